"""GB300-native DGSEM p-multigrid with anisotropic truncation-error p-adaptation.

The compute path is the CUDA library libdgpmg.so behind the C ABI of
include/dg.h; ``paper_1806_11456_gb300.dg`` is its Python binding and
``paper_1806_11456_gb300.synthetic`` builds seeded meshes and states.
Importing this package loads nothing: the binding loads the library on first
use and raises if it is missing."""
