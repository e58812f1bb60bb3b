"""FP64 CPU oracle of the DGSEM p-multigrid / p-adaptation path.

Test infrastructure only: imported by tests/, the smoke check and the CPU
baseline leg of bench.py -- never by the product package."""
