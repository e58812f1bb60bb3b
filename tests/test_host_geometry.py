"""The library's geometry precompute (Sec. 2: the contravariant metric terms
Ja^i, 2D cross-product and 3D invariant-curl forms, and the Jacobian J)
against the oracle, on the CPU.  A host driver (tests/host/
geometry_host_test.cpp) runs the library's own element geometry, the code
build_level runs before the upload, on quadratic cubed-sphere elements
(some with permuted local axes), a rotated affine box and a stretched 2D
plate; the result must match oracle.geometry to 1e-12 of the largest metric
term of the mesh (the two codes evaluate the mapping with different
interpolation formulas)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1806_11456_gb300 import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-12


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cxx is None or not os.path.isdir(os.path.join(home, "include")):
        pytest.skip("no host compiler or CUDA headers")
    import __graft_entry__ as g
    from paper_1806_11456_gb300 import build
    g.build()
    exe = str(tmp_path_factory.mktemp("geometry") / "geometry_host_test")
    cmd = [cxx, "-std=c++17", "-O1", "-I", os.path.join(home, "include"),
           os.path.join(ROOT, "tests", "host", "geometry_host_test.cpp"), "-o", exe, build.LIB,
           "-Wl,-rpath," + os.path.dirname(build.LIB)]
    for d in (os.path.join(home, "lib64"), os.path.join(home, "lib")):
        if os.path.isdir(d):
            cmd += ["-L", d, "-Wl,-rpath," + d]
    subprocess.check_call(cmd + ["-lcudart", "-lpthread"])
    return exe


def _run(exe, mesh, orders):
    lines = [f"{mesh['dim']} {mesh['K']} {mesh['M']}",
             " ".join(float(v).hex() for v in np.asarray(mesh["xmap"], dtype=np.float64).reshape(-1)),
             " ".join(str(int(v)) for v in np.asarray(orders).reshape(-1))]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    vals = np.array([float.fromhex(x) for x in out.split()]).reshape(-1, 10)
    return vals[:, :9], vals[:, 9]


CASES = {
    "sphere_curved": lambda: (lambda m: (m, syn.random_orders(m["K"], 3, 1, 5, 7)))(
        syn.rotate_elements(syn.cubed_sphere_mesh(2, 2), seed=5, frac=0.6)),
    "box_rotated": lambda: (lambda m: (m, syn.random_orders(m["K"], 3, 1, 6, 8)))(
        syn.rotate_elements(syn.periodic_box(2, 2, 2), seed=4, frac=0.75)),
    "plate_2d": lambda: (lambda m: (m, syn.random_orders(m["K"], 2, 1, 8, 9)))(
        syn.flat_plate_mesh(nx=6, ny=4)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_library_geometry_equals_the_oracle(driver, name):
    mesh, o = CASES[name]()
    Ja, J = _run(driver, mesh, o)
    Ja_o, J_o = orc.geometry(mesh, o)
    scale = np.max(np.abs(Ja_o))
    assert Ja.shape == Ja_o.shape and np.max(np.abs(Ja - Ja_o)) <= TOL * scale, np.max(np.abs(Ja - Ja_o)) / scale
    assert np.max(np.abs(J - J_o)) <= TOL * np.max(np.abs(J_o))
    assert np.all(J > 0)
