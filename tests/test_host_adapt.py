"""The library's order adaptation (dg_adapt) against the oracle, on the CPU.

dg_adapt runs on the host: the per-element order selection of Sec. 3.3.2
(steps 3-6: the inner map first, then the extrapolated map, the fewest
degrees of freedom with the stated tie-breaks) and the order-jump fix-point
(Sec. 4.1.2 for 2D, Sec. 4.2.1 for 3D, with the conforming-wall rule).  A
small host driver (tests/host/adapt_host_test.cpp) builds a mesh handle with
only the host fields dg_adapt reads, so the library's own code runs here
without a GPU; its maps must equal oracle.adapt_orders bit for bit on tables
that exercise every branch: decaying and noisy estimates, unmeasured
entries, extrapolation above the reference order, caps, both jump rules,
rotated 3D faces and a tagged wall."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1806_11456_gb300 import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RULES = {0: None, 1: "2d", 2: "3d"}


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cxx is None or not os.path.isdir(os.path.join(home, "include")):
        pytest.skip("no host compiler or CUDA headers")
    import __graft_entry__ as g
    from paper_1806_11456_gb300 import build
    g.build()
    libdir = os.path.dirname(build.LIB)
    exe = str(tmp_path_factory.mktemp("adapt") / "adapt_host_test")
    cudalib = [d for d in (os.path.join(home, "lib64"), os.path.join(home, "lib")) if os.path.isdir(d)]
    cmd = [cxx, "-std=c++17", "-O1", "-I", os.path.join(home, "include"),
           os.path.join(ROOT, "tests", "host", "adapt_host_test.cpp"), "-o", exe, build.LIB,
           "-Wl,-rpath," + libdir]
    for d in cudalib:
        cmd += ["-L", d, "-Wl,-rpath," + d]
    cmd += ["-lcudart", "-lpthread"]
    subprocess.check_call(cmd)
    return exe


def _run(exe, mesh, P, tab, tau_max, n_min, n_max, cap, rule, conform_tag):
    K = mesh["K"]
    lines = [f"{mesh['dim']} {K}",
             " ".join(str(int(v)) for v in np.asarray(mesh["ftab"], dtype=np.int64).reshape(-1)),
             " ".join(str(int(v)) for v in np.asarray(P, dtype=np.int64).reshape(-1)),
             f"{float(tau_max).hex()} {n_min} {n_max} {cap} {rule} {conform_tag}",
             " ".join(float(v).hex() for v in np.asarray(tab, dtype=np.float64).reshape(-1))]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    assert not out.startswith("error"), out
    return np.array([int(x) for x in out.split()], dtype=np.int32).reshape(K, 3)


def _table(rng, K, P, dim, noisy=False, holes=False):
    """Directional estimates t_i(N) for N < P_i: log-linear decay with seeded
    rates, optionally with noise that breaks monotonicity and with entries
    left unmeasured (-1)."""
    tab = np.full((K, 3, 16), -1.0)
    for e in range(K):
        for i in range(dim):
            rate, base = rng.uniform(0.05, 1.2), 10 ** rng.uniform(-5, 0)
            for N in range(1, P[e, i]):
                j = rng.uniform(-1.0, 1.0) if noisy else rng.uniform(-0.3, 0.3)
                tab[e, i, N] = base * 10 ** (-rate * N) * 10 ** j
                if holes and rng.uniform() < 0.15:
                    tab[e, i, N] = -1.0
    return tab


def _cases():
    out = []
    rng = np.random.default_rng(11)
    m2 = syn.box_mesh(np.linspace(0, 1, 9), np.linspace(0, 1, 7), None)
    P2 = syn.random_orders(m2["K"], 2, 2, 7, 3)
    out.append(("2d", m2, P2, _table(rng, m2["K"], P2, 2), 1, 1, 9, 0, -1))
    out.append(("2d_noisy_holes", m2, P2, _table(rng, m2["K"], P2, 2, noisy=True, holes=True), 1, 1, 9, 0, -1))
    out.append(("2d_capped", m2, P2, _table(rng, m2["K"], P2, 2), 1, 1, 9, 4, -1))
    out.append(("2d_no_rule", m2, P2, _table(rng, m2["K"], P2, 2, noisy=True), 0, 2, 6, 0, -1))
    plate = syn.box_mesh(np.linspace(-0.2, 1, 7), [0, 0.02, 0.06, 0.15, 0.3],
                         bc=dict(xmin=1, xmax=2, ymin=lambda i, k: 3 if i < 1 else 4, ymax=1))
    Pp = syn.random_orders(plate["K"], 2, 2, 7, 5)
    out.append(("2d_wall_tag", plate, Pp, _table(rng, plate["K"], Pp, 2), 1, 1, 9, 0, 4))
    m3 = syn.rotate_elements(syn.box_mesh(np.linspace(0, 1, 5), np.linspace(0, 1, 4), np.linspace(0, 1, 4)), 2)
    P3 = syn.random_orders(m3["K"], 3, 2, 7, 3)
    out.append(("3d_rotated", m3, P3, _table(rng, m3["K"], P3, 3), 2, 2, 9, 0, -1))
    out.append(("3d_rotated_noisy_capped", m3, P3, _table(rng, m3["K"], P3, 3, noisy=True, holes=True), 2, 2, 9, 5,
                -1))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_library_adaptation_equals_the_oracle(driver, case):
    name, mesh, P, tab, rule, n_min, n_max, cap, tag = case
    kinds = set()
    for tau_max in (1e-1, 1e-3, 1e-5):
        got = _run(driver, mesh, P, tab, tau_max, n_min, n_max, cap, rule, tag)
        want = orc.adapt_orders(mesh, P, tab, tau_max, n_min, n_max, cap=cap or None, rule=RULES[rule],
                                conform_tag=None if tag < 0 else tag)
        assert np.array_equal(got, want), (name, tau_max)
        kinds |= {tuple(r) for r in got}
    assert len(kinds) > 3  # the maps are not trivially uniform
