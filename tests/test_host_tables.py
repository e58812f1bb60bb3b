"""The library's 1-D tables and transfer matrices against closed forms, on
the CPU (a host driver, tests/host/tables_host_test.cpp, prints the tables
the library builds and uploads).  For every node count n = 1 ... 13:

- the Gauss-Legendre nodes and weights equal numpy's leggauss;
- the collocation derivative D differentiates the Legendre polynomials
  P_0 ... P_{n-1} exactly at the nodes;
- summation by parts, W D + (W D)^T = l(1) l(1)^T - l(-1) l(-1)^T, pins D,
  the weights and the boundary rows together, and the weak-form matrix is
  Dhat[i][a] = -(w_a / w_i) D[a][i];
- the boundary rows reproduce P_p(-1) = (-1)^p and P_p(1) = 1 for p < n;
- the transfer from n_f to n_t nodes reproduces P_p for p < min(n_f, n_t)
  and, as an L2 projection (n_t < n_f), maps P_p for n_t <= p < n_f to zero
  (orthogonality); equal counts give the identity (Sec. 3.1, eq for I_P^N)."""
import os
import shutil
import subprocess

import numpy as np
import pytest
from numpy.polynomial import legendre as npl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-12


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    cxx = shutil.which("g++")
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cxx is None or not os.path.isdir(os.path.join(home, "include")):
        pytest.skip("no host compiler or CUDA headers")
    import __graft_entry__ as g
    from paper_1806_11456_gb300 import build
    g.build()
    exe = str(tmp_path_factory.mktemp("tables") / "tables_host_test")
    cmd = [cxx, "-std=c++17", "-O1", "-I", os.path.join(home, "include"),
           os.path.join(ROOT, "tests", "host", "tables_host_test.cpp"), "-o", exe, build.LIB,
           "-Wl,-rpath," + os.path.dirname(build.LIB)]
    for d in (os.path.join(home, "lib64"), os.path.join(home, "lib")):
        if os.path.isdir(d):
            cmd += ["-L", d, "-Wl,-rpath," + d]
    subprocess.check_call(cmd + ["-lcudart", "-lpthread"])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    tab = {}
    for line in out.splitlines():
        f = line.split()
        if f[0] == "T":
            nf, nt = int(f[1]), int(f[2])
            tab[("T", nf, nt)] = np.array([float.fromhex(v) for v in f[3:]]).reshape(nt, nf)
        else:
            n = int(f[1])
            v = np.array([float.fromhex(v) for v in f[2:]])
            tab[(f[0], n)] = v.reshape(n, n) if f[0] in ("D", "Dhat") else v
    return tab


def _P(p, x):
    return npl.legval(x, [0.0] * p + [1.0])


def _dP(p, x):
    return npl.legval(x, npl.legder([0.0] * p + [1.0])) if p > 0 else np.zeros_like(x)


NS = list(range(1, 14))


@pytest.mark.parametrize("n", NS)
def test_gauss_rule_derivative_and_boundary_rows(tables, n):
    x, w = tables[("x", n)], tables[("w", n)]
    xr, wr = npl.leggauss(n)
    assert np.max(np.abs(x - xr)) < 1e-15 and np.max(np.abs(w - wr)) < 1e-15
    D, Dh, lm, lp = tables[("D", n)], tables[("Dhat", n)], tables[("lm", n)], tables[("lp", n)]
    for p in range(n):
        assert np.max(np.abs(D @ _P(p, x) - _dP(p, x))) <= TOL * max(1.0, p * p), p
        assert abs(lm @ _P(p, x) - (-1.0) ** p) <= TOL and abs(lp @ _P(p, x) - 1.0) <= TOL, p
    WD = np.diag(w) @ D
    assert np.max(np.abs(WD + WD.T - (np.outer(lp, lp) - np.outer(lm, lm)))) <= TOL * n * n
    assert np.max(np.abs(Dh - (-(w[None, :] / w[:, None]) * D.T))) <= TOL * n * n


@pytest.mark.parametrize("nf", NS)
def test_transfer_matrices(tables, nf):
    for nt in NS:
        T = tables[("T", nf, nt)]
        xf, xt = npl.leggauss(nf)[0], npl.leggauss(nt)[0]
        if nf == nt:
            assert np.array_equal(T, np.eye(nf))
            continue
        for p in range(min(nf, nt)):
            assert np.max(np.abs(T @ _P(p, xf) - _P(p, xt))) <= TOL, (nf, nt, p)
        for p in range(nt, nf):  # projection: the higher Legendre modes vanish
            assert np.max(np.abs(T @ _P(p, xf))) <= TOL, (nf, nt, p)
