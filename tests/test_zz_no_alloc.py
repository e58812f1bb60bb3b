"""dg_transfer_noalloc -- the transfer for callers that cannot allocate device
memory -- against the allocating dg_transfer_state, through the C ABI, on two
calls in a row (the second call reuses the shared static record array the
first one filled), and against the oracle's tensor-product L2 projection /
interpolation (Sec. 3.1).  Tolerance: 1e-12 of max |q|, as for the other state
comparisons."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1806_11456_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1806_11456_gb300 import dg as mod
    return mod


def _noalloc(dgmod, dim, o_from, o_to, q_in, q_out):
    import torch
    of = np.ascontiguousarray(o_from, dtype=np.int32)
    ot = np.ascontiguousarray(o_to, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    return dgmod.lib().dg_transfer_noalloc(dim, len(of), of.ctypes.data_as(ip), ot.ctypes.data_as(ip), 5,
                                           ctypes.c_void_p(q_in.data_ptr()), ctypes.c_void_p(q_out.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_transfer_matches_allocating_transfer_two_calls(dg, dim):
    import torch
    if dim == 3:
        mesh = syn.rotate_elements(syn.periodic_box(3, 2, 2), seed=3, frac=0.5)
    else:
        mesh = syn.flat_plate_mesh(nx=12, ny=5)
    prm = syn.flow_params()
    o1 = syn.random_orders(mesh["K"], dim, 1, 7, 21)
    o2 = syn.random_orders(mesh["K"], dim, 1, 7, 22)
    o3 = syn.random_orders(mesh["K"], dim, 1, 7, 23)
    q1 = torch.tensor(syn.perturbed_state(mesh, o1, prm, 4), device="cuda")
    A, B, C = dg.Mesh(mesh, o1, prm), dg.Mesh(mesh, o2, prm), dg.Mesh(mesh, o3, prm)
    # first call: o1 -> o2
    ref12 = A.transfer_state_to(B, q1)
    out12 = torch.full((5 * B.nodes,), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(dg, dim, o1, o2, q1, out12) == 0
    torch.cuda.synchronize()
    scale = float(q1.abs().max())
    assert float((out12 - ref12).abs().max()) <= TOL * scale
    want12 = orc.transfer(dim, o1, o2, q1.cpu().numpy())
    assert float(np.max(np.abs(out12.cpu().numpy() - want12))) <= TOL * scale
    # second call in a row: o2 -> o3 on the first call's output
    ref23 = B.transfer_state_to(C, ref12)
    out23 = torch.full((5 * C.nodes,), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(dg, dim, o2, o3, out12, out23) == 0
    torch.cuda.synchronize()
    assert float((out23 - ref23).abs().max()) <= TOL * scale
    want23 = orc.transfer(dim, o2, o3, want12)
    assert float(np.max(np.abs(out23.cpu().numpy() - want23))) <= TOL * scale


def test_noalloc_rejects_more_elements_than_its_limit(dg):
    import torch
    K = 65537
    o = np.ones((K, 3), dtype=np.int32)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = _noalloc(dg, 3, o, o, buf, buf.clone())
    assert rc == -1
    assert "65536" in dg.lib().dg_last_error().decode()
