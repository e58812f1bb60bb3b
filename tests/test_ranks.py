"""Host logic of the N > 1 bench path on CPU: two gloo ranks with different
timings give the slowest rank's time and the job-total throughput."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_ranks(100.0 + 50.0 * rank, 1e6, world, "cpu")
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    import socket
    ctx = mp.get_context("spawn")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 150.0                      # max over ranks
        assert value == pytest.approx(2 * 1e6 / 0.150)  # both ranks' units over that time


def test_footprint_is_host_logic_and_grows_with_orders():
    import __graft_entry__ as g
    g.build()
    from paper_1806_11456_gb300 import dg, synthetic as syn
    mesh = syn.periodic_box(3, 3, 1, dim=2)
    prm = syn.flow_params()
    small = dg.solve_footprint(mesh, syn.uniform_orders(mesh["K"], 2, 2), prm)
    large = dg.solve_footprint(mesh, syn.uniform_orders(mesh["K"], 2, 6), prm)
    assert 0 < small < large
    m3 = syn.periodic_box(3, 3, 3)
    assert dg.solve_footprint(m3, syn.uniform_orders(m3["K"], 3, 4), prm) > large


def test_server_rejects_bad_parameters_without_touching_the_device():
    import ctypes
    import __graft_entry__ as g
    g.build()
    from paper_1806_11456_gb300 import dg
    L = dg.lib()
    h = ctypes.c_void_p()
    for budget, slots in ((1 << 30, 0), (0, 2), (1 << 30, 1000)):
        p = dg.ServerParams()
        p.hbm_budget, p.slots, p.device = budget, slots, 0
        assert L.dg_server_create(ctypes.byref(p), ctypes.byref(h)) == -1  # DG_EINVAL
    rid = ctypes.c_int64()
    sp = dg.solve_params()
    assert L.dg_server_submit(None, None, None, None, None, ctypes.byref(sp), ctypes.byref(rid)) == -1
    assert L.dg_server_wait(None, -1, 0.0) == -1
    assert L.dg_server_destroy(None) == 0
