"""Serving loop (dg_server_*): concurrent steady solves admitted by a memory
budget.  Each solve must give the same bits in the mix as alone."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1806_11456_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

MG = dict(beta1=1, beta2=1, beta_c=2, direction=-1, coarsest=1, delta_n=1, graph=1)


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1806_11456_gb300 import dg as mod
    return mod


def _requests(n, seed):
    """Mixed 2D/3D requests with sources, random orders and flow parameters;
    an unreachable tolerance makes every solve run exactly max_cycles."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        if k % 3 == 2:
            mesh = syn.rotate_elements(syn.periodic_box(2, 2, 2), seed=k, frac=0.5)
            o = syn.random_orders(mesh["K"], 3, 2, 4, seed * 10 + k)
        else:
            mesh = syn.periodic_box(int(rng.integers(2, 5)), int(rng.integers(2, 4)), 1, dim=2)
            o = syn.random_orders(mesh["K"], 2, 1, 5, seed * 10 + k)
        prm = syn.flow_params(mach=float(rng.uniform(0.1, 0.4)), re=float(10 ** rng.uniform(2, 4)))
        q = syn.perturbed_state(mesh, o, prm, k, amp=0.02)
        s = syn.random_source(mesh, o, k + 1, amp=1e-3)
        out.append((mesh, o, prm, q, s))
    return out


def _alone(dg, mesh, o, prm, q, s, **kw):
    import torch
    M = dg.Mesh(mesh, o, prm)
    qd = torch.tensor(q, device="cuda")
    sd = None if s is None else torch.tensor(s, device="cuda")
    qd2, rep = M.solve_steady(qd, sd, **kw)
    return qd2.cpu().numpy(), M.orders.copy(), rep


def test_server_results_equal_alone(dg):
    reqs = _requests(7, 1)
    kw = dict(tol=1e-30, max_cycles=3, fmg=True, fmg_tol=1e-30, mg=MG)
    with dg.Server(hbm_budget=8 << 30, slots=4) as S:
        ids = [S.submit(m, o, p, q0=q, s=s, **kw) for (m, o, p, q, s) in reqs]
        S.wait()
        for rid, (m, o, p, q, s) in zip(ids, reqs):
            info = S.info(rid)
            assert info["state"] == -5 and info["rep"]["cycles"] > 0  # ran to the cycle cap
            assert info["t_submit"] <= info["t_start"] <= info["t_end"]
            qs, os_ = S.result(rid)
            qa, oa, rep = _alone(dg, m, o, p, q, s, **kw)
            assert np.array_equal(os_, oa)
            assert np.array_equal(qs, qa), rid
            assert info["rep"]["cycles"] == rep["cycles"]
            if rid == ids[0]:  # the served solve against the oracle's steady driver (Sec. 3.1.1)
                oo, qo, orep = orc.solve_steady(m, o, p, q, s, kw["tol"], kw["max_cycles"], MG, fmg=True,
                                                fmg_tol=kw["fmg_tol"])
                assert np.array_equal(oo, os_) and orep["cycles"] == info["rep"]["cycles"]
                assert np.max(np.abs(qs - qo)) <= 1e-12 * np.max(np.abs(qo))
            S.release(rid)


def test_a_finished_request_carries_its_result(dg):
    """Waiting on one request and reading it at once, while other slots are
    still running, sees the whole outcome: a finished state comes with its
    end time, report and result (they are published together)."""
    reqs = _requests(7, 1)
    kw = dict(tol=1e-30, max_cycles=3, fmg=True, fmg_tol=1e-30, mg=MG)
    with dg.Server(hbm_budget=8 << 30, slots=4) as S:
        ids = [S.submit(m, o, p, q0=q, s=s, **kw) for (m, o, p, q, s) in reqs]
        for rid, (m, o, p, q, s) in zip(ids, reqs):
            S.wait(rid)
            info = S.info(rid)
            assert info["state"] == -5
            assert 0.0 <= info["t_submit"] <= info["t_start"] <= info["t_end"] and info["t_end"] > 0.0
            assert info["rep"]["cycles"] > 0 and info["rep"]["nodes"] == q.size // 5
            qs, os_ = S.result(rid)
            assert qs.size == q.size and np.any(qs != 0.0)
            assert np.array_equal(os_, o)
            S.release(rid)


def test_server_adaptation_equals_alone(dg):
    mesh = syn.periodic_box(3, 2, 1, dim=2)
    prm = syn.flow_params(mach=0.3, re=100.0)
    P = syn.uniform_orders(mesh["K"], 2, 5)
    q = syn.manufactured_state(mesh, P, 5, prm[2], prm[0], amp=0.05)
    kw = dict(tol=1e-30, max_cycles=2, mg=MG, adapt=True, tau_max=1e3, n_min=1, n_max=6, jump_rule=1)
    with dg.Server(hbm_budget=4 << 30, slots=2) as S:
        rid = S.submit(mesh, P, prm, q0=q, **kw)
        S.wait(rid)
        info = S.info(rid)
        qs, os_ = S.result(rid)
    qa, oa, rep = _alone(dg, mesh, P, prm, q, None, **kw)
    assert info["rep"]["adapted"] == rep["adapted"] >= 1
    assert np.array_equal(os_, oa) and not np.array_equal(os_, P)
    assert np.array_equal(qs, qa)


def test_server_admission_by_budget(dg):
    reqs = _requests(3, 2)[:2]
    kw = dict(tol=1e-30, max_cycles=4, mg=MG)
    est = [dg.solve_footprint(m, o, p) for (m, o, p, _, _) in reqs]
    # room for either request, not for both: the second waits for the first
    with dg.Server(hbm_budget=max(est) + min(est) // 2, slots=4) as S:
        ids = [S.submit(m, o, p, q0=q, s=s, **kw) for (m, o, p, q, s) in reqs]
        S.wait()
        a, b = (S.info(i) for i in ids)
        assert b["t_start"] >= a["t_end"]
        big = syn.periodic_box(12, 12, 1, dim=2)
        with pytest.raises(dg.DGError):  # larger than the whole budget
            S.submit(big, syn.uniform_orders(big["K"], 2, 8), reqs[0][2], **kw)


def test_footprint_bounds_the_memory_held(dg):
    kw = dict(tol=1e-30, max_cycles=1, mg=MG)
    with dg.Server(hbm_budget=8 << 30, slots=2) as S:
        for (m, o, p, q, s) in _requests(6, 3):
            rid = S.submit(m, o, p, q0=q, s=s, **kw)
            S.wait(rid)
            info = S.info(rid)
            assert info["dev_bytes"] > 0
            assert info["dev_bytes"] <= info["est_bytes"] <= 4 * info["dev_bytes"] + (2 << 20), info


def test_check_every_runs_whole_groups_of_cycles(dg):
    m, o, p, q, s = _requests(1, 5)[0]
    kw = dict(tol=1e-30, max_cycles=7, mg=MG)
    qa, _, rep1 = _alone(dg, m, o, p, q, s, **kw)
    qb, _, rep5 = _alone(dg, m, o, p, q, s, check_every=5, **kw)
    assert rep1["cycles"] == rep5["cycles"] == 7  # the cap still bounds the phase
    assert np.array_equal(qa, qb)                 # same cycles, fewer residual checks


def test_double_float_requests_equal_alone(dg):
    reqs = _requests(3, 6)
    kw = dict(tol=1e-30, max_cycles=3, mg=MG, arith="df32")
    with dg.Server(hbm_budget=8 << 30, slots=3) as S:
        ids = [S.submit(m, o, p, q0=q, s=s, **kw) for (m, o, p, q, s) in reqs]
        S.wait()
        for rid, (m, o, p, q, s) in zip(ids, reqs):
            qs, _ = S.result(rid)
            import torch
            M = dg.Mesh(m, o, p).set_arithmetic("df32")
            qd, _ = M.solve_steady(torch.tensor(q, device="cuda"), torch.tensor(s, device="cuda"),
                                   tol=1e-30, max_cycles=3, mg=MG)
            assert np.array_equal(qs, qd.cpu().numpy())


def _shared_requests(n, seed, top=3):
    """2D requests that can share launches (same top order) with different
    flow parameters, sizes and order maps, and a 3D one that cannot."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        mesh = syn.periodic_box(int(rng.integers(2, 5)), int(rng.integers(2, 4)), 1, dim=2)
        o = syn.random_orders(mesh["K"], 2, 1, top, seed * 10 + k)
        o[0, :2] = top
        prm = syn.flow_params(mach=float(rng.uniform(0.1, 0.4)), re=float(10 ** rng.uniform(2, 4)))
        q = syn.perturbed_state(mesh, o, prm, k, amp=0.02)
        s = syn.random_source(mesh, o, k + 1, amp=1e-3) if k % 2 == 0 else None
        out.append((mesh, o, prm, q, s))
    mesh = syn.rotate_elements(syn.periodic_box(2, 2, 2), seed=3, frac=0.5)
    o = syn.random_orders(mesh["K"], 3, 2, 3, 77)
    prm = syn.flow_params(mach=0.3, re=200.0)
    out.append((mesh, o, prm, syn.perturbed_state(mesh, o, prm, 9, amp=0.02), None))
    return out


def test_shared_launches_equal_alone(dg):
    """Shared launches (batch_max > 1): one slot runs the compatible requests
    as one batch, members with their own cycle caps, tolerances and check
    intervals leave at their own check points, and requests submitted while
    the batch runs join it.  Every result -- state, cycles and status -- is
    bit for bit that of the same request alone; the incompatible 3D request
    runs on its own."""
    import time
    reqs = _shared_requests(7, 3)
    kws = []
    for k in range(len(reqs)):
        kw = dict(tol=1e-30, max_cycles=3 + k % 4, check_every=1 + k % 3, mg=MG)
        if k == 2:
            kw["tol"] = 1e30  # stops at its first check, before any cycle
        kws.append(kw)
    with dg.Server(hbm_budget=8 << 30, slots=1, batch_max=4) as S:
        ids = []
        for k, ((m, o, p, q, s), kw) in enumerate(zip(reqs, kws)):
            ids.append(S.submit(m, o, p, q0=q, s=s, **kw))
            if k == 3:
                time.sleep(0.2)  # the rest arrive while the first batch runs
        S.wait()
        peers = []
        for rid, (m, o, p, q, s), kw in zip(ids, reqs, kws):
            info = S.info(rid)
            qs, os_ = S.result(rid)
            qa, oa, rep = _alone(dg, m, o, p, q, s, **kw)
            assert np.array_equal(os_, oa)
            assert info["rep"]["cycles"] == rep["cycles"] and info["state"] == rep["status"], (rid, info, rep)
            assert np.array_equal(qs, qa), rid
            peers.append(info["batch_peers"])
    assert max(peers[:-1]) >= 1      # the 2D requests shared launches
    assert peers[-1] == 0            # the 3D one could not
