"""Batched solves (dg_batch_create): every kernel runs once over the elements
of all solves, each solve keeping its own parameters, time step and norm.  A
solve inside a batch must advance exactly as it does alone."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1806_11456_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1806_11456_gb300 import dg as mod
    return mod


def _solves_2d(n, seed, top=5):
    rng = np.random.default_rng(seed)
    items = []
    for k in range(n):
        nx, ny = int(rng.integers(3, 7)), int(rng.integers(2, 5))
        mesh = syn.flat_plate_mesh(nx=nx, ny=ny, dy0=0.02, ratio=1.3)
        prm = syn.flow_params(mach=float(10 ** rng.uniform(-1, np.log10(0.4))),
                              re=float(10 ** rng.uniform(2, 5)))
        o = syn.random_orders(mesh["K"], 2, 1, top, seed * 100 + k)
        o[0, :2] = top  # every solve reaches the same top order
        q = syn.perturbed_state(mesh, o, prm, seed * 100 + k, amp=0.02)
        items.append((mesh, o, prm, q))
    return items


def _solves_3d(n, seed, top=4):
    # trilinear shells (M = 1 <= N/2 for every N >= 2): the free-stream
    # condition of Sec. 2 for p-nonconforming 3D meshes holds, so smoothing
    # from a perturbed state stays bounded
    rng = np.random.default_rng(seed)
    items = []
    for k in range(n):
        mesh = syn.rotate_elements(syn.cubed_sphere_mesh(2, int(rng.integers(2, 4)), M=1),
                                   seed=seed + k, frac=0.5)
        prm = syn.flow_params(mach=float(10 ** rng.uniform(-1, np.log10(0.4))),
                              re=float(10 ** rng.uniform(2, 5)))
        o = syn.random_orders(mesh["K"], 3, 2, top, seed * 100 + k)
        o[0] = top
        q = syn.smooth_state(mesh, o, prm, seed * 100 + k)
        items.append((mesh, o, prm, q))
    return items


def _dev(x):
    import torch
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("kind", ["2d", "3d"])
@pytest.mark.parametrize("arith", ["fp64", "df32"])
def test_batch_equals_alone(dg, kind, arith):
    import torch
    items = _solves_2d(4, 1) if kind == "2d" else _solves_3d(3, 2)
    B = dg.Mesh.batch([(m, o, p) for (m, o, p, _) in items]).set_arithmetic(arith)
    off = B.solve_slices()
    assert len(off) == len(items) + 1
    qb = _dev(np.concatenate([q for (*_, q) in items]))
    kw = dict(beta1=1, beta2=2, beta_c=3)
    # residuals and per-solve norms
    rb = B.residual(qb).cpu().numpy()
    norms = B.residual_norms(qb)
    for k, (m, o, p, q) in enumerate(items):
        A = dg.Mesh(m, o, p).set_arithmetic(arith)
        ra, na = A.residual(_dev(q), norm=True)
        ra = ra.cpu().numpy()
        assert np.array_equal(rb[5 * off[k]:5 * off[k + 1]], ra)
        assert norms[k] == na
        if k == 0:  # and the batched residual is the oracle's (Sec. 2), element by element
            ro = orc.residual(m, o, p, q)
            assert np.max(np.abs(rb[5 * off[k]:5 * off[k + 1]] - ro)) <= 1e-12 * orc.volume_scale(m, o, p, q)
    # V-cycles (graph replay) and the explicit time step per solve
    B.vcycle(qb, None, graph=True, **kw)
    B.vcycle(qb, None, graph=True, **kw)
    qbn = qb.cpu().numpy()
    for k, (m, o, p, q) in enumerate(items):
        A = dg.Mesh(m, o, p).set_arithmetic(arith)
        qa = _dev(q)
        A.vcycle(qa, None, **kw)
        A.vcycle(qa, None, **kw)
        assert np.array_equal(qbn[5 * off[k]:5 * off[k + 1]], qa.cpu().numpy()), k
        if k == 0 and kind == "2d":  # two batched V-cycles against Algorithm 1 in the oracle
            qo = orc.fas_vcycle(m, o, p, q, None, kw["beta1"], kw["beta2"], kw["beta_c"])
            qo = orc.fas_vcycle(m, o, p, qo, None, kw["beta1"], kw["beta2"], kw["beta_c"])
            assert np.max(np.abs(qbn[5 * off[k]:5 * off[k + 1]] - qo)) <= 1e-12 * np.max(np.abs(qo))


def test_batch_steady_solve_reports_every_solve(dg):
    items = _solves_2d(3, 7, top=3)
    B = dg.Mesh.batch([(m, o, p) for (m, o, p, _) in items])
    qb = _dev(np.concatenate([q for (*_, q) in items]))
    q2, rep = B.solve_steady(qb, None, tol=1e-30, max_cycles=3, mg=dict(beta1=1, beta2=1, beta_c=2))
    assert rep["cycles"] == 3 and rep["status"] == -5
    norms = B.residual_norms(q2)
    assert abs(max(norms) - rep["rnorm"]) <= 1e-14 * max(norms)


def test_batch_rejects_mixed_dimensions(dg):
    a = _solves_2d(1, 3)[0]
    b = _solves_3d(1, 4)[0]
    with pytest.raises(dg.DGError):
        dg.Mesh.batch([(a[0], a[1], a[2]), (b[0], b[1], b[2])])


@pytest.mark.parametrize("arith", ["fp64", "mixed"])
def test_held_solves_stay_put_and_the_others_advance_as_alone(dg, arith):
    """dg_batch_set_active: a held solve's state is bitwise unchanged by later
    cycles (its time step is 0 in every sweep, so every correction it gets is
    exactly 0), while the other solves advance as they do alone; with the
    smoothing control on, the held solve counts as satisfied."""
    items = _solves_2d(3, 11)
    B = dg.Mesh.batch([(m, o, p) for (m, o, p, _) in items]).set_arithmetic(arith)
    off = B.solve_slices()
    qb = _dev(np.concatenate([q for (*_, q) in items]))
    kw = dict(beta1=1, beta2=2, beta_c=3)
    B.vcycle(qb, None, graph=True, **kw)
    before = qb.cpu().numpy()
    B.set_active([1, 0, 1])
    for graph in (True, False):
        B.vcycle(qb, None, graph=graph, **kw)
    if arith == "fp64":
        B.vcycle(qb, None, control=2, **kw)
    after = qb.cpu().numpy()
    assert np.array_equal(after[5 * off[1]:5 * off[2]], before[5 * off[1]:5 * off[2]])
    for k in (0, 2):
        m, o, p, q = items[k]
        A = dg.Mesh(m, o, p).set_arithmetic(arith)
        qa = _dev(q)
        A.vcycle(qa, None, graph=True, **kw)
        A.vcycle(qa, None, graph=True, **kw)
        A.vcycle(qa, None, graph=False, **kw)
        if arith == "fp64":
            A.vcycle(qa, None, control=2, **kw)
        assert np.array_equal(after[5 * off[k]:5 * off[k + 1]], qa.cpu().numpy()), k
        assert not np.array_equal(after[5 * off[k]:5 * off[k + 1]], before[5 * off[k]:5 * off[k + 1]])
