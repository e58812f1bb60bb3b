"""The mixed-precision form (dg_set_arithmetic 'mixed') against the FP64
oracle.

Roles: the finest-level residual, the coarse right-hand sides and the tau
estimate stay FP64 (compared at the FP64 bar, 1e-12 of the term scale); the
smoother and every coarse-level operator evaluation are FP32 Jacobian-vector
products J(Q) dQ in tangent arithmetic.  Their bound, per variable v:
|J dQ (GPU) - J dQ (oracle)|_inf <= TOL_TF * s_v, with s_v the magnitude of
the tangent's volume term for variable v (max over nodes of the directional
derivative of the oracle's volume term) -- FP32 rounding of the terms, not of
the result, which cancels.  The oracle differentiates its FP64 residual by
fourth-order central differences (accurate to ~1e-9 of the term scale on
these smooth states); the states are oblique flows, so no face-normal
velocity sits at the kink of the Roe dissipation's |lambda|.  The mixed
V-cycle is compared with the oracle's restatement of the same cycle within
TOL_CYCLE of the size of the correction it applies, and a mixed steady solve
must satisfy the oracle's FP64 equations to its tolerance.  Measured on
GB300: tangent errors up to 2.5e-6 of s_v, cycle errors up to 1.3e-7 of the
correction."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1806_11456_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
TOL = 1e-12
TOL_TF = 2e-5
TOL_CYCLE = 1e-6


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1806_11456_gb300 import dg as mod
    return mod


def _dev(x):
    import torch
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _cases():
    c = {}

    def box2d():
        mesh = syn.periodic_box(3, 3, 1, dim=2)
        prm = syn.flow_params(mach=0.3, re=100.0)
        return mesh, syn.random_orders(mesh["K"], 2, 2, 5, 31), prm

    def mortars3d():
        mesh = syn.periodic_box(3, 2, 2)
        prm = syn.flow_params(mach=0.3, re=100.0)
        return mesh, syn.random_orders(mesh["K"], 3, 1, 4, 32), prm

    def plate():
        mesh = syn.box_mesh(np.linspace(-0.2, 1, 6), [0, 0.01, 0.05, 0.12, 0.3],
                            bc=dict(xmin=1, xmax=2, ymin=lambda i, k: 3 if i < 1 else 4, ymax=1))
        prm = syn.flow_params(mach=0.2, re=1e4)
        return mesh, syn.random_orders(mesh["K"], 2, 1, 6, 33), prm

    def sphere():
        mesh = syn.rotate_elements(syn.cubed_sphere_mesh(2, 2), seed=5, frac=0.6)
        prm = syn.flow_params(mach=0.2, re=200.0)
        return mesh, syn.random_orders(mesh["K"], 3, 1, 4, 34), prm

    c["box2d"], c["mortars3d"], c["plate2d_all_bcs"], c["curved_sphere"] = box2d, mortars3d, plate, sphere
    return c


CASES = _cases()


def _tangent_scale(mesh, o, prm, q, dq):
    """Per-variable magnitude of the tangent's volume term."""
    dV = orc.directional_derivative(lambda x: orc.volume_term(mesh, o, prm, x), q, dq)
    return np.abs(syn.from_blocked(dV, o, mesh["dim"])).max(axis=1)


@pytest.mark.parametrize("name", list(CASES))
def test_tangent_residual_matches_the_oracle_derivative(dg, name):
    mesh, o, prm = CASES[name]()
    q = syn.oblique_state(mesh, o, prm, 3)
    rng = np.random.default_rng(4)
    dq = rng.normal(size=q.size) * 1e-2 * np.abs(q)
    b = syn.random_source(mesh, o, 5, amp=1e-2)
    M = dg.Mesh(mesh, o, prm)
    r = M.residual_tangent(_dev(q), _dev(dq), _dev(b)).cpu().numpy()
    ro = orc.tangent_residual(mesh, o, prm, q, dq, b)
    err = np.abs(syn.from_blocked(r - ro, o, mesh["dim"])).max(axis=1)
    scale = _tangent_scale(mesh, o, prm, q, dq)
    live = scale > 0  # (w in 2D is identically zero on both sides)
    assert np.all(err[~live] == 0.0)
    print(name, "tangent error / scale per variable:", err[live] / scale[live])
    assert np.all(err[live] <= TOL_TF * scale[live]), err[live] / scale[live]


def test_mixed_mode_keeps_the_fp64_residual_and_tau(dg):
    """The roles that stay FP64: the residual (convergence) and the tau
    estimate give the same bits as the FP64 mode."""
    mesh, o, prm = CASES["box2d"]()
    q = syn.oblique_state(mesh, o, prm, 6)
    A = dg.Mesh(mesh, o, prm)
    B = dg.Mesh(mesh, o, prm).set_arithmetic("mixed")
    qd = _dev(q)
    assert np.array_equal(A.residual(qd).cpu().numpy(), B.residual(qd).cpu().numpy())
    assert np.array_equal(A.tau_estimate(qd, None, dir_mask=3), B.tau_estimate(qd, None, dir_mask=3))


@pytest.mark.parametrize("name,kw", [
    ("box2d", dict(beta1=2, beta2=1, beta_c=3)),
    ("plate2d_all_bcs", dict(beta1=1, beta2=2, beta_c=2)),
    ("mortars3d", dict(beta1=1, beta2=1, beta_c=2, delta_n=2)),
])
@pytest.mark.parametrize("graph", [False, True])
def test_mixed_vcycle_matches_the_oracle_cycle(dg, name, kw, graph):
    mesh, o, prm = CASES[name]()
    qs = syn.oblique_state(mesh, o, prm, 7, amp=0.01)
    S = orc.operator_A(mesh, o, prm, qs)          # qs solves A(q) = S
    q0 = syn.oblique_state(mesh, o, prm, 8, amp=0.01)  # a start near it
    M = dg.Mesh(mesh, o, prm).set_arithmetic("mixed")
    qd = _dev(q0)
    if graph:
        M.vcycle(qd.clone(), _dev(S), graph=True, **kw)
    rep = M.vcycle(qd, _dev(S), graph=graph, **kw)
    qo = orc.mixed_vcycle(mesh, o, prm, q0, S, kw["beta1"], kw["beta2"], kw["beta_c"], delta_n=kw.get("delta_n", 1))
    corr = np.max(np.abs(qo - q0))
    assert rep["levels"] >= 2 and corr > 0
    err = np.max(np.abs(qd.cpu().numpy() - qo))
    print(name, "mixed cycle error / correction:", err / corr)
    assert err <= TOL_CYCLE * corr


# the smoothing rules of Sec. 3.1.2 on the linear residual b - J d: the
# number of operator evaluations (sweeps and rule checks) must equal the
# oracle's, so every rule took the same decision on both sides
@pytest.mark.parametrize("name,kw", [
    ("box2d", dict(beta1=1, beta2=1, beta_c=3, control=5, eta=1.1)),
    ("box2d", dict(beta1=1, beta2=1, beta_c=3, control=5, eta=2.0)),
    ("plate2d_all_bcs", dict(beta1=1, beta2=1, beta_c=2, control=4, eta=1.5)),
    ("mortars3d", dict(beta1=1, beta2=1, beta_c=2, control=3, eta=1.1)),
])
def test_mixed_vcycle_with_smoothing_control_matches_the_oracle(dg, name, kw, monkeypatch):
    mesh, o, prm = CASES[name]()
    qs = syn.oblique_state(mesh, o, prm, 7, amp=0.01)
    S = orc.operator_A(mesh, o, prm, qs)
    q0 = syn.oblique_state(mesh, o, prm, 8, amp=0.01)
    M = dg.Mesh(mesh, o, prm).set_arithmetic("mixed")
    qd = _dev(q0)
    rep = M.vcycle(qd, _dev(S), **kw)
    calls = []
    tangent = orc.tangent_residual

    def counted(*a, **k):
        calls.append(1)
        return tangent(*a, **k)

    monkeypatch.setattr(orc, "tangent_residual", counted)
    qo = orc.mixed_vcycle(mesh, o, prm, q0, S, kw["beta1"], kw["beta2"], kw["beta_c"],
                          control=kw["control"], eta=kw["eta"])
    fixed = 3 * (kw["beta1"] + kw["beta2"]) + 1
    print(name, kw, "evaluations gpu / oracle:", rep["residual_evals"], 1 + len(calls))
    assert rep["residual_evals"] == 1 + len(calls)  # the FP64 defect + the tangent evaluations
    corr = np.max(np.abs(qo - q0))
    err = np.max(np.abs(qd.cpu().numpy() - qo))
    print(name, "controlled mixed cycle error / correction:", err / corr)
    assert corr > 0 and err <= TOL_CYCLE * corr
    assert len(calls) > (rep["levels"] - 1) * fixed + 3 * kw["beta_c"]  # the rules added blocks or checks


def test_mixed_smoothing_control_per_solve_in_a_batch(dg):
    """Three solves whose rules take different decisions: each comes out of
    the batched controlled mixed cycle with the bits it gets alone."""
    items = []
    for seed in (2, 0, 1):
        mesh = syn.box_mesh(np.linspace(-0.2, 1, 5), [0, 0.05, 0.12, 0.3], bc=dict(xmin=1, xmax=2, ymin=4, ymax=1))
        o = syn.uniform_orders(mesh["K"], 2, 3)
        prm = syn.flow_params(mach=0.3, re=100.0)
        items.append((mesh, o, prm, syn.perturbed_state(mesh, o, prm, seed, amp=0.05)))
    B = dg.Mesh.batch([(m, o, p) for (m, o, p, _) in items]).set_arithmetic("mixed")
    off = B.solve_slices()
    qb = _dev(np.concatenate([q for (*_, q) in items]))
    B.vcycle(qb, None, 1, 1, 2, control=6, eta=1.5)
    qbn = qb.cpu().numpy()
    for k, (m, o, p, q) in enumerate(items):
        qa = _dev(q)
        dg.Mesh(m, o, p).set_arithmetic("mixed").vcycle(qa, None, 1, 1, 2, control=6, eta=1.5)
        assert np.array_equal(qbn[5 * off[k]:5 * off[k + 1]], qa.cpu().numpy()), k


def test_mixed_steady_solve_satisfies_the_fp64_equations(dg):
    """A steady problem whose discrete solution is known (S = A(q*)): the
    mixed form cycles until its FP64 residual is below 1e-10; the oracle's
    FP64 residual of the result is then below that tolerance too (to the
    parity bar).  Its state lies within 1e-10 of max|q*| of q* (the FP64 form:
    1e-12).  The FP64 cycle conserves the discrete totals of a periodic box
    exactly, the FP32 corrections only to rounding, and the totals are a
    direction the residual barely sees (uniform changes of a periodic state);
    the deviation's weighted mean and remainder are printed apart."""
    import torch
    mesh, o, prm, q_star = syn.manufactured_box_4x4x1()
    S = orc.operator_A(mesh, o, prm, q_star)
    q0 = syn.zero_mean_wave(mesh, o, q_star, 11, amp=0.01)
    out = {}
    for arith in ("fp64", "mixed"):
        M = dg.Mesh(mesh, o, prm).set_arithmetic(arith)
        qd, rep = M.solve_steady(_dev(q0), _dev(S), tol=1e-10, max_cycles=3000,
                                 mg=dict(beta1=3, beta2=3, beta_c=10), check_every=10)
        assert rep["status"] == 0, (arith, rep)
        out[arith] = (qd.cpu().numpy(), rep)
    qm = out["mixed"][0]
    ro = orc.residual(mesh, o, prm, qm, S)
    assert np.max(np.abs(ro)) <= 1e-10 + TOL * orc.volume_scale(mesh, o, prm, qm)
    dev64 = np.max(np.abs(out["fp64"][0] - q_star))
    devm = np.max(np.abs(qm - q_star))
    # split the mixed deviation into its per-variable weighted mean and the rest
    D = syn.from_blocked(qm - q_star, o, mesh["dim"])
    W = []
    for e in range(mesh["K"]):  # tensor Gauss weights of the element (equal elements: J drops out)
        w = np.ones(1)
        for d in range(mesh["dim"]):
            w = np.multiply.outer(np.polynomial.legendre.leggauss(int(o[e, d]) + 1)[1], w)
        W.append(w.reshape(-1))
    W = np.concatenate(W)
    mean = D @ W / W.sum()
    rest = np.max(np.abs(D - mean[:, None]))
    print("cycles fp64 / mixed:", out["fp64"][1]["cycles"], out["mixed"][1]["cycles"], "deviation fp64 / mixed:",
          dev64, devm, "mixed mean part:", np.max(np.abs(mean)), "rest:", rest)
    scale = np.max(np.abs(q_star))
    assert dev64 <= 1e-12 * scale and devm <= 1e-10 * scale


def test_mixed_solve_starts_in_the_fas_form_above_mixed_from(dg):
    """dg_solve_params.mixed_from: on a mixed-form mesh, cycles whose last
    checked residual is at least mixed_from run the FP64 FAS cycle.  With a
    threshold below every residual the solve is the FP64 solve, bit for bit
    (same cycles, same state); with 1e-3 it starts in the FAS form, switches
    to the defect correction, and its result satisfies the oracle's FP64
    equations to the tolerance (from a start 20 % away, with full multigrid,
    from which the defect correction alone diverges)."""
    mesh, o, prm, q_star = syn.manufactured_box_4x4x1()
    S = orc.operator_A(mesh, o, prm, q_star)
    q0 = syn.zero_mean_wave(mesh, o, q_star, 11, amp=0.2)
    kw = dict(tol=1e-10, max_cycles=3000, fmg=True, fmg_tol=1e-1, mg=dict(beta1=3, beta2=3, beta_c=10),
              check_every=10)
    A = dg.Mesh(mesh, o, prm)
    qa, ra = A.solve_steady(_dev(q0), _dev(S), **kw)
    B = dg.Mesh(mesh, o, prm).set_arithmetic("mixed")
    qb, rb = B.solve_steady(_dev(q0), _dev(S), mixed_from=1e-300, **kw)
    assert ra["status"] == 0 and rb["cycles"] == ra["cycles"]
    assert np.array_equal(qa.cpu().numpy(), qb.cpu().numpy())
    C = dg.Mesh(mesh, o, prm).set_arithmetic("mixed")
    qc, rc = C.solve_steady(_dev(q0), _dev(S), mixed_from=1e-3, **kw)
    assert rc["status"] == 0, rc
    qcn = qc.cpu().numpy()
    ro = orc.residual(mesh, o, prm, qcn, S)
    D = dg.Mesh(mesh, o, prm).set_arithmetic("mixed")
    _, rd = D.solve_steady(_dev(q0), _dev(S), **kw)
    print("cycles fp64 / switched:", ra["cycles"], rc["cycles"], "defect correction alone:", rd)
    assert np.max(np.abs(ro)) <= 1e-10 + TOL * orc.volume_scale(mesh, o, prm, qcn)

