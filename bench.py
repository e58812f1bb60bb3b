"""Benchmark of the DGSEM p-multigrid hot path on GB300.

Workload: the 2D flat-plate boundary-layer mesh, 60 x 24 elements stretched
toward the wall (first cell 1e-3, ratio 1.15), uniform order N = 7
(92,160 Gauss nodes, 460,800 degrees of freedom), Mach 0.2, Re_L 1e5, FP64.
A step is one pass of the whole path on that state: one FAS V-cycle N = 7
-> 1 (Algorithm 1; RK3 smoothing 2 pre / 2 post / 4 coarsest sweeps, L2
transfers, CFL step per sweep), the anisotropic isolated tau estimate in both
directions (chained restrictions, 6 levels each), and the order adaptation
(tau_max 1e-4, orders in [1, 7], jump limit 1).  The state is freestream plus
a seeded 1% perturbation.

metric  DOF-residual evaluations per second: the sum over every operator
        evaluation issued in a step (smoother stages, FAS sources, restricted
        residuals, tau residuals) of that level's degrees of freedom (5 x
        nodes), divided by the step's device time.
e2e     the same through the C ABI with the state in pinned host memory:
        host->device copy in, step, device->host copy out, all timed.
L2      a 512 MB buffer is written between timed steps (the state fits in L2).

--impl reference times the oracle (the plain FP64 CPU implementation) on the
host cores on the same workload and metric: a step is one full-operator
residual evaluation of the flat-plate state.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "flat_plate_2d_60x24_N7"
METRIC = "DOF residual evals/s"
CYCLE = dict(beta1=2, beta2=2, beta_c=4)
TAU_MAX = 1e-4
FP64_PEAK_TFLOPS = 4 * 152 * 2.070e9 / 1e12  # 2 DFMA/clk/SM x 152 SMs at 2070 MHz


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _hbm_peak()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--c2-solve", action="store_true",
                    help="also run the steady driver with adaptation on the flat plate (several minutes)")
    ap.add_argument("--serving-large", action="store_true",
                    help="also serve larger requests (1e4-5e4 DOF, random order maps; a few minutes)")
    ap.add_argument("--steady-adapt", action="store_true",
                    help="also run the whole steady driver with adaptation to 1e-10 on the 24x8 plate, FP64 and "
                         "mixed (several minutes)")
    ap.add_argument("--mg-compare", type=int, default=0, metavar="CYCLES",
                    help="also compare isotropic and anisotropic V-cycles on the flat plate for CYCLES cycles "
                         "(about a second per cycle; off by default)")
    return ap.parse_args()


def workload():
    from paper_1806_11456_gb300 import synthetic as syn
    mesh = syn.flat_plate_mesh()
    prm = syn.flow_params(mach=0.2, re=1e5)
    orders = syn.uniform_orders(mesh["K"], 2, 7)
    q = syn.perturbed_state(mesh, orders, prm, seed=7, amp=0.01)
    return mesh, prm, orders, q


def base_config(mesh, orders):
    nodes = int(np.sum((orders[:, 0] + 1) * (orders[:, 1] + 1)))
    return {"workload": WORKLOAD, "elements": int(mesh["K"]), "N": 7, "nodes": nodes, "dof": 5 * nodes,
            "mach": 0.2, "re": 1e5, "step": "V-cycle 7->1 (b1=2,b2=2,bc=4) + tau (2 dirs) + adapt",
            "l2": "flushed between steps (512 MB write)"}


def tau_dof_evals(orders, dim):
    """DOFs of the operator evaluations of one tau estimate: the reference
    residual plus one per directional level below the top."""
    def nodes(o):
        n = o[:, :dim] + 1
        return int(np.sum(np.prod(n, axis=1)))
    total = nodes(orders)
    for i in range(dim):
        for lv in range(int(orders[:, i].max()) - 1, 0, -1):
            o = orders.copy()
            o[:, i] = np.minimum(o[:, i], lv)
            total += nodes(o)
    return 5.0 * total


def volume_flops_per_node(dim, n, affine):
    """Algorithmic FP64 flops per node of the volume kernel (FMA = 2, a
    division or square root 1), n nodes per direction.

    3D, per direction: BR1 gradient contraction 27 n (general metrics: 3
    metric products + 12 FMA per point) or 8 n + 24 (affine: 4 FMA per
    point, then the 12-term metric product once); lifting of U* 54 (general:
    two faces, 3 metric products + 12 FMA each) or 16 (affine: the two faces'
    U* join the contraction); gradient face traces 48 (12 values); nodal
    viscous + advective contravariant fluxes 68; divergence 10 n; and per
    node primitives, p, viscosity and the 1/J scalings 34.

    2D (one-element-thick extrusion: z-derivatives and the z-components of
    the in-plane metrics are zero and left out), per direction: contraction
    8 n + 16 (affine: 8-term metric product) or 18 n (general); lifting 16
    or 36; gradient face traces 32 (8 values); nodal fluxes 53 (viscous flux
    32, normal velocity 3, five flux components 18); divergence 10 n; per
    node primitives 14, p and viscosity 7, 1/J scaling of 8 values 8."""
    if dim == 2:
        grad = (8 * n + 16) if affine else 18 * n
        lift = 16 if affine else 36
        return 29 + 2 * (grad + lift + 32 + 53 + 10 * n)
    grad = (8 * n + 24) if affine else 27 * n
    lift = 16 if affine else 54
    return 34 + dim * (grad + 10 * n + lift + 48 + 68)


class ClockSampler:
    def __init__(self):
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except FileNotFoundError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self, gpu_index=0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r for r in self.samples if len(r) >= 9 and r[0] == str(gpu_index)]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, rank):
    if rank != 0:
        return
    from oracle import oracle as orc
    mesh, prm, orders, q = workload()
    dof = 5.0 * orc.nodes_total(orders, 2)
    for _ in range(args.warmup):
        orc.residual(mesh, orders, prm, q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.residual(mesh, orders, prm, q)
    dt = time.perf_counter() - t0
    v = dof * args.steps / dt
    cfg = base_config(mesh, orders)
    cfg["step"] = "one full-operator residual evaluation (oracle)"
    cfg.pop("l2", None)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DOF/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfg,
           "cpu_baseline": {"value": v, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} oracle residual evaluations of the full workload"},
           "e2e": {"value": v, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def steady_problem(dg, torch, dev, mesh, o, prm, q_target, seed, amp=0.01):
    """A steady problem whose discrete solution is q_target: S = A(q_target),
    evaluated by the library (the residual with no source is -A), and a
    start q_target plus a smooth zero-mean wave (synthetic.zero_mean_wave).
    Per-node noise as the start does not converge to 1e-10 with the
    fixed-count cycle on these boxes (it stalls near 1e-5), a smooth
    perturbation does in a few hundred cycles."""
    from paper_1806_11456_gb300 import synthetic as syn
    M = dg.Mesh(mesh, o, prm)
    r = M.residual(torch.tensor(q_target, device=dev))
    S = (-r).cpu().numpy()
    return S, syn.zero_mean_wave(mesh, o, q_target, seed, amp)


def cycle_to_tolerance(dg, torch, dev, mesh, o, prm, q0, S, arith, mg, tol, max_cycles, q_star=None):
    """Repeated V-cycles from q0 until max|S - A(q)| < tol (checked every 10
    cycles, and at the start), timed on the host with the device
    synchronised on both sides.  With mg["control"] = 0 the cycles replay a
    CUDA graph; with control > 0 the paper's residual-based smoothing rules
    decide the sweep counts on the host."""
    M = dg.Mesh(mesh, o, prm).set_arithmetic(arith)
    qd = torch.tensor(q0, device=dev)
    sd = torch.tensor(S, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k, evals = 0, 0
    rn = M.residual(qd, sd, norm=True)[1]
    while rn >= tol and k < max_cycles and np.isfinite(rn):
        evals += M.vcycle(qd, sd, graph=not mg.get("control", 0), **mg)["residual_evals"]
        k += 1
        if k % 10 == 0:
            rn = M.residual(qd, sd, norm=True)[1]
    torch.cuda.synchronize()
    out = {"seconds": time.perf_counter() - t0, "cycles": k, "final_rnorm": rn, "converged": rn < tol,
           "operator_evals_per_cycle": evals / max(k, 1)}
    if q_star is not None:
        out["max_dev_from_q_star"] = float(np.max(np.abs(qd.cpu().numpy() - q_star)))
    return out


def time_to_tolerance(dg, torch, dev, tol=1e-10, max_cycles=3000):
    """Time to max|r| < tol of a steady problem on the 4x4x1 periodic unit box
    (N = 3, Mach 0.3, Re 100) whose discrete solution is the manufactured
    field: S = A(q*), start q* plus a 1% smooth zero-mean wave; repeated
    V-cycles 3 -> 1 (3/3/10 sweeps), a residual check every 10 cycles; FP64,
    double-float and the mixed form (FP64 residual, FP32 tangent-linear
    correction cycle), with fixed sweep counts (CUDA graphs) and with the
    residual-based smoothing control of Sec. 3.1.2 (at most 10 blocks,
    eta 1.1)."""
    from paper_1806_11456_gb300 import synthetic as syn
    mesh, o, prm, q_star = syn.manufactured_box_4x4x1()
    S, q0 = steady_problem(dg, torch, dev, mesh, o, prm, q_star, seed=11)
    out = {"workload": "periodic box 4x4x1, N=3, S = A(q*) with q* the manufactured field, start q* + 1% smooth zero-mean wave",
           "tol": tol, "cycle": "V 3->1, 3/3/10 sweeps, graph replay, norm every 10 cycles"}
    fixed = dict(beta1=3, beta2=3, beta_c=10)
    for arith in ("fp64", "df32", "mixed"):
        out[arith] = cycle_to_tolerance(dg, torch, dev, mesh, o, prm, q0, S, arith, fixed, tol, max_cycles, q_star)
    ctl = dict(fixed, control=10, eta=1.1)
    out["controlled"] = {"cycle": "V 3->1, blocks of 3/3 sweeps (10 at the coarsest) under the smoothing control "
                                  "(at most 10 blocks, eta 1.1), norm every 10 cycles"}
    for arith in ("fp64", "mixed"):
        out["controlled"][arith] = cycle_to_tolerance(dg, torch, dev, mesh, o, prm, q0, S, arith, ctl, tol,
                                                      max_cycles, q_star)
    return out


def time_to_tolerance_plate(dg, torch, dev, tol=1e-10, max_cycles=40000):
    """Time to max|r| < tol on a plate-shaped steady problem, a variant of the
    flat-plate workload that explicit pseudo-time cycles converge: the
    flat-plate boundary conditions on 24 x 8 uniform elements (h = 0.05),
    N = 3, Mach 0.2, Re 1e4, S = A(q*) with q* a boundary-layer-like field,
    start q* + 1 % smooth wave; V-cycles 3 -> 1 (2/2/4 sweeps), residual
    every 10 cycles; FP64 against the mixed form, with fixed sweep counts
    (CUDA graphs) and with the smoothing control (at most 10 blocks,
    eta 1.1).  (The stretched 60 x 24 plate itself does not reach 1e-10 with
    the global time step: its 1e-3 wall cells set the step of the whole
    mesh.)"""
    from paper_1806_11456_gb300 import synthetic as syn
    mesh, o, prm, q_star, q0 = syn.plate_steady_case()
    S = (-dg.Mesh(mesh, o, prm).residual(torch.tensor(q_star, device=dev))).cpu().numpy()
    out = {"workload": "plate-shaped variant: 24x8 uniform elements h=0.05 with the flat-plate boundary conditions, "
                       "N=3, Mach 0.2, Re 1e4, S = A(q*) with q* a boundary-layer-like field, start q* + 1% smooth wave",
           "tol": tol, "cycle": "V 3->1, 2/2/4 sweeps, graph replay, norm every 10 cycles"}
    fixed = dict(beta1=2, beta2=2, beta_c=4)
    for arith in ("fp64", "mixed"):
        out[arith] = cycle_to_tolerance(dg, torch, dev, mesh, o, prm, q0, S, arith, fixed, tol, max_cycles, q_star)
    out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    ctl = dict(fixed, control=10, eta=1.1)
    out["controlled"] = {"cycle": "V 3->1, blocks of 2/2 sweeps (4 at the coarsest) under the smoothing control "
                                  "(at most 10 blocks, eta 1.1), norm every 10 cycles"}
    for arith in ("fp64", "mixed"):
        out["controlled"][arith] = cycle_to_tolerance(dg, torch, dev, mesh, o, prm, q0, S, arith, ctl, tol,
                                                      max_cycles, q_star)
    c = out["controlled"]
    c["speedup_mixed_vs_fp64"] = c["fp64"]["seconds"] / c["mixed"]["seconds"]
    return out


def batched_solves(dg, torch, dev, steps=5):
    """Many independent solves batched into one handle per dimension (one
    launch per kernel over the elements of all its solves, one CUDA graph per
    V-cycle), against the same solves run one at a time, each with its own
    graph, on the same stream.  Workload: 64 solves, half stretched 2D plates
    and half quadratic cubed-sphere shells, 200-4000 elements, orders uniform
    in [1, 8]^dim, Mach in [0.1, 0.4] and Re in [1e2, 1e5] log-uniform,
    freestream start.  A step is one V-cycle 8 -> 1 of every solve."""
    from paper_1806_11456_gb300 import synthetic as syn
    t0 = time.time()
    items = syn.batch_workload_64()
    q_np = [syn.freestream_state(m, o, p) for (m, o, p) in items]
    t_gen = time.time() - t0
    groups = [[k for k in range(len(items)) if items[k][0]["dim"] == d] for d in (2, 3)]
    t0 = time.time()
    handles = [dg.Mesh.batch([items[k] for k in g]) for g in groups]
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    offs = [H.solve_slices() for H in handles]
    q0 = [torch.tensor(np.concatenate([q_np[k] for k in g]), device=dev) for g in groups]
    q = [x.clone() for x in q0]
    stream = torch.cuda.current_stream()

    def timed(fn, n):
        ms, dofs = 0.0, 0.0
        for _ in range(n):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dofs += fn()
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / n, dofs / n

    def batch_step():
        d = 0.0
        for H, x, x0 in zip(handles, q, q0):
            x.copy_(x0)
            d += H.vcycle(x, None, graph=True, **CYCLE)["dof_evals"]
        return d

    for _ in range(2):
        batch_step()
    launches0 = dg.kernel_launches()
    b_ms, b_dofs = timed(batch_step, steps)
    b_launches = (dg.kernel_launches() - launches0) // steps
    batch_once = [x.cpu().numpy() for x in q]
    # the same batched step in the mixed form (FP32 tangent smoothing and
    # coarse operators, FP64 finest residual): config-4 precision
    for H in handles:
        H.set_arithmetic("mixed")
    for _ in range(2):
        batch_step()
    m_ms, m_dofs = timed(batch_step, steps)
    for H in handles:
        H.set_arithmetic("fp64")
    norms = np.concatenate([H.residual_norms(x) for H, x in zip(handles, q)])
    stage = {}
    for d, H, x0 in zip((2, 3), handles, q0):
        prof = H.profile_residual(x0, None, iters=5)
        n_d = int(H.solve_slices()[-1])
        stage[f"{d}d"] = {"nodes": n_d, "stage_ms": prof,
                          "residual_dof_per_s": 5.0 * n_d / (sum(v for k, v in prof.items() if k != "isolated") * 1e-3)}

    # the same solves one at a time
    alone = [dg.Mesh(m, o, p) for (m, o, p) in items]
    qa0 = [torch.tensor(x, device=dev) for x in q_np]
    qa = [x.clone() for x in qa0]

    def seq_step():
        d = 0.0
        for A, x, x0 in zip(alone, qa, qa0):
            x.copy_(x0)
            d += A.vcycle(x, None, graph=True, **CYCLE)["dof_evals"]
        return d

    for _ in range(2):
        seq_step()
    launches0 = dg.kernel_launches()
    ns = max(2, steps // 2)
    s_ms, s_dofs = timed(seq_step, ns)
    s_launches = (dg.kernel_launches() - launches0) // ns
    same = True
    for g, off, qb in zip(groups, offs, batch_once):
        for j, k in enumerate(g):
            same &= bool(np.array_equal(qb[5 * off[j]:5 * off[j + 1]], qa[k].cpu().numpy()))
    nodes = int(sum(off[-1] for off in offs))
    del alone, qa, qa0, handles, q, q0
    torch.cuda.empty_cache()
    return {"workload": "64 solves: 32 stretched 2D plates + 32 quadratic cubed-sphere shells, 200-4000 "
                        "elements, orders U[1,8]^d, Mach U_log[0.1,0.4], Re U_log[1e2,1e5], freestream start",
            "solves": len(items), "handles": "one per dimension (2D: 32 solves, 3D: 32 solves)",
            "elements": int(sum(m["K"] for (m, _, _) in items)), "nodes": nodes,
            "dof": 5 * nodes, "step": "one V-cycle 8->1 (b1=2,b2=2,bc=4) of every solve, CUDA graph per handle",
            "batched": {"value": b_dofs / (b_ms * 1e-3), "unit": "DOF/s", "ms_per_step": b_ms,
                        "launches_per_step": int(b_launches)},
            "batched_mixed": {"value": m_dofs / (m_ms * 1e-3), "unit": "DOF/s", "ms_per_step": m_ms,
                              "note": "one mixed-precision cycle of every solve (a different iteration from the FAS "
                                      "cycle; FP64 finest residual, FP32 tangent smoothing and coarse operators)"},
            "one_at_a_time": {"value": s_dofs / (s_ms * 1e-3), "unit": "DOF/s", "ms_per_step": s_ms,
                              "launches_per_step": int(s_launches)},
            "speedup": s_ms / b_ms, "bitwise_equal_alone": bool(same), "residual_stages": stage,
            "finite": bool(np.all(np.isfinite(norms))), "setup_s": t_setup, "generate_s": t_gen}


def serving_requests(dg, torch, dev, n, seed=4):
    """Steady-solve requests of the serving workload: periodic 2D boxes (2-6
    elements per side, uniform N in {2, 3}) and 3D boxes (3 per side,
    N = 2), Mach U[0.25, 0.4], Re U_log[50, 200] (problems the fixed-count
    FAS cycle converges to 1e-10 in ~10^3 cycles); each with a known discrete
    solution q* (the manufactured field with seeded phases), S = A(q*), start
    q* plus a 1% smooth zero-mean wave."""
    from paper_1806_11456_gb300 import synthetic as syn
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        mach = float(rng.uniform(0.25, 0.4))
        re = float(np.exp(rng.uniform(np.log(50.0), np.log(200.0))))
        prm = syn.flow_params(mach=mach, re=re)
        if k % 4 == 3:
            mesh = syn.periodic_box(3, 3, 3)
            o = syn.uniform_orders(mesh["K"], 3, 2)
        else:
            m = int(rng.integers(2, 7))
            mesh = syn.periodic_box(m, m, 1, dim=2)
            o = syn.uniform_orders(mesh["K"], 2, int(rng.integers(2, 4)))
        q_star = syn.manufactured_state(mesh, o, seed * 1000 + k, mach, prm[0], amp=0.05)
        S, q0 = steady_problem(dg, torch, dev, mesh, o, prm, q_star, seed=k)
        out.append((mesh, o, prm, q0, S))
    return out


def serving(dg, torch, dev, rate=4.0, window=4.0, slots=8, budget=150 << 30, seed=4, control=10, legs=None):
    """Serving loop: requests arrive as a seeded Poisson process (rate per
    second over `window` seconds) and are submitted at their arrival times;
    each is solved to max|r| < 1e-10 by V-cycles 3/3/10 under the paper's
    residual-based smoothing control of Sec. 3.1.2 (at most `control`
    blocks, eta 1.1; sweep counts decided on the host; control = 0 runs fixed
    counts with graph replay instead).  The same arrival stream is served by
    `slots` concurrent slots in double-float arithmetic, by the same slots in
    FP64, by two slots with shared launches (up to 8 compatible requests per
    batch, joining at check points) in FP64 and in the mixed form, and by one
    slot in FP64 (the plain form, one solve at a time; its per-request
    outcomes are listed).  `legs` picks a subset."""
    import threading as th
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * window * 3)))
    arrivals = arrivals[arrivals < window]
    reqs = serving_requests(dg, torch, dev, len(arrivals), seed)
    # at most 4000 cycles: under fixed counts one 720-DOF box diverges after ~3,300
    kw = dict(tol=1e-10, max_cycles=4000, check_every=10,
              mg=dict(beta1=3, beta2=3, beta_c=10, graph=1, control=control, eta=1.1))

    def run(n_slots, arith, batch_max=1, details=False):
        kwa = dict(kw, arith=arith)
        ids = [None] * len(reqs)
        with dg.Server(hbm_budget=budget, slots=n_slots, batch_max=batch_max) as S:
            t0 = time.perf_counter()

            def feed():
                for i, (t, (m, o, p, q0, src)) in enumerate(zip(arrivals, reqs)):
                    dt = t - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                    ids[i] = S.submit(m, o, p, q0=q0, s=src, **kwa)

            feeder = th.Thread(target=feed)
            feeder.start()
            feeder.join()
            S.wait()
            makespan = time.perf_counter() - t0
            infos = [S.info(i) for i in ids]
        lat = np.array([x["t_end"] - x["t_submit"] for x in infos])
        dofs = sum(x["rep"]["dof_evals"] for x in infos)
        ok = sum(1 for x in infos if x["state"] == 0)
        out = {"slots": n_slots, "arith": arith, "batch_max": batch_max, "p50_s": float(np.percentile(lat, 50)),
               "p99_s": float(np.percentile(lat, 99)),
               "mean_s": float(lat.mean()), "makespan_s": makespan, "dof_per_s": dofs / makespan,
               "converged": ok, "cycles_mean": float(np.mean([x["rep"]["cycles"] for x in infos])),
               "max_batch_peers": int(max(x["batch_peers"] for x in infos))}
        if details:
            out["requests"] = [{"dof": 5 * x["rep"]["nodes"], "cycles": x["rep"]["cycles"], "status": x["state"],
                                "rnorm": x["rep"]["rnorm"], "latency_s": float(l)} for x, l in zip(infos, lat)]
        return out

    plan = {"concurrent": (slots, "df32", 1), "concurrent_fp64": (slots, "fp64", 1), "shared_fp64": (2, "fp64", 8),
            "shared_mixed": (2, "mixed", 8), "one_at_a_time": (1, "fp64", 1)}
    res = {k: run(*v, details=(k == "one_at_a_time")) for k, v in plan.items() if legs is None or k in legs}
    nodes = [int(np.sum(np.prod(o[:, :m["dim"]] + 1, axis=1))) for (m, o, *_r) in reqs]
    return {"workload": f"{len(reqs)} requests, Poisson {rate}/s over {window} s: periodic 2D boxes 2-6 per side "
                        "N in {2,3} and 3D boxes 3 per side N = 2, Mach U[0.25,0.4], Re U_log[50,200], "
                        "S = A(q*), to max|r| < 1e-10 (at most 4000 V-cycles 3/3/10, residual checked every 10"
                        + (f", residual-based smoothing control of at most {control} blocks, eta 1.1)" if control
                           else ", fixed sweep counts)"),
            "requests": len(reqs), "dof_range": [5 * min(nodes), 5 * max(nodes)],
            "offered_dof_per_s": 5.0 * sum(nodes) / window,
            "control": control, **res}


def serving_large(dg, torch, dev, rate=2.0, window=4.0, seed=6, control=10, legs=None):
    """Serving with larger requests (opt-in, --serving-large): Poisson
    arrivals (rate per second over `window` seconds) of periodic 2D boxes of
    12-28 elements per side at orders U[2,3]^2 (top order 3) and 3D boxes of
    4 or 8 per side at orders U[1,2]^3 (top order 2), elements of size 0.25
    (the domain grows with the request), Mach U[0.25,0.4], Re U_log[50,200],
    each a steady problem S = A(q*) with q* the manufactured field, started
    at q* plus a 1 % smooth wave, solved to max|r| < 1e-10 (at most 6000
    V-cycles 3/3/10 under the smoothing control of at most `control` blocks,
    residual every 10).  Served one at a time in FP64, by 8 concurrent slots
    in FP64, and by 2 slots with shared launches (up to 8 per batch) in the
    mixed form."""
    from paper_1806_11456_gb300 import synthetic as syn
    import threading as th
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * window * 3)))
    arrivals = arrivals[arrivals < window]
    reqs = []
    for k in range(len(arrivals)):
        mach = float(rng.uniform(0.25, 0.4))
        re = float(np.exp(rng.uniform(np.log(50.0), np.log(200.0))))
        prm = syn.flow_params(mach=mach, re=re)
        if k % 3 == 2:
            n = int(rng.choice([4, 8]))
            mesh = syn.periodic_box(n, n, n, L=(n / 4, n / 4, n / 4))
            o = syn.random_orders(mesh["K"], 3, 1, 2, seed * 100 + k)
            o[0] = 2
        else:
            n = int(rng.choice([12, 16, 20, 24, 28]))
            mesh = syn.periodic_box(n, n, 1, L=(n / 4, n / 4, 1.0), dim=2)
            o = syn.random_orders(mesh["K"], 2, 2, 3, seed * 100 + k)
            o[0, :2] = 3
        q_star = syn.manufactured_state(mesh, o, seed * 1000 + k, mach, prm[0], amp=0.05)
        S, q0 = steady_problem(dg, torch, dev, mesh, o, prm, q_star, seed=k)
        reqs.append((mesh, o, prm, q0, S))
    kw = dict(tol=1e-10, max_cycles=6000, check_every=10,
              mg=dict(beta1=3, beta2=3, beta_c=10, graph=1, control=control, eta=1.1))

    def run(n_slots, arith, batch_max=1):
        ids = [None] * len(reqs)
        with dg.Server(hbm_budget=150 << 30, slots=n_slots, batch_max=batch_max) as S:
            t0 = time.perf_counter()

            def feed():
                for i, (t, (m, o, p, q0, src)) in enumerate(zip(arrivals, reqs)):
                    dt = t - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                    ids[i] = S.submit(m, o, p, q0=q0, s=src, arith=arith, **kw)

            feeder = th.Thread(target=feed)
            feeder.start()
            feeder.join()
            S.wait()
            makespan = time.perf_counter() - t0
            infos = [S.info(i) for i in ids]
        lat = np.array([x["t_end"] - x["t_submit"] for x in infos])
        return {"slots": n_slots, "arith": arith, "batch_max": batch_max, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "makespan_s": makespan,
                "served_dof_evals_per_s": sum(x["rep"]["dof_evals"] for x in infos) / makespan,
                "converged": sum(1 for x in infos if x["state"] == 0),
                "cycles": [x["rep"]["cycles"] for x in infos], "max_batch_peers": max(x["batch_peers"] for x in infos)}

    nodes = [int(np.sum(np.prod(o[:, :m["dim"]] + 1, axis=1))) for (m, o, *_r) in reqs]
    return {"workload": f"{len(reqs)} requests, Poisson {rate}/s over {window} s: periodic 2D boxes 12-28 per side "
                        "orders U[2,3]^2 and 3D boxes 4 or 8 per side orders U[1,2]^3, element size 0.25, "
                        "S = A(q*), to max|r| < 1e-10 (scaled down from 20/s over 120 s and 1e4-2e7 DOF)"
                        + (f"; smoothing control of at most {control} blocks, eta 1.1" if control else ""),
            "dof": [5 * n for n in nodes], "offered_dof_per_s": 5.0 * sum(nodes) / window,
            **{k: run(*v) for k, v in {"one_at_a_time": (1, "fp64"), "concurrent_fp64": (8, "fp64"),
                                        "shared_mixed": (2, "mixed", 8)}.items() if legs is None or k in legs}}


def precision_report(dg, torch, dev):
    """Error of each double-float output against the FP64 path on the
    sphere workload (13,824 quadratic hexes, orders U[1,6]^3, Mach 0.2,
    Re 200; the FP64 path matches the oracle to 1e-12 in the parity tests):
    the residual, one V-cycle 6 -> 1 (1/1/2 sweeps) and the tau table; and
    the mixed form's outputs on the same workload (mixed_precision_report)."""
    from paper_1806_11456_gb300 import synthetic as syn
    mesh, o, prm = syn.sphere_shell_13824()
    q = syn.smooth_state(mesh, o, prm, 5, amp=0.02)
    out = {"workload": "cubed-sphere shell 6x12x12x16 = 13,824 quadratic hexes, orders U[1,6]^3, Mach 0.2, Re 200"}
    M = {a: dg.Mesh(mesh, o, prm).set_arithmetic(a) for a in ("fp64", "df32")}
    r = {a: M[a].residual(torch.tensor(q, device=dev)).cpu().numpy() for a in M}
    out["residual_max_abs_err"] = float(np.max(np.abs(r["df32"] - r["fp64"])))
    out["residual_rel_err"] = out["residual_max_abs_err"] / float(np.max(np.abs(r["fp64"])))
    qs = {}
    for a in M:
        qd = torch.tensor(q, device=dev)
        M[a].vcycle(qd, None, beta1=1, beta2=1, beta_c=2)
        qs[a] = qd.cpu().numpy()
    out["vcycle_state_rel_err"] = float(np.max(np.abs(qs["df32"] - qs["fp64"])) / np.max(np.abs(qs["fp64"])))
    t = {a: M[a].tau_estimate(torch.tensor(q, device=dev), None, dir_mask=7) for a in M}
    meas = t["fp64"] >= 0
    out["tau_rel_err"] = float(np.max(np.abs(t["df32"] - t["fp64"])[meas]) / np.max(t["fp64"][meas]))
    out["tau_measured_same"] = bool(np.array_equal(t["df32"] >= 0, meas))
    out["mixed"] = mixed_precision_report(dg, torch, dev, mesh, o, prm, q, M["fp64"], r["fp64"], t["fp64"])
    return out


def mixed_precision_report(dg, torch, dev, mesh, o, prm, q, M64, r64, t64):
    """Errors of the mixed form's outputs on the sphere workload against the
    FP64 path (which matches the oracle to 1e-12 in the parity tests).  Its
    FP64 roles (residual, tau) must give the FP64 bits.  Its FP32 tangent
    J(q) dq is compared with the fourth-order central difference of the FP64
    residual along dq (the oracle's definition of the derivative, relative
    step 1e-4), per variable relative to max |J dq| of that variable.  One
    mixed V-cycle 6 -> 1 (1/1/2 sweeps) is compared with one FAS V-cycle:
    the two are different iterations, so that difference holds the
    linearisation error besides FP32 rounding."""
    from paper_1806_11456_gb300 import synthetic as syn
    Mm = dg.Mesh(mesh, o, prm).set_arithmetic("mixed")
    qd = torch.tensor(q, device=dev)
    out = {"residual_bitwise": bool(np.array_equal(Mm.residual(qd).cpu().numpy(), r64)),
           "tau_bitwise": bool(np.array_equal(Mm.tau_estimate(qd, None, dir_mask=7), t64))}
    dq = np.random.default_rng(4).normal(size=q.size) * 1e-2 * np.abs(q)
    dqd = torch.tensor(dq, device=dev)
    jdq = -Mm.residual_tangent(qd, dqd).cpu().numpy()
    h = 1e-4 * float(np.max(np.abs(q))) / float(np.max(np.abs(dq)))
    A = lambda x: -M64.residual(torch.tensor(x, device=dev)).cpu().numpy()
    fd = (-A(q + 2 * h * dq) + 8 * A(q + h * dq) - 8 * A(q - h * dq) + A(q - 2 * h * dq)) / (12 * h)
    err = np.abs(syn.from_blocked(jdq - fd, o, 3)).max(axis=1)
    scale = np.abs(syn.from_blocked(fd, o, 3)).max(axis=1)
    out["tangent_rel_err_per_var"] = [float(e / s) for e, s in zip(err, scale)]
    qa, qb = torch.tensor(q, device=dev), torch.tensor(q, device=dev)
    M64.vcycle(qa, None, beta1=1, beta2=1, beta_c=2)
    Mm.vcycle(qb, None, beta1=1, beta2=1, beta_c=2)
    qa, qb = qa.cpu().numpy(), qb.cpu().numpy()
    out["vcycle_diff_rel_to_correction"] = float(np.max(np.abs(qb - qa)) / np.max(np.abs(qa - q)))
    return out


def c2_solve(dg, torch, dev, tau_max=1e-2, tol=1e-6, max_cycles=400):
    """The steady driver with adaptation on the flat plate (60x24, N = 7,
    Mach 0.2, Re 1e5, freestream start): controlled V-cycles (100/100/400,
    eta 1.1, at most 10 blocks per rule) to tau_max/10, the anisotropic
    isolated tau estimate, adaptation to orders in [1, 7]^2 (jump limit
    1), V-cycles on the adapted mesh to tol.  tau_max and tol are looser
    than the paper's 1e-4 and 1e-10 so the run fits in minutes."""
    from paper_1806_11456_gb300 import synthetic as syn
    mesh = syn.flat_plate_mesh()
    prm = syn.flow_params(mach=0.2, re=1e5)
    o = syn.uniform_orders(mesh["K"], 2, 7)
    M = dg.Mesh(mesh, o, prm)
    q = torch.tensor(syn.freestream_state(mesh, o, prm), device=dev)
    t0 = time.perf_counter()
    q2, rep = M.solve_steady(q, None, tol=tol, max_cycles=max_cycles, adapt=True, tau_max=tau_max, n_min=1,
                             n_max=7, jump_rule=1,
                             mg=dict(beta1=100, beta2=100, beta_c=400, control=10, eta=1.1, graph=0))
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    hist = {}
    for nx, ny in M.orders[:, :2]:
        hist[f"{nx},{ny}"] = hist.get(f"{nx},{ny}", 0) + 1
    return {"workload": "flat plate 60x24, N = 7 start, freestream", "tau_max": tau_max, "tol": tol,
            "seconds": secs, "report": rep, "nodes_before": int(mesh["K"] * 64), "orders_histogram": hist}


def steady_adapt_plate(dg, torch, dev, tau_max=1e-4, tol=1e-10, max_cycles=6000, mixed_from=1e-3):
    """The whole steady driver with adaptation (Sec. 3.1.1 full multigrid,
    Sec. 3.3.2) on the physical flat-plate problem (S = 0) of the
    plate-shaped variant's mesh: 24 x 8 uniform elements of size 0.05 with
    the flat-plate boundary conditions, Mach 0.2, Re 1e4, impulsive
    freestream start at N = 4.  Full multigrid to 1e-1 per order, V-cycles
    of 10/10/40 sweeps under the smoothing control (at most 10 blocks,
    eta 1.1) to tau_max/10, the isolated anisotropic tau estimate, orders in
    [1, 6]^2 with the jump limit, V-cycles to tol.  FP64 against the mixed
    form, which runs the FAS cycle while max|r| >= mixed_from (its
    linearisation does not hold at the impulsive start)."""
    from paper_1806_11456_gb300 import synthetic as syn
    mesh = syn.flat_plate_mesh(nx=24, ny=8, dy0=0.05, ratio=1.0)
    prm = syn.flow_params(mach=0.2, re=1e4)
    o = syn.uniform_orders(mesh["K"], 2, 4)
    out = {"workload": "flat plate 24x8 uniform h=0.05, Mach 0.2, Re 1e4, S = 0, freestream start at N = 4",
           "driver": f"FMG (1e-1) -> V 10/10/40 controlled (10 blocks, eta 1.1) to tau_max/10 -> tau -> adapt "
                     f"[1,6]^2 (jump 1) -> V to {tol}", "tau_max": tau_max, "tol": tol}
    for arith in ("fp64", "mixed"):
        M = dg.Mesh(mesh, o, prm).set_arithmetic(arith)
        q = torch.tensor(syn.freestream_state(mesh, o, prm), device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q2, rep = M.solve_steady(q, None, tol=tol, max_cycles=max_cycles, fmg=True, fmg_tol=0.1, adapt=True,
                                 tau_max=tau_max, n_min=1, n_max=6, jump_rule=1, check_every=10,
                                 mixed_from=mixed_from if arith == "mixed" else 0.0,
                                 mg=dict(beta1=10, beta2=10, beta_c=40, control=10, eta=1.1, graph=0))
        torch.cuda.synchronize()
        hist = {}
        for nx, ny in M.orders[:, :2]:
            hist[f"{nx},{ny}"] = hist.get(f"{nx},{ny}", 0) + 1
        out[arith] = {"seconds": time.perf_counter() - t0, "report": rep, "orders_histogram": hist,
                      "mixed_from": mixed_from if arith == "mixed" else None}
    both = out["fp64"]["report"]["status"] == 0 and out["mixed"]["report"]["status"] == 0
    out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"] if both else None
    return out


def mg_compare(dg, torch, dev, cycles):
    """Isotropic vs anisotropic FAS V-cycles (Sec. 3.3.1: coarsening in one
    reference direction per cycle, alternating xi and eta) on the flat plate
    at N = 7 from the freestream start, both with the residual-based
    smoothing control (100/100/400 sweeps, eta = 1.1, at most 10 blocks per
    rule): max|r| after every cycle and the device time."""
    from paper_1806_11456_gb300 import synthetic as syn
    mesh = syn.flat_plate_mesh()
    prm = syn.flow_params(mach=0.2, re=1e5)
    o = syn.uniform_orders(mesh["K"], 2, 7)
    out = {"workload": "flat plate 60x24, N = 7, Mach 0.2, Re 1e5, freestream start",
           "cycle": "V 7->1, 100/100/400 sweeps, control 10 blocks, eta 1.1"}
    for name in ("isotropic", "anisotropic"):
        M = dg.Mesh(mesh, o, prm)
        q = torch.tensor(syn.freestream_state(mesh, o, prm), device=dev)
        hist, secs, dofs = [M.residual(q, norm=True)[1]], [0.0], [0.0]
        t0 = time.perf_counter()
        for c in range(cycles):
            d = -1 if name == "isotropic" else c % 2
            rep = M.vcycle(q, None, 100, 100, 400, direction=d, control=10, eta=1.1)
            torch.cuda.synchronize()
            secs.append(time.perf_counter() - t0)
            dofs.append(dofs[-1] + rep["dof_evals"])
            hist.append(M.residual(q, norm=True)[1])
            if not np.isfinite(hist[-1]):
                break
        out[name] = {"rnorm": hist, "seconds": secs, "dof_evals": dofs}
    return out


def roofline_sweep(dg, torch, dev):
    """Residual stages on 3D periodic affine boxes far larger than L2:
    N = 3, 5, 7 with 64^3, 43^3 and 32^3 elements (16.8-17.2 M Gauss nodes,
    ~0.7 GB of state, ~5x the 129 MB L2).  The state is freestream times
    (1 + 1% seeded uniform noise), generated on the device."""
    from paper_1806_11456_gb300 import synthetic as syn
    out = []
    for N, ne in ((3, 64), (5, 43), (7, 32)):
        mesh = syn.periodic_box(ne, ne, ne)
        orders = syn.uniform_orders(mesh["K"], 3, N)
        prm = syn.flow_params(mach=0.3, re=100.0)
        t0 = time.time()
        M = dg.Mesh(mesh, orders, prm)
        torch.cuda.synchronize()
        setup = time.time() - t0
        nodes, _ = M.layout()
        gen = torch.Generator(device=dev)
        gen.manual_seed(N)
        nn = (N + 1) ** 3
        qinf = torch.tensor(prm[7:12], device=dev, dtype=torch.float64)
        q = (qinf.view(1, 5, 1) * (1.0 + 0.01 * (2 * torch.rand(mesh["K"], 5, nn, device=dev, dtype=torch.float64,
                                                                 generator=gen) - 1))).reshape(-1)
        prof = M.profile_residual(q, None, iters=10)
        res_ms = sum(v for k, v in prof.items() if k != "isolated")
        flops = volume_flops_per_node(3, N + 1, affine=True) * nodes
        tf = flops / (prof["volume"] * 1e-3) / 1e12
        gbs = 80.0 * nodes / (res_ms * 1e-3) / 1e9  # Q in + r out, the residual's algorithmic bytes
        out.append({"N": N, "elements": int(mesh["K"]), "nodes": int(nodes), "setup_s": setup,
                    "residual_ms": res_ms, "residual_dof_per_s": 5.0 * nodes / (res_ms * 1e-3),
                    "k_volume": {"ms": prof["volume"], "tflops": tf, "frac_fp64_nominal": tf / FP64_PEAK_TFLOPS},
                    "residual_gbs": gbs, "residual_frac_hbm": gbs / HBM_PEAK_GBS, "stage_ms": prof})
        del M, q
        torch.cuda.empty_cache()
    return out


def captured_traffic(kernel="k_volume"):
    """DRAM bytes (read + write) per launch of `kernel` on the headline
    workload, from the committed ncu summary, when that capture was taken
    with the current kernel source (its sha256 is recorded beside the
    figure); None otherwise."""
    import hashlib
    import re
    src = os.path.join(ROOT, "paper_1806_11456_gb300", "csrc", "dg_kernels.cu")
    prof = os.path.join(ROOT, "profiles", "k_volume_flat_plate_N7.md")
    try:
        with open(src, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()[:16]
        with open(prof) as f:
            text = f.read()
    except OSError:
        return None
    m = re.search(r"traffic: %s dram_bytes_per_launch=(\d+) kernel_source_sha256=([0-9a-f]+)" % kernel, text)
    return int(m.group(1)) if m and m.group(2) == digest else None


def aggregate_ranks(ms, dofs, world, device):
    """Whole-job figures of replicas: the slowest rank's time (max over
    ranks) and the units all ranks processed over that time.  Every rank
    processes the same work, so the job total is world x the rank's."""
    if world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    return ms, world * dofs / (ms * 1e-3)


def cpu_baseline_sample(mesh, prm, orders, q, budget_s=15.0):
    from oracle import oracle as orc
    dof = 5.0 * orc.nodes_total(orders, 2)
    n, t0 = 0, time.perf_counter()
    while True:
        orc.residual(mesh, orders, prm, q)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 40:
            break
    return {"value": dof * n / el, "unit": "DOF/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} oracle residual evaluations of the full workload, single thread"}


def cpu_baseline_all_cores(budget_s=8.0, timeout_s=120.0):
    """The same oracle sample run as one independent single-thread process per
    host core, all started together: the host's aggregate DOF/s with every
    core busy (memory bandwidth shared as it would be).  The oracle itself is
    unchanged.  None if any process fails or outlives timeout_s (it is then
    killed)."""
    try:
        ncores = len(os.sched_getaffinity(0))
    except AttributeError:
        ncores = os.cpu_count() or 1
    code = ("import json, sys; sys.path.insert(0, %r); import bench; m, p, o, q = bench.workload(); "
            "print(json.dumps(bench.cpu_baseline_sample(m, p, o, q, budget_s=%r)))" % (ROOT, budget_s))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                              text=True, env=env) for _ in range(ncores)]
    deadline = time.monotonic() + timeout_s
    vals, evals = [], 0
    for pr in procs:
        try:
            out, _ = pr.communicate(timeout=max(1.0, deadline - time.monotonic()))
            res = json.loads(out.strip().splitlines()[-1])
            vals.append(float(res["value"]))
            evals += int(res["sample"].split()[0])
        except Exception:
            pr.kill()
            pr.wait()
    if len(vals) != ncores:
        return None
    return {"value": sum(vals), "unit": "DOF/s", "cores": ncores, "kind": "oracle",
            "sample": f"{ncores} concurrent single-thread oracle processes, {evals} residual evaluations of the "
                      f"full workload in all, about {budget_s:g} s each"}


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------
def run_gb300(args, rank, world):
    import torch
    import __graft_entry__ as g
    from paper_1806_11456_gb300 import dg
    g.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    mesh, prm, orders, q_np = workload()
    M = dg.Mesh(mesh, orders, prm)
    stream = torch.cuda.current_stream()
    q0 = torch.tensor(q_np, device=dev)
    q = q0.clone()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tau_dofs = tau_dof_evals(orders, 2)

    def step(qd):
        rep = M.vcycle(qd, None, graph=True, **CYCLE)
        tau = M.tau_estimate(qd, None, dir_mask=3)
        M.adapt(tau, TAU_MAX, 1, 7, jump_rule=1)
        return rep["dof_evals"] + tau_dofs, rep["residual_evals"]

    for _ in range(args.warmup):
        q.copy_(q0)
        step(q)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler()
    clocks.start()
    total_ms, total_dofs = 0.0, 0.0
    launches0 = dg.kernel_launches()
    for _ in range(args.steps):
        q.copy_(q0)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        dofs, evals = step(q)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        total_dofs += dofs
    launches = dg.kernel_launches() - launches0
    torch.cuda.synchronize()
    clk = clocks.stop(dev.index)
    total_ms, value = aggregate_ranks(total_ms, total_dofs, world, dev)

    # where a step's time goes (separate pass, CUDA events around each part)
    parts = {"vcycle": 0.0, "tau": 0.0, "adapt": 0.0}
    for _ in range(10):
        q.copy_(q0)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        M.vcycle(q, None, graph=True, **CYCLE)
        ev[1].record(stream)
        tau = M.tau_estimate(q, None, dir_mask=3)
        ev[2].record(stream)
        M.adapt(tau, TAU_MAX, 1, 7, jump_rule=1)
        ev[3].record(stream)
        ev[3].synchronize()
        for k, name in enumerate(("vcycle", "tau", "adapt")):
            parts[name] += ev[k].elapsed_time(ev[k + 1]) / 10

    # e2e through the C ABI with pinned host buffers
    qh = torch.tensor(q_np).pin_memory()
    qout = torch.empty_like(qh).pin_memory()
    qd = torch.empty_like(q0)
    e2e_ms, e2e_dofs = 0.0, 0.0
    tau_bytes = mesh["K"] * 3 * 16 * 8
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        qd.copy_(qh, non_blocking=True)
        dofs, _ = step(qd)
        qout.copy_(qd, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        e2e_dofs += dofs
    e2e = {"value": world * e2e_dofs / (e2e_ms * 1e-3), "unit": "DOF/s",
           "h2d_bytes_per_step": int(qh.numel() * 8), "d2h_bytes_per_step": int(qout.numel() * 8 + tau_bytes)}

    # dominant kernel: CUDA events around each launch of one residual
    prof = M.profile_residual(q0, None, iters=50)
    stages = {k: v for k, v in prof.items() if k != "isolated"}
    dom = max(stages, key=stages.get)
    nodes = int(np.sum((orders[:, 0] + 1) * (orders[:, 1] + 1)))
    flops = volume_flops_per_node(2, 8, affine=True) * nodes  # the flat-plate mesh is affine
    vol_ms = prof["volume"]
    achieved = flops / (vol_ms * 1e-3) / 1e12
    residual_ms = sum(stages.values())
    rates = dg.measure_fma_rates()  # FP64 / FP32 FMA probe on this device, right after the timed steps
    roof = {"kernel": "k_volume", "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": captured_traffic(),
            "traffic_unit": "DRAM bytes per launch (ncu capture of the current kernel source, else null)",
            "peak_source": "FP64 nominal derived: 2 DFMA/clk/SM x 152 SMs x 2070 MHz",
            "peak_measured": rates["fp64_tflops"], "frac_measured": achieved / rates["fp64_tflops"],
            "peak_measured_source": "dg_measure_fma_rates: independent FP64 FMA chains on every SM, best of 3",
            "fp32_peak_measured": rates["fp32_tflops"],
            "flops_per_launch": flops, "ms_per_launch": vol_ms, "dominant_stage": dom,
            "stage_ms": prof, "residual_dof_per_s": 5.0 * nodes / (residual_ms * 1e-3)}

    # the same residual with element tiles chosen by the autotuner
    MT = dg.Mesh(mesh, orders, prm).set_autotune(True)
    prof_t = MT.profile_residual(q0, None, iters=50)
    autotune = {"tuning": MT.tuning(), "stage_ms": prof_t,
                "volume_speedup": prof["volume"] / prof_t["volume"],
                "residual_dof_per_s": 5.0 * nodes / (sum(v for k, v in prof_t.items() if k != "isolated") * 1e-3)}
    del MT

    # the same step with the operator evaluated in double-float arithmetic
    # (FP32 pairs on the FP32 pipes; parity with the oracle at the same 1e-12
    # bar), reported beside the native FP64 headline
    M.set_arithmetic("df32")
    for _ in range(2):
        q.copy_(q0)
        step(q)
    df_ms, df_dofs = 0.0, 0.0
    for _ in range(args.steps):
        q.copy_(q0)
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dofs, _ = step(q)
        e1.record(stream)
        e1.synchronize()
        df_ms += e0.elapsed_time(e1)
        df_dofs += dofs
    prof_df = M.profile_residual(q0, None, iters=50)
    df_res_ms = sum(v for k, v in prof_df.items() if k != "isolated")
    df32 = {"value": world * df_dofs / (df_ms * 1e-3), "unit": "DOF/s", "ms_per_step": df_ms / args.steps,
            "dtype": "f32x2 (double-float, ~48-bit significand)", "stage_ms": prof_df,
            "residual_dof_per_s": 5.0 * nodes / (df_res_ms * 1e-3),
            "parity": "same 1e-12 bar against the FP64 oracle (tests/test_gpu_parity.py)"}
    # the same step in the mixed form: FP64 finest residual, coarse
    # right-hand sides and tau; FP32 tangent-linear correction cycle
    M.set_arithmetic("mixed")
    for _ in range(2):
        q.copy_(q0)
        step(q)
    mx_ms, mx_dofs = 0.0, 0.0
    for _ in range(args.steps):
        q.copy_(q0)
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dofs, _ = step(q)
        e1.record(stream)
        e1.synchronize()
        mx_ms += e0.elapsed_time(e1)
        mx_dofs += dofs
    prof_mx = M.profile_residual(q0, None, iters=50)
    mx_res_ms = sum(v for k, v in prof_mx.items() if k != "isolated")
    mixed = {"value": world * mx_dofs / (mx_ms * 1e-3), "unit": "DOF/s", "ms_per_step": mx_ms / args.steps,
             "dtype": "f64 finest residual, coarse right-hand sides and tau; f32 tangent smoothing and coarse operators",
             "stage_ms": prof_mx, "tangent_residual_dof_per_s": 5.0 * nodes / (mx_res_ms * 1e-3),
             "note": "a step here is one defect-correction cycle (a different iteration from the FAS cycle of the "
                     "headline); errors against the oracle in tests/test_gpu_mixed.py"}
    M.set_arithmetic("fp64")

    if rank == 0:
        cfg = base_config(mesh, orders)
        out = {"metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": dict(cfg, parallelism=f"replicas{world}"), "e2e": e2e,
               "gpu_launches": None, "roofline": roof, "clocks": clk, "step_ms_parts": parts, "df32": df32,
               "mixed": mixed,
               "autotune": autotune}
        out["gpu_launches"] = int(launches)  # library kernels launched in the timed steps
        out["time_to_tol"] = time_to_tolerance(dg, torch, dev)
        out["time_to_tol_plate"] = time_to_tolerance_plate(dg, torch, dev)
        out["batched"] = batched_solves(dg, torch, dev)
        out["roofline_sweep"] = roofline_sweep(dg, torch, dev)
        out["serving"] = serving(dg, torch, dev)
        out["precision"] = precision_report(dg, torch, dev)
        if args.c2_solve:
            out["c2_solve"] = c2_solve(dg, torch, dev)
        if args.serving_large:
            out["serving_large"] = serving_large(dg, torch, dev)
        if args.steady_adapt:
            out["steady_adapt_plate"] = steady_adapt_plate(dg, torch, dev)
        if args.mg_compare > 0:
            out["mg_compare"] = mg_compare(dg, torch, dev, args.mg_compare)
        out["cpu_baseline"] = cpu_baseline_sample(mesh, prm, orders, q_np) if world == 1 else None
        if world == 1:
            try:
                out["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores()
            except (OSError, ValueError) as exc:  # no process could be started: report why
                out["cpu_baseline"]["all_cores"] = {"unavailable": str(exc)[:200]}
        print(json.dumps(out))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    run_gb300(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
