"""A small, fixed invocation of the residual for profilers (ncu): builds the
library, creates one workload and evaluates its residual `--warmup` + `--iters`
times on the current CUDA device, then exits.  Nothing is timed here.

    python -m paper_1806_11456_gb300.profile_case flat_plate --warmup 2 --iters 3
    python -m paper_1806_11456_gb300.profile_case box3d --arith df32

Workloads: flat_plate (60 x 24 stretched plate, N = 7, 92,160 nodes, the
bench's headline mesh); box3d (periodic 48^3 affine hexes, N = 3, 7.1 M nodes,
283 MB of state: larger than L2); sphere (13,824 quadratic hexes, orders
U[1,6]^3); tiny3d (periodic 3^3 box, N = 2: a serving-sized request).
--vcycles runs V-cycles instead of residuals.  --arith mixed evaluates the
linearised residual J(q) q in FP32 tangent arithmetic (the operator kernels of
the mixed-precision cycle) in place of the residual.
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def workload(name):
    from paper_1806_11456_gb300 import synthetic as syn
    if name == "flat_plate":
        mesh = syn.flat_plate_mesh()
        prm = syn.flow_params(mach=0.2, re=1e5)
        o = syn.uniform_orders(mesh["K"], 2, 7)
        return mesh, o, prm, syn.perturbed_state(mesh, o, prm, seed=7, amp=0.01)
    if name == "box3d":
        mesh = syn.periodic_box(48, 48, 48)
        prm = syn.flow_params(mach=0.3, re=100.0)
        o = syn.uniform_orders(mesh["K"], 3, 3)
        return mesh, o, prm, None
    if name == "tiny3d":
        mesh = syn.periodic_box(3, 3, 3)
        prm = syn.flow_params(mach=0.3, re=100.0)
        o = syn.uniform_orders(mesh["K"], 3, 2)
        return mesh, o, prm, syn.manufactured_state(mesh, o, 1, prm[2], prm[0], amp=0.05)
    if name == "sphere":
        mesh, o, prm = syn.sphere_shell_13824()
        return mesh, o, prm, syn.smooth_state(mesh, o, prm, 5, amp=0.02)
    raise SystemExit(f"unknown workload {name}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["flat_plate", "box3d", "sphere", "tiny3d"])
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--arith", default="fp64", choices=["fp64", "df32", "mixed"])
    ap.add_argument("--vcycles", action="store_true",
                    help="run V-cycles (3/3/10 sweeps, graph replay) instead of residual evaluations")
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1806_11456_gb300 import dg
    mesh, o, prm, q = workload(args.workload)
    M = dg.Mesh(mesh, o, prm).set_arithmetic(args.arith)
    if q is None:  # large box: freestream times (1 + 1% seeded noise), made on the device
        n, _ = M.layout()
        gen = torch.Generator(device="cuda")
        gen.manual_seed(3)
        qinf = torch.tensor(np.asarray(prm[7:12]), device="cuda", dtype=torch.float64)
        nn = int(np.prod(o[0, :mesh["dim"]] + 1))
        qd = (qinf.view(1, 5, 1) * (1 + 0.01 * (2 * torch.rand(mesh["K"], 5, nn, device="cuda", dtype=torch.float64,
                                                                 generator=gen) - 1))).reshape(-1)
    else:
        qd = torch.tensor(q, device="cuda")
    r = torch.empty_like(qd)

    def one():
        if args.vcycles:
            M.vcycle(qd, None, beta1=3, beta2=3, beta_c=10, graph=True)
        elif args.arith == "mixed":
            M.residual_tangent(qd, qd, None, r=r)
        else:
            M.residual(qd, None, r=r)

    for _ in range(args.warmup):
        one()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.iters):
        one()
    e1.record()
    torch.cuda.synchronize()
    what = "V-cycle" if args.vcycles else "residual"
    print(f"{args.workload} {args.arith}: {e0.elapsed_time(e1) / max(args.iters, 1):.4f} ms per {what} "
          f"(mean of {args.iters}, CUDA events, after {args.warmup} warm-up)")


if __name__ == "__main__":
    main()
