"""Writes the regression fixtures of this directory from the oracle alone.

All four record what the oracle computes today on one small case: a 2x2x1
periodic box with seeded random orders in [1, 3]^3, a seeded perturbed state
and a seeded source (Mach 0.3, Re 100).  A change to the oracle's arithmetic
shows up as a failing regression test and must be justified by the passage
it follows.

  oracle_residual_box2x2x1.txt  residual S - A(Q) (Sec. 2), element-blocked
  oracle_vcycle_box2x2x1.txt    state after one FAS V-cycle, 1/1/2 sweeps
                                (Algorithm 1)
  oracle_tau_box2x2x1.txt       anisotropic isolated tau table with
                                correction, K x 3 x 16, -1 where not measured
                                (Sec. 3.2.1)
  oracle_adapt_box2x2x1.txt     order map selected from that table with
                                tau_max 10, orders in [1, 6], 3D jump rule
                                (Sec. 3.3.2, Sec. 4.2.1)

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

HEADER = ("2x2x1 periodic box, orders U[1,3]^3 seed 11, state seed 12, source seed 13, Mach 0.3, Re 100 "
          "(written by make_golden.py from the oracle)")
TAU_MAX, N_MIN, N_MAX = 10.0, 1, 6  # the case's tau values are O(1-10): a mixed map


def case():
    from paper_1806_11456_gb300 import synthetic as syn
    mesh = syn.periodic_box(2, 2, 1)
    orders = syn.random_orders(mesh["K"], 3, 1, 3, 11)
    prm = syn.flow_params(mach=0.3, re=100.0)
    q = syn.perturbed_state(mesh, orders, prm, 12, amp=0.02)
    s = syn.random_source(mesh, orders, 13, amp=1e-3)
    return mesh, orders, prm, q, s


def compute():
    """The four oracle outputs of the case, by fixture file name."""
    from oracle import oracle as orc
    mesh, orders, prm, q, s = case()
    tau = orc.tau_estimate(mesh, orders, prm, q, s, dir_mask=7, with_correction=True, isolated=True)
    adapted = orc.adapt_orders(mesh, orders, tau, TAU_MAX, N_MIN, N_MAX, rule="3d")
    return {
        "oracle_residual_box2x2x1.txt": orc.residual(mesh, orders, prm, q, s),
        "oracle_vcycle_box2x2x1.txt": orc.fas_vcycle(mesh, orders, prm, q, s, 1, 1, 2),
        "oracle_tau_box2x2x1.txt": tau.reshape(-1),
        "oracle_adapt_box2x2x1.txt": adapted.reshape(-1).astype(np.float64),
    }


def main():
    for name, values in compute().items():
        np.savetxt(os.path.join(HERE, name), values, fmt="%.17e", header=name[:-4] + ": " + HEADER)


if __name__ == "__main__":
    main()
