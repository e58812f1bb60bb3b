"""Writes the regression fixtures of this directory from the oracle alone.

oracle_residual_box2x2x1.txt: the oracle's residual S - A(Q) (Sec. 2) on a
2x2x1 periodic box with seeded random orders in [1, 3]^3, a seeded
perturbed state and a seeded source (Mach 0.3, Re 100), one value per line
in the element-blocked layout.  It records what the oracle computes today; a
change to the oracle's arithmetic shows up as a failing regression test and
must be justified by the passage it follows.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def case():
    from paper_1806_11456_gb300 import synthetic as syn
    mesh = syn.periodic_box(2, 2, 1)
    orders = syn.random_orders(mesh["K"], 3, 1, 3, 11)
    prm = syn.flow_params(mach=0.3, re=100.0)
    q = syn.perturbed_state(mesh, orders, prm, 12, amp=0.02)
    s = syn.random_source(mesh, orders, 13, amp=1e-3)
    return mesh, orders, prm, q, s


def main():
    from oracle import oracle as orc
    mesh, orders, prm, q, s = case()
    r = orc.residual(mesh, orders, prm, q, s)
    np.savetxt(os.path.join(HERE, "oracle_residual_box2x2x1.txt"), r, fmt="%.17e",
               header="oracle residual S - A(Q), 2x2x1 periodic box, orders U[1,3]^3 seed 11, state seed 12, "
                      "source seed 13, Mach 0.3, Re 100 (written by make_golden.py)")


if __name__ == "__main__":
    main()
