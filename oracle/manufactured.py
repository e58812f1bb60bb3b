"""Exact manufactured source for the smooth periodic state of the input
generator (TEST INFRASTRUCTURE, oracle side).

For a steady state q(x, y) the source that makes it an exact solution of
q_t + div(F^a - F^v / Re) = s (Appendix A) is s = div(F^a - F^v / Re)(q).
It is formed here symbolically with sympy (exact derivatives, no finite
differences) from the closed-form fields, and sampled at given points.
"""
from __future__ import annotations

import functools

import numpy as np
import sympy as sp


@functools.lru_cache(maxsize=8)
def _source_functions(phases_key, mach, gamma, re, pr, suth, amp):
    phases = np.array(phases_key).reshape(4, 2, 2)
    x, y = sp.symbols("x y", real=True)

    def g(m):
        return sum(sp.sin(2 * sp.pi * k * x + phases[m, k - 1, 0]) * sp.cos(2 * sp.pi * k * y + phases[m, k - 1, 1])
                   for k in (1, 2))

    rho = 1 + amp * g(0)
    u = 1 + amp * g(1)
    v = amp * g(2)
    w = sp.Integer(0)
    p = (1 + amp * g(3)) / (gamma * mach ** 2)
    E = p / (gamma - 1) + rho * (u ** 2 + v ** 2 + w ** 2) / 2
    T = gamma * mach ** 2 * p / rho
    mu = T ** sp.Rational(3, 2) * (1 + suth) / (T + suth)
    kappa = mu
    vel = [u, v, w]
    X = [x, y]

    def dvel(i, j):  # d v_i / d x_j, z-derivatives vanish
        return sp.diff(vel[i], X[j]) if j < 2 else sp.Integer(0)

    div = dvel(0, 0) + dvel(1, 1) + dvel(2, 2)

    def tau(i, j):
        t = mu * (dvel(i, j) + dvel(j, i))
        if i == j:
            t = t - sp.Rational(2, 3) * mu * div
        return t

    hc = kappa / ((gamma - 1) * pr * mach ** 2)
    # advective and viscous flux columns in x and y
    Fa = [[rho * vel[c], rho * u * vel[c] + (p if c == 0 else 0), rho * v * vel[c] + (p if c == 1 else 0),
           rho * w * vel[c], (E + p) * vel[c]] for c in range(2)]
    Fv = [[0, tau(0, c), tau(1, c), tau(2, c),
           u * tau(0, c) + v * tau(1, c) + w * tau(2, c) + hc * sp.diff(T, X[c])] for c in range(2)]
    src = []
    for comp in range(5):
        s = 0
        for c in range(2):
            s += sp.diff(Fa[c][comp] - Fv[c][comp] / re, X[c])
        src.append(s)
    return [sp.lambdify((x, y), s, "numpy") for s in src]


def source_at(points, phases, mach, gamma, re, pr, suth, amp=0.1):
    """(5, npts) exact source at the points' (x, y)."""
    fns = _source_functions(tuple(np.asarray(phases).ravel().tolist()), float(mach), float(gamma),
                            float(re), float(pr), float(suth), float(amp))
    x, y = points[:, 0], points[:, 1]
    out = np.zeros((5, len(x)))
    for c, f in enumerate(fns):
        out[c] = np.broadcast_to(f(x, y), x.shape)
    return out
