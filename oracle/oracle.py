"""Oracle: plain, slow FP64 CPU reference of the p-multigrid / anisotropic
p-adaptation path.  TEST INFRASTRUCTURE ONLY -- only tests, the smoke check and
the CPU-baseline leg of the benchmark may import it.  It shares no code with
the CUDA library (its residual lives in dg_oracle.c, compiled with gcc).

Sections of the paper each function follows:
  residual / isolated residual   Sec. 2 (weak form, DiscretNSElem), Sec. 3.2.1
  cfl_dt                         Sec. 2 (CFL restrictions)
  rk3_sweep                      Sec. 3.1 (Williamson low-storage RK3 smoother)
  fas_vcycle                     Sec. 3.1, Algorithm 1 (FAS V-cycle), eqs
                                 FAScoarseSource, FASIterError, FASCorrectSol
  level_orders                   Sec. 3.3.3 (high-order coarsening)
  tau_estimate                   Sec. 3.2.1 (TruncError!, AnisTruncError),
                                 Sec. 3.3.1 (anisotropic coarsening)
  adapt_orders                   Sec. 3.3.2 (six-step order selection),
                                 Sec. 4.1.2 / 4.2.1 (order-jump rules)
  tangent_residual, mixed_vcycle the linearised residual b - J(q) dq (Sec. 3.1,
                                 nonlinRes, differentiated along dq) and the
                                 library's mixed-precision defect-correction
                                 cycle built on it; not a method of the paper
                                 but a restatement, for parity, of how the
                                 library splits precision around Algorithm 1
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build_oracle

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.or_residual.argtypes = [ctypes.c_int] * 3 + [_dp, _ip, _ip, _dp, _dp, _dp, _dp, ctypes.c_int]
        L.or_residual.restype = ctypes.c_int
        L.or_gradients.argtypes = [ctypes.c_int] * 3 + [_dp, _ip, _ip, _dp, _dp, _dp]
        L.or_geometry.argtypes = [ctypes.c_int] * 3 + [_dp, _ip, _dp, _dp]
        L.or_node_coords.argtypes = [ctypes.c_int] * 3 + [_dp, _ip, _dp]
        L.or_cfl_dt.argtypes = [ctypes.c_int] * 3 + [_dp, _ip, _dp, _dp]
        L.or_cfl_dt.restype = ctypes.c_double
        L.or_transfer.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _ip, ctypes.c_int, _dp, _dp]
        L.or_gauss.argtypes = [ctypes.c_int, _dp, _dp]
        L.or_lagrange_table.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
        L.or_roe.argtypes = [_dp] * 5
        L.or_adv_flux.argtypes = [_dp] * 4
        L.or_visc_flux.argtypes = [_dp] * 5
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(_dp)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32).ctypes.data_as(_ip)


def nodes_total(orders, dim):
    n = orders.astype(np.int64) + 1
    if dim == 2:
        n[:, 2] = 1
    return int(np.sum(n[:, 0] * n[:, 1] * n[:, 2]))


# ---------------------------------------------------------------------------
# thin wrappers over the C part
# ---------------------------------------------------------------------------
def gauss(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().or_gauss(n, _d(x), _d(w))
    return x, w


def lagrange_at(n, x):
    l, dl = np.zeros(n), np.zeros(n)
    lib().or_lagrange_table(n, float(x), _d(l), _d(dl))
    return l, dl


def residual(mesh, orders, prm, q, s=None, isolated=False):
    """r = S - A(Q) with A = M^{-1} F (or the isolated F-hat); S None = 0."""
    orders = np.ascontiguousarray(orders, dtype=np.int32)
    xmap = np.ascontiguousarray(mesh["xmap"], dtype=np.float64)
    ftab = np.ascontiguousarray(mesh["ftab"], dtype=np.int32)
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.zeros_like(q)
    sp = _d(s) if s is not None else ctypes.cast(None, _dp)
    keep = (xmap, ftab, orders, q, s)
    lib().or_residual(mesh["dim"], mesh["K"], mesh["M"], _d(xmap), _i(ftab), _i(orders), _d(prm),
                      _d(q), sp, r.ctypes.data_as(_dp), int(bool(isolated)))
    del keep
    return r


def operator_A(mesh, orders, prm, q, isolated=False):
    return -residual(mesh, orders, prm, q, None, isolated)


def volume_scale(mesh, orders, prm, q):
    """max |volume term of A(q)|: the magnitude of the operator's terms, the
    scale against which residual differences are measured."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.zeros_like(q)
    lib().or_residual(mesh["dim"], mesh["K"], mesh["M"], _d(mesh["xmap"]), _i(mesh["ftab"]), _i(orders),
                      _d(prm), _d(q), ctypes.cast(None, _dp), r.ctypes.data_as(_dp), 2)
    return float(np.max(np.abs(r)))


def volume_term(mesh, orders, prm, q):
    """The volume term of A(q) alone (M^{-1} of the volume integral)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.zeros_like(q)
    lib().or_residual(mesh["dim"], mesh["K"], mesh["M"], _d(mesh["xmap"]), _i(mesh["ftab"]), _i(orders),
                      _d(prm), _d(q), ctypes.cast(None, _dp), r.ctypes.data_as(_dp), 2)
    return -r


def gradients(mesh, orders, prm, q):
    G = np.zeros((nodes_total(orders, mesh["dim"]), 12))
    lib().or_gradients(mesh["dim"], mesh["K"], mesh["M"], _d(mesh["xmap"]), _i(mesh["ftab"]),
                       _i(orders), _d(prm), _d(q), G.ctypes.data_as(_dp))
    return G


def geometry(mesh, orders):
    Nt = nodes_total(orders, mesh["dim"])
    Ja, J = np.zeros((Nt, 9)), np.zeros(Nt)
    lib().or_geometry(mesh["dim"], mesh["K"], mesh["M"], _d(mesh["xmap"]), _i(orders),
                      Ja.ctypes.data_as(_dp), J.ctypes.data_as(_dp))
    return Ja, J


def node_coords(mesh, orders):
    X = np.zeros((nodes_total(orders, mesh["dim"]), 3))
    lib().or_node_coords(mesh["dim"], mesh["K"], mesh["M"], _d(mesh["xmap"]), _i(orders),
                         X.ctypes.data_as(_dp))
    return X


def cfl_dt(mesh, orders, prm, q):
    return lib().or_cfl_dt(mesh["dim"], mesh["K"], mesh["M"], _d(mesh["xmap"]), _i(orders), _d(prm), _d(q))


def transfer(dim, orders_from, orders_to, vec, nvar=5):
    out = np.zeros(nodes_total(orders_to, dim) * nvar)
    lib().or_transfer(dim, len(orders_from), _i(orders_from), _i(orders_to), nvar, _d(vec),
                      out.ctypes.data_as(_dp))
    return out


def roe(prm, qL, qR, n):
    f = np.zeros(5)
    lib().or_roe(_d(prm), _d(qL), _d(qR), _d(n), f.ctypes.data_as(_dp))
    return f


def adv_flux(prm, q, n):
    f = np.zeros(5)
    lib().or_adv_flux(_d(prm), _d(q), _d(n), f.ctypes.data_as(_dp))
    return f


def visc_flux(prm, q, G, n):
    f = np.zeros(5)
    lib().or_visc_flux(_d(prm), _d(q), _d(G), _d(n), f.ctypes.data_as(_dp))
    return f


# ---------------------------------------------------------------------------
# smoother (Sec. 3.1): Williamson 2N-storage third-order Runge-Kutta
# ---------------------------------------------------------------------------
RK3_A = (0.0, -5.0 / 9.0, -153.0 / 128.0)
RK3_B = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)


def rk3_sweep(mesh, orders, prm, q, s, dt=None):
    """One sweep = one RK3 step of dQ/dt = S - A(Q); dt from the CFL rule at the
    start of the sweep unless given."""
    if dt is None:
        dt = cfl_dt(mesh, orders, prm, q)
    q = q.copy()
    g = np.zeros_like(q)
    for k in range(3):
        r = residual(mesh, orders, prm, q, s)
        g = RK3_A[k] * g + dt * r
        q = q + RK3_B[k] * g
    return q


def smooth(mesh, orders, prm, q, s, sweeps):
    for _ in range(sweeps):
        q = rk3_sweep(mesh, orders, prm, q, s)
    return q


# ---------------------------------------------------------------------------
# multigrid levels (Sec. 3.3.3, high-order coarsening with N_coarse = dN = 1)
# ---------------------------------------------------------------------------
def level_orders(orders, level, dim, direction=None):
    """Orders at multigrid level `level`: each coarsened direction is capped at
    `level` (maximum order at that level); direction=None coarsens all (isotropic)."""
    o = orders.copy()
    dirs = range(dim) if direction is None else [direction]
    for d in dirs:
        o[:, d] = np.minimum(o[:, d], level)
    return o


def n_levels(orders, dim, direction=None):
    dirs = range(dim) if direction is None else [direction]
    return int(max(orders[:, d].max() for d in dirs))


# ---------------------------------------------------------------------------
# FAS V-cycle (Algorithm 1)
# ---------------------------------------------------------------------------
def fas_vcycle(mesh, orders, prm, q, s, beta1, beta2, beta_c, direction=None, coarsest=1, delta_n=1,
               control=0, eta=1.1):
    """One FAS V-cycle from the finest level (orders) down to level `coarsest`,
    the order dropping by delta_n per level (Sec. 3.1 uses 1).

    Follows Algorithm 1 with the sign of eq FASIterError (eps = Q - Q0).  At the
    finest level S is the physical source; below it S = A(Q0) + r (eq
    FAScoarseSource).  The coarsest level runs a single block of beta_c sweeps
    in place of pre + post smoothing.  Returns the new finest-level Q.

    control > 0 applies the residual-based smoothing design of Sec. 3.1.2 on
    every level above the coarsest, with at most `control` blocks per rule:
    pre-smoothing repeats blocks of beta1 sweeps until the level's residual
    is below eta times its restriction to the next coarser level,
    max|r^P| < eta max|I r^P| (P the level, N = P - dN the coarser one, as in
    the FAS equations; eta = 1.1 in the paper), i.e. until what is left is
    mostly representable on the coarser level; post-smoothing repeats blocks
    of beta2 sweeps until max|r| is no larger than it was after the
    pre-smoothing."""
    dim = mesh["dim"]
    top = n_levels(orders, dim, direction)
    seq = [top]
    while seq[-1] - delta_n >= coarsest:
        seq.append(seq[-1] - delta_n)
    lv_orders = {lv: level_orders(orders, lv, dim, direction) for lv in seq}
    below = {seq[k]: seq[k + 1] for k in range(len(seq) - 1)}
    bottom = seq[-1]

    def cycle(level, q, r_or_s, finest):
        o = lv_orders[level]
        if finest:
            S = r_or_s
        else:
            S = operator_A(mesh, o, prm, q) + r_or_s
        q0 = q.copy()
        if level == bottom:
            q = smooth(mesh, o, prm, q, S, beta_c)
        else:
            oc = lv_orders[below[level]]
            blocks = 0
            while True:  # pre-smoothing
                q = smooth(mesh, o, prm, q, S, beta1)
                blocks += 1
                r = residual(mesh, o, prm, q, S)
                rc = transfer(dim, o, oc, r)
                if control <= 0 or blocks >= control or np.max(np.abs(r)) < eta * np.max(np.abs(rc)):
                    break
            r_pre = np.max(np.abs(r))
            qc = transfer(dim, o, oc, q)
            epsc = cycle(below[level], qc, rc, False)
            q = q + transfer(dim, oc, o, epsc)
            blocks = 0
            while True:  # post-smoothing
                q = smooth(mesh, o, prm, q, S, beta2)
                blocks += 1
                if control <= 0 or blocks >= control:
                    break
                if np.max(np.abs(residual(mesh, o, prm, q, S))) <= r_pre:
                    break
        if finest:
            return q
        return q - q0

    return cycle(top, q.copy(), s, True)


# ---------------------------------------------------------------------------
# linearised residual and the mixed-precision defect-correction cycle
# ---------------------------------------------------------------------------
TANGENT_STEP = 1e-4  # finite-difference step, relative to max|q| / max|dq|


def directional_derivative(f, q, dq, step=TANGENT_STEP):
    """d/dh f(q + h dq) at h = 0 by the fourth-order central difference
    (-f(q+2h) + 8 f(q+h) - 8 f(q-h) + f(q-2h)) / (12 h), with h dq a
    relative perturbation of size `step` of q."""
    nq, nd = float(np.max(np.abs(q))), float(np.max(np.abs(dq)))
    if nd == 0.0:
        return np.zeros_like(q)
    h = step * nq / nd
    return (-f(q + 2 * h * dq) + 8 * f(q + h * dq) - 8 * f(q - h * dq) + f(q - 2 * h * dq)) / (12 * h)


def tangent_residual(mesh, orders, prm, q, dq, b=None):
    """b - J(q) dq, J the Jacobian of A at q, by directional differences of
    the residual (b None = 0)."""
    Jdq = directional_derivative(lambda x: operator_A(mesh, orders, prm, x), q, dq)
    return (0.0 if b is None else b) - Jdq


def mixed_vcycle(mesh, orders, prm, q, s, beta1, beta2, beta_c, direction=None, coarsest=1, delta_n=1,
                 control=0, eta=1.1):
    """One defect-correction cycle: r = S - A(q) at the finest level, one
    V-cycle of Algorithm 1's shape (levels, sweeps, RK3 smoother, L2
    restriction and prolongation) on the linearised problem J d = r in which
    level l is linearised at the restriction of q, its right-hand side is the
    restriction of the finer level's linear residual b - J d, and its
    correction starts from 0; then q + d.  The RK3 step of a level comes from
    its linearisation point.  Returns the new q.

    control > 0 applies the residual-based smoothing design of Sec. 3.1.2 to
    the linear residual b - J d of each level above the coarsest, with the
    same rules and block limit as fas_vcycle: pre-smoothing repeats blocks of
    beta1 sweeps until max|b - J d| < eta max|I (b - J d)|, post-smoothing
    repeats blocks of beta2 sweeps until max|b - J d| is no larger than after
    the pre-smoothing.  For a linear operator these are the FAS rules'
    residuals exactly (b - J d = S - A(q0 + d))."""
    dim = mesh["dim"]
    top = n_levels(orders, dim, direction)
    seq = [top]
    while seq[-1] - delta_n >= coarsest:
        seq.append(seq[-1] - delta_n)
    lv_orders = {lv: level_orders(orders, lv, dim, direction) for lv in seq}

    def smooth_linear(o, base, d, b, sweeps):
        dt = cfl_dt(mesh, o, prm, base)
        for _ in range(sweeps):
            g = np.zeros_like(d)
            for k in range(3):
                rk = tangent_residual(mesh, o, prm, base, d, b)
                g = RK3_A[k] * g + dt * rk
                d = d + RK3_B[k] * g
        return d

    def cycle(k, base, b):
        o = lv_orders[seq[k]]
        d = np.zeros_like(base)
        if k + 1 == len(seq):
            return smooth_linear(o, base, d, b, beta_c)
        oc = lv_orders[seq[k + 1]]
        blocks = 0
        while True:  # pre-smoothing
            d = smooth_linear(o, base, d, b, beta1)
            blocks += 1
            rl = tangent_residual(mesh, o, prm, base, d, b)
            rc = transfer(dim, o, oc, rl)
            if control <= 0 or blocks >= control or np.max(np.abs(rl)) < eta * np.max(np.abs(rc)):
                break
        r_pre = np.max(np.abs(rl))
        dc = cycle(k + 1, transfer(dim, o, oc, base), rc)
        d = d + transfer(dim, oc, o, dc)
        blocks = 0
        while True:  # post-smoothing
            d = smooth_linear(o, base, d, b, beta2)
            blocks += 1
            if control <= 0 or blocks >= control:
                break
            if np.max(np.abs(tangent_residual(mesh, o, prm, base, d, b))) <= r_pre:
                break
        return d

    r = residual(mesh, orders, prm, q, s)
    return q + cycle(0, q, r)


# ---------------------------------------------------------------------------
# anisotropic truncation-error estimate (Sec. 3.2.1, 3.3.1)
# ---------------------------------------------------------------------------
NOT_MEASURED = -1.0


def tau_estimate(mesh, orders, prm, q, s, dir_mask=7, with_correction=True, isolated=True):
    """Directional estimates t[e, i, N] = max over nodes and variables of
    |tau_i| at order N_i < P_i in direction i (other directions at P).

    tau_i at level l is  R^l(I q) - I R^P(q)  (with correction) or R^l(I q)
    (without), R = S - A, with I the chained level-by-level L2 restriction in
    direction i only; the source at level l is the chained restriction of S.
    Entries never measured hold -1."""
    dim = mesh["dim"]
    K = mesh["K"]
    Nmax_tab = 16
    t = np.full((K, 3, Nmax_tab), NOT_MEASURED)
    if s is None:
        s = np.zeros_like(q)
    rP = residual(mesh, orders, prm, q, s, isolated)
    for i in range(dim):
        if not (dir_mask >> i) & 1:
            continue
        top = int(orders[:, i].max())
        o_prev, q_l, s_l, r_l = orders, q, s, rP
        for lv in range(top - 1, 0, -1):
            o_l = level_orders(orders, lv, dim, i)
            q_l = transfer(dim, o_prev, o_l, q_l)
            s_l = transfer(dim, o_prev, o_l, s_l)
            r_l = transfer(dim, o_prev, o_l, r_l)
            tau = residual(mesh, o_l, prm, q_l, s_l, isolated)
            if with_correction:
                tau = tau - r_l
            nn = (o_l.astype(np.int64) + 1)
            if dim == 2:
                nn[:, 2] = 1
            nn = nn[:, 0] * nn[:, 1] * nn[:, 2]
            off = np.concatenate([[0], np.cumsum(5 * nn)])
            for e in range(K):
                if orders[e, i] > lv:
                    t[e, i, lv] = np.max(np.abs(tau[off[e]:off[e + 1]]))
            o_prev = o_l
    return t


# ---------------------------------------------------------------------------
# p-adaptation (Sec. 3.3.2) and order-jump rules (Sec. 4.1.2, 4.2.1)
# ---------------------------------------------------------------------------
def _fit_directional(tvals, P):
    """Linear-log least-squares fit of log10 t against N over the measured
    orders 1..P-1.  Returns a function N -> t_i(N): measured values below P,
    the extrapolation 10**(a + b N) at and above P.  With fewer than two points
    or a non-negative slope the extrapolated value is t(P-1) (non-decaying);
    with no measurement at all it is 0."""
    xs, ys = [], []
    for N in range(1, P):
        v = tvals[N]
        if v > 0.0:
            xs.append(float(N))
            ys.append(math.log10(v))
    slope = intercept = None
    if len(xs) >= 2:
        xm = sum(xs) / len(xs)
        ym = sum(ys) / len(ys)
        sxx = sum((x - xm) * (x - xm) for x in xs)
        sxy = sum((x - xm) * (y - ym) for x, y in zip(xs, ys))
        b = sxy / sxx
        if b < 0.0:
            slope, intercept = b, ym - b * xm
    last = tvals[P - 1] if P >= 2 and tvals[P - 1] >= 0.0 else 0.0

    def f(N):
        if N < P:
            return tvals[N] if tvals[N] >= 0.0 else 0.0
        if slope is None:
            return last
        return 10.0 ** (intercept + slope * N)

    return f


def select_orders(ttab, P, tau_max, n_min, n_max, dim, cap=None):
    """Steps 3-6 of the order selection for one element.  P: the element's
    reference orders (3,), ttab: (3, >=n_max+1) directional table.
    Candidates N_i in [n_min, min(n_max, cap)]; tau(N) = sum_i t_i(N_i).
    Step 4 searches the inner map (all N_i < P_i) first; steps 5/6 the full
    map with extrapolated values; if nothing reaches tau < tau_max, N_i = the
    upper bound in every direction.  Among candidates the fewest degrees of
    freedom win, then the smaller tau, then the lexicographically smaller
    (N1, N2, N3)."""
    hi = n_max if cap is None else min(n_max, cap)
    fits = [_fit_directional(ttab[i], int(P[i])) for i in range(dim)]

    def tau_of(N):
        s = 0.0
        for i in range(dim):
            s += fits[i](N[i])
        return s

    def best(ranges):
        bestkey, bestN = None, None
        for N in _product(ranges):
            tv = tau_of(N)
            if not (tv < tau_max):
                continue
            dof = 1
            for i in range(dim):
                dof *= N[i] + 1
            key = (dof, tv, tuple(N))
            if bestkey is None or key < bestkey:
                bestkey, bestN = key, N
        return bestN

    inner = [range(n_min, min(int(P[i]) - 1, hi) + 1) for i in range(dim)]
    N = best(inner) if all(len(r) > 0 for r in inner) else None
    if N is None:
        N = best([range(n_min, hi + 1) for _ in range(dim)])
    if N is None:
        N = [hi] * dim
    out = [0, 0, 0]
    for i in range(dim):
        out[i] = int(N[i])
    return out


def _product(ranges):
    if not ranges:
        yield []
        return
    for v in ranges[0]:
        for rest in _product(ranges[1:]):
            yield [v] + rest


def face_direction_map(f_self, f_nb, o):
    """For a face seen from element A (face f_self) and its neighbour B (face
    f_nb, orientation o from A's face frame to B's), the direction of B that
    corresponds to each reference direction of A."""
    dA, dB = f_self // 2, f_nb // 2
    tA = [t for t in range(3) if t != dA]
    tB = [t for t in range(3) if t != dB]
    m = {dA: dB}
    if o & 1:
        m[tA[0]], m[tA[1]] = tB[1], tB[0]
    else:
        m[tA[0]], m[tA[1]] = tB[0], tB[1]
    return m


def limit_jumps(mesh, orders, rule="2d", conform_tag=None):
    """Order-jump fix-point: only raises orders.  rule '2d': |N+ - N-| <= 1;
    rule '3d': N+ >= floor(2/3 N-).  Directions are matched through each face's
    orientation.  conform_tag: faces between two elements that both touch a
    boundary of that tag get equal orders in every direction.  Jacobi sweeps
    (all raises computed from the previous map) until nothing changes."""
    dim = mesh["dim"]
    ftab = mesh["ftab"]
    K = mesh["K"]
    o = orders.copy()
    touches = np.zeros(K, dtype=bool)
    if conform_tag is not None:
        for e in range(K):
            for f in range(2 * dim):
                if ftab[e, f, 0] < 0 and ftab[e, f, 3] == conform_tag:
                    touches[e] = True
    for _ in range(10000):
        new = o.copy()
        for e in range(K):
            for f in range(2 * dim):
                nb, fn, ori, _ = ftab[e, f]
                if nb < 0:
                    continue
                m = face_direction_map(f, fn, ori)
                for i in range(dim):
                    other = o[nb, m[i]]
                    if rule == "2d":
                        need = other - 1
                    elif rule == "3d":
                        need = (2 * other) // 3
                    else:
                        need = 0
                    if conform_tag is not None and touches[e] and touches[nb]:
                        need = max(need, other)
                    if need > new[e, i]:
                        new[e, i] = need
        if np.array_equal(new, o):
            return o
        o = new
    raise RuntimeError("order-jump fix-point did not settle")


def adapt_orders(mesh, P, ttab, tau_max, n_min, n_max, cap=None, rule="2d", conform_tag=None):
    """Per-element selection followed by the order-jump fix-point."""
    dim = mesh["dim"]
    K = mesh["K"]
    new = np.zeros((K, 3), dtype=np.int32)
    for e in range(K):
        new[e] = select_orders(ttab[e], P[e], tau_max, n_min, n_max, dim, cap)
    if rule is None and conform_tag is None:
        return new
    return limit_jumps(mesh, new, rule, conform_tag)


# ---------------------------------------------------------------------------
# steady driver (Sec. 3.1.1 FMG and V-cycling, Sec. 3.3.2 adaptation)
# ---------------------------------------------------------------------------
def _max_norm(mesh, orders, prm, q, s):
    return float(np.max(np.abs(residual(mesh, orders, prm, q, s))))


def _cycle_until(mesh, orders, prm, q, s, mg, target, cap):
    """V-cycles until max|r| < target or `cap` cycles.  Returns (q, cycles,
    final norm, status) with status 'ok', 'cap' or 'diverged'."""
    rn = _max_norm(mesh, orders, prm, q, s)
    c = 0
    while True:
        if rn < target:
            return q, c, rn, "ok"
        if not math.isfinite(rn):
            return q, c, rn, "diverged"
        if c >= cap:
            return q, c, rn, "cap"
        q = fas_vcycle(mesh, orders, prm, q, s, mg["beta1"], mg["beta2"], mg["beta_c"],
                       direction=None if mg.get("direction", -1) < 0 else mg["direction"],
                       coarsest=mg.get("coarsest", 1), delta_n=mg.get("delta_n", 1))
        c += 1
        rn = _max_norm(mesh, orders, prm, q, s)


def solve_steady(mesh, orders, prm, q, s, tol, max_cycles, mg, fmg=False, fmg_tol=1e-1, adapt=None):
    """FMG start from order 1 (each level cycled to fmg_tol, then interpolated
    up), V-cycles at the reference orders to tol -- or, with `adapt` (dict of
    select/jump parameters), to tau_max/10, then the isolated tau estimate,
    the new order map, the state transferred, and V-cycles to tol.
    Returns (orders, q, report)."""
    dim = mesh["dim"]
    rep = dict(cycles=0, fmg_cycles=0, adapted=0)
    status = "ok"
    if fmg:
        top = int(orders[:, :dim].max())
        prev_o, prev_q = None, None
        for lv in range(1, top):
            o = level_orders(orders, lv, dim)
            ql = transfer(dim, orders, o, q) if prev_o is None else transfer(dim, prev_o, o, prev_q)
            sl = transfer(dim, orders, o, s) if s is not None else None
            ql, c, rn, st = _cycle_until(mesh, o, prm, ql, sl, mg, fmg_tol, max_cycles)
            rep["cycles"] += c
            rep["fmg_cycles"] += c
            if st == "diverged":
                status = st
                break
            prev_o, prev_q = o, ql
        if status == "ok" and prev_o is not None:
            q = transfer(dim, prev_o, orders, prev_q)
    rn = float("nan")
    if status == "ok":
        target = adapt["tau_max"] * adapt.get("ref_factor", 0.1) if adapt else tol
        q, c, rn, status = _cycle_until(mesh, orders, prm, q, s, mg, target, max_cycles)
        rep["cycles"] += c
    if status == "ok" and adapt:
        rep["adapted"] = 0
        stages = list(adapt.get("stages", ()))
        nst = max(1, len(stages))
        rule = {0: None, 1: "2d", 2: "3d"}[adapt.get("jump_rule", 0)]
        for st_i in range(nst):
            if st_i > 0:  # each stage starts from a state converged to tau_max/10
                q, c, rn, status = _cycle_until(mesh, orders, prm, q, None, mg, adapt["tau_max"] * adapt.get("ref_factor", 0.1),
                                                max_cycles)
                rep["cycles"] += c
                if status != "ok":
                    break
            rep["rnorm_adapt"] = rn
            t = tau_estimate(mesh, orders, prm, q, None, dir_mask=(1 << dim) - 1)
            cap = stages[st_i] if stages else (adapt.get("cap") or None)
            last = True
            if stages:
                free = adapt_orders(mesh, orders, t, adapt["tau_max"], adapt["n_min"], adapt["n_max"], cap=None,
                                    rule=rule)
                last = st_i == nst - 1 or int(free.max()) <= cap
            new = adapt_orders(mesh, orders, t, adapt["tau_max"], adapt["n_min"], adapt["n_max"], cap=cap, rule=rule)
            if not np.array_equal(new, orders):
                q = transfer(dim, orders, new, q)
                orders = new
                rep["adapted"] += 1
            if last:
                break
        if status == "ok":
            q, c, rn, status = _cycle_until(mesh, orders, prm, q, None, mg, tol, max_cycles)
            rep["cycles"] += c
    rep["rnorm"] = rn
    rep["status"] = status
    return orders, q, rep
