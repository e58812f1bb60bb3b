"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no arithmetic of the discretisation: it builds hexahedral
mesh topologies (element mapping nodes, face-neighbour tables, boundary tags),
order maps and flow states sampled from closed-form fields.  Both the CUDA
library and the oracle receive these arrays as plain data.

Mesh dictionary keys
--------------------
dim   : 2 or 3 (2 = one-element-thick extrusion, N3 = 0)
K     : element count
M     : mapping order (mapping nodes equispaced on [-1, 1] per direction)
xmap  : float64 (K, (M+1)**dim, 3) mapping nodes, node (a, b[, c]) at
        index (c*(M+1) + b)*(M+1) + a
ftab  : int32 (K, 6, 4) per face (neighbour element or -1, neighbour face,
        orientation code, boundary tag); faces 4, 5 unused in 2D
Faces: 0 xi=-1, 1 xi=+1, 2 eta=-1, 3 eta=+1, 4 zeta=-1, 5 zeta=+1.
Orientation code o maps the first side's face coordinates (s, t) (the two
tangential reference directions in increasing order) to the second side's:
bit0 swaps them, bit1 negates the first, bit2 negates the second.
Boundary tags: 0 interior, 1 freestream, 2 subsonic outflow (far-field
pressure), 3 free-slip, 4 no-slip adiabatic wall.
"""
from __future__ import annotations

import numpy as np

BC_INTERIOR, BC_FREESTREAM, BC_OUTFLOW, BC_SLIP, BC_WALL = 0, 1, 2, 3, 4


def flow_params(mach=0.3, re=100.0, pr=0.72, gamma=1.4, ca=0.2, cnu=0.2):
    """Parameter vector (16 doubles) understood by both implementations.

    0 gamma, 1 Pr, 2 Mach, 3 Re, 4 Sutherland constant (110.4 K / 288.15 K),
    5 C_a, 6 C_nu, 7..11 freestream conserved state (rho=1, |v|=1 along x,
    p = 1/(gamma M^2)), 12..15 reserved.
    """
    p_inf = 1.0 / (gamma * mach * mach)
    qinf = [1.0, 1.0, 0.0, 0.0, p_inf / (gamma - 1.0) + 0.5]
    v = np.zeros(16)
    v[:12] = [gamma, pr, mach, re, 110.4 / 288.15, ca, cnu] + qinf
    return v


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
def box_mesh(xs, ys, zs=None, periodic=(False, False, False), bc=None):
    """Structured box of axis-aligned hexahedra on the tensor grid xs x ys x zs.

    zs=None gives a 2D mesh (dim=2).  ``bc`` maps 'xmin','xmax','ymin','ymax',
    'zmin','zmax' to a boundary tag or to a callable(i_or_j, k) -> tag taking
    the element's tangential indices, for non-periodic sides.
    Elements are numbered e = (k*ny + j)*nx + i.
    """
    xs, ys = np.asarray(xs, float), np.asarray(ys, float)
    dim = 2 if zs is None else 3
    zs = np.asarray([0.0, 1.0] if zs is None else zs, float)
    nx, ny, nz = len(xs) - 1, len(ys) - 1, len(zs) - 1
    if dim == 2:
        nz = 1
    bc = dict(bc or {})
    K = nx * ny * nz
    npe = 8 if dim == 3 else 4
    xmap = np.zeros((K, npe, 3))
    ftab = np.full((K, 6, 4), -1, dtype=np.int32)
    ftab[:, :, 2:] = 0

    def eid(i, j, k):
        return (k * ny + j) * nx + i

    def tag(side, a, b):
        t = bc.get(side, BC_FREESTREAM)
        return int(t(a, b)) if callable(t) else int(t)

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = eid(i, j, k)
                if dim == 3:
                    for c in range(2):
                        for b in range(2):
                            for a in range(2):
                                xmap[e, (c * 2 + b) * 2 + a] = (xs[i + a], ys[j + b], zs[k + c])
                else:
                    for b in range(2):
                        for a in range(2):
                            xmap[e, b * 2 + a] = (xs[i + a], ys[j + b], 0.0)
                # neighbours in each direction
                idx = [i, j, k]
                ncell = [nx, ny, nz]
                for d in range(dim):
                    for side in range(2):
                        f = 2 * d + side
                        nb = list(idx)
                        nb[d] += 1 if side else -1
                        if 0 <= nb[d] < ncell[d] or periodic[d]:
                            nb[d] %= ncell[d]
                            ftab[e, f] = (eid(*nb), 2 * d + (1 - side), 0, BC_INTERIOR)
                        else:
                            name = "xyz"[d] + ("max" if side else "min")
                            tang = [idx[t] for t in range(3) if t != d]
                            ftab[e, f] = (-1, -1, 0, tag(name, tang[0], tang[1]))
    return dict(dim=dim, K=K, M=1, xmap=xmap, ftab=ftab)


def periodic_box(nx, ny, nz, L=(1.0, 1.0, 1.0), dim=3):
    """Fully periodic uniform box [0,Lx]x[0,Ly]x[0,Lz] (2D if dim == 2)."""
    xs = np.linspace(0.0, L[0], nx + 1)
    ys = np.linspace(0.0, L[1], ny + 1)
    zs = np.linspace(0.0, L[2], nz + 1) if dim == 3 else None
    return box_mesh(xs, ys, zs, periodic=(True, True, True))


def flat_plate_mesh(nx=60, ny=24, x0=-0.2, x1=1.0, dy0=1e-3, ratio=1.15):
    """2D flat-plate boundary-layer mesh: uniform in x on [x0, x1] with the
    leading edge x = 0 at a vertex, geometric growth in y from the wall.
    Inflow x = x0 and top: freestream; outflow x = x1: far-field pressure;
    y = 0: free-slip for x < 0, adiabatic no-slip wall for x > 0."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.concatenate([[0.0], np.cumsum(dy0 * ratio ** np.arange(ny))])

    def wall(i, _k):
        return BC_WALL if 0.5 * (xs[i] + xs[i + 1]) > 0.0 else BC_SLIP

    return box_mesh(xs, ys, None, bc=dict(xmin=BC_FREESTREAM, xmax=BC_OUTFLOW,
                                          ymin=wall, ymax=BC_FREESTREAM))


_PERMS = [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)]


def rotate_elements(mesh, seed, frac=0.5):
    """Re-label the local reference axes of a random subset of the elements of
    a 3D mesh (axis permutations and reversals), keeping the geometry.  The
    face table and its orientation codes are rebuilt from the geometry, so
    neighbouring elements see each other through non-trivial orientations;
    boundary faces keep their tags."""
    assert mesh["dim"] == 3
    M = mesh["M"]
    Mp = M + 1
    rng = np.random.default_rng(seed)
    K = mesh["K"]
    xmap = mesh["xmap"].copy()
    for e in range(K):
        if rng.random() >= frac:
            continue
        perm = _PERMS[rng.integers(len(_PERMS))]
        flips = rng.integers(0, 2, size=3)
        old = xmap[e].reshape(Mp, Mp, Mp, 3)  # [c][b][a]
        new = np.empty_like(old)
        for c in range(Mp):
            for b in range(Mp):
                for a in range(Mp):
                    loc = [a, b, c]          # index along the new axes
                    src = [0, 0, 0]
                    for nd in range(3):      # new axis nd is old axis perm[nd]
                        v = loc[nd]
                        src[perm[nd]] = M - v if flips[nd] else v
                    new[c, b, a] = old[src[2], src[1], src[0]]
        # keep a right-handed frame: reverse the first axis if the relabelling
        # inverted the element
        det = np.linalg.det(np.stack([new[0, 0, M] - new[0, 0, 0], new[0, M, 0] - new[0, 0, 0],
                                      new[M, 0, 0] - new[0, 0, 0]]))
        if det < 0:
            new = new[:, :, ::-1].copy()
        xmap[e] = new.reshape(Mp ** 3, 3)
    scale = np.max(np.abs(mesh["xmap"]))
    old_tags = {}
    for e in range(K):
        for f in range(6):
            if mesh["ftab"][e, f, 0] < 0:
                old_tags[_corner_key(_face_corners(mesh["xmap"][e], f, M), scale)] = int(mesh["ftab"][e, f, 3])
    out = dict(mesh)
    out["xmap"] = xmap
    out["ftab"] = _connect_periodic_aware(mesh, xmap, old_tags, scale)
    return out


def _connect_periodic_aware(mesh, xmap, old_tags, scale):
    """Faces of the relabelled mesh.  Geometric matching handles every face
    pair whose corners coincide; a periodic pair (corners one period apart) is
    found through the old table: the relabelled face has the corner key of
    one old face of the same element, whose old neighbour face is located in
    the neighbour's relabelled faces by its corner key."""
    M = mesh["M"]
    K = mesh["K"]
    xold = mesh["xmap"]
    ftab = connect_faces(xmap, M, 3, None, tag_of_key=(old_tags, scale), allow_unmatched_keys=True)
    for e in range(K):
        for f in range(6):
            if ftab[e, f, 0] >= 0 or ftab[e, f, 3] != -99:
                continue
            A = _face_corners(xmap[e], f, M)
            key = _corner_key(A, scale)
            f_old = [g for g in range(6) if _corner_key(_face_corners(xold[e], g, M), scale) == key]
            assert len(f_old) == 1
            nb, g_old = mesh["ftab"][e, f_old[0], 0], mesh["ftab"][e, f_old[0], 1]
            key_nb = _corner_key(_face_corners(xold[nb], g_old, M), scale)
            g_new = [g for g in range(6) if _corner_key(_face_corners(xmap[nb], g, M), scale) == key_nb]
            assert len(g_new) == 1
            B = _face_corners(xmap[nb], g_new[0], M)
            Bs = B + (A.mean(axis=0) - B.mean(axis=0))  # remove the period
            ftab[e, f] = (nb, g_new[0], _orientation(A, Bs, scale), 0)
    return ftab


def _orientation(X, Y, scale):
    for o in range(8):
        ok = True
        for bt in range(2):
            for at in range(2):
                s_, t_ = 2 * at - 1, 2 * bt - 1
                s2, t2 = (t_, s_) if (o & 1) else (s_, t_)
                if o & 2:
                    s2 = -s2
                if o & 4:
                    t2 = -t2
                ia, ib = (s2 + 1) // 2, (t2 + 1) // 2
                if np.linalg.norm(X[bt * 2 + at] - Y[ib * 2 + ia]) > 1e-9 * scale:
                    ok = False
        if ok:
            return o
    raise AssertionError("face corners do not match")


# cube faces of the cubed sphere: outward normal n and tangent axes with e1 x e2 = n
_CUBE_FACES = [((1, 0, 0), (0, 1, 0), (0, 0, 1)), ((-1, 0, 0), (0, 0, 1), (0, 1, 0)),
               ((0, 1, 0), (0, 0, 1), (1, 0, 0)), ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
               ((0, 0, 1), (1, 0, 0), (0, 1, 0)), ((0, 0, -1), (0, 1, 0), (1, 0, 0))]


def cubed_sphere_mesh(nt, nr, r0=1.0, r1=20.0, M=2, inner_tag=BC_WALL, outer_tag=BC_FREESTREAM):
    """Equiangular cubed-sphere shell r0 <= r <= r1: 6 patches of nt x nt
    elements, nr layers with geometric radii r_k = r0 (r1/r0)^(k/nr).  Element
    axes: (xi, eta) along the patch's equiangular angles, zeta outward.  The
    mapping of order M interpolates the exact sphere at the equispaced
    reference nodes; faces are connected by matching corner positions (with
    the orientation codes this implies across cube edges)."""
    Mp = M + 1
    ang = np.linspace(-np.pi / 4, np.pi / 4, nt + 1)
    rad = r0 * (r1 / r0) ** (np.arange(nr + 1) / nr)
    ref = np.linspace(0.0, 1.0, Mp)
    K = 6 * nt * nt * nr
    xmap = np.zeros((K, Mp ** 3, 3))
    e = 0
    for (n, e1, e2) in _CUBE_FACES:
        n, e1, e2 = np.array(n, float), np.array(e1, float), np.array(e2, float)
        for k in range(nr):
            for j in range(nt):
                for i in range(nt):
                    for c in range(Mp):
                        r = rad[k] * (rad[k + 1] / rad[k]) ** ref[c]
                        for b in range(Mp):
                            be = ang[j] + (ang[j + 1] - ang[j]) * ref[b]
                            for a in range(Mp):
                                al = ang[i] + (ang[i + 1] - ang[i]) * ref[a]
                                v = n + np.tan(al) * e1 + np.tan(be) * e2
                                xmap[e, (c * Mp + b) * Mp + a] = r * v / np.linalg.norm(v)
                    e += 1
    ftab = connect_faces(xmap, M, 3, lambda cen: inner_tag if np.linalg.norm(cen) < 0.5 * (r0 + rad[1]) else outer_tag)
    return dict(dim=3, K=K, M=M, xmap=xmap, ftab=ftab)


def _face_corners(xm, f, M):
    """Corner positions of face f of an element with (M+1)^3 mapping nodes,
    in the face's (s, t) corner order (-,-), (+,-), (-,+), (+,+)."""
    Mp = M + 1
    v = xm.reshape(Mp, Mp, Mp, 3)  # [c][b][a]
    d, side = f // 2, f % 2
    ta, tb = [t for t in range(3) if t != d]
    out = []
    for bt in range(2):
        for at in range(2):
            idx = [0, 0, 0]
            idx[d] = side * M
            idx[ta] = at * M
            idx[tb] = bt * M
            out.append(v[idx[2], idx[1], idx[0]])
    return np.array(out)


def _corner_key(C, scale):
    return tuple(sorted(tuple(np.round(c / scale, 9)) for c in C))


def connect_faces(xmap, M, dim, boundary_tag, tag_of_key=None, allow_unmatched_keys=False):
    """Face table of a conforming hexahedral mesh from its geometry: faces
    that share their four corners are neighbours; the orientation code maps
    one side's face coordinates to the other's.  Unmatched faces get
    boundary_tag(face centroid), or the tag stored for their corner key (tag
    -99 marks an unmatched face with no stored tag when allowed)."""
    K = xmap.shape[0]
    ftab = np.full((K, 6, 4), -1, dtype=np.int32)
    ftab[:, :, 2:] = 0
    scale = np.max(np.abs(xmap))
    key_of = {}
    corners = {}
    for e in range(K):
        for f in range(2 * dim):
            C = _face_corners(xmap[e], f, M)
            corners[(e, f)] = C
            key_of.setdefault(_corner_key(C, scale), []).append((e, f))
    for key, lst in key_of.items():
        if len(lst) == 1:
            e, f = lst[0]
            if tag_of_key is not None:
                k2 = _corner_key(corners[(e, f)], tag_of_key[1])
                if k2 in tag_of_key[0]:
                    tag = tag_of_key[0][k2]
                elif allow_unmatched_keys:
                    tag = -99
                else:
                    raise AssertionError("unmatched face without a boundary tag")
            else:
                tag = boundary_tag(corners[(e, f)].mean(axis=0))
            ftab[e, f] = (-1, -1, 0, tag)
            continue
        assert len(lst) == 2, "a face shared by more than two elements"
        (eA, fA), (eB, fB) = lst
        A, B = corners[(eA, fA)], corners[(eB, fB)]
        ftab[eA, fA] = (eB, fB, _orientation(A, B, scale), 0)
        ftab[eB, fB] = (eA, fA, _orientation(B, A, scale), 0)
    return ftab


# --------------------------------------------------------------------------
# order maps
# --------------------------------------------------------------------------
def uniform_orders(K, dim, N):
    o = np.full((K, 3), N, dtype=np.int32)
    if dim == 2:
        o[:, 2] = 0
    return o


def random_orders(K, dim, lo, hi, seed):
    rng = np.random.default_rng(seed)
    o = rng.integers(lo, hi + 1, size=(K, 3)).astype(np.int32)
    if dim == 2:
        o[:, 2] = 0
    return o


def layout_offsets(orders, dim):
    """Node count per element and its prefix sum (element-blocked layout)."""
    n = orders.astype(np.int64) + 1
    if dim == 2:
        n[:, 2] = 1
    nn = n[:, 0] * n[:, 1] * n[:, 2]
    off = np.concatenate([[0], np.cumsum(nn)])
    return nn, off


# --------------------------------------------------------------------------
# states
# --------------------------------------------------------------------------
def _gauss(n):
    return np.polynomial.legendre.leggauss(n)


def node_coordinates(mesh, orders):
    """Physical coordinates of every element's tensor Gauss nodes, node-major
    (total_nodes, 3): used only to sample closed-form fields."""
    dim, M = mesh["dim"], mesh["M"]
    nn, off = layout_offsets(orders, dim)
    X = np.zeros((off[-1], 3))
    eq = np.linspace(-1.0, 1.0, M + 1)

    def lag(x):
        L = np.ones((len(x), M + 1))
        for a in range(M + 1):
            for b in range(M + 1):
                if b != a:
                    L[:, a] *= (x - eq[b]) / (eq[a] - eq[b])
        return L

    for e in range(mesh["K"]):
        n = orders[e] + 1
        if dim == 2:
            n = [n[0], n[1], 1]
        x0, x1 = _gauss(n[0])[0], _gauss(n[1])[0]
        x2 = _gauss(n[2])[0] if dim == 3 else np.zeros(1)
        L0, L1 = lag(x0), lag(x1)
        if dim == 3:
            L2 = lag(x2)
            P = mesh["xmap"][e].reshape(M + 1, M + 1, M + 1, 3)
            pts = np.einsum("ia,jb,kc,cbax->kjix", L0, L1, L2, P)
        else:
            P = mesh["xmap"][e].reshape(M + 1, M + 1, 3)
            pts = np.einsum("ia,jb,bax->jix", L0, L1, P)[None]
            pts = pts.copy()
            pts[..., 2] = x2[:, None, None]
        X[off[e]:off[e + 1]] = pts.reshape(-1, 3)
    return X


def conserved(rho, u, v, w, p, gamma):
    return np.stack([rho, rho * u, rho * v, rho * w, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])


def to_blocked(fields, orders, dim):
    """(nvar, total_nodes) node-major fields -> element-blocked flat vector."""
    nvar = fields.shape[0]
    nn, off = layout_offsets(orders, dim)
    out = np.empty(off[-1] * nvar)
    for e in range(len(nn)):
        out[nvar * off[e]: nvar * off[e + 1]] = fields[:, off[e]:off[e + 1]].reshape(-1)
    return out


def from_blocked(vec, orders, dim, nvar=5):
    nn, off = layout_offsets(orders, dim)
    out = np.empty((nvar, off[-1]))
    for e in range(len(nn)):
        out[:, off[e]:off[e + 1]] = vec[nvar * off[e]: nvar * off[e + 1]].reshape(nvar, nn[e])
    return out


def manufactured_phases(seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 2.0 * np.pi, size=(4, 2, 2))


def manufactured_primitives(X, phases, mach, gamma, amp=0.1):
    """rho, u, v, w, p of the smooth periodic field
    g_m(x,y) = sum_{k=1,2} sin(2 pi k x + phi_mk) cos(2 pi k y + psi_mk):
    rho = 1 + a g_0, u = 1 + a g_1, v = a g_2, w = 0, p = (1 + a g_3)/(gamma M^2)."""
    x, y = X[:, 0], X[:, 1]

    def g(m):
        s = 0.0
        for k in (1, 2):
            s = s + np.sin(2 * np.pi * k * x + phases[m, k - 1, 0]) * np.cos(2 * np.pi * k * y + phases[m, k - 1, 1])
        return s

    rho = 1.0 + amp * g(0)
    u = 1.0 + amp * g(1)
    v = amp * g(2)
    w = np.zeros_like(x)
    p = (1.0 + amp * g(3)) / (gamma * mach * mach)
    return rho, u, v, w, p


def manufactured_state(mesh, orders, seed, mach, gamma, amp=0.1):
    X = node_coordinates(mesh, orders)
    rho, u, v, w, p = manufactured_primitives(X, manufactured_phases(seed), mach, gamma, amp)
    return to_blocked(conserved(rho, u, v, w, p, gamma), orders, mesh["dim"])


def freestream_state(mesh, orders, prm):
    nn, off = layout_offsets(orders, mesh["dim"])
    q = np.tile(np.asarray(prm[7:12])[:, None], (1, off[-1]))
    return to_blocked(q, orders, mesh["dim"])


def perturbed_state(mesh, orders, prm, seed, amp=0.05):
    """Freestream plus independent seeded perturbations of rho, u, v, (w), p at
    every node (not smooth: exercises every term of the operator)."""
    rng = np.random.default_rng(seed)
    gamma, mach = prm[0], prm[2]
    nn, off = layout_offsets(orders, mesh["dim"])
    Nt = off[-1]
    rho = 1.0 + amp * rng.uniform(-1, 1, Nt)
    u = 1.0 + amp * rng.uniform(-1, 1, Nt)
    v = amp * rng.uniform(-1, 1, Nt)
    w = amp * rng.uniform(-1, 1, Nt) if mesh["dim"] == 3 else np.zeros(Nt)
    p = (1.0 + amp * rng.uniform(-1, 1, Nt)) / (gamma * mach * mach)
    return to_blocked(conserved(rho, u, v, w, p, gamma), orders, mesh["dim"])


def oblique_state(mesh, orders, prm, seed, amp=0.02, vel=(0.8, 0.5, 0.3)):
    """A uniform flow of velocity `vel` (oblique to every face of an
    axis-aligned mesh) with independent seeded per-node perturbations of
    relative size `amp` of rho, the velocity components and p: no face-normal
    velocity comes near zero, so comparisons of derivatives of the operator
    stay clear of the kinks of |lambda| in an upwind flux."""
    dim = mesh["dim"]
    X = node_coordinates(mesh, orders)
    g, M = prm[0], prm[2]
    rng = np.random.default_rng(seed)
    n = X.shape[0]

    def f(c):
        return c + amp * rng.uniform(-1, 1, n)

    w = f(vel[2]) if dim == 3 else 0.0 * X[:, 0]
    return to_blocked(conserved(f(1.0), f(vel[0]), f(vel[1]), w, f(1.0) / (g * M * M), g), orders, dim)


def zero_mean_wave(mesh, orders, q_target, seed, amp=0.01):
    """q_target plus amp * |q_target| * w, w the smooth periodic wave
    sin(2 pi (x + 2y) + phase_v) with seeded phases (resolved on every mesh
    used here, including the one-element-thick 4x4x1 box).  On a periodic mesh
    the pseudo-time iteration conserves the discrete totals of the five
    variables, so w is given zero weighted mean per variable (Gauss weights;
    meshes of equal elements)."""
    rng = np.random.default_rng(seed)
    dim = mesh["dim"]
    W = []
    for e in range(mesh["K"]):
        w = np.ones(1)
        for d in range(dim):
            w = np.multiply.outer(np.polynomial.legendre.leggauss(int(orders[e, d]) + 1)[1], w)
        W.append(w.reshape(-1))
    W = np.concatenate(W)
    X = node_coordinates(mesh, orders)
    phase = rng.uniform(0.0, 2.0 * np.pi, 5)
    wave = np.stack([np.sin(2.0 * np.pi * (X[:, 0] + 2.0 * X[:, 1]) + phase[v]) for v in range(5)])
    wave -= (wave @ W / W.sum())[:, None]
    scale = np.abs(from_blocked(q_target, orders, dim)).max(axis=1)[:, None]
    return q_target + amp * to_blocked(wave * scale, orders, dim)


def boundary_layer_state(mesh, orders, prm, delta=0.05):
    """rho = 1, p = p_inf, u = 1 - exp(-y / delta), v = w = 0: a smooth
    boundary-layer-like field, zero velocity on the wall y = 0."""
    X = node_coordinates(mesh, orders)
    g, M = prm[0], prm[2]
    y = X[:, 1]
    one = np.ones_like(y)
    u = 1.0 - np.exp(-y / delta)
    return to_blocked(conserved(one, u, 0 * y, 0 * y, one / (g * M * M), g), orders, mesh["dim"])


def plate_steady_case(seed=3):
    """A plate-shaped steady problem that explicit pseudo-time cycles can
    converge to 1e-10 (a variant of the stretched flat-plate workload): the
    flat-plate boundary conditions on 24 x 8 uniform elements of size 0.05
    (x in [-0.2, 1], y in [0, 0.4]), N = 3, Mach 0.2, Re 1e4.  Its discrete
    solution is the boundary-layer-like field q* of boundary_layer_state: the
    caller forms S = A(q*).  The start is q* plus a 1 % smooth wave
    (zero_mean_wave).  Returns mesh, orders, params, q*, start."""
    mesh = flat_plate_mesh(nx=24, ny=8, dy0=0.05, ratio=1.0)
    prm = flow_params(mach=0.2, re=1e4)
    o = uniform_orders(mesh["K"], 2, 3)
    qs = boundary_layer_state(mesh, o, prm)
    return mesh, o, prm, qs, zero_mean_wave(mesh, o, qs, seed, amp=0.01)


def smooth_state(mesh, orders, prm, seed, amp=0.05, wavelength=5.0):
    """Freestream plus smooth seeded perturbations of rho, u, v, w, p: each a
    sum of three plane waves with random directions, wavelength ~ `wavelength`
    and random phases (resolved by the mesh, unlike per-node noise)."""
    rng = np.random.default_rng(seed)
    gamma, mach = prm[0], prm[2]
    X = node_coordinates(mesh, orders)
    if mesh["dim"] == 2:
        X = X.copy()
        X[:, 2] = 0.0

    def field():
        out = np.zeros(len(X))
        for _ in range(3):
            kdir = rng.normal(size=3)
            if mesh["dim"] == 2:
                kdir[2] = 0.0
            kdir *= 2 * np.pi / wavelength / np.linalg.norm(kdir)
            out += np.sin(X @ kdir + rng.uniform(0, 2 * np.pi)) / 3.0
        return out

    rho = 1.0 + amp * field()
    u = 1.0 + amp * field()
    v = amp * field()
    w = amp * field() if mesh["dim"] == 3 else np.zeros(len(X))
    p = (1.0 + amp * field()) / (gamma * mach * mach)
    return to_blocked(conserved(rho, u, v, w, p, gamma), orders, mesh["dim"])


def random_source(mesh, orders, seed, amp=1e-2):
    rng = np.random.default_rng(seed + 1000)
    nn, off = layout_offsets(orders, mesh["dim"])
    s = amp * rng.uniform(-1, 1, (5, off[-1]))
    if mesh["dim"] == 2:
        s[3] = 0.0
    return to_blocked(s, orders, mesh["dim"])


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def manufactured_box_4x4x1(seed=0):
    """4x4x1 periodic unit box, N=3, manufactured state (Mach 0.3, Re 100)."""
    mesh = periodic_box(4, 4, 1)
    prm = flow_params(mach=0.3, re=100.0)
    orders = uniform_orders(mesh["K"], 3, 3)
    q = manufactured_state(mesh, orders, seed, prm[2], prm[0])
    return mesh, orders, prm, q


def sphere_shell_13824(seed=2, nt=12, nr=16):
    """Cubed-sphere shell r in [1, 20], 6 x nt x nt x nr quadratic hexes
    (13,824 at nt=12, nr=16), orders uniform in [1, 6]^3 from the seed, Mach
    0.2, Re 200, no-slip adiabatic sphere, freestream outer boundary."""
    mesh = cubed_sphere_mesh(nt, nr)
    prm = flow_params(mach=0.2, re=200.0)
    orders = random_orders(mesh["K"], 3, 1, 6, seed)
    return mesh, orders, prm


def compatible_source(mesh, orders, S, weights_times_J):
    """Remove from each variable of the source its mean with respect to the
    given nodal weights w J (node-major over the element-blocked layout): on a
    periodic domain a steady state exists only for a source of zero integral."""
    F = from_blocked(S, orders, mesh["dim"])
    F = F - (F @ weights_times_J / weights_times_J.sum())[:, None]
    return to_blocked(F, orders, mesh["dim"])


def flat_plate_60x24(N=7):
    """60x24 stretched 2D flat plate, uniform N, freestream start (Mach 0.2, Re 1e5)."""
    mesh = flat_plate_mesh()
    prm = flow_params(mach=0.2, re=1e5)
    orders = uniform_orders(mesh["K"], 2, N)
    q = freestream_state(mesh, orders, prm)
    return mesh, orders, prm, q


def batch_workload_64(seed=3, nsolves=64, kmin=200, kmax=4000, nmax=8, sphere_M=2):
    """Many independent steady solves: half stretched 2D plate-type meshes,
    half cubed-sphere shells.  Element counts log-uniform in [kmin, kmax],
    orders i.i.d. uniform in [1, nmax]^dim, Mach log-uniform in [0.1, 0.4],
    Re log-uniform in [1e2, 1e5].  Returns [(mesh, orders, params), ...]."""
    rng = np.random.default_rng(seed)
    items, shells = [], {}
    for k in range(nsolves):
        target = float(np.exp(rng.uniform(np.log(kmin), np.log(kmax))))
        mach = float(np.exp(rng.uniform(np.log(0.1), np.log(0.4))))
        re = float(np.exp(rng.uniform(np.log(1e2), np.log(1e5))))
        if k % 2 == 0:
            # plate-type: nx : ny = 5 : 2 as in the 60 x 24 plate
            ny = max(2, int(round(np.sqrt(target / 2.5))))
            nx = max(2, int(round(target / ny)))
            mesh = flat_plate_mesh(nx=nx, ny=ny, dy0=float(10 ** rng.uniform(-3, -2)), ratio=1.15)
            orders = random_orders(mesh["K"], 2, 1, nmax, seed * 1000 + k)
        else:
            # shell: 6 nt^2 nr elements with nr ~ 4/3 nt as in 6 x 12 x 12 x 16
            nt = max(1, int(round((target / 8.0) ** (1.0 / 3.0))))
            nr = max(2, int(round(target / (6.0 * nt * nt))))
            if (nt, nr) not in shells:  # same shape, same mesh: built once
                shells[(nt, nr)] = cubed_sphere_mesh(nt, nr, M=sphere_M)
            mesh = shells[(nt, nr)]
            orders = random_orders(mesh["K"], 3, 1, nmax, seed * 1000 + k)
        items.append((mesh, orders, flow_params(mach=mach, re=re)))
    return items
