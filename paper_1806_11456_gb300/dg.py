"""Python binding of the C ABI in include/dg.h (argument marshalling only).

Every computation runs in the CUDA library libdgpmg.so; this module loads it
(failing loudly when it is missing or no CUDA device is present), converts
torch tensors to device pointers and the current torch stream to a
cudaStream_t, and maps status codes to exceptions.  State tensors are float64
CUDA tensors in the element-blocked layout of ``Mesh.layout()``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgpmg.so")

DG_ISOLATED = 1
DG_NORM = 2
TAU_SLOTS = 16


class DGError(RuntimeError):
    pass


class MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("K", ctypes.c_int32), ("M", ctypes.c_int32),
                ("xmap", ctypes.POINTER(ctypes.c_double)), ("ftab", ctypes.POINTER(ctypes.c_int32)),
                ("params", ctypes.c_double * 16)]


class MGParams(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_int32), ("beta2", ctypes.c_int32), ("beta_c", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("coarsest", ctypes.c_int32), ("delta_n", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("control", ctypes.c_int32), ("eta", ctypes.c_double)]


class SolveReport(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int32), ("fmg_cycles", ctypes.c_int32), ("adapted", ctypes.c_int32),
                ("status", ctypes.c_int32), ("rnorm", ctypes.c_double), ("rnorm_adapt", ctypes.c_double),
                ("dof_evals", ctypes.c_double), ("nodes", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class ServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("slots", ctypes.c_int32), ("device", ctypes.c_int32),
                ("batch_max", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("K", ctypes.c_int32), ("rep", SolveReport),
                ("est_bytes", ctypes.c_int64), ("dev_bytes", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double), ("batch_peers", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


REQ_QUEUED, REQ_RUNNING = 1, 2


class CycleReport(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("residual_evals", ctypes.c_int32), ("dof_evals", ctypes.c_double),
                ("rnorm", ctypes.c_double)]


class AdaptParams(ctypes.Structure):
    _fields_ = [("tau_max", ctypes.c_double), ("n_min", ctypes.c_int32), ("n_max", ctypes.c_int32),
                ("cap", ctypes.c_int32), ("jump_rule", ctypes.c_int32), ("conform_tag", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_cycles", ctypes.c_int32), ("fmg", ctypes.c_int32),
                ("fmg_tol", ctypes.c_double), ("mg", MGParams), ("adapt", ctypes.c_int32),
                ("n_stages", ctypes.c_int32), ("ap", AdaptParams), ("stage_orders", ctypes.c_int32 * 4),
                ("ref_factor", ctypes.c_double), ("check_every", ctypes.c_int32), ("arith", ctypes.c_int32),
                ("mixed_from", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)

EXPORTS = ["dg_mesh_create", "dg_mesh_destroy", "dg_mesh_layout", "dg_residual", "dg_cfl_dt", "dg_smooth",
           "dg_pmg_vcycle", "dg_tau_estimate", "dg_adapt", "dg_transfer_state", "dg_profile_residual",
           "dg_kernel_launches", "dg_transfer_noalloc", "dg_solve_steady", "dg_mesh_orders", "dg_set_arithmetic",
           "dg_batch_create", "dg_batch_info", "dg_residual_norms", "dg_solve_footprint", "dg_server_create",
           "dg_server_submit", "dg_server_wait", "dg_server_info", "dg_server_result", "dg_server_release",
           "dg_server_destroy", "dg_set_autotune", "dg_mesh_tuning", "dg_measure_fma_rates", "dg_residual_tangent",
           "dg_batch_set_active", "dg_last_error"]
ARITH = {"fp64": 0, "df32": 1, "mixed": 2}
KERNEL_STAGES = ["trace_q", "mortar_u_star", "volume", "mortar_flux", "surface", "isolated"]


def lib(path=LIB_PATH):
    """Load libdgpmg.so (no CUDA call is made here)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise DGError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    L.dg_last_error.restype = ctypes.c_char_p
    L.dg_mesh_create.argtypes = [ctypes.POINTER(MeshDesc), _ip, ctypes.POINTER(_vp)]
    L.dg_mesh_destroy.argtypes = [_vp]
    L.dg_mesh_layout.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.dg_residual.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, _dp, _vp]
    L.dg_cfl_dt.argtypes = [_vp, _vp, _dp, _vp]
    L.dg_smooth.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp]
    L.dg_pmg_vcycle.argtypes = [_vp, _vp, _vp, ctypes.POINTER(MGParams), ctypes.c_int, ctypes.POINTER(CycleReport), _vp]
    L.dg_tau_estimate.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _vp]
    L.dg_adapt.argtypes = [_vp, _dp, ctypes.POINTER(AdaptParams), _ip]
    L.dg_transfer_state.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.dg_profile_residual.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, _dp, _vp]
    L.dg_kernel_launches.argtypes = [ctypes.POINTER(ctypes.c_int64)]
    L.dg_solve_steady.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, ctypes.POINTER(SolveParams), ALLOC_FN,
                                  _vp, ctypes.POINTER(SolveReport), _vp]
    L.dg_mesh_orders.argtypes = [_vp, _ip]
    L.dg_set_arithmetic.argtypes = [_vp, ctypes.c_int]
    L.dg_batch_create.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(_ip), ctypes.c_int32, ctypes.POINTER(_vp)]
    L.dg_batch_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]
    L.dg_residual_norms.argtypes = [_vp, _vp, _vp, _dp, _vp]
    L.dg_transfer_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, _ip, _ip, ctypes.c_int32, _vp, _vp, _vp]
    L.dg_set_autotune.argtypes = [_vp, ctypes.c_int, _vp]
    L.dg_mesh_tuning.argtypes = [_vp, _ip]
    L.dg_solve_footprint.argtypes = [ctypes.POINTER(MeshDesc), _ip, ctypes.POINTER(ctypes.c_int64)]
    L.dg_server_create.argtypes = [ctypes.POINTER(ServerParams), ctypes.POINTER(_vp)]
    L.dg_server_submit.argtypes = [_vp, ctypes.POINTER(MeshDesc), _ip, _dp, _dp, ctypes.POINTER(SolveParams),
                                   ctypes.POINTER(ctypes.c_int64)]
    L.dg_server_wait.argtypes = [_vp, ctypes.c_int64, ctypes.c_double]
    L.dg_server_info.argtypes = [_vp, ctypes.c_int64, ctypes.POINTER(RequestInfo)]
    L.dg_server_result.argtypes = [_vp, ctypes.c_int64, _dp, _ip]
    L.dg_server_release.argtypes = [_vp, ctypes.c_int64]
    L.dg_server_destroy.argtypes = [_vp]
    L.dg_measure_fma_rates.argtypes = [_dp, _dp, _vp]
    L.dg_residual_tangent.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.dg_batch_set_active.argtypes = [_vp, _ip, _vp]
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise DGError(f"dg error {rc}: {lib().dg_last_error().decode()}")


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise DGError("state tensors must be contiguous float64 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def measure_fma_rates(stream=None):
    """FP64 and FP32 FMA throughput of the current device in TFLOP/s."""
    import torch
    if not torch.cuda.is_available():
        raise DGError("no CUDA device: the DGSEM library has no CPU path")
    L = lib()
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    _check(L.dg_measure_fma_rates(ctypes.byref(f64), ctypes.byref(f32), _stream(stream)))
    return {"fp64_tflops": f64.value, "fp32_tflops": f32.value}


def kernel_launches():
    """Cumulative count of kernels the library has launched in this process."""
    c = ctypes.c_int64()
    _check(lib().dg_kernel_launches(ctypes.byref(c)))
    return int(c.value)


def solve_params(tol=1e-10, max_cycles=200, fmg=False, fmg_tol=1e-1, mg=None, adapt=False, tau_max=1e-4, n_min=1,
                 n_max=7, jump_rule=1, conform_tag=-1, cap=0, stages=(), ref_factor=0.1, check_every=1, arith="fp64",
                 mixed_from=0.0):
    """dg_solve_params from keyword arguments (mg: dict of dg_mg_params fields)."""
    sp = SolveParams()
    sp.tol, sp.max_cycles, sp.fmg, sp.fmg_tol, sp.adapt = float(tol), int(max_cycles), int(bool(fmg)), \
        float(fmg_tol), int(bool(adapt))
    m = dict(beta1=3, beta2=3, beta_c=6, direction=-1, coarsest=1, delta_n=1, graph=1, control=0, eta=1.1)
    m.update(mg or {})
    for k, v in m.items():
        setattr(sp.mg, k, float(v) if k == "eta" else int(v))
    sp.ap.tau_max, sp.ap.n_min, sp.ap.n_max, sp.ap.cap, sp.ap.jump_rule, sp.ap.conform_tag = \
        float(tau_max), n_min, n_max, cap, jump_rule, conform_tag
    if len(stages) > 4:
        raise DGError("at most 4 adaptation stages")
    sp.n_stages = len(stages)
    sp.ref_factor = float(ref_factor)
    for i, v in enumerate(stages):
        sp.stage_orders[i] = int(v)
    sp.check_every = int(check_every)
    sp.arith = ARITH[arith]
    sp.mixed_from = float(mixed_from)
    return sp


def _desc(mesh, params, keep):
    d = MeshDesc()
    xmap = np.ascontiguousarray(mesh["xmap"], dtype=np.float64)
    ftab = np.ascontiguousarray(mesh["ftab"], dtype=np.int32)
    keep += [xmap, ftab]
    d.dim, d.K, d.M = int(mesh["dim"]), int(mesh["K"]), int(mesh["M"])
    d.xmap = xmap.ctypes.data_as(_dp)
    d.ftab = ftab.ctypes.data_as(_ip)
    for i in range(16):
        d.params[i] = float(params[i])
    return d


class Mesh:
    """A mesh with an order map: geometry, faces and multigrid levels live on
    the device inside the library."""

    @classmethod
    def batch(cls, items):
        """One handle for several independent solves [(mesh, orders, params),
        ...] (dg_batch_create).  ``solve_slices()`` gives each solve's range
        of the batch state vector."""
        import torch
        if not torch.cuda.is_available():
            raise DGError("no CUDA device: the DGSEM library has no CPU path")
        keep = []
        descs = (MeshDesc * len(items))()
        ords = (_ip * len(items))()
        for k, (mesh, orders, params) in enumerate(items):
            descs[k] = _desc(mesh, params, keep)
            o = np.ascontiguousarray(orders, dtype=np.int32)
            keep.append(o)
            ords[k] = o.ctypes.data_as(_ip)
        h = _vp()
        torch.cuda.current_device()
        _check(lib().dg_batch_create(descs, ords, len(items), ctypes.byref(h)))
        self = cls.__new__(cls)
        self.h = h
        self.dim = int(items[0][0]["dim"])
        self.K = sum(int(it[0]["K"]) for it in items)
        self.M = int(items[0][0]["M"])
        self.orders = np.concatenate([np.asarray(it[1], dtype=np.int32) for it in items])
        self.params = np.asarray(items[0][2], dtype=np.float64)
        self.mesh = None
        self.arith = "fp64"
        return self

    def solve_slices(self):
        """Node offsets of the solves (5 values per node in the state)."""
        n = ctypes.c_int32()
        _check(lib().dg_batch_info(self.h, ctypes.byref(n), None))
        off = np.zeros(n.value + 1, dtype=np.int64)
        _check(lib().dg_batch_info(self.h, ctypes.byref(n), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return off

    def set_active(self, active, stream=None):
        """Hold the solves whose flag is 0 (dg_batch_set_active)."""
        a = np.ascontiguousarray(active, dtype=np.int32)
        _check(lib().dg_batch_set_active(self.h, a.ctypes.data_as(_ip), _stream(stream)))
        return self

    def residual_norms(self, q, s=None, stream=None):
        n = ctypes.c_int32()
        _check(lib().dg_batch_info(self.h, ctypes.byref(n), None))
        out = np.zeros(n.value)
        _check(lib().dg_residual_norms(self.h, _ptr(q), _ptr(s), out.ctypes.data_as(_dp), _stream(stream)))
        return out

    def __init__(self, mesh, orders, params):
        import torch
        if not torch.cuda.is_available():
            raise DGError("no CUDA device: the DGSEM library has no CPU path")
        self.dim, self.K, self.M = int(mesh["dim"]), int(mesh["K"]), int(mesh["M"])
        self._xmap = np.ascontiguousarray(mesh["xmap"], dtype=np.float64)
        self._ftab = np.ascontiguousarray(mesh["ftab"], dtype=np.int32)
        self.orders = np.ascontiguousarray(orders, dtype=np.int32)
        self.params = np.asarray(params, dtype=np.float64)
        self.mesh = mesh
        d = MeshDesc()
        d.dim, d.K, d.M = self.dim, self.K, self.M
        d.xmap = self._xmap.ctypes.data_as(_dp)
        d.ftab = self._ftab.ctypes.data_as(_ip)
        for i in range(16):
            d.params[i] = float(self.params[i])
        h = _vp()
        torch.cuda.current_device()  # make sure the CUDA context exists
        _check(lib().dg_mesh_create(ctypes.byref(d), self.orders.ctypes.data_as(_ip), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().dg_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_autotune(self, on=True, stream=None):
        """Choose the element tiles of every level by timing (dg_set_autotune)."""
        _check(lib().dg_set_autotune(self.h, int(bool(on)), _stream(stream)))
        return self

    def tuning(self):
        """Finest level's tiles: nodes per CTA for small elements, CTA sizes per class."""
        out = np.zeros(4, dtype=np.int32)
        _check(lib().dg_mesh_tuning(self.h, out.ctypes.data_as(_ip)))
        return dict(pack=int(out[0]), class_threads=[int(x) for x in out[1:]])

    def set_arithmetic(self, mode):
        """'fp64' (native FP64), 'df32' (double-float pairs on the FP32 pipes)
        or 'mixed' (FP64 finest residual, coarse right-hand sides and tau;
        FP32 tangent-linear correction cycle) for the operator kernels."""
        _check(lib().dg_set_arithmetic(self.h, ARITH[mode]))
        self.arith = mode
        return self

    def layout(self):
        n = ctypes.c_int64()
        off = np.zeros(self.K + 1, dtype=np.int64)
        _check(lib().dg_mesh_layout(self.h, ctypes.byref(n), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return int(n.value), off

    @property
    def nodes(self):
        return self.layout()[0]

    def residual(self, q, s=None, r=None, isolated=False, norm=False, stream=None):
        import torch
        if r is None:
            r = torch.empty_like(q)
        flags = (DG_ISOLATED if isolated else 0) | (DG_NORM if norm else 0)
        rn = ctypes.c_double(0.0)
        _check(lib().dg_residual(self.h, _ptr(q), _ptr(s), _ptr(r), flags, ctypes.byref(rn), _stream(stream)))
        return (r, rn.value) if norm else r

    def residual_tangent(self, q, dq, b=None, r=None, stream=None):
        """b - J(q) dq with the operator's Jacobian at q applied in FP32 tangent
        arithmetic (b None: 0)."""
        import torch
        if r is None:
            r = torch.empty_like(q)
        _check(lib().dg_residual_tangent(self.h, _ptr(q), _ptr(dq), _ptr(b), _ptr(r), _stream(stream)))
        return r

    def cfl_dt(self, q, stream=None):
        dt = ctypes.c_double()
        _check(lib().dg_cfl_dt(self.h, _ptr(q), ctypes.byref(dt), _stream(stream)))
        return dt.value

    def smooth(self, q, s=None, sweeps=1, stream=None):
        _check(lib().dg_smooth(self.h, _ptr(q), _ptr(s), int(sweeps), _stream(stream)))
        return q

    def vcycle(self, q, s=None, beta1=3, beta2=3, beta_c=3, direction=-1, coarsest=1, delta_n=1,
               graph=False, want_norm=False, control=0, eta=1.1, stream=None):
        mg = MGParams()
        mg.beta1, mg.beta2, mg.beta_c, mg.direction, mg.coarsest, mg.delta_n, mg.graph = \
            beta1, beta2, beta_c, direction, coarsest, delta_n, int(bool(graph))
        mg.control, mg.eta = int(control), float(eta)
        rep = CycleReport()
        _check(lib().dg_pmg_vcycle(self.h, _ptr(q), _ptr(s), ctypes.byref(mg), int(bool(want_norm)),
                                   ctypes.byref(rep), _stream(stream)))
        return dict(levels=rep.levels, residual_evals=rep.residual_evals, dof_evals=rep.dof_evals,
                    rnorm=rep.rnorm)

    def tau_estimate(self, q, s=None, dir_mask=7, with_correction=True, isolated=True, stream=None):
        tab = np.zeros((self.K, 3, TAU_SLOTS))
        _check(lib().dg_tau_estimate(self.h, _ptr(q), _ptr(s), int(dir_mask), int(bool(with_correction)),
                                     int(bool(isolated)), tab.ctypes.data_as(_dp), _stream(stream)))
        return tab

    def adapt(self, tau, tau_max, n_min, n_max, cap=0, jump_rule=0, conform_tag=-1):
        ap = AdaptParams()
        ap.tau_max, ap.n_min, ap.n_max, ap.cap, ap.jump_rule, ap.conform_tag = \
            float(tau_max), n_min, n_max, cap, jump_rule, conform_tag
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        out = np.zeros((self.K, 3), dtype=np.int32)
        _check(lib().dg_adapt(self.h, tau.ctypes.data_as(_dp), ctypes.byref(ap), out.ctypes.data_as(_ip)))
        return out

    def profile_residual(self, q, s=None, iters=20, stream=None):
        """Mean ms per residual stage (CUDA events on the launching stream)."""
        import torch
        r = torch.empty_like(q)
        ms = np.zeros(6)
        _check(lib().dg_profile_residual(self.h, _ptr(q), _ptr(s), _ptr(r), int(iters), ms.ctypes.data_as(_dp),
                                         _stream(stream)))
        return dict(zip(KERNEL_STAGES, ms.tolist()))

    def solve_steady(self, q, s=None, tol=1e-10, max_cycles=200, fmg=False, fmg_tol=1e-1, mg=None, adapt=False,
                     tau_max=1e-4, n_min=1, n_max=7, jump_rule=1, conform_tag=-1, cap=0, stages=(), ref_factor=0.1,
                     check_every=1, mixed_from=0.0, stream=None):
        """Steady solve through dg_solve_steady.  Returns (q, report); with
        adaptation q is a new tensor on the adapted mesh, which this object
        then wraps (its orders are updated)."""
        import torch
        sp = solve_params(tol, max_cycles, fmg, fmg_tol, mg, adapt, tau_max, n_min, n_max, jump_rule, conform_tag,
                          cap, stages, ref_factor, check_every, mixed_from=mixed_from)
        keep = []

        def _alloc(nbytes, _ctx):
            t = torch.empty(int(nbytes) // 8, dtype=torch.float64, device=q.device)
            keep.append(t)
            return t.data_ptr()

        cb = ALLOC_FN(_alloc)
        hp = _vp(self.h.value)
        qp = _vp(q.data_ptr())
        rep = SolveReport()
        _ptr(q)
        rc = lib().dg_solve_steady(ctypes.byref(hp), ctypes.byref(qp), _ptr(s), ctypes.byref(sp), cb, None,
                                   ctypes.byref(rep), _stream(stream))
        out = q
        if rep.adapted:
            self.h = hp
            orders = np.zeros((self.K, 3), dtype=np.int32)
            _check(lib().dg_mesh_orders(self.h, orders.ctypes.data_as(_ip)))
            self.orders = orders
            out = keep[-1]
        report = dict(cycles=rep.cycles, fmg_cycles=rep.fmg_cycles, adapted=int(rep.adapted), status=rep.status,
                      rnorm=rep.rnorm, rnorm_adapt=rep.rnorm_adapt, dof_evals=rep.dof_evals, nodes=rep.nodes)
        if rc not in (0, -4, -5):
            _check(rc)
        return out, report

    def transfer_state_to(self, other, q_from, q_to=None, stream=None):
        import torch
        if q_to is None:
            q_to = torch.empty(5 * other.nodes, dtype=torch.float64, device=q_from.device)
        _check(lib().dg_transfer_state(self.h, _ptr(q_from), other.h, _ptr(q_to), _stream(stream)))
        return q_to


def solve_footprint(mesh, orders, params):
    """Device bytes a steady solve of this mesh and order map is estimated to
    hold (dg_solve_footprint; the serving admission estimate)."""
    keep = []
    d = _desc(mesh, params, keep)
    o = np.ascontiguousarray(orders, dtype=np.int32)
    b = ctypes.c_int64()
    _check(lib().dg_solve_footprint(ctypes.byref(d), o.ctypes.data_as(_ip), ctypes.byref(b)))
    return int(b.value)


class Server:
    """Serving loop (dg_server_*): steady solves submitted as host arrays run
    in `slots` concurrent workers, admitted while their memory estimates fit
    in `hbm_budget` bytes; with batch_max > 1 each worker runs up to
    batch_max compatible requests in shared launches."""

    def __init__(self, hbm_budget, slots=4, device=None, batch_max=1):
        import torch
        if not torch.cuda.is_available():
            raise DGError("no CUDA device: the DGSEM library has no CPU path")
        p = ServerParams()
        p.hbm_budget, p.slots, p.batch_max = int(hbm_budget), int(slots), int(batch_max)
        p.device = torch.cuda.current_device() if device is None else int(device)
        self.h = _vp()
        _check(lib().dg_server_create(ctypes.byref(p), ctypes.byref(self.h)))

    def submit(self, mesh, orders, params, q0=None, s=None, **solve_kw):
        keep = []
        d = _desc(mesh, params, keep)
        o = np.ascontiguousarray(orders, dtype=np.int32)
        qa = None if q0 is None else np.ascontiguousarray(q0, dtype=np.float64)
        sa = None if s is None else np.ascontiguousarray(s, dtype=np.float64)
        sp = solve_params(**solve_kw)
        rid = ctypes.c_int64()
        _check(lib().dg_server_submit(self.h, ctypes.byref(d), o.ctypes.data_as(_ip),
                                      None if qa is None else qa.ctypes.data_as(_dp),
                                      None if sa is None else sa.ctypes.data_as(_dp), ctypes.byref(sp),
                                      ctypes.byref(rid)))
        return int(rid.value)

    def wait(self, rid=-1, timeout=-1.0):
        _check(lib().dg_server_wait(self.h, int(rid), float(timeout)))

    def info(self, rid):
        i = RequestInfo()
        _check(lib().dg_server_info(self.h, int(rid), ctypes.byref(i)))
        r = i.rep
        return dict(state=i.state, K=i.K, est_bytes=i.est_bytes, dev_bytes=i.dev_bytes, t_submit=i.t_submit,
                    t_start=i.t_start, t_end=i.t_end, batch_peers=i.batch_peers,
                    rep=dict(cycles=r.cycles, fmg_cycles=r.fmg_cycles, adapted=r.adapted, status=r.status,
                             rnorm=r.rnorm, rnorm_adapt=r.rnorm_adapt, dof_evals=r.dof_evals, nodes=r.nodes))

    def result(self, rid):
        i = self.info(rid)
        q = np.zeros(5 * i["rep"]["nodes"])
        o = np.zeros((i["K"], 3), dtype=np.int32)
        _check(lib().dg_server_result(self.h, int(rid), q.ctypes.data_as(_dp), o.ctypes.data_as(_ip)))
        return q, o

    def release(self, rid):
        _check(lib().dg_server_release(self.h, int(rid)))

    def close(self):
        if self.h:
            lib().dg_server_destroy(self.h)
            self.h = _vp()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
