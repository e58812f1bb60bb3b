// CUDA kernels of the DGSEM residual, smoother and transfers (sm_103a, FP64).
//
// One residual evaluation r = S - M^{-1} F(Q) (Sec. 2, DiscretNSElem; Sec. 3.1)
// is five launches:
//   k_trace_q      element tiles: conserved state interpolated to every face
//   k_mortar<1>    mortar tiles : BR1 average U* of (u,v,w,T) at mortar nodes,
//                                 L2-projected back onto both faces
//   k_volume       element tiles: BR1 gradient (weak form + lifting of U*),
//                                 its face traces, nodal NS fluxes, weak-form
//                                 volume divergence
//   k_mortar<2>    mortar tiles : Roe + BR1 viscous flux, projected back
//   k_surface      element tiles: surface terms, 1/J, r = S - A; optionally
//                                 fused RK3 stage update and max |r|
// The isolated operator (Sec. 3.2.1) is one element-local launch
// (k_isolated), strong form, optionally fused with the tau epilogue.
//
// Work decomposition: a CTA owns whole elements of one order triple
// (elements-per-CTA so that the tile has <= 256 nodes, one element per CTA
// above that); one thread per node; the element's state, metrics and the
// 1-D derivative tables of its orders are staged in shared memory, where the
// tensor-product contractions read them.  Mortar CTAs own whole mortars, one
// thread per mortar node.  FP64 throughput (2 DFMA/clk/SM on GB300) bounds
// these kernels: the code is written to minimise FP64 instructions (one
// reciprocal of rho per node, T^1.5 as T*sqrt(T), contravariant fluxes formed
// directly from the contravariant velocity).
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cstdio>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <type_traits>

#include "dg_internal.h"
#include "dg_real.h"

namespace dg {

__constant__ DevTables c_tab;
__constant__ double* c_Dhat;  // [kNP][kNP][kNP]
__constant__ double* c_D;     // [kNP][kNP][kNP]
__constant__ double* c_T;     // [kNP][kNP][kNP*kNP] transfer matrices (n_from, n_to)

// the same tables as float pairs (hi, lo) for the double-float kernels
struct DevTables2 {
  float2 lm[kNP][kNP], lp[kNP][kNP];
  float2 lmw[kNP][kNP], lpw[kNP][kNP];
};
__constant__ DevTables2 c_tab2;
__constant__ float2* c_Dhat2;
__constant__ float2* c_D2;
__constant__ float2* c_T2;
// the same tables as tangent pairs (value, 0) for the tangent kernels; the
// boundary interpolation vectors are read from c_tab2's leading parts
__constant__ float2* c_DhatT;
__constant__ float2* c_DT;
__constant__ float2* c_TT;

static float2 split2(double x) {
  float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// Kernels launched by this library: a process total and a per-thread count
// (a graph capture measures its own launches with the latter).
static std::atomic<unsigned long long> g_launches_total{0};
static thread_local unsigned long long t_launches = 0;
static inline void count_launch() {
  g_launches_total.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
unsigned long long launches() { return t_launches; }
unsigned long long launches_total() { return g_launches_total.load(std::memory_order_relaxed); }
void add_launches(unsigned long long n) {
  g_launches_total.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
// Device copies of the derivative and transfer tables, one set per device:
// the __constant__ pointers above are per-device symbols, and each device's
// must point at that device's own copy.
struct DeviceTables {
  double *Dhat = nullptr, *D = nullptr, *T = nullptr;
  float2 *Dhat2 = nullptr, *D2 = nullptr, *T2 = nullptr;
  float2 *DhatT = nullptr, *DT = nullptr, *TT = nullptr;
  bool ready = false;       // tables uploaded and symbols set on this device
  bool smem_ready = false;  // kernel shared-memory attributes set on this device
};
static PerDevice<DeviceTables> g_dev_tables;

static std::mutex g_setup_mutex;  // one-time per-device setup (tables, kernel attributes)

int upload_tables() {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  int dev = 0;
  DG_CUDA_TRY(cudaGetDevice(&dev));
  DeviceTables* dt = g_dev_tables.get(dev);
  if (!dt) {
    set_error("device index " + std::to_string(dev) + " beyond the library's limit of " +
              std::to_string(PerDevice<DeviceTables>::kMax) + " devices");
    return DG_EINVAL;
  }
  if (dt->ready) return DG_OK;
  const Tables1D& T = tables();
  DevTables h;
  memset(&h, 0, sizeof(h));
  for (int n = 1; n < kNP; ++n)
    for (int j = 0; j < n; ++j) {
      h.x[n][j] = T.x[n][j];
      h.w[n][j] = T.w[n][j];
      h.lm[n][j] = T.lm[n][j];
      h.lp[n][j] = T.lp[n][j];
      h.lmw[n][j] = T.lm[n][j] / T.w[n][j];
      h.lpw[n][j] = T.lp[n][j] / T.w[n][j];
    }
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_tab, &h, sizeof(h)));
  std::vector<double> Dh((size_t)kNP * kNP * kNP, 0.0), Dc((size_t)kNP * kNP * kNP, 0.0);
  for (int n = 1; n < kNP; ++n)
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < n; ++a) {
        Dh[((size_t)n * kNP + i) * kNP + a] = T.Dhat[n][i][a];
        Dc[((size_t)n * kNP + i) * kNP + a] = T.D[n][i][a];
      }
  std::vector<double> Tm((size_t)kNP * kNP * kNP * kNP, 0.0);
  for (int nf = 1; nf < kNP; ++nf)
    for (int nt = 1; nt < kNP; ++nt) transfer_matrix(nf, nt, &Tm[((size_t)nf * kNP + nt) * kNP * kNP]);
  if (!dt->Dhat) {
    DG_CUDA_TRY(cudaMalloc(&dt->Dhat, Dh.size() * sizeof(double)));
    DG_CUDA_TRY(cudaMalloc(&dt->D, Dc.size() * sizeof(double)));
    DG_CUDA_TRY(cudaMalloc(&dt->T, Tm.size() * sizeof(double)));
  }
  DG_CUDA_TRY(cudaMemcpy(dt->Dhat, Dh.data(), Dh.size() * sizeof(double), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpy(dt->D, Dc.data(), Dc.size() * sizeof(double), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpy(dt->T, Tm.data(), Tm.size() * sizeof(double), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_Dhat, &dt->Dhat, sizeof(double*)));
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_D, &dt->D, sizeof(double*)));
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_T, &dt->T, sizeof(double*)));
  // float-pair copies
  DevTables2 h2;
  memset(&h2, 0, sizeof(h2));
  for (int n = 1; n < kNP; ++n)
    for (int j = 0; j < n; ++j) {
      h2.lm[n][j] = split2(h.lm[n][j]);
      h2.lp[n][j] = split2(h.lp[n][j]);
      h2.lmw[n][j] = split2(h.lmw[n][j]);
      h2.lpw[n][j] = split2(h.lpw[n][j]);
    }
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_tab2, &h2, sizeof(h2)));
  std::vector<float2> Dh2(Dh.size()), Dc2(Dc.size()), Tm2(Tm.size());
  for (size_t i = 0; i < Dh.size(); ++i) Dh2[i] = split2(Dh[i]);
  for (size_t i = 0; i < Dc.size(); ++i) Dc2[i] = split2(Dc[i]);
  for (size_t i = 0; i < Tm.size(); ++i) Tm2[i] = split2(Tm[i]);
  if (!dt->Dhat2) {
    DG_CUDA_TRY(cudaMalloc(&dt->Dhat2, Dh2.size() * sizeof(float2)));
    DG_CUDA_TRY(cudaMalloc(&dt->D2, Dc2.size() * sizeof(float2)));
    DG_CUDA_TRY(cudaMalloc(&dt->T2, Tm2.size() * sizeof(float2)));
  }
  DG_CUDA_TRY(cudaMemcpy(dt->Dhat2, Dh2.data(), Dh2.size() * sizeof(float2), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpy(dt->D2, Dc2.data(), Dc2.size() * sizeof(float2), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpy(dt->T2, Tm2.data(), Tm2.size() * sizeof(float2), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_Dhat2, &dt->Dhat2, sizeof(float2*)));
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_D2, &dt->D2, sizeof(float2*)));
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_T2, &dt->T2, sizeof(float2*)));
  // value-only pairs (derivative 0) for the tangent arithmetic
  for (size_t i = 0; i < Dh.size(); ++i) Dh2[i] = make_float2((float)Dh[i], 0.0f);
  for (size_t i = 0; i < Dc.size(); ++i) Dc2[i] = make_float2((float)Dc[i], 0.0f);
  for (size_t i = 0; i < Tm.size(); ++i) Tm2[i] = make_float2((float)Tm[i], 0.0f);
  if (!dt->DhatT) {
    DG_CUDA_TRY(cudaMalloc(&dt->DhatT, Dh2.size() * sizeof(float2)));
    DG_CUDA_TRY(cudaMalloc(&dt->DT, Dc2.size() * sizeof(float2)));
    DG_CUDA_TRY(cudaMalloc(&dt->TT, Tm2.size() * sizeof(float2)));
  }
  DG_CUDA_TRY(cudaMemcpy(dt->DhatT, Dh2.data(), Dh2.size() * sizeof(float2), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpy(dt->DT, Dc2.data(), Dc2.size() * sizeof(float2), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpy(dt->TT, Tm2.data(), Tm2.size() * sizeof(float2), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_DhatT, &dt->DhatT, sizeof(float2*)));
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_DT, &dt->DT, sizeof(float2*)));
  DG_CUDA_TRY(cudaMemcpyToSymbol(c_TT, &dt->TT, sizeof(float2*)));
  dt->ready = true;
  return DG_OK;
}

// ---------------------------------------------------------------------------
// device physics (Appendix A), generic over the arithmetic type R
// ---------------------------------------------------------------------------
#define DEV __device__ __forceinline__

// Programmatic dependent launch.  The kernels of the operator chain are
// launched with the programmatic-serialisation attribute (launch_k below),
// so the GPU processes the launch of a kernel while its predecessor in the
// stream still runs, instead of after it.  Each such kernel starts with
// pdl_enter(): griddepcontrol.wait returns once the preceding kernel has
// completed and its writes are visible (the kernel reads and writes nothing
// before it).  No kernel triggers its dependents early: they launch as its
// CTAs exit, so a dependent's CTAs are not placed on whichever SMs happened
// to have room while this kernel ran (the FP64 kernels' time follows their
// most loaded SM).  On a launch without a programmatic predecessor the wait
// returns at once.
DEV void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Where the attribute is set: DG_LAUNCH_PDL=0 never, 1 on streams that are
// not being captured, 2 (default) also inside captured graphs.  Measured on
// GB300, flat plate 60x24 at N = 7, one V-cycle 7 -> 1 (2/2/4 sweeps):
//   FP64   direct 8.54 -> 7.52 ms, graph 7.58 -> 7.52 ms
//   mixed  direct 4.75 -> 3.61 ms, graph 3.83 -> 3.62 ms
// (an earlier form that triggered dependents at kernel entry made the FP64
// cycle slower, 10.3 ms, through the placement of the dependents' CTAs).
// The knob selects the launch mode only; the work is the same.
static int pdl_mode() {
  static const int mode = [] {
    const char* e = std::getenv("DG_LAUNCH_PDL");
    return e ? std::atoi(e) : 2;
  }();
  return mode;
}

template <typename... KArgs, typename... Args>
static void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 0;
  const int mode = pdl_mode();
  if (mode == 2) {
    cfg.numAttrs = 1;
  } else if (mode == 1) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) cfg.numAttrs = 1;
  }
  (void)cudaLaunchKernelEx(&cfg, kern, args...);  // a launch error is read by the caller's cudaGetLastError
}

template <typename R>
DEV R cst(float x);
template <>
DEV double cst<double>(float x) {
  return (double)x;
}
template <>
DEV dd cst<dd>(float x) {
  return dd(x, 0.0f);
}
template <>
DEV tf cst<tf>(float x) {
  return tf(x, 0.0f);
}

// Gas constants in R (split into float pairs on the host for R = dd).
template <typename R>
struct GasT {
  R g1;      // gamma - 1
  R gM2;     // gamma M^2
  R igM2;    // 1 / (gamma M^2)
  R Su, Su1; // Sutherland S and 1 + S
  R hc;      // 1/((gamma-1) Pr M^2)
  R invRe;
  R two3;    // 2/3
  R qinf[5];
  R pinf;
  R ig1;     // 1/(gamma - 1)
};


template <typename R>
R host_r(double x);
template <>
double host_r<double>(double x) {
  return x;
}
template <>
dd host_r<dd>(double x) {
  dd v;
  v.hi = (float)x;
  v.lo = (float)(x - (double)v.hi);
  return v;
}
template <>
tf host_r<tf>(double x) {
  tf v;
  v.v = (float)x;
  v.t = 0.0f;  // constants of the gas do not depend on the state
  return v;
}

template <typename R>
GasT<R> make_gas(const Params& P) {
  GasT<R> G;
  G.g1 = host_r<R>(P.g - 1.0);
  G.gM2 = host_r<R>(P.gM2);
  G.igM2 = host_r<R>(1.0 / P.gM2);
  G.Su = host_r<R>(P.Su);
  G.Su1 = host_r<R>(1.0 + P.Su);
  G.hc = host_r<R>(P.hc);
  G.invRe = host_r<R>(P.invRe);
  G.two3 = host_r<R>(2.0 / 3.0);
  for (int v = 0; v < 5; ++v) G.qinf[v] = host_r<R>(P.qinf[v]);
  G.pinf = host_r<R>(P.pinf);
  G.ig1 = host_r<R>(1.0 / (P.g - 1.0));
  return G;
}

static GasD make_gas_d(const Params& P) {
  GasD G;
  G.g = P.g;
  G.g1 = P.g - 1.0;
  G.gM2 = P.gM2;
  G.Su = P.Su;
  G.Su1 = 1.0 + P.Su;
  G.invRe = P.invRe;
  G.Ca = P.Ca;
  G.Cnu = P.Cnu;
  return G;
}

// primitives: 1/rho, velocity, pressure, temperature
template <typename R>
DEV void to_prim(const R* q, const GasT<R>& G, R& ir, R* u, R& p, R& T) {
  ir = cst<R>(1.0f) / q[0];
  u[0] = q[1] * ir;
  u[1] = q[2] * ir;
  u[2] = q[3] * ir;
  p = G.g1 * (q[4] - cst<R>(0.5f) * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
  T = G.gM2 * p * ir;
}

template <typename R>
DEV R mu_of_T(R T, const GasT<R>& G) {
  return T * sqrt(T) * G.Su1 / (T + G.Su);
}

// viscous flux (no 1/Re) on vector nv; grad[v*3+c] = d(u,v,w,T)_v / dx_c.
// DIM = 2: a field of the one-element-thick extrusion, whose z-derivatives
// (grad[v*3+2]) and z-components of the face and metric vectors (nv[2]) are
// exactly zero: their terms are left out (the same values; the velocity w
// and its in-plane derivatives stay).
template <typename R, int DIM = 3>
DEV void visc_flux(const R* u, R mu, const R* grad, const R* nv, const GasT<R>& G, bool heat, R* f) {
  if (DIM == 2) {
    const R div = grad[0] + grad[4];
    const R lam = -(G.two3 * mu * div);
    const R mu2 = cst<R>(2.0f) * mu;
    const R t00 = mu2 * grad[0] + lam, t11 = mu2 * grad[4] + lam;
    const R t01 = mu * (grad[1] + grad[3]), t02 = mu * grad[6], t12 = mu * grad[7];
    const R tn0 = t00 * nv[0] + t01 * nv[1];
    const R tn1 = t01 * nv[0] + t11 * nv[1];
    const R tn2 = t02 * nv[0] + t12 * nv[1];
    f[0] = cst<R>(0.0f);
    f[1] = tn0;
    f[2] = tn1;
    f[3] = tn2;
    R e = u[0] * tn0 + u[1] * tn1 + u[2] * tn2;
    if (heat) e += G.hc * mu * (grad[9] * nv[0] + grad[10] * nv[1]);
    f[4] = e;
    return;
  }
  const R div = grad[0] + grad[4] + grad[8];
  const R lam = -(G.two3 * mu * div);
  const R mu2 = cst<R>(2.0f) * mu;
  const R t00 = mu2 * grad[0] + lam, t11 = mu2 * grad[4] + lam, t22 = mu2 * grad[8] + lam;
  const R t01 = mu * (grad[1] + grad[3]), t02 = mu * (grad[2] + grad[6]), t12 = mu * (grad[5] + grad[7]);
  const R tn0 = t00 * nv[0] + t01 * nv[1] + t02 * nv[2];
  const R tn1 = t01 * nv[0] + t11 * nv[1] + t12 * nv[2];
  const R tn2 = t02 * nv[0] + t12 * nv[1] + t22 * nv[2];
  f[0] = cst<R>(0.0f);
  f[1] = tn0;
  f[2] = tn1;
  f[3] = tn2;
  R e = u[0] * tn0 + u[1] * tn1 + u[2] * tn2;
  if (heat) e += G.hc * mu * (grad[9] * nv[0] + grad[10] * nv[1] + grad[11] * nv[2]);
  f[4] = e;
}

// visc_flux for a dimension known at run time (the mortar kernels serve both)
template <typename R>
DEV void visc_flux_dim(int dim, const R* u, R mu, const R* grad, const R* nv, const GasT<R>& G, bool heat, R* f) {
  if (dim == 2)
    visc_flux<R, 2>(u, mu, grad, nv, G, heat, f);
  else
    visc_flux<R, 3>(u, mu, grad, nv, G, heat, f);
}

// Roe flux for unit normal n (textbook averages, five waves, no entropy fix)
// (the primitives 1/rho, u, p of both states are passed in: the mortar kernel
// reuses them for the viscous fluxes)
template <typename R>
DEV void roe(const R* qL, const R* qR, R irL, const R* uL, R pL, R irR, const R* uR, R pR, const R* n,
             const GasT<R>& G, R* f) {
  const R half = cst<R>(0.5f);
  const R unL = uL[0] * n[0] + uL[1] * n[1] + uL[2] * n[2];
  const R unR = uR[0] * n[0] + uR[1] * n[1] + uR[2] * n[2];
  const R HL = (qL[4] + pL) * irL, HR = (qR[4] + pR) * irR;
  const R pLR = pL + pR;
  f[0] = half * (qL[0] * unL + qR[0] * unR);
  f[1] = half * (qL[1] * unL + qR[1] * unR + pLR * n[0]);
  f[2] = half * (qL[2] * unL + qR[2] * unR + pLR * n[1]);
  f[3] = half * (qL[3] * unL + qR[3] * unR + pLR * n[2]);
  f[4] = half * (qL[0] * HL * unL + qR[0] * HR * unR);
  const R sL = sqrt(qL[0]), sR = sqrt(qR[0]);
  const R iw = cst<R>(1.0f) / (sL + sR);
  const R ut0 = (sL * uL[0] + sR * uR[0]) * iw, ut1 = (sL * uL[1] + sR * uR[1]) * iw,
          ut2 = (sL * uL[2] + sR * uR[2]) * iw;
  const R Ht = (sL * HL + sR * HR) * iw;
  const R rt = sL * sR;
  const R q2 = ut0 * ut0 + ut1 * ut1 + ut2 * ut2;
  const R c2 = G.g1 * (Ht - half * q2);
  const R ct = sqrt(c2);
  const R ic2 = cst<R>(1.0f) / c2;
  const R unt = ut0 * n[0] + ut1 * n[1] + ut2 * n[2];
  const R dp = pR - pL, dr = qR[0] - qL[0];
  const R du0 = uR[0] - uL[0], du1 = uR[1] - uL[1], du2 = uR[2] - uL[2];
  const R dun = unR - unL;
  const R rcd = rt * ct * dun;
  const R a1 = half * (dp - rcd) * ic2;
  const R a5 = half * (dp + rcd) * ic2;
  const R a2 = dr - dp * ic2;
  const R l1 = fabs(unt - ct) * a1, l5 = fabs(unt + ct) * a5, l2 = fabs(unt);
  const R e2 = l2 * a2;
  const R dt0 = du0 - dun * n[0], dt1 = du1 - dun * n[1], dt2 = du2 - dun * n[2];
  const R sh = l2 * rt;
  const R cn0 = ct * n[0], cn1 = ct * n[1], cn2 = ct * n[2];
  const R d0 = l1 + l5 + e2;
  const R d1 = l1 * (ut0 - cn0) + l5 * (ut0 + cn0) + e2 * ut0 + sh * dt0;
  const R d2 = l1 * (ut1 - cn1) + l5 * (ut1 + cn1) + e2 * ut1 + sh * dt1;
  const R d3 = l1 * (ut2 - cn2) + l5 * (ut2 + cn2) + e2 * ut2 + sh * dt2;
  const R uc = unt * ct;
  const R d4 = l1 * (Ht - uc) + l5 * (Ht + uc) + e2 * half * q2 + sh * (ut0 * dt0 + ut1 * dt1 + ut2 * dt2);
  f[0] -= half * d0;
  f[1] -= half * d1;
  f[2] -= half * d2;
  f[3] -= half * d3;
  f[4] -= half * d4;
}

template <typename R>
DEV void ghost(int bc, const R* qi, const R* nu, const GasT<R>& G, R* qg) {
  if (bc == DG_BC_FREESTREAM) {
#pragma unroll
    for (int v = 0; v < 5; ++v) qg[v] = G.qinf[v];
    return;
  }
  if (bc == DG_BC_OUTFLOW) {
    const R ke = cst<R>(0.5f) * (qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]) / qi[0];
    qg[0] = qi[0];
    qg[1] = qi[1];
    qg[2] = qi[2];
    qg[3] = qi[3];
    qg[4] = G.pinf * G.ig1 + ke;
    return;
  }
  if (bc == DG_BC_SLIP) {
    const R mn2 = cst<R>(2.0f) * (qi[1] * nu[0] + qi[2] * nu[1] + qi[3] * nu[2]);
    qg[0] = qi[0];
    qg[1] = qi[1] - mn2 * nu[0];
    qg[2] = qi[2] - mn2 * nu[1];
    qg[3] = qi[3] - mn2 * nu[2];
    qg[4] = qi[4];
    return;
  }
  // wall: negated velocity, same density and internal energy
  qg[0] = qi[0];
  qg[1] = -qi[1];
  qg[2] = -qi[2];
  qg[3] = -qi[3];
  qg[4] = qi[4];
}

// Reduce v into dst[slot] for the active lanes of a warp: one atomic when all
// participating lanes share a slot (single solves, sorted batches), one per
// lane otherwise.  Every lane of the warp must call it.
template <bool MAX>
DEV void warp_slot_reduce(double* dst, int slot, double v, bool active);

DEV void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}
DEV void atomic_min_pos(double* addr, double v) {
  atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <bool MAX>
DEV void warp_slot_reduce(double* dst, int slot, double v, bool active) {
  const unsigned act = __ballot_sync(0xffffffffu, active);
  if (act == 0u) return;
  const int lead = __ffs(act) - 1;
  const int s0 = __shfl_sync(0xffffffffu, slot, lead);
  const bool uniform = __all_sync(0xffffffffu, !active || slot == s0);
  if (uniform) {
    double w = active ? v : (MAX ? 0.0 : 1e300);
    for (int o = 16; o > 0; o >>= 1) {
      const double x = __shfl_xor_sync(0xffffffffu, w, o);
      w = MAX ? fmax(w, x) : fmin(w, x);
    }
    if ((int)(threadIdx.x & 31) == lead) {
      if (MAX)
        atomic_max_nonneg(dst + s0, w);
      else
        atomic_min_pos(dst + s0, w);
    }
  } else if (active) {
    if (MAX)
      atomic_max_nonneg(dst + slot, v);
    else
      atomic_min_pos(dst + slot, v);
  }
}

// ---- tables in R ----
template <typename R>
struct Tab;
template <>
struct Tab<double> {
  static DEV double lp(int n, int j) { return c_tab.lp[n][j]; }
  static DEV double lm(int n, int j) { return c_tab.lm[n][j]; }
  static DEV double lpw(int n, int j) { return c_tab.lpw[n][j]; }
  static DEV double lmw(int n, int j) { return c_tab.lmw[n][j]; }
  static DEV const double* Dhat() { return c_Dhat; }
  static DEV const double* Dcol() { return c_D; }
  static DEV const double* T() { return c_T; }
};
template <>
struct Tab<dd> {
  static DEV dd lp(int n, int j) { return dd(c_tab2.lp[n][j].x, c_tab2.lp[n][j].y); }
  static DEV dd lm(int n, int j) { return dd(c_tab2.lm[n][j].x, c_tab2.lm[n][j].y); }
  static DEV dd lpw(int n, int j) { return dd(c_tab2.lpw[n][j].x, c_tab2.lpw[n][j].y); }
  static DEV dd lmw(int n, int j) { return dd(c_tab2.lmw[n][j].x, c_tab2.lmw[n][j].y); }
  static DEV const float2* Dhat() { return c_Dhat2; }
  static DEV const float2* Dcol() { return c_D2; }
  static DEV const float2* T() { return c_T2; }
};
template <>
struct Tab<tf> {
  static DEV tf lp(int n, int j) { return tf(c_tab2.lp[n][j].x, 0.0f); }
  static DEV tf lm(int n, int j) { return tf(c_tab2.lm[n][j].x, 0.0f); }
  static DEV tf lpw(int n, int j) { return tf(c_tab2.lpw[n][j].x, 0.0f); }
  static DEV tf lmw(int n, int j) { return tf(c_tab2.lmw[n][j].x, 0.0f); }
  static DEV const float2* Dhat() { return c_DhatT; }
  static DEV const float2* Dcol() { return c_DT; }
  static DEV const float2* T() { return c_TT; }
};

// ---------------------------------------------------------------------------
// shared helpers for element tiles
// ---------------------------------------------------------------------------
template <typename R>
struct LevelArgsT {
  using ST = typename Store<R>::T;
  const int32_t* n;
  const int32_t* off;
  const ST* geo;  // 10 x nodes
  int64_t nodes;
  const int32_t* fo;
  int64_t fn;  // face nodes
  const ST* fnS;
  const ElemTile* tiles;
  const int32_t* tile_elems;
  const int32_t* slot;  // solve slot of each element (batched meshes; all 0 otherwise)
  int dim;
  const double* base;   // tangent arithmetic: the linearisation point (the state argument is then the correction)
};

template <typename R>
static LevelArgsT<R> largs(const Level* L);
template <>
LevelArgsT<double> largs<double>(const Level* L) {
  LevelArgsT<double> a;
  a.n = L->d_n;
  a.off = L->d_off;
  a.geo = L->d_geo;
  a.nodes = L->nodes;
  a.fo = L->d_fo;
  a.fn = L->face_nodes;
  a.fnS = L->d_fnS;
  a.tiles = L->d_tiles;
  a.tile_elems = L->d_tile_elems;
  a.slot = L->d_slot;
  a.dim = L->dim;
  a.base = nullptr;
  return a;
}
template <>
LevelArgsT<dd> largs<dd>(const Level* L) {
  LevelArgsT<dd> a;
  a.n = L->d_n;
  a.off = L->d_off;
  a.geo = reinterpret_cast<const float2*>(L->d_geo2);
  a.nodes = L->nodes;
  a.fo = L->d_fo;
  a.fn = L->face_nodes;
  a.fnS = reinterpret_cast<const float2*>(L->d_fnS2);
  a.tiles = L->d_tiles;
  a.tile_elems = L->d_tile_elems;
  a.slot = L->d_slot;
  a.dim = L->dim;
  a.base = nullptr;
  return a;
}
template <>
LevelArgsT<tf> largs<tf>(const Level* L) {
  LevelArgsT<tf> a;
  a.n = L->d_n;
  a.off = L->d_off;
  a.geo = reinterpret_cast<const float2*>(L->d_geoT);
  a.nodes = L->nodes;
  a.fo = L->d_fo;
  a.fn = L->face_nodes;
  a.fnS = reinterpret_cast<const float2*>(L->d_fnST);
  a.tiles = L->d_tiles;
  a.tile_elems = L->d_tile_elems;
  a.slot = L->d_slot;
  a.dim = L->dim;
  a.base = nullptr;
  return a;
}

DEV void face_dirs(int f, int& d, int& ta, int& tb, int& side) {
  d = f >> 1;
  side = f & 1;
  ta = (d == 0) ? 1 : 0;
  tb = (d == 2) ? 1 : 2;
}

// component k of a 3-vector held in scalars (avoids local-memory arrays)
DEV int pick(int k, int a0, int a1, int a2) { return k == 0 ? a0 : (k == 1 ? a1 : a2); }

// Interpolate face values (NVAR comps, stride fs) of an na x nb face to the
// mortar point (ia, ib) of an ma x mb rule.
// Value at mortar node (ia, ib) (face frame of the trace) of a face trace with
// na x nb nodes, interpolated to ma x mb mortar nodes.  A direction in which
// the face already has the mortar's order is the identity and is skipped.
template <typename R, int NVAR>
DEV void face_interp(const typename Store<R>::T* X, int64_t fs, int na, int nb, int ma, int mb, int ia, int ib,
                     R* out) {
  using SR = Store<R>;
  if (na == ma && nb == mb) {
    int p = ib * na + ia;
#pragma unroll
    for (int v = 0; v < NVAR; ++v) out[v] = SR::get(X, v * fs + p);
    return;
  }
  const typename Store<R>::T* Ta = Tab<R>::T() + ((size_t)na * kNP + ma) * kNP * kNP + ia * na;
  const typename Store<R>::T* Tb = Tab<R>::T() + ((size_t)nb * kNP + mb) * kNP * kNP + ib * nb;
  const bool ida = (na == ma), idb = (nb == mb);
  const int a0 = ida ? ia : 0, a1 = ida ? ia + 1 : na;
  const int b0 = idb ? ib : 0, b1 = idb ? ib + 1 : nb;
#pragma unroll
  for (int v = 0; v < NVAR; ++v) out[v] = cst<R>(0.0f);
  for (int kb = b0; kb < b1; ++kb) {
    const R wb = idb ? cst<R>(1.0f) : SR::get(Tb, kb);
    for (int ka = a0; ka < a1; ++ka) {
      const R wgt = ida ? wb : wb * SR::get(Ta, ka);
      int p = kb * na + ka;
#pragma unroll
      for (int v = 0; v < NVAR; ++v) out[v] = madd(out[v], wgt, SR::get(X, v * fs + p));
    }
  }
}

// Node-count of face f of an element with node counts (n0, n1, n2)
DEV int face_size(int f, int n0, int n1, int n2) {
  int d = f >> 1;
  return d == 0 ? n1 * n2 : (d == 1 ? n0 * n2 : n0 * n1);
}

// ---------------------------------------------------------------------------
// k_trace_q: conserved state at every face node of every element
// ---------------------------------------------------------------------------
// Conserved state at every face node of the tile's elements from the staged
// state sq (5 x T, variable-major): interpolation to xi_d = -1 / +1 along
// the face's normal direction.
template <typename R, int DIM>
DEV void write_face_traces(const LevelArgsT<R>& A, const ElemTile& t, const R* sq, int T,
                           typename Store<R>::T* __restrict__ trq) {
  const int n0 = t.n[0], n1 = t.n[1], n2 = t.n[2];
  const int nn = n0 * n1 * n2;
  int FE = 0;
#pragma unroll
  for (int f = 0; f < 2 * DIM; ++f) FE += face_size(f, n0, n1, n2);
  for (int i = threadIdx.x; i < t.count * FE; i += blockDim.x) {
    int le = i / FE, r = i - le * FE;
    int f = 0;
    while (r >= face_size(f, n0, n1, n2)) {
      r -= face_size(f, n0, n1, n2);
      ++f;
    }
    int d, ta, tb, side;
    face_dirs(f, d, ta, tb, side);
    const int nta = pick(ta, n0, n1, n2), nd = pick(d, n0, n1, n2);
    int ia = r % nta, ib = r / nta;
    int i0 = (d == 0) ? 0 : ia;
    int i1 = (d == 1) ? 0 : (d == 0 ? ia : ib);
    int i2 = (d == 2) ? 0 : ib;
    int base = (i2 * n1 + i1) * n0 + i0;
    int sd = (d == 0) ? 1 : (d == 1 ? n0 : n0 * n1);
    int e = A.tile_elems[t.first + le];
    int64_t p = A.fo[e * 6 + f] + r;
    const R* s0 = sq + le * nn + base;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R acc = cst<R>(0.0f);
      for (int k = 0; k < nd; ++k) acc = madd(acc, (side ? Tab<R>::lp(nd, k) : Tab<R>::lm(nd, k)), s0[v * T + k * sd]);
      Store<R>::put(trq, v * A.fn + p, acc);
    }
  }
}

// face traces of the state of one element tile (sq: 5 x tile nodes of shared memory)
template <typename R, int DIM>
DEV void trace_tile(const LevelArgsT<R>& A, int tile, const double* __restrict__ q,
                    typename Store<R>::T* __restrict__ trq, R* sq) {
  const ElemTile t = A.tiles[tile];
  const int nn = t.n[0] * t.n[1] * t.n[2];
  const int T = t.count * nn;
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    int le = i / nn, node = i - le * nn;
    int e = A.tile_elems[t.first + le];
#pragma unroll
    for (int v = 0; v < 5; ++v) sq[v * T + i] = state_value<R>(q, A.base, (size_t)5 * A.off[e] + v * nn + node);
  }
  __syncthreads();
  write_face_traces<R, DIM>(A, t, sq, T, trq);
}

template <typename R, int DIM>
__global__ void __launch_bounds__(kTileNodes) k_trace_q(LevelArgsT<R> A, const double* __restrict__ q,
                                                        typename Store<R>::T* __restrict__ trq) {
  pdl_enter();
  extern __shared__ double smem_raw[];
  trace_tile<R, DIM>(A, blockIdx.x, q, trq, reinterpret_cast<R*>(smem_raw));
}

// ---------------------------------------------------------------------------
// k_mortar<PASS>: PASS 1 = BR1 average U*, PASS 2 = Roe + BR1 viscous flux
// ---------------------------------------------------------------------------
template <typename R>
struct MortarArgsT {
  const MortarDev* mortars;
  const int32_t* mnode_mortar;
  const typename Store<R>::T* mnS;
  int64_t mnodes;
  const MortarTile* tiles;
};

template <typename R>
static MortarArgsT<R> margs(const Level* L) {
  MortarArgsT<R> a;
  a.mortars = L->d_mortars;
  a.mnode_mortar = L->d_mnode_mortar;
  a.mnS = std::is_same<R, dd>::value   ? reinterpret_cast<const typename Store<R>::T*>(L->d_mnS2)
          : std::is_same<R, tf>::value ? reinterpret_cast<const typename Store<R>::T*>(L->d_mnST)
                                       : reinterpret_cast<const typename Store<R>::T*>(L->d_mnS);
  a.mnodes = L->mortar_nodes;
  a.tiles = L->d_mtiles;
  return a;
}

// value at one mortar node: U* (PASS 1) or F* S-hat (PASS 2)
template <typename R, int PASS>
DEV void mortar_node_value(const LevelArgsT<R>& A, const MortarArgsT<R>& MA, const GasT<R>& G,
                           const typename Store<R>::T* __restrict__ trq, const typename Store<R>::T* __restrict__ trg,
                           int64_t gp, R* o) {
  using SR = Store<R>;
  const R half = cst<R>(0.5f);
  const MortarDev M = MA.mortars[MA.mnode_mortar[gp]];
  const int loc = (int)(gp - M.node_off);
  const int a = loc % M.ma, b = loc / M.ma;
  int dL, taL, tbL, sL;
  face_dirs(M.fL, dL, taL, tbL, sL);
  const int nLa = A.n[M.eL * 3 + taL], nLb = A.n[M.eL * 3 + tbL];
  const int64_t pL = A.fo[M.eL * 6 + M.fL];
  R qL[5], qR[5];
  face_interp<R, 5>(trq + pL, A.fn, nLa, nLb, M.ma, M.mb, a, b, qL);
  const R nS0 = SR::get(MA.mnS, gp), nS1 = SR::get(MA.mnS, MA.mnodes + gp), nS2 = SR::get(MA.mnS, 2 * MA.mnodes + gp);
  const R S = sqrt(nS0 * nS0 + nS1 * nS1 + nS2 * nS2);
  const R iS = cst<R>(1.0f) / S;
  const R nu[3] = {nS0 * iS, nS1 * iS, nS2 * iS};
  int Ra = 0, Rb = 0, Ma = 0, Mb = 0, ia = 0, ib = 0;
  int64_t pR = 0;
  if (M.eR >= 0) {
    int dR, taR, tbR, sR;
    face_dirs(M.fR, dR, taR, tbR, sR);
    Ra = A.n[M.eR * 3 + taR];
    Rb = A.n[M.eR * 3 + tbR];
    const bool sw = M.orient & 1;
    Ma = sw ? M.mb : M.ma;
    Mb = sw ? M.ma : M.mb;
    ia = sw ? b : a;
    ib = sw ? a : b;
    if (M.orient & 2) ia = Ma - 1 - ia;
    if (M.orient & 4) ib = Mb - 1 - ib;
    pR = A.fo[M.eR * 6 + M.fR];
    face_interp<R, 5>(trq + pR, A.fn, Ra, Rb, Ma, Mb, ia, ib, qR);
  } else {
    ghost(M.bc, qL, nu, G, qR);
  }
  if (PASS == 1) {
    R ir, u[3], p, T, u2[3], T2;
    to_prim(qL, G, ir, u, p, T);
    to_prim(qR, G, ir, u2, p, T2);
    o[0] = half * (u[0] + u2[0]);
    o[1] = half * (u[1] + u2[1]);
    o[2] = half * (u[2] + u2[2]);
    o[3] = half * (T + T2);
    return;
  }
  R f[5];
  R irL, uL[3], pLs, TL, irR, uR[3], pRs, TR;
  to_prim(qL, G, irL, uL, pLs, TL);
  to_prim(qR, G, irR, uR, pRs, TR);
  roe(qL, qR, irL, uL, pLs, irR, uR, pRs, nu, G, f);
  if (!(M.eR < 0 && M.bc == DG_BC_SLIP)) {
    R g[12], fv[5];
    face_interp<R, 12>(trg + pL, A.fn, nLa, nLb, M.ma, M.mb, a, b, g);
    const R mu = mu_of_T(TL, G);
    if (M.eR < 0 && M.bc == DG_BC_WALL) {
      const R z[3] = {cst<R>(0.0f), cst<R>(0.0f), cst<R>(0.0f)};
      visc_flux_dim(A.dim, z, mu, g, nu, G, false, fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) f[v] -= G.invRe * fv[v];
    } else {
      const R hre = half * G.invRe;
      visc_flux_dim(A.dim, uL, mu, g, nu, G, true, fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) f[v] -= hre * fv[v];
      if (M.eR >= 0) face_interp<R, 12>(trg + pR, A.fn, Ra, Rb, Ma, Mb, ia, ib, g);  // else: interior gradient
      visc_flux_dim(A.dim, uR, mu_of_T(TR, G), g, nu, G, true, fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) f[v] -= hre * fv[v];
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) o[v] = S * f[v];
}

// L2 projection of mortar values (ma x mb nodes in the mortar's L frame,
// stride 5 per node) onto face node (ka, kb) of a side with na x nb nodes.
// (Ma, Mb) are the mortar's node counts in that side's frame and `orient`
// the face orientation code from the L frame to it (0 for the L side).  A
// direction in which the side has the mortar's order is the identity.
template <typename R, int NV>
DEV void mortar_project(const R* vals, int ma, int mb, int Ma, int Mb, int orient, int na, int nb, int ka, int kb,
                        R* acc) {
  using SR = Store<R>;
  const bool ida = (na == Ma), idb = (nb == Mb);
  const typename SR::T* Pa = Tab<R>::T() + ((size_t)Ma * kNP + na) * kNP * kNP + ka * Ma;
  const typename SR::T* Pb = Tab<R>::T() + ((size_t)Mb * kNP + nb) * kNP * kNP + kb * Mb;
  const int a0 = ida ? ka : 0, a1 = ida ? ka + 1 : Ma;
  const int b0 = idb ? kb : 0, b1 = idb ? kb + 1 : Mb;
  const bool sw = orient & 1;
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = cst<R>(0.0f);
  for (int ib = b0; ib < b1; ++ib) {
    const R wb = idb ? cst<R>(1.0f) : SR::get(Pb, ib);
    const int jb = (orient & 4) ? Mb - 1 - ib : ib;
    for (int ia = a0; ia < a1; ++ia) {
      const R wgt = ida ? wb : wb * SR::get(Pa, ia);
      const int ja = (orient & 2) ? Ma - 1 - ia : ia;
      const int aa = sw ? jb : ja, bb = sw ? ja : jb;  // back to the L frame
      const R* x = vals + (bb * ma + aa) * 5;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = madd(acc[v], wgt, x[v]);
    }
  }
}

template <typename R, int PASS>
__global__ void __launch_bounds__(kMortarTile, 8) k_mortar(LevelArgsT<R> A, MortarArgsT<R> MA,
                                                           const GasT<R>* __restrict__ gas,
                                                           const typename Store<R>::T* __restrict__ trq,
                                                           const typename Store<R>::T* __restrict__ trg,
                                                           typename Store<R>::T* __restrict__ out) {
  pdl_enter();
  using SR = Store<R>;
  constexpr int NV = (PASS == 1) ? 4 : 5;
  __shared__ R sval[kMortarTileMax * 5];
  __shared__ int scum[kMortarTileMax + 1];
  const MortarTile mt = MA.tiles[blockIdx.x];
  for (int i = threadIdx.x; i < mt.nodes; i += blockDim.x) {
    const int64_t gp = mt.node_first + i;
    const GasT<R>& G = gas[A.slot[MA.mortars[MA.mnode_mortar[gp]].eL]];
    mortar_node_value<R, PASS>(A, MA, G, trq, trg, gp, sval + i * 5);
  }
  for (int m = threadIdx.x; m < mt.count; m += blockDim.x) scum[m] = MA.mortars[mt.first + m].out_off;
  if (threadIdx.x == 0) scum[mt.count] = mt.outs;
  __syncthreads();
  // L2 projection of the mortar values back onto each side's face nodes
  for (int i = threadIdx.x; i < mt.outs; i += blockDim.x) {
    int lo = 0, hi = mt.count - 1;  // the mortar whose outputs hold i
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (scum[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    const MortarDev M = MA.mortars[mt.first + lo];
    int r = i - scum[lo];
    const R* vals = sval + (M.node_off - mt.node_first) * 5;
    int dL, taL, tbL, sL;
    face_dirs(M.fL, dL, taL, tbL, sL);
    const int nLa = A.n[M.eL * 3 + taL], nLb = A.n[M.eL * 3 + tbL];
    R acc[NV];
    int64_t dst;
    bool neg = false;
    if (r < nLa * nLb) {
      dst = A.fo[M.eL * 6 + M.fL] + r;
      mortar_project<R, NV>(vals, M.ma, M.mb, M.ma, M.mb, 0, nLa, nLb, r % nLa, r / nLa, acc);
    } else {
      r -= nLa * nLb;
      int dR, taR, tbR, sR;
      face_dirs(M.fR, dR, taR, tbR, sR);
      const int Ra = A.n[M.eR * 3 + taR], Rb = A.n[M.eR * 3 + tbR];
      const bool sw = M.orient & 1;
      dst = A.fo[M.eR * 6 + M.fR] + r;
      neg = (PASS == 2);
      mortar_project<R, NV>(vals, M.ma, M.mb, sw ? M.mb : M.ma, sw ? M.ma : M.mb, M.orient, Ra, Rb, r % Ra, r / Ra,
                            acc);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) SR::put(out, v * A.fn + dst, neg ? -acc[v] : acc[v]);
  }
}

// k_mortar_conf<PASS>: the same two passes on a level whose mortars are all
// conforming (both sides carry the mortar's order in each tangential
// direction, e.g. every level of a uniform-order mesh).  The L2 projection
// back is then the identity, so each thread computes one mortar node and
// writes it to the L side's face node and, through the face orientation, to
// the R side's (negated for the flux): no shared memory, no barrier, no
// search for the owning mortar, and CTAs of any size.  Same bits as the tile
// kernel, whose identity projection is an exact copy.
constexpr int kMortarConfThreads = 32;  // one warp: spreads a level's warps evenly over the SMs

// mortar node gp of a conforming level (no-op past the last node)
template <typename R, int PASS>
DEV void mortar_conf_node(const LevelArgsT<R>& A, const MortarArgsT<R>& MA, const GasT<R>* __restrict__ gas,
                          const typename Store<R>::T* __restrict__ trq, const typename Store<R>::T* __restrict__ trg,
                          typename Store<R>::T* __restrict__ out, int64_t gp) {
  using SR = Store<R>;
  constexpr int NV = (PASS == 1) ? 4 : 5;
  if (gp >= MA.mnodes) return;
  const MortarDev M = MA.mortars[MA.mnode_mortar[gp]];
  R o[5];
  mortar_node_value<R, PASS>(A, MA, gas[A.slot[M.eL]], trq, trg, gp, o);
  const int loc = (int)(gp - M.node_off);
  const int a = loc % M.ma, b = loc / M.ma;
  const int64_t dL = A.fo[M.eL * 6 + M.fL] + b * M.ma + a;  // L face node = mortar node (L frame)
#pragma unroll
  for (int v = 0; v < NV; ++v) SR::put(out, v * A.fn + dL, o[v]);
  if (M.eR >= 0) {
    const bool sw = M.orient & 1;
    const int Ma = sw ? M.mb : M.ma, Mb = sw ? M.ma : M.mb;
    int ia = sw ? b : a, ib = sw ? a : b;
    if (M.orient & 2) ia = Ma - 1 - ia;
    if (M.orient & 4) ib = Mb - 1 - ib;
    const int64_t dR = A.fo[M.eR * 6 + M.fR] + ib * Ma + ia;
#pragma unroll
    for (int v = 0; v < NV; ++v) SR::put(out, v * A.fn + dR, PASS == 2 ? -o[v] : o[v]);
  }
}

template <typename R, int PASS>
__global__ void __launch_bounds__(kMortarConfThreads, 12)
    k_mortar_conf(LevelArgsT<R> A, MortarArgsT<R> MA, const GasT<R>* __restrict__ gas,
                  const typename Store<R>::T* __restrict__ trq, const typename Store<R>::T* __restrict__ trg,
                  typename Store<R>::T* __restrict__ out) {
  pdl_enter();
  mortar_conf_node<R, PASS>(A, MA, gas, trq, trg, out, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// k_mortar_conf_flux: the flux pass of k_mortar_conf with each node's work
// on two warps: 32 mortar nodes per CTA, the first warp forms the Roe flux,
// the second the BR1 viscous fluxes of both sides; both then combine them
// in the order of mortar_node_value (Roe, minus the L viscous term, minus
// the R one), so the bits are the same, and write the L and the R face
// node.  Each warp's serial FP64 chain is about half of one thread's in
// k_mortar_conf<2>, and an SM holds twice the warps.
template <typename R>
__global__ void __launch_bounds__(64, 6)
    k_mortar_conf_flux(LevelArgsT<R> A, MortarArgsT<R> MA, const GasT<R>* __restrict__ gas,
                       const typename Store<R>::T* __restrict__ trq, const typename Store<R>::T* __restrict__ trg,
                       typename Store<R>::T* __restrict__ out) {
  pdl_enter();
  using SR = Store<R>;
  __shared__ R s_roe[32][5], s_vl[32][5], s_vr[32][5];
  const int lane = threadIdx.x & 31, part = threadIdx.x >> 5;
  const int64_t gp = blockIdx.x * (int64_t)32 + lane;
  const bool act = gp < MA.mnodes;
  const R half = cst<R>(0.5f);
  MortarDev M{};
  int a = 0, b = 0, Ma = 0, ia = 0, ib = 0;
  R S = cst<R>(0.0f);
  if (act) {
    M = MA.mortars[MA.mnode_mortar[gp]];
    const GasT<R>& G = gas[A.slot[M.eL]];
    const int loc = (int)(gp - M.node_off);
    a = loc % M.ma;
    b = loc / M.ma;
    int dL, taL, tbL, sL;
    face_dirs(M.fL, dL, taL, tbL, sL);
    const int nLa = A.n[M.eL * 3 + taL], nLb = A.n[M.eL * 3 + tbL];
    const int64_t pL = A.fo[M.eL * 6 + M.fL];
    R qL[5], qR[5];
    face_interp<R, 5>(trq + pL, A.fn, nLa, nLb, M.ma, M.mb, a, b, qL);
    const R nS0 = SR::get(MA.mnS, gp), nS1 = SR::get(MA.mnS, MA.mnodes + gp), nS2 = SR::get(MA.mnS, 2 * MA.mnodes + gp);
    S = sqrt(nS0 * nS0 + nS1 * nS1 + nS2 * nS2);
    const R iS = cst<R>(1.0f) / S;
    const R nu[3] = {nS0 * iS, nS1 * iS, nS2 * iS};
    int Ra = 0, Rb = 0, Mb = 0;
    int64_t pR = 0;
    if (M.eR >= 0) {
      int dR, taR, tbR, sR;
      face_dirs(M.fR, dR, taR, tbR, sR);
      Ra = A.n[M.eR * 3 + taR];
      Rb = A.n[M.eR * 3 + tbR];
      const bool sw = M.orient & 1;
      Ma = sw ? M.mb : M.ma;
      Mb = sw ? M.ma : M.mb;
      ia = sw ? b : a;
      ib = sw ? a : b;
      if (M.orient & 2) ia = Ma - 1 - ia;
      if (M.orient & 4) ib = Mb - 1 - ib;
      pR = A.fo[M.eR * 6 + M.fR];
      face_interp<R, 5>(trq + pR, A.fn, Ra, Rb, Ma, Mb, ia, ib, qR);
    } else {
      ghost(M.bc, qL, nu, G, qR);
    }
    R irL, uL[3], pLs, TL, irR, uR[3], pRs, TR;
    to_prim(qL, G, irL, uL, pLs, TL);
    to_prim(qR, G, irR, uR, pRs, TR);
    if (part == 0) {
      R f[5];
      roe(qL, qR, irL, uL, pLs, irR, uR, pRs, nu, G, f);
#pragma unroll
      for (int v = 0; v < 5; ++v) s_roe[lane][v] = f[v];
    } else if (!(M.eR < 0 && M.bc == DG_BC_SLIP)) {
      R g[12], fv[5];
      face_interp<R, 12>(trg + pL, A.fn, nLa, nLb, M.ma, M.mb, a, b, g);
      const R mu = mu_of_T(TL, G);
      if (M.eR < 0 && M.bc == DG_BC_WALL) {
        const R z[3] = {cst<R>(0.0f), cst<R>(0.0f), cst<R>(0.0f)};
        visc_flux_dim(A.dim, z, mu, g, nu, G, false, fv);
#pragma unroll
        for (int v = 0; v < 5; ++v) s_vl[lane][v] = fv[v];
      } else {
        visc_flux_dim(A.dim, uL, mu, g, nu, G, true, fv);
#pragma unroll
        for (int v = 0; v < 5; ++v) s_vl[lane][v] = fv[v];
        if (M.eR >= 0) face_interp<R, 12>(trg + pR, A.fn, Ra, Rb, Ma, Mb, ia, ib, g);  // else: interior gradient
        visc_flux_dim(A.dim, uR, mu_of_T(TR, G), g, nu, G, true, fv);
#pragma unroll
        for (int v = 0; v < 5; ++v) s_vr[lane][v] = fv[v];
      }
    }
  }
  __syncthreads();
  if (!act) return;
  const GasT<R>& G = gas[A.slot[M.eL]];
  R o[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) o[v] = s_roe[lane][v];
  if (!(M.eR < 0 && M.bc == DG_BC_SLIP)) {
    if (M.eR < 0 && M.bc == DG_BC_WALL) {
#pragma unroll
      for (int v = 0; v < 5; ++v) o[v] -= G.invRe * s_vl[lane][v];
    } else {
      const R hre = half * G.invRe;
#pragma unroll
      for (int v = 0; v < 5; ++v) o[v] -= hre * s_vl[lane][v];
#pragma unroll
      for (int v = 0; v < 5; ++v) o[v] -= hre * s_vr[lane][v];
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) o[v] = S * o[v];
  if (part == 0) {  // L face node = mortar node (L frame)
    const int64_t dL = A.fo[M.eL * 6 + M.fL] + b * M.ma + a;
#pragma unroll
    for (int v = 0; v < 5; ++v) SR::put(out, v * A.fn + dL, o[v]);
  } else if (M.eR >= 0) {  // R face node through the orientation, negated
    const int64_t dR = A.fo[M.eR * 6 + M.fR] + ib * Ma + ia;
#pragma unroll
    for (int v = 0; v < 5; ++v) SR::put(out, v * A.fn + dR, -o[v]);
  }
}

// ---------------------------------------------------------------------------
// element kernels: staging, BR1 gradient, fluxes, divergence
// ---------------------------------------------------------------------------
template <typename R>
DEV void load_dtables(R* sD, const typename Store<R>::T* src, int n0, int n1, int n2, int dim) {
  // sD[d][i][a] with stride kNP*kNP per direction
  for (int d = 0; d < dim; ++d) {
    const int nd = pick(d, n0, n1, n2);
    for (int k = threadIdx.x; k < nd * nd; k += blockDim.x) {
      int i = k / nd, a = k - i * nd;
      sD[d * kNP * kNP + i * kNP + a] = Store<R>::get(src, ((size_t)nd * kNP + i) * kNP + a);
    }
  }
}

// Stage the tile: conserved state (sq), primitives u,v,w,T (sA[0..3]) and the
// nine metric components (sA[4..12]).
template <typename R, int DIM>
DEV void stage_tile(const LevelArgsT<R>& A, const ElemTile& t, int nn, int T, const GasT<R>* __restrict__ gas,
                    const double* __restrict__ q, R* sq, R* sA) {
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    int le = i / nn, node = i - le * nn;
    int e = A.tile_elems[t.first + le];
    const GasT<R>& G = gas[A.slot[e]];
    const int64_t gn = A.off[e] + node;
    R qq[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      qq[v] = state_value<R>(q, A.base, (size_t)5 * A.off[e] + v * nn + node);
      sq[v * T + i] = qq[v];
    }
    R ir, u[3], p, Tt;
    to_prim(qq, G, ir, u, p, Tt);
    sA[0 * T + i] = u[0];
    sA[1 * T + i] = u[1];
    sA[2 * T + i] = u[2];
    sA[3 * T + i] = Tt;
    // a 2D field reads only the in-plane components of Ja^1 and Ja^2
#pragma unroll
    for (int c = 0; c < 9; ++c)
      if (DIM == 3 || c == 0 || c == 1 || c == 3 || c == 4) sA[(4 + c) * T + i] = Store<R>::get(A.geo, c * A.nodes + gn);
  }
}

// Volume part of the gradient at node i of the tile: sum_d D^d (Ja^d U).
// AFFINE: the metrics are constant in the element, so Ja^d is factored out
// of the contraction (same value, 4 instead of 15 operations per point).
// LIFT (affine elements only): the surface part of the BR1 gradient joins the
// same per-direction sum.  On an affine element the outward face metric of
// faces 2d and 2d+1 is -Ja^d and +Ja^d (the face value of a constant field),
// so the lifted U* of those two faces (weights l(-1)/w and l(+1)/w) is added
// to the contraction before the one metric product: 8 FMA per direction
// instead of 30 operations.  ust: U* at the element's face nodes (4
// variables, stride fn), fo_e: the element's six face offsets.
template <typename R, int DIM, bool AFFINE, bool LIFT = false>
DEV void gradient_volume(const R* sD, const R* sA, int T, int nn, int i, int n0, int n1, int n2, R* g,
                         const typename Store<R>::T* __restrict__ ust = nullptr, const int32_t* fo_e = nullptr,
                         int64_t fn = 0) {
  static_assert(AFFINE || !LIFT, "the folded lifting needs constant metrics");
  const int le = i / nn, node = i - le * nn;
  const int idx0 = node % n0, idx1 = (node / n0) % n1, idx2 = node / (n0 * n1);
#pragma unroll
  for (int k = 0; k < 12; ++k) g[k] = cst<R>(0.0f);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int id = pick(d, idx0, idx1, idx2), nd = pick(d, n0, n1, n2);
    const int sd = (d == 0) ? 1 : (d == 1 ? n0 : n0 * n1);
    const int base = le * nn + node - id * sd;
    const R* Drow = sD + d * kNP * kNP + id * kNP;
    if (AFFINE) {
      R cu[4] = {cst<R>(0.0f), cst<R>(0.0f), cst<R>(0.0f), cst<R>(0.0f)};
      for (int a = 0; a < nd; ++a) {
        const int la = base + a * sd;
        const R c = Drow[a];
#pragma unroll
        for (int v = 0; v < 4; ++v) cu[v] = madd(cu[v], c, sA[v * T + la]);
      }
      if (LIFT) {
        const int ta = (d == 0) ? 1 : 0, tb = (d == 2) ? 1 : 2;  // face_dirs of faces 2d, 2d+1
        const int fp = pick(tb, idx0, idx1, idx2) * pick(ta, n0, n1, n2) + pick(ta, idx0, idx1, idx2);
        const int64_t pm = fo_e[2 * d] + fp, pp = fo_e[2 * d + 1] + fp;
        const R wm = -Tab<R>::lmw(nd, id), wp = Tab<R>::lpw(nd, id);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          cu[v] = madd(cu[v], wm, Store<R>::get(ust, v * fn + pm));
          cu[v] = madd(cu[v], wp, Store<R>::get(ust, v * fn + pp));
        }
      }
      const R j0 = sA[(4 + d * 3 + 0) * T + i], j1 = sA[(4 + d * 3 + 1) * T + i];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        g[v * 3 + 0] = madd(g[v * 3 + 0], j0, cu[v]);
        g[v * 3 + 1] = madd(g[v * 3 + 1], j1, cu[v]);
      }
      if (DIM == 3) {  // (2D: the metric's z-column is zero, so is every z-derivative)
        const R j2 = sA[(4 + d * 3 + 2) * T + i];
#pragma unroll
        for (int v = 0; v < 4; ++v) g[v * 3 + 2] = madd(g[v * 3 + 2], j2, cu[v]);
      }
    } else {
      for (int a = 0; a < nd; ++a) {
        const int la = base + a * sd;
        const R c = Drow[a];
        const R j0 = c * sA[(4 + d * 3 + 0) * T + la];
        const R j1 = c * sA[(4 + d * 3 + 1) * T + la];
        const R j2 = (DIM == 3) ? c * sA[(4 + d * 3 + 2) * T + la] : cst<R>(0.0f);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const R uv = sA[v * T + la];
          g[v * 3 + 0] = madd(g[v * 3 + 0], j0, uv);
          g[v * 3 + 1] = madd(g[v * 3 + 1], j1, uv);
          if (DIM == 3) g[v * 3 + 2] = madd(g[v * 3 + 2], j2, uv);
        }
      }
    }
  }
}

// Nodal contravariant fluxes Ftilde^d = Ja^d . (F^a - F^v / Re) of node i,
// written over its own sA slots (reads its own slots first).
template <typename R, int DIM>
DEV void nodal_fluxes(const R* sq, R* sA, const R* sG, int T, int i, const GasT<R>& G) {
  R qq[5], u[3], Ja[3 * DIM], gr[12];
#pragma unroll
  for (int v = 0; v < 5; ++v) qq[v] = sq[v * T + i];
  u[0] = sA[0 * T + i];
  u[1] = sA[1 * T + i];
  u[2] = sA[2 * T + i];
  const R Tt = sA[3 * T + i];
#pragma unroll
  for (int c = 0; c < 3 * DIM; ++c) Ja[c] = (DIM == 3 || c % 3 != 2) ? sA[(4 + c) * T + i] : cst<R>(0.0f);
#pragma unroll
  for (int k = 0; k < 12; ++k) gr[k] = sG[k * T + i];
  const R p = Tt * qq[0] * G.igM2;
  const R mu = mu_of_T(Tt, G);
  R F[5 * DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const R* nv = Ja + 3 * d;
    R fv[5];
    visc_flux<R, DIM>(u, mu, gr, nv, G, true, fv);
    if (DIM == 2) {  // nv[2] = 0
      const R un = u[0] * nv[0] + u[1] * nv[1];
      F[d * 5 + 0] = qq[0] * un;
      F[d * 5 + 1] = qq[1] * un + p * nv[0] - G.invRe * fv[1];
      F[d * 5 + 2] = qq[2] * un + p * nv[1] - G.invRe * fv[2];
      F[d * 5 + 3] = qq[3] * un - G.invRe * fv[3];
      F[d * 5 + 4] = (qq[4] + p) * un - G.invRe * fv[4];
    } else {
      const R un = u[0] * nv[0] + u[1] * nv[1] + u[2] * nv[2];
      F[d * 5 + 0] = qq[0] * un;
      F[d * 5 + 1] = qq[1] * un + p * nv[0] - G.invRe * fv[1];
      F[d * 5 + 2] = qq[2] * un + p * nv[1] - G.invRe * fv[2];
      F[d * 5 + 3] = qq[3] * un + p * nv[2] - G.invRe * fv[3];
      F[d * 5 + 4] = (qq[4] + p) * un - G.invRe * fv[4];
    }
  }
#pragma unroll
  for (int k = 0; k < 5 * DIM; ++k) sA[k * T + i] = F[k];
}

// sum_d D^d Ftilde^d at node i
template <typename R, int DIM>
DEV void divergence(const R* sD, const R* sA, int T, int nn, int i, int n0, int n1, int n2, R* acc) {
  const int le = i / nn, node = i - le * nn;
  const int idx0 = node % n0, idx1 = (node / n0) % n1, idx2 = node / (n0 * n1);
#pragma unroll
  for (int v = 0; v < 5; ++v) acc[v] = cst<R>(0.0f);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int id = pick(d, idx0, idx1, idx2), nd = pick(d, n0, n1, n2);
    const int sd = (d == 0) ? 1 : (d == 1 ? n0 : n0 * n1);
    const int base = le * nn + node - id * sd;
    const R* Drow = sD + d * kNP * kNP + id * kNP;
    for (int a = 0; a < nd; ++a) {
      const int la = base + a * sd;
      const R c = Drow[a];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = madd(acc[v], c, sA[(d * 5 + v) * T + la]);
    }
  }
}

// Register caps: 96 in 2D keeps five 128-thread CTAs per SM (a 100-register
// build rounds to 104 and fits only four); 104 in 3D, 128 for the isolated
// kernel in 3D (it spills at 104).
// volume stage of one element tile: BR1 gradient (volume part + lifting of
// U*), the gradient face traces, the nodal fluxes and the weak-form
// divergence (smem_raw: 3 kNP^2 + 32 x tile nodes of shared memory)
template <typename R, int DIM, bool AFFINE>
DEV void volume_tile(const LevelArgsT<R>& A, int tile, const GasT<R>* __restrict__ gas,
                     const double* __restrict__ q, const typename Store<R>::T* __restrict__ ust,
                     typename Store<R>::T* __restrict__ trg, typename Store<R>::T* __restrict__ vol,
                     double* smem_raw) {
  using SR = Store<R>;
  const ElemTile t = A.tiles[tile];
  const int n0 = t.n[0], n1 = t.n[1], n2 = t.n[2];
  const int nn = n0 * n1 * n2;
  const int T = t.count * nn;
  R* sD = reinterpret_cast<R*>(smem_raw);     // 3 * kNP * kNP
  R* sq = sD + 3 * kNP * kNP;                  // 5 * T
  R* sA = sq + 5 * T;                          // 15 * T: U(4) + Ja(9) | Ftilde(15)
  R* sG = sA + 15 * T;                         // 12 * T
  load_dtables<R>(sD, Tab<R>::Dhat(), n0, n1, n2, DIM);
  stage_tile<R, DIM>(A, t, nn, T, gas, q, sq, sA);
  __syncthreads();
  // ---- gradient: volume part + lifting of U*, times 1/J ----
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    R g[12];
    const int le = i / nn, node = i - le * nn;
    const int e = A.tile_elems[t.first + le];
    if (AFFINE) {
      gradient_volume<R, DIM, true, true>(sD, sA, T, nn, i, n0, n1, n2, g, ust, A.fo + e * 6, A.fn);
    } else {
      gradient_volume<R, DIM, false>(sD, sA, T, nn, i, n0, n1, n2, g);
      // lifting of U* n S from every face (curved metrics: per face node)
      const int idx0 = node % n0, idx1 = (node / n0) % n1, idx2 = node / (n0 * n1);
#pragma unroll
      for (int f = 0; f < 2 * DIM; ++f) {
        int d, ta, tb, side;
        face_dirs(f, d, ta, tb, side);
        const int nd = pick(d, n0, n1, n2), id = pick(d, idx0, idx1, idx2);
        const R lw = side ? Tab<R>::lpw(nd, id) : Tab<R>::lmw(nd, id);
        const int64_t p =
            A.fo[e * 6 + f] + pick(tb, idx0, idx1, idx2) * pick(ta, n0, n1, n2) + pick(ta, idx0, idx1, idx2);
        const R m0 = lw * SR::get(A.fnS, p), m1 = lw * SR::get(A.fnS, A.fn + p);
        const R m2 = (DIM == 3) ? lw * SR::get(A.fnS, 2 * A.fn + p) : cst<R>(0.0f);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const R us = SR::get(ust, v * A.fn + p);
          g[v * 3 + 0] = madd(g[v * 3 + 0], m0, us);
          g[v * 3 + 1] = madd(g[v * 3 + 1], m1, us);
          if (DIM == 3) g[v * 3 + 2] = madd(g[v * 3 + 2], m2, us);
        }
      }
    }
    const R iJ = SR::get(A.geo, 9 * A.nodes + A.off[e] + node);
#pragma unroll
    for (int k = 0; k < 12; ++k) sG[k * T + i] = (DIM == 2 && k % 3 == 2) ? cst<R>(0.0f) : g[k] * iJ;
  }
  __syncthreads();
  // ---- gradient face traces ----
  {
    int FE = 0;
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) FE += face_size(f, n0, n1, n2);
    for (int i = threadIdx.x; i < t.count * FE; i += blockDim.x) {
      int le = i / FE, r = i - le * FE;
      int f = 0;
      while (r >= face_size(f, n0, n1, n2)) {
        r -= face_size(f, n0, n1, n2);
        ++f;
      }
      int d, ta, tb, side;
      face_dirs(f, d, ta, tb, side);
      const int nta = pick(ta, n0, n1, n2), nd = pick(d, n0, n1, n2);
      int ia = r % nta, ib = r / nta;
      int i0 = (d == 0) ? 0 : ia;
      int i1 = (d == 1) ? 0 : (d == 0 ? ia : ib);
      int i2 = (d == 2) ? 0 : ib;
      int base = (i2 * n1 + i1) * n0 + i0;
      int sdd = (d == 0) ? 1 : (d == 1 ? n0 : n0 * n1);
      int e = A.tile_elems[t.first + le];
      int64_t p = A.fo[e * 6 + f] + r;
      const R* s0 = sG + le * nn + base;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        R acc = cst<R>(0.0f);
        if (DIM == 3 || k % 3 != 2)  // (2D: the z-derivatives are zero)
          for (int j = 0; j < nd; ++j) acc = madd(acc, (side ? Tab<R>::lp(nd, j) : Tab<R>::lm(nd, j)), s0[k * T + j * sdd]);
        SR::put(trg, k * A.fn + p, acc);
      }
    }
  }
  // ---- nodal contravariant fluxes (own node only: no cross-node hazard) ----
  for (int i = threadIdx.x; i < T; i += blockDim.x)
    nodal_fluxes<R, DIM>(sq, sA, sG, T, i, gas[A.slot[A.tile_elems[t.first + i / nn]]]);
  __syncthreads();
  // ---- weak-form divergence ----
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    R acc[5];
    divergence<R, DIM>(sD, sA, T, nn, i, n0, n1, n2, acc);
    const int le = i / nn, node = i - le * nn;
    const int e = A.tile_elems[t.first + le];
    const size_t ve = (size_t)5 * A.off[e] + node;
#pragma unroll
    for (int v = 0; v < 5; ++v) SR::put(vol, ve + v * nn, acc[v]);
  }
}

template <typename R, int DIM, bool AFFINE>
__global__ void __launch_bounds__(kVolThreads) __maxnreg__(DIM == 2 ? 96 : 104) k_volume(LevelArgsT<R> A, int tile0, const GasT<R>* __restrict__ gas,
                                                        const double* __restrict__ q,
                                                        const typename Store<R>::T* __restrict__ ust,
                                                        typename Store<R>::T* __restrict__ trg,
                                                        typename Store<R>::T* __restrict__ vol) {
  pdl_enter();
  extern __shared__ double smem_raw[];
  volume_tile<R, DIM, AFFINE>(A, tile0 + blockIdx.x, gas, q, ust, trg, vol, smem_raw);
}

// ---------------------------------------------------------------------------
// k_volume_split: the same volume stage for levels with few warps per SM
// ---------------------------------------------------------------------------
// On a coarse level a tile holds few nodes and the SMs hold about one warp
// each, so a launch lasts as long as one thread's serial FP64 instruction
// stream.  This variant gives each phase more independent work items -- one
// per (node, variable) in the gradient and the divergence, per (node,
// direction) in the nodal fluxes, per (face node, component) in the traces
// -- so that four to five times as many warps share the SM's FP64 pipe.
// Every output is computed by the same operations in the same order as in
// k_volume, so the results are the same bits.

// BR1 gradient of variable v of (u, v, w, T) at node i before the 1/J
// scaling: the work of gradient_volume (and, on curved elements, of the
// lifting of U*) for one variable.
template <typename R, int DIM, bool AFFINE>
DEV void gradient_var(const LevelArgsT<R>& A, const R* sD, const R* sA, int T, int nn, int i, int n0, int n1,
                      int n2, int v, int e, const typename Store<R>::T* __restrict__ ust, R* g) {
  using SR = Store<R>;
  const int le = i / nn, node = i - le * nn;
  const int idx0 = node % n0, idx1 = (node / n0) % n1, idx2 = node / (n0 * n1);
  g[0] = cst<R>(0.0f);
  g[1] = cst<R>(0.0f);
  g[2] = cst<R>(0.0f);
  const int32_t* fo_e = A.fo + e * 6;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int id = pick(d, idx0, idx1, idx2), nd = pick(d, n0, n1, n2);
    const int sd = (d == 0) ? 1 : (d == 1 ? n0 : n0 * n1);
    const int base = le * nn + node - id * sd;
    const R* Drow = sD + d * kNP * kNP + id * kNP;
    if (AFFINE) {
      R cu = cst<R>(0.0f);
      for (int a = 0; a < nd; ++a) cu = madd(cu, Drow[a], sA[v * T + base + a * sd]);
      const int ta = (d == 0) ? 1 : 0, tb = (d == 2) ? 1 : 2;
      const int fp = pick(tb, idx0, idx1, idx2) * pick(ta, n0, n1, n2) + pick(ta, idx0, idx1, idx2);
      const int64_t pm = fo_e[2 * d] + fp, pp = fo_e[2 * d + 1] + fp;
      const R wm = -Tab<R>::lmw(nd, id), wp = Tab<R>::lpw(nd, id);
      cu = madd(cu, wm, SR::get(ust, v * A.fn + pm));
      cu = madd(cu, wp, SR::get(ust, v * A.fn + pp));
      const R j0 = sA[(4 + d * 3 + 0) * T + i], j1 = sA[(4 + d * 3 + 1) * T + i];
      g[0] = madd(g[0], j0, cu);
      g[1] = madd(g[1], j1, cu);
      if (DIM == 3) g[2] = madd(g[2], sA[(4 + d * 3 + 2) * T + i], cu);
    } else {
      for (int a = 0; a < nd; ++a) {
        const int la = base + a * sd;
        const R c = Drow[a];
        const R j0 = c * sA[(4 + d * 3 + 0) * T + la];
        const R j1 = c * sA[(4 + d * 3 + 1) * T + la];
        const R j2 = (DIM == 3) ? c * sA[(4 + d * 3 + 2) * T + la] : cst<R>(0.0f);
        const R uv = sA[v * T + la];
        g[0] = madd(g[0], j0, uv);
        g[1] = madd(g[1], j1, uv);
        if (DIM == 3) g[2] = madd(g[2], j2, uv);
      }
    }
  }
  if (!AFFINE) {
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
      int d, ta, tb, side;
      face_dirs(f, d, ta, tb, side);
      const int nd = pick(d, n0, n1, n2), id = pick(d, idx0, idx1, idx2);
      const R lw = side ? Tab<R>::lpw(nd, id) : Tab<R>::lmw(nd, id);
      const int64_t p = fo_e[f] + pick(tb, idx0, idx1, idx2) * pick(ta, n0, n1, n2) + pick(ta, idx0, idx1, idx2);
      const R m0 = lw * SR::get(A.fnS, p), m1 = lw * SR::get(A.fnS, A.fn + p);
      const R us = SR::get(ust, v * A.fn + p);
      g[0] = madd(g[0], m0, us);
      g[1] = madd(g[1], m1, us);
      if (DIM == 3) g[2] = madd(g[2], lw * SR::get(A.fnS, 2 * A.fn + p), us);
    }
  }
}

// The blockDim must be at least DIM x (the tile's nodes): the nodal-flux
// phase reads every input of its item before a barrier and writes after it.
template <typename R, int DIM, bool AFFINE>
DEV void volume_split_tile(const LevelArgsT<R>& A, int tile, const GasT<R>* __restrict__ gas,
                           const double* __restrict__ q, const typename Store<R>::T* __restrict__ ust,
                           typename Store<R>::T* __restrict__ trg, typename Store<R>::T* __restrict__ vol,
                           double* smem_raw) {
  using SR = Store<R>;
  const ElemTile t = A.tiles[tile];
  const int n0 = t.n[0], n1 = t.n[1], n2 = t.n[2];
  const int nn = n0 * n1 * n2;
  const int T = t.count * nn;
  R* sD = reinterpret_cast<R*>(smem_raw);
  R* sq = sD + 3 * kNP * kNP;
  R* sA = sq + 5 * T;
  R* sG = sA + 15 * T;
  load_dtables<R>(sD, Tab<R>::Dhat(), n0, n1, n2, DIM);
  stage_tile<R, DIM>(A, t, nn, T, gas, q, sq, sA);
  __syncthreads();
  // ---- gradient: one (node, variable) per item ----
  for (int w = threadIdx.x; w < 4 * T; w += blockDim.x) {
    const int i = w % T, v = w / T;
    const int le = i / nn, node = i - le * nn;
    const int e = A.tile_elems[t.first + le];
    R g[3];
    gradient_var<R, DIM, AFFINE>(A, sD, sA, T, nn, i, n0, n1, n2, v, e, ust, g);
    const R iJ = SR::get(A.geo, 9 * A.nodes + A.off[e] + node);
#pragma unroll
    for (int c = 0; c < 3; ++c) sG[(v * 3 + c) * T + i] = (DIM == 2 && c == 2) ? cst<R>(0.0f) : g[c] * iJ;
  }
  __syncthreads();
  // ---- gradient face traces: one (face node, component) per item ----
  {
    int FE = 0;
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) FE += face_size(f, n0, n1, n2);
    const int nf = t.count * FE;
    for (int w = threadIdx.x; w < 12 * nf; w += blockDim.x) {
      const int fi = w % nf, k = w / nf;
      int le = fi / FE, r = fi - le * FE;
      int f = 0;
      while (r >= face_size(f, n0, n1, n2)) {
        r -= face_size(f, n0, n1, n2);
        ++f;
      }
      int d, ta, tb, side;
      face_dirs(f, d, ta, tb, side);
      const int nta = pick(ta, n0, n1, n2), nd = pick(d, n0, n1, n2);
      int ia = r % nta, ib = r / nta;
      int i0 = (d == 0) ? 0 : ia;
      int i1 = (d == 1) ? 0 : (d == 0 ? ia : ib);
      int i2 = (d == 2) ? 0 : ib;
      int base = (i2 * n1 + i1) * n0 + i0;
      int sdd = (d == 0) ? 1 : (d == 1 ? n0 : n0 * n1);
      int e = A.tile_elems[t.first + le];
      int64_t p = A.fo[e * 6 + f] + r;
      const R* s0 = sG + le * nn + base;
      R acc = cst<R>(0.0f);
      if (DIM == 3 || k % 3 != 2)  // (2D: the z-derivatives are zero)
        for (int j = 0; j < nd; ++j) acc = madd(acc, (side ? Tab<R>::lp(nd, j) : Tab<R>::lm(nd, j)), s0[k * T + j * sdd]);
      SR::put(trg, k * A.fn + p, acc);
    }
  }
  // ---- nodal contravariant fluxes: one (node, direction) per item ----
  {
    const int w = threadIdx.x;
    const bool act = w < DIM * T;
    const int i = act ? w % T : 0, d = act ? w / T : 0;
    R qq[5], u[3], Tt, nv[3], gr[12];
    if (act) {
#pragma unroll
      for (int v = 0; v < 5; ++v) qq[v] = sq[v * T + i];
      u[0] = sA[0 * T + i];
      u[1] = sA[1 * T + i];
      u[2] = sA[2 * T + i];
      Tt = sA[3 * T + i];
#pragma unroll
      for (int c = 0; c < 3; ++c) nv[c] = (DIM == 3 || c != 2) ? sA[(4 + 3 * d + c) * T + i] : cst<R>(0.0f);
#pragma unroll
      for (int k = 0; k < 12; ++k) gr[k] = sG[k * T + i];
    }
    __syncthreads();  // every item has read its inputs before any overwrites them
    if (act) {
      const GasT<R>& G = gas[A.slot[A.tile_elems[t.first + i / nn]]];
      const R p = Tt * qq[0] * G.igM2;
      const R mu = mu_of_T(Tt, G);
      R fv[5];
      visc_flux<R, DIM>(u, mu, gr, nv, G, true, fv);
      if (DIM == 2) {  // as nodal_fluxes: nv[2] = 0
        const R un = u[0] * nv[0] + u[1] * nv[1];
        sA[(d * 5 + 0) * T + i] = qq[0] * un;
        sA[(d * 5 + 1) * T + i] = qq[1] * un + p * nv[0] - G.invRe * fv[1];
        sA[(d * 5 + 2) * T + i] = qq[2] * un + p * nv[1] - G.invRe * fv[2];
        sA[(d * 5 + 3) * T + i] = qq[3] * un - G.invRe * fv[3];
        sA[(d * 5 + 4) * T + i] = (qq[4] + p) * un - G.invRe * fv[4];
      } else {
        const R un = u[0] * nv[0] + u[1] * nv[1] + u[2] * nv[2];
        sA[(d * 5 + 0) * T + i] = qq[0] * un;
        sA[(d * 5 + 1) * T + i] = qq[1] * un + p * nv[0] - G.invRe * fv[1];
        sA[(d * 5 + 2) * T + i] = qq[2] * un + p * nv[1] - G.invRe * fv[2];
        sA[(d * 5 + 3) * T + i] = qq[3] * un + p * nv[2] - G.invRe * fv[3];
        sA[(d * 5 + 4) * T + i] = (qq[4] + p) * un - G.invRe * fv[4];
      }
    }
  }
  __syncthreads();
  // ---- weak-form divergence: one (node, variable) per item ----
  for (int w = threadIdx.x; w < 5 * T; w += blockDim.x) {
    const int i = w % T, v = w / T;
    const int le = i / nn, node = i - le * nn;
    const int idx0 = node % n0, idx1 = (node / n0) % n1, idx2 = node / (n0 * n1);
    R acc = cst<R>(0.0f);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int id = pick(d, idx0, idx1, idx2), nd = pick(d, n0, n1, n2);
      const int sd = (d == 0) ? 1 : (d == 1 ? n0 : n0 * n1);
      const int base = le * nn + node - id * sd;
      const R* Drow = sD + d * kNP * kNP + id * kNP;
      for (int a = 0; a < nd; ++a) acc = madd(acc, Drow[a], sA[(d * 5 + v) * T + base + a * sd]);
    }
    const int e = A.tile_elems[t.first + le];
    SR::put(vol, (size_t)5 * A.off[e] + node + v * nn, acc);
  }
}
template <typename R, int DIM, bool AFFINE>
__global__ void __launch_bounds__(kVolThreads) __maxnreg__(DIM == 2 ? 96 : 104)
    k_volume_split(LevelArgsT<R> A, int tile0, const GasT<R>* __restrict__ gas, const double* __restrict__ q,
                   const typename Store<R>::T* __restrict__ ust, typename Store<R>::T* __restrict__ trg,
                   typename Store<R>::T* __restrict__ vol) {
  pdl_enter();
  extern __shared__ double smem_raw[];
  volume_split_tile<R, DIM, AFFINE>(A, tile0 + blockIdx.x, gas, q, ust, trg, vol, smem_raw);
}

// ---------------------------------------------------------------------------
// k_surface: surface terms, r = S - A; optional RK3 stage and max|r|
// ---------------------------------------------------------------------------
// CFL limit of Sec. 2 at one node: min over directions d with N_d > 0 of
// C_a h_d / ((|v| + c) N_d^2) and C_nu h_d^2 / (nu N_d^4), h_d = 2 / |a^d|,
// from the conserved state qq and the FP64 geometry (geo, SoA over nodes).
template <int DIM>
DEV double node_dt(const GasD& G, const double* qq, const double* __restrict__ geo, int64_t nodes, int64_t gn,
                   int n0, int n1, int n2) {
  double best = 1e300;
  const double ir = 1.0 / qq[0];
  const double u0 = qq[1] * ir, u1 = qq[2] * ir, u2 = qq[3] * ir;
  const double p = G.g1 * (qq[4] - 0.5 * (qq[1] * u0 + qq[2] * u1 + qq[3] * u2));
  const double Tt = G.gM2 * p * ir;
  const double c = sqrt(G.g * p * ir);
  const double vel = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
  const double nu = Tt * sqrt(Tt) * G.Su1 / (Tt + G.Su) * ir * G.invRe;
  const double iJ = geo[9 * nodes + gn];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int N = pick(d, n0, n1, n2) - 1;
    if (N <= 0) continue;
    double j0 = geo[(3 * d + 0) * nodes + gn], j1 = geo[(3 * d + 1) * nodes + gn],
           j2 = geo[(3 * d + 2) * nodes + gn];
    double h = 2.0 / (sqrt(j0 * j0 + j1 * j1 + j2 * j2) * iJ);
    double N2 = (double)N * (double)N;
    best = fmin(best, G.Ca * h / ((vel + c) * N2));
    best = fmin(best, G.Cnu * h * h / (nu * N2 * N2));
  }
  return best;
}

struct RKArgs {
  int stage;          // -1: plain residual, 0..2 RK3 stage
  double a, b;
  double* g;          // RK register
  const double* dt;   // device scalar
  double* qupd;       // state updated in place
  void* trq_next;     // if set: face traces of the updated state (the next stage's traces)
  // if set: the next sweep's time step per slot, reset in stage 1 and reduced
  // from the updated state in stage 2 (the work of k_cfl on that state)
  double* dt_next;
  const GasD* gasd;
  const double* geo64;  // FP64 geometry (the dt must not depend on the arithmetic mode)
  int nslots;
};

// surface stage of one element tile: the lifting of the face fluxes, 1/J,
// r = S - A (or the RK3 stage update), optionally the updated state's face
// traces and the next sweep's time step (smem_raw: 5 x tile nodes)
template <typename R, int DIM>
DEV void surface_tile(const LevelArgsT<R>& A, int tile, const typename Store<R>::T* __restrict__ vol,
                      const typename Store<R>::T* __restrict__ fst, const double* __restrict__ s,
                      double* __restrict__ r, double* norm, const RKArgs& rk, double* smem_raw) {
  using SR = Store<R>;
  R* sq = reinterpret_cast<R*>(smem_raw);  // updated state (5 x T) when rk.trq_next is set
  const bool traces = rk.stage >= 0 && rk.trq_next != nullptr;
  const ElemTile t = A.tiles[tile];
  if (rk.dt_next && rk.stage == 1 && tile == 0)
    for (int k = threadIdx.x; k < rk.nslots; k += blockDim.x) rk.dt_next[k] = 1e300;
  const bool cfl = rk.dt_next && rk.stage == 2;
  const int n0 = t.n[0], n1 = t.n[1], n2 = t.n[2];
  const int nn = n0 * n1 * n2;
  const int T = t.count * nn;
  for (int i0 = 0; i0 < T; i0 += blockDim.x) {  // all lanes iterate together (warp reductions)
    const int i = i0 + threadIdx.x;
    const bool active = i < T;
    double lmax = 0.0, best = 1e300;
    int slot = 0;
    if (active) {
      const int le = i / nn, node = i - le * nn;
      const int e = A.tile_elems[t.first + le];
      slot = A.slot[e];
      const int idx0 = node % n0, idx1 = (node / n0) % n1, idx2 = node / (n0 * n1);
      const size_t base = (size_t)5 * A.off[e] + node;
      R acc[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = SR::get(vol, base + v * nn);
#pragma unroll
      for (int f = 0; f < 2 * DIM; ++f) {
        int d, ta, tb, side;
        face_dirs(f, d, ta, tb, side);
        const int nd = pick(d, n0, n1, n2), id = pick(d, idx0, idx1, idx2);
        const R lw = side ? Tab<R>::lpw(nd, id) : Tab<R>::lmw(nd, id);
        const int64_t p = A.fo[e * 6 + f] + pick(tb, idx0, idx1, idx2) * pick(ta, n0, n1, n2) + pick(ta, idx0, idx1, idx2);
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] = madd(acc[v], lw, SR::get(fst, v * A.fn + p));
      }
      const R iJ = SR::get(A.geo, 9 * A.nodes + A.off[e] + node);
      const double dt = (rk.stage >= 0) ? rk.dt[slot] : 0.0;
      // every load of the node's source, state and RK register before any
      // store (the stores go through pointers the compiler cannot tell apart)
      double sv[5], qo[5], go[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) sv[v] = s ? s[base + v * nn] : 0.0;
      if (rk.stage >= 0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) qo[v] = rk.qupd[base + v * nn];
#pragma unroll
        for (int v = 0; v < 5; ++v) go[v] = (dt != 0.0 && rk.stage != 0) ? rk.g[base + v * nn] : 0.0;
      }
      double qnew[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double rv = sv[v] - to_double(acc[v] * iJ);
        lmax = (rv != rv) ? INFINITY : fmax(lmax, fabs(rv));  // a NaN residual reads as +inf
        if (rk.stage < 0) {
          r[base + v * nn] = rv;
        } else {
          double qn = qo[v];
          if (dt != 0.0) {  // dt = 0: the solve is held (smoothing control)
            double gv = (rk.stage == 0 ? 0.0 : rk.a * go[v]) + dt * rv;
            rk.g[base + v * nn] = gv;
            qn += rk.b * gv;
            rk.qupd[base + v * nn] = qn;
          }
          if (traces) sq[v * T + i] = state_of<R>(qn, A.base, base + v * nn);
          qnew[v] = qn;
        }
      }
      if (cfl) best = node_dt<DIM>(rk.gasd[slot], qnew, rk.geo64, A.nodes, A.off[e] + node, n0, n1, n2);
    }
    if (norm) warp_slot_reduce<true>(norm, slot, lmax, active);
    if (cfl) warp_slot_reduce<false>(rk.dt_next, slot, best, active);
  }
  if (traces) {
    __syncthreads();
    write_face_traces<R, DIM>(A, t, sq, T, static_cast<typename Store<R>::T*>(rk.trq_next));
  }
}

// (at least five CTAs per SM: a 720-tile level stays in one wave)
template <typename R, int DIM>
__global__ void __launch_bounds__(kTileNodes, 5) k_surface(LevelArgsT<R> A, const typename Store<R>::T* __restrict__ vol,
                                                        const typename Store<R>::T* __restrict__ fst,
                                                        const double* __restrict__ s, double* __restrict__ r,
                                                        double* norm, RKArgs rk) {
  pdl_enter();
  extern __shared__ double smem_raw[];
  surface_tile<R, DIM>(A, blockIdx.x, vol, fst, s, r, norm, rk, smem_raw);
}

// ---------------------------------------------------------------------------
// k_isolated: strong-form element-local operator; r = S - A, optional tau
// ---------------------------------------------------------------------------
struct TauArgs {
  const double* rho;     // chained restriction of the finest isolated residual (or null)
  double* table;         // K x 3 x 16
  const int32_t* fine_orders;  // K x 3
  int dir, slot;
};

template <typename R, int DIM, bool AFFINE>
__global__ void __launch_bounds__(kVolThreads) __maxnreg__(DIM == 2 ? 96 : 128) k_isolated(LevelArgsT<R> A, int tile0, const GasT<R>* __restrict__ gas,
                                                          const double* __restrict__ q,
                                                          const double* __restrict__ s, double* __restrict__ r,
                                                          TauArgs tau) {
  pdl_enter();
  using SR = Store<R>;
  extern __shared__ double smem_raw[];
  const ElemTile t = A.tiles[tile0 + blockIdx.x];
  const int n0 = t.n[0], n1 = t.n[1], n2 = t.n[2];
  const int nn = n0 * n1 * n2;
  const int T = t.count * nn;
  R* sD = reinterpret_cast<R*>(smem_raw);
  R* sq = sD + 3 * kNP * kNP;
  R* sA = sq + 5 * T;
  R* sG = sA + 15 * T;
  load_dtables<R>(sD, Tab<R>::Dcol(), n0, n1, n2, DIM);
  stage_tile<R, DIM>(A, t, nn, T, gas, q, sq, sA);
  __syncthreads();
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    R g[12];
    gradient_volume<R, DIM, AFFINE>(sD, sA, T, nn, i, n0, n1, n2, g);
    const int le = i / nn, node = i - le * nn;
    const int e = A.tile_elems[t.first + le];
    const R iJ = SR::get(A.geo, 9 * A.nodes + A.off[e] + node);
#pragma unroll
    for (int k = 0; k < 12; ++k) sG[k * T + i] = (DIM == 2 && k % 3 == 2) ? cst<R>(0.0f) : g[k] * iJ;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < T; i += blockDim.x)
    nodal_fluxes<R, DIM>(sq, sA, sG, T, i, gas[A.slot[A.tile_elems[t.first + i / nn]]]);
  __syncthreads();
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    R acc[5];
    divergence<R, DIM>(sD, sA, T, nn, i, n0, n1, n2, acc);
    const int le = i / nn, node = i - le * nn;
    const int e = A.tile_elems[t.first + le];
    const R iJ = SR::get(A.geo, 9 * A.nodes + A.off[e] + node);
    const size_t base = (size_t)5 * A.off[e] + node;
    double tmax = 0.0;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double rv = (s ? s[base + v * nn] : 0.0) - to_double(acc[v] * iJ);
      if (tau.table) {
        double tv = tau.rho ? rv - tau.rho[base + v * nn] : rv;
        tmax = fmax(tmax, fabs(tv));
      } else {
        r[base + v * nn] = rv;
      }
    }
    if (tau.table && tau.fine_orders[e * 3 + tau.dir] > tau.slot)
      atomic_max_nonneg(tau.table + ((size_t)e * 3 + tau.dir) * kTauSlots + tau.slot, tmax);
  }
}

// ---------------------------------------------------------------------------
// k_cfl: global minimum of the explicit step (FP64)
// ---------------------------------------------------------------------------
// per-slot minimum of the explicit step over the nodes of one element tile
template <int DIM>
DEV void cfl_tile(const LevelArgsT<double>& A, int tile, const GasD* __restrict__ gasd, const double* __restrict__ q,
                  double* dtmin) {
  const ElemTile t = A.tiles[tile];
  const int n0 = t.n[0], n1 = t.n[1], n2 = t.n[2];
  const int nn = n0 * n1 * n2;
  const int T = t.count * nn;
  for (int i0 = 0; i0 < T; i0 += blockDim.x) {  // all lanes iterate together (warp reductions)
    const int i = i0 + threadIdx.x;
    const bool active = i < T;
    double best = 1e300;
    int slot = 0;
    if (active) {
      int le = i / nn, node = i - le * nn;
      int e = A.tile_elems[t.first + le];
      slot = A.slot[e];
      const double* qe = q + (size_t)5 * A.off[e];
      double qq[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qq[v] = qe[v * nn + node];
      best = node_dt<DIM>(gasd[slot], qq, A.geo, A.nodes, A.off[e] + node, n0, n1, n2);
    }
    warp_slot_reduce<false>(dtmin, slot, best, active);
  }
}

template <int DIM>
__global__ void __launch_bounds__(kTileNodes) k_cfl(LevelArgsT<double> A, const GasD* __restrict__ gasd,
                                                    const double* __restrict__ q, double* dtmin) {
  pdl_enter();
  cfl_tile<DIM>(A, blockIdx.x, gasd, q, dtmin);
}

// ---------------------------------------------------------------------------
// transfers between order maps: out_e = (T2 x T1 x T0) (in_e - sub_e),
// sum-factorised through shared memory, one direction per pass.  A pass
// covers `vgroup` variables at once (all five unless an element's slab is
// too large for that), and a flat direction (one node on both sides, the z
// direction of a 2D mesh) is skipped: its factor is the 1 x 1 identity.
// ---------------------------------------------------------------------------
constexpr int kTransferThreads = 128;
// largest per-variable slab: 3D elements have <= 729 nodes and n <= 13 per
// direction, so f1*f2 <= 364 and t0 <= 13 bound the x-pass intermediate;
// the shared memory holds two slabs of that size (or more smaller ones)
constexpr int kTransferMaxSlab = 4800;

DEV int transfer_slab(int f0, int f1, int f2, int t0, int t1, int t2) {
  return max(max(f0 * f1 * f2, t0 * t1 * t2), max(f2 * f1 * t0, f2 * t1 * t0));
}

__global__ void __launch_bounds__(kTransferThreads) k_transfer(const int32_t* __restrict__ nf,
                                                               const int32_t* __restrict__ offf,
                                                               const int32_t* __restrict__ nt,
                                                               const int32_t* __restrict__ offt, int nvar,
                                                               int vgroup, const double* __restrict__ in,
                                                               const double* __restrict__ sub,
                                                               double* __restrict__ out, int accumulate) {
  pdl_enter();
  extern __shared__ double sbuf[];
  const int e = blockIdx.x;
  const int f0 = nf[e * 3], f1 = nf[e * 3 + 1], f2 = nf[e * 3 + 2];
  const int t0 = nt[e * 3], t1 = nt[e * 3 + 1], t2 = nt[e * 3 + 2];
  const int nnf = f0 * f1 * f2, nnt = t0 * t1 * t2;
  const double* T0 = c_T + ((size_t)f0 * kNP + t0) * kNP * kNP;
  const double* T1 = c_T + ((size_t)f1 * kNP + t1) * kNP * kNP;
  const double* T2 = c_T + ((size_t)f2 * kNP + t2) * kNP * kNP;
  const int slab = transfer_slab(f0, f1, f2, t0, t1, t2);
  double* bA = sbuf;
  double* bB = sbuf + (size_t)vgroup * slab;
  const int n1x = f2 * f1 * t0, n2y = f2 * t1 * t0;
  const bool flat = (f2 == 1 && t2 == 1);
  for (int v0 = 0; v0 < nvar; v0 += vgroup) {
    const int nv = min(vgroup, nvar - v0);
    const size_t ib = (size_t)nvar * offf[e] + (size_t)v0 * nnf;
    double* oe = out + (size_t)nvar * offt[e] + (size_t)v0 * nnt;
    for (int i = threadIdx.x; i < nv * nnf; i += blockDim.x) {
      const int v = i / nnf, k = i - v * nnf;
      bA[v * slab + k] = sub ? in[ib + i] - sub[ib + i] : in[ib + i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv * n1x; i += blockDim.x) {  // x pass: [k2][k1][j0]
      const int v = i / n1x, r = i - v * n1x;
      const int j0 = r % t0, k12 = r / t0;
      const double* src = bA + v * slab + k12 * f0;
      double acc = 0.0;
      for (int k0 = 0; k0 < f0; ++k0) acc += T0[j0 * f0 + k0] * src[k0];
      bB[v * slab + r] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv * n2y; i += blockDim.x) {  // y pass: [k2][j1][j0]
      const int v = i / n2y, r = i - v * n2y;
      const int j0 = r % t0, j1 = (r / t0) % t1, k2 = r / (t0 * t1);
      const double* src = bB + v * slab + k2 * f1 * t0 + j0;
      double acc = 0.0;
      for (int k1 = 0; k1 < f1; ++k1) acc += T1[j1 * f1 + k1] * src[k1 * t0];
      if (!flat) {
        bA[v * slab + r] = acc;
      } else if (accumulate) {  // flat: [j1][j0] is the output layout
        oe[v * nnt + r] += acc;
      } else {
        oe[v * nnt + r] = acc;
      }
    }
    __syncthreads();
    if (flat) continue;
    for (int i = threadIdx.x; i < nv * nnt; i += blockDim.x) {  // z pass: [j2][j1][j0]
      const int v = i / nnt, r = i - v * nnt;
      const int j01 = r % (t0 * t1), j2 = r / (t0 * t1);
      const double* src = bA + v * slab + j01;
      double acc = 0.0;
      for (int k2 = 0; k2 < f2; ++k2) acc += T2[j2 * f2 + k2] * src[k2 * t1 * t0];
      if (accumulate)
        oe[v * nnt + r] += acc;
      else
        oe[v * nnt + r] = acc;
    }
    __syncthreads();
  }
}

__global__ void k_fill(double* p, double v, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_axpby(double* y, double a, const double* x, double b, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
__global__ void k_sub3(double* o, const double* a, const double* b, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = a[i] - b[i];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename R, int DIM, bool AFF>
static int set_attrs() {
  const int big = (int)((3 * kNP * kNP + 32 * kMaxElemNodes) * sizeof(double));
  DG_CUDA_TRY(cudaFuncSetAttribute(k_volume<R, DIM, AFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DG_CUDA_TRY(cudaFuncSetAttribute(k_volume_split<R, DIM, AFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DG_CUDA_TRY(cudaFuncSetAttribute(k_isolated<R, DIM, AFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return DG_OK;
}

static int configure_smem() {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  int dev = 0;
  DG_CUDA_TRY(cudaGetDevice(&dev));
  DeviceTables* dt = g_dev_tables.get(dev);
  if (!dt) {
    set_error("device index " + std::to_string(dev) + " beyond the library's device limit");
    return DG_EINVAL;
  }
  if (dt->smem_ready) return DG_OK;
  int rc;
  if ((rc = set_attrs<double, 2, false>()) != DG_OK) return rc;
  if ((rc = set_attrs<double, 2, true>()) != DG_OK) return rc;
  if ((rc = set_attrs<double, 3, false>()) != DG_OK) return rc;
  if ((rc = set_attrs<double, 3, true>()) != DG_OK) return rc;
  if ((rc = set_attrs<dd, 2, false>()) != DG_OK) return rc;
  if ((rc = set_attrs<dd, 2, true>()) != DG_OK) return rc;
  if ((rc = set_attrs<dd, 3, false>()) != DG_OK) return rc;
  if ((rc = set_attrs<dd, 3, true>()) != DG_OK) return rc;
  {
    const int big = (int)((3 * kNP * kNP + 32 * kMaxElemNodes) * sizeof(double));
    DG_CUDA_TRY(cudaFuncSetAttribute(k_volume<tf, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    DG_CUDA_TRY(cudaFuncSetAttribute(k_volume<tf, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    DG_CUDA_TRY(cudaFuncSetAttribute(k_volume<tf, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    DG_CUDA_TRY(cudaFuncSetAttribute(k_volume<tf, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    DG_CUDA_TRY(cudaFuncSetAttribute(k_volume_split<tf, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    DG_CUDA_TRY(cudaFuncSetAttribute(k_volume_split<tf, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    DG_CUDA_TRY(cudaFuncSetAttribute(k_volume_split<tf, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    DG_CUDA_TRY(cudaFuncSetAttribute(k_volume_split<tf, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  }
  DG_CUDA_TRY(cudaFuncSetAttribute(k_transfer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(2 * kTransferMaxSlab * sizeof(double))));
  dt->smem_ready = true;
  return DG_OK;
}

int prepare_capture() { return configure_smem(); }

// max |x| over the nodes and 5 variables of every solve slot (x in the
// level's layout) into out[slot]; out must be zeroed first
__global__ void __launch_bounds__(kTileNodes) k_slot_maxabs(LevelArgsT<double> A, const double* __restrict__ x,
                                                            double* out) {
  pdl_enter();
  const ElemTile t = A.tiles[blockIdx.x];
  const int nn = t.n[0] * t.n[1] * t.n[2];
  const int T = t.count * nn;
  for (int i0 = 0; i0 < T; i0 += blockDim.x) {  // all lanes iterate together (warp reductions)
    const int i = i0 + threadIdx.x;
    const bool active = i < T;
    double m = 0.0;
    int slot = 0;
    if (active) {
      const int le = i / nn, node = i - le * nn;
      const int e = A.tile_elems[t.first + le];
      slot = A.slot[e];
      const size_t base = (size_t)5 * A.off[e] + node;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double a = x[base + v * nn];
        m = (a != a) ? INFINITY : fmax(m, fabs(a));
      }
    }
    warp_slot_reduce<true>(out, slot, m, active);
  }
}

// dt[k] = 0 for every slot k whose mask is 0 (k_surface then leaves it unchanged)
__global__ void k_mask_dt(double* dt, const double* mask, int n) {
  pdl_enter();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n && mask[k] == 0.0) dt[k] = 0.0;
}

static int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)std::max<int64_t>(1, b);
}

int slot_maxabs(const dg_mesh* m, const Level* L, const double* x, double* out, cudaStream_t st) {
  const int rc = fill(out, 0.0, m->nslots, st);
  if (rc != DG_OK) return rc;
  count_launch();
  launch_k(k_slot_maxabs, L->n_tiles, kTileNodes, 0, st, largs<double>(L), x, out);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int mask_dt(const dg_mesh* m, double* dt, const double* mask, cudaStream_t st) {
  count_launch();
  launch_k(k_mask_dt, (m->nslots + 127) / 128, 128, 0, st, dt, mask, m->nslots);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int fill(double* p, double v, int64_t n, cudaStream_t st) {
  count_launch();
  launch_k(k_fill, grid_for(n), 256, 0, st, p, v, n);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}
int axpby(double* y, double a, const double* x, double b, int64_t n, cudaStream_t st) {
  count_launch();
  launch_k(k_axpby, grid_for(n), 256, 0, st, y, a, x, b, n);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}
int sub3(double* o, const double* a, const double* b, int64_t n, cudaStream_t st) {
  count_launch();
  launch_k(k_sub3, grid_for(n), 256, 0, st, o, a, b, n);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}
int reset_max(double* d, cudaStream_t st) { return fill(d, 0.0, 1, st); }
int reset_min(double* d, cudaStream_t st) { return fill(d, 1e300, 1, st); }
int read_scalar(const double* d, double* h, cudaStream_t st) {
  DG_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, st));
  DG_CUDA_TRY(cudaStreamSynchronize(st));
  return DG_OK;
}

// float-pair copies of a level's geometry (double-float kernels), made once
__global__ void k_split(const double* __restrict__ x, float2* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = (float)v;
    y[i] = make_float2(h, (float)(v - (double)h));
  }
}
static int split_array(const double* x, double** y, int64_t n, cudaStream_t st) {
  DG_CUDA_TRY(cudaMalloc((void**)y, std::max<int64_t>(1, n) * sizeof(float2)));
  count_launch();
  k_split<<<grid_for(n), 256, 0, st>>>(x, reinterpret_cast<float2*>(*y), n);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}
static int ensure_dd(Level* L, cudaStream_t st) {
  if (L->d_geo2) return DG_OK;
  int rc;
  if ((rc = split_array(L->d_geo, &L->d_geo2, 10 * L->nodes, st)) != DG_OK) return rc;
  if ((rc = split_array(L->d_fnS, &L->d_fnS2, 3 * L->face_nodes, st)) != DG_OK) return rc;
  if ((rc = split_array(L->d_mnS, &L->d_mnS2, 3 * L->mortar_nodes, st)) != DG_OK) return rc;
  L->bytes += (int64_t)sizeof(float2) * (10 * L->nodes + 3 * L->face_nodes + 3 * L->mortar_nodes);
  return DG_OK;
}

// value-only pairs (derivative 0) of a level's geometry for the tangent
// kernels, made once
__global__ void k_split_value(const double* __restrict__ x, float2* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = make_float2((float)x[i], 0.0f);
}
static int value_array(const double* x, double** y, int64_t n, cudaStream_t st) {
  DG_CUDA_TRY(cudaMalloc((void**)y, std::max<int64_t>(1, n) * sizeof(float2)));
  count_launch();
  k_split_value<<<grid_for(n), 256, 0, st>>>(x, reinterpret_cast<float2*>(*y), n);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}
static int ensure_tf(Level* L, cudaStream_t st) {
  if (L->d_geoT) return DG_OK;
  int rc;
  if ((rc = value_array(L->d_geo, &L->d_geoT, 10 * L->nodes, st)) != DG_OK) return rc;
  if ((rc = value_array(L->d_fnS, &L->d_fnST, 3 * L->face_nodes, st)) != DG_OK) return rc;
  if ((rc = value_array(L->d_mnS, &L->d_mnST, 3 * L->mortar_nodes, st)) != DG_OK) return rc;
  L->bytes += (int64_t)sizeof(float2) * (10 * L->nodes + 3 * L->face_nodes + 3 * L->mortar_nodes);
  return DG_OK;
}

template <typename R>
static const GasT<R>* gas_table(const dg_mesh* m);
template <>
const GasT<double>* gas_table<double>(const dg_mesh* m) {
  return reinterpret_cast<const GasT<double>*>(m->d_gas64);
}
template <>
const GasT<dd>* gas_table<dd>(const dg_mesh* m) {
  return reinterpret_cast<const GasT<dd>*>(m->d_gas32x2);
}
template <>
const GasT<tf>* gas_table<tf>(const dg_mesh* m) {
  return reinterpret_cast<const GasT<tf>*>(m->d_gastf);
}

// per-slot gas constants on the device (FP64, float pairs, CFL)
int upload_gas(dg_mesh* m) {
  const int S = m->nslots;
  std::vector<GasT<double>> g64(S);
  std::vector<GasT<dd>> g2(S);
  std::vector<GasD> gd(S);
  std::vector<GasT<tf>> gt(S);
  for (int k = 0; k < S; ++k) {
    g64[k] = make_gas<double>(m->slot_prm[k]);
    g2[k] = make_gas<dd>(m->slot_prm[k]);
    gd[k] = make_gas_d(m->slot_prm[k]);
    gt[k] = make_gas<tf>(m->slot_prm[k]);
  }
  DG_CUDA_TRY(cudaMalloc(&m->d_gas64, S * sizeof(GasT<double>)));
  DG_CUDA_TRY(cudaMalloc(&m->d_gas32x2, S * sizeof(GasT<dd>)));
  DG_CUDA_TRY(cudaMalloc((void**)&m->d_gasd, S * sizeof(GasD)));
  DG_CUDA_TRY(cudaMemcpy(m->d_gas64, g64.data(), S * sizeof(GasT<double>), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpy(m->d_gas32x2, g2.data(), S * sizeof(GasT<dd>), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpy(m->d_gasd, gd.data(), S * sizeof(GasD), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMalloc(&m->d_gastf, S * sizeof(GasT<tf>)));
  DG_CUDA_TRY(cudaMemcpy(m->d_gastf, gt.data(), S * sizeof(GasT<tf>), cudaMemcpyHostToDevice));
  return DG_OK;
}

int prepare_arith(const dg_mesh* m, Level* L, cudaStream_t st) {
  if (m->arith == DG_ARITH_DF32) return ensure_dd(L, st);
  if (m->arith == DG_ARITH_MIXED) return ensure_tf(L, st);
  return DG_OK;
}

// ---- per-kernel launch helpers (arithmetic / dimension / affine dispatch) ----
template <typename R>
using ST = typename Store<R>::T;

template <typename R>
static ST<R>* buf(double* p) {
  return reinterpret_cast<ST<R>*>(p);
}

template <typename R>
static void launch_trace(const Level* L, const double* q, cudaStream_t st, const double* base = nullptr) {
  count_launch();
  const size_t sm = 5 * L->tile_smem_nodes * sizeof(double);
  LevelArgsT<R> A = largs<R>(L);
  A.base = base;
  if (L->dim == 2)
    launch_k(k_trace_q<R, 2>, L->n_tiles, kTileNodes, sm, st, A, q, buf<R>(L->d_trq));
  else
    launch_k(k_trace_q<R, 3>, L->n_tiles, kTileNodes, sm, st, A, q, buf<R>(L->d_trq));
}
// The staged element kernels run once per tile class: tiles of <= 128 nodes
// with 128 threads, <= 256 with 256, larger (one element of up to 729 nodes)
// with 512, each class with the shared memory of its own largest tile.
template <typename F>
static void for_tile_classes(const Level* L, F launch, int only = -1, int threads_override = 0) {
  int begin = 0;
  for (int c = 0; c < kTileClasses; ++c) {
    const int end = L->tile_class_end[c];
    if (end > begin && (only < 0 || only == c)) {
      count_launch();
      const int th = threads_override > 0 ? threads_override : L->class_threads[c];
      launch(begin, end - begin, th, (size_t)(3 * kNP * kNP + 32 * L->tile_class_nodes[c]) * sizeof(double));
    }
    begin = end;
  }
}

// Whether a level's small-element tiles (class 0) take k_volume_split:
// DG_VOLUME_SPLIT=0 never, 2 always, 1 (default) for FP64 tiles of at most
// 32 nodes that give the plain kernel fewer than 8 warps per SM.  Measured
// on the flat plate (FP64 volume stage per level, plain / split): N = 1
// 14.8 / 12.4 us, N = 2 15.9 / 16.2, N = 3 23.2 / 32.7, N = 7 62.7 / 90.9;
// the tangent arithmetic was never faster split.  Larger tiles make
// 5 x 128-thread CTAs, one per SM, in two waves.  The results are the same
// bits either way; the knob selects the kernel only.
static int volume_split_mode() {
  static const int mode = [] {
    const char* e = std::getenv("DG_VOLUME_SPLIT");
    return e ? std::atoi(e) : 1;
  }();
  return mode;
}
// DG_MORTAR_FLUX_SPLIT=0 runs the flux pass of conforming levels in
// k_mortar_conf<2> (one warp per 32 nodes), 2 always in k_mortar_conf_flux
// (two), 1 (default) in k_mortar_conf_flux for the FP32-pipe arithmetics
// and, in FP64, on levels with fewer than 3 warps of mortar nodes per SM.
// Measured on the flat plate (FP64 flux pass, one / two warps): N = 1 14.4 /
// 10.4 us, N = 3 14.4 / 13.5, N = 4 14.6 / 15.9, N = 7 18.2 / 20.4 (above
// ~3 warps per SM the duplicated trace and primitive work outweighs the
// latency it hides); the tangent form gains on every level (N = 7: 5.4 /
// 5.2 us).  Same bits; the knob selects the kernel only.
static int mortar_flux_split_mode() {
  static const int mode = [] {
    const char* e = std::getenv("DG_MORTAR_FLUX_SPLIT");
    return e ? std::atoi(e) : 1;
  }();
  return mode;
}
static int sm_count_cached();
static bool mortar_flux_split(const Level* L, bool fp64) {
  const int mode = mortar_flux_split_mode();
  if (mode == 0) return false;
  if (mode == 2 || !fp64) return true;
  return (L->mortar_nodes + 31) / 32 < 3 * (int64_t)sm_count_cached();
}
static int sm_count_cached() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 152;
    return v > 0 ? v : 152;
  }();
  return n;
}
static bool volume_split(const Level* L, bool fp64) {
  const int mode = volume_split_mode();
  if (mode == 0 || L->tile_class_end[0] == 0) return false;
  if (mode == 2) return true;
  if (!fp64 || L->tile_class_nodes[0] > 32) return false;
  const int64_t warps = (int64_t)L->tile_class_end[0] * ((L->tile_class_nodes[0] + 31) / 32);
  return warps < 8 * (int64_t)sm_count_cached();
}

template <typename R>
static void launch_volume(const Level* L, const GasT<R>* G, const double* q, cudaStream_t st, int only = -1,
                          int threads_override = 0, const double* base = nullptr) {
  LevelArgsT<R> A = largs<R>(L);
  A.base = base;
  const ST<R>* ust = buf<R>(L->d_ust);
  ST<R>* trg = buf<R>(L->d_trg);
  ST<R>* vol = buf<R>(L->d_vol);
  const bool split =
      threads_override == 0 && (only < 0 || only == 0) && volume_split(L, std::is_same<R, double>::value);
  if (split) {  // class 0 in the split kernel; the other classes below
    const int T0 = L->tile_class_nodes[0];
    const int th = std::min(kVolThreads, std::max(((5 * T0 + 31) / 32) * 32, 32));
    const size_t sm = (size_t)(3 * kNP * kNP + 32 * T0) * sizeof(double);
    const int nt = L->tile_class_end[0];
    if (only == 0) count_launch();  // (otherwise for_tile_classes counts class 0 below)
    if (L->dim == 2) {
      if (L->affine)
        launch_k(k_volume_split<R, 2, true>, nt, th, sm, st, A, 0, G, q, ust, trg, vol);
      else
        launch_k(k_volume_split<R, 2, false>, nt, th, sm, st, A, 0, G, q, ust, trg, vol);
    } else {
      if (L->affine)
        launch_k(k_volume_split<R, 3, true>, nt, th, sm, st, A, 0, G, q, ust, trg, vol);
      else
        launch_k(k_volume_split<R, 3, false>, nt, th, sm, st, A, 0, G, q, ust, trg, vol);
    }
    if (only == 0) return;
  }
  for_tile_classes(L, [&](int t0, int nt, int th, size_t sm) {
    if (split && t0 == 0) return;  // class 0 ran in the split kernel
    if (L->dim == 2) {
      if (L->affine)
        launch_k(k_volume<R, 2, true>, nt, th, sm, st, A, t0, G, q, ust, trg, vol);
      else
        launch_k(k_volume<R, 2, false>, nt, th, sm, st, A, t0, G, q, ust, trg, vol);
    } else {
      if (L->affine)
        launch_k(k_volume<R, 3, true>, nt, th, sm, st, A, t0, G, q, ust, trg, vol);
      else
        launch_k(k_volume<R, 3, false>, nt, th, sm, st, A, t0, G, q, ust, trg, vol);
    }
  }, only, threads_override);
}
template <typename R>
static void launch_isolated(const Level* L, const GasT<R>* G, const double* q, const double* s, double* r,
                            const TauArgs& ta, cudaStream_t st) {
  LevelArgsT<R> A = largs<R>(L);
  for_tile_classes(L, [&](int t0, int nt, int th, size_t sm) {
    if (L->dim == 2) {
      if (L->affine)
        launch_k(k_isolated<R, 2, true>, nt, th, sm, st, A, t0, G, q, s, r, ta);
      else
        launch_k(k_isolated<R, 2, false>, nt, th, sm, st, A, t0, G, q, s, r, ta);
    } else {
      if (L->affine)
        launch_k(k_isolated<R, 3, true>, nt, th, sm, st, A, t0, G, q, s, r, ta);
      else
        launch_k(k_isolated<R, 3, false>, nt, th, sm, st, A, t0, G, q, s, r, ta);
    }
  });
}
template <typename R>
static void launch_surface(const Level* L, const double* s, double* r, double* norm, const RKArgs& rk,
                           cudaStream_t st, const double* base = nullptr) {
  count_launch();
  LevelArgsT<R> A = largs<R>(L);
  A.base = base;
  const size_t sm = rk.trq_next ? 5 * L->tile_smem_nodes * sizeof(double) : 0;
  if (L->dim == 2)
    launch_k(k_surface<R, 2>, L->n_tiles, kTileNodes, sm, st, A, buf<R>(L->d_vol), buf<R>(L->d_fst), s, r, norm, rk);
  else
    launch_k(k_surface<R, 3>, L->n_tiles, kTileNodes, sm, st, A, buf<R>(L->d_vol), buf<R>(L->d_fst), s, r, norm, rk);
}
template <typename R>
static void launch_mortar(int pass, const Level* L, const GasT<R>* G, cudaStream_t st) {
  count_launch();
  LevelArgsT<R> A = largs<R>(L);
  MortarArgsT<R> MA = margs<R>(L);
  if (L->mortars_conforming) {
    const int grid = (int)std::max<int64_t>(1, (L->mortar_nodes + kMortarConfThreads - 1) / kMortarConfThreads);
    if (pass == 1)
      launch_k(k_mortar_conf<R, 1>, grid, kMortarConfThreads, 0, st, A, MA, G, buf<R>(L->d_trq), nullptr,
                                                               buf<R>(L->d_ust));
    else if (mortar_flux_split(L, std::is_same<R, double>::value))  // two warps per 32 nodes (same bits)
      launch_k(k_mortar_conf_flux<R>, grid, 64, 0, st, A, MA, G, buf<R>(L->d_trq), buf<R>(L->d_trg),
               buf<R>(L->d_fst));
    else
      launch_k(k_mortar_conf<R, 2>, grid, kMortarConfThreads, 0, st, A, MA, G, buf<R>(L->d_trq), buf<R>(L->d_trg),
                                                               buf<R>(L->d_fst));
    return;
  }
  if (pass == 1)
    launch_k(k_mortar<R, 1>, L->n_mtiles, kMortarTile, 0, st, A, MA, G, buf<R>(L->d_trq), nullptr, buf<R>(L->d_ust));
  else
    launch_k(k_mortar<R, 2>, L->n_mtiles, kMortarTile, 0, st, A, MA, G, buf<R>(L->d_trq), buf<R>(L->d_trg),
                                                        buf<R>(L->d_fst));
}

static RKArgs rk_args(int rk_stage, double* rk_g, const double* d_dt, const double* q) {
  RKArgs rk;
  rk.stage = rk_stage;
  rk.a = (rk_stage == 1) ? -5.0 / 9.0 : (rk_stage == 2 ? -153.0 / 128.0 : 0.0);
  rk.b = (rk_stage == 0) ? 1.0 / 3.0 : (rk_stage == 1 ? 15.0 / 16.0 : 8.0 / 15.0);
  rk.g = rk_g;
  rk.dt = d_dt;
  rk.qupd = const_cast<double*>(q);
  rk.trq_next = nullptr;
  rk.dt_next = nullptr;
  rk.gasd = nullptr;
  rk.geo64 = nullptr;
  rk.nslots = 0;
  return rk;
}

template <typename R>
static int residual_t(const dg_mesh* m, Level* L, const double* q, const double* s, double* r, bool isolated,
                      cudaStream_t st, double* d_norm, int rk_stage, double* rk_g, const double* d_dt,
                      int trace_flags, double* dt_next, const double* base = nullptr) {
  const GasT<R>* G = gas_table<R>(m);
  if (isolated) {
    TauArgs ta{nullptr, nullptr, nullptr, 0, 0};
    launch_isolated<R>(L, G, q, s, r, ta, st);
    DG_CUDA_TRY(cudaGetLastError());
    return DG_OK;
  }
  if (!(trace_flags & kTracesCurrent)) launch_trace<R>(L, q, st, base);
  launch_mortar<R>(1, L, G, st);
  launch_volume<R>(L, G, q, st, -1, 0, base);
  launch_mortar<R>(2, L, G, st);
  RKArgs rk = rk_args(rk_stage, rk_g, d_dt, q);
  if (rk_stage >= 0 && (trace_flags & kTracesNext)) rk.trq_next = buf<R>(L->d_trq);
  if (rk_stage >= 0 && dt_next) {
    rk.dt_next = dt_next;
    rk.gasd = m->d_gasd;
    rk.geo64 = L->d_geo;
    rk.nslots = m->nslots;
  }
  launch_surface<R>(L, s, r, d_norm, rk, st, base);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int residual_tangent(const dg_mesh* m, Level* L, const double* base, const double* dq, const double* b, double* r,
                     cudaStream_t st, double* d_norm, int rk_stage, double* rk_g, const double* d_dt,
                     int trace_flags) {
  int rc = configure_smem();
  if (rc != DG_OK) return rc;
  if ((rc = ensure_tf(L, st)) != DG_OK) return rc;
  return residual_t<tf>(m, L, dq, b, r, false, st, d_norm, rk_stage, rk_g, d_dt, trace_flags, nullptr, base);
}

int residual(const dg_mesh* m, Level* L, const double* q, const double* s, double* r, bool isolated,
             cudaStream_t st, double* d_norm, int rk_stage, double* rk_g, const double* d_dt, int trace_flags,
             double* dt_next) {
  int rc = configure_smem();
  if (rc != DG_OK) return rc;
  if (m->arith == DG_ARITH_DF32) {
    if ((rc = ensure_dd(L, st)) != DG_OK) return rc;
    return residual_t<dd>(m, L, q, s, r, isolated, st, d_norm, rk_stage, rk_g, d_dt, trace_flags, dt_next);
  }
  return residual_t<double>(m, L, q, s, r, isolated, st, d_norm, rk_stage, rk_g, d_dt, trace_flags, dt_next);
}

// ---------------------------------------------------------------------------
// k_smooth_block: one smoothing block (the CFL step, then `sweeps` RK3 sweeps
// of trace / U* / volume / flux / surface stages) of a small conforming level
// in one cooperative launch.  On such a level every kernel of the chain runs
// a few CTAs whose time is one CTA's latency chain, and the launch gaps
// between the ~13 launches of a sweep cost as much as the work.  Here the
// stages are phases of one persistent kernel: each phase loops over its work
// items (element tiles or 128 mortar nodes) with the per-item code of the
// separate kernels, and phases are separated by a grid barrier.  Each output
// is computed by the same operations in the same order as in the separate
// kernels, so the results are the same bits.
// ---------------------------------------------------------------------------
// Grid barrier state (16 bytes of device memory per mesh, zeroed at
// creation).  A cooperative launch makes every block resident, so a barrier
// always completes; the wait is still bounded: a block that polls
// kGridSyncSpins times records `failed` and the kernel returns, and later
// launches return at entry until the host reads and clears the flag
// (fused_sync_check).
struct GridSync {
  unsigned int count;
  unsigned int gen;
  int failed;
  int pad;
};
constexpr unsigned int kGridSyncSpins = 1u << 21;  // about a second of polling (two L2 round trips a poll)

// The block's writes are ordered before its arrival by the barrier and
// thread 0's release (cumulative over the CTA); the others' writes are
// visible after thread 0's acquire of the new generation and the barrier
// that follows.
DEV unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
DEV bool grid_sync(GridSync* gs, unsigned int nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int g, old;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(&gs->gen) : "memory");
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(&gs->count) : "memory");
    if (old == nblocks - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&gs->count) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&gs->gen) : "memory");  // release the others
    } else {
      unsigned int spins = 0;
      volatile int* vfail = &gs->failed;
      while (ld_acquire(&gs->gen) == g) {
        if (++spins > kGridSyncSpins || *vfail) {
          atomicExch(&gs->failed, 1);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename R>
struct FusedArgs {
  using ST = typename Store<R>::T;
  LevelArgsT<R> A;    // A.base: the linearisation point of the tangent form (else null)
  MortarArgsT<R> MA;
  const GasT<R>* gas;
  LevelArgsT<double> A64;  // FP64 geometry for the time step
  const GasD* gasd;
  const double* cfl_q;  // state the block's time step is computed from
  double* q;            // state (or correction) updated in place
  const double* s;      // source (or linear right-hand side)
  double* g;            // RK register
  double* dt0;
  double* dt1;          // the next sweep's step (FAS form); unused when !dt_next
  const double* mask;   // per slot: 0 holds the slot (smoothing control), or null
  const double* hold;   // per slot: 0 holds the slot (held solves), or null
  const double* geo64;
  ST* trq;
  ST* trg;
  ST* ust;
  ST* vol;
  ST* fst;
  double a[3], b[3];    // RK3 coefficients of the three stages
  int64_t mnodes;
  int mper;             // mortar nodes per block (a contiguous run: the level's nodes spread over every block)
  int ntiles;
  int nslots;
  int sweeps;
  int dt_next;          // 1: reduce the next sweep's step in the last stage (FAS form); 0: one step per block
  int vsplit;           // 1: the volume phase takes the split form (the one k_volume_split runs)
  GridSync* sync;
};

template <typename R, int DIM, bool AFFINE>
__global__ void __launch_bounds__(kTileNodes, 1) k_smooth_block(FusedArgs<R> F) {
  pdl_enter();
  extern __shared__ double smem_raw[];
  GridSync* gs = F.sync;
  if (*reinterpret_cast<volatile int*>(&gs->failed)) return;
  const unsigned int nb = gridDim.x;
  const int64_t m0 = (int64_t)blockIdx.x * F.mper;  // this block's run of mortar nodes
  // the block's first time step (the work of k_fill and k_cfl)
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < F.nslots; j += blockDim.x) F.dt0[j] = 1e300;
  if (!grid_sync(gs, nb)) return;
  for (int w = blockIdx.x; w < F.ntiles; w += gridDim.x) cfl_tile<DIM>(F.A64, w, F.gasd, F.cfl_q, F.dt0);
  if (!grid_sync(gs, nb)) return;
  for (int k = 0; k < F.sweeps; ++k) {
    double* dt = (F.dt_next && (k & 1)) ? F.dt1 : F.dt0;
    double* dtn = (F.dt_next && k + 1 < F.sweeps) ? ((k & 1) ? F.dt0 : F.dt1) : nullptr;
    if (F.mask || F.hold) {  // (the work of k_mask_dt)
      if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < F.nslots; j += blockDim.x) {
          if (F.mask && F.mask[j] == 0.0) dt[j] = 0.0;
          if (F.hold && F.hold[j] == 0.0) dt[j] = 0.0;
        }
      if (!grid_sync(gs, nb)) return;
    }
    for (int stage = 0; stage < 3; ++stage) {
      if (k == 0 && stage == 0) {  // the block's first traces; later ones come from the surface phase
        for (int w = blockIdx.x; w < F.ntiles; w += gridDim.x) {
          trace_tile<R, DIM>(F.A, w, F.q, F.trq, reinterpret_cast<R*>(smem_raw));
          __syncthreads();
        }
        if (!grid_sync(gs, nb)) return;
      }
      for (int i = threadIdx.x; i < F.mper; i += blockDim.x)
        mortar_conf_node<R, 1>(F.A, F.MA, F.gas, F.trq, nullptr, F.ust, m0 + i);
      if (!grid_sync(gs, nb)) return;
      for (int w = blockIdx.x; w < F.ntiles; w += gridDim.x) {
        if (F.vsplit)
          volume_split_tile<R, DIM, AFFINE>(F.A, w, F.gas, F.q, F.ust, F.trg, F.vol, smem_raw);
        else
          volume_tile<R, DIM, AFFINE>(F.A, w, F.gas, F.q, F.ust, F.trg, F.vol, smem_raw);
        __syncthreads();
      }
      if (!grid_sync(gs, nb)) return;
      for (int i = threadIdx.x; i < F.mper; i += blockDim.x)
        mortar_conf_node<R, 2>(F.A, F.MA, F.gas, F.trq, F.trg, F.fst, m0 + i);
      if (!grid_sync(gs, nb)) return;
      RKArgs rk;
      rk.stage = stage;
      rk.a = F.a[stage];
      rk.b = F.b[stage];
      rk.g = F.g;
      rk.dt = dt;
      rk.qupd = F.q;
      rk.trq_next = F.trq;
      rk.dt_next = dtn;
      rk.gasd = dtn ? F.gasd : nullptr;
      rk.geo64 = dtn ? F.geo64 : nullptr;
      rk.nslots = dtn ? F.nslots : 0;
      for (int w = blockIdx.x; w < F.ntiles; w += gridDim.x) {
        surface_tile<R, DIM>(F.A, w, F.vol, F.fst, F.s, nullptr, nullptr, rk, smem_raw);
        __syncthreads();
      }
      if (k + 1 < F.sweeps || stage < 2)
        if (!grid_sync(gs, nb)) return;
    }
  }
}

// DG_FUSED_SMOOTH=0 (default) never fuses, 1 fuses levels with at most
// kFusedMaxTiles element tiles, 2 every level that qualifies.  The results
// are the same bits either way; the knob selects the launch form only.
// Measured on GB300 (CUDA events, V-cycles replayed from graphs), separate
// launches / fused blocks (1):
//   periodic 3x3x3 box, N = 2, V 2 -> 1, 3/3/10 sweeps: FP64 2.00 / 2.41 ms,
//     mixed form 1.52 / 1.90 ms
//   flat plate 60x24, N = 7, V 7 -> 1, 2/2/4 sweeps (N <= 3 fused): FP64
//     6.60 / 6.98 ms, mixed form 3.20 / 3.64 ms
//   4x4x1 box to 1e-10 (550 cycles): FP64 1.59 / 1.92 s
// A grid barrier costs about 2 us more than the gap between two kernels
// launched back to back with programmatic dependent launch (in a graph or
// not), so fusing does not pay while each phase is one warp's latency chain.
static int fused_mode() {
  static const int mode = [] {
    const char* e = std::getenv("DG_FUSED_SMOOTH");
    return e ? std::atoi(e) : 0;
  }();
  return mode;
}
constexpr int kFusedMaxTiles = 304;  // two tiles per SM

static GridSync* fused_sync(const dg_mesh* m) { return reinterpret_cast<GridSync*>(m->d_scalars + 7 * m->nslots); }

template <typename R, int DIM, bool AFF>
static int launch_fused(const dg_mesh* m, const Level* L, FusedArgs<R> F, cudaStream_t st) {
  // shared memory: the volume phase's staging of a tile of at most 128 nodes
  // (37.5 KB, below the default limit, so no attribute is set per device)
  static_assert((3 * kNP * kNP + 32 * kTileNodes) * sizeof(double) <= 48 * 1024, "fused kernel shared memory");
  const size_t smem = std::max((size_t)(3 * kNP * kNP + 32 * L->tile_smem_nodes), (size_t)(5 * L->tile_smem_nodes)) *
                      sizeof(double);
  // resident blocks per SM at the largest shared memory (the grid never exceeds what is co-resident)
  static const int occ = [] {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_smooth_block<R, DIM, AFF>, kTileNodes,
                                                      (3 * kNP * kNP + 32 * kTileNodes) * sizeof(double)) !=
        cudaSuccess)
      return 0;
    return v;
  }();
  if (occ < 1) return kNotFused;
  // one block per tile, or per 32 mortar nodes where those are more (the
  // separate kernels' one-warp mortar CTAs), up to what is co-resident
  const int64_t mwarps = (F.mnodes + 31) / 32;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(F.ntiles, mwarps),
                                                                (int64_t)occ * sm_count_cached()));
  F.mper = (int)((F.mnodes + grid - 1) / grid);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kTileNodes);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  DG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_smooth_block<R, DIM, AFF>, F));
  return DG_OK;
}

template <typename R>
static int smooth_fused_t(const dg_mesh* m, Level* L, double* q, const double* s, const double* cfl_q,
                          const double* base, int sweeps, bool dt_next, const double* mask, const double* hold,
                          double* dt0, double* dt1, cudaStream_t st) {
  FusedArgs<R> F;
  F.A = largs<R>(L);
  F.A.base = base;
  F.MA = margs<R>(L);
  F.gas = gas_table<R>(m);
  F.A64 = largs<double>(L);
  F.gasd = m->d_gasd;
  F.cfl_q = cfl_q;
  F.q = q;
  F.s = s;
  F.g = L->d_G;
  F.dt0 = dt0;
  F.dt1 = dt1;
  F.mask = mask;
  F.hold = hold;
  F.geo64 = L->d_geo;
  F.trq = buf<R>(L->d_trq);
  F.trg = buf<R>(L->d_trg);
  F.ust = buf<R>(L->d_ust);
  F.vol = buf<R>(L->d_vol);
  F.fst = buf<R>(L->d_fst);
  for (int k = 0; k < 3; ++k) {
    const RKArgs rk = rk_args(k, nullptr, nullptr, nullptr);
    F.a[k] = rk.a;
    F.b[k] = rk.b;
  }
  F.mnodes = L->mortar_nodes;
  F.ntiles = L->n_tiles;
  F.nslots = m->nslots;
  F.sweeps = sweeps;
  F.dt_next = dt_next ? 1 : 0;
  // (the split form needs at least DIM threads per tile node: 128 threads cover tiles of up to 128 / DIM nodes;
  // larger tiles take the plain form, the same bits)
  F.vsplit = (volume_split(L, std::is_same<R, double>::value) && L->tile_class_nodes[0] * L->dim <= kTileNodes) ? 1 : 0;
  F.mper = 0;
  F.sync = fused_sync(m);
  if (L->dim == 2)
    return L->affine ? launch_fused<R, 2, true>(m, L, F, st) : launch_fused<R, 2, false>(m, L, F, st);
  return L->affine ? launch_fused<R, 3, true>(m, L, F, st) : launch_fused<R, 3, false>(m, L, F, st);
}

static bool fused_eligible(const Level* L) {
  const int mode = fused_mode();
  if (mode == 0 || !L->mortars_conforming || L->n_tiles < 1) return false;
  if (L->tile_class_end[0] != L->n_tiles || L->tile_class_nodes[0] > kTileNodes) return false;  // 128-node tiles only
  if (mode == 1 && L->n_tiles > kFusedMaxTiles) return false;
  static const int coop = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
      return 0;
    return v;
  }();
  return coop != 0;
}

int smooth_block_fused(const dg_mesh* m, Level* L, double* q, const double* s, int sweeps, const double* mask,
                       const double* hold, double* dt0, double* dt1, cudaStream_t st) {
  if (sweeps < 1 || m->arith == DG_ARITH_DF32 || !fused_eligible(L)) return kNotFused;  // FP64 operator only
  int rc = configure_smem();
  if (rc != DG_OK) return rc;
  return smooth_fused_t<double>(m, L, q, s, q, nullptr, sweeps, true, mask, hold, dt0, dt1, st);
}

int smooth_tangent_fused(const dg_mesh* m, Level* L, const double* base, double* d, const double* b, int sweeps,
                         const double* mask, const double* hold, double* dt, cudaStream_t st) {
  if (sweeps < 1 || !fused_eligible(L)) return kNotFused;
  int rc = configure_smem();
  if (rc != DG_OK) return rc;
  if ((rc = ensure_tf(L, st)) != DG_OK) return rc;
  return smooth_fused_t<tf>(m, L, d, b, base, base, sweeps, false, mask, hold, dt, dt, st);
}

int fused_sync_check(const dg_mesh* m, cudaStream_t st) {
  GridSync h{};
  DG_CUDA_TRY(cudaMemcpyAsync(&h, fused_sync(m), sizeof(h), cudaMemcpyDeviceToHost, st));
  DG_CUDA_TRY(cudaStreamSynchronize(st));
  if (h.failed) {
    DG_CUDA_TRY(cudaMemsetAsync(fused_sync(m), 0, sizeof(GridSync), st));
    DG_CUDA_TRY(cudaStreamSynchronize(st));
    set_error("fused smoothing kernel: a grid barrier wait ran out (results of the cycle are void)");
    return DG_ECUDA;
  }
  return DG_OK;
}

template <typename R>
static int profile_t(const dg_mesh* m, Level* L, const double* q, const double* s, double* r, int iters,
                     double* ms_out, cudaStream_t st, const double* base = nullptr) {
  const GasT<R>* G = gas_table<R>(m);
  RKArgs rk = rk_args(-1, nullptr, nullptr, nullptr);
  TauArgs ta{nullptr, nullptr, nullptr, 0, 0};
  cudaEvent_t e0, e1;
  DG_CUDA_TRY(cudaEventCreate(&e0));
  DG_CUDA_TRY(cudaEventCreate(&e1));
  for (int k = 0; k < 6; ++k) {
    DG_CUDA_TRY(cudaEventRecord(e0, st));
    for (int it = 0; it < iters; ++it) {
      switch (k) {
        case 0: launch_trace<R>(L, q, st, base); break;
        case 1: launch_mortar<R>(1, L, G, st); break;
        case 2: launch_volume<R>(L, G, q, st, -1, 0, base); break;
        case 3: launch_mortar<R>(2, L, G, st); break;
        case 4: launch_surface<R>(L, s, r, nullptr, rk, st, base); break;
        default:
          if (std::is_same<R, tf>::value) break;  // tau stays FP64 in the mixed form: timed in FP64 below
          launch_isolated<R>(L, G, q, s, r, ta, st);
          break;
      }
    }
    DG_CUDA_TRY(cudaEventRecord(e1, st));
    DG_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    DG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    ms_out[k] = ms / std::max(1, iters);
  }
  DG_CUDA_TRY(cudaGetLastError());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return DG_OK;
}

// scratch state for tuning: every node at its solve's freestream
__global__ void __launch_bounds__(kTileNodes) k_fill_freestream(LevelArgsT<double> A, const double* __restrict__ qinf,
                                                                double* __restrict__ q) {
  const ElemTile t = A.tiles[blockIdx.x];
  const int nn = t.n[0] * t.n[1] * t.n[2];
  for (int i = threadIdx.x; i < t.count * nn; i += blockDim.x) {
    const int le = i / nn, node = i - le * nn;
    const int e = A.tile_elems[t.first + le];
    const size_t base = (size_t)5 * A.off[e] + node;
#pragma unroll
    for (int v = 0; v < 5; ++v) q[base + v * nn] = qinf[A.slot[e] * 5 + v];
  }
}

template <typename R>
static int residual_t(const dg_mesh* m, Level* L, const double* q, const double* s, double* r, bool isolated,
                      cudaStream_t st, double* d_norm, int rk_stage, double* rk_g, const double* d_dt,
                      int trace_flags, double* dt_next, const double* base);

template <typename R>
static int tune_t(dg_mesh* m, Level* L, const double* q, cudaStream_t st) {
  static const int packs[3] = {64, 128, 256};
  static const int options[kTileClasses][2] = {{64, 128}, {128, 256}, {256, 512}};
  const GasT<R>* G = gas_table<R>(m);
  cudaEvent_t e0, e1;
  DG_CUDA_TRY(cudaEventCreate(&e0));
  DG_CUDA_TRY(cudaEventCreate(&e1));
  double best_total = 1e300;
  int best_pack = L->pack, best_threads[kTileClasses] = {L->class_threads[0], L->class_threads[1],
                                                         L->class_threads[2]};
  int rc = DG_OK;
  for (int pk : packs) {
    if ((rc = build_tiles(L, pk)) != DG_OK) break;
    int th_c[kTileClasses] = {kTileNodes, 2 * kTileNodes, kVolThreads};
    for (int c = 0; c < kTileClasses; ++c) {
      const int begin = c ? L->tile_class_end[c - 1] : 0;
      if (L->tile_class_end[c] == begin) continue;
      double best_c = 1e300;
      for (int th : options[c]) {
        launch_volume<R>(L, G, q, st, c, th);  // warm-up
        DG_CUDA_TRY(cudaEventRecord(e0, st));
        for (int k = 0; k < 5; ++k) launch_volume<R>(L, G, q, st, c, th);
        DG_CUDA_TRY(cudaEventRecord(e1, st));
        DG_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        DG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_c) {
          best_c = ms;
          th_c[c] = th;
        }
      }
    }
    // packings are compared on the whole residual: the other tile kernels
    // (traces, surface) see the same tiles
    for (int c = 0; c < kTileClasses; ++c) L->class_threads[c] = th_c[c];
    if ((rc = residual_t<R>(m, L, q, nullptr, L->d_R, false, st, nullptr, -1, nullptr, nullptr, 0, nullptr)) !=
        DG_OK)
      break;
    DG_CUDA_TRY(cudaEventRecord(e0, st));
    for (int k = 0; k < 5; ++k)
      if ((rc = residual_t<R>(m, L, q, nullptr, L->d_R, false, st, nullptr, -1, nullptr, nullptr, 0, nullptr)) !=
          DG_OK)
        break;
    if (rc != DG_OK) break;
    DG_CUDA_TRY(cudaEventRecord(e1, st));
    DG_CUDA_TRY(cudaEventSynchronize(e1));
    float ms_res = 0.f;
    DG_CUDA_TRY(cudaEventElapsedTime(&ms_res, e0, e1));
    const double total = ms_res;
    if (total < best_total) {
      best_total = total;
      best_pack = pk;
      for (int c = 0; c < kTileClasses; ++c) best_threads[c] = th_c[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DG_OK) return rc;
  if (L->pack != best_pack && (rc = build_tiles(L, best_pack)) != DG_OK) return rc;
  for (int c = 0; c < kTileClasses; ++c) L->class_threads[c] = best_threads[c];
  L->tuned = true;
  return DG_OK;
}

int tune_level(dg_mesh* m, Level* L, cudaStream_t st) {
  int rc = configure_smem();
  if (rc != DG_OK) return rc;
  if ((rc = ensure_work(L)) != DG_OK) return rc;
  if ((rc = prepare_arith(m, L, st)) != DG_OK) return rc;
  std::vector<double> qinf((size_t)5 * m->nslots);
  for (int k = 0; k < m->nslots; ++k)
    for (int v = 0; v < 5; ++v) qinf[k * 5 + v] = m->slot_raw[k][7 + v];
  double *q = nullptr, *dq = nullptr;
  DG_CUDA_TRY(cudaMalloc(&q, (size_t)5 * L->nodes * sizeof(double)));
  DG_CUDA_TRY(cudaMalloc(&dq, qinf.size() * sizeof(double)));
  DG_CUDA_TRY(cudaMemcpyAsync(dq, qinf.data(), qinf.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  count_launch();
  k_fill_freestream<<<L->n_tiles, kTileNodes, 0, st>>>(largs<double>(L), dq, q);
  DG_CUDA_TRY(cudaGetLastError());
  rc = (m->arith == DG_ARITH_DF32) ? tune_t<dd>(m, L, q, st) : tune_t<double>(m, L, q, st);
  DG_CUDA_TRY(cudaStreamSynchronize(st));
  {
    std::lock_guard<std::mutex> lock(device_sync_mutex());
    cudaFree(q);
    cudaFree(dq);
  }
  return rc;
}

int profile_residual(const dg_mesh* m, Level* L, const double* q, const double* s, double* r, int iters,
                     double* ms_out, cudaStream_t st) {
  // One full evaluation fills every intermediate buffer; then each stage is
  // launched `iters` times back to back between two events on `st` (each
  // stage rewrites only its own outputs, so repeats are idempotent) and the
  // mean duration per launch is reported.
  int rc = residual(m, L, q, s, r, false, st, nullptr, -1, nullptr, nullptr);
  if (rc != DG_OK) return rc;
  if (m->arith == DG_ARITH_DF32) return profile_t<dd>(m, L, q, s, r, iters, ms_out, st);
  if (m->arith == DG_ARITH_MIXED) {
    // the operator stages as the mixed cycle runs them: tangent kernels,
    // J(q) dq with dq = q (any direction costs the same); the isolated
    // operator in FP64
    if ((rc = residual_tangent(m, L, q, q, s, r, st, nullptr, -1, nullptr, nullptr)) != DG_OK) return rc;
    double iso[6];
    if ((rc = profile_t<double>(m, L, q, s, r, iters, iso, st)) != DG_OK) return rc;
    if ((rc = profile_t<tf>(m, L, q, s, r, iters, ms_out, st, q)) != DG_OK) return rc;
    ms_out[5] = iso[5];
    return DG_OK;
  }
  return profile_t<double>(m, L, q, s, r, iters, ms_out, st);
}

int cfl_dt(const dg_mesh* m, Level* L, const double* q, double* d_dt, cudaStream_t st) {
  int rc = fill(d_dt, 1e300, m->nslots, st);
  if (rc != DG_OK) return rc;
  count_launch();
  if (L->dim == 2)
    launch_k(k_cfl<2>, L->n_tiles, kTileNodes, 0, st, largs<double>(L), m->d_gasd, q, d_dt);
  else
    launch_k(k_cfl<3>, L->n_tiles, kTileNodes, 0, st, largs<double>(L), m->d_gasd, q, d_dt);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

int transfer(const dg_mesh* m, const Level* from, const Level* to, int nvar, const double* in, double* out,
             cudaStream_t st, const double* sub, bool accumulate) {
  (void)m;
  int rc = configure_smem();
  if (rc != DG_OK) return rc;
  // shared memory: two slabs of the largest per-variable intermediate
  size_t slab = 0;
  for (int e = 0; e < from->K; ++e) {
    const int* f = &from->nvec_host[e * 3];
    const int* t = &to->nvec_host[e * 3];
    size_t a = std::max((size_t)f[0] * f[1] * f[2], (size_t)t[0] * t[1] * t[2]);
    size_t b = std::max((size_t)f[2] * f[1] * t[0], (size_t)f[2] * t[1] * t[0]);
    slab = std::max(slab, std::max(a, b));
  }
  if (slab > (size_t)kTransferMaxSlab || nvar < 1) {
    set_error("transfer: element too large for the shared-memory slab");
    return DG_EINVAL;
  }
  // as many variables per pass as two slabs each fit in the reserved shared memory
  const int vgroup = std::max(1, std::min(nvar, (int)(kTransferMaxSlab / slab)));
  count_launch();
  launch_k(k_transfer, from->K, kTransferThreads, 2 * (size_t)vgroup * slab * sizeof(double), st, from->d_n,
           from->d_off, to->d_n, to->d_off, nvar, vgroup, in, sub, out, accumulate ? 1 : 0);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

static int tau_reduce(const Level* L, const double* r, const double* rho, int dir, int slot,
                      const int32_t* fine_orders, double* table, cudaStream_t st);

int tau_accumulate(const dg_mesh* m, Level* L, const double* q, const double* s, const double* rho, bool isolated,
                   int dir, int slot, const int32_t* fine_orders_dev, double* d_tau, cudaStream_t st) {
  int rc = configure_smem();
  if (rc != DG_OK) return rc;
  if (!isolated) {
    // full operator: residual into the level's scratch, then reduce
    rc = residual(m, L, q, s, L->d_R, false, st, nullptr, -1, nullptr, nullptr);
    if (rc != DG_OK) return rc;
    return tau_reduce(L, L->d_R, rho, dir, slot, fine_orders_dev, d_tau, st);
  }
  TauArgs ta{rho, d_tau, fine_orders_dev, dir, slot};
  if (m->arith == DG_ARITH_DF32) {
    if ((rc = ensure_dd(L, st)) != DG_OK) return rc;
    launch_isolated<dd>(L, gas_table<dd>(m), q, s, nullptr, ta, st);
  } else {
    launch_isolated<double>(L, gas_table<double>(m), q, s, nullptr, ta, st);
  }
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

__global__ void k_tau_reduce(LevelArgsT<double> A, const double* __restrict__ r, const double* __restrict__ rho, int dir,
                             int slot, const int32_t* __restrict__ fine_orders, double* table) {
  pdl_enter();
  const ElemTile t = A.tiles[blockIdx.x];
  const int nn = t.n[0] * t.n[1] * t.n[2];
  const int T = t.count * nn;
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    int le = i / nn, node = i - le * nn;
    int e = A.tile_elems[t.first + le];
    const size_t base = (size_t)5 * A.off[e] + node;
    double tmax = 0.0;
    for (int v = 0; v < 5; ++v) {
      double tv = r[base + v * nn] - (rho ? rho[base + v * nn] : 0.0);
      tmax = fmax(tmax, fabs(tv));
    }
    if (fine_orders[e * 3 + dir] > slot) atomic_max_nonneg(table + ((size_t)e * 3 + dir) * kTauSlots + slot, tmax);
  }
}

static int tau_reduce(const Level* L, const double* r, const double* rho, int dir, int slot,
                      const int32_t* fine_orders, double* table, cudaStream_t st) {
  count_launch();
  launch_k(k_tau_reduce, L->n_tiles, kTileNodes, 0, st, largs<double>(L), r, rho, dir, slot, fine_orders, table);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free order-map transfer (dg_transfer_noalloc in dg.h)
//
// Some callers cannot allocate device memory when they need a transfer: a
// host code that reserves all device memory up front in its own pool leaves
// none for a library.  This variant of k_transfer needs no
// mesh handle and no library-allocated buffer: its only scratch -- one
// 8-int record per element (both node-count triples and both node offsets) --
// lives in the static device array below, and its 1-D projection /
// interpolation matrices are formed in shared memory from the Gauss nodes in
// constant memory.  The array is reserved on every GPU that loads the library
// and stays reserved until the process exits.  Every call shares it, so
// calls whose kernels overlap on the GPU race; each call rewrites the records
// of all the elements it uses, so nothing has to start at zero.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxElems = 65536;  // 65,536 elements -> 2 MiB of records
constexpr int kNoAllocRec = 8;
constexpr int kNoAllocMaxVars = 64;      // variables per node
static __device__ __align__(256) int32_t g_noalloc_records[kNoAllocMaxElems * kNoAllocRec];

namespace {
constexpr int kMaxDevices = 64;
int32_t* g_noalloc_dev_ptr[kMaxDevices] = {nullptr};
bool g_noalloc_ready[kMaxDevices] = {false};
std::mutex g_noalloc_mutex;
}  // namespace

// l_j(x) on the n Gauss nodes of c_tab, from the product formula
DEV double noalloc_lagrange(int n, int j, double x) {
  double v = 1.0;
  for (int i = 0; i < n; ++i)
    if (i != j) v *= (x - c_tab.x[n][i]) / (c_tab.x[n][j] - c_tab.x[n][i]);
  return v;
}

__global__ void k_transfer_noalloc(int nvar, const int32_t* __restrict__ rec_all, const double* __restrict__ in,
                                   double* __restrict__ out) {
  __shared__ double sT[3][kNP * kNP];
  const int e = blockIdx.x;
  const int32_t* rec = rec_all + (size_t)e * kNoAllocRec;
  const int nf[3] = {rec[0], rec[1], rec[2]};
  const int nt[3] = {rec[3], rec[4], rec[5]};
  // 1-D matrices: L2 projection when the order drops, interpolation when it
  // rises, identity when equal
  for (int d = 0; d < 3; ++d)
    for (int k = threadIdx.x; k < nt[d] * nf[d]; k += blockDim.x) {
      int j = k / nf[d], i = k - j * nf[d];
      double v;
      if (nt[d] < nf[d])
        v = c_tab.w[nf[d]][i] * noalloc_lagrange(nt[d], j, c_tab.x[nf[d]][i]) / c_tab.w[nt[d]][j];
      else if (nt[d] > nf[d])
        v = noalloc_lagrange(nf[d], i, c_tab.x[nt[d]][j]);
      else
        v = (i == j) ? 1.0 : 0.0;
      sT[d][k] = v;
    }
  __syncthreads();
  const int nnf = nf[0] * nf[1] * nf[2], nnt = nt[0] * nt[1] * nt[2];
  const double* ie = in + (size_t)nvar * rec[6];
  double* oe = out + (size_t)nvar * rec[7];
  for (int i = threadIdx.x; i < nnt * nvar; i += blockDim.x) {
    int v = i / nnt, j = i - v * nnt;
    int j0 = j % nt[0], j1 = (j / nt[0]) % nt[1], j2 = j / (nt[0] * nt[1]);
    double acc = 0.0;
    for (int k2 = 0; k2 < nf[2]; ++k2)
      for (int k1 = 0; k1 < nf[1]; ++k1) {
        double w21 = sT[2][j2 * nf[2] + k2] * sT[1][j1 * nf[1] + k1];
        for (int k0 = 0; k0 < nf[0]; ++k0)
          acc += w21 * sT[0][j0 * nf[0] + k0] * ie[v * nnf + (k2 * nf[1] + k1) * nf[0] + k0];
      }
    oe[v * nnt + j] = acc;
  }
}

// Once per device, with that device current: resolve the static array's
// device address and make sure the Gauss tables are in constant memory
// (cudaMemcpyToSymbol writes them; it allocates nothing).
static int noalloc_setup(int32_t** ptr) {
  int dev = 0;
  DG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("dg_transfer_noalloc: device index out of range");
    return DG_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ready[dev]) {
    int32_t* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_records);
    if (e != cudaSuccess || p == nullptr) {
      set_error(std::string("dg_transfer_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return DG_ECUDA;
    }
    const Tables1D& T = tables();
    DevTables h;
    memset(&h, 0, sizeof(h));
    for (int n = 1; n < kNP; ++n)
      for (int j = 0; j < n; ++j) {
        h.x[n][j] = T.x[n][j];
        h.w[n][j] = T.w[n][j];
        h.lm[n][j] = T.lm[n][j];
        h.lp[n][j] = T.lp[n][j];
        h.lmw[n][j] = T.lm[n][j] / T.w[n][j];
        h.lpw[n][j] = T.lp[n][j] / T.w[n][j];
      }
    DG_CUDA_TRY(cudaMemcpyToSymbol(c_tab, &h, sizeof(h)));
    g_noalloc_dev_ptr[dev] = p;
    g_noalloc_ready[dev] = true;
  }
  *ptr = g_noalloc_dev_ptr[dev];
  return DG_OK;
}

int transfer_noalloc(int dim, int K, const int32_t* orders_from, const int32_t* orders_to, int nvar,
                     const double* in, double* out, cudaStream_t st) {
  if ((dim != 2 && dim != 3) || K < 1 || !orders_from || !orders_to || !in || !out) {
    set_error("dg_transfer_noalloc: bad argument");
    return DG_EINVAL;
  }
  if (nvar < 1 || nvar > kNoAllocMaxVars) {  // keeps nodes x nvar far inside 32 bits in the kernel
    set_error("dg_transfer_noalloc: nvar must lie in [1, " + std::to_string(kNoAllocMaxVars) + "]");
    return DG_EINVAL;
  }
  if (K > kNoAllocMaxElems) {
    set_error("dg_transfer_noalloc: " + std::to_string(K) + " elements exceed the static limit of " +
              std::to_string(kNoAllocMaxElems));
    return DG_EINVAL;
  }
  std::vector<int32_t> rec((size_t)K * kNoAllocRec);
  int64_t of = 0, ot = 0;
  for (int e = 0; e < K; ++e) {
    int32_t* r = &rec[(size_t)e * kNoAllocRec];
    for (int d = 0; d < 3; ++d) {
      int a = orders_from[e * 3 + d], b = orders_to[e * 3 + d];
      bool active = d < dim;
      if ((active && (a < 1 || a > kNMax || b < 1 || b > kNMax)) || (!active && (a != 0 || b != 0))) {
        set_error("dg_transfer_noalloc: order out of range at element " + std::to_string(e));
        return DG_EINVAL;
      }
      r[d] = active ? a + 1 : 1;
      r[3 + d] = active ? b + 1 : 1;
    }
    if (of + (int64_t)r[0] * r[1] * r[2] > INT32_MAX || ot + (int64_t)r[3] * r[4] * r[5] > INT32_MAX) {
      set_error("dg_transfer_noalloc: node offsets exceed 32 bits");
      return DG_EINVAL;
    }
    r[6] = (int32_t)of;
    r[7] = (int32_t)ot;
    of += (int64_t)r[0] * r[1] * r[2];
    ot += (int64_t)r[3] * r[4] * r[5];
  }
  int32_t* dev_rec = nullptr;
  int rc = noalloc_setup(&dev_rec);
  if (rc != DG_OK) return rc;
  DG_CUDA_TRY(cudaMemcpyAsync(dev_rec, rec.data(), rec.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  count_launch();
  k_transfer_noalloc<<<K, 128, 0, st>>>(nvar, dev_rec, in, out);
  DG_CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

}  // namespace dg
