// Internal declarations of the GB300 DGSEM library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dg.h"

namespace dg {

constexpr int kNMax = 12;               // highest polynomial order
constexpr int kNP = kNMax + 2;          // table stride (n = 1 .. kNMax+1)
constexpr int kMaxElemNodes = 729;      // 3D element node cap (smem staging)
constexpr int kTileNodes = 128;         // element-kernel CTA size (threads) and tile target
constexpr int kVolThreads = 512;        // launch bound of the element-tile kernels with staged tiles
constexpr int kTileClasses = 3;         // tiles of <= 128, <= 256 and more nodes (one element)
constexpr int kMortarTile = 64;         // mortar-kernel CTA size (threads) and tile target
constexpr int kMortarTileMax = 169;     // a single mortar of 13 x 13 nodes forms its own tile
constexpr int kTauSlots = 16;           // orders per direction in the tau table

void set_error(const std::string& msg);

// Process-wide state kept once per CUDA device (device tables, one-time
// set-up flags): get(dev) is the entry of device `dev`, or nullptr for an
// index outside [0, kMax).  Pure host bookkeeping; callers serialise access.
template <typename T>
class PerDevice {
 public:
  static constexpr int kMax = 64;
  T* get(int dev) { return (dev >= 0 && dev < kMax) ? &slots_[dev] : nullptr; }

 private:
  T slots_[kMax] = {};
};

#define DG_CUDA_TRY(call)                                                              \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess) {                                                           \
      ::dg::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));             \
      return DG_ECUDA;                                                                 \
    }                                                                                  \
  } while (0)

// ---------------------------------------------------------------------------
// 1-D tables (host, FP64) for n = 1 .. kNMax+1 Legendre-Gauss nodes
// ---------------------------------------------------------------------------
struct Tables1D {
  double x[kNP][kNP], w[kNP][kNP];   // nodes, weights
  double bw[kNP][kNP];               // barycentric weights
  double Dhat[kNP][kNP][kNP];        // weak-form derivative: -(w_a/w_i) l_i'(x_a)  [n][i][a]
  double D[kNP][kNP][kNP];           // collocation derivative: l_a'(x_i)          [n][i][a]
  double lm[kNP][kNP], lp[kNP][kNP]; // l_j(-1), l_j(+1)
};
const Tables1D& tables();
double lagrange_bary(int n, int j, double x);  // l_j(x) on n Gauss nodes
// transfer matrix between n_from and n_to Gauss nodes: L2 projection (down),
// interpolation (up), identity (equal); T[j*n_from + k]
void transfer_matrix(int n_from, int n_to, double* T);

// ---------------------------------------------------------------------------
// device-side descriptors
// ---------------------------------------------------------------------------
// Device constant tables (defined in dg_kernels.cu)
struct DevTables {
  double x[kNP][kNP];
  double w[kNP][kNP];
  double lm[kNP][kNP], lp[kNP][kNP];
  double lmw[kNP][kNP], lpw[kNP][kNP];   // l(-1)/w, l(+1)/w
};

struct ElemTile {      // one CTA of an element kernel: `count` elements of one order
  int32_t first;       // index into the level's tile_elems list
  int32_t count;
  int16_t n[3];
  int16_t pad;
};

struct MortarDev {     // one mortar (a face pair or a boundary face)
  int32_t eL, fL, eR, fR;
  int32_t orient, bc;
  int32_t ma, mb;      // mortar nodes per tangential direction (L frame)
  int32_t node_off;    // first mortar node
  int32_t flags;       // bit0: both sides conforming with the mortar
  int32_t out_off;     // first of its face nodes (L side, then R side) within its tile
  int32_t pad;
};

struct MortarTile {    // one CTA of a mortar kernel
  int32_t first, count;     // mortars
  int32_t node_first, nodes;
  int32_t outs;             // face nodes written (both sides of every mortar)
};

struct GasD {  // FP64 constants of the CFL kernel
  double g, g1, gM2, Su, Su1, invRe, Ca, Cnu;
};

struct Params {
  double g, Pr, Ma, Re, Su, Ca, Cnu;
  double qinf[5];
  double pinf;
  double gM2;      // gamma M^2
  double hc;       // 1/((gamma-1) Pr M^2)
  double invRe;
};

// A level: one order map of the mesh with its geometry, tables and buffers.
struct Level {
  int dim = 3, K = 0;
  std::vector<int32_t> orders;          // K x 3
  std::vector<int64_t> off;             // K+1 node offsets
  int64_t nodes = 0;
  int64_t bytes = 0;                    // device memory this level holds
  // device
  int32_t* d_n = nullptr;               // K x 3 node counts
  int32_t* d_off = nullptr;             // K+1 (int32 suffices: < 2^31 nodes)
  double* d_geo = nullptr;              // 10 x nodes: Ja (9, [i*3+c]) then 1/J, SoA
  int32_t* d_fo = nullptr;              // K*6 element-face node offsets
  int64_t face_nodes = 0;
  double* d_fnS = nullptr;              // 3 x face_nodes: own outward metric
  double* d_trq = nullptr;              // 5 x face_nodes: q traces
  double* d_ust = nullptr;              // 4 x face_nodes: projected U*
  double* d_trg = nullptr;              // 12 x face_nodes: gradient traces
  double* d_fst = nullptr;              // 5 x face_nodes: projected F* S
  MortarDev* d_mortars = nullptr;
  int n_mortars = 0;
  int64_t mortar_nodes = 0;
  int32_t* d_mnode_mortar = nullptr;    // mortar node -> mortar
  double* d_mnS = nullptr;              // 3 x mortar_nodes
  MortarTile* d_mtiles = nullptr;
  int n_mtiles = 0;
  bool mortars_conforming = false;      // every mortar conforming: one-pass mortar kernels
  int32_t* d_tile_elems = nullptr;
  int32_t* d_slot = nullptr;            // solve slot of each element
  ElemTile* d_tiles = nullptr;
  int n_tiles = 0;
  size_t tile_smem_nodes = 0;           // max nodes of a tile
  int pack = kTileNodes;                           // tile target for small elements (nodes)
  int class_threads[kTileClasses] = {kTileNodes, 2 * kTileNodes, kVolThreads};  // per launch class
  bool tuned = false;                              // pack and threads chosen by timing
  int tile_class_end[kTileClasses] = {0, 0, 0};    // tiles are ordered by class; cumulative ends
  int tile_class_nodes[kTileClasses] = {0, 0, 0};  // max nodes of a tile of each class
  double* d_vol = nullptr;              // 5 x nodes volume part
  bool affine = false;                  // metrics constant within every element
  double* d_geo2 = nullptr;             // float-pair copies for the double-float kernels (lazy)
  double* d_fnS2 = nullptr;
  double* d_mnS2 = nullptr;
  double* d_geoT = nullptr;             // value-only float pairs for the tangent kernels (lazy)
  double* d_fnST = nullptr;
  double* d_mnST = nullptr;
  std::vector<int32_t> nvec_host;       // K x 3 node counts (host copy)
  // multigrid work arrays (allocated on first use)
  double *d_Q = nullptr, *d_S = nullptr, *d_Q0 = nullptr, *d_G = nullptr, *d_R = nullptr;
  ~Level();
};

}  // namespace dg

struct dg_mesh {
  int dim = 3, K = 0, M = 1;
  int arith = DG_ARITH_FP64;     // arithmetic of the operator kernels
  std::vector<double> xmap;
  std::vector<int32_t> ftab;
  dg::Params prm;                // slot 0 (single solves)
  double raw_params[16];
  int nslots = 1;                // independent solves batched in this mesh
  std::vector<dg::Params> slot_prm;
  std::vector<std::vector<double>> slot_raw;  // per-slot raw parameter vectors
  bool autotune = false;                       // tune every level's tiles when it is built
  std::vector<int32_t> elem_slot;             // K
  std::vector<int32_t> slot_elem_off;         // nslots + 1
  void* d_gas64 = nullptr;       // per-slot gas constants (FP64)
  void* d_gas32x2 = nullptr;     // per-slot gas constants (float pairs)
  void* d_gastf = nullptr;       // per-slot gas constants (tangent pairs, derivative 0)
  dg::GasD* d_gasd = nullptr;    // per-slot CFL constants
  std::vector<int32_t> orders;
  std::unique_ptr<dg::Level> fine;
  std::map<std::vector<int32_t>, std::unique_ptr<dg::Level>> levels;  // coarse levels by order map
  bool freeze = false;           // some solves may be held (dg_batch_set_active): every sweep masks their dt
  std::vector<int32_t> active;   // per solve 1 = advanced, 0 = held (when freeze)
  double* d_scalars = nullptr;   // per slot: [6n, 7n) the active mask; [0, n) dt, [n, 2n) max|r|, [2n, 3n) and [3n, 4n) the
                                 // smoothing-control norms, [4n, 5n) 1/0 smoothing mask, [5n, 6n) the
                                 // alternate dt of every other sweep (n = nslots)
  double* d_tau = nullptr;       // K x 3 x 16 tau table
  int32_t* d_orders = nullptr;   // K x 3 orders on the device
  cudaStream_t cap_stream = nullptr;  // stream used to capture cycle graphs
  cudaStream_t tau_st[3] = {nullptr, nullptr, nullptr};  // one per direction of the tau estimate
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int evals = 0;
    double dofs = 0.0;
    unsigned long long launches = 0;
  };
  std::map<std::string, Graph> graphs;  // captured V-cycles by (orders, pointers, parameters)
};

namespace dg {
int build_level(const dg_mesh* m, const std::vector<int32_t>& orders, Level* L);
// The metric terms of one element as build_level computes them (host only):
// Ja[node][i][c] = (J a^i)_c (9 per node) and J[node] at the element's Gauss
// nodes, node counts n[3], from its (M+1)^dim mapping nodes (3 doubles each).
void element_geometry_host(int M, int dim, const double* xmap_elem, const int n[3], double* Ja, double* J);
Level* get_level(dg_mesh* m, const std::vector<int32_t>& orders);
int ensure_work(Level* L);
// (re)build a level's element tile lists with `pack` nodes per tile for small elements
int build_tiles(Level* L, int pack);
// time the staged element kernels over tile packings and class thread counts and
// keep the fastest (results do not change: the per-node arithmetic is the same)
int tune_level(dg_mesh* m, Level* L, cudaStream_t st);
Params make_params(const double* p);

// kernels (dg_kernels.cu)
int upload_tables();
int upload_gas(dg_mesh* m);
// Held while a V-cycle is captured into a graph and around cudaFree calls:
// a cudaFree in one thread synchronises the device and would break a capture
// running in another (serving runs solves in several threads).
std::mutex& device_sync_mutex();
// device bytes held by a mesh's levels and scalars
int64_t mesh_device_bytes(const dg_mesh* m);
unsigned long long launches();        // launched by the calling thread
unsigned long long launches_total();  // launched by all threads
void add_launches(unsigned long long n);
int prepare_capture();  // one-time per-device set-up that may not run inside a capture
int prepare_arith(const dg_mesh* m, Level* L, cudaStream_t st);  // per-level data the arithmetic mode needs
// trace_flags for residual(): the face traces of q are already in the level's
// buffer (skip computing them) / an RK stage also writes the traces of the
// updated state there (the next stage then passes kTracesCurrent)
constexpr int kTracesCurrent = 1;
constexpr int kTracesNext = 2;
// dt_next (RK stages only): the next sweep's per-slot time step, reset by
// stage 1 and reduced from the updated state by stage 2 (what cfl_dt would
// compute from that state)
int residual(const dg_mesh* m, Level* L, const double* q, const double* s, double* r, bool isolated,
             cudaStream_t st, double* d_norm, int rk_stage, double* rk_g, const double* d_dt,
             int trace_flags = 0, double* dt_next = nullptr);
int cfl_dt(const dg_mesh* m, Level* L, const double* q, double* d_dt, cudaStream_t st);
// The linearised residual r = b - J(base) dq with J the Jacobian of the
// operator A at `base`, evaluated in FP32 tangent arithmetic (the correction
// solves of the mixed-precision cycle); the RK arguments as in residual()
// (an RK stage updates dq in place).
int residual_tangent(const dg_mesh* m, Level* L, const double* base, const double* dq, const double* b, double* r,
                     cudaStream_t st, double* d_norm, int rk_stage, double* rk_g, const double* d_dt,
                     int trace_flags = 0);
int profile_residual(const dg_mesh* m, Level* L, const double* q, const double* s, double* r, int iters,
                     double* ms_out, cudaStream_t st);
int transfer(const dg_mesh* m, const Level* from, const Level* to, int nvar, const double* in, double* out,
             cudaStream_t st, const double* sub = nullptr, bool accumulate = false);
// max |x| per solve slot over a level vector (out zeroed here; device)
int slot_maxabs(const dg_mesh* m, const Level* L, const double* x, double* out, cudaStream_t st);
// Runs f(begin, end) on contiguous blocks of [0, n) on up to 16 host threads,
// at least `grain` items a thread (one block, on the calling thread, when n
// is small).  Every f must write only its own block.
template <class F>
void parallel_for(int n, F f, int grain = 256) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nt = (int)std::min<unsigned>(std::min(hw, 16u), (unsigned)std::max(1, n / std::max(1, grain)));
  if (nt <= 1) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) {
    const int b = (int)((int64_t)n * t / nt), e = (int)((int64_t)n * (t + 1) / nt);
    th.emplace_back([=, &f] { f(b, e); });
  }
  f(0, (int)((int64_t)n / nt));
  for (auto& x : th) x.join();
}

// One smoothing block of a small conforming level in a single cooperative
// launch (k_smooth_block), the same bits as the separate launches.  They
// return kNotFused, with nothing launched, when the level or the arithmetic
// does not qualify; the caller then launches the stages one by one.
constexpr int kNotFused = 1;
int smooth_block_fused(const dg_mesh* m, Level* L, double* q, const double* s, int sweeps, const double* mask,
                       const double* hold, double* dt0, double* dt1, cudaStream_t st);
int smooth_tangent_fused(const dg_mesh* m, Level* L, const double* base, double* d, const double* b, int sweeps,
                         const double* mask, const double* hold, double* dt, cudaStream_t st);
// Reads (and clears) the fused kernel's barrier-failure flag: DG_ECUDA if a
// grid barrier wait ran out since the last check.  Synchronises the stream.
int fused_sync_check(const dg_mesh* m, cudaStream_t st);
// dt[k] = 0 where mask[k] == 0 (nslots entries, device)
int mask_dt(const dg_mesh* m, double* dt, const double* mask, cudaStream_t st);
int fill(double* p, double v, int64_t n, cudaStream_t st);
int axpby(double* y, double a, const double* x, double b, int64_t n, cudaStream_t st);  // y = a x + b y
int sub3(double* out, const double* a, const double* b, int64_t n, cudaStream_t st);    // out = a - b
int tau_accumulate(const dg_mesh* m, Level* L, const double* q, const double* s, const double* rho,
                   bool isolated, int dir, int order_slot, const int32_t* fine_orders_dev, double* d_tau,
                   cudaStream_t st);
int read_scalar(const double* d, double* h, cudaStream_t st);
int transfer_noalloc(int dim, int K, const int32_t* orders_from, const int32_t* orders_to, int nvar,
                     const double* in, double* out, cudaStream_t st);
int reset_max(double* d, cudaStream_t st);
// FMA rates of the current device in TFLOP/s (dg_peaks.cu)
int measure_fma_rates(double* fp64_tflops, double* fp32_tflops, cudaStream_t st);
int reset_min(double* d, cudaStream_t st);
}  // namespace dg
