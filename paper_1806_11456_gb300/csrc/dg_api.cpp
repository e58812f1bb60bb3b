// C ABI entry points and host orchestration of the multigrid cycle, the tau
// estimate and the order adaptation.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dg_internal.h"

namespace dg {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

#define DG_TRY(x)                 \
  do {                            \
    int _rc = (x);                \
    if (_rc != DG_OK) return _rc; \
  } while (0)

static int check_desc(const dg_mesh_desc* d, const int32_t* orders) {
  if (!d || !orders || !d->xmap || !d->ftab) {
    set_error("null argument");
    return DG_EINVAL;
  }
  if (d->dim != 2 && d->dim != 3) {
    set_error("dim must be 2 or 3");
    return DG_EINVAL;
  }
  if (d->K <= 0 || d->M < 1 || d->M > 8) {
    set_error("need K > 0 and 1 <= M <= 8");
    return DG_EINVAL;
  }
  for (int e = 0; e < d->K; ++e) {
    for (int i = 0; i < 3; ++i) {
      int N = orders[e * 3 + i];
      bool active = i < d->dim;
      if ((active && (N < 1 || N > kNMax)) || (!active && N != 0)) {
        set_error("order out of range at element " + std::to_string(e));
        return DG_EINVAL;
      }
    }
    for (int f = 0; f < 2 * d->dim; ++f) {
      const int32_t* ft = d->ftab + (size_t)(e * 6 + f) * 4;
      if (ft[0] >= 0) {
        if (ft[0] >= d->K || ft[1] < 0 || ft[1] >= 2 * d->dim || ft[2] < 0 || ft[2] > 7) {
          set_error("bad face entry at element " + std::to_string(e));
          return DG_EINVAL;
        }
        const int32_t* bk = d->ftab + (size_t)(ft[0] * 6 + ft[1]) * 4;
        if (bk[0] != e || bk[1] != f) {
          set_error("face table not symmetric at element " + std::to_string(e));
          return DG_EINVAL;
        }
      } else if (ft[3] < DG_BC_FREESTREAM || ft[3] > DG_BC_WALL) {
        set_error("bad boundary tag at element " + std::to_string(e));
        return DG_EINVAL;
      }
    }
  }
  return DG_OK;
}

static cudaStream_t S(void* p) { return reinterpret_cast<cudaStream_t>(p); }

// ---------------------------------------------------------------------------
// multigrid
// ---------------------------------------------------------------------------
struct Cycle {
  dg_mesh* m;
  cudaStream_t st;
  dg_mg_params mg;
  std::vector<Level*> lv;  // lv[k]: k-th level from the top (lv[0] = finest)
  int evals = 0;
  double dofs = 0.0;
  const double* q_fine = nullptr;  // mixed-precision cycle: the finest state (linearisation point)
};

// `sweeps` RK3 sweeps; with a mask (per slot 1/0, device) the slots whose
// mask is 0 get dt = 0 and are left unchanged.
static int smooth_level(Cycle& C, Level* L, double* Q, const double* Sv, int sweeps,
                        const double* mask = nullptr) {
  DG_TRY(ensure_work(L));
  // The sweeps alternate two per-slot dt buffers: the last stage of a sweep
  // reduces the next sweep's dt from the state it produces, so only the
  // block's first sweep launches the CFL kernel; likewise every stage's
  // surface kernel writes the traces of the state it updates, so only the
  // block's first stage computes them from Q.
  double* dtb[2] = {C.m->d_scalars, C.m->d_scalars + 5 * C.m->nslots};
  const double* hold = C.m->freeze ? C.m->d_scalars + 6 * C.m->nslots : nullptr;
  if (sweeps > 0) {  // a small conforming level: the whole block in one cooperative launch
    const int rc = smooth_block_fused(C.m, L, Q, Sv, sweeps, mask, hold, dtb[0], dtb[1], C.st);
    if (rc == DG_OK) {
      C.evals += 3 * sweeps;
      C.dofs += 15.0 * sweeps * L->nodes;
      return DG_OK;
    }
    if (rc != kNotFused) return rc;
  }
  if (sweeps > 0) DG_TRY(cfl_dt(C.m, L, Q, dtb[0], C.st));
  for (int k = 0; k < sweeps; ++k) {
    double* dt = dtb[k & 1];
    double* dt_next = (k + 1 < sweeps) ? dtb[(k + 1) & 1] : nullptr;
    if (mask) DG_TRY(mask_dt(C.m, dt, mask, C.st));
    if (hold) DG_TRY(mask_dt(C.m, dt, hold, C.st));  // held solves
    for (int stage = 0; stage < 3; ++stage) {
      const int tf = kTracesNext | ((k > 0 || stage > 0) ? kTracesCurrent : 0);
      DG_TRY(residual(C.m, L, Q, Sv, nullptr, false, C.st, nullptr, stage, L->d_G, dt, tf, dt_next));
      C.evals++;
      C.dofs += 5.0 * L->nodes;
    }
  }
  return DG_OK;
}

// Residual-based smoothing of Sec. 3.1.2 on one level, decided per solve slot
// on the host.  d_scalars holds per slot [2n, 3n) max|r^P|, [3n, 4n)
// max|I r^P|, [4n, 5n) the mask of the slots still smoothing.  Held solves
// (dg_batch_set_active) take no part in the rules: they count as done.
struct SmoothingRules {
  Cycle& C;
  const int ns;
  const bool on;
  const double eta;
  double* const dN;
  double* const dP;
  double* const dmask;
  std::vector<double> h, rpre;
  std::vector<char> held, done;
  const double* mask = nullptr;  // null while every slot still smooths

  explicit SmoothingRules(Cycle& c)
      : C(c), ns(c.m->nslots), on(c.mg.control > 0), eta(c.mg.eta > 0.0 ? c.mg.eta : 1.1),
        dN(c.m->d_scalars + 2 * ns), dP(c.m->d_scalars + 3 * ns), dmask(c.m->d_scalars + 4 * ns),
        h(2 * ns), rpre(ns, 0.0), held(ns, 0) {
    if (C.m->freeze)
      for (int j = 0; j < ns; ++j) held[j] = C.m->active[j] ? 0 : 1;
    done = held;
  }
  // hold the slots that are done for the next block
  int hold_done() {
    std::vector<double> hm(ns);
    for (int j = 0; j < ns; ++j) hm[j] = done[j] ? 0.0 : 1.0;
    DG_CUDA_TRY(cudaMemcpyAsync(dmask, hm.data(), ns * sizeof(double), cudaMemcpyHostToDevice, C.st));
    DG_CUDA_TRY(cudaStreamSynchronize(C.st));
    mask = dmask;
    return DG_OK;
  }
  // after pre-smoothing block `blk`, with dN and dP filled: a slot is done
  // once max|r^P| < eta max|I r^P| or after `control` blocks
  int pre(int blk, bool* all) {
    DG_CUDA_TRY(cudaMemcpyAsync(h.data(), dN, 2 * ns * sizeof(double), cudaMemcpyDeviceToHost, C.st));
    DG_CUDA_TRY(cudaStreamSynchronize(C.st));
    return decide([&](int j) {
      rpre[j] = h[j];
      return h[j] < eta * h[ns + j] || blk >= C.mg.control;
    }, all);
  }
  // the post-smoothing rule starts afresh
  void restart() {
    done = held;
    mask = nullptr;
  }
  // after a post-smoothing block, with dN filled: a slot is done once max|r|
  // is no larger than after its pre-smoothing
  int post(bool* all) {
    DG_CUDA_TRY(cudaMemcpyAsync(h.data(), dN, ns * sizeof(double), cudaMemcpyDeviceToHost, C.st));
    DG_CUDA_TRY(cudaStreamSynchronize(C.st));
    return decide([&](int j) { return h[j] <= rpre[j]; }, all);
  }

 private:
  template <typename F>
  int decide(F&& rule, bool* all) {
    bool a = true, any = false;
    for (int j = 0; j < ns; ++j) {
      if (!done[j] && rule(j)) done[j] = 1;
      a = a && done[j];
      any = any || done[j];
    }
    *all = a;
    if (!a && any) return hold_done();
    return DG_OK;
  }
};

static int vcycle_level(Cycle& C, size_t k, double* Qf, const double* Sf) {
  const bool finest = (k == 0);
  Level* L = C.lv[k];
  DG_TRY(ensure_work(L));
  double* Q = finest ? Qf : L->d_Q;
  const double* Sv = finest ? Sf : L->d_S;
  const int64_t n5 = 5 * L->nodes;
  if (!finest) {
    // S = A(Q0) + r  (r was restricted into d_S)
    DG_TRY(residual(C.m, L, Q, nullptr, L->d_R, false, C.st, nullptr, -1, nullptr, nullptr));
    C.evals++;
    C.dofs += 5.0 * L->nodes;
    DG_TRY(sub3(L->d_S, L->d_S, L->d_R, n5, C.st));
    DG_CUDA_TRY(cudaMemcpyAsync(L->d_Q0, Q, n5 * sizeof(double), cudaMemcpyDeviceToDevice, C.st));
  }
  if (k + 1 == C.lv.size()) {
    DG_TRY(smooth_level(C, L, Q, Sv, C.mg.beta_c));
    return DG_OK;
  }
  Level* Cc = C.lv[k + 1];
  DG_TRY(ensure_work(Cc));
  SmoothingRules R(C);
  // pre-smoothing: blocks of beta1 sweeps until max|r^P| < eta max|I r^P|
  for (int blk = 1;; ++blk) {
    DG_TRY(smooth_level(C, L, Q, Sv, C.mg.beta1, R.mask));
    if (R.on) DG_TRY(fill(R.dN, 0.0, R.ns, C.st));
    DG_TRY(residual(C.m, L, Q, Sv, L->d_R, false, C.st, R.on ? R.dN : nullptr, -1, nullptr, nullptr));
    C.evals++;
    C.dofs += 5.0 * L->nodes;
    DG_TRY(transfer(C.m, L, Cc, 5, L->d_R, Cc->d_S, C.st));
    if (!R.on) break;
    DG_TRY(slot_maxabs(C.m, Cc, Cc->d_S, R.dP, C.st));
    bool all = false;
    DG_TRY(R.pre(blk, &all));
    if (all) break;
  }
  DG_TRY(transfer(C.m, L, Cc, 5, Q, Cc->d_Q, C.st));
  DG_TRY(vcycle_level(C, k + 1, nullptr, nullptr));
  DG_TRY(transfer(C.m, Cc, L, 5, Cc->d_Q, Q, C.st, Cc->d_Q0, true));
  // post-smoothing: blocks of beta2 sweeps until max|r| <= its value after the pre-smoothing
  R.restart();
  for (int blk = 1;; ++blk) {
    DG_TRY(smooth_level(C, L, Q, Sv, C.mg.beta2, R.mask));
    if (!R.on || blk >= C.mg.control) break;
    DG_TRY(fill(R.dN, 0.0, R.ns, C.st));
    DG_TRY(residual(C.m, L, Q, Sv, L->d_R, false, C.st, R.dN, -1, nullptr, nullptr));
    C.evals++;
    C.dofs += 5.0 * L->nodes;
    bool all = false;
    DG_TRY(R.post(&all));
    if (all) break;
  }
  return DG_OK;
}

// ---------------------------------------------------------------------------
// mixed precision: FP64 defect, FP32 tangent-linear correction cycle
// ---------------------------------------------------------------------------
// One mixed cycle is a defect correction.  The finest residual r = S - A(Q)
// is formed in FP64 (it is also the residual that defines convergence); a
// V-cycle with the levels, sweeps and transfers of Algorithm 1 then solves
// the linearised problem J(Q) d = r approximately, every operator evaluation
// in it being the Jacobian-vector product J(Q_l) d_l in FP32 tangent
// arithmetic, whose rounding error scales with |d| (no floor from the FP32
// evaluation of the full operator); Q += d.  On level l the linearisation
// point is the restriction of the finest state, Q_l = I Q, and the coarse
// right-hand side I (b - J d) is formed in FP64 -- the linear counterpart of
// the FAS source A_c(I Q) + I r, whose A_c(I Q) term cancels against the
// coarse operator's value at Q_l.  Near convergence the cycle contracts like
// the FAS cycle; far from it the linearisation error is O(|d|^2).
static int smooth_tangent(Cycle& C, Level* L, const double* base, double* d, const double* b, int sweeps,
                          const double* mask = nullptr) {
  // pseudo-time step of the linear problem from its linearisation point,
  // fixed during the block; slots whose mask is 0 get dt = 0 (held)
  double* dt = C.m->d_scalars;
  const double* hold = C.m->freeze ? C.m->d_scalars + 6 * C.m->nslots : nullptr;
  if (sweeps > 0) {  // a small conforming level: the whole block in one cooperative launch
    const int rc = smooth_tangent_fused(C.m, L, base, d, b, sweeps, mask, hold, dt, C.st);
    if (rc == DG_OK) {
      C.evals += 3 * sweeps;
      C.dofs += 15.0 * sweeps * L->nodes;
      return DG_OK;
    }
    if (rc != kNotFused) return rc;
  }
  if (sweeps > 0) DG_TRY(cfl_dt(C.m, L, base, dt, C.st));
  if (sweeps > 0 && mask) DG_TRY(mask_dt(C.m, dt, mask, C.st));
  if (sweeps > 0 && hold) DG_TRY(mask_dt(C.m, dt, hold, C.st));
  for (int k = 0; k < sweeps; ++k)
    for (int stage = 0; stage < 3; ++stage) {
      const int tfl = kTracesNext | ((k > 0 || stage > 0) ? kTracesCurrent : 0);
      DG_TRY(residual_tangent(C.m, L, base, d, b, nullptr, C.st, nullptr, stage, L->d_G, dt, tfl));
      C.evals++;
      C.dofs += 5.0 * L->nodes;
    }
  return DG_OK;
}

// The linear V-cycle on level k: J(base) d = b with d starting at 0.  With
// mg.control > 0 the smoothing rules of Sec. 3.1.2 read the linear residual
// b - J d, as the FAS rules read S - A(Q) (for a linear operator they are the
// same vectors).
static int tangent_level(Cycle& C, size_t k) {
  Level* L = C.lv[k];
  DG_TRY(ensure_work(L));
  const double* base = (k == 0) ? C.q_fine : L->d_Q0;
  double* d = L->d_Q;
  const double* b = L->d_S;
  DG_TRY(fill(d, 0.0, 5 * L->nodes, C.st));
  if (k + 1 == C.lv.size()) return smooth_tangent(C, L, base, d, b, C.mg.beta_c);
  Level* Cc = C.lv[k + 1];
  DG_TRY(ensure_work(Cc));
  SmoothingRules R(C);
  for (int blk = 1;; ++blk) {  // pre-smoothing
    DG_TRY(smooth_tangent(C, L, base, d, b, C.mg.beta1, R.mask));
    if (R.on) DG_TRY(fill(R.dN, 0.0, R.ns, C.st));
    DG_TRY(residual_tangent(C.m, L, base, d, b, L->d_R, C.st, R.on ? R.dN : nullptr, -1, nullptr, nullptr));
    C.evals++;
    C.dofs += 5.0 * L->nodes;
    DG_TRY(transfer(C.m, L, Cc, 5, L->d_R, Cc->d_S, C.st));  // coarse right-hand side I (b - J d), FP64
    if (!R.on) break;
    DG_TRY(slot_maxabs(C.m, Cc, Cc->d_S, R.dP, C.st));
    bool all = false;
    DG_TRY(R.pre(blk, &all));
    if (all) break;
  }
  DG_TRY(transfer(C.m, L, Cc, 5, base, Cc->d_Q0, C.st));  // coarse linearisation point I Q
  DG_TRY(tangent_level(C, k + 1));
  DG_TRY(transfer(C.m, Cc, L, 5, Cc->d_Q, d, C.st, nullptr, true));  // d += I d_c
  R.restart();
  for (int blk = 1;; ++blk) {  // post-smoothing
    DG_TRY(smooth_tangent(C, L, base, d, b, C.mg.beta2, R.mask));
    if (!R.on || blk >= C.mg.control) break;
    DG_TRY(fill(R.dN, 0.0, R.ns, C.st));
    DG_TRY(residual_tangent(C.m, L, base, d, b, L->d_R, C.st, R.dN, -1, nullptr, nullptr));
    C.evals++;
    C.dofs += 5.0 * L->nodes;
    bool all = false;
    DG_TRY(R.post(&all));
    if (all) break;
  }
  return DG_OK;
}

static int mixed_cycle(Cycle& C, double* Q, const double* Sv) {
  Level* L = C.lv[0];
  DG_TRY(ensure_work(L));
  DG_TRY(residual(C.m, L, Q, Sv, L->d_S, false, C.st, nullptr, -1, nullptr, nullptr));  // FP64 defect
  C.evals++;
  C.dofs += 5.0 * L->nodes;
  C.q_fine = Q;
  DG_TRY(tangent_level(C, 0));
  return axpby(Q, 1.0, L->d_Q, 1.0, 5 * L->nodes, C.st);  // Q += d
}

static std::vector<int32_t> capped(const std::vector<int32_t>& o, int dim, int level, int direction) {
  std::vector<int32_t> r = o;
  size_t K = o.size() / 3;
  for (size_t e = 0; e < K; ++e)
    for (int d = 0; d < dim; ++d)
      if (direction < 0 || direction == d) r[e * 3 + d] = std::min(r[e * 3 + d], level);
  return r;
}

// max |S - A(Q)| per solve slot into norms (host, nslots values); *out gets the max over slots
static int level_norms(dg_mesh* m, Level* L, const double* Q, const double* Sv, cudaStream_t st, double* norms,
                       double* out) {
  DG_TRY(ensure_work(L));
  double* dn = m->d_scalars + m->nslots;
  DG_TRY(fill(dn, 0.0, m->nslots, st));
  DG_TRY(residual(m, L, Q, Sv, L->d_R, false, st, dn, -1, nullptr, nullptr));
  std::vector<double> tmp(m->nslots);
  double* h = norms ? norms : tmp.data();
  DG_CUDA_TRY(cudaMemcpyAsync(h, dn, m->nslots * sizeof(double), cudaMemcpyDeviceToHost, st));
  DG_CUDA_TRY(cudaStreamSynchronize(st));
  DG_TRY(fused_sync_check(m, st));
  double mx = 0.0;
  for (int k = 0; k < m->nslots; ++k) mx = (h[k] != h[k]) ? h[k] : std::max(mx, h[k]);
  if (out) *out = mx;
  return DG_OK;
}

static int level_norm(dg_mesh* m, Level* L, const double* Q, const double* Sv, cudaStream_t st, double* out) {
  return level_norms(m, L, Q, Sv, st, nullptr, out);
}

static std::vector<int32_t> capped(const std::vector<int32_t>& o, int dim, int level, int direction);

// The levels of a cycle whose finest level has orders `top_orders`.
static int cycle_levels(dg_mesh* m, const std::vector<int32_t>& top_orders, const dg_mg_params& mg,
                        std::vector<Level*>* lv) {
  int top = 0;
  for (int e = 0; e < m->K; ++e)
    for (int d = 0; d < m->dim; ++d)
      if (mg.direction < 0 || mg.direction == d) top = std::max(top, (int)top_orders[e * 3 + d]);
  const int coarsest = std::min((int)mg.coarsest, top);
  const int dN = mg.delta_n > 0 ? mg.delta_n : 1;
  lv->clear();
  for (int l = top; l >= coarsest; l -= dN) {
    Level* L = get_level(m, capped(top_orders, m->dim, l, mg.direction));
    if (!L) return DG_ECUDA;
    DG_TRY(ensure_work(L));
    lv->push_back(L);
  }
  return DG_OK;
}

// One V-cycle on (Q, Sv) whose finest level has orders `top_orders`.  With
// mg.graph the launch sequence is captured once per (orders, Q, Sv,
// parameters) on a library stream and replayed on `st` afterwards.
static int run_vcycle(dg_mesh* m, const std::vector<int32_t>& top_orders, double* Q, const double* Sv,
                      const dg_mg_params& mg, cudaStream_t st, int* evals, double* dofs, int* nlev,
                      bool fas = false) {
  Cycle C{m, st, mg, {}, 0, 0.0};
  DG_TRY(cycle_levels(m, top_orders, mg, &C.lv));
  *nlev = (int)C.lv.size();
  for (Level* L : C.lv) DG_TRY(prepare_arith(m, L, st));  // never allocate inside a capture
  const bool mixed = m->arith == DG_ARITH_MIXED && !fas;  // fas: the FP64 FAS cycle on a mixed-form mesh
  if (!mg.graph || mg.control > 0) {  // controlled sweep counts are decided on the host
    DG_TRY(mixed ? mixed_cycle(C, Q, Sv) : vcycle_level(C, 0, Q, Sv));
    *evals = C.evals;
    *dofs = C.dofs;
    return DG_OK;
  }
  std::string key((const char*)top_orders.data(), top_orders.size() * sizeof(int32_t));
  const void* ptrs[2] = {Q, Sv};
  key.append((const char*)ptrs, sizeof(ptrs));
  key.append((const char*)&mg, sizeof(mg));
  key.push_back(m->freeze ? 'h' : '-');
  key.push_back(mixed ? 'm' : 'f');
  auto it = m->graphs.find(key);
  if (it == m->graphs.end()) {
    DG_TRY(prepare_capture());
    if (!m->cap_stream) DG_CUDA_TRY(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
    Cycle G{m, m->cap_stream, mg, C.lv, 0, 0.0};
    unsigned long long l0 = launches();
    std::unique_lock<std::mutex> lock(device_sync_mutex());  // no cudaFree elsewhere while capturing
    DG_CUDA_TRY(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = mixed ? mixed_cycle(G, Q, Sv) : vcycle_level(G, 0, Q, Sv);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(m->cap_stream, &graph);
    lock.unlock();
    if (rc != DG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) {
      set_error(std::string("V-cycle capture: ") + cudaGetErrorString(e));
      return DG_ECUDA;
    }
    dg_mesh::Graph gr;
    e = cudaGraphInstantiate(&gr.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_error(std::string("V-cycle graph instantiate: ") + cudaGetErrorString(e));
      return DG_ECUDA;
    }
    gr.evals = G.evals;
    gr.dofs = G.dofs;
    gr.launches = launches() - l0;
    add_launches(0ULL - gr.launches);  // captured, not launched
    it = m->graphs.emplace(key, gr).first;
  }
  DG_CUDA_TRY(cudaGraphLaunch(it->second.exec, st));
  add_launches(it->second.launches);
  *evals = it->second.evals;
  *dofs = it->second.dofs;
  return DG_OK;
}

// ---------------------------------------------------------------------------
// adaptation (host, deterministic)
// ---------------------------------------------------------------------------
struct DirFit {
  bool has_slope = false;
  double slope = 0.0, intercept = 0.0, last = 0.0;
  int P = 0;
  const double* t = nullptr;
  double at(int N) const {
    if (N < P) return t[N] >= 0.0 ? t[N] : 0.0;
    if (!has_slope) return last;
    return std::pow(10.0, intercept + slope * N);
  }
};

static DirFit fit_dir(const double* t, int P) {
  DirFit F;
  F.P = P;
  F.t = t;
  double xs[kTauSlots], ys[kTauSlots];
  int np = 0;
  for (int N = 1; N < P && N < kTauSlots; ++N)
    if (t[N] > 0.0) {
      xs[np] = (double)N;
      ys[np] = std::log10(t[N]);
      ++np;
    }
  if (np >= 2) {
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < np; ++k) sx += xs[k];
    for (int k = 0; k < np; ++k) sy += ys[k];
    double xm = sx / np, ym = sy / np;
    double sxx = 0.0, sxy = 0.0;
    for (int k = 0; k < np; ++k) sxx += (xs[k] - xm) * (xs[k] - xm);
    for (int k = 0; k < np; ++k) sxy += (xs[k] - xm) * (ys[k] - ym);
    double b = sxy / sxx;
    if (b < 0.0) {
      F.has_slope = true;
      F.slope = b;
      F.intercept = ym - b * xm;
    }
  }
  F.last = (P >= 2 && t[P - 1] >= 0.0) ? t[P - 1] : 0.0;
  return F;
}

static void select_element(const double* tab /* 3 x 16 */, const int32_t* P, const dg_adapt_params& ap, int dim,
                           int32_t* out) {
  int hi = ap.n_max;
  if (ap.cap > 0) hi = std::min(hi, (int)ap.cap);
  DirFit F[3];
  for (int i = 0; i < dim; ++i) F[i] = fit_dir(tab + i * kTauSlots, P[i]);
  // each direction's estimate over the candidate range, evaluated once
  double tab_at[3][kTauSlots + 1];  // (orders <= n_max < kTauSlots, checked by dg_adapt)
  const int top = std::max(hi, 1);
  for (int i = 0; i < dim; ++i)
    for (int N = 0; N <= top && N <= kTauSlots; ++N) tab_at[i][N] = F[i].at(N);
  // Candidates in lexicographic order (the last direction fastest); the
  // first one with the fewest degrees of freedom and, among those, the
  // smallest estimate wins, so a later candidate never wins a full tie.  The
  // estimate is summed over the directions in order (0 + t_0 + t_1 + t_2).
  auto search = [&](const int* lo, const int* up, int32_t* best) -> bool {
    for (int i = 0; i < dim; ++i)
      if (up[i] < lo[i]) return false;
    bool found = false;
    long bestdof = 0;
    double besttau = 0.0;
    auto consider = [&](double tv, long dof, int a, int b, int c) {
      if (!(tv < ap.tau_max)) return;
      if (found && !(dof < bestdof || (dof == bestdof && tv < besttau))) return;
      found = true;
      bestdof = dof;
      besttau = tv;
      best[0] = a;
      best[1] = b;
      best[2] = c;
    };
    if (dim == 1) {
      for (int a = lo[0]; a <= up[0]; ++a) consider(0.0 + tab_at[0][a], a + 1, a, 0, 0);
    } else if (dim == 2) {
      for (int a = lo[0]; a <= up[0]; ++a) {
        const double ta = 0.0 + tab_at[0][a];
        for (int b = lo[1]; b <= up[1]; ++b) consider(ta + tab_at[1][b], (long)(a + 1) * (b + 1), a, b, 0);
      }
    } else {
      for (int a = lo[0]; a <= up[0]; ++a) {
        const double ta = 0.0 + tab_at[0][a];
        for (int b = lo[1]; b <= up[1]; ++b) {
          const double tb = ta + tab_at[1][b];
          for (int c = lo[2]; c <= up[2]; ++c)
            consider(tb + tab_at[2][c], (long)(a + 1) * (b + 1) * (c + 1), a, b, c);
        }
      }
    }
    return found;
  };
  int lo[3], up[3];
  int32_t best[3] = {0, 0, 0};
  bool ok = false;
  bool inner_ok = true;
  for (int i = 0; i < dim; ++i) {
    lo[i] = ap.n_min;
    up[i] = std::min(P[i] - 1, hi);
    if (up[i] < lo[i]) inner_ok = false;
  }
  if (inner_ok) ok = search(lo, up, best);
  if (!ok) {
    for (int i = 0; i < dim; ++i) up[i] = hi;
    ok = search(lo, up, best);
  }
  if (!ok)
    for (int i = 0; i < dim; ++i) best[i] = hi;
  for (int i = 0; i < 3; ++i) out[i] = (i < dim) ? best[i] : 0;
}

static void face_map(int fA, int fB, int o, int* m) {
  int dA = fA / 2, dB = fB / 2;
  int tA[2], tB[2], k = 0;
  for (int t = 0; t < 3; ++t)
    if (t != dA) tA[k++] = t;
  k = 0;
  for (int t = 0; t < 3; ++t)
    if (t != dB) tB[k++] = t;
  m[dA] = dB;
  if (o & 1) {
    m[tA[0]] = tB[1];
    m[tA[1]] = tB[0];
  } else {
    m[tA[0]] = tB[0];
    m[tA[1]] = tB[1];
  }
}

// Jacobi sweeps of the order-jump rules until nothing changes.  The rules only
// raise orders and never above the largest order of the map, so the sweeps
// settle within K x max order of them; the cap only guards that argument.
static int limit_jumps(const dg_mesh* m, std::vector<int32_t>& o, int rule, int conform_tag) {
  const int dim = m->dim, K = m->K;
  std::vector<char> touches(K, 0);
  if (conform_tag >= 0)
    for (int e = 0; e < K; ++e)
      for (int f = 0; f < 2 * dim; ++f) {
        const int32_t* ft = &m->ftab[(size_t)(e * 6 + f) * 4];
        if (ft[0] < 0 && ft[3] == conform_tag) touches[e] = 1;
      }
  // each interior face once: the neighbour and, per direction, the
  // neighbour's direction it faces (fixed across the sweeps)
  struct Link {
    int e, nb, mp[3];
    bool conform;
  };
  std::vector<Link> links;
  links.reserve((size_t)K * 2 * dim);
  for (int e = 0; e < K; ++e)
    for (int f = 0; f < 2 * dim; ++f) {
      const int32_t* ft = &m->ftab[(size_t)(e * 6 + f) * 4];
      if (ft[0] < 0) continue;
      Link l;
      l.e = e;
      l.nb = ft[0];
      face_map(f, ft[1], ft[2], l.mp);
      l.conform = conform_tag >= 0 && touches[e] && touches[ft[0]];
      links.push_back(l);
    }
  std::vector<int32_t> nw(o.size());
  for (int it = 0; it < 100000; ++it) {
    nw = o;
    for (const Link& l : links)
      for (int i = 0; i < dim; ++i) {
        const int other = o[l.nb * 3 + l.mp[i]];
        int need = (rule == 1) ? other - 1 : (rule == 2 ? (2 * other) / 3 : 0);
        if (l.conform) need = std::max(need, other);
        if (need > nw[l.e * 3 + i]) nw[l.e * 3 + i] = need;
      }
    if (nw == o) return DG_OK;
    o.swap(nw);
  }
  set_error("dg_adapt: the order-jump fix-point did not settle within 100000 sweeps");
  return DG_ENOTCONVERGED;
}

}  // namespace dg

using namespace dg;

// A C++ exception never leaves the C ABI: a host allocation failure comes back
// as DG_ENOMEM, anything else as DG_EINVAL with its message.
template <class F>
static int guarded(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    set_error("out of host memory");
    return DG_ENOMEM;
  } catch (const std::exception& e) {
    set_error(std::string("internal error: ") + e.what());
    return DG_EINVAL;
  }
}

extern "C" {

const char* dg_last_error(void) { return g_err.c_str(); }

int dg_kernel_launches(int64_t* count) {
  return guarded([&]() -> int {
    if (!count) {
      set_error("dg_kernel_launches: null argument");
      return DG_EINVAL;
    }
    *count = (int64_t)launches_total();
    return DG_OK;
  });
}

int dg_mesh_create(const dg_mesh_desc* desc, const int32_t* orders, dg_mesh** out) {
  return guarded([&]() -> int {
    if (!out) {
      set_error("null output");
      return DG_EINVAL;
    }
    DG_TRY(check_desc(desc, orders));
    DG_TRY(upload_tables());
    dg_mesh* m = new (std::nothrow) dg_mesh();
    if (!m) return DG_ENOMEM;
    m->dim = desc->dim;
    m->K = desc->K;
    m->M = desc->M;
    int Mp = desc->M + 1;
    size_t npe = desc->dim == 3 ? (size_t)Mp * Mp * Mp : (size_t)Mp * Mp;
    m->xmap.assign(desc->xmap, desc->xmap + (size_t)desc->K * npe * 3);
    m->ftab.assign(desc->ftab, desc->ftab + (size_t)desc->K * 24);
    m->prm = make_params(desc->params);
    std::memcpy(m->raw_params, desc->params, sizeof(m->raw_params));
    m->nslots = 1;
    m->slot_prm.assign(1, m->prm);
    m->slot_raw.assign(1, std::vector<double>(desc->params, desc->params + 16));
    m->elem_slot.assign(desc->K, 0);
    m->slot_elem_off = {0, desc->K};
    m->orders.assign(orders, orders + (size_t)desc->K * 3);
    m->fine.reset(new Level());
    int rc = build_level(m, m->orders, m->fine.get());
    if (rc == DG_OK) rc = upload_gas(m);
    if (rc == DG_OK) {
      cudaError_t e1 = cudaMalloc(&m->d_scalars, (7 * m->nslots + 16) * sizeof(double));
      if (e1 == cudaSuccess) e1 = cudaMemset(m->d_scalars, 0, (7 * m->nslots + 16) * sizeof(double));
      cudaError_t e2 = cudaMalloc(&m->d_tau, (size_t)m->K * 3 * kTauSlots * sizeof(double));
      cudaError_t e3 = cudaMalloc(&m->d_orders, m->orders.size() * sizeof(int32_t));
      if (e3 == cudaSuccess)
        e3 = cudaMemcpy(m->d_orders, m->orders.data(), m->orders.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        set_error("cudaMalloc failed for mesh scalars");
        rc = DG_ECUDA;
      }
    }
    if (rc != DG_OK) {
      dg_mesh_destroy(m);
      return rc;
    }
    *out = m;
    return DG_OK;
  });
}

int dg_batch_create(const dg_mesh_desc* descs, const int32_t* const* orders, int32_t nsolves, dg_mesh** out) {
  return guarded([&]() -> int {
    if (!descs || !orders || !out || nsolves < 1) {
      set_error("dg_batch_create: bad argument");
      return DG_EINVAL;
    }
    for (int k = 0; k < nsolves; ++k) {
      DG_TRY(check_desc(&descs[k], orders[k]));
      if (descs[k].dim != descs[0].dim || descs[k].M != descs[0].M) {
        set_error("dg_batch_create: all solves need the same dim and mapping order");
        return DG_EINVAL;
      }
    }
    DG_TRY(upload_tables());
    dg_mesh* m = new (std::nothrow) dg_mesh();
    if (!m) return DG_ENOMEM;
    const int dim = descs[0].dim, Mp = descs[0].M + 1;
    const size_t npe = dim == 3 ? (size_t)Mp * Mp * Mp : (size_t)Mp * Mp;
    m->dim = dim;
    m->M = descs[0].M;
    m->nslots = nsolves;
    m->slot_elem_off.assign(1, 0);
    for (int k = 0; k < nsolves; ++k) {
      const dg_mesh_desc& d = descs[k];
      const int e0 = m->K;
      m->xmap.insert(m->xmap.end(), d.xmap, d.xmap + (size_t)d.K * npe * 3);
      for (int i = 0; i < d.K * 24; ++i) {
        int32_t v = d.ftab[i];
        if (i % 4 == 0 && v >= 0) v += e0;  // neighbour index into the batch
        m->ftab.push_back(v);
      }
      m->orders.insert(m->orders.end(), orders[k], orders[k] + (size_t)d.K * 3);
      m->elem_slot.insert(m->elem_slot.end(), d.K, k);
      m->slot_prm.push_back(make_params(d.params));
      m->slot_raw.push_back(std::vector<double>(d.params, d.params + 16));
      m->K += d.K;
      m->slot_elem_off.push_back(m->K);
    }
    m->prm = m->slot_prm[0];
    std::memcpy(m->raw_params, descs[0].params, sizeof(m->raw_params));
    m->fine.reset(new Level());
    int rc = build_level(m, m->orders, m->fine.get());
    if (rc == DG_OK) rc = upload_gas(m);
    if (rc == DG_OK) {
      cudaError_t e1 = cudaMalloc(&m->d_scalars, (7 * m->nslots + 16) * sizeof(double));
      if (e1 == cudaSuccess) e1 = cudaMemset(m->d_scalars, 0, (7 * m->nslots + 16) * sizeof(double));
      cudaError_t e2 = cudaMalloc(&m->d_tau, (size_t)m->K * 3 * kTauSlots * sizeof(double));
      cudaError_t e3 = cudaMalloc(&m->d_orders, m->orders.size() * sizeof(int32_t));
      if (e3 == cudaSuccess)
        e3 = cudaMemcpy(m->d_orders, m->orders.data(), m->orders.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        set_error("cudaMalloc failed for batch scalars");
        rc = DG_ECUDA;
      }
    }
    if (rc != DG_OK) {
      dg_mesh_destroy(m);
      return rc;
    }
    *out = m;
    return DG_OK;
  });
}

int dg_batch_set_active(dg_mesh* m, const int32_t* active, void* stream) {
  return guarded([&]() -> int {
    if (!m || !active) {
      set_error("dg_batch_set_active: null argument");
      return DG_EINVAL;
    }
    const int ns = m->nslots;
    std::vector<double> h(ns);
    m->active.assign(active, active + ns);
    for (int k = 0; k < ns; ++k) h[k] = active[k] ? 1.0 : 0.0;
    cudaStream_t st = S(stream);
    DG_CUDA_TRY(cudaMemcpyAsync(m->d_scalars + 6 * ns, h.data(), ns * sizeof(double), cudaMemcpyHostToDevice, st));
    DG_CUDA_TRY(cudaStreamSynchronize(st));  // h is a local buffer
    m->freeze = true;  // (held from now on; cached graphs were captured without the mask)
    return DG_OK;
  });
}

int dg_batch_info(const dg_mesh* m, int32_t* nsolves, int64_t* offs) {
  return guarded([&]() -> int {
    if (!m) {
      set_error("dg_batch_info: null mesh");
      return DG_EINVAL;
    }
    if (nsolves) *nsolves = m->nslots;
    if (offs)
      for (int k = 0; k <= m->nslots; ++k) offs[k] = m->fine->off[m->slot_elem_off[k]];
    return DG_OK;
  });
}

int dg_residual_norms(dg_mesh* m, const double* q, const double* s, double* norms, void* stream) {
  return guarded([&]() -> int {
    if (!m || !q || !norms) {
      set_error("dg_residual_norms: null argument");
      return DG_EINVAL;
    }
    double mx = 0.0;
    return level_norms(m, m->fine.get(), q, s, S(stream), norms, &mx);
  });
}

int dg_mesh_destroy(dg_mesh* m) {
  return guarded([&]() -> int {
    if (!m) return DG_OK;
    {
      std::lock_guard<std::mutex> lock(device_sync_mutex());
      for (auto& kv : m->graphs) cudaGraphExecDestroy(kv.second.exec);
      if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
      for (cudaStream_t t : m->tau_st)
        if (t) cudaStreamDestroy(t);
      if (m->d_scalars) cudaFree(m->d_scalars);
      if (m->d_tau) cudaFree(m->d_tau);
      if (m->d_orders) cudaFree(m->d_orders);
      if (m->d_gas64) cudaFree(m->d_gas64);
      if (m->d_gas32x2) cudaFree(m->d_gas32x2);
      if (m->d_gastf) cudaFree(m->d_gastf);
      if (m->d_gasd) cudaFree(m->d_gasd);
    }
    delete m;  // the levels lock again while they free
    return DG_OK;
  });
}

int dg_set_autotune(dg_mesh* m, int on, void* stream) {
  return guarded([&]() -> int {
    if (!m) {
      set_error("dg_set_autotune: null mesh");
      return DG_EINVAL;
    }
    m->autotune = on != 0;
    if (!m->autotune) return DG_OK;
    {
      std::lock_guard<std::mutex> lock(device_sync_mutex());
      for (auto& kv : m->graphs) cudaGraphExecDestroy(kv.second.exec);  // they hold the old tile lists
    }
    m->graphs.clear();
    cudaStream_t st = S(stream);
    DG_TRY(tune_level(m, m->fine.get(), st));
    for (auto& kv : m->levels) DG_TRY(tune_level(m, kv.second.get(), st));
    return DG_OK;
  });
}

int dg_mesh_tuning(const dg_mesh* m, int32_t* out) {
  return guarded([&]() -> int {
    if (!m || !out) {
      set_error("dg_mesh_tuning: bad argument");
      return DG_EINVAL;
    }
    out[0] = m->fine->pack;
    for (int c = 0; c < kTileClasses; ++c) out[1 + c] = m->fine->class_threads[c];
    return DG_OK;
  });
}

int dg_mesh_layout(const dg_mesh* m, int64_t* total_nodes, int64_t* elem_offsets) {
  return guarded([&]() -> int {
    if (!m) {
      set_error("null mesh");
      return DG_EINVAL;
    }
    if (total_nodes) *total_nodes = m->fine->nodes;
    if (elem_offsets)
      for (int e = 0; e <= m->K; ++e) elem_offsets[e] = m->fine->off[e];
    return DG_OK;
  });
}

int dg_set_arithmetic(dg_mesh* m, int mode) {
  return guarded([&]() -> int {
    if (!m || (mode != DG_ARITH_FP64 && mode != DG_ARITH_DF32 && mode != DG_ARITH_MIXED)) {
      set_error("dg_set_arithmetic: bad argument");
      return DG_EINVAL;
    }
    if (m->arith != mode) {
      for (auto& kv : m->graphs) cudaGraphExecDestroy(kv.second.exec);
      m->graphs.clear();
    }
    m->arith = mode;
    return DG_OK;
  });
}

int dg_mesh_orders(const dg_mesh* m, int32_t* out) {
  return guarded([&]() -> int {
    if (!m || !out) {
      set_error("dg_mesh_orders: null argument");
      return DG_EINVAL;
    }
    std::memcpy(out, m->orders.data(), m->orders.size() * sizeof(int32_t));
    return DG_OK;
  });
}

int dg_residual(dg_mesh* m, const double* q, const double* s, double* r, int flags, double* rnorm_host,
                void* stream) {
  return guarded([&]() -> int {
    if (!m || !q || !r || q == r) {
      set_error("dg_residual: null or aliased arrays");
      return DG_EINVAL;
    }
    if ((flags & DG_NORM) && !rnorm_host) {
      set_error("dg_residual: DG_NORM needs rnorm_host");
      return DG_EINVAL;
    }
    cudaStream_t st = S(stream);
    bool iso = flags & DG_ISOLATED;
    double* dnorm = nullptr;
    if (flags & DG_NORM) {
      dnorm = m->d_scalars + m->nslots;
      DG_TRY(fill(dnorm, 0.0, m->nslots, st));
    }
    DG_TRY(residual(m, m->fine.get(), q, s, r, iso, st, iso ? nullptr : dnorm, -1, nullptr, nullptr));
    if (flags & DG_NORM) {
      if (iso) {
        // norm of the isolated residual: reduce it with the tau reduction over one slot
        set_error("DG_NORM with DG_ISOLATED is not supported");
        return DG_EINVAL;
      }
      std::vector<double> h(m->nslots);
      DG_CUDA_TRY(cudaMemcpyAsync(h.data(), dnorm, m->nslots * sizeof(double), cudaMemcpyDeviceToHost, st));
      DG_CUDA_TRY(cudaStreamSynchronize(st));
      DG_TRY(fused_sync_check(m, st));  // a fused smoothing block that failed voids the state
      double mx = 0.0;
      for (double v : h) mx = (v != v) ? v : std::max(mx, v);
      *rnorm_host = mx;
    }
    return DG_OK;
  });
}

int dg_residual_tangent(dg_mesh* m, const double* q, const double* dq, const double* b, double* r, void* stream) {
  return guarded([&]() -> int {
    if (!m || !q || !dq || !r || r == q || r == dq) {
      set_error("dg_residual_tangent: null or aliased arrays");
      return DG_EINVAL;
    }
    return residual_tangent(m, m->fine.get(), q, dq, b, r, S(stream), nullptr, -1, nullptr, nullptr);
  });
}

int dg_cfl_dt(dg_mesh* m, const double* q, double* dt, void* stream) {
  return guarded([&]() -> int {
    if (!m || !q || !dt) {
      set_error("dg_cfl_dt: null argument");
      return DG_EINVAL;
    }
    cudaStream_t st = S(stream);
    DG_TRY(cfl_dt(m, m->fine.get(), q, m->d_scalars, st));
    return read_scalar(m->d_scalars, dt, st);
  });
}

int dg_smooth(dg_mesh* m, double* q, const double* s, int sweeps, void* stream) {
  return guarded([&]() -> int {
    if (!m || !q || sweeps < 0) {
      set_error("dg_smooth: bad argument");
      return DG_EINVAL;
    }
    Cycle C{m, S(stream), dg_mg_params{}, {}, 0, 0.0};
    return smooth_level(C, m->fine.get(), q, s, sweeps);
  });
}

int dg_pmg_vcycle(dg_mesh* m, double* q, const double* s, const dg_mg_params* mg, int want_norm,
                  dg_cycle_report* rep, void* stream) {
  return guarded([&]() -> int {
    if (!m || !q || !mg || mg->beta1 < 0 || mg->beta2 < 0 || mg->beta_c < 0 || mg->coarsest < 1 ||
        mg->direction < -1 || mg->direction >= m->dim || mg->control < 0 ||
        (mg->control > 0 && (mg->beta1 < 1 || mg->beta2 < 1))) {
      set_error("dg_pmg_vcycle: bad argument");
      return DG_EINVAL;
    }
    cudaStream_t st = S(stream);
    int evals = 0;
    double dofs = 0.0;
    int nlev = 0;
    DG_TRY(run_vcycle(m, m->orders, q, s, *mg, st, &evals, &dofs, &nlev));
    double rn = 0.0;
    if (want_norm) DG_TRY(level_norm(m, m->fine.get(), q, s, st, &rn));
    if (rep) {
      rep->levels = nlev;
      rep->residual_evals = evals;
      rep->dof_evals = dofs;
      rep->rnorm = rn;
    }
    return DG_OK;
  });
}

int dg_tau_estimate(dg_mesh* m, const double* q, const double* s, int dir_mask, int with_correction, int isolated,
                    double* tau_host, void* stream) {
  return guarded([&]() -> int {
    if (!m || !q || !tau_host) {
      set_error("dg_tau_estimate: null argument");
      return DG_EINVAL;
    }
    cudaStream_t st = S(stream);
    Level* F = m->fine.get();
    DG_TRY(ensure_work(F));
    const size_t tsz = (size_t)m->K * 3 * kTauSlots;
    DG_TRY(fill(m->d_tau, 0.0, (int64_t)tsz, st));
    // R^P(q) at the reference orders
    if (with_correction) DG_TRY(residual(m, F, q, s, F->d_R, isolated != 0, st, nullptr, -1, nullptr, nullptr));
    const int32_t* d_fine_orders = m->d_orders;
    // The directions are independent (their levels, buffers and table slots
    // differ): each runs on its own stream, forked from and joined back to st.
    cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
    DG_CUDA_TRY(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    DG_CUDA_TRY(cudaEventRecord(ev_fork, st));
    int rc = DG_OK;
    for (int i = 0; i < m->dim && rc == DG_OK; ++i) {
      if (!((dir_mask >> i) & 1)) continue;
      if (!m->tau_st[i] && cudaStreamCreateWithFlags(&m->tau_st[i], cudaStreamNonBlocking) != cudaSuccess) {
        rc = DG_ECUDA;
        break;
      }
      cudaStream_t sti = m->tau_st[i];
      if (cudaStreamWaitEvent(sti, ev_fork, 0) != cudaSuccess) {
        rc = DG_ECUDA;
        break;
      }
      int top = 0;
      for (int e = 0; e < m->K; ++e) top = std::max(top, (int)m->orders[e * 3 + i]);
      Level* prev = F;
      const double* Qp = q;
      const double* Sp = s;
      const double* Rp = with_correction ? F->d_R : nullptr;
      for (int l = top - 1; l >= 1 && rc == DG_OK; --l) {
        Level* Ll = get_level(m, capped(m->orders, m->dim, l, i));
        if (!Ll) {
          rc = DG_ECUDA;
          break;
        }
        if ((rc = ensure_work(Ll)) != DG_OK) break;
        if ((rc = transfer(m, prev, Ll, 5, Qp, Ll->d_Q, sti)) != DG_OK) break;
        if (s && (rc = transfer(m, prev, Ll, 5, Sp, Ll->d_S, sti)) != DG_OK) break;
        if (Rp && (rc = transfer(m, prev, Ll, 5, Rp, Ll->d_G, sti)) != DG_OK) break;
        rc = tau_accumulate(m, Ll, Ll->d_Q, s ? Ll->d_S : nullptr, Rp ? Ll->d_G : nullptr, isolated != 0, i, l,
                            d_fine_orders, m->d_tau, sti);
        prev = Ll;
        Qp = Ll->d_Q;
        Sp = Ll->d_S;
        Rp = Rp ? Ll->d_G : nullptr;
      }
      if (cudaEventCreateWithFlags(&ev_join[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(ev_join[i], sti) != cudaSuccess || cudaStreamWaitEvent(st, ev_join[i], 0) != cudaSuccess)
        rc = DG_ECUDA;
    }
    cudaEventDestroy(ev_fork);
    for (cudaEvent_t e : ev_join)
      if (e) cudaEventDestroy(e);
    if (rc == DG_OK) {
      cudaError_t e = cudaMemcpyAsync(tau_host, m->d_tau, tsz * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        set_error(std::string("tau copy: ") + cudaGetErrorString(e));
        rc = DG_ECUDA;
      }
    }
    if (rc != DG_OK) return rc;
    for (int e = 0; e < m->K; ++e)
      for (int i = 0; i < 3; ++i)
        for (int N = 0; N < kTauSlots; ++N) {
          bool measured = i < m->dim && ((dir_mask >> i) & 1) && N >= 1 && N < m->orders[e * 3 + i];
          if (!measured) tau_host[((size_t)e * 3 + i) * kTauSlots + N] = -1.0;
        }
    return DG_OK;
  });
}

int dg_adapt(const dg_mesh* m, const double* tau_host, const dg_adapt_params* ap, int32_t* new_orders) {
  return guarded([&]() -> int {
    if (!m || !tau_host || !ap || !new_orders || ap->n_min < 1 || ap->n_max > kNMax || ap->n_min > ap->n_max ||
        ap->n_max >= kTauSlots) {
      set_error("dg_adapt: bad argument");
      return DG_EINVAL;
    }
    std::vector<int32_t> o((size_t)m->K * 3, 0);
    // (on the calling thread: at a few hundred ns an element, starting host
    // threads costs more than it saves for meshes of a few thousand elements)
    for (int e = 0; e < m->K; ++e)
      select_element(tau_host + (size_t)e * 3 * kTauSlots, &m->orders[e * 3], *ap, m->dim, &o[e * 3]);
    if (ap->jump_rule == 1 || ap->jump_rule == 2 || ap->conform_tag >= 0)
      DG_TRY(limit_jumps(m, o, ap->jump_rule, ap->conform_tag));
    std::memcpy(new_orders, o.data(), o.size() * sizeof(int32_t));
    return DG_OK;
  });
}

int dg_profile_residual(dg_mesh* m, const double* q, const double* s, double* r, int iters, double* ms_out,
                        void* stream) {
  return guarded([&]() -> int {
    if (!m || !q || !r || !ms_out || iters < 1 || q == r) {
      set_error("dg_profile_residual: bad argument");
      return DG_EINVAL;
    }
    return profile_residual(m, m->fine.get(), q, s, r, iters, ms_out, S(stream));
  });
}

// Cycle (Q, Sv) with top orders `o` until max|r| < target or `cap` cycles;
// *cycles counts them.  Returns DG_OK, DG_ENOTCONVERGED or DG_EDIVERGED.
// V-cycles until max|r| < target (checked every `every` cycles).  On a
// mixed-form mesh with mixed_from > 0, cycles whose last checked residual is
// at least mixed_from run the FP64 FAS cycle instead of the defect
// correction, whose linearisation holds only near a solution.
static int cycle_until(dg_mesh* m, const std::vector<int32_t>& o, Level* L, double* Q, const double* Sv,
                       const dg_mg_params& mg, double target, int cap, cudaStream_t st, int* cycles, double* dofs,
                       double* rn, int every = 1, double mixed_from = 0.0) {
  DG_TRY(level_norm(m, L, Q, Sv, st, rn));
  dofs[0] += 5.0 * L->nodes;
  every = std::max(1, every);
  for (int c = 0; c < cap;) {
    if (!(*rn < target)) {
      if (std::isnan(*rn) || std::isinf(*rn)) return DG_EDIVERGED;
    } else {
      return DG_OK;
    }
    const bool fas = m->arith == DG_ARITH_MIXED && mixed_from > 0.0 && !(*rn < mixed_from);
    for (int k = 0; k < every && c < cap; ++k, ++c) {
      int ev = 0, nl = 0;
      double dd = 0.0;
      DG_TRY(run_vcycle(m, o, Q, Sv, mg, st, &ev, &dd, &nl, fas));
      dofs[0] += dd;
      (*cycles)++;
    }
    DG_TRY(level_norm(m, L, Q, Sv, st, rn));
    dofs[0] += 5.0 * L->nodes;
  }
  if (std::isnan(*rn) || std::isinf(*rn)) return DG_EDIVERGED;
  return (*rn < target) ? DG_OK : DG_ENOTCONVERGED;
}

int dg_solve_steady(dg_mesh** meshp, double** qp, const double* s, const dg_solve_params* sp, dg_alloc_fn alloc,
                    void* alloc_ctx, dg_solve_report* rep, void* stream) {
  return guarded([&]() -> int {
    if (!meshp || !*meshp || !qp || !*qp || !sp || !rep || sp->max_cycles < 0 || !(sp->tol > 0.0) ||
        (sp->adapt && (!alloc || s)) || (sp->fmg && !(sp->fmg_tol > 0.0))) {
      set_error("dg_solve_steady: bad argument (adaptation needs alloc and s == NULL)");
      return DG_EINVAL;
    }
    std::memset(rep, 0, sizeof(*rep));
    dg_mesh* m = *meshp;
    if (sp->adapt && m->nslots > 1) {
      set_error("dg_solve_steady: adaptation of a batch is not supported (adapt each solve)");
      return DG_EINVAL;
    }
    double* q = *qp;
    cudaStream_t st = S(stream);
    dg_mg_params mg = sp->mg;
    int rc = DG_OK;
    double rn = 0.0;
    // ---- full multigrid ramp (Sec. 3.1.1) ----
    if (sp->fmg) {
      int top = 0;
      for (int e = 0; e < m->K; ++e)
        for (int d = 0; d < m->dim; ++d) top = std::max(top, (int)m->orders[e * 3 + d]);
      Level* prev = nullptr;
      for (int l = 1; l < top; ++l) {
        std::vector<int32_t> o = capped(m->orders, m->dim, l, -1);
        Level* L = get_level(m, o);
        if (!L) return DG_ECUDA;
        DG_TRY(ensure_work(L));
        if (!prev)
          DG_TRY(transfer(m, m->fine.get(), L, 5, q, L->d_Q, st));  // initial state, L2-projected down
        else
          DG_TRY(transfer(m, prev, L, 5, prev->d_Q, L->d_Q, st));   // interpolated up
        if (s) DG_TRY(transfer(m, m->fine.get(), L, 5, s, L->d_S, st));
        int cyc = 0;
        rc = cycle_until(m, o, L, L->d_Q, s ? L->d_S : nullptr, mg, sp->fmg_tol, sp->max_cycles, st, &cyc,
                         &rep->dof_evals, &rn, sp->check_every, sp->mixed_from);
        rep->cycles += cyc;
        rep->fmg_cycles += cyc;
        if (rc == DG_EDIVERGED) break;
        rc = DG_OK;  // a FMG level that stalls still hands its state up
        prev = L;
      }
      if (rc == DG_OK && prev) DG_TRY(transfer(m, prev, m->fine.get(), 5, prev->d_Q, q, st));
    }
    // ---- reference orders ----
    if (rc == DG_OK) {
      const double ref = sp->ref_factor > 0.0 ? sp->ref_factor : 0.1;
      double target = sp->adapt ? sp->ap.tau_max * ref : sp->tol;
      int cyc = 0;
      rc = cycle_until(m, m->orders, m->fine.get(), q, s, mg, target, sp->max_cycles, st, &cyc, &rep->dof_evals, &rn, sp->check_every, sp->mixed_from);
      rep->cycles += cyc;
    }
    // ---- adaptation (Sec. 3.3.2), possibly in stages (Sec. 3.3.4) ----
    if (rc == DG_OK && sp->adapt) {
      const int nst = std::max(1, (int)sp->n_stages);
      for (int stage = 0; stage < nst && rc == DG_OK; ++stage) {
        if (stage > 0) {  // every stage starts from a state converged to tau_max/10
          int cyc = 0;
          const double ref = sp->ref_factor > 0.0 ? sp->ref_factor : 0.1;
          rc = cycle_until(m, m->orders, m->fine.get(), q, nullptr, mg, sp->ap.tau_max * ref, sp->max_cycles, st,
                           &cyc, &rep->dof_evals, &rn, sp->check_every, sp->mixed_from);
          rep->cycles += cyc;
          if (rc != DG_OK) break;
        }
        rep->rnorm_adapt = rn;
        std::vector<double> tau((size_t)m->K * 3 * kTauSlots);
        DG_TRY(dg_tau_estimate(m, q, nullptr, (1 << m->dim) - 1, 1, 1, tau.data(), stream));
        dg_adapt_params ap = sp->ap;
        bool last = true;
        if (sp->n_stages > 0) {
          ap.cap = sp->stage_orders[stage];
          dg_adapt_params un = sp->ap;
          un.cap = 0;
          std::vector<int32_t> free_orders(m->orders.size());
          DG_TRY(dg_adapt(m, tau.data(), &un, free_orders.data()));
          int need = 0;
          for (int32_t v : free_orders) need = std::max(need, (int)v);
          last = (stage == nst - 1) || need <= ap.cap;
        }
        std::vector<int32_t> no(m->orders.size());
        DG_TRY(dg_adapt(m, tau.data(), &ap, no.data()));
        if (no != m->orders) {
          dg_mesh_desc d;
          d.dim = m->dim;
          d.K = m->K;
          d.M = m->M;
          d.xmap = m->xmap.data();
          d.ftab = m->ftab.data();
          std::memcpy(d.params, m->raw_params, sizeof(d.params));
          dg_mesh* nm = nullptr;
          DG_TRY(dg_mesh_create(&d, no.data(), &nm));
          nm->arith = m->arith;
          double* nq = (double*)alloc((size_t)5 * nm->fine->nodes * sizeof(double), alloc_ctx);
          if (!nq) {
            dg_mesh_destroy(nm);
            set_error("dg_solve_steady: allocator returned NULL");
            return DG_ENOMEM;
          }
          rc = transfer(m, m->fine.get(), nm->fine.get(), 5, q, nq, st);
          if (rc != DG_OK) {
            dg_mesh_destroy(nm);
            return rc;
          }
          DG_CUDA_TRY(cudaStreamSynchronize(st));
          dg_mesh_destroy(m);
          m = nm;
          q = nq;
          *meshp = m;
          *qp = q;
          rep->adapted += 1;
        }
        if (last) break;
      }
      if (rc == DG_OK) {
        int cyc = 0;
        rc = cycle_until(m, m->orders, m->fine.get(), q, nullptr, mg, sp->tol, sp->max_cycles, st, &cyc,
                         &rep->dof_evals, &rn, sp->check_every, sp->mixed_from);
        rep->cycles += cyc;
      }
    }
    rep->rnorm = rn;
    rep->status = rc;
    rep->nodes = m->fine->nodes;
    if (rc != DG_OK) set_error(rc == DG_EDIVERGED ? "dg_solve_steady: residual diverged"
                                                  : "dg_solve_steady: cycle cap reached before the tolerance");
    return rc;
  });
}

int dg_measure_fma_rates(double* fp64_tflops, double* fp32_tflops, void* stream) {
  return guarded([&]() -> int {
    if (!fp64_tflops || !fp32_tflops) {
      set_error("dg_measure_fma_rates: null argument");
      return DG_EINVAL;
    }
    return measure_fma_rates(fp64_tflops, fp32_tflops, S(stream));
  });
}

int dg_transfer_noalloc(int32_t dim, int32_t K, const int32_t* orders_from, const int32_t* orders_to,
                        int32_t nvar, const double* in, double* out, void* stream) {
  return guarded([&]() -> int {
    return transfer_noalloc(dim, K, orders_from, orders_to, nvar, in, out, S(stream));
  });
}

int dg_transfer_state(const dg_mesh* from, const double* q_from, const dg_mesh* to, double* q_to, void* stream) {
  return guarded([&]() -> int {
    if (!from || !to || !q_from || !q_to || from->K != to->K || from->dim != to->dim) {
      set_error("dg_transfer_state: meshes do not match");
      return DG_EINVAL;
    }
    return transfer(from, from->fine.get(), to->fine.get(), 5, q_from, q_to, S(stream));
  });
}

}  // extern "C"
