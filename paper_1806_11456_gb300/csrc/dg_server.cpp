// Serving loop: steady solves admitted as they arrive.
//
// Each slot is a host worker thread with its own CUDA stream.  A request
// waits in a FIFO queue until a slot is free and its device-memory estimate
// fits in what the running solves leave of the budget; the worker then builds
// the request's mesh (its multigrid hierarchy stays resident while it runs),
// uploads the state and source, runs the steady driver (Sec. 3.1 cycling,
// Sec. 3.3.2 adaptation) on its stream, and copies the result back.  The
// kernels of concurrent solves overlap on the device; requests share no
// device data, so a solve gives the same bits alone and among others.
#include <algorithm>
#include <climits>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <exception>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dg_internal.h"

using dg::set_error;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  int dim = 0, K = 0, M = 0;
  std::vector<double> xmap;
  std::vector<int32_t> ftab, orders;
  double params[16];
  std::vector<double> q0, s;
  dg_solve_params sp;
  int64_t est = 0;
  // results
  int state = DG_REQ_QUEUED;
  dg_solve_report rep;
  std::vector<double> q;
  std::vector<int32_t> orders_out;
  int64_t dev_bytes = 0;
  double t_submit = 0, t_start = 0, t_end = 0;
  int batch_peers = 0;  // most other requests it shared launches with
};

// Device bytes of one multigrid level with the given order map (the buffers
// build_level and ensure_work allocate), from the face table alone.
int64_t level_bytes(int dim, int K, const int32_t* ftab, const std::vector<int32_t>& o) {
  auto n = [&](int e, int d) { return (d < dim) ? o[e * 3 + d] + 1 : 1; };
  auto tang = [&](int e, int f, int k) {  // node count of face f's k-th tangential direction
    const int d = f >> 1;
    const int a = (d == 0) ? 1 : 0, b = (d == 2) ? 1 : 2;
    return (int64_t)n(e, k == 0 ? a : b);
  };
  int64_t nodes = 0, fnodes = 0, mnodes = 0, mortars = 0;
  for (int e = 0; e < K; ++e) {
    nodes += (int64_t)n(e, 0) * n(e, 1) * n(e, 2);
    for (int f = 0; f < 2 * dim; ++f) {
      fnodes += tang(e, f, 0) * tang(e, f, 1);
      const int32_t* ft = ftab + (size_t)(e * 6 + f) * 4;
      if (ft[0] >= 0 && (int64_t)ft[0] * 6 + ft[1] < (int64_t)e * 6 + f) continue;
      ++mortars;
      if (ft[0] < 0) {
        mnodes += tang(e, f, 0) * tang(e, f, 1);
      } else {  // ma x mb <= (largest tangential count of either side)^2
        const int64_t m = std::max(std::max(tang(e, f, 0), tang(e, f, 1)),
                                   std::max(tang(ft[0], ft[1], 0), tang(ft[0], ft[1], 1)));
        mnodes += (dim == 2) ? m : m * m;
      }
    }
  }
  // per node: 10 geometry, 5 volume part, 5 x 5 work arrays; per face node:
  // 5 + 4 + 12 + 5 traces and fluxes, 3 metric; per mortar node: 3 metric
  // + node map; mortar records and tiles; element tables
  return 8 * (nodes * 40 + fnodes * 29 + mnodes * 3) + 4 * mnodes + 72 * mortars + 64 * (int64_t)K;
}

// the mesh's own per-element tables (tau table, orders)
int64_t mesh_bytes(int K) { return (int64_t)K * (3 * 16 * 8 + 3 * 4); }

int64_t footprint(int dim, int K, const int32_t* ftab, const int32_t* orders, int n_over) {
  std::vector<int32_t> o(orders, orders + (size_t)K * 3);
  int top = 1;
  for (int e = 0; e < K; ++e)
    for (int d = 0; d < dim; ++d) top = std::max(top, (int)o[e * 3 + d]);
  if (n_over > 0) {  // adaptation may raise every order up to n_over
    for (int e = 0; e < K; ++e)
      for (int d = 0; d < dim; ++d) o[e * 3 + d] = std::max(o[e * 3 + d], n_over);
    top = std::max(top, n_over);
  }
  int64_t total = 0;
  for (int l = top; l >= 1; --l) {
    std::vector<int32_t> c = o;
    for (int e = 0; e < K; ++e)
      for (int d = 0; d < dim; ++d) c[e * 3 + d] = std::min(c[e * 3 + d], l);
    total += level_bytes(dim, K, ftab, c);
  }
  int64_t fine_nodes = 0;
  for (int e = 0; e < K; ++e) {
    int64_t nn = 1;
    for (int d = 0; d < dim; ++d) nn *= o[e * 3 + d] + 1;
    fine_nodes += nn;
  }
  return total + mesh_bytes(K) + 2 * 5 * 8 * fine_nodes + (1 << 20);  // + state and source, slack
}

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

}  // namespace

struct dg_server {
  dg_server_params p{};
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_id = 1;
  int64_t used = 0;
  bool stop = false;
  std::vector<std::thread> workers;
};

namespace {

struct AllocCtx {
  std::vector<void*> ptrs;
  int64_t bytes = 0;
};

void* alloc_cb(size_t bytes, void* ctx) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  static_cast<AllocCtx*>(ctx)->ptrs.push_back(p);
  static_cast<AllocCtx*>(ctx)->bytes += (int64_t)bytes;
  return p;
}

void free_all(AllocCtx& a) {
  std::lock_guard<std::mutex> lock(dg::device_sync_mutex());
  for (void* p : a.ptrs) cudaFree(p);
  a.ptrs.clear();
}

// What a finished request hands back; the worker publishes it under the
// server lock in one step, so a waiter that sees a finished state also sees
// the result, the report and the timings that go with it.
struct Outcome {
  int state = DG_EINVAL;
  dg_solve_report rep{};
  std::vector<double> q;
  std::vector<int32_t> orders;
  int64_t dev_bytes = 0;
};

// Runs one request on stream st.  Reads the request's inputs only (they do
// not change after submission); everything it produces goes to the outcome.
Outcome run_request(const Request& r, cudaStream_t st) {
  Outcome out;
  AllocCtx ac;
  dg_mesh* m = nullptr;
  dg_mesh_desc d;
  d.dim = r.dim;
  d.K = r.K;
  d.M = r.M;
  d.xmap = r.xmap.data();
  d.ftab = r.ftab.data();
  std::memcpy(d.params, r.params, sizeof(d.params));
  int rc = dg_mesh_create(&d, r.orders.data(), &m);
  if (rc == DG_OK && r.sp.arith != DG_ARITH_FP64) rc = dg_set_arithmetic(m, r.sp.arith);
  if (rc != DG_OK) {
    if (m) dg_mesh_destroy(m);
    out.state = rc;
    return out;
  }
  int64_t nodes = 0;
  dg_mesh_layout(m, &nodes, nullptr);
  const size_t n5 = (size_t)5 * nodes;
  double* q = static_cast<double*>(alloc_cb(n5 * sizeof(double), &ac));
  double* s = nullptr;
  if (!r.s.empty()) s = static_cast<double*>(alloc_cb(n5 * sizeof(double), &ac));
  if (!q || (!r.s.empty() && !s)) {
    out.state = DG_ENOMEM;
    dg_mesh_destroy(m);
    free_all(ac);
    return out;
  }
  std::vector<double> fs;  // freestream of the parameters, element-blocked
  const double* q0 = r.q0.data();
  if (r.q0.empty()) {
    std::vector<int64_t> off(r.K + 1);
    dg_mesh_layout(m, &nodes, off.data());
    fs.resize(n5);
    for (int e = 0; e < r.K; ++e) {
      const int64_t nn = off[e + 1] - off[e];
      for (int v = 0; v < 5; ++v)
        for (int64_t i = 0; i < nn; ++i) fs[5 * off[e] + v * nn + i] = r.params[7 + v];
    }
    q0 = fs.data();
  }
  cudaMemcpyAsync(q, q0, n5 * sizeof(double), cudaMemcpyHostToDevice, st);
  if (s) cudaMemcpyAsync(s, r.s.data(), n5 * sizeof(double), cudaMemcpyHostToDevice, st);
  double* qf = q;
  out.state = dg_solve_steady(&m, &qf, s, &r.sp, alloc_cb, &ac, &out.rep, st);
  int64_t fn = 0;
  dg_mesh_layout(m, &fn, nullptr);
  out.q.resize((size_t)5 * fn);
  cudaMemcpyAsync(out.q.data(), qf, out.q.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  out.orders.resize((size_t)r.K * 3);
  dg_mesh_orders(m, out.orders.data());
  cudaStreamSynchronize(st);
  out.dev_bytes = dg::mesh_device_bytes(m) + ac.bytes;
  dg_mesh_destroy(m);
  free_all(ac);
  return out;
}

// ---------------------------------------------------------------------------
// Shared launches (batch_max > 1): requests that can share a V-cycle run as
// one batch; each keeps its own stopping rule (that of the steady driver
// without full multigrid or adaptation: residual checked before the first
// cycle, after every check_every cycles and at the cap).
// ---------------------------------------------------------------------------
int top_order(const Request& r) {
  int top = 1;
  for (int e = 0; e < r.K; ++e)
    for (int d = 0; d < r.dim; ++d) top = std::max(top, (int)r.orders[e * 3 + d]);
  return top;
}

// (a mixed-form request that starts in the FAS form switches per its own
// residual, which a shared cycle cannot do for each member: it runs alone)
bool batchable(const Request& r) {
  return !r.sp.adapt && !r.sp.fmg && !(r.sp.arith == DG_ARITH_MIXED && r.sp.mixed_from > 0.0);
}

bool same_cycle(const dg_mg_params& a, const dg_mg_params& b) {
  return a.beta1 == b.beta1 && a.beta2 == b.beta2 && a.beta_c == b.beta_c && a.direction == b.direction &&
         a.coarsest == b.coarsest && a.delta_n == b.delta_n && a.graph == b.graph && a.control == b.control &&
         a.eta == b.eta;
}

// Requests whose solves a batch advances exactly as alone: same dimension and
// mapping order (a batch's geometry), arithmetic and cycle, and the same top
// order (a batch cycle visits the levels of its largest top order).
bool compatible(const Request& a, const Request& b) {
  return batchable(a) && batchable(b) && a.dim == b.dim && a.M == b.M && a.sp.arith == b.sp.arith &&
         same_cycle(a.sp.mg, b.sp.mg) && top_order(a) == top_order(b);
}

struct Member {
  std::shared_ptr<Request> r;
  int cycles = 0;         // V-cycles run for it
  double rn = 0.0;        // max |r| at its last check
  double dofs = 0.0;      // its share of the operator evaluations
  int64_t nodes = 0;
  int checked_at = -1;    // cycle count at its last residual check (-1: none yet)
  int slot = -1;          // index in the current batch
};

// One slot's batch of requests that share launches.
struct Cohort {
  dg_server* S;
  cudaStream_t st;
  std::vector<Member> mem;     // running members, in batch order
  dg_mesh* b = nullptr;        // current batch
  double* q = nullptr;         // its state and source (5 x nodes each)
  double* s = nullptr;
  AllocCtx ac;                 // q and s
  int64_t nodes = 0;
  std::vector<int64_t> off;    // node offsets of the solves
  std::vector<int32_t> active; // per batch slot: 1 running, 0 finished (held)

  Cohort(dg_server* srv, cudaStream_t stream) : S(srv), st(stream) {}

  // Take queued requests that can join (in arrival order), up to batch_max
  // running members and the memory budget.  Needs the server lock.
  bool gather_locked() {
    bool took = false;
    const Request& ref = *mem.front().r;
    for (auto it = S->queue.begin(); it != S->queue.end() && (int)mem.size() < S->p.batch_max;) {
      const std::shared_ptr<Request>& c = *it;
      if (compatible(ref, *c) && S->used + c->est <= S->p.hbm_budget) {
        S->used += c->est;
        c->state = DG_REQ_RUNNING;
        c->t_start = seconds_since(S->t0);
        Member m;
        m.r = c;
        mem.push_back(m);
        it = S->queue.erase(it);
        took = true;
      } else {
        ++it;
      }
    }
    return took;
  }

  // The running members' current states (or their starts) in a new batch of
  // the running members; the old batch and arrays are freed.
  int rebuild() {
    const int n = (int)mem.size();
    std::vector<dg_mesh_desc> descs(n);
    std::vector<const int32_t*> ords(n);
    for (int k = 0; k < n; ++k) {
      const Request& r = *mem[k].r;
      descs[k].dim = r.dim;
      descs[k].K = r.K;
      descs[k].M = r.M;
      descs[k].xmap = r.xmap.data();
      descs[k].ftab = r.ftab.data();
      std::memcpy(descs[k].params, r.params, sizeof(r.params));
      ords[k] = r.orders.data();
    }
    dg_mesh* nb = nullptr;
    int rc = dg_batch_create(descs.data(), ords.data(), n, &nb);
    if (rc == DG_OK && mem.front().r->sp.arith != DG_ARITH_FP64) rc = dg_set_arithmetic(nb, mem.front().r->sp.arith);
    if (rc != DG_OK) {
      if (nb) dg_mesh_destroy(nb);
      return rc;
    }
    int32_t ns = 0;
    std::vector<int64_t> noff(n + 1);
    dg_batch_info(nb, &ns, noff.data());
    const int64_t nn = noff[n];
    AllocCtx nac;
    double* nq = static_cast<double*>(alloc_cb((size_t)5 * nn * sizeof(double), &nac));
    double* nsrc = static_cast<double*>(alloc_cb((size_t)5 * nn * sizeof(double), &nac));
    if (!nq || !nsrc) {
      dg_mesh_destroy(nb);
      free_all(nac);
      return DG_ENOMEM;
    }
    std::vector<std::vector<double>> staged;  // host starts, alive until the copies are done
    for (int k = 0; k < n; ++k) {
      Member& m = mem[k];
      const Request& r = *m.r;
      const int64_t len = noff[k + 1] - noff[k];
      m.nodes = len;
      double* dq = nq + 5 * noff[k];
      if (m.slot >= 0) {  // a running member: its current state, exactly
        cudaMemcpyAsync(dq, q + 5 * off[m.slot], (size_t)5 * len * sizeof(double), cudaMemcpyDeviceToDevice, st);
      } else if (!r.q0.empty()) {
        cudaMemcpyAsync(dq, r.q0.data(), (size_t)5 * len * sizeof(double), cudaMemcpyHostToDevice, st);
      } else {  // the freestream of its parameters
        std::vector<double> fs((size_t)5 * len);
        int64_t o = 0;
        for (int e = 0; e < r.K; ++e) {
          int64_t ne = 1;
          for (int d = 0; d < r.dim; ++d) ne *= r.orders[e * 3 + d] + 1;
          for (int v = 0; v < 5; ++v)
            for (int64_t i = 0; i < ne; ++i) fs[(size_t)(5 * o + v * ne + i)] = r.params[7 + v];
          o += ne;
        }
        staged.push_back(std::move(fs));
        cudaMemcpyAsync(dq, staged.back().data(), (size_t)5 * len * sizeof(double), cudaMemcpyHostToDevice, st);
      }
      double* ds = nsrc + 5 * noff[k];
      if (!r.s.empty())
        cudaMemcpyAsync(ds, r.s.data(), (size_t)5 * len * sizeof(double), cudaMemcpyHostToDevice, st);
      else  // no source: zeros give the same bits as a NULL source
        cudaMemsetAsync(ds, 0, (size_t)5 * len * sizeof(double), st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      dg_mesh_destroy(nb);
      free_all(nac);
      return DG_ECUDA;
    }
    release_batch();
    b = nb;
    q = nq;
    s = nsrc;
    ac = std::move(nac);
    nodes = nn;
    off = noff;
    active.assign(n, 1);
    for (int k = 0; k < n; ++k) mem[k].slot = k;
    const int peers = n - 1;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (Member& m : mem) m.r->batch_peers = std::max(m.r->batch_peers, peers);
    }
    return DG_OK;
  }

  void release_batch() {
    if (b) dg_mesh_destroy(b);
    b = nullptr;
    free_all(ac);
    ac = AllocCtx();
    q = s = nullptr;
  }

  // Hand a member's result back (copy of its state, report), hold its solve
  // in the batch and drop it from the running members.
  void finish(size_t k, int status) {
    Member& m = mem[k];
    Outcome out;
    out.state = status;
    out.rep.cycles = m.cycles;
    out.rep.status = status;
    out.rep.rnorm = m.rn;
    out.rep.dof_evals = m.dofs;
    out.rep.nodes = m.nodes;
    out.q.resize((size_t)5 * m.nodes);
    cudaMemcpyAsync(out.q.data(), q + 5 * off[m.slot], out.q.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    out.orders = m.r->orders;
    out.dev_bytes = (int64_t)((double)(dg::mesh_device_bytes(b) + ac.bytes) * (double)m.nodes / (double)nodes);
    active[m.slot] = 0;
    publish(*m.r, out);
    mem.erase(mem.begin() + (long)k);
  }

  void publish(Request& r, Outcome& out) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->used -= r.est;
      r.rep = out.rep;
      r.q.swap(out.q);
      r.orders_out.swap(out.orders);
      r.dev_bytes = out.dev_bytes;
      r.state = out.state;
      r.t_end = seconds_since(S->t0);
      r.q0.clear();
      r.q0.shrink_to_fit();
      r.s.clear();
      r.s.shrink_to_fit();
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }

  // Fail every running member with rc.
  void fail_all(int rc) {
    for (Member& m : mem) {
      Outcome out;
      out.state = rc;
      out.rep.status = rc;
      out.rep.cycles = m.cycles;
      publish(*m.r, out);
    }
    mem.clear();
  }

  // The check of the steady driver at a member's check point: stop when
  // max |r| < tol, on a NaN/inf residual, or at the cycle cap.
  int decide(const Member& m) const {
    const dg_solve_params& sp = m.r->sp;
    if (m.rn < sp.tol) return DG_OK;
    if (std::isnan(m.rn) || std::isinf(m.rn)) return DG_EDIVERGED;
    if (m.cycles >= sp.max_cycles) return DG_ENOTCONVERGED;
    return 1;  // go on
  }

  static int every(const Member& m) { return std::max(1, (int)m.r->sp.check_every); }

  bool at_check(const Member& m) const {
    if (m.checked_at == m.cycles) return false;  // (a rebuild at a check point: already checked)
    return m.checked_at < 0 || m.cycles % every(m) == 0 || m.cycles >= m.r->sp.max_cycles;
  }

  // Residual checks of the members at a check point; members that stop are
  // handed back.  Returns DG_OK or an error of the library.
  int checks() {
    std::vector<double> norms(active.size());
    int rc = dg_residual_norms(b, q, s, norms.data(), st);
    if (rc != DG_OK) return rc;
    bool held = false;
    for (size_t k = 0; k < mem.size();) {
      Member& m = mem[k];
      if (at_check(m)) {
        m.rn = norms[m.slot];
        m.checked_at = m.cycles;
        m.dofs += 5.0 * (double)m.nodes;
        const int d = decide(m);
        if (d <= 0) {
          finish(k, d);
          held = true;
          continue;
        }
      }
      ++k;
    }
    if (held && !mem.empty()) rc = dg_batch_set_active(b, active.data(), st);
    return rc;
  }

  // Cycles until the next member reaches a check point.
  int cycles_to_next_check() const {
    int n = INT32_MAX;
    for (const Member& m : mem) {
      const int cap = m.r->sp.max_cycles;
      const int next = std::min((m.cycles / every(m) + 1) * every(m), cap);
      n = std::min(n, next - m.cycles);
    }
    return std::max(1, n);
  }

  void run() {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      gather_locked();
    }
    int rc = rebuild();
    while (rc == DG_OK && !mem.empty()) {
      if ((rc = checks()) != DG_OK) break;
      bool joined;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        joined = !mem.empty() ? gather_locked() : false;
      }
      const int held = (int)active.size() - (int)std::count(active.begin(), active.end(), 1);
      if (joined || (held > 0 && held >= (int)mem.size() && !mem.empty())) {
        if ((rc = rebuild()) != DG_OK) break;
        continue;  // new members take their first check before any cycle
      }
      if (mem.empty()) {  // all done: take a new compatible group if one waits
        break;
      }
      const int n = cycles_to_next_check();
      const dg_mg_params mg = mem.front().r->sp.mg;
      for (int c = 0; c < n && rc == DG_OK; ++c) {
        dg_cycle_report crep{};
        rc = dg_pmg_vcycle(b, q, s, &mg, 0, &crep, st);
        for (Member& m : mem) {
          m.cycles += 1;
          m.dofs += crep.dof_evals * (double)m.nodes / (double)nodes;
        }
      }
    }
    if (rc != DG_OK) fail_all(rc);
    release_batch();
  }
};

void worker(dg_server* S) {
  cudaSetDevice(S->p.device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        return S->stop || (!S->queue.empty() && S->used + S->queue.front()->est <= S->p.hbm_budget);
      });
      if (S->stop) break;
      r = S->queue.front();
      S->queue.pop_front();
      S->used += r->est;
      r->state = DG_REQ_RUNNING;
      r->t_start = seconds_since(S->t0);
    }
    if (S->p.batch_max > 1 && batchable(*r)) {  // shared launches with compatible requests
      Cohort c(S, st);
      Member m;
      m.r = r;
      c.mem.push_back(m);
      try {
        c.run();
      } catch (const std::exception&) {  // host allocation failure: its requests fail, the server lives
        c.fail_all(DG_ENOMEM);
        c.release_batch();
      }
      continue;
    }
    Outcome out;
    try {
      out = run_request(*r, st);
    } catch (const std::exception&) {  // host allocation failure: the request fails, the server lives
      out = Outcome();
      out.state = DG_ENOMEM;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->used -= r->est;
      r->rep = out.rep;
      r->q.swap(out.q);
      r->orders_out.swap(out.orders);
      r->dev_bytes = out.dev_bytes;
      r->state = out.state;
      r->t_end = seconds_since(S->t0);
      r->q0.clear();
      r->q0.shrink_to_fit();
      r->s.clear();
      r->s.shrink_to_fit();
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

std::shared_ptr<Request> find(dg_server* S, int64_t id) {
  auto it = S->all.find(id);
  return it == S->all.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

int dg_solve_footprint(const dg_mesh_desc* desc, const int32_t* orders, int64_t* bytes) {
  if (!desc || !orders || !bytes || desc->K <= 0 || (desc->dim != 2 && desc->dim != 3) || !desc->ftab) {
    set_error("dg_solve_footprint: bad argument");
    return DG_EINVAL;
  }
  *bytes = footprint(desc->dim, desc->K, desc->ftab, orders, 0);
  return DG_OK;
}

int dg_server_create(const dg_server_params* p, dg_server** out) {
  if (!p || !out || p->slots < 1 || p->slots > 256 || p->hbm_budget <= 0) {
    set_error("dg_server_create: bad argument");
    return DG_EINVAL;
  }
  dg_server* S = new dg_server();
  S->p = *p;
  S->t0 = Clock::now();
  for (int i = 0; i < p->slots; ++i) S->workers.emplace_back(worker, S);
  *out = S;
  return DG_OK;
}

static int submit_impl(dg_server* S, const dg_mesh_desc* desc, const int32_t* orders, const double* q0,
                       const double* s, const dg_solve_params* sp, int64_t* id);

int dg_server_submit(dg_server* S, const dg_mesh_desc* desc, const int32_t* orders, const double* q0,
                     const double* s, const dg_solve_params* sp, int64_t* id) {
  try {
    return submit_impl(S, desc, orders, q0, s, sp, id);
  } catch (const std::exception&) {
    set_error("dg_server_submit: out of host memory");
    return DG_ENOMEM;
  }
}

static int submit_impl(dg_server* S, const dg_mesh_desc* desc, const int32_t* orders, const double* q0,
                       const double* s, const dg_solve_params* sp, int64_t* id) {
  if (!S || !desc || !orders || !sp || !id || desc->K <= 0 || (desc->dim != 2 && desc->dim != 3) ||
      desc->M < 1 || !desc->xmap || !desc->ftab || (sp->adapt && s)) {
    set_error("dg_server_submit: bad argument");
    return DG_EINVAL;
  }
  auto r = std::make_shared<Request>();
  r->dim = desc->dim;
  r->K = desc->K;
  r->M = desc->M;
  const int Mp = desc->M + 1;
  const size_t npe = (desc->dim == 3) ? (size_t)Mp * Mp * Mp : (size_t)Mp * Mp;
  r->xmap.assign(desc->xmap, desc->xmap + (size_t)desc->K * npe * 3);
  r->ftab.assign(desc->ftab, desc->ftab + (size_t)desc->K * 24);
  r->orders.assign(orders, orders + (size_t)desc->K * 3);
  std::memcpy(r->params, desc->params, sizeof(r->params));
  int64_t nodes = 0;
  for (int e = 0; e < desc->K; ++e) {
    int64_t nn = 1;
    for (int d = 0; d < desc->dim; ++d) nn *= orders[e * 3 + d] + 1;
    nodes += nn;
  }
  if (q0) r->q0.assign(q0, q0 + (size_t)5 * nodes);
  if (s) r->s.assign(s, s + (size_t)5 * nodes);
  r->sp = *sp;
  r->est = footprint(desc->dim, desc->K, desc->ftab, orders, sp->adapt ? sp->ap.n_max : 0);
  std::memset(&r->rep, 0, sizeof(r->rep));
  if (r->est > S->p.hbm_budget) {
    set_error("dg_server_submit: the request's memory estimate exceeds the budget");
    return DG_EBUDGET;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    r->t_submit = seconds_since(S->t0);
    S->all.emplace(r->id, r);
    S->queue.push_back(r);
    *id = r->id;
  }
  S->cv_work.notify_all();
  return DG_OK;
}

int dg_server_wait(dg_server* S, int64_t id, double timeout_s) {
  if (!S) {
    set_error("dg_server_wait: null server");
    return DG_EINVAL;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto finished = [&] {
    if (id >= 0) {
      auto r = find(S, id);
      return !r || r->state <= 0;
    }
    for (auto& kv : S->all)
      if (kv.second->state > 0) return false;
    return true;
  };
  if (id >= 0 && !find(S, id)) {
    set_error("dg_server_wait: unknown request");
    return DG_EINVAL;
  }
  if (timeout_s < 0) {
    S->cv_done.wait(lk, finished);
    return DG_OK;
  }
  if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished)) {
    set_error("dg_server_wait: timed out");
    return DG_ETIMEOUT;
  }
  return DG_OK;
}

int dg_server_info(dg_server* S, int64_t id, dg_request_info* info) {
  if (!S || !info) {
    set_error("dg_server_info: bad argument");
    return DG_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto r = find(S, id);
  if (!r) {
    set_error("dg_server_info: unknown request");
    return DG_EINVAL;
  }
  info->state = r->state;
  info->K = r->K;
  info->rep = r->rep;
  info->est_bytes = r->est;
  info->dev_bytes = r->dev_bytes;
  info->t_submit = r->t_submit;
  info->t_start = r->t_start;
  info->t_end = r->t_end;
  info->batch_peers = r->batch_peers;
  info->reserved = 0;
  return DG_OK;
}

int dg_server_result(dg_server* S, int64_t id, double* q, int32_t* orders) {
  if (!S) {
    set_error("dg_server_result: null server");
    return DG_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto r = find(S, id);
  if (!r || r->state > 0) {
    set_error("dg_server_result: unknown or unfinished request");
    return DG_EINVAL;
  }
  if (q) std::copy(r->q.begin(), r->q.end(), q);
  if (orders) std::copy(r->orders_out.begin(), r->orders_out.end(), orders);
  return DG_OK;
}

int dg_server_release(dg_server* S, int64_t id) {
  if (!S) {
    set_error("dg_server_release: null server");
    return DG_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto r = find(S, id);
  if (!r || r->state > 0) {
    set_error("dg_server_release: unknown or unfinished request");
    return DG_EINVAL;
  }
  S->all.erase(id);
  return DG_OK;
}

int dg_server_destroy(dg_server* S) {
  if (!S) return DG_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto& r : S->queue) r->state = DG_ENOTCONVERGED;  // cancelled before it ran
    S->queue.clear();
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
  return DG_OK;
}

}  // extern "C"
