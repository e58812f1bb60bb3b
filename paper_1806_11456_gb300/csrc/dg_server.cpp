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
