// Host side of the library: 1-D tables, geometry precompute, face/mortar
// tables and CTA work lists for one order map (a "level").
//
// Geometry follows Sec. 2 of Rueda-Ramirez et al.: x(xi) of order M,
// covariant vectors a_i = dx/dxi_i, J = a_1 . (a_2 x a_3), contravariant
// metrics J a^i by the cross-product form in 2D and the invariant curl form
// in 3D (interpolant I^N at the order's Gauss nodes).  Face metrics are the
// interpolant of the element's nodal J a^d at the face; a mortar carries the
// first side's face metric interpolated to the mortar nodes.
#include <algorithm>
#include <array>
#include <cmath>
#include <atomic>
#include <cstring>
#include <mutex>
#include <thread>

#include "dg_internal.h"

namespace dg {

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
static Tables1D g_tab;
static std::once_flag g_tab_once;

// Roots of P_n by Newton on the Legendre recurrence (initial guess from the
// asymptotic cosine formula), symmetrised; weights 2/((1-x^2)P_n'^2).
static void gauss_rule(int n, double* x, double* w) {
  for (int k = 0; k < (n + 1) / 2; ++k) {
    double z = std::cos(M_PI * (k + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 60; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pm = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pm = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
    }
    double wk = 2.0 / ((1.0 - z * z) * dp * dp);
    if (2 * k + 1 == n) z = 0.0;
    x[n - 1 - k] = z;
    x[k] = -z;
    w[k] = w[n - 1 - k] = wk;
  }
}

static double bary_eval(const Tables1D& T, int n, int j, double xx) {
  const double* x = T.x[n];
  const double* bw = T.bw[n];
  for (int k = 0; k < n; ++k)
    if (xx == x[k]) return (k == j) ? 1.0 : 0.0;
  double den = 0.0;
  for (int k = 0; k < n; ++k) den += bw[k] / (xx - x[k]);
  return (bw[j] / (xx - x[j])) / den;
}

double lagrange_bary(int n, int j, double xx) { return bary_eval(tables(), n, j, xx); }

static void init_tables() {
  Tables1D& T = g_tab;
  std::memset(&T, 0, sizeof(T));
  for (int n = 1; n < kNP; ++n) {
    gauss_rule(n, T.x[n], T.w[n]);
    for (int j = 0; j < n; ++j) {
      double p = 1.0;
      for (int k = 0; k < n; ++k)
        if (k != j) p *= (T.x[n][j] - T.x[n][k]);
      T.bw[n][j] = 1.0 / p;
    }
  }
  for (int n = 1; n < kNP; ++n) {
    // collocation derivative via barycentric weights
    for (int i = 0; i < n; ++i) {
      double diag = 0.0;
      for (int a = 0; a < n; ++a) {
        if (a == i) continue;
        double v = (T.bw[n][a] / T.bw[n][i]) / (T.x[n][i] - T.x[n][a]);
        T.D[n][i][a] = v;
        diag -= v;
      }
      T.D[n][i][i] = diag;
    }
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < n; ++a) T.Dhat[n][i][a] = -(T.w[n][a] / T.w[n][i]) * T.D[n][a][i];
  }
}

const Tables1D& tables() {
  std::call_once(g_tab_once, [] {
    init_tables();
    // boundary values need the finished barycentric weights
    for (int n = 1; n < kNP; ++n)
      for (int j = 0; j < n; ++j) {
        g_tab.lm[n][j] = bary_eval(g_tab, n, j, -1.0);
        g_tab.lp[n][j] = bary_eval(g_tab, n, j, 1.0);
      }
  });
  return g_tab;
}

void transfer_matrix(int nf, int nt, double* Tm) {
  const Tables1D& T = tables();
  for (int j = 0; j < nt; ++j)
    for (int k = 0; k < nf; ++k) {
      double v;
      if (nt < nf)  // L2 projection onto the lower order, by the finer quadrature
        v = T.w[nf][k] * lagrange_bary(nt, j, T.x[nf][k]) / T.w[nt][j];
      else if (nt > nf)  // interpolation
        v = lagrange_bary(nf, k, T.x[nt][j]);
      else
        v = (j == k) ? 1.0 : 0.0;
      Tm[j * nf + k] = v;
    }
}

Params make_params(const double* p) {
  Params P;
  P.g = p[0]; P.Pr = p[1]; P.Ma = p[2]; P.Re = p[3]; P.Su = p[4]; P.Ca = p[5]; P.Cnu = p[6];
  for (int v = 0; v < 5; ++v) P.qinf[v] = p[7 + v];
  double ke = 0.5 * (P.qinf[1] * P.qinf[1] + P.qinf[2] * P.qinf[2] + P.qinf[3] * P.qinf[3]) / P.qinf[0];
  P.pinf = (P.g - 1.0) * (P.qinf[4] - ke);
  P.gM2 = P.g * P.Ma * P.Ma;
  P.hc = 1.0 / ((P.g - 1.0) * P.Pr * P.Ma * P.Ma);
  P.invRe = 1.0 / P.Re;
  return P;
}

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
namespace {

struct MapEval {
  int M, dim;
  std::vector<double> eq, bw;  // equispaced nodes, barycentric weights
  explicit MapEval(int M_, int dim_) : M(M_), dim(dim_) {
    for (int a = 0; a <= M; ++a) eq.push_back(M == 0 ? 0.0 : -1.0 + 2.0 * a / M);
    for (int a = 0; a <= M; ++a) {
      double p = 1.0;
      for (int b = 0; b <= M; ++b)
        if (b != a) p *= eq[a] - eq[b];
      bw.push_back(1.0 / p);
    }
  }
  // values and derivatives of the M+1 mapping basis functions at x
  void basis(double x, double* L, double* dL) const {
    int n = M + 1;
    int hit = -1;
    for (int k = 0; k < n; ++k)
      if (x == eq[k]) hit = k;
    if (hit >= 0) {
      for (int k = 0; k < n; ++k) L[k] = (k == hit) ? 1.0 : 0.0;
      // derivative at a node: barycentric differentiation formula
      double diag = 0.0;
      for (int k = 0; k < n; ++k) {
        if (k == hit) continue;
        double v = (bw[k] / bw[hit]) / (eq[hit] - eq[k]);
        dL[k] = v;
        diag -= v;
      }
      dL[hit] = diag;
      return;
    }
    double s = 0.0, sd = 0.0;
    for (int k = 0; k < n; ++k) {
      double t = bw[k] / (x - eq[k]);
      s += t;
      sd += t / (x - eq[k]);
    }
    for (int k = 0; k < n; ++k) {
      double t = bw[k] / (x - eq[k]);
      L[k] = t / s;
      // d/dx [t/s] = (-t/(x-x_k) s + t sd) / s^2
      dL[k] = (-t / (x - eq[k]) * s + t * sd) / (s * s);
    }
  }
  // x(xi) and dx[c][j] = d x_c / d xi_j for element nodes X
  void eval(const double* X, const double* xi, double* x, double dx[3][3]) const {
    int n = M + 1;
    double L[3][16], dL[3][16];
    for (int d = 0; d < dim; ++d) basis(xi[d], L[d], dL[d]);
    for (int c = 0; c < 3; ++c) {
      x[c] = 0.0;
      dx[c][0] = dx[c][1] = dx[c][2] = 0.0;
    }
    if (dim == 3) {
      for (int cc = 0; cc < n; ++cc)
        for (int b = 0; b < n; ++b)
          for (int a = 0; a < n; ++a) {
            const double* P = X + 3 * ((cc * n + b) * n + a);
            double f = L[0][a] * L[1][b] * L[2][cc];
            double g0 = dL[0][a] * L[1][b] * L[2][cc];
            double g1 = L[0][a] * dL[1][b] * L[2][cc];
            double g2 = L[0][a] * L[1][b] * dL[2][cc];
            for (int c = 0; c < 3; ++c) {
              x[c] += f * P[c];
              dx[c][0] += g0 * P[c];
              dx[c][1] += g1 * P[c];
              dx[c][2] += g2 * P[c];
            }
          }
    } else {
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          const double* P = X + 3 * (b * n + a);
          double f = L[0][a] * L[1][b];
          double g0 = dL[0][a] * L[1][b];
          double g1 = L[0][a] * dL[1][b];
          for (int c = 0; c < 2; ++c) {
            x[c] += f * P[c];
            dx[c][0] += g0 * P[c];
            dx[c][1] += g1 * P[c];
          }
        }
      x[2] = xi[2];
      dx[2][2] = 1.0;
    }
  }
};

inline void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Ja[node][i][c] and J[node] for one element with node counts n[3]
void element_geometry(const MapEval& ME, const double* Xabs, const int n[3], int dim, std::vector<double>& Ja,
                      std::vector<double>& J) {
  const Tables1D& T = tables();
  int nn = n[0] * n[1] * n[2];
  // Work with coordinates relative to the element's first mapping node: the
  // metrics are unchanged (the curl of the discrete gradient of a constant
  // vanishes when M <= N) and the curl-form products no longer cancel large
  // absolute coordinates.
  const int npe = (dim == 3) ? (ME.M + 1) * (ME.M + 1) * (ME.M + 1) : (ME.M + 1) * (ME.M + 1);
  std::vector<double> Xrel((size_t)npe * 3);
  for (int a = 0; a < npe; ++a)
    for (int c = 0; c < 3; ++c) Xrel[a * 3 + c] = Xabs[a * 3 + c] - Xabs[c];
  const double* X = Xrel.data();
  Ja.assign((size_t)nn * 9, 0.0);
  J.assign(nn, 0.0);
  std::vector<double> xs((size_t)nn * 3), dxs((size_t)nn * 9);
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int nd = (k * n[1] + j) * n[0] + i;
        double xi[3] = {T.x[n[0]][i], T.x[n[1]][j], dim == 3 ? T.x[n[2]][k] : 0.0};
        double x[3], dx[3][3];
        ME.eval(X, xi, x, dx);
        double a[3][3];
        for (int jj = 0; jj < 3; ++jj)
          for (int c = 0; c < 3; ++c) a[jj][c] = dx[c][jj];
        double c23[3];
        cross(a[1], a[2], c23);
        J[nd] = a[0][0] * c23[0] + a[0][1] * c23[1] + a[0][2] * c23[2];
        for (int c = 0; c < 3; ++c) {
          xs[nd * 3 + c] = x[c];
          for (int jj = 0; jj < 3; ++jj) dxs[nd * 9 + c * 3 + jj] = dx[c][jj];
        }
        if (dim == 2) {
          double c31[3], c12[3];
          cross(a[2], a[0], c31);
          cross(a[0], a[1], c12);
          for (int c = 0; c < 3; ++c) {
            Ja[nd * 9 + 0 * 3 + c] = c23[c];
            Ja[nd * 9 + 1 * 3 + c] = c31[c];
            Ja[nd * 9 + 2 * 3 + c] = c12[c];
          }
        }
      }
  if (dim == 3) {
    // invariant curl form: component n of J a^i = -1/2 (curl_xi V^n)_i,
    // V^n = I^N(X_l grad X_m - X_m grad X_l), (n, m, l) cyclic
    std::vector<double> V((size_t)nn * 3);
    for (int cn = 0; cn < 3; ++cn) {
      int cm = (cn + 1) % 3, cl = (cn + 2) % 3;
      for (int nd = 0; nd < nn; ++nd)
        for (int jj = 0; jj < 3; ++jj)
          V[nd * 3 + jj] = xs[nd * 3 + cl] * dxs[nd * 9 + cm * 3 + jj] - xs[nd * 3 + cm] * dxs[nd * 9 + cl * 3 + jj];
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            int nd = (k * n[1] + j) * n[0] + i;
            double g[3][3];  // g[comp][dir]
            for (int comp = 0; comp < 3; ++comp) {
              double s0 = 0, s1 = 0, s2 = 0;
              for (int a = 0; a < n[0]; ++a) s0 += T.D[n[0]][i][a] * V[((k * n[1] + j) * n[0] + a) * 3 + comp];
              for (int a = 0; a < n[1]; ++a) s1 += T.D[n[1]][j][a] * V[((k * n[1] + a) * n[0] + i) * 3 + comp];
              for (int a = 0; a < n[2]; ++a) s2 += T.D[n[2]][k][a] * V[((a * n[1] + j) * n[0] + i) * 3 + comp];
              g[comp][0] = s0;
              g[comp][1] = s1;
              g[comp][2] = s2;
            }
            double curl[3] = {g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]};
            for (int ii = 0; ii < 3; ++ii) Ja[nd * 9 + ii * 3 + cn] = -0.5 * curl[ii];
          }
    }
  }
}

inline void face_dirs(int f, int* d, int* ta, int* tb, int* side) {
  *d = f / 2;
  *side = f % 2;
  if (*d == 0) { *ta = 1; *tb = 2; }
  else if (*d == 1) { *ta = 0; *tb = 2; }
  else { *ta = 0; *tb = 1; }
}

template <typename T>
int dev_upload(int64_t* acc, T** dst, const std::vector<T>& src) {
  size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  DG_CUDA_TRY(cudaMalloc((void**)dst, bytes));
  *acc += (int64_t)bytes;
  if (!src.empty()) DG_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return DG_OK;
}

int dev_zeros(int64_t* acc, double** dst, size_t n) {
  DG_CUDA_TRY(cudaMalloc((void**)dst, std::max<size_t>(1, n) * sizeof(double)));
  *acc += (int64_t)(std::max<size_t>(1, n) * sizeof(double));
  DG_CUDA_TRY(cudaMemset(*dst, 0, std::max<size_t>(1, n) * sizeof(double)));
  return DG_OK;
}

}  // namespace

#define DG_TRY(x)                \
  do {                           \
    int _rc = (x);               \
    if (_rc != DG_OK) return _rc; \
  } while (0)

void element_geometry_host(int M, int dim, const double* xmap_elem, const int n[3], double* Ja, double* J) {
  MapEval ME(M, dim);
  std::vector<double> a, j;
  element_geometry(ME, xmap_elem, n, dim, a, j);
  std::copy(a.begin(), a.end(), Ja);
  std::copy(j.begin(), j.end(), J);
}

std::mutex& device_sync_mutex() {
  static std::mutex mu;
  return mu;
}

int64_t mesh_device_bytes(const dg_mesh* m) {
  int64_t b = m->fine ? m->fine->bytes : 0;
  for (const auto& kv : m->levels) b += kv.second->bytes;
  return b + (int64_t)(5 * m->nslots + 16) * (int64_t)sizeof(double);
}

Level::~Level() {
  std::lock_guard<std::mutex> lock(device_sync_mutex());  // cudaFree synchronises the device
  void* ptrs[] = {d_n,   d_off,   d_geo,       d_fo,    d_fnS,          d_trq,  d_ust,  d_trg,
                  d_fst, d_mortars, d_mnode_mortar, d_mnS, d_mtiles, d_tile_elems, d_tiles, d_vol,
                  d_Q,   d_S,     d_Q0,        d_G,     d_R,            d_geo2, d_fnS2, d_mnS2, d_slot,
                  d_geoT, d_fnST, d_mnST};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// CTA work lists of a level: whole elements of one order triple per tile,
// `pack` nodes per tile at most for elements that fit (one element per tile
// otherwise), ordered by launch class: tiles of <= 128 nodes, <= 256, larger.
// Replaces any earlier lists of the level (graphs captured with them must be
// dropped by the caller).
// SMs of the current device (1 if it cannot be queried)
static int sm_count() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    return 1;
  return nsm;
}

// Element tiles that build_tiles makes with the given packing (whole
// elements of one order triple per tile, pack / nodes-per-element of them)
static int64_t count_tiles(const std::vector<int32_t>& nvec, int K, int pack) {
  std::map<std::array<int, 3>, int64_t> groups;
  for (int e = 0; e < K; ++e) groups[{nvec[e * 3], nvec[e * 3 + 1], nvec[e * 3 + 2]}]++;
  int64_t tiles = 0;
  for (const auto& kv : groups) {
    const int per = std::max(1, pack / (kv.first[0] * kv.first[1] * kv.first[2]));
    tiles += (kv.second + per - 1) / per;
  }
  return tiles;
}

int build_tiles(Level* L, int pack) {
  const int K = L->K;
  const std::vector<int32_t>& nvec = L->nvec_host;
  std::map<std::array<int, 3>, std::vector<int32_t>> groups;
  for (int e = 0; e < K; ++e) groups[{nvec[e * 3], nvec[e * 3 + 1], nvec[e * 3 + 2]}].push_back(e);
  std::vector<int32_t> tile_elems;
  std::vector<ElemTile> tiles;
  size_t max_nodes = 0;
  for (auto& kv : groups) {
    int nn = kv.first[0] * kv.first[1] * kv.first[2];
    if (nn > kMaxElemNodes) {
      set_error("element with more than 729 nodes");
      return DG_EINVAL;
    }
    int per = std::max(1, pack / nn);
    const auto& els = kv.second;
    for (size_t i = 0; i < els.size(); i += per) {
      ElemTile t;
      t.first = (int32_t)tile_elems.size();
      t.count = (int32_t)std::min<size_t>(per, els.size() - i);
      t.n[0] = (int16_t)kv.first[0];
      t.n[1] = (int16_t)kv.first[1];
      t.n[2] = (int16_t)kv.first[2];
      t.pad = 0;
      for (int c = 0; c < t.count; ++c) tile_elems.push_back(els[i + c]);
      tiles.push_back(t);
      max_nodes = std::max(max_nodes, (size_t)t.count * nn);
    }
  }
  auto tile_class = [](const ElemTile& t) {
    const int T = t.count * t.n[0] * t.n[1] * t.n[2];
    return T <= kTileNodes ? 0 : (T <= 2 * kTileNodes ? 1 : 2);
  };
  std::stable_sort(tiles.begin(), tiles.end(),
                   [&](const ElemTile& a, const ElemTile& b) { return tile_class(a) < tile_class(b); });
  for (int c = 0; c < kTileClasses; ++c) L->tile_class_end[c] = L->tile_class_nodes[c] = 0;
  for (const ElemTile& t : tiles) {
    const int c = tile_class(t);
    L->tile_class_end[c]++;
    L->tile_class_nodes[c] = std::max(L->tile_class_nodes[c], t.count * t.n[0] * t.n[1] * t.n[2]);
  }
  for (int c = 1; c < kTileClasses; ++c) L->tile_class_end[c] += L->tile_class_end[c - 1];
  {
    std::lock_guard<std::mutex> lock(device_sync_mutex());
    if (L->d_tiles) cudaFree(L->d_tiles);
    if (L->d_tile_elems) cudaFree(L->d_tile_elems);
  }
  L->d_tiles = nullptr;
  L->d_tile_elems = nullptr;
  int64_t scratch = 0;  // the lists' bytes are counted once, at the first build
  int64_t* acc = (L->n_tiles == 0) ? &L->bytes : &scratch;
  DG_TRY(dev_upload(acc, &L->d_tile_elems, tile_elems));
  DG_TRY(dev_upload(acc, &L->d_tiles, tiles));
  L->n_tiles = (int)tiles.size();
  L->tile_smem_nodes = max_nodes;
  L->pack = pack;
  return DG_OK;
}

int build_level(const dg_mesh* m, const std::vector<int32_t>& orders, Level* L) {
  const Tables1D& T = tables();
  const int dim = m->dim, K = m->K;
  const int nf = 2 * dim;
  L->dim = dim;
  L->K = K;
  L->orders = orders;
  std::vector<int32_t> nvec((size_t)K * 3);
  L->off.assign(K + 1, 0);
  for (int e = 0; e < K; ++e) {
    for (int d = 0; d < 3; ++d) nvec[e * 3 + d] = orders[e * 3 + d] + 1;
    if (dim == 2) nvec[e * 3 + 2] = 1;
    L->off[e + 1] = L->off[e] + (int64_t)nvec[e * 3] * nvec[e * 3 + 1] * nvec[e * 3 + 2];
  }
  L->nodes = L->off[K];
  if (L->nodes >= (int64_t(1) << 31) / 16) {
    set_error("mesh too large for 32-bit node offsets");
    return DG_EINVAL;
  }
  // ---- per-node geometry (SoA: 9 Ja then 1/J) ----
  MapEval ME(m->M, dim);
  int Mp = m->M + 1;
  int npe = (dim == 3) ? Mp * Mp * Mp : Mp * Mp;
  std::vector<double> geo((size_t)10 * L->nodes);
  std::vector<std::vector<double>> elemJa(K);
  std::atomic<int> bad{K};             // smallest element with J <= 0
  std::atomic<bool> affine_all{true};
  parallel_for(K, [&](int e0, int e1) {
    bool affine = true;
    for (int e = e0; e < e1; ++e) {
      std::vector<double> Ja, J;
      int n[3] = {nvec[e * 3], nvec[e * 3 + 1], nvec[e * 3 + 2]};
      element_geometry(ME, m->xmap.data() + (size_t)e * npe * 3, n, dim, Ja, J);
      int nn = n[0] * n[1] * n[2];
      for (int nd = 0; nd < nn; ++nd) {
        if (!(J[nd] > 0.0)) {
          int cur = bad.load();
          while (e < cur && !bad.compare_exchange_weak(cur, e)) {
          }
          break;
        }
        for (int c = 0; c < 9; ++c) geo[(size_t)c * L->nodes + L->off[e] + nd] = Ja[nd * 9 + c];
        geo[(size_t)9 * L->nodes + L->off[e] + nd] = 1.0 / J[nd];
      }
      // affine element: every metric component equal to its value at node 0
      double scale = 0.0, dev = 0.0;
      for (int c = 0; c < 9; ++c) scale = std::max(scale, std::fabs(Ja[c]));
      for (int nd = 1; nd < nn; ++nd)
        for (int c = 0; c < 9; ++c) dev = std::max(dev, std::fabs(Ja[nd * 9 + c] - Ja[c]));
      if (dev > 1e-13 * scale) affine = false;
      elemJa[e] = std::move(Ja);
    }
    if (!affine) affine_all.store(false);
  });
  if (bad.load() < K) {
    set_error("element " + std::to_string(bad.load()) + " has a non-positive Jacobian");
    return DG_EINVAL;
  }
  bool affine = affine_all.load();
  L->affine = affine;
  L->nvec_host = nvec;
  // ---- element-face offsets and own outward face metrics ----
  std::vector<int32_t> fo((size_t)K * 6, 0);
  int64_t acc = 0;
  for (int e = 0; e < K; ++e)
    for (int f = 0; f < 6; ++f) {
      fo[e * 6 + f] = (int32_t)acc;
      if (f < nf) {
        int d, ta, tb, side;
        face_dirs(f, &d, &ta, &tb, &side);
        acc += nvec[e * 3 + ta] * nvec[e * 3 + tb];
      }
    }
  L->face_nodes = acc;
  std::vector<double> fnS((size_t)3 * acc);
  parallel_for(K, [&](int e0, int e1) {
    for (int e = e0; e < e1; ++e) {
      const int* n = &nvec[e * 3];
      for (int f = 0; f < nf; ++f) {
        int d, ta, tb, side;
        face_dirs(f, &d, &ta, &tb, &side);
        const double* lb = side ? T.lp[n[d]] : T.lm[n[d]];
        double sg = side ? 1.0 : -1.0;
        for (int ib = 0; ib < n[tb]; ++ib)
          for (int ia = 0; ia < n[ta]; ++ia) {
            double v[3] = {0, 0, 0};
            for (int k = 0; k < n[d]; ++k) {
              int idx[3];
              idx[d] = k;
              idx[ta] = ia;
              idx[tb] = ib;
              int nd = (idx[2] * n[1] + idx[1]) * n[0] + idx[0];
              for (int c = 0; c < 3; ++c) v[c] += lb[k] * elemJa[e][nd * 9 + d * 3 + c];
            }
            int64_t p = fo[e * 6 + f] + ib * n[ta] + ia;
            for (int c = 0; c < 3; ++c) fnS[(size_t)c * acc + p] = sg * v[c];
          }
      }
    }
  });
  // ---- mortars ----
  std::vector<MortarDev> mortars;
  std::vector<double> mnS;
  std::vector<int32_t> mnode_mortar;
  int64_t mnodes = 0;
  std::vector<std::array<double, 3>> mgeo;
  for (int e = 0; e < K; ++e)
    for (int f = 0; f < nf; ++f) {
      const int32_t* ft = &m->ftab[(size_t)(e * 6 + f) * 4];
      int eR = ft[0], fR = ft[1], o = ft[2], bc = ft[3];
      if (eR >= 0 && eR * 6 + fR < e * 6 + f) continue;
      int d, ta, tb, side;
      face_dirs(f, &d, &ta, &tb, &side);
      int nLa = nvec[e * 3 + ta], nLb = nvec[e * 3 + tb];
      int ma = nLa, mb = nLb;
      bool conf = true;
      if (eR >= 0) {
        int dR, taR, tbR, sR;
        face_dirs(fR, &dR, &taR, &tbR, &sR);
        int ra = (o & 1) ? nvec[eR * 3 + tbR] : nvec[eR * 3 + taR];
        int rb = (o & 1) ? nvec[eR * 3 + taR] : nvec[eR * 3 + tbR];
        ma = std::max(ma, ra);
        mb = std::max(mb, rb);
        conf = (ra == ma && rb == mb);
      }
      conf = conf && nLa == ma && nLb == mb;
      MortarDev M;
      M.eL = e; M.fL = f; M.eR = eR; M.fR = eR >= 0 ? fR : -1;
      M.orient = eR >= 0 ? o : 0;
      M.bc = eR >= 0 ? 0 : bc;
      M.ma = ma; M.mb = mb;
      M.node_off = (int32_t)mnodes;
      M.flags = conf ? 1 : 0;
      M.out_off = 0;  // set with the tiles
      M.pad = 0;
      mortars.push_back(M);
      // mortar-node metric: L face metric interpolated to the mortar nodes
      std::vector<double> Ia((size_t)ma * nLa), Ib((size_t)mb * nLb);
      transfer_matrix(nLa, ma, Ia.data());
      transfer_matrix(nLb, mb, Ib.data());
      for (int b = 0; b < mb; ++b)
        for (int a = 0; a < ma; ++a) {
          std::array<double, 3> v = {0, 0, 0};
          for (int kb = 0; kb < nLb; ++kb)
            for (int ka = 0; ka < nLa; ++ka) {
              double wgt = Ia[a * nLa + ka] * Ib[b * nLb + kb];
              int64_t p = fo[e * 6 + f] + kb * nLa + ka;
              for (int c = 0; c < 3; ++c) v[c] += wgt * fnS[(size_t)c * acc + p];
            }
          mgeo.push_back(v);
          mnode_mortar.push_back((int32_t)(mortars.size() - 1));
        }
      mnodes += (int64_t)ma * mb;
    }
  L->n_mortars = (int)mortars.size();
  L->mortar_nodes = mnodes;
  L->mortars_conforming = true;
  for (const MortarDev& M : mortars) L->mortars_conforming = L->mortars_conforming && (M.flags & 1);
  mnS.assign((size_t)3 * mnodes, 0.0);
  for (int64_t p = 0; p < mnodes; ++p)
    for (int c = 0; c < 3; ++c) mnS[(size_t)c * mnodes + p] = mgeo[p][c];
  // mortar tiles: whole mortars, at most `target` nodes each (a larger
  // mortar forms its own tile); every mortar records where its face nodes
  // start among the tile's outputs
  auto pack_mortars = [&](int target) {
    std::vector<MortarTile> tiles;
    MortarTile cur{0, 0, 0, 0, 0};
    for (int i = 0; i < (int)mortars.size(); ++i) {
      MortarDev& M = mortars[i];
      int sz = M.ma * M.mb;
      if (cur.count > 0 && cur.nodes + sz > target) {
        tiles.push_back(cur);
        cur = MortarTile{i, 0, M.node_off, 0, 0};
      }
      if (cur.count == 0) {
        cur.first = i;
        cur.node_first = M.node_off;
      }
      int d, ta, tb, side;
      face_dirs(M.fL, &d, &ta, &tb, &side);
      int outs = nvec[M.eL * 3 + ta] * nvec[M.eL * 3 + tb];
      if (M.eR >= 0) {
        face_dirs(M.fR, &d, &ta, &tb, &side);
        outs += nvec[M.eR * 3 + ta] * nvec[M.eR * 3 + tb];
      }
      M.out_off = cur.outs;
      cur.count++;
      cur.nodes += sz;
      cur.outs += outs;
    }
    if (cur.count > 0) tiles.push_back(cur);
    return tiles;
  };
  // The mortar kernels run one thread per mortar node and are latency bound
  // on small levels, where their time follows the most loaded SM.  Half-size
  // tiles are taken when they lower that load (nodes of the fullest tile x
  // tiles per SM, rounded up) by a tenth or more and all of them are resident
  // at once (8 CTAs per SM: the mortar kernels' launch bounds).
  std::vector<MortarTile> mtiles = pack_mortars(kMortarTile / 2);
  {
    const int64_t nsm = sm_count();
    auto load = [&](const std::vector<MortarTile>& t) {
      int64_t mx = 0;
      for (const MortarTile& x : t) mx = std::max<int64_t>(mx, x.nodes);
      return ((int64_t)t.size() + nsm - 1) / nsm * mx;
    };
    const int64_t half_load = load(mtiles);
    const bool fits = (int64_t)mtiles.size() <= 8 * nsm;
    std::vector<MortarTile> full = pack_mortars(kMortarTile);  // (also restores the full tiles' out_off)
    if (fits && 10 * half_load <= 9 * load(full))
      mtiles = pack_mortars(kMortarTile / 2);
    else
      mtiles = std::move(full);
  }
  L->n_mtiles = (int)mtiles.size();
  // ---- upload ----
  std::vector<int32_t> off32(L->off.begin(), L->off.end());
  DG_TRY(dev_upload(&L->bytes, &L->d_n, nvec));
  DG_TRY(dev_upload(&L->bytes, &L->d_off, off32));
  DG_TRY(dev_upload(&L->bytes, &L->d_geo, geo));
  DG_TRY(dev_upload(&L->bytes, &L->d_fo, fo));
  DG_TRY(dev_upload(&L->bytes, &L->d_fnS, fnS));
  DG_TRY(dev_upload(&L->bytes, &L->d_mortars, mortars));
  DG_TRY(dev_upload(&L->bytes, &L->d_mnode_mortar, mnode_mortar));
  DG_TRY(dev_upload(&L->bytes, &L->d_mnS, mnS));
  DG_TRY(dev_upload(&L->bytes, &L->d_mtiles, mtiles));
  DG_TRY(dev_upload(&L->bytes, &L->d_slot, m->elem_slot));
  // Element tiles: kTileNodes nodes each, halved (down to a quarter) while
  // the level has fewer tiles than SMs.  The element kernels run one thread
  // per node and an SM's FP64 pipe serialises its tiles' arithmetic, so a
  // coarse level (N = 1: 32 elements per 128-node tile) packed at full size
  // would leave most SMs idle.
  int pack = kTileNodes;
  const int64_t nsm_tiles = sm_count();
  while (pack > kTileNodes / 4 && count_tiles(nvec, K, pack) < nsm_tiles) pack /= 2;
  DG_TRY(build_tiles(L, pack));
  DG_TRY(dev_zeros(&L->bytes, &L->d_trq, (size_t)5 * acc));
  DG_TRY(dev_zeros(&L->bytes, &L->d_ust, (size_t)4 * acc));
  DG_TRY(dev_zeros(&L->bytes, &L->d_trg, (size_t)12 * acc));
  DG_TRY(dev_zeros(&L->bytes, &L->d_fst, (size_t)5 * acc));
  DG_TRY(dev_zeros(&L->bytes, &L->d_vol, (size_t)5 * L->nodes));
  return DG_OK;
}

int ensure_work(Level* L) {
  if (L->d_Q) return DG_OK;
  size_t n = (size_t)5 * L->nodes;
  DG_TRY(dev_zeros(&L->bytes, &L->d_Q, n));
  DG_TRY(dev_zeros(&L->bytes, &L->d_S, n));
  DG_TRY(dev_zeros(&L->bytes, &L->d_Q0, n));
  DG_TRY(dev_zeros(&L->bytes, &L->d_G, n));
  DG_TRY(dev_zeros(&L->bytes, &L->d_R, n));
  return DG_OK;
}

Level* get_level(dg_mesh* m, const std::vector<int32_t>& orders) {
  if (orders == m->orders) return m->fine.get();
  auto it = m->levels.find(orders);
  if (it != m->levels.end()) return it->second.get();
  std::unique_ptr<Level> L(new Level());
  if (build_level(m, orders, L.get()) != DG_OK) return nullptr;
  if (m->autotune && tune_level(m, L.get(), nullptr) != DG_OK) return nullptr;
  Level* raw = L.get();
  m->levels.emplace(orders, std::move(L));
  return raw;
}

}  // namespace dg
