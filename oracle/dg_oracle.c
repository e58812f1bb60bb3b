/*
 * dg_oracle.c -- plain, slow, FP64 CPU oracle of the DGSEM compressible
 * Navier-Stokes operator with per-element, per-direction polynomial orders.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (paper section / equation it follows):
 *   - Legendre-Gauss nodes and weights, Lagrange basis and derivative
 *     (Sec. 2, tensor-product nodal basis on Gauss points).
 *   - Element mapping x(xi) of order M, covariant vectors, J, contravariant
 *     metrics Ja^i: 2D cross-product form, 3D invariant curl form (Sec. 2,
 *     mapping and metric equations).
 *   - The element operator F^e(Q) of the weak form (Sec. 2, DiscretNSElem)
 *     evaluated literally: for every test function, an explicit Gauss
 *     quadrature sum over every volume point and every face point, with the
 *     basis functions evaluated from their definition.  No sum
 *     factorisation, no strong-form rewrite.
 *   - Roe advective flux and Bassi-Rebay 1 viscous flux and gradient
 *     (Sec. 2, numerical fluxes), projection mortars on faces whose sides
 *     carry different orders (Sec. 2, non-conforming remark).  The paper
 *     gives no mortar detail; the reading used: per tangential direction
 *     max(N+, N-) + 1 Gauss points in the first side's face frame, both
 *     traces interpolated there, U* and F*.S formed there and L2-projected
 *     back onto each side's face space.
 *   - The isolated operator F-hat: the element's own flux in place of the
 *     numerical flux on its boundary (Sec. 3.2.1, isolated truncation error).
 *   - A(Q) = M^{-1} F(Q) and the residual r = S - A(Q) (Sec. 3.1, nonlinRes).
 *   - The CFL time step (Sec. 2, advective and diffusive restrictions).
 *   - Tensor-product L2 restriction and interpolation between orders
 *     (Sec. 3.1, FASCoarseSol/FASCoarseRes).
 * The Navier-Stokes fluxes follow Appendix A.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_NMAX 12              /* highest polynomial order handled */
#define OR_NP (OR_NMAX + 2)

/* ------------------------------------------------------------------ */
/* 1-D Legendre-Gauss quadrature                                       */
/* ------------------------------------------------------------------ */
static double g_x[OR_NP][OR_NP], g_w[OR_NP][OR_NP];
static int g_ready = 0;

/* Legendre polynomial P_n(x) and its derivative by the three-term recurrence. */
static void legendre_eval(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = p2;
  }
  *P = p1;
  *dP = n * (x * p1 - p0) / (x * x - 1.0);
}

/* Nodes are the roots of P_n (Newton from the Chebyshev-like guess),
 * weights 2 / ((1 - x^2) P_n'(x)^2).  The set is made exactly symmetric. */
static void gauss_init(void) {
  if (g_ready) return;
  for (int n = 1; n < OR_NP; ++n) {
    for (int k = 0; k < (n + 1) / 2; ++k) {
      double x = -cos(M_PI * (k + 0.75) / (n + 0.5));
      double P, dP;
      for (int it = 0; it < 100; ++it) {
        legendre_eval(n, x, &P, &dP);
        double dx = P / dP;
        x -= dx;
        if (fabs(dx) < 1e-17) break;
      }
      legendre_eval(n, x, &P, &dP);
      double w = 2.0 / ((1.0 - x * x) * dP * dP);
      if (2 * k + 1 == n) x = 0.0;
      g_x[n][k] = x;           g_w[n][k] = w;
      g_x[n][n - 1 - k] = -x;  g_w[n][n - 1 - k] = w;
    }
  }
  g_ready = 1;
}

void or_gauss(int n, double* x, double* w) {
  gauss_init();
  for (int k = 0; k < n; ++k) { x[k] = g_x[n][k]; w[k] = g_w[n][k]; }
}

/* Lagrange basis l_j on nodes xs[0..n-1], evaluated at x, from its product
 * definition. */
static double lag(int n, const double* xs, int j, double x) {
  double v = 1.0;
  for (int i = 0; i < n; ++i)
    if (i != j) v *= (x - xs[i]) / (xs[j] - xs[i]);
  return v;
}

/* Derivative of l_j at x: sum over the dropped factor (product rule). */
static double lagd(int n, const double* xs, int j, double x) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == j) continue;
    double v = 1.0 / (xs[j] - xs[m]);
    for (int i = 0; i < n; ++i)
      if (i != j && i != m) v *= (x - xs[i]) / (xs[j] - xs[i]);
    s += v;
  }
  return s;
}

void or_lagrange_table(int n, double x, double* l, double* dl) {
  gauss_init();
  for (int j = 0; j < n; ++j) {
    l[j] = lag(n, g_x[n], j, x);
    dl[j] = lagd(n, g_x[n], j, x);
  }
}

/* ------------------------------------------------------------------ */
/* Parameters                                                          */
/* ------------------------------------------------------------------ */
/* prm layout (double[16]):
 *  0 gamma, 1 Pr, 2 Mach, 3 Re, 4 Sutherland S (T_ref-scaled), 5 C_a, 6 C_nu,
 *  7..11 freestream conserved state, 12 wall_bc_uses_zero_heat_flux (unused) */
typedef struct {
  double g, Pr, Ma, Re, Su, Ca, Cnu;
  double qinf[5];
} prm_t;

static prm_t unpack(const double* p) {
  prm_t r;
  r.g = p[0]; r.Pr = p[1]; r.Ma = p[2]; r.Re = p[3]; r.Su = p[4];
  r.Ca = p[5]; r.Cnu = p[6];
  for (int v = 0; v < 5; ++v) r.qinf[v] = p[7 + v];
  return r;
}

/* ------------------------------------------------------------------ */
/* Navier-Stokes fluxes (Appendix A)                                   */
/* ------------------------------------------------------------------ */
static double pressure(const double* q, const prm_t* P) {
  double ke = 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0];
  return (P->g - 1.0) * (q[4] - ke);
}

/* Primitive set used by the BR1 gradients: (u, v, w, T), T = gamma M^2 p / rho. */
static void primitives(const double* q, const prm_t* P, double* U) {
  double p = pressure(q, P);
  U[0] = q[1] / q[0];
  U[1] = q[2] / q[0];
  U[2] = q[3] / q[0];
  U[3] = P->g * P->Ma * P->Ma * p / q[0];
}

static double sutherland(double T, const prm_t* P) {
  return pow(T, 1.5) * (1.0 + P->Su) / (T + P->Su);
}

/* Advective flux projected on a (not necessarily unit) vector nv. */
static void adv_flux_n(const double* q, const double* nv, const prm_t* P, double* f) {
  double p = pressure(q, P);
  double un = (q[1] * nv[0] + q[2] * nv[1] + q[3] * nv[2]) / q[0];
  f[0] = q[0] * un;
  f[1] = q[1] * un + p * nv[0];
  f[2] = q[2] * un + p * nv[1];
  f[3] = q[3] * un + p * nv[2];
  f[4] = (q[4] + p) * un;
}

/* Viscous flux (without the 1/Re factor) projected on nv.  G[v*3+c] is the
 * derivative of primitive v in Cartesian direction c.  heat = 0 drops the
 * heat-flux term (adiabatic wall). */
static void visc_flux_n(const double* q, const double* G, const double* nv, const prm_t* P,
                        int heat, double* f) {
  double U[4];
  primitives(q, P, U);
  double mu = sutherland(U[3], P);
  double kap = mu;
  double div = G[0 * 3 + 0] + G[1 * 3 + 1] + G[2 * 3 + 2];
  double tau[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      tau[i][j] = mu * (G[i * 3 + j] + G[j * 3 + i]);
      if (i == j) tau[i][j] -= 2.0 / 3.0 * mu * div;
    }
  double hc = kap / ((P->g - 1.0) * P->Pr * P->Ma * P->Ma);
  f[0] = 0.0;
  for (int i = 0; i < 3; ++i) {
    f[1 + i] = 0.0;
    for (int c = 0; c < 3; ++c) f[1 + i] += tau[i][c] * nv[c];
  }
  f[4] = 0.0;
  for (int c = 0; c < 3; ++c) {
    double e = U[0] * tau[0][c] + U[1] * tau[1][c] + U[2] * tau[2][c];
    if (heat) e += hc * G[3 * 3 + c];
    f[4] += e * nv[c];
  }
}

/* Roe approximate Riemann solver, unit normal n: textbook Roe averages
 * (sqrt(rho)-weighted velocity and total enthalpy), |lambda| on the five
 * waves, no entropy fix. */
static void roe_flux(const double* qL, const double* qR, const double* n, const prm_t* P,
                     double* f) {
  double fL[5], fR[5];
  adv_flux_n(qL, n, P, fL);
  adv_flux_n(qR, n, P, fR);
  double rL = qL[0], rR = qR[0];
  double uL[3] = {qL[1] / rL, qL[2] / rL, qL[3] / rL};
  double uR[3] = {qR[1] / rR, qR[2] / rR, qR[3] / rR};
  double pL = pressure(qL, P), pR = pressure(qR, P);
  double HL = (qL[4] + pL) / rL, HR = (qR[4] + pR) / rR;
  double sL = sqrt(rL), sR = sqrt(rR);
  double ut[3];
  for (int c = 0; c < 3; ++c) ut[c] = (sL * uL[c] + sR * uR[c]) / (sL + sR);
  double Ht = (sL * HL + sR * HR) / (sL + sR);
  double rt = sL * sR;
  double q2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  double ct = sqrt((P->g - 1.0) * (Ht - 0.5 * q2));
  double unt = ut[0] * n[0] + ut[1] * n[1] + ut[2] * n[2];
  double dr = rR - rL, dp = pR - pL;
  double du[3] = {uR[0] - uL[0], uR[1] - uL[1], uR[2] - uL[2]};
  double dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2];
  double a1 = (dp - rt * ct * dun) / (2.0 * ct * ct);
  double a5 = (dp + rt * ct * dun) / (2.0 * ct * ct);
  double a2 = dr - dp / (ct * ct);
  double l1 = fabs(unt - ct), l2 = fabs(unt), l5 = fabs(unt + ct);
  double d[5];
  /* acoustic wave u_n - c */
  d[0] = l1 * a1;
  for (int c = 0; c < 3; ++c) d[1 + c] = l1 * a1 * (ut[c] - ct * n[c]);
  d[4] = l1 * a1 * (Ht - unt * ct);
  /* acoustic wave u_n + c */
  d[0] += l5 * a5;
  for (int c = 0; c < 3; ++c) d[1 + c] += l5 * a5 * (ut[c] + ct * n[c]);
  d[4] += l5 * a5 * (Ht + unt * ct);
  /* entropy wave */
  d[0] += l2 * a2;
  for (int c = 0; c < 3; ++c) d[1 + c] += l2 * a2 * ut[c];
  d[4] += l2 * a2 * 0.5 * q2;
  /* shear waves */
  double ush = 0.0;
  for (int c = 0; c < 3; ++c) {
    double dt = du[c] - dun * n[c];
    d[1 + c] += l2 * rt * dt;
    ush += ut[c] * dt;
  }
  d[4] += l2 * rt * ush;
  for (int v = 0; v < 5; ++v) f[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * d[v];
}

/* exported for the consistency/symmetry pins */
void or_roe(const double* prm, const double* qL, const double* qR, const double* n, double* f) {
  prm_t P = unpack(prm);
  roe_flux(qL, qR, n, &P, f);
}
void or_adv_flux(const double* prm, const double* q, const double* n, double* f) {
  prm_t P = unpack(prm);
  adv_flux_n(q, n, &P, f);
}
void or_visc_flux(const double* prm, const double* q, const double* G, const double* n, double* f) {
  prm_t P = unpack(prm);
  visc_flux_n(q, G, n, &P, 1, f);
}

/* Boundary ghost state (tags: 1 freestream, 2 subsonic outflow with the
 * far-field pressure, 3 free-slip, 4 no-slip adiabatic wall). nu = unit normal. */
static void ghost_state(int bc, const double* qi, const double* nu, const prm_t* P, double* qg) {
  if (bc == 1) {
    for (int v = 0; v < 5; ++v) qg[v] = P->qinf[v];
    return;
  }
  double r = qi[0];
  double u[3] = {qi[1] / r, qi[2] / r, qi[3] / r};
  double p = pressure(qi, P);
  if (bc == 2) {
    double pinf = pressure(P->qinf, P);
    qg[0] = r; qg[1] = qi[1]; qg[2] = qi[2]; qg[3] = qi[3];
    qg[4] = pinf / (P->g - 1.0) + 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    return;
  }
  double ug[3];
  if (bc == 3) {
    double un = u[0] * nu[0] + u[1] * nu[1] + u[2] * nu[2];
    for (int c = 0; c < 3; ++c) ug[c] = u[c] - 2.0 * un * nu[c];
  } else {
    for (int c = 0; c < 3; ++c) ug[c] = -u[c];
  }
  qg[0] = r;
  for (int c = 0; c < 3; ++c) qg[1 + c] = r * ug[c];
  qg[4] = p / (P->g - 1.0) + 0.5 * r * (ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
}

/* ------------------------------------------------------------------ */
/* Mesh, geometry                                                      */
/* ------------------------------------------------------------------ */
/* Mesh arguments shared by the entry points:
 *   dim      2 or 3
 *   K        element count
 *   M        mapping order; mapping nodes are equispaced on [-1,1]
 *   xmap     K x (M+1)^dim x 3 doubles, node (a,b[,c]) at ((c*(M+1)+b)*(M+1)+a)
 *   ftab     K x 6 x 4 ints: (neighbour element or -1, neighbour face,
 *            orientation, boundary tag); faces 4,5 ignored in 2D
 *   ord      K x 3 ints: (N1,N2,N3); N3 = 0 in 2D
 * State arrays: element-blocked, element e occupies 5*nn_e doubles starting at
 * 5*off_e, variable-major: q[5*off_e + v*nn_e + node], node = (k*n2+j)*n1+i. */
typedef struct {
  int dim, K, M;
  const double* xmap;
  const int* ftab;
  const int* ord;
  int* off;   /* K+1 node offsets */
} mesh_t;

static void elem_n(const mesh_t* m, int e, int n[3]) {
  for (int d = 0; d < 3; ++d) n[d] = m->ord[3 * e + d] + 1;
  if (m->dim == 2) n[2] = 1;
}

static void build_offsets(mesh_t* m) {
  m->off = (int*)malloc(sizeof(int) * (m->K + 1));
  m->off[0] = 0;
  for (int e = 0; e < m->K; ++e) {
    int n[3];
    elem_n(m, e, n);
    m->off[e + 1] = m->off[e] + n[0] * n[1] * n[2];
  }
}

/* Mapping x(xi) - o and dx/dxi_j at reference point xi for element e, with
 * o = shift (NULL: no shift) subtracted from every mapping node first. */
static void mapping_eval_shift(const mesh_t* m, int e, const double* xi, const double* shift, double* x,
                               double dx[3][3]);
static void mapping_eval(const mesh_t* m, int e, const double* xi, double* x, double dx[3][3]) {
  mapping_eval_shift(m, e, xi, NULL, x, dx);
}
static void mapping_eval_shift(const mesh_t* m, int e, const double* xi, const double* shift, double* x,
                               double dx[3][3]) {
  int M = m->M, Mp = M + 1;
  double eq[OR_NP];
  for (int a = 0; a <= M; ++a) eq[a] = (M == 0) ? 0.0 : -1.0 + 2.0 * a / M;
  double L[3][OR_NP], D[3][OR_NP];
  int nd = m->dim;
  for (int d = 0; d < nd; ++d)
    for (int a = 0; a <= M; ++a) {
      L[d][a] = lag(Mp, eq, a, xi[d]);
      D[d][a] = lagd(Mp, eq, a, xi[d]);
    }
  for (int c = 0; c < 3; ++c) {
    x[c] = 0.0;
    for (int j = 0; j < 3; ++j) dx[c][j] = 0.0;
  }
  const double* X = m->xmap + (size_t)e * (nd == 3 ? Mp * Mp * Mp : Mp * Mp) * 3;
  if (nd == 3) {
    for (int cc = 0; cc <= M; ++cc)
      for (int b = 0; b <= M; ++b)
        for (int a = 0; a <= M; ++a) {
          const double* p0 = X + 3 * ((cc * Mp + b) * Mp + a);
          double p[3] = {p0[0], p0[1], p0[2]};
          if (shift)
            for (int c = 0; c < 3; ++c) p[c] -= shift[c];
          double f = L[0][a] * L[1][b] * L[2][cc];
          double f0 = D[0][a] * L[1][b] * L[2][cc];
          double f1 = L[0][a] * D[1][b] * L[2][cc];
          double f2 = L[0][a] * L[1][b] * D[2][cc];
          for (int c = 0; c < 3; ++c) {
            x[c] += p[c] * f;
            dx[c][0] += p[c] * f0;
            dx[c][1] += p[c] * f1;
            dx[c][2] += p[c] * f2;
          }
        }
  } else {
    /* 2D: x, y from the planar mapping; the extrusion is z = zeta. */
    for (int b = 0; b <= M; ++b)
      for (int a = 0; a <= M; ++a) {
        const double* p0 = X + 3 * (b * Mp + a);
        double p[3] = {p0[0], p0[1], p0[2]};
        if (shift)
          for (int c = 0; c < 2; ++c) p[c] -= shift[c];
        double f = L[0][a] * L[1][b];
        double f0 = D[0][a] * L[1][b];
        double f1 = L[0][a] * D[1][b];
        for (int c = 0; c < 2; ++c) {
          x[c] += p[c] * f;
          dx[c][0] += p[c] * f0;
          dx[c][1] += p[c] * f1;
        }
      }
    x[2] = xi[2];
    dx[2][2] = 1.0;
  }
}

/* Metric terms at the Gauss nodes of element e:
 *   Ja[node*9 + i*3 + c] = c-th Cartesian component of J a^i,  J[node].
 * 2D: cross-product form.  3D: invariant curl form with I^N interpolation at
 * the element's Gauss nodes. */
static void element_metrics(const mesh_t* m, int e, double* Ja, double* J) {
  int n[3];
  elem_n(m, e, n);
  const double *x0 = g_x[n[0]], *x1 = g_x[n[1]], *x2 = g_x[n[2]];
  int nn = n[0] * n[1] * n[2];
  double* dxs = (double*)malloc(sizeof(double) * nn * 9);
  double* xs = (double*)malloc(sizeof(double) * nn * 3);
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int nd = (k * n[1] + j) * n[0] + i;
        double xi[3] = {x0[i], x1[j], (m->dim == 3) ? x2[k] : 0.0};
        double x[3], dx[3][3];
        /* coordinates relative to the element's first mapping node */
        mapping_eval_shift(m, e, xi, m->xmap + (size_t)e * (m->dim == 3 ? (m->M + 1) * (m->M + 1) * (m->M + 1)
                                                                          : (m->M + 1) * (m->M + 1)) * 3,
                           x, dx);
        for (int c = 0; c < 3; ++c) {
          xs[nd * 3 + c] = x[c];
          for (int jj = 0; jj < 3; ++jj) dxs[nd * 9 + c * 3 + jj] = dx[c][jj];
        }
        /* J = a_1 . (a_2 x a_3), a_j = dx/dxi_j */
        double a1[3] = {dx[0][0], dx[1][0], dx[2][0]};
        double a2[3] = {dx[0][1], dx[1][1], dx[2][1]};
        double a3[3] = {dx[0][2], dx[1][2], dx[2][2]};
        double c23[3] = {a2[1] * a3[2] - a2[2] * a3[1], a2[2] * a3[0] - a2[0] * a3[2],
                         a2[0] * a3[1] - a2[1] * a3[0]};
        J[nd] = a1[0] * c23[0] + a1[1] * c23[1] + a1[2] * c23[2];
        if (m->dim == 2) {
          double c31[3] = {a3[1] * a1[2] - a3[2] * a1[1], a3[2] * a1[0] - a3[0] * a1[2],
                           a3[0] * a1[1] - a3[1] * a1[0]};
          double c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2],
                           a1[0] * a2[1] - a1[1] * a2[0]};
          for (int c = 0; c < 3; ++c) {
            Ja[nd * 9 + 0 * 3 + c] = c23[c];
            Ja[nd * 9 + 1 * 3 + c] = c31[c];
            Ja[nd * 9 + 2 * 3 + c] = c12[c];
          }
        }
      }
  if (m->dim == 3) {
    /* For Cartesian component cn (n in the curl formula), with (n,m,l) cyclic:
     * V = I^N( X_l grad X_m - X_m grad X_l ),  Ja^i_n = -1/2 (curl_xi V)_i.
     * X is taken relative to the element's first mapping node o (xs holds
     * x - o): the extra terms -o_l grad X_m + o_m grad X_l have zero discrete
     * curl whenever M <= N, and the products no longer cancel large absolute
     * coordinates. */
    double* V = (double*)malloc(sizeof(double) * nn * 3);
    for (int cn = 0; cn < 3; ++cn) {
      int cm = (cn + 1) % 3, cl = (cn + 2) % 3;
      for (int nd = 0; nd < nn; ++nd)
        for (int jj = 0; jj < 3; ++jj)
          V[nd * 3 + jj] = xs[nd * 3 + cl] * dxs[nd * 9 + cm * 3 + jj] -
                           xs[nd * 3 + cm] * dxs[nd * 9 + cl * 3 + jj];
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            int nd = (k * n[1] + j) * n[0] + i;
            /* dV[comp][dir]: derivative of the interpolant of V_comp along xi_dir */
            double dV[3][3];
            for (int comp = 0; comp < 3; ++comp) {
              double s0 = 0, s1 = 0, s2 = 0;
              for (int a = 0; a < n[0]; ++a)
                s0 += lagd(n[0], x0, a, x0[i]) * V[((k * n[1] + j) * n[0] + a) * 3 + comp];
              for (int a = 0; a < n[1]; ++a)
                s1 += lagd(n[1], x1, a, x1[j]) * V[((k * n[1] + a) * n[0] + i) * 3 + comp];
              for (int a = 0; a < n[2]; ++a)
                s2 += lagd(n[2], x2, a, x2[k]) * V[((a * n[1] + j) * n[0] + i) * 3 + comp];
              dV[comp][0] = s0; dV[comp][1] = s1; dV[comp][2] = s2;
            }
            double curl[3] = {dV[2][1] - dV[1][2], dV[0][2] - dV[2][0], dV[1][0] - dV[0][1]};
            for (int ii = 0; ii < 3; ++ii) Ja[nd * 9 + ii * 3 + cn] = -0.5 * curl[ii];
          }
    }
    free(V);
  }
  free(dxs);
  free(xs);
}

/* Face f of an element: normal direction d = f/2, side +1 for odd f.
 * Tangential directions (ta, tb): the two remaining directions in increasing
 * order. */
static void face_dirs(int f, int* d, int* ta, int* tb, double* side) {
  *d = f / 2;
  *side = (f % 2) ? 1.0 : -1.0;
  if (*d == 0) { *ta = 1; *tb = 2; }
  else if (*d == 1) { *ta = 0; *tb = 2; }
  else { *ta = 0; *tb = 1; }
}

/* Value at reference point xi of the element's nodal interpolant of a field
 * with nv components stored as F[node*nv + v]. */
static void interp_point(const int n[3], const double* F, int nv, const double* xi, double* out) {
  double L0[OR_NP], L1[OR_NP], L2[OR_NP];
  for (int a = 0; a < n[0]; ++a) L0[a] = lag(n[0], g_x[n[0]], a, xi[0]);
  for (int a = 0; a < n[1]; ++a) L1[a] = lag(n[1], g_x[n[1]], a, xi[1]);
  for (int a = 0; a < n[2]; ++a) L2[a] = lag(n[2], g_x[n[2]], a, xi[2]);
  for (int v = 0; v < nv; ++v) out[v] = 0.0;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        double phi = L0[i] * L1[j] * L2[k];
        int nd = (k * n[1] + j) * n[0] + i;
        for (int v = 0; v < nv; ++v) out[v] += F[nd * nv + v] * phi;
      }
}

/* Reference coordinates of face point (s,t) (face-tangential coordinates) on face f. */
static void face_point(int dim, int f, double s, double t, double* xi) {
  int d, ta, tb;
  double side;
  face_dirs(f, &d, &ta, &tb, &side);
  xi[d] = side;
  xi[ta] = s;
  xi[tb] = t;
  if (dim == 2) xi[2] = 0.0;
}

/* Orientation o maps the first side's face coordinates (s,t) to the second
 * side's (s',t'): bit0 swaps, bit1 negates s', bit2 negates t'. */
static void orient_map(int o, double s, double t, double* s2, double* t2) {
  double a = (o & 1) ? t : s, b = (o & 1) ? s : t;
  if (o & 2) a = -a;
  if (o & 4) b = -b;
  *s2 = a;
  *t2 = b;
}

/* ------------------------------------------------------------------ */
/* The residual                                                        */
/* ------------------------------------------------------------------ */
typedef struct {
  double* Ja;  /* per node 9 */
  double* J;   /* per node */
  double* U;   /* per node 4 primitives */
  double* qn;  /* per node 5 conserved, node-major copy */
  double* G;   /* per node 12 gradients */
  int* fo;     /* K*6+1 face point offsets */
  double* us;  /* per face point 4: projected U* */
  double* fs;  /* per face point 5: projected F* S-hat */
} work_t;

static int face_count(int dim) { return 2 * dim; }

/* number of quadrature points on face f of element e, tangential sizes */
static void face_sizes(const mesh_t* m, int e, int f, int* na, int* nb) {
  int n[3], d, ta, tb;
  double side;
  elem_n(m, e, n);
  face_dirs(f, &d, &ta, &tb, &side);
  *na = n[ta];
  *nb = n[tb];
}

/* Outward own-face metric s * Ja^d at reference point xi (interpolant of the
 * nodal metric). */
static void own_face_metric(const mesh_t* m, const work_t* W, int e, int f, const double* xi,
                            double* nv) {
  int n[3], d, ta, tb;
  double side;
  elem_n(m, e, n);
  face_dirs(f, &d, &ta, &tb, &side);
  int nn = n[0] * n[1] * n[2];
  double* tmp = (double*)malloc(sizeof(double) * nn * 3);
  for (int nd = 0; nd < nn; ++nd)
    for (int c = 0; c < 3; ++c) tmp[nd * 3 + c] = W->Ja[(m->off[e] + nd) * 9 + d * 3 + c];
  interp_point(n, tmp, 3, xi, nv);
  for (int c = 0; c < 3; ++c) nv[c] *= side;
  free(tmp);
}

/* Nodal field of element e (node-major, nv comps) from a per-node global array. */
static const double* elem_field(const mesh_t* m, const double* A, int nv, int e) {
  return A + (size_t)m->off[e] * nv;
}

/*
 * Mortar treatment of one face (pass = 1: BR1 state average U*, pass = 2:
 * Roe + BR1 viscous flux).  The mortar carries, per tangential direction,
 * max(N+, N-) + 1 Gauss points laid out in the first side's face frame.
 * Both sides' polynomials are evaluated at the mortar points, the numerical
 * quantity is formed there, and it is L2-projected back onto each side's
 * face space (the second side receives the negated flux for pass 2).
 */
static void mortar(const mesh_t* m, work_t* W, const prm_t* P, int eL, int fL, int pass) {
  const int* ft = m->ftab + (size_t)(eL * 6 + fL) * 4;
  int eR = ft[0], fR = ft[1], o = ft[2], bc = ft[3];
  int nL[3];
  elem_n(m, eL, nL);
  int dL, taL, tbL;
  double sideL;
  face_dirs(fL, &dL, &taL, &tbL, &sideL);
  int ma = nL[taL], mb = nL[tbL];
  int nR[3], dR = 0, taR = 0, tbR = 0;
  double sideR = 0;
  if (eR >= 0) {
    elem_n(m, eR, nR);
    face_dirs(fR, &dR, &taR, &tbR, &sideR);
    int ra = (o & 1) ? nR[tbR] : nR[taR];
    int rb = (o & 1) ? nR[taR] : nR[tbR];
    if (ra > ma) ma = ra;
    if (rb > mb) mb = rb;
  }
  const double *sa = g_x[ma], *sb = g_x[mb], *wa = g_w[ma], *wb = g_w[mb];
  int nvo = (pass == 1) ? 4 : 5;
  double* val = (double*)malloc(sizeof(double) * ma * mb * 5);
  int nnL = nL[0] * nL[1] * nL[2];
  double* qLn = W->qn + (size_t)m->off[eL] * 5;
  double* GLn = W->G + (size_t)m->off[eL] * 12;
  for (int b = 0; b < mb; ++b)
    for (int a = 0; a < ma; ++a) {
      double xiL[3];
      face_point(m->dim, fL, sa[a], sb[b], xiL);
      double qL[5], nv[3];
      interp_point(nL, qLn, 5, xiL, qL);
      own_face_metric(m, W, eL, fL, xiL, nv);
      double S = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
      double nu[3] = {nv[0] / S, nv[1] / S, nv[2] / S};
      double qR[5], GL[12], GR[12];
      if (eR >= 0) {
        double s2, t2, xiR[3];
        orient_map(o, sa[a], sb[b], &s2, &t2);
        face_point(m->dim, fR, s2, t2, xiR);
        interp_point(nR, W->qn + (size_t)m->off[eR] * 5, 5, xiR, qR);
        if (pass == 2) interp_point(nR, W->G + (size_t)m->off[eR] * 12, 12, xiR, GR);
      } else {
        ghost_state(bc, qL, nu, P, qR);
      }
      if (pass == 2) {
        interp_point(nL, GLn, 12, xiL, GL);
        if (eR < 0) memcpy(GR, GL, sizeof(GL));
      }
      double* out = val + (size_t)(b * ma + a) * 5;
      if (pass == 1) {
        double UL[4], UR[4];
        primitives(qL, P, UL);
        primitives(qR, P, UR);
        for (int v = 0; v < 4; ++v) out[v] = 0.5 * (UL[v] + UR[v]);
      } else {
        double fr[5], fvL[5], fvR[5];
        roe_flux(qL, qR, nu, P, fr);
        if (eR < 0 && bc == 3) {
          for (int v = 0; v < 5; ++v) fvL[v] = fvR[v] = 0.0;
        } else if (eR < 0 && bc == 4) {
          /* adiabatic no-slip wall: stresses from the interior gradient at the
           * wall state (zero velocity), no heat flux */
          double qw[5] = {qL[0], 0.0, 0.0, 0.0, qL[4] - 0.5 * (qL[1] * qL[1] + qL[2] * qL[2] + qL[3] * qL[3]) / qL[0]};
          visc_flux_n(qw, GL, nu, P, 0, fvL);
          memcpy(fvR, fvL, sizeof(fvL));
        } else {
          visc_flux_n(qL, GL, nu, P, 1, fvL);
          visc_flux_n(qR, GR, nu, P, 1, fvR);
        }
        for (int v = 0; v < 5; ++v) out[v] = S * (fr[v] - 0.5 * (fvL[v] + fvR[v]) / P->Re);
      }
    }
  /* L2 projection onto side L's face space: node (ka,kb) */
  double* dst = (pass == 1) ? W->us : W->fs;
  {
    int na = nL[taL], nb = nL[tbL];
    for (int kb = 0; kb < nb; ++kb)
      for (int ka = 0; ka < na; ++ka) {
        double acc[5] = {0, 0, 0, 0, 0};
        for (int b = 0; b < mb; ++b)
          for (int a = 0; a < ma; ++a) {
            double wgt = wa[a] * wb[b] * lag(na, g_x[na], ka, sa[a]) * lag(nb, g_x[nb], kb, sb[b]);
            for (int v = 0; v < nvo; ++v) acc[v] += wgt * val[(b * ma + a) * 5 + v];
          }
        double* o2 = dst + (size_t)(W->fo[eL * 6 + fL] + kb * na + ka) * nvo;
        for (int v = 0; v < nvo; ++v) o2[v] = acc[v] / (g_w[na][ka] * g_w[nb][kb]);
      }
  }
  if (eR >= 0) {
    int na = nR[taR], nb = nR[tbR];
    double sgn = (pass == 1) ? 1.0 : -1.0;
    for (int kb = 0; kb < nb; ++kb)
      for (int ka = 0; ka < na; ++ka) {
        double acc[5] = {0, 0, 0, 0, 0};
        for (int b = 0; b < mb; ++b)
          for (int a = 0; a < ma; ++a) {
            double s2, t2;
            orient_map(o, sa[a], sb[b], &s2, &t2);
            double wgt = wa[a] * wb[b] * lag(na, g_x[na], ka, s2) * lag(nb, g_x[nb], kb, t2);
            for (int v = 0; v < nvo; ++v) acc[v] += wgt * val[(b * ma + a) * 5 + v];
          }
        double* o2 = dst + (size_t)(W->fo[eR * 6 + fR] + kb * na + ka) * nvo;
        for (int v = 0; v < nvo; ++v) o2[v] = sgn * acc[v] / (g_w[na][ka] * g_w[nb][kb]);
      }
  }
  (void)nnL; (void)dR; (void)sideR;
  free(val);
}

/* Setup shared by the residual-type entry points. */
static void setup(mesh_t* m, work_t* W, const prm_t* P, const double* q) {
  gauss_init();
  build_offsets(m);
  int N = m->off[m->K];
  W->Ja = (double*)calloc((size_t)N * 9, sizeof(double));
  W->J = (double*)calloc((size_t)N, sizeof(double));
  W->U = (double*)calloc((size_t)N * 4, sizeof(double));
  W->qn = (double*)calloc((size_t)N * 5, sizeof(double));
  W->G = (double*)calloc((size_t)N * 12, sizeof(double));
  W->fo = (int*)calloc((size_t)m->K * 6 + 1, sizeof(int));
  for (int e = 0; e < m->K; ++e) {
    element_metrics(m, e, W->Ja + (size_t)m->off[e] * 9, W->J + m->off[e]);
    int n[3];
    elem_n(m, e, n);
    int nn = n[0] * n[1] * n[2];
    for (int nd = 0; nd < nn; ++nd) {
      double qq[5];
      for (int v = 0; v < 5; ++v) qq[v] = q[(size_t)5 * m->off[e] + (size_t)v * nn + nd];
      memcpy(W->qn + (size_t)(m->off[e] + nd) * 5, qq, sizeof(qq));
      primitives(qq, P, W->U + (size_t)(m->off[e] + nd) * 4);
    }
  }
  int acc = 0;
  for (int e = 0; e < m->K; ++e)
    for (int f = 0; f < 6; ++f) {
      W->fo[e * 6 + f] = acc;
      if (f < face_count(m->dim)) {
        int na, nb;
        face_sizes(m, e, f, &na, &nb);
        acc += na * nb;
      }
    }
  W->fo[m->K * 6] = acc;
  W->us = (double*)calloc((size_t)acc * 4 + 1, sizeof(double));
  W->fs = (double*)calloc((size_t)acc * 5 + 1, sizeof(double));
}

static void teardown(mesh_t* m, work_t* W) {
  free(W->Ja); free(W->J); free(W->U); free(W->qn); free(W->G);
  free(W->fo); free(W->us); free(W->fs); free(m->off);
}

/* Visit each face pair once (the side with the smaller (element, face) key
 * leads) and every boundary face. */
static void all_mortars(const mesh_t* m, work_t* W, const prm_t* P, int pass) {
  for (int e = 0; e < m->K; ++e)
    for (int f = 0; f < face_count(m->dim); ++f) {
      const int* ft = m->ftab + (size_t)(e * 6 + f) * 4;
      if (ft[0] >= 0 && ft[0] * 6 + ft[1] < e * 6 + f) continue;
      mortar(m, W, P, e, f, pass);
    }
}

/* 1-D quantities on n nodes used by the element quadratures. */
typedef struct {
  double L[OR_NP][OR_NP];   /* L[j][q] = l_j(x_q) */
  double Dp[OR_NP][OR_NP];  /* Dp[j][q] = l_j'(x_q) */
  double Lm[OR_NP], Lp[OR_NP];  /* l_j(-1), l_j(+1) */
} basis1_t;

static void basis1(int n, basis1_t* B) {
  for (int j = 0; j < n; ++j) {
    for (int q = 0; q < n; ++q) {
      B->L[j][q] = lag(n, g_x[n], j, g_x[n][q]);
      B->Dp[j][q] = lagd(n, g_x[n], j, g_x[n][q]);
    }
    B->Lm[j] = lag(n, g_x[n], j, -1.0);
    B->Lp[j] = lag(n, g_x[n], j, 1.0);
  }
}

/*
 * Weak-form element quadrature shared by the gradient and the flux
 * divergence.  For every test function phi_j (node j) of element e:
 *   out_j = ( - sum_q W_q sum_d  Fd_q(d) . dphi_j/dxi_d (q)
 *             + sum_faces sum_p w_p Fs_p phi_j(p) ) / (W_j J_j)
 * where Fd (volume, nv comps per direction) and Fs (surface, nv comps per
 * face point, already multiplied by the outward metric) are supplied.
 */
static void weak_form(const mesh_t* m, const work_t* W, int e, int nv, const double* Fd /* node*3*nv */,
                      const double* Fs /* per face point nv, indexed by W->fo */, double* out /* node*nv */) {
  int n[3];
  elem_n(m, e, n);
  basis1_t B[3];
  for (int d = 0; d < 3; ++d) basis1(n[d], &B[d]);
  const double *w0 = g_w[n[0]], *w1 = g_w[n[1]], *w2 = g_w[n[2]];
  int nn = n[0] * n[1] * n[2];
  for (int jk = 0; jk < n[2]; ++jk)
    for (int jj = 0; jj < n[1]; ++jj)
      for (int ji = 0; ji < n[0]; ++ji) {
        int jn = (jk * n[1] + jj) * n[0] + ji;
        double acc[12];
        for (int v = 0; v < nv; ++v) acc[v] = 0.0;
        /* volume: every quadrature point */
        for (int qk = 0; qk < n[2]; ++qk)
          for (int qj = 0; qj < n[1]; ++qj)
            for (int qi = 0; qi < n[0]; ++qi) {
              int qn = (qk * n[1] + qj) * n[0] + qi;
              double Wq = w0[qi] * w1[qj] * w2[qk];
              double dphi[3];
              dphi[0] = B[0].Dp[ji][qi] * B[1].L[jj][qj] * B[2].L[jk][qk];
              dphi[1] = B[0].L[ji][qi] * B[1].Dp[jj][qj] * B[2].L[jk][qk];
              dphi[2] = B[0].L[ji][qi] * B[1].L[jj][qj] * B[2].Dp[jk][qk];
              for (int d = 0; d < m->dim; ++d)
                for (int v = 0; v < nv; ++v) acc[v] -= Wq * Fd[((size_t)qn * 3 + d) * nv + v] * dphi[d];
            }
        /* surface: every face point */
        for (int f = 0; f < face_count(m->dim); ++f) {
          int d, ta, tb;
          double side;
          face_dirs(f, &d, &ta, &tb, &side);
          int jidx[3] = {ji, jj, jk};
          double lend = (side > 0) ? B[d].Lp[jidx[d]] : B[d].Lm[jidx[d]];
          int na = n[ta], nb = n[tb];
          for (int pb = 0; pb < nb; ++pb)
            for (int pa = 0; pa < na; ++pa) {
              double phi = lend * B[ta].L[jidx[ta]][pa] * B[tb].L[jidx[tb]][pb];
              double wp = g_w[na][pa] * g_w[nb][pb];
              const double* fsv = Fs + (size_t)(W->fo[e * 6 + f] + pb * na + pa) * nv;
              for (int v = 0; v < nv; ++v) acc[v] += wp * fsv[v] * phi;
            }
        }
        double mass = w0[ji] * w1[jj] * w2[jk] * W->J[m->off[e] + jn];
        for (int v = 0; v < nv; ++v) out[(size_t)jn * nv + v] = acc[v] / mass;
      }
  (void)nn;
}

/* Own (isolated) surface values: interpolant of the nodal contravariant field
 * Fd(d) at each face point, times the face side sign. */
static void own_surface(const mesh_t* m, const work_t* W, int e, int nv, const double* Fd, double* Fs) {
  int n[3];
  elem_n(m, e, n);
  int nn = n[0] * n[1] * n[2];
  double* tmp = (double*)malloc(sizeof(double) * nn * nv);
  for (int f = 0; f < face_count(m->dim); ++f) {
    int d, ta, tb;
    double side;
    face_dirs(f, &d, &ta, &tb, &side);
    for (int nd = 0; nd < nn; ++nd)
      for (int v = 0; v < nv; ++v) tmp[nd * nv + v] = Fd[((size_t)nd * 3 + d) * nv + v];
    int na = n[ta], nb = n[tb];
    for (int pb = 0; pb < nb; ++pb)
      for (int pa = 0; pa < na; ++pa) {
        double xi[3];
        face_point(m->dim, f, g_x[na][pa], g_x[nb][pb], xi);
        double* o = Fs + (size_t)(W->fo[e * 6 + f] + pb * na + pa) * nv;
        interp_point(n, tmp, nv, xi, o);
        for (int v = 0; v < nv; ++v) o[v] *= side;
      }
  }
  free(tmp);
}

/*
 * or_residual: r = S - A(Q), A = M^{-1} F(Q) (isolated = 0) or
 * A = M^{-1} F-hat(Q) (isolated = 1).  S may be NULL (zero source).
 * isolated = 2 returns the volume term alone (M^{-1} of the volume integral,
 * surface integrals dropped): the magnitude scale of the operator's terms.
 * Returns 0 on success.
 */
int or_residual(int dim, int K, int M, const double* xmap, const int* ftab, const int* ord,
                const double* prm, const double* q, const double* s, double* r, int isolated) {
  mesh_t m = {dim, K, M, xmap, ftab, ord, NULL};
  prm_t P = unpack(prm);
  work_t W;
  setup(&m, &W, &P, q);
  int iso_grad = (isolated == 1);
  /* ---- BR1 pass 1: U* on every face, projected to each side ---- */
  if (!iso_grad) all_mortars(&m, &W, &P, 1);
  /* ---- gradients ---- */
  for (int e = 0; e < K; ++e) {
    int n[3];
    elem_n(&m, e, n);
    int nn = n[0] * n[1] * n[2];
    double* Fd = (double*)calloc((size_t)nn * 3 * 12, sizeof(double));
    for (int nd = 0; nd < nn; ++nd) {
      const double* Ja = W.Ja + (size_t)(m.off[e] + nd) * 9;
      const double* U = W.U + (size_t)(m.off[e] + nd) * 4;
      for (int d = 0; d < 3; ++d)
        for (int v = 0; v < 4; ++v)
          for (int c = 0; c < 3; ++c) Fd[((size_t)nd * 3 + d) * 12 + v * 3 + c] = Ja[d * 3 + c] * U[v];
    }
    double* Fs = (double*)calloc((size_t)W.fo[K * 6] * 12 + 1, sizeof(double));
    if (iso_grad) {
      own_surface(&m, &W, e, 12, Fd, Fs);
    } else {
      for (int f = 0; f < face_count(dim); ++f) {
        int na, nb, d, ta, tb;
        double side;
        face_sizes(&m, e, f, &na, &nb);
        face_dirs(f, &d, &ta, &tb, &side);
        for (int pb = 0; pb < nb; ++pb)
          for (int pa = 0; pa < na; ++pa) {
            int p = W.fo[e * 6 + f] + pb * na + pa;
            double xi[3], nv[3];
            face_point(dim, f, g_x[na][pa], g_x[nb][pb], xi);
            own_face_metric(&m, &W, e, f, xi, nv);
            for (int v = 0; v < 4; ++v)
              for (int c = 0; c < 3; ++c) Fs[(size_t)p * 12 + v * 3 + c] = W.us[(size_t)p * 4 + v] * nv[c];
          }
      }
    }
    weak_form(&m, &W, e, 12, Fd, Fs, W.G + (size_t)m.off[e] * 12);
    free(Fd);
    free(Fs);
  }
  /* ---- BR1 pass 2 + Roe: numerical flux on every face ---- */
  if (!isolated) all_mortars(&m, &W, &P, 2);
  /* (the volume-only mode keeps the BR1 gradient of the full operator) */
  /* ---- flux divergence, residual ---- */
  for (int e = 0; e < K; ++e) {
    int n[3];
    elem_n(&m, e, n);
    int nn = n[0] * n[1] * n[2];
    double* Fd = (double*)calloc((size_t)nn * 3 * 5, sizeof(double));
    for (int nd = 0; nd < nn; ++nd) {
      const double* Ja = W.Ja + (size_t)(m.off[e] + nd) * 9;
      const double* qq = W.qn + (size_t)(m.off[e] + nd) * 5;
      const double* G = W.G + (size_t)(m.off[e] + nd) * 12;
      for (int d = 0; d < 3; ++d) {
        double fa[5], fv[5];
        adv_flux_n(qq, Ja + d * 3, &P, fa);
        visc_flux_n(qq, G, Ja + d * 3, &P, 1, fv);
        for (int v = 0; v < 5; ++v) Fd[((size_t)nd * 3 + d) * 5 + v] = fa[v] - fv[v] / P.Re;
      }
    }
    double* Fs;
    if (isolated == 2) {
      Fs = (double*)calloc((size_t)W.fo[K * 6] * 5 + 1, sizeof(double));
    } else if (isolated) {
      Fs = (double*)calloc((size_t)W.fo[K * 6] * 5 + 1, sizeof(double));
      own_surface(&m, &W, e, 5, Fd, Fs);
    } else {
      Fs = W.fs;
    }
    double* A = (double*)malloc(sizeof(double) * nn * 5);
    weak_form(&m, &W, e, 5, Fd, Fs, A);
    for (int nd = 0; nd < nn; ++nd)
      for (int v = 0; v < 5; ++v) {
        size_t gi = (size_t)5 * m.off[e] + (size_t)v * nn + nd;
        r[gi] = (s ? s[gi] : 0.0) - A[nd * 5 + v];
      }
    free(A);
    free(Fd);
    if (isolated) free(Fs);
  }
  teardown(&m, &W);
  return 0;
}

/* Gradients of (u,v,w,T) as computed inside or_residual (BR1), exported for
 * the viscous pins: G[node*12 + v*3 + c], node-major over the element-blocked
 * node numbering. */
int or_gradients(int dim, int K, int M, const double* xmap, const int* ftab, const int* ord,
                 const double* prm, const double* q, double* Gout) {
  mesh_t m = {dim, K, M, xmap, ftab, ord, NULL};
  prm_t P = unpack(prm);
  work_t W;
  setup(&m, &W, &P, q);
  all_mortars(&m, &W, &P, 1);
  for (int e = 0; e < K; ++e) {
    int n[3];
    elem_n(&m, e, n);
    int nn = n[0] * n[1] * n[2];
    double* Fd = (double*)calloc((size_t)nn * 3 * 12, sizeof(double));
    for (int nd = 0; nd < nn; ++nd) {
      const double* Ja = W.Ja + (size_t)(m.off[e] + nd) * 9;
      const double* U = W.U + (size_t)(m.off[e] + nd) * 4;
      for (int d = 0; d < 3; ++d)
        for (int v = 0; v < 4; ++v)
          for (int c = 0; c < 3; ++c) Fd[((size_t)nd * 3 + d) * 12 + v * 3 + c] = Ja[d * 3 + c] * U[v];
    }
    double* Fs = (double*)calloc((size_t)W.fo[K * 6] * 12 + 1, sizeof(double));
    for (int f = 0; f < face_count(dim); ++f) {
      int na, nb;
      face_sizes(&m, e, f, &na, &nb);
      for (int pb = 0; pb < nb; ++pb)
        for (int pa = 0; pa < na; ++pa) {
          int p = W.fo[e * 6 + f] + pb * na + pa;
          double xi[3], nv[3];
          face_point(dim, f, g_x[na][pa], g_x[nb][pb], xi);
          own_face_metric(&m, &W, e, f, xi, nv);
          for (int v = 0; v < 4; ++v)
            for (int c = 0; c < 3; ++c) Fs[(size_t)p * 12 + v * 3 + c] = W.us[(size_t)p * 4 + v] * nv[c];
        }
    }
    weak_form(&m, &W, e, 12, Fd, Fs, W.G + (size_t)m.off[e] * 12);
    free(Fd);
    free(Fs);
  }
  memcpy(Gout, W.G, sizeof(double) * (size_t)m.off[K] * 12);
  teardown(&m, &W);
  return 0;
}

/* Geometry export (node-major): Ja[node*9 + i*3 + c], J[node]. */
int or_geometry(int dim, int K, int M, const double* xmap, const int* ord, double* Ja, double* J) {
  mesh_t m = {dim, K, M, xmap, NULL, ord, NULL};
  gauss_init();
  build_offsets(&m);
  for (int e = 0; e < K; ++e) element_metrics(&m, e, Ja + (size_t)m.off[e] * 9, J + m.off[e]);
  free(m.off);
  return 0;
}

/* Physical node coordinates (node-major, 3 per node). */
int or_node_coords(int dim, int K, int M, const double* xmap, const int* ord, double* X) {
  mesh_t m = {dim, K, M, xmap, NULL, ord, NULL};
  gauss_init();
  build_offsets(&m);
  for (int e = 0; e < K; ++e) {
    int n[3];
    elem_n(&m, e, n);
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          double xi[3] = {g_x[n[0]][i], g_x[n[1]][j], dim == 3 ? g_x[n[2]][k] : 0.0};
          double dx[3][3];
          mapping_eval(&m, e, xi, X + (size_t)(m.off[e] + (k * n[1] + j) * n[0] + i) * 3, dx);
        }
  }
  free(m.off);
  return 0;
}

/*
 * CFL time step (Sec. 2): at every Gauss point and every reference direction
 * i with N_i > 0,
 *   dt_a = C_a / ( (|v| + c) N_i^2 / h_i ),  dt_nu = C_nu / ( nu N_i^4 / h_i^2 ),
 * h_i = 2 / |a^i| (a^i = Ja^i / J), nu = mu(T) / (rho Re); the global minimum.
 */
double or_cfl_dt(int dim, int K, int M, const double* xmap, const int* ord, const double* prm,
                 const double* q) {
  mesh_t m = {dim, K, M, xmap, NULL, ord, NULL};
  prm_t P = unpack(prm);
  gauss_init();
  build_offsets(&m);
  double dt = 1e300;
  for (int e = 0; e < K; ++e) {
    int n[3];
    elem_n(&m, e, n);
    int nn = n[0] * n[1] * n[2];
    double* Ja = (double*)malloc(sizeof(double) * nn * 9);
    double* J = (double*)malloc(sizeof(double) * nn);
    element_metrics(&m, e, Ja, J);
    for (int nd = 0; nd < nn; ++nd) {
      double qq[5], U[4];
      for (int v = 0; v < 5; ++v) qq[v] = q[(size_t)5 * m.off[e] + (size_t)v * nn + nd];
      primitives(qq, &P, U);
      double c = sqrt(P.g * pressure(qq, &P) / qq[0]);
      double vel = sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
      double nu = sutherland(U[3], &P) / (qq[0] * P.Re);
      for (int i = 0; i < dim; ++i) {
        int Ni = ord[3 * e + i];
        if (Ni <= 0) continue;
        double a2 = 0.0;
        for (int cc = 0; cc < 3; ++cc) {
          double ai = Ja[nd * 9 + i * 3 + cc] / J[nd];
          a2 += ai * ai;
        }
        double h = 2.0 / sqrt(a2);
        double N2 = (double)Ni * (double)Ni;
        double dta = P.Ca / ((vel + c) * N2 / h);
        double dtv = P.Cnu / (nu * N2 * N2 / (h * h));
        if (dta < dt) dt = dta;
        if (dtv < dt) dt = dtv;
      }
    }
    free(Ja);
    free(J);
  }
  free(m.off);
  return dt;
}

/*
 * Tensor-product transfer between order maps (Sec. 3.1): per element and
 * direction, the L2 projection onto the lower order,
 *   v_j = (1/w^c_j) sum_k w^f_k l^c_j(x^f_k) u_k,
 * or the interpolation onto the higher order, u(x^f_j) = sum_k l^c_k(x^f_j) u_k,
 * or the identity.  Applied as the full Kronecker product per element.
 * in/out: element-blocked with nvar variables.
 */
static double t1d(int nfrom, int nto, int j, int k) {
  if (nto < nfrom)
    return g_w[nfrom][k] * lag(nto, g_x[nto], j, g_x[nfrom][k]) / g_w[nto][j];
  if (nto > nfrom) return lag(nfrom, g_x[nfrom], k, g_x[nto][j]);
  return (j == k) ? 1.0 : 0.0;
}

int or_transfer(int dim, int K, const int* ord_from, const int* ord_to, int nvar, const double* in,
                double* out) {
  gauss_init();
  size_t ofrom = 0, oto = 0;
  for (int e = 0; e < K; ++e) {
    int nf[3], nt[3];
    for (int d = 0; d < 3; ++d) {
      nf[d] = ord_from[3 * e + d] + 1;
      nt[d] = ord_to[3 * e + d] + 1;
    }
    if (dim == 2) { nf[2] = 1; nt[2] = 1; }
    int nnf = nf[0] * nf[1] * nf[2], nnt = nt[0] * nt[1] * nt[2];
    for (int v = 0; v < nvar; ++v)
      for (int jk = 0; jk < nt[2]; ++jk)
        for (int jj = 0; jj < nt[1]; ++jj)
          for (int ji = 0; ji < nt[0]; ++ji) {
            double acc = 0.0;
            for (int kk = 0; kk < nf[2]; ++kk)
              for (int kj = 0; kj < nf[1]; ++kj)
                for (int ki = 0; ki < nf[0]; ++ki) {
                  double T = t1d(nf[0], nt[0], ji, ki) * t1d(nf[1], nt[1], jj, kj) *
                             t1d(nf[2], nt[2], jk, kk);
                  acc += T * in[ofrom * nvar + (size_t)v * nnf + (kk * nf[1] + kj) * nf[0] + ki];
                }
            out[oto * nvar + (size_t)v * nnt + (jk * nt[1] + jj) * nt[0] + ji] = acc;
          }
    ofrom += nnf;
    oto += nnt;
  }
  return 0;
}
