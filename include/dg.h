/*
 * dg.h -- C ABI of the GB300 DGSEM p-multigrid library.
 *
 * The library evaluates the discontinuous Galerkin spectral element (DGSEM)
 * discretisation of the compressible Navier-Stokes equations on hexahedral
 * meshes whose elements carry per-direction polynomial orders (N1,N2,N3), and
 * runs the nonlinear FAS p-multigrid cycle, the anisotropic truncation-error
 * estimate and the order adaptation built on it (Rueda-Ramirez et al.,
 * "A p-multigrid strategy with anisotropic p-adaptation based on truncation
 * errors for high-order DG methods").
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every function returns an int status: DG_OK (0) or a negative DG_E*
 *    code; dg_last_error() then gives a thread-local message.
 *  - Handles (dg_mesh) are library-owned: create/destroy pairs.
 *  - State arrays (q, s, r) are caller-owned DEVICE pointers to doubles in the
 *    element-blocked layout: element e occupies 5*nn_e doubles starting at
 *    5*off_e (off_e from dg_mesh_layout), variable-major inside the element:
 *    q[5*off_e + v*nn_e + node], node = (k*n2 + j)*n1 + i over the element's
 *    tensor Legendre-Gauss nodes, n_d = N_d + 1 (n3 = 1 in 2D).  The five
 *    variables are the conserved (rho, rho u, rho v, rho w, rho e).
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls are asynchronous on that stream unless they return host
 *    data (then they synchronise it).  No call frees caller memory.
 *  - Internal scratch (face traces, multigrid levels) is allocated by the
 *    library on dg_mesh_create / first use and freed by dg_mesh_destroy.
 *  - Invalid arguments give DG_EINVAL without touching any output.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK 0
#define DG_EINVAL (-1)
#define DG_ENOMEM (-2)
#define DG_ECUDA (-3)
#define DG_EDIVERGED (-4)
#define DG_ENOTCONVERGED (-5)
#define DG_EBUDGET (-6)  /* a request does not fit the serving memory budget */
#define DG_ETIMEOUT (-7) /* dg_server_wait ran out of time */

/* dg_residual flags */
#define DG_ISOLATED 1 /* the isolated operator F-hat (own flux on the element boundary) */
#define DG_NORM 2     /* also return max |r| over all nodes and variables */

/* Boundary tags of the face table. */
#define DG_BC_INTERIOR 0
#define DG_BC_FREESTREAM 1 /* ghost = freestream state */
#define DG_BC_OUTFLOW 2    /* ghost = interior state with the far-field pressure */
#define DG_BC_SLIP 3       /* ghost = mirrored normal velocity, no viscous flux */
#define DG_BC_WALL 4       /* no-slip adiabatic wall: ghost = negated velocity, no heat flux */

/*
 * Mesh description (all host pointers, copied by dg_mesh_create).
 *  dim     2 (one-element-thick extrusion, N3 = 0, faces 4/5 ignored) or 3.
 *  K       number of hexahedral elements.
 *  M       order of the element mapping x(xi) (Sec. 2, mapping equation); the
 *          mapping nodes are equispaced on [-1,1] per direction.
 *  xmap    K x (M+1)^dim x 3 doubles; node (a,b[,c]) of element e at
 *          e*(M+1)^dim + (c*(M+1)+b)*(M+1)+a.  2D: x,y used, z = zeta.
 *  ftab    K x 6 x 4 int32 per face (faces 0/1: xi=-1/+1, 2/3: eta, 4/5: zeta):
 *          (neighbour element or -1, neighbour face, orientation, bc tag).
 *          Orientation o maps this side's face coordinates (s,t) -- the two
 *          tangential reference directions in increasing order -- to the
 *          neighbour's: bit0 swaps them, bit1 negates the first, bit2 the
 *          second.  Each interior face must be listed consistently from both sides.
 *  params  0 gamma, 1 Pr, 2 Mach, 3 Re, 4 Sutherland constant S/T_ref,
 *          5 C_a, 6 C_nu (CFL constants), 7..11 freestream conserved state,
 *          12..15 reserved (0).  Nondimensionalisation of Appendix A.
 */
typedef struct {
  int32_t dim;
  int32_t K;
  int32_t M;
  const double* xmap;
  const int32_t* ftab;
  double params[16];
} dg_mesh_desc;

typedef struct dg_mesh dg_mesh;

/*
 * dg_mesh_create -- build the mesh for a per-element order map.
 * Implements the geometry of Sec. 2 (mapping, covariant/contravariant metrics,
 * cross-product form in 2D, invariant curl form in 3D) at the order map's
 * Gauss nodes, the face/mortar tables and the device tables.
 *  orders  K x 3 int32 host array (N1,N2,N3), 1 <= N_d <= 12 (N3 = 0 in 2D);
 *          3D elements are limited to (N1+1)(N2+1)(N3+1) <= 729 nodes.
 *  out     receives the handle.
 * Errors: DG_EINVAL (bad sizes/orders/face table), DG_ENOMEM, DG_ECUDA.
 */
int dg_mesh_create(const dg_mesh_desc* desc, const int32_t* orders, dg_mesh** out);

/*
 * dg_batch_create -- one handle for `nsolves` independent problems (the
 * batched form): their elements are concatenated in solve order, each solve
 * keeping its own flow parameters, explicit time step and residual norm, so
 * every kernel of the path runs once per launch over the elements of all
 * solves and each solve advances exactly as it would alone.  Element groups
 * of equal order triples are shared across solves.  All descriptions must
 * have the same dim and mapping order M.  The state of solve k occupies the
 * node range returned by dg_batch_info.  The batch cycles with every call
 * above (dg_residual, dg_smooth, dg_pmg_vcycle, dg_solve_steady without
 * adaptation); dg_residual's DG_NORM and the driver's checks take the maximum
 * over solves, dg_residual_norms gives them per solve.  Not part of the paper:
 * the batching of independent solves is this library's.
 *  descs   nsolves descriptions; orders: nsolves pointers to K_k x 3 maps.
 */
int dg_batch_create(const dg_mesh_desc* descs, const int32_t* const* orders, int32_t nsolves, dg_mesh** out);

/* dg_batch_info -- number of solves and their node offsets (nsolves + 1
 * values, host; may be NULL) in the batch layout. */
int dg_batch_info(const dg_mesh* mesh, int32_t* nsolves, int64_t* solve_node_offsets);

/*
 * dg_batch_set_active -- hold solves of a batch: active is a host array of
 * nsolves flags; a solve whose flag is 0 is not advanced by any later call
 * (its time step is 0 in every sweep, so its state stays bitwise unchanged,
 * and the smoothing-control rules count it as satisfied), while the others
 * advance exactly as before.  Lets solves of a batch finish at different
 * times.  Not part of the paper (batching is this library's).  Synchronises
 * the stream.
 */
int dg_batch_set_active(dg_mesh* mesh, const int32_t* active, void* stream);

/* dg_residual_norms -- max |S - A(Q)| of every solve of the mesh (host
 * array of nsolves doubles; 1 for a plain mesh).  Synchronises the stream. */
int dg_residual_norms(dg_mesh* mesh, const double* q, const double* s, double* norms, void* stream);

/* dg_mesh_destroy -- free the handle and all library-owned device memory. */
int dg_mesh_destroy(dg_mesh* mesh);

/*
 * dg_mesh_layout -- node count of the layout (state arrays hold 5x that many
 * doubles) and, if elem_offsets != NULL, the K+1 node offsets off_e (host).
 */
int dg_mesh_layout(const dg_mesh* mesh, int64_t* total_nodes, int64_t* elem_offsets);

/* Arithmetic of the operator kernels (dg_set_arithmetic). */
#define DG_ARITH_FP64 0 /* native FP64 */
#define DG_ARITH_DF32 1 /* double-float: pairs of FP32 numbers, ~48-bit significands, on the FP32 pipes */
#define DG_ARITH_MIXED 2 /* FP64 defect, FP32 tangent-linear correction cycle (see dg_set_arithmetic) */

/*
 * dg_set_arithmetic -- choose how the operator kernels evaluate A(Q):
 *  DG_ARITH_FP64 (default) native FP64 everywhere.
 *  DG_ARITH_DF32  double-float on every level (residual, isolated residual,
 *                 tau, smoother).
 *  DG_ARITH_MIXED precision by role: FP64 for the finest-level residual (the
 *                 one that defines convergence and feeds every residual check
 *                 and dg_residual), for the right-hand sides of the coarse
 *                 problems, and for the tau estimate (a difference of
 *                 residuals that cancels); FP32 for every smoother sweep and
 *                 every coarse-level operator evaluation.  dg_pmg_vcycle then
 *                 runs a defect-correction cycle: r = S - A(Q) in FP64, one
 *                 V-cycle of Algorithm 1's shape (same levels, sweeps and L2
 *                 transfers) on the linearised problem J(Q) d = r with the
 *                 Jacobian-vector products J(I Q) d evaluated in FP32 tangent
 *                 arithmetic (their rounding error scales with |d|, so the
 *                 cycle converges to the FP64 solution), and Q += d.  With
 *                 mg->control > 0 the smoothing rules of Sec. 3.1.2 read
 *                 each level's linear residual b - J d (FP64 norms).
 * Memory formats do not change (FP64 state, source and residual arrays) and
 * the smoother's state update stays FP64.  Cached V-cycle graphs are dropped.
 */
int dg_set_arithmetic(dg_mesh* mesh, int mode);

/* dg_mesh_orders -- copy the mesh's K x 3 order map to orders_out (host). */
int dg_mesh_orders(const dg_mesh* mesh, int32_t* orders_out);

/*
 * dg_residual -- r = S - A(Q), A = M^{-1} F(Q) (Sec. 3.1, nonlinRes; F the
 * DGSEM operator of Sec. 2, DiscretNSElem, with Roe and BR1 fluxes and
 * projection mortars on faces whose sides carry different orders).
 *  q, r    device arrays (5 x total_nodes), r may not alias q.
 *  s       device source array or NULL for S = 0.
 *  flags   DG_ISOLATED: the isolated operator (Sec. 3.2.1); DG_NORM: write
 *          max |r| to *rnorm_host (synchronises the stream).
 */
int dg_residual(dg_mesh* mesh, const double* q, const double* s, double* r, int flags,
                double* rnorm_host, void* stream);

/*
 * dg_residual_tangent -- the linearised residual r = b - J(q) dq, J(q) the
 * Jacobian of the operator A at q (Sec. 3.1, nonlinRes, linearised; the
 * correction equation of the mixed-precision cycle), evaluated in FP32
 * tangent arithmetic: every operation of the DGSEM operator carries the
 * directional derivative along dq.  Inputs and output are FP64.
 *  q, dq   device arrays (5 x total_nodes): linearisation point and
 *          correction.  b: device array or NULL for 0.  r may alias neither.
 */
int dg_residual_tangent(dg_mesh* mesh, const double* q, const double* dq, const double* b, double* r, void* stream);

/*
 * dg_cfl_dt -- the explicit time step of Sec. 2: minimum over Gauss points
 * and reference directions with N_i > 0 of C_a h_i / ((|v|+c) N_i^2) and
 * C_nu h_i^2 / (nu N_i^4), h_i = 2/|a^i|, nu = mu(T)/(rho Re).
 * Result on the host in *dt (synchronises the stream).
 */
int dg_cfl_dt(dg_mesh* mesh, const double* q, double* dt, void* stream);

/*
 * dg_smooth -- `sweeps` steps of the Williamson low-storage RK3 smoother
 * (Sec. 3.1) on dQ/dt = S - A(Q), the CFL step recomputed at every sweep.
 *  q       device state, updated in place.  s: device source or NULL.
 */
int dg_smooth(dg_mesh* mesh, double* q, const double* s, int sweeps, void* stream);

/* Multigrid parameters (Sec. 3.1, Algorithm 1). */
typedef struct {
  int32_t beta1;      /* pre-smoothing sweeps per level */
  int32_t beta2;      /* post-smoothing sweeps per level */
  int32_t beta_c;     /* sweeps at the coarsest level (replaces pre + post) */
  int32_t direction;  /* -1: isotropic coarsening; 0/1/2: coarsen that reference direction only */
  int32_t coarsest;   /* lowest level order (1 = N_coarse = 1) */
  int32_t delta_n;    /* order drop between consecutive levels (Sec. 3.1 uses 1); <= 0 means 1 */
  int32_t graph;      /* 1: capture the cycle's launches as a CUDA graph on the first call with these
                         arrays and parameters, replay it on later calls (same result); ignored
                         when control > 0 (the sweep counts are then decided on the host) */
  int32_t control;    /* 0: fixed sweep counts.  n > 0: residual-based smoothing of Sec. 3.1.2 on
                         every level above the coarsest, at most n blocks per rule: pre-smoothing
                         repeats blocks of beta1 sweeps until max|r^P| < eta max|I r^P| (r^P the
                         level's residual, I the restriction to the next coarser level), post-
                         smoothing repeats blocks of beta2 sweeps until max|r| is no larger than
                         after the pre-smoothing.  Decided per solve of a batch (a solve that
                         meets its rule is not advanced by the other solves' extra blocks). */
  double eta;         /* pre-smoothing threshold of the rule above (the paper uses 1.1); <= 0: 1.1 */
} dg_mg_params;

/* What a cycle reports. */
typedef struct {
  int32_t levels;         /* levels visited */
  int32_t residual_evals; /* operator evaluations issued */
  double dof_evals;       /* sum over evaluations of the level's degrees of freedom (5 x nodes) */
  double rnorm;           /* max |S - A(Q)| on the finest level after the cycle (if requested) */
} dg_cycle_report;

/*
 * dg_pmg_vcycle -- one FAS V-cycle (Algorithm 1) from the mesh's orders down
 * to level `coarsest` with high-order coarsening (Sec. 3.3.3: at level l each
 * coarsened direction is capped at l; levels top, top - delta_n, ... >=
 * coarsest), L2 restriction / interpolation between consecutive levels, coarse source S_c = A_c(I Q) + I r (eq FAScoarseSource),
 * correction Q += I (Q_c - Q_c0) (eqs FASIterError, FASCorrectSol).
 *  q       device finest-level state, updated in place.  s: source or NULL.
 *  rep     optional report; with want_norm != 0 rep->rnorm is filled
 *          (synchronises the stream).
 * With the environment variable DG_FUSED_SMOOTH=1 or 2, a smoothing block of
 * a small level whose mortars are all conforming runs as one cooperative
 * launch whose phases meet at grid barriers (same results; off by default).
 * Their waits are bounded: should one run out, the cycle's state is void and
 * the next call that reads a residual norm (want_norm, dg_residual with
 * DG_NORM, dg_residual_norms, dg_solve_steady) returns DG_ECUDA.
 */
int dg_pmg_vcycle(dg_mesh* mesh, double* q, const double* s, const dg_mg_params* mg,
                  int want_norm, dg_cycle_report* rep, void* stream);

/*
 * dg_tau_estimate -- anisotropic truncation-error estimate (Sec. 3.2.1 eqs
 * TruncError! and AnisTruncError, Sec. 3.3.1): for every reference direction i
 * in dir_mask and every level l < P_i, with Q_l the chained L2 restriction of
 * q in direction i only and S_l that of s,
 *   tau_i = R^l(Q_l) - I R^P(q)   (with_correction = 1)  or  R^l(Q_l)  (0),
 * R = S - A with the isolated operator (isolated = 1) or the full operator.
 *  tau_host  K x 3 x 16 doubles (host): tau_host[(e*3+i)*16 + N] = max over
 *            the element's nodes and variables of |tau_i| at order N_i = N;
 *            -1 where nothing was measured (N >= P_i of that element).
 * Synchronises the stream.
 */
int dg_tau_estimate(dg_mesh* mesh, const double* q, const double* s, int dir_mask,
                    int with_correction, int isolated, double* tau_host, void* stream);

/* Adaptation parameters (Sec. 3.3.2 and the order-jump rules of Sec. 4). */
typedef struct {
  double tau_max;      /* truncation-error threshold */
  int32_t n_min;       /* lowest order allowed after adaptation */
  int32_t n_max;       /* highest order allowed */
  int32_t cap;         /* stage cap (multi-stage), <= 0 for none */
  int32_t jump_rule;   /* 0 none, 1: |N+ - N-| <= 1, 2: N+ >= floor(2/3 N-) */
  int32_t conform_tag; /* boundary tag whose touching elements are made conforming, -1 none */
  int32_t reserved[3];
} dg_adapt_params;

/*
 * dg_adapt -- new order map from a tau table (host, layout of
 * dg_tau_estimate) and the mesh's current orders as the reference P:
 * linear-log least-squares extrapolation of each directional estimate,
 * inner-map search then full-map search for the fewest degrees of freedom
 * with sum_i t_i(N_i) < tau_max (ties: smaller estimate, then
 * lexicographically smaller orders), N_max where nothing qualifies, then the
 * order-jump fix-point (only raises orders).
 *  new_orders  K x 3 int32 host output.
 * Pure host computation; deterministic.  DG_ENOTCONVERGED (new_orders
 * untouched) if the jump fix-point has not settled after 100,000 sweeps.
 */
int dg_adapt(const dg_mesh* mesh, const double* tau_host, const dg_adapt_params* ap,
             int32_t* new_orders);

/* Steady-solve parameters (Sec. 3.1.1 cycling, Sec. 3.3.2 adaptation). */
typedef struct {
  double tol;              /* stop when max |S - A(Q)| < tol */
  int32_t max_cycles;      /* V-cycle cap per phase (FMG level, reference solve, final solve) */
  int32_t fmg;             /* 1: full-multigrid start from order 1, raising one order at a time */
  double fmg_tol;          /* residual to reach on a FMG level before raising the order (paper: 1e-1) */
  dg_mg_params mg;         /* cycle used in every phase */
  int32_t adapt;           /* 1: converge to tau_max/10, estimate tau, adapt, then converge to tol */
  int32_t n_stages;        /* multi-stage adaptation (Sec. 3.3.4): 0 = single stage */
  dg_adapt_params ap;      /* adaptation parameters (jump rule etc.; ap.cap = single-stage cap) */
  int32_t stage_orders[4]; /* caps of the successive stages P_2 < P_3 < ... (the mesh enters at P_1) */
  double ref_factor;       /* reference solves converge to ref_factor * tau_max (paper: 1/10; <= 0 means 0.1) */
  int32_t check_every;     /* residual checked after every k-th V-cycle (<= 1: every cycle); a phase
                              may run up to k - 1 cycles past its target */
  int32_t arith;           /* DG_ARITH_FP64, DG_ARITH_DF32 or DG_ARITH_MIXED for a solve run by the serving
                              loop (which owns the mesh); dg_solve_steady itself uses the mesh's setting */
  double mixed_from;       /* DG_ARITH_MIXED only: > 0 runs the FP64 FAS cycle while the last checked
                              max |r| >= mixed_from (full multigrid, the start of each phase) and the
                              mixed defect correction below it, whose linearisation holds only near a
                              solution; <= 0: the mixed cycle throughout */
} dg_solve_params;

typedef struct {
  int32_t cycles;          /* V-cycles in all phases */
  int32_t fmg_cycles;      /* of which on FMG levels below the reference orders */
  int32_t adapted;         /* number of adaptations that changed the order map */
  int32_t status;          /* DG_OK, DG_ENOTCONVERGED or DG_EDIVERGED */
  double rnorm;            /* final max |r| */
  double rnorm_adapt;      /* max |r| when the tau estimate was taken */
  double dof_evals;        /* sum over operator evaluations of the level's degrees of freedom */
  int64_t nodes;           /* nodes of the final mesh */
} dg_solve_report;

/* Allocator for the state array of an adapted mesh: returns a device pointer
 * of at least `bytes` bytes that the caller owns, or NULL. */
typedef void* (*dg_alloc_fn)(size_t bytes, void* ctx);

/*
 * dg_solve_steady -- steady solve A(Q) = S (Sec. 3.1) with the FAS cycle:
 * optional full-multigrid start (orders 1, 2, ... each cycled until max |r| <
 * fmg_tol, then interpolated up; Sec. 3.1.1), V-cycles at the mesh's orders
 * until max |r| < tol -- or, with adapt = 1, until max |r| < tau_max/10
 * (Sec. 3.3.2 step 1), then the isolated anisotropic tau estimate, the order
 * selection and jump rules, a new mesh and the state transferred to it, and
 * V-cycles until max |r| < tol.  With n_stages > 0 the adaptation repeats in
 * stages (Sec. 3.3.4): stage i caps the new orders at stage_orders[i] and is
 * the last one when the largest uncapped required order is <= that cap (or
 * when the stages run out); each stage first converges to tau_max/10.
 *  mesh, q   in/out: on adaptation *mesh is replaced by a new handle (the old
 *            one is destroyed) and *q by an array obtained from `alloc` (the
 *            old array stays the caller's).  s must be NULL when adapt = 1.
 *  alloc     required when adapt = 1.
 * Returns DG_OK when converged, DG_ENOTCONVERGED when a cycle cap was hit,
 * DG_EDIVERGED when the residual became NaN/inf; rep is filled in every case.
 * Synchronises the stream at every residual check.
 */
int dg_solve_steady(dg_mesh** mesh, double** q, const double* s, const dg_solve_params* sp, dg_alloc_fn alloc,
                    void* alloc_ctx, dg_solve_report* rep, void* stream);

/*
 * dg_transfer_state -- move a state between two meshes of the same geometry
 * and topology but different order maps (per element and direction: L2
 * projection when the order drops, interpolation when it rises).
 *  q_from  device array in `from`'s layout; q_to device array in `to`'s.
 */
int dg_transfer_state(const dg_mesh* from, const double* q_from, const dg_mesh* to, double* q_to,
                      void* stream);

/*
 * dg_transfer_noalloc -- the order-map transfer of dg_transfer_state for
 * callers that cannot allocate device memory at the time of the call (a host
 * code that hands all device memory to its own pool at start-up and has none
 * left for a library): it takes no mesh handle and allocates nothing.
 * The paper has no counterpart to this entry point; it is a service of this
 * library.
 *  dim          2 or 3.
 *  K            element count, 1 <= K <= 65,536 (larger K: DG_EINVAL with a
 *               message naming the limit).
 *  orders_from, orders_to  K x 3 int32 HOST arrays of the two order maps
 *               (N3 = 0 in 2D); read before the call returns.
 *  nvar         variables per node (5 for a state), 1 <= nvar <= 64
 *               (larger: DG_EINVAL).
 *  in, out      caller-owned DEVICE arrays in the element-blocked layout of
 *               the two order maps (nvar values per node, variable-major per
 *               element); out may not alias in.
 * Per element and direction it applies the L2 projection (order drops), the
 * interpolation (order rises) or the identity, exactly as dg_transfer_state.
 * Its per-element records live in one statically reserved device array of
 * 2 MiB that every GPU loading the library holds until the process exits.
 * The first call on a device resolves that array's address and writes the
 * Gauss tables to constant memory (synchronous set-up); make that first call
 * before any stream capture.  Calls share the array: calls whose work
 * overlaps on the GPU race, so serialise them (one stream, or events).
 */
int dg_transfer_noalloc(int32_t dim, int32_t K, const int32_t* orders_from, const int32_t* orders_to,
                        int32_t nvar, const double* in, double* out, void* stream);

/*
 * dg_profile_residual -- measurement aid: evaluates the full residual
 * r = S - A(q) once (as dg_residual), then launches each of its stages
 * `iters` times back to back between two CUDA events recorded on `stream`
 * and writes the mean duration per launch in ms to ms_out[0..5]: face
 * traces, mortar pass 1 (BR1 U*), volume (BR1 gradient + flux divergence),
 * mortar pass 2 (Roe + BR1 flux), surface + residual, and ms_out[5] the
 * isolated operator.  r receives the residual.  With DG_ARITH_MIXED the
 * five operator stages are timed as the mixed cycle runs them, in FP32
 * tangent arithmetic (J(q) q), and the isolated operator in FP64.
 * Synchronises the stream.
 */
int dg_profile_residual(dg_mesh* mesh, const double* q, const double* s, double* r, int iters,
                        double* ms_out, void* stream);

/*
 * ---------------------------------------------------------------------------
 * Serving loop: steady solves admitted as they arrive (continuous admission)
 * ---------------------------------------------------------------------------
 * A server runs up to `slots` solves at once, each in its own host worker
 * thread with its own CUDA stream, mesh hierarchy and state, so the kernels
 * of concurrent solves overlap on the device.  A submitted request waits in a
 * FIFO queue until a slot is free and its device-memory estimate
 * (dg_solve_footprint) fits in what the running solves leave of the budget;
 * it then runs dg_solve_steady with its own parameters and keeps its
 * hierarchy resident until it finishes.  Requests share no device data, so a
 * solve gives bit for bit the same result alone and among others.  Not part
 * of the paper: serving many steady solves is this library's addition
 * around the solver of Sec. 3.
 *
 * Shared launches (batch_max > 1).  A slot that takes a request which needs
 * neither full multigrid nor adaptation also takes the queued requests that
 * can share its cycle -- same dimension, mapping order, arithmetic, multigrid
 * parameters and top order -- up to batch_max and the memory budget, and runs
 * them as one batch (dg_batch_create): every kernel of a V-cycle is one
 * launch over the elements of all of them.  Each member keeps its own
 * tolerance, cycle cap and residual-check interval: its residual is checked
 * at its own check points, and a member that stops is held
 * (dg_batch_set_active) and handed back at once.  Requests that arrive while
 * the batch runs join it at the next check point (the batch is rebuilt with
 * the running members' states copied over exactly), and held members are
 * dropped at such rebuilds.  A batch advances each solve exactly as it does
 * alone, so every result is bit for bit the one of the same request alone.
 */
typedef struct dg_server dg_server;

typedef struct {
  int64_t hbm_budget; /* bytes of device memory the running solves may hold together (by estimate) */
  int32_t slots;      /* solves that run at the same time (>= 1) */
  int32_t device;     /* CUDA device of every solve */
  int32_t batch_max;  /* > 1: shared launches, up to batch_max requests per slot (see below); <= 1: one per slot */
  int32_t reserved;
} dg_server_params;

#define DG_REQ_QUEUED 1  /* dg_request_info.state: waiting for a slot or for memory */
#define DG_REQ_RUNNING 2 /* in a slot; finished requests hold their solve's status (<= 0) */

typedef struct {
  int32_t state;          /* DG_REQ_QUEUED, DG_REQ_RUNNING, or DG_OK / DG_E* when finished */
  int32_t K;              /* elements */
  dg_solve_report rep;    /* of the finished solve (rep.nodes sizes the result) */
  int64_t est_bytes;      /* admission estimate */
  int64_t dev_bytes;      /* device bytes the solve's mesh hierarchy and arrays held at its end */
  double t_submit;        /* seconds since dg_server_create */
  double t_start;
  double t_end;
  int32_t batch_peers;    /* most other requests it shared launches with (0: it ran alone) */
  int32_t reserved;
} dg_request_info;

/* Estimate of the device bytes a steady solve of this mesh and order map
 * holds: every multigrid level 1..max order (geometry, face and mortar
 * buffers, work arrays) plus its state and source. */
int dg_solve_footprint(const dg_mesh_desc* desc, const int32_t* orders, int64_t* bytes);

int dg_server_create(const dg_server_params* p, dg_server** out);

/*
 * dg_server_submit -- queue a steady solve.  Host inputs, all copied:
 *  desc, orders  the mesh (as dg_mesh_create).
 *  q0            initial state in the mesh's layout (5 x nodes), or NULL for
 *                the freestream of desc->params.
 *  s             source in the same layout, or NULL.
 *  sp            steady-driver parameters (as dg_solve_steady).
 * DG_EBUDGET when the estimate alone exceeds the budget.
 */
int dg_server_submit(dg_server* srv, const dg_mesh_desc* desc, const int32_t* orders, const double* q0,
                     const double* s, const dg_solve_params* sp, int64_t* id);

/* Wait until request `id` (or every request, id = -1) has finished; DG_ETIMEOUT
 * after timeout_s seconds (< 0: no limit). */
int dg_server_wait(dg_server* srv, int64_t id, double timeout_s);

int dg_server_info(dg_server* srv, int64_t id, dg_request_info* info);

/* Final state (5 x rep.nodes doubles, the final mesh's layout) and order map
 * (K x 3) of a finished request into host arrays (either may be NULL). */
int dg_server_result(dg_server* srv, int64_t id, double* q, int32_t* orders);

/* Drop a finished request's host copies. */
int dg_server_release(dg_server* srv, int64_t id);

/* Cancel queued requests, wait for the running ones, stop the workers. */
int dg_server_destroy(dg_server* srv);

/*
 * dg_set_autotune -- with on != 0, choose each multigrid level's element CTA
 * tiles by timing: for every packing of small elements (64, 128 or 256 nodes
 * per CTA) the volume kernel of every launch class (tiles of <= 128, <= 256,
 * <= 729 nodes) is timed with two CTA sizes on a freestream state, the
 * faster size kept, and the packings are compared on the time of the whole
 * residual (the other tile kernels see the same tiles); the fastest is kept.
 * Levels that exist are tuned now (synchronises the stream; captured V-cycle
 * graphs are dropped), later ones when they are built.  Results do not
 * change: every node's arithmetic is the same whatever CTA computes it.
 * on = 0 keeps the current tiles.  Without tuning a level packs 128 nodes
 * per CTA, or 64 or 32 when it has fewer such tiles than the device has SMs.
 * Not part of the paper (a choice of GPU work decomposition).
 */
int dg_set_autotune(dg_mesh* mesh, int on, void* stream);

/* dg_mesh_tuning -- the finest level's tiles: out[0] nodes per CTA for small
 * elements, out[1..3] CTA sizes of the three launch classes. */
int dg_mesh_tuning(const dg_mesh* mesh, int32_t* out);

/*
 * dg_measure_fma_rates -- measurement aid (the paper has no counterpart): the
 * device's fused multiply-add throughput in FP64 and in FP32, in TFLOP/s
 * (an FMA counts 2 flops), best of three timed launches of independent FMA
 * chains on every SM (CUDA events on `stream`).  These are the denominators
 * of the roofline of the ALU-bound operator kernels.  Allocates and frees a
 * small device buffer; takes about 0.2 s; synchronises the stream.
 */
int dg_measure_fma_rates(double* fp64_tflops, double* fp32_tflops, void* stream);

/* dg_kernel_launches -- cumulative number of CUDA kernels this library has
 * launched in the process (host-side count; a measurement aid). */
int dg_kernel_launches(int64_t* count);

const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
