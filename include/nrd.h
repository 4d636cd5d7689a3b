/*
 * nrd.h -- C ABI of the GB300 implementation of the implicit non-equilibrium
 * radiation diffusion hot path of arXiv 1302.6303 ("Dynamic Implicit 3D
 * Adaptive Mesh Refinement for Non-Equilibrium Radiation Diffusion").
 *
 * The library computes, on one GPU, for a 3D patch hierarchy with refinement
 * ratio 2:
 *   - the two-field (E, T) finite-volume residual of Sec. 3.2/3.3
 *     (Eqs. E_int, diffusion_coeffs1-6, bdf2, be, nonlinearsystem);
 *   - its Jacobian-vector product, as the finite difference of Sec. 4.1
 *     (Eq. Jac-free) or as the exact tangent;
 *   - the physics-based preconditioner P = P1 P2 of Sec. 4.2 with FAC
 *     V-cycles (Sec. 4.3, Algorithm 1) on the diffusion blocks;
 *   - right-preconditioned GMRES inside an inexact Newton solve (Sec. 4.1);
 *   - a BE / BDF2 implicit time step (Sec. 3.3) and the pieces of adaptive
 *     step control (Sec. 3.4-3.5: predictor, local error, controllers);
 *   - the refinement indicators, Berger-Rigoutsos clustering and the
 *     conservative linear transfer between hierarchies of Sec. 5;
 *   - the transposed Jacobian and adjoint solve of one implicit step
 *     (gradients through time steps).
 *
 * Conventions
 *   - Every call returns an int status: NRD_OK (0) or a negative NRD_E* code;
 *     nrd_last_error() then describes the failure.  A NULL context returns
 *     NRD_EINVAL.
 *   - Array arguments are DEVICE pointers owned by the caller (for example
 *     torch CUDA tensors), unless the argument name ends in _host.  Arrays
 *     must not alias unless a call says so.
 *   - Calls taking a cudaStream_t are asynchronous on that stream, except
 *     where a call documents that it synchronises (it then returns results
 *     through host pointers).
 *   - The context owns its internal device work buffers (allocated in
 *     nrd_set_hierarchy and on first use by the solver calls) and frees them
 *     in nrd_destroy.  A context is used by one host thread at a time.
 *
 * Data layout (the "hierarchy layout")
 *   - A hierarchy has L levels; level 0 is one box [0,n0x) x [0,n0y) x
 *     [0,n0z) covering the unit cube; level l has spacing h_d = 1/(n0d 2^l).
 *   - Boxes are given as lo[3], hi[3] (inclusive) in their level's index
 *     space.  Boxes of a level must not overlap.  Boxes of level l >= 1 must
 *     be aligned to ratio 2 (lo even, hi odd) and properly nested: the box
 *     coarsened to level l-1 and grown by one cell (clipped to the domain)
 *     must lie inside level l-1.
 *   - One field on the hierarchy is a vector of ncells values: level 0
 *     first, then level 1, ..., boxes in the given order, x fastest inside a
 *     box.  Cells covered by a finer level are present but are not unknowns:
 *     the residual and Jv return 0 there and their input values are ignored
 *     (except where a call says otherwise).
 *   - A state u is E (ncells values) followed by T (ncells values), FP64.
 *   - Ghost buffers hold one value per face cell of every box, boxes in
 *     layout order, faces x-, x+, y-, y+, z-, z+; on a face normal to axis d
 *     the cells run with axis (d+1)%3 fastest, then axis (d+2)%3.
 *
 * Readings of points where the paper is silent (all implemented exactly this
 * way): Wilson-consistent limiter D_E = D_h/(1 + D_h |dE|/(h E_f)) with
 * D_h = 2 T_f^3/(3 (z_a^3 + z_b^3)) (NRD_LIM_PAPER_LITERAL selects the printed
 * 2 D_r/(1 + D_r g)); face D_T = k T_f^(5/2); Neumann ghost = interior value;
 * Robin ghost from the discrete Robin relation with the unlimited
 * D_b = T^3/(3 z^3); coarse-fine ghost g = (f + 2 i)/3 with i the bilinear
 * interpolation (9,3,3,1)/16 of the four nearest coarse cells; residual per
 * unit volume F = a0 u - b - dt f(u); dots and norms weighted by cell volume
 * over leaf cells.
 */
#ifndef NRD_H
#define NRD_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
enum {
  NRD_OK = 0,
  NRD_EINVAL = -1,   /* bad argument, hierarchy or state */
  NRD_ENOMEM = -2,   /* device or host allocation failed */
  NRD_ENONCONV = -3, /* Newton or GMRES hit its iteration cap (stats filled) */
  NRD_ENEG = -4,     /* a state lost positivity */
  NRD_ENAN = -5,     /* a NaN or Inf appeared in a norm */
  NRD_ECUDA = -6,    /* a CUDA runtime call failed */
  NRD_ESTATE = -7    /* call order: e.g. no hierarchy or no material yet */
};

enum { NRD_BC_NEUMANN = 0, NRD_BC_ROBIN = 1 };
enum { NRD_LIM_WILSON = 0, NRD_LIM_PAPER_LITERAL = 1 };
/* Jv forms: NRD_JV_FD finite difference of Sec. 4.1 (the plain form);
 * NRD_JV_ANALYTIC exact tangent.  Inside nrd_newton / nrd_step the analytic
 * form evaluates the tangent's face coefficients once per Newton iterate
 * (nrd_linearise) and applies them per Krylov iteration (NRD_JV_FROZEN). */
enum { NRD_JV_FD = 0, NRD_JV_ANALYTIC = 1, NRD_JV_FROZEN = 2 };
enum { NRD_PC_F64 = 0, NRD_PC_F32 = 1 };
/* V-cycle smoothers (Sec. 4.3): red-black Gauss-Seidel (the paper's runs),
 * damped point Jacobi, e <- e + omega ((f + off(e)) / diag - e), or block
 * Gauss-Seidel with x-line blocks on the box levels (each line solved
 * exactly, lines coloured by the parity of j + k; the patch levels then keep
 * red-black point sweeps) */
enum { NRD_SMOOTH_RBGS = 0, NRD_SMOOTH_JACOBI = 1, NRD_SMOOTH_LINE = 2 };

/* Solver and model parameters.  nrd_params_default() fills the values used
 * by the paper (Sec. 3.1: k = 0.01; Sec. 4.1: u_min = 1e-6) and the
 * benchmark defaults (GMRES(30), V(2,2), 4 GMG levels, Newton rtol 1e-8). */
typedef struct {
  double k;            /* material conduction constant: D_T = k T^(5/2) */
  int limiter;         /* NRD_LIM_* */
  double u_min;        /* differencing parameter floor of Sec. 4.1 */
  int restart;         /* GMRES restart length m */
  int max_krylov;      /* cap on Krylov iterations per Newton step */
  int jv_mode;         /* NRD_JV_FD (plain) or NRD_JV_ANALYTIC */
  int pc_precision;    /* NRD_PC_F64 or NRD_PC_F32 V-cycle arithmetic */
  int nu1, nu2;        /* pre-/post-smoothing sweeps */
  int nmg;             /* GMG levels on the base box, including the base */
  int coarse_sweeps;   /* smoothing sweeps on the coarsest GMG grid */
  double rtol, atol;   /* Newton stop: ||F|| <= rtol ||F(u0)|| + atol */
  int max_newton;      /* Newton iteration cap */
  double eta_max;      /* Eisenstat-Walker forcing cap */
  double ew_gamma;     /* Eisenstat-Walker gamma */
  int tile_x, tile_y, tile_z;  /* stencil tile shape (0,0,0: 32 x 4 x 4); one of
                                  32x4x4, 32x8x4, 32x4x8, 32x2x4, 16x8x4, 16x4x8,
                                  16x8x8, 16x4x4, 8x8x8, 8x8x4 */
  int graph;           /* 1 (default): with NRD_JV_ANALYTIC, nrd_newton / nrd_step run
                          the whole Newton solve as one CUDA graph whose Newton,
                          GMRES-cycle and Arnoldi loops are conditional graph nodes
                          driven by device-side tests (one read-back per solve);
                          0: host-driven loop, one read-back per Krylov iteration.
                          The host-driven loop is also used while kernel timing is
                          on.  Both give the same iterates up to rounding. */
  int smoother;        /* NRD_SMOOTH_RBGS (default) or NRD_SMOOTH_JACOBI, on every AMR
                          level and GMG grid, or NRD_SMOOTH_LINE */
  double omega;        /* damping of NRD_SMOOTH_JACOBI, 0 < omega <= 1 (default 6/7) */
  double eta0;         /* Eisenstat-Walker forcing of the first Newton iteration,
                          0 < eta0 <= eta_max (default 0.3) */
} nrd_params;

/* Statistics of one Newton solve (nrd_newton / nrd_step). */
typedef struct {
  int status;          /* 0 converged, NRD_ENONCONV otherwise */
  int newton_its;      /* Newton iterations taken */
  int krylov_its;      /* total GMRES iterations (Jv + P^{-1} applications) */
  int pc_setups;       /* preconditioner set-ups (one per Newton iteration) */
  double fnorm0;       /* ||F(u0)|| (volume-weighted 2-norm over leaf cells) */
  double fnorm;        /* final ||F|| */
  double min_lambda;   /* smallest positivity damping factor used (Sec. 4.1) */
  int64_t kernels;     /* graph form: kernel launches the solve executed (kernel nodes
                          of each loop body times the iterations of that loop);
                          host-driven form: 0 (not counted) */
} nrd_stats;

typedef struct nrd_ctx nrd_ctx;

/* Fill *p with defaults.  Returns NRD_EINVAL if p is NULL. */
int nrd_params_default(nrd_params* p);

/* Create a context on the current CUDA device.  *out receives the handle.
 * Errors: NRD_EINVAL (bad parameter), NRD_ENOMEM. */
int nrd_create(const nrd_params* p, nrd_ctx** out);

/* Free the context and every device buffer it owns. */
int nrd_destroy(nrd_ctx* ctx);

/* Message of the last failed call on ctx (owned by ctx; valid until the
 * next call).  NULL ctx gives a static message. */
const char* nrd_last_error(const nrd_ctx* ctx);

/* Replace the parameters of an existing context (takes effect on the next
 * call). */
int nrd_set_params(nrd_ctx* ctx, const nrd_params* p);

/* Define the patch hierarchy (Sec. 3.2.1 SAMR hierarchy).
 *   nlevels      number of levels L >= 1
 *   nboxes_host  [L] boxes per level (nboxes_host[0] must be 1)
 *   boxes_host   6 ints per box, levels in order: lo[3], hi[3] inclusive
 *   bc_type_host [6] NRD_BC_* for faces x-, x+, y-, y+, z-, z+ (for E; T is
 *                Neumann everywhere, Sec. 3.1 Eq. bcs)
 *   bc_R_host    [6] Robin data R of Sec. 3.1 Eq. robinbc
 * Builds every ghost, flux-matching, coarsening and tile work-list on the
 * host and uploads them.  Synchronises the device.  Errors: NRD_EINVAL
 * (alignment, nesting, overlap, domain), NRD_ENOMEM, NRD_ECUDA. */
int nrd_set_hierarchy(nrd_ctx* ctx, int nlevels, const int* nboxes_host, const int* boxes_host,
                      const int* bc_type_host, const double* bc_R_host);

/* Sizes of the hierarchy layout: ncells per field, ghost cells per field,
 * leaf cells. */
int nrd_layout(const nrd_ctx* ctx, int64_t* ncells_host, int64_t* nghosts_host,
               int64_t* nleaf_host);

/* Material atomic number z per cell (hierarchy layout, ncells floats,
 * Sec. 3.1 sigma_a = z^3/T^3).  Copied; the caller may free z afterwards. */
int nrd_set_material(nrd_ctx* ctx, const float* z, cudaStream_t stream);

/* Ghost values of a state (Sec. 3.2 first-order physical ghosts, sibling
 * copies, Sec. 3.2.1 linear coarse-fine interpolation), written to gE, gT
 * (nghosts doubles each) and gz (nghosts floats, z of the ghost cell; may be
 * NULL).  u: 2*ncells doubles. */
int nrd_ghost_fill(nrd_ctx* ctx, const double* u, double* gE, double* gT, float* gz,
                   cudaStream_t stream);

/* Nonlinear residual (Eq. nonlinearsystem per unit volume):
 *   F = a0 u - b - dt f(u),  f from Eqs. E_td, T_td discretised as in
 * Sec. 3.2 with flux matching at coarse-fine faces (Sec. 3.2.1).
 *   u, b, F: 2*ncells doubles (b = history combination, e.g. u_n for BE).
 * F is 0 on covered cells. */
int nrd_residual(nrd_ctx* ctx, const double* u, const double* b, double a0, double dt, double* F,
                 cudaStream_t stream);

/* Jacobian-vector product J v of the residual at u.
 *   mode NRD_JV_ANALYTIC: exact tangent a0 v - dt f'(u) v (b, F0 unused,
 *                         may be NULL);
 *   mode NRD_JV_FD:       (F(u + eps v) - F0)/eps of Sec. 4.1 Eq. Jac-free
 *                         with the two-branch eps of Sec. 4.1 (b required;
 *                         F0 = F(u) required);
 *   mode NRD_JV_FROZEN:   the exact tangent at the state of the last
 *                         nrd_linearise (u, b, F0 unused and may be NULL;
 *                         NRD_ESTATE if there was none).
 * Jv: 2*ncells doubles, 0 on covered cells. */
int nrd_jv(nrd_ctx* ctx, const double* u, const double* v, const double* b, const double* F0,
           double a0, double dt, int mode, double* Jv, cudaStream_t stream);

/* Residual plus linearisation at u: writes F (as nrd_residual) and freezes
 * (a) the partial derivatives of every face flux and of the coupling term at
 * u (the exact Jacobian of Sec. 4.1, applied later by nrd_jv with
 * NRD_JV_FROZEN), and (b) the preconditioner of Sec. 4.2 at u (as
 * nrd_precond_setup).  u, b, F: 2*ncells doubles. */
int nrd_linearise(nrd_ctx* ctx, const double* u, const double* b, double a0, double dt, double* F,
                  cudaStream_t stream);

/* Adjoint of the residual at the state of the last nrd_linearise (the
 * transpose of the exact Jacobian of Sec. 4.1; not in the paper, used to
 * differentiate through implicit steps):
 *   JTw = (dF/du)^T w   (2*ncells doubles; 0 on covered cells)
 *   dz  = (dF/dz)^T w   (ncells doubles, may be NULL): sensitivity to the
 *                       material z of each cell (0 on covered cells).  Needs
 *                       the material partials, which nrd_linearise forms and
 *                       the Newton solves of nrd_newton / nrd_step do not
 *                       (NRD_ESTATE after those).
 * Gather form (no atomics), deterministic.  a0, dt as in the linearisation. */
int nrd_vjp(nrd_ctx* ctx, const double* w, double a0, double dt, double* JTw, double* dz,
            cudaStream_t stream);

/* Adjoint solve at the last nrd_linearise: J^T lam = g to
 * ||g - J^T lam|| <= rtol ||g|| (volume-weighted norms), by restarted GMRES
 * with the preconditioner of nrd_precond_apply on the right.  g, lam:
 * 2*ncells doubles.  Returns NRD_ENONCONV if the tolerance is not reached
 * within max_krylov iterations (lam holds the last iterate). */
int nrd_adjoint_solve(nrd_ctx* ctx, const double* g, double a0, double dt, double rtol,
                      double* lam, nrd_stats* stats, cudaStream_t stream);

/* The differencing parameter eps(u, v) of Sec. 4.1 (synchronises; result in
 * *eps_host). */
int nrd_fd_eps(nrd_ctx* ctx, const double* u, const double* v, double* eps_host,
               cudaStream_t stream);

/* Volume-weighted inner product over leaf cells of both fields
 * (synchronises; result in *out_host). */
int nrd_dot(nrd_ctx* ctx, const double* x, const double* y, double* out_host,
            cudaStream_t stream);

/* Freeze the preconditioner at the iterate u (Sec. 4.2): face D_E^k, D_T^k
 * for every AMR level, their coarsening to the GMG levels, and the P2 data.
 * beta = dt/a0 = (alpha+1)/(2 alpha+1) dt. */
int nrd_precond_setup(nrd_ctx* ctx, const double* u, double a0, double dt, cudaStream_t stream);

/* y = P^{-1} w = P2^{-1} (P1^{-1} w): one FAC V(nu1,nu2) cycle per diffusion
 * block (Algorithm 1) in the precision chosen by pc_precision, then the
 * cell-local 2x2 P2 solve in FP64.  w, y: 2*ncells doubles; y is 0 on
 * covered cells.  Requires nrd_precond_setup. */
int nrd_precond_apply(nrd_ctx* ctx, const double* w, double* y, cudaStream_t stream);

/* Solve F(u) = 0 (Eq. nonlinearsystem) by inexact Newton with
 * Eisenstat-Walker forcing, positivity-damped updates and right-
 * preconditioned restarted GMRES (Sec. 4.1-4.2).
 *   u: in initial guess, out solution (covered cells set to the mean of
 *      their children);  b: history combination;  stats: may be NULL.
 * Host-driven loop: synchronises once per Krylov iteration.
 * Returns NRD_ENONCONV if the Newton cap is hit (u holds the last iterate). */
int nrd_newton(nrd_ctx* ctx, double* u, const double* b, double a0, double dt, nrd_stats* stats,
               cudaStream_t stream);

/* One implicit time step (Sec. 3.3): backward Euler when u_nm1 is NULL
 * (Eq. be), else variable-step BDF2 (Eq. bdf2) with alpha = dt/dt_prev.
 *   u: in initial guess for u_{n+1}, out u_{n+1};  u_n, u_nm1: history. */
int nrd_step(nrd_ctx* ctx, double* u, const double* u_n, const double* u_nm1, double dt,
             double dt_prev, nrd_stats* stats, cudaStream_t stream);

/* nrd_step in two halves, so that work using the step's result can be
 * enqueued before the host waits for it.  nrd_step_begin checks the
 * arguments as nrd_step does and enqueues the whole step on `stream` (the
 * device-loop form; the host-driven form runs to the end here and keeps its
 * result).  Until nrd_step_end the step is pending: only nrd_time_derivative,
 * nrd_predict, nrd_lte, nrd_tag and nrd_dot may be called on the context, on
 * the same stream (they are ordered after the step); any other call returns
 * NRD_ESTATE, as does a second nrd_step_begin.  nrd_step_end waits for the
 * stream and returns what nrd_step would have (status and stats; stats may
 * be NULL); NRD_ESTATE if no step is pending.  u is complete when
 * nrd_step_end returns (stream-ordered uses may read it earlier). */
int nrd_step_begin(nrd_ctx* ctx, double* u, const double* u_n, const double* u_nm1, double dt,
                   double dt_prev, cudaStream_t stream);
int nrd_step_end(nrd_ctx* ctx, nrd_stats* stats);

/* Refinement indicators of Sec. 5 on every cell (covered cells use the mean
 * of their children): bit 0: tau^c > thr_c (curvature), bit 1: tau^g > thr_g
 * (gradient), bit 2: h |grad E| / E > thr_r.  tags: ncells bytes. */
int nrd_tag(nrd_ctx* ctx, const double* u, double thr_c, double thr_g, double thr_r,
            uint8_t* tags, cudaStream_t stream);

/* ------------------------------------------------------- regridding (Sec. 5)
 * Berger-Rigoutsos clustering of tagged cells into the boxes of a new
 * hierarchy on the same base grid (host C++; the paper names the algorithm
 * but gives no parameters).  Level by level from the coarsest, cells of the
 * new level l whose tag byte has a bit of tag_bits (cells absent from the
 * current level l inherit the tag of the finest current cell holding them)
 * are dilated by `buffer` cells, kept where the finer level is properly
 * nested (the cell's 26 neighbours inside the domain lie in the new level l),
 * and clustered: a box is shrunk to its tags and accepted when
 * tags/volume >= efficiency, it is properly nested and no side exceeds
 * max_side/2; otherwise it is cut at a zero of a tag signature (nearest the
 * middle, longest axis first), else at the strongest inflection of the
 * signatures, else in the middle of its longest side, each part keeping at
 * least min_side/2 planes unless proper nesting forces a narrower cut.  The
 * accepted boxes refined by 2 form level l+1.
 *   tags: device, ncells bytes (nrd_tag's output);  min_side, max_side: even,
 *   2 <= min_side <= max_side, in cells of the new level;  max_levels: 1 ..
 *   NRD_MAX_LEVELS, levels of the new hierarchy at most;  out (host):
 *   *nlevels_out levels, nboxes_out[max_levels] boxes per level (0 past the
 *   last), boxes_out[6*max_boxes] inclusive lo/hi per box in layout order
 *   (level 0 is the base box), *total_out the total box count (also set when
 *   it exceeds max_boxes, which returns NRD_EINVAL, as does a level whose
 *   index space has 2^31 cells or more).  Synchronises. */
int nrd_regrid_boxes(nrd_ctx* ctx, const uint8_t* tags, int tag_bits, int buffer,
                     double efficiency, int min_side, int max_side, int max_levels,
                     int max_boxes, int* nlevels_out, int* nboxes_out, int* boxes_out,
                     int* total_out);

/* Conservative linear refinement of Sec. 5: moves nvec state vectors from the
 * hierarchy of ctx_src to that of ctx_dst (same base grid).  The old vectors
 * are made composite first (covered cells := mean of their 8 children, on a
 * private copy: u_src is not modified).  A new cell that exists on the same
 * old level copies it; any other new cell takes, at its centre, the
 * minmod-limited linear reconstruction of the finest old cell holding it
 * (slope 0 along an axis where an old neighbour on that level is missing), so
 * leaf sums of V u are conserved and no value leaves the range of the old
 * neighbours (E, T stay positive).
 *   u_src: device, nvec x 2*ncells(src) doubles;  u_dst: device,
 *   nvec x 2*ncells(dst) doubles (every cell written).  Allocates and frees
 *   one device buffer: a copy of u_src, 4 bytes per new cell (the old cell it
 *   copies, or -1) and 44 bytes per reconstructed cell (the source list is
 *   built on host threads).  Synchronises.
 * Errors: NRD_ESTATE (a context without hierarchy), NRD_EINVAL (different
 * base grids, null pointers, nvec < 1, a new cell in no old cell),
 * NRD_ENOMEM, NRD_ECUDA; the message is stored in ctx_dst. */
int nrd_transfer(nrd_ctx* ctx_src, nrd_ctx* ctx_dst, const double* u_src, double* u_dst,
                 int nvec, cudaStream_t stream);

/* Tile-shape autotuner: times the linearisation stencil, one frozen-Jacobian
 * Jv and one preconditioner application at the state u for every supported
 * tile shape (3 repetitions each, CUDA events, after one warm-up) and keeps
 * the fastest for this context.  Synchronises.  tile_out_host[3] receives the
 * chosen shape and ms_out_host the best time (either may be NULL). */
int nrd_autotune(nrd_ctx* ctx, const double* u, const double* b, double a0, double dt,
                 int* tile_out_host, double* ms_out_host, cudaStream_t stream);

/* Allocation-free weighted inner product (no counterpart in the paper: an
 * interface addition for callers that cannot allocate device memory where
 * they need the product -- code under an external memory manager that owns
 * all device memory, or latency-critical paths where an allocation, which
 * can synchronise the device, is not acceptable).
 *   out[0] = sum_{i<n} w[i] (x[i] y[i] + x[n+i] y[n+i])   (device pointers:
 *   x, y: 2n doubles; w: n floats; out: one double, written asynchronously).
 * With w = leaf-cell volumes (0 on covered cells) this equals nrd_dot.
 * Needs no context and allocates nothing: its block partials live in a
 * file-scope device array of 65,536 doubles (512 KiB), held by every GPU that
 * loads the library until the process exits; n is therefore limited to
 * 2^26 = 67,108,864 (NRD_EINVAL beyond, nothing launched).  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) and
 * keeps it for later calls.  All calls share the array:
 * calls that overlap on the GPU (different streams without ordering) race
 * and give wrong results; calls ordered on one stream are safe.  Every
 * partial a call reads it has written itself, so nothing needs clearing.
 * Errors: NRD_EINVAL (null pointer, n < 0, n too large), NRD_ECUDA. */
int nrd_wdot_noalloc(const double* x, const double* y, const float* w, int64_t n, double* out,
                     cudaStream_t stream);

/* Check of the arithmetic the linearisation stencil uses instead of FP64
 * division and square root (no counterpart in the paper): for n doubles x
 * (device), out (device, 4n doubles) receives rcp(x), 1.0/x, rsqrt(x) and
 * 1.0/sqrt(x), where rcp and rsqrt are the PTX approximate FP64 reciprocal
 * (square root) refined with the second-order series of the correction and
 * the others CUDA's correctly rounded operations.  Relative error bound of
 * the refinements for 1e-300 < x < 1e300: 1e-15 (outside, the rounded
 * values).
 * Asynchronous.  Errors: NRD_EINVAL, NRD_ECUDA. */
int nrd_check_fastmath(const double* x, int64_t n, double* out, cudaStream_t stream);

/* Check of the FP64 -> FP32 narrowing the linearisation stencil forms with
 * integer instructions (no counterpart in the paper): for n doubles x
 * (device), out (device, 2n floats) receives the integer-instruction
 * round-to-nearest-even narrowing of each x and CUDA's __double2float_rn of
 * it; the two are bit-identical for every input.
 * Asynchronous.  Errors: NRD_EINVAL (null pointer, n < 0), NRD_ECUDA. */
int nrd_check_narrow(const double* x, int64_t n, float* out, cudaStream_t stream);

/* Machine rates used as roofline denominators, measured on the current
 * device: FP64 and FP32 FMA throughput in TFLOP/s (an FMA counts 2 flops;
 * independent FMA chains on every SM) and device-to-device copy bandwidth in
 * GB/s (read + write bytes of a 1 GiB copy), each the best of 3 runs timed with
 * CUDA events.  Allocates and frees 2 GiB of scratch.  Synchronises. */
int nrd_measure_peaks(double* fp64_tflops_host, double* fp32_tflops_host, double* copy_gbs_host,
                      cudaStream_t stream);

/* FP64 operation rates of the current device, for charging the divisions and
 * square roots of a kernel's algorithmic work (the paper has no counterpart):
 * rates_host[0] = fused multiply-adds per second, [1] = correctly rounded
 * divisions per second, [2] = correctly rounded square roots per second, each
 * from independent chains on every SM, the best of 3 runs timed with CUDA
 * events.  Allocates and frees a small scratch array.  Synchronises. */
int nrd_measure_fp64_ops(double* rates_host, cudaStream_t stream);

/* ---------------------------------------------- time-step control (Sec. 3.4-3.5) */
enum { NRD_DT_EPS = 0, NRD_DT_PC47 = 1 };

/* Time derivative at t_{n+1} from the left-hand side of Eq. bdf2 (Remark 2 of
 * Sec. 3.5): udot = (a0 u_{n+1} - (1+al) u_n + al^2/(1+al) u_{n-1}) / dt with
 * al = dt/dt_prev; backward Euler (u_nm1 NULL): (u_{n+1} - u_n)/dt.
 * All vectors 2*ncells doubles. */
int nrd_time_derivative(nrd_ctx* ctx, const double* u_np1, const double* u_n,
                        const double* u_nm1, double dt, double dt_prev, double* udot,
                        cudaStream_t stream);

/* Generalised leapfrog predictor (Eq. leapfrog), initial guess and error
 * reference: u_p = u_n + (1+al) dt udot_n - al^2 (u_n - u_{n-1}), al = dt/dt_prev. */
int nrd_predict(nrd_ctx* ctx, const double* u_n, const double* u_nm1, const double* udot_n,
                double dt, double dt_prev, double* u_p, cudaStream_t stream);

/* Local error estimate (Eq. bdf2le) e = (al+1)/(3 al+2) (u_{n+1} - u_p) in the
 * scaled max norm of Sec. 3.5: max over leaf cells of |e_E/(E+eta_E)| and
 * |e_T/(T+eta_T)|, with E, T from u_{n+1} (synchronises; *err_host). */
int nrd_lte(nrd_ctx* ctx, const double* u_np1, const double* u_p, double alpha, double eta_E,
            double eta_T, double* err_host, cudaStream_t stream);

/* Step-size controllers (host arithmetic, no context): NRD_DT_EPS, Eq. odets,
 * dt_{n+1} = (eps_t/err_n)^(1/3) dt_n; NRD_DT_PC47, Eq. pc47 with k kI = 0.4,
 * k kP = 0.7, k = 3: alpha_{n+1} = (eps_t/err_n)^kI (err_{n-1}/err_n)^kP alpha_n,
 * alpha_n = dt_n/dt_{n-1}, dt_{n+1} = alpha_{n+1} dt_n. */
int nrd_dt_control(int kind, double eps_t, double err_n, double err_nm1, double dt_n,
                   double dt_nm1, double* dt_next_host);

/* Smoother autotuner: for (nu1, nu2, coarse_sweeps) in {(1,0,2) (the paper's
 * V(1,0)), (1,1,2), (2,1,3), (2,2,4), (3,3,6)}, each with red-black
 * Gauss-Seidel and with damped Jacobi (the context's omega), times one
 * implicit step from u_n (BE when u_nm1 is NULL, else BDF2) with CUDA events
 * (second of two runs) and keeps the fastest combination that converges.
 * Synchronises; uses the context's scratch for the trial states.
 * nu_out_host[4] receives the choice: nu1, nu2, coarse_sweeps, smoother. */
int nrd_autotune_sweeps(nrd_ctx* ctx, const double* u_n, const double* u_nm1, double dt,
                        double dt_prev, int* nu_out_host, double* ms_out_host,
                        cudaStream_t stream);

/* ------------------------------------------------------- kernel timing
 * Optional CUDA-event timing of the library's kernel groups, recorded on the
 * stream each group is launched on (a start/stop event pair around every
 * launch).  Off by default; nrd_timing_enable(ctx, 1) turns it on and clears
 * the counters.  nrd_timing_read synchronises on the recorded events and
 * returns the summed device time (ms) and the number of launches. */
enum {
  NRD_TK_RESIDUAL = 0,   /* residual-only stencil (all levels, one launch) */
  NRD_TK_JV = 1,         /* analytic-tangent stencil */
  NRD_TK_JV_FD = 2,      /* finite-difference Jv stencil (incl. eps reduction) */
  NRD_TK_PC_APPLY = 3,   /* one P^{-1} application: FAC/GMG V-cycles + P2 */
  NRD_TK_PC_SETUP = 4,   /* coefficient freeze and coarsening */
  NRD_TK_ORTHO = 5,      /* CGS2 orthogonalisation of one Krylov vector */
  NRD_TK_GHOST = 6,      /* ghost fill of a direction vector */
  NRD_TK_TRANSFER = 7,   /* regrid transfer: composite copy + gather (ctx_dst) */
  NRD_TK_LINEARISE = 8,  /* residual + linearisation stencil (nrd_linearise, Newton) */
  NRD_TK_COUNT = 9
};
int nrd_timing_enable(nrd_ctx* ctx, int enable);
int nrd_timing_read(nrd_ctx* ctx, int group, double* ms_host, int64_t* launches_host);

#ifdef __cplusplus
}
#endif
#endif /* NRD_H */
