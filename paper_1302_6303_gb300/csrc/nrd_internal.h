// Internal declarations of the nrd CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nrd.h"

#define NRD_MAX_LEVELS 8
#define NRD_MAX_MG 12

// Ghost cell kinds (one per face cell of every patch).
enum : uint8_t { GT_NEUMANN = 0, GT_ROBIN = 1, GT_SIBLING = 2, GT_CF = 3 };

// Cell mask bits: bit 0 covered by a finer level; bit 1+f: face f of this leaf
// cell is the coarse side of a coarse-fine face (its flux comes from flux
// matching).  Faces f = 0..5 are x-, x+, y-, y+, z-, z+.
enum : uint8_t { MASK_COVERED = 1 };

struct PatchDev {
  int n[3];     // cells per axis
  int lo[3];    // level index of the first cell
  int level;
  int off;      // first cell (hierarchy layout)
  int goff;     // first ghost of this patch
  int fo[6];    // ghost offset of each face, relative to goff
};

struct TileDev {
  int patch;
  int i0, j0, k0;
  int k1;       // end plane (exclusive): k0 + tile_z, or less at the patch top
                // and for tiles split in two along z
  int flags;    // bit 0: every cell of the tile is covered
};

struct LevelInfo {
  int n[3];
  double h[3];
  int off, ncell;      // cell range of the level
  int p0, np;          // patch range
  int g0, ng;          // ghost range
  int t0, nt;          // tile range
};

// Host-built hierarchy metadata mirrored on the device.
struct Hier {
  int L = 0;
  LevelInfo lev[NRD_MAX_LEVELS];
  int N = 0, G = 0, nleaf = 0;
  int bc_type[6];
  double bc_R[6];
  int tile_x = 32, tile_y = 4, tile_z = 4;
  bool ragged = false;                    // a tile narrower than the tile shape in x or y
  std::vector<uint8_t> hmask;             // host copy of the cell masks

  // host copies
  std::vector<PatchDev> patches;
  std::vector<TileDev> tiles;
  std::vector<int> cell_patch;            // per cell
  std::vector<std::vector<int>> lmap;     // dense level maps (all levels, host)

  // device arrays
  PatchDev* d_patches = nullptr;
  TileDev* d_tiles = nullptr;
  uint8_t* d_mask = nullptr;              // N
  float* d_wvol = nullptr;                // N: cell volume for leaf cells, 0 if covered
  // ghosts
  uint8_t* d_gtype = nullptr;             // G
  uint8_t* d_gface = nullptr;             // G: face 0..5 of the owning patch
  int* d_gcell = nullptr;                 // G: interior cell adjacent to the ghost
  int* d_gzsrc = nullptr;                 // G: cell whose z the ghost takes
  int* d_gt0 = nullptr;                   // G+1: term ranges (sibling and CF)
  int* d_gidx = nullptr;                  // terms: source cells
  double* d_gw = nullptr;                 // terms: weights
  int nterm = 0;
  // flux matching: coarse leaf cells with coarse-side CF faces
  int nrf = 0;
  int* d_rf_cell = nullptr;               // nrf
  int* d_rf_off = nullptr;                // nrf+1, entries per cell
  int* d_rf_face = nullptr;               // entries: face 0..5 of the coarse cell
  int4* d_rf_g = nullptr;                 // entries: ghost slots of the 4 fine fluxes
  int* d_rf_level = nullptr;              // nrf: level of the coarse cell
  int rf_lstart[NRD_MAX_LEVELS + 1] = {}; // first entry of each level (cells ascend by level)
  // transposed ghost stencils (adjoint): cell -> (ghost, weight), and the
  // sibling / coarse-fine ghosts that take their z from a cell
  int* d_ts_off = nullptr;
  int* d_ts_g = nullptr;
  double* d_ts_w = nullptr;
  int* d_tz_off = nullptr;
  int* d_tz_g = nullptr;
  // coefficient coarsening (per level l < L-1; sources on level l+1)
  int ncz[NRD_MAX_LEVELS] = {0};
  int* d_cz_tgt[NRD_MAX_LEVELS] = {nullptr};
  int4* d_cz_src[NRD_MAX_LEVELS] = {nullptr};
  // dense level maps (device) for levels 0..L-2
  int* d_lmap[NRD_MAX_LEVELS] = {nullptr};
  // covered cells per level (for average-down): cell, first child, strides
  int ncov[NRD_MAX_LEVELS] = {0};
  int4* d_cov[NRD_MAX_LEVELS] = {nullptr};  // x: cell, y: child base, z: sx, w: sxy
  // leaf cells where fine-side CF ghosts live: none needed separately
};

// Parameters copied to kernels.
struct ModelParams {
  double k;
  int limiter;
  double bc_R[6];
  int bc_type[6];
};

struct nrd_ctx_s;

// host helpers (hier.cu)
int hier_build(Hier& H, int nlevels, const int* nboxes, const int* boxes, const int* bc_type,
               const double* bc_R, std::string& err);
int hier_upload(Hier& H, std::string& err);
// (re)build and upload the stencil tile list for shape tile_x x tile_y x tile_z
int hier_tiles(Hier& H, std::string& err);
void hier_free(Hier& H);

// Kernel launchers (k_stencil.cu)
// stencil modes; ST_JVF applies the Jacobian frozen by ST_LIN (jc, cc) to v;
// ST_LINZ is ST_LIN that also forms the partials with respect to z^3
// ST_LINF / ST_LINC (ST_RESF / ST_RESC): ST_LIN (ST_RESIDUAL) in two launches,
// every face once (face fluxes to StencilIO::pef), then the cell balance from them
enum { ST_RESIDUAL = 0, ST_JV = 1, ST_FD = 2, ST_LIN = 3, ST_JVF = 4, ST_LINZ = 5, ST_LINF = 6,
       ST_LINC = 7, ST_RESF = 8, ST_RESC = 9 };
struct StencilIO {
  const double* u;      // state (E then T)
  const double* v;      // direction (JV, FD)
  const double* gu;     // ghosts of u: [2][G]
  const double* gv;     // ghosts of v: [2][G]
  const double* b;      // history (RESIDUAL, FD)
  const double* F0;     // F(u) (FD)
  const double* eps;    // device scalar (FD)
  double a0, dt;
  double* out;          // F or Jv
  double* cfflux;       // [2][G] fine-side coarse-fine fluxes
  // ST_LIN outputs (face slots: [3N low faces | G boundary faces])
  double* jc;           // [6][3N+G] flux partial derivatives (5: d Phi_E / d z^3)
  double* craw;         // [2][3N+G] frozen D_E, D_T (Robin slots: D_b)
  double* cc;           // [3][N] coupling partials (E, T, z^3)
  double beta;          // dt / a0
  float* a32;           // [2][3N+G] scaled P1 coefficients (FP32 V-cycle), or
  double* a64;          //   the FP64 array when a32 is null
  double* p2;           // [3][N] P2 data (FP64 V-cycle), or
  float* p2f;           //   FP32 (FP32 V-cycle)
  const double* par;    // device [a0, dt, beta] overriding a0, dt, beta (or null)
  double* pef = nullptr;  // [2][3N+G] face fluxes: ST_LIN / ST_RESIDUAL run split when set
};
void launch_ghost_fill(const Hier& H, const ModelParams& mp, const float* z, const double* u,
                       double* g, int nonlinear, cudaStream_t s);
void launch_ghost_z(const Hier& H, const float* z, float* gz, cudaStream_t s);
// z3 (optional): z^3 in FP64 for the cells followed by the ghosts (N + G)
void launch_stencil(const Hier& H, const ModelParams& mp, const float* z, const float* gz,
                    int mode, const StencilIO& io, cudaStream_t s, const double* z3 = nullptr);
// z3[c] = z[c]^3 (cells), z3[N + g] = gz[g]^3 (ghosts), in FP64
void launch_cube(const Hier& H, const float* z, const float* gz, double* z3, cudaStream_t s);
void launch_reflux(const Hier& H, const StencilIO& io, int mode, cudaStream_t s);
void launch_jv_frozen(const Hier& H, const ModelParams& mp, const double* jc, const double* cc,
                      const StencilIO& io, cudaStream_t s);
// k_vjp.cu: JTw = (dF/du)^T w, dz = (dF/dz)^T w (dz may be null)
void launch_vjp(const Hier& H, const double* jc, const double* cc, const float* z, const double* w,
                double* lam, double* gam, double a0, double dt, double* out, double* dz,
                cudaStream_t s);
void launch_tag(const Hier& H, const double* E, const double* gE, double thr_c, double thr_g,
                double thr_r, const double* emax, uint8_t* tags, cudaStream_t s);
void launch_average_down(const Hier& H, double* x, int nfield, int fstride, cudaStream_t s);

// BLAS / reductions (k_blas.cu)
struct Reducer {
  int nblk = 0;
  double* d_part = nullptr;   // partials [nblk * NVMAX]
  double* d_res = nullptr;    // results [64]
  double* h_res = nullptr;    // pinned host mirror [64]
  unsigned* d_count = nullptr;  // last-block ticket counter (0 between launches)
  unsigned* d_bar = nullptr;    // grid barrier: arrival count, generation
  double* d_part2 = nullptr;    // second partial buffer (cooperative reductions)
  int* d_err = nullptr;         // set when a grid barrier wait gave up
  int coop_blocks = 0;          // grid of the cooperative CGS2 (0: unavailable)
};
int reducer_init(Reducer& R, int N);
void reducer_free(Reducer& R);
// res[slot] = sum over leaf cells of both fields of wvol * x * y
void launch_wdot(const Hier& H, Reducer& R, const double* x, const double* y, int slot,
                 cudaStream_t s);
// eps of Sec. 4.1 into R.d_res[slot]
void launch_fd_eps(const Hier& H, Reducer& R, const double* u, const double* v, double u_min,
                   int slot, cudaStream_t s);
// max |E| over leaf cells into R.d_res[slot]
void launch_emax(const Hier& H, Reducer& R, const double* E, int slot, cudaStream_t s);
// multi-dot: res[slot + i] = <w, V_i> for i < nv (V given as base + i*stride)
// w -= sum_i h[i] V_i  (h device)
void launch_axpy(int n, double a, const double* x, double* y, cudaStream_t s);
void launch_scale_dev(int n, const double* num, const double* den_sq, double* x, cudaStream_t s);
void launch_lincomb_dev(int n, double* x, const double* Z, long stride, int nv, const double* y,
                        cudaStream_t s);
void launch_zero_covered(const Hier& H, double* x, cudaStream_t s);
void launch_pos_cap(const Hier& H, Reducer& R, const double* u, const double* v, int slot,
                    cudaStream_t s);
// x += sum_q y_q Z_q over nv = (jd ? *jd : nv) columns, and the positivity cap
// of x at u (as launch_pos_cap) into res[slot]; one launch
void launch_lincomb_cap(const Hier& H, Reducer& R, double* x, const double* Z, long stride,
                        const int* jd, int nv, const double* y, const double* u, int slot,
                        cudaStream_t s);
// vector counts *jd + add (device values) for graph-captured solves
void launch_mdot_dyn(const Hier& H, Reducer& R, const double* w, const double* V, long stride,
                     const int* jd, int add, int slot, cudaStream_t s);
void launch_lincomb_dyn(int n, double* x, const double* Z, long stride, const int* jd,
                        const double* y, cudaStream_t s);
void launch_axpy_dev(int n, const double* a, const double* x, double* y, cudaStream_t s);
// res[slot] = volume-weighted <x, y> for vectors that vanish on covered cells
// (level volumes times FMA chains; one launch)
void launch_wdot_lv(const Hier& H, Reducer& R, const double* x, const double* y, int slot,
                    cudaStream_t s);
// CGS2 against the nv = (jd ? *jd : 0) + add columns of V: res[slot_h1..] and
// res[slot_h2..] receive the two passes' coefficients, res[slot_nrm] the
// squared norm of the orthogonalised w (three launches)
void launch_cgs2(const Hier& H, Reducer& R, double* w, const double* V, long stride,
                 const int* jd, int add, int slot_h1, int slot_h2, int slot_nrm, cudaStream_t s);
// one cooperative kernel: classical Gram-Schmidt with a second pass only
// when the first removed more than 1 - 1e-4 of |w|^2 (one grid-wide
// reduction in the common case, two otherwise; norms by the Pythagorean
// identity), writing V[nv] = w' / |w'|.  For vectors that vanish on covered
// cells.  always2: the second pass every time (CGS2).
// Returns NRD_ECUDA if a cooperative launch is not possible.
int launch_cgs2_coop(const Hier& H, Reducer& R, double* w, double* V, long stride, const int* jd,
                     int add, int slot_h1, int slot_h2, int slot_nrm, cudaStream_t s,
                     bool always2 = false);

// Preconditioner (k_pc.cu)
struct PcState;
int pc_alloc(PcState** ps, const Hier& H, const nrd_params& p, std::string& err);
void pc_free(PcState* ps);
int pc_setup(PcState* ps, const Hier& H, const ModelParams& mp, const double* u, const double* gu,
             const float* z, const float* gz, double a0, double dt, cudaStream_t s);
int pc_apply(PcState* ps, const Hier& H, const double* w, double* y, cudaStream_t s);
int pc_apply_ex(PcState* ps, const Hier& H, const double* w, double* y, bool transposed,
                cudaStream_t s);
// raw coefficient array [2][3N+G] the linearisation writes into
double* pc_craw(PcState* ps);
void pc_drop_graphs(PcState* ps);
void pc_set_sweeps(PcState* ps, int nu1, int nu2, int csw);
void pc_set_smoother(PcState* ps, int kind, double omega);
// coarsen (and, unless the linearisation already did, scale) after the raw
// coefficients were written at u
int pc_finish(PcState* ps, const Hier& H, const double* u, const float* z, double a0, double dt,
              bool from_lin, cudaStream_t s, bool beta_on_device = false);
// P^{-1} applied to column *jd of the basis V (columns jstride apart) into
// column *jd of Z, and into zcopy; jd is a device index (graph capture).
int pc_apply_indexed(PcState* ps, const Hier& H, const double* V, double* Z, const int* jd,
                     long jstride, double* zcopy, cudaStream_t s);
// device copy of beta = dt / a0 read by the set-up kernels
double* pc_beta_device(PcState* ps);
// where the linearisation writes scaled coefficients and P2 data
void pc_lin_targets(PcState* ps, float** a32, double** a64, double** p2, float** p2f);

#define CUDA_TRY(x)                                         \
  do {                                                      \
    cudaError_t e_ = (x);                                   \
    if (e_ != cudaSuccess) {                                \
      err = std::string(#x) + ": " + cudaGetErrorString(e_); \
      return NRD_ECUDA;                                     \
    }                                                       \
  } while (0)

// CUDA-event timing of kernel groups (off unless enabled).
struct Timer {
  bool on = false;
  std::vector<cudaEvent_t> ev[NRD_TK_COUNT];   // start/stop pairs
  size_t used[NRD_TK_COUNT] = {0};
  void begin(int k, cudaStream_t s) {
    if (!on) return;
    if (used[k] + 2 > ev[k].size()) {
      for (int i = 0; i < 64; i++) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ev[k].push_back(e);
      }
    }
    cudaEventRecord(ev[k][used[k]], s);
  }
  void end(int k, cudaStream_t s) {
    if (!on) return;
    cudaEventRecord(ev[k][used[k] + 1], s);
    used[k] += 2;
  }
  void reset() {
    for (int k = 0; k < NRD_TK_COUNT; k++) used[k] = 0;
  }
  void destroy() {
    for (int k = 0; k < NRD_TK_COUNT; k++) {
      for (auto e : ev[k]) cudaEventDestroy(e);
      ev[k].clear();
      used[k] = 0;
    }
  }
};

// The context behind the opaque nrd_ctx handle.
struct nrd_ctx {
  Timer timer;
  nrd_params p;
  ModelParams mp;
  Hier H;
  bool have_hier = false, have_mat = false;
  float* d_z = nullptr;        // N: material z
  float* d_gz = nullptr;       // G: z of ghost cells
  double* d_gu = nullptr;      // 2G: ghosts of the state
  double* d_gv = nullptr;      // 2G: ghosts of a direction
  double* d_cf = nullptr;      // 2G: fine-side coarse-fine fluxes
  double* d_tmp = nullptr;     // 2N scratch
  double* d_jc = nullptr;      // [6][3N+G] frozen flux partial derivatives
  double* d_pef = nullptr;     // [2][3N+G] face fluxes of the split linearisation
  double* d_cc = nullptr;      // [3][N] frozen coupling partials
  double* d_lam = nullptr;     // [2][3N+G] adjoint face scratch
  double* d_gam = nullptr;     // [3][G] adjoint ghost scratch
  double* d_z3 = nullptr;      // [N + G] z^3 of cells and ghost cells (FP64)
  bool lin_ready = false;
  bool lin_dz = false;         // the last linearisation holds the d/dz^3 partials
  Reducer R;
  PcState* pc = nullptr;
  bool pc_ready = false;
  // Krylov / Newton work space (allocated on first solver call)
  int kry_m = 0;
  double* d_V = nullptr;       // (m+1) x 2N
  double* d_Z = nullptr;       // m x 2N
  double* d_F = nullptr;       // 2N
  double* d_dx = nullptr;      // 2N
  double* d_w = nullptr;       // 2N
  double* d_r = nullptr;       // 2N
  double* d_b = nullptr;       // 2N
  double* d_small = nullptr;   // Hessenberg, rotations, g, y
  // Newton solve captured as one CUDA graph (nk_graph.cu)
  struct NkGraph* nk = nullptr;
  unsigned gen = 0;            // bumped whenever captured state may change
  // a step begun by nrd_step_begin and not yet ended: 0 none, 1 the Newton
  // graph in flight on pend_s, 2 finished by the host-driven loop
  int pend = 0;
  cudaStream_t pend_s = nullptr;
  int pend_rc = 0;
  nrd_stats pend_st{};
  std::string err;
};

// solver.cu
int solver_newton(nrd_ctx* c, double* u, const double* b, double a0, double dt, nrd_stats* st,
                  cudaStream_t s);
int solver_alloc(nrd_ctx* c);
int solver_adjoint(nrd_ctx* c, const double* g, double a0, double dt, double rtol, double* lam,
                   nrd_stats* st, cudaStream_t s);
void solver_free(nrd_ctx* c);
// nk_graph.cu: the whole Newton solve as one graph with device-side loops
// (analytic Jv form, timing off).  Same contract as solver_newton.
int nk_graph_solve(nrd_ctx* c, double* u, const double* b, double a0, double dt, nrd_stats* st,
                   cudaStream_t s);
// the same in two halves: enqueue without waiting, then wait and report
int nk_graph_launch(nrd_ctx* c, double* u, const double* b, double a0, double dt,
                    cudaStream_t s);
int nk_graph_collect(nrd_ctx* c, nrd_stats* st, cudaStream_t s);
// solver_newton in two halves (nrd_step_begin / nrd_step_end): the graph
// form is enqueued and collected later; the host-driven loop runs to the end
// in the first half and keeps its result for the second
int solver_newton_begin(nrd_ctx* c, double* u, const double* b, double a0, double dt,
                        cudaStream_t s);
int solver_newton_end(nrd_ctx* c, nrd_stats* st);
// capi.cu: NRD_OK when no step is pending, or when pending_ok and s is the
// stream of the pending step; otherwise NRD_ESTATE with the context's error set
int step_pending_check(nrd_ctx* c, bool pending_ok, cudaStream_t s);
void nk_graph_free(nrd_ctx* c);
// capi.cu helpers used by the solver
// par: optional device [a0, dt, beta] read instead of a0, dt (graph-captured
// solves).  The residual is bit-identical to the one ctx_linearise writes.
int ctx_residual(nrd_ctx* c, const double* u, const double* b, double a0, double dt, double* F,
                 bool fill_ghosts, cudaStream_t s, const double* par = nullptr);
// par: optional device [a0, dt, beta] read by the kernels instead of a0, dt
// (graph-captured solves; the frozen Jv and the linearisation only)
int ctx_jv(nrd_ctx* c, const double* u, const double* v, const double* b, const double* F0,
           double a0, double dt, int mode, double* Jv, bool fill_u_ghosts, cudaStream_t s,
           const double* par = nullptr);
int ctx_linearise(nrd_ctx* c, const double* u, const double* b, double a0, double dt, double* F,
                  cudaStream_t s, const double* par = nullptr, bool with_dz = false);

#ifdef __CUDACC__
// Candidate test of the positivity cap (Sec. 4.1 remark: lambda =
// min(1, 0.9 min over x_i < 0 of u_i / (-x_i))): true when x < 0 (not -0, not
// NaN) and u / (-x) may be below 2, read from the exponent fields with integer
// instructions.  An entry with u / (-x) > 2 cannot set lambda (0.9 x 2 > 1), so
// leaving it out gives the same lambda as the full minimum, and most entries of
// a Newton update are decided without FP64 instructions, which issue on
// GB300's narrow FP64 pipe.  (With e_u >= e_x + 2, u >= 2^(e_u - 1023) and
// -x < 2^(e_x - 1022), so u / (-x) > 2.)  A negative u always counts: it
// makes lambda <= 0, the failure the callers report.
__device__ __forceinline__ bool cap_candidate(double u, double x) {
  const unsigned xh = (unsigned)__double2hiint(x), xl = (unsigned)__double2loint(x);
  const unsigned ax = xh & 0x7fffffffu;
  if (!(xh >> 31) || (ax | xl) == 0u) return false;                       // x >= 0 or -0
  if (ax > 0x7ff00000u || (ax == 0x7ff00000u && xl != 0u)) return false;  // NaN
  const unsigned uh = (unsigned)__double2hiint(u);
  if (uh >> 31) return true;
  return (uh >> 20) <= (ax >> 20) + 1u;
}
// a thread's best candidate so far as the pair (a, b) = (u, -x): a/b < c/d
// compared as a d < c b (both b > 0), one division at the end
__device__ __forceinline__ void cap_take(double u, double x, bool& have, double& ba, double& bb) {
  const double b = -x;
  if (!have || u * bb < ba * b) { ba = u; bb = b; have = true; }
}
#endif
