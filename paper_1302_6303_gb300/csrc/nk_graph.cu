// The inexact Newton solve of one implicit step (Sec. 4.1-4.3) as ONE CUDA
// graph with device-side control flow, so that a time step costs one graph
// launch and one read-back instead of a host round trip per Krylov
// iteration:
//
//   evaluate F(u^0); init                                  (stop, eta_0)
//   while (||F|| > stop and k < max_newton):               Newton
//     r_0 = -F, v_0 = r_0/||r_0||, dx = 0
//     while (not converged and Krylov its < max_krylov):   GMRES cycles
//       if (restart): r = -F - J dx, v_0 = r/||r||
//       while (|g_{j+1}| > tol and j < m):                 Arnoldi steps
//         z_j = P^{-1} v_j; w = J z_j; CGS2 against v_0..v_j;
//         v_{j+1} = w/||w||; Givens update of the least-squares problem
//       dx += sum_i y_i z_i (back substitution on the device)
//     lambda = min(1, 0.9 min u/(-dx)); u += lambda dx    (positivity cap)
//     if (lambda = 1 and the solve aimed at the forcing floor):
//       F(u) alone; re-linearise only if ||F|| > stop
//     else re-linearise at u
//     Eisenstat-Walker forcing eta_{k+1}
//   covered cells := mean of their children
//
// The loops are conditional WHILE / IF graph nodes whose conditions are set
// by one-thread control kernels; a0, dt and beta = dt/a0 are device values,
// so one instantiated graph serves every step size.  Every control kernel
// also counts against a global cap of kMaxTicks loop iterations and ends
// all loops when it is reached (a bound independent of the tolerances).
// The arithmetic is that of the host-driven solver in solver.cu (same
// kernels, same reduction orders, the same forcing and cap rules).
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "nrd_internal.h"

namespace {

constexpr int kMaxTicks = 1 << 16;
constexpr int NVMAXG = 32;
// result slots in the reducer's device array (disjoint from solver.cu's)
enum { G_F = 100, G_CAP = 101, G_R = 102, G_NRM = 103, G_H1 = 104, G_H2 = 140 };
enum { NK_NAN = 1, NK_NEG = 2 };

struct NkCtl {
  double a0, dt, beta;            // read by the stencil kernels (par)
  double fn, fn0, fold, stop, eta, tol, lam, min_lambda, gres, rn2;
  double rtol, atol, eta_max, ew_gamma, eta0;
  int j, total, it, krylov, flags, ticks;
  int max_newton, max_krylov;
  int cycles, restarts;           // executions of the cycle and restart bodies
  int nres, nlin;                 // residual-only and linearising evaluations in the loop
  int lin_last;                   // the last evaluation linearised (frozen J at u)
};

struct SmallG {
  double* Hm;   // (m+1) x m, column j at Hm + (m+1) j
  double* cs;
  double* sn;
  double* g;    // m+1
  double* y;    // m
};

__device__ __forceinline__ bool tick(NkCtl* c) { return ++c->ticks < kMaxTicks; }

__global__ void k_nk_params(NkCtl* c, double a0, double dt, double rtol, double atol,
                            double eta_max, double ew_gamma, double eta0, int max_newton,
                            int max_krylov, double* dbeta) {
  c->a0 = a0;
  c->dt = dt;
  c->beta = dt / a0;
  *dbeta = c->beta;
  c->rtol = rtol;
  c->atol = atol;
  c->eta_max = eta_max;
  c->ew_gamma = ew_gamma;
  c->eta0 = eta0;
  c->max_newton = max_newton;
  c->max_krylov = max_krylov;
  c->ticks = 0;
}

__global__ void k_nk_init(NkCtl* c, const double* res, cudaGraphConditionalHandle hN) {
  const double fn = sqrt(res[G_F]);
  c->fn = fn;
  c->fn0 = fn;
  c->stop = c->rtol * fn + c->atol;
  c->eta = c->eta0;
  c->it = 0;
  c->krylov = 0;
  c->cycles = 0;
  c->restarts = 0;
  c->min_lambda = 1.0;
  c->lam = 1.0;
  c->nres = 0;
  c->nlin = 0;
  c->lin_last = 1;
  c->flags = isfinite(fn) ? 0 : NK_NAN;
  const bool go = tick(c) && !c->flags && fn > c->stop && c->it < c->max_newton;
  cudaGraphSetConditional(hN, go ? 1u : 0u);
}

// restart from the true residual r = -F - J dx (its squared norm in res)
__global__ void k_gm_restart(NkCtl* c, SmallG S, int m, const double* res) {
  c->restarts += 1;
  c->rn2 = res[G_R];
  c->j = 0;
  for (int i = 0; i <= m; i++) S.g[i] = 0.0;
  S.g[0] = sqrt(c->rn2);
  c->gres = S.g[0];
  if (!isfinite(c->gres)) c->flags |= NK_NAN;
}

__global__ void k_arn_start(NkCtl* c, int m, cudaGraphConditionalHandle hA) {
  const bool go = tick(c) && !c->flags && c->gres > c->tol && c->j < m &&
                  c->total < c->max_krylov;
  cudaGraphSetConditional(hA, go ? 1u : 0u);
}

// v = sign r / sqrt(nrm2), into column (*jd + add) of V (jd may be null)
__global__ void k_normalize_g(int n, const double* r, double* V, long stride, const int* jd,
                              int add, const double* nrm2, double sign) {
  double* v = V + (long)((jd ? *jd : 0) + add) * stride;
  __shared__ double sc_s;
  if (threadIdx.x == 0) {
    const double d = sqrt(*nrm2);
    sc_s = (d > 0.0) ? sign / d : 0.0;
  }
  __syncthreads();
  const double sc = sc_s;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v[i] = sc * r[i];
}

// r = -F - Ax
__global__ void k_resid_g(int n, const double* F, const double* Ax, double* r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    r[i] = -F[i] - Ax[i];
}

// Hessenberg column j from the two CGS passes, Givens update, residual
// estimate |g_{j+1}|; j and the iteration count advance.
__global__ void k_arnoldi_g(NkCtl* c, SmallG S, int m, const double* res, const int* err,
                            cudaGraphConditionalHandle hA) {
  const int j = c->j;
  double* col = S.Hm + (size_t)(m + 1) * j;
  for (int i = 0; i <= j; i++) col[i] = res[G_H1 + i] + res[G_H2 + i];
  col[j + 1] = sqrt(res[G_NRM]);
  for (int i = 0; i < j; i++) {
    double a = col[i], b = col[i + 1];
    col[i] = S.cs[i] * a + S.sn[i] * b;
    col[i + 1] = -S.sn[i] * a + S.cs[i] * b;
  }
  double a = col[j], b = col[j + 1];
  double den = sqrt(a * a + b * b);
  double cs = (den > 0.0) ? a / den : 1.0;
  double sn = (den > 0.0) ? b / den : 0.0;
  S.cs[j] = cs;
  S.sn[j] = sn;
  col[j] = den;
  col[j + 1] = 0.0;
  double gj = S.g[j];
  S.g[j + 1] = -sn * gj;
  S.g[j] = cs * gj;
  c->gres = fabs(S.g[j + 1]);
  c->j = j + 1;
  c->total += 1;
  if (!isfinite(c->gres) || *err) c->flags |= NK_NAN;
  const bool go = tick(c) && !c->flags && c->gres > c->tol && c->j < m &&
                  c->total < c->max_krylov;
  cudaGraphSetConditional(hA, go ? 1u : 0u);
}

// Predicted convergence: a full step (lambda = 1) whose linear solve was
// asked to reach the forcing floor (tol = eta ||F|| = stop/2) leaves a new
// residual of about stop/2 plus the nonlinear remainder, so the iterate is
// probably the last one: evaluate F alone first and linearise only if
// ||F|| > stop after all (the residual is bit-identical either way).
__device__ __forceinline__ bool nk_predict(const NkCtl* c) {
  return !c->flags && c->lam == 1.0 && c->tol <= 0.5 * c->stop * (1.0 + 1e-12);
}

// after the residual-only evaluation: linearise unless converged
__global__ void k_nk_checkres(NkCtl* c, const double* res, cudaGraphConditionalHandle hL) {
  const bool need = !(sqrt(res[G_F]) <= c->stop);
  if (need) {
    c->lin_last = 1;
    c->nlin += 1;
  }
  cudaGraphSetConditional(hL, need ? 1u : 0u);
}

// new residual norm, Eisenstat-Walker forcing (Kelley's safeguarded choice)
__global__ void k_nk_update(NkCtl* c, const double* res, cudaGraphConditionalHandle hN) {
  c->fold = c->fn;
  const double fn = sqrt(res[G_F]);
  c->fn = fn;
  c->it += 1;
  if (!isfinite(fn)) c->flags |= NK_NAN;
  if (!c->flags) {
    const double rat = fn / c->fold;
    const double g = c->ew_gamma, eta = c->eta;
    const double etaA = g * rat * rat;
    double etaN;
    if (g * eta * eta <= 0.1) etaN = fmin(c->eta_max, etaA);
    else etaN = fmin(c->eta_max, fmax(etaA, g * eta * eta));
    c->eta = fmin(c->eta_max, fmax(etaN, 0.5 * c->stop / fn));
  }
  const bool go = tick(c) && !c->flags && fn > c->stop && c->it < c->max_newton;
  cudaGraphSetConditional(hN, go ? 1u : 0u);
}

int grid1(long n) {
  long b = (n + 255) / 256;
  return (int)std::max(1L, std::min(b, 152L * 8));
}

// ---- vector kernels fused with the one-thread control steps around them
// (the graph form; the host-driven loop in solver.cu does the same
// arithmetic in separate kernels and on the host).

// block minimum (tree), valid in every thread; blockDim.x a power of two
__device__ double blk_min(double v, double* sh) {
  const int t = threadIdx.x;
  __syncthreads();
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (t < s) sh[t] = fmin(sh[t], sh[t + s]);
    __syncthreads();
  }
  return sh[0];
}

// true in the block that arrives last (ticket on a counter left at 0)
__device__ bool last_block(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  return last;
}

// The start of a Newton iteration's GMRES: dx = 0, v_0 = -F / ||F|| and, in
// block 0, the solve's set-up: tolerance eta ||F||, least-squares right-hand
// side g = ||r_0|| e_0, the first cycle (no restart).
__global__ void k_gm_start_g(NkCtl* c, SmallG S, int m, int n, const double* __restrict__ F,
                             double* __restrict__ V, double* __restrict__ dx,
                             cudaGraphConditionalHandle hC, cudaGraphConditionalHandle hR) {
  const double fn = c->fn;
  __shared__ double sc_s;
  if (threadIdx.x == 0) {
    const double d = sqrt(fn * fn);
    sc_s = (d > 0.0) ? -1.0 / d : 0.0;
  }
  __syncthreads();
  const double sc = sc_s;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    V[i] = sc * F[i];
    dx[i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->rn2 = fn * fn;
    c->tol = c->eta * fn;
    c->j = 0;
    c->total = 0;
    for (int i = 0; i <= m; i++) S.g[i] = 0.0;
    S.g[0] = sqrt(c->rn2);
    c->gres = S.g[0];
    cudaGraphSetConditional(hC, tick(c) ? 1u : 0u);
    cudaGraphSetConditional(hR, 0u);
  }
}

// The end of a GMRES cycle: every block solves the k x k triangular system
// R y = g (back substitution) into shared memory, dx += Z y with the
// positivity cap of dx at u (as k_lincomb_cap), and the last block finishes
// the cap's minimum into res[G_CAP] and decides whether another cycle
// (restart) follows.  256 threads.
__global__ void __launch_bounds__(256) k_cycle_update_g(
    NkCtl* c, SmallG S, int m, const uint8_t* __restrict__ mask, int N,
    double* __restrict__ dx, const double* __restrict__ Z, long stride,
    const double* __restrict__ u, double* part, unsigned* counter, double* res,
    cudaGraphConditionalHandle hC, cudaGraphConditionalHandle hR) {
  __shared__ double ys[NVMAXG];
  __shared__ double sh[256];
  const int k = min(c->j, NVMAXG);
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; i--) {
      double s = S.g[i];
      for (int t = i + 1; t < k; t++) s -= S.Hm[i + (size_t)(m + 1) * t] * ys[t];
      ys[i] = s / S.Hm[i + (size_t)(m + 1) * i];
    }
    if (blockIdx.x == 0)
      for (int i = 0; i < k; i++) S.y[i] = ys[i];
  }
  __syncthreads();
  double ba = 1.0, bb = 0.0;
  bool have = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    // u and the mask are fetched with dx and Z, not after the sign test
    const double u0 = u[i], u1 = u[N + i];
    const bool leaf = !(mask[i] & MASK_COVERED);
    double s0 = dx[i], s1 = dx[N + i];
    // 4 basis vectors in flight; fuller unrolling takes the registers of a
    // fourth resident block (80 instead of 60), and the grid then runs in two waves
#pragma unroll 4
    for (int q = 0; q < k; q++) {
      s0 += ys[q] * Z[q * stride + i];
      s1 += ys[q] * Z[q * stride + N + i];
    }
    dx[i] = s0;
    dx[N + i] = s1;
    // candidates screened with integer instructions (cap_candidate)
    if (leaf && cap_candidate(u0, s0)) cap_take(u0, s0, have, ba, bb);
    if (leaf && cap_candidate(u1, s1)) cap_take(u1, s1, have, ba, bb);
  }
  double r = DBL_MAX;
  if (__syncthreads_or(have)) {
    double mq = DBL_MAX;
    if (have) mq = ba / bb;
    r = blk_min(mq, sh);
  }
  if (threadIdx.x == 0) part[blockIdx.x] = r;
  if (last_block(counter)) {
    double acc = DBL_MAX;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) acc = fmin(acc, __ldcg(&part[b]));
    const double mm = blk_min(acc, sh);
    if (threadIdx.x == 0) {
      res[G_CAP] = mm;
      *counter = 0u;
      c->cycles += 1;
      const bool conv = c->gres <= c->tol;
      const bool go = tick(c) && !conv && !c->flags && c->total < c->max_krylov;
      cudaGraphSetConditional(hC, go ? 1u : 0u);
      cudaGraphSetConditional(hR, go ? 1u : 0u);
    }
  }
}

// u += lambda dx with lambda = min(1, 0.9 cap) (the positivity-constrained
// step, Sec. 4.1 remark) and, in block 0, the step's bookkeeping (lambda,
// its minimum, a vanished cap, the Krylov count) and the last-iterate
// prediction (nk_predict).
__global__ void k_nk_step_g(NkCtl* c, const double* res, int n, const double* __restrict__ dx,
                            double* __restrict__ u, cudaGraphConditionalHandle hP,
                            cudaGraphConditionalHandle hL) {
  double lam = fmin(1.0, 0.9 * res[G_CAP]);
  const bool neg = !(lam > 0.0);
  if (neg) lam = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    u[i] += lam * dx[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (neg) c->flags |= NK_NEG;
    c->lam = lam;
    c->min_lambda = fmin(c->min_lambda, lam);
    c->krylov += c->total;
    const bool pred = nk_predict(c);
    c->lin_last = pred ? 0 : 1;
    if (pred) c->nres += 1;
    else c->nlin += 1;
    cudaGraphSetConditional(hP, pred ? 1u : 0u);
    cudaGraphSetConditional(hL, pred ? 0u : 1u);
  }
}

}  // namespace

struct NkGraph {
  unsigned gen = 0;
  const double* b = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  NkCtl* ctl = nullptr;      // device
  NkCtl* h_ctl = nullptr;    // pinned host mirror
  double* uw = nullptr;      // the iterate (2N)
  double* zf = nullptr;      // the current preconditioned direction (2N)
  cudaStream_t cs[4] = {nullptr, nullptr, nullptr, nullptr};
  // kernel nodes per execution of: the top level, the Newton body, the cycle
  // body, the restart body, the Arnoldi body, the residual-only evaluation,
  // the linearising evaluation
  long kn[7] = {0, 0, 0, 0, 0, 0, 0};
};

namespace {

// Add a conditional node at the current position of the capture on `s`;
// returns its body graph (to be captured on another stream).
cudaError_t add_conditional(cudaStream_t s, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams p = {};   // aggregate initialisation: all bytes zero
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                             cudaStreamSetCaptureDependencies);
}

struct Builder {
  nrd_ctx* c;
  NkGraph* G;
  const double* b;
  cudaGraphConditionalHandle hN, hC, hR, hA, hP, hL;
  cudaError_t err = cudaSuccess;
  int rc = NRD_OK;

  SmallG small() const {
    const int m = c->kry_m;
    SmallG S;
    S.Hm = c->d_small;
    S.cs = S.Hm + (m + 1) * m;
    S.sn = S.cs + m;
    S.g = S.sn + m;
    S.y = S.g + m + 1;
    return S;
  }
  const double* par() const { return &G->ctl->a0; }
  double* res() const { return c->R.d_res; }

  // F(u), the frozen Jacobian and the preconditioner at u; ||F||^2 -> G_F
  void evaluate(cudaStream_t s) {
    int r = ctx_linearise(c, G->uw, b, 1.0, 1.0, c->d_F, s, par());
    if (r != NRD_OK) rc = r;
    launch_wdot_lv(c->H, c->R, c->d_F, c->d_F, G_F, s);
  }

  void jv(const double* v, double* out, cudaStream_t s) {
    int r = ctx_jv(c, G->uw, v, b, c->d_F, 1.0, 1.0, NRD_JV_FROZEN, out, false, s, par());
    if (r != NRD_OK) rc = r;
  }

  // one Arnoldi step (body of the innermost loop)
  void arnoldi(cudaStream_t s) {
    Hier& H = c->H;
    const int n2 = 2 * H.N;
    const long stride = n2;
    const int m = c->kry_m;
    int r = pc_apply_indexed(c->pc, H, c->d_V, c->d_Z, &G->ctl->j, stride, G->zf, s);
    if (r != NRD_OK) rc = r;
    jv(G->zf, c->d_w, s);
    const int* jd = &G->ctl->j;
    if (launch_cgs2_coop(H, c->R, c->d_w, c->d_V, stride, jd, 1, G_H1, G_H2, G_NRM, s) !=
        NRD_OK) {
      cudaGetLastError();
      launch_cgs2(H, c->R, c->d_w, c->d_V, stride, jd, 1, G_H1, G_H2, G_NRM, s);
      k_normalize_g<<<grid1(n2), 256, 0, s>>>(n2, c->d_w, c->d_V, stride, jd, 1, res() + G_NRM,
                                              1.0);
    }
    k_arnoldi_g<<<1, 1, 0, s>>>(G->ctl, small(), m, res(), c->R.d_err, hA);
  }

  // restart from the true residual (body of the IF node)
  void restart(cudaStream_t s) {
    Hier& H = c->H;
    const int n2 = 2 * H.N;
    jv(c->d_dx, c->d_w, s);
    k_resid_g<<<grid1(n2), 256, 0, s>>>(n2, c->d_F, c->d_w, c->d_r);
    launch_wdot_lv(H, c->R, c->d_r, c->d_r, G_R, s);
    k_gm_restart<<<1, 1, 0, s>>>(G->ctl, small(), c->kry_m, res());
    k_normalize_g<<<grid1(n2), 256, 0, s>>>(n2, c->d_r, c->d_V, n2, nullptr, 0, &G->ctl->rn2, 1.0);
  }

  bool ok(cudaError_t e) {
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    return e == cudaSuccess;
  }

  // capture `fn` into the body graph `body` on stream index `lvl`; *nk
  // receives the number of kernel nodes directly in the body
  template <class Fn>
  void capture_body(cudaGraph_t body, int lvl, long* nk, Fn fn) {
    cudaStream_t s = G->cs[lvl];
    if (!ok(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal)))
      return;
    fn(s);
    cudaGraph_t out;
    if (ok(cudaStreamEndCapture(s, &out))) *nk = count_kernels(body);
  }

  long count_kernels(cudaGraph_t g) {
    size_t n = 0;
    if (!ok(cudaGraphGetNodes(g, nullptr, &n))) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n == 0 || !ok(cudaGraphGetNodes(g, nodes.data(), &n))) return 0;
    long k = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (ok(cudaGraphNodeGetType(nd, &t)) && t == cudaGraphNodeTypeKernel) k++;
    }
    return k;
  }

  // the GMRES cycle loop body
  void cycle(cudaStream_t s) {
    cudaGraph_t bR, bA;
    if (!ok(add_conditional(s, hR, cudaGraphCondTypeIf, &bR))) return;
    capture_body(bR, 3, &G->kn[3], [&](cudaStream_t s3) { restart(s3); });
    k_arn_start<<<1, 1, 0, s>>>(G->ctl, c->kry_m, hA);
    if (!ok(add_conditional(s, hA, cudaGraphCondTypeWhile, &bA))) return;
    capture_body(bA, 3, &G->kn[4], [&](cudaStream_t s3) { arnoldi(s3); });
    const int n2 = 2 * c->H.N;
    // back substitution, dx += Z y with the positivity cap of dx at u (the
    // last cycle's stands), the cycle-end test
    k_cycle_update_g<<<c->R.nblk, 256, 0, s>>>(G->ctl, small(), c->kry_m, c->H.d_mask, c->H.N,
                                               c->d_dx, c->d_Z, n2, G->uw, c->R.d_part,
                                               c->R.d_count, res(), hC, hR);
  }

  // the Newton loop body
  void newton(cudaStream_t s) {
    Hier& H = c->H;
    const int n2 = 2 * H.N;
    k_gm_start_g<<<grid1(n2), 256, 0, s>>>(G->ctl, small(), c->kry_m, n2, c->d_F, c->d_V,
                                           c->d_dx, hC, hR);
    cudaGraph_t bC;
    if (!ok(add_conditional(s, hC, cudaGraphCondTypeWhile, &bC))) return;
    capture_body(bC, 2, &G->kn[2], [&](cudaStream_t s2) { cycle(s2); });
    k_nk_step_g<<<grid1(n2), 256, 0, s>>>(G->ctl, res(), n2, c->d_dx, G->uw, hP, hL);
    cudaGraph_t bP, bL;
    if (!ok(add_conditional(s, hP, cudaGraphCondTypeIf, &bP))) return;
    capture_body(bP, 2, &G->kn[5], [&](cudaStream_t s2) {
      int r = ctx_residual(c, G->uw, b, 1.0, 1.0, c->d_F, true, s2, par());
      if (r != NRD_OK) rc = r;
      launch_wdot_lv(c->H, c->R, c->d_F, c->d_F, G_F, s2);
      k_nk_checkres<<<1, 1, 0, s2>>>(G->ctl, res(), hL);
    });
    if (!ok(add_conditional(s, hL, cudaGraphCondTypeIf, &bL))) return;
    capture_body(bL, 2, &G->kn[6], [&](cudaStream_t s2) { evaluate(s2); });
    k_nk_update<<<1, 1, 0, s>>>(G->ctl, res(), hN);
  }

  int build() {
    if (!ok(cudaGraphCreate(&G->graph, 0))) return NRD_ECUDA;
    const unsigned dflt = cudaGraphCondAssignDefault;
    if (!ok(cudaGraphConditionalHandleCreate(&hN, G->graph, 0, dflt)) ||
        !ok(cudaGraphConditionalHandleCreate(&hC, G->graph, 0, dflt)) ||
        !ok(cudaGraphConditionalHandleCreate(&hR, G->graph, 0, dflt)) ||
        !ok(cudaGraphConditionalHandleCreate(&hA, G->graph, 0, dflt)) ||
        !ok(cudaGraphConditionalHandleCreate(&hP, G->graph, 0, dflt)) ||
        !ok(cudaGraphConditionalHandleCreate(&hL, G->graph, 0, dflt)))
      return NRD_ECUDA;
    cudaStream_t s = G->cs[0];
    if (!ok(cudaStreamBeginCaptureToGraph(s, G->graph, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal)))
      return NRD_ECUDA;
    evaluate(s);
    k_nk_init<<<1, 1, 0, s>>>(G->ctl, res(), hN);
    cudaGraph_t bN;
    if (ok(add_conditional(s, hN, cudaGraphCondTypeWhile, &bN)))
      capture_body(bN, 1, &G->kn[1], [&](cudaStream_t s1) { newton(s1); });
    launch_average_down(c->H, G->uw, 2, c->H.N, s);
    cudaGraph_t out;
    if (ok(cudaStreamEndCapture(s, &out))) G->kn[0] = count_kernels(G->graph);
    if (err != cudaSuccess || rc != NRD_OK) return rc != NRD_OK ? rc : NRD_ECUDA;
    if (!ok(cudaGraphInstantiate(&G->exec, G->graph, 0))) return NRD_ECUDA;
    return NRD_OK;
  }
};

void destroy(NkGraph* G) {
  if (!G) return;
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->graph) cudaGraphDestroy(G->graph);
  if (G->ctl) cudaFree(G->ctl);
  if (G->h_ctl) cudaFreeHost(G->h_ctl);
  if (G->uw) cudaFree(G->uw);
  if (G->zf) cudaFree(G->zf);
  for (auto& q : G->cs)
    if (q) cudaStreamDestroy(q);
  delete G;
}

}  // namespace

void nk_graph_free(nrd_ctx* c) {
  destroy(c->nk);
  c->nk = nullptr;
}

int nk_graph_solve(nrd_ctx* c, double* u, const double* b, double a0, double dt, nrd_stats* st,
                   cudaStream_t s) {
  const int rc = nk_graph_launch(c, u, b, a0, dt, s);
  if (rc != NRD_OK) return rc;
  return nk_graph_collect(c, st, s);
}

// Enqueue the whole Newton solve (graph, result copy, control read-back) on
// s without waiting for it.
int nk_graph_launch(nrd_ctx* c, double* u, const double* b, double a0, double dt,
                    cudaStream_t s) {
  int rc = solver_alloc(c);
  if (rc != NRD_OK) return rc;
  if (c->kry_m > NVMAXG - 1) {
    c->err = "graph form needs restart < 32";
    return NRD_EINVAL;
  }
  Hier& H = c->H;
  const size_t n2 = 2 * (size_t)H.N;
  NkGraph* G = c->nk;
  if (G && (G->gen != c->gen || G->b != b)) {
    nk_graph_free(c);
    G = nullptr;
  }
  if (!G) {
    G = new NkGraph();
    bool okm = cudaMalloc(&G->ctl, sizeof(NkCtl)) == cudaSuccess &&
               cudaMallocHost(&G->h_ctl, sizeof(NkCtl)) == cudaSuccess &&
               cudaMalloc(&G->uw, n2 * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&G->zf, n2 * sizeof(double)) == cudaSuccess;
    for (auto& q : G->cs)
      okm = okm && cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) == cudaSuccess;
    if (!okm) {
      destroy(G);
      c->err = "allocation of the Newton graph work space failed";
      return NRD_ENOMEM;
    }
    G->gen = c->gen;
    G->b = b;
    // one eager linearisation first: sets kernel attributes outside capture
    // and leaves valid preconditioner data behind
    cudaMemcpyAsync(G->uw, u, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    rc = ctx_linearise(c, G->uw, b, a0, dt, c->d_F, s);
    // and one frozen Jv: first launches set kernel attributes, which must
    // not happen inside the capture
    if (rc == NRD_OK)
      rc = ctx_jv(c, G->uw, c->d_F, b, c->d_F, a0, dt, NRD_JV_FROZEN, c->d_w, false, s);
    if (rc == NRD_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = NRD_ECUDA;
    if (rc == NRD_OK) {
      Builder B{c, G, b};
      rc = B.build();
      if (rc != NRD_OK) {
        c->err = std::string("building the Newton graph failed: ") +
                 (B.err != cudaSuccess ? cudaGetErrorString(B.err) : "launch error");
        cudaGetLastError();
      }
    }
    if (rc != NRD_OK) {
      destroy(G);
      return rc;
    }
    c->nk = G;
  }
  cudaMemcpyAsync(G->uw, u, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  k_nk_params<<<1, 1, 0, s>>>(G->ctl, a0, dt, c->p.rtol, c->p.atol, c->p.eta_max, c->p.ew_gamma,
                              c->p.eta0, c->p.max_newton, c->p.max_krylov,
                              pc_beta_device(c->pc));
  if (cudaGraphLaunch(G->exec, s) != cudaSuccess) {
    c->err = "launch of the Newton graph failed";
    return NRD_ECUDA;
  }
  cudaMemcpyAsync(u, G->uw, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(G->h_ctl, G->ctl, sizeof(NkCtl), cudaMemcpyDeviceToHost, s);
  return NRD_OK;
}

// Wait for the solve nk_graph_launch enqueued on s and report it.
int nk_graph_collect(nrd_ctx* c, nrd_stats* st, cudaStream_t s) {
  NkGraph* G = c->nk;
  if (!G) return NRD_ESTATE;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    c->err = "Newton graph execution failed";
    return NRD_ECUDA;
  }
  const NkCtl& h = *G->h_ctl;
  // the frozen Jacobian belongs to u unless the last evaluation was F alone
  c->lin_ready = h.lin_last != 0;
  c->lin_dz = false;
  c->pc_ready = true;
  nrd_stats loc{};
  loc.newton_its = h.it;
  loc.krylov_its = h.krylov;
  loc.pc_setups = h.it;
  loc.fnorm0 = h.fn0;
  loc.fnorm = h.fn;
  loc.min_lambda = h.min_lambda;
  loc.kernels = G->kn[0] + (long)h.it * G->kn[1] + (long)h.cycles * G->kn[2] +
                (long)h.restarts * G->kn[3] + (long)h.krylov * G->kn[4] +
                (long)h.nres * G->kn[5] + (long)h.nlin * G->kn[6];
  if (h.flags & NK_NEG) {
    loc.status = NRD_ENEG;
    c->err = "positivity cap vanished";
  } else if (h.flags & NK_NAN) {
    loc.status = NRD_ENAN;
    c->err = "non-finite residual";
  } else if (h.ticks >= kMaxTicks) {
    loc.status = NRD_ENONCONV;
    c->err = "Newton graph hit its loop cap";
  } else if (h.fn > h.stop) {
    loc.status = NRD_ENONCONV;
    c->err = "Newton did not converge within max_newton";
  } else {
    loc.status = NRD_OK;
  }
  if (st) *st = loc;
  return loc.status;
}
