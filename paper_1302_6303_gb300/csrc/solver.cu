// Inexact Newton with Eisenstat-Walker forcing and right-preconditioned
// restarted GMRES (Sec. 4.1, 4.2).  All vectors stay on the device; the
// Hessenberg column, Givens rotations and the residual estimate are updated
// by a one-thread kernel, and the host reads back one scalar per Krylov
// iteration to decide convergence.  Orthogonalisation is classical
// Gram-Schmidt applied twice (CGS2), each pass one multi-dot and one update.
// The preconditioned directions z_j = P^{-1} v_j are kept (flexible form), so
// the update is x = sum_j y_j z_j; for a fixed preconditioner this is
// right-preconditioned GMRES, and it stays valid for the FP32 V-cycle.
#include <cmath>
#include <cstdio>

#include "nrd_internal.h"

namespace {

enum {
  SL_EPS = 0, SL_DOT = 1, SL_NRM = 2, SL_G = 3, SL_F = 4, SL_CAP = 5, SL_R = 6,
  SL_H1 = 8, SL_H2 = 48
};

struct Small {
  double* Hm;   // (m+1) x m, column-major by j: Hm[i + (m+1) j]
  double* cs;
  double* sn;
  double* g;    // m+1
  double* y;    // m
};

Small small_of(nrd_ctx* c) {
  int m = c->kry_m;
  Small S;
  S.Hm = c->d_small;
  S.cs = S.Hm + (m + 1) * m;
  S.sn = S.cs + m;
  S.g = S.sn + m;
  S.y = S.g + m + 1;
  return S;
}

// Column j of the Hessenberg matrix from the two CGS passes, then the Givens
// update of the least-squares problem; res[SL_G] = |g_{j+1}|.
// (err: set by a grid barrier that gave up; the estimate then reads NaN)
__global__ void k_arnoldi(Small S, int m, int j, double* res, const int* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = S.Hm + (size_t)(m + 1) * j;
  for (int i = 0; i <= j; i++) col[i] = res[SL_H1 + i] + res[SL_H2 + i];
  double hn = sqrt(res[SL_NRM]);
  col[j + 1] = hn;
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
  res[SL_G] = (*err) ? nan("") : fabs(S.g[j + 1]);
}

__global__ void k_ginit(Small S, int m, const double* nrm2, double* res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i <= m; i++) S.g[i] = 0.0;
  S.g[0] = sqrt(*nrm2);
}

__global__ void k_backsub(Small S, int m, int k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; i--) {
    double s = S.g[i];
    for (int t = i + 1; t < k; t++) s -= S.Hm[i + (size_t)(m + 1) * t] * S.y[t];
    S.y[i] = s / S.Hm[i + (size_t)(m + 1) * i];
  }
}

// v0 = sign * r / sqrt(nrm2)
__global__ void k_normalize(int n, const double* r, double* v, const double* nrm2, double sign) {
  // the scale once per block (FP64 square root and division are slow)
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

// r = sign * rhs - Ax
__global__ void k_resid(int n, const double* rhs, double sign, const double* Ax, double* r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    r[i] = sign * rhs[i] - Ax[i];
}

int grid1(long n) {
  long b = (n + 255) / 256;
  return (int)std::max(1L, std::min(b, 152L * 8));
}

double read_slot(nrd_ctx* c, int slot, cudaStream_t s) {
  cudaMemcpyAsync(c->R.h_res + slot, c->R.d_res + slot, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return c->R.h_res[slot];
}

}  // namespace

int solver_alloc(nrd_ctx* c) {
  int m = c->p.restart;
  if (c->d_V && c->kry_m == m) return NRD_OK;
  solver_free(c);
  size_t n2 = 2 * (size_t)c->H.N;
  bool ok = cudaMalloc(&c->d_V, (m + 1) * n2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_Z, m * n2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_F, n2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_dx, n2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_w, n2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_r, n2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_b, n2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_small, ((m + 1) * m + 5 * m + 8) * sizeof(double)) == cudaSuccess;
  if (!ok) {
    solver_free(c);
    c->err = "solver work-space allocation failed";
    return NRD_ENOMEM;
  }
  c->kry_m = m;
  return NRD_OK;
}

static int solver_newton_host(nrd_ctx* c, double* u, const double* b, double a0, double dt,
                              nrd_stats* st, cudaStream_t s);

static bool use_graph(const nrd_ctx* c) {
  return c->p.graph && c->p.jv_mode == NRD_JV_ANALYTIC && !c->timer.on && c->p.restart < 32;
}

int solver_newton(nrd_ctx* c, double* u, const double* b, double a0, double dt, nrd_stats* st,
                  cudaStream_t s) {
  const int rc = solver_newton_begin(c, u, b, a0, dt, s);
  if (rc != NRD_OK) {
    c->pend = 0;
    return rc;
  }
  return solver_newton_end(c, st);
}

int solver_newton_begin(nrd_ctx* c, double* u, const double* b, double a0, double dt,
                        cudaStream_t s) {
  if (use_graph(c)) {
    int rc = solver_alloc(c);
    if (rc != NRD_OK) return rc;
    // the graph reads the history from the context's own buffer
    if (b != c->d_b)
      cudaMemcpyAsync(c->d_b, b, 2 * (size_t)c->H.N * sizeof(double), cudaMemcpyDeviceToDevice,
                      s);
    rc = nk_graph_launch(c, u, c->d_b, a0, dt, s);
    if (rc != NRD_OK) return rc;
    c->pend = 1;
    c->pend_s = s;
    return NRD_OK;
  }
  c->pend_st = nrd_stats{};
  c->pend_rc = solver_newton_host(c, u, b, a0, dt, &c->pend_st, s);
  c->pend = 2;
  c->pend_s = s;
  return NRD_OK;
}

int solver_newton_end(nrd_ctx* c, nrd_stats* st) {
  const int pend = c->pend;
  c->pend = 0;
  if (pend == 1) return nk_graph_collect(c, st, c->pend_s);
  if (pend == 2) {
    if (st) *st = c->pend_st;
    return c->pend_rc;
  }
  c->err = "no step pending";
  return NRD_ESTATE;
}

void solver_free(nrd_ctx* c) {
  nk_graph_free(c);
  auto F = [](void* p) { if (p) cudaFree(p); };
  F(c->d_V); F(c->d_Z); F(c->d_F); F(c->d_dx); F(c->d_w); F(c->d_r); F(c->d_b); F(c->d_small);
  c->d_V = c->d_Z = c->d_F = c->d_dx = c->d_w = c->d_r = c->d_b = c->d_small = nullptr;
  c->kry_m = 0;
}

// GMRES for A x = sign * rhs to ||sign rhs - A x|| <= tol, with A = J (the
// configured Jv form) or, when transposed, A = J^T at the last linearisation.
// x: c->d_dx.  Returns iterations in *its.
static int gmres(nrd_ctx* c, const double* u, const double* b, double a0, double dt,
                 const double* rhs, double rhs_sign, double fn, double tol, bool transposed,
                 int* its, cudaStream_t s) {
  Hier& H = c->H;
  const int n2 = 2 * H.N;
  const long stride = n2;
  const int m = c->kry_m;
  Small S = small_of(c);
  const int mode = (c->p.jv_mode == NRD_JV_ANALYTIC) ? NRD_JV_FROZEN : NRD_JV_FD;
  auto apply = [&](const double* v, double* out) -> int {
    if (transposed) {
      launch_vjp(H, c->d_jc, c->d_cc, c->d_z, v, c->d_lam, c->d_gam, a0, dt, out, nullptr, s);
      return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
    }
    return ctx_jv(c, u, v, b, c->d_F, a0, dt, mode, out, false, s);
  };
  cudaMemsetAsync(c->d_dx, 0, n2 * sizeof(double), s);
  double rn2 = fn * fn;
  const double* r0 = rhs;
  double sign = rhs_sign;
  int total = 0;
  *its = 0;
  if (fn <= tol) return NRD_OK;
  bool first = true;
  while (total < c->p.max_krylov) {
    // V0 = r / ||r||
    cudaMemcpyAsync(c->R.d_res + SL_R, &rn2, sizeof(double), cudaMemcpyHostToDevice, s);
    k_normalize<<<grid1(n2), 256, 0, s>>>(n2, r0, c->d_V, c->R.d_res + SL_R, sign);
    k_ginit<<<1, 1, 0, s>>>(S, m, c->R.d_res + SL_R, c->R.d_res);
    int j = 0;
    bool conv = false;
    for (; j < m && total < c->p.max_krylov; j++) {
      double* Vj = c->d_V + (size_t)j * stride;
      double* Zj = c->d_Z + (size_t)j * stride;
      c->timer.begin(NRD_TK_PC_APPLY, s);
      int rc = pc_apply_ex(c->pc, H, Vj, Zj, transposed, s);
      c->timer.end(NRD_TK_PC_APPLY, s);
      if (rc != NRD_OK) return rc;
      rc = apply(Zj, c->d_w);
      if (rc != NRD_OK) return rc;
      total++;
      // CGS2
      c->timer.begin(NRD_TK_ORTHO, s);
      // the adjoint solve runs to a tight tolerance: always two passes
      if (launch_cgs2_coop(H, c->R, c->d_w, c->d_V, stride, nullptr, j + 1, SL_H1, SL_H2,
                           SL_NRM, s, transposed) != NRD_OK) {
        cudaGetLastError();
        launch_cgs2(H, c->R, c->d_w, c->d_V, stride, nullptr, j + 1, SL_H1, SL_H2, SL_NRM, s);
        k_normalize<<<grid1(n2), 256, 0, s>>>(n2, c->d_w, c->d_V + (size_t)(j + 1) * stride,
                                               c->R.d_res + SL_NRM, 1.0);
      }
      c->timer.end(NRD_TK_ORTHO, s);
      k_arnoldi<<<1, 1, 0, s>>>(S, m, j, c->R.d_res, c->R.d_err);
      double gres = read_slot(c, SL_G, s);
      double hn2 = c->R.h_res[SL_NRM];
      (void)hn2;
      if (!std::isfinite(gres)) {
        c->err = "non-finite GMRES residual";
        return NRD_ENAN;
      }
      if (gres <= tol) {
        j++;
        conv = true;
        break;
      }
    }
    k_backsub<<<1, 1, 0, s>>>(S, m, j);
    // the forward solve's update comes with its positivity cap at u
    if (transposed) launch_lincomb_dev(n2, c->d_dx, c->d_Z, stride, j, S.y, s);
    else launch_lincomb_cap(H, c->R, c->d_dx, c->d_Z, stride, nullptr, j, S.y, u, SL_CAP, s);
    if (conv) break;
    if (total >= c->p.max_krylov) break;
    // restart from the true residual r = sign * rhs - A dx
    int rc = apply(c->d_dx, c->d_w);
    if (rc != NRD_OK) return rc;
    k_resid<<<grid1(n2), 256, 0, s>>>(n2, rhs, rhs_sign, c->d_w, c->d_r);
    launch_wdot_lv(H, c->R, c->d_r, c->d_r, SL_R, s);
    rn2 = read_slot(c, SL_R, s);
    r0 = c->d_r;
    sign = 1.0;
    first = false;
    if (std::sqrt(rn2) <= tol) break;
  }
  (void)first;
  *its = total;
  return (cudaGetLastError() == cudaSuccess) ? NRD_OK : NRD_ECUDA;
}

// Host-driven form: one read-back per Krylov iteration.  Used when the
// graph form is off, for the finite-difference Jv, and while kernel timing
// is recorded (event records cannot sit inside the graph's loops).
static int solver_newton_host(nrd_ctx* c, double* u, const double* b, double a0, double dt,
                              nrd_stats* st, cudaStream_t s) {
  int rc = solver_alloc(c);
  if (rc != NRD_OK) return rc;
  Hier& H = c->H;
  const int n2 = 2 * H.N;
  nrd_stats loc{};
  loc.min_lambda = 1.0;
  // analytic form: residual, exact-Jacobian face coefficients and the
  // preconditioner are produced together at every iterate
  const bool lin = (c->p.jv_mode == NRD_JV_ANALYTIC);
  auto evaluate = [&](void) -> int {
    if (lin) return ctx_linearise(c, u, b, a0, dt, c->d_F, s);
    return ctx_residual(c, u, b, a0, dt, c->d_F, true, s);
  };
  rc = evaluate();
  if (rc != NRD_OK) return rc;
  launch_wdot_lv(H, c->R, c->d_F, c->d_F, SL_F, s);
  double fn = std::sqrt(read_slot(c, SL_F, s));
  if (!std::isfinite(fn)) {
    c->err = "non-finite initial residual";
    return NRD_ENAN;
  }
  loc.fnorm0 = fn;
  const double stop = c->p.rtol * fn + c->p.atol;
  double eta = c->p.eta0;
  int it = 0;
  while (fn > stop && it < c->p.max_newton) {
    if (!lin) {
      c->timer.begin(NRD_TK_PC_SETUP, s);
      rc = pc_setup(c->pc, H, c->mp, u, c->d_gu, c->d_z, c->d_gz, a0, dt, s);
      c->timer.end(NRD_TK_PC_SETUP, s);
      if (rc != NRD_OK) { c->err = "preconditioner set-up failed"; return rc; }
      c->pc_ready = true;
    }
    loc.pc_setups++;
    int its = 0;
    rc = gmres(c, u, b, a0, dt, c->d_F, -1.0, fn, eta * fn, false, &its, s);
    if (rc != NRD_OK) return rc;
    loc.krylov_its += its;
    // positivity-constrained update (Sec. 4.1 remark, reading R7): the cap
    // came with the last update of dx (none without Krylov iterations)
    if (its == 0) launch_pos_cap(H, c->R, u, c->d_dx, SL_CAP, s);
    double m = read_slot(c, SL_CAP, s);
    double lam = std::min(1.0, 0.9 * m);
    if (!(lam > 0.0)) {
      c->err = "positivity cap vanished";
      return NRD_ENEG;
    }
    loc.min_lambda = std::min(loc.min_lambda, lam);
    launch_axpy(n2, lam, c->d_dx, u, s);
    double fold = fn;
    // predicted last iterate (a full step whose solve aimed at the forcing
    // floor, stop/2): F alone first, the linearisation only if still needed;
    // the residual is bit-identical to the linearisation's
    bool done = false;
    if (lin && lam == 1.0 && eta * fold <= 0.5 * stop * (1.0 + 1e-12)) {
      rc = ctx_residual(c, u, b, a0, dt, c->d_F, true, s);
      if (rc != NRD_OK) return rc;
      launch_wdot_lv(H, c->R, c->d_F, c->d_F, SL_F, s);
      fn = std::sqrt(read_slot(c, SL_F, s));
      done = fn <= stop;
      if (done) c->lin_ready = false;   // the frozen Jacobian is the previous iterate's
    }
    if (!done) {
      rc = evaluate();
      if (rc != NRD_OK) return rc;
      launch_wdot_lv(H, c->R, c->d_F, c->d_F, SL_F, s);
      fn = std::sqrt(read_slot(c, SL_F, s));
    }
    if (!std::isfinite(fn)) {
      c->err = "non-finite residual";
      return NRD_ENAN;
    }
    // Eisenstat-Walker forcing term (Kelley's safeguarded choice)
    double rat = fn / fold;
    double g = c->p.ew_gamma;
    double etaA = g * rat * rat;
    double etaN;
    if (g * eta * eta <= 0.1) etaN = std::min(c->p.eta_max, etaA);
    else etaN = std::min(c->p.eta_max, std::max(etaA, g * eta * eta));
    eta = std::min(c->p.eta_max, std::max(etaN, 0.5 * stop / fn));
    it++;
  }
  launch_average_down(H, u, 2, H.N, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    c->err = "synchronisation failed";
    return NRD_ECUDA;
  }
  loc.newton_its = it;
  loc.fnorm = fn;
  loc.status = (fn > stop) ? NRD_ENONCONV : NRD_OK;
  if (st) *st = loc;
  if (loc.status != NRD_OK) c->err = "Newton did not converge within max_newton";
  return loc.status;
}

// Solve J^T lam = g at the last linearisation (adjoint of one implicit step)
// by GMRES with the forward preconditioner on the right.
int solver_adjoint(nrd_ctx* c, const double* g, double a0, double dt, double rtol, double* lam,
                   nrd_stats* st, cudaStream_t s) {
  int rc = solver_alloc(c);
  if (rc != NRD_OK) return rc;
  Hier& H = c->H;
  const int n2 = 2 * H.N;
  // covered entries of g are not unknowns: a copy with them zeroed keeps
  // every Krylov vector zero there (the level-weighted dots rely on it)
  cudaMemcpyAsync(c->d_tmp, g, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  launch_zero_covered(H, c->d_tmp, s);
  g = c->d_tmp;
  launch_wdot_lv(H, c->R, g, g, SL_F, s);
  double gn = std::sqrt(read_slot(c, SL_F, s));
  nrd_stats loc{};
  loc.fnorm0 = gn;
  int its = 0;
  rc = gmres(c, nullptr, nullptr, a0, dt, g, 1.0, gn, rtol * gn, true, &its, s);
  if (rc != NRD_OK) return rc;
  cudaMemcpyAsync(lam, c->d_dx, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  // final residual of the adjoint system
  launch_vjp(H, c->d_jc, c->d_cc, c->d_z, lam, c->d_lam, c->d_gam, a0, dt, c->d_w, nullptr, s);
  k_resid<<<grid1(n2), 256, 0, s>>>(n2, g, 1.0, c->d_w, c->d_r);
  launch_wdot_lv(H, c->R, c->d_r, c->d_r, SL_R, s);
  double rn = std::sqrt(read_slot(c, SL_R, s));
  loc.krylov_its = its;
  loc.fnorm = rn;
  loc.status = (rn <= 100.0 * rtol * gn || gn == 0.0) ? NRD_OK : NRD_ENONCONV;
  if (st) *st = loc;
  if (loc.status != NRD_OK) c->err = "adjoint GMRES did not reach the tolerance";
  return loc.status;
}
