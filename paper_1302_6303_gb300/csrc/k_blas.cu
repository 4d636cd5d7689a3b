// Device-resident reductions and vector updates for GMRES and Newton
// (Sec. 4.1): volume-weighted dots over leaf cells, the differencing
// parameter of Eq. Jac-free, classical Gram-Schmidt multi-dots and updates,
// and the positivity cap.  Reductions are two-stage with a fixed grid
// (warp shuffles, then a fixed-order block tree), so results are
// deterministic run to run.
#include <algorithm>
#include <cfloat>
#include <utility>

#include "nrd_internal.h"

namespace {

constexpr int RB = 256;
constexpr int NVMAX = 32;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
// block reduction; result valid in thread 0.  op: 0 sum, 1 min, 2 max.
// A shared-memory tree whose active warps halve (then one warp of shuffles):
// GB300 issues an FP64 instruction at the same cost however many lanes are
// active, so this needs 12 FP64 warp instructions for 256 threads where a
// shuffle tree in every warp needs 45.  sh: at least blockDim.x doubles;
// blockDim.x a power of two >= 32.
template <int OP>
__device__ double block_red(double v, double* sh) {
  const int t = threadIdx.x;
  __syncthreads();   // sh may still be read by a previous call
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x >> 1; s >= 32; s >>= 1) {
    if (t < s) {
      const double a = sh[t], b = sh[t + s];
      sh[t] = (OP == 0) ? a + b : (OP == 1 ? fmin(a, b) : fmax(a, b));
    }
    __syncthreads();
  }
  double r = (OP == 0) ? 0.0 : (OP == 1 ? DBL_MAX : -DBL_MAX);
  if (t < 32) {
    r = sh[t];
    r = (OP == 0) ? warp_sum(r) : (OP == 1 ? warp_min(r) : warp_max(r));
  }
  return r;
}

// ---- last-block finishing: every block writes its partials, takes a ticket;
// the block holding the last ticket sums the partials in block order (a fixed
// order, so the result does not depend on which block finished last) and
// resets the ticket counter for the next launch.
__device__ bool lb_arrive(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  return last;
}

template <int OP>
__device__ void lb_finish(const double* part, int nq, int pstride, double* res, int slot,
                          unsigned* counter) {
  __shared__ double sh[1024];
  for (int q = 0; q < nq; q++) {
    double acc = (OP == 0) ? 0.0 : (OP == 1 ? DBL_MAX : -DBL_MAX);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      const double v = __ldcg(&part[(long)b * pstride + q]);
      acc = (OP == 0) ? acc + v : (OP == 1 ? fmin(acc, v) : fmax(acc, v));
    }
    const double r = block_red<OP>(acc, sh);
    if (threadIdx.x == 0) res[slot + q] = r;
    __syncthreads();
  }
  if (threadIdx.x == 0) *counter = 0u;
}

__global__ void k_wdot(const float* __restrict__ wv, const double* __restrict__ x,
                       const double* __restrict__ y, int N, double* part, unsigned* counter,
                       double* res, int slot) {
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double w = (double)wv[i];
    acc += w * (x[i] * y[i] + x[N + i] * y[N + i]);
  }
  double r = block_red<0>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
  if (lb_arrive(counter)) lb_finish<0>(part, 1, 1, res, slot, counter);
}

// sum (or min/max) of nblk partials per quantity -> res[slot + q]
template <int OP>
__global__ void k_finish(const double* part, int nblk, int nq, double* res, int slot) {
  __shared__ double sh[1024];
  for (int q = 0; q < nq; q++) {
    double acc = (OP == 0) ? 0.0 : (OP == 1 ? DBL_MAX : -DBL_MAX);
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      double v = part[(long)b * nq + q];
      acc = (OP == 0) ? acc + v : (OP == 1 ? fmin(acc, v) : fmax(acc, v));
    }
    double r = block_red<OP>(acc, sh);
    if (threadIdx.x == 0) res[slot + q] = r;
    __syncthreads();
  }
}

// Differencing-parameter reductions (Sec. 4.1): <u,v>, ||v||_1, ||v||_2^2
// (volume weighted, leaf cells), and for the positivity rule the minima of
// u/(-v) over v<0, u/v over v>0 and u over leaf cells.
__global__ void k_eps_part(const float* __restrict__ wv, const uint8_t* __restrict__ mask,
                           const double* __restrict__ u, const double* __restrict__ v, int N,
                           double* part) {
  __shared__ double sh[1024];
  double suv = 0.0, sv1 = 0.0, svv = 0.0, mneg = DBL_MAX, mpos = DBL_MAX, mu = DBL_MAX;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (mask[i] & MASK_COVERED) continue;
    double w = (double)wv[i];
    for (int f = 0; f < 2; f++) {
      double uu = u[f * N + i], vv = v[f * N + i];
      suv += w * uu * vv;
      sv1 += w * fabs(vv);
      svv += w * vv * vv;
      if (vv < 0.0) mneg = fmin(mneg, uu / (-vv));
      if (vv > 0.0) mpos = fmin(mpos, uu / vv);
      mu = fmin(mu, uu);
    }
  }
  double r;
  r = block_red<0>(suv, sh); if (threadIdx.x == 0) part[blockIdx.x * 6 + 0] = r;
  r = block_red<0>(sv1, sh); if (threadIdx.x == 0) part[blockIdx.x * 6 + 1] = r;
  r = block_red<0>(svv, sh); if (threadIdx.x == 0) part[blockIdx.x * 6 + 2] = r;
  r = block_red<1>(mneg, sh); if (threadIdx.x == 0) part[blockIdx.x * 6 + 3] = r;
  r = block_red<1>(mpos, sh); if (threadIdx.x == 0) part[blockIdx.x * 6 + 4] = r;
  r = block_red<1>(mu, sh); if (threadIdx.x == 0) part[blockIdx.x * 6 + 5] = r;
}

__global__ void k_eps_finish(const double* part, int nblk, double u_min, double* res, int slot) {
  __shared__ double sh[1024];
  double q[6];
  for (int k = 0; k < 6; k++) {
    double acc = (k < 3) ? 0.0 : DBL_MAX;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      double v = part[b * 6 + k];
      acc = (k < 3) ? acc + v : fmin(acc, v);
    }
    q[k] = (k < 3) ? block_red<0>(acc, sh) : block_red<1>(acc, sh);
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double uv = q[0], v1 = q[1], vv = q[2], mneg = q[3], mpos = q[4], mu = q[5];
  double eps = 0.0;
  if (vv > 0.0) {
    const double sq = 1.4901161193847656e-08;  // sqrt(2^-52) = 2^-26
    if (fabs(uv) > u_min * v1)
      eps = sq * uv / vv;
    else
      eps = sq * u_min * (uv >= 0.0 ? 1.0 : -1.0) * v1 / vv;
    for (int t = 0; t < 10; t++) {
      bool pos = (mu > 0.0) && ((eps > 0.0) ? (eps < mneg) : (-eps < mpos));
      if (pos) break;
      eps *= 0.5;
    }
  }
  res[slot] = eps;
}

__global__ void k_emax(const uint8_t* __restrict__ mask, const double* __restrict__ E, int N,
                       double* part) {
  __shared__ double sh[1024];
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    if (!(mask[i] & MASK_COVERED)) m = fmax(m, fabs(E[i]));
  double r = block_red<2>(m, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void k_axpy(int n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

// x = num * x / sqrt(den_sq)   (num may be null -> 1)
__global__ void k_scale_dev(int n, const double* num, const double* den_sq, double* x) {
  __shared__ double s_s;
  if (threadIdx.x == 0) {
    const double nn = num ? *num : 1.0;
    const double d = sqrt(*den_sq);
    s_s = (d > 0.0) ? nn / d : 0.0;
  }
  __syncthreads();
  const double s = s_s;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] *= s;
}

__global__ void k_lincomb(int n, double* __restrict__ x, const double* __restrict__ Z, long stride,
                          int nv, const double* __restrict__ y) {
  __shared__ double ys[NVMAX];
  if (threadIdx.x < nv) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = x[i];
    for (int q = 0; q < nv; q++) s += ys[q] * Z[q * stride + i];
    x[i] = s;
  }
}

__global__ void k_zero_cov(const uint8_t* __restrict__ mask, int N, double* x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    if (mask[i] & MASK_COVERED) {
      x[i] = 0.0;
      x[N + i] = 0.0;
    }
}

// positivity cap of the Newton update (Sec. 4.1 remark): min over leaf
// components with v < 0 of u/(-v).  Each thread keeps its best ratio as a
// pair (a, b) = (u, -v), compared by cross-multiplication (both b > 0), and
// divides once at the end: FP64 division is a long instruction sequence on
// GB300.  (a/b < c/d <=> a d < c b; a near-tie may pick the other element,
// whose quotient then differs in the last bit at most.)
// Entries are screened by cap_candidate (integer instructions); blocks with
// no candidate skip the FP64 minimum tree.

__global__ void k_poscap(const uint8_t* __restrict__ mask, const double* __restrict__ u,
                         const double* __restrict__ v, int N, double* part, unsigned* counter,
                         double* res, int slot) {
  __shared__ double sh[1024];
  double ba = 1.0, bb = 0.0;
  bool have = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const bool leaf = !(mask[i] & MASK_COVERED);
    const double v0 = v[i], v1 = v[N + i];
    const double u0 = u[i], u1 = u[N + i];   // fetched with v, not after the sign test
    if (leaf && cap_candidate(u0, v0)) cap_take(u0, v0, have, ba, bb);
    if (leaf && cap_candidate(u1, v1)) cap_take(u1, v1, have, ba, bb);
  }
  double r = DBL_MAX;
  if (__syncthreads_or(have)) {
    double m = DBL_MAX;
    if (have) m = ba / bb;
    r = block_red<1>(m, sh);
  }
  if (threadIdx.x == 0) part[blockIdx.x] = r;
  if (lb_arrive(counter)) lb_finish<1>(part, 1, 1, res, slot, counter);
}

// x += sum_q y_q Z_q (the Newton update from the Krylov basis, both fields of
// a cell per thread, the same per-element sums as k_lincomb) fused with the
// positivity cap of the result: min over leaf components with x < 0 of
// u / (-x), pairs compared by cross-multiplication as in k_poscap, into
// res[slot] by last-block finishing.  nv = *jd when jd is given (device
// count), else nvh.
__global__ void __launch_bounds__(256) k_lincomb_cap(const uint8_t* __restrict__ mask, int N, double* __restrict__ x,
                              const double* __restrict__ Z, long stride, const int* jd, int nvh,
                              const double* __restrict__ y, const double* __restrict__ u,
                              double* part, unsigned* counter, double* res, int slot) {
  __shared__ double sh[1024];
  __shared__ double ys[NVMAX];
  const int nv = min(jd ? *jd : nvh, NVMAX);
  if (threadIdx.x < nv) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  double ba = 1.0, bb = 0.0;
  bool have = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    // u and the mask are fetched with dx and Z, not after the sign test
    const double u0 = u[i], u1 = u[N + i];
    const bool leaf = !(mask[i] & MASK_COVERED);
    double s0 = x[i], s1 = x[N + i];
    // 4 basis vectors in flight; fuller unrolling takes the registers of a
    // fourth resident block (80 instead of 60), and the grid then runs in two waves
#pragma unroll 4
    for (int q = 0; q < nv; q++) {
      s0 += ys[q] * Z[q * stride + i];
      s1 += ys[q] * Z[q * stride + N + i];
    }
    x[i] = s0;
    x[N + i] = s1;
    if (leaf && cap_candidate(u0, s0)) cap_take(u0, s0, have, ba, bb);
    if (leaf && cap_candidate(u1, s1)) cap_take(u1, s1, have, ba, bb);
  }
  double r = DBL_MAX;
  if (__syncthreads_or(have)) {
    double m = DBL_MAX;
    if (have) m = ba / bb;
    r = block_red<1>(m, sh);
  }
  if (threadIdx.x == 0) part[blockIdx.x] = r;
  if (lb_arrive(counter)) lb_finish<1>(part, 1, 1, res, slot, counter);
}

// ---- variants whose vector count is a device value (graph-captured solves)

// res[q] = <w, V_q>, q < *jd + add, in groups of 4 vectors (w re-read per
// group), a thread-strided sum per block, a block tree, then the last block
// sums the block partials in block order.
__global__ void k_mdot_dyn(const float* __restrict__ wv, const double* __restrict__ w,
                           const double* __restrict__ V, long stride, int N, const int* jd,
                           int add, double* part, unsigned* counter, double* res, int slot) {
  __shared__ double sh[1024];
  const int nv = min((jd ? *jd : 0) + add, NVMAX);
  for (int q0 = 0; q0 < nv; q0 += 4) {
    const int nq = min(4, nv - q0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const double* Vq = V + (long)q0 * stride;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
      double vol = (double)wv[i];
      double wE = vol * w[i], wT = vol * w[N + i];
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (q < nq) acc[q] += wE * Vq[q * stride + i] + wT * Vq[q * stride + N + i];
    }
    for (int q = 0; q < nq; q++) {
      double r = block_red<0>(acc[q], sh);
      if (threadIdx.x == 0) part[(long)blockIdx.x * NVMAX + q0 + q] = r;
      __syncthreads();
    }
  }
  if (lb_arrive(counter)) lb_finish<0>(part, nv, NVMAX, res, slot, counter);
}

// CGS pass 2 fused with pass 1's update: w <- w - sum_q h_q V_q, then the
// partial dots <w, V_q> (volume weighted) of the updated w; q < *jd + add.
// The first 8 dots ride on the update; more are formed from the stored w.
__global__ void k_cgs_upd_dots(const float* __restrict__ wv, double* __restrict__ w,
                               const double* __restrict__ V, long stride, int N, const int* jd,
                               int add, const double* __restrict__ h, double* part,
                               unsigned* counter, double* res, int slot) {
  __shared__ double sh[1024];
  __shared__ double hs[NVMAX];
  const int nv = min((jd ? *jd : 0) + add, NVMAX);
  if (threadIdx.x < nv) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; q++) acc[q] = 0.0;
  const int n8 = min(nv, 8);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double sE = w[i], sT = w[N + i];
    for (int q = 0; q < nv; q++) {
      sE -= hs[q] * V[q * stride + i];
      sT -= hs[q] * V[q * stride + N + i];
    }
    w[i] = sE;
    w[N + i] = sT;
    const double vol = (double)wv[i];
    const double wE = vol * sE, wT = vol * sT;
#pragma unroll
    for (int q = 0; q < 8; q++)
      if (q < n8) acc[q] += wE * V[q * stride + i] + wT * V[q * stride + N + i];
  }
  for (int q = 0; q < n8; q++) {
    const double r = block_red<0>(acc[q], sh);
    if (threadIdx.x == 0) part[(long)blockIdx.x * NVMAX + q] = r;
    __syncthreads();
  }
  for (int q0 = 8; q0 < nv; q0 += 8) {
    const int nq = min(8, nv - q0);
#pragma unroll
    for (int q = 0; q < 8; q++) acc[q] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
      const double vol = (double)wv[i];
      const double wE = vol * w[i], wT = vol * w[N + i];
#pragma unroll
      for (int q = 0; q < 8; q++)
        if (q < nq)
          acc[q] += wE * V[(q0 + q) * stride + i] + wT * V[(q0 + q) * stride + N + i];
    }
    for (int q = 0; q < nq; q++) {
      const double r = block_red<0>(acc[q], sh);
      if (threadIdx.x == 0) part[(long)blockIdx.x * NVMAX + q0 + q] = r;
      __syncthreads();
    }
  }
  if (lb_arrive(counter)) lb_finish<0>(part, nv, NVMAX, res, slot, counter);
}

// CGS pass 2's update fused with the squared norm of the result
__global__ void k_cgs_upd_norm(const float* __restrict__ wv, double* __restrict__ w,
                               const double* __restrict__ V, long stride, int N, const int* jd,
                               int add, const double* __restrict__ h, double* part,
                               unsigned* counter, double* res, int slot) {
  __shared__ double sh[1024];
  __shared__ double hs[NVMAX];
  const int nv = min((jd ? *jd : 0) + add, NVMAX);
  if (threadIdx.x < nv) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double sE = w[i], sT = w[N + i];
    for (int q = 0; q < nv; q++) {
      sE -= hs[q] * V[q * stride + i];
      sT -= hs[q] * V[q * stride + N + i];
    }
    w[i] = sE;
    w[N + i] = sT;
    acc += (double)wv[i] * (sE * sE + sT * sT);
  }
  const double r = block_red<0>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
  if (lb_arrive(counter)) lb_finish<0>(part, 1, 1, res, slot, counter);
}

__global__ void k_lincomb_dyn(int n, double* __restrict__ x, const double* __restrict__ Z,
                              long stride, const int* jd, const double* __restrict__ y) {
  __shared__ double ys[NVMAX];
  const int nv = min(*jd, NVMAX);
  if (threadIdx.x < nv) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = x[i];
    for (int q = 0; q < nv; q++) s += ys[q] * Z[q * stride + i];
    x[i] = s;
  }
}

__global__ void k_axpy_dev(int n, const double* __restrict__ a, const double* __restrict__ x,
                           double* __restrict__ y) {
  const double av = *a;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] += av * x[i];
}

// ---- CGS2 of one Arnoldi step as one cooperative kernel
// Grid-wide barrier for a cooperative launch (all blocks resident).  The
// wait is bounded: after kSpinLimit polls the block records an error in
// err[0] and carries on, so a launch that is not co-resident cannot hang.
constexpr long kSpinLimit = 1L << 24;

__device__ void grid_barrier(unsigned* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long it = 0;
      while (*gen == g) {
        if (++it > kSpinLimit) {
          atomicOr(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// every block sums the nq block partials (stride NVMAX) in block order into
// out[0..nq) (shared); the same order in every block, so all agree
__device__ void coop_reduce(const double* part, int nq, double* out, double* sh) {
  for (int q = 0; q < nq; q++) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      acc += __ldcg(&part[(long)b * NVMAX + q]);
    const double r = block_red<0>(acc, sh);
    if (threadIdx.x == 0) out[q] = r;
    __syncthreads();
  }
}

// Volume weights of a level-major vector whose covered cells are zero (every
// Krylov vector, F and the Newton directions): the leaf-cell volume is
// constant on a level, so a weighted dot is, per level, an FMA chain over
// the level's cells times the level volume.  A thread's cells increase, so
// it meets the level boundaries in order.
struct LevW {
  int L;
  int end[NRD_MAX_LEVELS];     // one past the last cell of level l
  double w[NRD_MAX_LEVELS];    // cell volume of level l
};

// One sweep over a thread's cells (level-weighted, see LevW): with UPD first
// w -= sum_{q<nv} hu_q V_q (stored back), then the NQ dots
// <w, V_{q0+q}> and, with NORM, <w, w>.  NQ, UPD and NORM are compile-time,
// so no FP64 instruction is issued for an unused accumulator.  Block
// partials to part[blockIdx.x * NVMAX + col0 + q] (the norm after the dots).
template <int NQ, bool UPD, bool NORM>
__device__ void orth_sweep(const LevW& lw, int l0, double* __restrict__ w,
                           const double* __restrict__ V, long stride, int N, int nv,
                           const double* hu, int q0, double* part, int col0, double* sh) {
  constexpr int NA = NQ + (NORM ? 1 : 0);
  double acc[NA > 0 ? NA : 1], tot[NA > 0 ? NA : 1];
#pragma unroll
  for (int q = 0; q < NA; q++) acc[q] = tot[q] = 0.0;
  const int T = gridDim.x * blockDim.x;
  int l = l0, lend = lw.end[l0];
  double lwt = lw.w[l0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += T) {
    while (i >= lend) {
#pragma unroll
      for (int q = 0; q < NA; q++) {
        tot[q] = fma(lwt, acc[q], tot[q]);
        acc[q] = 0.0;
      }
      l++;
      lend = lw.end[l];
      lwt = lw.w[l];
    }
    double wE = w[i], wT = w[N + i];
    if (UPD) {
      for (int q = 0; q < nv; q++) {
        wE = fma(-hu[q], V[q * stride + i], wE);
        wT = fma(-hu[q], V[q * stride + N + i], wT);
      }
      w[i] = wE;
      w[N + i] = wT;
    }
#pragma unroll
    for (int q = 0; q < NQ; q++)
      acc[q] = fma(wE, V[(q0 + q) * stride + i], fma(wT, V[(q0 + q) * stride + N + i], acc[q]));
    if (NORM) acc[NA - 1] = fma(wE, wE, fma(wT, wT, acc[NA - 1]));
  }
#pragma unroll
  for (int q = 0; q < NA; q++) {
    tot[q] = fma(lwt, acc[q], tot[q]);
    const double r = block_red<0>(tot[q], sh);
    if (threadIdx.x == 0) part[(long)blockIdx.x * NVMAX + col0 + q] = r;
  }
}

// the dots <w, V_q>, q < nv, in chunks of 4 (UPD and NORM on the first chunk)
template <bool UPD, bool NORM>
__device__ void orth_dots(const LevW& lw, int l0, double* w, const double* V, long stride, int N,
                          int nv, const double* hu, double* part, double* sh) {
  for (int q0 = 0; q0 < nv; q0 += 4) {
    const int nq = min(4, nv - q0);
    const bool first = (q0 == 0);
    // norm column: right after the last dot (col nv)
    if (first) {
      switch (nq) {
        case 1: orth_sweep<1, UPD, NORM>(lw, l0, w, V, stride, N, nv, hu, 0, part, 0, sh); break;
        case 2: orth_sweep<2, UPD, NORM>(lw, l0, w, V, stride, N, nv, hu, 0, part, 0, sh); break;
        case 3: orth_sweep<3, UPD, NORM>(lw, l0, w, V, stride, N, nv, hu, 0, part, 0, sh); break;
        default: orth_sweep<4, UPD, NORM>(lw, l0, w, V, stride, N, nv, hu, 0, part, 0, sh);
      }
      if (NORM && nq < nv && threadIdx.x == 0) {
        // move the norm partial from column nq to column nv
        part[(long)blockIdx.x * NVMAX + nv] = part[(long)blockIdx.x * NVMAX + nq];
      }
    } else {
      switch (nq) {
        case 1: orth_sweep<1, false, false>(lw, l0, w, V, stride, N, nv, hu, q0, part, q0, sh); break;
        case 2: orth_sweep<2, false, false>(lw, l0, w, V, stride, N, nv, hu, q0, part, q0, sh); break;
        case 3: orth_sweep<3, false, false>(lw, l0, w, V, stride, N, nv, hu, q0, part, q0, sh); break;
        default: orth_sweep<4, false, false>(lw, l0, w, V, stride, N, nv, hu, q0, part, q0, sh);
      }
    }
  }
}

// sums of block partials in block order (the same in every block) -> out
__device__ void coop_sum(const double* part, int nq, double* out, double* sh) {
  for (int q = 0; q < nq; q++) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      acc += __ldcg(&part[(long)b * NVMAX + q]);
    const double r = block_red<0>(acc, sh);
    if (threadIdx.x == 0) out[q] = r;
  }
  __syncthreads();
}

// V[nv] = (w - V h) * sc, one sweep
__device__ void orth_final(double* __restrict__ w, double* __restrict__ V, long stride, int N,
                           int nv, const double* h, double sc) {
  const int T = gridDim.x * blockDim.x;
  double* vn = V + (long)nv * stride;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += T) {
    double wE = w[i], wT = w[N + i];
    for (int q = 0; q < nv; q++) {
      wE = fma(-h[q], V[q * stride + i], wE);
      wT = fma(-h[q], V[q * stride + N + i], wT);
    }
    vn[i] = sc * wE;
    vn[N + i] = sc * wT;
  }
}

// A second Gram-Schmidt pass runs when the first one removed more than this
// fraction of |w|^2 (|w'| < |w| / 100): then one classical pass may have
// lost orthogonality (its error grows like eps |w| / |w'|) and the
// Pythagorean norm below would cancel.
constexpr double kReorthFrac = 1e-4;

// Orthogonalisation of w against the nv = (jd ? *jd : 0) + add columns of V
// by classical Gram-Schmidt with a conditional second pass:
//   pass 1: h1 = V^T W w and s0 = w^T W w                    (barrier)
//   s1 = s0 - |h1|^2 = |w - V h1|^2 (Pythagoras, V orthonormal)
//   if s1 > 1e-4 s0:  V[nv] = (w - V h1) / sqrt(s1)          (h2 = 0)
//   else:  pass 2: w <- w - V h1; h2 = V^T W w and s = w^T W w  (barrier)
//          V[nv] = (w - V h2) / sqrt(s - |h2|^2)
// The first branch is the common one: one grid barrier and two sweeps over
// V.  The Pythagorean norms are well conditioned where they are used (s1 >
// 1e-4 s0; |h2| << |w| in the second pass: low-synchronisation
// Gram-Schmidt, Swirydowicz et al., Numer. Linear Algebra Appl. 2021).  W:
// leaf volumes (level-weighted dots; w and V vanish on covered cells).
// res[slot_h1 + q] = h1, res[slot_h2 + q] = h2 (0 without a second pass),
// res[slot_nrm] = the squared norm of the orthogonalised w.  Partials
// ping-pong between pa and pb so that each reduction needs one barrier.
// Every block sums the partials in the same order, so all take the same
// branch.  always2: the second pass every time (CGS2; solves that need an
// orthogonal basis to working precision, such as the adjoint's).
__global__ void __launch_bounds__(256) k_orth_coop(LevW lw, double* __restrict__ w,
                                                   double* __restrict__ V, long stride, int N,
                                                   const int* jd, int add, double* pa, double* pb,
                                                   unsigned* bar, int* err, double* res,
                                                   int slot_h1, int slot_h2, int slot_nrm,
                                                   int always2) {
  __shared__ double sh[1024];
  __shared__ double h[NVMAX + 1];
  __shared__ double hu[NVMAX];
  __shared__ double s_sc, s_nrm;
  __shared__ int s_re;
  const int nv = min((jd ? *jd : 0) + add, NVMAX - 1);
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  int l0 = 0;
  while (l0 < lw.L - 1 && i0 >= lw.end[l0]) l0++;

  orth_dots<false, true>(lw, l0, w, V, stride, N, nv, nullptr, pa, sh);
  grid_barrier(bar, err);
  coop_sum(pa, nv + 1, h, sh);                   // h = h1, h[nv] = |w|^2
  if (threadIdx.x == 0) {
    double q2 = 0.0;
    for (int q = 0; q < nv; q++) q2 = fma(h[q], h[q], q2);
    const double s0 = h[nv], s1 = s0 - q2;
    const bool re = always2 || !(s1 > kReorthFrac * s0);   // (NaN: the second pass reports it)
    s_re = re ? 1 : 0;
    s_nrm = re ? 0.0 : s1;
    s_sc = re ? 0.0 : 1.0 / sqrt(s1);
  }
  if (threadIdx.x < nv) hu[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x < nv) res[slot_h1 + threadIdx.x] = hu[threadIdx.x];
  if (!s_re) {
    if (blockIdx.x == 0) {
      if (threadIdx.x < nv) res[slot_h2 + threadIdx.x] = 0.0;
      if (threadIdx.x == 0) res[slot_nrm] = s_nrm;
    }
    orth_final(w, V, stride, N, nv, hu, s_sc);
    return;
  }
  orth_dots<true, true>(lw, l0, w, V, stride, N, nv, hu, pb, sh);
  grid_barrier(bar, err);
  coop_sum(pb, nv + 1, h, sh);                   // h = h2, h[nv] = |w|^2
  if (threadIdx.x == 0) {
    double q2 = 0.0;
    for (int q = 0; q < nv; q++) q2 = fma(h[q], h[q], q2);
    const double nrm = fmax(h[nv] - q2, 0.0);   // (a breakdown rounds to 0, not below)
    s_nrm = nrm;
    s_sc = (nrm > 0.0) ? 1.0 / sqrt(nrm) : 0.0;
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    if (threadIdx.x < nv) res[slot_h2 + threadIdx.x] = h[threadIdx.x];
    if (threadIdx.x == 0) res[slot_nrm] = s_nrm;
  }
  orth_final(w, V, stride, N, nv, h, s_sc);
}

// level-weighted <x, y> over both fields for vectors that vanish on covered
// cells; last-block finish into res[slot]
__global__ void k_wdot_lv(LevW lw, const double* __restrict__ x, const double* __restrict__ y,
                          int N, double* part, unsigned* counter, double* res, int slot) {
  __shared__ double sh[1024];
  const int T = gridDim.x * blockDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  int l = 0;
  while (l < lw.L - 1 && i0 >= lw.end[l]) l++;
  int lend = lw.end[l];
  double lwt = lw.w[l];
  double acc = 0.0, tot = 0.0;
  for (int i = i0; i < N; i += T) {
    while (i >= lend) {
      tot = fma(lwt, acc, tot);
      acc = 0.0;
      l++;
      lend = lw.end[l];
      lwt = lw.w[l];
    }
    acc = fma(x[i], y[i], fma(x[N + i], y[N + i], acc));
  }
  tot = fma(lwt, acc, tot);
  const double r = block_red<0>(tot, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
  if (lb_arrive(counter)) lb_finish<0>(part, 1, 1, res, slot, counter);
}

int grid_for(long n) {
  long b = (n + RB - 1) / RB;
  return (int)std::max(1L, std::min(b, (long)152 * 8));
}

}  // namespace

int reducer_init(Reducer& R, int N) {
  R.nblk = std::max(1, std::min((N + RB * 4 - 1) / (RB * 4), 152 * 4));
  if (cudaMalloc(&R.d_part, sizeof(double) * (size_t)R.nblk * NVMAX) != cudaSuccess) return NRD_ENOMEM;
  if (cudaMalloc(&R.d_res, sizeof(double) * 256) != cudaSuccess) return NRD_ENOMEM;
  if (cudaMallocHost(&R.h_res, sizeof(double) * 256) != cudaSuccess) return NRD_ENOMEM;
  if (cudaMalloc(&R.d_count, sizeof(unsigned)) != cudaSuccess) return NRD_ENOMEM;
  if (cudaMalloc(&R.d_bar, 2 * sizeof(unsigned)) != cudaSuccess) return NRD_ENOMEM;
  if (cudaMalloc(&R.d_part2, sizeof(double) * (size_t)R.nblk * NVMAX) != cudaSuccess)
    return NRD_ENOMEM;
  if (cudaMalloc(&R.d_err, sizeof(int)) != cudaSuccess) return NRD_ENOMEM;
  cudaMemset(R.d_res, 0, sizeof(double) * 256);
  cudaMemset(R.d_count, 0, sizeof(unsigned));
  cudaMemset(R.d_bar, 0, 2 * sizeof(unsigned));
  cudaMemset(R.d_err, 0, sizeof(int));
  // cooperative CGS2: every block resident, at most the partial buffer's rows
  {
    int dev = 0, nsm = 0, per = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_orth_coop, RB, 0);
    int want = std::max(1, (N + RB - 1) / RB);
    R.coop_blocks = coop ? std::min(std::min(nsm * std::min(per, 4), want), R.nblk) : 0;
  }
  return NRD_OK;
}

void reducer_free(Reducer& R) {
  if (R.d_part) cudaFree(R.d_part);
  if (R.d_res) cudaFree(R.d_res);
  if (R.h_res) cudaFreeHost(R.h_res);
  if (R.d_count) cudaFree(R.d_count);
  if (R.d_bar) cudaFree(R.d_bar);
  if (R.d_part2) cudaFree(R.d_part2);
  R.d_part2 = nullptr;
  if (R.d_err) cudaFree(R.d_err);
  R.d_part = R.d_res = R.h_res = nullptr;
  R.d_count = nullptr;
  R.d_bar = nullptr;
  R.d_err = nullptr;
}

void launch_wdot(const Hier& H, Reducer& R, const double* x, const double* y, int slot,
                 cudaStream_t s) {
  k_wdot<<<R.nblk, RB, 0, s>>>(H.d_wvol, x, y, H.N, R.d_part, R.d_count, R.d_res, slot);
}

void launch_fd_eps(const Hier& H, Reducer& R, const double* u, const double* v, double u_min,
                   int slot, cudaStream_t s) {
  k_eps_part<<<R.nblk, RB, 0, s>>>(H.d_wvol, H.d_mask, u, v, H.N, R.d_part);
  k_eps_finish<<<1, 1024, 0, s>>>(R.d_part, R.nblk, u_min, R.d_res, slot);
}

void launch_emax(const Hier& H, Reducer& R, const double* E, int slot, cudaStream_t s) {
  k_emax<<<R.nblk, RB, 0, s>>>(H.d_mask, E, H.N, R.d_part);
  k_finish<2><<<1, 1024, 0, s>>>(R.d_part, R.nblk, 1, R.d_res, slot);
}

void launch_axpy(int n, double a, const double* x, double* y, cudaStream_t s) {
  k_axpy<<<grid_for(n), RB, 0, s>>>(n, a, x, y);
}

void launch_scale_dev(int n, const double* num, const double* den_sq, double* x, cudaStream_t s) {
  k_scale_dev<<<grid_for(n), RB, 0, s>>>(n, num, den_sq, x);
}

void launch_lincomb_dev(int n, double* x, const double* Z, long stride, int nv, const double* y,
                        cudaStream_t s) {
  k_lincomb<<<grid_for(n), RB, 0, s>>>(n, x, Z, stride, nv, y);
}

void launch_zero_covered(const Hier& H, double* x, cudaStream_t s) {
  k_zero_cov<<<grid_for(H.N), RB, 0, s>>>(H.d_mask, H.N, x);
}

void launch_pos_cap(const Hier& H, Reducer& R, const double* u, const double* v, int slot,
                    cudaStream_t s) {
  k_poscap<<<R.nblk, RB, 0, s>>>(H.d_mask, u, v, H.N, R.d_part, R.d_count, R.d_res, slot);
}

void launch_lincomb_cap(const Hier& H, Reducer& R, double* x, const double* Z, long stride,
                        const int* jd, int nv, const double* y, const double* u, int slot,
                        cudaStream_t s) {
  k_lincomb_cap<<<R.nblk, RB, 0, s>>>(H.d_mask, H.N, x, Z, stride, jd, nv, y, u, R.d_part,
                                      R.d_count, R.d_res, slot);
}

void launch_mdot_dyn(const Hier& H, Reducer& R, const double* w, const double* V, long stride,
                     const int* jd, int add, int slot, cudaStream_t s) {
  k_mdot_dyn<<<R.nblk, RB, 0, s>>>(H.d_wvol, w, V, stride, H.N, jd, add, R.d_part, R.d_count,
                                   R.d_res, slot);
}

LevW levw_of(const Hier& H) {
  LevW lw;
  lw.L = H.L;
  for (int l = 0; l < NRD_MAX_LEVELS; l++) {
    lw.end[l] = (l < H.L) ? H.lev[l].off + H.lev[l].ncell : H.N;
    lw.w[l] = (l < H.L) ? H.lev[l].h[0] * H.lev[l].h[1] * H.lev[l].h[2] : 0.0;
  }
  return lw;
}

int launch_cgs2_coop(const Hier& H, Reducer& R, double* w, double* V, long stride, const int* jd,
                     int add, int slot_h1, int slot_h2, int slot_nrm, cudaStream_t s,
                     bool always2) {
  if (R.coop_blocks <= 0) return NRD_ECUDA;
  LevW lw = levw_of(H);
  int N = H.N;
  double* pa = R.d_part;
  double* pb = R.d_part2;
  unsigned* bar = R.d_bar;
  int* err = R.d_err;
  double* res = R.d_res;
  int a2 = always2 ? 1 : 0;
  void* args[] = {(void*)&lw, (void*)&w, (void*)&V, (void*)&stride, (void*)&N, (void*)&jd,
                  (void*)&add, (void*)&pa, (void*)&pb, (void*)&bar, (void*)&err, (void*)&res,
                  (void*)&slot_h1, (void*)&slot_h2, (void*)&slot_nrm, (void*)&a2};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_orth_coop, dim3(R.coop_blocks),
                                              dim3(RB), args, 0, s);
  return e == cudaSuccess ? NRD_OK : NRD_ECUDA;
}

void launch_wdot_lv(const Hier& H, Reducer& R, const double* x, const double* y, int slot,
                    cudaStream_t s) {
  k_wdot_lv<<<R.nblk, RB, 0, s>>>(levw_of(H), x, y, H.N, R.d_part, R.d_count, R.d_res, slot);
}

void launch_cgs2(const Hier& H, Reducer& R, double* w, const double* V, long stride,
                 const int* jd, int add, int slot_h1, int slot_h2, int slot_nrm, cudaStream_t s) {
  k_mdot_dyn<<<R.nblk, RB, 0, s>>>(H.d_wvol, w, V, stride, H.N, jd, add, R.d_part, R.d_count,
                                   R.d_res, slot_h1);
  k_cgs_upd_dots<<<R.nblk, RB, 0, s>>>(H.d_wvol, w, V, stride, H.N, jd, add, R.d_res + slot_h1,
                                       R.d_part, R.d_count, R.d_res, slot_h2);
  k_cgs_upd_norm<<<R.nblk, RB, 0, s>>>(H.d_wvol, w, V, stride, H.N, jd, add, R.d_res + slot_h2,
                                       R.d_part, R.d_count, R.d_res, slot_nrm);
}

void launch_lincomb_dyn(int n, double* x, const double* Z, long stride, const int* jd,
                        const double* y, cudaStream_t s) {
  k_lincomb_dyn<<<grid_for(n), RB, 0, s>>>(n, x, Z, stride, jd, y);
}

void launch_axpy_dev(int n, const double* a, const double* x, double* y, cudaStream_t s) {
  k_axpy_dev<<<grid_for(n), RB, 0, s>>>(n, a, x, y);
}
