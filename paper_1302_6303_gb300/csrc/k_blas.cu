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
// block reduction; result valid in thread 0.  op: 0 sum, 1 min, 2 max
template <int OP>
__device__ double block_red(double v, double* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = (OP == 0) ? warp_sum(v) : (OP == 1 ? warp_min(v) : warp_max(v));
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = (OP == 0) ? 0.0 : (OP == 1 ? DBL_MAX : -DBL_MAX);
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : r;
    r = (OP == 0) ? warp_sum(r) : (OP == 1 ? warp_min(r) : warp_max(r));
  }
  return r;
}

__global__ void k_wdot(const float* __restrict__ wv, const double* __restrict__ x,
                       const double* __restrict__ y, int N, double* part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double w = (double)wv[i];
    acc += w * (x[i] * y[i] + x[N + i] * y[N + i]);
  }
  double r = block_red<0>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// sum (or min/max) of nblk partials per quantity -> res[slot + q]
template <int OP>
__global__ void k_finish(const double* part, int nblk, int nq, double* res, int slot) {
  __shared__ double sh[32];
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
  __shared__ double sh[32];
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
  __shared__ double sh[32];
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
  __shared__ double sh[32];
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    if (!(mask[i] & MASK_COVERED)) m = fmax(m, fabs(E[i]));
  double r = block_red<2>(m, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// res[i] = <w, V_i>, i < NV: w read once, each V_i once; NV is a template
// parameter so the accumulators stay in registers.
template <int NV>
__global__ void k_mdot(const float* __restrict__ wv, const double* __restrict__ w,
                       const double* __restrict__ V, long stride, int N, double* part) {
  __shared__ double sh[32];
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; q++) acc[q] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double vol = (double)wv[i];
    double wE = vol * w[i], wT = vol * w[N + i];
#pragma unroll
    for (int q = 0; q < NV; q++) acc[q] += wE * V[q * stride + i] + wT * V[q * stride + N + i];
  }
#pragma unroll
  for (int q = 0; q < NV; q++) {
    double r = block_red<0>(acc[q], sh);
    if (threadIdx.x == 0) part[(long)blockIdx.x * NV + q] = r;
  }
}

template <int NV>
void mdot_launch(int nblk, cudaStream_t s, const float* wv, const double* w, const double* V,
                 long stride, int N, double* part) {
  k_mdot<NV><<<nblk, RB, 0, s>>>(wv, w, V, stride, N, part);
}

template <int... I>
void mdot_dispatch(std::integer_sequence<int, I...>, int nv, int nblk, cudaStream_t s,
                   const float* wv, const double* w, const double* V, long stride, int N,
                   double* part) {
  using Fn = void (*)(int, cudaStream_t, const float*, const double*, const double*, long, int,
                      double*);
  static const Fn table[] = {&mdot_launch<I + 1>...};
  table[nv - 1](nblk, s, wv, w, V, stride, N, part);
}

__global__ void k_mupdate(int n2, double* __restrict__ w, const double* __restrict__ V, long stride,
                          int nv, const double* __restrict__ h) {
  __shared__ double hs[NVMAX];
  if (threadIdx.x < nv) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    double s = w[i];
    for (int q = 0; q < nv; q++) s -= hs[q] * V[q * stride + i];
    w[i] = s;
  }
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
// components with v < 0 of u/(-v)
__global__ void k_poscap(const uint8_t* __restrict__ mask, const double* __restrict__ u,
                         const double* __restrict__ v, int N, double* part) {
  __shared__ double sh[32];
  double m = DBL_MAX;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (mask[i] & MASK_COVERED) continue;
    for (int f = 0; f < 2; f++) {
      // divide only when the ratio beats the running minimum
      // (u/(-v) < m  <=>  u < m (-v) for v < 0), so the result is the same
      const double vv = v[f * N + i];
      if (vv < 0.0) {
        const double uu = u[f * N + i];
        if (uu < m * (-vv)) m = fmin(m, uu / (-vv));
      }
    }
  }
  double r = block_red<1>(m, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// ---- variants whose vector count is a device value (graph-captured solves)

// res[q] = <w, V_q>, q < *jd + add, in groups of 4 vectors (w re-read per
// group); the per-thread and block summation orders are those of k_mdot.
__global__ void k_mdot_dyn(const float* __restrict__ wv, const double* __restrict__ w,
                           const double* __restrict__ V, long stride, int N, const int* jd,
                           int add, double* part) {
  __shared__ double sh[32];
  const int nv = min(*jd + add, NVMAX);
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
}

__global__ void k_finish_dyn(const double* part, int nblk, const int* jd, int add, double* res,
                             int slot) {
  __shared__ double sh[32];
  const int nq = min(*jd + add, NVMAX);
  for (int q = 0; q < nq; q++) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[(long)b * NVMAX + q];
    double r = block_red<0>(acc, sh);
    if (threadIdx.x == 0) res[slot + q] = r;
    __syncthreads();
  }
}

__global__ void k_mupdate_dyn(int n2, double* __restrict__ w, const double* __restrict__ V,
                              long stride, const int* jd, int add, const double* __restrict__ h) {
  __shared__ double hs[NVMAX];
  const int nv = min(*jd + add, NVMAX);
  if (threadIdx.x < nv) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    double s = w[i];
    for (int q = 0; q < nv; q++) s -= hs[q] * V[q * stride + i];
    w[i] = s;
  }
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
  cudaMemset(R.d_res, 0, sizeof(double) * 256);
  return NRD_OK;
}

void reducer_free(Reducer& R) {
  if (R.d_part) cudaFree(R.d_part);
  if (R.d_res) cudaFree(R.d_res);
  if (R.h_res) cudaFreeHost(R.h_res);
  R.d_part = R.d_res = R.h_res = nullptr;
}

void launch_wdot(const Hier& H, Reducer& R, const double* x, const double* y, int slot,
                 cudaStream_t s) {
  k_wdot<<<R.nblk, RB, 0, s>>>(H.d_wvol, x, y, H.N, R.d_part);
  k_finish<0><<<1, 1024, 0, s>>>(R.d_part, R.nblk, 1, R.d_res, slot);
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

void launch_mdot(const Hier& H, Reducer& R, const double* w, const double* V, long stride, int nv,
                 int slot, cudaStream_t s) {
  mdot_dispatch(std::make_integer_sequence<int, NVMAX>{}, nv, R.nblk, s, H.d_wvol, w, V, stride,
                H.N, R.d_part);
  k_finish<0><<<1, 1024, 0, s>>>(R.d_part, R.nblk, nv, R.d_res, slot);
}

void launch_mupdate(int n2, double* w, const double* V, long stride, int nv, const double* h,
                    cudaStream_t s) {
  k_mupdate<<<grid_for(n2), RB, 0, s>>>(n2, w, V, stride, nv, h);
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
  k_poscap<<<R.nblk, RB, 0, s>>>(H.d_mask, u, v, H.N, R.d_part);
  k_finish<1><<<1, 1024, 0, s>>>(R.d_part, R.nblk, 1, R.d_res, slot);
}

void launch_mdot_dyn(const Hier& H, Reducer& R, const double* w, const double* V, long stride,
                     const int* jd, int add, int slot, cudaStream_t s) {
  k_mdot_dyn<<<R.nblk, RB, 0, s>>>(H.d_wvol, w, V, stride, H.N, jd, add, R.d_part);
  k_finish_dyn<<<1, 1024, 0, s>>>(R.d_part, R.nblk, jd, add, R.d_res, slot);
}

void launch_mupdate_dyn(int n2, double* w, const double* V, long stride, const int* jd, int add,
                        const double* h, cudaStream_t s) {
  k_mupdate_dyn<<<grid_for(n2), RB, 0, s>>>(n2, w, V, stride, jd, add, h);
}

void launch_lincomb_dyn(int n, double* x, const double* Z, long stride, const int* jd,
                        const double* y, cudaStream_t s) {
  k_lincomb_dyn<<<grid_for(n), RB, 0, s>>>(n, x, Z, stride, jd, y);
}

void launch_axpy_dev(int n, const double* a, const double* x, double* y, cudaStream_t s) {
  k_axpy_dev<<<grid_for(n), RB, 0, s>>>(n, a, x, y);
}
