// Allocation-free variant of the volume-weighted inner product (nrd_dot).
//
// nrd_dot reduces through block partials held in device memory that the
// context allocated.  Some callers cannot allocate device memory at the point
// where they need a dot product: code running under an external memory
// manager that owns every device byte, or a latency-critical path where an
// allocation (which can synchronise the device) is not acceptable.  nrd_wdot_noalloc serves them:
// its block partials live in the file-scope array below, so the call itself
// allocates nothing and needs no context.
#include <mutex>

#include "nrd_internal.h"

namespace {

constexpr int kBlock = 256;             // threads per block
constexpr int kPerBlock = 1024;         // elements reduced by one block
constexpr int kMaxPartials = 65536;     // 512 KiB of partials -> n <= 2^26

// Shared by every call on a device; kept by the device until the process
// exits.  Every slot a call reads is written earlier in the same call, so
// nothing has to be cleared between calls.
static __device__ __align__(256) double g_partials[kMaxPartials];

std::mutex g_mu;
double* g_addr[256] = {nullptr};        // device address of g_partials, per device ordinal

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v) {
  __shared__ double sh[kBlock / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (lane < kBlock / 32) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// partial b = sum over i in [b*kPerBlock, (b+1)*kPerBlock) of
// w_i (x_i y_i + x_{n+i} y_{n+i})
__global__ void __launch_bounds__(kBlock) k_wdot_part(const double* __restrict__ x,
                                                      const double* __restrict__ y,
                                                      const float* __restrict__ w, long n,
                                                      double* part) {
  const long base = (long)blockIdx.x * kPerBlock;
  double acc = 0.0;
  for (int k = threadIdx.x; k < kPerBlock; k += kBlock) {
    long i = base + k;
    if (i < n) acc += (double)w[i] * (x[i] * y[i] + x[n + i] * y[n + i]);
  }
  double r = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// out = sum of the first nblk partials, fixed order
__global__ void __launch_bounds__(kBlock) k_wdot_final(const double* part, int nblk, double* out) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kBlock) acc += part[b];
  double r = block_sum(acc);
  if (threadIdx.x == 0) out[0] = r;
}

}  // namespace

extern "C" int nrd_wdot_noalloc(const double* x, const double* y, const float* w, int64_t n,
                                double* out, cudaStream_t s) {
  if (!x || !y || !w || !out || n < 0) return NRD_EINVAL;
  const long nblk = (n + kPerBlock - 1) / kPerBlock;
  if (nblk > kMaxPartials) return NRD_EINVAL;   // beyond the static scratch capacity
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NRD_ECUDA;
  double* part;
  {
    // first call on a device: look up the device address of the scratch array
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return NRD_ECUDA;
      g_addr[dev] = (double*)p;
    }
    part = g_addr[dev];
  }
  if (nblk > 0) k_wdot_part<<<(unsigned)nblk, kBlock, 0, s>>>(x, y, w, (long)n, part);
  k_wdot_final<<<1, kBlock, 0, s>>>(part, (int)nblk, out);
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}
