// Machine-rate measurement used as roofline denominators: FP64 and FP32 FMA
// throughput (independent FMA chains, all SMs busy), FP64 division and square
// root throughput, and device copy bandwidth.  Timed with CUDA events on the
// caller's stream.
#include <algorithm>

#include "nrd_internal.h"

namespace {

template <class T>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; i++) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// independent chains of FP64 divisions (op 0) or square roots (op 1), CUDA's
// correctly rounded operations
__global__ void k_div_sqrt_chains(double* out, int iters, int op, double a) {
  double x0 = 1.0 + threadIdx.x * 1e-6, x1 = x0 + 0.25, x2 = x0 + 0.5, x3 = x0 + 0.75;
  if (op == 0) {
    for (int i = 0; i < iters; i++) {
      x0 = a / x0; x1 = a / x1; x2 = a / x2; x3 = a / x3;
    }
  } else {
    for (int i = 0; i < iters; i++) {
      x0 = sqrt(x0 + a); x1 = sqrt(x1 + a); x2 = sqrt(x2 + a); x3 = sqrt(x3 + a);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}

__global__ void k_copy(const double2* __restrict__ a, double2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

}  // namespace

extern "C" int nrd_measure_peaks(double* fp64_tflops, double* fp32_tflops, double* copy_gbs,
                                 cudaStream_t s) {
  if (!fp64_tflops || !fp32_tflops || !copy_gbs) return NRD_EINVAL;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nb = nsm * 8, nt = 256;
  const size_t nthr = (size_t)nb * nt;
  double* od = nullptr;
  float* of = nullptr;
  double2 *a = nullptr, *b = nullptr;
  const size_t ncopy = (size_t)1 << 26;   // 2 x 1 GiB of double2
  if (cudaMalloc(&od, nthr * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&of, nthr * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&a, ncopy * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&b, ncopy * sizeof(double2)) != cudaSuccess) {
    cudaFree(od); cudaFree(of); cudaFree(a); cudaFree(b);
    return NRD_ENOMEM;
  }
  cudaMemsetAsync(a, 0, ncopy * sizeof(double2), s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms;
  double best64 = 0, best32 = 0, bestc = 0;
  const int it64 = 4000, it32 = 16000;
  for (int rep = 0; rep < 3; rep++) {
    cudaEventRecord(e0, s);
    k_fma_chains<double><<<nb, nt, 0, s>>>(od, it64, 0.9999999, 1e-9);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best64 = std::max(best64, 2.0 * 8 * it64 * (double)nthr / (ms * 1e-3) / 1e12);
    cudaEventRecord(e0, s);
    k_fma_chains<float><<<nb, nt, 0, s>>>(of, it32, 0.9999999f, 1e-9f);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best32 = std::max(best32, 2.0 * 8 * it32 * (double)nthr / (ms * 1e-3) / 1e12);
    cudaEventRecord(e0, s);
    k_copy<<<nsm * 16, 512, 0, s>>>(a, b, ncopy);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    bestc = std::max(bestc, 2.0 * ncopy * sizeof(double2) / (ms * 1e-3) / 1e9);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(od); cudaFree(of); cudaFree(a); cudaFree(b);
  *fp64_tflops = best64;
  *fp32_tflops = best32;
  *copy_gbs = bestc;
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}

extern "C" int nrd_measure_fp64_ops(double* rates, cudaStream_t s) {
  if (!rates) return NRD_EINVAL;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nb = nsm * 8, nt = 256;
  const size_t nthr = (size_t)nb * nt;
  double* od = nullptr;
  if (cudaMalloc(&od, nthr * sizeof(double)) != cudaSuccess) return NRD_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms;
  double best[3] = {0, 0, 0};
  const int itf = 4000, itd = 500;
  for (int rep = 0; rep < 3; rep++) {
    cudaEventRecord(e0, s);
    k_fma_chains<double><<<nb, nt, 0, s>>>(od, itf, 0.9999999, 1e-9);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best[0] = std::max(best[0], 8.0 * itf * (double)nthr / (ms * 1e-3));
    for (int op = 0; op < 2; op++) {
      cudaEventRecord(e0, s);
      k_div_sqrt_chains<<<nb, nt, 0, s>>>(od, itd, op, 1.0000001);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      best[1 + op] = std::max(best[1 + op], 4.0 * itd * (double)nthr / (ms * 1e-3));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(od);
  for (int q = 0; q < 3; q++) rates[q] = best[q];
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}
