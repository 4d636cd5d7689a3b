// Time-step control of Sec. 3.4-3.5: the BDF2 time derivative (left-hand
// side of Eq. bdf2 over dt), the generalised leapfrog predictor (Eq.
// leapfrog), the local error estimate (Eq. bdf2le) in the scaled max norm, and
// the EPS (Eq. odets) and PC.4.7 (Eq. pc47) controllers.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "nrd_internal.h"

namespace {

// udot = (a0 u1 - c1 u0 - c2 um1) / dt  with (a0, c1, c2) of the step that
// produced u1 (backward Euler: 1, 1, 0)
__global__ void k_time_deriv(int n, const double* u1, const double* u0, const double* um1,
                             double a0, double c1, double c2, double rdt, double* ud) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = a0 * u1[i] - c1 * u0[i];
    if (um1) v -= c2 * um1[i];
    ud[i] = v * rdt;
  }
}

// up = u_n + (1 + al) dt udot_n - al^2 (u_n - u_nm1)
__global__ void k_predict(int n, const double* un, const double* unm1, const double* ud, double al,
                          double dt, double* up) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    up[i] = un[i] + (1.0 + al) * dt * ud[i] - al * al * (un[i] - unm1[i]);
}

// max over leaf cells of |c (u - up) / (u + eta)| per field
__global__ void k_lte(const uint8_t* mask, int N, const double* u, const double* up, double c,
                      double etaE, double etaT, double* part) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (mask[i] & MASK_COVERED) continue;
    double eE = c * (u[i] - up[i]), eT = c * (u[N + i] - up[N + i]);
    m = fmax(m, fabs(eE / (u[i] + etaE)));
    m = fmax(m, fabs(eT / (u[N + i] + etaT)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
    if (threadIdx.x == 0) part[blockIdx.x] = r;
  }
}

__global__ void k_max_finish(const double* part, int n, double* out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, part[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
    if (threadIdx.x == 0) *out = r;
  }
}

int gridn(long n) { return (int)std::max(1L, std::min((n + 255) / 256, 152L * 8)); }

}  // namespace

extern "C" {

int nrd_time_derivative(nrd_ctx* c, const double* u_np1, const double* u_n, const double* u_nm1,
                        double dt, double dt_prev, double* udot, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  if (!c->have_hier) { c->err = "no hierarchy"; return NRD_ESTATE; }
  if (step_pending_check(c, true, s)) return NRD_ESTATE;
  if (!u_np1 || !u_n || !udot || !(dt > 0.0)) { c->err = "bad argument"; return NRD_EINVAL; }
  double a0 = 1.0, c1 = 1.0, c2 = 0.0;
  if (u_nm1) {
    if (!(dt_prev > 0.0)) { c->err = "dt_prev must be positive"; return NRD_EINVAL; }
    double al = dt / dt_prev;
    a0 = (1.0 + 2.0 * al) / (1.0 + al);
    c1 = 1.0 + al;
    c2 = -al * al / (1.0 + al);
  }
  const int n2 = 2 * c->H.N;
  k_time_deriv<<<gridn(n2), 256, 0, s>>>(n2, u_np1, u_n, u_nm1, a0, c1, c2, 1.0 / dt, udot);
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}

int nrd_predict(nrd_ctx* c, const double* u_n, const double* u_nm1, const double* udot_n,
                double dt, double dt_prev, double* u_p, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  if (!c->have_hier) { c->err = "no hierarchy"; return NRD_ESTATE; }
  if (step_pending_check(c, true, s)) return NRD_ESTATE;
  if (!u_n || !u_nm1 || !udot_n || !u_p || !(dt > 0.0) || !(dt_prev > 0.0)) {
    c->err = "bad argument";
    return NRD_EINVAL;
  }
  const int n2 = 2 * c->H.N;
  k_predict<<<gridn(n2), 256, 0, s>>>(n2, u_n, u_nm1, udot_n, dt / dt_prev, dt, u_p);
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}

int nrd_lte(nrd_ctx* c, const double* u_np1, const double* u_p, double alpha, double eta_E,
            double eta_T, double* err_host, cudaStream_t s) {
  if (!c) return NRD_EINVAL;
  if (!c->have_hier) { c->err = "no hierarchy"; return NRD_ESTATE; }
  if (step_pending_check(c, true, s)) return NRD_ESTATE;
  if (!u_np1 || !u_p || !err_host || !(alpha >= 0.0)) { c->err = "bad argument"; return NRD_EINVAL; }
  const double coef = (alpha + 1.0) / (3.0 * alpha + 2.0);
  const int nb = c->R.nblk;
  k_lte<<<nb, 256, 0, s>>>(c->H.d_mask, c->H.N, u_np1, u_p, coef, eta_E, eta_T, c->R.d_part);
  k_max_finish<<<1, 1024, 0, s>>>(c->R.d_part, nb, c->R.d_res + 7);
  cudaMemcpyAsync(c->R.h_res + 7, c->R.d_res + 7, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) { c->err = "sync failed"; return NRD_ECUDA; }
  *err_host = c->R.h_res[7];
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}

int nrd_dt_control(int kind, double eps_t, double err_n, double err_nm1, double dt_n,
                   double dt_nm1, double* dt_next) {
  if (!dt_next || !(eps_t > 0.0) || !(err_n > 0.0) || !(dt_n > 0.0)) return NRD_EINVAL;
  const double k = 3.0;   // BDF2: local error O(dt^3)
  if (kind == NRD_DT_EPS) {
    *dt_next = std::pow(eps_t / err_n, 1.0 / k) * dt_n;
    return NRD_OK;
  }
  if (kind == NRD_DT_PC47) {
    if (!(err_nm1 > 0.0) || !(dt_nm1 > 0.0)) return NRD_EINVAL;
    const double kI = 0.4 / k, kP = 0.7 / k;
    const double alpha_n = dt_n / dt_nm1;
    const double alpha_next = std::pow(eps_t / err_n, kI) * std::pow(err_nm1 / err_n, kP) * alpha_n;
    *dt_next = alpha_next * dt_n;
    return NRD_OK;
  }
  return NRD_EINVAL;
}

}  // extern "C"
