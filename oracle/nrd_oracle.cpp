// Plain FP64 CPU oracle for the implicit non-equilibrium radiation diffusion
// method of "Dynamic Implicit 3D Adaptive Mesh Refinement for Non-Equilibrium
// Radiation Diffusion" (arXiv 1302.6303).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
// restatement of the method that the CUDA path is checked against.  Only the
// test-suite, the smoke check and the benchmark's CPU-baseline leg may load
// it.  It shares no code, header or table with the CUDA library.
//
// Everything is scalar loops over cells in FP64, following the paper's
// equations in order:
//   Sec. 3.1  model:       Eqs. E_td, T_td, sigma_a = z^3/T^3, D_T = k T^(5/2),
//                          Wilson-limited D_E, Robin/Neumann boundaries.
//   Sec. 3.2  space:       finite-volume cell balance (Eq. E_int), face fluxes
//                          (Eqs. diffusion_coeffs1-6), face T average,
//                          harmonic D_r, flux-limited D_E, first-order ghosts.
//   Sec. 3.2.1 AMR:        linear coarse-fine ghost interpolation (bilinear
//                          tangential, then linear normal), flux matching.
//   Sec. 3.3  time:        BDF2 / backward Euler residual (Eqs. bdf2, be,
//                          nonlinearsystem).
//   Sec. 4.1  JFNK:        inexact Newton with Eisenstat-Walker forcing,
//                          positivity-constrained update, FD Jv (Eq. Jac-free)
//                          with the two-branch differencing parameter,
//                          right-preconditioned GMRES.
//   Sec. 4.2  precond.:    P = P1 P2 split, frozen D_E^k, D_T^k.
//   Sec. 4.3  FAC:         Algorithm 1 with red-black Gauss-Seidel, averaging
//                          restriction, (tri)linear prolongation; geometric
//                          multigrid V-cycle on the coarsest AMR level.
//   Sec. 5    regridding:  tau^c, tau^g error indicators.
//
// Readings where the paper is silent or garbled (the CUDA path takes the
// same readings):
//   R1 limiter: default D_E = D_h/(1 + D_h g) with D_h = 2 D_r (Wilson form of
//      Sec. 3.1); LIM_PAPER_LITERAL gives the printed 2 D_r/(1 + D_r g).
//   R2 face D_T = k T_f^(5/2) with the arithmetic face T, not limited.
//   R3 cell sigma_a = z^3/T^3 at the cell centre.
//   R4 physical ghosts: Neumann ghost = interior value (zero flux); Robin
//      ghost from the discrete Robin relation with the unlimited
//      D_b = T_0^3/(3 z_0^3); the Robin face flux uses D_b.
//   R5 residual per unit volume: F = a0 u - b - dt f(u); dots and norms are
//      volume weighted over leaf cells.
//   R6 differencing parameter: b = 1, |<u,v>| compared, eps_mach = 2^-52,
//      sign(0) = +1, eps halved (at most 10 times) until u + eps v > 0.
//   R7 positivity cap: lambda = min(1, 0.9 min_{v_i<0} u_i/|v_i|).
//   R8 Eisenstat-Walker forcing with eta_max = 0.9, gamma = 0.9 and the
//      safeguards of Kelley's choice; first forcing eta_0 = 0.3.
//   R9 FAC: level error equations start from zero with homogeneous
//      coarse-fine ghosts (coarse value 0); corrections are interpolated to
//      every finer level; the composite residual is recomputed before every
//      smoothing pass, including those of the up-leg.
//   R10 coarsest AMR level: GMG V(nu1,nu2) with coarse_sweeps sweeps on the
//      coarsest grid.
//   R11 coarsened coefficients: mean of the 4 coincident fine faces; Robin
//      D_b averaged and re-discretised with the coarse spacing.
//   R12 red-black colour = parity of (i+j+k) in level index space, red
//      first for pre-smoothing, black first for post-smoothing.
//   R13 tangential coarse neighbours outside the domain are replaced by the
//      in-domain coarse cell (constant extrapolation); the same rule is used
//      for trilinear prolongation.
//   R14 d|x|/dx at x = 0 is taken as 0.
//   R15 z in a coarse-fine ghost is the z of the coarse parent cell.
//
// Parity pins: see tests/test_oracle_pins.py.  Every public function here is
// pinned by at least one closed form, invariant or brute-force check there.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

// Threads: built with OpenMP, the loops over cells whose iterations are
// independent (every cell written by exactly one iteration, reading only
// values no iteration of the same loop writes: the residual and its tangent
// per cell, one colour of a red-black pass, a Jacobi sweep into a second
// array, restriction, prolongation, averaging, the frozen-coefficient
// set-up) run on several threads.  Each result is the same expression in
// the same order as on one thread, so results are bit-identical for any
// thread count.  Sums over cells (the inner products) stay serial, in cell
// order.
#define ORC_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")

namespace {

enum { BC_NEUMANN = 0, BC_ROBIN = 1 };
enum { LIM_WILSON = 0, LIM_PAPER_LITERAL = 1 };
enum { JV_FD = 0, JV_ANALYTIC = 1 };

// ---------------------------------------------------------------- dual numbers
// Forward-mode tangent: the directional derivative of the exact same residual
// code, used for the analytic Jacobian-vector product.
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(double a, Dual b) { return Dual(a) + b; }
inline Dual operator+(Dual a, double b) { return a + Dual(b); }
inline Dual operator-(Dual a, double b) { return a - Dual(b); }
inline Dual operator/(double a, Dual b) { return Dual(a) / b; }
inline Dual operator-(double a, Dual b) { return Dual(a) - b; }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
// R14: derivative of |x| at 0 taken as 0.
inline Dual fabs(Dual a) {
  if (a.v > 0) return a;
  if (a.v < 0) return -a;
  return Dual(0.0, 0.0);
}
using std::sqrt;
using std::fabs;

// Sparse forward mode: a value with its derivatives with respect to every
// input of the residual (sorted (input, derivative) pairs).  Evaluating the
// residual code once with every input seeded by its own index gives every
// row of the Jacobian, with its sparsity, by the same chain rule as Dual.
struct SDual {
  double v;
  std::vector<std::pair<long, double>> d;
  SDual() : v(0) {}
  SDual(double a) : v(a) {}
};
// ca * a + cb * b on sorted derivative lists
inline std::vector<std::pair<long, double>> sd_comb(const std::vector<std::pair<long, double>>& a,
                                                    double ca,
                                                    const std::vector<std::pair<long, double>>& b,
                                                    double cb) {
  std::vector<std::pair<long, double>> o;
  o.reserve(a.size() + b.size());
  size_t i = 0, j = 0;
  while (i < a.size() || j < b.size()) {
    if (j == b.size() || (i < a.size() && a[i].first < b[j].first)) {
      o.push_back({a[i].first, ca * a[i].second});
      i++;
    } else if (i == a.size() || b[j].first < a[i].first) {
      o.push_back({b[j].first, cb * b[j].second});
      j++;
    } else {
      o.push_back({a[i].first, ca * a[i].second + cb * b[j].second});
      i++;
      j++;
    }
  }
  return o;
}
inline SDual sd_make(double v, std::vector<std::pair<long, double>> d) {
  SDual r(v);
  r.d = std::move(d);
  return r;
}
inline SDual sd_scale(const SDual& a, double v, double c) {
  SDual r(v);
  r.d = a.d;
  for (auto& e : r.d) e.second *= c;
  return r;
}
inline SDual operator+(const SDual& a, const SDual& b) { return sd_make(a.v + b.v, sd_comb(a.d, 1.0, b.d, 1.0)); }
inline SDual operator-(const SDual& a, const SDual& b) { return sd_make(a.v - b.v, sd_comb(a.d, 1.0, b.d, -1.0)); }
inline SDual operator-(const SDual& a) { return sd_scale(a, -a.v, -1.0); }
inline SDual operator*(const SDual& a, const SDual& b) { return sd_make(a.v * b.v, sd_comb(a.d, b.v, b.d, a.v)); }
inline SDual operator/(const SDual& a, const SDual& b) {
  return sd_make(a.v / b.v, sd_comb(a.d, 1.0 / b.v, b.d, -a.v / (b.v * b.v)));
}
inline SDual operator+(double a, const SDual& b) { return sd_scale(b, a + b.v, 1.0); }
inline SDual operator+(const SDual& a, double b) { return sd_scale(a, a.v + b, 1.0); }
inline SDual operator-(const SDual& a, double b) { return sd_scale(a, a.v - b, 1.0); }
inline SDual operator-(double a, const SDual& b) { return sd_scale(b, a - b.v, -1.0); }
inline SDual operator*(double a, const SDual& b) { return sd_scale(b, a * b.v, a); }
inline SDual operator*(const SDual& a, double b) { return sd_scale(a, a.v * b, b); }
inline SDual operator/(const SDual& a, double b) { return sd_scale(a, a.v / b, 1.0 / b); }
inline SDual operator/(double a, const SDual& b) { return SDual(a) / b; }
inline SDual& operator+=(SDual& a, const SDual& b) { a = a + b; return a; }
inline SDual sqrt(const SDual& a) {
  double s = std::sqrt(a.v);
  return sd_scale(a, s, 1.0 / (2.0 * s));
}
// R14: derivative of |x| at 0 taken as 0.
inline SDual fabs(const SDual& a) {
  if (a.v > 0) return a;
  if (a.v < 0) return -a;
  return SDual(0.0);
}

// --------------------------------------------------------------- hierarchy
struct Level {
  int n[3];
  double h[3];
  std::vector<int> box;    // 6 ints per patch: lo[3], hi[3] (inclusive)
  std::vector<long> off;   // first hierarchy-vector index of each patch
  std::vector<long> map;   // dense level index -> hierarchy index or -1
};

struct Hier {
  int L = 0;
  std::vector<Level> lev;
  long N = 0;                       // cells over all levels (one field)
  std::vector<int> cell_level;      // per hierarchy index
  std::vector<int> cell_ijk;        // 3 per hierarchy index
  int bc_type[6];
  double bc_R[6];
  double kcond = 0.01;
  int limiter = LIM_WILSON;
  std::vector<double> z;            // material z per cell (double copy of input)
  std::string err;

  // solver settings
  int restart = 30, max_krylov = 300, jv_mode = JV_FD;
  int nu1 = 2, nu2 = 2, nmg = 4, coarse_sweeps = 4;
  int smoother = 0;                 // 0 red-black Gauss-Seidel, 1 damped point Jacobi,
                                    // 2 block (x-line) Gauss-Seidel on the box levels
  double omega = 6.0 / 7.0;         // Jacobi damping
  double rtol = 1e-8, atol = 0.0;
  int max_newton = 20;
  double eta_max = 0.9, ew_gamma = 0.9, eta0 = 0.3, u_min = 1e-6;

  // preconditioner state (frozen at the Newton iterate)
  bool pc_ready = false;
  double beta = 0.0;
  std::vector<double> uk;           // frozen iterate (2N)
  // per field (0 = E, 1 = T), per operator level: AMR levels 0..L-1 then
  // GMG levels below level 0 are stored separately.
  struct OpLevel {
    int n[3];
    double h[3];
    int amr;                        // AMR level index, or -1 for a GMG-only grid
    std::vector<double> C[3];       // face coefficients (dense face arrays)
    std::vector<double> Db[6];      // Robin D_b on each domain face plane
  };
  std::vector<OpLevel> opl[2];      // AMR levels
  std::vector<OpLevel> mg[2];       // GMG levels m = 0..nmg-1 (m = 0 mirrors AMR level 0)

  long cell(int l, int i, int j, int k) const {
    const Level& Lv = lev[l];
    if (i < 0 || j < 0 || k < 0 || i >= Lv.n[0] || j >= Lv.n[1] || k >= Lv.n[2]) return -2;
    return Lv.map[(long)i + (long)Lv.n[0] * ((long)j + (long)Lv.n[1] * k)];
  }
  long cell(int l, const int c[3]) const { return cell(l, c[0], c[1], c[2]); }
  bool inside(int l, const int c[3]) const {
    for (int d = 0; d < 3; d++) if (c[d] < 0 || c[d] >= lev[l].n[d]) return false;
    return true;
  }
  bool covered(int l, const int c[3]) const {
    if (l + 1 >= L) return false;
    return cell(l + 1, 2 * c[0], 2 * c[1], 2 * c[2]) >= 0;
  }
  bool covered_idx(long idx) const {
    int l = cell_level[idx];
    return covered(l, &cell_ijk[3 * idx]);
  }
};

[[noreturn]] void fatal(const char* msg) {
  std::fprintf(stderr, "oracle internal error: %s\n", msg);
  std::abort();
}

inline double cube(double a) { return a * a * a; }
inline Dual cube(Dual a) { return a * a * a; }
inline SDual cube(const SDual& a) { return a * a * a; }

// Composite value of a field at an existing level-l cell: its own value when
// it is a leaf, the mean of its 8 children when covered by level l+1.
template <class S>
S comp_value(const Hier& H, const S* x, int l, const int c[3]) {
  long idx = H.cell(l, c);
  if (idx < 0) fatal("comp_value: cell does not exist (nesting violated)");
  if (!H.covered(l, c)) return x[idx];
  S sum = S(0.0);
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++)
      for (int e = 0; e < 2; e++) {
        int q[3] = {2 * c[0] + a, 2 * c[1] + b, 2 * c[2] + e};
        sum += comp_value(H, x, l + 1, q);
      }
  return sum / 8.0;
}

// Coarse-fine ghost (Sec. 3.2.1, Fig. interp): fine cell c at level l >= 1,
// ghost g = c + s e_d lies outside level l.  Bilinear interpolation of the
// four coarse values around the ghost's parent gives a value aligned with c;
// linear interpolation along the normal between it (coarse centre at 3h/2
// from c's centre) and c gives the ghost at distance h: g = (x_c + 2 i)/3.
template <class S>
S cf_ghost(const Hier& H, const S* x, int l, const int c[3], int d, int s) {
  if (l < 1) fatal("cf_ghost on level 0");
  int g[3] = {c[0], c[1], c[2]};
  g[d] += s;
  int P[3] = {g[0] / 2, g[1] / 2, g[2] / 2};
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const Level& C = H.lev[l - 1];
  int o1 = (g[t1] % 2 == 0) ? -1 : 1;
  int o2 = (g[t2] % 2 == 0) ? -1 : 1;
  if (P[t1] + o1 < 0 || P[t1] + o1 >= C.n[t1]) o1 = 0;  // R13
  if (P[t2] + o2 < 0 || P[t2] + o2 >= C.n[t2]) o2 = 0;
  int q10[3] = {P[0], P[1], P[2]}; q10[t1] += o1;
  int q01[3] = {P[0], P[1], P[2]}; q01[t2] += o2;
  int q11[3] = {P[0], P[1], P[2]}; q11[t1] += o1; q11[t2] += o2;
  S c00 = comp_value(H, x, l - 1, P);
  S c10 = comp_value(H, x, l - 1, q10);
  S c01 = comp_value(H, x, l - 1, q01);
  S c11 = comp_value(H, x, l - 1, q11);
  S iv = (9.0 * c00 + 3.0 * c10 + 3.0 * c01 + c11) / 16.0;
  long ic = H.cell(l, c);
  return (x[ic] + 2.0 * iv) / 3.0;
}

template <class Z>
Z cf_ghost_z(const Hier& H, const Z* z, int l, const int c[3], int d, int s) {
  int g[3] = {c[0], c[1], c[2]};
  g[d] += s;
  int P[3] = {g[0] / 2, g[1] / 2, g[2] / 2};
  long ip = H.cell(l - 1, P);
  if (ip < 0) fatal("cf_ghost_z: parent missing");
  return z[ip];  // R15
}
double cf_ghost_z(const Hier& H, int l, const int c[3], int d, int s) {
  return cf_ghost_z<double>(H, H.z.data(), l, c, d, s);
}

// Face fluxes D (b - a)/h between cell a (low side) and b (high side).
// Sec. 3.2: T_f = (T_a + T_b)/2; D_r = T_f^3 / (3 (z_a^3 + z_b^3));
// D_E limited (R1); D_T = k T_f^(5/2) (R2).
template <class S>
struct FluxPair { S E, T; };

template <class S>
FluxPair<S> pair_flux(const Hier& H, S Ea, S Eb, S Ta, S Tb, S za, S zb, double h) {
  S Tf = 0.5 * (Ta + Tb);
  S Dr = Tf * Tf * Tf / (3.0 * (cube(za) + cube(zb)));
  S g = fabs(Eb - Ea) / (0.5 * h * (Ea + Eb));
  S DE;
  if (H.limiter == LIM_WILSON) {
    S Dh = 2.0 * Dr;
    DE = Dh / (1.0 + Dh * g);
  } else {
    DE = 2.0 * Dr / (1.0 + Dr * g);
  }
  S DT = H.kcond * Tf * Tf * sqrt(Tf);
  FluxPair<S> f;
  f.E = DE * (Eb - Ea) / h;
  f.T = DT * (Tb - Ta) / h;
  return f;
}

// Robin ghost of Sec. 3.1 Eq. robinbc discretised at the face (R4):
// (1/2) D_b (E_g - E_0)/h + (E_g + E_0)/8 = R.
template <class S, class Z>
S robin_ghost(S E0, S T0, Z z0, double h, double R) {
  S Db = T0 * T0 * T0 / (3.0 * cube(z0));
  S a = Db / (2.0 * h);
  return (R + E0 * (a - 0.125)) / (a + 0.125);
}

// Flux (in the +e_d direction) through face (c, d, s) of the leaf cell c at
// level l, for the nonlinear residual.
template <class S>
FluxPair<S> face_flux(const Hier& H, const S* E, const S* T, const S* z, int l, const int c[3], int d,
                      int s) {
  const Level& Lv = H.lev[l];
  double h = Lv.h[d];
  long ic = H.cell(l, c);
  int g[3] = {c[0], c[1], c[2]};
  g[d] += s;
  FluxPair<S> f;
  if (!H.inside(l, g)) {
    int face = 2 * d + (s > 0 ? 1 : 0);
    f.T = S(0.0);
    if (H.bc_type[face] == BC_ROBIN) {
      S Eg = robin_ghost(E[ic], T[ic], z[ic], h, H.bc_R[face]);
      S Db = T[ic] * T[ic] * T[ic] / (3.0 * cube(z[ic]));
      f.E = (s > 0) ? Db * (Eg - E[ic]) / h : Db * (E[ic] - Eg) / h;
    } else {
      f.E = S(0.0);
    }
    return f;
  }
  long ig = H.cell(l, g);
  S Eg, Tg, zg;
  if (ig >= 0) {
    if (H.covered(l, g)) {
      // Flux matching (Sec. 3.2.1, Fig. flux): the coarse face flux is the
      // average of the four fine fluxes computed on the fine side.
      int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      FluxPair<S> sum;
      sum.E = S(0.0);
      sum.T = S(0.0);
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
          int q[3];
          q[d] = (s > 0) ? 2 * g[d] : 2 * g[d] + 1;
          q[t1] = 2 * c[t1] + a;
          q[t2] = 2 * c[t2] + b;
          FluxPair<S> ff = face_flux(H, E, T, z, l + 1, q, d, -s);
          sum.E += ff.E;
          sum.T += ff.T;
        }
      f.E = 0.25 * sum.E;
      f.T = 0.25 * sum.T;
      return f;
    }
    Eg = E[ig];
    Tg = T[ig];
    zg = z[ig];
  } else {
    Eg = cf_ghost(H, E, l, c, d, s);
    Tg = cf_ghost(H, T, l, c, d, s);
    zg = cf_ghost_z<S>(H, z, l, c, d, s);
  }
  if (s > 0) return pair_flux(H, E[ic], Eg, T[ic], Tg, z[ic], zg, h);
  return pair_flux(H, Eg, E[ic], Tg, T[ic], zg, z[ic], h);
}

// F(u) = a0 u - b - dt f(u)  (Eq. nonlinearsystem per unit volume, R5), with
// f_E = sum_d (F_{d+} - F_{d-})/h_d + sigma (T^4 - E),
// f_T = sum_d (G_{d+} - G_{d-})/h_d - sigma (T^4 - E).  Covered cells: 0.
// mag != nullptr receives, per cell and field, the sum of absolute values of
// the terms (a scale for rounding-level comparisons).
template <class S>
void residual_t(const Hier& H, const S* u, const S* z, const double* b, double a0, double dt, S* F,
                S* mag) {
  const long N = H.N;
  const S* E = u;
  const S* T = u + N;
  ORC_PARALLEL_FOR
  for (long idx = 0; idx < N; idx++) {
    int l = H.cell_level[idx];
    const int* c = &H.cell_ijk[3 * idx];
    if (H.covered(l, c)) {
      F[idx] = S(0.0);
      F[N + idx] = S(0.0);
      if (mag) { mag[idx] = S(0.0); mag[N + idx] = S(0.0); }
      continue;
    }
    S divE = S(0.0), divT = S(0.0);
    S absE = S(0.0), absT = S(0.0);
    for (int d = 0; d < 3; d++) {
      double h = H.lev[l].h[d];
      for (int s = -1; s <= 1; s += 2) {
        FluxPair<S> f = face_flux(H, E, T, z, l, c, d, s);
        divE += double(s) * f.E / h;
        divT += double(s) * f.T / h;
        if (mag) { absE += fabs(f.E) / h; absT += fabs(f.T) / h; }
      }
    }
    S zc = cube(z[idx]);
    S Tc = T[idx];
    S sigma = zc / (Tc * Tc * Tc);
    S T4 = Tc * Tc * Tc * Tc;
    S coup = sigma * (T4 - E[idx]);
    F[idx] = a0 * E[idx] - b[idx] - dt * (divE + coup);
    F[N + idx] = a0 * T[idx] - b[N + idx] - dt * (divT - coup);
    if (mag) {
      S st4 = fabs(sigma * T4), se = fabs(sigma * E[idx]);
      mag[idx] = a0 * fabs(E[idx]) + fabs(S(b[idx])) + dt * (absE + st4 + se);
      mag[N + idx] = a0 * fabs(T[idx]) + fabs(S(b[N + idx])) + dt * (absT + st4 + se);
    }
  }
}

// Weighted inner product over leaf cells of both fields: weight = cell volume
// (R5).
double wdot(const Hier& H, const double* x, const double* y) {
  double s = 0.0;
  for (int f = 0; f < 2; f++)
    for (long i = 0; i < H.N; i++) {
      if (H.covered_idx(i)) continue;
      const double* hh = H.lev[H.cell_level[i]].h;
      s += hh[0] * hh[1] * hh[2] * x[f * H.N + i] * y[f * H.N + i];
    }
  return s;
}

double wnorm1(const Hier& H, const double* x) {
  double s = 0.0;
  for (int f = 0; f < 2; f++)
    for (long i = 0; i < H.N; i++) {
      if (H.covered_idx(i)) continue;
      const double* hh = H.lev[H.cell_level[i]].h;
      s += hh[0] * hh[1] * hh[2] * std::fabs(x[f * H.N + i]);
    }
  return s;
}

// Differencing parameter of Sec. 4.1 (R6).
double fd_eps(const Hier& H, const double* u, const double* v) {
  double uv = wdot(H, u, v);
  double vv = wdot(H, v, v);
  double v1 = wnorm1(H, v);
  if (vv == 0.0) return 0.0;
  const double sq = std::sqrt(std::ldexp(1.0, -52));
  double eps;
  if (std::fabs(uv) > H.u_min * v1)
    eps = sq * uv / vv;
  else
    eps = sq * H.u_min * (uv >= 0.0 ? 1.0 : -1.0) * v1 / vv;
  for (int t = 0; t < 10; t++) {
    bool pos = true;
    for (long i = 0; i < 2 * H.N && pos; i++) {
      if (H.covered_idx(i % H.N)) continue;
      if (!(u[i] + eps * v[i] > 0.0)) pos = false;
    }
    if (pos) break;
    eps *= 0.5;
  }
  return eps;
}

void residual(const Hier& H, const double* u, const double* b, double a0, double dt, double* F) {
  residual_t<double>(H, u, H.z.data(), b, a0, dt, F, nullptr);
}

std::vector<Dual> zconst(const Hier& H) {
  std::vector<Dual> z(H.N);
  for (long i = 0; i < H.N; i++) z[i] = Dual(H.z[i], 0.0);
  return z;
}

void jv_analytic(const Hier& H, const double* u, const double* v, double a0, double dt, double* Jv) {
  const long n2 = 2 * H.N;
  std::vector<Dual> ud(n2), Fd(n2);
  std::vector<double> b0(n2, 0.0);
  for (long i = 0; i < n2; i++) ud[i] = Dual(u[i], v[i]);
  std::vector<Dual> zd = zconst(H);
  residual_t<Dual>(H, ud.data(), zd.data(), b0.data(), a0, dt, Fd.data(), nullptr);
  for (long i = 0; i < n2; i++) Jv[i] = Fd[i].d;
}

// (dF/du)^T w and (dF/dz)^T w by their definition: one Jacobian column per
// unknown (forward-mode tangent along a unit vector), each dotted with w.
// O(N^2): for small hierarchies only.
void vjp_bruteforce(const Hier& H, const double* u, const double* w, double a0, double dt,
                    double* JTw, double* dz, double* JTw_abs) {
  const long N = H.N, n2 = 2 * N;
  std::vector<Dual> ud(n2), Fd(n2);
  std::vector<double> b0(n2, 0.0);
  std::vector<Dual> zd = zconst(H);
  for (long i = 0; i < n2; i++) ud[i] = Dual(u[i], 0.0);
  for (long j = 0; j < n2; j++) {
    ud[j].d = 1.0;
    residual_t<Dual>(H, ud.data(), zd.data(), b0.data(), a0, dt, Fd.data(), nullptr);
    ud[j].d = 0.0;
    double s = 0.0, sa = 0.0;
    for (long i = 0; i < n2; i++) {
      s += w[i] * Fd[i].d;
      sa += std::fabs(w[i] * Fd[i].d);
    }
    JTw[j] = s;
    if (JTw_abs) JTw_abs[j] = sa;
  }
  if (!dz) return;
  for (long k = 0; k < N; k++) {
    zd[k].d = 1.0;
    residual_t<Dual>(H, ud.data(), zd.data(), b0.data(), a0, dt, Fd.data(), nullptr);
    zd[k].d = 0.0;
    double s = 0.0;
    for (long i = 0; i < n2; i++) s += w[i] * Fd[i].d;
    dz[k] = s;
  }
}

void jv_fd(const Hier& H, const double* u, const double* v, const double* b, double a0, double dt,
           const double* F0, double* Jv, double* eps_out) {
  const long n2 = 2 * H.N;
  double eps = fd_eps(H, u, v);
  if (eps_out) *eps_out = eps;
  if (eps == 0.0) {
    for (long i = 0; i < n2; i++) Jv[i] = 0.0;
    return;
  }
  std::vector<double> up(n2), Fp(n2), F0own;
  for (long i = 0; i < n2; i++) up[i] = u[i] + eps * v[i];
  if (!F0) {
    F0own.resize(n2);
    residual(H, u, b, a0, dt, F0own.data());
    F0 = F0own.data();
  }
  residual(H, up.data(), b, a0, dt, Fp.data());
  for (long i = 0; i < n2; i++) Jv[i] = (Fp[i] - F0[i]) / eps;
}

// ----------------------------------------------------- frozen coefficients
// D_E and D_T at a face from cell values (the same formulas as pair_flux).
void face_coefs(const Hier& H, double Ea, double Eb, double Ta, double Tb, double za, double zb,
                double h, double* DE, double* DT) {
  double Tf = 0.5 * (Ta + Tb);
  double Dr = Tf * Tf * Tf / (3.0 * (cube(za) + cube(zb)));
  double g = std::fabs(Eb - Ea) / (0.5 * h * (Ea + Eb));
  if (H.limiter == LIM_WILSON) {
    double Dh = 2.0 * Dr;
    *DE = Dh / (1.0 + Dh * g);
  } else {
    *DE = 2.0 * Dr / (1.0 + Dr * g);
  }
  *DT = H.kcond * Tf * Tf * std::sqrt(Tf);
}

inline int fdim(const int n[3], int d, int a) { return n[a] + (a == d ? 1 : 0); }
inline long fidx(const int n[3], int d, int i, int j, int k) {
  return (long)i + (long)fdim(n, d, 0) * ((long)j + (long)fdim(n, d, 1) * k);
}
inline int plane_t1(int d) { return (d + 1) % 3; }
inline int plane_t2(int d) { return (d + 2) % 3; }
// index of a cell position on the domain-face plane normal to d
inline long pidx(const int n[3], int d, const int c[3]) {
  return (long)c[plane_t1(d)] + (long)n[plane_t1(d)] * c[plane_t2(d)];
}

// pc_setup (Sec. 4.2): freeze D_E^k, D_T^k at the Newton iterate and build
// the level operators of P1 (R9-R11).
void pc_setup(Hier& H, const double* u, double a0, double dt) {
  const long N = H.N;
  H.uk.assign(u, u + 2 * N);
  H.beta = dt / a0;  // beta_n = (alpha+1)/(2 alpha+1) dt = dt / a0
  const double* E = H.uk.data();
  const double* T = H.uk.data() + N;
  for (int fld = 0; fld < 2; fld++) {
    H.opl[fld].assign(H.L, Hier::OpLevel());
    for (int l = H.L - 1; l >= 0; l--) {
      Hier::OpLevel& O = H.opl[fld][l];
      const Level& Lv = H.lev[l];
      for (int d = 0; d < 3; d++) { O.n[d] = Lv.n[d]; O.h[d] = Lv.h[d]; }
      O.amr = l;
      for (int d = 0; d < 3; d++) {
        long nf = (long)fdim(O.n, d, 0) * fdim(O.n, d, 1) * fdim(O.n, d, 2);
        O.C[d].assign(nf, 0.0);
        int t1 = plane_t1(d), t2 = plane_t2(d);
        ORC_PARALLEL_FOR
        for (int k = 0; k < fdim(O.n, d, 2); k++)
          for (int j = 0; j < fdim(O.n, d, 1); j++)
            for (int i = 0; i < fdim(O.n, d, 0); i++) {
              int bcell[3] = {i, j, k};              // high-side cell of the face
              int acell[3] = {i, j, k};
              acell[d] -= 1;                         // low-side cell
              if (!H.inside(l, acell) || !H.inside(l, bcell)) continue;  // physical
              long ia = H.cell(l, acell), ib = H.cell(l, bcell);
              if (ia < 0 && ib < 0) continue;
              bool cov = (ia >= 0 && H.covered(l, acell)) || (ib >= 0 && H.covered(l, bcell));
              double C;
              if (cov) {
                // R11: mean of the four coincident fine faces
                const Hier::OpLevel& F = H.opl[fld][l + 1];
                double s = 0.0;
                for (int a = 0; a < 2; a++)
                  for (int bb = 0; bb < 2; bb++) {
                    int q[3];
                    q[d] = 2 * bcell[d];
                    q[t1] = 2 * bcell[t1] + a;
                    q[t2] = 2 * bcell[t2] + bb;
                    s += F.C[d][fidx(F.n, d, q[0], q[1], q[2])];
                  }
                C = 0.25 * s;
              } else {
                double Ea, Eb, Ta, Tb, za, zb;
                if (ia >= 0) { Ea = E[ia]; Ta = T[ia]; za = H.z[ia]; }
                else {
                  Ea = cf_ghost(H, E, l, bcell, d, -1);
                  Ta = cf_ghost(H, T, l, bcell, d, -1);
                  za = cf_ghost_z(H, l, bcell, d, -1);
                }
                if (ib >= 0) { Eb = E[ib]; Tb = T[ib]; zb = H.z[ib]; }
                else {
                  Eb = cf_ghost(H, E, l, acell, d, +1);
                  Tb = cf_ghost(H, T, l, acell, d, +1);
                  zb = cf_ghost_z(H, l, acell, d, +1);
                }
                double DE, DT;
                face_coefs(H, Ea, Eb, Ta, Tb, za, zb, Lv.h[d], &DE, &DT);
                C = (fld == 0) ? DE : DT;
              }
              O.C[d][fidx(O.n, d, i, j, k)] = C;
            }
      }
      // Robin D_b on the six domain faces (E only; T is Neumann everywhere)
      for (int face = 0; face < 6; face++) {
        int d = face / 2, t1 = plane_t1(d), t2 = plane_t2(d);
        O.Db[face].assign((long)O.n[t1] * O.n[t2], 0.0);
        if (fld != 0 || H.bc_type[face] != BC_ROBIN) continue;
        for (int b2 = 0; b2 < O.n[t2]; b2++)
          for (int b1 = 0; b1 < O.n[t1]; b1++) {
            int c[3];
            c[d] = (face % 2 == 0) ? 0 : O.n[d] - 1;
            c[t1] = b1;
            c[t2] = b2;
            long ic = H.cell(l, c);
            if (ic < 0) continue;
            double v;
            if (H.covered(l, c)) {
              const Hier::OpLevel& F = H.opl[fld][l + 1];
              double s = 0.0;
              for (int a = 0; a < 2; a++)
                for (int bb = 0; bb < 2; bb++) {
                  int q[3];
                  q[d] = (face % 2 == 0) ? 0 : F.n[d] - 1;
                  q[t1] = 2 * b1 + a;
                  q[t2] = 2 * b2 + bb;
                  s += F.Db[face][pidx(F.n, d, q)];
                }
              v = 0.25 * s;
            } else {
              v = cube(T[ic]) / (3.0 * cube(H.z[ic]));
            }
            O.Db[face][pidx(O.n, d, c)] = v;
          }
      }
    }
    // GMG levels below AMR level 0 (level 0 is a single box covering the
    // domain); m = 0 is AMR level 0 itself.
    H.mg[fld].assign(H.nmg, Hier::OpLevel());
    H.mg[fld][0] = H.opl[fld][0];
    H.mg[fld][0].amr = -1;
    for (int m = 1; m < H.nmg; m++) {
      const Hier::OpLevel& F = H.mg[fld][m - 1];
      Hier::OpLevel& O = H.mg[fld][m];
      for (int d = 0; d < 3; d++) { O.n[d] = F.n[d] / 2; O.h[d] = 2.0 * F.h[d]; }
      O.amr = -1;
      for (int d = 0; d < 3; d++) {
        int t1 = plane_t1(d), t2 = plane_t2(d);
        long nf = (long)fdim(O.n, d, 0) * fdim(O.n, d, 1) * fdim(O.n, d, 2);
        O.C[d].assign(nf, 0.0);
        ORC_PARALLEL_FOR
        for (int k = 0; k < fdim(O.n, d, 2); k++)
          for (int j = 0; j < fdim(O.n, d, 1); j++)
            for (int i = 0; i < fdim(O.n, d, 0); i++) {
              int f[3] = {i, j, k};
              double s = 0.0;
              for (int a = 0; a < 2; a++)
                for (int bb = 0; bb < 2; bb++) {
                  int q[3];
                  q[d] = 2 * f[d];
                  q[t1] = 2 * f[t1] + a;
                  q[t2] = 2 * f[t2] + bb;
                  s += F.C[d][fidx(F.n, d, q[0], q[1], q[2])];
                }
              O.C[d][fidx(O.n, d, i, j, k)] = 0.25 * s;
            }
      }
      for (int face = 0; face < 6; face++) {
        int d = face / 2, t1 = plane_t1(d), t2 = plane_t2(d);
        O.Db[face].assign((long)O.n[t1] * O.n[t2], 0.0);
        for (int b2 = 0; b2 < O.n[t2]; b2++)
          for (int b1 = 0; b1 < O.n[t1]; b1++) {
            double s = 0.0;
            for (int a = 0; a < 2; a++)
              for (int bb = 0; bb < 2; bb++) {
                int q[3];
                q[d] = 0;
                q[t1] = 2 * b1 + a;
                q[t2] = 2 * b2 + bb;
                s += F.Db[face][pidx(F.n, d, q)];
              }
            int c[3];
            c[d] = 0;
            c[t1] = b1;
            c[t2] = b2;
            O.Db[face][pidx(O.n, d, c)] = 0.25 * s;
          }
      }
    }
  }
  H.pc_ready = true;
}

// ------------------------------------------------------ P1 level operators
// A level grid: either AMR level `amr` (cells that exist in its patches) or a
// full GMG box.  Values are stored densely over the level index space.
struct Grid {
  const Hier* H;
  const Hier::OpLevel* O;
  int fld;
  bool exists(const int c[3]) const {
    for (int d = 0; d < 3; d++) if (c[d] < 0 || c[d] >= O->n[d]) return false;
    if (O->amr < 0) return true;
    return H->cell(O->amr, c) >= 0;
  }
  bool in_domain(const int c[3]) const {
    for (int d = 0; d < 3; d++) if (c[d] < 0 || c[d] >= O->n[d]) return false;
    return true;
  }
  long di(const int c[3]) const {
    return (long)c[0] + (long)O->n[0] * ((long)c[1] + (long)O->n[1] * c[2]);
  }
  long ncell() const { return (long)O->n[0] * O->n[1] * O->n[2]; }
};

// Diagonal and off-diagonal sum of (I - beta div D grad) at cell c of a level
// grid, with homogeneous coarse-fine ghosts e_g = e_c/3 (R9), zero-flux
// Neumann faces and the linearised homogeneous Robin ghost.
void level_row(const Grid& G, const std::vector<double>& e, const int c[3], double* diag,
               double* off) {
  const Hier& H = *G.H;
  const Hier::OpLevel& O = *G.O;
  double beta = H.beta;
  double dg = 1.0, of = 0.0;
  for (int d = 0; d < 3; d++) {
    double h = O.h[d];
    for (int s = -1; s <= 1; s += 2) {
      int g[3] = {c[0], c[1], c[2]};
      g[d] += s;
      int face = 2 * d + (s > 0 ? 1 : 0);
      if (!G.in_domain(g)) {
        if (G.fld == 0 && H.bc_type[face] == BC_ROBIN) {
          double Db = O.Db[face][pidx(O.n, d, c)];
          dg += beta * 2.0 * Db / (h * (4.0 * Db + h));
        }
        continue;
      }
      int fc[3] = {c[0], c[1], c[2]};
      if (s > 0) fc[d] += 1;
      double C = O.C[d][fidx(O.n, d, fc[0], fc[1], fc[2])];
      if (G.exists(g)) {
        dg += beta * C / (h * h);
        of += beta * C / (h * h) * e[G.di(g)];
      } else {
        dg += beta * (2.0 / 3.0) * C / (h * h);
      }
    }
  }
  *diag = dg;
  *off = of;
}

void level_apply(const Grid& G, const std::vector<double>& e, std::vector<double>& y) {
  y.assign(G.ncell(), 0.0);
  ORC_PARALLEL_FOR
  for (int k = 0; k < G.O->n[2]; k++)
    for (int j = 0; j < G.O->n[1]; j++)
      for (int i = 0; i < G.O->n[0]; i++) {
        int c[3] = {i, j, k};
        if (!G.exists(c)) continue;
        double dg, of;
        level_row(G, e, c, &dg, &of);
        y[G.di(c)] = dg * e[G.di(c)] - of;
      }
}

// Red-black Gauss-Seidel sweep (R12): colour = (i+j+k) % 2.
void rbgs(const Grid& G, std::vector<double>& e, const std::vector<double>& f, int sweeps,
          bool red_first) {
  for (int sw = 0; sw < sweeps; sw++)
    for (int pass = 0; pass < 2; pass++) {
      int colour = red_first ? pass : 1 - pass;
      ORC_PARALLEL_FOR
      for (int k = 0; k < G.O->n[2]; k++)
        for (int j = 0; j < G.O->n[1]; j++)
          for (int i = 0; i < G.O->n[0]; i++) {
            if ((i + j + k) % 2 != colour) continue;
            int c[3] = {i, j, k};
            if (!G.exists(c)) continue;
            double dg, of;
            level_row(G, e, c, &dg, &of);
            e[G.di(c)] = (f[G.di(c)] + of) / dg;
          }
    }
}

// Damped point Jacobi sweeps (Sec. 4.3 names damped point Jacobi as an
// alternative smoother): every cell from the previous iterate,
//   e <- e + omega ((f + off(e)) / diag - e).
void jacobi(const Grid& G, std::vector<double>& e, const std::vector<double>& f, int sweeps,
            double omega) {
  std::vector<double> en;
  for (int sw = 0; sw < sweeps; sw++) {
    en = e;
    ORC_PARALLEL_FOR
    for (int k = 0; k < G.O->n[2]; k++)
      for (int j = 0; j < G.O->n[1]; j++)
        for (int i = 0; i < G.O->n[0]; i++) {
          int c[3] = {i, j, k};
          if (!G.exists(c)) continue;
          double dg, of;
          level_row(G, e, c, &dg, &of);
          const long q = G.di(c);
          en[q] = e[q] + omega * ((f[q] + of) / dg - e[q]);
        }
    e.swap(en);
  }
}

// Block Gauss-Seidel (Sec. 4.3 names it without saying what the blocks are;
// reading R26): the blocks are the x-lines of a box level, each solved
// exactly (a tridiagonal system: the line's cells coupled through their x
// faces, the y- and z-neighbours taken at their current values), the lines
// coloured by the parity of j + k, red lines first in pre-smoothing and
// black lines first in post-smoothing.  A colour's lines do not couple, so
// one colour is a block Jacobi pass and the two colours a block
// Gauss-Seidel sweep.  The AMR patch levels keep point red-black sweeps.
void xline_gs(const Grid& G, std::vector<double>& e, const std::vector<double>& f, int sweeps,
              bool red_first) {
  const Hier& H = *G.H;
  const Hier::OpLevel& O = *G.O;
  const double beta = H.beta;
  const int n0 = O.n[0], n1 = O.n[1], n2 = O.n[2];
  for (int sw = 0; sw < sweeps; sw++)
    for (int pass = 0; pass < 2; pass++) {
      int colour = red_first ? pass : 1 - pass;
      ORC_PARALLEL_FOR
      for (int k = 0; k < n2; k++)
        for (int j = 0; j < n1; j++) {
          if ((j + k) % 2 != colour) continue;
          // the line's tridiagonal system: lo e_{i-1} + dg e_i + hi e_{i+1} = rhs
          std::vector<double> lo(n0, 0.0), dg(n0, 1.0), hi(n0, 0.0), rhs(n0, 0.0);
          for (int i = 0; i < n0; i++) {
            int c[3] = {i, j, k};
            double d = 1.0, of = 0.0;
            for (int dd = 0; dd < 3; dd++) {
              double h = O.h[dd];
              for (int s = -1; s <= 1; s += 2) {
                int g[3] = {c[0], c[1], c[2]};
                g[dd] += s;
                int face = 2 * dd + (s > 0 ? 1 : 0);
                if (!G.in_domain(g)) {
                  if (G.fld == 0 && H.bc_type[face] == BC_ROBIN) {
                    double Db = O.Db[face][pidx(O.n, dd, c)];
                    d += beta * 2.0 * Db / (h * (4.0 * Db + h));
                  }
                  continue;
                }
                int fc[3] = {c[0], c[1], c[2]};
                if (s > 0) fc[dd] += 1;
                double a = beta * O.C[dd][fidx(O.n, dd, fc[0], fc[1], fc[2])] / (h * h);
                d += a;
                if (dd == 0) {
                  if (s < 0) lo[i] = -a; else hi[i] = -a;
                } else {
                  of += a * e[G.di(g)];
                }
              }
            }
            dg[i] = d;
            rhs[i] = f[G.di(c)] + of;
          }
          // Thomas algorithm
          std::vector<double> cp(n0), dp(n0);
          cp[0] = hi[0] / dg[0];
          dp[0] = rhs[0] / dg[0];
          for (int i = 1; i < n0; i++) {
            double m = dg[i] - lo[i] * cp[i - 1];
            cp[i] = hi[i] / m;
            dp[i] = (rhs[i] - lo[i] * dp[i - 1]) / m;
          }
          int cl[3] = {n0 - 1, j, k};
          e[G.di(cl)] = dp[n0 - 1];
          for (int i = n0 - 2; i >= 0; i--) {
            int c[3] = {i, j, k}, c1[3] = {i + 1, j, k};
            e[G.di(c)] = dp[i] - cp[i] * e[G.di(c1)];
          }
        }
    }
}

// the smoother selected for the V-cycle
void smooth(const Grid& G, std::vector<double>& e, const std::vector<double>& f, int sweeps,
            bool red_first) {
  if (G.H->smoother == 1) jacobi(G, e, f, sweeps, G.H->omega);
  else if (G.H->smoother == 2 && G.O->amr < 0) xline_gs(G, e, f, sweeps, red_first);
  else rbgs(G, e, f, sweeps, red_first);
}

// Trilinear prolongation of a coarse dense array to one fine cell q (R13).
double prolong_at(const int cn[3], const std::vector<double>& ec, const int q[3]) {
  int p[3], o[3];
  for (int d = 0; d < 3; d++) {
    p[d] = q[d] / 2;
    o[d] = (q[d] % 2 == 0) ? -1 : 1;
    if (p[d] + o[d] < 0 || p[d] + o[d] >= cn[d]) o[d] = 0;
  }
  double s = 0.0;
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++)
      for (int e = 0; e < 2; e++) {
        double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (e ? 0.25 : 0.75);
        int i = p[0] + (a ? o[0] : 0), j = p[1] + (b ? o[1] : 0), k = p[2] + (e ? o[2] : 0);
        s += w * ec[(long)i + (long)cn[0] * ((long)j + (long)cn[1] * k)];
      }
  return s;
}

// Geometric multigrid V(nu1, nu2) on the base box (R10).
void gmg_vcycle(const Hier& H, int fld, int m, std::vector<double>& e, const std::vector<double>& f) {
  Grid G{&H, &H.mg[fld][m], fld};
  if (m == H.nmg - 1) {
    smooth(G, e, f, H.coarse_sweeps, true);
    return;
  }
  smooth(G, e, f, H.nu1, true);
  std::vector<double> Le;
  level_apply(G, e, Le);
  const Hier::OpLevel& Oc = H.mg[fld][m + 1];
  Grid Gc{&H, &Oc, fld};
  std::vector<double> fc(Gc.ncell(), 0.0), ec(Gc.ncell(), 0.0);
  ORC_PARALLEL_FOR
  for (int k = 0; k < Oc.n[2]; k++)
    for (int j = 0; j < Oc.n[1]; j++)
      for (int i = 0; i < Oc.n[0]; i++) {
        double s = 0.0;
        for (int a = 0; a < 2; a++)
          for (int b = 0; b < 2; b++)
            for (int c2 = 0; c2 < 2; c2++) {
              int q[3] = {2 * i + a, 2 * j + b, 2 * k + c2};
              s += f[G.di(q)] - Le[G.di(q)];
            }
        int cc[3] = {i, j, k};
        fc[Gc.di(cc)] = s / 8.0;
      }
  gmg_vcycle(H, fld, m + 1, ec, fc);
  ORC_PARALLEL_FOR
  for (int k = 0; k < G.O->n[2]; k++)
    for (int j = 0; j < G.O->n[1]; j++)
      for (int i = 0; i < G.O->n[0]; i++) {
        int q[3] = {i, j, k};
        e[G.di(q)] += prolong_at(Oc.n, ec, q);
      }
  smooth(G, e, f, H.nu2, false);
}

// Composite operator L^c of one P1 block applied to a leaf vector x (Sec. 4.3):
// the same face classification as the residual, with frozen coefficients.
double comp_flux(const Hier& H, int fld, const double* x, int l, const int c[3], int d, int s) {
  const Hier::OpLevel& O = H.opl[fld][l];
  double h = O.h[d];
  long ic = H.cell(l, c);
  int g[3] = {c[0], c[1], c[2]};
  g[d] += s;
  int face = 2 * d + (s > 0 ? 1 : 0);
  if (!H.inside(l, g)) {
    if (fld == 0 && H.bc_type[face] == BC_ROBIN) {
      double Db = O.Db[face][pidx(O.n, d, c)];
      double a = Db / (2.0 * h);
      double xg = x[ic] * (a - 0.125) / (a + 0.125);
      return (s > 0) ? Db * (xg - x[ic]) / h : Db * (x[ic] - xg) / h;
    }
    return 0.0;
  }
  int fc[3] = {c[0], c[1], c[2]};
  if (s > 0) fc[d] += 1;
  double C = O.C[d][fidx(O.n, d, fc[0], fc[1], fc[2])];
  long ig = H.cell(l, g);
  double xg;
  if (ig >= 0) {
    if (H.covered(l, g)) {
      int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      double sum = 0.0;
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
          int q[3];
          q[d] = (s > 0) ? 2 * g[d] : 2 * g[d] + 1;
          q[t1] = 2 * c[t1] + a;
          q[t2] = 2 * c[t2] + b;
          sum += comp_flux(H, fld, x, l + 1, q, d, -s);
        }
      return 0.25 * sum;
    }
    xg = x[ig];
  } else {
    xg = cf_ghost(H, x, l, c, d, s);
  }
  return (s > 0) ? C * (xg - x[ic]) / h : C * (x[ic] - xg) / h;
}

// y = L^c x for one field (x, y of length N); covered cells get 0.
void comp_apply(const Hier& H, int fld, const double* x, double* y) {
  ORC_PARALLEL_FOR
  for (long idx = 0; idx < H.N; idx++) {
    int l = H.cell_level[idx];
    const int* c = &H.cell_ijk[3 * idx];
    if (H.covered(l, c)) { y[idx] = 0.0; continue; }
    double div = 0.0;
    for (int d = 0; d < 3; d++)
      for (int s = -1; s <= 1; s += 2)
        div += double(s) * comp_flux(H, fld, x, l, c, d, s) / H.lev[l].h[d];
    y[idx] = x[idx] - H.beta * div;
  }
}

// Replace covered values by the mean of their children, finest first.
void average_down(const Hier& H, double* x) {
  for (int l = H.L - 2; l >= 0; l--) {
    ORC_PARALLEL_FOR
    for (long idx = 0; idx < H.N; idx++) {
      if (H.cell_level[idx] != l) continue;
      const int* c = &H.cell_ijk[3 * idx];
      if (!H.covered(l, c)) continue;
      double s = 0.0;
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
          for (int e = 0; e < 2; e++)
            s += x[H.cell(l + 1, 2 * c[0] + a, 2 * c[1] + b, 2 * c[2] + e)];
      x[idx] = s / 8.0;
    }
  }
}

// Dense level array <-> hierarchy vector helpers
void gather_level(const Hier& H, int l, const double* x, std::vector<double>& out) {
  const Level& Lv = H.lev[l];
  out.assign((long)Lv.n[0] * Lv.n[1] * Lv.n[2], 0.0);
  ORC_PARALLEL_FOR
  for (long idx = 0; idx < H.N; idx++) {
    if (H.cell_level[idx] != l) continue;
    const int* c = &H.cell_ijk[3 * idx];
    out[(long)c[0] + (long)Lv.n[0] * ((long)c[1] + (long)Lv.n[1] * c[2])] = x[idx];
  }
}

// u^c += P^c_l e^l: add e to leaf cells of level l and its trilinear
// interpolation to every finer level (R9).
void correct_composite(const Hier& H, int l, const std::vector<double>& e, double* u) {
  std::vector<double> cur = e, next;
  for (int m = l; m < H.L; m++) {
    const Level& Lv = H.lev[m];
    if (m > l) {
      const Level& Lc = H.lev[m - 1];
      next.assign((long)Lv.n[0] * Lv.n[1] * Lv.n[2], 0.0);
      ORC_PARALLEL_FOR
      for (long idx = 0; idx < H.N; idx++) {
        if (H.cell_level[idx] != m) continue;
        const int* q = &H.cell_ijk[3 * idx];
        next[(long)q[0] + (long)Lv.n[0] * ((long)q[1] + (long)Lv.n[1] * q[2])] =
            prolong_at(Lc.n, cur, q);
      }
      cur.swap(next);
    }
    ORC_PARALLEL_FOR
    for (long idx = 0; idx < H.N; idx++) {
      if (H.cell_level[idx] != m) continue;
      const int* c = &H.cell_ijk[3 * idx];
      if (H.covered(m, c)) continue;
      u[idx] += cur[(long)c[0] + (long)Lv.n[0] * ((long)c[1] + (long)Lv.n[1] * c[2])];
    }
  }
}

// One FAC V(nu1, nu2) cycle (Algorithm 1, readings R9/R10) for
// L^c u = f, from u = 0.  f, u: one field, hierarchy layout.
void fac_vcycle(const Hier& H, int fld, const double* f, double* u) {
  const long N = H.N;
  std::vector<double> r(N), Lu(N), fl, el;
  for (long i = 0; i < N; i++) u[i] = 0.0;
  auto update_residual = [&]() {
    comp_apply(H, fld, u, Lu.data());
    for (long i = 0; i < N; i++) r[i] = f[i] - Lu[i];
    average_down(H, r.data());  // R^c_l r^c for every level at once
  };
  update_residual();
  for (int l = H.L - 1; l >= 1; l--) {
    gather_level(H, l, r.data(), fl);
    el.assign(fl.size(), 0.0);
    Grid G{&H, &H.opl[fld][l], fld};
    smooth(G, el, fl, H.nu1, true);
    correct_composite(H, l, el, u);
    update_residual();
  }
  gather_level(H, 0, r.data(), fl);
  el.assign(fl.size(), 0.0);
  gmg_vcycle(H, fld, 0, el, fl);
  correct_composite(H, 0, el, u);
  for (int l = 1; l < H.L; l++) {
    update_residual();
    gather_level(H, l, r.data(), fl);
    el.assign(fl.size(), 0.0);
    Grid G{&H, &H.opl[fld][l], fld};
    smooth(G, el, fl, H.nu2, false);
    correct_composite(H, l, el, u);
  }
  for (long i = 0; i < N; i++)
    if (H.covered_idx(i)) u[i] = 0.0;
}

// y = P^{-1} w = P2^{-1} (P1^{-1} w)  (Sec. 4.2).
void pc_apply(const Hier& H, const double* w, double* y) {
  const long N = H.N;
  std::vector<double> zE(N), zT(N);
  fac_vcycle(H, 0, w, zE.data());
  fac_vcycle(H, 1, w + N, zT.data());
  const double beta = H.beta;
  ORC_PARALLEL_FOR
  for (long i = 0; i < N; i++) {
    if (H.covered_idx(i)) { y[i] = 0.0; y[N + i] = 0.0; continue; }
    double T = H.uk[N + i];
    double T3 = T * T * T;
    double sigma = cube(H.z[i]) / T3;
    // P2 = [[1 + sigma beta, -sigma beta T^3], [-sigma beta, 1 + sigma beta T^3]]
    double a = 1.0 + sigma * beta, bb = -sigma * beta * T3;
    double c = -sigma * beta, dd = 1.0 + sigma * beta * T3;
    double det = a * dd - bb * c;
    y[i] = (dd * zE[i] - bb * zT[i]) / det;
    y[N + i] = (a * zT[i] - c * zE[i]) / det;
  }
}

// ------------------------------------------------------------ GMRES, Newton
struct Stats {
  int newton_its = 0, krylov_its = 0, status = 0;
  double fnorm0 = 0, fnorm = 0;
};

// Right-preconditioned restarted GMRES (Sec. 4.1-4.2) with modified
// Gram-Schmidt and Givens rotations, for J x = rhs to ||rhs - J x|| <= tol.
// The preconditioned directions z_j = P^{-1} v_j are kept, so the update is
// x = x0 + sum_j y_j z_j.
int gmres(Hier& H, const double* u, const double* b, double a0, double dt, const double* F0,
          const double* rhs, double tol, double* x, int* its) {
  const long n2 = 2 * H.N;
  const int m = H.restart;
  std::vector<std::vector<double>> V(m + 1, std::vector<double>(n2)), Z(m, std::vector<double>(n2));
  std::vector<double> Hm((m + 1) * m), cs(m), sn(m), g(m + 1), w(n2), r(n2), yv(m);
  auto J = [&](const double* v, double* out) {
    if (H.jv_mode == JV_ANALYTIC) jv_analytic(H, u, v, a0, dt, out);
    else jv_fd(H, u, v, b, a0, dt, F0, out, nullptr);
  };
  for (long i = 0; i < n2; i++) { x[i] = 0.0; r[i] = rhs[i]; }
  int total = 0;
  double rn = std::sqrt(wdot(H, r.data(), r.data()));
  if (rn <= tol) { *its = 0; return 0; }
  while (total < H.max_krylov) {
    for (long i = 0; i < n2; i++) V[0][i] = r[i] / rn;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = rn;
    int j = 0;
    bool conv = false;
    for (; j < m && total < H.max_krylov; j++) {
      pc_apply(H, V[j].data(), Z[j].data());
      J(Z[j].data(), w.data());
      total++;
      for (int i = 0; i <= j; i++) {
        double hij = wdot(H, w.data(), V[i].data());
        Hm[i * m + j] = hij;
        for (long t = 0; t < n2; t++) w[t] -= hij * V[i][t];
      }
      double hn = std::sqrt(wdot(H, w.data(), w.data()));
      Hm[(j + 1) * m + j] = hn;
      for (long t = 0; t < n2; t++) V[j + 1][t] = (hn > 0.0) ? w[t] / hn : 0.0;
      for (int i = 0; i < j; i++) {
        double t0 = cs[i] * Hm[i * m + j] + sn[i] * Hm[(i + 1) * m + j];
        double t1 = -sn[i] * Hm[i * m + j] + cs[i] * Hm[(i + 1) * m + j];
        Hm[i * m + j] = t0;
        Hm[(i + 1) * m + j] = t1;
      }
      double a = Hm[j * m + j], bb = Hm[(j + 1) * m + j];
      double den = std::sqrt(a * a + bb * bb);
      cs[j] = (den > 0.0) ? a / den : 1.0;
      sn[j] = (den > 0.0) ? bb / den : 0.0;
      Hm[j * m + j] = den;
      Hm[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (std::fabs(g[j + 1]) <= tol || hn == 0.0) { j++; conv = true; break; }
    }
    // back substitution H y = g
    for (int i = j - 1; i >= 0; i--) {
      double s = g[i];
      for (int t = i + 1; t < j; t++) s -= Hm[i * m + t] * yv[t];
      yv[i] = s / Hm[i * m + i];
    }
    for (int i = 0; i < j; i++)
      for (long t = 0; t < n2; t++) x[t] += yv[i] * Z[i][t];
    J(x, w.data());
    for (long t = 0; t < n2; t++) r[t] = rhs[t] - w[t];
    rn = std::sqrt(wdot(H, r.data(), r.data()));
    if (conv || rn <= tol) { *its = total; return 0; }
  }
  *its = total;
  return 1;
}

// Inexact Newton (Sec. 4.1) with Eisenstat-Walker forcing (R8) and the
// positivity-constrained update (R7).  u: initial guess in, solution out.
int newton(Hier& H, double* u, const double* b, double a0, double dt, Stats* st) {
  const long n2 = 2 * H.N;
  std::vector<double> F(n2), v(n2), rhs(n2);
  residual(H, u, b, a0, dt, F.data());
  double fn = std::sqrt(wdot(H, F.data(), F.data()));
  st->fnorm0 = fn;
  double stop = H.rtol * fn + H.atol;
  double eta = H.eta0;
  int it = 0, kits = 0, status = 0;
  while (fn > stop && it < H.max_newton) {
    pc_setup(H, u, a0, dt);
    for (long i = 0; i < n2; i++) rhs[i] = -F[i];
    int its = 0;
    gmres(H, u, b, a0, dt, F.data(), rhs.data(), eta * fn, v.data(), &its);
    kits += its;
    double lam = 1.0;
    for (long i = 0; i < n2; i++) {
      if (H.covered_idx(i % H.N)) continue;
      if (v[i] < 0.0) lam = std::min(lam, 0.9 * u[i] / (-v[i]));
    }
    for (long i = 0; i < n2; i++) u[i] += lam * v[i];
    residual(H, u, b, a0, dt, F.data());
    double fold = fn;
    fn = std::sqrt(wdot(H, F.data(), F.data()));
    double rat = fn / fold;
    double etaA = H.ew_gamma * rat * rat;
    double etaN;
    if (H.ew_gamma * eta * eta <= 0.1) etaN = std::min(H.eta_max, etaA);
    else etaN = std::min(H.eta_max, std::max(etaA, H.ew_gamma * eta * eta));
    eta = std::min(H.eta_max, std::max(etaN, 0.5 * stop / fn));
    it++;
  }
  if (fn > stop) status = 1;
  for (int f = 0; f < 2; f++) average_down(H, u + f * H.N);
  st->newton_its = it;
  st->krylov_its = kits;
  st->fnorm = fn;
  st->status = status;
  return status;
}

// -------------------------------------------------------------- ghosts
// Ghost value of E, T, z at face (c, d, s) of a level-l cell, as seen by the
// residual: physical (R4), sibling (composite value), coarse-fine.
void ghost_of(const Hier& H, const double* u, int l, const int c[3], int d, int s, double* Eg,
              double* Tg, double* zg) {
  const long N = H.N;
  const double* E = u;
  const double* T = u + N;
  long ic = H.cell(l, c);
  int g[3] = {c[0], c[1], c[2]};
  g[d] += s;
  if (!H.inside(l, g)) {
    int face = 2 * d + (s > 0 ? 1 : 0);
    *Tg = T[ic];
    *zg = H.z[ic];
    if (H.bc_type[face] == BC_ROBIN)
      *Eg = robin_ghost(E[ic], T[ic], H.z[ic], H.lev[l].h[d], H.bc_R[face]);
    else
      *Eg = E[ic];
    return;
  }
  long ig = H.cell(l, g);
  if (ig >= 0) {
    // sibling: the stored value (a covered sibling is never used by the
    // residual, whose flux there comes from flux matching)
    *Eg = E[ig];
    *Tg = T[ig];
    *zg = H.z[ig];
    return;
  }
  *Eg = cf_ghost(H, E, l, c, d, s);
  *Tg = cf_ghost(H, T, l, c, d, s);
  *zg = cf_ghost_z(H, l, c, d, s);
}

}  // namespace

// =================================================================== C API
extern "C" {

struct orc_hier;

orc_hier* orc_create(int nlevels, const int* nboxes, const int* boxes, const int* bc_type,
                     const double* bc_R, double kcond, int limiter) {
  Hier* H = new Hier();
  H->L = nlevels;
  H->kcond = kcond;
  H->limiter = limiter;
  for (int f = 0; f < 6; f++) { H->bc_type[f] = bc_type[f]; H->bc_R[f] = bc_R[f]; }
  H->lev.resize(nlevels);
  int bi = 0;
  // level 0 must be one box starting at the origin: it defines the domain
  const int* b0 = boxes;
  if (nboxes[0] != 1 || b0[0] != 0 || b0[1] != 0 || b0[2] != 0) {
    std::fprintf(stderr, "orc_create: level 0 must be one box at the origin\n");
    delete H;
    return nullptr;
  }
  long off = 0;
  for (int l = 0; l < nlevels; l++) {
    Level& Lv = H->lev[l];
    for (int d = 0; d < 3; d++) {
      Lv.n[d] = (b0[3 + d] + 1) << l;
      Lv.h[d] = 1.0 / Lv.n[d];
    }
    Lv.map.assign((long)Lv.n[0] * Lv.n[1] * Lv.n[2], -1);
    for (int p = 0; p < nboxes[l]; p++, bi++) {
      const int* bx = boxes + 6 * bi;
      for (int t = 0; t < 6; t++) Lv.box.push_back(bx[t]);
      Lv.off.push_back(off);
      for (int k = bx[2]; k <= bx[5]; k++)
        for (int j = bx[1]; j <= bx[4]; j++)
          for (int i = bx[0]; i <= bx[3]; i++) {
            if (i < 0 || j < 0 || k < 0 || i >= Lv.n[0] || j >= Lv.n[1] || k >= Lv.n[2]) {
              std::fprintf(stderr, "orc_create: box outside the domain\n");
              delete H;
              return nullptr;
            }
            long di = (long)i + (long)Lv.n[0] * ((long)j + (long)Lv.n[1] * k);
            if (Lv.map[di] >= 0) {
              std::fprintf(stderr, "orc_create: overlapping boxes\n");
              delete H;
              return nullptr;
            }
            Lv.map[di] = off;
            H->cell_level.push_back(l);
            H->cell_ijk.push_back(i);
            H->cell_ijk.push_back(j);
            H->cell_ijk.push_back(k);
            off++;
          }
    }
  }
  H->N = off;
  H->z.assign(H->N, 1.0);
  // Fine boxes must be aligned to the refinement ratio 2 and properly nested:
  // the coarsened box grown by one coarse cell (clipped to the domain) must lie
  // inside level l-1.
  for (int l = 1; l < nlevels; l++) {
    const Level& Lv = H->lev[l];
    for (size_t p = 0; p < Lv.off.size(); p++) {
      const int* bx = &Lv.box[6 * p];
      for (int d = 0; d < 3; d++)
        if (bx[d] % 2 != 0 || bx[3 + d] % 2 != 1) {
          std::fprintf(stderr, "orc_create: box not aligned to ratio 2\n");
          delete H;
          return nullptr;
        }
      for (int k = bx[2] / 2 - 1; k <= bx[5] / 2 + 1; k++)
        for (int j = bx[1] / 2 - 1; j <= bx[4] / 2 + 1; j++)
          for (int i = bx[0] / 2 - 1; i <= bx[3] / 2 + 1; i++) {
            int c[3] = {i, j, k};
            if (!H->inside(l - 1, c)) continue;
            if (H->cell(l - 1, c) < 0) {
              std::fprintf(stderr, "orc_create: level %d not properly nested\n", l);
              delete H;
              return nullptr;
            }
          }
    }
  }
  return reinterpret_cast<orc_hier*>(H);
}

void orc_destroy(orc_hier* h) { delete reinterpret_cast<Hier*>(h); }

// Host threads for the cell loops (1 without OpenMP); returns the count used.
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

long orc_ncells(orc_hier* h) { return reinterpret_cast<Hier*>(h)->N; }

void orc_set_material(orc_hier* h, const float* z) {
  Hier* H = reinterpret_cast<Hier*>(h);
  for (long i = 0; i < H->N; i++) H->z[i] = z[i];
}

void orc_set_solver(orc_hier* h, int restart, int max_krylov, int jv_mode, int nu1, int nu2,
                    int nmg, int coarse_sweeps, double rtol, double atol, int max_newton) {
  Hier* H = reinterpret_cast<Hier*>(h);
  H->restart = restart;
  H->max_krylov = max_krylov;
  H->jv_mode = jv_mode;
  H->nu1 = nu1;
  H->nu2 = nu2;
  H->nmg = nmg;
  H->coarse_sweeps = coarse_sweeps;
  H->rtol = rtol;
  H->atol = atol;
  H->max_newton = max_newton;
}

// smoother of the V-cycle: 0 red-black Gauss-Seidel, 1 damped point Jacobi,
// 2 x-line block Gauss-Seidel on the box levels (R26)
void orc_set_smoother(orc_hier* h, int kind, double omega) {
  Hier* H = reinterpret_cast<Hier*>(h);
  H->smoother = kind;
  H->omega = omega;
}

void orc_leaf_mask(orc_hier* h, unsigned char* leaf) {
  Hier* H = reinterpret_cast<Hier*>(h);
  for (long i = 0; i < H->N; i++) leaf[i] = H->covered_idx(i) ? 0 : 1;
}

void orc_residual(orc_hier* h, const double* u, const double* b, double a0, double dt, double* F) {
  residual(*reinterpret_cast<Hier*>(h), u, b, a0, dt, F);
}

void orc_residual_scale(orc_hier* h, const double* u, const double* b, double a0, double dt,
                        double* S) {
  Hier* H = reinterpret_cast<Hier*>(h);
  std::vector<double> F(2 * H->N);
  residual_t<double>(*H, u, H->z.data(), b, a0, dt, F.data(), S);
}

void orc_jv_analytic(orc_hier* h, const double* u, const double* v, double a0, double dt,
                     double* Jv) {
  jv_analytic(*reinterpret_cast<Hier*>(h), u, v, a0, dt, Jv);
}

// Scale for tangent comparisons: per cell, a0|v| + dt * sum of |tangent| of
// every face flux and coupling term.
void orc_jv_scale(orc_hier* h, const double* u, const double* v, double a0, double dt, double* S) {
  Hier* H = reinterpret_cast<Hier*>(h);
  const long N = H->N, n2 = 2 * N;
  std::vector<Dual> ud(n2);
  for (long i = 0; i < n2; i++) ud[i] = Dual(u[i], v[i]);
  std::vector<Dual> zd = zconst(*H);
  const Dual* E = ud.data();
  const Dual* T = ud.data() + N;
  for (long idx = 0; idx < N; idx++) {
    int l = H->cell_level[idx];
    const int* c = &H->cell_ijk[3 * idx];
    if (H->covered(l, c)) { S[idx] = 0.0; S[N + idx] = 0.0; continue; }
    double aE = 0.0, aT = 0.0;
    for (int d = 0; d < 3; d++)
      for (int s = -1; s <= 1; s += 2) {
        FluxPair<Dual> f = face_flux(*H, E, T, zd.data(), l, c, d, s);
        aE += std::fabs(f.E.d) / H->lev[l].h[d];
        aT += std::fabs(f.T.d) / H->lev[l].h[d];
      }
    double zc = cube(H->z[idx]);
    Dual Tc = T[idx];
    Dual sigma = zc / (Tc * Tc * Tc);
    Dual st4 = sigma * (Tc * Tc * Tc * Tc);
    Dual se = sigma * E[idx];
    double cpl = std::fabs(st4.d) + std::fabs(se.d);
    S[idx] = a0 * std::fabs(v[idx]) + dt * (aE + cpl);
    S[N + idx] = a0 * std::fabs(v[N + idx]) + dt * (aT + cpl);
  }
}

void orc_vjp(orc_hier* h, const double* u, const double* w, double a0, double dt, double* JTw,
             double* dz, double* JTw_abs) {
  vjp_bruteforce(*reinterpret_cast<Hier*>(h), u, w, a0, dt, JTw, dz, JTw_abs);
}

// The Jacobian of F(u) = a0 u - b - dt f(u) with respect to u and z, every
// entry the residual code reaches, as triplets: rows 0 .. 2N-1, columns
// 0 .. 2N-1 for u and 2N + k for z_k.  Returns the number of entries, or
// -(that number) when cap is too small (nothing written then).
long orc_jacobian(orc_hier* h, const double* u, double a0, double dt, long cap, int* rows,
                  int* cols, double* vals) {
  const Hier& H = *reinterpret_cast<Hier*>(h);
  const long N = H.N, n2 = 2 * N;
  std::vector<SDual> ud(n2), zd(N), Fd(n2);
  for (long i = 0; i < n2; i++) {
    ud[i] = SDual(u[i]);
    ud[i].d.push_back({i, 1.0});
  }
  for (long k = 0; k < N; k++) {
    zd[k] = SDual(H.z[k]);
    zd[k].d.push_back({n2 + k, 1.0});
  }
  std::vector<double> b0(n2, 0.0);
  residual_t<SDual>(H, ud.data(), zd.data(), b0.data(), a0, dt, Fd.data(), nullptr);
  long nnz = 0;
  for (long r = 0; r < n2; r++) nnz += (long)Fd[r].d.size();
  if (nnz > cap) return -nnz;
  long q = 0;
  for (long r = 0; r < n2; r++)
    for (const auto& e : Fd[r].d) {
      rows[q] = (int)r;
      cols[q] = (int)e.first;
      vals[q] = e.second;
      q++;
    }
  return nnz;
}

// material in double precision (for finite-difference pins in z)
void orc_set_material_f64(orc_hier* h, const double* z) {
  Hier* H = reinterpret_cast<Hier*>(h);
  for (long i = 0; i < H->N; i++) H->z[i] = z[i];
}

// Sec. 3.5 Remark 2: time derivative at t_{n+1} from the left-hand side of
// Eq. bdf2 (backward Euler when u_nm1 is null).
void orc_time_derivative(orc_hier* h, const double* u_np1, const double* u_n,
                         const double* u_nm1, double dt, double dt_prev, double* udot) {
  Hier* H = reinterpret_cast<Hier*>(h);
  for (long i = 0; i < 2 * H->N; i++) {
    if (u_nm1) {
      double al = dt / dt_prev;
      double lhs = (1.0 + 2.0 * al) / (1.0 + al) * u_np1[i] - (1.0 + al) * u_n[i] +
                   al * al / (1.0 + al) * u_nm1[i];
      udot[i] = lhs / dt;
    } else {
      udot[i] = (u_np1[i] - u_n[i]) / dt;
    }
  }
}

// Eq. leapfrog: generalised leapfrog predictor.
void orc_predict(orc_hier* h, const double* u_n, const double* u_nm1, const double* udot_n,
                 double dt, double dt_prev, double* u_p) {
  Hier* H = reinterpret_cast<Hier*>(h);
  double al = dt / dt_prev;
  for (long i = 0; i < 2 * H->N; i++)
    u_p[i] = u_n[i] + (1.0 + al) * dt * udot_n[i] - al * al * (u_n[i] - u_nm1[i]);
}

// Eq. bdf2le with the scaled max norm of Sec. 3.5 over leaf cells.
double orc_lte(orc_hier* h, const double* u_np1, const double* u_p, double alpha, double eta_E,
               double eta_T) {
  Hier* H = reinterpret_cast<Hier*>(h);
  const long N = H->N;
  double m = 0.0;
  for (long i = 0; i < N; i++) {
    if (H->covered_idx(i)) continue;
    double eE = (alpha + 1.0) / (3.0 * alpha + 2.0) * (u_np1[i] - u_p[i]);
    double eT = (alpha + 1.0) / (3.0 * alpha + 2.0) * (u_np1[N + i] - u_p[N + i]);
    m = std::max(m, std::fabs(eE / (u_np1[i] + eta_E)));
    m = std::max(m, std::fabs(eT / (u_np1[N + i] + eta_T)));
  }
  return m;
}

double orc_fd_eps(orc_hier* h, const double* u, const double* v) {
  return fd_eps(*reinterpret_cast<Hier*>(h), u, v);
}

double orc_jv_fd(orc_hier* h, const double* u, const double* v, const double* b, double a0,
                 double dt, const double* F0, double* Jv) {
  double eps = 0.0;
  jv_fd(*reinterpret_cast<Hier*>(h), u, v, b, a0, dt, F0, Jv, &eps);
  return eps;
}

double orc_dot(orc_hier* h, const double* x, const double* y) {
  return wdot(*reinterpret_cast<Hier*>(h), x, y);
}

// Ghost values in the per-patch face layout: patches in hierarchy order; for
// each patch faces x-, x+, y-, y+, z-, z+; on a face normal to d the cells
// are ordered with t1 = (d+1)%3 fastest, then t2 = (d+2)%3.
long orc_ghosts(orc_hier* h, const double* u, double* gE, double* gT, float* gz) {
  Hier* H = reinterpret_cast<Hier*>(h);
  long gi = 0;
  for (int l = 0; l < H->L; l++) {
    const Level& Lv = H->lev[l];
    for (size_t p = 0; p < Lv.off.size(); p++) {
      const int* bx = &Lv.box[6 * p];
      for (int face = 0; face < 6; face++) {
        int d = face / 2, s = (face % 2) ? 1 : -1;
        int t1 = plane_t1(d), t2 = plane_t2(d);
        for (int b2 = bx[t2]; b2 <= bx[3 + t2]; b2++)
          for (int b1 = bx[t1]; b1 <= bx[3 + t1]; b1++) {
            int c[3];
            c[d] = (s < 0) ? bx[d] : bx[3 + d];
            c[t1] = b1;
            c[t2] = b2;
            double Eg, Tg, zg;
            ghost_of(*H, u, l, c, d, s, &Eg, &Tg, &zg);
            if (gE) gE[gi] = Eg;
            if (gT) gT[gi] = Tg;
            if (gz) gz[gi] = (float)zg;
            gi++;
          }
      }
    }
  }
  return gi;
}

void orc_pc_setup(orc_hier* h, const double* u, double a0, double dt) {
  pc_setup(*reinterpret_cast<Hier*>(h), u, a0, dt);
}

void orc_pc_apply(orc_hier* h, const double* w, double* y) {
  pc_apply(*reinterpret_cast<Hier*>(h), w, y);
}

void orc_comp_apply(orc_hier* h, int fld, const double* x, double* y) {
  comp_apply(*reinterpret_cast<Hier*>(h), fld, x, y);
}

// y = the level-l operator of the FAC V-cycle (R9: homogeneous coarse-fine
// ghosts) applied to x; x and y dense over level l's index space, 0 where
// the level has no cell.  Needs orc_pc_setup.
void orc_level_apply(orc_hier* h, int fld, int l, const double* x, double* y) {
  Hier& H = *reinterpret_cast<Hier*>(h);
  if (!H.pc_ready || l < 0 || l >= H.L) fatal("orc_level_apply: no set-up or bad level");
  Grid G{&H, &H.opl[fld][l], fld};
  std::vector<double> e(x, x + G.ncell()), out;
  level_apply(G, e, out);
  std::copy(out.begin(), out.end(), y);
}

void orc_fac(orc_hier* h, int fld, const double* f, double* u) {
  fac_vcycle(*reinterpret_cast<Hier*>(h), fld, f, u);
}

// One GMG V-cycle on the base box alone (single-level operator), for tests.
void orc_gmg(orc_hier* h, int fld, const double* f, double* e) {
  Hier* H = reinterpret_cast<Hier*>(h);
  const Hier::OpLevel& O = H->mg[fld][0];
  long n = (long)O.n[0] * O.n[1] * O.n[2];
  std::vector<double> ff(f, f + n), ee(n, 0.0);
  gmg_vcycle(*H, fld, 0, ee, ff);
  for (long i = 0; i < n; i++) e[i] = ee[i];
}

void orc_average_down(orc_hier* h, double* x) {
  Hier* H = reinterpret_cast<Hier*>(h);
  average_down(*H, x);
}

int orc_newton(orc_hier* h, double* u, const double* b, double a0, double dt, int* newton_its,
               int* krylov_its, double* fnorm0, double* fnorm) {
  Stats st;
  int rc = newton(*reinterpret_cast<Hier*>(h), u, b, a0, dt, &st);
  if (newton_its) *newton_its = st.newton_its;
  if (krylov_its) *krylov_its = st.krylov_its;
  if (fnorm0) *fnorm0 = st.fnorm0;
  if (fnorm) *fnorm = st.fnorm;
  return rc;
}

// Error indicators of Sec. 5 plus the relative gradient h |grad E| / E, on
// every cell of every level (covered cells use composite values).
// The three refinement indicators of every cell (Sec. 5; R16): ind[3 idx]
// = tau^c / (0.1 max|E|), ind[3 idx + 1] = tau^g / (0.1 max|E|),
// ind[3 idx + 2] = h|grad E| / E, on composite values.
void orc_tag_values(orc_hier* h, const double* u, double* ind) {
  Hier* H = reinterpret_cast<Hier*>(h);
  const long N = H->N;
  double emax = 0.0;
  for (long i = 0; i < N; i++)
    if (!H->covered_idx(i)) emax = std::max(emax, std::fabs(u[i]));
  // the indicators see composite values: covered cells (and the physical
  // ghosts next to them) take the mean of their children
  std::vector<double> uc(u, u + 2 * N);
  average_down(*H, uc.data());
  average_down(*H, uc.data() + N);
  u = uc.data();
  for (long idx = 0; idx < N; idx++) {
    int l = H->cell_level[idx];
    const int* c = &H->cell_ijk[3 * idx];
    double Ec = comp_value(*H, u, l, c);
    double tc = 0.0, tg = 0.0, gr2 = 0.0;
    for (int d = 0; d < 3; d++) {
      double Ev[2];
      for (int si = 0; si < 2; si++) {
        int s = si ? 1 : -1;
        int g[3] = {c[0], c[1], c[2]};
        g[d] += s;
        if (H->inside(l, g) && H->cell(l, g) >= 0) {
          Ev[si] = comp_value(*H, u, l, g);
        } else {
          double Eg, Tg, zg;
          ghost_of(*H, u, l, c, d, s, &Eg, &Tg, &zg);
          Ev[si] = Eg;
        }
      }
      tc += std::fabs(Ev[1] - 2.0 * Ec + Ev[0]);
      tg += 0.5 * std::fabs(Ev[1] - Ev[0]);
      gr2 += 0.25 * (Ev[1] - Ev[0]) * (Ev[1] - Ev[0]);
    }
    ind[3 * idx] = tc / (0.1 * emax);
    ind[3 * idx + 1] = tg / (0.1 * emax);
    ind[3 * idx + 2] = std::sqrt(gr2) / Ec;
  }
}

// Refinement tags of Sec. 5 from the indicators above, thresholds strict:
// bit 0 tau^c > thr_c; bit 1 tau^g > thr_g; bit 2 h|grad E|/E > thr_r.
void orc_tag(orc_hier* h, const double* u, double thr_c, double thr_g, double thr_r,
             unsigned char* tags) {
  Hier* H = reinterpret_cast<Hier*>(h);
  std::vector<double> ind(3 * H->N);
  orc_tag_values(h, u, ind.data());
  for (long idx = 0; idx < H->N; idx++) {
    unsigned char t = 0;
    if (ind[3 * idx] > thr_c) t |= 1;
    if (ind[3 * idx + 1] > thr_g) t |= 2;
    if (ind[3 * idx + 2] > thr_r) t |= 4;
    tags[idx] = t;
  }
}

}  // extern "C"
