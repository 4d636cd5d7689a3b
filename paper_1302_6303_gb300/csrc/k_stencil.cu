// Stencil kernels of the radiation-diffusion residual (Sec. 3.2, 3.2.1, 3.3)
// and its Jacobian-vector products (Sec. 4.1), all FP64:
//   ghost fill     physical / sibling / coarse-fine ghosts from a work-list
//   k_stencil      one persistent launch over the tiles of every level:
//                  halo staged in shared memory, each face flux computed
//                  once and shared by its two cells, then the cell balance
//   k_reflux       flux matching at coarse-fine faces
//   k_tag          Sec. 5 refinement indicators
//   k_avgdown      covered cells := mean of their children
#include <algorithm>
#include <cstdio>

#include "nrd_internal.h"

namespace {

struct LevelH {
  double h[NRD_MAX_LEVELS][3];
  double rh[NRD_MAX_LEVELS][3];   // 1/h
  double h3[NRD_MAX_LEVELS][3];   // 3h
  double kh[NRD_MAX_LEVELS][3];   // k/h
  double kh5[NRD_MAX_LEVELS][3];  // 1.25 k/h
  double bh2[NRD_MAX_LEVELS][3];  // beta/h^2 (linearisation only)
  // the face fluxes' constants in terms of Ts = T_a + T_b (face_core)
  double h12[NRD_MAX_LEVELS][3];  // 12h
  double khs[NRD_MAX_LEVELS][3];  // 2^(-5/2) k/h
  double kh5s[NRD_MAX_LEVELS][3]; // 2^(-3/2) 1.25 k/h
};

// 2^(-5/2) and 2^(-3/2): Tf^(5/2) = 2^(-5/2) Ts^(5/2), Tf^(3/2) = 2^(-3/2) Ts^(3/2)
constexpr double kP52 = 0.17677669529663688;
constexpr double kP32 = 0.35355339059327376;

struct GhostArgs {
  const uint8_t* gtype;
  const uint8_t* gface;   // face | level << 3
  const int* gcell;
  const int* gt0;
  const int* gidx;
  const double* gw;
  const float* z;
  int N, G;
  double R[6];
  LevelH lh;
};

// Fill ghosts of a two-field vector u (E = u[0..N), T = u[N..2N)) into
// g[0..G) (E) and g[G..2G) (T).  nonlinear = 1 evaluates the Robin ghost of
// Sec. 3.1 Eq. robinbc; nonlinear = 0 copies the interior value there (linear
// uses never read physical ghosts).
__global__ void k_ghost_fill(GhostArgs a, const double* __restrict__ u, double* __restrict__ g,
                             int nonlinear) {
  const int N = a.N, G = a.G;
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < G; gi += gridDim.x * blockDim.x) {
    uint8_t t = a.gtype[gi];
    int c = a.gcell[gi];
    double e, tt;
    if (t == GT_NEUMANN) {
      e = u[c];
      tt = u[N + c];
    } else if (t == GT_ROBIN) {
      e = u[c];
      tt = u[N + c];
      if (nonlinear) {
        int f = a.gface[gi] & 7, lvl = a.gface[gi] >> 3;
        double h = a.lh.h[lvl][f / 2];
        double T = tt;
        double zc = (double)a.z[c];
        double Db = T * T * T / (3.0 * (zc * zc * zc));
        double aa = Db / (2.0 * h);
        e = (a.R[f] + e * (aa - 0.125)) / (aa + 0.125);
      }
    } else {
      int t0 = a.gt0[gi], t1 = a.gt0[gi + 1];
      double se = 0.0, st = 0.0;
      for (int q = t0; q < t1; q++) {
        int s = a.gidx[q];
        double w = a.gw[q];
        se += w * u[s];
        st += w * u[N + s];
      }
      e = se;
      tt = st;
    }
    g[gi] = e;
    g[G + gi] = tt;
  }
}

__global__ void k_ghost_z(const int* __restrict__ zsrc, const float* __restrict__ z,
                          float* __restrict__ gz, int G) {
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < G; gi += gridDim.x * blockDim.x)
    gz[gi] = z[zsrc[gi]];
}

struct StArgs {
  const TileDev* tiles;
  const PatchDev* patches;
  const uint8_t* mask;
  const uint8_t* gtype;
  const float* z;     // material z per cell
  const float* gz;    // z of every ghost cell
  const double* z3;   // z^3 of cells then ghosts (FP64), or null
  int ntiles, N, G;
  double k;       // D_T = k T^(5/2)
  double cL;      // limiter constant: 4 (Wilson form) or 2 (printed form)
  double cL2;     // cL / 2 (face_core's Ts form)
  double m15cL;   // -1.5 cL
  double R[6];
  LevelH lh;
  StencilIO io;
};

// Linearisation of one face at the iterate: the fluxes, the frozen
// coefficients D_E = 2 Tf^3 S h / den and D_T = k Tf^(5/2) of Sec. 4.2, and
// the partial derivatives of Phi_E w.r.t. E_a, E_b and T_a (= w.r.t. T_b) and
// of Phi_T w.r.t. T_a, T_b (sign(0) = 0).
struct FaceLin {
  double PE, PT, aEa, aEb, aT, bTa, bTb, aZ;
  double X, T25;   // C_E = X h, C_D = k 2^(-5/2) T25
};

// 1/x from the PTX approximate FP64 reciprocal (rcp.approx.ftz.f64, a
// seed of about 20 good bits) refined with the second-order series of the
// correction: with e = 1 - x r0, 1/x = r0 / (1 - e) = r0 (1 + e + e^2 + ...),
// so r1 = r0 + r0 (e + e^2) leaves a relative error of e^3 (iterative
// refinement of reciprocals, see e.g. Muller et al., Handbook of
// Floating-Point Arithmetic): about 1e-18 before rounding.  For positive
// x in [2^-997, 2^997) (about 7.5e-301 to 1.3e300); elsewhere (zero,
// subnormal, negative, huge, inf, NaN) the correctly rounded 1/x.  The range
// test looks at the high word of x with integer instructions: FP64 compares
// would take FP64-pipe issue slots, the scarce resource of these kernels.
__device__ __forceinline__ bool in_refine_range(double x) {
  // biased exponent in [26, 2020) and sign bit clear
  const unsigned hi = (unsigned)__double2hiint(x);
  return hi - (26u << 20) < ((2020u - 26u) << 20);
}
__device__ __forceinline__ double rcp_approx(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rsqrt_approx(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rcp_nr(double x) {
  if (!in_refine_range(x)) return 1.0 / x;
  const double r = rcp_approx(x);
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// 1/sqrt(x) from the PTX approximate FP64 reciprocal square root
// (rsqrt.approx.ftz.f64) refined with the second-order series: with
// e = 1 - x y0^2, 1/sqrt(x) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3 e^2/8 + ...),
// a relative error of about (5/16) e^3 before rounding.  For x in the range
// of rcp_nr; elsewhere the correctly rounded 1/sqrt(x).
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!in_refine_range(x)) return 1.0 / sqrt(x);
  const double y = rsqrt_approx(x);
  const double e = fma(-x * y, y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}

// FP64 -> FP32 with round-to-nearest-even (the IEEE narrowing conversion,
// bit-identical to the (float) cast) from integer instructions: on GB300 the
// conversion instruction issues on the FP64 pipe, which bounds the
// linearisation.  With the FP64 exponent field e in [897, 1150] the result is a
// normal float: its exponent is e - 896 and its 23 mantissa bits are the top
// 23 of the 52; the 29 dropped bits d round up when d > 2^28, or d = 2^28 and
// the kept lsb is odd, i.e. exactly when d + (2^28 - 1) + lsb >= 2^29.  A
// mantissa carry runs into the exponent (up to infinity when the rounded value
// overflows, as IEEE narrowing gives).  Other exponents (zero, subnormal or
// overflowing results, inf, NaN) take the conversion instruction, in a
// function of its own: inlined, the compiler predicates the conversion instead
// of branching around it, and a predicated-off instruction still takes its
// FP64-pipe issue slot.
__device__ __noinline__ float narrow_slow(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float narrow_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u > 253u) return narrow_slow(x);
  const unsigned top = __funnelshift_l(lo, hi & 0x7fffffffu, 3);   // exponent+mantissa bits
  const unsigned rnd = ((lo & 0x1fffffffu) + 0x0fffffffu + (top & 1u)) >> 29;
  return __uint_as_float((hi & 0x80000000u) | (top - (896u << 23) + rnd));
}

// Face flux in the +e_d direction between cells a (low) and b (high):
//   Phi_E = D_E (E_b - E_a)/h with D_E = D_h/(1 + D_h g) (or the printed form)
//         = 2 Tf^3 S dE / (3 h Zs S + cL Tf^3 |dE|),  S = E_a + E_b,
//           Zs = z_a^3 + z_b^3, dE = E_b - E_a, Tf = (T_a + T_b)/2
//   Phi_T = k Tf^(5/2) (T_b - T_a)/h,
// with the intermediate quantities the partial derivatives reuse.  The
// residual and the linearisation both take their fluxes from here, so the
// two produce bit-identical residuals.
// Evaluated in Ts = T_a + T_b = 2 Tf with the powers of 2 folded into the
// constants (two FP64 multiplies fewer per face): with
//   den' = 4 den = 12h Zs S + (cL/2) Ts^3 |dE|,   X = 2 Tf^3 S / den = Ts^3 S / den',
//   Tf^(5/2) = 2^(-5/2) Ts^(5/2)  (2^(-5/2) in khs = 2^(-5/2) k/h).
// rden = 1/den', hz = 12h Zs, ltadE = (cL/2) Ts^3 |dE| (4 times the Tf-form
// terms), T15 = Ts^(3/2), T25 = Ts^(5/2), khT25 = (k/h) Tf^(5/2).
struct FaceCore {
  double Ts, Ts2, Ts3, dE, adE, S, hz, ltadE, rden, X, PE, T15, T25, dT, khT25, PT;
};
__device__ __forceinline__ FaceCore face_core(double Ea, double Eb, double Ta, double Tb,
                                              double za, double zb, double h12, double khs,
                                              double cL2) {
  FaceCore q;
  q.Ts = Ta + Tb;
  q.Ts2 = q.Ts * q.Ts;
  q.Ts3 = q.Ts2 * q.Ts;
  q.dE = Eb - Ea;
  q.S = Ea + Eb;
  q.hz = h12 * (za + zb);
  q.adE = fabs(q.dE);
  q.ltadE = (cL2 * q.Ts3) * q.adE;
  q.rden = rcp_nr(fma(q.hz, q.S, q.ltadE));
  q.X = (q.Ts3 * q.S) * q.rden;
  q.PE = q.X * q.dE;
  const double y = rsqrt_nr(q.Ts);
  q.T15 = q.Ts2 * y;     // Ts^(3/2)
  q.T25 = q.Ts * q.T15;  // Ts^(5/2)
  q.dT = Tb - Ta;
  q.khT25 = khs * q.T25;
  q.PT = q.khT25 * q.dT;
  return q;
}

// Face flux of face_core and its partial derivatives at one iterate (the
// frozen Jacobian), with X = 2 Tf^3 S / den, den = 3h Zs S + cL Tf^3 |dE|:
//   PE = X dE (the P1 coefficient C_E = D_E h is X h)
//   d PE / d E_a = (-4 Tf^3 E_a - PE (3h Zs - cL Tf^3 sg)) / den
//   d PE / d E_b = ( 4 Tf^3 E_b - PE (3h Zs + cL Tf^3 sg)) / den
//   d PE / d T_a = d PE / d T_b = Tf^2 (3 S dE - 1.5 cL |dE| PE) / den
//   d PE / d Zs  = -PE 3h S / den
//   PT = (k/h) Tf^(5/2) dT, d PT / d T_{a,b} = (k/h)(1.25 Tf^(3/2) dT -/+ Tf^(5/2))
// (sg = sign(dE), sign(0) = 0), each evaluated in face_core's Ts form (the
// factor 4 of den' cancels against the factor 4 of the Ts-form terms:
// 4 Tf^3 = Ts^3 / 2, Tf^2 / den = Ts^2 / den').  The reciprocal and
// Ts^(-1/2) come from rcp_nr / rsqrt_nr (within ~1e-13 relative of correctly
// rounded arithmetic).  T25 is Ts^(5/2): C_D = k 2^(-5/2) T25.
__device__ __forceinline__ FaceLin flux_lin(double Ea, double Eb, double Ta, double Tb, double za,
                                            double zb, double h12, double khs, double kh5s,
                                            double cL2, double m15cL, bool with_dz) {
  const FaceCore q = face_core(Ea, Eb, Ta, Tb, za, zb, h12, khs, cL2);
  FaceLin r;
  r.PE = q.PE;
  r.X = q.X;
  const double A = q.PE * q.hz;
  const double Bs = q.X * q.ltadE;      // = 4 PE cL Tf^3 sign(dE)
  const double t16 = q.Ts3 + q.Ts3;     // 16 Tf^3
  r.aEa = (fma(-t16, Ea, Bs) - A) * q.rden;
  r.aEb = (fma(t16, Eb, -Bs) - A) * q.rden;
  r.aT = (q.Ts2 * q.rden) * fma(m15cL, q.adE * q.PE, 3.0 * (q.S * q.dE));
  r.aZ = with_dz ? -(q.PE * q.rden) * (h12 * q.S) : 0.0;
  r.T25 = q.T25;
  r.PT = q.PT;
  const double khq = kh5s * q.T15 * q.dT;
  r.bTa = khq - q.khT25;
  r.bTb = khq + q.khT25;
  return r;
}

// Balance of one cell (Eq. nonlinearsystem, per unit volume):
//   F_E = a0 E - b_E - dt (div_E + c),  F_T = a0 T - b_T - dt (div_T - c),
//   c = sigma (T^4 - E), sigma = z^3 / T^3,
// shared by the residual and the linearisation (bit-identical F); returns
// 1/T and sigma for the partial derivatives.
__device__ __forceinline__ void cell_balance(double a0, double dt, double E, double T, double z3,
                                             double bE, double bT, double divE, double divT,
                                             double& FE, double& FT, double& rT, double& sig) {
  rT = rcp_nr(T);
  sig = z3 * rT * rT * rT;
  const double T2 = T * T;
  const double cp = sig * (T2 * T2 - E);
  FE = a0 * E - bE - dt * (divE + cp);
  FT = a0 * T - bT - dt * (divT - cp);
}

// Tangent of the face fluxes in the direction (dEa, dEb, dTa, dTb); sign(0) = 0.
__device__ __forceinline__ void flux_tan(double Ea, double Eb, double Ta, double Tb, double za,
                                         double zb, double h3, double kh, double cL, double vEa,
                                         double vEb, double vTa, double vTb, double& dPE,
                                         double& dPT) {
  double Tf = 0.5 * (Ta + Tb);
  double dTf = 0.5 * (vTa + vTb);
  double Tf2 = Tf * Tf;
  double Tf3 = Tf2 * Tf;
  double dTf3 = 3.0 * Tf2 * dTf;
  double dE = Eb - Ea, ddE = vEb - vEa;
  double S = Ea + Eb, dS = vEa + vEb;
  double Zs = za + zb;
  double sg = (dE > 0.0) ? 1.0 : ((dE < 0.0) ? -1.0 : 0.0);
  double num = 2.0 * Tf3 * dE * S;
  double dnum = 2.0 * (dTf3 * dE * S + Tf3 * (ddE * S + dE * dS));
  double den = h3 * Zs * S + cL * Tf3 * fabs(dE);
  double dden = h3 * Zs * dS + cL * (dTf3 * fabs(dE) + Tf3 * sg * ddE);
  double rden = 1.0 / den;
  double PE = num * rden;
  dPE = (dnum - PE * dden) * rden;
  double sq = sqrt(Tf);
  dPT = kh * ((2.5 * Tf * sq * dTf) * (Tb - Ta) + Tf2 * sq * (vTb - vTa));
}

// Robin face (Sec. 3.1 Eq. robinbc, unlimited D_b = T^3/(3 z^3)): the +e_d
// flux through the boundary face on side s of the cell is
//   Phi = -s D_b (2 E - 8 R) / (4 D_b + h).
__device__ __forceinline__ double robin_flux(double E, double T, double z, double h, double R,
                                             int s) {
  double Db = T * T * T / (3.0 * z);
  return -(double)s * Db * (2.0 * E - 8.0 * R) / (4.0 * Db + h);
}

__device__ __forceinline__ double robin_tan(double E, double T, double z, double h, double R,
                                            int s, double vE, double vT) {
  double Db = T * T * T / (3.0 * z);
  double dDb = T * T * vT / z;
  double m = 2.0 * E - 8.0 * R, dm = 2.0 * vE;
  double q = 4.0 * Db + h;
  return -(double)s * (dDb * m * h + Db * dm * q) / (q * q);
}

// scaled P1 coefficient a = beta C / h^2 (or the Robin diagonal term) in the
// V-cycle precision
__device__ __forceinline__ void put_scaled(const StencilIO& io, long NS, long slot, double aE,
                                           double aT) {
  if (io.a32) {
    io.a32[slot] = (float)aE;
    io.a32[NS + slot] = (float)aT;
  } else {
    io.a64[slot] = aE;
    io.a64[NS + slot] = aT;
  }
}

// The linearisation's cell outputs (shared by the fused and the split form):
// F from cell_balance, the coupling partials and the P2 data.
template <bool DZ>
__device__ __forceinline__ void lin_cell(const StencilIO& io, int N, int idx, double a0v,
                                         double dtv, double betav, float betaf, double E,
                                         double T, double z, double divE, double divT) {
  const double T2 = T * T, T3 = T2 * T;
  double FE, FT, rT, sig;
  cell_balance(a0v, dtv, E, T, z, io.b[idx], io.b[N + idx], divE, divT, FE, FT, rT, sig);
  io.out[idx] = FE;
  io.out[N + idx] = FT;
  // coupling tangent dc = cE vE + cT vT
  io.cc[idx] = -sig;
  io.cc[N + idx] = sig * fma(3.0 * E, rT, T3);
  if (DZ) io.cc[2L * N + idx] = (T2 * T2 - E) * rT * rT * rT;   // d coupling / d z^3
  // P2 of Sec. 4.2 at this iterate: [[1 + sb, -sbt], [-sb, 1 + sbt]]
  // (det = (1 + sb)(1 + sbt) - sbt sb = 1 + sb + sbt), in the
  // preconditioner's precision
  if (io.p2f) {
    const float sb = narrow_rn(sig) * betaf, sbt = sb * narrow_rn(T3);
    io.p2f[idx] = sb;
    io.p2f[N + idx] = sbt;
    io.p2f[2L * N + idx] = 1.0f / (1.0f + sb + sbt);
  } else {
    const double sb = sig * betav, sbt = sb * T3;
    io.p2[idx] = sb;
    io.p2[N + idx] = sbt;
    io.p2[2L * N + idx] = rcp_nr(1.0 + sb + sbt);
  }
}

// covered cell: not an unknown
template <bool DZ>
__device__ __forceinline__ void lin_cell_covered(const StencilIO& io, int N, int idx) {
  io.out[idx] = 0.0;
  io.out[N + idx] = 0.0;
  io.cc[idx] = 0.0;
  io.cc[N + idx] = 0.0;
  if (DZ) io.cc[2L * N + idx] = 0.0;
  if (io.p2f) {
    io.p2f[idx] = 0.0f;
    io.p2f[N + idx] = 0.0f;
    io.p2f[2L * N + idx] = 0.0f;
  } else {
    io.p2[idx] = 0.0;
    io.p2[N + idx] = 0.0;
    io.p2[2L * N + idx] = 0.0;
  }
}

// CMP: the cell loops (and the fused forms' face loop) run over the cells of
// a tile inside its patch only, with index arithmetic in the tile's runtime
// extent; used where the hierarchy has tiles narrower than the tile shape
// (patches whose sides are not multiples of it), so that no lane of a warp
// idles on a cell outside its patch.  Without CMP the extents are the
// compile-time shape (fewer registers: the form for hierarchies without
// such tiles).
template <int MODE, int TX, int TY, int TZ, bool CMP = false>
__global__ void __launch_bounds__(256) k_stencil(StArgs A) {
  constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
  constexpr int NH = HX * HY * HZ;
  constexpr int NFX = (TX + 1) * TY * TZ, NFY = TX * (TY + 1) * TZ, NFZ = TX * TY * (TZ + 1);
  constexpr int NC = TX * TY * TZ;
  constexpr bool TAN = (MODE == ST_JV);
  constexpr bool LINF = (MODE == ST_LINF);     // the split linearisation's face launch
  constexpr bool LINC = (MODE == ST_LINC);     // and its cell launch
  constexpr bool FACES = LINF || MODE == ST_RESF;   // split forms: faces only
  constexpr bool CELLS = LINC || MODE == ST_RESC;   // split forms: cells only
  constexpr bool LIN = (MODE == ST_LIN || MODE == ST_LINZ || LINF);   // writes the face data
  constexpr bool DZ = (MODE == ST_LINZ);       // also the d/dz^3 partials
  constexpr bool JVF = (MODE == ST_JVF);       // frozen-Jacobian Jv: sE, sT hold v
  extern __shared__ double smem[];
  double* sE = smem;
  double* sT = sE + NH;
  double* svE = sT + NH;                       // tangent direction (JV only)
  double* svT = svE + (TAN ? NH : 0);
  double* fxE = svT + (TAN ? NH : 0);
  double* fxT = fxE + NFX;
  double* fyE = fxT + NFX;
  double* fyT = fyE + NFY;
  double* fzE = fyT + NFY;
  double* fzT = fzE + NFZ;
  double* sZ = fzT + NFZ;                     // z^3 of the halo cells

  const int N = A.N, G = A.G;
  const long NS = 3L * N + G;                  // face slots per coefficient array
  const StencilIO& io = A.io;
  // a0, dt, beta: kernel arguments, or device values (graph-captured solves)
  double a0v = io.a0, dtv = io.dt, betav = io.beta;
  if (io.par) {
    a0v = io.par[0];
    dtv = io.par[1];
    betav = io.par[2];
  }
  double eps = 0.0, reps = 0.0;
  if (MODE == ST_FD) {
    eps = *io.eps;
    reps = 1.0 / eps;
  }
  // FP32 scale factors of the V-cycle coefficients per level and axis:
  // beta C_E / h^2 = X (beta / h), beta C_T / h^2 = Ts^(5/2) (2^(-5/2) beta k / h^2)
  __shared__ float s_bh[LIN ? NRD_MAX_LEVELS * 3 : 1], s_bk[LIN ? NRD_MAX_LEVELS * 3 : 1];
  if (LIN && threadIdx.x < NRD_MAX_LEVELS * 3) {
    const double rh = A.lh.rh[threadIdx.x / 3][threadIdx.x % 3];
    s_bh[threadIdx.x] = (float)(betav * rh);
    s_bk[threadIdx.x] = (float)(kP52 * (betav * A.k * rh * rh));
  }
  const float betaf = (float)betav;

  for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
    const TileDev tile = A.tiles[t];
    const PatchDev P = A.patches[tile.patch];
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int lvl = P.level;
    if (tile.flags & 1) {
      // every cell covered: not unknowns
      for (int c = threadIdx.x; c < NC; c += blockDim.x) {
        int ci = c % TX, cj = (c / TX) % TY, ck = c / (TX * TY);
        int i = tile.i0 + ci, j = tile.j0 + cj, k = tile.k0 + ck;
        if (i >= nx || j >= ny || k >= tile.k1) continue;
        int idx = P.off + i + nx * (j + ny * k);
        io.out[idx] = 0.0;
        io.out[N + idx] = 0.0;
      }
      continue;
    }
    if (CELLS) {
      // the split forms' cell launch: the face fluxes come from pef (written
      // by the face launch, each face once), the divergence is formed in the
      // fused kernel's order, so F is bit-identical to it
      const double rhx = A.lh.rh[lvl][0], rhy = A.lh.rh[lvl][1], rhz = A.lh.rh[lvl][2];
      const double* pE = io.pef;
      const double* pT = io.pef + NS;
      const int cex = CMP ? min(TX, nx - tile.i0) : TX, cey = CMP ? min(TY, ny - tile.j0) : TY;
      const int nce = CMP ? cex * cey * (tile.k1 - tile.k0) : NC;
      for (int c = threadIdx.x; c < nce; c += blockDim.x) {
        const int ci = c % cex, cj = (c / cex) % cey, ck = c / (cex * cey);
        const int i = tile.i0 + ci, j = tile.j0 + cj, k = tile.k0 + ck;
        if (i >= nx || j >= ny || k >= tile.k1) continue;
        const int idx = P.off + i + nx * (j + ny * k);
        const uint8_t m = A.mask[idx];
        if (m & MASK_COVERED) {
          if (LINC) {
            lin_cell_covered<false>(io, N, idx);
          } else {
            io.out[idx] = 0.0;
            io.out[N + idx] = 0.0;
          }
          continue;
        }
        // face slots: an interior face at dir N + the index of the cell on its
        // high side (the face is that cell's low face: cell idx has its low x
        // face at idx and its high x face at idx + 1); patch faces at 3N +
        // their ghost index
        auto gslot = [&](int ff, int a, int b) {
          return 3L * N + P.goff + P.fo[ff] + a + P.n[((ff >> 1) + 1) % 3] * b;
        };
        const long xl = (i == 0) ? gslot(0, j, k) : (long)idx;
        const long xh = (i == nx - 1) ? gslot(1, j, k) : (long)idx + 1;
        const long yl = (j == 0) ? gslot(2, k, i) : (long)N + idx;
        const long yh = (j == ny - 1) ? gslot(3, k, i) : (long)N + idx + nx;
        const long zl = (k == 0) ? gslot(4, i, j) : 2L * N + idx;
        const long zh = (k == nz - 1) ? gslot(5, i, j) : 2L * N + idx + (long)nx * ny;
        auto pick = [](bool skip, double v) { return skip ? 0.0 : v; };
        const double divE = (pick(m & 4, pE[xh]) - pick(m & 2, pE[xl])) * rhx +
                            (pick(m & 16, pE[yh]) - pick(m & 8, pE[yl])) * rhy +
                            (pick(m & 64, pE[zh]) - pick(m & 32, pE[zl])) * rhz;
        const double divT = (pick(m & 4, pT[xh]) - pick(m & 2, pT[xl])) * rhx +
                            (pick(m & 16, pT[yh]) - pick(m & 8, pT[yl])) * rhy +
                            (pick(m & 64, pT[zh]) - pick(m & 32, pT[zl])) * rhz;
        const double E = io.u[idx], T = io.u[N + idx];
        const double z = A.z3 ? A.z3[idx] : (double)A.z[idx];
        const double z3c = A.z3 ? z : z * z * z;
        if (LINC) {
          lin_cell<false>(io, N, idx, a0v, dtv, betav, betaf, E, T, z3c, divE, divT);
        } else {
          double FE, FT, rT, sig;
          cell_balance(a0v, dtv, E, T, z3c, io.b[idx], io.b[N + idx], divE, divT, FE, FT, rT,
                       sig);
          io.out[idx] = FE;
          io.out[N + idx] = FT;
        }
      }
      continue;
    }
    // ---- halo load (face halos only; edges and corners are never read)
    for (int hh = threadIdx.x; hh < NH; hh += blockDim.x) {
      int hx_ = hh % HX, hy_ = (hh / HX) % HY, hz_ = hh / (HX * HY);
      int i = tile.i0 + hx_ - 1, j = tile.j0 + hy_ - 1, k = tile.k0 + hz_ - 1;
      int ox = (i < 0) ? -1 : ((i >= nx) ? 1 : 0);
      int oy = (j < 0) ? -1 : ((j >= ny) ? 1 : 0);
      int oz = (k < 0) ? -1 : ((k >= nz) ? 1 : 0);
      if ((ox != 0) + (oy != 0) + (oz != 0) > 1) continue;
      if (i > nx || j > ny || k > tile.k1) continue;
      double e, tt, ve = 0.0, vt = 0.0;
      double z = 0.0;
      if (JVF) {
        if (!ox && !oy && !oz) {
          int idx = P.off + i + nx * (j + ny * k);
          e = io.v[idx];
          tt = io.v[N + idx];
        } else {
          int f = ox ? (ox < 0 ? 0 : 1) : (oy ? (oy < 0 ? 2 : 3) : (oz < 0 ? 4 : 5));
          int a = ox ? j : (oy ? k : i), b = ox ? k : (oy ? i : j);
          int gi = P.goff + P.fo[f] + a + P.n[(f / 2 + 1) % 3] * b;
          e = io.gv[gi];
          tt = io.gv[G + gi];
        }
        sE[hh] = e;
        sT[hh] = tt;
        continue;
      }
      if (!ox && !oy && !oz) {
        int idx = P.off + i + nx * (j + ny * k);
        e = io.u[idx];
        tt = io.u[N + idx];
        z = A.z3 ? A.z3[idx] : (double)A.z[idx];
        if (MODE == ST_JV || MODE == ST_FD) {
          ve = io.v[idx];
          vt = io.v[N + idx];
        }
      } else {
        int f, a, b;
        if (ox) { f = ox < 0 ? 0 : 1; a = j; b = k; }
        else if (oy) { f = oy < 0 ? 2 : 3; a = k; b = i; }
        else { f = oz < 0 ? 4 : 5; a = i; b = j; }
        int d = f / 2;
        int nt1 = P.n[(d + 1) % 3];
        int gi = P.goff + P.fo[f] + a + nt1 * b;
        e = io.gu[gi];
        tt = io.gu[G + gi];
        z = A.z3 ? A.z3[(long)N + gi] : (double)A.gz[gi];
        if (MODE == ST_JV || MODE == ST_FD) {
          ve = io.gv[gi];
          vt = io.gv[G + gi];
        }
      }
      if (MODE == ST_FD) {
        e += eps * ve;
        tt += eps * vt;
      }
      sE[hh] = e;
      sT[hh] = tt;
      sZ[hh] = A.z3 ? z : z * z * z;
      if (TAN) {
        svE[hh] = ve;
        svT[hh] = vt;
      }
    }
    __syncthreads();
    // ---- face fluxes, each computed once per tile (split forms: once in the launch:
    // the low faces of the tile's cells, and the patch's high boundary faces
    // where the tile ends the patch, enumerated without gaps so that whole
    // warps skip what is not there)
    const int tzl = tile.k1 - tile.k0;
    // the tile's extent inside its patch (a tile at a patch's high end may be
    // narrower than TX x TY): only its cells' faces are enumerated, so that
    // no lane of a warp idles on a face outside the patch (an idle lane
    // still costs its warp's FP64 issue slots)
    const int ex = min(TX, nx - tile.i0), ey = min(TY, ny - tile.j0);
    const bool full = (ex == TX && ey == TY);
    const int nlow = FACES ? ex * ey * tzl : 0;
    const int nbx = (FACES && tile.i0 + ex == nx) ? ey * tzl : 0;
    const int nby = (FACES && tile.j0 + ey == ny) ? ex * tzl : 0;
    const int nbz = (FACES && tile.k1 == nz) ? ex * ey : 0;
    const int nfxe = (ex + 1) * ey * tzl, nfye = ex * (ey + 1) * tzl;
    const int nfaces = FACES ? 3 * nlow + nbx + nby + nbz
                             : (CMP ? nfxe + nfye + ex * ey * (tzl + 1) : NFX + NFY + NFZ);
    for (int f = threadIdx.x; f < nfaces; f += blockDim.x) {
      int dir, fi, fj, fk, slot = 0;
      double* outE = nullptr;
      double* outT = nullptr;
      if (FACES) {
        int q = f;
        if (q < 3 * nlow) {
          dir = q / nlow;
          q -= dir * nlow;
          if (full) {
            fi = q % TX; fj = (q / TX) % TY; fk = q / (TX * TY);
          } else {
            fi = q % ex; fj = (q / ex) % ey; fk = q / (ex * ey);
          }
        } else if ((q -= 3 * nlow) < nbx) {
          dir = 0; fi = ex; fj = q % ey; fk = q / ey;
        } else if ((q -= nbx) < nby) {
          dir = 1; fj = ey; fi = q % ex; fk = q / ex;
        } else {
          q -= nby;
          dir = 2; fk = tzl; fi = q % ex; fj = q / ex;
        }
      } else if (CMP) {
        // the faces of the tile's cells inside the patch, each written to its
        // full-tile slot (the cell loop reads them there)
        int q = f;
        if (q < nfxe) {
          dir = 0; fi = q % (ex + 1); fj = (q / (ex + 1)) % ey; fk = q / ((ex + 1) * ey);
          slot = fi + (TX + 1) * (fj + TY * fk);
          outE = fxE; outT = fxT;
        } else if ((q -= nfxe) < nfye) {
          dir = 1; fi = q % ex; fj = (q / ex) % (ey + 1); fk = q / (ex * (ey + 1));
          slot = fi + TX * (fj + (TY + 1) * fk);
          outE = fyE; outT = fyT;
        } else {
          q -= nfye;
          dir = 2; fi = q % ex; fj = (q / ex) % ey; fk = q / (ex * ey);
          slot = fi + TX * (fj + TY * fk);
          outE = fzE; outT = fzT;
        }
      } else if (f < NFX) {
        dir = 0; slot = f;
        fi = f % (TX + 1); fj = (f / (TX + 1)) % TY; fk = f / ((TX + 1) * TY);
        outE = fxE; outT = fxT;
      } else if (f < NFX + NFY) {
        dir = 1; slot = f - NFX;
        fi = slot % TX; fj = (slot / TX) % (TY + 1); fk = slot / (TX * (TY + 1));
        outE = fyE; outT = fyT;
      } else {
        dir = 2; slot = f - NFX - NFY;
        fi = slot % TX; fj = (slot / TX) % TY; fk = slot / (TX * TY);
        outE = fzE; outT = fzT;
      }
      // face on the low side of tile cell (fi, fj, fk) along dir
      int i = tile.i0 + fi, j = tile.j0 + fj, k = tile.k0 + fk;
      if (i > nx || j > ny || k > tile.k1) continue;
      if ((dir != 0 && i >= nx) || (dir != 1 && j >= ny) || (dir != 2 && k >= tile.k1)) continue;
      int pos = (dir == 0) ? i : ((dir == 1) ? j : k);
      int nd = P.n[dir];
      int hb = (fi + 1) + HX * ((fj + 1) + HY * (fk + 1));   // high-side cell
      int st = (dir == 0) ? 1 : ((dir == 1) ? HX : HX * HY);
      int ha = hb - st;                                      // low-side cell
      const double h = A.lh.h[lvl][dir], h3 = A.lh.h3[lvl][dir], kh = A.lh.kh[lvl][dir];
      double PE = 0.0, PT = 0.0;
      uint8_t gt = GT_SIBLING;
      int gi = -1;
      long fslot;                                            // coefficient slot
      if (pos == 0 || pos == nd) {
        int ff = 2 * dir + (pos == nd ? 1 : 0);
        int a, b;
        if (dir == 0) { a = j; b = k; }
        else if (dir == 1) { a = k; b = i; }
        else { a = i; b = j; }
        gi = P.goff + P.fo[ff] + a + P.n[(dir + 1) % 3] * b;
        gt = A.gtype[gi];
        fslot = 3L * N + gi;
      } else {
        fslot = (long)dir * N + P.off + i + (long)nx * (j + (long)ny * k);
      }
      if (JVF) {
        // tangent flux = stored partials times the direction (sE, sT hold v)
        if (gt == GT_ROBIN) {
          const int hc = (pos == 0) ? hb : ha;
          PE = io.jc[fslot] * sE[hc] + io.jc[NS + fslot] * sT[hc];
        } else if (gt != GT_NEUMANN) {
          PE = io.jc[fslot] * sE[ha] + io.jc[NS + fslot] * sE[hb] +
               io.jc[2 * NS + fslot] * (sT[ha] + sT[hb]);
          PT = io.jc[3 * NS + fslot] * sT[ha] + io.jc[4 * NS + fslot] * sT[hb];
          if (gt == GT_CF) {
            io.cfflux[gi] = PE;
            io.cfflux[G + gi] = PT;
          }
        }
      } else if (gt == GT_NEUMANN) {
        PE = 0.0;
        PT = 0.0;
        if (LIN) {
          for (int q = 0; q < 6; q++) io.jc[q * NS + fslot] = 0.0;
          put_scaled(io, NS, fslot, 0.0, 0.0);
        }
      } else if (gt == GT_ROBIN) {
        int s = (pos == 0) ? -1 : 1;
        int hc = (pos == 0) ? hb : ha;      // the interior cell
        int ff = 2 * dir + (pos == nd ? 1 : 0);
        if (TAN) {
          PE = robin_tan(sE[hc], sT[hc], sZ[hc], h, A.R[ff], s, svE[hc], svT[hc]);
        } else {
          PE = robin_flux(sE[hc], sT[hc], sZ[hc], h, A.R[ff], s);
        }
        if (LIN) {
          // dPhi/dE_c and dPhi/dT_c in slots 0 and 1; raw P1 slot holds D_b
          double Ec = sE[hc], Tc = sT[hc], zc = sZ[hc];
          double Db = Tc * Tc * Tc / (3.0 * zc);
          double qd = 4.0 * Db + h;
          double rq = 1.0 / qd;
          double m = 2.0 * Ec - 8.0 * A.R[ff];
          io.jc[fslot] = -(double)s * 2.0 * Db * rq;
          io.jc[NS + fslot] = -(double)s * (Tc * Tc / zc) * m * h * rq * rq;
          io.jc[2 * NS + fslot] = 0.0;
          io.jc[3 * NS + fslot] = 0.0;
          io.jc[4 * NS + fslot] = 0.0;
          if (DZ) io.jc[5 * NS + fslot] = (double)s * m * h * rq * rq * Db / zc;  // d Phi / d z_c^3
          io.craw[fslot] = Db;
          io.craw[NS + fslot] = 0.0;
          put_scaled(io, NS, fslot, betav * 2.0 * Db * rq / h, 0.0);
        }
        PT = 0.0;
      } else {
        if (TAN) {
          flux_tan(sE[ha], sE[hb], sT[ha], sT[hb], sZ[ha], sZ[hb], h3, kh, A.cL, svE[ha], svE[hb],
                   svT[ha], svT[hb], PE, PT);
        } else if (LIN) {
          FaceLin L = flux_lin(sE[ha], sE[hb], sT[ha], sT[hb], sZ[ha], sZ[hb],
                               A.lh.h12[lvl][dir], A.lh.khs[lvl][dir], A.lh.kh5s[lvl][dir], A.cL2,
                               A.m15cL, DZ);
          PE = L.PE;
          PT = L.PT;
          io.jc[fslot] = L.aEa;
          io.jc[NS + fslot] = L.aEb;
          io.jc[2 * NS + fslot] = L.aT;
          io.jc[3 * NS + fslot] = L.bTa;
          io.jc[4 * NS + fslot] = L.bTb;
          if (DZ) io.jc[5 * NS + fslot] = L.aZ;
          // only the scaled P1 coefficients: the coarsening averages them
          // (raw values are kept for Robin faces alone)
          if (io.a32) {
            io.a32[fslot] = narrow_rn(L.X) * s_bh[3 * lvl + dir];
            io.a32[NS + fslot] = narrow_rn(L.T25) * s_bk[3 * lvl + dir];
          } else {
            // beta D_E / h^2 = X beta / h, beta D_T / h^2 = Ts^(5/2) 2^(-5/2) beta k / h^2
            const double bh = betav * A.lh.rh[lvl][dir];
            io.a64[fslot] = L.X * bh;
            io.a64[NS + fslot] = L.T25 * (kP52 * (bh * A.k * A.lh.rh[lvl][dir]));
          }
        } else {
          const FaceCore q = face_core(sE[ha], sE[hb], sT[ha], sT[hb], sZ[ha], sZ[hb],
                                       A.lh.h12[lvl][dir], A.lh.khs[lvl][dir], A.cL2);
          PE = q.PE;
          PT = q.PT;
        }
        if (gt == GT_CF) {
          io.cfflux[gi] = PE;
          io.cfflux[G + gi] = PT;
        }
      }
      if (FACES) {
        io.pef[fslot] = PE;
        io.pef[NS + fslot] = PT;
      } else {
        outE[slot] = PE;
        outT[slot] = PT;
      }
    }
    __syncthreads();
    if (FACES) continue;   // the cell launch forms the balance
    // ---- cell balance
    const double rhx = A.lh.rh[lvl][0], rhy = A.lh.rh[lvl][1], rhz = A.lh.rh[lvl][2];
    const int fex = CMP ? ex : TX, fey = CMP ? ey : TY;
    const int nce = CMP ? ex * ey * tzl : NC;
    for (int c = threadIdx.x; c < nce; c += blockDim.x) {
      int ci = c % fex, cj = (c / fex) % fey, ck = c / (fex * fey);
      int i = tile.i0 + ci, j = tile.j0 + cj, k = tile.k0 + ck;
      if (i >= nx || j >= ny || k >= tile.k1) continue;
      int idx = P.off + i + nx * (j + ny * k);
      uint8_t m = A.mask[idx];
      if (m & MASK_COVERED) {
        if (LIN) {
          lin_cell_covered<DZ>(io, N, idx);
        } else {
          io.out[idx] = 0.0;
          io.out[N + idx] = 0.0;
        }
        continue;
      }
      int xl = ci + (TX + 1) * (cj + TY * ck);
      int yl = ci + TX * (cj + (TY + 1) * ck);
      int zl = ci + TX * (cj + TY * ck);
      // coarse-side coarse-fine faces take their flux from flux matching
      auto pick = [](bool skip, double v) { return skip ? 0.0 : v; };
      double divE = (pick(m & 4, fxE[xl + 1]) - pick(m & 2, fxE[xl])) * rhx +
                    (pick(m & 16, fyE[yl + TX]) - pick(m & 8, fyE[yl])) * rhy +
                    (pick(m & 64, fzE[zl + TX * TY]) - pick(m & 32, fzE[zl])) * rhz;
      double divT = (pick(m & 4, fxT[xl + 1]) - pick(m & 2, fxT[xl])) * rhx +
                    (pick(m & 16, fyT[yl + TX]) - pick(m & 8, fyT[yl])) * rhy +
                    (pick(m & 64, fzT[zl + TX * TY]) - pick(m & 32, fzT[zl])) * rhz;
      int hc = (ci + 1) + HX * ((cj + 1) + HY * (ck + 1));
      double E = sE[hc], T = sT[hc], z = sZ[hc];
      double T2 = T * T, T3 = T2 * T;
      if (JVF) {
        const double dc = io.cc[idx] * E + io.cc[N + idx] * T;
        io.out[idx] = a0v * E - dtv * (divE + dc);
        io.out[N + idx] = a0v * T - dtv * (divT - dc);
      } else if (MODE == ST_JV) {
        double rT = 1.0 / T;
        double sig = z * rT * rT * rT;
        double vE = svE[hc], vT = svT[hc];
        double dc = sig * ((T3 + 3.0 * E * rT) * vT - vE);
        io.out[idx] = a0v * vE - dtv * (divE + dc);
        io.out[N + idx] = a0v * vT - dtv * (divT - dc);
      } else if (LIN) {
        lin_cell<DZ>(io, N, idx, a0v, dtv, betav, betaf, E, T, z, divE, divT);
      } else {
        double FE, FT, rT, sig;
        cell_balance(a0v, dtv, E, T, z, io.b[idx], io.b[N + idx], divE, divT, FE, FT, rT, sig);
        if (MODE == ST_FD) {
          FE = (FE - io.F0[idx]) * reps;
          FT = (FT - io.F0[N + idx]) * reps;
        }
        io.out[idx] = FE;
        io.out[N + idx] = FT;
      }
    }
    __syncthreads();
  }
}

struct RfArgs {
  const int* cell;
  const int* off;
  const int* face;
  const int4* g;
  const PatchDev* patches;
  int nrf, N, G;
  LevelH lh;
};

// Flux matching (Sec. 3.2.1): the coarse face flux is the average of the four
// fine fluxes stored by the fine-side stencil; scale = -dt (RESIDUAL, JV) or
// -dt/eps (FD).
__global__ void k_reflux(RfArgs a, const int* __restrict__ rf_level, const double* cf,
                         double* out, double dt, const double* par, const double* eps,
                         int mode) {
  if (par) dt = par[1];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.nrf; r += gridDim.x * blockDim.x) {
    int c = a.cell[r];
    int lvl = rf_level[r];
    double sc = -dt;
    if (mode == ST_FD) sc /= *eps;
    double dE = 0.0, dT = 0.0;
    for (int q = a.off[r]; q < a.off[r + 1]; q++) {
      int f = a.face[q];
      int d = f / 2;
      double s = (f % 2) ? 1.0 : -1.0;
      int4 g = a.g[q];
      double PE = 0.25 * (cf[g.x] + cf[g.y] + cf[g.z] + cf[g.w]);
      double PT = 0.25 * (cf[a.G + g.x] + cf[a.G + g.y] + cf[a.G + g.z] + cf[a.G + g.w]);
      const double rh = a.lh.rh[lvl][d];   // 1/h: no FP64 division per face
      dE += s * PE * rh;
      dT += s * PT * rh;
    }
    out[c] += sc * dE;
    out[a.N + c] += sc * dT;
  }
}

// Sec. 5 indicators on every cell.  E holds composite values (covered cells
// already averaged from their children); gE its ghosts.
// The indicator decisions sqrt(s) / b > t (and a / b > t) exactly as the
// correctly rounded formula takes them, with the rounded square root and
// division evaluated only near the threshold: the rounded quotient is within
// 3e-16 relative of the exact one, and t b, (t b)^2 within 7e-16, so away
// from a band of 1e-12 around the threshold the squared comparison decides
// the same.  FP64 square roots and divisions are long instruction sequences
// on GB300's FP64 pipe.
// For non-negative doubles (not NaN) the order of the values is the order of
// their bit patterns as signed 64-bit integers, so the comparisons below take
// integer instructions instead of FP64 compares (which issue on GB300's narrow
// FP64 pipe).  A band of 2^14 units in the last place around the threshold is
// at least 1.8e-12 relative (an ulp step is between 2^-53 and 2^-52
// relative), wider than the 1e-12 the exact-decision argument needs.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
constexpr long long kBits1em290 = 0x03b8f2b061aea072LL;   // 1e-290
constexpr long long kBits1e290 = 0x7c2485ce9e7a065fLL;    // 1e290
constexpr long long kBits1e300 = 0x7e37e43c8800759cLL;    // 1e300
constexpr long long kBand = 1LL << 14;
__device__ __forceinline__ bool fast_range(double x) {
  const long long xb = dbits(x);
  return xb > kBits1em290 && xb < kBits1e290;
}
__device__ __forceinline__ bool sqrt_ratio_gt(double s, double b, double t) {
  const double tb = t * b, tb2 = tb * tb;
  const long long sb = dbits(s), t2b = dbits(tb2);
  if (dbits(b) > 0 && t >= 0.0 && sb >= 0 && fast_range(tb2) && sb < kBits1e300) {
    if (sb > t2b + kBand) return true;
    if (sb < t2b - kBand) return false;
  }
  return sqrt(s) / b > t;
}
__device__ __forceinline__ bool ratio_gt(double a, double b, double t) {
  const double tb = t * b;
  const long long ab = dbits(a), tbb = dbits(tb);
  if (b > 0.0 && t >= 0.0 && ab >= 0 && fast_range(tb) && ab < kBits1e300) {
    if (ab > tbb + kBand) return true;
    if (ab < tbb - kBand) return false;
  }
  return a / b > t;
}

// x 2^k (k = 1, -1, -2) exactly, by adding k to the exponent field when x is
// normal and stays normal (the product of a power of 2 is then exact, so the
// result is bit-identical to the multiplication), x itself for +-0; other
// values (subnormal, near overflow, inf, NaN) take the multiplication.
__device__ __noinline__ double scale2_slow(double x, double f) { return __dmul_rn(f, x); }
template <int K>
__device__ __forceinline__ double scale2(double x) {
  const long long xb = dbits(x);
  const long long e = (xb >> 52) & 0x7ff;
  if (e >= 3 && e <= 2044) return __longlong_as_double(xb + ((long long)K << 52));
  if ((xb & 0x7fffffffffffffffLL) == 0) return x;
  return scale2_slow(x, K == 1 ? 2.0 : (K == -1 ? 0.5 : 0.25));
}

__global__ void k_tag(const TileDev* tiles, const PatchDev* patches, int ntiles, int tx, int ty, int tz,
                      const double* E, const double* gE, double thr_c, double thr_g,
                      double thr_r, const double* emax_p, uint8_t* tags) {
  const double emax = *emax_p;
  const double sc = 0.1 * emax;
  // an infinite threshold never tags: skip that indicator (uniform branch;
  // the enabled ones keep the plain formulas, so decisions are unchanged)
  const bool want_c = thr_c < INFINITY, want_g = thr_g < INFINITY, want_r = thr_r < INFINITY;
  const int nc = tx * ty * tz;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const TileDev tile = tiles[t];
    const PatchDev P = patches[tile.patch];
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int i = tile.i0 + c % tx, j = tile.j0 + (c / tx) % ty, k = tile.k0 + c / (tx * ty);
      if (i >= nx || j >= ny || k >= tile.k1) continue;
      int idx = P.off + i + nx * (j + ny * k);
      double Ec = E[idx];
      double tc = 0.0, tg = 0.0, gr2 = 0.0;
      int pos[3] = {i, j, k};
      for (int d = 0; d < 3; d++) {
        double Ev[2];
        for (int si = 0; si < 2; si++) {
          int q[3] = {i, j, k};
          q[d] += si ? 1 : -1;
          if (q[d] >= 0 && q[d] < P.n[d]) {
            Ev[si] = E[P.off + q[0] + nx * (q[1] + ny * q[2])];
          } else {
            int f = 2 * d + si;
            int a = pos[(d + 1) % 3], b = pos[(d + 2) % 3];
            Ev[si] = gE[P.goff + P.fo[f] + a + P.n[(d + 1) % 3] * b];
          }
        }
        // no contraction: the same roundings as a plain evaluation (the
        // power-of-2 scalings are exact either way)
        if (want_c) tc += fabs(__dadd_rn(__dsub_rn(Ev[1], scale2<1>(Ec)), Ev[0]));
        const double df = __dsub_rn(Ev[1], Ev[0]);
        if (want_g) tg += scale2<-1>(fabs(df));
        if (want_r) gr2 = __dadd_rn(gr2, __dmul_rn(scale2<-2>(df), df));
      }
      uint8_t tag = 0;
      if (want_c && ratio_gt(tc, sc, thr_c)) tag |= 1;
      if (want_g && ratio_gt(tg, sc, thr_g)) tag |= 2;
      if (want_r && sqrt_ratio_gt(gr2, Ec, thr_r)) tag |= 4;
      tags[idx] = tag;
    }
  }
}

// covered cell := mean of its 8 children (children order: x slowest ... as
// listed), for nfield fields stored fstride apart.
__global__ void k_avgdown(const int4* __restrict__ cov, int n, double* x, int nfield,
                          int fstride) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int4 c = cov[r];
    for (int f = 0; f < nfield; f++) {
      double* xf = x + (long)f * fstride;
      double s = 0.0;
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
          for (int e = 0; e < 2; e++) s += xf[c.y + a + b * c.z + e * c.w];
      xf[c.x] = s / 8.0;
    }
  }
}

int blocks_for(long n, int bs) {
  long b = (n + bs - 1) / bs;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

__global__ void k_check_fastmath(const double* x, long n, double* out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[i] = rcp_nr(v);
    out[n + i] = 1.0 / v;
    out[2 * n + i] = rsqrt_nr(v);
    out[3 * n + i] = 1.0 / sqrt(v);
  }
}

__global__ void k_check_narrow(const double* x, long n, float* out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[i] = narrow_rn(v);
    out[n + i] = __double2float_rn(v);
  }
}

LevelH level_h(const Hier& H, double k = 0.01, double beta = 0.0) {
  LevelH lh;
  for (int l = 0; l < NRD_MAX_LEVELS; l++)
    for (int d = 0; d < 3; d++) {
      double h = (l < H.L) ? H.lev[l].h[d] : 1.0;
      lh.h[l][d] = h;
      lh.rh[l][d] = 1.0 / h;
      lh.h3[l][d] = 3.0 * h;
      lh.kh[l][d] = k / h;
      lh.kh5[l][d] = 1.25 * k / h;
      lh.bh2[l][d] = beta / (h * h);
      lh.h12[l][d] = 12.0 * h;
      lh.khs[l][d] = kP52 * (k / h);
      lh.kh5s[l][d] = kP32 * (1.25 * k / h);
    }
  return lh;
}

template <int MODE, int TX, int TY, int TZ>
size_t stencil_smem() {
  if (MODE == ST_LINC || MODE == ST_RESC) return 0;   // cells and faces from global memory
  constexpr int NH = (TX + 2) * (TY + 2) * (TZ + 2);
  constexpr int NF = (TX + 1) * TY * TZ + TX * (TY + 1) * TZ + TX * TY * (TZ + 1);
  size_t d = (size_t)NH * (MODE == ST_JV ? 5 : (MODE == ST_JVF ? 2 : 3)) + 2 * (size_t)NF;
  return d * sizeof(double);
}

template <int MODE, int TX, int TY, int TZ, bool CMP>
void run_stencil(const StArgs& a, cudaStream_t s) {
  size_t sm = stencil_smem<MODE, TX, TY, TZ>();
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(k_stencil<MODE, TX, TY, TZ, CMP>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    init = true;
  }
  // one tile per CTA: the block scheduler balances tiles of uneven cost
  int grid = a.ntiles;
  if (grid < 1) return;
  k_stencil<MODE, TX, TY, TZ, CMP><<<grid, 256, sm, s>>>(a);
}

template <int MODE, bool CMP = false>
void dispatch_tile(const StArgs& a, int tx, int ty, int tz, cudaStream_t s) {
  if (tx == 32 && ty == 8 && tz == 4) run_stencil<MODE, 32, 8, 4, CMP>(a, s);
  else if (tx == 32 && ty == 4 && tz == 8) run_stencil<MODE, 32, 4, 8, CMP>(a, s);
  else if (tx == 32 && ty == 2 && tz == 4) run_stencil<MODE, 32, 2, 4, CMP>(a, s);
  else if (tx == 16 && ty == 8 && tz == 4) run_stencil<MODE, 16, 8, 4, CMP>(a, s);
  else if (tx == 16 && ty == 4 && tz == 8) run_stencil<MODE, 16, 4, 8, CMP>(a, s);
  else if (tx == 16 && ty == 8 && tz == 8) run_stencil<MODE, 16, 8, 8, CMP>(a, s);
  else if (tx == 16 && ty == 4 && tz == 4) run_stencil<MODE, 16, 4, 4, CMP>(a, s);
  else if (tx == 8 && ty == 8 && tz == 8) run_stencil<MODE, 8, 8, 8, CMP>(a, s);
  else if (tx == 8 && ty == 8 && tz == 4) run_stencil<MODE, 8, 8, 4, CMP>(a, s);
  else run_stencil<MODE, 32, 4, 4, CMP>(a, s);
}

// the compact-cell form where the hierarchy has ragged tiles, for the launches
// of the Newton and Krylov loops (the cell launches and the frozen Jv)
template <int MODE>
void dispatch_tile_h(const Hier& H, const StArgs& a, cudaStream_t s) {
  if (H.ragged) dispatch_tile<MODE, true>(a, H.tile_x, H.tile_y, H.tile_z, s);
  else dispatch_tile<MODE, false>(a, H.tile_x, H.tile_y, H.tile_z, s);
}

}  // namespace

void launch_ghost_fill(const Hier& H, const ModelParams& mp, const float* z, const double* u,
                       double* g, int nonlinear, cudaStream_t s) {
  GhostArgs a;
  a.gtype = H.d_gtype;
  a.gface = H.d_gface;
  a.gcell = H.d_gcell;
  a.gt0 = H.d_gt0;
  a.gidx = H.d_gidx;
  a.gw = H.d_gw;
  a.z = z;
  a.N = H.N;
  a.G = H.G;
  for (int f = 0; f < 6; f++) a.R[f] = mp.bc_R[f];
  a.lh = level_h(H);
  if (H.G == 0) return;
  k_ghost_fill<<<blocks_for(H.G, 256), 256, 0, s>>>(a, u, g, nonlinear);
}

__global__ void k_cube(const float* z, long n, double* z3) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const double v = (double)z[i];
    z3[i] = v * v * v;
  }
}

void launch_cube(const Hier& H, const float* z, const float* gz, double* z3, cudaStream_t s) {
  k_cube<<<blocks_for(H.N, 256), 256, 0, s>>>(z, H.N, z3);
  if (H.G) k_cube<<<blocks_for(H.G, 256), 256, 0, s>>>(gz, H.G, z3 + H.N);
}

void launch_ghost_z(const Hier& H, const float* z, float* gz, cudaStream_t s) {
  if (H.G == 0) return;
  k_ghost_z<<<blocks_for(H.G, 256), 256, 0, s>>>(H.d_gzsrc, z, gz, H.G);
}

void launch_stencil(const Hier& H, const ModelParams& mp, const float* z, const float* gz,
                    int mode, const StencilIO& io, cudaStream_t s, const double* z3) {
  StArgs a;
  a.z3 = z3;
  a.tiles = H.d_tiles;
  a.patches = H.d_patches;
  a.mask = H.d_mask;
  a.gtype = H.d_gtype;
  a.z = z;
  a.gz = gz;
  a.ntiles = (int)H.tiles.size();
  a.N = H.N;
  a.G = H.G;
  a.k = mp.k;
  a.cL = (mp.limiter == NRD_LIM_PAPER_LITERAL) ? 2.0 : 4.0;
  a.cL2 = 0.5 * a.cL;
  a.m15cL = -1.5 * a.cL;
  for (int f = 0; f < 6; f++) a.R[f] = mp.bc_R[f];
  a.lh = level_h(H, mp.k, io.beta);
  a.io = io;
  if (mode == ST_RESIDUAL && io.pef) {
    dispatch_tile<ST_RESF>(a, H.tile_x, H.tile_y, H.tile_z, s);
    dispatch_tile_h<ST_RESC>(H, a, s);
  } else if (mode == ST_RESIDUAL) dispatch_tile<ST_RESIDUAL>(a, H.tile_x, H.tile_y, H.tile_z, s);
  else if (mode == ST_JV) dispatch_tile<ST_JV>(a, H.tile_x, H.tile_y, H.tile_z, s);
  else if (mode == ST_LIN && io.pef) {
    dispatch_tile<ST_LINF>(a, H.tile_x, H.tile_y, H.tile_z, s);
    dispatch_tile_h<ST_LINC>(H, a, s);
  } else if (mode == ST_LIN) dispatch_tile<ST_LIN>(a, H.tile_x, H.tile_y, H.tile_z, s);
  else if (mode == ST_LINZ) dispatch_tile<ST_LINZ>(a, H.tile_x, H.tile_y, H.tile_z, s);
  else if (mode == ST_JVF) dispatch_tile_h<ST_JVF>(H, a, s);
  else dispatch_tile<ST_FD>(a, H.tile_x, H.tile_y, H.tile_z, s);
}

void launch_reflux(const Hier& H, const StencilIO& io, int mode, cudaStream_t s) {
  if (H.nrf == 0) return;
  RfArgs a;
  a.cell = H.d_rf_cell;
  a.off = H.d_rf_off;
  a.face = H.d_rf_face;
  a.g = H.d_rf_g;
  a.patches = H.d_patches;
  a.nrf = H.nrf;
  a.N = H.N;
  a.G = H.G;
  a.lh = level_h(H);
  k_reflux<<<blocks_for(H.nrf, 128), 128, 0, s>>>(a, H.d_rf_level, io.cfflux, io.out, io.dt,
                                                   io.par, io.eps, mode);
}

void launch_jv_frozen(const Hier& H, const ModelParams& mp, const double* jc, const double* cc,
                      const StencilIO& io, cudaStream_t s) {
  // the tiled stencil in ST_JVF mode: v staged in shared memory, each face's
  // tangent flux formed once from the stored partials
  StencilIO q = io;
  q.jc = const_cast<double*>(jc);
  q.cc = const_cast<double*>(cc);
  launch_stencil(H, mp, nullptr, nullptr, ST_JVF, q, s);
}

void launch_tag(const Hier& H, const double* E, const double* gE, double thr_c, double thr_g,
                double thr_r, const double* emax, uint8_t* tags, cudaStream_t s) {
  // tag tiles: reuse the stencil tile list (tiles are at most 32 x 8 x 8)
  k_tag<<<std::min((int)H.tiles.size(), 152 * 8), 256, 0, s>>>(
      H.d_tiles, H.d_patches, (int)H.tiles.size(), H.tile_x, H.tile_y, H.tile_z, E, gE, thr_c, thr_g, thr_r,
      emax, tags);
}

void launch_average_down(const Hier& H, double* x, int nfield, int fstride, cudaStream_t s) {
  for (int l = H.L - 2; l >= 0; l--) {
    if (H.ncov[l] == 0) continue;
    k_avgdown<<<blocks_for(H.ncov[l], 256), 256, 0, s>>>(H.d_cov[l], H.ncov[l], x, nfield,
                                                          fstride);
  }
}

extern "C" int nrd_check_fastmath(const double* x, int64_t n, double* out, cudaStream_t s) {
  if (!x || !out || n < 0) return NRD_EINVAL;
  if (n == 0) return NRD_OK;
  const int grid = (int)std::min<long>(152L * 8, (n + 255) / 256);
  k_check_fastmath<<<grid, 256, 0, s>>>(x, n, out);
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}

extern "C" int nrd_check_narrow(const double* x, int64_t n, float* out, cudaStream_t s) {
  if (!x || !out || n < 0) return NRD_EINVAL;
  if (n == 0) return NRD_OK;
  const int grid = (int)std::min<long>(152L * 8, (n + 255) / 256);
  k_check_narrow<<<grid, 256, 0, s>>>(x, n, out);
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}
