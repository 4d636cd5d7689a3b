// Physics-based preconditioner P = P1 P2 (Sec. 4.2) with FAC (Sec. 4.3,
// Algorithm 1) on the two diffusion blocks of P1 and a geometric multigrid
// V-cycle on the base box.
//
//   set-up   face coefficients D_E^k, D_T^k frozen at the Newton iterate
//            (same face formulas as the residual), coarsened to covered
//            faces and to the GMG levels as the mean of the 4 coincident fine
//            faces, then scaled to a = beta C / h^2 in the V-cycle precision;
//            Robin faces carry beta 2 D_b / (h (4 D_b + h)) on the diagonal.
//   apply    FAC V(nu1, nu2): red-black Gauss-Seidel on each AMR level with
//            homogeneous coarse-fine ghosts (e_g = e_c/3), correction of the
//            composite solution interpolated to every finer level, composite
//            residual (with coarse-fine interpolation and flux matching)
//            recomputed before every smoothing pass; GMG V-cycle on level 0;
//            then the cell-local 2x2 P2 solve in FP64.
// Both fields (E, T) are processed by every launch (blockIdx.y = field).
#include <algorithm>
#include <cstdio>

#include "nrd_internal.h"

namespace {

constexpr int BS = 256;

int g1(long n) {
  long b = (n + BS - 1) / BS;
  return (int)std::max(1L, std::min(b, 152L * 16));
}

struct LevelHP {
  double h[NRD_MAX_LEVELS][3];
};

// ------------------------------------------------------------- box levels
template <class P>
struct BoxV {
  int n[3];
  int fo[6];
  const P* A;     // coefficients of field 0; field f at A + f * Afs
  long Afs;
  long NA;        // stride of the low-face blocks
  long gbase;     // index of the first boundary slot
  long cell0;     // first cell of the box in the vectors
  P* e;           // correction, field f at e + f * vfs
  const P* f;     // right-hand side
  long vfs;
};

template <class P>
__device__ __forceinline__ void box_row(const BoxV<P>& V, int fld, int i, int j, int k, const P* e,
                                        P& dg, P& of) {
  const P* A = V.A + fld * V.Afs;
  const int n0 = V.n[0], n1 = V.n[1], n2 = V.n[2];
  long idx = i + (long)n0 * (j + (long)n1 * k);
  long ci = V.cell0 + idx;
  P d = P(1), o = P(0), a;
  if (i > 0) { a = A[ci]; d += a; o += a * e[idx - 1]; }
  else d += A[V.gbase + V.fo[0] + j + n1 * k];
  if (i < n0 - 1) { a = A[ci + 1]; d += a; o += a * e[idx + 1]; }
  else d += A[V.gbase + V.fo[1] + j + n1 * k];
  if (j > 0) { a = A[V.NA + ci]; d += a; o += a * e[idx - n0]; }
  else d += A[V.gbase + V.fo[2] + k + n2 * i];
  if (j < n1 - 1) { a = A[V.NA + ci + n0]; d += a; o += a * e[idx + n0]; }
  else d += A[V.gbase + V.fo[3] + k + n2 * i];
  long s2 = (long)n0 * n1;
  if (k > 0) { a = A[2 * V.NA + ci]; d += a; o += a * e[idx - s2]; }
  else d += A[V.gbase + V.fo[4] + i + n0 * j];
  if (k < n2 - 1) { a = A[2 * V.NA + ci + s2]; d += a; o += a * e[idx + s2]; }
  else d += A[V.gbase + V.fo[5] + i + n0 * j];
  dg = d;
  of = o;
}

// one colour of a red-black Gauss-Seidel sweep on a box level
template <class P>
__global__ void k_box_rbgs(BoxV<P> V, int colour) {
  const int fld = blockIdx.y;
  P* e = V.e + fld * V.vfs;
  const P* f = V.f + fld * V.vfs;
  const long nc = (long)V.n[0] * V.n[1] * V.n[2];
  // thread t handles the t-th cell of the requested colour
  const long nhalf = (nc + 1) / 2;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nhalf;
       t += (long)gridDim.x * blockDim.x) {
    long idx = 2 * t;
    int i = (int)(idx % V.n[0]);
    long r = idx / V.n[0];
    int j = (int)(r % V.n[1]);
    int k = (int)(r / V.n[1]);
    if (((i + j + k) & 1) != colour) {
      i += 1;
      if (i >= V.n[0]) continue;  // only when n0 is odd; the cell is picked up elsewhere
    }
    long c = i + (long)V.n[0] * (j + (long)V.n[1] * k);
    P dg, of;
    box_row(V, fld, i, j, k, e, dg, of);
    e[c] = (f[c] + of) / dg;
  }
}

// same, for boxes with odd n0: one thread per cell
template <class P>
__global__ void k_box_rbgs_odd(BoxV<P> V, int colour) {
  const int fld = blockIdx.y;
  P* e = V.e + fld * V.vfs;
  const P* f = V.f + fld * V.vfs;
  const long nc = (long)V.n[0] * V.n[1] * V.n[2];
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < nc;
       c += (long)gridDim.x * blockDim.x) {
    int i = (int)(c % V.n[0]);
    long r = c / V.n[0];
    int j = (int)(r % V.n[1]);
    int k = (int)(r / V.n[1]);
    if (((i + j + k) & 1) != colour) continue;
    P dg, of;
    box_row(V, fld, i, j, k, e, dg, of);
    e[c] = (f[c] + of) / dg;
  }
}

// coarse f = 8-cell average of the fine residual f - L e (Sec. 4.3: simple
// averaging restriction)
template <class P>
__global__ void k_box_restrict(BoxV<P> F, P* fc, long cfs) {
  const int fld = blockIdx.y;
  const P* e = F.e + fld * F.vfs;
  const P* f = F.f + fld * F.vfs;
  const int cn0 = F.n[0] / 2, cn1 = F.n[1] / 2, cn2 = F.n[2] / 2;
  const long ncc = (long)cn0 * cn1 * cn2;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncc;
       c += (long)gridDim.x * blockDim.x) {
    int ci = (int)(c % cn0);
    long r = c / cn0;
    int cj = (int)(r % cn1), ck = (int)(r / cn1);
    P s = P(0);
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int d = 0; d < 2; d++) {
          int i = 2 * ci + a, j = 2 * cj + b, k = 2 * ck + d;
          long q = i + (long)F.n[0] * (j + (long)F.n[1] * k);
          P dg, of;
          box_row(F, fld, i, j, k, e, dg, of);
          s += f[q] - (dg * e[q] - of);
        }
    fc[fld * cfs + c] = s / P(8);
  }
}

// trilinear interpolation weight along one axis: (3/4 parent, 1/4 neighbour);
// neighbours outside the domain fall back to the parent
template <class P>
__device__ __forceinline__ P tri_interp(const P* src, const int cn[3], const int q[3],
                                        const int* map, long moff) {
  int p[3], o[3];
  for (int d = 0; d < 3; d++) {
    p[d] = q[d] >> 1;
    o[d] = (q[d] & 1) ? 1 : -1;
    if (p[d] + o[d] < 0 || p[d] + o[d] >= cn[d]) o[d] = 0;
  }
  P s = P(0);
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++)
      for (int d = 0; d < 2; d++) {
        P w = (a ? P(0.25) : P(0.75)) * (b ? P(0.25) : P(0.75)) * (d ? P(0.25) : P(0.75));
        int i = p[0] + (a ? o[0] : 0), j = p[1] + (b ? o[1] : 0), k = p[2] + (d ? o[2] : 0);
        long li = i + (long)cn[0] * (j + (long)cn[1] * k);
        long si = map ? (long)map[li] : li + moff;
        if (si < 0) si = map[p[0] + (long)cn[0] * (p[1] + (long)cn[1] * p[2])];  // nesting guard
        s += w * src[si];
      }
  return s;
}

template <class P>
__global__ void k_box_prolong_add(const P* ec, long cfs, int cn0, int cn1, int cn2, BoxV<P> F) {
  const int fld = blockIdx.y;
  P* e = F.e + fld * F.vfs;
  const P* src = ec + fld * cfs;
  const int cn[3] = {cn0, cn1, cn2};
  const long nc = (long)F.n[0] * F.n[1] * F.n[2];
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < nc;
       c += (long)gridDim.x * blockDim.x) {
    int q[3];
    q[0] = (int)(c % F.n[0]);
    long r = c / F.n[0];
    q[1] = (int)(r % F.n[1]);
    q[2] = (int)(r / F.n[1]);
    e[c] += tri_interp(src, cn, q, (const int*)nullptr, 0);
  }
}

// ------------------------------------------------- AMR (multi-patch) levels
template <class P>
struct HierV {
  const TileDev* tiles;
  const PatchDev* patches;
  const uint8_t* mask;
  const uint8_t* gtype;
  const int* gt0;      // sibling ghost -> its source cell is gidx[gt0[g]]
  const int* gidx;
  const P* A;        // field f at A + f * Afs; slots [3N | G]
  long Afs;
  int N, G;
};

// level-l row of I - beta div D grad (homogeneous coarse-fine ghosts)
template <class P>
__device__ __forceinline__ void lev_row(const HierV<P>& V, const PatchDev& Pt, int fld, int i,
                                        int j, int k, const P* e, const P* gh, P& dg, P& of) {
  const P* A = V.A + fld * V.Afs;
  const int nx = Pt.n[0], ny = Pt.n[1], nz = Pt.n[2];
  const long N = V.N;
  long idx = Pt.off + i + (long)nx * (j + (long)ny * k);
  P d = P(1), o = P(0);
  auto bnd = [&](int f, int a, int b) {
    int g = Pt.goff + Pt.fo[f] + a + Pt.n[((f >> 1) + 1) % 3] * b;
    uint8_t t = V.gtype[g];
    P av = A[3 * N + g];
    // a sibling cell has the other colour: read it directly
    if (t == GT_SIBLING) { d += av; o += av * e[V.gidx[V.gt0[g]]]; }
    else if (t == GT_CF) d += P(2.0 / 3.0) * av;
    else d += av;   // Robin diagonal term, or 0 for Neumann
  };
  P a;
  if (i > 0) { a = A[idx]; d += a; o += a * e[idx - 1]; } else bnd(0, j, k);
  if (i < nx - 1) { a = A[idx + 1]; d += a; o += a * e[idx + 1]; } else bnd(1, j, k);
  if (j > 0) { a = A[N + idx]; d += a; o += a * e[idx - nx]; } else bnd(2, k, i);
  if (j < ny - 1) { a = A[N + idx + nx]; d += a; o += a * e[idx + nx]; } else bnd(3, k, i);
  long s2 = (long)nx * ny;
  if (k > 0) { a = A[2 * N + idx]; d += a; o += a * e[idx - s2]; } else bnd(4, i, j);
  if (k < nz - 1) { a = A[2 * N + idx + s2]; d += a; o += a * e[idx + s2]; } else bnd(5, i, j);
  dg = d;
  of = o;
}

template <class P>
__global__ void k_lev_rbgs(HierV<P> V, int t0, int nt, int tx, int ty, int tz, P* e, const P* f,
                           const P* gh, int colour) {
  const int fld = blockIdx.y;
  P* ef = e + (long)fld * V.N;
  const P* ff = f + (long)fld * V.N;
  const P* gf = gh + (long)fld * V.G;
  // one thread per x-pair of cells: exactly one of the two has the colour
  const int hx = tx >> 1;
  const int np = hx * ty * tz;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const TileDev tile = V.tiles[t0 + t];
    const PatchDev Pt = V.patches[tile.patch];
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
      int j = tile.j0 + (q / hx) % ty, k = tile.k0 + q / (hx * ty);
      int i = tile.i0 + 2 * (q % hx);
      if (((Pt.lo[0] + i + Pt.lo[1] + j + Pt.lo[2] + k) & 1) != colour) i += 1;
      if (i >= Pt.n[0] || j >= Pt.n[1] || k >= Pt.n[2]) continue;
      long idx = Pt.off + i + (long)Pt.n[0] * (j + (long)Pt.n[1] * k);
      P dg, of;
      lev_row(V, Pt, fld, i, j, k, ef, gf, dg, of);
      ef[idx] = (ff[idx] + of) / dg;
    }
  }
}

// sibling ghosts of a level vector (raw copies)
template <class P>
__global__ void k_sib_ghost(const uint8_t* gtype, const int* gt0, const int* gidx, int g0, int ng,
                            int N, int G, const P* e, P* gh) {
  const int fld = blockIdx.y;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ng; q += gridDim.x * blockDim.x) {
    int g = g0 + q;
    if (gtype[g] != GT_SIBLING) continue;
    gh[(long)fld * G + g] = e[(long)fld * N + gidx[gt0[g]]];
  }
}

// sibling and coarse-fine ghosts of a composite vector
template <class P>
__global__ void k_lin_ghost(const uint8_t* gtype, const int* gt0, const int* gidx, const double* gw,
                            int N, int G, const P* u, P* gh) {
  const int fld = blockIdx.y;
  const P* uf = u + (long)fld * N;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    uint8_t t = gtype[g];
    if (t != GT_SIBLING && t != GT_CF) continue;
    double s = 0.0;
    for (int q = gt0[g]; q < gt0[g + 1]; q++) s += gw[q] * (double)uf[gidx[q]];
    gh[(long)fld * G + g] = (P)s;
  }
}

// r = f - L^c u on leaf cells (composite operator with coarse-fine
// interpolation); fine-side coarse-fine fluxes a (u_g - u_c) go to cf.
template <class P>
__global__ void k_comp_resid(HierV<P> V, int ntiles, int tx, int ty, int tz, const P* u, const P* f,
                             const P* gh, P* r, P* cf) {
  const int fld = blockIdx.y;
  const long N = V.N;
  const P* A = V.A + fld * V.Afs;
  const P* uf = u + fld * N;
  const P* ff = f + fld * N;
  const P* gf = gh + (long)fld * V.G;
  P* rf = r + fld * N;
  P* cff = cf + (long)fld * V.G;
  const int nc = tx * ty * tz;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const TileDev tile = V.tiles[t];
    const PatchDev Pt = V.patches[tile.patch];
    const int nx = Pt.n[0], ny = Pt.n[1], nz = Pt.n[2];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int i = tile.i0 + c % tx, j = tile.j0 + (c / tx) % ty, k = tile.k0 + c / (tx * ty);
      if (i >= nx || j >= ny || k >= nz) continue;
      long idx = Pt.off + i + (long)nx * (j + (long)ny * k);
      uint8_t m = V.mask[idx];
      if (m & MASK_COVERED) { rf[idx] = P(0); continue; }
      P uc = uf[idx];
      P Lu = uc;
      auto bnd = [&](int f, int a, int b) {
        int g = Pt.goff + Pt.fo[f] + a + Pt.n[((f >> 1) + 1) % 3] * b;
        uint8_t t = V.gtype[g];
        P av = A[3 * N + g];
        if (t == GT_SIBLING || t == GT_CF) {
          P ug = gf[g];
          Lu += av * (uc - ug);
          if (t == GT_CF) cff[g] = av * (ug - uc);
        } else {
          Lu += av * uc;   // Robin term (0 for Neumann)
        }
      };
      P a;
      if (!(m & 2)) { if (i > 0) { a = A[idx]; Lu += a * (uc - uf[idx - 1]); } else bnd(0, j, k); }
      if (!(m & 4)) { if (i < nx - 1) { a = A[idx + 1]; Lu += a * (uc - uf[idx + 1]); } else bnd(1, j, k); }
      if (!(m & 8)) { if (j > 0) { a = A[N + idx]; Lu += a * (uc - uf[idx - nx]); } else bnd(2, k, i); }
      if (!(m & 16)) { if (j < ny - 1) { a = A[N + idx + nx]; Lu += a * (uc - uf[idx + nx]); } else bnd(3, k, i); }
      long s2 = (long)nx * ny;
      if (!(m & 32)) { if (k > 0) { a = A[2 * N + idx]; Lu += a * (uc - uf[idx - s2]); } else bnd(4, i, j); }
      if (!(m & 64)) { if (k < nz - 1) { a = A[2 * N + idx + s2]; Lu += a * (uc - uf[idx + s2]); } else bnd(5, i, j); }
      rf[idx] = ff[idx] - Lu;
    }
  }
}

// flux matching for the composite operator: coarse cell gets sum(phi)/8 per
// coarse-fine face
template <class P>
__global__ void k_comp_reflux(const int* cell, const int* off, const int4* gq, int nrf, int N,
                              int G, const P* cf, P* r) {
  const int fld = blockIdx.y;
  const P* c = cf + (long)fld * G;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nrf; q += gridDim.x * blockDim.x) {
    P s = P(0);
    for (int e = off[q]; e < off[q + 1]; e++) {
      int4 g = gq[e];
      s += c[g.x] + c[g.y] + c[g.z] + c[g.w];
    }
    r[(long)fld * N + cell[q]] -= s / P(8);
  }
}

template <class P>
__global__ void k_avgdown_p(const int4* __restrict__ cov, int n, P* x, int N) {
  const int fld = blockIdx.y;
  P* xf = x + (long)fld * N;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int4 c = cov[q];
    P s = P(0);
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int e = 0; e < 2; e++) s += xf[c.y + a + b * c.z + e * c.w];
    xf[c.x] = s / P(8);
  }
}

// u += e on the uncovered cells of [c0, c0 + n)
template <class P>
__global__ void k_add_leaf(const uint8_t* mask, int c0, int n, int N, const P* e, P* u) {
  const int fld = blockIdx.y;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int c = c0 + q;
    if (!(mask[c] & MASK_COVERED)) u[(long)fld * N + c] += e[(long)fld * N + c];
  }
}

// pv(level m) = trilinear interpolation of src(level m-1) via the dense map;
// u += pv on uncovered level-m cells
template <class P>
__global__ void k_prolong_level(const TileDev* tiles, const PatchDev* patches, int t0, int nt, int tx,
                                int ty, int tz, const uint8_t* mask, const int* cmap, int cn0, int cn1,
                                int cn2, int N, const P* src, P* pv, P* u) {
  const int fld = blockIdx.y;
  const int cn[3] = {cn0, cn1, cn2};
  const P* s = src + (long)fld * N;
  const int nc = tx * ty * tz;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const TileDev tile = tiles[t0 + t];
    const PatchDev Pt = patches[tile.patch];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int i = tile.i0 + c % tx, j = tile.j0 + (c / tx) % ty, k = tile.k0 + c / (tx * ty);
      if (i >= Pt.n[0] || j >= Pt.n[1] || k >= Pt.n[2]) continue;
      long idx = Pt.off + i + (long)Pt.n[0] * (j + (long)Pt.n[1] * k);
      int q[3] = {Pt.lo[0] + i, Pt.lo[1] + j, Pt.lo[2] + k};
      P v = tri_interp(s, cn, q, cmap, 0);
      pv[(long)fld * N + idx] = v;
      if (!(mask[idx] & MASK_COVERED)) u[(long)fld * N + idx] += v;
    }
  }
}

// y = P2^{-1} z per leaf cell, P2 = [[1 + s b, -s b T^3], [-s b, 1 + s b T^3]],
// s = z^3/T^3 at the frozen iterate (Sec. 4.2)
// P2 data frozen at the iterate: p[c] = sigma beta, p[N+c] = sigma beta T^3,
// p[2N+c] = 1/det with P2 = [[1 + p0, -p1], [-p0, 1 + p1]].
// det P2 = (1 + p0)(1 + p1) - p0 p1 = 1 + p0 + p1 (formed without the
// cancellation).  Stored in the V-cycle precision P.
template <class P>
__global__ void k_p2_setup(const uint8_t* mask, int N, const double* Tk, const float* zm,
                           const double* beta_p, P* p) {
  const double beta = *beta_p;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    double T = Tk[c];
    double T3 = T * T * T;
    double z = (double)zm[c];
    double sig = z * z * z / T3;
    double sb = sig * beta, sbt = sb * T3;
    bool cov = mask[c] & MASK_COVERED;
    p[c] = cov ? P(0) : (P)sb;
    p[N + c] = cov ? P(0) : (P)sbt;
    p[2L * N + c] = cov ? P(0) : (P)(1.0 / (1.0 + sb + sbt));
  }
}

// y = P2^{-1} z per leaf cell (Sec. 4.2); covered cells get 0
template <class P>
__global__ void k_p2(int N, const P* zin, const P* p, double* y, const int* jd, long jstride,
                     double* y2) {
  if (jd) y += (long)(*jd) * jstride;   // y = column *jd of a basis (device index)
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const P sb = p[c], sbt = p[N + c], rd = p[2L * N + c];
    const P zE = zin[c], zT = zin[N + c];
    const double yE = (double)(((P(1) + sbt) * zE + sbt * zT) * rd);
    const double yT = (double)(((P(1) + sb) * zT + sb * zE) * rd);
    y[c] = yE;
    y[N + c] = yT;
    if (y2) {
      y2[c] = yE;
      y2[N + c] = yT;
    }
  }
}

// transposed P2 solve fused with the cast into the V-cycle precision:
// P2^T = [[1 + sb, -sb], [-sbt, 1 + sbt]]
template <class P>
__global__ void k_p2t_cast(int N, const double* w, const P* p, P* out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const P sb = p[c], sbt = p[N + c], rd = p[2L * N + c];
    const P wE = (P)w[c], wT = (P)w[N + c];
    out[c] = ((P(1) + sbt) * wE + sb * wT) * rd;
    out[N + c] = (sbt * wE + (P(1) + sb) * wT) * rd;
  }
}

// y = V-cycle output in FP64; covered cells get 0
template <class P>
__global__ void k_out_cast(const uint8_t* mask, int N, const P* u, double* y) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    bool cov = mask[c] & MASK_COVERED;
    y[c] = cov ? 0.0 : (double)u[c];
    y[N + c] = cov ? 0.0 : (double)u[N + c];
  }
}

template <class P>
__global__ void k_cast(int n, const double* w, P* out, const int* jd, long jstride) {
  if (jd) w += (long)(*jd) * jstride;   // w = column *jd of a basis (device index)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (P)w[i];
}

// ----------------------------------------------------------- set-up kernels
struct SetupArgs {
  double bh2[NRD_MAX_LEVELS][3];   // beta / h^2
  const TileDev* tiles;
  const PatchDev* patches;
  const uint8_t* mask;
  const uint8_t* gtype;
  const uint8_t* gface;
  const int* gidx;
  const int* gt0;
  const double* u;     // frozen iterate
  const double* gu;    // its ghosts
  const float* z;
  const float* gz;
  int N, G, ntiles, tx, ty, tz;
  double k, cL, beta;
  LevelHP lh;
  double* Craw;        // [2][3N+G]
};

__device__ __forceinline__ void coef_pair(double Ea, double Eb, double Ta, double Tb, double za,
                                          double zb, double h, double k, double cL, double& CE,
                                          double& CT) {
  // D_E = D_h/(1 + D_h |dE|/(h E_f)), D_h = 2 T_f^3/(3 (z_a^3 + z_b^3))
  // (or the printed form, cL = 2); D_T = k T_f^(5/2)
  double Tf = 0.5 * (Ta + Tb);
  double Tf3 = Tf * Tf * Tf;
  double Zs = za * za * za + zb * zb * zb;
  double Dr = Tf3 / (3.0 * Zs);
  double g = fabs(Eb - Ea) / (0.5 * h * (Ea + Eb));
  CE = (cL == 4.0) ? (2.0 * Dr) / (1.0 + 2.0 * Dr * g) : 2.0 * Dr / (1.0 + Dr * g);
  CT = k * Tf * Tf * sqrt(Tf);
}

// raw face coefficients of every face whose two sides are uncovered leaf
// cells (or a leaf cell and a coarse-fine ghost); Robin slots get D_b.
__global__ void k_coef(SetupArgs a) {
  const int N = a.N, G = a.G;
  const long AF = 3L * N + G;
  const int nc = a.tx * a.ty * a.tz;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const TileDev tile = a.tiles[t];
    const PatchDev Pt = a.patches[tile.patch];
    const int nx = Pt.n[0], ny = Pt.n[1], nz = Pt.n[2];
    const double* hh = a.lh.h[Pt.level];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int i = tile.i0 + c % a.tx, j = tile.j0 + (c / a.tx) % a.ty, k = tile.k0 + c / (a.tx * a.ty);
      if (i >= nx || j >= ny || k >= nz) continue;
      long idx = Pt.off + i + (long)nx * (j + (long)ny * k);
      bool cov = a.mask[idx] & MASK_COVERED;
      double Ec = a.u[idx], Tc = a.u[N + idx], zc = (double)a.z[idx];
      int loc[3] = {i, j, k};
      long st[3] = {1, nx, (long)nx * ny};
      for (int d = 0; d < 3; d++) {
        // low face of this cell inside the patch
        if (loc[d] > 0) {
          long nb = idx - st[d];
          if (!cov && !(a.mask[nb] & MASK_COVERED)) {
            double CE, CT;
            coef_pair(a.u[nb], Ec, a.u[N + nb], Tc, (double)a.z[nb], zc, hh[d], a.k, a.cL, CE, CT);
            a.Craw[d * (long)N + idx] = CE;
            a.Craw[AF + d * (long)N + idx] = CT;
          }
        }
        // patch-boundary faces of this cell
        for (int s = 0; s < 2; s++) {
          bool at = s ? (loc[d] == Pt.n[d] - 1) : (loc[d] == 0);
          if (!at) continue;
          int f = 2 * d + s;
          int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          int g = Pt.goff + Pt.fo[f] + loc[t1] + Pt.n[t1] * loc[t2];
          uint8_t ty = a.gtype[g];
          double CE = 0.0, CT = 0.0;
          if (cov) continue;  // covered cells: coarsened from the finer level
          if (ty == GT_ROBIN) {
            CE = Tc * Tc * Tc / (3.0 * (zc * zc * zc));   // D_b
          } else if (ty == GT_SIBLING) {
            int nb = a.gidx[a.gt0[g]];
            if (a.mask[nb] & MASK_COVERED) continue;       // coarsened
            coef_pair(Ec, a.gu[g], Tc, a.gu[G + g], zc, (double)a.gz[g], hh[d], a.k, a.cL, CE, CT);
          } else if (ty == GT_CF) {
            coef_pair(Ec, a.gu[g], Tc, a.gu[G + g], zc, (double)a.gz[g], hh[d], a.k, a.cL, CE, CT);
          }
          a.Craw[3L * N + g] = CE;
          a.Craw[AF + 3L * N + g] = CT;
        }
      }
    }
  }
}

// covered faces of level l: mean of the 4 coincident faces on level l+1;
// with A non-null also the scaled coefficient of the target (level l)
template <class P>
__global__ void k_coef_coarsen(const int* tgt, const int4* src, int n, long AF, int N,
                               const uint8_t* gtype, const uint8_t* gface,
                               const double* dbeta, LevelHP lh, int lvl, double* Craw, P* A) {
  const double beta = *dbeta;
  const int fld = blockIdx.y;
  double* C = Craw + fld * AF;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int4 s = src[q];
    int t = tgt[q];
    double c = 0.25 * (C[s.x] + C[s.y] + C[s.z] + C[s.w]);
    C[t] = c;
    if (!A) continue;
    double v;
    if (t < 3L * N) {
      double h = lh.h[lvl][t / N];
      v = c * beta / (h * h);
    } else {
      int g = t - 3 * N;
      int d = (gface[g] & 7) / 2;
      double h = lh.h[lvl][d];
      uint8_t ty = gtype[g];
      if (ty == GT_NEUMANN) v = 0.0;
      else if (ty == GT_ROBIN) v = (fld == 0) ? beta * 2.0 * c / (h * (4.0 * c + h)) : 0.0;
      else v = c * beta / (h * h);
    }
    A[fld * AF + t] = (P)v;
  }
}

// scale raw coefficients of the hierarchy: a = beta C / h^2; Robin slots:
// beta 2 D_b / (h (4 D_b + h)) for E and 0 for T; Neumann slots: 0.
template <class P>
__global__ void k_scale_hier(SetupArgs a, const int* cell_level_unused, P* A) {
  const int N = a.N, G = a.G;
  const long AF = 3L * N + G;
  const int nc = a.tx * a.ty * a.tz;
  const int fld = blockIdx.y;
  const double* C = a.Craw + fld * AF;
  P* Af = A + fld * AF;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const TileDev tile = a.tiles[t];
    const PatchDev Pt = a.patches[tile.patch];
    const int nx = Pt.n[0], ny = Pt.n[1], nz = Pt.n[2];
    const double* hh = a.lh.h[Pt.level];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int i = tile.i0 + c % a.tx, j = tile.j0 + (c / a.tx) % a.ty, k = tile.k0 + c / (a.tx * a.ty);
      if (i >= nx || j >= ny || k >= nz) continue;
      long idx = Pt.off + i + (long)nx * (j + (long)ny * k);
      int loc[3] = {i, j, k};
      const double* bh2 = a.bh2[Pt.level];
      for (int d = 0; d < 3; d++) {
        double h = hh[d];
        if (loc[d] > 0) Af[d * (long)N + idx] = (P)(C[d * (long)N + idx] * bh2[d]);
        for (int s = 0; s < 2; s++) {
          bool at = s ? (loc[d] == Pt.n[d] - 1) : (loc[d] == 0);
          if (!at) continue;
          int f = 2 * d + s;
          int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          int g = Pt.goff + Pt.fo[f] + loc[t1] + Pt.n[t1] * loc[t2];
          uint8_t ty = a.gtype[g];
          double v;
          if (ty == GT_NEUMANN) v = 0.0;
          else if (ty == GT_ROBIN) {
            double Db = C[3L * N + g];
            v = (fld == 0) ? a.beta * 2.0 * Db / (h * (4.0 * Db + h)) : 0.0;
          } else {
            v = C[3L * N + g] * bh2[d];
          }
          Af[3L * N + g] = (P)v;
        }
      }
    }
  }
}

// GMG level m >= 1 from level m-1 (boxes): raw coefficients averaged over
// the 4 coincident fine faces, Robin D_b averaged, then scaled.
struct BoxRaw {
  int n[3];
  int fo[6];
  long NA, gbase, cell0, AF;
};

// fused with the scaling of the coarse level:
// A = beta C / h^2 on interior faces, beta 2 D_b / (h (4 D_b + h)) on Robin
// faces of E, 0 elsewhere; rh2 = 1/h^2 per axis of the coarse level.
template <class P>
__global__ void k_box_coarsen(BoxRaw F, const double* Cf, BoxRaw Cc, double* Cc_raw,
                              const int* gtype_box, const double* dbeta, double hx, double hy,
                              double hz, double rh2x, double rh2y, double rh2z, P* A) {
  const int fld = blockIdx.y;
  const double* cf = Cf + fld * F.AF;
  double* cc = Cc_raw + fld * Cc.AF;
  P* Af = A + fld * Cc.AF;
  const double beta = *dbeta;
  const double hh[3] = {hx, hy, hz};
  const double bh2[3] = {beta * rh2x, beta * rh2y, beta * rh2z};
  const long ncc = (long)Cc.n[0] * Cc.n[1] * Cc.n[2];
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncc;
       c += (long)gridDim.x * blockDim.x) {
    int q[3];
    q[0] = (int)(c % Cc.n[0]);
    long r = c / Cc.n[0];
    q[1] = (int)(r % Cc.n[1]);
    q[2] = (int)(r / Cc.n[1]);
    for (int d = 0; d < 3; d++) {
      int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      if (q[d] > 0) {
        double s = 0.0;
        for (int a = 0; a < 2; a++)
          for (int b = 0; b < 2; b++) {
            int p[3];
            p[d] = 2 * q[d];
            p[t1] = 2 * q[t1] + a;
            p[t2] = 2 * q[t2] + b;
            long fi = F.cell0 + p[0] + (long)F.n[0] * (p[1] + (long)F.n[1] * p[2]);
            s += cf[d * F.NA + fi];
          }
        cc[d * Cc.NA + c] = 0.25 * s;
        Af[d * Cc.NA + c] = (P)(0.25 * s * bh2[d]);
      }
      for (int sd = 0; sd < 2; sd++) {
        bool at = sd ? (q[d] == Cc.n[d] - 1) : (q[d] == 0);
        if (!at) continue;
        int f = 2 * d + sd;
        double s = 0.0;
        for (int a = 0; a < 2; a++)
          for (int b = 0; b < 2; b++) {
            int p1 = 2 * q[t1] + a, p2 = 2 * q[t2] + b;
            s += cf[F.gbase + F.fo[f] + p1 + F.n[t1] * p2];
          }
        const long g = Cc.gbase + Cc.fo[f] + q[t1] + Cc.n[t1] * q[t2];
        cc[g] = 0.25 * s;
        double v = 0.0;
        if (gtype_box[f] == 1 && fld == 0) {
          const double Db = 0.25 * s, h = hh[d];
          v = beta * 2.0 * Db / (h * (4.0 * Db + h));
        }
        Af[g] = (P)v;
      }
    }
  }
}

}  // namespace

// ------------------------------------------------------------------ state
struct PcState {
  int prec = NRD_PC_F32;
  int nmg = 1, nu1 = 2, nu2 = 2, csw = 4;
  size_t esz = 4;
  double beta = 0.0;
  long AF = 0;           // hierarchy coefficient slots per field
  double* Craw = nullptr;
  void* A = nullptr;     // [2][AF] in precision P
  void* fu = nullptr;    // composite solution [2][N]
  void* fr = nullptr;    // composite residual / level rhs
  void* fe = nullptr;    // level corrections
  void* fp = nullptr;    // prolongation scratch
  void* ff = nullptr;    // rhs
  void* gh = nullptr;    // [2][G] ghosts
  void* cf = nullptr;    // [2][G] coarse-fine fluxes
  double* Tk = nullptr;  // frozen T [N]
  const float* z = nullptr;
  // GMG levels m = 1..nmg-1
  BoxRaw box[NRD_MAX_MG];
  double bh[NRD_MAX_MG][3];
  double* bCraw[NRD_MAX_MG] = {nullptr};
  void* bA[NRD_MAX_MG] = {nullptr};
  void* be[NRD_MAX_MG] = {nullptr};
  void* bf[NRD_MAX_MG] = {nullptr};
  int* bgt = nullptr;    // [6] boundary type per box face (1 = Robin)
  double* d_beta = nullptr;
  void* p2 = nullptr;    // [3][N] frozen P2 data, V-cycle precision
  // CUDA graphs of one apply, per (w, y) pair, captured on a private stream
  struct Graph {
    const double* w;
    double* y;
    bool tr;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap = nullptr;
  bool use_graph = true;
  // GMG levels tail_m.. run as one shared-memory kernel (0: off)
  int tail_m = 0;
  size_t tail_smem = 0;
};

namespace {

BoxRaw level0_box(const Hier& H) {
  BoxRaw B;
  const PatchDev& P0 = H.patches[0];
  for (int d = 0; d < 3; d++) B.n[d] = P0.n[d];
  for (int f = 0; f < 6; f++) B.fo[f] = P0.fo[f];
  B.NA = H.N;
  B.cell0 = 0;
  B.gbase = 3L * H.N + P0.goff;
  B.AF = 3L * H.N + H.G;
  return B;
}

template <class P>
BoxV<P> view_of(const BoxRaw& B, const void* A, void* e, const void* f, long vfs) {
  BoxV<P> V;
  for (int d = 0; d < 3; d++) V.n[d] = B.n[d];
  for (int q = 0; q < 6; q++) V.fo[q] = B.fo[q];
  V.A = (const P*)A;
  V.Afs = B.AF;
  V.NA = B.NA;
  V.gbase = B.gbase;
  V.cell0 = B.cell0;
  V.e = (P*)e;
  V.f = (const P*)f;
  V.vfs = vfs;
  return V;
}

template <class P>
void box_smooth(const BoxV<P>& V, int sweeps, bool red_first, cudaStream_t s) {
  long nc = (long)V.n[0] * V.n[1] * V.n[2];
  bool odd = (V.n[0] & 1);
  dim3 grid(g1(odd ? nc : (nc + 1) / 2), 2);
  for (int sw = 0; sw < sweeps; sw++)
    for (int pass = 0; pass < 2; pass++) {
      int colour = red_first ? pass : 1 - pass;
      if (odd) k_box_rbgs_odd<P><<<grid, BS, 0, s>>>(V, colour);
      else k_box_rbgs<P><<<grid, BS, 0, s>>>(V, colour);
    }
}

// ---- the coarse end of the GMG V-cycle in one kernel
// Levels tail_m .. nmg-1 are small (at most 8,192 cells per field): one CTA
// per field copies their coefficients and the rhs of level tail_m into
// shared memory and runs the rest of the V-cycle there (the same smoothing,
// restriction and prolongation arithmetic as the per-level kernels above),
// with block barriers where the per-level form has kernel boundaries.
constexpr int kTailThreads = 1024;
constexpr size_t kTailSmemMax = 200 * 1024;

template <class P>
struct TailArgs {
  int nlev;                       // levels tail_m .. nmg-1
  BoxRaw B[NRD_MAX_MG];
  const P* A[NRD_MAX_MG];         // coefficients (field f at + f * B.AF)
  long offA[NRD_MAX_MG], offE[NRD_MAX_MG], offF[NRD_MAX_MG];   // in elements
  const P* f0;                    // rhs of the first tail level (field stride vfs0)
  P* e0;                          // its correction (output)
  long vfs0;
  int nu1, nu2, csw;
};

template <class P>
__device__ BoxV<P> tail_view(const TailArgs<P>& a, P* sm, int l) {
  BoxV<P> V;
  const BoxRaw& B = a.B[l];
  for (int d = 0; d < 3; d++) V.n[d] = B.n[d];
  for (int q = 0; q < 6; q++) V.fo[q] = B.fo[q];
  V.A = sm + a.offA[l];
  V.Afs = 0;
  V.NA = B.NA;
  V.gbase = B.gbase;
  V.cell0 = 0;
  V.e = sm + a.offE[l];
  V.f = sm + a.offF[l];
  V.vfs = 0;
  return V;
}

template <class P>
__device__ void tail_smooth(const BoxV<P>& V, int sweeps, bool red_first) {
  const long nc = (long)V.n[0] * V.n[1] * V.n[2];
  for (int sw = 0; sw < sweeps; sw++)
    for (int pass = 0; pass < 2; pass++) {
      const int colour = red_first ? pass : 1 - pass;
      for (long c = threadIdx.x; c < nc; c += blockDim.x) {
        int i = (int)(c % V.n[0]);
        long r = c / V.n[0];
        int j = (int)(r % V.n[1]);
        int k = (int)(r / V.n[1]);
        if (((i + j + k) & 1) != colour) continue;
        P dg, of;
        box_row(V, 0, i, j, k, V.e, dg, of);
        V.e[c] = (V.f[c] + of) / dg;
      }
      __syncthreads();
    }
}

template <class P>
__global__ void __launch_bounds__(kTailThreads) k_box_tail(TailArgs<P> a) {
  extern __shared__ __align__(16) unsigned char tail_raw[];
  P* sm = reinterpret_cast<P*>(tail_raw);
  const int fld = blockIdx.x;
  for (int l = 0; l < a.nlev; l++) {
    const BoxRaw& B = a.B[l];
    const P* A = a.A[l] + fld * B.AF;
    for (long q = threadIdx.x; q < B.AF; q += blockDim.x) sm[a.offA[l] + q] = A[q];
    const long nc = (long)B.n[0] * B.n[1] * B.n[2];
    for (long q = threadIdx.x; q < nc; q += blockDim.x) sm[a.offE[l] + q] = P(0);
  }
  {
    const long nc = (long)a.B[0].n[0] * a.B[0].n[1] * a.B[0].n[2];
    for (long q = threadIdx.x; q < nc; q += blockDim.x)
      sm[a.offF[0] + q] = a.f0[fld * a.vfs0 + q];
  }
  __syncthreads();
  // down: smooth, restrict (8-cell average of f - L e)
  for (int l = 0; l + 1 < a.nlev; l++) {
    BoxV<P> V = tail_view(a, sm, l);
    tail_smooth(V, a.nu1, true);
    BoxV<P> C = tail_view(a, sm, l + 1);
    const long ncc = (long)C.n[0] * C.n[1] * C.n[2];
    for (long c = threadIdx.x; c < ncc; c += blockDim.x) {
      int ci = (int)(c % C.n[0]);
      long r = c / C.n[0];
      int cj = (int)(r % C.n[1]), ck = (int)(r / C.n[1]);
      P s = P(0);
      for (int x = 0; x < 2; x++)
        for (int y = 0; y < 2; y++)
          for (int z = 0; z < 2; z++) {
            int i = 2 * ci + x, j = 2 * cj + y, k = 2 * ck + z;
            long q = i + (long)V.n[0] * (j + (long)V.n[1] * k);
            P dg, of;
            box_row(V, 0, i, j, k, V.e, dg, of);
            s += V.f[q] - (dg * V.e[q] - of);
          }
      sm[a.offF[l + 1] + c] = s / P(8);
    }
    __syncthreads();
  }
  tail_smooth(tail_view(a, sm, a.nlev - 1), a.csw, true);
  // up: trilinear prolongation of the coarse correction, smooth
  for (int l = a.nlev - 2; l >= 0; l--) {
    BoxV<P> V = tail_view(a, sm, l);
    const BoxRaw& C = a.B[l + 1];
    const int cn[3] = {C.n[0], C.n[1], C.n[2]};
    const P* src = sm + a.offE[l + 1];
    const long nf = (long)V.n[0] * V.n[1] * V.n[2];
    for (long c = threadIdx.x; c < nf; c += blockDim.x) {
      int q[3];
      q[0] = (int)(c % V.n[0]);
      long r = c / V.n[0];
      q[1] = (int)(r % V.n[1]);
      q[2] = (int)(r / V.n[1]);
      V.e[c] += tri_interp(src, cn, q, (const int*)nullptr, 0);
    }
    __syncthreads();
    tail_smooth(V, a.nu2, false);
  }
  const long nc0 = (long)a.B[0].n[0] * a.B[0].n[1] * a.B[0].n[2];
  for (long q = threadIdx.x; q < nc0; q += blockDim.x) a.e0[fld * a.vfs0 + q] = sm[a.offE[0] + q];
}

template <class P>
void run_tail(PcState* ps, cudaStream_t s) {
  TailArgs<P> a;
  const int m0 = ps->tail_m;
  a.nlev = ps->nmg - m0;
  long off = 0;
  for (int l = 0; l < a.nlev; l++) {
    const BoxRaw& B = ps->box[m0 + l];
    const long nc = (long)B.n[0] * B.n[1] * B.n[2];
    a.B[l] = B;
    a.A[l] = (const P*)ps->bA[m0 + l];
    a.offA[l] = off;
    off += B.AF;
    a.offE[l] = off;
    off += nc;
    a.offF[l] = off;
    off += nc;
  }
  a.f0 = (const P*)ps->bf[m0];
  a.e0 = (P*)ps->be[m0];
  a.vfs0 = (long)ps->box[m0].n[0] * ps->box[m0].n[1] * ps->box[m0].n[2];
  a.nu1 = ps->nu1;
  a.nu2 = ps->nu2;
  a.csw = ps->csw;
  k_box_tail<P><<<2, kTailThreads, ps->tail_smem, s>>>(a);
}

// GMG V-cycle on box level m (m = 0: AMR level 0 inside the hierarchy vectors)
template <class P>
void gmg_vcycle(PcState* ps, const Hier& H, int m, cudaStream_t s) {
  if (m > 0 && m == ps->tail_m) {
    run_tail<P>(ps, s);
    return;
  }
  BoxRaw B = (m == 0) ? level0_box(H) : ps->box[m];
  const void* A = (m == 0) ? ps->A : ps->bA[m];
  void* e = (m == 0) ? ps->fe : ps->be[m];
  const void* f = (m == 0) ? ps->fr : ps->bf[m];
  long vfs = (m == 0) ? H.N : (long)B.n[0] * B.n[1] * B.n[2];
  BoxV<P> V = view_of<P>(B, A, e, f, vfs);
  if (m == ps->nmg - 1) {
    box_smooth(V, ps->csw, true, s);
    return;
  }
  box_smooth(V, ps->nu1, true, s);
  BoxRaw C = ps->box[m + 1];
  long cn = (long)C.n[0] * C.n[1] * C.n[2];
  dim3 gc(g1(cn), 2);
  k_box_restrict<P><<<gc, BS, 0, s>>>(V, (P*)ps->bf[m + 1], cn);
  if (m + 1 != ps->tail_m) cudaMemsetAsync(ps->be[m + 1], 0, 2 * cn * ps->esz, s);
  gmg_vcycle<P>(ps, H, m + 1, s);
  long nf = (long)B.n[0] * B.n[1] * B.n[2];
  dim3 gf(g1(nf), 2);
  k_box_prolong_add<P><<<gf, BS, 0, s>>>((const P*)ps->be[m + 1], cn, C.n[0], C.n[1], C.n[2], V);
  box_smooth(V, ps->nu2, false, s);
}

template <class P>
HierV<P> hview(PcState* ps, const Hier& H) {
  HierV<P> V;
  V.tiles = H.d_tiles;
  V.patches = H.d_patches;
  V.mask = H.d_mask;
  V.gtype = H.d_gtype;
  V.gt0 = H.d_gt0;
  V.gidx = H.d_gidx;
  V.A = (const P*)ps->A;
  V.Afs = ps->AF;
  V.N = H.N;
  V.G = H.G;
  return V;
}

// r = ff - L^c fu, then covered cells := mean of their children
template <class P>
void composite_residual(PcState* ps, const Hier& H, cudaStream_t s) {
  dim3 gg(g1(std::max(H.G, 1)), 2);
  if (H.G) k_lin_ghost<P><<<gg, BS, 0, s>>>(H.d_gtype, H.d_gt0, H.d_gidx, H.d_gw, H.N, H.G,
                                           (const P*)ps->fu, (P*)ps->gh);
  HierV<P> V = hview<P>(ps, H);
  int nt = (int)H.tiles.size();
  dim3 gt(std::min(nt, 152 * 8), 2);
  k_comp_resid<P><<<gt, BS, 0, s>>>(V, nt, H.tile_x, H.tile_y, H.tile_z, (const P*)ps->fu,
                                    (const P*)ps->ff, (const P*)ps->gh, (P*)ps->fr, (P*)ps->cf);
  if (H.nrf) {
    dim3 gr(g1(H.nrf), 2);
    k_comp_reflux<P><<<gr, BS, 0, s>>>(H.d_rf_cell, H.d_rf_off, H.d_rf_g, H.nrf, H.N, H.G,
                                       (const P*)ps->cf, (P*)ps->fr);
  }
  for (int l = H.L - 2; l >= 0; l--) {
    if (!H.ncov[l]) continue;
    dim3 ga(g1(H.ncov[l]), 2);
    k_avgdown_p<P><<<ga, BS, 0, s>>>(H.d_cov[l], H.ncov[l], (P*)ps->fr, H.N);
  }
}

// u^c += P^c_l e^l: add on uncovered level-l cells, then interpolate to every
// finer level
template <class P>
void correct(PcState* ps, const Hier& H, int l, cudaStream_t s) {
  const LevelInfo& Lv = H.lev[l];
  dim3 g(g1(Lv.ncell), 2);
  k_add_leaf<P><<<g, BS, 0, s>>>(H.d_mask, Lv.off, Lv.ncell, H.N, (const P*)ps->fe, (P*)ps->fu);
  const void* src = ps->fe;
  for (int m = l + 1; m < H.L; m++) {
    const LevelInfo& Lm = H.lev[m];
    const LevelInfo& Lc = H.lev[m - 1];
    dim3 gt(std::max(1, std::min(Lm.nt, 152 * 8)), 2);
    k_prolong_level<P><<<gt, BS, 0, s>>>(H.d_tiles, H.d_patches, Lm.t0, Lm.nt, H.tile_x, H.tile_y, H.tile_z,
                                         H.d_mask, H.d_lmap[m - 1], Lc.n[0], Lc.n[1], Lc.n[2], H.N,
                                         (const P*)src, (P*)ps->fp, (P*)ps->fu);
    src = ps->fp;
  }
}

template <class P>
void level_smooth(PcState* ps, const Hier& H, int l, int sweeps, bool red_first, cudaStream_t s) {
  const LevelInfo& Lv = H.lev[l];
  HierV<P> V = hview<P>(ps, H);
  dim3 gt(std::max(1, std::min(Lv.nt, 152 * 8)), 2);
  for (int sw = 0; sw < sweeps; sw++)
    for (int pass = 0; pass < 2; pass++) {
      int colour = red_first ? pass : 1 - pass;
      k_lev_rbgs<P><<<gt, BS, 0, s>>>(V, Lv.t0, Lv.nt, H.tile_x, H.tile_y, H.tile_z, (P*)ps->fe,
                                      (const P*)ps->fr, (const P*)ps->gh, colour);
    }
}

template <class P>
void zero_level(PcState* ps, const Hier& H, int l, cudaStream_t s) {
  const LevelInfo& Lv = H.lev[l];
  for (int f = 0; f < 2; f++)
    cudaMemsetAsync((char*)ps->fe + ((long)f * H.N + Lv.off) * sizeof(P), 0,
                    (size_t)Lv.ncell * sizeof(P), s);
}

// y = P^{-1} w.  With jd non-null (forward only) w and y are bases of
// columns jstride apart and the column *jd (a device index) is used; y2, if
// non-null, receives a second copy of the result.
template <class P>
int apply_t(PcState* ps, const Hier& H, const double* w, double* y, bool transposed,
            cudaStream_t s, const int* jd = nullptr, long jstride = 0, double* y2 = nullptr) {
  const long n2 = 2L * H.N;
  if (transposed)
    k_p2t_cast<P><<<g1(H.N), BS, 0, s>>>(H.N, w, (const P*)ps->p2, (P*)ps->ff);
  else
    k_cast<P><<<g1(n2), BS, 0, s>>>((int)n2, w, (P*)ps->ff, jd, jstride);
  cudaMemsetAsync(ps->fu, 0, n2 * sizeof(P), s);
  // r = f (u = 0); covered := mean of children
  cudaMemcpyAsync(ps->fr, ps->ff, n2 * sizeof(P), cudaMemcpyDeviceToDevice, s);
  for (int l = H.L - 2; l >= 0; l--) {
    if (!H.ncov[l]) continue;
    dim3 ga(g1(H.ncov[l]), 2);
    k_avgdown_p<P><<<ga, BS, 0, s>>>(H.d_cov[l], H.ncov[l], (P*)ps->fr, H.N);
  }
  for (int l = H.L - 1; l >= 1; l--) {
    zero_level<P>(ps, H, l, s);
    level_smooth<P>(ps, H, l, ps->nu1, true, s);
    correct<P>(ps, H, l, s);
    composite_residual<P>(ps, H, s);
  }
  zero_level<P>(ps, H, 0, s);
  gmg_vcycle<P>(ps, H, 0, s);
  correct<P>(ps, H, 0, s);
  for (int l = 1; l < H.L; l++) {
    composite_residual<P>(ps, H, s);
    zero_level<P>(ps, H, l, s);
    level_smooth<P>(ps, H, l, ps->nu2, false, s);
    correct<P>(ps, H, l, s);
  }
  if (transposed)
    k_out_cast<P><<<g1(H.N), BS, 0, s>>>(H.d_mask, H.N, (const P*)ps->fu, y);
  else
    k_p2<P><<<g1(H.N), BS, 0, s>>>(H.N, (const P*)ps->fu, (const P*)ps->p2, y, jd, jstride, y2);
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}

template <class P>
void scale_all(PcState* ps, const Hier& H, SetupArgs& a, cudaStream_t s) {
  int nt = (int)H.tiles.size();
  dim3 gt(std::min(nt, 152 * 8), 2);
  k_scale_hier<P><<<gt, BS, 0, s>>>(a, nullptr, (P*)ps->A);
}

}  // namespace

int pc_alloc(PcState** out, const Hier& H, const nrd_params& p, std::string& err) {
  PcState* ps = new PcState();
  ps->prec = p.pc_precision;
  ps->esz = (ps->prec == NRD_PC_F32) ? 4 : 8;
  ps->nmg = p.nmg;
  ps->nu1 = p.nu1;
  ps->nu2 = p.nu2;
  ps->csw = p.coarse_sweeps;
  const PatchDev& P0 = H.patches[0];
  for (int m = 1; m < ps->nmg; m++)
    for (int d = 0; d < 3; d++)
      if (P0.n[d] % (1 << m) != 0) {
        err = "base box sides must be divisible by 2^(nmg-1)";
        delete ps;
        return NRD_EINVAL;
      }
  const long N = H.N, G = H.G;
  ps->AF = 3 * N + G;
  size_t e = ps->esz;
  bool ok = cudaMalloc(&ps->Craw, 2 * ps->AF * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ps->A, 2 * ps->AF * e) == cudaSuccess &&
            cudaMalloc(&ps->fu, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->fr, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->fe, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->fp, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->ff, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->gh, 2 * std::max(G, 1L) * e) == cudaSuccess &&
            cudaMalloc(&ps->cf, 2 * std::max(G, 1L) * e) == cudaSuccess &&
            cudaMalloc(&ps->Tk, N * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ps->bgt, 6 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&ps->d_beta, sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ps->p2, 3 * N * e) == cudaSuccess &&
            cudaStreamCreateWithFlags(&ps->cap, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) {
    cudaMemset(ps->Craw, 0, 2 * ps->AF * sizeof(double));
    cudaMemset(ps->A, 0, 2 * ps->AF * e);
    cudaMemset(ps->gh, 0, 2 * std::max(G, 1L) * e);
    cudaMemset(ps->cf, 0, 2 * std::max(G, 1L) * e);
    int bt[6];
    for (int f = 0; f < 6; f++) bt[f] = (H.bc_type[f] == NRD_BC_ROBIN) ? 1 : 0;
    cudaMemcpy(ps->bgt, bt, sizeof bt, cudaMemcpyHostToDevice);
  }
  ps->box[0] = level0_box(H);
  for (int m = 1; ok && m < ps->nmg; m++) {
    BoxRaw& B = ps->box[m];
    int fo = 0;
    for (int d = 0; d < 3; d++) B.n[d] = P0.n[d] >> m;
    for (int f = 0; f < 6; f++) {
      int d = f / 2;
      B.fo[f] = fo;
      fo += B.n[(d + 1) % 3] * B.n[(d + 2) % 3];
    }
    long nc = (long)B.n[0] * B.n[1] * B.n[2];
    B.NA = nc;
    B.cell0 = 0;
    B.gbase = 3 * nc;
    B.AF = 3 * nc + fo;
    for (int d = 0; d < 3; d++) ps->bh[m][d] = H.lev[0].h[d] * (double)(1 << m);
    ok = cudaMalloc(&ps->bCraw[m], 2 * B.AF * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&ps->bA[m], 2 * B.AF * e) == cudaSuccess &&
         cudaMalloc(&ps->be[m], 2 * nc * e) == cudaSuccess &&
         cudaMalloc(&ps->bf[m], 2 * nc * e) == cudaSuccess;
    if (ok) {
      cudaMemset(ps->bCraw[m], 0, 2 * B.AF * sizeof(double));
      cudaMemset(ps->bA[m], 0, 2 * B.AF * e);
    }
  }
  if (!ok) {
    pc_free(ps);
    err = "preconditioner allocation failed";
    return NRD_ENOMEM;
  }
  // the coarsest box levels whose data fit one CTA's shared memory run as
  // one kernel (the first such level with at most 8,192 cells per field);
  // FP32 V-cycles only: one SM's FP64 rate is too low for it
  ps->tail_m = 0;
  for (int m = 1; m < ps->nmg && !ps->tail_m && ps->prec == NRD_PC_F32; m++) {
    const long nc = (long)ps->box[m].n[0] * ps->box[m].n[1] * ps->box[m].n[2];
    if (nc > 8192) continue;
    size_t need = 0;
    for (int l = m; l < ps->nmg; l++) {
      const BoxRaw& B = ps->box[l];
      need += (size_t)(B.AF + 2L * B.n[0] * B.n[1] * B.n[2]) * e;
    }
    if (need <= kTailSmemMax) {
      ps->tail_m = m;
      ps->tail_smem = need;
    }
  }
  // (set here, outside any stream capture)
  if (ps->tail_m) {
    cudaFuncSetAttribute(k_box_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kTailSmemMax);
    cudaFuncSetAttribute(k_box_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kTailSmemMax);
  }
  *out = ps;
  return NRD_OK;
}

void pc_drop_graphs(PcState* ps);

void pc_free(PcState* ps) {
  if (!ps) return;
  auto F = [](void* p) { if (p) cudaFree(p); };
  F(ps->Craw); F(ps->A); F(ps->fu); F(ps->fr); F(ps->fe); F(ps->fp); F(ps->ff); F(ps->gh);
  F(ps->cf); F(ps->Tk); F(ps->bgt); F(ps->d_beta); F(ps->p2);
  pc_drop_graphs(ps);
  if (ps->cap) cudaStreamDestroy(ps->cap);
  for (int m = 0; m < NRD_MAX_MG; m++) { F(ps->bCraw[m]); F(ps->bA[m]); F(ps->be[m]); F(ps->bf[m]); }
  delete ps;
}

double* pc_craw(PcState* ps) { return ps->Craw; }

static SetupArgs setup_args(PcState* ps, const Hier& H, const ModelParams* mp, const double* u,
                            const double* gu, const float* z, const float* gz) {
  SetupArgs a;
  a.tiles = H.d_tiles;
  a.patches = H.d_patches;
  a.mask = H.d_mask;
  a.gtype = H.d_gtype;
  a.gface = H.d_gface;
  a.gidx = H.d_gidx;
  a.gt0 = H.d_gt0;
  a.u = u;
  a.gu = gu;
  a.z = z;
  a.gz = gz;
  a.N = H.N;
  a.G = H.G;
  a.ntiles = (int)H.tiles.size();
  a.tx = H.tile_x;
  a.ty = H.tile_y;
  a.tz = H.tile_z;
  a.k = mp ? mp->k : 0.0;
  a.cL = (mp && mp->limiter == NRD_LIM_PAPER_LITERAL) ? 2.0 : 4.0;
  a.beta = ps->beta;
  for (int l = 0; l < NRD_MAX_LEVELS; l++)
    for (int d = 0; d < 3; d++) {
      a.lh.h[l][d] = (l < H.L) ? H.lev[l].h[d] : 1.0;
      a.bh2[l][d] = a.beta / (a.lh.h[l][d] * a.lh.h[l][d]);
    }
  a.Craw = ps->Craw;
  return a;
}

void pc_lin_targets(PcState* ps, float** a32, double** a64, double** p2, float** p2f) {
  *a32 = (ps->prec == NRD_PC_F32) ? (float*)ps->A : nullptr;
  *a64 = (ps->prec == NRD_PC_F32) ? nullptr : (double*)ps->A;
  *p2 = (ps->prec == NRD_PC_F32) ? nullptr : (double*)ps->p2;
  *p2f = (ps->prec == NRD_PC_F32) ? (float*)ps->p2 : nullptr;
}

int pc_finish(PcState* ps, const Hier& H, const double* u, const float* z, double a0, double dt,
              bool from_lin, cudaStream_t s, bool beta_on_device) {
  ps->beta = dt / a0;
  if (ps->z != z) pc_drop_graphs(ps);
  ps->z = z;
  // beta = dt / a0 for the set-up kernels; a graph-captured solve writes it
  // to the device itself before the launch
  if (!beta_on_device)
    cudaMemcpyAsync(ps->d_beta, &ps->beta, sizeof(double), cudaMemcpyHostToDevice, s);
  SetupArgs a = setup_args(ps, H, nullptr, u, nullptr, z, nullptr);
  if (!from_lin) {
    cudaMemcpyAsync(ps->Tk, u + H.N, (size_t)H.N * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (ps->prec == NRD_PC_F32)
      k_p2_setup<float><<<g1(H.N), BS, 0, s>>>(H.d_mask, H.N, ps->Tk, z, ps->d_beta,
                                               (float*)ps->p2);
    else
      k_p2_setup<double><<<g1(H.N), BS, 0, s>>>(H.d_mask, H.N, ps->Tk, z, ps->d_beta,
                                                (double*)ps->p2);
  }
  for (int l = H.L - 2; l >= 0; l--) {
    if (!H.ncz[l]) continue;
    dim3 g(g1(H.ncz[l]), 2);
    if (from_lin && ps->prec == NRD_PC_F32)
      k_coef_coarsen<float><<<g, BS, 0, s>>>(H.d_cz_tgt[l], H.d_cz_src[l], H.ncz[l], ps->AF, H.N,
                                             H.d_gtype, H.d_gface, ps->d_beta, a.lh, l, ps->Craw,
                                             (float*)ps->A);
    else if (from_lin)
      k_coef_coarsen<double><<<g, BS, 0, s>>>(H.d_cz_tgt[l], H.d_cz_src[l], H.ncz[l], ps->AF, H.N,
                                              H.d_gtype, H.d_gface, ps->d_beta, a.lh, l, ps->Craw,
                                              (double*)ps->A);
    else
      k_coef_coarsen<float><<<g, BS, 0, s>>>(H.d_cz_tgt[l], H.d_cz_src[l], H.ncz[l], ps->AF, H.N,
                                             H.d_gtype, H.d_gface, ps->d_beta, a.lh, l, ps->Craw,
                                             (float*)nullptr);
  }
  // GMG levels
  for (int m = 1; m < ps->nmg; m++) {
    const BoxRaw& F = (m == 1) ? ps->box[0] : ps->box[m - 1];
    const double* Cf = (m == 1) ? ps->Craw : ps->bCraw[m - 1];
    const BoxRaw& C = ps->box[m];
    long nc = (long)C.n[0] * C.n[1] * C.n[2];
    dim3 g(g1(nc), 2);
    const double* hb = ps->bh[m];
    const double r2[3] = {1.0 / (hb[0] * hb[0]), 1.0 / (hb[1] * hb[1]), 1.0 / (hb[2] * hb[2])};
    if (ps->prec == NRD_PC_F32)
      k_box_coarsen<float><<<g, BS, 0, s>>>(F, Cf, C, ps->bCraw[m], ps->bgt, ps->d_beta, hb[0],
                                            hb[1], hb[2], r2[0], r2[1], r2[2],
                                            (float*)ps->bA[m]);
    else
      k_box_coarsen<double><<<g, BS, 0, s>>>(F, Cf, C, ps->bCraw[m], ps->bgt, ps->d_beta, hb[0],
                                             hb[1], hb[2], r2[0], r2[1], r2[2],
                                             (double*)ps->bA[m]);
  }
  if (!from_lin) {
    if (ps->prec == NRD_PC_F32) scale_all<float>(ps, H, a, s);
    else scale_all<double>(ps, H, a, s);
  }
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}

int pc_setup(PcState* ps, const Hier& H, const ModelParams& mp, const double* u, const double* gu,
             const float* z, const float* gz, double a0, double dt, cudaStream_t s) {
  ps->beta = dt / a0;
  SetupArgs a = setup_args(ps, H, &mp, u, gu, z, gz);
  int nt = (int)H.tiles.size();
  k_coef<<<std::min(nt, 152 * 8), BS, 0, s>>>(a);
  return pc_finish(ps, H, u, z, a0, dt, false, s);
}

int pc_apply_indexed(PcState* ps, const Hier& H, const double* V, double* Z, const int* jd,
                     long jstride, double* zcopy, cudaStream_t s) {
  if (ps->prec == NRD_PC_F32)
    return apply_t<float>(ps, H, V, Z, false, s, jd, jstride, zcopy);
  return apply_t<double>(ps, H, V, Z, false, s, jd, jstride, zcopy);
}

double* pc_beta_device(PcState* ps) { return ps->d_beta; }

static int apply_any(PcState* ps, const Hier& H, const double* w, double* y, bool tr,
                     cudaStream_t s) {
  if (ps->prec == NRD_PC_F32) return apply_t<float>(ps, H, w, y, tr, s);
  return apply_t<double>(ps, H, w, y, tr, s);
}

void pc_drop_graphs(PcState* ps) {
  for (auto& g : ps->graphs) cudaGraphExecDestroy(g.exec);
  ps->graphs.clear();
}

void pc_set_sweeps(PcState* ps, int nu1, int nu2, int csw) {
  if (ps->nu1 != nu1 || ps->nu2 != nu2 || ps->csw != csw) pc_drop_graphs(ps);
  ps->nu1 = nu1;
  ps->nu2 = nu2;
  ps->csw = csw;
}

// One apply is a fixed sequence of about a hundred small launches; it is
// captured once per (w, y) pair into a CUDA graph and replayed.  Everything
// the launches read besides w is at fixed addresses (beta in device memory).
int pc_apply(PcState* ps, const Hier& H, const double* w, double* y, cudaStream_t s) {
  return pc_apply_ex(ps, H, w, y, false, s);
}

// transposed: P^{-T} = P1^{-T} P2^{-T}, with one V-cycle for P1^{-T} (the
// red-black V-cycle with reversed post-smoothing is used as is)
int pc_apply_ex(PcState* ps, const Hier& H, const double* w, double* y, bool tr, cudaStream_t s) {
  if (!ps->use_graph) return apply_any(ps, H, w, y, tr, s);
  cudaGraphExec_t exec = nullptr;
  for (auto& g : ps->graphs)
    if (g.w == w && g.y == y && g.tr == tr) { exec = g.exec; break; }
  if (!exec) {
    if (ps->graphs.size() >= 64) pc_drop_graphs(ps);
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(ps->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return NRD_ECUDA;
    int rc = apply_any(ps, H, w, y, tr, ps->cap);
    cudaError_t e = cudaStreamEndCapture(ps->cap, &graph);
    if (rc != NRD_OK || e != cudaSuccess) return NRD_ECUDA;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return NRD_ECUDA;
    ps->graphs.push_back({w, y, tr, exec});
  }
  return cudaGraphLaunch(exec, s) == cudaSuccess ? NRD_OK : NRD_ECUDA;
}
