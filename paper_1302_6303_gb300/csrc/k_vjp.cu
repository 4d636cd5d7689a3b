// Transposed Jacobian of the residual (the adjoint / vector-Jacobian
// product), at the state of the last linearisation.  Gather form, no atomics,
// deterministic:
//   1. face adjoints   lambda_f = sum over the cells whose balance uses face f
//                      of (+-1/h) w_cell, including the coarse cell of a
//                      coarse-fine face through flux matching (1/4 of the fine
//                      face, on the coarse side);
//   2. ghost adjoints  gamma_g = the ghost side's flux partials times lambda;
//   3. cell gather     (J^T w)_c = a0 w_c - dt (sum of the cell's own face
//                      partials times lambda + the ghost adjoints of every
//                      ghost that reads c, with the ghost's stencil weight +
//                      coupling partials), and the same for d/dz.
#include <algorithm>

#include "nrd_internal.h"

namespace {

struct VjpArgs {
  const TileDev* tiles;
  const PatchDev* patches;
  const uint8_t* mask;
  const uint8_t* gtype;
  const uint8_t* gface;
  const int* gcell;
  const int* gzsrc;
  const int* ts_off;   // transposed ghost stencil: cell -> (ghost, weight)
  const int* ts_g;
  const double* ts_w;
  const int* tz_off;   // ghosts taking their z from a cell
  const int* tz_g;
  const double* jc;    // [6][NS] face partials (5: d Phi_E / d z^3)
  const double* cc;    // [3][N] coupling partials (2: d coupling / d z^3)
  const float* z;
  const double* w;     // [2][N]
  double* lam;         // [2][NS]
  double* gam;         // [3][G]
  double* out;         // [2][N]
  double* dz;          // [N] or null
  double a0, dt;
  int N, G, ntiles, tx, ty, tz;
  double rh[NRD_MAX_LEVELS][3];
};

__device__ __forceinline__ bool leaf(const uint8_t* mask, int c) {
  return !(mask[c] & MASK_COVERED);
}

// 1. face adjoints of the low faces and boundary faces of every cell
__global__ void k_vjp_faces(VjpArgs a) {
  const int N = a.N, G = a.G;
  const long NS = 3L * N + G;
  const int nc = a.tx * a.ty * a.tz;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const TileDev tile = a.tiles[t];
    const PatchDev P = a.patches[tile.patch];
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int i = tile.i0 + c % a.tx, j = tile.j0 + (c / a.tx) % a.ty, k = tile.k0 + c / (a.tx * a.ty);
      if (i >= nx || j >= ny || k >= tile.k1) continue;
      const int idx = P.off + i + nx * (j + ny * k);
      const int loc[3] = {i, j, k};
      const int st[3] = {1, nx, nx * ny};
      const uint8_t m = a.mask[idx];
      const bool lf = leaf(a.mask, idx);
      const double wE = a.w[idx], wT = a.w[N + idx];
      for (int d = 0; d < 3; d++) {
        const double rh = a.rh[P.level][d];
        if (loc[d] > 0) {
          // interior face between a = idx - st (low) and b = idx (high)
          const int ia = idx - st[d];
          const uint8_t ma = a.mask[ia];
          double lE = 0.0, lT = 0.0;
          if (leaf(a.mask, ia) && !(ma & (2 << (2 * d + 1)))) {
            lE += a.w[ia] * rh;
            lT += a.w[N + ia] * rh;
          }
          if (lf && !(m & (2 << (2 * d)))) {
            lE -= wE * rh;
            lT -= wT * rh;
          }
          const long slot = (long)d * N + idx;
          a.lam[slot] = lE;
          a.lam[NS + slot] = lT;
        }
        for (int sd = 0; sd < 2; sd++) {
          const bool at = sd ? (loc[d] == P.n[d] - 1) : (loc[d] == 0);
          if (!at) continue;
          const int f = 2 * d + sd;
          const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          const int g = P.goff + P.fo[f] + loc[t1] + P.n[t1] * loc[t2];
          const uint8_t ty = a.gtype[g];
          const long slot = 3L * N + g;
          double lE = 0.0, lT = 0.0;
          if (ty != GT_NEUMANN && lf && !(m & (2 << f))) {
            // this cell is the low side of its high face (sd = 1), the high
            // side of its low face (sd = 0)
            const double sg = sd ? 1.0 : -1.0;
            lE += sg * wE * rh;
            lT += sg * wT * rh;
            if (ty == GT_CF) {
              // the coarse cell across the face takes 1/4 of this fine flux
              const int C = a.gzsrc[g];
              const double rhc = a.rh[P.level - 1][d];
              lE -= sg * 0.25 * a.w[C] * rhc;
              lT -= sg * 0.25 * a.w[N + C] * rhc;
            }
          }
          a.lam[slot] = lE;
          a.lam[NS + slot] = lT;
        }
      }
    }
  }
}

// 2. ghost adjoints: the ghost side's partials times the face adjoint
__global__ void k_vjp_ghosts(VjpArgs a) {
  const int N = a.N, G = a.G;
  const long NS = 3L * N + G;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const uint8_t ty = a.gtype[g];
    double gE = 0.0, gT = 0.0, gZ = 0.0;
    if (ty == GT_SIBLING || ty == GT_CF) {
      const long slot = 3L * N + g;
      const bool hi = (a.gface[g] & 7) % 2;   // ghost on the high side of the face
      const double lE = a.lam[slot], lT = a.lam[NS + slot];
      gE = (hi ? a.jc[NS + slot] : a.jc[slot]) * lE;
      gT = a.jc[2 * NS + slot] * lE + (hi ? a.jc[4 * NS + slot] : a.jc[3 * NS + slot]) * lT;
      gZ = a.jc[5 * NS + slot] * lE;
    }
    a.gam[g] = gE;
    a.gam[G + g] = gT;
    a.gam[2L * G + g] = gZ;
  }
}

// 3. per-cell gather
__global__ void k_vjp_cells(VjpArgs a) {
  const int N = a.N, G = a.G;
  const long NS = 3L * N + G;
  const int nc = a.tx * a.ty * a.tz;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const TileDev tile = a.tiles[t];
    const PatchDev P = a.patches[tile.patch];
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      int i = tile.i0 + c % a.tx, j = tile.j0 + (c / a.tx) % a.ty, k = tile.k0 + c / (a.tx * a.ty);
      if (i >= nx || j >= ny || k >= tile.k1) continue;
      const int idx = P.off + i + nx * (j + ny * k);
      const uint8_t m = a.mask[idx];
      if (m & MASK_COVERED) {
        a.out[idx] = 0.0;
        a.out[N + idx] = 0.0;
        if (a.dz) a.dz[idx] = 0.0;
        continue;
      }
      const int loc[3] = {i, j, k};
      const int st[3] = {1, nx, nx * ny};
      double accE = 0.0, accT = 0.0, accZ = 0.0;
      for (int d = 0; d < 3; d++) {
        for (int sd = 0; sd < 2; sd++) {
          const int f = 2 * d + sd;
          if (m & (2 << f)) continue;                      // flux matching face
          const bool bnd = sd ? (loc[d] == P.n[d] - 1) : (loc[d] == 0);
          long slot;
          uint8_t ty = GT_SIBLING;
          if (!bnd) {
            slot = (long)d * N + (sd ? idx + st[d] : idx);
          } else {
            const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            const int g = P.goff + P.fo[f] + loc[t1] + P.n[t1] * loc[t2];
            ty = a.gtype[g];
            slot = 3L * N + g;
          }
          if (ty == GT_NEUMANN) continue;
          const double lE = a.lam[slot], lT = a.lam[NS + slot];
          if (ty == GT_ROBIN) {
            accE += a.jc[slot] * lE;
            accT += a.jc[NS + slot] * lE;
            accZ += a.jc[5 * NS + slot] * lE;
            continue;
          }
          // this cell is the low side ('a') of its high face, 'b' of its low face
          accE += (sd ? a.jc[slot] : a.jc[NS + slot]) * lE;
          accT += a.jc[2 * NS + slot] * lE + (sd ? a.jc[3 * NS + slot] : a.jc[4 * NS + slot]) * lT;
          accZ += a.jc[5 * NS + slot] * lE;
        }
      }
      // ghosts that read this cell (sibling copies, coarse-fine stencils)
      for (int q = a.ts_off[idx]; q < a.ts_off[idx + 1]; q++) {
        const int g = a.ts_g[q];
        const double wq = a.ts_w[q];
        accE += wq * a.gam[g];
        accT += wq * a.gam[G + g];
      }
      const double wE = a.w[idx], wT = a.w[N + idx];
      const double dw = wE - wT;
      a.out[idx] = a.a0 * wE - a.dt * (accE + a.cc[idx] * dw);
      a.out[N + idx] = a.a0 * wT - a.dt * (accT + a.cc[N + idx] * dw);
      if (a.dz) {
        for (int q = a.tz_off[idx]; q < a.tz_off[idx + 1]; q++) accZ += a.gam[2L * G + a.tz_g[q]];
        const double zc = (double)a.z[idx];
        a.dz[idx] = -a.dt * 3.0 * zc * zc * (accZ + a.cc[2L * N + idx] * dw);
      }
    }
  }
}

}  // namespace

void launch_vjp(const Hier& H, const double* jc, const double* cc, const float* z, const double* w,
                double* lam, double* gam, double a0, double dt, double* out, double* dz,
                cudaStream_t s) {
  VjpArgs a;
  a.tiles = H.d_tiles;
  a.patches = H.d_patches;
  a.mask = H.d_mask;
  a.gtype = H.d_gtype;
  a.gface = H.d_gface;
  a.gcell = H.d_gcell;
  a.gzsrc = H.d_gzsrc;
  a.ts_off = H.d_ts_off;
  a.ts_g = H.d_ts_g;
  a.ts_w = H.d_ts_w;
  a.tz_off = H.d_tz_off;
  a.tz_g = H.d_tz_g;
  a.jc = jc;
  a.cc = cc;
  a.z = z;
  a.w = w;
  a.lam = lam;
  a.gam = gam;
  a.out = out;
  a.dz = dz;
  a.a0 = a0;
  a.dt = dt;
  a.N = H.N;
  a.G = H.G;
  a.ntiles = (int)H.tiles.size();
  a.tx = H.tile_x;
  a.ty = H.tile_y;
  a.tz = H.tile_z;
  for (int l = 0; l < NRD_MAX_LEVELS; l++)
    for (int d = 0; d < 3; d++) a.rh[l][d] = (l < H.L) ? 1.0 / H.lev[l].h[d] : 1.0;
  const int nt = std::max(1, (int)H.tiles.size());
  k_vjp_faces<<<nt, 256, 0, s>>>(a);
  int gb = (int)std::min(152L * 8, (H.G + 255L) / 256);
  k_vjp_ghosts<<<std::max(gb, 1), 256, 0, s>>>(a);
  k_vjp_cells<<<nt, 256, 0, s>>>(a);
}
