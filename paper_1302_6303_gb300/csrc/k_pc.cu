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

#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "nrd_internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int BS = 256;

int g1(long n) {
  long b = (n + BS - 1) / BS;
  return (int)std::max(1L, std::min(b, 152L * 16));
}

struct LevelHP {
  double h[NRD_MAX_LEVELS][3];
  double r2[NRD_MAX_LEVELS][3];   // 1 / h^2
};

// ---------------------------------------------------------------- V-cycle
// All apply kernels work on 8x8x8 tiles (ragged at patch and box edges):
// one tile per block of 256 threads, so every in-tile coordinate is a shift
// or a mask and every index is 32-bit (pc_alloc rejects hierarchies whose
// coefficient slots exceed 2^31).  Red-black passes give each thread one
// x-pair of cells, exactly one of which has the pass colour.
constexpr int VT = 8;
constexpr int VTHREADS = 256;
constexpr int kTilePatch = 0x3fffffff;
constexpr int kTileCovered = 1 << 30;

// thread -> x-pair of a red-black pass: pair (t & 3), row (t >> 2) & 7,
// plane t >> 5
__device__ __forceinline__ int rb_px(int t) { return 2 * (t & 3); }
__device__ __forceinline__ int rb_j(int t) { return (t >> 2) & 7; }
__device__ __forceinline__ int rb_k(int t) { return t >> 5; }
// thread -> cell of a full-tile sweep (512 threads): x (t & 7), row
// (t >> 3) & 7, plane t >> 6
constexpr int FTHREADS = 512;
__device__ __forceinline__ int ft_i(int t) { return t & 7; }
__device__ __forceinline__ int ft_j(int t) { return (t >> 3) & 7; }
__device__ __forceinline__ int ft_k(int t) { return t >> 6; }

// ---- box levels (level 0 inside the hierarchy vectors, and the GMG boxes)
template <class P>
struct BoxK {
  int n0, n1, n2;
  int fo[6];      // boundary slot offset of each face, relative to gbase
  const P* A;     // coefficients of field 0; field f at A + f * Afs
  long Afs;
  int NA;         // stride of the low-face blocks
  int gbase;      // index of the first boundary slot
  P* e;           // correction, field f at e + f * vfs
  const P* f;     // right-hand side
  long vfs;
};

// diagonal and off-diagonal sum of row (i, j, k) of I - beta div D grad on a
// box (all box faces physical); ZERO: the neighbours are 0
template <class P, bool ZERO>
__device__ __forceinline__ void box_row(const BoxK<P>& B, const P* A, const P* e, int i, int j,
                                        int k, P& dg, P& of) {
  const int n0 = B.n0, n1 = B.n1, n2 = B.n2;
  const int idx = i + n0 * (j + n1 * k);
  const int s2 = n0 * n1;
  P d = P(1), o = P(0), a;
  if (i > 0) { a = A[idx]; d += a; if (!ZERO) o += a * e[idx - 1]; }
  else d += A[B.gbase + B.fo[0] + j + n1 * k];
  if (i < n0 - 1) { a = A[idx + 1]; d += a; if (!ZERO) o += a * e[idx + 1]; }
  else d += A[B.gbase + B.fo[1] + j + n1 * k];
  if (j > 0) { a = A[B.NA + idx]; d += a; if (!ZERO) o += a * e[idx - n0]; }
  else d += A[B.gbase + B.fo[2] + k + n2 * i];
  if (j < n1 - 1) { a = A[B.NA + idx + n0]; d += a; if (!ZERO) o += a * e[idx + n0]; }
  else d += A[B.gbase + B.fo[3] + k + n2 * i];
  if (k > 0) { a = A[2 * B.NA + idx]; d += a; if (!ZERO) o += a * e[idx - s2]; }
  else d += A[B.gbase + B.fo[4] + i + n0 * j];
  if (k < n2 - 1) { a = A[2 * B.NA + idx + s2]; d += a; if (!ZERO) o += a * e[idx + s2]; }
  else d += A[B.gbase + B.fo[5] + i + n0 * j];
  dg = d;
  of = o;
}

// one colour of a red-black Gauss-Seidel pass on a box; grid (tiles x,
// tiles y, 2 x tiles z), the upper half of z for field 1.
// ZERO: the correction starts from 0 (the pass writes 0 to the other colour);
// ADD:  last pass of the level: u += e on both cells of the pair where the
//       cell is not covered (level 0 inside the hierarchy vectors)
template <class P, bool ZERO, bool ADD>
__global__ void __launch_bounds__(VTHREADS) k_bsmooth(BoxK<P> B, int colour, const uint8_t* mask,
                                                       P* u) {
  const int ntz = gridDim.z >> 1;
  const int fld = blockIdx.z >= ntz;
  const int t = threadIdx.x;
  const int j = blockIdx.y * VT + rb_j(t), k = (blockIdx.z - fld * ntz) * VT + rb_k(t);
  if (j >= B.n1 || k >= B.n2) return;
  const int ib = blockIdx.x * VT + rb_px(t);
  const int par = (j + k + colour) & 1;          // box cells: colour = parity of i + j + k
  const int i = ib + par, ip = ib + 1 - par;     // this colour, the other one
  P* e = B.e + fld * B.vfs;
  const P* A = B.A + fld * B.Afs;
  const int row = B.n0 * (j + B.n1 * k);
  P ev = P(0);
  if (i < B.n0) {
    P dg, of;
    box_row<P, ZERO>(B, A, e, i, j, k, dg, of);
    ev = (B.f[fld * B.vfs + row + i] + of) / dg;
    e[row + i] = ev;
    if (ADD && !(mask[row + i] & MASK_COVERED)) u[fld * B.vfs + row + i] += ev;
  }
  if (ip < B.n0) {
    if (ZERO) e[row + ip] = P(0);
    if (ADD && !(mask[row + ip] & MASK_COVERED)) u[fld * B.vfs + row + ip] += e[row + ip];
  }
}

// ---- one red-black Gauss-Seidel sweep on a box, both colours in one launch
// (FP32 boxes whose arrays TMA can address).  The sweep reads the correction
// es (or zero) and writes ed (ed != es): first every cell of colour c0 from
// the old values of its neighbours (which have the other colour), then every
// cell of colour 1 - c0 from the new ones, as two colour passes of
// k_bsmooth do (the division as a multiplication by the reciprocal of the
// diagonal, which is at least 1).  A CTA owns a 32 x 8 x 4 tile.  One thread
// starts five TMA box loads into shared memory: the old correction over the
// tile and a two-cell ring, and the rhs and the three low-face coefficient
// arrays over the tile and a one-cell ring (plus the high faces of the
// ring); all threads wait on one mbarrier (bounded: a wait that runs out
// sets err and the CTA stops after a second bounded wait for its copies).
// Then the first colour is updated on the tile and the ring (the values the
// tile's second colour reads), the second colour on the tile, and the tile
// is written.  Nothing another CTA writes is read (es and ed differ), so
// tiles are independent; the ring loads of neighbouring tiles mostly hit
// L2.  A sweep thus moves the coefficients, the rhs and es from DRAM about
// once and writes ed once, where two colour passes move them twice.
// The boxes start 4 cells before the tile in x (TMA wants the innermost
// coordinate at a 16-byte boundary) and are 40 wide; cells outside the
// array read as zero and are never used (domain faces take the boundary
// slot coefficient, read from global memory).
// ZERO: es = 0 (the first sweep of a level; no load).  ADD: u += ed on
// uncovered cells (the last sweep on level 0, in the hierarchy vectors).
constexpr int SX = 32, SY = 8, SZ = 4;
constexpr int SW_THREADS = SX * SY;                          // one tile column per thread
constexpr int TBX = 40;                                      // box width in x (from x0 - 4)
constexpr int EBY = SY + 4, EBZ = SZ + 4;                    // correction box: two-cell ring
constexpr int FBY = SY + 2, FBZ = SZ + 2;                    // rhs / coefficient boxes
constexpr int E_BYTES = TBX * EBY * EBZ * 4;                 // correction
constexpr int F_BYTES = TBX * FBY * FBZ * 4;                 // rhs, x faces
constexpr int AY_BYTES = TBX * (FBY + 1) * FBZ * 4;          // y faces (one more row)
constexpr int AZ_BYTES = TBX * FBY * (FBZ + 1) * 4;          // z faces (one more plane)
constexpr int up128(int b) { return (b + 127) / 128 * 128; }
constexpr int OFF_F = up128(E_BYTES);
constexpr int OFF_AX = OFF_F + up128(F_BYTES);
constexpr int OFF_AY = OFF_AX + up128(F_BYTES);
constexpr int OFF_AZ = OFF_AY + up128(AY_BYTES);
constexpr int STAGE_BYTES = OFF_AZ + up128(AZ_BYTES);      // one tile's boxes
constexpr int SWEEP_SMEM = STAGE_BYTES + 16;                // the boxes + the mbarrier
constexpr long kTmaSpinLimit = 1L << 20;   // polls of mbarrier.try_wait

struct SweepMaps {                 // per field: old correction, rhs, x/y/z low faces
  CUtensorMap es[2], f[2], ax[2], ay[2], az[2];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                          int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];"
      :
      : "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// wait for the phase of the given parity of the mbarrier to complete, at
// most kTmaSpinLimit polls; false if the wait ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < kTmaSpinLimit; it++) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// row (i, j, k) of I - beta div D grad with the six face coefficients and
// neighbour values given; domain faces take the boundary slot (the same
// operations in the same order as box_row)
__device__ __forceinline__ void box_row_s(const BoxK<float>& B, const float* A, int i, int j,
                                          int k, float axl, float axh, float ayl, float ayh,
                                          float azl, float azh, float xm, float xp, float ym,
                                          float yp, float zm, float zp, float& dg, float& of) {
  const int n0 = B.n0, n1 = B.n1, n2 = B.n2;
  float d = 1.0f, o = 0.0f;
  if (i > 0) { d += axl; o += axl * xm; }
  else d += A[B.gbase + B.fo[0] + j + n1 * k];
  if (i < n0 - 1) { d += axh; o += axh * xp; }
  else d += A[B.gbase + B.fo[1] + j + n1 * k];
  if (j > 0) { d += ayl; o += ayl * ym; }
  else d += A[B.gbase + B.fo[2] + k + n2 * i];
  if (j < n1 - 1) { d += ayh; o += ayh * yp; }
  else d += A[B.gbase + B.fo[3] + k + n2 * i];
  if (k > 0) { d += azl; o += azl * zm; }
  else d += A[B.gbase + B.fo[4] + i + n0 * j];
  if (k < n2 - 1) { d += azh; o += azh * zp; }
  else d += A[B.gbase + B.fo[5] + i + n0 * j];
  dg = d;
  of = o;
}

constexpr int EPL = EBY * TBX;          // plane strides of the boxes in shared memory
constexpr int FPL = FBY * TBX;
constexpr int YPL = (FBY + 1) * TBX;

// one Gauss-Seidel update of cell (i, j, k) from the shared boxes: oe its
// offset in the correction box, of in the rhs / x-face / z-face boxes, oy in
// the y-face box.  CHECK: the cell may lie on a domain face (box_row_s);
// else all six neighbours are in the box (the same operations in the same
// order).  ZERO: the neighbours' old values are zero.
template <bool CHECK, bool ZERO>
__device__ __forceinline__ void rb_update(const BoxK<float>& B, const float* A, float* Se,
                                          const float* Sf, const float* Sx, const float* Sy,
                                          const float* Sz, int oe, int of, int oy, int i, int j,
                                          int k) {
  const float axl = Sx[of], axh = Sx[of + 1], ayl = Sy[oy], ayh = Sy[oy + TBX];
  const float azl = Sz[of], azh = Sz[of + FPL];
  float xm = 0.0f, xp = 0.0f, ym = 0.0f, yp = 0.0f, zm = 0.0f, zp = 0.0f;
  if (!ZERO) {
    xm = Se[oe - 1];
    xp = Se[oe + 1];
    ym = Se[oe - TBX];
    yp = Se[oe + TBX];
    zm = Se[oe - EPL];
    zp = Se[oe + EPL];
  }
  float dg, o;
  if (CHECK) {
    box_row_s(B, A, i, j, k, axl, axh, ayl, ayh, azl, azh, xm, xp, ym, yp, zm, zp, dg, o);
  } else {
    float d = 1.0f;
    o = 0.0f;
    d += axl; o += axl * xm;
    d += axh; o += axh * xp;
    d += ayl; o += ayl * ym;
    d += ayh; o += ayh * yp;
    d += azl; o += azl * zm;
    d += azh; o += azh * zp;
    dg = d;
  }
  Se[oe] = __fdividef(Sf[of] + o, dg);
}

// Grid (ntx, nty, 2 ntz), one tile per CTA, the upper half of z for field 1;
// SWEEP_SMEM bytes of dynamic shared memory, four CTAs per SM (some compute
// while the others' loads land).  The tile origin is even on every axis, so
// the colour of the cell at (x, y, z) in the one-ring frame (origin one cell
// before the tile) is (x + y + z + 1) mod 2.
// ADD stores the correction into u: on level 0's uncovered cells the
// composite solution is still zero when level 0 is corrected (the finer
// levels' corrections touch only their own cells), so u += e there is u = e.
template <bool ZERO, bool ADD>
__global__ void __launch_bounds__(SW_THREADS, 4) k_bsweep(const __grid_constant__ SweepMaps M,
                                                           BoxK<float> B, int c0,
                                                           float* __restrict__ ed,
                                                           const uint8_t* __restrict__ mask,
                                                           float* __restrict__ u,
                                                           int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t bar = smem_u32(smem + STAGE_BYTES);
  const int t = threadIdx.x;
  const int n0 = B.n0, n1 = B.n1, n2 = B.n2;
  const int ntz = gridDim.z >> 1;
  const int fld = blockIdx.z >= ntz;
  const int x0 = blockIdx.x * SX, y0 = blockIdx.y * SY, z0 = (blockIdx.z - fld * ntz) * SZ;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint32_t bytes = (ZERO ? 0 : E_BYTES) + 2 * F_BYTES + AY_BYTES + AZ_BYTES;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    if (!ZERO) tma_load3(smem_u32(smem), &M.es[fld], x0 - 4, y0 - 2, z0 - 2, bar);
    tma_load3(smem_u32(smem + OFF_F), &M.f[fld], x0 - 4, y0 - 1, z0 - 1, bar);
    tma_load3(smem_u32(smem + OFF_AX), &M.ax[fld], x0 - 4, y0 - 1, z0 - 1, bar);
    tma_load3(smem_u32(smem + OFF_AY), &M.ay[fld], x0 - 4, y0 - 1, z0 - 1, bar);
    tma_load3(smem_u32(smem + OFF_AZ), &M.az[fld], x0 - 4, y0 - 1, z0 - 1, bar);
  }
  // thread -> cells (tile origins are even, so this is the same for every
  // tile): first colour: columns t and t + SW_THREADS of the 34 x 10 ring
  // frame, all planes, those of the colour every other plane; second colour
  // and write: column (x2, y2) = t of the tile, all planes
  const int x2 = t & (SX - 1), y2 = t / SX;
  const int z2s = (c0 + 1 + x2 + y2) & 1;
  const int oe2 = 2 * EPL + (y2 + 2) * TBX + x2 + 4, of2 = FPL + (y2 + 1) * TBX + x2 + 4,
            oy2 = YPL + (y2 + 1) * TBX + x2 + 4;
  // everyone waits for the loads (the barrier's first phase); bounded
  __syncthreads();
  const bool late = !mbar_wait(bar, 0);
  if (__syncthreads_or(late)) {
    // the copies did not land in time: report, give them a second bounded
    // wait (they write this CTA's shared memory), and stop
    if (t == 0) atomicOr(err, 2);
    mbar_wait(bar, 0);
    return;
  }
  float* Se = reinterpret_cast<float*>(smem);
  const float* Sf = reinterpret_cast<const float*>(smem + OFF_F);
  const float* Sx = reinterpret_cast<const float*>(smem + OFF_AX);
  const float* Sy = reinterpret_cast<const float*>(smem + OFF_AY);
  const float* Sz = reinterpret_cast<const float*>(smem + OFF_AZ);
  const float* A = B.A + fld * B.Afs;
  // tiles whose cells and ring all have six in-box neighbours skip the
  // boundary tests
  const bool inner = x0 >= 2 && x0 + SX + 1 < n0 && y0 >= 2 && y0 + SY + 1 < n1 && z0 >= 2 &&
                     z0 + SZ + 1 < n2;
  // first colour on the tile and the one-cell ring
  for (int c = t; c < FBY * (SX + 2); c += SW_THREADS) {
    const int x1 = c % (SX + 2), y1 = c / (SX + 2);
    const int z1s = (c0 + 1 + x1 + y1) & 1;
    const int oe1 = EPL + (y1 + 1) * TBX + x1 + 3, of1 = y1 * TBX + x1 + 3;
    const int i = x0 - 1 + x1, j = y0 - 1 + y1;
    if (inner) {
#pragma unroll
      for (int zz = 0; zz < FBZ; zz += 2) {
        const int z = z1s + zz;
        rb_update<false, ZERO>(B, A, Se, Sf, Sx, Sy, Sz, oe1 + z * EPL, of1 + z * FPL,
                               of1 + z * YPL, i, j, z0 - 1 + z);
      }
    } else if (i >= 0 && i < n0 && j >= 0 && j < n1) {
      for (int z = z1s; z < FBZ; z += 2) {
        const int k = z0 - 1 + z;
        if (k >= 0 && k < n2)
          rb_update<true, ZERO>(B, A, Se, Sf, Sx, Sy, Sz, oe1 + z * EPL, of1 + z * FPL,
                                of1 + z * YPL, i, j, k);
      }
    }
  }
  __syncthreads();
  // second colour on the tile
  {
    const int i = x0 + x2, j = y0 + y2;
    if (inner) {
#pragma unroll
      for (int zz = 0; zz < SZ; zz += 2) {
        const int z = z2s + zz;
        rb_update<false, false>(B, A, Se, Sf, Sx, Sy, Sz, oe2 + z * EPL, of2 + z * FPL,
                                oy2 + z * YPL, i, j, z0 + z);
      }
    } else if (i < n0 && j < n1) {
      for (int z = z2s; z < SZ; z += 2)
        if (z0 + z < n2)
          rb_update<true, false>(B, A, Se, Sf, Sx, Sy, Sz, oe2 + z * EPL, of2 + z * FPL,
                                 oy2 + z * YPL, i, j, z0 + z);
    }
  }
  __syncthreads();
  // the tile, both colours: rows of 32, every plane
  const long fo = (long)fld * B.vfs;
  const int i = x0 + x2, j = y0 + y2;
  if (i < n0 && j < n1) {
#pragma unroll
    for (int dz = 0; dz < SZ; dz++) {
      const int k = z0 + dz;
      if (k >= n2) break;
      const int idx = i + n0 * (j + n1 * k);
      const float v = Se[2 * EPL + (y2 + 2) * TBX + x2 + 4 + dz * EPL];
      ed[fo + idx] = v;
      if (ADD && !(mask[idx] & MASK_COVERED)) u[fo + idx] = v;
    }
  }
}

// ---- block (x-line) Gauss-Seidel on a box (Sec. 4.3 names block
// Gauss-Seidel; the blocks are the box's x-lines, reading R26).  One colour
// of lines per launch: each thread solves one x-line (j, k) with
// (j + k) % 2 == colour exactly by the Thomas algorithm, the line's cells
// coupled through their x faces and the y- and z-neighbours (lines of the
// other colour) at their current values.  The forward elimination keeps c'
// in cp (a scratch vector of the correction's layout) and d' in e; the back
// substitution overwrites e.  Grid (lines / 128, 2 fields).
// ZERO: the neighbours are 0 (the first pass of a level).  (On level 0 the
// caller adds the correction of both colours' lines to the composite
// solution after the last pass.)
template <class P, bool ZERO>
__global__ void __launch_bounds__(128) k_bline(BoxK<P> B, int colour, P* cpbuf) {
  const int fld = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B.n1 * B.n2) return;
  const int n0 = B.n0, n1 = B.n1, n2 = B.n2;
  const int j = q % n1, k = q / n1;
  if (((j + k) & 1) != colour) return;
  P* e = B.e + fld * B.vfs;
  P* cp = cpbuf + fld * B.vfs;
  const P* f = B.f + fld * B.vfs;
  const P* A = B.A + fld * B.Afs;
  const int s2 = n0 * n1;
  const int base = n0 * (j + n1 * k);
  P cprev = P(0), dprev = P(0);
  for (int i = 0; i < n0; i++) {
    const int idx = base + i;
    P d = P(1), lo = P(0), hi = P(0), of = P(0), a;
    if (i > 0) { a = A[idx]; d += a; lo = -a; }
    else d += A[B.gbase + B.fo[0] + j + n1 * k];
    if (i < n0 - 1) { a = A[idx + 1]; d += a; hi = -a; }
    else d += A[B.gbase + B.fo[1] + j + n1 * k];
    if (j > 0) { a = A[B.NA + idx]; d += a; if (!ZERO) of += a * e[idx - n0]; }
    else d += A[B.gbase + B.fo[2] + k + n2 * i];
    if (j < n1 - 1) { a = A[B.NA + idx + n0]; d += a; if (!ZERO) of += a * e[idx + n0]; }
    else d += A[B.gbase + B.fo[3] + k + n2 * i];
    if (k > 0) { a = A[2 * B.NA + idx]; d += a; if (!ZERO) of += a * e[idx - s2]; }
    else d += A[B.gbase + B.fo[4] + i + n0 * j];
    if (k < n2 - 1) { a = A[2 * B.NA + idx + s2]; d += a; if (!ZERO) of += a * e[idx + s2]; }
    else d += A[B.gbase + B.fo[5] + i + n0 * j];
    const P m = d - lo * cprev;
    cprev = hi / m;
    dprev = (f[idx] + of - lo * dprev) / m;
    cp[idx] = cprev;
    e[idx] = dprev;
  }
  P x = dprev;
  for (int i = n0 - 2; i >= 0; i--) {
    const int idx = base + i;
    x = e[idx] - cp[idx] * x;
    e[idx] = x;
  }
}

// one damped point Jacobi sweep on a box (Sec. 4.3): ed = es + omega
// ((f + off(es)) / diag - es); ZERO: es = 0; ADD: u += ed on uncovered cells
// (level 0).  One cell per thread; grid (tiles x, tiles y, 2 x tiles z).
template <class P, bool ZERO, bool ADD>
__global__ void __launch_bounds__(FTHREADS) k_bjacobi(BoxK<P> B, P omega,
                                                       const P* __restrict__ es,
                                                       P* __restrict__ ed,
                                                       const uint8_t* __restrict__ mask,
                                                       P* __restrict__ u) {
  const int ntz = gridDim.z >> 1;
  const int fld = blockIdx.z >= ntz;
  const int t = threadIdx.x;
  const int i = blockIdx.x * VT + ft_i(t), j = blockIdx.y * VT + ft_j(t);
  const int k = (blockIdx.z - fld * ntz) * VT + ft_k(t);
  if (i >= B.n0 || j >= B.n1 || k >= B.n2) return;
  const long fo = fld * B.vfs;
  const P* e = es + fo;
  P dg, of;
  box_row<P, ZERO>(B, B.A + fld * B.Afs, e, i, j, k, dg, of);
  const int idx = i + B.n0 * (j + B.n1 * k);
  const P fv = B.f[fo + idx];
  const P ev = ZERO ? omega * (fv / dg) : e[idx] + omega * ((fv + of) / dg - e[idx]);
  ed[fo + idx] = ev;
  if (ADD && !(mask[idx] & MASK_COVERED)) u[fo + idx] += ev;
}

// coarse rhs = 8-cell average of the fine residual f - L e (Sec. 4.3: simple
// averaging restriction).  BLACK0: the last pass on the fine box was black,
// so the residual of the black children is zero (up to rounding) and only
// the 4 red children are summed.  Four consecutive threads share a coarse
// cell, one red child (and one black child unless BLACK0) each, and sum by
// shuffles; a block covers 8 x 4 x 2 coarse cells.
constexpr int RX = 8, RY = 4, RZ = 2;
dim3 restrict_grid(int cn0, int cn1, int cn2) {
  return dim3((cn0 + RX - 1) / RX, (cn1 + RY - 1) / RY, 2 * ((cn2 + RZ - 1) / RZ));
}

template <class P, bool BLACK0>
__global__ void __launch_bounds__(VTHREADS) k_brestrict(BoxK<P> F, P* fc, int cn0, int cn1,
                                                         int cn2) {
  const int ntz = gridDim.z >> 1;
  const int fld = blockIdx.z >= ntz;
  const int t = threadIdx.x;
  const int q = t & 3;
  const int ci = blockIdx.x * RX + ((t >> 2) & 7), cj = blockIdx.y * RY + ((t >> 5) & 3);
  const int ck = (blockIdx.z - fld * ntz) * RZ + (t >> 7);
  const bool in = ci < cn0 && cj < cn1 && ck < cn2;
  P s = P(0);
  if (in) {
    const P* e = F.e + fld * F.vfs;
    const P* f = F.f + fld * F.vfs;
    const P* A = F.A + fld * F.Afs;
    // red children (0,0,0) (1,1,0) (1,0,1) (0,1,1); black (1,0,0) (0,1,0) (0,0,1) (1,1,1)
    const int rx = (q == 1 || q == 2), ry = (q == 1 || q == 3), rz = (q >= 2);
    const int bx = (q == 0 || q == 3), by = (q == 1 || q == 3), bz = (q == 2 || q == 3);
#pragma unroll
    for (int c = 0; c < (BLACK0 ? 1 : 2); c++) {
      const int i = 2 * ci + (c ? bx : rx), j = 2 * cj + (c ? by : ry), k = 2 * ck + (c ? bz : rz);
      P dg, of;
      box_row<P, false>(F, A, e, i, j, k, dg, of);
      const int idx = i + F.n0 * (j + F.n1 * k);
      s += f[idx] - (dg * e[idx] - of);
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  if (in && q == 0) fc[fld * ((long)cn0 * cn1 * cn2) + ci + cn0 * (cj + cn1 * ck)] = s / P(8);
}

// trilinear interpolation weight along one axis: (3/4 parent, 1/4 neighbour);
// neighbours outside the domain fall back to the parent.  map: dense level
// map of the coarse level (cell or -1), else src is the coarse box itself.
template <class P>
__device__ __forceinline__ P tri_interp(const P* src, int cn0, int cn1, int cn2, int q0, int q1,
                                        int q2, const int* map) {
  const int p0 = q0 >> 1, p1 = q1 >> 1, p2 = q2 >> 1;
  int o0 = (q0 & 1) ? 1 : -1, o1 = (q1 & 1) ? 1 : -1, o2 = (q2 & 1) ? 1 : -1;
  if (p0 + o0 < 0 || p0 + o0 >= cn0) o0 = 0;
  if (p1 + o1 < 0 || p1 + o1 >= cn1) o1 = 0;
  if (p2 + o2 < 0 || p2 + o2 >= cn2) o2 = 0;
  int parent = -1;
  P s = P(0);
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int a = q & 1, b = (q >> 1) & 1, d = q >> 2;
    const P w = (a ? P(0.25) : P(0.75)) * (b ? P(0.25) : P(0.75)) * (d ? P(0.25) : P(0.75));
    const int li = (p0 + a * o0) + cn0 * ((p1 + b * o1) + cn1 * (p2 + d * o2));
    int si = map ? map[li] : li;
    if (si < 0) {   // nesting guard: a missing neighbour takes the parent
      if (parent < 0) parent = map[p0 + cn0 * (p1 + cn1 * p2)];
      si = parent;
    }
    s += w * src[si];
  }
  return s;
}

// e(fine box) += trilinear interpolation of the coarse correction
// out = e + P ec (out may be e itself).  One thread per coarse cell p and its
// 2x2x2 children: the 27 coarse values around p are loaded once and shared
// by the children, each of which sums its 8 terms in tri_interp's order and
// with its weights (parent 3/4, the neighbour on the child's side 1/4 per
// axis; the parent itself where that neighbour is outside the box), so the
// result is bit-identical to tri_interp per fine cell.  grid (coarse x / 8,
// y / 8, 2 fields x z / 4), 256 threads.
constexpr int PX = 8, PY = 8, PZ = 4;
template <class P>
__global__ void __launch_bounds__(PX * PY * PZ) k_bprolong(const P* ec, int cn0, int cn1,
                                                            int cn2, BoxK<P> F, P* out) {
  const int ntz = gridDim.z >> 1;
  const int fld = blockIdx.z >= ntz;
  const int t = threadIdx.x;
  const int p0 = blockIdx.x * PX + t % PX, p1 = blockIdx.y * PY + (t / PX) % PY;
  const int p2 = (blockIdx.z - fld * ntz) * PZ + t / (PX * PY);
  if (p0 >= cn0 || p1 >= cn1 || p2 >= cn2) return;
  const P* src = ec + fld * ((long)cn0 * cn1 * cn2);
  const long fo = fld * F.vfs;
  // coarse coordinates of the low / centre / high neighbours per axis
  const int cx[3] = {p0 > 0 ? p0 - 1 : p0, p0, p0 < cn0 - 1 ? p0 + 1 : p0};
  const int cy[3] = {p1 > 0 ? p1 - 1 : p1, p1, p1 < cn1 - 1 ? p1 + 1 : p1};
  const int cz[3] = {p2 > 0 ? p2 - 1 : p2, p2, p2 < cn2 - 1 ? p2 + 1 : p2};
  P c[3][3][3];
#pragma unroll
  for (int z = 0; z < 3; z++)
#pragma unroll
    for (int y = 0; y < 3; y++)
#pragma unroll
      for (int x = 0; x < 3; x++) c[z][y][x] = src[cx[x] + cn0 * (cy[y] + cn1 * cz[z])];
#pragma unroll
  for (int sz = 0; sz < 2; sz++)
#pragma unroll
    for (int sy = 0; sy < 2; sy++)
#pragma unroll
      for (int sx = 0; sx < 2; sx++) {
        const int i = 2 * p0 + sx, j = 2 * p1 + sy, k = 2 * p2 + sz;
        if (i >= F.n0 || j >= F.n1 || k >= F.n2) continue;
        P v = P(0);
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int a = q & 1, b = (q >> 1) & 1, d = q >> 2;
          const P w = (a ? P(0.25) : P(0.75)) * (b ? P(0.25) : P(0.75)) * (d ? P(0.25) : P(0.75));
          // term a of axis x: the parent (centre) or the neighbour on the child's side
          const int xs = a ? 2 * sx : 1, ys = b ? 2 * sy : 1, zs = d ? 2 * sz : 1;
          v += w * c[zs][ys][xs];
        }
        const long idx = fo + i + F.n0 * (j + (long)F.n1 * k);
        out[idx] = F.e[idx] + v;
      }
}

// ------------------------------------------------- AMR (multi-patch) levels
template <class P>
struct VLev {
  const int4* vt;          // tiles: x patch | kTileCovered, y i0, z j0, w k0
  const PatchDev* patches;
  const uint8_t* mask;
  const int2* gsrc;        // per ghost: (sibling source cell, 0), (-1, 0) physical,
                           // (-2 - first term, end of terms) coarse-fine
  const int* gidx;         // coarse-fine ghost terms: source cells and weights
  const P* gw;
  const P* A;              // field f at A + f * Afs; slots [3N | G]
  long Afs;
  int N, G;
};

// ghost slot of face fc of cell (a, b) in the face's (t1, t2) coordinates
__device__ __forceinline__ int ghost_slot(const PatchDev& Pt, int fc, int a, int b) {
  return Pt.goff + Pt.fo[fc] + a + Pt.n[((fc >> 1) + 1) % 3] * b;
}

// one colour of a red-black pass of the level-l error equation (homogeneous
// coarse-fine ghosts e_g = e_c/3; sibling cells have the other colour and
// are read directly); one level tile per block and loop iteration
// (level_grid), both fields per thread.  ZERO / ADD as for k_bsmooth.
template <class P, bool ZERO, bool ADD>
__device__ __forceinline__ void k_lsmooth_tile(int tt, VLev<P> V, int t0, int colour,
                                               P* __restrict__ e,
                                               const P* __restrict__ f,
                                               P* __restrict__ u) {
  const int4 tl = V.vt[t0 + tt];
  const PatchDev Pt = V.patches[tl.x & kTilePatch];   // a register copy: no reloads after stores
  const int nx = Pt.n[0], ny = Pt.n[1], nz = Pt.n[2];
  const int t = threadIdx.x;
  const int j = tl.z + rb_j(t), k = tl.w + rb_k(t);
  if (j >= ny || k >= nz) return;
  const int ib = tl.y + rb_px(t);
  const int par = (Pt.lo[0] + Pt.lo[1] + Pt.lo[2] + j + k + colour) & 1;
  const int i = ib + par, ip = ib + 1 - par;
  const int N = V.N;
  P* e0 = e;
  P* e1 = e + N;
  const P* A0 = V.A;
  const P* A1 = V.A + V.Afs;
  const int row = Pt.off + nx * (j + ny * k);
  if (i < nx) {
    const int idx = row + i;
    P d0 = P(1), o0 = P(0), d1 = P(1), o1 = P(0);
    auto face = [&](int off, int nb) {
      const P a0 = A0[off], a1 = A1[off];
      d0 += a0;
      d1 += a1;
      if (!ZERO) {
        o0 += a0 * e0[nb];
        o1 += a1 * e1[nb];
      }
    };
    auto bnd = [&](int fc, int a1, int b1) {
      const int g = ghost_slot(Pt, fc, a1, b1);
      const P av0 = A0[3 * N + g], av1 = A1[3 * N + g];
      const int src = V.gsrc[g].x;
      if (src >= 0) {
        d0 += av0;
        d1 += av1;
        if (!ZERO) {
          o0 += av0 * e0[src];
          o1 += av1 * e1[src];
        }
      } else if (src < -1) {
        d0 += P(2.0 / 3.0) * av0;
        d1 += P(2.0 / 3.0) * av1;
      } else {   // Robin diagonal term, or 0 for Neumann
        d0 += av0;
        d1 += av1;
      }
    };
    const int s2 = nx * ny;
    if (i > 0) face(idx, idx - 1); else bnd(0, j, k);
    if (i < nx - 1) face(idx + 1, idx + 1); else bnd(1, j, k);
    if (j > 0) face(N + idx, idx - nx); else bnd(2, k, i);
    if (j < ny - 1) face(N + idx + nx, idx + nx); else bnd(3, k, i);
    if (k > 0) face(2 * N + idx, idx - s2); else bnd(4, i, j);
    if (k < nz - 1) face(2 * N + idx + s2, idx + s2); else bnd(5, i, j);
    const P ev0 = (f[idx] + o0) / d0, ev1 = (f[N + idx] + o1) / d1;
    e0[idx] = ev0;
    e1[idx] = ev1;
    if (ADD && !(V.mask[idx] & MASK_COVERED)) {
      u[idx] += ev0;
      u[N + idx] += ev1;
    }
  }
  if (ip < nx) {
    const int idx = row + ip;
    if (ZERO) {
      e0[idx] = P(0);
      e1[idx] = P(0);
    }
    if (ADD && !(V.mask[idx] & MASK_COVERED)) {
      u[idx] += e0[idx];
      u[N + idx] += e1[idx];
    }
  }
}

template <class P, bool ZERO, bool ADD>
__global__ void __launch_bounds__(VTHREADS) k_lsmooth(int ntl, VLev<P> V, int t0, int colour,
                                                      P* __restrict__ e,
                                                      const P* __restrict__ f,
                                                      P* __restrict__ u) {
  for (int tt = blockIdx.x; tt < ntl; tt += gridDim.x)
    k_lsmooth_tile<P, ZERO, ADD>(tt, V, t0, colour, e, f, u);
}

// one damped point Jacobi sweep of the level-l error equation (Sec. 4.3):
// ed = es + omega ((f + off(es)) / diag - es) with the level operator of
// k_lsmooth; ZERO: es = 0, ed = omega (f / diag); ADD: u += ed on uncovered
// cells.  One cell per thread, both fields; one level tile per block and
// loop iteration (level_grid).
template <class P, bool ZERO, bool ADD>
__device__ __forceinline__ void k_ljacobi_tile(int tt, VLev<P> V, int t0, P omega,
                                               const P* __restrict__ es,
                                               P* __restrict__ ed,
                                               const P* __restrict__ f,
                                               P* __restrict__ u) {
  const int4 tl = V.vt[t0 + tt];
  const PatchDev Pt = V.patches[tl.x & kTilePatch];   // a register copy: no reloads after stores
  const int nx = Pt.n[0], ny = Pt.n[1], nz = Pt.n[2];
  const int t = threadIdx.x;
  const int i = tl.y + ft_i(t), j = tl.z + ft_j(t), k = tl.w + ft_k(t);
  if (i >= nx || j >= ny || k >= nz) return;
  const int N = V.N;
  const int idx = Pt.off + i + nx * (j + ny * k);
  const P* e0 = es;
  const P* e1 = es + N;
  const P* A0 = V.A;
  const P* A1 = V.A + V.Afs;
  P d0 = P(1), o0 = P(0), d1 = P(1), o1 = P(0);
  auto face = [&](int off, int nb) {
    const P a0 = A0[off], a1 = A1[off];
    d0 += a0;
    d1 += a1;
    if (!ZERO) {
      o0 += a0 * e0[nb];
      o1 += a1 * e1[nb];
    }
  };
  auto bnd = [&](int fc, int a1, int b1) {
    const int g = ghost_slot(Pt, fc, a1, b1);
    const P av0 = A0[3 * N + g], av1 = A1[3 * N + g];
    const int src = V.gsrc[g].x;
    if (src >= 0) {
      d0 += av0;
      d1 += av1;
      if (!ZERO) {
        o0 += av0 * e0[src];
        o1 += av1 * e1[src];
      }
    } else if (src < -1) {
      d0 += P(2.0 / 3.0) * av0;
      d1 += P(2.0 / 3.0) * av1;
    } else {   // Robin diagonal term, or 0 for Neumann
      d0 += av0;
      d1 += av1;
    }
  };
  const int s2 = nx * ny;
  if (i > 0) face(idx, idx - 1); else bnd(0, j, k);
  if (i < nx - 1) face(idx + 1, idx + 1); else bnd(1, j, k);
  if (j > 0) face(N + idx, idx - nx); else bnd(2, k, i);
  if (j < ny - 1) face(N + idx + nx, idx + nx); else bnd(3, k, i);
  if (k > 0) face(2 * N + idx, idx - s2); else bnd(4, i, j);
  if (k < nz - 1) face(2 * N + idx + s2, idx + s2); else bnd(5, i, j);
  P ev0, ev1;
  if (ZERO) {
    ev0 = omega * (f[idx] / d0);
    ev1 = omega * (f[N + idx] / d1);
  } else {
    ev0 = e0[idx] + omega * ((f[idx] + o0) / d0 - e0[idx]);
    ev1 = e1[idx] + omega * ((f[N + idx] + o1) / d1 - e1[idx]);
  }
  ed[idx] = ev0;
  ed[N + idx] = ev1;
  if (ADD && !(V.mask[idx] & MASK_COVERED)) {
    u[idx] += ev0;
    u[N + idx] += ev1;
  }
}

template <class P, bool ZERO, bool ADD>
__global__ void __launch_bounds__(FTHREADS) k_ljacobi(int ntl, VLev<P> V, int t0, P omega,
                                                      const P* __restrict__ es,
                                                      P* __restrict__ ed,
                                                      const P* __restrict__ f,
                                                      P* __restrict__ u) {
  for (int tt = blockIdx.x; tt < ntl; tt += gridDim.x)
    k_ljacobi_tile<P, ZERO, ADD>(tt, V, t0, omega, es, ed, f, u);
}

// r = f - L^c u on the leaf cells of every tile (composite operator): the
// sibling and coarse-fine ghosts of u are formed here (the coarse-fine one
// from its interpolation terms, Sec. 3.2.1); the fine-side coarse-fine
// fluxes a (u_g - u_c) go to cf for flux matching.  Faces marked in the mask
// as coarse sides of coarse-fine faces are left to flux matching; covered
// cells are left to the average-down.  One tile per block and loop
// iteration (level_grid); both fields per thread.
template <class P>
__device__ __forceinline__ void k_cresid_tile(int tt, VLev<P> V, const P* __restrict__ u,
                                              const P* __restrict__ f,
                                              P* __restrict__ r, P* __restrict__ cf) {
  const int4 tl = V.vt[tt];
  if (tl.x & kTileCovered) return;
  const PatchDev Pt = V.patches[tl.x & kTilePatch];   // a register copy: no reloads after stores
  const int nx = Pt.n[0], ny = Pt.n[1], nz = Pt.n[2];
  const int t = threadIdx.x;
  const int i = tl.y + ft_i(t), j = tl.z + ft_j(t), k = tl.w + ft_k(t);
  if (i >= nx || j >= ny || k >= nz) return;
  const int N = V.N;
  const int idx = Pt.off + i + nx * (j + ny * k);
  // both fields in one thread: independent loads, shared index work
  const P* A0 = V.A;
  const P* A1 = V.A + V.Afs;
  const P* u0 = u;
  const P* u1 = u + N;
  const int s2 = nx * ny;
  // the in-patch faces' coefficients and neighbour values are fetched before
  // the mask is known (it only selects which of them count)
  const int off6[6] = {idx, idx + 1, N + idx, N + idx + nx, 2 * N + idx, 2 * N + idx + s2};
  const int nb6[6] = {idx - 1, idx + 1, idx - nx, idx + nx, idx - s2, idx + s2};
  const bool in6[6] = {i > 0, i < nx - 1, j > 0, j < ny - 1, k > 0, k < nz - 1};
  P fa0[6], fa1[6], fv0[6], fv1[6];
#pragma unroll
  for (int q = 0; q < 6; q++) {
    fa0[q] = in6[q] ? A0[off6[q]] : P(0);
    fa1[q] = in6[q] ? A1[off6[q]] : P(0);
    fv0[q] = in6[q] ? u0[nb6[q]] : P(0);
    fv1[q] = in6[q] ? u1[nb6[q]] : P(0);
  }
  const uint8_t m = V.mask[idx];
  const P uc0 = u0[idx], uc1 = u1[idx];
  if (m & MASK_COVERED) return;
  P L0 = uc0, L1 = uc1;
  auto face = [&](int q) {
    L0 += fa0[q] * (uc0 - fv0[q]);
    L1 += fa1[q] * (uc1 - fv1[q]);
  };
  auto bnd = [&](int fc, int a1, int b1) {
    const int g = ghost_slot(Pt, fc, a1, b1);
    const P av0 = A0[3 * N + g], av1 = A1[3 * N + g];
    const int2 src = V.gsrc[g];
    if (src.x >= 0) {
      L0 += av0 * (uc0 - u0[src.x]);
      L1 += av1 * (uc1 - u1[src.x]);
    } else if (src.x < -1) {
      P ug0 = P(0), ug1 = P(0);
      for (int q = -2 - src.x; q < src.y; q++) {
        const int c = V.gidx[q];
        const P w = V.gw[q];
        ug0 += w * u0[c];
        ug1 += w * u1[c];
      }
      L0 += av0 * (uc0 - ug0);
      L1 += av1 * (uc1 - ug1);
      cf[g] = av0 * (ug0 - uc0);
      cf[(long)V.G + g] = av1 * (ug1 - uc1);
    } else {
      L0 += av0 * uc0;   // Robin term (0 for Neumann)
      L1 += av1 * uc1;
    }
  };
  if (!(m & 2)) { if (in6[0]) face(0); else bnd(0, j, k); }
  if (!(m & 4)) { if (in6[1]) face(1); else bnd(1, j, k); }
  if (!(m & 8)) { if (in6[2]) face(2); else bnd(2, k, i); }
  if (!(m & 16)) { if (in6[3]) face(3); else bnd(3, k, i); }
  if (!(m & 32)) { if (in6[4]) face(4); else bnd(4, i, j); }
  if (!(m & 64)) { if (in6[5]) face(5); else bnd(5, i, j); }
  r[idx] = f[idx] - L0;
  r[N + idx] = f[N + idx] - L1;
}

template <class P>
__global__ void __launch_bounds__(FTHREADS) k_cresid(int ntl, VLev<P> V, const P* __restrict__ u,
                                                     const P* __restrict__ f,
                                                     P* __restrict__ r, P* __restrict__ cf) {
  for (int tt = blockIdx.x; tt < ntl; tt += gridDim.x)
    k_cresid_tile<P>(tt, V, u, f, r, cf);
}

// flux matching of the composite operator (each coarse cell with coarse-fine
// faces gets -sum(fine fluxes)/8 per face) fused with the average-down of the
// finest covered level: the two write disjoint cells, and the covered cells
// of the level below the finest read only finest-level cells, which flux
// matching never writes.
template <class P>
__global__ void k_reflux_avg(const int* cell, const int* off, const int4* gq, int nrf,
                             const int4* __restrict__ cov, int ncov, int N, int G, const P* cf,
                             P* r) {
  const int fld = blockIdx.y;
  const P* c = cf + (long)fld * G;
  P* rf = r + (long)fld * N;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nrf + ncov;
       q += gridDim.x * blockDim.x) {
    if (q < nrf) {
      P s = P(0);
      for (int e = off[q]; e < off[q + 1]; e++) {
        const int4 g = gq[e];
        s += c[g.x] + c[g.y] + c[g.z] + c[g.w];
      }
      rf[cell[q]] -= s / P(8);
    } else {
      const int4 v = cov[q - nrf];
      P s = P(0);
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
          for (int e = 0; e < 2; e++) s += rf[v.y + a + b * v.z + e * v.w];
      rf[v.x] = s / P(8);
    }
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

// u += e on the uncovered cells of [c0, c0 + n) (a level whose last pass
// could not do it: no smoothing sweeps)
template <class P>
__global__ void k_add_leaf(const uint8_t* mask, int c0, int n, int N, const P* e, P* u) {
  const int fld = blockIdx.y;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int c = c0 + q;
    if (!(mask[c] & MASK_COVERED)) u[(long)fld * N + c] += e[(long)fld * N + c];
  }
}

// v(level m) = trilinear interpolation of src(level m-1) via its dense map;
// u += v on uncovered level-m cells; PV: also keep v for the next level.
// Both fields per thread (the map lookups are shared).
template <class P, bool PV>
__device__ __forceinline__ void k_vprolong_tile(int tt, VLev<P> V, int t0, const int* cmap,
                                                int cn0, int cn1, int cn2,
                                                const P* __restrict__ src,
                                                P* __restrict__ pv, P* __restrict__ u) {
  const int4 tl = V.vt[t0 + tt];
  const PatchDev Pt = V.patches[tl.x & kTilePatch];   // a register copy: no reloads after stores
  const int t = threadIdx.x;
  const int i = tl.y + ft_i(t), j = tl.z + ft_j(t), k = tl.w + ft_k(t);
  if (i >= Pt.n[0] || j >= Pt.n[1] || k >= Pt.n[2]) return;
  const int N = V.N;
  const int idx = Pt.off + i + Pt.n[0] * (j + Pt.n[1] * k);
  const int q0 = Pt.lo[0] + i, q1 = Pt.lo[1] + j, q2 = Pt.lo[2] + k;
  const int p0 = q0 >> 1, p1 = q1 >> 1, p2 = q2 >> 1;
  int o0 = (q0 & 1) ? 1 : -1, o1 = (q1 & 1) ? 1 : -1, o2 = (q2 & 1) ? 1 : -1;
  if (p0 + o0 < 0 || p0 + o0 >= cn0) o0 = 0;
  if (p1 + o1 < 0 || p1 + o1 >= cn1) o1 = 0;
  if (p2 + o2 < 0 || p2 + o2 >= cn2) o2 = 0;
  int parent = -1;
  P v0 = P(0), v1 = P(0);
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int a = q & 1, b = (q >> 1) & 1, d = q >> 2;
    const P w = (a ? P(0.25) : P(0.75)) * (b ? P(0.25) : P(0.75)) * (d ? P(0.25) : P(0.75));
    int si = cmap[(p0 + a * o0) + cn0 * ((p1 + b * o1) + cn1 * (p2 + d * o2))];
    if (si < 0) {   // nesting guard: a missing neighbour takes the parent
      if (parent < 0) parent = cmap[p0 + cn0 * (p1 + cn1 * p2)];
      si = parent;
    }
    v0 += w * src[si];
    v1 += w * src[N + si];
  }
  if (PV) {
    pv[idx] = v0;
    pv[N + idx] = v1;
  }
  if (!(V.mask[idx] & MASK_COVERED)) {
    u[idx] += v0;
    u[N + idx] += v1;
  }
}

template <class P, bool PV>
__global__ void __launch_bounds__(FTHREADS) k_vprolong(int ntl, VLev<P> V, int t0, const int* cmap,
                                                       int cn0, int cn1, int cn2,
                                                       const P* __restrict__ src,
                                                       P* __restrict__ pv, P* __restrict__ u) {
  for (int tt = blockIdx.x; tt < ntl; tt += gridDim.x)
    k_vprolong_tile<P, PV>(tt, V, t0, cmap, cn0, cn1, cn2, src, pv, u);
}

// V-cycle input: fr = w (the residual of u = 0) and, with finer levels (ff
// non-null), ff = w and u = 0; TR: w goes through the transposed P2 solve
// first, P2^T = [[1 + sb, -sb], [-sbt, 1 + sbt]]
template <class P, bool TR>
__global__ void k_vc_init(int N, const double* w, const P* p, P* ff, P* fr, P* fu, const int* jd,
                          long jstride) {
  if (jd) w += (long)(*jd) * jstride;   // w = column *jd of a basis (device index)
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    P xE, xT;
    if (TR) {
      const P sb = p[c], sbt = p[N + c], rd = p[2L * N + c];
      const P wE = (P)w[c], wT = (P)w[N + c];
      xE = ((P(1) + sbt) * wE + sb * wT) * rd;
      xT = (sbt * wE + (P(1) + sb) * wT) * rd;
    } else {
      xE = (P)w[c];
      xT = (P)w[N + c];
    }
    if (ff) {   // the composite rhs and solution exist only with finer levels
      ff[c] = xE;
      ff[N + c] = xT;
      fu[c] = P(0);
      fu[N + c] = P(0);
    }
    fr[c] = xE;
    fr[N + c] = xT;
  }
}

// ghost descriptors for the V-cycle: sibling (source cell, 0), physical
// (-1, 0), coarse-fine (-2 - first term, end of terms); the coarse-fine
// weights in the V-cycle precision
template <class P>
__global__ void k_vc_ghosts(const uint8_t* gtype, const int* gt0, const int* gidx, int G,
                            const double* gw, int nterm, int2* gsrc, P* gwp) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const uint8_t t = gtype[g];
    gsrc[g] = (t == GT_SIBLING) ? make_int2(gidx[gt0[g]], 0)
              : (t == GT_CF)    ? make_int2(-2 - gt0[g], gt0[g + 1])
                                : make_int2(-1, 0);
  }
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nterm; q += gridDim.x * blockDim.x)
    gwp[q] = (P)gw[q];
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
// (err set: a TMA wait of this V-cycle gave up, and y reads NaN)
template <class P>
__global__ void k_p2(int N, const P* zin, const P* p, double* y, const int* jd, long jstride,
                     double* y2, const int* err) {
  if (jd) y += (long)(*jd) * jstride;   // y = column *jd of a basis (device index)
  if (*err) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 2 * N; c += gridDim.x * blockDim.x) {
      y[c] = nan;
      if (y2) y2[c] = nan;
    }
    return;
  }
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

// y = V-cycle output in FP64; covered cells get 0
template <class P>
__global__ void k_out_cast(const uint8_t* mask, int N, const P* u, double* y, const int* err) {
  if (*err) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 2 * N; c += gridDim.x * blockDim.x)
      y[c] = nan;
    return;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    bool cov = mask[c] & MASK_COVERED;
    y[c] = cov ? 0.0 : (double)u[c];
    y[N + c] = cov ? 0.0 : (double)u[N + c];
  }
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
      if (i >= nx || j >= ny || k >= tile.k1) continue;
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
// with A non-null also the scaled coefficient of the target (level l).
// SCALED (after the linearisation, which writes scaled coefficients and raw
// values on Robin faces only): the scaled coefficient of a non-Robin face is
// the mean of the 4 fine scaled ones over 4 (beta C / h^2 with C the mean of
// the fine C and h twice the fine h), the Robin faces average the raw D_b.
// (a + b + c + d) / 16: the mean of four scaled P1 coefficients over 4
template <class P>
__device__ __forceinline__ P mean16(P a, P b, P c, P d) {
  return P(0.0625) * ((a + b) + (c + d));
}

template <class P, bool SCALED>
__global__ void k_coef_coarsen(const int* tgt, const int4* src, int n, long AF, int N,
                               const uint8_t* gtype, const uint8_t* gface,
                               const double* dbeta, LevelHP lh, int lvl, double* Craw, P* A) {
  const double beta = *dbeta;
  const int fld = blockIdx.y;
  double* C = Craw + fld * AF;
  const double bx = beta * lh.r2[lvl][0], by = beta * lh.r2[lvl][1], bz = beta * lh.r2[lvl][2];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int4 s = src[q];
    int t = tgt[q];
    if (SCALED) {
      const P* Af = A + fld * AF;
      double v;
      const uint8_t ty = (t < 3 * N) ? GT_SIBLING : gtype[t - 3 * N];
      if (ty == GT_NEUMANN) {
        v = 0.0;
      } else if (ty == GT_ROBIN) {
        const double c = 0.25 * (C[s.x] + C[s.y] + C[s.z] + C[s.w]);
        C[t] = c;
        const double h = lh.h[lvl][(gface[t - 3 * N] & 7) / 2];
        v = (fld == 0) ? beta * 2.0 * c / (h * (4.0 * c + h)) : 0.0;
      } else {
        // the mean of four scaled coefficients over 4, in their own precision
        A[fld * AF + t] = mean16<P>(Af[s.x], Af[s.y], Af[s.z], Af[s.w]);
        continue;
      }
      A[fld * AF + t] = (P)v;
      continue;
    }
    double c = 0.25 * (C[s.x] + C[s.y] + C[s.z] + C[s.w]);
    C[t] = c;
    if (!A) continue;
    double v;
    if (t < 3 * N) {   // low-face slot of axis t / N (3N + G < 2^31)
      v = c * ((t >= 2 * N) ? bz : (t >= N) ? by : bx);
    } else {
      int g = t - 3 * N;
      int d = (gface[g] & 7) / 2;
      double h = lh.h[lvl][d];
      uint8_t ty = gtype[g];
      if (ty == GT_NEUMANN) v = 0.0;
      else if (ty == GT_ROBIN) v = (fld == 0) ? beta * 2.0 * c / (h * (4.0 * c + h)) : 0.0;
      else v = c * beta * lh.r2[lvl][d];
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
      if (i >= nx || j >= ny || k >= tile.k1) continue;
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

// Every GMG level m >= 1 of the base box in one launch, each straight from
// the base level: a level-m face covers S^2 base faces (S = 2^m), and the
// level-by-level rule (coarse C = mean of the 4 finer C; scaled
// A = beta C / h^2 with h doubling per level) composes to
//   C_m = mean of the S^2 base C,   A_m = (sum of the S^2 base A) / S^4,
// so no level waits for the one above it.  Fused with the scaling: A = beta C
// / h^2 on interior faces, beta 2 D_b / (h (4 D_b + h)) on Robin faces of E
// (D_b the mean of the S^2 base D_b), 0 elsewhere.  SCALED (after the
// linearisation): interior faces from the base level's scaled coefficients
// Ain, box faces from the raw Robin D_b.  One thread per (level, coarse cell,
// axis); FP32 coefficients are summed in FP32 (FP64 arithmetic and
// conversions issue on GB300's narrow FP64 pipe).
template <class P>
struct CoarsenAll {
  int nlev;                        // levels 1 .. nlev
  BoxRaw F;                        // the base box (level 0 of the GMG hierarchy)
  BoxRaw C[NRD_MAX_MG];            // level m at C[m]
  P* A[NRD_MAX_MG];                // scaled coefficients of level m (field f at + f AF)
  double h[NRD_MAX_MG][3];
  int item0[NRD_MAX_MG + 1];       // first item of level m (3 per coarse cell); the
                                   // coarsest level first (its items sum the most terms)
};

template <class P, bool SCALED>
__global__ void k_box_coarsen(CoarsenAll<P> a, const double* Cf, const P* Ain,
                              const int* gtype_box, const double* dbeta) {
  const int fld = blockIdx.y;
  const BoxRaw& F = a.F;
  const double* cf = Cf + fld * F.AF;
  const P* ain = SCALED ? Ain + fld * F.AF : nullptr;
  // indices are 32-bit (3N + G < 2^31 for the hierarchy, which bounds every box)
  const int fNA = (int)F.NA, fgb = (int)F.gbase;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a.item0[0];
       t += gridDim.x * blockDim.x) {
    int m = a.nlev;
    while (t >= a.item0[m - 1]) m--;
    const BoxRaw& Cc = a.C[m];
    const int ncc = Cc.n[0] * Cc.n[1] * Cc.n[2];
    const int it = t - a.item0[m];
    const int d = it / ncc, c = it - d * ncc;
    int q[3];
    const int r = c / Cc.n[0];
    q[0] = c - r * Cc.n[0];
    q[2] = r / Cc.n[1];
    q[1] = r - q[2] * Cc.n[1];
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int S = 1 << m, S2 = S * S;
    const int cNA = (int)Cc.NA, cgb = (int)Cc.gbase;
    P* Af = a.A[m] + fld * Cc.AF;
    const double beta = *dbeta;
    const double hd = a.h[m][d];
    if (q[d] > 0) {
      int p[3];
      p[d] = S * q[d];
      if (SCALED) {
        P acc[4] = {P(0), P(0), P(0), P(0)};
#pragma unroll 4
        for (int u = 0; u < S2; u++) {
          p[t1] = S * q[t1] + (u & (S - 1));
          p[t2] = S * q[t2] + (u >> m);
          acc[u & 3] += ain[d * fNA + p[0] + F.n[0] * (p[1] + F.n[1] * p[2])];
        }
        // 1 / S^4 is a power of 2: the scaling is exact
        Af[d * cNA + c] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) * (P(1) / (P(S2) * P(S2)));
      } else {
        double acc = 0.0;
        for (int u = 0; u < S2; u++) {
          p[t1] = S * q[t1] + (u & (S - 1));
          p[t2] = S * q[t2] + (u >> m);
          acc += cf[d * fNA + p[0] + F.n[0] * (p[1] + F.n[1] * p[2])];
        }
        Af[d * cNA + c] = (P)((acc / S2) * (beta / (hd * hd)));
      }
    }
    for (int sd = 0; sd < 2; sd++) {
      const bool at = sd ? (q[d] == Cc.n[d] - 1) : (q[d] == 0);
      if (!at) continue;
      const int f = 2 * d + sd;
      double v = 0.0;
      if (gtype_box[f] == 1 && fld == 0) {
        double acc = 0.0;
        for (int u = 0; u < S2; u++) {
          const int p1 = S * q[t1] + (u & (S - 1)), p2 = S * q[t2] + (u >> m);
          acc += cf[fgb + F.fo[f] + p1 + F.n[t1] * p2];
        }
        const double Db = acc / S2;
        v = beta * 2.0 * Db / (hd * (4.0 * Db + hd));
      }
      Af[cgb + Cc.fo[f] + q[t1] + Cc.n[t1] * q[t2]] = (P)v;
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
  int tail_cl = 1;   // CTAs per field of the tail's cluster
  // 8^3 tiles of all patches for the V-cycle kernels, level by level
  int4* vt = nullptr;
  int vt0[NRD_MAX_LEVELS] = {0}, vnt[NRD_MAX_LEVELS] = {0};
  int ntile = 0;
  int2* gsrc = nullptr;  // [G] V-cycle ghost descriptors
  // smoother (NRD_SMOOTH_*) and the damped-Jacobi scratch vectors
  int smoother = NRD_SMOOTH_RBGS;
  double omega = 6.0 / 7.0;
  void* fj = nullptr;    // [2][N]
  void* bj[NRD_MAX_MG] = {nullptr};
  void* gwp = nullptr;   // [nterm] coarse-fine weights in precision P
  // FP32 box levels whose arrays TMA can address run the one-launch
  // red-black sweep (k_bsweep); their tensor maps: correction [buffer: e,
  // scratch][field], rhs [field], low-face coefficients [axis][field]
  bool tma_ok[NRD_MAX_MG] = {false};
  CUtensorMap tm_e[NRD_MAX_MG][2][2];
  CUtensorMap tm_f[NRD_MAX_MG][2];
  CUtensorMap tm_a[NRD_MAX_MG][3][2];
  int* d_err = nullptr;  // set when a TMA wait of the V-cycle gave up
  int nsm = 152;         // SMs of the device (persistent sweep grid)
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
BoxK<P> boxk(const BoxRaw& B, const void* A, void* e, const void* f, long vfs) {
  BoxK<P> V;
  V.n0 = B.n[0];
  V.n1 = B.n[1];
  V.n2 = B.n[2];
  for (int q = 0; q < 6; q++) V.fo[q] = B.fo[q];
  V.A = (const P*)A;
  V.Afs = B.AF;
  V.NA = (int)B.NA;
  V.gbase = (int)B.gbase;
  V.e = (P*)e;
  V.f = (const P*)f;
  V.vfs = vfs;
  return V;
}

// 8^3 tiles of an n0 x n1 x n2 box, both fields (field 1 in the upper half of z)
dim3 tile_grid(int n0, int n1, int n2) {
  return dim3((n0 + VT - 1) / VT, (n1 + VT - 1) / VT, 2 * ((n2 + VT - 1) / VT));
}

// red-black sweeps on a box; zero: the first pass starts from e = 0; addu:
// the last pass adds e to u on uncovered cells (level 0)
// damped Jacobi sweeps between e and a scratch vector of the same layout:
// from zero, the first sweep writes whichever buffer makes the last land in
// e; from the current e, the sweeps alternate starting e -> scratch, and the
// caller arranges an even count or a start in the scratch (see
// start_in_scratch)
template <class P>
void box_jacobi(const BoxK<P>& V, P omega, P* scratch, int sweeps, bool zero, bool from_scratch,
                const uint8_t* mask, P* addu, cudaStream_t s) {
  const dim3 g = tile_grid(V.n0, V.n1, V.n2);
  P* buf[2] = {V.e, scratch};
  int cur = zero ? (((sweeps - 1) % 2 == 0) ? 0 : 1) : (from_scratch ? 1 : 0);
  for (int sw = 0; sw < sweeps; sw++) {
    const bool D = addu && sw == sweeps - 1;
    if (zero && sw == 0) {
      if (D) k_bjacobi<P, true, true><<<g, FTHREADS, 0, s>>>(V, omega, nullptr, buf[cur], mask, addu);
      else k_bjacobi<P, true, false><<<g, FTHREADS, 0, s>>>(V, omega, nullptr, buf[cur], mask, addu);
      continue;
    }
    if (D) k_bjacobi<P, false, true><<<g, FTHREADS, 0, s>>>(V, omega, buf[cur], buf[1 - cur], mask, addu);
    else k_bjacobi<P, false, false><<<g, FTHREADS, 0, s>>>(V, omega, buf[cur], buf[1 - cur], mask, addu);
    cur = 1 - cur;
  }
}


// red-black sweeps on FP32 box level m with k_bsweep, alternating between
// e and a scratch vector of the same layout (as box_jacobi); c0 = first
// colour (0: red first); zero: the first sweep starts from e = 0 and its
// target is chosen so that the last sweep writes e; otherwise the sweeps
// start from e, or from the scratch when from_scratch (the caller starts an
// odd count there, so that the last sweep writes e); addu: the last sweep
// adds the correction to u on uncovered cells (level 0)
void box_sweeps(const PcState* ps, int m, const BoxK<float>& V, float* scratch, int sweeps, int c0,
                bool zero, bool from_scratch, const uint8_t* mask, float* addu, cudaStream_t s) {
  const dim3 g((V.n0 + SX - 1) / SX, (V.n1 + SY - 1) / SY, 2 * ((V.n2 + SZ - 1) / SZ));
  float* buf[2] = {V.e, scratch};
  SweepMaps M;
  for (int fld = 0; fld < 2; fld++) {
    M.f[fld] = ps->tm_f[m][fld];
    M.ax[fld] = ps->tm_a[m][0][fld];
    M.ay[fld] = ps->tm_a[m][1][fld];
    M.az[fld] = ps->tm_a[m][2][fld];
  }
  auto src = [&](int b) {
    for (int fld = 0; fld < 2; fld++) M.es[fld] = ps->tm_e[m][b][fld];
  };
  int cur = zero ? (((sweeps - 1) % 2 == 0) ? 0 : 1) : (from_scratch ? 1 : 0);
  for (int sw = 0; sw < sweeps; sw++) {
    const bool D = addu && sw == sweeps - 1;
    if (zero && sw == 0) {
      if (D) k_bsweep<true, true><<<g, SW_THREADS, SWEEP_SMEM, s>>>(M, V, c0, buf[cur], mask, addu, ps->d_err);
      else k_bsweep<true, false><<<g, SW_THREADS, SWEEP_SMEM, s>>>(M, V, c0, buf[cur], mask, addu, ps->d_err);
      continue;
    }
    src(cur);
    if (D) k_bsweep<false, true><<<g, SW_THREADS, SWEEP_SMEM, s>>>(M, V, c0, buf[1 - cur], mask, addu, ps->d_err);
    else k_bsweep<false, false><<<g, SW_THREADS, SWEEP_SMEM, s>>>(M, V, c0, buf[1 - cur], mask, addu, ps->d_err);
    cur = 1 - cur;
  }
}

// a nonzero start for `sweeps` Gauss-Seidel or Jacobi sweeps that must end
// in e: in the scratch when the count is odd
inline bool start_in_scratch(int sweeps) { return (sweeps % 2) == 1; }

// red-black sweeps on a box in place, two colour passes each (k_bsmooth)
template <class P>
void box_smooth(const BoxK<P>& V, int sweeps, bool red_first, bool zero, const uint8_t* mask,
                P* addu, cudaStream_t s) {
  const dim3 g = tile_grid(V.n0, V.n1, V.n2);
  for (int sw = 0; sw < sweeps; sw++)
    for (int pass = 0; pass < 2; pass++) {
      const int colour = red_first ? pass : 1 - pass;
      const bool Z = zero && sw == 0 && pass == 0;
      const bool D = addu && sw == sweeps - 1 && pass == 1;
      if (Z) k_bsmooth<P, true, false><<<g, VTHREADS, 0, s>>>(V, colour, mask, addu);
      else if (D) k_bsmooth<P, false, true><<<g, VTHREADS, 0, s>>>(V, colour, mask, addu);
      else k_bsmooth<P, false, false><<<g, VTHREADS, 0, s>>>(V, colour, mask, addu);
    }
}

// block Gauss-Seidel sweeps on a box in place: two colours of x-lines each
// (k_bline); c' in the scratch
template <class P>
void box_lines(const BoxK<P>& V, P* scratch, int sweeps, bool red_first, bool zero,
               const uint8_t* mask, P* addu, cudaStream_t s) {
  const dim3 g((V.n1 * V.n2 + 127) / 128, 2);
  for (int sw = 0; sw < sweeps; sw++)
    for (int pass = 0; pass < 2; pass++) {
      const int colour = red_first ? pass : 1 - pass;
      const bool Z = zero && sw == 0 && pass == 0;
      if (Z) k_bline<P, true><<<g, 128, 0, s>>>(V, colour, scratch);
      else k_bline<P, false><<<g, 128, 0, s>>>(V, colour, scratch);
    }
  // the correction of both colours' lines into the composite solution
  if (addu) {
    const int n = V.n0 * V.n1 * V.n2;
    k_add_leaf<P><<<dim3(g1(n), 2), BS, 0, s>>>(mask, 0, n, (int)V.vfs, V.e, addu);
  }
}

// does box level m smooth with the one-launch sweep (ping-pong buffers)?
template <class P>
bool fused_sweeps(const PcState* ps, int m) {
  return sizeof(P) == 4 && ps->tma_ok[m] && ps->smoother == NRD_SMOOTH_RBGS;
}

// red-black sweeps on box level m: the one-launch TMA sweep where the level
// allows it, else two colour passes in place (from_scratch is then false)
template <class P>
void rb_sweeps(const PcState* ps, int m, const BoxK<P>& V, P* scratch, int sweeps, int c0,
               bool zero, bool from_scratch, const uint8_t* mask, P* addu, cudaStream_t s) {
  if (ps->smoother == NRD_SMOOTH_LINE) {
    box_lines(V, scratch, sweeps, c0 == 0, zero, mask, addu, s);
    return;
  }
  if constexpr (sizeof(P) == 4) {
    if (ps->tma_ok[m]) {
      box_sweeps(ps, m, V, scratch, sweeps, c0, zero, from_scratch, mask, addu, s);
      return;
    }
  }
  box_smooth(V, sweeps, c0 == 0, zero, mask, addu, s);
}



// ---- the coarse end of the GMG V-cycle in one kernel
// Levels tail_m .. nmg-1 are small (at most 8,192 cells per field): one CTA
// per field copies their coefficients and the rhs of level tail_m into
// shared memory and runs the rest of the V-cycle there (the same smoothing,
// restriction and prolongation arithmetic as the per-level kernels above),
// with block barriers where the per-level form has kernel boundaries.
constexpr int kTailThreads = 1024;
constexpr size_t kTailSmemMax = 200 * 1024;
constexpr int kTailClusterMax = 4;   // CTAs per field (4 measured fastest; 8 is portable)

template <class P>
struct TailArgs {
  int nlev;                       // levels tail_m .. nmg-1
  BoxRaw B[NRD_MAX_MG];
  const P* A[NRD_MAX_MG];         // coefficients (field f at + f * B.AF)
  int offA[NRD_MAX_MG], offE[NRD_MAX_MG], offF[NRD_MAX_MG];   // in elements
  const P* f0;                    // rhs of the first tail level (field stride vfs0)
  P* e0;                          // its correction (output)
  int vfs0;
  int nu1, nu2, csw;
  int jacobi;                     // smoother: 0 red-black Gauss-Seidel, 1 damped Jacobi
  P omega;
  int pb[NRD_MAX_MG + 1];         // first z-plane of each level in the plane lists
};

template <class P>
__device__ BoxK<P> tail_view(const TailArgs<P>& a, P* sm, int l) {
  BoxK<P> V;
  const BoxRaw& B = a.B[l];
  V.n0 = B.n[0];
  V.n1 = B.n[1];
  V.n2 = B.n[2];
  for (int q = 0; q < 6; q++) V.fo[q] = B.fo[q];
  V.A = sm + a.offA[l];
  V.Afs = 0;
  V.NA = (int)B.NA;
  V.gbase = (int)B.gbase;
  V.e = sm + a.offE[l];
  V.f = sm + a.offF[l];
  V.vfs = 0;
  return V;
}

// body(a, b, c) over an na x nb x nc grid by one CTA.  When a whole number of
// (a, b) planes fits the block, each thread keeps its (a, b) and steps c (no
// division in the loop); otherwise a flat index is split per item.  Plane
// sides that are powers of 2 (the usual coarse boxes) take shifts and masks
// instead of the integer divisions, which cost about 20 instructions each and
// dominated the one-CTA levels.
__device__ __forceinline__ bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
template <class F>
__device__ __forceinline__ void cta_for3(int na, int nb, int nc, F body) {
  const int plane = na * nb, bd = blockDim.x, t = threadIdx.x;
  if (is_pow2(na) && is_pow2(nb) && plane <= bd && is_pow2(bd)) {
    const int la = __ffs(na) - 1, lp = la + __ffs(nb) - 1;
    const int a = t & (na - 1), b = (t >> la) & (nb - 1);
    for (int c = t >> lp; c < nc; c += bd >> lp) body(a, b, c);
  } else if (plane <= bd && bd % plane == 0) {
    const int a = t % na, b = (t / na) % nb;
    for (int c = t / plane; c < nc; c += bd / plane) body(a, b, c);
  } else {
    for (int q = t; q < plane * nc; q += bd) {
      const int r = q / na, a = q - r * na;
      const int c = r / nb, b = r - c * nb;
      body(a, b, c);
    }
  }
}

// The tail's cluster: every CTA holds a replica of all tail levels in its
// shared memory and forms the values of its share of the z-planes of each
// level; a value it writes goes into the replicas of the CTAs that read its
// plane (distributed shared memory stores are slow: about 2 per clock per
// SM), and a cluster barrier ends each phase.  Readers of a plane of level X:
// for the correction e the CTAs owning a plane within 1 of it (smoothing),
// restricting from it (the fine planes 2 c0 - 1 .. 2 c1 of their coarse planes
// [c0, c1)) or prolonging from it (the coarse planes (f0 >> 1) - 1 ..
// ((f1 - 1) >> 1) + 1 of their fine planes [f0, f1)); for the rhs f its owner
// and the CTAs restricting from it (fine planes 2 c0 .. 2 c1 - 1).
constexpr int kTailPlanes = 256;   // plane-reader masks kept for up to this many planes

template <class P>
struct TailCl {
  P* sm;          // this CTA's replica
  P* const* rb;   // every CTA's replica, by rank (shared memory of this CTA)
  const uint8_t* me;   // reader masks of the e planes (null: every CTA)
  const uint8_t* mf;   // reader masks of the f planes
  const int* pb;       // first plane of each level in the masks
  int r, C, lgC;  // rank, cluster size (a power of 2), log2 of it
  __device__ __forceinline__ void put(P* p, P v, unsigned mask) const {
    const long o = p - sm;
    for (int q = 0; q < C; q++) {
      if (!((mask >> q) & 1u)) continue;
      if (q == r) *p = v;
      else rb[q][o] = v;
    }
  }
  // write a value of plane k of level l to its readers
  __device__ __forceinline__ void put_e(int l, int k, P* p, P v) const {
    put(p, v, me ? me[pb[l] + k] : 0xffu);
  }
  __device__ __forceinline__ void put_f(int l, int k, P* p, P v) const {
    put(p, v, mf ? mf[pb[l] + k] : 0xffu);
  }
  __device__ __forceinline__ void sync() const {
    if (C > 1) cg::this_cluster().sync();
    else __syncthreads();
  }
  __device__ __forceinline__ void own(int nz, int rank, int& c0, int& c1) const {
    c0 = (rank * nz) >> lgC;
    c1 = ((rank + 1) * nz) >> lgC;
  }
};

// cta_for3 over this CTA's planes [r nc / C, (r + 1) nc / C) of c
template <class P, class F>
__device__ __forceinline__ void cl_for3(const TailCl<P>& cl, int na, int nb, int nc, F body) {
  const int c0 = (cl.r * nc) >> cl.lgC, c1 = ((cl.r + 1) * nc) >> cl.lgC;
  cta_for3(na, nb, c1 - c0, [&](int a, int b, int c) { body(a, b, c0 + c); });
}

// damped Jacobi sweeps: every thread forms the new values of its cells (at
// most 8: tail levels hold at most 8,192 cells) from the old iterate, then,
// once every CTA has read the old iterate, all write
template <class P>
__device__ void tail_jacobi(const TailCl<P>& cl, int l, const BoxK<P>& V, int sweeps, P omega) {
  const int n0 = V.n0, n1 = V.n1;
  for (int sw = 0; sw < sweeps; sw++) {
    P nv[8];
    int cnt = 0;
    cl_for3(cl, n0, n1, V.n2, [&](int i, int j, int k) {
      P dg, of;
      box_row<P, false>(V, V.A, V.e, i, j, k, dg, of);
      const int idx = i + n0 * (j + n1 * k);
      if (cnt < 8) nv[cnt] = V.e[idx] + omega * ((V.f[idx] + of) / dg - V.e[idx]);
      cnt++;
    });
    cl.sync();
    cnt = 0;
    cl_for3(cl, n0, n1, V.n2, [&](int i, int j, int k) {
      if (cnt < 8) cl.put_e(l, k, V.e + i + n0 * (j + n1 * k), nv[cnt]);
      cnt++;
    });
    cl.sync();
  }
}

// red-black sweeps, each thread over x-pairs of its CTA's planes (or damped
// Jacobi sweeps); a pass reads only the other colour, so its writes can go
// out while it runs
template <class P>
__device__ void tail_smooth(const TailCl<P>& cl, const TailArgs<P>& a, int l, const BoxK<P>& V,
                            int sweeps, bool red_first) {
  if (a.jacobi) {
    tail_jacobi(cl, l, V, sweeps, a.omega);
    return;
  }
  const int n0 = V.n0, n1 = V.n1;
  const int hx = (n0 + 1) >> 1;
  for (int sw = 0; sw < sweeps; sw++)
    for (int pass = 0; pass < 2; pass++) {
      const int colour = red_first ? pass : 1 - pass;
      cl_for3(cl, hx, n1, V.n2, [&](int px, int j, int k) {
        const int i = 2 * px + ((j + k + colour) & 1);
        if (i >= n0) return;
        P dg, of;
        box_row<P, false>(V, V.A, V.e, i, j, k, dg, of);
        const int idx = i + n0 * (j + n1 * k);
        cl.put_e(l, k, V.e + idx, (V.f[idx] + of) / dg);
      });
      cl.sync();
    }
}

// dst[0, n) = src[0, n) by one CTA, 8 loads in flight per thread
template <class P>
__device__ void cta_copy(P* dst, const P* __restrict__ src, int n) {
  const int bd = blockDim.x;
  int q = threadIdx.x;
  for (; q + 7 * bd < n; q += 8 * bd) {
    P v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) v[u] = src[q + u * bd];
#pragma unroll
    for (int u = 0; u < 8; u++) dst[q + u * bd] = v[u];
  }
  for (; q < n; q += bd) dst[q] = src[q];
}

// grid: 2 clusters of C CTAs (field = cluster; C a power of 2), launched
// with cluster dimension C (C = 1: one CTA per field)
template <class P>
__global__ void __launch_bounds__(kTailThreads) k_box_tail(TailArgs<P> a) {
  extern __shared__ __align__(16) unsigned char tail_raw[];
  __shared__ P* s_rb[kTailClusterMax];
  P* sm = reinterpret_cast<P*>(tail_raw);
  cg::cluster_group cluster = cg::this_cluster();
  TailCl<P> cl;
  cl.sm = sm;
  cl.rb = s_rb;
  cl.C = (int)cluster.num_blocks();
  cl.r = (int)cluster.block_rank();
  cl.lgC = 31 - __clz(cl.C);
  const int fld = blockIdx.x / cl.C;
  if (threadIdx.x < cl.C) s_rb[threadIdx.x] = cluster.map_shared_rank(sm, (int)threadIdx.x);
  __shared__ uint8_t s_me[kTailPlanes], s_mf[kTailPlanes];
  const int npl = a.pb[a.nlev];
  cl.pb = a.pb;
  cl.me = (cl.C > 1 && npl <= kTailPlanes) ? s_me : nullptr;
  cl.mf = cl.me ? s_mf : nullptr;
  if (cl.me) {
    for (int q = threadIdx.x; q < npl; q += blockDim.x) {
      int X = 0;
      while (q >= a.pb[X + 1]) X++;
      const int p = q - a.pb[X];
      unsigned me = 0u, mf = 0u;
      for (int rr = 0; rr < cl.C; rr++) {
        int o0, o1;
        cl.own(a.B[X].n[2], rr, o0, o1);
        if (o0 < o1 && p >= o0 - 1 && p <= o1) me |= 1u << rr;
        if (p >= o0 && p < o1) mf |= 1u << rr;
        if (X + 1 < a.nlev) {
          int c0, c1;
          cl.own(a.B[X + 1].n[2], rr, c0, c1);
          if (c0 < c1 && p >= 2 * c0 - 1 && p <= 2 * c1) me |= 1u << rr;
          if (c0 < c1 && p >= 2 * c0 && p < 2 * c1) mf |= 1u << rr;
        }
        if (X > 0) {
          int f0, f1;
          cl.own(a.B[X - 1].n[2], rr, f0, f1);
          if (f0 < f1 && p >= (f0 >> 1) - 1 && p <= ((f1 - 1) >> 1) + 1) me |= 1u << rr;
        }
      }
      s_me[q] = (uint8_t)me;
      s_mf[q] = (uint8_t)mf;
    }
  }
  for (int l = 0; l < a.nlev; l++) {
    const BoxRaw& B = a.B[l];
    cta_copy(sm + a.offA[l], a.A[l] + fld * B.AF, (int)B.AF);
    const int nc = B.n[0] * B.n[1] * B.n[2];
    for (int q = threadIdx.x; q < nc; q += blockDim.x) sm[a.offE[l] + q] = P(0);
  }
  cta_copy(sm + a.offF[0], a.f0 + fld * a.vfs0, a.B[0].n[0] * a.B[0].n[1] * a.B[0].n[2]);
  // every replica initialised (and every CTA of the cluster running) before
  // the first remote write
  cl.sync();
  // down: smooth, restrict (8-cell average of f - L e; after a red-first
  // sweep the black children's residual is zero)
  for (int l = 0; l + 1 < a.nlev; l++) {
    BoxK<P> V = tail_view(a, sm, l);
    tail_smooth(cl, a, l, V, a.nu1, true);
    const BoxRaw& C = a.B[l + 1];
    const int c0 = C.n[0], c1 = C.n[1];
    const bool black0 = a.nu1 > 0 && !a.jacobi;
    P* fc = sm + a.offF[l + 1];
    cl_for3(cl, c0, c1, C.n[2], [&](int ci, int cj, int ck) {
      P s = P(0);
      for (int q = 0; q < 8; q++) {
        const int x = q & 1, y = (q >> 1) & 1, z = q >> 2;
        if (black0 && ((x + y + z) & 1)) continue;
        const int i = 2 * ci + x, j = 2 * cj + y, k = 2 * ck + z;
        const int idx = i + V.n0 * (j + V.n1 * k);
        P dg, of;
        box_row<P, false>(V, V.A, V.e, i, j, k, dg, of);
        s += V.f[idx] - (dg * V.e[idx] - of);
      }
      cl.put_f(l + 1, ck, fc + ci + c0 * (cj + c1 * ck), s / P(8));
    });
    cl.sync();
  }
  tail_smooth(cl, a, a.nlev - 1, tail_view(a, sm, a.nlev - 1), a.csw, true);
  // up: trilinear prolongation of the coarse correction, smooth
  for (int l = a.nlev - 2; l >= 0; l--) {
    BoxK<P> V = tail_view(a, sm, l);
    const BoxRaw& C = a.B[l + 1];
    const P* src = sm + a.offE[l + 1];
    cl_for3(cl, V.n0, V.n1, V.n2, [&](int i, int j, int k) {
      P* pe = V.e + i + V.n0 * (j + V.n1 * k);
      cl.put_e(l, k, pe,
               *pe + tri_interp(src, C.n[0], C.n[1], C.n[2], i, j, k, (const int*)nullptr));
    });
    cl.sync();
    tail_smooth(cl, a, l, V, a.nu2, false);
  }
  // every replica is complete: each CTA stores its planes of level 0
  const BoxRaw& B0 = a.B[0];
  cl_for3(cl, B0.n[0], B0.n[1], B0.n[2], [&](int i, int j, int k) {
    const int q = i + B0.n[0] * (j + B0.n[1] * k);
    a.e0[fld * a.vfs0 + q] = sm[a.offE[0] + q];
  });
}

template <class P>
void run_tail(PcState* ps, cudaStream_t s) {
  TailArgs<P> a;
  const int m0 = ps->tail_m;
  a.nlev = ps->nmg - m0;
  int off = 0;
  for (int l = 0; l < a.nlev; l++) {
    const BoxRaw& B = ps->box[m0 + l];
    const int nc = B.n[0] * B.n[1] * B.n[2];
    a.B[l] = B;
    a.A[l] = (const P*)ps->bA[m0 + l];
    a.offA[l] = off;
    off += (int)B.AF;
    a.offE[l] = off;
    off += nc;
    a.offF[l] = off;
    off += nc;
  }
  a.pb[0] = 0;
  for (int l = 0; l < a.nlev; l++) a.pb[l + 1] = a.pb[l] + ps->box[m0 + l].n[2];
  a.f0 = (const P*)ps->bf[m0];
  a.e0 = (P*)ps->be[m0];
  a.vfs0 = ps->box[m0].n[0] * ps->box[m0].n[1] * ps->box[m0].n[2];
  a.nu1 = ps->nu1;
  a.nu2 = ps->nu2;
  a.csw = ps->csw;
  a.jacobi = ps->smoother == NRD_SMOOTH_JACOBI;
  a.omega = (P)ps->omega;
  const int C = std::max(1, ps->tail_cl);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * C);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = ps->tail_smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_box_tail<P>, a);
}

template <class P>
VLev<P> vlev(PcState* ps, const Hier& H) {
  VLev<P> V;
  V.vt = ps->vt;
  V.patches = H.d_patches;
  V.mask = H.d_mask;
  V.gsrc = ps->gsrc;
  V.gidx = H.d_gidx;
  V.gw = (const P*)ps->gwp;
  V.A = (const P*)ps->A;
  V.Afs = ps->AF;
  V.N = H.N;
  V.G = H.G;
  return V;
}

// u += e on the uncovered cells of level l (used when no pass of the level
// could do it)
template <class P>
void add_level(PcState* ps, const Hier& H, int l, cudaStream_t s) {
  const LevelInfo& Lv = H.lev[l];
  dim3 g(g1(Lv.ncell), 2);
  k_add_leaf<P><<<g, BS, 0, s>>>(H.d_mask, Lv.off, Lv.ncell, H.N, (const P*)ps->fe, (P*)ps->fu);
}

// GMG V-cycle on box level m (m = 0: AMR level 0 inside the hierarchy
// vectors).  Every level's correction starts from zero; on level 0 the last
// pass also adds the correction to the composite solution.
template <class P>
void gmg_vcycle(PcState* ps, const Hier& H, int m, cudaStream_t s) {
  if (m > 0 && m == ps->tail_m && ps->smoother != NRD_SMOOTH_LINE) {
    run_tail<P>(ps, s);
    return;
  }
  const BoxRaw B = (m == 0) ? level0_box(H) : ps->box[m];
  const void* A = (m == 0) ? ps->A : ps->bA[m];
  void* e = (m == 0) ? ps->fe : ps->be[m];
  const void* f = (m == 0) ? ps->fr : ps->bf[m];
  const long nc = (long)B.n[0] * B.n[1] * B.n[2];
  const long vfs = (m == 0) ? H.N : nc;
  const BoxK<P> V = boxk<P>(B, A, e, f, vfs);
  const uint8_t* mask = (m == 0) ? H.d_mask : nullptr;
  // one level: the level-0 correction is the V-cycle's result (read from fe),
  // no composite solution to add it to
  P* addu = (m == 0 && H.L > 1) ? (P*)ps->fu : nullptr;
  auto zero_e = [&]() {
    for (int fld = 0; fld < 2; fld++)
      cudaMemsetAsync((char*)e + fld * vfs * (long)sizeof(P), 0, nc * sizeof(P), s);
  };
  const bool jac = ps->smoother == NRD_SMOOTH_JACOBI;
  const P omega = (P)ps->omega;
  P* scratch = (P*)((m == 0) ? ps->fj : ps->bj[m]);
  if (m == ps->nmg - 1) {
    if (ps->csw == 0) zero_e();   // no correction
    else if (jac) box_jacobi(V, omega, scratch, ps->csw, true, false, mask, addu, s);
    else rb_sweeps<P>(ps, m, V, scratch, ps->csw, 0, true, false, mask, addu, s);
    return;
  }
  if (ps->nu1 == 0) zero_e();
  else if (jac) box_jacobi(V, omega, scratch, ps->nu1, true, false, nullptr, (P*)nullptr, s);
  else rb_sweeps<P>(ps, m, V, scratch, ps->nu1, 0, true, false, nullptr, (P*)nullptr, s);
  const BoxRaw& C = ps->box[m + 1];
  const dim3 gc = restrict_grid(C.n[0], C.n[1], C.n[2]);
  // after a red-first point Gauss-Seidel sweep the black residuals are zero
  if (ps->nu1 > 0 && !jac && ps->smoother != NRD_SMOOTH_LINE)
    k_brestrict<P, true><<<gc, VTHREADS, 0, s>>>(V, (P*)ps->bf[m + 1], C.n[0], C.n[1], C.n[2]);
  else
    k_brestrict<P, false><<<gc, VTHREADS, 0, s>>>(V, (P*)ps->bf[m + 1], C.n[0], C.n[1], C.n[2]);
  gmg_vcycle<P>(ps, H, m + 1, s);
  // e + P e_c: into the scratch when an odd number of sweeps follows, so
  // that the last one writes e
  const bool to_scratch =
      (jac || fused_sweeps<P>(ps, m)) && ps->nu2 > 0 && start_in_scratch(ps->nu2);
  k_bprolong<P><<<dim3((C.n[0] + PX - 1) / PX, (C.n[1] + PY - 1) / PY,
                       2 * ((C.n[2] + PZ - 1) / PZ)), PX * PY * PZ, 0, s>>>(
      (const P*)ps->be[m + 1], C.n[0], C.n[1], C.n[2], V, to_scratch ? scratch : V.e);
  if (ps->nu2 == 0) {
    if (m == 0 && H.L > 1) add_level<P>(ps, H, 0, s);
  } else if (jac) {
    box_jacobi(V, omega, scratch, ps->nu2, false, to_scratch, mask, addu, s);
  } else {
    rb_sweeps<P>(ps, m, V, scratch, ps->nu2, 1, false, to_scratch, mask, addu, s);
  }
}

// Grid of the AMR-level kernels, which loop over their tiles with a grid
// stride: at most per_sm blocks per SM, so that a warp done with one tile
// starts the loads of its next one instead of waiting for its block to be
// replaced.  Measured on a 3-level hierarchy of 1,913 patches (45.6M cells),
// against one block per tile: the composite residual best at 32 per SM, the
// point Jacobi sweep and the prolongation at 16, the red-black pass at 32
// (a V(1,0) Jacobi apply 5.6 -> 4.2 ms, a V(1,1) red-black one 10.7 -> 8.6).
inline int level_grid(const PcState* ps, int ntiles, int per_sm) {
  return std::max(1, std::min(ntiles, per_sm * ps->nsm));
}

// r = ff - L^c fu on the leaf cells of levels lmin and finer; flux matching;
// covered cells of those levels := mean of their children.  The caller
// needs the residual on levels >= lmin only (a level's covered cells take
// the means of the finer levels): lmin = l - 1 before smoothing level l - 1
// on the down-leg, lmin = l before smoothing level l on the up-leg, which on
// the finest level leaves one sweep over that level's tiles.
// With zero_base (lmin = 0, on the down-leg) the correction is still zero on
// the base level, which has no coarse-fine ghosts: there L u = 0, so the
// residual of its uncovered cells is the rhs that fr already holds, and only
// the flux matching (the fine fluxes at its coarse-fine faces) and the
// covered means change it.  That needs fr = ff on the base level's uncovered
// cells, which holds because flux matching only touches levels >= lmin.  (A
// finer level has no such shortcut: its coarse-fine ghosts interpolate
// composite values of covered coarse cells, i.e. means of finer values.)
template <class P>
void composite_residual(PcState* ps, const Hier& H, int lmin, cudaStream_t s,
                        bool zero_base = false) {
  const VLev<P> V = vlev<P>(ps, H);
  const int t0 = ps->vt0[(zero_base && lmin == 0) ? 1 : lmin];
  VLev<P> Vs = V;
  Vs.vt = V.vt + t0;
  if (ps->ntile > t0)
    k_cresid<P><<<level_grid(ps, ps->ntile - t0, 32), FTHREADS, 0, s>>>(
        ps->ntile - t0, Vs, (const P*)ps->fu, (const P*)ps->ff, (P*)ps->fr, (P*)ps->cf);
  if (H.L < 2 || lmin > H.L - 2) return;
  const int lc = H.L - 2;
  // flux matching of the coarse cells on levels >= lmin only (the levels
  // below are not read before the next residual that covers them)
  const int r0 = H.rf_lstart[lmin];
  const int nrf = H.nrf - r0;
  const int n = nrf + H.ncov[lc];
  if (n)
    k_reflux_avg<P><<<dim3(g1(n), 2), BS, 0, s>>>(H.d_rf_cell + r0, H.d_rf_off + r0, H.d_rf_g,
                                                  nrf, H.d_cov[lc], H.ncov[lc], H.N, H.G,
                                                  (const P*)ps->cf, (P*)ps->fr);
  for (int l = H.L - 3; l >= lmin; l--) {
    if (!H.ncov[l]) continue;
    dim3 ga(g1(H.ncov[l]), 2);
    k_avgdown_p<P><<<ga, BS, 0, s>>>(H.d_cov[l], H.ncov[l], (P*)ps->fr, H.N);
  }
}

// the level-l correction (already added on level l) interpolated to every
// finer level and added on its uncovered cells
template <class P>
void prolong_finer(PcState* ps, const Hier& H, int l, cudaStream_t s) {
  const VLev<P> V = vlev<P>(ps, H);
  const void* src = ps->fe;
  for (int m = l + 1; m < H.L; m++) {
    const LevelInfo& Lc = H.lev[m - 1];
    const dim3 gs(level_grid(ps, ps->vnt[m], 16));
    if (m + 1 < H.L)
      k_vprolong<P, true><<<gs, FTHREADS, 0, s>>>(ps->vnt[m], V, ps->vt0[m], H.d_lmap[m - 1],
                                                  Lc.n[0], Lc.n[1], Lc.n[2], (const P*)src,
                                                  (P*)ps->fp, (P*)ps->fu);
    else
      k_vprolong<P, false><<<gs, FTHREADS, 0, s>>>(ps->vnt[m], V, ps->vt0[m], H.d_lmap[m - 1],
                                                   Lc.n[0], Lc.n[1], Lc.n[2], (const P*)src,
                                                   (P*)ps->fp, (P*)ps->fu);
    src = ps->fp;
  }
}

// sweeps > 0 red-black sweeps of the level-l error equation from e = 0; the
// last pass adds e to the composite solution
template <class P>
void level_smooth(PcState* ps, const Hier& H, int l, int sweeps, bool red_first, cudaStream_t s) {
  if (ps->smoother == NRD_SMOOTH_JACOBI) {
    // from zero; the first sweep writes whichever of fe / fj makes the last
    // land in fe, which also adds the correction to the composite solution
    const VLev<P> V = vlev<P>(ps, H);
    const int ntl = ps->vnt[l];
    const dim3 gs(level_grid(ps, ntl, 16));
    const int t0 = ps->vt0[l];
    const P omega = (P)ps->omega;
    P* buf[2] = {(P*)ps->fe, (P*)ps->fj};
    const P* f = (const P*)ps->fr;
    P* u = (P*)ps->fu;
    int cur = ((sweeps - 1) % 2 == 0) ? 0 : 1;
    for (int sw = 0; sw < sweeps; sw++) {
      const bool D = sw == sweeps - 1;
      if (sw == 0) {
        if (D) k_ljacobi<P, true, true><<<gs, FTHREADS, 0, s>>>(ntl, V, t0, omega, nullptr, buf[cur], f, u);
        else k_ljacobi<P, true, false><<<gs, FTHREADS, 0, s>>>(ntl, V, t0, omega, nullptr, buf[cur], f, u);
        continue;
      }
      if (D) k_ljacobi<P, false, true><<<gs, FTHREADS, 0, s>>>(ntl, V, t0, omega, buf[cur], buf[1 - cur], f, u);
      else k_ljacobi<P, false, false><<<gs, FTHREADS, 0, s>>>(ntl, V, t0, omega, buf[cur], buf[1 - cur], f, u);
      cur = 1 - cur;
    }
    return;
  }
  const VLev<P> V = vlev<P>(ps, H);
  const int ntl = ps->vnt[l];
  const dim3 gs(level_grid(ps, ntl, 32));
  P* e = (P*)ps->fe;
  const P* f = (const P*)ps->fr;
  P* u = (P*)ps->fu;
  for (int sw = 0; sw < sweeps; sw++)
    for (int pass = 0; pass < 2; pass++) {
      const int colour = red_first ? pass : 1 - pass;
      const bool Z = sw == 0 && pass == 0;
      const bool D = sw == sweeps - 1 && pass == 1;
      if (Z) k_lsmooth<P, true, false><<<gs, VTHREADS, 0, s>>>(ntl, V, ps->vt0[l], colour, e, f, u);
      else if (D) k_lsmooth<P, false, true><<<gs, VTHREADS, 0, s>>>(ntl, V, ps->vt0[l], colour, e, f, u);
      else k_lsmooth<P, false, false><<<gs, VTHREADS, 0, s>>>(ntl, V, ps->vt0[l], colour, e, f, u);
    }
}

// y = P^{-1} w.  With jd non-null (forward only) w and y are bases of
// columns jstride apart and the column *jd (a device index) is used; y2, if
// non-null, receives a second copy of the result.
template <class P>
int apply_t(PcState* ps, const Hier& H, const double* w, double* y, bool transposed,
            cudaStream_t s, const int* jd = nullptr, long jstride = 0, double* y2 = nullptr) {
  // r = f (u = 0).  The covered cells' residual is not averaged down here:
  // the finest level has none, and every coarser level's covered cells are
  // re-averaged by the down-leg composite residual that precedes its smoothing
  // one level: the V-cycle is the GMG cycle on level 0 alone, whose rhs is fr
  // and whose correction (fe) is the result; the composite rhs ff and solution
  // fu are neither written nor read
  const bool one = H.L == 1;
  P* ffp = one ? nullptr : (P*)ps->ff;
  if (transposed)
    k_vc_init<P, true><<<g1(H.N), BS, 0, s>>>(H.N, w, (const P*)ps->p2, ffp, (P*)ps->fr,
                                              (P*)ps->fu, nullptr, 0);
  else
    k_vc_init<P, false><<<g1(H.N), BS, 0, s>>>(H.N, w, (const P*)ps->p2, ffp, (P*)ps->fr,
                                               (P*)ps->fu, jd, jstride);
  // down: finest to level 1 (no sweeps: a zero correction)
  for (int l = H.L - 1; l >= 1; l--) {
    if (ps->nu1 > 0) {
      level_smooth<P>(ps, H, l, ps->nu1, true, s);
      prolong_finer<P>(ps, H, l, s);
    }
    composite_residual<P>(ps, H, l - 1, s, l == 1);
  }
  gmg_vcycle<P>(ps, H, 0, s);
  prolong_finer<P>(ps, H, 0, s);
  // up: level 1 to finest (without post-smoothing nothing reads the
  // up-leg residuals: the correction is complete after the coarse solve's
  // prolongation)
  for (int l = 1; l < H.L && ps->nu2 > 0; l++) {
    composite_residual<P>(ps, H, l, s);
    level_smooth<P>(ps, H, l, ps->nu2, false, s);
    prolong_finer<P>(ps, H, l, s);
  }
  const P* res = (const P*)(one ? ps->fe : ps->fu);
  if (transposed)
    k_out_cast<P><<<g1(H.N), BS, 0, s>>>(H.d_mask, H.N, res, y, ps->d_err);
  else
    k_p2<P><<<g1(H.N), BS, 0, s>>>(H.N, res, (const P*)ps->p2, y, jd, jstride, y2,
                                   ps->d_err);
  return cudaGetLastError() == cudaSuccess ? NRD_OK : NRD_ECUDA;
}

template <class P>
void scale_all(PcState* ps, const Hier& H, SetupArgs& a, cudaStream_t s) {
  int nt = (int)H.tiles.size();
  dim3 gt(std::min(nt, 152 * 8), 2);
  k_scale_hier<P><<<gt, BS, 0, s>>>(a, nullptr, (P*)ps->A);
}

}  // namespace

// cuTensorMapEncodeTiled of the CUDA driver API, found through the runtime's
// entry-point query (no link to libcuda); null when the installed CUDA driver
// does not offer it
using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;
EncodeFn tmap_encoder() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

// tensor map of an FP32 n0 x n1 x n2 array (x fastest) at base, with a
// TBX x by x bz box; false when TMA cannot address it (base or row stride
// not 16-byte aligned) or the encoding is refused
bool tmap3(CUtensorMap* m, const float* base, const int n[3], int by, int bz) {
  EncodeFn enc = tmap_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) || (n[0] % 4) != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2]};
  cuuint64_t strides[2] = {(cuuint64_t)n[0] * 4, (cuuint64_t)n[0] * n[1] * 4};
  cuuint32_t box[3] = {(cuuint32_t)TBX, (cuuint32_t)by, (cuuint32_t)bz};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tensor maps of FP32 box level m for k_bsweep (levels of at least 32 x 8 x 8
// cells; the smaller ones keep the two-pass kernel)
void setup_sweep_maps(PcState* ps, const Hier& H, int m) {
  ps->tma_ok[m] = false;
  if (ps->prec != NRD_PC_F32) return;
  const BoxRaw B = (m == 0) ? level0_box(H) : ps->box[m];
  if (B.n[0] < 32 || B.n[1] < 8 || B.n[2] < 8) return;
  const long vfs = (m == 0) ? H.N : (long)B.n[0] * B.n[1] * B.n[2];
  const float* e = (const float*)((m == 0) ? ps->fe : ps->be[m]);
  const float* sc = (const float*)((m == 0) ? ps->fj : ps->bj[m]);
  const float* f = (const float*)((m == 0) ? ps->fr : ps->bf[m]);
  const float* A = (const float*)((m == 0) ? ps->A : ps->bA[m]);
  bool ok = true;
  for (int fld = 0; fld < 2 && ok; fld++) {
    ok = tmap3(&ps->tm_e[m][0][fld], e + fld * vfs, B.n, SY + 4, SZ + 4) &&
         tmap3(&ps->tm_e[m][1][fld], sc + fld * vfs, B.n, SY + 4, SZ + 4) &&
         tmap3(&ps->tm_f[m][fld], f + fld * vfs, B.n, SY + 2, SZ + 2) &&
         tmap3(&ps->tm_a[m][0][fld], A + fld * B.AF, B.n, SY + 2, SZ + 2) &&
         tmap3(&ps->tm_a[m][1][fld], A + fld * B.AF + B.NA, B.n, SY + 3, SZ + 2) &&
         tmap3(&ps->tm_a[m][2][fld], A + fld * B.AF + 2 * B.NA, B.n, SY + 2, SZ + 3);
  }
  ps->tma_ok[m] = ok;
}

int pc_alloc(PcState** out, const Hier& H, const nrd_params& p, std::string& err) {
  PcState* ps = new PcState();
  ps->prec = p.pc_precision;
  ps->esz = (ps->prec == NRD_PC_F32) ? 4 : 8;
  ps->nmg = p.nmg;
  ps->nu1 = p.nu1;
  ps->nu2 = p.nu2;
  ps->csw = p.coarse_sweeps;
  ps->smoother = p.smoother;
  ps->omega = p.omega;
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
  if (ps->AF >= (1L << 31)) {
    err = "hierarchy too large for the V-cycle's 32-bit indices (3N + G >= 2^31)";
    delete ps;
    return NRD_EINVAL;
  }
  size_t e = ps->esz;
  bool ok = cudaMalloc(&ps->Craw, 2 * ps->AF * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ps->A, 2 * ps->AF * e) == cudaSuccess &&
            cudaMalloc(&ps->fu, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->fr, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->fe, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->fp, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->fj, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->ff, 2 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->gh, 2 * std::max(G, 1L) * e) == cudaSuccess &&
            cudaMalloc(&ps->cf, 2 * std::max(G, 1L) * e) == cudaSuccess &&
            cudaMalloc(&ps->Tk, N * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ps->bgt, 6 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&ps->d_beta, sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ps->p2, 3 * N * e) == cudaSuccess &&
            cudaMalloc(&ps->gsrc, std::max(G, 1L) * sizeof(int2)) == cudaSuccess &&
            cudaMalloc(&ps->gwp, std::max(H.nterm, 1) * e) == cudaSuccess &&
            cudaStreamCreateWithFlags(&ps->cap, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) {
    cudaMemset(ps->Craw, 0, 2 * ps->AF * sizeof(double));
    cudaMemset(ps->A, 0, 2 * ps->AF * e);
    cudaMemset(ps->gh, 0, 2 * std::max(G, 1L) * e);
    cudaMemset(ps->cf, 0, 2 * std::max(G, 1L) * e);
    int bt[6];
    for (int f = 0; f < 6; f++) bt[f] = (H.bc_type[f] == NRD_BC_ROBIN) ? 1 : 0;
    cudaMemcpy(ps->bgt, bt, sizeof bt, cudaMemcpyHostToDevice);
    if (G) {
      if (ps->prec == NRD_PC_F32)
        k_vc_ghosts<float><<<g1(G), BS>>>(H.d_gtype, H.d_gt0, H.d_gidx, (int)G, H.d_gw, H.nterm,
                                          ps->gsrc, (float*)ps->gwp);
      else
        k_vc_ghosts<double><<<g1(G), BS>>>(H.d_gtype, H.d_gt0, H.d_gidx, (int)G, H.d_gw, H.nterm,
                                           ps->gsrc, (double*)ps->gwp);
    }
    // V-cycle tiles: 8^3 blocks of every patch, level by level; a tile all
    // of whose cells are covered is flagged (no composite residual there)
    std::vector<int4> vt;
    for (int l = 0; l < H.L; l++) {
      const LevelInfo& Lv = H.lev[l];
      ps->vt0[l] = (int)vt.size();
      for (int p = Lv.p0; p < Lv.p0 + Lv.np; p++) {
        const PatchDev& Q = H.patches[p];
        for (int k0 = 0; k0 < Q.n[2]; k0 += VT)
          for (int j0 = 0; j0 < Q.n[1]; j0 += VT)
            for (int i0 = 0; i0 < Q.n[0]; i0 += VT) {
              bool all = true;
              for (int k = k0; k < std::min(k0 + VT, Q.n[2]) && all; k++)
                for (int j = j0; j < std::min(j0 + VT, Q.n[1]) && all; j++)
                  for (int i = i0; i < std::min(i0 + VT, Q.n[0]) && all; i++)
                    if (!(H.hmask[Q.off + i + Q.n[0] * (j + Q.n[1] * k)] & MASK_COVERED))
                      all = false;
              vt.push_back(make_int4(p | (all ? kTileCovered : 0), i0, j0, k0));
            }
      }
      ps->vnt[l] = (int)vt.size() - ps->vt0[l];
    }
    ps->ntile = (int)vt.size();
    ok = cudaMalloc(&ps->vt, vt.size() * sizeof(int4)) == cudaSuccess &&
         cudaMemcpy(ps->vt, vt.data(), vt.size() * sizeof(int4), cudaMemcpyHostToDevice) ==
             cudaSuccess;
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
    ok = cudaMalloc(&ps->bA[m], 2 * B.AF * e) == cudaSuccess &&
         cudaMalloc(&ps->be[m], 2 * nc * e) == cudaSuccess &&
         cudaMalloc(&ps->bj[m], 2 * nc * e) == cudaSuccess &&
         cudaMalloc(&ps->bf[m], 2 * nc * e) == cudaSuccess;
    if (ok) {
      cudaMemset(ps->bA[m], 0, 2 * B.AF * e);
    }
  }
  if (ok) ok = cudaMalloc(&ps->d_err, sizeof(int)) == cudaSuccess &&
               cudaMemset(ps->d_err, 0, sizeof(int)) == cudaSuccess;
  if (!ok) {
    pc_free(ps);
    err = "preconditioner allocation failed";
    return NRD_ENOMEM;
  }
  // the one-launch red-black sweep on the FP32 box levels TMA can address
  // (attributes set here, outside any stream capture)
  if (ps->prec == NRD_PC_F32) {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&ps->nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_bsweep<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SWEEP_SMEM);
    cudaFuncSetAttribute(k_bsweep<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SWEEP_SMEM);
    cudaFuncSetAttribute(k_bsweep<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SWEEP_SMEM);
    cudaFuncSetAttribute(k_bsweep<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SWEEP_SMEM);
    for (int m = 0; m < ps->nmg; m++) setup_sweep_maps(ps, H, m);
  }
  // the coarsest box levels whose data fit one CTA's shared memory run as
  // one kernel (the first such level with at most 8,192 cells per field),
  // one thread-block cluster per field; FP32 V-cycles only: the few SMs'
  // FP64 rate is too low for it
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
    // the largest cluster (up to kTailClusterMax CTAs, one per SM) that can be resident
    ps->tail_cl = 1;
    for (int C = kTailClusterMax; C > 1; C /= 2) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(2 * C);
      cfg.blockDim = dim3(kTailThreads);
      cfg.dynamicSmemBytes = ps->tail_smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, k_box_tail<float>, &cfg) == cudaSuccess &&
          ncl >= 1) {
        ps->tail_cl = C;
        break;
      }
      cudaGetLastError();   // clear a refused query
    }
  }
  *out = ps;
  return NRD_OK;
}

void pc_drop_graphs(PcState* ps);

void pc_free(PcState* ps) {
  if (!ps) return;
  auto F = [](void* p) { if (p) cudaFree(p); };
  F(ps->Craw); F(ps->A); F(ps->fu); F(ps->fr); F(ps->fe); F(ps->fp); F(ps->fj); F(ps->ff); F(ps->gh);
  F(ps->cf); F(ps->Tk); F(ps->bgt); F(ps->d_beta); F(ps->p2); F(ps->vt); F(ps->gsrc); F(ps->gwp);
  F(ps->d_err);
  pc_drop_graphs(ps);
  if (ps->cap) cudaStreamDestroy(ps->cap);
  for (int m = 0; m < NRD_MAX_MG; m++) {
    F(ps->bA[m]); F(ps->be[m]); F(ps->bj[m]); F(ps->bf[m]);
  }
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
      a.lh.r2[l][d] = 1.0 / (a.lh.h[l][d] * a.lh.h[l][d]);
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

template <class P>
void coarsen_all(PcState* ps, bool scaled, cudaStream_t s) {
  CoarsenAll<P> a;
  a.nlev = ps->nmg - 1;
  a.F = ps->box[0];
  // items of level m: [item0[m], item0[m - 1]), item0[nlev] = 0, item0[0] = all
  a.item0[ps->nmg - 1] = 0;
  for (int m = ps->nmg - 1; m >= 1; m--) {
    a.C[m] = ps->box[m];
    a.A[m] = (P*)ps->bA[m];
    for (int d = 0; d < 3; d++) a.h[m][d] = ps->bh[m][d];
    a.item0[m - 1] = a.item0[m] + 3 * ps->box[m].n[0] * ps->box[m].n[1] * ps->box[m].n[2];
  }
  const dim3 g(g1(a.item0[0]), 2);
  if (scaled)
    k_box_coarsen<P, true><<<g, BS, 0, s>>>(a, ps->Craw, (const P*)ps->A, ps->bgt, ps->d_beta);
  else
    k_box_coarsen<P, false><<<g, BS, 0, s>>>(a, ps->Craw, (const P*)nullptr, ps->bgt,
                                             ps->d_beta);
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
      k_coef_coarsen<float, true><<<g, BS, 0, s>>>(H.d_cz_tgt[l], H.d_cz_src[l], H.ncz[l], ps->AF,
                                                   H.N, H.d_gtype, H.d_gface, ps->d_beta, a.lh,
                                                   l, ps->Craw, (float*)ps->A);
    else if (from_lin)
      k_coef_coarsen<double, true><<<g, BS, 0, s>>>(H.d_cz_tgt[l], H.d_cz_src[l], H.ncz[l],
                                                    ps->AF, H.N, H.d_gtype, H.d_gface,
                                                    ps->d_beta, a.lh, l, ps->Craw,
                                                    (double*)ps->A);
    else
      k_coef_coarsen<float, false><<<g, BS, 0, s>>>(H.d_cz_tgt[l], H.d_cz_src[l], H.ncz[l],
                                                    ps->AF, H.N, H.d_gtype, H.d_gface,
                                                    ps->d_beta, a.lh, l, ps->Craw,
                                                    (float*)nullptr);
  }
  // GMG levels, all from the base level in one launch
  if (ps->nmg > 1) {
    if (ps->prec == NRD_PC_F32) coarsen_all<float>(ps, from_lin, s);
    else coarsen_all<double>(ps, from_lin, s);
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

void pc_set_smoother(PcState* ps, int kind, double omega) {
  if (ps->smoother != kind || ps->omega != omega) pc_drop_graphs(ps);
  ps->smoother = kind;
  ps->omega = omega;
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
