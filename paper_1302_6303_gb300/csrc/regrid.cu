// Dynamic regridding (Sec. 5).
//
// nrd_regrid_boxes: Berger-Rigoutsos clustering of tagged cells into the
// boxes of a new hierarchy (host C++, off the stepping path).  Level by level
// from the coarsest: the cells of the new level l that carry a selected tag
// (a cell that does not exist on level l of the current hierarchy inherits
// the tag of the finest current cell that contains it) are dilated by
// `buffer` cells and kept only where a finer level can be properly nested
// (every level-l neighbour of the cell, inside the domain, belongs to the new
// level l).  The tagged set is clustered recursively:
//   shrink the box to the bounding box of its tags (drop it if none);
//   accept it when tags/volume >= efficiency, every cell may hold the finer
//   level, and no side exceeds max_side/2 cells;
//   otherwise cut it, trying in turn
//     (1) a zero of a tag signature (the count of tags per plane), axes taken
//         longest first, the zero nearest the middle (lower one on a tie);
//         the empty plane itself is dropped,
//     (2) the strongest sign change of the signature's second difference,
//         over all axes with at least 4 planes (first one on a tie),
//     (3) the middle of the longest side,
//   where a cut must leave both parts at least min_side/2 planes wide unless
//   the box holds cells that cannot take the finer level (then any cut is
//   allowed); a box that cannot be cut is accepted as it is.
// Accepted boxes, refined by 2, are the boxes of level l+1, in the order the
// recursion accepts them (lower part first).
//
// nrd_transfer: conservative limited-linear transfer of state vectors from an
// old to a new hierarchy (device gather, descriptor built on the host).  The
// old vectors are first made composite (covered cells := mean of their
// children).  A new cell that exists on the same level of the old hierarchy
// copies it; any other new cell evaluates, at its centre, the limited linear
// reconstruction of the old cell that contains it on the finest old level
// present there:
//   u = u_c + sum_d s_d (x_d - x_{c,d}) / h_{c,d},
//   s_d = minmod(u_c - u_{c-e_d}, u_{c+e_d} - u_c)  (0 if a neighbour is missing),
// whose mean over the children of the coarse cell is u_c (conservative) and
// which takes no value outside the neighbouring old values (no new extrema,
// so positivity is kept).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "nrd_internal.h"

namespace {

struct IBox {
  int lo[3], hi[3];
  long vol() const {
    return (long)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
  }
  int side(int d) const { return hi[d] - lo[d] + 1; }
};

struct Clusterer {
  const std::vector<uint8_t>& tag;   // dense level-l tags
  const std::vector<uint8_t>& ok;    // dense: cell may hold the finer level
  int n[3];
  double eff;
  int max_side, min_side;            // in level-l cells
  std::vector<IBox>& out;

  long at(int i, int j, int k) const { return i + (long)n[0] * (j + (long)n[1] * k); }

  bool shrink(IBox& b, long& cnt) const {
    int lo[3] = {b.hi[0], b.hi[1], b.hi[2]}, hi[3] = {b.lo[0], b.lo[1], b.lo[2]};
    cnt = 0;
    for (int k = b.lo[2]; k <= b.hi[2]; k++)
      for (int j = b.lo[1]; j <= b.hi[1]; j++)
        for (int i = b.lo[0]; i <= b.hi[0]; i++)
          if (tag[at(i, j, k)]) {
            cnt++;
            const int c[3] = {i, j, k};
            for (int d = 0; d < 3; d++) {
              lo[d] = std::min(lo[d], c[d]);
              hi[d] = std::max(hi[d], c[d]);
            }
          }
    if (!cnt) return false;
    for (int d = 0; d < 3; d++) {
      b.lo[d] = lo[d];
      b.hi[d] = hi[d];
    }
    return true;
  }

  bool all_ok(const IBox& b) const {
    for (int k = b.lo[2]; k <= b.hi[2]; k++)
      for (int j = b.lo[1]; j <= b.hi[1]; j++)
        for (int i = b.lo[0]; i <= b.hi[0]; i++)
          if (!ok[at(i, j, k)]) return false;
    return true;
  }

  void signature(const IBox& b, int d, std::vector<long>& sig) const {
    sig.assign(b.side(d), 0);
    for (int k = b.lo[2]; k <= b.hi[2]; k++)
      for (int j = b.lo[1]; j <= b.hi[1]; j++)
        for (int i = b.lo[0]; i <= b.hi[0]; i++)
          if (tag[at(i, j, k)]) {
            const int c[3] = {i, j, k};
            sig[c[d] - b.lo[d]]++;
          }
  }

  void run(IBox b) {
    long cnt;
    if (!shrink(b, cnt)) return;
    int longest = 0;
    for (int d = 1; d < 3; d++)
      if (b.side(d) > b.side(longest)) longest = d;
    const bool nested = all_ok(b);
    if (nested && b.side(longest) <= max_side && (double)cnt >= eff * (double)b.vol()) {
      out.push_back(b);
      return;
    }
    const int mn = nested ? std::max(1, min_side) : 1;
    const int order[3] = {longest, (longest + 1) % 3, (longest + 2) % 3};
    std::vector<long> sig;
    // (1) a hole of a signature: parts [lo, lo+i-1] and [lo+i+1, hi]
    for (int q = 0; q < 3; q++) {
      const int d = order[q], s = b.side(d), mid = s / 2;
      if (s < 3) continue;
      signature(b, d, sig);
      int best = -1, bestdist = 1 << 30;
      for (int i = 1; i + 1 < s; i++)
        if (sig[i] == 0 && i >= mn && s - 1 - i >= mn && std::abs(i - mid) < bestdist) {
          best = i;
          bestdist = std::abs(i - mid);
        }
      if (best >= 0) {
        IBox a = b, c = b;
        a.hi[d] = b.lo[d] + best - 1;
        c.lo[d] = b.lo[d] + best + 1;
        run(a);
        run(c);
        return;
      }
    }
    // (2) an inflection: parts [lo, lo+i] and [lo+i+1, hi]
    int sd = -1, cut = -1;
    long bestv = 0;
    for (int q = 0; q < 3; q++) {
      const int d = order[q], s = b.side(d);
      if (s < 4) continue;
      signature(b, d, sig);
      for (int i = 1; i + 2 < s; i++) {
        const long l1 = sig[i + 1] - 2 * sig[i] + sig[i - 1];
        const long l2 = sig[i + 2] - 2 * sig[i + 1] + sig[i];
        if ((l1 < 0) == (l2 < 0)) continue;
        if (i + 1 < mn || s - 1 - i < mn) continue;
        const long v = std::labs(l2 - l1);
        if (v > bestv) {
          bestv = v;
          sd = d;
          cut = i;
        }
      }
    }
    if (sd >= 0) {
      IBox a = b, c = b;
      a.hi[sd] = b.lo[sd] + cut;
      c.lo[sd] = b.lo[sd] + cut + 1;
      run(a);
      run(c);
      return;
    }
    // (3) bisection of the longest side: [lo, lo+s/2-1] and [lo+s/2, hi]
    const int s = b.side(longest);
    if (s >= 2 && s / 2 >= mn && s - s / 2 >= mn) {
      IBox a = b, c = b;
      a.hi[longest] = b.lo[longest] + s / 2 - 1;
      c.lo[longest] = b.lo[longest] + s / 2;
      run(a);
      run(c);
      return;
    }
    out.push_back(b);
  }
};

struct TransferDesc {
  int src;          // old cell (copy) or old coarse cell (reconstruction)
  int nb[6];        // old neighbours of src on its level (-1: none), x-, x+, y-, ...
  float off[3];     // (x - x_c) / h_c of the new cell centre per axis (exact in float)
};

__device__ __forceinline__ double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return (fabs(a) < fabs(b)) ? a : b;
}

__global__ void k_transfer(const TransferDesc* __restrict__ d, int N, int Nold, int nvec,
                           const double* __restrict__ uo, double* __restrict__ un) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const TransferDesc t = d[c];
    for (int f = 0; f < 2 * nvec; f++) {
      const double* u = uo + (long)f * Nold;
      const double uc = u[t.src];
      double v = uc;
      for (int a = 0; a < 3; a++) {
        const int im = t.nb[2 * a], ip = t.nb[2 * a + 1];
        if (im >= 0 && ip >= 0) v += minmod(uc - u[im], u[ip] - uc) * (double)t.off[a];
      }
      un[(long)f * N + c] = v;
    }
  }
}

}  // namespace

extern "C" {

int nrd_regrid_boxes(nrd_ctx* c, const uint8_t* tags, int tag_bits, int buffer,
                     double efficiency, int min_side, int max_side, int max_levels,
                     int max_boxes, int* nlevels_out, int* nboxes_out, int* boxes_out,
                     int* total_out) {
  if (!c) return NRD_EINVAL;
  if (!c->have_hier) {
    c->err = "no hierarchy";
    return NRD_ESTATE;
  }
  if (step_pending_check(c, false, nullptr)) return NRD_ESTATE;
  if (!tags || !nlevels_out || !nboxes_out || !boxes_out || !total_out || buffer < 0 ||
      !(efficiency > 0.0 && efficiency <= 1.0) || min_side < 2 || max_side < min_side ||
      (min_side % 2) || (max_side % 2) || max_levels < 1 || max_levels > NRD_MAX_LEVELS ||
      max_boxes < 1 || (tag_bits & 0xff) == 0) {
    c->err = "bad argument to nrd_regrid_boxes";
    return NRD_EINVAL;
  }
  const Hier& H = c->H;
  std::vector<uint8_t> htags(H.N);
  if (cudaMemcpy(htags.data(), tags, H.N, cudaMemcpyDeviceToHost) != cudaSuccess) {
    c->err = "copy of the tags failed";
    return NRD_ECUDA;
  }
  const int n0[3] = {H.lev[0].n[0], H.lev[0].n[1], H.lev[0].n[2]};
  // tag of the current cell (l, q), or -1 if the current hierarchy has none
  auto cur_tag = [&](int l, const int q[3]) -> int {
    if (l >= H.L) return -1;
    const LevelInfo& Lv = H.lev[l];
    const int ci = H.lmap[l][q[0] + (long)Lv.n[0] * (q[1] + (long)Lv.n[1] * q[2])];
    return ci < 0 ? -1 : ((htags[ci] & tag_bits) ? 1 : 0);
  };
  std::vector<std::vector<IBox>> levels(1);
  levels[0].push_back(IBox{{0, 0, 0}, {n0[0] - 1, n0[1] - 1, n0[2] - 1}});
  for (int l = 0; l + 1 < max_levels; l++) {
    const int n[3] = {n0[0] << l, n0[1] << l, n0[2] << l};
    const long lsize = (long)n[0] * n[1] * n[2];
    auto li = [&](int i, int j, int k) { return i + (long)n[0] * (j + (long)n[1] * k); };
    std::vector<uint8_t> in(lsize, 0), raw(lsize, 0), tg(lsize, 0), ok(lsize, 0);
    for (const IBox& b : levels[l])
      for (int k = b.lo[2]; k <= b.hi[2]; k++)
        for (int j = b.lo[1]; j <= b.hi[1]; j++)
          for (int i = b.lo[0]; i <= b.hi[0]; i++) {
            in[li(i, j, k)] = 1;
            int t = -1;
            for (int lc = std::min(l, H.L - 1); lc >= 0 && t < 0; lc--) {
              const int q[3] = {i >> (l - lc), j >> (l - lc), k >> (l - lc)};
              t = cur_tag(lc, q);
            }
            raw[li(i, j, k)] = t > 0 ? 1 : 0;
          }
    for (int k = 0; k < n[2]; k++)
      for (int j = 0; j < n[1]; j++)
        for (int i = 0; i < n[0]; i++) {
          if (!in[li(i, j, k)]) continue;
          bool nest = true;
          for (int dk = -1; dk <= 1 && nest; dk++)
            for (int dj = -1; dj <= 1 && nest; dj++)
              for (int di = -1; di <= 1 && nest; di++) {
                const int q[3] = {i + di, j + dj, k + dk};
                if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= n[0] || q[1] >= n[1] ||
                    q[2] >= n[2])
                  continue;
                if (!in[li(q[0], q[1], q[2])]) nest = false;
              }
          ok[li(i, j, k)] = nest ? 1 : 0;
          if (!nest) continue;
          bool hit = false;
          for (int dk = -buffer; dk <= buffer && !hit; dk++)
            for (int dj = -buffer; dj <= buffer && !hit; dj++)
              for (int di = -buffer; di <= buffer && !hit; di++) {
                const int q[3] = {i + di, j + dj, k + dk};
                if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= n[0] || q[1] >= n[1] ||
                    q[2] >= n[2])
                  continue;
                if (raw[li(q[0], q[1], q[2])]) hit = true;
              }
          tg[li(i, j, k)] = hit ? 1 : 0;
        }
    std::vector<IBox> coarse;
    Clusterer C{tg, ok, {n[0], n[1], n[2]}, efficiency, max_side / 2, min_side / 2, coarse};
    C.run(IBox{{0, 0, 0}, {n[0] - 1, n[1] - 1, n[2] - 1}});
    if (coarse.empty()) break;
    levels.emplace_back();
    for (const IBox& b : coarse) {
      IBox f;
      for (int d = 0; d < 3; d++) {
        f.lo[d] = 2 * b.lo[d];
        f.hi[d] = 2 * b.hi[d] + 1;
      }
      levels[l + 1].push_back(f);
    }
  }
  int total = 0;
  for (const auto& lv : levels) total += (int)lv.size();
  *total_out = total;
  *nlevels_out = (int)levels.size();
  if (total > max_boxes) {
    c->err = "the new hierarchy has more than max_boxes boxes";
    return NRD_EINVAL;
  }
  int q = 0;
  for (int l = 0; l < max_levels; l++) {
    nboxes_out[l] = l < (int)levels.size() ? (int)levels[l].size() : 0;
    if (l >= (int)levels.size()) continue;
    for (const IBox& b : levels[l]) {
      for (int d = 0; d < 3; d++) boxes_out[6 * q + d] = b.lo[d];
      for (int d = 0; d < 3; d++) boxes_out[6 * q + 3 + d] = b.hi[d];
      q++;
    }
  }
  return NRD_OK;
}

int nrd_transfer(nrd_ctx* src, nrd_ctx* dst, const double* u_src, double* u_dst, int nvec,
                 cudaStream_t s) {
  if (!src || !dst) return NRD_EINVAL;
  if (!src->have_hier || !dst->have_hier) {
    dst->err = "both contexts need a hierarchy";
    return NRD_ESTATE;
  }
  if (step_pending_check(src, false, nullptr) || step_pending_check(dst, false, nullptr))
    return NRD_ESTATE;
  if (!u_src || !u_dst || nvec < 1) {
    dst->err = "bad argument to nrd_transfer";
    return NRD_EINVAL;
  }
  const Hier& A = src->H;
  const Hier& B = dst->H;
  for (int d = 0; d < 3; d++)
    if (A.lev[0].n[d] != B.lev[0].n[d]) {
      dst->err = "the hierarchies have different base grids";
      return NRD_EINVAL;
    }
  auto old_cell = [&](int l, const int q[3]) -> int {
    if (l < 0 || l >= A.L) return -1;
    for (int d = 0; d < 3; d++)
      if (q[d] < 0 || q[d] >= A.lev[l].n[d]) return -1;
    return A.lmap[l][q[0] + (long)A.lev[l].n[0] * (q[1] + (long)A.lev[l].n[1] * q[2])];
  };
  std::vector<TransferDesc> desc(B.N);
  for (const PatchDev& P : B.patches) {
    const int l = P.level;
    for (int k = 0; k < P.n[2]; k++)
      for (int j = 0; j < P.n[1]; j++)
        for (int i = 0; i < P.n[0]; i++) {
          const int q[3] = {P.lo[0] + i, P.lo[1] + j, P.lo[2] + k};
          TransferDesc t;
          for (int f = 0; f < 6; f++) t.nb[f] = -1;
          for (int d = 0; d < 3; d++) t.off[d] = 0.0f;
          t.src = old_cell(l, q);
          if (t.src < 0) {
            int lc = std::min(l, A.L) - 1, cq[3] = {0, 0, 0};
            for (; lc >= 0; lc--) {
              for (int d = 0; d < 3; d++) cq[d] = q[d] >> (l - lc);
              if (old_cell(lc, cq) >= 0) break;
            }
            if (lc < 0) {
              dst->err = "transfer: a new cell lies in no old cell";
              return NRD_EINVAL;
            }
            t.src = old_cell(lc, cq);
            const int r = 1 << (l - lc);
            for (int d = 0; d < 3; d++) {
              // centre of the new cell relative to the old one, in old cells
              t.off[d] = (float)((2.0 * (q[d] - cq[d] * r) + 1.0 - r) / (2.0 * r));
              for (int sd = 0; sd < 2; sd++) {
                int nq[3] = {cq[0], cq[1], cq[2]};
                nq[d] += sd ? 1 : -1;
                t.nb[2 * d + sd] = old_cell(lc, nq);
              }
            }
          }
          desc[P.off + i + P.n[0] * (j + P.n[1] * k)] = t;
        }
  }
  const size_t No = (size_t)A.N, Nn = (size_t)B.N;
  TransferDesc* d_desc = nullptr;
  double* d_comp = nullptr;
  if (cudaMalloc(&d_desc, Nn * sizeof(TransferDesc)) != cudaSuccess ||
      cudaMalloc(&d_comp, 2 * No * nvec * sizeof(double)) != cudaSuccess) {
    cudaFree(d_desc);
    dst->err = "allocation failed";
    return NRD_ENOMEM;
  }
  cudaMemcpyAsync(d_desc, desc.data(), Nn * sizeof(TransferDesc), cudaMemcpyHostToDevice, s);
  dst->timer.begin(NRD_TK_TRANSFER, s);
  cudaMemcpyAsync(d_comp, u_src, 2 * No * nvec * sizeof(double), cudaMemcpyDeviceToDevice, s);
  launch_average_down(A, d_comp, 2 * nvec, (int)No, s);
  const int grid = (int)std::max(1L, std::min(152L * 8, ((long)Nn + 255) / 256));
  k_transfer<<<grid, 256, 0, s>>>(d_desc, (int)Nn, (int)No, nvec, d_comp, u_dst);
  dst->timer.end(NRD_TK_TRANSFER, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(d_desc);
  cudaFree(d_comp);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    dst->err = "transfer kernel failed";
    return NRD_ECUDA;
  }
  return NRD_OK;
}

}  // extern "C"
