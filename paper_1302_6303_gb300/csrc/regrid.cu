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
// old to a new hierarchy (device gather; the per-cell source list is built on
// host threads).  The
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
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
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

// One axis of a box filter of a dense 0/1 field of n[0] x n[1] x n[2] cells:
// v[c] := AND (MIN) or OR (!MIN) of v over the cells within r of c along
// axis d that lie inside the field.  v is viewed as [outer][n[d]][inner],
// and each output row along the contiguous inner index combines 2r + 1
// input rows.
template <bool MIN>
void box_filter_t(std::vector<uint8_t>& v, const int n[3], int d, int r) {
  const long inner = d == 0 ? 1 : (d == 1 ? (long)n[0] : (long)n[0] * n[1]);
  const long outer = (long)v.size() / (inner * n[d]);
  const int m = n[d];
  std::vector<uint8_t> w(v.size());
  auto op = [](uint8_t a, uint8_t b) -> uint8_t { return MIN ? (a & b) : (a | b); };
  for (long o = 0; o < outer; o++) {
    const uint8_t* vo = &v[o * m * inner];
    uint8_t* wo = &w[o * m * inner];
    if (inner == 1) {  // along the row: combine the row with its shifts
      std::memcpy(wo, vo, m);
      for (int s = 1; s <= r && s < m; s++) {
        for (int x = 0; x + s < m; x++) wo[x] = op(wo[x], vo[x + s]);
        for (int x = s; x < m; x++) wo[x] = op(wo[x], vo[x - s]);
      }
      continue;
    }
    for (int x = 0; x < m; x++) {
      const int y0 = std::max(0, x - r), y1 = std::min(m - 1, x + r);
      uint8_t* dst = wo + x * inner;
      std::memcpy(dst, vo + y0 * inner, inner);
      for (int y = y0 + 1; y <= y1; y++) {
        const uint8_t* src = vo + y * inner;
        for (long t = 0; t < inner; t++) dst[t] = op(dst[t], src[t]);
      }
    }
  }
  v.swap(w);
}

void box_filter(std::vector<uint8_t>& v, const int n[3], int d, int r, bool take_min) {
  if (take_min)
    box_filter_t<true>(v, n, d, r);
  else
    box_filter_t<false>(v, n, d, r);
}

// Counts over boxes in O(1): a summed-area table of a dense 0/1 field,
// S(i, j, k) = number of set cells in [0, i) x [0, j) x [0, k).
struct BoxSum {
  int n[3];
  std::vector<int> S;
  BoxSum(const std::vector<uint8_t>& v, const int nn[3]) {
    for (int d = 0; d < 3; d++) n[d] = nn[d];
    const long sx = n[0] + 1, sxy = sx * (n[1] + 1);
    S.assign(sxy * (n[2] + 1), 0);
    for (int k = 0; k < n[2]; k++)
      for (int j = 0; j < n[1]; j++) {
        const uint8_t* row = &v[(long)n[0] * (j + (long)n[1] * k)];
        int* o = &S[(k + 1) * sxy + (j + 1) * sx];
        const int* dn = o - sx;        // (j, k + 1)
        const int* bk = o - sxy;       // (j + 1, k)
        const int* db = o - sx - sxy;  // (j, k)
        int line = 0;                  // running sum along the row
        for (int i = 0; i < n[0]; i++) {
          line += row[i] ? 1 : 0;
          o[i + 1] = line + dn[i + 1] + bk[i + 1] - db[i + 1];
        }
      }
  }
  long count(const int lo[3], const int hi[3]) const {
    const long sx = n[0] + 1, sxy = sx * (n[1] + 1);
    auto at = [&](int i, int j, int k) { return (long)S[k * sxy + j * sx + i]; };
    const int a0 = lo[0], a1 = lo[1], a2 = lo[2], b0 = hi[0] + 1, b1 = hi[1] + 1, b2 = hi[2] + 1;
    return at(b0, b1, b2) - at(a0, b1, b2) - at(b0, a1, b2) - at(b0, b1, a2) + at(a0, a1, b2) +
           at(a0, b1, a2) + at(b0, a1, a2) - at(a0, a1, a2);
  }
};

struct Clusterer {
  const BoxSum& tag;   // level-l tags
  const BoxSum& ok;    // level-l cells that may hold the finer level
  int n[3];
  double eff;
  int max_side, min_side;            // in level-l cells
  std::vector<IBox>& out;

  // sig[x] = tags in the plane lo[d] + x of the box, along axis d
  void signature(const IBox& b, int d, std::vector<long>& sig) const {
    sig.assign(b.side(d), 0);
    int lo[3] = {b.lo[0], b.lo[1], b.lo[2]}, hi[3] = {b.hi[0], b.hi[1], b.hi[2]};
    for (int x = 0; x < b.side(d); x++) {
      lo[d] = hi[d] = b.lo[d] + x;
      sig[x] = tag.count(lo, hi);
    }
  }

  // the box cut down to the bounding box of its tags; false if it has none
  bool shrink(IBox& b, long& cnt) const {
    cnt = tag.count(b.lo, b.hi);
    if (!cnt) return false;
    std::vector<long> sig;
    for (int d = 0; d < 3; d++) {
      signature(b, d, sig);
      int f = 0, l = b.side(d) - 1;
      while (!sig[f]) f++;
      while (!sig[l]) l--;
      const int lo = b.lo[d];
      b.lo[d] = lo + f;
      b.hi[d] = lo + l;
    }
    return true;
  }

  bool all_ok(const IBox& b) const { return ok.count(b.lo, b.hi) == b.vol(); }

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

// A new cell that is not a copy of an old cell on its own level: the old
// coarse cell src, its six neighbours on that level (-1: none; x-, x+, y-,
// ...) and the new cell centre relative to src's, (x - x_c) / h_c per axis
// (a multiple of 1/2^(l - lc + 1), exact in float).
struct ReconDesc {
  int cell;         // the new cell
  int src;
  int nb[6];
  float off[3];
};

__device__ __forceinline__ double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return (fabs(a) < fabs(b)) ? a : b;
}

// Threads [0, N): new cells with code >= 0 copy old cell code for every
// field.  Threads [N, N + nrec): the reconstruction entries.
__global__ void k_transfer(const int* __restrict__ code, const ReconDesc* __restrict__ rec,
                           int N, int nrec, int Nold, int nvec, const double* __restrict__ uo,
                           double* __restrict__ un) {
  const long total = (long)N + nrec;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    if (t < N) {
      const int src = code[t];
      if (src < 0) continue;
      for (int f = 0; f < 2 * nvec; f++) un[(long)f * N + t] = uo[(long)f * Nold + src];
      continue;
    }
    const ReconDesc r = rec[t - N];
    for (int f = 0; f < 2 * nvec; f++) {
      const double* u = uo + (long)f * Nold;
      const double uc = u[r.src];
      double v = uc;
      for (int a = 0; a < 3; a++) {
        const int im = r.nb[2 * a], ip = r.nb[2 * a + 1];
        if (im >= 0 && ip >= 0) v += minmod(uc - u[im], u[ip] - uc) * (double)r.off[a];
      }
      un[(long)f * N + r.cell] = v;
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
    if ((long)(n[0] + 1) * (n[1] + 1) * (n[2] + 1) > (long)INT32_MAX) {
      c->err = "nrd_regrid_boxes: a level is too large for int32 box counts";
      return NRD_EINVAL;
    }
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
    // ok: every neighbour of the 3x3x3 block inside the domain is in the new
    // level (proper nesting); tg: a raw tag within `buffer` cells (inside the
    // domain), on ok cells.  Both are box filters, done one axis at a time:
    // the minimum of `in` over windows of 3 (outside the domain counts as
    // in), the maximum of `raw` over windows of 2 buffer + 1 (outside counts
    // as untagged).
    ok = in;
    for (int d = 0; d < 3; d++) box_filter(ok, n, d, 1, true);
    std::vector<uint8_t> hit = raw;
    for (int d = 0; d < 3; d++) box_filter(hit, n, d, buffer, false);
    for (long q = 0; q < lsize; q++) tg[q] = (ok[q] && hit[q]) ? 1 : 0;
    std::vector<IBox> coarse;
    const BoxSum tsum(tg, n), osum(ok, n);
    Clusterer C{tsum, osum, {n[0], n[1], n[2]}, efficiency, max_side / 2, min_side / 2, coarse};
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
  // Per new cell: the old cell on the same level (a copy), else -1 and a
  // reconstruction entry.  Patches are split over host threads; each thread
  // keeps its own entries, concatenated afterwards.
  std::vector<int> code(B.N);
  const int np = (int)B.patches.size();
  int nth = (int)std::min<long>(16, std::max<long>(1, (long)B.N / 65536));
  nth = std::max(1, std::min(nth, (int)std::thread::hardware_concurrency()));
  std::vector<std::vector<ReconDesc>> recs(nth);
  std::vector<int> fail(nth, 0);
  auto work = [&](int th) {
    // patches of thread th: a contiguous range holding about 1/nth of the cells
    const long lo_cell = (long)B.N * th / nth, hi_cell = (long)B.N * (th + 1) / nth;
    for (int p = 0; p < np; p++) {
      const PatchDev& P = B.patches[p];
      if (P.off < lo_cell || P.off >= hi_cell) continue;
      const int l = P.level;
      for (int k = 0; k < P.n[2]; k++)
        for (int j = 0; j < P.n[1]; j++)
          for (int i = 0; i < P.n[0]; i++) {
            const int q[3] = {P.lo[0] + i, P.lo[1] + j, P.lo[2] + k};
            const int c = P.off + i + P.n[0] * (j + P.n[1] * k);
            code[c] = old_cell(l, q);
            if (code[c] >= 0) continue;
            int lc = std::min(l, A.L) - 1, cq[3] = {0, 0, 0};
            for (; lc >= 0; lc--) {
              for (int d = 0; d < 3; d++) cq[d] = q[d] >> (l - lc);
              if (old_cell(lc, cq) >= 0) break;
            }
            if (lc < 0) {
              fail[th] = 1;
              return;
            }
            ReconDesc t;
            t.cell = c;
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
            recs[th].push_back(t);
          }
    }
  };
  if (nth == 1) {
    work(0);
  } else {
    // a part whose thread cannot be started (the system refuses it) runs here
    std::vector<std::thread> pool;
    int started = 0;
    try {
      for (; started < nth; started++) pool.emplace_back(work, started);
    } catch (...) {
    }
    for (int th = started; th < nth; th++) work(th);
    for (auto& t : pool) t.join();
  }
  for (int th = 0; th < nth; th++)
    if (fail[th]) {
      dst->err = "transfer: a new cell lies in no old cell";
      return NRD_EINVAL;
    }
  size_t nrec = 0;
  for (const auto& v : recs) nrec += v.size();
  std::vector<ReconDesc> rec;
  rec.reserve(nrec);
  for (const auto& v : recs) rec.insert(rec.end(), v.begin(), v.end());
  const size_t No = (size_t)A.N, Nn = (size_t)B.N;
  // one device buffer: the old vectors (made composite), the codes and the
  // reconstruction entries
  const size_t comp_bytes = 2 * No * nvec * sizeof(double);
  const size_t code_bytes = (Nn * sizeof(int) + 15) / 16 * 16;
  const size_t rec_bytes = nrec * sizeof(ReconDesc);
  char* d_buf = nullptr;
  if (cudaMalloc(&d_buf, comp_bytes + code_bytes + rec_bytes) != cudaSuccess) {
    dst->err = "allocation failed";
    return NRD_ENOMEM;
  }
  double* d_comp = (double*)d_buf;
  int* d_code = (int*)(d_buf + comp_bytes);
  ReconDesc* d_rec = (ReconDesc*)(d_buf + comp_bytes + code_bytes);
  cudaMemcpyAsync(d_code, code.data(), Nn * sizeof(int), cudaMemcpyHostToDevice, s);
  if (nrec) cudaMemcpyAsync(d_rec, rec.data(), rec_bytes, cudaMemcpyHostToDevice, s);
  dst->timer.begin(NRD_TK_TRANSFER, s);
  cudaMemcpyAsync(d_comp, u_src, comp_bytes, cudaMemcpyDeviceToDevice, s);
  launch_average_down(A, d_comp, 2 * nvec, (int)No, s);
  const long work_items = (long)Nn + (long)nrec;
  const int grid = (int)std::max(1L, std::min(152L * 8, (work_items + 255) / 256));
  k_transfer<<<grid, 256, 0, s>>>(d_code, d_rec, (int)Nn, (int)nrec, (int)No, nvec, d_comp,
                                  u_dst);
  dst->timer.end(NRD_TK_TRANSFER, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(d_buf);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    dst->err = "transfer kernel failed";
    return NRD_ECUDA;
  }
  return NRD_OK;
}

}  // extern "C"
