// Host-side construction of the patch hierarchy work-lists (Sec. 3.2.1 SAMR
// hierarchy): patch table, cell masks, ghost descriptors (physical, sibling,
// coarse-fine interpolation stencils), flux-matching lists, coefficient
// coarsening lists, dense level maps and stencil tiles.  Built once per
// hierarchy and uploaded; every kernel then runs from these lists.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <thread>

#include "nrd_internal.h"

namespace {

// The per-cell and per-patch loops below are independent across cells
// (patches): they run over contiguous chunks on host threads, each chunk
// with its own output lists, joined in chunk order, so every list is the
// one a serial loop builds.
int host_chunks(long n, long min_per_chunk) {
  const long hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  return (int)std::max(1L, std::min(hw, n / std::max(1L, min_per_chunk)));
}
// fn(lo, hi, k) for chunk k = [n k / nch, n (k + 1) / nch)
template <class F>
void host_parallel(long n, int nch, const F& fn) {
  if (nch <= 1) {
    fn(0L, n, 0);
    return;
  }
  // a chunk whose thread cannot be started (the system refuses it) runs here
  std::vector<std::thread> th;
  th.reserve(nch);
  int started = 0;
  try {
    for (; started < nch; started++) {
      const int k = started;
      th.emplace_back([&fn, n, nch, k] { fn(n * k / nch, n * (k + 1) / nch, k); });
    }
  } catch (...) {
  }
  for (int k = started; k < nch; k++) fn(n * k / nch, n * (k + 1) / nch, k);
  for (auto& t : th) t.join();
}

struct Builder {
  Hier& H;
  std::vector<int> box;   // 6 per patch
  explicit Builder(Hier& h) : H(h) {}

  long lidx(int l, int i, int j, int k) const {
    const LevelInfo& Lv = H.lev[l];
    return (long)i + (long)Lv.n[0] * ((long)j + (long)Lv.n[1] * k);
  }
  bool inside(int l, const int c[3]) const {
    for (int d = 0; d < 3; d++)
      if (c[d] < 0 || c[d] >= H.lev[l].n[d]) return false;
    return true;
  }
  int cell(int l, const int c[3]) const {
    if (!inside(l, c)) return -2;
    return H.lmap[l][lidx(l, c[0], c[1], c[2])];
  }
  bool covered(int l, const int c[3]) const {
    if (l + 1 >= H.L) return false;
    int q[3] = {2 * c[0], 2 * c[1], 2 * c[2]};
    return cell(l + 1, q) >= 0;
  }
  void ijk_of(int idx, int c[3]) const {
    const PatchDev& P = H.patches[H.cell_patch[idx]];
    int r = idx - P.off;
    c[0] = P.lo[0] + r % P.n[0];
    r /= P.n[0];
    c[1] = P.lo[1] + r % P.n[1];
    c[2] = P.lo[2] + r / P.n[1];
  }
  // ghost index of the face cell of patch p on face f at level position c
  // (c is the interior cell adjacent to the face)
  int ghost_index(int p, int f, const int c[3]) const {
    const PatchDev& P = H.patches[p];
    int d = f / 2, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int a = c[t1] - P.lo[t1], b = c[t2] - P.lo[t2];
    return P.goff + P.fo[f] + a + P.n[t1] * b;
  }
  // Expand a coarse source cell into leaf terms: a covered cell is the mean
  // of its 8 children (recursively).
  void expand(int l, const int c[3], double w, std::vector<int>& idx, std::vector<double>& ws) {
    if (covered(l, c)) {
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
          for (int e = 0; e < 2; e++) {
            int q[3] = {2 * c[0] + a, 2 * c[1] + b, 2 * c[2] + e};
            expand(l + 1, q, w / 8.0, idx, ws);
          }
      return;
    }
    idx.push_back(cell(l, c));
    ws.push_back(w);
  }
  // Address of the face between level-l cells a (low) and b = a + e_d (high)
  // in the coefficient space [3N low faces | G boundary faces].
  int face_addr(int l, int d, const int a[3], const int b[3]) const {
    int ib = inside(l, b) ? cell(l, b) : -2;
    if (ib >= 0) {
      int p = H.cell_patch[ib];
      const PatchDev& P = H.patches[p];
      if (b[d] > P.lo[d]) return d * H.N + ib;           // interior low face of b
      return 3 * H.N + ghost_index(p, 2 * d, b);         // b's patch, face d-
    }
    int ia = cell(l, a);
    int p = H.cell_patch[ia];
    return 3 * H.N + ghost_index(p, 2 * d + 1, a);       // a's patch, face d+
  }
};

}  // namespace

int hier_build(Hier& H, int nlevels, const int* nboxes, const int* boxes, const int* bc_type,
               const double* bc_R, std::string& err) {
  if (nlevels < 1 || nlevels > NRD_MAX_LEVELS) {
    err = "nlevels must be in [1, 8]";
    return NRD_EINVAL;
  }
  if (nboxes[0] != 1) {
    err = "level 0 must be exactly one box covering the domain";
    return NRD_EINVAL;
  }
  const int* b0 = boxes;
  if (b0[0] != 0 || b0[1] != 0 || b0[2] != 0 || b0[3] < 0 || b0[4] < 0 || b0[5] < 0) {
    err = "level 0 box must start at the origin";
    return NRD_EINVAL;
  }
  for (int f = 0; f < 6; f++) {
    if (bc_type[f] != NRD_BC_NEUMANN && bc_type[f] != NRD_BC_ROBIN) {
      err = "bad boundary type";
      return NRD_EINVAL;
    }
    H.bc_type[f] = bc_type[f];
    H.bc_R[f] = bc_R[f];
  }
  H.L = nlevels;
  H.patches.clear();
  H.tiles.clear();
  H.cell_patch.clear();
  H.lmap.assign(nlevels, std::vector<int>());
  Builder B(H);
  long off = 0, goff = 0;
  int bi = 0;
  for (int l = 0; l < nlevels; l++) {
    LevelInfo& Lv = H.lev[l];
    for (int d = 0; d < 3; d++) {
      long n = (long)(b0[3 + d] + 1) << l;
      if (n > (1 << 20)) {
        err = "level index space too large";
        return NRD_EINVAL;
      }
      Lv.n[d] = (int)n;
      Lv.h[d] = 1.0 / (double)n;
    }
    long lsize = (long)Lv.n[0] * Lv.n[1] * Lv.n[2];
    if (lsize > (1L << 31) - 1) {
      err = "level index space exceeds 2^31 cells";
      return NRD_EINVAL;
    }
    H.lmap[l].assign(lsize, -1);
    Lv.off = (int)off;
    Lv.p0 = (int)H.patches.size();
    Lv.g0 = (int)goff;
    if (nboxes[l] < 1) {
      err = "every level needs at least one box";
      return NRD_EINVAL;
    }
    for (int p = 0; p < nboxes[l]; p++, bi++) {
      const int* bx = boxes + 6 * bi;
      PatchDev P;
      P.level = l;
      for (int d = 0; d < 3; d++) {
        if (bx[d] < 0 || bx[3 + d] >= Lv.n[d] || bx[3 + d] < bx[d]) {
          err = "box outside the domain or empty";
          return NRD_EINVAL;
        }
        if (l > 0 && (bx[d] % 2 != 0 || bx[3 + d] % 2 != 1)) {
          err = "fine box not aligned to refinement ratio 2";
          return NRD_EINVAL;
        }
        P.lo[d] = bx[d];
        P.n[d] = bx[3 + d] - bx[d] + 1;
      }
      long pc = (long)P.n[0] * P.n[1] * P.n[2];
      if (off + pc > (1L << 30)) {
        err = "more than 2^30 cells";
        return NRD_EINVAL;
      }
      P.off = (int)off;
      P.goff = (int)goff;
      int fo = 0;
      for (int f = 0; f < 6; f++) {
        int d = f / 2;
        P.fo[f] = fo;
        fo += P.n[(d + 1) % 3] * P.n[(d + 2) % 3];
      }
      int pid = (int)H.patches.size();
      for (int k = 0; k < P.n[2]; k++)
        for (int j = 0; j < P.n[1]; j++)
          for (int i = 0; i < P.n[0]; i++) {
            long li = B.lidx(l, P.lo[0] + i, P.lo[1] + j, P.lo[2] + k);
            if (H.lmap[l][li] >= 0) {
              err = "overlapping boxes on a level";
              return NRD_EINVAL;
            }
            H.lmap[l][li] = (int)(off + i + (long)P.n[0] * (j + (long)P.n[1] * k));
          }
      H.cell_patch.insert(H.cell_patch.end(), pc, pid);
      H.patches.push_back(P);
      off += pc;
      goff += fo;
    }
    Lv.ncell = (int)(off - Lv.off);
    Lv.np = (int)H.patches.size() - Lv.p0;
    Lv.ng = (int)(goff - Lv.g0);
  }
  H.N = (int)off;
  H.G = (int)goff;
  // proper nesting
  for (int l = 1; l < nlevels; l++) {
    const LevelInfo& Lv = H.lev[l];
    for (int p = Lv.p0; p < Lv.p0 + Lv.np; p++) {
      const PatchDev& P = H.patches[p];
      for (int k = P.lo[2] / 2 - 1; k <= (P.lo[2] + P.n[2] - 1) / 2 + 1; k++)
        for (int j = P.lo[1] / 2 - 1; j <= (P.lo[1] + P.n[1] - 1) / 2 + 1; j++)
          for (int i = P.lo[0] / 2 - 1; i <= (P.lo[0] + P.n[0] - 1) / 2 + 1; i++) {
            int c[3] = {i, j, k};
            if (!B.inside(l - 1, c)) continue;
            if (B.cell(l - 1, c) < 0) {
              char buf[128];
              std::snprintf(buf, sizeof buf, "level %d is not properly nested in level %d", l,
                            l - 1);
              err = buf;
              return NRD_EINVAL;
            }
          }
    }
  }
  return NRD_OK;
}

namespace {
template <class T>
int upload(T** dptr, const std::vector<T>& v, std::string& err) {
  *dptr = nullptr;
  if (v.empty()) return NRD_OK;
  CUDA_TRY(cudaMalloc((void**)dptr, v.size() * sizeof(T)));
  CUDA_TRY(cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return NRD_OK;
}
}  // namespace

#define UP(ptr, vec)                          \
  do {                                        \
    int rc_ = upload(&(ptr), (vec), err);     \
    if (rc_ != NRD_OK) return rc_;            \
  } while (0)

int hier_upload(Hier& H, std::string& err) {
  Builder B(H);
  const int N = H.N, G = H.G, L = H.L;
  // masks and leaf volumes
  std::vector<uint8_t> mask(N, 0);
  std::vector<float> wvol(N, 0.0f);
  std::vector<int> cellijk(3 * (size_t)N);
  const int nchc = host_chunks(N, 32768);
  std::vector<int> leaf_k(nchc, 0);
  host_parallel(N, nchc, [&](long lo, long hi, int k) {
    int nl = 0;
    for (long idx = lo; idx < hi; idx++) {
      int c[3];
      B.ijk_of((int)idx, c);
      cellijk[3 * idx] = c[0];
      cellijk[3 * idx + 1] = c[1];
      cellijk[3 * idx + 2] = c[2];
      int l = H.patches[H.cell_patch[idx]].level;
      if (B.covered(l, c)) {
        mask[idx] = MASK_COVERED;
        continue;
      }
      nl++;
      const double* h = H.lev[l].h;
      wvol[idx] = (float)(h[0] * h[1] * h[2]);
      for (int f = 0; f < 6; f++) {
        int d = f / 2, s = (f % 2) ? 1 : -1;
        int g[3] = {c[0], c[1], c[2]};
        g[d] += s;
        if (B.inside(l, g) && B.cell(l, g) >= 0 && B.covered(l, g))
          mask[idx] |= (uint8_t)(2 << f);
      }
    }
    leaf_k[k] = nl;
  });
  int nleaf = 0;
  for (int v : leaf_k) nleaf += v;
  H.nleaf = nleaf;
  // ghosts
  std::vector<uint8_t> gtype(G), gface(G);
  std::vector<int> gcell(G), gzsrc(G), gt0(G + 1);
  std::vector<int> gidx;
  std::vector<double> gw;
  {
    const int np = (int)H.patches.size();
    const int nch = host_chunks(np, 8);
    std::vector<std::vector<int>> gxk(nch);
    std::vector<std::vector<double>> wxk(nch);
    std::vector<int> bad(nch, 0);
    host_parallel(np, nch, [&](long plo, long phi, int k) {
      std::vector<int>& gx = gxk[k];
      std::vector<double>& wx = wxk[k];
      for (int p = (int)plo; p < (int)phi; p++) {
        const PatchDev& P = H.patches[p];
        int l = P.level;
        for (int f = 0; f < 6; f++) {
          int d = f / 2, s = (f % 2) ? 1 : -1, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          for (int b = 0; b < P.n[t2]; b++)
            for (int a = 0; a < P.n[t1]; a++) {
              int c[3];
              c[d] = (s < 0) ? P.lo[d] : P.lo[d] + P.n[d] - 1;
              c[t1] = P.lo[t1] + a;
              c[t2] = P.lo[t2] + b;
              int gi = P.goff + P.fo[f] + a + P.n[t1] * b;
              int ic = B.cell(l, c);
              int g[3] = {c[0], c[1], c[2]};
              g[d] += s;
              gface[gi] = (uint8_t)(f | (l << 3));
              gcell[gi] = ic;
              gt0[gi] = (int)gx.size();
              if (!B.inside(l, g)) {
                gtype[gi] = (H.bc_type[f] == NRD_BC_ROBIN) ? GT_ROBIN : GT_NEUMANN;
                gzsrc[gi] = ic;
                continue;
              }
              int ig = B.cell(l, g);
              if (ig >= 0) {
                gtype[gi] = GT_SIBLING;
                gzsrc[gi] = ig;
                gx.push_back(ig);
                wx.push_back(1.0);
                continue;
              }
              // coarse-fine: g = (x_c + 2 i)/3, i = (9 c00 + 3 c10 + 3 c01 + c11)/16
              gtype[gi] = GT_CF;
              int Pc[3] = {g[0] / 2, g[1] / 2, g[2] / 2};
              const LevelInfo& C = H.lev[l - 1];
              int o1 = (g[t1] % 2 == 0) ? -1 : 1, o2 = (g[t2] % 2 == 0) ? -1 : 1;
              if (Pc[t1] + o1 < 0 || Pc[t1] + o1 >= C.n[t1]) o1 = 0;
              if (Pc[t2] + o2 < 0 || Pc[t2] + o2 >= C.n[t2]) o2 = 0;
              gzsrc[gi] = B.cell(l - 1, Pc);
              gx.push_back(ic);
              wx.push_back(1.0 / 3.0);
              const double wq[4] = {9.0, 3.0, 3.0, 1.0};
              for (int q = 0; q < 4; q++) {
                int cc[3] = {Pc[0], Pc[1], Pc[2]};
                if (q == 1 || q == 3) cc[t1] += o1;
                if (q == 2 || q == 3) cc[t2] += o2;
                if (B.cell(l - 1, cc) < 0) {
                  bad[k] = 1;
                  return;
                }
                B.expand(l - 1, cc, (2.0 / 3.0) * wq[q] / 16.0, gx, wx);
              }
            }
        }
      }
    });
    for (int k = 0; k < nch; k++)
      if (bad[k]) {
        err = "coarse-fine interpolation source missing (nesting)";
        return NRD_EINVAL;
      }
    // chunk k's term offsets start at the terms of the chunks before it
    for (int k = 0; k < nch; k++) {
      const int base = (int)gidx.size();
      const int plo = (int)((long)np * k / nch), phi = (int)((long)np * (k + 1) / nch);
      if (plo < phi) {
        const int g0 = H.patches[plo].goff;
        const int g1 = (phi < np) ? H.patches[phi].goff : G;
        for (int g = g0; g < g1; g++) gt0[g] += base;
      }
      gidx.insert(gidx.end(), gxk[k].begin(), gxk[k].end());
      gw.insert(gw.end(), wxk[k].begin(), wxk[k].end());
    }
  }
  gt0[G] = (int)gidx.size();
  H.nterm = (int)gidx.size();
  // transposed ghost stencils for the adjoint
  std::vector<int> ts_off(N + 1, 0), ts_g, tz_off(N + 1, 0), tz_g;
  std::vector<double> ts_w;
  {
    std::vector<int> cnt(N, 0), zc(N, 0);
    for (int g = 0; g < G; g++) {
      if (gtype[g] != GT_SIBLING && gtype[g] != GT_CF) continue;
      for (int q = gt0[g]; q < gt0[g + 1]; q++) cnt[gidx[q]]++;
      zc[gzsrc[g]]++;
    }
    for (int c = 0; c < N; c++) {
      ts_off[c + 1] = ts_off[c] + cnt[c];
      tz_off[c + 1] = tz_off[c] + zc[c];
    }
    ts_g.assign(ts_off[N], 0);
    ts_w.assign(ts_off[N], 0.0);
    tz_g.assign(tz_off[N], 0);
    std::vector<int> p1(ts_off.begin(), ts_off.end() - 1), p2(tz_off.begin(), tz_off.end() - 1);
    for (int g = 0; g < G; g++) {
      if (gtype[g] != GT_SIBLING && gtype[g] != GT_CF) continue;
      for (int q = gt0[g]; q < gt0[g + 1]; q++) {
        int c = gidx[q];
        ts_g[p1[c]] = g;
        ts_w[p1[c]] = gw[q];
        p1[c]++;
      }
      tz_g[p2[gzsrc[g]]++] = g;
    }
  }
  // flux matching lists
  std::vector<int> rf_cell, rf_off, rf_face, rf_level;
  std::vector<int4> rf_g;
  for (int idx = 0; idx < N; idx++) {
    if (!(mask[idx] & 0x7e)) continue;
    const int* c = &cellijk[3 * idx];
    int l = H.patches[H.cell_patch[idx]].level;
    rf_cell.push_back(idx);
    rf_level.push_back(l);
    rf_off.push_back((int)rf_face.size());
    for (int f = 0; f < 6; f++) {
      if (!(mask[idx] & (2 << f))) continue;
      int d = f / 2, s = (f % 2) ? 1 : -1, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      int g[3] = {c[0], c[1], c[2]};
      g[d] += s;
      int gs[4];
      int n = 0;
      for (int bb = 0; bb < 2; bb++)
        for (int aa = 0; aa < 2; aa++) {
          int q[3];
          q[d] = (s > 0) ? 2 * g[d] : 2 * g[d] + 1;
          q[t1] = 2 * c[t1] + aa;
          q[t2] = 2 * c[t2] + bb;
          int iq = B.cell(l + 1, q);
          if (iq < 0) {
            err = "flux matching: fine cell missing";
            return NRD_EINVAL;
          }
          int fq = 2 * d + (s > 0 ? 0 : 1);   // fine face pointing back at c
          gs[n++] = B.ghost_index(H.cell_patch[iq], fq, q);
        }
      rf_face.push_back(f);
      rf_g.push_back(make_int4(gs[0], gs[1], gs[2], gs[3]));
    }
  }
  H.nrf = (int)rf_cell.size();
  for (int l = 0; l <= NRD_MAX_LEVELS; l++) {
    int q = 0;
    while (q < H.nrf && rf_level[q] < l) q++;
    H.rf_lstart[l] = q;
  }
  rf_off.push_back((int)rf_face.size());
  // coefficient coarsening lists: faces of level l with a covered side
  std::vector<std::vector<int>> cz_tgt(L);
  std::vector<std::vector<int4>> cz_src(L);
  for (int l = 0; l + 1 < L; l++) {
    const LevelInfo& Lv = H.lev[l];
    const int nch = host_chunks(Lv.ncell, 4096);
    std::vector<std::vector<int>> tk(nch);
    std::vector<std::vector<int4>> sk(nch);
    host_parallel(Lv.ncell, nch, [&](long lo, long hi, int k) {
      for (long q = lo; q < hi; q++) {
        const int idx = Lv.off + (int)q;
        const int* c = &cellijk[3 * idx];
        const PatchDev& P = H.patches[H.cell_patch[idx]];
        const bool cov_c = B.covered(l, c);
        for (int f = 0; f < 6; f++) {
          int d = f / 2, s = (f % 2) ? 1 : -1, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          int g[3] = {c[0], c[1], c[2]};
          g[d] += s;
          bool patch_bnd = (s < 0) ? (c[d] == P.lo[d]) : (c[d] == P.lo[d] + P.n[d] - 1);
          if (!patch_bnd && s > 0) continue;  // interior faces listed once (as low faces)
          bool in = B.inside(l, g);
          bool cov_g = in && B.cell(l, g) >= 0 && B.covered(l, g);
          if (!cov_c && !cov_g) continue;
          int tgt;
          if (patch_bnd)
            tgt = 3 * N + B.ghost_index(H.cell_patch[idx], f, c);
          else
            tgt = d * N + idx;
          int src[4];
          int n = 0;
          for (int bb = 0; bb < 2; bb++)
            for (int aa = 0; aa < 2; aa++) {
              int qa[3], qb[3];
              // fine cells on both sides of the coincident fine face
              int plane = (s > 0) ? 2 * g[d] : 2 * c[d];   // fine index of the high-side cell
              qb[d] = plane;
              qa[d] = plane - 1;
              qa[t1] = qb[t1] = 2 * c[t1] + aa;
              qa[t2] = qb[t2] = 2 * c[t2] + bb;
              if (!in) {
                // physical face: Robin D_b lives in the boundary slot of the
                // fine boundary cell
                int* qc = (s > 0) ? qa : qb;
                int iq = B.cell(l + 1, qc);
                src[n++] = 3 * N + B.ghost_index(H.cell_patch[iq], f, qc);
              } else {
                src[n++] = B.face_addr(l + 1, d, qa, qb);
              }
            }
          tk[k].push_back(tgt);
          sk[k].push_back(make_int4(src[0], src[1], src[2], src[3]));
        }
      }
    });
    for (int k = 0; k < nch; k++) {
      cz_tgt[l].insert(cz_tgt[l].end(), tk[k].begin(), tk[k].end());
      cz_src[l].insert(cz_src[l].end(), sk[k].begin(), sk[k].end());
    }
  }
  // covered lists for average-down
  std::vector<std::vector<int4>> cov(L);
  for (int idx = 0; idx < N; idx++) {
    if (!(mask[idx] & MASK_COVERED)) continue;
    const int* c = &cellijk[3 * idx];
    int l = H.patches[H.cell_patch[idx]].level;
    int q[3] = {2 * c[0], 2 * c[1], 2 * c[2]};
    int iq = B.cell(l + 1, q);
    const PatchDev& Q = H.patches[H.cell_patch[iq]];
    cov[l].push_back(make_int4(idx, iq, Q.n[0], Q.n[0] * Q.n[1]));
  }
  H.hmask = mask;
  // upload
  UP(H.d_patches, H.patches);
  UP(H.d_mask, mask);
  UP(H.d_wvol, wvol);
  UP(H.d_gtype, gtype);
  UP(H.d_gface, gface);
  UP(H.d_gcell, gcell);
  UP(H.d_gzsrc, gzsrc);
  UP(H.d_gt0, gt0);
  UP(H.d_gidx, gidx);
  UP(H.d_gw, gw);
  UP(H.d_rf_cell, rf_cell);
  UP(H.d_rf_off, rf_off);
  UP(H.d_rf_face, rf_face);
  UP(H.d_rf_g, rf_g);
  UP(H.d_rf_level, rf_level);
  UP(H.d_ts_off, ts_off);
  UP(H.d_ts_g, ts_g);
  UP(H.d_ts_w, ts_w);
  UP(H.d_tz_off, tz_off);
  UP(H.d_tz_g, tz_g);
  {
    int rc = hier_tiles(H, err);
    if (rc != NRD_OK) return rc;
  }
  for (int l = 0; l < L; l++) {
    H.ncz[l] = (int)cz_tgt[l].size();
    UP(H.d_cz_tgt[l], cz_tgt[l]);
    UP(H.d_cz_src[l], cz_src[l]);
    H.ncov[l] = (int)cov[l].size();
    UP(H.d_cov[l], cov[l]);
    if (l + 1 < L) UP(H.d_lmap[l], H.lmap[l]);
  }
  return NRD_OK;
}

// Stencil tiles of shape tile_x x tile_y x tile_z over every patch.  One
// tile is one CTA, and the block scheduler starts CTAs in index order, so
// the list runs from the most to the least expensive item: whole tiles,
// then the last kSplit whole tiles cut into two halves along z (the last
// wave then holds half tiles and ends sooner), then the tiles whose cells
// are all covered (they only write zeros).  Per-level ranges are not kept:
// every consumer of the list works on single tiles.
int hier_tiles(Hier& H, std::string& err) {
  (void)err;
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int kSplit = 3 * std::max(nsm, 1);   // about one wave of the linearisation stencil
  const int TX = H.tile_x, TY = H.tile_y, TZ = H.tile_z;
  std::vector<TileDev> full, covered;
  H.ragged = false;
  for (int l = 0; l < H.L; l++) {
    LevelInfo& Lv = H.lev[l];
    Lv.t0 = 0;
    Lv.nt = 0;
    for (int p = Lv.p0; p < Lv.p0 + Lv.np; p++) {
      const PatchDev& P = H.patches[p];
      for (int k0 = 0; k0 < P.n[2]; k0 += TZ)
        for (int j0 = 0; j0 < P.n[1]; j0 += TY)
          for (int i0 = 0; i0 < P.n[0]; i0 += TX) {
            const int k1 = std::min(k0 + TZ, P.n[2]);
            bool all = true;
            for (int k = k0; k < k1 && all; k++)
              for (int j = j0; j < std::min(j0 + TY, P.n[1]) && all; j++)
                for (int i = i0; i < std::min(i0 + TX, P.n[0]) && all; i++)
                  if (!(H.hmask[P.off + i + P.n[0] * (j + P.n[1] * k)] & MASK_COVERED)) all = false;
            TileDev t{p, i0, j0, k0, k1, all ? 1 : 0};
            (all ? covered : full).push_back(t);
            if (!all && (i0 + TX > P.n[0] || j0 + TY > P.n[1])) H.ragged = true;
          }
    }
  }
  H.tiles.clear();
  const int nsplit = std::min((int)full.size(), kSplit);
  const int nkeep = (int)full.size() - nsplit;
  H.tiles.insert(H.tiles.end(), full.begin(), full.begin() + nkeep);
  for (int q = nkeep; q < (int)full.size(); q++) {
    TileDev t = full[q];
    const int depth = t.k1 - t.k0;
    if (depth < 2) {
      H.tiles.push_back(t);
      continue;
    }
    const int km = t.k0 + depth / 2;
    TileDev lo = t, hi = t;
    lo.k1 = km;
    hi.k0 = km;
    H.tiles.push_back(lo);
    H.tiles.push_back(hi);
  }
  H.tiles.insert(H.tiles.end(), covered.begin(), covered.end());
  if (H.d_tiles) cudaFree(H.d_tiles);
  H.d_tiles = nullptr;
  UP(H.d_tiles, H.tiles);
  return NRD_OK;
}

void hier_free(Hier& H) {
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  F(H.d_patches); F(H.d_tiles); F(H.d_mask); F(H.d_wvol); F(H.d_gtype); F(H.d_gface);
  F(H.d_gcell); F(H.d_gzsrc); F(H.d_gt0); F(H.d_gidx); F(H.d_gw); F(H.d_rf_cell);
  F(H.d_rf_off); F(H.d_rf_face); F(H.d_rf_g); F(H.d_rf_level);
  F(H.d_ts_off); F(H.d_ts_g); F(H.d_ts_w); F(H.d_tz_off); F(H.d_tz_g);
  H.d_ts_off = nullptr; H.d_ts_g = nullptr; H.d_ts_w = nullptr; H.d_tz_off = nullptr;
  H.d_tz_g = nullptr;
  for (int l = 0; l < NRD_MAX_LEVELS; l++) {
    F(H.d_cz_tgt[l]); F(H.d_cz_src[l]); F(H.d_cov[l]); F(H.d_lmap[l]);
    H.d_cz_tgt[l] = nullptr; H.d_cz_src[l] = nullptr; H.d_cov[l] = nullptr; H.d_lmap[l] = nullptr;
    H.ncz[l] = 0; H.ncov[l] = 0;
  }
  H.d_patches = nullptr; H.d_tiles = nullptr; H.d_mask = nullptr; H.d_wvol = nullptr;
  H.d_gtype = nullptr; H.d_gface = nullptr; H.d_gcell = nullptr; H.d_gzsrc = nullptr;
  H.d_gt0 = nullptr; H.d_gidx = nullptr; H.d_gw = nullptr; H.d_rf_cell = nullptr;
  H.d_rf_off = nullptr; H.d_rf_face = nullptr; H.d_rf_g = nullptr; H.d_rf_level = nullptr;
}
