"""Plain CPU restatement of the regridding step of Sec. 5 (arXiv 1302.6303).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone.  It shares no code
with the CUDA library.

The paper groups tagged cells into patches with the Berger-Rigoutsos
algorithm and moves data to the new hierarchy by conservative linear
refinement, without giving parameters.  The reading followed here (R18-R20,
the same on the CUDA side):

R18 clustering, level by level from the coarsest.  Tags of level l are those
    of the current hierarchy; a cell missing there inherits the tag of the
    finest current cell containing it.  They are dilated by `buffer` cells
    and kept only on cells whose whole 3x3x3 neighbourhood (inside the
    domain) lies in the new level l (proper nesting).  Then, recursively on
    a box: shrink to the bounding box of its tags (drop if empty); accept if
    every cell may hold the finer level, no side exceeds max_side/2 and
    tags/volume >= efficiency; else cut at (1) a zero of a signature, axes
    longest first, zero nearest the middle, the empty plane dropped; (2) the
    strongest sign change of the second difference of the signatures (axes
    of at least 4 planes); (3) the middle of the longest side.  Cuts leave
    both parts at least min_side/2 planes wide unless the box holds cells
    that may not hold the finer level.  A box that cannot be cut is kept.
R19 transfer: old vectors are made composite (covered := mean of children);
    a new cell present on the same old level copies it; any other new cell
    takes the minmod-limited linear reconstruction of the finest old cell
    containing it, evaluated at its centre (slope 0 on an axis where an old
    neighbour on that level is missing).
R20 warm restart: the step that produced u_n is solved again on the new
    hierarchy from the transferred u_n with the transferred history, and the
    next local error estimate is not used (Sec. 5).
"""
from __future__ import annotations

import numpy as np


# ------------------------------------------------------------------ clustering
def _signature(tag, b, d):
    lo, hi = b
    sub = tag[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1]
    axes = tuple(a for a in range(3) if a != d)
    return sub.sum(axis=axes).astype(np.int64)


def _cluster(tag, ok, b, eff, max_side, min_side, out):
    lo, hi = b
    sub = tag[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1]
    if not sub.any():
        return
    # shrink to the bounding box of the tags
    nz = np.nonzero(sub)
    lo = tuple(int(lo[d] + nz[d].min()) for d in range(3))
    hi = tuple(int(b[0][d] + nz[d].max()) for d in range(3))
    b = (lo, hi)
    side = [hi[d] - lo[d] + 1 for d in range(3)]
    cnt = int(tag[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1].sum())
    vol = side[0] * side[1] * side[2]
    longest = int(np.argmax(side))          # first axis of the largest side
    nested = bool(ok[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1].all())
    if nested and side[longest] <= max_side and cnt >= eff * vol:
        out.append(b)
        return
    mn = max(1, min_side) if nested else 1
    order = [longest, (longest + 1) % 3, (longest + 2) % 3]

    def split(d, a_hi, c_lo):
        a = (lo, tuple(a_hi if e == d else hi[e] for e in range(3)))
        c = (tuple(c_lo if e == d else lo[e] for e in range(3)), hi)
        _cluster(tag, ok, a, eff, max_side, min_side, out)
        _cluster(tag, ok, c, eff, max_side, min_side, out)

    # (1) holes
    for d in order:
        s = side[d]
        if s < 3:
            continue
        sig = _signature(tag, b, d)
        cands = [i for i in range(1, s - 1) if sig[i] == 0 and i >= mn and s - 1 - i >= mn]
        if cands:
            mid = s // 2
            best = min(cands, key=lambda i: (abs(i - mid), i))
            split(d, lo[d] + best - 1, lo[d] + best + 1)
            return
    # (2) inflection
    best = None
    for d in order:
        s = side[d]
        if s < 4:
            continue
        sig = _signature(tag, b, d)
        lap = sig[2:] - 2 * sig[1:-1] + sig[:-2]      # lap[i-1] at plane i
        for i in range(1, s - 2):
            l1, l2 = lap[i - 1], lap[i]
            if (l1 < 0) == (l2 < 0):
                continue
            if i + 1 < mn or s - 1 - i < mn:
                continue
            v = abs(int(l2) - int(l1))
            if v > 0 and (best is None or v > best[0]):
                best = (v, d, i)
    if best is not None:
        _, d, i = best
        split(d, lo[d] + i, lo[d] + i + 1)
        return
    # (3) bisection
    s = side[longest]
    if s >= 2 and s // 2 >= mn and s - s // 2 >= mn:
        split(longest, lo[longest] + s // 2 - 1, lo[longest] + s // 2)
        return
    out.append(b)


def cluster_level(tag, ok, efficiency, max_side, min_side):
    """Boxes (inclusive lo/hi, level-l index) covering the tags of one level."""
    out = []
    n = tag.shape
    _cluster(tag.astype(bool), ok.astype(bool), ((0, 0, 0), tuple(x - 1 for x in n)),
             efficiency, max_side, min_side, out)
    return out


def _dense_tags(hier, tags, tag_bits):
    """Per current level: dense int8 array, -1 where the level has no cell."""
    out = []
    off = 0
    dense = [np.full(hier.level_n(l), -1, dtype=np.int8) for l in range(hier.nlevels)]
    for l, lev in enumerate(hier.levels):
        for lo, hi in lev:
            n = [hi[d] - lo[d] + 1 for d in range(3)]
            cnt = n[0] * n[1] * n[2]
            t = ((tags[off:off + cnt] & tag_bits) != 0).astype(np.int8)
            dense[l][lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] = \
                t.reshape(n[2], n[1], n[0]).transpose(2, 1, 0)
            off += cnt
    out = dense
    return out


def _dilate(mask, r):
    if r == 0:
        return mask.copy()
    p = np.pad(mask, r, constant_values=False)
    out = np.zeros_like(mask)
    n = mask.shape
    for dk in range(-r, r + 1):
        for dj in range(-r, r + 1):
            for di in range(-r, r + 1):
                out |= p[r + di:r + di + n[0], r + dj:r + dj + n[1], r + dk:r + dk + n[2]]
    return out


def _nestable(inmask):
    p = np.pad(inmask, 1, constant_values=True)
    out = inmask.copy()
    n = inmask.shape
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                out &= p[1 + di:1 + di + n[0], 1 + dj:1 + dj + n[1], 1 + dk:1 + dk + n[2]]
    return out


def regrid_boxes(hier, tags, tag_bits=1, buffer=1, efficiency=0.7, min_side=4, max_side=32,
                 max_levels=None):
    """Boxes of every level of the new hierarchy (level 0 = the base box)."""
    if max_levels is None:
        max_levels = hier.nlevels
    cur = _dense_tags(hier, np.asarray(tags, dtype=np.uint8), tag_bits)
    n0 = tuple(hier.n0)
    levels = [[((0, 0, 0), tuple(x - 1 for x in n0))]]
    for l in range(max_levels - 1):
        n = tuple(x << l for x in n0)
        inmask = np.zeros(n, dtype=bool)
        for lo, hi in levels[l]:
            inmask[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] = True
        raw = np.full(n, -1, dtype=np.int8)
        for lc in range(min(l, hier.nlevels - 1), -1, -1):
            s = l - lc
            up = cur[lc]
            for ax in range(3):
                up = np.repeat(up, 1 << s, axis=ax)
            raw = np.where(raw < 0, up, raw)
        raw = (raw > 0) & inmask
        ok = _nestable(inmask)
        tg = _dilate(raw, buffer) & ok
        coarse = cluster_level(tg, ok, efficiency, max_side // 2, min_side // 2)
        if not coarse:
            break
        levels.append([(tuple(2 * x for x in lo), tuple(2 * x + 1 for x in hi))
                       for lo, hi in coarse])
    return levels


# -------------------------------------------------------------------- transfer
def _cells(hier):
    """Per level: dict (i,j,k) -> cell index, plus the list of cells."""
    maps = [dict() for _ in range(hier.nlevels)]
    cells = []
    off = 0
    for l, lev in enumerate(hier.levels):
        for lo, hi in lev:
            for k in range(lo[2], hi[2] + 1):
                for j in range(lo[1], hi[1] + 1):
                    for i in range(lo[0], hi[0] + 1):
                        maps[l][(i, j, k)] = off
                        cells.append((l, i, j, k))
                        off += 1
    return maps, cells


def composite(hier, x):
    """Covered cells := mean of their 8 children, finest level first."""
    maps, cells = _cells(hier)
    x = np.array(x, dtype=np.float64)
    for l in range(hier.nlevels - 2, -1, -1):
        for (i, j, k), c in maps[l].items():
            kids = [maps[l + 1].get((2 * i + a, 2 * j + b, 2 * k + e))
                    for e in (0, 1) for b in (0, 1) for a in (0, 1)]
            if kids[0] is not None:
                x[c] = sum(x[q] for q in kids) / 8.0
    return x


def _minmod(a, b):
    if a * b <= 0.0:
        return 0.0
    return a if abs(a) < abs(b) else b


def transfer(old, new, u_old):
    """Transfer a state vector [E, T] from hierarchy `old` to `new`."""
    No, Nn = old.ncells, new.ncells
    u_old = np.asarray(u_old, dtype=np.float64)
    omaps, _ = _cells(old)
    _, ncells = _cells(new)
    out = np.empty(2 * Nn)
    for f in range(2):
        uo = composite(old, u_old[f * No:(f + 1) * No])
        for c, (l, i, j, k) in enumerate(ncells):
            q = (i, j, k)
            if l < old.nlevels and q in omaps[l]:
                out[f * Nn + c] = uo[omaps[l][q]]
                continue
            lc = min(l, old.nlevels) - 1
            while lc >= 0:
                cq = tuple(x >> (l - lc) for x in q)
                if cq in omaps[lc]:
                    break
                lc -= 1
            if lc < 0:
                raise ValueError("a new cell lies in no old cell")
            r = 1 << (l - lc)
            uc = uo[omaps[lc][cq]]
            v = uc
            for d in range(3):
                m = list(cq); m[d] -= 1
                p = list(cq); p[d] += 1
                im, ip = omaps[lc].get(tuple(m)), omaps[lc].get(tuple(p))
                if im is None or ip is None:
                    continue
                # centre of the new cell minus the centre of the old one, in old cells
                off = ((q[d] - cq[d] * r) + 0.5) / r - 0.5
                v += _minmod(uc - uo[im], uo[ip] - uc) * off
            out[f * Nn + c] = v
    return out
