"""Readers for the hand-worked clustering cases in tests/golden/br_*.txt and
seeded hierarchies for the transfer tests (layout only, no arithmetic of the
method)."""
from __future__ import annotations

import glob
import os

import numpy as np

from paper_1302_6303_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_case(path):
    base, levels, tagboxes, params, expect = None, {}, [], {}, {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        w = line.split()
        if w[0] == "base":
            base = tuple(int(x) for x in w[1:4])
        elif w[0] == "level":
            l = int(w[1])
            v = [int(x) for x in w[2:8]]
            levels.setdefault(l, []).append((tuple(v[:3]), tuple(v[3:])))
        elif w[0] == "tag":
            v = [int(x) for x in w[1:8]]
            tagboxes.append((v[0], tuple(v[1:4]), tuple(v[4:7])))
        elif w[0] == "params":
            for kv in w[1:]:
                k, v = kv.split("=")
                params[k] = float(v) if "." in v else int(v)
        elif w[0] == "expect":
            l = int(w[1])
            v = [int(x) for x in w[2:8]]
            expect.setdefault(l, []).append((tuple(v[:3]), tuple(v[3:])))
    lev = [[((0, 0, 0), tuple(n - 1 for n in base))]]
    for l in sorted(levels):
        lev.append(levels[l])
    hier = W.Hierarchy(n0=base, levels=lev)
    L, I, J, K = hier.cell_ijk()
    tags = np.zeros(hier.ncells, dtype=np.uint8)
    for l, lo, hi in tagboxes:
        sel = (L == l)
        for d, idx in enumerate((I, J, K)):
            sel &= (idx >= lo[d]) & (idx <= hi[d])
        tags[sel] = 1
    exp = [[((0, 0, 0), tuple(n - 1 for n in base))]]
    for l in sorted(expect):
        exp.append(expect[l])
    return hier, tags, params, exp


def golden_cases():
    return sorted(glob.glob(os.path.join(GOLDEN, "br_*.txt")))


def random_hierarchy(rng, n0, nlevels, count=3, side_lo=2, side_hi=5):
    """Properly nested random hierarchy (one coarse cell of buffer)."""
    levels = [[((0, 0, 0), tuple(n - 1 for n in n0))]]
    for l in range(1, nlevels):
        parent = levels[l - 1]
        n_par = tuple(n << (l - 1) for n in n0)
        inside = np.zeros(n_par, dtype=bool)
        for lo, hi in parent:
            inside[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] = True
        # cells whose 26 neighbours (inside the domain) lie in the parent level
        p = np.pad(inside, 1, constant_values=True)
        ok = inside.copy()
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    ok &= p[1 + di:1 + di + n_par[0], 1 + dj:1 + dj + n_par[1],
                            1 + dk:1 + dk + n_par[2]]
        taken = np.zeros(n_par, dtype=bool)
        boxes = []
        for _ in range(200):
            if len(boxes) == count:
                break
            s = rng.integers(side_lo, side_hi + 1, size=3)
            lo = [int(rng.integers(0, max(1, n_par[d] - s[d] + 1))) for d in range(3)]
            hi = [min(n_par[d] - 1, lo[d] + int(s[d]) - 1) for d in range(3)]
            sl = (slice(lo[0], hi[0] + 1), slice(lo[1], hi[1] + 1), slice(lo[2], hi[2] + 1))
            if ok[sl].all() and not taken[sl].any():
                taken[sl] = True
                boxes.append((tuple(2 * x for x in lo), tuple(2 * x + 1 for x in hi)))
        if not boxes:
            break
        levels.append(boxes)
    return W.Hierarchy(n0=tuple(n0), levels=levels)
