"""Seeded synthetic workloads: patch hierarchies, material fields and states.

This module holds no arithmetic of the method.  It only lays out boxes and
draws seeded inputs (numpy PCG64) shaped like the Marshak-wave problem of
arXiv 1302.6303 Sec. 6 (unit cube, z = 10 blocks in a z = 1 background,
E0 = 1e-5, T0 = E0^(1/4), incoming-flux Robin face at x = 0).  Both the CUDA
path and the CPU oracle consume exactly these arrays.

Vector layout (shared interface): cells of all levels, level-major, patches in
the given order, x fastest inside a patch.  A state vector u holds E for all
cells followed by T for all cells.  Ghost buffers hold, per patch, the six
faces x-, x+, y-, y+, z-, z+; on a face normal to axis d the cells run with
axis (d+1)%3 fastest, then (d+2)%3.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BC_NEUMANN, BC_ROBIN = 0, 1


@dataclass
class Hierarchy:
    """Boxes per level (inclusive lo/hi in that level's index space, ratio 2)."""

    n0: tuple
    levels: list                      # levels[l] = [(lo(3), hi(3)), ...]
    bc_type: list = field(default_factory=lambda: [BC_ROBIN, 0, 0, 0, 0, 0])
    bc_R: list = field(default_factory=lambda: [1.0, 0, 0, 0, 0, 0])

    @property
    def nlevels(self):
        return len(self.levels)

    @property
    def nboxes(self):
        return [len(b) for b in self.levels]

    def boxes_flat(self):
        out = []
        for lev in self.levels:
            for lo, hi in lev:
                out.extend(list(lo) + list(hi))
        return out

    def level_n(self, l):
        return tuple(n << l for n in self.n0)

    def patches(self):
        """(level, lo, hi, cell offset) for every patch in layout order."""
        out, off = [], 0
        for l, lev in enumerate(self.levels):
            for lo, hi in lev:
                out.append((l, tuple(lo), tuple(hi), off))
                off += int(np.prod([hi[d] - lo[d] + 1 for d in range(3)]))
        return out

    @property
    def ncells(self):
        return sum(int(np.prod([hi[d] - lo[d] + 1 for d in range(3)]))
                   for lev in self.levels for lo, hi in lev)

    @property
    def nghosts(self):
        g = 0
        for lev in self.levels:
            for lo, hi in lev:
                n = [hi[d] - lo[d] + 1 for d in range(3)]
                g += 2 * (n[1] * n[2] + n[0] * n[2] + n[0] * n[1])
        return g

    def cell_ijk(self):
        """(level, i, j, k) arrays over all cells in layout order."""
        Ls, Is, Js, Ks = [], [], [], []
        for l, lo, hi, _ in self.patches():
            k, j, i = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1),
                                  np.arange(lo[0], hi[0] + 1), indexing="ij")
            Is.append(i.ravel()); Js.append(j.ravel()); Ks.append(k.ravel())
            Ls.append(np.full(i.size, l))
        return (np.concatenate(Ls), np.concatenate(Is), np.concatenate(Js), np.concatenate(Ks))

    def cell_centres(self):
        """Physical cell centres on [0,1]^3 and the level of each cell."""
        L, I, J, K = self.cell_ijk()
        out = []
        for d, idx in enumerate((I, J, K)):
            n = np.array([self.n0[d] << l for l in range(self.nlevels)])[L]
            out.append((idx + 0.5) / n)
        return L, out[0], out[1], out[2]

    def covered_mask(self):
        """True for cells covered by the next finer level (layout only)."""
        L, I, J, K = self.cell_ijk()
        cov = np.zeros(I.size, dtype=bool)
        for l in range(self.nlevels - 1):
            fine = np.zeros(self.level_n(l + 1), dtype=bool)
            for lo, hi in self.levels[l + 1]:
                fine[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] = True
            sel = L == l
            cov[sel] = fine[2 * I[sel], 2 * J[sel], 2 * K[sel]]
        return cov

    def ghost_count_per_patch(self):
        out = []
        for lev in self.levels:
            for lo, hi in lev:
                n = [hi[d] - lo[d] + 1 for d in range(3)]
                out.append(2 * (n[1] * n[2] + n[0] * n[2] + n[0] * n[1]))
        return out


def uniform(n, bc_type=None, bc_R=None):
    bt = bc_type if bc_type is not None else [BC_ROBIN, 0, 0, 0, 0, 0]
    br = bc_R if bc_R is not None else [1.0, 0, 0, 0, 0, 0]
    if np.isscalar(n):
        n = (n, n, n)
    return Hierarchy(tuple(n), [[((0, 0, 0), tuple(x - 1 for x in n))]], list(bt), list(br))


def all_neumann(h: Hierarchy) -> Hierarchy:
    return Hierarchy(h.n0, h.levels, [0] * 6, [0.0] * 6)


# ------------------------------------------------------------ material fields
def material_from_cubes(hier: Hierarchy, cubes, background=1.0):
    """z per cell: the value of the last cube (in base-cell units, half-open
    [lo, lo+side)) containing the cell centre, else the background."""
    integral = all(float(v).is_integer() for lo, side, _ in cubes
                   for v in list(lo) + list(side if np.ndim(side) else (side,)))
    if not integral:
        return _material_from_centres(hier, cubes, background)
    # integer cube corners: a level-l cell i (centre (i + 1/2) / 2^l base
    # cells, never an integer) lies in [lo, lo + side) exactly when
    # lo 2^l <= i <= (lo + side) 2^l - 1, so each cube is a slice of a patch
    zval = np.full(hier.ncells, background, dtype=np.float32)
    for l, lo, hi, off in hier.patches():
        n = [hi[d] - lo[d] + 1 for d in range(3)]
        zp = zval[off:off + n[0] * n[1] * n[2]].reshape(n[2], n[1], n[0])
        r = 1 << l
        for clo, side, val in cubes:
            sd = side if np.ndim(side) else (side,) * 3
            sl = []
            for d in range(3):
                a = max(int(clo[d]) * r, lo[d])
                b = min((int(clo[d]) + int(sd[d])) * r - 1, hi[d])
                if a > b:
                    break
                sl.append(slice(a - lo[d], b - lo[d] + 1))
            else:
                zp[sl[2], sl[1], sl[0]] = val
    return zval


def _material_from_centres(hier: Hierarchy, cubes, background=1.0):
    L, x, y, zc = hier.cell_centres()
    nb = np.array(hier.n0, dtype=np.float64)
    zval = np.full(x.size, background, dtype=np.float32)
    for lo, side, val in cubes:
        lo = np.asarray(lo, dtype=np.float64)
        sd = np.asarray(side if np.ndim(side) else (side,) * 3, dtype=np.float64)
        inside = np.ones(x.size, dtype=bool)
        for d, c in enumerate((x, y, zc)):
            inside &= (c * nb[d] >= lo[d]) & (c * nb[d] < lo[d] + sd[d])
        zval[inside] = val
    return zval


def random_cubes(rng, n0, count, side_lo, side_hi, values=(10.0,)):
    cubes = []
    for _ in range(count):
        side = int(rng.integers(side_lo, side_hi + 1))
        lo = [int(rng.integers(0, max(1, n0[d] - side + 1))) for d in range(3)]
        val = float(values[int(rng.integers(0, len(values)))])
        cubes.append((lo, side, val))
    return cubes


def paper_blocks(n0):
    """The three z = 10 blocks of the paper's Sec. 6 material layout, in base
    cells (rounded to the base grid)."""
    def blk(x0, x1, y0, y1, z0, z1):
        lo = [int(round(x0 * n0[0])), int(round(y0 * n0[1])), int(round(z0 * n0[2]))]
        hi = [int(round(x1 * n0[0])), int(round(y1 * n0[1])), int(round(z1 * n0[2]))]
        return (lo, [max(1, hi[d] - lo[d]) for d in range(3)], 10.0)
    return [blk(0.0625, 0.2, 0.375, 0.625, 0.375, 0.625),
            blk(0.125, 0.375, 0.0, 1.0, 0.0, 0.125),
            blk(0.125, 0.375, 0.0, 1.0, 0.875, 1.0)]


# -------------------------------------------------------------------- states
E0 = 1e-5


def initial_state(hier: Hierarchy, E0=E0):
    """Sec. 3.1 initial condition: E = E0, T = E0^(1/4) everywhere."""
    N = hier.ncells
    u = np.empty(2 * N)
    u[:N] = E0
    u[N:] = E0 ** 0.25
    return u


def front_state(hier: Hierarchy, seed=0, noise=0.05, front=0.3, width=0.08):
    """A positive Marshak-like state: a smooth front in x plus seeded
    cell-wise noise, E in [~1e-5, ~1], T near E^(1/4)."""
    rng = np.random.default_rng(seed)
    L, x, y, z = hier.cell_centres()
    N = x.size
    prof = 0.5 * (1.0 + np.tanh((front - x) / width))
    wob = 1.0 + 0.2 * np.sin(2 * np.pi * y) * np.cos(2 * np.pi * z)
    E = E0 + (1.0 - E0) * prof * wob
    E = E * (1.0 + noise * rng.uniform(-1, 1, N))
    T = np.abs(E) ** 0.25 * (1.0 + noise * rng.uniform(-1, 1, N))
    return np.concatenate([E, T])


def random_direction(hier: Hierarchy, seed=1):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(2 * hier.ncells)


# --------------------------------------------------------------- hierarchies
def split_extent(length, lo, hi, rng):
    """Seeded split of `length` into even parts with sizes in [lo, hi]."""
    for _ in range(1000):
        parts, rem = [], length
        while rem > 0:
            if rem <= hi and rem >= lo:
                if rng.random() < 0.5 or rem - lo < lo:
                    parts.append(rem)
                    break
            s = int(rng.integers(lo // 2, hi // 2 + 1)) * 2
            s = min(s, rem)
            parts.append(s)
            rem -= s
        if all(lo <= p <= hi and p % 2 == 0 for p in parts) and sum(parts) == length:
            return parts
    raise ValueError("cannot split %d into [%d,%d]" % (length, lo, hi))


def tile_region(lo, hi, side_lo, side_hi, rng):
    """Tile the box [lo, hi] (inclusive, even-aligned) with boxes whose sides
    lie in [side_lo, side_hi]."""
    cuts = []
    for d in range(3):
        ln = hi[d] - lo[d] + 1
        if ln <= side_hi:
            cuts.append([ln])
        else:
            cuts.append(split_extent(ln, side_lo, side_hi, rng))
    boxes = []
    z0 = lo[2]
    for sz in cuts[2]:
        y0 = lo[1]
        for sy in cuts[1]:
            x0 = lo[0]
            for sx in cuts[0]:
                boxes.append(((x0, y0, z0), (x0 + sx - 1, y0 + sy - 1, z0 + sz - 1)))
                x0 += sx
            y0 += sy
        z0 += sz
    return boxes


def config_single_level(n=32, seed=0, ncubes=2, cube_side=8, values=(10.0,)):
    """One level n^3: z = 1 plus `ncubes` seeded cubes, Robin R = 1 at x = 0."""
    rng = np.random.default_rng(seed)
    h = uniform(n)
    cubes = random_cubes(rng, h.n0, ncubes, cube_side, cube_side, values)
    return h, material_from_cubes(h, cubes)


def config_256(n=256, seed=0):
    """Single level: 64 cubes with z in {1, 5, 10}, sides U{8..32} (scaled to n)."""
    rng = np.random.default_rng(seed)
    h = uniform(n)
    s_lo, s_hi = max(1, 8 * n // 256), max(1, 32 * n // 256)
    cubes = random_cubes(rng, h.n0, 64, s_lo, s_hi, (1.0, 5.0, 10.0))
    return h, material_from_cubes(h, cubes)


def config_amr2_cubes(n0=64, seed=0, band=8, ncubes=20):
    """Hierarchy and material cubes of `config_amr2` (the cubes re-evaluate
    the same material on any other hierarchy of the same base grid)."""
    rng = np.random.default_rng(seed)
    fine_lo = (0, 0, 0)
    fine_hi = (2 * band - 1, 2 * n0 - 1, 2 * n0 - 1)
    side_lo, side_hi = (16, 32) if n0 >= 16 else (4, 8)
    boxes = tile_region(fine_lo, fine_hi, side_lo, side_hi, rng)
    h = Hierarchy((n0, n0, n0), [[((0, 0, 0), (n0 - 1,) * 3)], boxes])
    s_lo, s_hi = max(1, 4 * n0 // 64), max(1, 12 * n0 // 64)
    cubes = random_cubes(rng, h.n0, ncubes, s_lo, s_hi)
    return h, cubes


def config_amr2(n0=64, seed=0, band=8, ncubes=20):
    """Two levels, base n0^3, ratio 2: the fine level tiles the Marshak band
    x in [0, band) base cells with patches of 16^3-32^3 fine cells; z = 10 in
    `ncubes` seeded cubes of side 4-12 base cells on z = 1."""
    h, cubes = config_amr2_cubes(n0, seed, band, ncubes)
    return h, material_from_cubes(h, cubes)


def tiny_amr(n0=8, three_levels=False, concave=True):
    """Small hierarchies for oracle pins and parity: an L-shaped pair of fine
    patches (a concave corner) and optionally a third level."""
    lv1 = [((4, 4, 4), (11, 11, 7))]
    if concave:
        lv1.append(((4, 4, 8), (7, 7, 11)))
    levels = [[((0, 0, 0), (n0 - 1,) * 3)], lv1]
    if three_levels:
        levels.append([((12, 12, 10), (17, 17, 13))])
    return Hierarchy((n0, n0, n0), levels)


def boundary_amr(n0=8):
    """Fine patches touching the physical boundary (Robin face x = 0) and a
    sibling pair sharing a face."""
    lv1 = [((0, 0, 0), (5, 7, 7)), ((6, 0, 0), (9, 7, 7)), ((0, 8, 0), (3, 11, 5))]
    return Hierarchy((n0, n0, n0), [[((0, 0, 0), (n0 - 1,) * 3)], lv1])


def random_nested_level(rng, parent_boxes, n_fine, count, side_lo, side_hi, tries=200000,
                        margin=1):
    """Seeded rejection sampling of `count` non-overlapping fine boxes (sides
    U{side_lo..side_hi}, even, aligned to ratio 2) properly nested in the
    parent level (its boxes in parent index space): every fine box coarsened
    and grown by `margin` coarse cells must lie inside one parent box."""
    occ = np.zeros(n_fine, dtype=bool)
    boxes = []
    pb = [(np.array(lo), np.array(hi)) for lo, hi in parent_boxes]
    t = 0
    while len(boxes) < count and t < tries:
        t += 1
        p = pb[int(rng.integers(0, len(pb)))]
        side = [2 * int(rng.integers((side_lo + 1) // 2, side_hi // 2 + 1)) for _ in range(3)]
        # coarse extent of the fine box must fit inside the parent box with margin
        clo = p[0] + margin
        chi = p[1] - margin
        span = [int(chi[d] - clo[d] + 1) for d in range(3)]
        csd = [s // 2 for s in side]
        if any(csd[d] > span[d] for d in range(3)):
            continue
        c0 = [int(clo[d] + rng.integers(0, span[d] - csd[d] + 1)) for d in range(3)]
        lo = tuple(2 * c0[d] for d in range(3))
        hi = tuple(lo[d] + side[d] - 1 for d in range(3))
        sl = tuple(slice(lo[d], hi[d] + 1) for d in range(3))
        if occ[sl].any():
            continue
        occ[sl] = True
        boxes.append((lo, hi))
    return boxes


def tile_region_guillotine(lo, hi, side_lo, side_hi, rng):
    """Tile the box [lo, hi] (inclusive, even-aligned, even extents) with
    boxes whose sides lie in [side_lo, side_hi]: seeded slabs along z, each
    slab cut into seeded rows along y, each row into seeded lengths along x.
    Each box draws its own x side and shares its y side with its row and its
    z side with its slab; every side is even, so the boxes align to ratio 2."""
    boxes = []
    z0 = lo[2]
    for sz in split_extent(hi[2] - lo[2] + 1, side_lo, side_hi, rng):
        y0 = lo[1]
        for sy in split_extent(hi[1] - lo[1] + 1, side_lo, side_hi, rng):
            x0 = lo[0]
            for sx in split_extent(hi[0] - lo[0] + 1, side_lo, side_hi, rng):
                boxes.append(((x0, y0, z0), (x0 + sx - 1, y0 + sy - 1, z0 + sz - 1)))
                x0 += sx
            y0 += sy
        z0 += sz
    return boxes


def config_batching(n0=128, seed=0, side_lo=8, side_hi=48):
    """Three levels, base n0^3, ratio 2, patches with sides drawn uniformly
    (even) from [side_lo, side_hi] per axis.  Level 1 tiles the slab
    x < 168/256 of the domain (at n0 = 128: 256 x 256 x 168 level-1 cells,
    about 500 patches); level 2 tiles x < 124/512 of the domain inside it
    (124 x 512 x 512 level-2 cells, about 1,450 patches), which keeps one
    level-1 cell between the level-2 region and the level-1 boundary inside
    the domain (proper nesting).  About 2,000 patches and 44M fine cells at
    n0 = 128.  z = 10 in 64 seeded cubes of side 4-12 (scaled) base cells on
    z = 1."""
    rng = np.random.default_rng(seed)
    base = [((0, 0, 0), (n0 - 1,) * 3)]
    n1, n2 = 2 * n0, 4 * n0
    x1 = max(2, 2 * int(round(168 * n1 / 256 / 2)))
    x2 = max(2, min(2 * (x1 - 1), 2 * int(round(124 * n2 / 512 / 2))))
    l1 = tile_region_guillotine((0, 0, 0), (x1 - 1, n1 - 1, n1 - 1), side_lo, side_hi, rng)
    l2 = tile_region_guillotine((0, 0, 0), (x2 - 1, n2 - 1, n2 - 1), side_lo, side_hi, rng)
    h = Hierarchy((n0, n0, n0), [base, l1, l2])
    s_lo, s_hi = max(1, 4 * n0 // 64), max(1, 12 * n0 // 64)
    cubes = random_cubes(rng, h.n0, 64, s_lo, s_hi)
    return h, material_from_cubes(h, cubes)


def config_adjoint(n0=96, seed=0, nbox=8):
    """Two levels, base n0^3: `nbox` fine boxes of 16^3-32^3 fine cells near
    x = 0 (seeded), z = 10 in 20 seeded cubes; the functional box is an
    interior 16^3 (base-cell) box."""
    rng = np.random.default_rng(seed)
    base = [((0, 0, 0), (n0 - 1,) * 3)]
    region = [((0, 0, 0), (max(3, n0 // 6), n0 - 1, n0 - 1))]
    s_lo, s_hi = (16, 32) if n0 >= 64 else (4, 8)
    l1 = random_nested_level(rng, region, (2 * n0,) * 3, nbox, s_lo, s_hi, margin=0)
    h = Hierarchy((n0, n0, n0), [base, l1])
    s_lo, s_hi = max(1, 4 * n0 // 64), max(1, 12 * n0 // 64)
    cubes = random_cubes(rng, h.n0, 20, s_lo, s_hi)
    c = n0 // 2 - n0 // 12
    fbox = ((c,) * 3, (c + max(1, n0 // 6) - 1,) * 3)
    return h, material_from_cubes(h, cubes), fbox
