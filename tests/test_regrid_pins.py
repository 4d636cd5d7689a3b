"""Pins of the oracle's regridding (Sec. 5) against hand-worked cases and the
properties the paper fixes: clustering covers every tag with disjoint,
properly nested boxes; the conservative linear refinement conserves the leaf
integral of E and T, creates no new extrema (no negative undershoots), is
exact for linear data and the identity on an unchanged hierarchy."""
import numpy as np
import pytest

from oracle import regrid as R
from paper_1302_6303_gb300 import workloads as W
from regrid_cases import golden_cases, load_case, random_hierarchy


def vols(h):
    L = h.cell_ijk()[0]
    return np.array([1.0 / np.prod(h.level_n(l)) for l in range(h.nlevels)])[L]


# ------------------------------------------------------------------ clustering
@pytest.mark.parametrize("path", golden_cases(), ids=lambda p: p.split("/")[-1])
def test_clustering_hand_worked(path):
    hier, tags, params, expect = load_case(path)
    got = R.regrid_boxes(hier, tags, **params)
    assert [[(tuple(lo), tuple(hi)) for lo, hi in lev] for lev in got] == expect


def _check_cover_nesting(hier, tags, levels, buffer, max_side):
    """Every dilated tag that may hold a finer level is covered; boxes are
    disjoint, inside their level, properly nested and within max_side."""
    n0 = hier.n0
    for l in range(1, len(levels)):
        nl = tuple(n << l for n in n0)
        occ = np.zeros(nl, dtype=np.int32)
        for lo, hi in levels[l]:
            assert all(hi[d] - lo[d] + 1 <= max_side for d in range(3))
            assert all(lo[d] % 2 == 0 and hi[d] % 2 == 1 for d in range(3))
            occ[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] += 1
        assert occ.max() == 1                              # disjoint
        # proper nesting: the coarse footprint grown by one cell (clipped to
        # the domain) lies in level l-1
        npar = tuple(n << (l - 1) for n in n0)
        par = np.zeros(npar, dtype=bool)
        for lo, hi in levels[l - 1]:
            par[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] = True
        for lo, hi in levels[l]:
            clo = [max(0, lo[d] // 2 - 1) for d in range(3)]
            chi = [min(npar[d] - 1, hi[d] // 2 + 1) for d in range(3)]
            assert par[clo[0]:chi[0] + 1, clo[1]:chi[1] + 1, clo[2]:chi[2] + 1].all()
    # level-0 tags (dilated) are all refined when level 0 is the whole domain
    L, I, J, K = hier.cell_ijk()
    if len(levels) > 1:
        fine = np.zeros(tuple(2 * n for n in n0), dtype=bool)
        for lo, hi in levels[1]:
            fine[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] = True
        sel = (L == 0) & (tags > 0)
        for i, j, k in zip(I[sel], J[sel], K[sel]):
            assert fine[2 * i, 2 * j, 2 * k]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_clustering_random_properties(seed):
    rng = np.random.default_rng(seed)
    hier = W.uniform(16)
    # tags: a few random blobs
    L, I, J, K = hier.cell_ijk()
    tags = np.zeros(hier.ncells, dtype=np.uint8)
    for _ in range(4):
        c = rng.integers(2, 14, size=3)
        r = rng.integers(1, 3)
        sel = (abs(I - c[0]) <= r) & (abs(J - c[1]) <= r) & (abs(K - c[2]) <= r)
        tags[sel] = 1
    for eff in (0.5, 0.7, 0.9):
        levels = R.regrid_boxes(hier, tags, buffer=1, efficiency=eff, min_side=2, max_side=16,
                                max_levels=2)
        _check_cover_nesting(hier, tags, levels, 1, 16)
        # each accepted box is the bounding box of its tags: every face plane
        # holds a tag of the dilated set, so the box cannot shrink
        dil = np.zeros(hier.n0, dtype=bool)
        for i, j, k in zip(I[tags > 0], J[tags > 0], K[tags > 0]):
            dil[max(0, i - 1):i + 2, max(0, j - 1):j + 2, max(0, k - 1):k + 2] = True
        for lo, hi in levels[1]:
            clo, chi = [x // 2 for x in lo], [x // 2 for x in hi]
            sub = dil[clo[0]:chi[0] + 1, clo[1]:chi[1] + 1, clo[2]:chi[2] + 1]
            for d in range(3):
                s = np.moveaxis(sub, d, 0)
                assert s[0].any() and s[-1].any()
    # higher efficiency never covers more cells than lower
    vol = []
    for eff in (0.3, 0.95):
        levels = R.regrid_boxes(hier, tags, buffer=1, efficiency=eff, min_side=2, max_side=32,
                                max_levels=2)
        vol.append(sum(np.prod([hi[d] - lo[d] + 1 for d in range(3)]) for lo, hi in levels[1]))
    assert vol[1] <= vol[0]


def test_clustering_three_levels_nesting():
    rng = np.random.default_rng(5)
    hier = random_hierarchy(rng, (12, 12, 12), 3, count=3, side_lo=3, side_hi=5)
    L, I, J, K = hier.cell_ijk()
    tags = (rng.random(hier.ncells) < 0.08).astype(np.uint8)
    levels = R.regrid_boxes(hier, tags, buffer=1, efficiency=0.6, min_side=2, max_side=16,
                            max_levels=4)
    assert len(levels) >= 2
    _check_cover_nesting(hier, tags, levels, 1, 16)
    # the result is itself a valid hierarchy
    W.Hierarchy(n0=hier.n0, levels=levels).covered_mask()


def test_clustering_no_tags_gives_base_only():
    hier = W.uniform(8)
    levels = R.regrid_boxes(hier, np.zeros(hier.ncells, np.uint8), max_levels=3)
    assert levels == [[((0, 0, 0), (7, 7, 7))]]


def test_clustering_min_side():
    """Cuts that would leave a part narrower than min_side/2 are not taken:
    two blobs 3 planes apart stay in one box when min_side/2 = 4."""
    hier = W.uniform(16)
    L, I, J, K = hier.cell_ijk()
    tags = np.zeros(hier.ncells, np.uint8)
    tags[(I <= 1) & (J <= 1) & (K <= 1)] = 1
    tags[(I >= 5) & (I <= 6) & (J <= 1) & (K <= 1)] = 1
    lv = R.regrid_boxes(hier, tags, buffer=0, efficiency=0.9, min_side=8, max_side=32,
                        max_levels=2)
    assert lv[1] == [((0, 0, 0), (13, 3, 3))]
    lv = R.regrid_boxes(hier, tags, buffer=0, efficiency=0.9, min_side=2, max_side=32,
                        max_levels=2)
    assert lv[1] == [((0, 0, 0), (3, 3, 3)), ((10, 0, 0), (13, 3, 3))]


# -------------------------------------------------------------------- transfer
def _state(h, rng):
    N = h.ncells
    return np.concatenate([rng.uniform(0.1, 2.0, N), rng.uniform(0.5, 1.5, N)])


def _leaf(h):
    return ~h.covered_mask()


def test_transfer_identity():
    rng = np.random.default_rng(0)
    h = W.tiny_amr(8, three_levels=True)
    u = _state(h, rng)
    v = R.transfer(h, h, u)
    leaf = np.concatenate([_leaf(h)] * 2)
    assert np.array_equal(v[leaf], u[leaf])
    # covered cells hold the mean of their children
    N = h.ncells
    for f in range(2):
        c = R.composite(h, u[f * N:(f + 1) * N])
        assert np.array_equal(v[f * N:(f + 1) * N], c)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_transfer_conserves_leaf_integral(seed):
    rng = np.random.default_rng(seed)
    a = random_hierarchy(rng, (8, 8, 8), 3)
    b = random_hierarchy(rng, (8, 8, 8), 3)
    u = _state(a, rng)
    v = R.transfer(a, b, u)
    Va, Vb = vols(a), vols(b)
    la, lb = _leaf(a), _leaf(b)
    for f in range(2):
        ua = u[f * a.ncells:(f + 1) * a.ncells]
        vb = v[f * b.ncells:(f + 1) * b.ncells]
        assert abs(np.sum((Va * ua)[la]) - np.sum((Vb * vb)[lb])) <= 1e-14 * np.sum(Va * ua)
        # no new extrema, positivity kept
        assert vb.min() >= ua[la].min() * (1 - 1e-15) and vb.max() <= ua[la].max() * (1 + 1e-15)


def test_transfer_linear_exact():
    """Minmod slopes of linear data are the exact slopes: refined cells away
    from the domain boundary take the linear function at their centres."""
    a = W.uniform(8)
    b = W.Hierarchy(n0=(8, 8, 8), levels=[[((0, 0, 0), (7, 7, 7))],
                                          [((4, 4, 4), (11, 11, 11))],
                                          [((10, 10, 10), (13, 13, 13))]])
    La, x, y, z = a.cell_centres()
    f = lambda x, y, z: 1.0 + 0.5 * x - 0.25 * y + 0.75 * z
    u = np.concatenate([f(x, y, z), 2.0 + f(x, y, z)])
    v = R.transfer(a, b, u)
    Lb, xb, yb, zb = b.cell_centres()
    N = b.ncells
    assert np.allclose(v[:N], f(xb, yb, zb), rtol=0, atol=4e-15)
    assert np.allclose(v[N:], 2.0 + f(xb, yb, zb), rtol=0, atol=4e-15)


def test_transfer_extremum_flat():
    """At a local maximum minmod gives zero slopes: the children copy it."""
    a = W.uniform(6)
    La, I, J, K = a.cell_ijk()
    E = np.ones(a.ncells)
    E[(I == 2) & (J == 2) & (K == 2)] = 5.0
    u = np.concatenate([E, E])
    b = W.Hierarchy(n0=(6, 6, 6), levels=[[((0, 0, 0), (5, 5, 5))], [((2, 2, 2), (7, 7, 7))]])
    v = R.transfer(a, b, u)
    Lb, Ib, Jb, Kb = b.cell_ijk()
    kids = (Lb == 1) & (Ib // 2 == 2) & (Jb // 2 == 2) & (Kb // 2 == 2)
    assert np.all(v[:b.ncells][kids] == 5.0)
    # neighbours of the peak: one-sided slopes of opposite sign on the
    # peak's axis -> zero slope there, exact copies too
    nb = (Lb == 1) & (Ib // 2 == 3) & (Jb // 2 == 2) & (Kb // 2 == 2)
    assert np.all(v[:b.ncells][nb] == 1.0)


def test_transfer_coarsening_takes_means():
    rng = np.random.default_rng(3)
    a = W.tiny_amr(8)
    u = _state(a, rng)
    b = W.uniform(8)
    v = R.transfer(a, b, u)
    N = a.ncells
    La, I, J, K = a.cell_ijk()
    for c in np.nonzero(La == 0)[0][:50]:
        kids = (La == 1) & (I // 2 == I[c]) & (J // 2 == J[c]) & (K // 2 == K[c])
        if kids.any():
            assert kids.sum() == 8
            assert abs(v[c] - u[:N][kids].mean()) <= 1e-15 * u[:N][kids].mean()
        else:
            assert v[c] == u[c]
