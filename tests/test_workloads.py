"""Seeded input generators: the layouts the configurations state."""
import numpy as np

from paper_1302_6303_gb300 import workloads as W


def test_material_slices_equal_centre_tests():
    """Integer cube corners are applied as patch slices; that must give the
    same material as testing every cell centre against every cube."""
    for n0 in (16, 32):
        for seed in range(3):
            rng = np.random.default_rng(seed)
            h, _ = W.config_batching(n0, seed=seed, side_lo=4, side_hi=12)
            cubes = W.random_cubes(rng, h.n0, 30, 1, 9, (1.0, 5.0, 10.0))
            cubes.append(((1, 2, 3), [3, 4, 5], 7.0))
            assert np.array_equal(W.material_from_cubes(h, cubes),
                                  W._material_from_centres(h, cubes))
    h = W.tiny_amr(8, three_levels=True)
    cubes = W.paper_blocks(h.n0)
    assert np.array_equal(W.material_from_cubes(h, cubes), W._material_from_centres(h, cubes))


def test_batching_layout_at_full_size():
    """Base 128^3, 3 levels: about 2,000 patches with sides in 8..48 (even,
    aligned to ratio 2), about 44M fine cells, disjoint per level and
    properly nested (each level-2 box, coarsened and grown by one level-1
    cell inside the domain, lies in level 1)."""
    h, z = W.config_batching(128, seed=0)
    assert h.nlevels == 3 and 1800 <= sum(h.nboxes) - 1 <= 2200
    fine = h.ncells - 128 ** 3
    assert 40e6 <= fine <= 48e6
    sides = np.array([[hi[d] - lo[d] + 1 for d in range(3)]
                      for lev in h.levels[1:] for lo, hi in lev])
    assert sides.min() >= 8 and sides.max() <= 48 and np.all(sides % 2 == 0)
    assert 24 <= sides.mean() <= 32
    for l in (1, 2):
        occ = np.zeros(h.level_n(l), dtype=np.uint8)
        for lo, hi in h.levels[l]:
            assert all(lo[d] % 2 == 0 for d in range(3))
            occ[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] += 1
        assert occ.max() == 1
    l1 = np.zeros(h.level_n(1), dtype=bool)
    for lo, hi in h.levels[1]:
        l1[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] = True
    n1 = h.level_n(1)
    for lo, hi in h.levels[2]:
        a = [max(0, lo[d] // 2 - 1) for d in range(3)]
        b = [min(n1[d] - 1, hi[d] // 2 + 1) for d in range(3)]
        assert l1[a[0]:b[0] + 1, a[1]:b[1] + 1, a[2]:b[2] + 1].all()
    assert set(np.unique(z)) <= {1.0, 10.0}
