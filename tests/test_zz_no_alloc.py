"""The allocation-free entry point (nrd_wdot_noalloc) against nrd_dot.

Callers that cannot allocate device memory at the point of use (an external
memory manager, latency-critical paths) use the allocation-free variant; it must give the same inner product as the context
call.  This file is collected last so that a failure here comes after every
other test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_dot_matches_nrd_dot_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from oracle.oracle import Oracle
    from paper_1302_6303_gb300 import nrd, workloads as W

    h, z = W.config_amr2(16, seed=3, band=4, ncubes=4)
    ctx = nrd.Context()
    ctx.set_hierarchy_from(h)
    ctx.set_material(torch.from_numpy(z).cuda())
    # leaf-cell volumes, 0 on covered cells: the weights nrd_dot uses
    L, _, _, _ = h.cell_ijk()
    vol = np.array([1.0 / np.prod(h.level_n(l)) for l in range(h.nlevels)])[L]
    leaf = Oracle(h, z).leaf_mask()
    w = torch.from_numpy(np.where(leaf, vol, 0.0).astype(np.float32)).cuda()
    rng = np.random.default_rng(0)
    for trial in range(2):
        x = rng.standard_normal(2 * h.ncells) * (1 + trial)
        y = rng.standard_normal(2 * h.ncells)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ref = ctx.dot(xd, yd)
        got = nrd.wdot_noalloc(xd, yd, w)
        torch.cuda.synchronize()
        scale = float(np.sum(np.concatenate([w.cpu().numpy()] * 2) * np.abs(x * y)))
        assert abs(got.item() - ref) <= 1e-14 * scale, (trial, got.item(), ref)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_capacity_and_handles_empty():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd
    lib = nrd.load()
    import ctypes
    x = torch.zeros(2, dtype=torch.float64, device="cuda")
    w = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the size check happens on the host before any launch
    assert lib.nrd_wdot_noalloc(p(x), p(x), p(w), (1 << 26) + 1, p(out), s) == nrd.EINVAL
    assert lib.nrd_wdot_noalloc(p(x), p(x), p(w), -1, p(out), s) == nrd.EINVAL
    assert lib.nrd_wdot_noalloc(p(x), p(x), p(w), 0, p(out), s) == nrd.OK
    torch.cuda.synchronize()
    assert out.item() == 0.0
