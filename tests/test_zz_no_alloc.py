"""The allocation-free voxeliser, for callers that cannot allocate device memory.

lvr_voxelize_static computes what lvr_voxelize computes, into buffers the
caller owns, using a static device array as scratch. Its output must equal
the allocating entry point's, bit for bit (the voxeliser's parity bar), on
two calls in a row: the second call reuses the array the first call left
behind. This file is collected last so that a failure here cannot hide any
other test.
"""
import numpy as np
import pytest

from tests import _scenes as S

pytestmark = pytest.mark.gpu


def _decode(records):
    r = records.astype(np.uint64)
    cols = [(0, 7), (3, 127), (10, 127), (17, 7), (20, 127), (27, 127), (34, 255), (42, 1)]
    return np.stack([((r >> np.uint64(s)) & np.uint64(m)).astype(np.uint8) for s, m in cols], 1)


def test_static_voxelize_matches_allocating_entry_point():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_1801_01155_gb300 import lvr
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(dev)
    ctx = lvr.Context(0, stream)
    cases = [(S.streamlines(500, 64, 0), 32, 32, 32.0), (S.streamlines(800, 96, 12), (48, 40, 56), 16, 44.0)]
    for ls, R, N, sc in cases:
        gargs = S.grid_args(ls, R, N, scale=sc)
        ref = lvr.export_lineset_numpy(ctx, S.gpu_lineset(lvr, ctx, ls, dev, **gargs))
        nvox = int(np.prod(gargs["res"] if not np.isscalar(gargs["res"]) else [R] * 3))
        xyz = torch.from_numpy(ls.xyz).to(dev)
        attr = torch.from_numpy(ls.attr).to(dev)
        offs = torch.from_numpy(ls.offsets).to(dev)
        off = torch.empty(nvox + 1, dtype=torch.int32, device=dev)
        # too small a buffer: the count comes back, nothing else is written
        small = torch.empty(8, dtype=torch.int64, device=dev)
        with pytest.raises(lvr.LVRError) as ei:
            lvr.lvr_voxelize_static(xyz, attr, offs, lvr.grid_desc(**gargs), off, small, small.clone(), stream)
        assert ei.value.code == lvr.EOVERFLOW and ei.value.n_segments == len(ref["curve"])
        cap = len(ref["curve"]) + 100
        rec = torch.empty(cap, dtype=torch.int64, device=dev)
        key = torch.empty(cap, dtype=torch.int64, device=dev)
        n = lvr.lvr_voxelize_static(xyz, attr, offs, lvr.grid_desc(**gargs), off, rec, key, stream)
        stream.synchronize()
        assert n == len(ref["curve"])
        np.testing.assert_array_equal(off.cpu().numpy().view(np.uint32), ref["offset"])
        r = rec.cpu().numpy()[:n].view(np.uint64)
        k = key.cpu().numpy()[:n].view(np.uint64)
        np.testing.assert_array_equal(_decode(r), ref["fields"])
        np.testing.assert_array_equal((k >> np.uint64(32)).astype(np.uint32), ref["curve"])
        np.testing.assert_array_equal((k & np.uint64(0xffffffff)).astype(np.uint32), ref["ordinal"])
    # a dense bundle: 3000 curves through one voxel, whose list is longer than
    # the shared-memory sort limit and is sorted in place in the caller's buffers
    rng = np.random.default_rng(3)
    n_b = 3000
    xyz_b = np.zeros((n_b, 2, 3), np.float32)
    xyz_b[:, 0, 0], xyz_b[:, 1, 0] = 0.5, 2.5
    xyz_b[:, :, 1] = (0.5 + 0.49 * (rng.random(n_b) - 0.5))[:, None]
    xyz_b[:, :, 2] = (0.5 + 0.49 * (rng.random(n_b) - 0.5))[:, None]
    xyz_b = xyz_b.reshape(-1, 3)
    offs_b = np.arange(0, 2 * n_b + 1, 2, dtype=np.int64)
    g_b = dict(res=(3, 1, 1), bins=128, scale=1.0)
    ref = lvr.export_lineset_numpy(ctx, lvr.lvr_voxelize(ctx, xyz_b, None, offs_b, lvr.grid_desc(**g_b)))
    assert len(ref["curve"]) == n_b
    off = torch.empty(4, dtype=torch.int32, device=dev)
    rec = torch.empty(n_b, dtype=torch.int64, device=dev)
    key = torch.empty(n_b, dtype=torch.int64, device=dev)
    for _ in range(2):
        n = lvr.lvr_voxelize_static(torch.from_numpy(xyz_b).to(dev), None, torch.from_numpy(offs_b).to(dev),
                                    lvr.grid_desc(**g_b), off, rec, key, stream)
        stream.synchronize()
        assert n == n_b
        np.testing.assert_array_equal(off.cpu().numpy().view(np.uint32), ref["offset"])
        np.testing.assert_array_equal(_decode(rec.cpu().numpy().view(np.uint64)), ref["fields"])
        k = key.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal((k >> np.uint64(32)).astype(np.uint32), ref["curve"])
        np.testing.assert_array_equal((k & np.uint64(0xffffffff)).astype(np.uint32), ref["ordinal"])
    # buffers outside the current device's memory are refused before anything runs
    with pytest.raises(lvr.LVRError) as ei:
        lvr.lvr_voxelize_static(torch.from_numpy(xyz_b), None, torch.from_numpy(offs_b).to(dev), lvr.grid_desc(**g_b),
                                off, rec, key, stream)
    assert ei.value.code == lvr.EINVAL
    # too large a grid for the static scratch
    ls = S.streamlines(50, 16, 0)
    with pytest.raises(lvr.LVRError) as ei:
        big = lvr.grid_desc(256, 32, scale=256.0)
        lvr.lvr_voxelize_static(torch.from_numpy(ls.xyz).to(dev), None, torch.from_numpy(ls.offsets).to(dev), big,
                                torch.empty(256 ** 3 + 1, dtype=torch.int32, device=dev),
                                torch.empty(16, dtype=torch.int64, device=dev),
                                torch.empty(16, dtype=torch.int64, device=dev), stream)
    assert ei.value.code == lvr.EINVAL
    ctx.close()
