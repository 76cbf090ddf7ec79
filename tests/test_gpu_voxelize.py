"""CUDA voxeliser and LoD against the FP64 oracle: bit-exact (Secs. 3.1-3.4)."""
import json
import os

import numpy as np
import pytest

from tests import _scenes as S

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g
    g.build()
    from oracle import oracle as O
    from paper_1801_01155_gb300 import lvr
    assert torch.cuda.is_available()
    dev = torch.device("cuda:0")
    ctx = lvr.Context(0, torch.cuda.Stream(dev))
    return lvr, O, ctx, dev


def test_c1_bit_exact(env):
    lvr, O, ctx, dev = env
    ls = S.streamlines(500, 64, 0)
    g = S.grid_args(ls, 32, 32)
    n = S.compare_lineset(lvr, ctx, S.gpu_lineset(lvr, ctx, ls, dev, **g), S.oracle_lineset(O, ls, **g))
    assert n > 3000


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "vox_hand_cases.json")))["cases"],
                         ids=lambda c: c["name"])
def test_hand_cases(env, case):
    lvr, O, ctx, dev = env
    g = lvr.grid_desc(case["res"], case["bins"], scale=1.0, attr_min=case["attr_range"][0],
                      attr_max=case["attr_range"][1])
    attr = None if case["attr"] is None else np.array(case["attr"], np.float32)
    ls = lvr.lvr_voxelize(ctx, np.array(case["xyz"], np.float32), attr, np.array(case["offsets"], np.int64), g)
    e = lvr.export_lineset_numpy(ctx, ls)
    got = [[int(np.searchsorted(e["offset"], i, side="right") - 1), int(e["curve"][i]), int(e["ordinal"][i])]
           + [int(x) for x in e["fields"][i]] for i in range(len(e["curve"]))]
    assert got == case["segments"]


@pytest.mark.parametrize("res,bins,origin,scale,attr", [
    ((20, 33, 17), 2, (-0.1, 0.05, 0.2), 25.0, True),
    ((48, 16, 40), 8, (0.0, 0.0, 0.0), 40.0, False),
    ((24, 24, 24), 128, (0.3, -0.2, 0.1), 31.0, True),
    ((7, 5, 3), 4, (0.0, 0.0, 0.0), 6.0, True),
    ((1, 1, 1), 16, (0.25, 0.25, 0.25), 2.0, True),
])
def test_varied_grids_bit_exact(env, res, bins, origin, scale, attr):
    """Non-cubic grids, offsets and scales that put curves outside the grid,
    every bin count class, with and without attributes."""
    lvr, O, ctx, dev = env
    ls = S.streamlines(300, 80, 11)
    g = dict(res=res, bins=bins, origin=origin, scale=scale,
             attr_min=float(ls.attr.min()) if attr else 0.0, attr_max=float(ls.attr.max()) if attr else 0.0)
    S.compare_lineset(lvr, ctx, S.gpu_lineset(lvr, ctx, ls, dev, **g), S.oracle_lineset(O, ls, **g))


def test_fit_mode(env):
    """Grid fitted to the bounding box keeping its aspect ratio (Sec. 3.1)."""
    lvr, O, ctx, dev = env
    ls = S.streamlines(200, 64, 5)
    gd = lvr.grid_desc(40, 16, fit=True, attr_min=0.0, attr_max=5.0)
    gl = lvr.lvr_voxelize(ctx, ls.xyz, ls.attr, ls.offsets, gd)
    og = O.fit_grid(ls.xyz, 40, 16)
    assert list(gd.res) == list(og.res) and max(gd.res) == 40
    assert list(gd.origin) == list(og.origin) and gd.scale == og.scale
    og.attr_min, og.attr_max = 0.0, 5.0
    S.compare_lineset(lvr, ctx, gl, O.VoxSet(ls.xyz, ls.attr, ls.offsets, og))


def test_empty_and_degenerate(env):
    lvr, O, ctx, dev = env
    g = lvr.grid_desc(8, 8, scale=8.0)
    ls = lvr.lvr_voxelize(ctx, np.zeros((0, 3), np.float32), None, np.zeros(1, np.int64), g)
    assert ls.info().n_segments == 0
    e = lvr.export_lineset_numpy(ctx, ls)
    assert not e["offset"].any()
    # empty curves, single-vertex curves, a curve entirely outside, a curve inside one voxel
    xyz = np.array([[0.5, 0.5, 0.5], [5.0, 5.0, 5.0], [6.0, 5.0, 5.0], [0.31, 0.32, 0.33], [0.34, 0.35, 0.36],
                    [0.05, 0.5, 0.5], [0.95, 0.5, 0.5]], np.float32)
    offs = np.array([0, 0, 1, 3, 5, 5, 7], np.int64)
    gl = lvr.lvr_voxelize(ctx, xyz, None, offs, g)
    ov = O.VoxSet(xyz, None, offs, O.make_grid(8, 8, scale=8.0))
    assert S.compare_lineset(lvr, ctx, gl, ov) == ov.nseg > 0


def test_invalid_inputs_rejected(env):
    lvr, O, ctx, dev = env
    xyz = np.array([[0.1, 0.1, 0.1], [0.9, 0.9, 0.9]], np.float32)
    offs = np.array([0, 2], np.int64)
    g = lambda **k: lvr.grid_desc(**{**dict(res=8, bins=8, scale=8.0), **k})   # noqa: E731
    cases = [
        (np.array([[np.nan, 0, 0], [1, 1, 1]], np.float32), offs, g()),
        (np.array([[0, 0, 0], [np.inf, 1, 1]], np.float32), offs, g()),
        (np.array([[0, 0, 0], [3000.0, 1, 1]], np.float32), offs, g()),      # 24000 voxels away
        (xyz, np.array([0, 3], np.int64), g()),                               # wrong end
        (xyz, np.array([1, 2], np.int64), g()),                               # wrong start
        (xyz, offs, g(bins=12)),
        (xyz, offs, g(bins=256)),
        (xyz, offs, g(res=0)),
        (xyz, offs, g(scale=-1.0)),
        (xyz, offs, g(res=(4096, 4096, 4096))),
    ]
    for x, o, gd in cases:
        with pytest.raises(lvr.LVRError) as ei:
            lvr.lvr_voxelize(ctx, x, None, o, gd)
        assert ei.value.code == lvr.EINVAL
    # non-monotone offsets across three curves
    x3 = np.repeat(xyz, 2, 0)
    with pytest.raises(lvr.LVRError):
        lvr.lvr_voxelize(ctx, x3, None, np.array([0, 3, 2, 4], np.int64), g())
    with pytest.raises(lvr.LVRError):
        lvr.lvr_voxelize(ctx, xyz, np.array([0.0, np.nan], np.float32), offs, g(attr_min=0.0, attr_max=1.0))
    # the context stays usable
    assert lvr.lvr_voxelize(ctx, xyz, None, offs, g()).info().n_segments > 0


def test_host_and_device_inputs_agree(env):
    lvr, O, ctx, dev = env
    ls = S.streamlines(200, 64, 6)
    g = S.grid_args(ls, 24, 16)
    a = lvr.export_lineset_numpy(ctx, S.gpu_lineset(lvr, ctx, ls, dev, **g))
    b = lvr.export_lineset_numpy(ctx, lvr.lvr_voxelize(ctx, ls.xyz, ls.attr, ls.offsets, lvr.grid_desc(**g)))
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_long_lists_sorted(env):
    """Many curves through one voxel: per-voxel lists longer than the
    one-thread and the shared-memory sort limits stay canonical."""
    lvr, O, ctx, dev = env
    rng = np.random.default_rng(3)
    for n in (40, 3000):
        y = 0.5 + 0.49 * (rng.random(n) - 0.5)
        z = 0.5 + 0.49 * (rng.random(n) - 0.5)
        xyz = np.zeros((n, 2, 3), np.float32)
        xyz[:, 0, 0], xyz[:, 1, 0] = 0.5, 2.5
        xyz[:, :, 1] = y[:, None]
        xyz[:, :, 2] = z[:, None]
        xyz = xyz.reshape(-1, 3)
        offs = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
        g = lvr.grid_desc((3, 1, 1), 128, scale=1.0)
        gl = lvr.lvr_voxelize(ctx, xyz, None, offs, g)
        ov = O.VoxSet(xyz, None, offs, O.make_grid((3, 1, 1), 128, scale=1.0))
        assert S.compare_lineset(lvr, ctx, gl, ov) == n


def test_c2_full_size_bit_exact(env):
    """The full 100k x 200 streamline set in a 256^3 grid (N = 32)."""
    lvr, O, ctx, dev = env
    ls = S.streamlines(100_000, 200, 1)
    g = S.grid_args(ls, 256, 32)
    n = S.compare_lineset(lvr, ctx, S.gpu_lineset(lvr, ctx, ls, dev, **g), S.oracle_lineset(O, ls, **g))
    assert n > 10_000_000


def test_512_grid_bit_exact(env):
    """Largest grid of the batched workload (512^3) with a sample of curves."""
    lvr, O, ctx, dev = env
    ls = S.streamlines(4000, 150, 4)
    g = S.grid_args(ls, 512, 32)
    S.compare_lineset(lvr, ctx, S.gpu_lineset(lvr, ctx, ls, dev, **g), S.oracle_lineset(O, ls, **g))


def test_512_full_set_sampled_curves(env):
    """The batched workload's largest set at full size: 2M streamlines x 150
    vertices (seed 23) in a 512^3 grid (N = 32), voxelised in one call as the
    benchmark does. Every segment of 2000 sampled curves, located in the full
    voxelisation, equals the oracle's voxelisation of those curves alone, bit
    for bit (voxel, fields, ordinal, canonical order), and each sampled curve
    has exactly the segments the oracle gives it."""
    import torch

    from paper_1801_01155_gb300 import synth
    lvr, O, ctx, dev = env
    n, nv = 2_000_000, 150
    xyz, attr, offs = synth.make_streamlines_device(n, nv, 23, dev)
    g = dict(res=512, bins=32, origin=(0.0, 0.0, 0.0), scale=512.0,
             attr_min=float(attr.min()), attr_max=float(attr.max()))
    gls = lvr.lvr_voxelize(ctx, xyz, attr, offs, lvr.grid_desc(**g))
    inf = gls.info()
    nseg, nvox = int(inf.n_segments), int(inf.n_voxels)
    assert nseg > 300_000_000
    off = torch.empty(nvox + 1, dtype=torch.int32, device=dev)
    fields = torch.empty((nseg, 8), dtype=torch.uint8, device=dev)
    curve = torch.empty(nseg, dtype=torch.int32, device=dev)
    ordn = torch.empty(nseg, dtype=torch.int32, device=dev)
    lvr.lvr_export_lineset(ctx, gls, off, fields, curve, ordn)
    ctx.sync()
    gls.free()
    sample = np.sort(np.random.default_rng(7).choice(n, 2000, replace=False))
    pick = torch.isin(curve, torch.from_numpy(sample.astype(np.int32)).to(dev)).nonzero().squeeze(1)
    gvox = torch.searchsorted(off[1:].to(torch.int64), pick, right=True).cpu().numpy()
    gfields = fields[pick].cpu().numpy()
    gcurve = curve[pick].cpu().numpy().astype(np.int64)
    gord = ordn[pick].cpu().numpy()
    del fields, curve, ordn, off
    sub = torch.from_numpy(sample).to(dev)
    sxyz = xyz.view(n, nv, 3)[sub].reshape(-1, 3).cpu().numpy()
    sattr = attr.view(n, nv)[sub].reshape(-1).cpu().numpy()
    soffs = np.arange(0, (len(sample) + 1) * nv, nv, dtype=np.int64)
    o = O.VoxSet(sxyz, sattr, soffs, O.make_grid(**g)).export()
    ovox = np.repeat(np.arange(nvox, dtype=np.int64), np.diff(o["offset"].astype(np.int64)))
    assert len(ovox) == len(gvox) > 100_000
    np.testing.assert_array_equal(gvox, ovox)
    np.testing.assert_array_equal(gfields, o["fields"])
    np.testing.assert_array_equal(gcurve, sample[o["curve"].astype(np.int64)])
    np.testing.assert_array_equal(gord, o["ordinal"])


@pytest.mark.parametrize("R,levels", [(32, 3), (37, 4), (256, 3)])
def test_lod(env, R, levels):
    """Counts bit-exact. Float32 sums of n positive terms carry a relative error
    of at most about n * 2^-24; a level sums at most ~14 segments per voxel and
    then 8 children per level, so 4e-6 bounds it."""
    lvr, O, ctx, dev = env
    ls = S.streamlines(100_000, 200, 1) if R == 256 else S.streamlines(500, 64, 0)
    g = S.grid_args(ls, R, 32)
    tf = __import__("paper_1801_01155_gb300.synth", fromlist=["x"]).tf_ramp(0.05, 0.3)
    sig = tf[:, 3].copy()
    gl = S.gpu_lineset(lvr, ctx, ls, dev, **g)
    glod = lvr.lvr_build_lod(ctx, gl, levels, sig)
    olod = O.Lod(S.oracle_lineset(O, ls, **g), levels, sig)
    assert glod.info().levels == levels
    for l in range(levels):
        a, b = lvr.export_lod_numpy(ctx, glod, l), olod.export(l)
        assert tuple(a["dims"]) == b["dims"]
        np.testing.assert_array_equal(a["cnt"], b["cnt"])
        for k in ("len", "dens"):
            np.testing.assert_allclose(a[k], b[k], rtol=4e-6, atol=1e-7)
