"""Pins of the oracle's traversal counters, which fix the algorithmic bytes of
the roofline (8 B per voxel visited, one record per record tested).

With early termination off and translucent tubes every primary ray walks
the grid from entry to exit, so the voxels it visits are exactly the cells
whose box the ray crosses over an interval of positive length after leaving
the eye, and the records it tests are those cells' stored segments. Both are
recounted here by a slab test of the ray against every cell of the grid.
"""
import numpy as np

from paper_1801_01155_gb300 import synth


def test_voxels_and_records_equal_a_slab_test_over_all_cells(orc):
    R = 12
    ls = synth.make_streamlines(200, 48, seed=4)
    g = orc.make_grid(R, 32, scale=float(R), attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))
    vs = orc.VoxSet(ls.xyz, ls.attr, ls.offsets, g)
    counts = np.diff(vs.export()["offset"].astype(np.int64))
    W, H = 40, 30
    cam = synth.orbit_view((R, R, R), W, H)
    view = orc.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], W, H, cam["light_dir"])
    pix = orc.pixel_grid(0, 0, W, H)
    tf = synth.tf_ramp(0.01, 0.02)
    _, tie, cnt = orc.render(vs, None, view, orc.make_rdesc(0.2, tf, ert_alpha=2.0), pix)
    idx = np.arange(R ** 3)
    lo = np.stack([idx % R, (idx // R) % R, idx // (R * R)], 1).astype(np.float64)
    hi = lo + 1.0
    nvox = nrec = 0
    for i, j in pix:
        o, d = orc.primary_ray(view, int(i), int(j))
        o, d = o.astype(np.float64), d.astype(np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            t1, t2 = (lo - o) / d, (hi - o) / d
        tn = np.maximum(np.nanmax(np.minimum(t1, t2), 1), 0.0)
        tf_ = np.nanmin(np.maximum(t1, t2), 1)
        crossed = tf_ - tn > 1e-9
        nvox += int(crossed.sum())
        nrec += int(counts[crossed].sum())
    assert nvox > 5000 and nrec > 1000
    assert int(cnt[0]) == nvox
    assert int(cnt[1]) == nrec


def test_lod_samples_of_shadow_marches_in_closed_form(orc):
    """One straight opaque tube along x at y = z = 8 + 16.5/32 (its quantised
    axis) in a 16^3 grid with a 3-level LoD, lit straight from +y, at a density
    so low that no march reaches O = 1. By the soft-shadow reading (samples at
    s = 1, 2, 4 on levels 0, 1, 2, then every 4 voxels, ending where a sample
    would leave the density's support [-2, 18]) every hit, whose y lies in
    [axis - r, axis + r], takes its samples at y + 1, 2, 4 and 8 and stops
    before y + 12: exactly 4 per hit."""
    R, r = 16, 0.2
    xyz = np.array([[0.5, 8.5, 8.5], [15.5, 8.5, 8.5]], np.float32)
    attr = np.zeros(2, np.float32)
    vs = orc.VoxSet(xyz, attr, np.array([0, 2], np.int64), orc.make_grid(R, 32, scale=1.0))
    tf = synth.tf_ramp(1.0, 1.0)
    lod = orc.Lod(vs, 3, np.full(256, 1e-3, np.float32))
    W, H = 64, 48
    view = orc.make_view((8.0, 8.5, 40.0), (8.0, 8.5, 8.5), (0.0, 1.0, 0.0), 20.0, W, H, (0.0, -1.0, 0.0))
    pix = orc.pixel_grid(0, 0, W, H)
    _, tie, cnt = orc.render(vs, lod, view, orc.make_rdesc(r, tf, opaque=True, shadows=True), pix)
    assert int(cnt[3]) > 100
    assert int(cnt[2]) == 4 * int(cnt[3])


def test_lod_samples_with_ao_in_closed_form(orc):
    """The same kind of tube in the middle of a 32^3 grid (support [-2, 34]),
    now with 16 AO rays of radius 15 per hit as well: an AO ray samples at
    s = 1, 2, 4, 8, 12 and stops because s = 16 exceeds the radius (no sample
    point can leave the support), a shadow march toward +y at s = 1, 2, 4,
    8, 12, 16 and stops before leaving at y + 20: 6 + 16 x 5 = 86 per hit."""
    R, r = 32, 0.2
    xyz = np.array([[12.5, 16.5, 16.5], [20.5, 16.5, 16.5]], np.float32)
    attr = np.zeros(2, np.float32)
    vs = orc.VoxSet(xyz, attr, np.array([0, 2], np.int64), orc.make_grid(R, 32, scale=1.0))
    lod = orc.Lod(vs, 3, np.full(256, 1e-3, np.float32))
    W, H = 64, 48
    view = orc.make_view((16.5, 16.5, 60.0), (16.5, 16.5, 16.5), (0.0, 1.0, 0.0), 6.0, W, H, (0.0, -1.0, 0.0))
    pix = orc.pixel_grid(0, 0, W, H)
    rd = orc.make_rdesc(r, synth.tf_ramp(1.0, 1.0), opaque=True, shadows=True, ao=True, ao_rays=16, ao_radius=15.0)
    _, tie, cnt = orc.render(vs, lod, view, rd, pix)
    assert int(cnt[3]) > 100
    assert int(cnt[2]) == 86 * int(cnt[3])
