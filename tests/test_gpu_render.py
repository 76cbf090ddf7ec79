"""CUDA ray-caster against the FP64 oracle (Secs. 4-5).

RGBA must agree within 2e-3 per channel outside near-tie pixels, which the
oracle flags (silhouettes, voxel-face ownership, depth order) and which are
capped at 0.1 % of the pixels.
"""
import numpy as np
import pytest

from paper_1801_01155_gb300 import synth
from tests import _scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g
    g.build()
    from oracle import oracle as O
    from paper_1801_01155_gb300 import lvr
    dev = torch.device("cuda:0")
    ctx = lvr.Context(0, torch.cuda.Stream(dev))
    return lvr, O, ctx, dev


class Scene:
    def __init__(self, env, n, nv, seed, R, N=32, levels=3, alpha=(0.05, 0.3)):
        lvr, O, ctx, dev = env
        self.ls = S.streamlines(n, nv, seed)
        g = S.grid_args(self.ls, R, N)
        self.R = R
        self.tf = synth.tf_ramp(*alpha)
        self.gls = S.gpu_lineset(lvr, ctx, self.ls, dev, **g)
        self.ovs = S.oracle_lineset(O, self.ls, **g)
        sig = synth.sigma_lut(self.tf)
        self.glod = lvr.lvr_build_lod(ctx, self.gls, levels, sig)
        self.olod = O.Lod(self.ovs, levels, sig)

    def render(self, env, cam, crop=None, radius=0.15, tile=(0, 0), counters=False, flips=False, **kw):
        import torch
        lvr, O, ctx, dev = env
        lv, ov, pix = S.views(cam, crop)
        w, h = (crop[2], crop[3]) if crop else (cam["width"], cam["height"])
        out = torch.empty((h, w, 4), dtype=torch.float32, device=dev)
        cnt = torch.zeros(4, dtype=torch.int64, device=dev) if counters else None
        reps = kw.pop("reps_oracle", None)
        okw = {k: v for k, v in kw.items() if k != "ao_mode"}
        if kw.get("ao_mode"):
            okw["ao"] = True
        if reps is not None:
            okw["reps"] = reps
        desc = lvr.make_desc(radius, self.tf, tile=tile, **kw)
        lvr.lvr_render(ctx, self.gls, self.glod, lv, desc, out, counters=cnt)
        ctx.sync()
        rd = O.make_rdesc(radius, self.tf, **okw)
        # kept for check_image: the oracle's flip budget of hard-shadow
        # near-ties and its second right answer of one-pair depth ties
        ref, tie, ocnt, self.flip, self.alt = O.render(self.ovs, self.olod, ov, rd, pix, flips=True, alts=True)
        got = out.cpu().numpy().reshape(-1, 4)
        return got, ref, tie, (cnt.cpu().numpy() if counters else None), ocnt


@pytest.fixture(scope="module")
def c1(env):
    return Scene(env, 500, 64, 0, 32, alpha=(1.0, 1.0))


@pytest.fixture(scope="module")
def c1t(env):
    return Scene(env, 500, 64, 0, 32)


@pytest.fixture(scope="module")
def c2(env):
    return Scene(env, 100_000, 200, 1, 256)


def test_c1_opaque_full_image(env, c1):
    """Config 1: 500 x 64 streamlines, 32^3, r = 0.2, opaque, 128 x 128."""
    cam = synth.orbit_view((32, 32, 32), 128, 128)
    got, ref, tie, gc, oc = c1.render(env, cam, radius=0.2, opaque=True, counters=True)
    S.check_image(got, ref, tie, what="c1 opaque", alt=c1.alt)
    assert (ref[:, 3] > 0).mean() > 0.3
    # the same voxels and records are read (float32 may pass a voxel edge on
    # the other side, so allow a few extra or fewer)
    np.testing.assert_allclose(gc, oc.astype(np.float64), rtol=2e-3)


def test_c3_illumination_small(env, c1t):
    """Config 3 at reduced size: c1 set + 3-level LoD, transparent, soft
    shadows and 16 traced AO rays per hit."""
    cam = synth.orbit_view((32, 32, 32), 192, 108)
    got, ref, tie, gc, oc = c1t.render(env, cam, radius=0.2, ert_alpha=0.99, shadows=True, ao_mode=1,
                                       counters=True)
    S.check_image(got, ref, tie, what="c3 small", alt=c1t.alt)
    # traversal counters match the oracle's within the tie pixels' share
    np.testing.assert_allclose(gc, oc.astype(np.float64), rtol=2e-3)


def test_c3_full_frame_sampled(env, c1t):
    """Config 3 at 1920 x 1080, launched as the benchmark launches it; the
    oracle checks a sample of 3000 pixels."""
    import torch
    lvr, O, ctx, dev = env
    cam = synth.orbit_view((32, 32, 32), 1920, 1080)
    lv, ov, _ = S.views(cam)
    out = torch.empty((1080, 1920, 4), dtype=torch.float32, device=dev)
    lvr.lvr_render(ctx, c1t.gls, c1t.glod, lv, lvr.make_desc(0.2, c1t.tf, ert_alpha=0.99, shadows=True, ao_mode=1), out)
    ctx.sync()
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(0, 1920, 3000), rng.integers(0, 1080, 3000)], 1).astype(np.int32)
    ref, tie, _, alt = O.render(c1t.ovs, c1t.olod, ov, O.make_rdesc(0.2, c1t.tf, ert_alpha=0.99, shadows=True, ao=True),
                                pix, alts=True)
    got = out.cpu().numpy()[pix[:, 1], pix[:, 0]]
    S.check_image(got, ref, tie, what="c3 sampled", alt=alt)


def test_c2_crop_transparent(env, c2):
    """Config 2: 100k x 200 streamlines, 256^3, r = 0.15, alpha 0.05-0.3,
    termination at 0.99, 1920 x 1080 view; the central 256 x 256 crop."""
    cam = synth.orbit_view((256, 256, 256), 1920, 1080)
    got, ref, tie, gc, oc = c2.render(env, cam, crop=(832, 412, 256, 256), ert_alpha=0.99, counters=True)
    S.check_image(got, ref, tie, what="c2 crop", alt=c2.alt)
    assert (ref[:, 3] > 0.9).mean() > 0.5
    np.testing.assert_allclose(gc, oc.astype(np.float64), rtol=2e-3)


def test_c2_crop_shadows_ao(env, c2):
    """The benchmark workload (config 2 set, transparent, soft shadows, 16 AO
    rays) on a 128 x 128 crop."""
    cam = synth.orbit_view((256, 256, 256), 1920, 1080)
    got, ref, tie, gc, oc = c2.render(env, cam, crop=(896, 476, 128, 128), ert_alpha=0.99, shadows=True,
                                      ao_mode=1, counters=True)
    S.check_image(got, ref, tie, what="c2 crop AO", alt=c2.alt)
    np.testing.assert_allclose(gc, oc.astype(np.float64), rtol=2e-3)


def test_c2_full_frame_sampled(env, c2):
    """Full 1080p frame of the benchmark workload in the benchmark's launch
    configurations (the default one, and the autotuner's usual pick: 16-byte
    records with 4x8 ray tiles); 2000 sampled pixels checked by the oracle."""
    import torch
    lvr, O, ctx, dev = env
    lvr.lvr_lineset_layout(ctx, c2.gls, lvr.LAYOUT_AOS16)
    cam = synth.orbit_view((256, 256, 256), 1920, 1080)
    lv, ov, _ = S.views(cam)
    rng = np.random.default_rng(1)
    pix = np.stack([rng.integers(0, 1920, 2000), rng.integers(0, 1080, 2000)], 1).astype(np.int32)
    ref, tie, _, alt = O.render(c2.ovs, c2.olod, ov, O.make_rdesc(0.15, c2.tf, ert_alpha=0.99, shadows=True, ao=True),
                                pix, alts=True)
    for kw in (dict(), dict(layout=lvr.LAYOUT_AOS16, tile=(4, 8))):
        out = torch.empty((1080, 1920, 4), dtype=torch.float32, device=dev)
        desc = lvr.make_desc(0.15, c2.tf, ert_alpha=0.99, shadows=True, ao_mode=1, **kw)
        lvr.lvr_render(ctx, c2.gls, c2.glod, lv, desc, out)
        ctx.sync()
        got = out.cpu().numpy()[pix[:, 1], pix[:, 0]]
        S.check_image(got, ref, tie, what=f"c2 sampled {kw}", alt=alt)


def test_counting_does_not_change_the_image(env, c1t):
    """A render that fills the traversal counters and one that does not run
    different kernels (the second drops the counting and the AO march's
    support tests, relying on the padded coarsest LoD copy): the same bits,
    on a 32^3 grid where many AO rays of radius 15 leave the grid, in both
    record layouts and in a batch (which never counts)."""
    import torch
    lvr, O, ctx, dev = env
    assert c1t.glod.info().levels == 3
    cam = synth.orbit_view((32, 32, 32), 96, 80)
    lv, _, _ = S.views(cam)
    for layout in (0, 1):
        if layout:
            lvr.lvr_lineset_layout(ctx, c1t.gls, lvr.LAYOUT_AOS16)
        desc = lvr.make_desc(0.2, c1t.tf, shadows=True, ao_mode=1, ao_radius=15.0, layout=layout)
        imgs = []
        for counted in (True, False):
            out = torch.empty((80, 96, 4), dtype=torch.float32, device=dev)
            cnt = torch.zeros(4, dtype=torch.int64, device=dev) if counted else None
            lvr.lvr_render(ctx, c1t.gls, c1t.glod, lv, desc, out, counters=cnt)
            ctx.sync()
            imgs.append(out.cpu().numpy())
        assert imgs[0][..., 3].max() > 0.5
        np.testing.assert_array_equal(imgs[1], imgs[0])
        out = torch.empty((80, 96, 4), dtype=torch.float32, device=dev)
        b = lvr.lvr_batch_create(ctx, [(c1t.gls, c1t.glod, lv, desc, None, out)])
        lvr.lvr_batch_render(ctx, b)
        ctx.sync()
        np.testing.assert_array_equal(out.cpu().numpy(), imgs[0])


def test_tile_shapes_bit_identical(env, c1t):
    import torch
    lvr, O, ctx, dev = env
    cam = synth.orbit_view((32, 32, 32), 100, 70)
    lv, _, _ = S.views(cam)
    imgs = []
    for tile in ((8, 4), (4, 8), (16, 2), (32, 1)):
        out = torch.empty((70, 100, 4), dtype=torch.float32, device=dev)
        lvr.lvr_render(ctx, c1t.gls, c1t.glod, lv, lvr.make_desc(0.2, c1t.tf, shadows=True, ao_mode=1, tile=tile), out)
        ctx.sync()
        imgs.append(out.cpu().numpy())
    for im in imgs[1:]:
        np.testing.assert_array_equal(im, imgs[0])


def test_host_output_and_crops_agree(env, c1t):
    """Host output buffers, and crops (including ragged ones at the image
    edge), reproduce the same pixels as a full device render."""
    import torch
    lvr, O, ctx, dev = env
    cam = synth.orbit_view((32, 32, 32), 77, 53)
    lv, _, _ = S.views(cam)
    desc = lvr.make_desc(0.2, c1t.tf, shadows=True, ao_mode=1)
    full = torch.empty((53, 77, 4), dtype=torch.float32, device=dev)
    lvr.lvr_render(ctx, c1t.gls, c1t.glod, lv, desc, full)
    ctx.sync()
    host = np.empty((53, 77, 4), np.float32)
    lvr.lvr_render(ctx, c1t.gls, c1t.glod, lv, desc, host)
    np.testing.assert_array_equal(host, full.cpu().numpy())
    for crop in ((0, 0, 13, 7), (60, 40, 17, 13), (5, 50, 72, 3)):
        lvc, _, _ = S.views(cam, crop)
        part = np.empty((crop[3], crop[2], 4), np.float32)
        lvr.lvr_render(ctx, c1t.gls, c1t.glod, lvc, desc, part)
        np.testing.assert_array_equal(part, full.cpu().numpy()[crop[1]:crop[1] + crop[3], crop[0]:crop[0] + crop[2]])


def test_edge_cases(env, c1t):
    """Camera inside the grid, rays that miss the grid, an empty line set."""
    import torch
    lvr, O, ctx, dev = env
    inside = dict(eye=np.array([16.3, 15.2, 17.1], np.float32), at=np.array([30.0, 2.0, 5.0], np.float32),
                  up=np.array([0, 1, 0], np.float32), fovy_deg=70.0, width=64, height=48,
                  light_dir=np.array([0.2, -1, 0.1], np.float32))
    got, ref, tie, _, _ = c1t.render(env, inside, radius=0.2, ert_alpha=0.99, shadows=True, ao_mode=1)
    S.check_image(got, ref, tie, what="camera inside", alt=c1t.alt)
    away = dict(inside, eye=np.array([100.0, 100.0, 100.0], np.float32), at=np.array([200.0, 100, 100], np.float32))
    got, ref, tie, _, _ = c1t.render(env, away, radius=0.2)
    np.testing.assert_array_equal(got, np.tile([1, 1, 1, 0], (64 * 48, 1)).astype(np.float32))
    empty = lvr.lvr_voxelize(ctx, np.zeros((0, 3), np.float32), None, np.zeros(1, np.int64),
                             lvr.grid_desc(16, 8, scale=16.0))
    cam = synth.orbit_view((16, 16, 16), 32, 32)
    lv, _, _ = S.views(cam)
    out = np.empty((32, 32, 4), np.float32)
    lvr.lvr_render(ctx, empty, None, lv, lvr.make_desc(0.2, c1t.tf, bg=(0.2, 0.3, 0.4)), out)
    np.testing.assert_array_equal(out.reshape(-1, 4), np.tile([0.2, 0.3, 0.4, 0], (1024, 1)).astype(np.float32))


def test_many_hits_in_one_voxel(env):
    """More hits per voxel than the shared-memory list holds: the overflow path
    must keep depth order. 60 parallel lines through a 3-voxel row, seen
    along the lines with wide tubes and no early termination."""
    import torch
    lvr, O, ctx, dev = env
    rng = np.random.default_rng(9)
    n = 60
    xyz = np.zeros((n, 2, 3), np.float32)
    xyz[:, 0, 0], xyz[:, 1, 0] = 0.2, 2.8
    xyz[:, :, 1] = (0.1 + 0.8 * rng.random(n))[:, None]
    xyz[:, :, 2] = (0.1 + 0.8 * rng.random(n))[:, None]
    attr = np.repeat(rng.random(n).astype(np.float32), 2)
    offs = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    g = dict(res=(3, 1, 1), bins=64, scale=1.0, attr_min=0.0, attr_max=1.0)
    gl = lvr.lvr_voxelize(ctx, xyz.reshape(-1, 3), attr, offs, lvr.grid_desc(**g))
    ov = O.VoxSet(xyz.reshape(-1, 3), attr, offs, O.make_grid(**g))
    tf = synth.tf_ramp(0.02, 0.05)
    cam = dict(eye=np.array([1.5, 0.5, 6.0], np.float32), at=np.array([1.5, 0.5, 0.5], np.float32),
               up=np.array([0, 1, 0], np.float32), fovy_deg=12.0, width=48, height=32,
               light_dir=np.array([0.3, -1, -0.2], np.float32))
    lv, ovw, pix = S.views(cam)
    out = np.empty((32, 48, 4), np.float32)
    lvr.lvr_render(ctx, gl, None, lv, lvr.make_desc(0.3, tf, ert_alpha=2.0), out)
    ref, tie, cnt, alt = O.render(ov, None, ovw, O.make_rdesc(0.3, tf, ert_alpha=2.0), pix, alts=True)
    assert cnt[3] / len(pix) > 10
    S.check_image(out, ref, tie, what="overflow path", alt=alt)


def test_invalid_render_arguments(env, c1t):
    lvr, O, ctx, dev = env
    cam = synth.orbit_view((32, 32, 32), 16, 16)
    lv, _, _ = S.views(cam)
    out = np.empty((16, 16, 4), np.float32)
    bad = [
        (lvr.make_desc(0.0, c1t.tf), c1t.glod, lv),
        (lvr.make_desc(0.2, c1t.tf, shadows=True), None, lv),
        (lvr.make_desc(0.2, c1t.tf, ao_mode=1, ao_rays=0), c1t.glod, lv),
        (lvr.make_desc(0.2, c1t.tf, ao_mode=1, ao_rays=33), c1t.glod, lv),
        (lvr.make_desc(0.2, c1t.tf, tile=(5, 5)), c1t.glod, lv),
        (lvr.make_desc(0.2, c1t.tf), c1t.glod, S.views(cam, (10, 10, 8, 8))[0]),
    ]
    for desc, lod, view in bad:
        with pytest.raises(lvr.LVRError) as ei:
            lvr.lvr_render(ctx, c1t.gls, lod, view, desc, out)
        assert ei.value.code == lvr.EINVAL


def test_still_camera_mode_matches_oracle(env, c1t, c1):
    """Camera at rest (Sec. 4.1): neighbouring voxels' segments and one hit per
    line id per voxel; transparent with shadows and AO, and opaque."""
    cam = synth.orbit_view((32, 32, 32), 192, 108)
    got, ref, tie, gc, oc = c1t.render(env, cam, radius=0.2, ert_alpha=0.99, shadows=True, ao_mode=1,
                                       still=True, counters=True)
    S.check_image(got, ref, tie, what="still transparent", alt=c1t.alt)
    # voxels visited, LoD samples, hits; records tested at rest are the
    # neighbour-list entries, a subset of the 27-voxel neighbourhoods
    # the oracle counts
    np.testing.assert_allclose(gc[[0, 2, 3]], oc[[0, 2, 3]].astype(np.float64), rtol=2e-3)
    assert 0 < gc[1] <= oc[1] * 1.002
    got, ref, tie, _, _ = c1.render(env, synth.orbit_view((32, 32, 32), 128, 128), radius=0.2, opaque=True,
                                    still=True)
    S.check_image(got, ref, tie, what="still opaque", alt=c1.alt)


def test_still_camera_neighbour_lists(env, c1t):
    """The camera-at-rest neighbour lists: lists built for a larger radius
    serve a smaller one with the same image as lists built for it; at radius
    0.45 (tubes reaching far into the neighbours) the image matches the
    oracle's search over all 26 neighbours; bad radii are refused."""
    import torch
    lvr, O, ctx, dev = env
    cam = synth.orbit_view((32, 32, 32), 96, 64)
    lv, _, _ = S.views(cam)

    def frame(gls, r):
        out = torch.empty((64, 96, 4), dtype=torch.float32, device=dev)
        lvr.lvr_render(ctx, gls, c1t.glod, lv, lvr.make_desc(r, c1t.tf, ert_alpha=0.99, shadows=True, still=True), out)
        ctx.sync()
        return out.cpu().numpy()

    wide = S.gpu_lineset(lvr, ctx, c1t.ls, dev, **S.grid_args(c1t.ls, 32, 32))
    lvr.lvr_lineset_neighbours(ctx, wide, 0.45)
    narrow = S.gpu_lineset(lvr, ctx, c1t.ls, dev, **S.grid_args(c1t.ls, 32, 32))
    lvr.lvr_lineset_neighbours(ctx, narrow, 0.2)
    assert np.array_equal(frame(wide, 0.2), frame(narrow, 0.2))
    # a larger radius than the lists hold rebuilds them
    assert np.array_equal(frame(narrow, 0.45), frame(wide, 0.45))
    got, ref, tie, _, _ = c1t.render(env, cam, radius=0.45, ert_alpha=0.99, shadows=True, still=True)
    # tubes of radius 0.45 overlap their neighbours' heavily, so more hits
    # have near-equal entry depths: 12 of these 6144 pixels hold one such
    # pair, and either order is right
    S.check_image(got, ref, tie, what="still r=0.45", alt=c1t.alt)
    for r in (0.0, -1.0, float("nan")):
        with pytest.raises(lvr.LVRError) as ei:
            lvr.lvr_lineset_neighbours(ctx, wide, r)
        assert ei.value.code == lvr.EINVAL


def test_still_camera_mode_layouts_agree(env, c1t):
    import torch
    lvr, O, ctx, dev = env
    lvr.lvr_lineset_layout(ctx, c1t.gls, lvr.LAYOUT_AOS16)
    cam = synth.orbit_view((32, 32, 32), 96, 64)
    lv, _, _ = S.views(cam)
    outs = []
    for layout in (0, 1):
        out = torch.empty((64, 96, 4), dtype=torch.float32, device=dev)
        lvr.lvr_render(ctx, c1t.gls, c1t.glod, lv, lvr.make_desc(0.2, c1t.tf, ert_alpha=0.99, shadows=True,
                                                                  ao_mode=1, still=True, layout=layout), out)
        ctx.sync()
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_sphere_ao_field_matches_oracle(env, c1t):
    """Sec. 5.3's spherical per-voxel AO (100 rays, radius 5): every voxel's
    value against the oracle's float64 field."""
    lvr, O, ctx, dev = env
    lvr.lvr_lod_ao_field(ctx, c1t.glod, 100, 5.0)
    got = lvr.export_ao_field_numpy(ctx, c1t.glod).astype(np.float64)
    ref = O.ao_sphere_field(c1t.olod, 100, 5.0)
    assert ref.min() < 0.9 and ref.max() > 0.99
    assert np.abs(got - ref).max() <= 1e-5


def test_render_with_sphere_ao_field(env, c1t):
    import torch
    lvr, O, ctx, dev = env
    lvr.lvr_lod_ao_field(ctx, c1t.glod, 100, 5.0)
    field = O.ao_sphere_field(c1t.olod, 100, 5.0)
    cam = synth.orbit_view((32, 32, 32), 192, 108)
    lv, ov, pix = S.views(cam)
    out = torch.empty((108, 192, 4), dtype=torch.float32, device=dev)
    lvr.lvr_render(ctx, c1t.gls, c1t.glod, lv, lvr.make_desc(0.2, c1t.tf, ert_alpha=0.99, shadows=True, ao_mode=3),
                   out)
    ctx.sync()
    ref, tie, _ = O.render(c1t.ovs, c1t.olod, ov, O.make_rdesc(0.2, c1t.tf, ert_alpha=0.99, shadows=True,
                                                                 ao_field=field), pix)
    S.check_image(out.cpu().numpy().reshape(-1, 4), ref, tie, what="spherical AO field")
    with pytest.raises(lvr.LVRError):     # the field must be built first
        other = lvr.lvr_build_lod(ctx, c1t.gls, 3, synth.sigma_lut(c1t.tf))
        lvr.lvr_render(ctx, c1t.gls, other, lv, lvr.make_desc(0.2, c1t.tf, ao_mode=3), out)


@pytest.mark.parametrize("scene", ["c1t", "c2"])
def test_rep_lines_bit_exact(env, scene, request):
    """Representative lines of every LoD level (Sec. 3.4) equal the oracle's
    byte for byte (integer arithmetic on both sides)."""
    sc = request.getfixturevalue(scene)
    lvr, O, ctx, dev = env
    lvr.lvr_lod_rep_lines(ctx, sc.glod, sc.gls)
    reps = O.Reps(sc.ovs, 3)
    for level in range(3):
        got = lvr.export_rep_lines_numpy(ctx, sc.glod, level)
        ref = reps.export(level)
        assert np.array_equal(got[:, :7], ref), f"level {level}"
        assert not got[:, 7].any()
        assert 0.01 < ref[:, 0].mean()


@pytest.mark.parametrize("level", [0, 1, 2])
def test_rep_line_shadows_match_oracle(env, c1, c1t, level):
    """Hard shadows against the representative lines of one level (Sec. 5.2,
    first approach), opaque and transparent with traced AO."""
    lvr, O, ctx, dev = env
    for sc in (c1, c1t):
        lvr.lvr_lod_rep_lines(ctx, sc.glod, sc.gls)
        if not hasattr(sc, "oreps"):
            sc.oreps = O.Reps(sc.ovs, 3)
    cam = synth.orbit_view((32, 32, 32), 128, 128)
    import torch
    for sc, dkw, okw in ((c1, dict(opaque=True), dict(opaque=True)),
                         (c1t, dict(ert_alpha=0.99, ao_mode=1), dict(ert_alpha=0.99, ao=True))):
        lv, ov, pix = S.views(cam)
        out = torch.empty((128, 128, 4), dtype=torch.float32, device=dev)
        lvr.lvr_render(ctx, sc.gls, sc.glod, lv, lvr.make_desc(0.2, sc.tf, shadow_level=level, **dkw), out)
        ctx.sync()
        ref, tie, _, flip = O.render(sc.ovs, sc.olod, ov,
                                     O.make_rdesc(0.2, sc.tf, reps=sc.oreps, shadow_level=level, **okw), pix,
                                     flips=True)
        got = out.cpu().numpy().reshape(-1, 4)
        # binary visibility: pixels with a hit within 1e-3 voxel of a shadow
        # edge are compared within the oracle's flip budget
        S.check_image(got, ref, tie, flip=flip, what=f"rep shadows level {level}")
        # the shadows are there: against the unshadowed frame some pixels darken
        plain, _, _ = O.render(sc.ovs, sc.olod, ov, O.make_rdesc(0.2, sc.tf, **okw), pix)
        assert (ref[:, :3] < plain[:, :3] - 1e-3).any(1).mean() > 0.01


def test_rep_line_shadows_c2_crop(env, c2):
    """The config-2 set (256^3) with level-1 representative-line shadows on a
    128 x 128 crop of the 1080p view. Opaque: about 1 % of the pixels hold a
    hit within 1e-3 voxel of a shadow edge. Transparent: 20-40 hits per pixel
    each walk tens of densely filled cells, so about 40 % of the pixels hold
    such a hit. A hit's visibility is binary and enters only its own diffuse
    term, so those pixels are compared within 2e-3 plus the oracle's bound on
    what their near-tie visibilities can change (Sec. 5.2, first approach);
    pixels with any other near-tie stay under the usual 0.1 % cap."""
    lvr, O, ctx, dev = env
    lvr.lvr_lod_rep_lines(ctx, c2.glod, c2.gls)
    reps = O.Reps(c2.ovs, 3)
    cam = synth.orbit_view((256, 256, 256), 1920, 1080)
    got, ref, tie, _, _ = c2.render(env, cam, crop=(896, 476, 128, 128), opaque=True, shadow_level=1,
                                    reps_oracle=reps, flips=True)
    S.check_image(got, ref, tie, flip=c2.flip, what="c2 crop rep shadows, opaque", alt=c2.alt)
    got, ref, tie, _, _ = c2.render(env, cam, crop=(896, 476, 128, 128), ert_alpha=0.99, shadow_level=1,
                                    reps_oracle=reps, flips=True)
    S.check_image(got, ref, tie, flip=c2.flip, what="c2 crop rep shadows, transparent", alt=c2.alt)


def test_rep_line_shadows_invalid(env, c1t):
    import torch
    lvr, O, ctx, dev = env
    cam = synth.orbit_view((32, 32, 32), 16, 16)
    lv, _, _ = S.views(cam)
    out = torch.empty((16, 16, 4), dtype=torch.float32, device=dev)
    fresh = lvr.lvr_build_lod(ctx, c1t.gls, 3, synth.sigma_lut(c1t.tf))
    bad = [(fresh, lvr.make_desc(0.2, c1t.tf, shadow_level=0)),          # lines not built
           (c1t.glod, lvr.make_desc(0.2, c1t.tf, shadow_level=3)),       # level outside the LoD
           (c1t.glod, lvr.make_desc(0.2, c1t.tf, shadow_level=-1)),
           (None, lvr.make_desc(0.2, c1t.tf, shadow_level=0)),
           (c1t.glod, lvr.make_desc(0.2, c1t.tf, shadow_level=0, still=True))]   # no camera-at-rest variant
    lvr.lvr_lod_rep_lines(ctx, c1t.glod, c1t.gls)
    for lod, desc in bad:
        with pytest.raises(lvr.LVRError) as ei:
            lvr.lvr_render(ctx, c1t.gls, lod, lv, desc, out)
        assert ei.value.code == lvr.EINVAL
    d = lvr.make_desc(0.2, c1t.tf)
    d.shadows = 3
    with pytest.raises(lvr.LVRError):
        lvr.lvr_render(ctx, c1t.gls, c1t.glod, lv, d, out)
    with pytest.raises(lvr.LVRError):
        lvr.export_rep_lines_numpy(ctx, fresh, 0)


def test_rep_line_shadows_tiles_agree(env, c1t):
    """The lighting phase splits a walk over 1-8 lanes depending on how many
    hits a warp holds, which changes with the ray tile: the images agree bit
    for bit."""
    import torch
    lvr, O, ctx, dev = env
    lvr.lvr_lod_rep_lines(ctx, c1t.glod, c1t.gls)
    cam = synth.orbit_view((32, 32, 32), 160, 96)
    lv, _, _ = S.views(cam)
    outs = []
    for tile in ((8, 4), (32, 1), (4, 8)):
        out = torch.empty((96, 160, 4), dtype=torch.float32, device=dev)
        lvr.lvr_render(ctx, c1t.gls, c1t.glod, lv, lvr.make_desc(0.2, c1t.tf, ert_alpha=0.99, shadow_level=1,
                                                                  tile=tile), out)
        ctx.sync()
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_rep_lines_of_an_empty_line_set(env):
    """Curves entirely outside the grid: no segments, no representative
    lines, and shadows 2 leave the (empty) frame unshadowed."""
    import torch
    lvr, O, ctx, dev = env
    xyz = torch.tensor([[40.0, 40.0, 40.0], [41.0, 40.5, 40.0]], dtype=torch.float32, device=dev)
    offs = torch.tensor([0, 2], dtype=torch.int64, device=dev)
    ls = lvr.lvr_voxelize(ctx, xyz, None, offs, lvr.grid_desc(res=16, bins=32, scale=1.0))
    lod = lvr.lvr_build_lod(ctx, ls, 2, synth.sigma_lut(synth.tf_ramp()))
    lvr.lvr_lod_rep_lines(ctx, lod, ls)
    for level in (0, 1):
        assert not lvr.export_rep_lines_numpy(ctx, lod, level).any()
    out = torch.empty((16, 16, 4), dtype=torch.float32, device=dev)
    lvr.lvr_render(ctx, ls, lod, S.views(synth.orbit_view((16, 16, 16), 16, 16))[0],
                   lvr.make_desc(0.2, synth.tf_ramp(), shadow_level=1), out)
    ctx.sync()
    assert np.all(out.cpu().numpy()[..., 3] == 0.0)
