"""Ray casting on the largest grid of the batched-views workload: 512^3
voxels (134 M), tube radius 0.1 (Secs. 4-5 at that size).

100k streamlines x 150 vertices are voxelised into a 512^3 grid with 32^2
face bins; a 1920 x 1080 view with transparency (alpha 0.05-0.3, early
termination at 0.99), soft shadows and 16 traced AO rays per hit is rendered
in the default launch configuration and in the autotuner's usual pick
(16-byte records, 4x8 ray tiles), and 2000 sampled pixels are compared with
the FP64 oracle. One batched view of the same frame must equal its single
render bit for bit.
"""
import numpy as np
import pytest

from paper_1801_01155_gb300 import synth
from tests import _scenes as S

pytestmark = pytest.mark.gpu

R, RADIUS = 512, 0.1


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g
    g.build()
    from oracle import oracle as O
    from paper_1801_01155_gb300 import lvr
    dev = torch.device("cuda:0")
    return lvr, O, lvr.Context(0, torch.cuda.Stream(dev)), dev


@pytest.fixture(scope="module")
def c5(env):
    lvr, O, ctx, dev = env
    ls = S.streamlines(100_000, 150, 23)
    g = S.grid_args(ls, R, 32)
    tf = synth.tf_ramp(0.05, 0.3)
    sig = synth.sigma_lut(tf)
    gls = S.gpu_lineset(lvr, ctx, ls, dev, **g)
    ovs = S.oracle_lineset(O, ls, **g)
    nseg = S.compare_lineset(lvr, ctx, gls, ovs)
    glod = lvr.lvr_build_lod(ctx, gls, 3, sig)
    olod = O.Lod(ovs, 3, sig)
    yield dict(ls=ls, tf=tf, gls=gls, ovs=ovs, glod=glod, olod=olod, nseg=nseg)
    glod.free()
    gls.free()


def test_grid_512_full_frame_sampled(env, c5):
    import torch
    lvr, O, ctx, dev = env
    assert c5["nseg"] > 10_000_000   # the grid is well filled: tens of millions of segments
    lvr.lvr_lineset_layout(ctx, c5["gls"], lvr.LAYOUT_AOS16)
    cam = synth.orbit_view((R, R, R), 1920, 1080)
    lv, ov, _ = S.views(cam)
    rng = np.random.default_rng(5)
    pix = np.stack([rng.integers(0, 1920, 2000), rng.integers(0, 1080, 2000)], 1).astype(np.int32)
    rd = O.make_rdesc(RADIUS, c5["tf"], ert_alpha=0.99, shadows=True, ao=True)
    ref, tie, _, alt = O.render(c5["ovs"], c5["olod"], ov, rd, pix, alts=True)
    assert (ref[:, 3] > 0.5).mean() > 0.3
    frames = []
    for kw in (dict(), dict(layout=lvr.LAYOUT_AOS16, tile=(4, 8))):
        out = torch.empty((1080, 1920, 4), dtype=torch.float32, device=dev)
        desc = lvr.make_desc(RADIUS, c5["tf"], ert_alpha=0.99, shadows=True, ao_mode=1, **kw)
        lvr.lvr_render(ctx, c5["gls"], c5["glod"], lv, desc, out)
        ctx.sync()
        frames.append(out.cpu().numpy())
        got = frames[-1][pix[:, 1], pix[:, 0]]
        S.check_image(got, ref, tie, what=f"512^3 sampled {kw}", alt=alt)
    # record layouts decode to the same face points: the two frames are identical
    assert np.array_equal(frames[0], frames[1])
    # the same view as a one-item batch equals its single render
    desc = lvr.make_desc(RADIUS, c5["tf"], ert_alpha=0.99, shadows=True, ao_mode=1,
                         layout=lvr.LAYOUT_AOS16, tile=(4, 8))
    outb = torch.empty((1080, 1920, 4), dtype=torch.float32, device=dev)
    b = lvr.lvr_batch_create(ctx, [(c5["gls"], c5["glod"], lv, desc, None, outb)])
    lvr.lvr_batch_render(ctx, b)
    ctx.sync()
    assert np.array_equal(outb.cpu().numpy(), frames[1])
    b.free()
