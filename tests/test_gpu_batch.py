"""Batched persistent rendering, record layouts and the autotuner.

A batch renders every view exactly as lvr_render renders it alone (same
kernel code per tile, deterministic per pixel), so outputs are compared
bit for bit with single renders, which the oracle pins elsewhere; one view
is also checked against the oracle directly. The 16-byte record layout
decodes to the same face points as the packed one for power-of-two bin
counts, so its images are bit-identical too.
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
    return lvr, O, lvr.Context(0, torch.cuda.Stream(dev)), dev


class Set:
    def __init__(self, env, n, nv, seed, R, N=32):
        lvr, O, ctx, dev = env
        self.ls = S.streamlines(n, nv, seed)
        self.g = S.grid_args(self.ls, R, N)
        self.R = R
        self.tf = synth.tf_ramp(0.05, 0.3)
        self.gls = S.gpu_lineset(lvr, ctx, self.ls, dev, **self.g)
        self.glod = lvr.lvr_build_lod(ctx, self.gls, 3, synth.sigma_lut(self.tf))


@pytest.fixture(scope="module")
def sets(env):
    lvr, O, ctx, dev = env
    a, b = Set(env, 500, 64, 0, 32), Set(env, 800, 64, 3, 48)
    for s in (a, b):
        lvr.lvr_lineset_layout(ctx, s.gls, lvr.LAYOUT_AOS16)
    return a, b


def _view(lvr, st, w, h, k, crop=None):
    cam = synth.orbit_view((st.R,) * 3, w, h)
    ang = 0.7 * k
    c = np.array([st.R / 2.0] * 3)
    eye = c + (np.array(cam["eye"]) - c) @ np.array([[np.cos(ang), 0, -np.sin(ang)], [0, 1, 0],
                                                      [np.sin(ang), 0, np.cos(ang)]])
    cam["eye"] = [float(x) for x in eye]
    return lvr.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], w, h, cam["light_dir"], crop=crop), cam


def _single(env, st, view, desc, model, h, w):
    import torch
    lvr, O, ctx, dev = env
    out = torch.full((h, w, 4), -1.0, dtype=torch.float32, device=dev)
    lvr.lvr_render(ctx, st.gls, st.glod, view, desc, out, ao_model=model)
    ctx.sync()
    return out.cpu().numpy()


def test_aos16_layout_is_bit_identical(env, sets):
    lvr, O, ctx, dev = env
    st = sets[0]
    view, _ = _view(lvr, st, 160, 96, 0)
    for kw in (dict(shadows=True, ao_mode=1), dict(opaque=True)):
        a = _single(env, st, view, lvr.make_desc(0.2, st.tf, layout=0, **kw), None, 96, 160)
        b = _single(env, st, view, lvr.make_desc(0.2, st.tf, layout=1, **kw), None, 96, 160)
        assert np.array_equal(a, b)
        assert (a[..., 3] > 0).mean() > 0.2


def test_layout_argument_checks(env):
    lvr, O, ctx, dev = env
    st = Set(env, 200, 32, 5, 24)
    with pytest.raises(lvr.LVRError):      # unknown layout
        lvr.lvr_lineset_layout(ctx, st.gls, 7)
    with pytest.raises(lvr.LVRError):      # rendering with 16-byte records needs them built
        _single(env, st, _view(lvr, st, 32, 32, 0)[0], lvr.make_desc(0.2, st.tf, layout=1), None, 32, 32)


def _entries(env, sets, desc_kw, model=None, layout=0):
    import torch
    lvr, O, ctx, dev = env
    shapes = [(96, 64, (8, 4), None), (200, 120, (32, 1), None), (33, 17, (4, 8), None),
              (256, 144, (16, 2), (40, 20, 100, 70)), (64, 64, (8, 4), None), (120, 90, (4, 8), None)]
    ents, singles = [], []
    for k, (w, h, tile, crop) in enumerate(shapes):
        st = sets[k % 2]
        view, _ = _view(lvr, st, w, h, k, crop=crop)
        desc = lvr.make_desc(0.2 if k % 2 == 0 else 0.15, st.tf, tile=tile, layout=layout, **desc_kw)
        ow, oh = (crop[2], crop[3]) if crop else (w, h)
        out = torch.full((oh, ow, 4), -1.0, dtype=torch.float32, device=dev)
        ents.append((st.gls, st.glod, view, desc, model, out))
        singles.append(_single(env, st, view, desc, model, oh, ow))
    return ents, singles


def test_batch_matches_single_renders(env, sets):
    lvr, O, ctx, dev = env
    ents, singles = _entries(env, sets, dict(ert_alpha=0.99, shadows=True, ao_mode=1))
    b = lvr.lvr_batch_create(ctx, ents)
    tiles, rays = b.size()
    assert rays == sum(e[5].shape[0] * e[5].shape[1] for e in ents)
    for _ in range(2):                      # graph replays give the same images
        b.render()
        ctx.sync()
        for e, ref in zip(ents, singles):
            assert np.array_equal(e[5].cpu().numpy(), ref)


def test_batch_with_views_of_their_own(env, sets):
    """Views large enough to fill the GPU on their own (1920 x 1080: 64 800
    tiles) get their own launch inside the batch's graph, beside the queue of
    the small ones: every view still equals its single render bit for bit,
    for traced and for learned AO, and over two replays."""
    import torch
    lvr, O, ctx, dev = env
    rng = np.random.default_rng(5)
    model = lvr.lvr_ao_model_create(ctx, (rng.standard_normal(lvr.lvr_ao_nparams()) * 0.05).astype(np.float32))
    for kw, m in ((dict(ert_alpha=0.99, shadows=True, ao_mode=1), None), (dict(ert_alpha=0.99, ao_mode=2), model)):
        ents, singles = [], []
        for k, (w, h) in enumerate(((1920, 1080), (96, 64), (1920, 1080), (200, 120))):
            st = sets[k % 2]
            view, _ = _view(lvr, st, w, h, k)
            desc = lvr.make_desc(0.2, st.tf, layout=1, **kw)
            out = torch.full((h, w, 4), -1.0, dtype=torch.float32, device=dev)
            ents.append((st.gls, st.glod, view, desc, m, out))
            singles.append(_single(env, st, view, desc, m, h, w))
        b = lvr.lvr_batch_create(ctx, ents)
        tiles, rays = b.size()
        assert rays == sum(e[5].shape[0] * e[5].shape[1] for e in ents)
        for _ in range(2):
            for e in ents:
                e[5].fill_(-1.0)
            b.render()
            ctx.sync()
            for e, ref in zip(ents, singles):
                assert np.array_equal(e[5].cpu().numpy(), ref)
        assert (singles[0][..., 3] > 0).mean() > 0.2


def test_batch_view_against_oracle(env, sets):
    import torch
    lvr, O, ctx, dev = env
    st = sets[0]
    view, cam = _view(lvr, st, 128, 96, 2)
    desc = lvr.make_desc(0.2, st.tf, ert_alpha=0.99, shadows=True, ao_mode=1)
    out = torch.empty((96, 128, 4), dtype=torch.float32, device=dev)
    other = torch.empty((40, 50, 4), dtype=torch.float32, device=dev)
    v2, _ = _view(lvr, sets[1], 50, 40, 3)
    b = lvr.lvr_batch_create(ctx, [(st.gls, st.glod, view, desc, None, out),
                                   (sets[1].gls, sets[1].glod, v2, desc, None, other)])
    b.render()
    ctx.sync()
    ovs = S.oracle_lineset(O, st.ls, **st.g)
    olod = O.Lod(ovs, 3, synth.sigma_lut(st.tf))
    _, ov, pix = S.views(cam)
    ref, tie, _ = O.render(ovs, olod, ov, O.make_rdesc(0.2, st.tf, ert_alpha=0.99, shadows=True, ao=True), pix)
    S.check_image(out.cpu().numpy().reshape(-1, 4), ref, tie, what="batched view")


def test_batch_learned_and_layouts(env, sets):
    from tests.test_gpu_learned_ao import random_params
    lvr, O, ctx, dev = env
    model = lvr.lvr_ao_model_create(ctx, random_params(21))
    for layout in (0, 1):
        ents, singles = _entries(env, sets, dict(ert_alpha=0.99, ao_mode=2), model=model, layout=layout)
        b = lvr.lvr_batch_create(ctx, ents)
        b.render()
        ctx.sync()
        for e, ref in zip(ents, singles):
            assert np.array_equal(e[5].cpu().numpy(), ref)


def test_batch_argument_checks(env, sets):
    import torch
    from tests.test_gpu_learned_ao import random_params
    lvr, O, ctx, dev = env
    st = sets[0]
    model = lvr.lvr_ao_model_create(ctx, random_params(22))
    view, _ = _view(lvr, st, 32, 32, 0)
    out = torch.empty((32, 32, 4), dtype=torch.float32, device=dev)
    learned = lvr.make_desc(0.2, st.tf, ao_mode=2)
    traced = lvr.make_desc(0.2, st.tf, ao_mode=1)
    with pytest.raises(lvr.LVRError):       # mixed AO kinds
        lvr.lvr_batch_create(ctx, [(st.gls, st.glod, view, learned, model, out),
                                   (st.gls, st.glod, view, traced, None, out)])
    with pytest.raises(lvr.LVRError):       # mixed layouts
        lvr.lvr_batch_create(ctx, [(st.gls, st.glod, view, traced, None, out),
                                   (st.gls, st.glod, view, lvr.make_desc(0.2, st.tf, ao_mode=1, layout=1), None, out)])
    with pytest.raises(lvr.LVRError):       # host output
        lvr.lvr_batch_create(ctx, [(st.gls, st.glod, view, traced, None, np.empty((32, 32, 4), np.float32))])
    with pytest.raises(lvr.LVRError):
        lvr.lvr_batch_create(ctx, [])


def test_autotune_picks_a_candidate(env, sets):
    lvr, O, ctx, dev = env
    ents, _ = _entries(env, sets, dict(ert_alpha=0.99, shadows=True, ao_mode=1))
    r = lvr.lvr_autotune(ctx, ents, reps=2)
    assert r["tile"] in [(8, 4), (4, 8), (16, 2), (32, 1)]
    assert r["layout"] in (0, 1)
    ms = r["ms"]
    assert all(m > 0 for m in ms)           # both layouts available: every candidate ran
    assert min(ms) == ms[r["layout"] * 4 + [(8, 4), (4, 8), (16, 2), (32, 1)].index(r["tile"])]


def test_batch_with_rep_line_shadows(env, sets):
    """Views with hard shadows against representative lines run in a batch
    of their own kernel variant and equal their single renders bit for bit;
    mixing them with soft-shadow views in one batch is refused."""
    lvr, O, ctx, dev = env
    for st in sets:
        lvr.lvr_lod_rep_lines(ctx, st.glod, st.gls)
    ents, singles = _entries(env, sets, dict(ert_alpha=0.99, ao_mode=1, shadow_level=1))
    b = lvr.lvr_batch_create(ctx, ents)
    b.render()
    ctx.sync()
    for e, ref in zip(ents, singles):
        assert np.array_equal(e[5].cpu().numpy(), ref)
    soft = _entries(env, sets, dict(ert_alpha=0.99, shadows=True, ao_mode=1))[0]
    with pytest.raises(lvr.LVRError):
        lvr.lvr_batch_create(ctx, [ents[0], soft[1]])
