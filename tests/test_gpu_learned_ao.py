"""Learned AO surrogate on the GPU against the oracle (aomlp.c, aotrain.py).

Model inputs must equal the oracle's bfloat16 inputs except where the oracle
value lies within the float32 error of a bfloat16 rounding boundary (those
may land on either neighbour; they are counted and capped). The model output
and the fused render agree within 2e-3: bfloat16 products are exact in both,
float32 against float64 sums differ by ~1e-6 relative, and a rare flip of
one bfloat16 activation moves the output by ~1e-4. The training step is
compared block by block: loss within 1e-5 relative, gradients within 2e-3 of
each block's largest magnitude.
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


class Set:
    def __init__(self, env, n, nv, seed, R, alpha=(0.05, 0.3), levels=3):
        lvr, O, ctx, dev = env
        self.ls = S.streamlines(n, nv, seed)
        g = S.grid_args(self.ls, R, 32)
        self.R = R
        self.tf = synth.tf_ramp(*alpha)
        self.gls = S.gpu_lineset(lvr, ctx, self.ls, dev, **g)
        self.ovs = S.oracle_lineset(O, self.ls, **g)
        sig = synth.sigma_lut(self.tf)
        self.glod = lvr.lvr_build_lod(ctx, self.gls, levels, sig)
        self.olod = O.Lod(self.ovs, levels, sig)


@pytest.fixture(scope="module")
def c1t(env):
    return Set(env, 500, 64, 0, 32)


def random_params(seed, scale=3.0):
    """Uniform +-scale/sqrt(fan_in) weights and biases, padding inputs zero."""
    from oracle import aotrain as T
    rng = np.random.default_rng(seed)
    p = np.empty(T.NPARAM)
    p[:T.OW2] = rng.uniform(-1, 1, T.OW2) * scale / 20.0
    p[T.OW2:] = rng.uniform(-1, 1, T.NPARAM - T.OW2) * scale / 8.0
    W1 = p[T.OW1:T.OB1].reshape(64, 400)
    W1[:, 15] = 0.0
    W1[:, 391:] = 0.0
    return p.astype(np.float32)


def hit_queries(st, n, seed):
    """Voxels (mostly non-empty, some empty, the corners), directions (random,
    axis-aligned, zero, negative first components), points inside the voxel
    and unit normals."""
    rng = np.random.default_rng(seed)
    cnt = st.olod.export(0)["cnt"]
    nz = np.flatnonzero(cnt)
    vox = np.where(rng.random(n) < 0.85, rng.choice(nz, n), rng.integers(0, cnt.size, n)).astype(np.int32)
    vox[:2] = [0, cnt.size - 1]
    d = rng.standard_normal((n, 3))
    d[2:8] = [[1, 0, 0], [0, -1, 0], [0, 0, 2.5], [0, 0, 0], [-1, 2, 0], [0, -3, 4]]
    R = st.R
    v = np.stack([vox % R, (vox // R) % R, vox // (R * R)], 1)
    pos = v + rng.uniform(0.0, 1.0, (n, 3))
    pos[8] = v[8]                                   # a voxel corner
    nrm = rng.standard_normal((n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return vox, d.astype(np.float32), pos.astype(np.float32), nrm.astype(np.float32)


def oracle_inputs(O, st, vox, d, pos, nrm):
    return np.stack([O.ao_features(st.olod, int(v), O.ao_tangent([0, 0, 0], dd), nn, pp)
                     for v, dd, pp, nn in zip(vox, d.astype(np.float64), pos.astype(np.float64),
                                              nrm.astype(np.float64))])


def _dev(torch, dev, *arrs):
    return [torch.from_numpy(a).to(dev) for a in arrs]


def bf16_margin_flags(x, rel):
    """True where x is within `rel` (relative) of a bfloat16 rounding boundary."""
    from oracle import aotrain as T
    x = np.asarray(x, np.float64)
    lo = T.bf16(x)
    ulp = np.abs(T.bf16(np.abs(x) * (1 + 2.0 ** -7)) - np.abs(lo))
    ulp = np.where(ulp > 0, ulp, 2.0 ** -133)
    frac = np.abs(np.abs(x) - np.abs(lo)) / ulp          # distance to the kept value, in ulps
    return np.abs(frac - 0.5) * ulp < rel * np.abs(x)


def test_features_match_oracle(env, c1t):
    import torch
    from oracle import aotrain as T
    lvr, O, ctx, dev = env
    q = hit_queries(c1t, 3000, 1)
    X = torch.empty((len(q[0]), 400), dtype=torch.int16, device=dev)
    lvr.lvr_ao_features(ctx, c1t.glod, *_dev(torch, dev, *q), X)
    ctx.sync()
    got = X.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    got = got.view(np.float32).astype(np.float64)
    ref = oracle_inputs(O, c1t, *q)
    want = T.bf16(ref)
    # margins: per-hit inputs from float32 directions and points (~2^-21
    # relative); densities are float32 sums over up to a few hundred
    # segments, pooled twice, then log1pf (~2^-17)
    flag = bf16_margin_flags(ref, 2.0 ** -19)
    flag[:, 16:391] |= bf16_margin_flags(ref[:, 16:391], 2.0 ** -17)
    bad = (got != want) & ~flag
    assert not bad.any(), f"{bad.sum()} inputs differ, first at {np.argwhere(bad)[:3]}"
    near = (got != want) & flag
    ulp = np.abs(T.bf16(np.abs(want) * (1 + 2.0 ** -7)) - np.abs(want))
    assert np.all(np.abs(got - want)[near] <= ulp[near] + 1e-300)
    assert flag.mean() < 0.01, flag.mean()
    assert (got[:, 16:391] != 0).mean() > 0.2


def test_infer_matches_oracle(env, c1t):
    import torch
    lvr, O, ctx, dev = env
    p = random_params(7)
    m = lvr.lvr_ao_model_create(ctx, p)
    q = hit_queries(c1t, 4000, 2)
    ao = torch.empty(len(q[0]), dtype=torch.float32, device=dev)
    lvr.lvr_ao_infer(ctx, m, c1t.glod, *_dev(torch, dev, *q), ao)
    ctx.sync()
    got = ao.cpu().numpy().astype(np.float64)
    ref = np.array([O.ao_mlp(p, x) for x in oracle_inputs(O, c1t, *q)])
    assert ref.std() > 0.05, "the random model should spread its outputs"
    err = np.abs(got - ref)
    assert err.max() <= S.TOL, f"max {err.max():.3e}"
    # host buffers give the same values
    got_h = np.empty(len(q[0]), np.float32)
    lvr.lvr_ao_infer(ctx, m, c1t.glod, *q, got_h)
    assert np.array_equal(got_h, got.astype(np.float32))


def test_infer_out_of_range_voxels(env, c1t):
    import torch
    lvr, O, ctx, dev = env
    m = lvr.lvr_ao_model_create(ctx, random_params(8))
    nvox = 32 ** 3
    vox = np.array([-1, nvox, 5], np.int32)
    d = np.ones((3, 3), np.float32)
    pos = np.full((3, 3), 5.5, np.float32)
    nrm = np.tile(np.array([0, 0, 1.0], np.float32), (3, 1))
    with pytest.raises(lvr.LVRError):
        lvr.lvr_ao_infer(ctx, m, c1t.glod, vox, d, pos, nrm, np.empty(3, np.float32))
    ao = torch.empty(3, dtype=torch.float32, device=dev)
    lvr.lvr_ao_infer(ctx, m, c1t.glod, *_dev(torch, dev, vox, d, pos, nrm), ao)
    ctx.sync()
    a = ao.cpu().numpy()
    assert np.isnan(a[0]) and np.isnan(a[1]) and np.isfinite(a[2])


def _render_pair(env, st, cam, p, crop=None, model=None, **kw):
    import torch
    lvr, O, ctx, dev = env
    lv, ov, pix = S.views(cam, crop)
    w, h = (crop[2], crop[3]) if crop else (cam["width"], cam["height"])
    m = model if model is not None else lvr.lvr_ao_model_create(ctx, p)
    out = torch.empty((h, w, 4), dtype=torch.float32, device=dev)
    lvr.lvr_render(ctx, st.gls, st.glod, lv, lvr.make_desc(0.2, st.tf, ao_mode=2, **kw), out, ao_model=m)
    ctx.sync()
    ref, tie, _ = O.render(st.ovs, st.olod, ov, O.make_rdesc(0.2, st.tf, ao_params=p, **kw), pix)
    return out.cpu().numpy().reshape(-1, 4), ref, tie


def test_render_learned_opaque(env, c1t):
    cam = synth.orbit_view((32, 32, 32), 128, 128)
    got, ref, tie = _render_pair(env, c1t, cam, random_params(9), opaque=True, ka=0.6, kd=0.4)
    S.check_image(got, ref, tie, what="learned AO opaque")


def test_render_learned_transparent_with_shadows(env, c1t):
    cam = synth.orbit_view((32, 32, 32), 192, 108)
    got, ref, tie = _render_pair(env, c1t, cam, random_params(10), ert_alpha=0.99, shadows=True)
    S.check_image(got, ref, tie, what="learned AO transparent")


def test_learned_model_rebinds_to_a_new_lod(env, c1t):
    """The cached per-voxel term follows the LoD the call names."""
    lvr, O, ctx, dev = env
    other = Set(env, 300, 48, 3, 32)
    cam = synth.orbit_view((32, 32, 32), 64, 64)
    p = random_params(11)
    m = lvr.lvr_ao_model_create(ctx, p)
    for st in (c1t, other, c1t):
        got, ref, tie = _render_pair(env, st, cam, p, model=m, opaque=True)
        S.check_image(got, ref, tie, what="rebind")


def _oracle_rows(st, n, seed):
    from oracle import aotrain as T
    from oracle import oracle as O
    X = oracle_inputs(O, st, *hit_queries(st, n, seed))
    Xb = T.bf16(X)
    bits = (Xb.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    t = np.random.default_rng(seed + 100).uniform(0.2, 1.0, n)
    return Xb, bits, t


def test_train_step_matches_oracle(env, c1t):
    import torch
    from oracle import aotrain as T
    lvr, O, ctx, dev = env
    p = random_params(12, scale=1.0)
    Xb, bits, t = _oracle_rows(c1t, 1500, 3)
    assert bits.shape == (1500, 400)
    m = lvr.lvr_ao_model_create(ctx, p)
    Xd = torch.from_numpy(bits.view(np.int16)).to(dev)
    yd = torch.from_numpy(t.astype(np.float32)).to(dev)
    g = np.empty(T.NPARAM, np.float32)
    loss = lvr.lvr_ao_train_step(ctx, m, Xd, yd, 0.0, g)
    l_ref, g_ref = T.loss_and_grad(p, Xb, t.astype(np.float32).astype(np.float64))
    assert loss == pytest.approx(l_ref, rel=1e-5)
    blocks = {"W1": (T.OW1, T.OB1), "b1": (T.OB1, T.OW2), "W2": (T.OW2, T.OB2), "b2": (T.OB2, T.OW3),
              "W3": (T.OW3, T.OB3), "b3": (T.OB3, T.OW4), "W4": (T.OW4, T.OB4), "b4": (T.OB4, T.NPARAM)}
    for name, (lo, hi) in blocks.items():
        a, b = g[lo:hi].astype(np.float64), g_ref[lo:hi]
        scale = np.abs(b).max()
        assert scale > 0, name
        assert np.abs(a - b).max() <= 2e-3 * scale, (name, np.abs(a - b).max() / scale)
    # one Adam step: where the gradient's sign is certain the update matches
    # the oracle's; elsewhere it is bounded by the step size
    lr = 1e-3
    lvr.lvr_ao_train_step(ctx, m, Xd, yd, lr, None)
    p1 = m.params().astype(np.float64)
    p_ref, _, _ = T.adam(p.astype(np.float64), g_ref, np.zeros(T.NPARAM), np.zeros(T.NPARAM), 1, lr)
    sure = np.zeros(T.NPARAM, bool)
    for lo, hi in blocks.values():
        sure[lo:hi] = np.abs(g_ref[lo:hi]) > 0.02 * np.abs(g_ref[lo:hi]).max()
    assert np.abs(p1 - p_ref)[sure].max() <= 1e-6 + 1e-3 * lr
    assert np.abs(p1 - p)[~sure].max() <= lr * 1.001


def test_train_step_argument_checks(env, c1t):
    import torch
    lvr, O, ctx, dev = env
    m = lvr.lvr_ao_model_create(ctx, random_params(13))
    with pytest.raises(lvr.LVRError):
        lvr.lvr_ao_train_step(ctx, m, np.zeros((4, 400), np.int16), np.zeros(4, np.float32))
    with pytest.raises(ValueError):
        lvr.lvr_ao_model_create(ctx, np.zeros(10, np.float32))
    bad = random_params(13)
    bad[5] = np.nan
    with pytest.raises(lvr.LVRError):
        lvr.lvr_ao_model_create(ctx, bad)
    # a batch of one row works (bias and output-layer reductions of length 1)
    X = torch.zeros((1, 400), dtype=torch.int16, device=dev)
    y = torch.full((1,), 0.5, dtype=torch.float32, device=dev)
    assert np.isfinite(lvr.lvr_ao_train_step(ctx, m, X, y))


def test_samples_record_the_target_hit(env, c1t):
    """Depth 1 records the first hit: its voxel is the one the opaque render
    sees, and its traced AO is the oracle's opaque AO factor there."""
    import torch
    lvr, O, ctx, dev = env
    cam = synth.orbit_view((32, 32, 32), 64, 64)
    lv, ov, pix = S.views(cam)
    n = 64 * 64
    vox = torch.empty(n, dtype=torch.int32, device=dev)
    d = torch.empty((n, 3), dtype=torch.float32, device=dev)
    ao = torch.empty(n, dtype=torch.float32, device=dev)
    desc = lvr.make_desc(0.2, c1t.tf, opaque=True, ao_mode=1, ka=1.0, kd=0.0, bg=(0, 0, 0))
    pos = torch.empty((n, 3), dtype=torch.float32, device=dev)
    nrm = torch.empty((n, 3), dtype=torch.float32, device=dev)
    lvr.lvr_ao_samples(ctx, c1t.gls, c1t.glod, lv, desc, 1, 5, vox, d, ao, pos, nrm)
    ctx.sync()
    v, a = vox.cpu().numpy(), ao.cpu().numpy()
    # the point lies in its voxel (to float32 rounding), the normal is unit and
    # perpendicular to the segment unless the hit is on an end cap
    hv = v >= 0
    R = c1t.R
    vc = np.stack([v % R, (v // R) % R, v // (R * R)], 1)[hv]
    pp, nn, uu = pos.cpu().numpy()[hv], nrm.cpu().numpy()[hv], d.cpu().numpy()[hv]
    assert np.all(pp >= vc - 1e-4) and np.all(pp <= vc + 1 + 1e-4)
    assert np.allclose(np.linalg.norm(nn, axis=1), 1.0, atol=1e-5)
    assert np.median(np.abs((nn * uu).sum(1))) < 1e-4
    # opaque, ka = 1, kd = 0, white TF, black background: pixel = AO at the first hit
    tf = np.ones((256, 4), np.float32)
    ref, tie, _ = O.render(c1t.ovs, c1t.olod, ov, O.make_rdesc(0.2, tf, opaque=True, ao=True, ka=1.0, kd=0.0,
                                                                bg=(0, 0, 0)), pix)
    hit = ref[:, 3] > 0
    assert not (((v >= 0) != hit) & (tie == 0)).any()
    ok = hit & (tie == 0)
    assert np.abs(a[ok] - ref[ok, 0]).max() <= S.TOL
    assert ok.sum() > 500
    dd = d.cpu().numpy()[v >= 0]
    assert np.allclose(np.linalg.norm(dd, axis=1), 1.0, atol=1e-6)
    # deeper targets record fewer pixels (rays that end earlier give none)
    lvr.lvr_ao_samples(ctx, c1t.gls, c1t.glod, lv, lvr.make_desc(0.2, c1t.tf, ert_alpha=0.99, ao_mode=1), 16, 5,
                       vox, d, ao)
    ctx.sync()
    assert 0 < (vox.cpu().numpy() >= 0).sum() < (v >= 0).sum()
