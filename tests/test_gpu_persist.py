"""Saving and restoring (voxel model, density LoD, learned-AO training
state) and the allocation-failure paths.

- A line set and a LoD exported and imported again are the same arrays and
  render the same image bit for bit; malformed imports are refused.
- Training continued from a checkpoint takes exactly the steps training that
  never stopped takes.
- Every call that allocates device memory returns LVR_ENOMEM when one of its
  allocations fails (injected on the host by the library's allocation hook)
  and holds no more device allocations afterwards than before.
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
    from paper_1801_01155_gb300 import lvr
    dev = torch.device("cuda:0")
    return lvr, lvr.Context(0, torch.cuda.Stream(dev)), dev


@pytest.fixture(scope="module")
def scene(env):
    lvr, ctx, dev = env
    ls = S.streamlines(500, 64, 0)
    g = S.grid_args(ls, 32, 32)
    tf = synth.tf_ramp(0.05, 0.3)
    gls = S.gpu_lineset(lvr, ctx, ls, dev, **g)
    lod = lvr.lvr_build_lod(ctx, gls, 3, synth.sigma_lut(tf))
    return dict(ls=ls, g=g, tf=tf, gls=gls, lod=lod)


def _frame(lvr, ctx, dev, ls, lod, tf, **kw):
    import torch
    cam = synth.orbit_view((32, 32, 32), 96, 64)
    v = lvr.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 96, 64, cam["light_dir"])
    out = torch.empty((64, 96, 4), dtype=torch.float32, device=dev)
    lvr.lvr_render(ctx, ls, lod, v, lvr.make_desc(0.2, tf, ert_alpha=0.99, **kw), out)
    ctx.sync()
    return out.cpu().numpy()


def test_lineset_round_trip(env, scene):
    import torch
    lvr, ctx, dev = env
    e = lvr.export_lineset_numpy(ctx, scene["gls"])
    g = scene["g"]
    imp = lvr.lvr_import_lineset(ctx, g["res"], g["bins"], g["origin"], g["scale"], e["offset"], e["fields"],
                                 e["curve"], e["ordinal"])
    e2 = lvr.export_lineset_numpy(ctx, imp)
    for k in e:
        np.testing.assert_array_equal(e2[k], e[k])
    assert np.array_equal(_frame(lvr, ctx, dev, imp, None, scene["tf"]),
                          _frame(lvr, ctx, dev, scene["gls"], None, scene["tf"]))
    # device arrays work the same
    dv = [torch.from_numpy(np.ascontiguousarray(e[k])).to(dev) for k in ("offset", "fields", "curve", "ordinal")]
    imp2 = lvr.lvr_import_lineset(ctx, g["res"], g["bins"], g["origin"], g["scale"], *dv)
    np.testing.assert_array_equal(lvr.export_lineset_numpy(ctx, imp2)["fields"], e["fields"])
    imp.free()
    imp2.free()
    # malformed arrays are refused, nothing kept
    live = lvr.lvr_test_live_allocations()
    bad_face = e["fields"].copy()
    bad_face[5, 0] = 6
    bad_off = e["offset"].copy()
    bad_off[-1] += 1
    k = int(np.flatnonzero(np.diff(e["offset"]) >= 2)[0])   # a voxel with two segments
    i0 = int(e["offset"][k])
    bad_order = [a.copy() for a in (e["fields"], e["curve"], e["ordinal"])]
    for a in bad_order:
        a[[i0, i0 + 1]] = a[[i0 + 1, i0]]
    for off, f, c, o in ((e["offset"], bad_face, e["curve"], e["ordinal"]),
                         (bad_off, e["fields"], e["curve"], e["ordinal"]),
                         (e["offset"], *bad_order)):
        with pytest.raises(lvr.LVRError) as ei:
            lvr.lvr_import_lineset(ctx, g["res"], g["bins"], g["origin"], g["scale"], off, f, c, o)
        assert ei.value.code == lvr.EINVAL
    assert lvr.lvr_test_live_allocations() == live


def test_lod_round_trip(env, scene):
    lvr, ctx, dev = env
    lod = scene["lod"]
    lv = [lvr.export_lod_numpy(ctx, lod, l) for l in range(3)]
    imp = lvr.lvr_import_lod(ctx, lv[0]["dims"], [x["cnt"] for x in lv], [x["len"] for x in lv],
                             [x["dens"] for x in lv])
    for l in range(3):
        e = lvr.export_lod_numpy(ctx, imp, l)
        assert e["dims"] == lv[l]["dims"]
        for k in ("cnt", "len", "dens"):
            np.testing.assert_array_equal(e[k], lv[l][k])
    kw = dict(shadows=True, ao_mode=1)
    assert np.array_equal(_frame(lvr, ctx, dev, scene["gls"], imp, scene["tf"], **kw),
                          _frame(lvr, ctx, dev, scene["gls"], lod, scene["tf"], **kw))
    imp.free()
    bad = lv[1]["dens"].copy()
    bad[3] = np.nan
    with pytest.raises(lvr.LVRError) as ei:
        lvr.lvr_import_lod(ctx, lv[0]["dims"], [x["cnt"] for x in lv], [x["len"] for x in lv],
                           [lv[0]["dens"], bad, lv[2]["dens"]])
    assert ei.value.code == lvr.EINVAL


def test_training_resumes_from_a_checkpoint(env):
    import torch
    lvr, ctx, dev = env
    rng = np.random.default_rng(11)
    n, nin = 1024, 400
    x = (rng.standard_normal((n, nin)) * 0.5).astype(np.float32)
    X = torch.from_numpy(x).to(dev).to(torch.bfloat16).view(torch.int16)
    y = torch.from_numpy(rng.random(n).astype(np.float32)).to(dev)
    p0 = (rng.uniform(-1, 1, lvr.lvr_ao_nparams()) * 0.05).astype(np.float32)

    def steps(m, k):
        for _ in range(k):
            lvr.lvr_ao_train_step(ctx, m, X, y, lr=2e-3)

    a = lvr.lvr_ao_model_create(ctx, p0)
    steps(a, 10)
    pa = a.params()
    b = lvr.lvr_ao_model_create(ctx, p0)
    steps(b, 6)
    params, mm, vv, step = lvr.lvr_ao_model_state(ctx, b)
    assert step == 6 and np.abs(mm).max() > 0 and np.abs(vv).max() > 0
    c = lvr.lvr_ao_model_create(ctx, params)
    lvr.lvr_ao_model_set_state(ctx, c, params, mm, vv, step)
    steps(c, 4)
    assert np.array_equal(c.params(), pa)
    # before any Adam step: zero moments and step 0
    _, m0, v0, s0 = lvr.lvr_ao_model_state(ctx, lvr.lvr_ao_model_create(ctx, p0))
    assert s0 == 0 and not m0.any() and not v0.any()


def test_allocation_failures_return_enomem(env, scene):
    """Each allocating call, with each of its device allocations failing in
    turn: LVR_ENOMEM and no device allocation left behind; with none failing
    it succeeds. (The context's grow-only buffers are sized by a first call.)"""
    import torch
    lvr, ctx, dev = env
    ls, g, tf = scene["ls"], scene["g"], scene["tf"]
    sig = synth.sigma_lut(tf)
    xyz, attr, offs = (torch.from_numpy(a).to(dev) for a in (ls.xyz, ls.attr, ls.offsets))
    e = lvr.export_lineset_numpy(ctx, scene["gls"])
    lv = [lvr.export_lod_numpy(ctx, scene["lod"], l) for l in range(3)]
    params = (np.random.default_rng(2).uniform(-1, 1, lvr.lvr_ao_nparams()) * 0.05).astype(np.float32)
    cam = synth.orbit_view((32, 32, 32), 64, 48)
    view = lvr.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 64, 48, cam["light_dir"])
    out = torch.empty((48, 64, 4), dtype=torch.float32, device=dev)

    def fresh_set():
        return lvr.lvr_voxelize(ctx, xyz, attr, offs, lvr.grid_desc(**g))

    calls = {
        "voxelize": lambda: fresh_set(),
        "build_lod": lambda: lvr.lvr_build_lod(ctx, scene["gls"], 3, sig),
        "layout": lambda: lvr.lvr_lineset_layout(ctx, fresh_set(), lvr.LAYOUT_AOS16),
        "neighbours": lambda: lvr.lvr_lineset_neighbours(ctx, fresh_set(), 0.2),
        "import_lineset": lambda: lvr.lvr_import_lineset(ctx, g["res"], g["bins"], g["origin"], g["scale"],
                                                        e["offset"], e["fields"], e["curve"], e["ordinal"]),
        "import_lod": lambda: lvr.lvr_import_lod(ctx, lv[0]["dims"], [x["cnt"] for x in lv],
                                                 [x["len"] for x in lv], [x["dens"] for x in lv]),
        "ao_model_create": lambda: lvr.lvr_ao_model_create(ctx, params),
        "learned_bind": lambda: lvr.lvr_render(ctx, scene["gls"], lvr.lvr_build_lod(ctx, scene["gls"], 3, sig), view,
                                               lvr.make_desc(0.2, tf, ao_mode=2), out,
                                               ao_model=lvr.lvr_ao_model_create(ctx, params)),
    }
    for name, call in calls.items():
        call()   # grow-only buffers at size
        ctx.sync()
        failed = 0
        for k in range(64):
            live = lvr.lvr_test_live_allocations()
            lvr.lvr_test_fail_allocation(k)
            try:
                call()
                ok = True
            except lvr.LVRError as err:
                ok = False
                assert err.code == lvr.ENOMEM, f"{name}, allocation {k}: {err}"
            finally:
                lvr.lvr_test_fail_allocation(-1)
            ctx.sync()
            import gc
            gc.collect()   # handles made before the failing allocation are freed by their wrappers
            ctx.sync()
            if ok:
                break
            failed += 1
            assert lvr.lvr_test_live_allocations() <= live, f"{name}: allocation {k} failing leaked"
        assert failed >= 1, f"{name} allocates nothing"
