"""Learned AO trained end to end, judged by the traced AO it replaces.

The model is trained by lvr_train_ao on 4M traced-AO samples from eight
seeded line sets of the small streamline workload (500 curves x 64 vertices,
32^3 grid, tube radius 0.2, seeds 100..107) and judged on a ninth set (seed
0, not seen in training) at 1920 x 1080 with transparency: over every
composited hit, the mean absolute difference between learned and traced AO
must not exceed 0.02; the 99th percentile is reported. Both AO values come
from kernels that the other GPU tests pin to the oracle.
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


def _set(lvr, ctx, dev, seed, sig):
    ls = S.streamlines(500, 64, seed)
    gls = S.gpu_lineset(lvr, ctx, ls, dev, **S.grid_args(ls, 32, 32))
    return gls, lvr.lvr_build_lod(ctx, gls, 3, sig)


def test_learned_ao_meets_the_error_bound(env):
    lvr, ctx, dev = env
    tf = synth.tf_ramp(0.05, 0.3)
    sig = synth.sigma_lut(tf)
    train = [_set(lvr, ctx, dev, s, sig) for s in range(100, 108)]
    gls, glod = _set(lvr, ctx, dev, 0, sig)
    desc = lvr.make_desc(0.2, tf, ert_alpha=0.99, shadows=True, ao_mode=1, ao_rays=16, ao_radius=15.0)
    td = lvr.ao_train_desc(4_000_000, 8, 8192, 3e-3, 1234, desc, view_size=256, depth=32)
    model, mse = lvr.lvr_train_ao(ctx, [t[0] for t in train], [t[1] for t in train], td)
    assert np.isfinite(mse) and mse < 0.01
    cam = synth.orbit_view((32, 32, 32), 1920, 1080)
    lv = lvr.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 1920, 1080, cam["light_dir"])
    err = lvr.lvr_ao_judge(ctx, gls, glod, lv, desc, model)
    print("learned vs traced AO:", err)
    assert err["hits"] > 100_000
    assert err["mean_abs"] <= 0.02, err
    assert err["p99_abs"] <= 0.15, err
