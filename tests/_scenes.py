"""Shared test scenes: one seeded input feeds both the CUDA path and the oracle."""
from __future__ import annotations

import json
import os

import numpy as np

from paper_1801_01155_gb300 import synth

TOL = 2e-3          # RGBA, absolute per channel
TIE_CAP = 1e-3      # fraction of pixels allowed to be flagged as near-ties

_CACHE = {}


def streamlines(n, nv, seed):
    key = (n, nv, seed)
    if key not in _CACHE:
        _CACHE[key] = synth.make_streamlines(n, nv, seed)
    return _CACHE[key]


def grid_args(ls, R, N, origin=(0.0, 0.0, 0.0), scale=None):
    scale = float(R) if scale is None else float(scale)
    return dict(res=R, bins=N, origin=origin, scale=scale,
                attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))


def gpu_lineset(lvr, ctx, ls, dev, **g):
    import torch
    xyz = torch.from_numpy(ls.xyz).to(dev)
    attr = torch.from_numpy(ls.attr).to(dev)
    offs = torch.from_numpy(ls.offsets).to(dev)
    return lvr.lvr_voxelize(ctx, xyz, attr, offs, lvr.grid_desc(**g))


def oracle_lineset(O, ls, **g):
    return O.VoxSet(ls.xyz, ls.attr, ls.offsets, O.make_grid(**g))


def compare_lineset(lvr, ctx, gls, ovs):
    e = lvr.export_lineset_numpy(ctx, gls)
    o = ovs.export()
    assert e["offset"].shape == o["offset"].shape
    np.testing.assert_array_equal(e["offset"], o["offset"])
    np.testing.assert_array_equal(e["fields"], o["fields"])
    np.testing.assert_array_equal(e["curve"], o["curve"])
    np.testing.assert_array_equal(e["ordinal"], o["ordinal"])
    return len(o["curve"])


def views(cam, crop=None):
    """(library view, oracle view, pixel list) for a synth camera dict."""
    from oracle import oracle as O
    from paper_1801_01155_gb300 import lvr
    W, H = cam["width"], cam["height"]
    lv = lvr.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], W, H, cam["light_dir"], crop=crop)
    ov = O.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], W, H, cam["light_dir"])
    if crop:
        pix = O.pixel_grid(*crop)
    else:
        pix = O.pixel_grid(0, 0, W, H)
    return lv, ov, pix


TIE_SHADOW = 64     # the oracle's flag bit of a near-tie hard-shadow visibility
TIE_SORT = 4        # the oracle's flag bit of two hits closer in depth than their error bounds


def check_image(got, ref, tie, tol=TOL, cap=TIE_CAP, what="", flip=None, alt=None):
    """Element-wise parity outside flagged pixels; flagged fraction capped.
    flip (the oracle's per-pixel flip budget, hard shadows): pixels whose only
    flag is a near-tie hard-shadow visibility are compared too, within tol
    plus the most those visibilities can move the colour, and do not count
    against the cap. alt (the oracle's second right answer of pixels whose
    only near-tie is one pair of hits in depth order, NaN elsewhere): those
    pixels must match one of the two answers within tol, and do not count
    against the cap either. With LVR_PARITY_REPORT set, each image's error
    statistics are appended to that file as one JSON line (before the
    checks, so failures show)."""
    got = np.asarray(got, np.float64).reshape(-1, 4)
    ok = tie == 0
    err = np.abs(got - ref)
    worst = err[ok].max() if ok.any() else 0.0
    nbad = int((err[ok].max(1) > tol).sum())
    shadow = (tie == TIE_SHADOW) if flip is not None else np.zeros(len(tie), bool)
    nbad_shadow = int((err[shadow].max(1) > tol + flip[shadow]).sum()) if shadow.any() else 0
    two = np.zeros(len(tie), bool)
    nbad_two = 0
    if alt is not None:
        alt = np.asarray(alt, np.float64).reshape(-1, 4)
        two = (tie == TIE_SORT) & np.isfinite(alt).all(1)
        if two.any():
            e_ref = err[two].max(1)
            e_alt = np.abs(got[two] - alt[two]).max(1)
            nbad_two = int((np.minimum(e_ref, e_alt) > tol).sum())
    frac = 1.0 - (ok | shadow | two).mean()
    report = os.environ.get("LVR_PARITY_REPORT")
    if report:
        rec = {"image": what, "pixels": int(len(got)), "max_abs": float(worst),
               "mean_abs": float(err[ok].mean()) if ok.any() else 0.0,
               "tie_pixels": int((~(ok | shadow | two)).sum()), "tie_frac": float(frac), "over_tol": nbad}
        if shadow.any():
            rec.update(shadow_tie_pixels=int(shadow.sum()), shadow_max_abs=float(err[shadow].max()),
                       shadow_median_budget=float(np.median(flip[shadow])), shadow_over_budget=nbad_shadow)
        if two.any():
            rec.update(two_answer_pixels=int(two.sum()),
                       two_answer_matched_alt=int((np.abs(got[two] - alt[two]).max(1) <= tol).sum()),
                       two_answer_over_tol=nbad_two)
        with open(report, "a") as f:
            f.write(json.dumps(rec) + "\n")
    assert nbad_shadow == 0, f"{what}: {nbad_shadow} shadow-tie pixels off by more than their flip budget"
    assert nbad_two == 0, f"{what}: {nbad_two} depth-tie pixels match neither order within {tol}"
    assert nbad == 0, f"{what}: {nbad} non-tie pixels off by > {tol} (worst {worst:.3e})"
    assert frac <= cap, f"{what}: {frac:.4%} tie pixels > {cap:.2%}"
    return worst, frac
