"""Named GPU cases for profiling one kernel on a reduced workload.

    python -m paper_1801_01155_gb300.cases render-crop [--reps K]
        the benchmark's render (config-2 set: 100k x 200 lines in 256^3,
        transparency with termination at 0.99, soft shadows, 16 traced AO
        rays, 16-byte records, 4x8 ray tiles) on the central 640 x 360 crop of
        the 1920 x 1080 view: one warm-up render, then K renders
    python -m paper_1801_01155_gb300.cases render-crop-learned [--reps K]
        the same crop with the learned AO surrogate in place of the traced AO
        rays (a model with seeded random weights: the work does not depend on
        them), after the model is bound to the LoD
    python -m paper_1801_01155_gb300.cases c1-traced [--reps K]
    python -m paper_1801_01155_gb300.cases c1-learned [--reps K]
        the learned-AO benchmark's test frame: a 500 x 64 streamline set
        (seed 0) in 32^3, 1920 x 1080, transparent tubes r = 0.2 with soft
        shadows and 16 traced AO rays per hit, or the learned AO surrogate (a
        model with seeded random weights) in their place: one warm-up render,
        then K renders
    python -m paper_1801_01155_gb300.cases voxel-term [--reps K]
        the learned-AO model bound to K fresh 3-level LoDs of the config-2 set
        (each bind computes the per-voxel term of every voxel on the tensor
        cores), after one warm-up bind

Each prints one line with its CUDA-event times. The inputs are the seeded
synthetic sets of the benchmark.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _setup(torch, lvr, synth):
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(dev)
    ctx = lvr.Context(0, st)
    ls = synth.make_streamlines(100_000, 200, 1)
    tf = synth.tf_ramp(0.05, 0.3)
    sig = synth.sigma_lut(tf)
    g = lvr.grid_desc(256, 32, scale=256.0, attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))
    with torch.cuda.stream(st):
        xyz, attr, offs = (torch.from_numpy(a).to(dev) for a in (ls.xyz, ls.attr, ls.offsets))
    s = lvr.lvr_voxelize(ctx, xyz, attr, offs, g)
    return dev, st, ctx, s, tf, sig


def render_crop(reps, learned=False):
    import torch

    from paper_1801_01155_gb300 import lvr, synth
    dev, st, ctx, s, tf, sig = _setup(torch, lvr, synth)
    model = None
    if learned:
        rng = np.random.default_rng(7)
        model = lvr.lvr_ao_model_create(ctx, (rng.standard_normal(lvr.lvr_ao_nparams()) * 0.05).astype(np.float32))
    lvr.lvr_lineset_layout(ctx, s, lvr.LAYOUT_AOS16)
    lod = lvr.lvr_build_lod(ctx, s, 3, sig)
    cam = synth.orbit_view((256, 256, 256), 1920, 1080)
    view = lvr.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 1920, 1080, cam["light_dir"],
                         crop=(640, 360, 640, 360))
    desc = lvr.make_desc(0.15, tf, ert_alpha=0.99, shadows=True, ao_mode=2 if learned else 1, ao_rays=16,
                         ao_radius=15.0, tile=(4, 8), layout=lvr.LAYOUT_AOS16)
    out = torch.empty((360, 640, 4), dtype=torch.float32, device=dev)
    lvr.lvr_render(ctx, s, lod, view, desc, out, ao_model=model)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lvr.lvr_render(ctx, s, lod, view, desc, out, ao_model=model)
        e1.record(st)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(f"render-crop{'-learned' if learned else ''}: {np.median(ms):.3f} ms per 640x360 crop render "
          f"(median of {reps})")


def c1_frame(reps, learned):
    import torch

    from paper_1801_01155_gb300 import lvr, synth
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(dev)
    ctx = lvr.Context(0, st)
    s = synth.make_streamlines(500, 64, 0)
    tf = synth.tf_ramp(0.05, 0.3)
    g = lvr.grid_desc(32, 32, scale=32.0, attr_min=float(s.attr.min()), attr_max=float(s.attr.max()))
    with torch.cuda.stream(st):
        xyz, attr, offs = (torch.from_numpy(a).to(dev) for a in (s.xyz, s.attr, s.offsets))
    ls = lvr.lvr_voxelize(ctx, xyz, attr, offs, g)
    lod = lvr.lvr_build_lod(ctx, ls, 3, synth.sigma_lut(tf))
    model = None
    if learned:
        rng = np.random.default_rng(7)
        model = lvr.lvr_ao_model_create(ctx, (rng.standard_normal(lvr.lvr_ao_nparams()) * 0.05).astype(np.float32))
    cam = synth.orbit_view((32, 32, 32), 1920, 1080)
    view = lvr.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 1920, 1080, cam["light_dir"])
    desc = lvr.make_desc(0.2, tf, ert_alpha=0.99, shadows=True, ao_mode=2 if learned else 1, ao_rays=16,
                         ao_radius=15.0)
    out = torch.empty((1080, 1920, 4), dtype=torch.float32, device=dev)
    lvr.lvr_render(ctx, ls, lod, view, desc, out, ao_model=model)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lvr.lvr_render(ctx, ls, lod, view, desc, out, ao_model=model)
        e1.record(st)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(f"c1-{'learned' if learned else 'traced'}: {np.median(ms):.3f} ms per 1920x1080 frame (median of {reps})")


def voxel_term(reps):
    import torch

    from paper_1801_01155_gb300 import lvr, synth
    dev, st, ctx, s, tf, sig = _setup(torch, lvr, synth)
    rng = np.random.default_rng(7)
    m = lvr.lvr_ao_model_create(ctx, (rng.standard_normal(lvr.lvr_ao_nparams()) * 0.05).astype(np.float32))
    hit = [torch.from_numpy(a).to(dev) for a in (np.zeros(1, np.int32), np.ones((1, 3), np.float32),
                                                 np.full((1, 3), 0.5, np.float32),
                                                 np.array([[0.0, 0.0, 1.0]], np.float32))]
    ao = torch.empty(1, dtype=torch.float32, device=dev)
    ms = []
    for k in range(reps + 1):
        lod = lvr.lvr_build_lod(ctx, s, 3, sig)
        st.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lvr.lvr_ao_infer(ctx, m, lod, *hit, ao)   # binds the model to the new LoD
        e1.record(st)
        e1.synchronize()
        if k > 0:
            ms.append(e0.elapsed_time(e1))
        lod.free()
    print(f"voxel-term: {np.median(ms):.3f} ms per bind to a 256^3 LoD (median of {reps}, allocation included)")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["render-crop", "render-crop-learned", "c1-traced", "c1-learned", "voxel-term"])
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args(argv)
    import __graft_entry__ as g
    g.build()
    if a.case == "voxel-term":
        voxel_term(a.reps)
    elif a.case.startswith("c1-"):
        c1_frame(a.reps, learned=a.case == "c1-learned")
    else:
        render_crop(a.reps, learned=a.case == "render-crop-learned")


if __name__ == "__main__":
    main()
