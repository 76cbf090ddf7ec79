"""The camera-at-rest cull's segment-to-voxel distance, built with the host
compiler from the same header the CUDA kernel includes, against brute-force
sampling: it must never exceed the true distance (an overestimate would drop
a record that can give the voxel a hit) and must be accurate.

Segments are the library's: end points on faces of a unit voxel at
bin centres (N = 32), shifted into a neighbour's frame by -1, 0 or 1 per axis.
"""
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1801_01155_gb300", "csrc")

DRIVER = r"""
#include <stdio.h>
#include "geom.cuh"
int main(void) {
    float a[3], b[3];
    while (scanf("%f %f %f %f %f %f", a, a + 1, a + 2, b, b + 1, b + 2) == 6)
        printf("%.9g\n", lvr_geom::segment_box_dist2(a, b));
    return 0;
}
"""


def _face_points(rng, n, N=32):
    face = rng.integers(0, 6, n)
    ax, side = face >> 1, (face & 1).astype(np.float64)
    u, v = (rng.integers(0, N, n) + 0.5) / N, (rng.integers(0, N, n) + 0.5) / N
    return np.stack([np.where(ax == 0, side, u), np.where(ax == 1, side, np.where(ax == 0, u, v)),
                     np.where(ax == 2, side, v)], 1)


def test_segment_box_distance_against_sampling(tmp_path):
    src = tmp_path / "geom_driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "geom_driver"
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    rng = np.random.default_rng(21)
    n = 4000
    shift = rng.integers(-1, 2, (n, 3)).astype(np.float64)
    a = (_face_points(rng, n) + shift).astype(np.float32)
    b = (_face_points(rng, n) + shift).astype(np.float32)
    # a few degenerate (zero-length) and axis-parallel segments
    b[:50] = a[:50]
    b[50:100, 1:] = a[50:100, 1:]
    text = "\n".join(" ".join(f"{x:.9g}" for x in np.concatenate([p, q])) for p, q in zip(a, b))
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
    got = np.sqrt(np.array([float(x) for x in out.split()]))
    assert len(got) == n
    s = np.linspace(0.0, 1.0, 4001)
    A, B = a.astype(np.float64), b.astype(np.float64)
    P = A[:, None, :] + s[None, :, None] * (B - A)[:, None, :]
    e = np.maximum(np.maximum(-P, P - 1.0), 0.0)
    brute = np.sqrt((e * e).sum(-1)).min(1)
    # sampling overestimates the true minimum by at most half a step times |b - a|
    slack = 0.5 / 4000 * np.linalg.norm(B - A, axis=1)
    assert np.all(got <= brute + 1e-6)
    assert np.all(got >= brute - slack - 1e-6)
    assert (got == 0).mean() > 0.05 and (got > 0.5).mean() > 0.05
