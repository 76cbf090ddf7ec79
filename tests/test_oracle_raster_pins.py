"""Pins of the oracle's rasterised comparison system (reading K1; Secs. 1,
5.1): every capsule between consecutive input vertices leaves one fragment
per pixel ray that enters it; fragments are sorted by depth and blended.

Pinned by closed forms (silhouette width, stacked tubes, the doubled joint
of two collinear capsules, the attribute byte), by an independent
per-pixel brute force over orc_capsule_entry, and by opaque = nearest.
"""
import math

import numpy as np
import pytest

from paper_1801_01155_gb300 import synth


def _flat_tf(alpha, rgb=(1.0, 1.0, 1.0)):
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = rgb
    tf[:, 3] = alpha
    return tf


def _ortho_view(orc, centre, dist, fov, W, H, light=(0.0, 0.0, -1.0)):
    cx, cy, cz = centre
    return orc.make_view([cx, cy, cz + dist], [cx, cy, cz], [0, 1, 0], fov, W, H, list(light))


def test_silhouette_width_is_two_radii(orc):
    """One straight tube along x seen head-on from far away: it covers 2r
    across its axis (within one pixel per edge), centred on the image."""
    r = 0.2
    xyz = np.array([[2.0, 8.0, 8.0], [14.0, 8.0, 8.0]], np.float32)
    offs = np.array([0, 2], np.int64)
    g = orc.make_grid(16, 32)
    W = H = 101
    dist, fov = 2000.0, 0.02
    v = _ortho_view(orc, (8.0, 8.0, 8.0), dist, fov, W, H)
    rgba, tie, cnt = orc.raster(xyz, None, offs, g, v, orc.make_rdesc(r, synth.tf_ramp(), opaque=True),
                                orc.pixel_grid(0, 0, W, H))
    cov = rgba[:, 3].reshape(H, W) > 0.5
    px = 2 * dist * math.tan(math.radians(fov / 2)) / H
    for col in (10, 50, 90):
        assert abs(cov[:, col].sum() - 2 * r / px) <= 2.0
        rows = np.nonzero(cov[:, col])[0]
        assert abs(rows.mean() - (H - 1) / 2) <= 0.5
    assert cnt[0] == cov.sum()          # one fragment per covered pixel


def test_stacked_tubes_compose_in_closed_form(orc):
    """k parallel tubes one behind the other along the view axis, alpha a:
    pixels that see all k have A = 1 - (1 - a)^k; with termination at A >= 0.5
    only the first m fragments blend, m the first with 1 - (1 - a)^m >= 0.5."""
    a, k = 0.2, 5
    xyz = np.array([[[2.0, 8.0, z], [14.0, 8.0, z]] for z in (2.0, 4.0, 6.0, 8.0, 10.0)], np.float32).reshape(-1, 3)
    offs = np.arange(0, 2 * k + 1, 2, dtype=np.int64)
    g = orc.make_grid(16, 32)
    v = _ortho_view(orc, (8.0, 8.0, 8.0), 1000.0, 0.05, 21, 21)
    pix = orc.pixel_grid(0, 0, 21, 21)
    rgba, _, cnt = orc.raster(xyz, None, offs, g, v, orc.make_rdesc(0.5, _flat_tf(a), ert_alpha=2.0), pix)
    centre = rgba.reshape(21, 21, 4)[10, 10]
    a = float(np.float32(a))            # the transfer function holds float32
    assert centre[3] == pytest.approx(1 - (1 - a) ** k, abs=1e-12)
    rgba2, _, cnt2 = orc.raster(xyz, None, offs, g, v, orc.make_rdesc(0.5, _flat_tf(a), ert_alpha=0.5), pix)
    m = next(i for i in range(1, k + 1) if 1 - (1 - a) ** i >= 0.5)
    assert rgba2.reshape(21, 21, 4)[10, 10, 3] == pytest.approx(1 - (1 - a) ** m, abs=1e-12)
    assert cnt2[0] == cnt[0] and cnt2[1] < cnt[1]


def test_collinear_joint_is_blended_twice(orc):
    """A straight line of two collinear capsules (joint at x = 8): rays that
    pass within r of the joint along the axis enter both capsules (two
    fragments), others one: A = 1 - (1 - a)^2 vs a."""
    a, r = 0.3, 0.5
    xyz = np.array([[2.0, 8.0, 8.0], [8.0, 8.0, 8.0], [14.0, 8.0, 8.0]], np.float32)
    offs = np.array([0, 3], np.int64)
    g = orc.make_grid(16, 32)
    W, H = 201, 11
    dist = 1000.0
    fov = 2 * math.degrees(math.atan(4.0 * H / W / dist))   # the image spans x = 4 .. 12
    v = _ortho_view(orc, (8.0, 8.0, 8.0), dist, fov, W, H)
    rgba, tie, _ = orc.raster(xyz, None, offs, g, v, orc.make_rdesc(r, _flat_tf(a), ert_alpha=2.0),
                              orc.pixel_grid(0, 0, W, H))
    row = rgba.reshape(H, W, 4)[H // 2]
    a = float(np.float32(a))
    ok = tie.reshape(H, W)[H // 2] == 0
    half_w = dist * math.tan(math.radians(fov / 2)) * W / H
    x = 8.0 + ((np.arange(W) + 0.5) * 2 / W - 1) * half_w
    inside = (np.abs(x - 8.0) < r - 0.02) & ok
    outside = (np.abs(x - 8.0) > r + 0.02) & (np.abs(x - 8.0) < 5.0) & ok
    assert inside.sum() >= 4 and outside.sum() > 20
    np.testing.assert_allclose(row[inside, 3], 1 - (1 - a) ** 2, atol=1e-12)
    np.testing.assert_allclose(row[outside, 3], a, atol=1e-12)


def test_segment_attribute_byte(orc):
    """Attribute codes A = rint(65535 (a - min) / (max - min)); a capsule's
    byte is floor(((A_0 + A_1) 255 + 65535) / 131070), read back through a
    transfer function whose alpha encodes the byte."""
    tf = np.zeros((256, 4), np.float32)
    tf[:, 3] = 1.0
    tf[:, 0] = np.arange(256) / 256.0
    g = orc.make_grid(16, 32, attr_min=0.0, attr_max=10.0)
    v = _ortho_view(orc, (8.0, 8.0, 8.0), 1000.0, 0.05, 5, 5)
    for a0, a1 in ((0.0, 10.0), (1.0, 2.0), (3.3, 3.3), (9.99, 10.0)):
        xyz = np.array([[2.0, 8.0, 8.0], [14.0, 8.0, 8.0]], np.float32)
        attr = np.array([a0, a1], np.float32)
        rgba, _, _ = orc.raster(xyz, attr, np.array([0, 2], np.int64), g, v,
                                orc.make_rdesc(0.5, tf, opaque=True, ka=1.0, kd=0.0), orc.pixel_grid(2, 2, 1, 1))
        A = [int(np.rint(np.float32(np.float32(x - 0.0) / np.float32(10.0)) * np.float32(65535.0))) for x in (a0, a1)]
        byte = ((A[0] + A[1]) * 255 + 65535) // 131070
        assert rgba[0, 0] == pytest.approx(byte / 256.0, abs=1e-12)


def test_fragments_against_brute_force(orc):
    """Per pixel: the number of fragments equals the number of capsules that
    orc_capsule_entry reports entered; the opaque colour is that of the
    nearest one; blended alpha follows the sorted entries."""
    ls = synth.make_streamlines(60, 24, seed=7)
    g = orc.make_grid(8, 32, scale=8.0, attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))
    cam = synth.orbit_view((8, 8, 8), 24, 20)
    v = orc.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 24, 20, cam["light_dir"])
    tf = synth.tf_ramp(0.1, 0.4)
    r = 0.25
    pix = orc.pixel_grid(0, 0, 24, 20)
    rgba, tie, cnt = orc.raster(ls.xyz, ls.attr, ls.offsets, g, v, orc.make_rdesc(r, tf, ert_alpha=0.6), pix)
    ld = np.asarray(cam["light_dir"], np.float64)
    Lt = (-ld / np.linalg.norm(ld)).astype(np.float32).astype(np.float64)
    # the segments in grid coordinates, as the oracle forms them (float32 steps)
    p = (ls.xyz.astype(np.float32) - np.float32(0.0)) * np.float32(8.0)
    A = np.rint(np.clip((ls.attr - ls.attr.min()) / (ls.attr.max() - ls.attr.min()), 0, 1) * 65535).astype(np.int64)
    segs = []
    for c in range(len(ls.offsets) - 1):
        for i in range(ls.offsets[c], ls.offsets[c + 1] - 1):
            segs.append((p[i].astype(np.float64), p[i + 1].astype(np.float64), ((A[i] + A[i + 1]) * 255 + 65535) // 131070))
    total = 0
    checked = 0
    for n, (i, j) in enumerate(pix):
        o, d = orc.primary_ray(v, int(i), int(j))
        ts = []
        for k, (a, b, byte) in enumerate(segs):
            hit, t, _ = orc.capsule_entry(o.astype(np.float64), d.astype(np.float64), a, b, r)
            if hit:
                ts.append((t, k, byte))
        total += len(ts)
        if tie[n]:
            continue
        ts.sort()
        A, A32, Cc = 0.0, np.float32(0.0), np.zeros(3)
        for t, k, byte in ts:
            a, b, _ = segs[k]
            P = o.astype(np.float64) + t * d.astype(np.float64)
            h = np.clip(np.dot(P - a, b - a) / max(np.dot(b - a, b - a), 1e-300), 0.0, 1.0)
            nrm = P - (a + h * (b - a))
            nrm /= np.linalg.norm(nrm)
            w = (1 - A) * float(tf[byte, 3])
            Cc += w * tf[byte, :3].astype(np.float64) * (0.3 + 0.7 * abs(np.dot(nrm, Lt)))
            A += w
            A32 = np.float32(A32 + np.float32(np.float32(1.0) - A32) * tf[byte, 3])
            if A32 >= np.float32(0.6):
                break
        assert rgba[n, 3] == pytest.approx(A, abs=1e-12)
        np.testing.assert_allclose(rgba[n, :3], Cc + (1 - A) * 1.0, atol=1e-9)
        checked += 1
    assert total == cnt[0] and checked > 400
