"""Pins of the oracle's second right answer for a pixel whose only near-tie
is one pair of hits in depth order (Secs. 4, 5.1: hits of a voxel are
composited in depth order; the rasterised comparison system sorts its
fragments by depth). Two straight tubes entered at exactly the same depth
by a ray: either order is right, and the two results have closed forms."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O

TIE_SORT = 4
R_TUBE = 0.3
# two lines along y through bin centres of a 32 x 32 face lattice, mirror
# images about x = 1 + 16.5 / 32 at depth z = 1 + 16.5 / 32: a ray along +z
# through that x passes both axes at distance 0.25, so it enters both tubes
# at z = zc - sqrt(r^2 - 0.25^2) (in voxel (1, 1, 1), away from its faces)
XC = 1.0 + 16.5 / 32.0
ZC = 1.0 + 16.5 / 32.0
XA, XB = 1.0 + 8.5 / 32.0, 1.0 + 24.5 / 32.0


def _scene():
    xyz = np.array([[XA, 0.5, ZC], [XA, 3.5, ZC], [XB, 0.5, ZC], [XB, 3.5, ZC]], np.float32) / 4.0
    attr = np.array([0.0, 0.0, 1.0, 1.0], np.float32)     # line A: byte 0, line B: byte 255
    offsets = np.array([0, 2, 4], np.int64)
    g = O.make_grid(4, 32, scale=4.0, attr_min=0.0, attr_max=1.0)
    tf = np.zeros((256, 4), np.float32)
    tf[0] = (1.0, 0.2, 0.0, 0.5)
    tf[255] = (0.0, 0.3, 1.0, 0.25)
    # a 1 x 1 image: the pixel centre's ray is the forward axis, exactly +z
    view = O.make_view((XC, 1.5, -5.0), (XC, 1.5, 0.0), (0.0, 1.0, 0.0), 30.0, 1, 1, (0.0, 0.0, -1.0))
    return xyz, attr, offsets, g, tf, view


def _expected(tf, opaque):
    """Closed forms: both entry normals are (+-0.25, 0, -h) / r, h =
    sqrt(r^2 - 0.25^2), so with the light along +z both hits are shaded by
    ka + kd h / r (the descriptor's float32 weights and radius); composited A
    then B, and B then A (Sec. 5.1)."""
    ka, kd, r = float(np.float32(0.3)), float(np.float32(0.7)), float(np.float32(R_TUBE))
    h = np.sqrt(r ** 2 - 0.25 ** 2)
    k = ka + kd * h / r
    cA, aA = tf[0, :3].astype(np.float64) * k, 1.0 if opaque else float(tf[0, 3])
    cB, aB = tf[255, :3].astype(np.float64) * k, 1.0 if opaque else float(tf[255, 3])
    A = 1.0 - (1.0 - aA) * (1.0 - aB)
    ab = aA * cA + (1.0 - aA) * aB * cB
    ba = aB * cB + (1.0 - aB) * aA * cA
    bg = np.ones(3)
    first = lambda c, a: np.concatenate([c + (1.0 - a) * bg, [a]])   # noqa: E731
    if opaque:
        return first(cA, 1.0), first(cB, 1.0)
    return first(ab, A), first(ba, A)


@pytest.mark.parametrize("opaque", [False, True])
def test_ray_caster_exact_tie_has_both_orders(opaque):
    xyz, attr, offsets, g, tf, view = _scene()
    vs = O.VoxSet(xyz, attr, offsets, g)
    rd = O.make_rdesc(R_TUBE, tf, opaque=opaque, ert_alpha=2.0)
    rgba, tie, cnt, alt = O.render(vs, None, view, rd, O.pixel_grid(0, 0, 1, 1), alts=True)
    assert tie[0] == TIE_SORT and int(cnt[3]) == (1 if opaque else 2)
    ab, ba = _expected(tf, opaque)
    # equal depths sort by record index: line A (curve 0) first
    np.testing.assert_allclose(rgba[0], ab, rtol=0, atol=1e-12)
    np.testing.assert_allclose(alt[0], ba, rtol=0, atol=1e-12)


@pytest.mark.parametrize("opaque", [False, True])
def test_rasteriser_exact_tie_has_both_orders(opaque):
    xyz, attr, offsets, g, tf, view = _scene()
    rd = O.make_rdesc(R_TUBE, tf, opaque=opaque, ert_alpha=2.0)
    rgba, tie, cnt, alt = O.raster(xyz, attr, offsets, g, view, rd, O.pixel_grid(0, 0, 1, 1), alts=True)
    assert tie[0] == TIE_SORT and int(cnt[0]) == 2
    ab, ba = _expected(tf, opaque)
    np.testing.assert_allclose(rgba[0], ab, rtol=0, atol=1e-12)
    np.testing.assert_allclose(alt[0], ba, rtol=0, atol=1e-12)


def test_no_second_answer_without_a_depth_tie():
    """A ray that sees one tube only (through x = XA) has no near-tie and no
    second answer."""
    xyz, attr, offsets, g, tf, _ = _scene()
    view = O.make_view((XA, 1.5, -5.0), (XA, 1.5, 0.0), (0.0, 1.0, 0.0), 30.0, 1, 1, (0.0, 0.0, -1.0))
    vs = O.VoxSet(xyz, attr, offsets, g)
    rgba, tie, _, alt = O.render(vs, None, view, O.make_rdesc(R_TUBE, tf, ert_alpha=2.0),
                                 O.pixel_grid(0, 0, 1, 1), alts=True)
    assert tie[0] == 0 and rgba[0, 3] > 0 and np.isnan(alt[0]).all()
