"""Pins of the representative lines (reading R3, Sec. 3.4) and of the
shadows against them (reading S5, Sec. 5.2's first approach).

Hand-built voxel sets with closed-form averages, the flip rule, the
connectivity step and the level above; the half-line/segment distance
against dense sampling; the shadow test against hand-placed occluders.
"""
import math

import numpy as np
import pytest


def _vs(orc, curves, res=4, bins=32):
    xyz = np.concatenate([np.asarray(c, np.float32) for c in curves])
    offs = np.cumsum([0] + [len(c) for c in curves])
    return orc.VoxSet(xyz, None, offs, orc.make_grid(res, bins, scale=1.0))


def _cell(res, x, y, z):
    return x + res * (y + res * z)


def test_single_segment_voxel_keeps_its_segment(orc):
    vs = _vs(orc, [[[0.2, 1.3, 2.6], [3.8, 1.7, 2.4]]])
    e = vs.export()
    reps = orc.Reps(vs, 1).export(0)
    for v in range(64):
        beg, end = e["offset"][v], e["offset"][v + 1]
        if end - beg == 1:
            f = e["fields"][beg]
            assert reps[v, 0] == 1 and tuple(reps[v, 1:]) == tuple(f[:6])
        if end == beg:
            assert reps[v, 0] == 0


def test_flip_rule_and_average(orc):
    """Voxel (1, 1, 1): a line along +x at bin 10 (curve 0) and the same
    line run backwards at bin 13 (curve 1). Flipped, both run along +x; the
    y bins average to floor((10 + 13 + 1) / 2) = 12 on both faces."""
    y10, y13 = 1 + 10.5 / 32, 1 + 13.5 / 32
    vs = _vs(orc, [[[0.2, y10, 1.5], [3.8, y10, 1.5]], [[3.8, y13, 1.5], [0.2, y13, 1.5]]])
    r = orc.Reps(vs, 1).export(0)[_cell(4, 1, 1, 1)]
    zb = 16   # z = 1.5 -> bin 16
    assert tuple(r) == (1, 0, 12, zb, 1, 12, zb)   # -x face (y 12, z 16) -> +x face


def test_connectivity_meets_in_the_middle(orc):
    """Voxel (1, 1, 1) holds curve 0 (y bin 10) and curve 1 (y bin 12); voxel
    (2, 1, 1) only curve 0 (curve 1 ends inside it, and its last partial
    piece is dropped). Averages in (1, 1, 1): y = (21 + 25) / (2 * 64) * 32
    -> bin 11 at both ends. Their shared face: 11 in (1, 1, 1), 10 in
    (2, 1, 1), joined at floor((11 + 10 + 1) / 2) = 11."""
    y10, y12 = 1 + 10.5 / 32, 1 + 12.5 / 32
    vs = _vs(orc, [[[0.2, y10, 1.5], [3.8, y10, 1.5]], [[0.2, y12, 1.5], [2.5, y12, 1.5]]])
    r = orc.Reps(vs, 1).export(0)
    a, b = r[_cell(4, 1, 1, 1)], r[_cell(4, 2, 1, 1)]
    assert a[4] == 1 and b[1] == 0          # A's +x end and B's -x start
    assert a[5] == 11 and b[2] == 11
    assert a[2] == 11 and b[5] == 10         # ends without a neighbour line keep their bins


def test_connectivity_takes_the_start_point_first(orc):
    """A curve makes a U-turn inside voxel (1, 1, 1): in and out through its
    +x face (bins 8 and 20); a second curve crosses voxel (2, 1, 1) at bin
    16. On the shared face the start point (bin 8) is joined with the
    neighbour's: floor((8 + 16 + 1) / 2) = 12; the end point keeps 20."""
    y8, y20, y16 = 1 + 8.5 / 32, 1 + 20.5 / 32, 1 + 16.5 / 32
    u_turn = [[2.5, y8, 1.5], [1.6, y8, 1.5], [1.6, y20, 1.5], [2.5, y20, 1.5]]
    vs = _vs(orc, [u_turn, [[1.9, y16, 1.5], [3.9, y16, 1.5]]])
    r = orc.Reps(vs, 1).export(0)
    a, b = r[_cell(4, 1, 1, 1)], r[_cell(4, 2, 1, 1)]
    assert tuple(a) == (1, 1, 12, 16, 1, 20, 16)
    assert tuple(b) == (1, 0, 12, 16, 1, 16, 16)


def test_level_above_from_the_children(orc):
    """A line along x at y = z = 1 + 8.5/32 (bin 8) through an 8^3 grid. The
    level-1 cell (1, 0, 0) holds the full lines of its children (2, 1, 1)
    and (3, 1, 1): the averaged start (x 1/4 of the parent) is nearest the
    -x face, the averaged end (x 3/4) the +x face, and y = z = (2N + 17) /
    4N of the parent fall in bin floor(81 * 32 / 128) = 20. The level-1
    cell (0, 0, 0) holds only child (1, 1, 1) (the first piece starts inside
    its voxel and is dropped): its start point, the parent's centre in x,
    is nearer the +y face (0.367) than the -x face (0.5) and snaps there."""
    c = 1 + 8.5 / 32
    vs = _vs(orc, [[[0.2, c, c], [7.8, c, c]]], res=8)
    r1 = orc.Reps(vs, 2).export(1)
    assert tuple(r1[_cell(4, 1, 0, 0)]) == (1, 0, 20, 20, 1, 20, 20)
    assert tuple(r1[_cell(4, 2, 0, 0)]) == (1, 0, 20, 20, 1, 20, 20)
    assert tuple(r1[_cell(4, 0, 0, 0)])[:2] == (1, 3) and tuple(r1[_cell(4, 0, 0, 0)])[4:] == (1, 20, 20)
    assert r1[:, 0].sum() == 4


def test_halfline_segment_distance_against_sampling(orc):
    rng = np.random.default_rng(3)
    for _ in range(40):
        o, a, b = rng.uniform(-2, 2, (3, 3))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        t = np.linspace(0.0, 8.0, 1601)[:, None, None]
        h = np.linspace(0.0, 1.0, 401)[None, :, None]
        pts = o + t * d - (a + h * (b - a))
        brute = np.sqrt((pts ** 2).sum(-1)).min()
        got = orc.halfline_segment_distance(o, d, a, b)
        assert got <= brute + 1e-12 and got == pytest.approx(brute, abs=6e-3)


def test_shadow_against_a_hand_placed_occluder(orc):
    """A level-0 representative line along x at y = 2 + 16.5/32, z = 2 +
    16.5/32 (the quantised line), radius 0.2. A point straight below it,
    lit from +y, is blocked when its z is within the radius of the line's z
    and visible otherwise; lit from -y (away from the line) always visible."""
    zq = 2 + 16.5 / 32
    vs = _vs(orc, [[[0.2, 2.5, 2.5], [3.8, 2.5, 2.5]]])
    reps = orc.Reps(vs, 1)
    up, down = [0.0, 1.0, 0.0], [0.0, -1.0, 0.0]
    assert orc.shadow_reps_visibility(vs, reps, 0.2, 0, [1.5, 0.3, zq + 0.1], up) == 0.0
    assert orc.shadow_reps_visibility(vs, reps, 0.2, 0, [1.5, 0.3, zq + 0.3], up) == 1.0
    assert orc.shadow_reps_visibility(vs, reps, 0.2, 0, [1.5, 0.3, zq + 0.1], down) == 1.0
    # the half-line starts one cell away: a point 0.5 below the line is not blocked by it
    assert orc.shadow_reps_visibility(vs, reps, 0.2, 0, [1.5, zq - 0.5, zq], up) == 1.0


def _rep_world(r, cell, dims, level, N):
    size = 2.0 ** level
    p = np.array([cell % dims[0], (cell // dims[0]) % dims[1], cell // (dims[0] * dims[1])], float)
    out = []
    for f, u, v in ((r[1], r[2], r[3]), (r[4], r[5], r[6])):
        ax = f >> 1
        others = [a for a in range(3) if a != ax]
        q = np.zeros(3)
        q[ax] = f & 1
        q[others[0]] = (u + 0.5) / N
        q[others[1]] = (v + 0.5) / N
        out.append((p + q) * size)
    return out


@pytest.mark.parametrize("level", [0, 1])
def test_shadow_walk_equals_brute_force(orc, level):
    """The level-l cell walk against testing every representative line whose
    cell the half-line (started one cell size toward the light) crosses."""
    rng = np.random.default_rng(11 + level)
    res, N, r = 8, 32, 0.15
    curves = []
    for _ in range(12):
        a, b = rng.uniform(0.1, res - 0.1, (2, 3))
        curves.append(np.linspace(a, b, 9))
    vs = _vs(orc, curves, res=res, bins=N)
    reps = orc.Reps(vs, 2)
    rl = r * 2.0 ** level
    dims = [(res + 2 ** level - 1) // 2 ** level] * 3
    rep = reps.export(level)
    checked = blocked = 0
    for _ in range(300):
        P = rng.uniform(0.0, res, 3)
        Lt = rng.standard_normal(3)
        Lt /= np.linalg.norm(Lt)
        S = P + 2.0 ** level * Lt
        want, near = 1.0, False
        for cell in np.nonzero(rep[:, 0])[0]:
            lo = np.array([cell % dims[0], (cell // dims[0]) % dims[1], cell // (dims[0] * dims[1])]) * 2.0 ** level
            hi = lo + 2.0 ** level
            with np.errstate(divide="ignore", invalid="ignore"):
                t1, t2 = (lo - S) / Lt, (hi - S) / Lt
            tn = max(0.0, np.nanmax(np.minimum(t1, t2)))
            tf = np.nanmin(np.maximum(t1, t2))
            if tf - tn < 1e-9:
                near |= abs(tf - tn) < 1e-6
                continue
            a, b = _rep_world(rep[cell], cell, dims, level, N)
            d = orc.halfline_segment_distance(S, Lt, a, b)
            near |= abs(d - rl) < 1e-6
            if d <= rl:
                want = 0.0
        if near:
            continue
        checked += 1
        blocked += want == 0.0
        assert orc.shadow_reps_visibility(vs, reps, r, level, P, Lt) == want
    assert checked > 250 and 10 < blocked < checked - 10


def test_image_with_rep_shadows_only_darkens(orc):
    """Opaque frame: with representative-line shadows every pixel is at most
    as bright as without (visibility only scales the diffuse term) and a
    visible share of the lit pixels falls into shadow."""
    from paper_1801_01155_gb300 import synth
    ls = synth.make_streamlines(150, 48, seed=5)
    g = orc.make_grid(16, 32, scale=16.0, attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))
    vs = orc.VoxSet(ls.xyz, ls.attr, ls.offsets, g)
    cam = synth.orbit_view((16, 16, 16), 48, 40)
    v = orc.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 48, 40, cam["light_dir"])
    pix = orc.pixel_grid(0, 0, 48, 40)
    reps = orc.Reps(vs, 3)
    base, tb, _ = orc.render(vs, None, v, orc.make_rdesc(0.2, synth.tf_ramp(), opaque=True), pix)
    for level in (0, 1, 2):
        sh, ts, _ = orc.render(vs, None, v, orc.make_rdesc(0.2, synth.tf_ramp(), opaque=True, reps=reps,
                                                           shadow_level=level), pix)
        ok = (tb == 0) & (ts == 0) & (base[:, 3] > 0)
        assert np.all(sh[ok, :3] <= base[ok, :3] + 1e-12)
        np.testing.assert_array_equal(sh[ok, 3], base[ok, 3])
        dark = (sh[ok, :3] < base[ok, :3] - 1e-6).any(1).mean()
        assert 0.02 < dark < 0.9


def test_flip_budget_is_the_diffuse_term(orc):
    """Opaque frame, uniform grey transfer function, no AO: a pixel's colour
    is c (ka + kd V |n.L|) with a binary V, so the most a flip of V can move
    it is kd |n.L| c, which the same frame without shadows gives as its
    colour minus ka c. Every pixel flagged with a near-tie visibility (bit
    64) carries exactly that budget; unflagged pixels carry at most the
    threshold below which near-ties are not flagged; each flagged pixel is
    either lit (colour without shadows) or dark (ka c)."""
    from paper_1801_01155_gb300 import synth
    ls = synth.make_streamlines(600, 48, seed=5)
    g = orc.make_grid(16, 32, scale=16.0, attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))
    vs = orc.VoxSet(ls.xyz, ls.attr, ls.offsets, g)
    W, H = 320, 240
    cam = synth.orbit_view((16, 16, 16), W, H)
    v = orc.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], W, H, cam["light_dir"])
    pix = orc.pixel_grid(0, 0, W, H)
    reps = orc.Reps(vs, 3)
    c, ka = float(np.float32(0.8)), float(np.float32(0.3))
    tf = np.tile(np.array([c, c, c, 1.0], np.float32), 256)
    plain, tp, _ = orc.render(vs, None, v, orc.make_rdesc(0.2, tf, opaque=True), pix)
    flagged = 0
    for level in (0, 1, 2):
        rgba, tie, _, flip = orc.render(vs, None, v, orc.make_rdesc(0.2, tf, opaque=True, reps=reps,
                                                                     shadow_level=level), pix, flips=True)
        sh = (tie & orc.TIE_SHADOW) != 0
        flagged += int(sh.sum())
        assert np.all(flip[~sh] < 5e-4)
        np.testing.assert_allclose(flip[sh], plain[sh, 0] - ka * c, rtol=0, atol=1e-12)
        lit = np.isclose(rgba[sh, 0], plain[sh, 0], rtol=0, atol=1e-12)
        dark = np.isclose(rgba[sh, 0], ka * c, rtol=0, atol=1e-12)
        assert np.all(lit | dark)
    assert flagged >= 10


def test_flip_budget_adds_up_along_the_ray(orc):
    """Transparent frames: the budget sums over every composited hit whose
    visibility is a near-tie, so terminating later (more hits composited)
    never lowers it, and it never exceeds the pixel's whole diffuse part
    (the frame without shadows minus its ambient part ka c A)."""
    from paper_1801_01155_gb300 import synth
    ls = synth.make_streamlines(1500, 64, seed=6)
    g = orc.make_grid(16, 32, scale=16.0, attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))
    vs = orc.VoxSet(ls.xyz, ls.attr, ls.offsets, g)
    W, H = 480, 360
    cam = synth.orbit_view((16, 16, 16), W, H)
    v = orc.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], W, H, cam["light_dir"])
    pix = orc.pixel_grid(0, 0, W, H)
    reps = orc.Reps(vs, 3)
    c, ka = float(np.float32(0.8)), float(np.float32(0.3))
    tf = np.tile(np.array([c, c, c, 0.2], np.float32), 256)
    plain, _, _ = orc.render(vs, None, v, orc.make_rdesc(0.2, tf, ert_alpha=2.0), pix)
    diffuse = plain[:, 0] - (1.0 - plain[:, 3]) * 1.0 - ka * c * plain[:, 3]   # minus background and ambient
    flips = []
    for ert in (0.5, 0.9, 2.0):
        _, tie, _, flip = orc.render(vs, None, v, orc.make_rdesc(0.2, tf, ert_alpha=ert, reps=reps,
                                                               shadow_level=1), pix, flips=True)
        flips.append(flip)
    assert np.all(flips[0] <= flips[1] + 1e-12) and np.all(flips[1] <= flips[2] + 1e-12)
    assert np.all(flips[2] <= diffuse + 1e-9)
    assert (flips[2] > flips[0] + 1e-6).sum() > 20
