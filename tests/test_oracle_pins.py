"""Pins of the FP64 oracle to facts other than itself.

Each test checks the oracle against something the paper or the mathematics
fixes: numbers printed in the paper, hand-derived cases, closed forms,
invariants, brute force on tiny inputs. None needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1801_01155_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(path):
    out = []
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            out.append([int(x) for x in line.split()])
    return out


# ------------------------------------------------------------ record budget (Sec. 6.2)
def test_record_bytes_match_paper(orc):
    rows = _rows(os.path.join(GOLDEN, "record_bytes.txt"))
    table = {n: b for n, b in rows[:6]}
    for n, b in table.items():
        assert orc.record_bytes(n) == b, n
    # 2 * 10 bin bits for 32^2: bits minus face ids (2*3), attribute (8), local id (5)
    n, binbits = rows[6]
    assert orc.record_bits(n) - 2 * 3 - 8 - 5 == binbits


# ------------------------------------------------------------ fixed point (reading V1)
def test_fixed_point_exact_values(orc):
    g = orc.make_grid(4, 4, scale=4.0)
    X = orc.fixed_point(np.array([[0.5, 0.25, 1.0]], np.float32), g)
    assert X.tolist() == [[2 * 65536, 65536, 4 * 65536]]
    # half-way cases round to even: 2^-17 -> 0.5 unit -> 0 ; 3*2^-17 -> 1.5 -> 2
    g1 = orc.make_grid(4, 4, scale=1.0)
    v = np.array([[2.0 ** -17, 3 * 2.0 ** -17, -(2.0 ** -17)]], np.float32)
    assert orc.fixed_point(v, g1).tolist() == [[0, 2, 0]]


def test_fixed_point_rejects_bad_vertices(orc):
    g = orc.make_grid(4, 4, scale=1.0)
    for bad in ([np.nan, 0, 0], [0, np.inf, 0], [0, 0, 20000.0]):
        with pytest.raises(orc.OracleError):
            orc.fixed_point(np.array([bad], np.float32), g)


def test_attr16_range(orc):
    a = np.array([-1.0, 0.0, 0.5, 1.0, 2.0], np.float32)
    A = orc.attr16(a, 0.0, 1.0)
    assert A.tolist() == [0, 0, 32768, 65535, 65535]   # 0.5*65535 = 32767.5 -> even 32768
    assert orc.attr16(a, 1.0, 1.0).tolist() == [0] * 5


# ------------------------------------------------------------ hand cases (Secs. 3.1, 3.2)
@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "vox_hand_cases.json")))["cases"],
                         ids=lambda c: c["name"])
def test_voxelize_hand_cases(orc, case):
    g = orc.make_grid(case["res"], case["bins"], scale=1.0,
                      attr_min=case["attr_range"][0], attr_max=case["attr_range"][1])
    attr = None if case["attr"] is None else np.array(case["attr"], np.float32)
    vs = orc.VoxSet(np.array(case["xyz"], np.float32), attr, np.array(case["offsets"]), g)
    e = vs.export()
    got = []
    for i in range(vs.nseg):
        got.append([int(np.searchsorted(e["offset"], i, side="right") - 1), int(e["curve"][i]),
                    int(e["ordinal"][i])] + [int(x) for x in e["fields"][i]])
    assert got == case["segments"]


# ------------------------------------------------------------ invariants on streamlines
@pytest.fixture(scope="module")
def c1set(orc):
    ls = synth.make_streamlines(200, 64, seed=0)
    g = orc.make_grid(32, 32, scale=32.0, attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))
    vs = orc.VoxSet(ls.xyz, ls.attr, ls.offsets, g)
    return ls, g, vs, vs.export()


def _decode(e, res, N):
    """World (grid-unit) endpoints of every segment."""
    off, f = e["offset"], e["fields"].astype(np.int64)
    vid = np.searchsorted(off, np.arange(len(f)), side="right") - 1
    base = np.stack([vid % res, (vid // res) % res, vid // (res * res)], 1).astype(np.float64)

    def pt(face, u, v):
        q = np.zeros((len(face), 3))
        ax = face // 2
        b0 = np.where(ax == 0, 1, 0)
        b1 = np.where(ax == 2, 1, 2)
        rows = np.arange(len(face))
        q[rows, ax] = (face & 1).astype(np.float64)
        q[rows, b0] = (u + 0.5) / N
        q[rows, b1] = (v + 0.5) / N
        return q

    return base + pt(f[:, 0], f[:, 1], f[:, 2]), base + pt(f[:, 3], f[:, 4], f[:, 5]), vid


def test_canonical_order_and_ranges(c1set):
    ls, g, vs, e = c1set
    assert e["offset"][0] == 0 and e["offset"][-1] == vs.nseg
    assert np.all(np.diff(e["offset"].astype(np.int64)) >= 0)
    f = e["fields"]
    assert f[:, [0, 3]].max() <= 5 and f[:, [1, 2, 4, 5]].max() < 32
    key = e["curve"].astype(np.int64) * 2 ** 32 + e["ordinal"]
    for v in range(vs.nvox):
        a, b = e["offset"][v], e["offset"][v + 1]
        assert np.all(np.diff(key[a:b]) > 0)


def test_continuity_exit_equals_next_entry(c1set):
    """Sec. 3.1: consecutive face points of a curve bound consecutive segments,
    so a continuing segment starts where its predecessor ends."""
    ls, g, vs, e = c1set
    a, b, vid = _decode(e, 32, 32)
    order = np.lexsort((e["ordinal"], e["curve"]))
    cur, ordn, cont = e["curve"][order], e["ordinal"][order], e["fields"][order, 7]
    nxt = np.nonzero((cur[1:] == cur[:-1]) & (ordn[1:] == ordn[:-1] + 1))[0]
    assert len(nxt) > 1000
    np.testing.assert_array_equal(b[order][nxt], a[order][nxt + 1])
    assert np.all(cont[nxt + 1] == 1)
    # neighbouring voxels share exactly one face
    va, vb = vid[order][nxt], vid[order][nxt + 1]
    dv = np.abs(np.stack([va % 32 - vb % 32, (va // 32) % 32 - (vb // 32) % 32, va // 1024 - vb // 1024], 1))
    assert np.all(dv.sum(1) == 1)


def _point_polyline_dist(p, poly):
    a, b = poly[:-1], poly[1:]
    ab = b - a
    t = np.clip(((p[:, None, :] - a[None]) * ab[None]).sum(-1) / np.maximum((ab * ab).sum(-1), 1e-30)[None], 0, 1)
    c = a[None] + t[..., None] * ab[None]
    return np.sqrt(((p[:, None, :] - c) ** 2).sum(-1)).min(1)


def test_deviation_bounded_by_voxel_diagonal(c1set):
    """Sec. 3.1: the deviation between a curve and its segments is bounded by the
    voxel diagonal."""
    ls, g, vs, e = c1set
    a, b, vid = _decode(e, 32, 32)
    grid_xyz = ls.xyz.astype(np.float64) * 32.0
    worst = 0.0
    for c in range(0, ls.n_curves, 7):
        m = e["curve"] == c
        if not m.any():
            continue
        poly = grid_xyz[ls.offsets[c]:ls.offsets[c + 1]]
        s = np.linspace(0, 1, 9)[:, None, None]
        pts = (a[m][None] * (1 - s) + b[m][None] * s).reshape(-1, 3)
        worst = max(worst, _point_polyline_dist(pts, poly).max())
    assert worst <= math.sqrt(3.0) + 1e-9
    assert worst > 0.1


def test_voxel_sequence_against_dense_sampling(c1set):
    """Brute force: sample every curve densely in fixed point and list the voxels
    it passes through; the oracle's voxel sequence (first and last partial
    voxels dropped) must contain that list in order, every step crossing one face."""
    ls, g, vs, e = c1set
    X = __import__("oracle.oracle", fromlist=["x"]).fixed_point(ls.xyz, g).astype(np.int64)
    a, b, vid = _decode(e, 32, 32)
    checked = 0
    for c in range(0, ls.n_curves, 5):
        P = X[ls.offsets[c]:ls.offsets[c + 1]]
        M = 256
        t = np.arange(M)[:, None]
        pts = (P[:-1, None, :] * (M - t)[None] + P[1:, None, :] * t[None]) // M   # exact floor
        pts = np.concatenate([pts.reshape(-1, 3), P[-1:]])
        vox = pts // 65536
        keep = np.concatenate([[True], np.any(vox[1:] != vox[:-1], 1)])
        seq = vox[keep]
        if len(seq) < 3:
            continue
        seq = seq[1:-1]                                       # partial first / last voxels
        inside = np.all((seq >= 0) & (seq < 32), 1)
        if not inside.all():
            continue                                          # keep to curves inside the grid
        m = np.nonzero(e["curve"] == c)[0]
        m = m[np.argsort(e["ordinal"][m])]
        ov = vid[m]
        ovx = np.stack([ov % 32, (ov // 32) % 32, ov // 1024], 1)
        assert np.all(np.abs(np.diff(ovx, axis=0)).sum(1) == 1)
        j = 0
        for s in seq:
            while j < len(ovx) and not np.array_equal(ovx[j], s):
                j += 1
            assert j < len(ovx), f"curve {c}: sampled voxel {s} missing from oracle sequence"
        checked += 1
    assert checked > 5


def test_quantised_length_bound(c1set):
    """Each quantised endpoint moves at most half a sub-square diagonal (Sec. 3.2),
    so the quantised chord of a voxel exceeds the exact chord, itself no longer
    than the curve inside the voxel, by at most sqrt(2)/N."""
    ls, g, vs, e = c1set
    a, b, vid = _decode(e, 32, 32)
    qlen = np.sqrt(((b - a) ** 2).sum(1))
    grid_xyz = ls.xyz.astype(np.float64) * 32.0
    seglen = np.sqrt((np.diff(grid_xyz, axis=0) ** 2).sum(1))
    seglen[ls.offsets[1:-1] - 1] = 0.0                        # no edges across curves
    total_poly = seglen.sum()
    assert qlen.sum() <= total_poly + vs.nseg * math.sqrt(2) / 32


# ------------------------------------------------------------ LoD (Sec. 3.4, Eq. 1)
def test_lod_sums_and_hand_density(orc, c1set):
    ls, g, vs, e = c1set
    sig = np.full(256, 0.5, np.float32)
    lod = orc.Lod(vs, 3, sig)
    l0 = lod.export(0)
    for l in range(3):
        x = lod.export(l)
        assert int(x["cnt"].sum()) == vs.nseg
        assert x["len"].sum() == pytest.approx(l0["len"].sum(), rel=1e-12)
        assert x["dens"].sum() == pytest.approx(0.5 * l0["len"].sum(), rel=1e-12)
    assert lod.dims(1) == (16, 16, 16) and lod.dims(2) == (8, 8, 8)

    # one straight x-segment through voxel (1,1,2) of a 5^3 grid: length 1, rho = sigma
    g5 = orc.make_grid(5, 4, scale=1.0)
    v1 = orc.VoxSet(np.array([[0.5, 1.5, 2.5], [2.5, 1.5, 2.5]], np.float32), None, np.array([0, 2]), g5)
    sig2 = np.zeros(256, np.float32)
    sig2[0] = 0.25
    L1 = orc.Lod(v1, 3, sig2)
    assert L1.dims(1) == (3, 3, 3) and L1.dims(2) == (2, 2, 2)      # ceil(5/2), ceil(3/2)
    d0, d1, d2 = (L1.export(l)["dens"] for l in range(3))
    assert d0[1 + 5 * (1 + 5 * 2)] == 0.25
    assert d1[0 + 3 * (0 + 3 * 1)] == 0.25
    assert d2[0] == 0.25
    assert L1.export(0)["len"].max() == 1.0
    # a diagonal segment from the -x face (bins (1,1)) to the +y face (bins (3,1)), N=4:
    # (0, .375, .375) -> (.875, 1, .375): length sqrt(.875^2 + .625^2)
    v2 = orc.VoxSet(np.array([[-0.6, -0.06, 0.375], [1.8, 1.65, 0.375]], np.float32), None,
                    np.array([0, 2]), orc.make_grid(2, 4, scale=1.0))
    x2 = v2.export()
    i = int(np.searchsorted(x2["offset"], 0, side="right") - 1)
    assert x2["fields"][0, :6].tolist() == [0, 1, 1, 3, 3, 1] and i == 0
    L2 = orc.Lod(v2, 1, np.ones(256, np.float32))
    assert L2.export(0)["len"][0] == pytest.approx(math.hypot(0.875, 0.625), abs=1e-15)


# ------------------------------------------------------------ capsule intersection (Secs. 4, 4.1)
@pytest.mark.parametrize("d", [0.0, 0.05, 0.1499])
def test_capsule_perpendicular_closed_form(orc, d):
    r = 0.15
    a, b = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0])
    o = np.array([0.4, d, -5.0])
    hit, t, dist = orc.capsule_entry(o, [0, 0, 1.0], a, b, r)
    assert hit
    assert t == pytest.approx(5.0 - math.sqrt(r * r - d * d), abs=1e-12)
    assert dist == pytest.approx(d, abs=1e-12)


def test_capsule_misses_and_caps(orc):
    r = 0.2
    a, b = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0])
    assert not orc.capsule_entry([0.4, 0.21, -5.0], [0, 0, 1.0], a, b, r)[0]
    # beyond the end point the cap sphere is hit: distance 0.1 past b
    hit, t, _ = orc.capsule_entry([1.1, 0.0, -5.0], [0, 0, 1.0], a, b, r)
    assert hit and t == pytest.approx(5.0 - math.sqrt(r * r - 0.01), abs=1e-12)
    # along the axis: enters the cap of a at distance |o - a| - r
    hit, t, _ = orc.capsule_entry([-3.0, 0.0, 0.0], [1.0, 0, 0], a, b, r)
    assert hit and t == pytest.approx(3.0 - r, abs=1e-12)
    # zero-length segment is a sphere
    hit, t, _ = orc.capsule_entry([0.0, 0.0, -2.0], [0, 0, 1.0], a, a, r)
    assert hit and t == pytest.approx(2.0 - r, abs=1e-12)
    # ray starting inside the tube: no entering intersection ahead
    assert not orc.capsule_entry([0.5, 0.0, 0.0], [0, 0, 1.0], a, b, r)[0]
    # tube behind the ray
    assert not orc.capsule_entry([0.4, 0.0, 5.0], [0, 0, 1.0], a, b, r)[0]


def test_capsule_far_origin_float32_direction(orc):
    """Primary rays start hundreds of voxels away with a float32 direction
    whose length is 1 only to ~1e-7. Closed form for a ray aimed 400 units
    along d at a sphere (zero-length segment) offset 0.1 perpendicular to d:
    |o + t d - c|^2 = (t - 400)^2 |d|^2 + 0.01, so t = 400 - sqrt(r^2 - 0.01) / |d|."""
    d32 = np.array([0.6, 0.0, 0.8], np.float64) * (1 + 3e-7)
    d = d32.astype(np.float32).astype(np.float64)          # |d| != 1
    o = np.array([0.25, -0.5, -300.0])
    c = o + 400.0 * d + np.array([0.0, 0.1, 0.0])          # (0,1,0) is exactly normal to d
    r = 0.15
    hit, t, dist = orc.capsule_entry(o, d, c, c, r)
    nd = math.sqrt(d[0] ** 2 + d[2] ** 2)
    assert hit and t == pytest.approx(400.0 - math.sqrt(r * r - 0.01) / nd, abs=1e-9)
    assert dist == pytest.approx(0.1, abs=1e-9)
    # the same through the body of a long tube along y (perpendicular to d)
    hit, t, dist = orc.capsule_entry(o, d, c - [0, 2.0, 0], c + [0, 2.0, 0], r)
    assert hit and t == pytest.approx(400.0 - r / nd, abs=1e-9)
    # and a near miss by 1e-6 is a miss
    cm = o + 400.0 * d + np.array([0.0, r + 1e-6, 0.0])
    assert not orc.capsule_entry(o, d, cm, cm, r)[0]


# ------------------------------------------------------------ primary rays (reading R0)
def test_primary_ray_geometry(orc):
    eye, at = np.array([10.0, 20.0, 30.0]), np.array([1.0, 2.0, 3.0])
    v = orc.make_view(eye, at, [0, 1, 0], 40.0, 1, 1, [0, -1, 0])
    o, d = orc.primary_ray(v, 0, 0)
    f = (at - eye) / np.linalg.norm(at - eye)
    np.testing.assert_allclose(d, f, atol=2e-7)
    np.testing.assert_array_equal(o, eye.astype(np.float32))
    # square image, far corner pixel: angle to the axis from tan(fovy/2) (1 - 1/W) sqrt(2)
    W = 64
    v = orc.make_view([0, 0, 10.0], [0, 0, 0], [0, 1, 0], 40.0, W, W, [0, -1, 0])
    o, d = orc.primary_ray(v, 0, 0)
    th = math.tan(math.radians(20.0)) * (1 - 1 / W)
    assert math.acos(-d[2]) == pytest.approx(math.atan(th * math.sqrt(2)), abs=1e-6)
    assert d[1] > 0 and d[0] < 0            # row 0 is the top, column 0 the left
    assert np.linalg.norm(d) == pytest.approx(1.0, abs=1e-7)


# ------------------------------------------------------------ density marches (readings S2, S3)
@pytest.fixture(scope="module")
def uniform_lod(orc):
    """64^3 grid where every voxel holds one straight -x -> +x segment of length 1:
    density sigma in every voxel at every level."""
    R = 64
    y, z = np.meshgrid(np.arange(R) + 0.5, np.arange(R) + 0.5, indexing="ij")
    n = R * R
    xyz = np.zeros((n, 2, 3), np.float32)
    xyz[:, 0, 0], xyz[:, 1, 0] = -0.5, R + 0.5
    xyz[:, :, 1] = y.reshape(-1, 1)
    xyz[:, :, 2] = z.reshape(-1, 1)
    vs = orc.VoxSet(xyz.reshape(-1, 3), None, np.arange(0, 2 * n + 1, 2), orc.make_grid(R, 4, scale=1.0))
    assert vs.nseg == R ** 3
    return vs, orc.Lod(vs, 3, np.full(256, 0.05, np.float32))


SIG = float(np.float32(0.05))      # sigma as stored (float32)


def test_trilinear_sample_uniform_and_outside(uniform_lod):
    vs, lod = uniform_lod
    for l in range(3):
        assert lod.sample(l, [32.3, 30.1, 33.7]) == pytest.approx(SIG, abs=1e-15)
    assert lod.sample(0, [-5.0, 10.0, 10.0]) == 0.0
    # half a cell outside the face: only the inner cell with weight 1/2
    assert lod.sample(0, [0.0, 10.5, 10.5]) == pytest.approx(SIG / 2, abs=1e-15)


def test_march_closed_form(uniform_lod):
    """Samples at s = 1, 2, 4, 8, 12, 16, 20 with steps 1, 2, 4, 4, ...: density 0.05
    gives O = 0.05 * (1 + 2 + 4 + 4 + 4) = 0.75 within a radius of 15, and the
    unbounded march stops at the first O >= 1 (after s = 20: 1.15)."""
    vs, lod = uniform_lod
    p = [32.2, 31.7, 32.9]
    assert lod.march(p, [0, 1.0, 0], 15.0) == pytest.approx(15 * SIG, abs=1e-12)
    assert lod.march(p, [0, 1.0, 0]) == pytest.approx(23 * SIG, abs=1e-12)
    # toward the +y face 2.5 voxels away (cell-centred samples, zero outside):
    # s=1 at y=62.5, level 0: one full cell -> 0.05 * 1
    # s=2 at y=63.5, level 1: 3/4 of cell 31, cell 32 outside -> 0.0375 * 2
    # s=4 at y=65.5, level 2: 1/8 of cell 15, cell 16 outside -> 0.00625 * 4
    # s=8 at y=69.5 is beyond the support (16.5 coarse cells = 66 voxels): stop
    p = [32.0, 61.5, 32.0]
    assert lod.march(p, [0, 1.0, 0], 15.0) == pytest.approx(SIG * (1 + 0.75 * 2 + 0.125 * 4), abs=1e-12)


def test_ao_directions_hemisphere(orc):
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    u = np.array([1.0, 0.2, -0.1])
    u /= np.linalg.norm(u)
    D = orc.ao_dirs(n, u, 16)
    np.testing.assert_allclose(np.linalg.norm(D, axis=1), 1.0, atol=1e-12)
    z = D @ n
    assert np.all(z > 0)
    np.testing.assert_allclose(np.sort(z)[::-1], 1 - (np.arange(16) + 0.5) / 16, atol=1e-12)
    # first direction leans toward the tube axis projected into the tangent plane
    t = u - (u @ n) * n
    assert (D[0] - z[0] * n) @ t > 0
    assert abs(D.sum(0) @ n - 8.0) < 1e-12


# ------------------------------------------------------------ images
def _tube_scene(orc, R=16, y=8.5, z=8.5):
    xyz = np.array([[-0.5, y, z], [R + 0.5, y, z]], np.float32)
    vs = orc.VoxSet(xyz, None, np.array([0, 2]), orc.make_grid(R, 32, scale=1.0))
    return vs


def test_silhouette_width_is_two_radii(orc):
    """A straight opaque tube seen from far away with a narrow field of view
    covers 2r of the image across its axis, within one pixel per edge."""
    R, r = 16, 0.2
    vs = _tube_scene(orc, R, 8.515625, 8.515625)
    W = H = 101
    dist, fov = 2000.0, 0.02                   # degrees: about 0.70 voxel across the image
    v = orc.make_view([8.0, 8.515625, 8.515625 + dist], [8.0, 8.515625, 8.515625], [0, 1, 0], fov, W, H, [0, 0, -1.0])
    tf = synth.tf_ramp()
    rd = orc.make_rdesc(r, tf, opaque=True)
    rgba, tie, _ = orc.render(vs, None, v, rd, orc.pixel_grid(0, 0, W, H))
    cov = rgba[:, 3].reshape(H, W) > 0.5
    px = 2 * dist * math.tan(math.radians(fov / 2)) / H
    for col in (10, 50, 90):
        assert abs(cov[:, col].sum() - 2 * r / px) <= 2.0
        # the tube axis sits at the bin centre the camera looks at: the image centre row
        rows = np.nonzero(cov[:, col])[0]
        assert abs(rows.mean() - (H - 1) / 2) <= 0.5
    assert cov.any(1).sum() == cov[:, 50].sum()


def test_dda_matches_brute_force(orc):
    ls = synth.make_streamlines(120, 48, seed=3)
    g = orc.make_grid(16, 32, scale=16.0, attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))
    vs = orc.VoxSet(ls.xyz, ls.attr, ls.offsets, g)
    tf = synth.tf_ramp(0.05, 0.3)
    lod = orc.Lod(vs, 3, synth.sigma_lut(tf))
    cam = synth.orbit_view((16, 16, 16), 48, 40)
    v = orc.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 48, 40, cam["light_dir"])
    pix = orc.pixel_grid(0, 0, 48, 40)
    for rd in (orc.make_rdesc(0.2, synth.tf_ramp(), opaque=True),
               orc.make_rdesc(0.3, tf, ert_alpha=0.99, shadows=True, ao=True)):
        a, ta, _ = orc.render(vs, lod, v, rd, pix)
        b, tb, _ = orc.render(vs, lod, v, rd, pix, mode="brute")
        ok = (ta == 0) & (tb == 0)
        assert ok.mean() > 0.99
        assert (a[:, 3] > 0).sum() > 100
        np.testing.assert_allclose(a[ok], b[ok], atol=1e-12)


def test_compositing_closed_forms(orc):
    ls = synth.make_streamlines(150, 48, seed=4)
    g = orc.make_grid(16, 32, scale=16.0)
    vs = orc.VoxSet(ls.xyz, None, ls.offsets, g)
    cam = synth.orbit_view((16, 16, 16), 40, 40)
    v = orc.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 40, 40, cam["light_dir"])
    pix = orc.pixel_grid(0, 0, 40, 40)
    alpha = 0.2
    tf = np.tile(np.array([[0.8, 0.4, 0.2, alpha]], np.float32), (256, 1))
    # ambient only, constant colour: rgb = c0 * A + (1 - A) * bg exactly
    rd = orc.make_rdesc(0.3, tf, ert_alpha=2.0, ka=1.0, kd=0.0, bg=(0.1, 0.2, 0.3))
    rgba, tie, cnt = orc.render(vs, None, v, rd, pix)
    A = rgba[:, 3]
    np.testing.assert_allclose(rgba[:, :3], np.outer(A, [0.8, 0.4, 0.2]) + np.outer(1 - A, [0.1, 0.2, 0.3]), atol=1e-12)
    # constant alpha, no termination: A = 1 - (1 - alpha)^k with k the hit count
    k = np.log1p(-A) / math.log1p(-alpha)
    np.testing.assert_allclose(k, np.round(k), atol=1e-9)
    assert int(np.round(k).sum()) == int(cnt[3]) and cnt[3] > 200
    # termination at tau: A >= tau wherever more hits were available, and no pixel is more opaque
    rd2 = orc.make_rdesc(0.3, tf, ert_alpha=0.6, ka=1.0, kd=0.0)
    A2 = orc.render(vs, None, v, rd2, pix)[0][:, 3]
    assert np.all(A2 <= A + 1e-15)
    more = A > A2 + 1e-12
    assert np.all(A2[more] >= 0.6 - 1e-6)
    # alpha = 1 everywhere in transparent mode equals opaque mode
    tf1 = tf.copy()
    tf1[:, 3] = 1.0
    o1 = orc.render(vs, None, v, orc.make_rdesc(0.3, tf1, ert_alpha=0.99), pix)[0]
    o2 = orc.render(vs, None, v, orc.make_rdesc(0.3, tf1, opaque=True), pix)[0]
    np.testing.assert_allclose(o1, o2, atol=1e-12)
