"""Pins of the oracle's camera-at-rest mode (reading R2, Sec. 4.1).

When the camera stands still, a ray also tests the segments stored in the 26
voxels around each voxel it visits (a hit still belongs to the voxel holding
its entry point), and among one voxel's hits only the first of each local
line id (curve index mod 32) is blended. Pinned by brute force over all
capsules (exact for tube radii <= 0.5 voxel), a hand-built overhang that the
interactive mode misses, and closed forms of the line-id rule.
"""
import numpy as np
import pytest

from paper_1801_01155_gb300 import synth


@pytest.mark.parametrize("radius", [0.2, 0.45])
def test_still_dda_matches_brute_force_over_all_capsules(orc, radius):
    ls = synth.make_streamlines(120, 48, seed=3)
    g = orc.make_grid(16, 32, scale=16.0, attr_min=float(ls.attr.min()), attr_max=float(ls.attr.max()))
    vs = orc.VoxSet(ls.xyz, ls.attr, ls.offsets, g)
    tf = synth.tf_ramp(0.05, 0.3)
    lod = orc.Lod(vs, 3, synth.sigma_lut(tf))
    cam = synth.orbit_view((16, 16, 16), 48, 40)
    v = orc.make_view(cam["eye"], cam["at"], cam["up"], cam["fovy_deg"], 48, 40, cam["light_dir"])
    pix = orc.pixel_grid(0, 0, 48, 40)
    for rd in (orc.make_rdesc(radius, synth.tf_ramp(), opaque=True, still=True),
               orc.make_rdesc(radius, tf, ert_alpha=0.99, shadows=True, still=True)):
        a, ta, _ = orc.render(vs, lod, v, rd, pix)
        b, tb, _ = orc.render(vs, lod, v, rd, pix, mode="brute")
        ok = (ta == 0) & (tb == 0)
        assert ok.mean() > 0.97
        np.testing.assert_allclose(a[ok], b[ok], atol=1e-12)
    # the interactive mode differs somewhere (overhangs), the still mode never loses coverage
    rd0 = orc.make_rdesc(radius, synth.tf_ramp(), opaque=True)
    c, tc, _ = orc.render(vs, lod, v, rd0, pix)
    s, ts, _ = orc.render(vs, lod, v, orc.make_rdesc(radius, synth.tf_ramp(), opaque=True, still=True), pix)
    ok = (tc == 0) & (ts == 0)
    assert np.all(s[ok, 3] >= c[ok, 3])
    assert (s[ok, 3] > c[ok, 3]).sum() > 0


def _one_ray(orc, eye, at):
    return orc.make_view(eye, at, (0.0, 1.0, 0.0), 10.0, 1, 1, (0.0, -1.0, 0.0))


def test_overhang_found_only_with_the_camera_at_rest(orc):
    """A straight line along x at y = 1.9, z = 2.5 (stored in voxels of row
    y = 1) is quantised to y = 1 + 28.5/32, z = 2 + 16.5/32. A ray along +z
    at x = 1.5, y = 2.1 passes 0.209 from the axis, inside radius 0.3, and
    enters the tube at z = 2 + 16.5/32 - sqrt(0.09 - 0.209375^2) = 2.3008,
    in voxel (1, 2, 2): no voxel on that ray stores the line."""
    xyz = np.array([[0.2, 1.9, 2.5], [3.8, 1.9, 2.5]], np.float32)
    vs = orc.VoxSet(xyz, None, np.array([0, 2]), orc.make_grid(4, 32, scale=1.0))
    v = _one_ray(orc, (1.5, 2.1, -20.0), (1.5, 2.1, 20.0))
    tf = synth.tf_ramp()
    pix = np.array([[0, 0]], np.int32)
    a, ta, _ = orc.render(vs, None, v, orc.make_rdesc(0.3, tf, opaque=True, ka=1.0, kd=0.0), pix)
    b, tb, _ = orc.render(vs, None, v, orc.make_rdesc(0.3, tf, opaque=True, ka=1.0, kd=0.0, still=True), pix)
    assert ta[0] == 0 and tb[0] == 0
    assert a[0, 3] == 0.0 and b[0, 3] == 1.0
    # ambient-only shading of attribute byte 0: the colour is the TF's
    np.testing.assert_allclose(b[0, :3], tf[0, :3], atol=1e-6)
    # the entry point of the closed form lies in voxel (1, 2, 2), not in row y = 1
    zq, yq = 2 + 16.5 / 32, 1 + 28.5 / 32
    z_entry = zq - np.sqrt(0.09 - (2.1 - yq) ** 2)
    assert 2.0 < z_entry < 3.0 and int(np.floor(2.1)) == 2


def test_line_id_rule_closed_forms(orc):
    """Two curves with identical geometry hit at the same depth. Curves 0 and
    32 share local id 0: at rest one hit is blended, A = alpha. Curves 0 and
    1 have different ids: both are, A = 1 - (1 - alpha)^2. The interactive
    mode blends both in either case."""
    line = np.array([[0.5, 1.5, 1.5], [3.5, 1.5, 1.5]], np.float32)
    filler = np.array([[0.3, 0.3, 3.6], [0.31, 0.3, 3.6]], np.float32)   # a curve far from the ray
    alpha = float(np.float32(0.25))
    tf = np.tile(np.array([1.0, 1.0, 1.0, alpha], np.float32), (256, 1))
    v = _one_ray(orc, (1.7, 1.5, -20.0), (1.7, 1.5, 20.0))
    pix = np.array([[0, 0]], np.int32)
    for second in (1, 32):
        curves = [line] + [filler] * (second - 1) + [line]
        xyz = np.concatenate(curves)
        offs = np.arange(0, 2 * len(curves) + 1, 2)
        vs = orc.VoxSet(xyz, None, offs, orc.make_grid(4, 32, scale=1.0))
        a, ta, _ = orc.render(vs, None, v, orc.make_rdesc(0.3, tf, ert_alpha=2.0), pix)
        b, tb, _ = orc.render(vs, None, v, orc.make_rdesc(0.3, tf, ert_alpha=2.0, still=True), pix)
        assert a[0, 3] == pytest.approx(1 - (1 - alpha) ** 2, abs=1e-12)
        want = alpha if second == 32 else 1 - (1 - alpha) ** 2
        assert b[0, 3] == pytest.approx(want, abs=1e-12)


# ---------------------------------------------------------------- spherical per-voxel AO (reading S4)
def _level0(orc, dens):
    """A one-level hand LoD over level-0 density sums [z][y][x]."""
    return orc.HandLod([dens])


def test_sphere_ao_field_linear_density_closed_form(orc):
    """Density linear in z, rho = alpha (k + 1/2) in voxel layer k: trilinear
    samples reproduce it, so a ray from a centre at height zc collects
    O = sum_{s=1..5} alpha (zc + s d_z) = alpha (5 zc + 15 d_z). The
    Fibonacci z values 1 - (2i+1)/K average to zero, so far from the grid's
    faces (and with every O below 1) AO = 1 - 5 alpha zc."""
    R = 24
    alpha = 0.004
    z = (np.arange(R) + 0.5)[:, None, None] * np.ones((1, R, R))
    lod = _level0(orc, alpha * z)
    f = orc.ao_sphere_field(lod, rays=100, radius=5.0).reshape(R, R, R)
    for k in (6, 9, 12, 17):
        zc = k + 0.5
        assert f[k, 10, 11] == pytest.approx(1.0 - 5 * alpha * zc, abs=1e-12)
        assert f[k, 7, 16] == pytest.approx(1.0 - 5 * alpha * zc, abs=1e-12)


def test_sphere_ao_field_saturates_and_empty_is_one(orc):
    """Uniform density 0.3: O = 0.3, 0.6, 0.9, 1.2 after four unit steps, so
    every interior ray saturates and AO = 0; an empty grid gives AO = 1."""
    R = 20
    lod = _level0(orc, np.full((R, R, R), 0.3))
    f = orc.ao_sphere_field(lod, rays=64, radius=5.0).reshape(R, R, R)
    assert f[10, 10, 10] == pytest.approx(0.0, abs=1e-12)
    lod0 = _level0(orc, np.zeros((R, R, R)))
    assert np.all(orc.ao_sphere_field(lod0, rays=64, radius=5.0) == 1.0)


def test_ao_field_sample_linear_and_clamped(orc):
    """Trilinear interpolation reproduces a linear field between voxel
    centres; beyond the outer centres the edge values hold."""
    dims = (7, 5, 6)
    zz, yy, xx = np.meshgrid(np.arange(6) + 0.5, np.arange(5) + 0.5, np.arange(7) + 0.5, indexing="ij")
    field = (0.1 * xx - 0.2 * yy + 0.05 * zz + 1.0).reshape(-1)
    lin = lambda x, y, z: 0.1 * x - 0.2 * y + 0.05 * z + 1.0
    for p in ([1.3, 2.2, 3.9], [0.5, 0.5, 0.5], [6.4, 4.1, 5.5], [3.0, 1.75, 2.25]):
        assert orc.ao_field_sample(field, dims, p) == pytest.approx(lin(*p), abs=1e-12)
    assert orc.ao_field_sample(field, dims, [0.1, 2.5, 2.5]) == pytest.approx(lin(0.5, 2.5, 2.5), abs=1e-12)
    assert orc.ao_field_sample(field, dims, [8.0, 6.0, -1.0]) == pytest.approx(lin(6.5, 4.5, 0.5), abs=1e-12)


def test_sphere_ao_field_single_ray_steps(orc):
    """One ray: z_0 = 0, phi_0 = 0, so it points along +x. With density
    alpha (i + 1/2) in voxel column i it collects alpha (5 xc + 1+2+3+4+5):
    the samples sit at unit steps 1..5 from the centre."""
    R = 24
    alpha = 0.003
    x = np.ones((R, R, 1)) * (np.arange(R) + 0.5)[None, None, :]
    f = orc.ao_sphere_field(_level0(orc, alpha * x), rays=1, radius=5.0).reshape(R, R, R)
    for i in (3, 8, 15):
        assert f[9, 11, i] == pytest.approx(1.0 - alpha * (5 * (i + 0.5) + 15), abs=1e-12)
