"""ctypes wrapper of the C oracle.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg. The product path never imports it.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class Grid(C.Structure):
    _fields_ = [("res", C.c_int32 * 3), ("bins", C.c_int32), ("origin", C.c_float * 3),
                ("scale", C.c_float), ("attr_min", C.c_float), ("attr_max", C.c_float)]


class View(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("at", C.c_float * 3), ("up", C.c_float * 3),
                ("fovy_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("light_dir", C.c_float * 3)]


class RDesc(C.Structure):
    _fields_ = [("radius", C.c_float), ("tf", C.c_float * 1024), ("opaque", C.c_int32),
                ("ert_alpha", C.c_float), ("shadows", C.c_int32), ("ao", C.c_int32),
                ("ao_rays", C.c_int32), ("ao_radius", C.c_float), ("ka", C.c_float),
                ("kd", C.c_float), ("bg", C.c_float * 3), ("ao_params", C.c_void_p), ("still", C.c_int32),
                ("ao_field", C.c_void_p), ("reps", C.c_void_p), ("shadow_level", C.c_int32)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.orc_last_error.restype = C.c_char_p
        L.orc_record_bits.argtypes = [C.c_int]
        L.orc_record_bytes.argtypes = [C.c_int]
        L.orc_fixed_point.argtypes = [vp, i64, vp, vp]
        L.orc_attr16.argtypes = [vp, i64, C.c_float, C.c_float, vp]
        L.orc_fit_grid.argtypes = [vp, i64, i32, i32, vp]
        L.orc_voxelize.argtypes = [vp, vp, vp, i64, i64, vp, C.POINTER(vp)]
        L.orc_voxset_free.argtypes = [vp]
        L.orc_voxset_nseg.argtypes = [vp]
        L.orc_voxset_nseg.restype = i64
        L.orc_voxset_nvox.argtypes = [vp]
        L.orc_voxset_nvox.restype = i64
        L.orc_voxset_export.argtypes = [vp, vp, vp, vp, vp]
        L.orc_build_lod.argtypes = [vp, C.c_int, vp, C.POINTER(vp)]
        L.orc_lod_free.argtypes = [vp]
        L.orc_lod_dims.argtypes = [vp, C.c_int, vp]
        L.orc_lod_export.argtypes = [vp, C.c_int, vp, vp, vp]
        L.orc_render.argtypes = [vp, vp, vp, vp, vp, i64, C.c_int, vp, vp, vp, vp, vp, vp, C.c_int]
        L.orc_primary_ray.argtypes = [vp, i32, i32, vp, vp]
        L.orc_capsule_entry.argtypes = [vp, vp, vp, vp, C.c_double, vp, vp]
        L.orc_march.argtypes = [vp, vp, vp, C.c_double]
        L.orc_march.restype = C.c_double
        L.orc_sample.argtypes = [vp, C.c_int, vp]
        L.orc_sample.restype = C.c_double
        L.orc_ao_dirs.argtypes = [vp, vp, C.c_int, vp]
        L.orc_reps_build.argtypes = [vp, C.c_int, C.POINTER(vp)]
        L.orc_reps_free.argtypes = [vp]
        L.orc_reps_export.argtypes = [vp, C.c_int, vp]
        L.orc_halfline_segment_distance.argtypes = [vp, vp, vp, vp]
        L.orc_halfline_segment_distance.restype = C.c_double
        L.orc_raster.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp, vp, C.c_int64, vp, vp, vp, vp, C.c_int]
        L.orc_raster.restype = C.c_int
        L.orc_shadow_reps_visibility.argtypes = [vp, vp, C.c_float, C.c_int, vp, vp]
        L.orc_shadow_reps_visibility.restype = C.c_double
        L.orc_ao_sphere_field.argtypes = [vp, C.c_int, C.c_double, vp]
        L.orc_ao_field_sample.argtypes = [vp, vp, vp]
        L.orc_ao_field_sample.restype = C.c_double
        L.orc_ao_nparams.restype = C.c_int
        L.orc_ao_ninputs.restype = C.c_int
        L.orc_bf16.argtypes = [C.c_double]
        L.orc_bf16.restype = C.c_double
        L.orc_ao_tangent.argtypes = [vp, vp, vp]
        L.orc_ao_features.argtypes = [vp, i64, vp, vp, vp, vp]
        L.orc_ao_features.restype = C.c_int
        L.orc_ao_mlp.argtypes = [vp, vp]
        L.orc_ao_mlp.restype = C.c_double
        _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"oracle error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != 0:
        raise OracleError(rc, lib().orc_last_error().decode())


def make_grid(res, bins, origin=(0.0, 0.0, 0.0), scale=1.0, attr_min=0.0, attr_max=0.0) -> Grid:
    g = Grid()
    r = (res, res, res) if np.isscalar(res) else tuple(res)
    g.res[:] = [int(x) for x in r]
    g.bins = int(bins)
    g.origin[:] = [float(x) for x in origin]
    g.scale = float(scale)
    g.attr_min = float(attr_min)
    g.attr_max = float(attr_max)
    return g


def record_bytes(bins: int) -> int:
    return lib().orc_record_bytes(bins)


def record_bits(bins: int) -> int:
    return lib().orc_record_bits(bins)


def fixed_point(xyz, grid: Grid):
    xyz = np.ascontiguousarray(xyz, np.float32)
    out = np.empty(xyz.shape, np.int32)
    _check(lib().orc_fixed_point(_p(xyz), len(xyz), C.byref(grid), _p(out)))
    return out


def attr16(attr, amin, amax):
    attr = np.ascontiguousarray(attr, np.float32)
    out = np.empty(attr.shape, np.uint16)
    _check(lib().orc_attr16(_p(attr), len(attr), amin, amax, _p(out)))
    return out


def fit_grid(xyz, rmax, bins) -> Grid:
    xyz = np.ascontiguousarray(xyz, np.float32)
    g = Grid()
    _check(lib().orc_fit_grid(_p(xyz), len(xyz), rmax, bins, C.byref(g)))
    return g


class VoxSet:
    """Oracle voxel model; fields decoded (face_in,u_in,v_in,face_out,u_out,v_out,attr,cont)."""

    def __init__(self, xyz, attr, offsets, grid: Grid):
        self.grid = grid
        xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
        attr = None if attr is None else np.ascontiguousarray(attr, np.float32)
        offsets = np.ascontiguousarray(offsets, np.int64)
        h = C.c_void_p()
        _check(lib().orc_voxelize(_p(xyz), _p(attr), _p(offsets), len(offsets) - 1, len(xyz),
                                  C.byref(grid), C.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_voxset_free(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    @property
    def nseg(self) -> int:
        return lib().orc_voxset_nseg(self._h)

    @property
    def nvox(self) -> int:
        return lib().orc_voxset_nvox(self._h)

    def export(self):
        n, v = self.nseg, self.nvox
        off = np.empty(v + 1, np.uint32)
        fields = np.empty((n, 8), np.uint8)
        curve = np.empty(n, np.uint32)
        ordn = np.empty(n, np.uint32)
        lib().orc_voxset_export(self._h, _p(off), _p(fields), _p(curve), _p(ordn))
        return dict(offset=off, fields=fields, curve=curve, ordinal=ordn)


class Lod:
    def __init__(self, vs: VoxSet, levels: int, sigma):
        self.vs = vs
        sigma = np.ascontiguousarray(sigma, np.float32)
        assert sigma.shape == (256,)
        h = C.c_void_p()
        _check(lib().orc_build_lod(vs.handle, levels, _p(sigma), C.byref(h)))
        self._h = h
        self.levels = levels

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_lod_free(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def dims(self, level):
        d = np.empty(3, np.int32)
        lib().orc_lod_dims(self._h, level, _p(d))
        return tuple(int(x) for x in d)

    def export(self, level):
        d = self.dims(level)
        n = d[0] * d[1] * d[2]
        cnt = np.empty(n, np.uint32)
        ln = np.empty(n, np.float64)
        dn = np.empty(n, np.float64)
        lib().orc_lod_export(self._h, level, _p(cnt), _p(ln), _p(dn))
        return dict(cnt=cnt, len=ln, dens=dn, dims=d)

    def sample(self, level, x):
        x = np.ascontiguousarray(x, np.float64)
        return lib().orc_sample(self._h, level, _p(x))

    def march(self, p, d, max_dist=-1.0):
        p = np.ascontiguousarray(p, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        return lib().orc_march(self._h, _p(p), _p(d), max_dist)


def make_view(eye, at, up, fovy_deg, width, height, light_dir) -> View:
    v = View()
    v.eye[:] = [float(x) for x in eye]
    v.at[:] = [float(x) for x in at]
    v.up[:] = [float(x) for x in up]
    v.fovy_deg = float(fovy_deg)
    v.width = int(width)
    v.height = int(height)
    v.light_dir[:] = [float(x) for x in light_dir]
    return v


def make_rdesc(radius, tf, opaque=False, ert_alpha=0.99, shadows=False, ao=False,
               ao_rays=16, ao_radius=15.0, ka=0.3, kd=0.7, bg=(1.0, 1.0, 1.0), ao_params=None,
               still=False, ao_field=None, reps=None, shadow_level=1) -> RDesc:
    """shadows: False/0 off, True/1 density cone march, 2 representative lines (reps, shadow_level)."""
    """ao: False/0 off, True/1 traced, 2 learned (ao_params: float32 [ao_nparams()])."""
    d = RDesc()
    d.radius = float(radius)
    tf = np.ascontiguousarray(tf, np.float32).reshape(-1)
    assert tf.size == 1024
    d.tf[:] = tf.tolist()
    d.opaque = int(bool(opaque))
    d.ert_alpha = float(ert_alpha)
    d.shadows = int(bool(shadows))
    d.ao = int(bool(ao))
    d.ao_rays = int(ao_rays)
    d.ao_radius = float(ao_radius)
    d.ka = float(ka)
    d.kd = float(kd)
    d.bg[:] = [float(x) for x in bg]
    d.still = int(bool(still))
    if reps is not None:
        d._keep_reps = reps
        d.reps = reps.handle.value
        d.shadow_level = int(shadow_level)
        d.shadows = 2
    if ao_field is not None:
        ao_field = np.ascontiguousarray(ao_field, np.float64)
        d._keep_field = ao_field
        d.ao_field = ao_field.ctypes.data
        d.ao = 3
    if ao_params is not None:
        ao_params = np.ascontiguousarray(ao_params, np.float32)
        assert ao_params.size == ao_nparams()
        d._keep = ao_params                       # keep the buffer alive with the struct
        d.ao_params = ao_params.ctypes.data
        d.ao = 2
    return d


def pixel_grid(x0, y0, w, h):
    jj, ii = np.meshgrid(np.arange(y0, y0 + h), np.arange(x0, x0 + w), indexing="ij")
    return np.stack([ii.reshape(-1), jj.reshape(-1)], 1).astype(np.int32)


# tie flag bits of render()
TIE_GRAZE, TIE_OWNER, TIE_SORT, TIE_FRAME, TIE_SLAB, TIE_SHADOW = 1, 2, 4, 16, 32, 64


def render(vs: VoxSet, lod: Lod | None, view: View, rd: RDesc, pix, mode="dda", nthreads=0,
           margins=False, flips=False, alts=False):
    """Render the listed pixels (int32 (n, 2) of (i, j)); returns rgba (n,4) f64,
    tie flags (n,) u8 and counters [voxels, records, lod samples, hits]; with
    margins=True also the per-pixel smallest normalised decision margin; with
    flips=True also the per-pixel bound on what near-tie hard-shadow
    visibilities can move a colour channel; with alts=True also, per pixel
    whose only near-tie is one pair of hits in depth order, the RGBA with
    that pair composited the other way round (NaN elsewhere), in that
    order."""
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    n = len(pix)
    rgba = np.empty((n, 4), np.float64)
    tie = np.empty(n, np.uint8)
    mg = np.empty(n, np.float64) if margins else None
    fl = np.empty(n, np.float64) if flips else None
    al = np.empty((n, 4), np.float64) if alts else None
    cnt = np.zeros(4, np.uint64)
    m = 1 if mode == "brute" else 0
    _check(lib().orc_render(vs.handle, lod.handle if lod is not None else None, C.byref(view),
                            C.byref(rd), _p(pix), n, m, _p(rgba), _p(tie), _p(mg), _p(fl), _p(al), _p(cnt),
                            int(nthreads)))
    out = (rgba, tie, cnt) + ((mg,) if margins else ()) + ((fl,) if flips else ()) + ((al,) if alts else ())
    return out


def primary_ray(view: View, i, j):
    o = np.empty(3, np.float32)
    d = np.empty(3, np.float32)
    lib().orc_primary_ray(C.byref(view), i, j, _p(o), _p(d))
    return o, d


def capsule_entry(o, d, a, b, r):
    arrs = [np.ascontiguousarray(x, np.float64) for x in (o, d, a, b)]
    t = np.zeros(1)
    dist = np.zeros(1)
    hit = lib().orc_capsule_entry(*[_p(x) for x in arrs], float(r), _p(t), _p(dist))
    return bool(hit), float(t[0]), float(dist[0])


def ao_dirs(n, u, k=16):
    n = np.ascontiguousarray(n, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    out = np.empty((k, 3))
    lib().orc_ao_dirs(_p(n), _p(u), k, _p(out))
    return out


def num_threads() -> int:
    return len(os.sched_getaffinity(0))


# ---------------------------------------------------------------- learned AO (reading L1)
def ao_nparams() -> int:
    return lib().orc_ao_nparams()


def bf16(x: float) -> float:
    return lib().orc_bf16(float(x))


def ao_tangent(a, b):
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    t = np.empty(3)
    lib().orc_ao_tangent(_p(a), _p(b), _p(t))
    return t


def ao_ninputs() -> int:
    return lib().orc_ao_ninputs()


def ao_features(lod: "Lod", voxel: int, t, n, p):
    """Model inputs of a hit in `voxel`: tangent t, unit normal n, hit point p."""
    t, n, p = (np.ascontiguousarray(a, np.float64) for a in (t, n, p))
    x = np.empty(ao_ninputs())
    if lib().orc_ao_features(lod.handle, int(voxel), _p(t), _p(n), _p(p), _p(x)) != 0:
        raise ValueError("the learned AO model needs a LoD of >= 3 levels")
    return x


def ao_mlp(params, x) -> float:
    params = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float64)
    return lib().orc_ao_mlp(_p(params), _p(x))


class _OrcLodStruct(C.Structure):
    _fields_ = [("levels", C.c_int), ("dims", (C.c_int32 * 3) * 4), ("cnt", C.c_void_p * 4),
                ("len", C.c_void_p * 4), ("dens", C.c_void_p * 4)]


class HandLod:
    """An orc_lod over given per-level density sums [z][y][x] (counts and
    lengths zero), for closed-form checks of the feature gather."""

    def __init__(self, dens_levels):
        self._keep = []
        s = _OrcLodStruct()
        s.levels = len(dens_levels)
        for l, d in enumerate(dens_levels):
            d = np.ascontiguousarray(d, np.float64)
            nz, ny, nx = d.shape
            c = np.zeros(d.shape, np.uint32)
            ln = np.zeros(d.shape)
            self._keep += [d, c, ln]
            s.dims[l][0], s.dims[l][1], s.dims[l][2] = nx, ny, nz
            s.cnt[l], s.len[l], s.dens[l] = c.ctypes.data, ln.ctypes.data, d.ctypes.data
        self._s = s

    @property
    def handle(self):
        return C.cast(C.pointer(self._s), C.c_void_p)

    def dims(self, level):
        return tuple(int(x) for x in self._s.dims[level])


# ---------------------------------------------------------------- spherical per-voxel AO (reading S4)
def ao_sphere_field(lod: "Lod", rays=100, radius=5.0):
    d = lod.dims(0)
    out = np.empty(int(d[0]) * int(d[1]) * int(d[2]), np.float64)
    lib().orc_ao_sphere_field(lod.handle, int(rays), float(radius), _p(out))
    return out


def ao_field_sample(field, dims, x):
    field = np.ascontiguousarray(field, np.float64)
    dm = np.ascontiguousarray(dims, np.int32)
    x = np.ascontiguousarray(x, np.float64)
    return lib().orc_ao_field_sample(_p(field), _p(dm), _p(x))


# ---------------------------------------------------------------- representative lines (reading R3)
class Reps:
    """Representative lines of every level of a voxel set."""

    def __init__(self, vs: "VoxSet", levels: int):
        h = C.c_void_p()
        _check(lib().orc_reps_build(vs.handle, int(levels), C.byref(h)))
        self.handle, self.vs, self.levels = h, vs, levels

    def export(self, level):
        """uint8 [cells][7]: valid, face_a, u_a, v_a, face_b, u_b, v_b."""
        dims = [int(x) for x in vs_dims(self.vs)]
        for _ in range(level):
            dims = [(d + 1) // 2 for d in dims]
        out = np.empty((dims[0] * dims[1] * dims[2], 7), np.uint8)
        lib().orc_reps_export(self.handle, int(level), _p(out))
        return out

    def __del__(self):
        if getattr(self, "handle", None):
            lib().orc_reps_free(self.handle)
            self.handle = None


def vs_dims(vs: "VoxSet"):
    return tuple(vs.grid.res)


def halfline_segment_distance(o, d, a, b) -> float:
    o, d, a, b = (np.ascontiguousarray(x, np.float64) for x in (o, d, a, b))
    return lib().orc_halfline_segment_distance(_p(o), _p(d), _p(a), _p(b))


def shadow_reps_visibility(vs: "VoxSet", reps: Reps, radius, level, P, Lt) -> float:
    P = np.ascontiguousarray(P, np.float64)
    Lt = np.ascontiguousarray(Lt, np.float64)
    return lib().orc_shadow_reps_visibility(vs.handle, reps.handle, float(radius), int(level), _p(P), _p(Lt))


def raster(xyz, attr, offsets, grid: "Grid", view: "View", rd: "RDesc", pix, nthreads=0, alts=False):
    """Reading K1 (rasterised comparison system) for the listed pixels: rgba
    (n, 4) f64, tie flags (n,) u8, counters [fragments, blended]; with
    alts=True also the RGBA of each pixel whose only near-tie is one pair of
    fragments in depth order, blended the other way round (NaN elsewhere)."""
    xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    attr = None if attr is None else np.ascontiguousarray(attr, np.float32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    n = len(pix)
    rgba = np.empty((n, 4), np.float64)
    tie = np.empty(n, np.uint8)
    cnt = np.zeros(2, np.uint64)
    al = np.empty((n, 4), np.float64) if alts else None
    _check(lib().orc_raster(_p(xyz), _p(attr), _p(offsets), len(offsets) - 1, C.byref(grid), C.byref(view),
                            C.byref(rd), _p(pix), n, _p(rgba), _p(tie), _p(al), _p(cnt), int(nthreads)))
    return (rgba, tie, cnt) + ((al,) if alts else ())
