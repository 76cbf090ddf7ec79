"""ctypes binding of liblvr.so (C ABI in include/lvr.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. The functions carry the C names (``lvr_voxelize``,
``lvr_build_lod``, ``lvr_render``, ...). Array arguments may be torch
tensors (CUDA or CPU) or numpy arrays; the library stages host memory
itself. Handles are wrapped so that they are freed with their Python
object. If the library has not been built this module raises on import:
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblvr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`")

_L = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, EOVERFLOW, ETIMEOUT, EDEVICE = range(7)
_NAMES = {0: "LVR_OK", 1: "LVR_EINVAL", 2: "LVR_ENOMEM", 3: "LVR_ECUDA", 4: "LVR_EOVERFLOW",
          5: "LVR_ETIMEOUT", 6: "LVR_EDEVICE"}


class LVRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("res", C.c_int32 * 3), ("bins", C.c_int32), ("fit", C.c_int32),
                ("origin", C.c_float * 3), ("scale", C.c_float),
                ("attr_min", C.c_float), ("attr_max", C.c_float)]


class LineSetInfo(C.Structure):
    _fields_ = [("res", C.c_int32 * 3), ("bins", C.c_int32), ("origin", C.c_float * 3),
                ("scale", C.c_float), ("n_voxels", C.c_int64), ("n_segments", C.c_int64),
                ("bytes", C.c_int64)]


class LodInfo(C.Structure):
    _fields_ = [("levels", C.c_int32), ("dims", (C.c_int32 * 3) * 4)]


class View(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("at", C.c_float * 3), ("up", C.c_float * 3),
                ("fovy_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("crop", C.c_int32 * 4), ("light_dir", C.c_float * 3)]


class RenderDesc(C.Structure):
    _fields_ = [("radius", C.c_float), ("tf_rgba", C.c_float * 1024), ("opaque", C.c_int32),
                ("ert_alpha", C.c_float), ("shadows", C.c_int32), ("ao_mode", C.c_int32),
                ("ao_rays", C.c_int32), ("ao_radius", C.c_float), ("ka", C.c_float),
                ("kd", C.c_float), ("bg", C.c_float * 3), ("tile_w", C.c_int32),
                ("tile_h", C.c_int32), ("layout", C.c_int32), ("still", C.c_int32),
                ("shadow_level", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("ls", C.c_void_p), ("lod", C.c_void_p), ("view", View), ("desc", C.POINTER(RenderDesc)),
                ("ao", C.c_void_p), ("rgba", C.c_void_p)]


class RasterStats(C.Structure):
    _fields_ = [("fragments", C.c_uint64), ("max_per_pixel", C.c_uint64), ("list_bytes", C.c_uint64)]


class Tune(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("layout", C.c_int32), ("ms", C.c_float * 8)]


LAYOUT_AOS8, LAYOUT_AOS16 = 0, 1


class AoTrainDesc(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("epochs", C.c_int32), ("batch", C.c_int32),
                ("lr", C.c_float), ("seed", C.c_uint64), ("view_size", C.c_int32),
                ("depth", C.c_int32), ("render", C.POINTER(RenderDesc))]


class AoError(C.Structure):
    _fields_ = [("hits", C.c_uint64), ("mean_abs", C.c_double), ("p99_abs", C.c_double),
                ("max_abs", C.c_double), ("mean_traced", C.c_double), ("mean_learned", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp, _i64, _i32 = C.c_void_p, C.c_int64, C.c_int32
_SIGS = {
    "lvr_version": ([], C.c_int),
    "lvr_create": ([C.c_int, _vp, C.POINTER(_vp)], C.c_int),
    "lvr_destroy": ([_vp], None),
    "lvr_last_error": ([_vp], C.c_char_p),
    "lvr_sync": ([_vp], C.c_int),
    "lvr_voxelize": ([_vp, _vp, _vp, _vp, _i64, _i64, C.POINTER(GridDesc), C.POINTER(_vp)], C.c_int),
    "lvr_lineset_info_get": ([_vp, C.POINTER(LineSetInfo)], C.c_int),
    "lvr_export_lineset": ([_vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "lvr_free_lineset": ([_vp], None),
    "lvr_build_lod": ([_vp, _vp, C.c_int, _vp, C.POINTER(_vp)], C.c_int),
    "lvr_lod_info_get": ([_vp, C.POINTER(LodInfo)], C.c_int),
    "lvr_export_lod": ([_vp, _vp, C.c_int, _vp, _vp, _vp], C.c_int),
    "lvr_free_lod": ([_vp], None),
    "lvr_render": ([_vp, _vp, _vp, C.POINTER(View), C.POINTER(RenderDesc), _vp, _vp, _vp], C.c_int),
    "lvr_voxelize_static": ([_vp, _vp, _vp, _i64, _i64, C.POINTER(GridDesc), _vp, _vp, _vp, _i64,
                             C.POINTER(_i64), _vp], C.c_int),
    "lvr_lineset_layout": ([_vp, _vp, C.c_int], C.c_int),
    "lvr_lineset_neighbours": ([_vp, _vp, C.c_float], C.c_int),
    "lvr_lod_ao_field": ([_vp, _vp, C.c_int, C.c_float], C.c_int),
    "lvr_export_ao_field": ([_vp, _vp, _vp], C.c_int),
    "lvr_lod_rep_lines": ([_vp, _vp, _vp], C.c_int),
    "lvr_raster": ([_vp, _vp, _vp, _vp, _i64, _i64, C.POINTER(GridDesc), C.POINTER(View), C.POINTER(RenderDesc),
                    _vp, C.POINTER(RasterStats)], C.c_int),
    "lvr_export_rep_lines": ([_vp, _vp, C.c_int, _vp], C.c_int),
    "lvr_batch_create": ([_vp, C.POINTER(BatchItem), C.c_int, C.POINTER(_vp)], C.c_int),
    "lvr_batch_render": ([_vp, _vp], C.c_int),
    "lvr_batch_size": ([_vp, C.POINTER(_i64), C.POINTER(_i64)], C.c_int),
    "lvr_free_batch": ([_vp], None),
    "lvr_autotune": ([_vp, C.POINTER(BatchItem), C.c_int, C.c_int, C.POINTER(Tune)], C.c_int),
    "lvr_ao_nparams": ([], C.c_int),
    "lvr_ao_model_create": ([_vp, _vp, C.POINTER(_vp)], C.c_int),
    "lvr_ao_model_params": ([_vp, _vp, _vp], C.c_int),
    "lvr_free_ao_model": ([_vp], None),
    "lvr_ao_infer": ([_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "lvr_ao_features": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "lvr_ao_samples": ([_vp, _vp, _vp, C.POINTER(View), C.POINTER(RenderDesc), _i32, C.c_uint32, _vp, _vp,
                        _vp, _vp, _vp], C.c_int),
    "lvr_ao_judge": ([_vp, _vp, _vp, C.POINTER(View), C.POINTER(RenderDesc), _vp, _vp, C.POINTER(AoError)],
                     C.c_int),
    "lvr_ao_train_step": ([_vp, _vp, _i64, _vp, _vp, C.c_float, C.POINTER(C.c_float), _vp], C.c_int),
    "lvr_train_ao": ([_vp, _vp, _vp, C.c_int, C.POINTER(AoTrainDesc), C.POINTER(_vp),
                      C.POINTER(C.c_float)], C.c_int),
    "lvr_import_lineset": ([_vp, C.POINTER(LineSetInfo), _vp, _vp, _vp, _vp, C.POINTER(_vp)], C.c_int),
    "lvr_import_lod": ([_vp, C.c_int, _vp, _vp, _vp, _vp, C.POINTER(_vp)], C.c_int),
    "lvr_ao_model_state": ([_vp, _vp, _vp, _vp, _vp, C.POINTER(_i64)], C.c_int),
    "lvr_ao_model_set_state": ([_vp, _vp, _vp, _vp, _vp, _i64], C.c_int),
    "lvr_test_fail_allocation": ([_i64], None),
    "lvr_test_live_allocations": ([], _i64),
}
STATIC_MAX_VOXELS = 2097152
for _n, (_a, _r) in _SIGS.items():
    _f = getattr(_L, _n)
    _f.argtypes = _a
    _f.restype = _r

ABI_SYMBOLS = tuple(_SIGS)


def _ptr(x):
    """Raw address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("arrays passed to lvr must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to lvr must be contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _check(ctx, rc):
    if rc != OK:
        msg = _L.lvr_last_error(ctx).decode() if ctx else ""
        raise LVRError(rc, msg)


# ---------------------------------------------------------------- handles
class Context:
    """lvr_ctx on a CUDA device; ``stream`` is a torch.cuda.Stream or raw handle."""

    def __init__(self, device: int = 0, stream=None):
        h = _vp()
        raw = None
        if stream is not None:
            raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = _L.lvr_create(int(device), raw, C.byref(h))
        if rc != OK:
            raise LVRError(rc, "lvr_create failed")
        self.handle = h
        self.device = device
        self.stream = stream

    def close(self):
        if getattr(self, "handle", None):
            _L.lvr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def sync(self):
        _check(self.handle, _L.lvr_sync(self.handle))


class LineSet:
    def __init__(self, ctx: Context, h):
        self.ctx, self.handle = ctx, h

    def info(self) -> LineSetInfo:
        inf = LineSetInfo()
        _check(self.ctx.handle, _L.lvr_lineset_info_get(self.handle, C.byref(inf)))
        return inf

    def free(self):
        if getattr(self, "handle", None):
            _L.lvr_free_lineset(self.handle)
            self.handle = None

    def __del__(self):
        if getattr(self, "ctx", None) is not None and self.ctx.handle:
            self.free()


class Lod:
    def __init__(self, ctx: Context, h):
        self.ctx, self.handle = ctx, h

    def info(self) -> LodInfo:
        inf = LodInfo()
        _check(self.ctx.handle, _L.lvr_lod_info_get(self.handle, C.byref(inf)))
        return inf

    def free(self):
        if getattr(self, "handle", None):
            _L.lvr_free_lod(self.handle)
            self.handle = None

    def __del__(self):
        if getattr(self, "ctx", None) is not None and self.ctx.handle:
            self.free()


class AoModel:
    """lvr_ao_model: learned AO surrogate parameters on the device."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.handle = ctx, h

    def params(self) -> np.ndarray:
        out = np.empty(lvr_ao_nparams(), np.float32)
        _check(self.ctx.handle, _L.lvr_ao_model_params(self.ctx.handle, self.handle, _ptr(out)))
        return out

    def free(self):
        if getattr(self, "handle", None):
            _L.lvr_free_ao_model(self.handle)
            self.handle = None

    def __del__(self):
        if getattr(self, "ctx", None) is not None and self.ctx.handle:
            self.free()


# ---------------------------------------------------------------- C-named calls
def lvr_version() -> int:
    return _L.lvr_version()


def lvr_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def lvr_sync(ctx: Context):
    ctx.sync()


def grid_desc(res, bins, origin=(0.0, 0.0, 0.0), scale=1.0, attr_min=0.0, attr_max=0.0,
              fit=False) -> GridDesc:
    g = GridDesc()
    r = (res, res, res) if np.isscalar(res) else tuple(res)
    g.res[:] = [int(x) for x in r]
    g.bins = int(bins)
    g.fit = int(bool(fit))
    g.origin[:] = [float(x) for x in origin]
    g.scale = float(scale)
    g.attr_min = float(attr_min)
    g.attr_max = float(attr_max)
    return g


def lvr_voxelize(ctx: Context, xyz, attr, curve_offsets, grid: GridDesc) -> LineSet:
    """xyz float32 (nv,3), attr float32 (nv,) or None, curve_offsets int64 (nc+1,)."""
    nv = int(xyz.shape[0]) if xyz is not None else 0
    nc = int(curve_offsets.shape[0]) - 1
    h = _vp()
    _check(ctx.handle, _L.lvr_voxelize(ctx.handle, _ptr(xyz), _ptr(attr), _ptr(curve_offsets), nc, nv,
                                       C.byref(grid), C.byref(h)))
    return LineSet(ctx, h)


def lvr_export_lineset(ctx: Context, ls: LineSet, offset=None, fields=None, curve=None, ordinal=None):
    _check(ctx.handle, _L.lvr_export_lineset(ctx.handle, ls.handle, _ptr(offset), _ptr(fields),
                                             _ptr(curve), _ptr(ordinal)))


def export_lineset_numpy(ctx: Context, ls: LineSet) -> dict:
    inf = ls.info()
    off = np.empty(inf.n_voxels + 1, np.uint32)
    fields = np.empty((inf.n_segments, 8), np.uint8)
    curve = np.empty(inf.n_segments, np.uint32)
    ordn = np.empty(inf.n_segments, np.uint32)
    lvr_export_lineset(ctx, ls, off, fields, curve, ordn)
    return dict(offset=off, fields=fields, curve=curve, ordinal=ordn)


def lvr_import_lineset(ctx: Context, res, bins, origin, scale, offset, fields, curve, ordinal) -> LineSet:
    """A line set from the arrays lvr_export_lineset writes (host or device)."""
    inf = LineSetInfo()
    r = (res, res, res) if np.isscalar(res) else tuple(res)
    inf.res[:] = [int(x) for x in r]
    inf.bins = int(bins)
    inf.origin[:] = [float(x) for x in origin]
    inf.scale = float(scale)
    inf.n_voxels = int(r[0]) * int(r[1]) * int(r[2])
    inf.n_segments = int(len(curve)) if curve is not None else 0
    h = _vp()
    _check(ctx.handle, _L.lvr_import_lineset(ctx.handle, C.byref(inf), _ptr(offset), _ptr(fields), _ptr(curve),
                                            _ptr(ordinal), C.byref(h)))
    return LineSet(ctx, h)


def lvr_free_lineset(ls: LineSet):
    ls.free()


def lvr_build_lod(ctx: Context, ls: LineSet, levels: int, sigma256) -> Lod:
    sigma256 = np.ascontiguousarray(np.asarray(sigma256, np.float32))
    assert sigma256.shape == (256,)
    h = _vp()
    _check(ctx.handle, _L.lvr_build_lod(ctx.handle, ls.handle, int(levels), _ptr(sigma256), C.byref(h)))
    return Lod(ctx, h)


def lvr_export_lod(ctx: Context, lod: Lod, level: int, cnt=None, len_=None, dens=None):
    _check(ctx.handle, _L.lvr_export_lod(ctx.handle, lod.handle, int(level), _ptr(cnt), _ptr(len_), _ptr(dens)))


def export_lod_numpy(ctx: Context, lod: Lod, level: int) -> dict:
    d = tuple(lod.info().dims[level])
    n = d[0] * d[1] * d[2]
    cnt = np.empty(n, np.uint32)
    ln = np.empty(n, np.float32)
    dn = np.empty(n, np.float32)
    lvr_export_lod(ctx, lod, level, cnt, ln, dn)
    return dict(cnt=cnt, len=ln, dens=dn, dims=d)


def lvr_import_lod(ctx: Context, dims0, cnt, len_, dens) -> Lod:
    """A LoD from per-level arrays (lists of host or device arrays, level 0 first)."""
    levels = len(cnt)
    d = (C.c_int32 * 3)(*[int(x) for x in dims0])
    arr = lambda xs: (_vp * levels)(*[_ptr(x) for x in xs])   # noqa: E731
    h = _vp()
    _check(ctx.handle, _L.lvr_import_lod(ctx.handle, levels, d, arr(cnt), arr(len_), arr(dens), C.byref(h)))
    return Lod(ctx, h)


def lvr_free_lod(lod: Lod):
    lod.free()


def make_view(eye, at, up, fovy_deg, width, height, light_dir, crop=None) -> View:
    v = View()
    v.eye[:] = [float(x) for x in eye]
    v.at[:] = [float(x) for x in at]
    v.up[:] = [float(x) for x in up]
    v.fovy_deg = float(fovy_deg)
    v.width = int(width)
    v.height = int(height)
    v.crop[:] = [int(x) for x in (crop or (0, 0, 0, 0))]
    v.light_dir[:] = [float(x) for x in light_dir]
    return v


def make_desc(radius, tf, opaque=False, ert_alpha=0.99, shadows=False, ao_mode=0, ao_rays=16,
              ao_radius=15.0, ka=0.3, kd=0.7, bg=(1.0, 1.0, 1.0), tile=(0, 0), layout=0,
              still=False, shadow_level=None) -> RenderDesc:
    """shadows: False/0 off, True/1 soft (density LoD); shadow_level given: 2, hard
    shadows against that LoD level's representative lines (lvr_lod_rep_lines)."""
    d = RenderDesc()
    d.radius = float(radius)
    tf = np.ascontiguousarray(np.asarray(tf, np.float32)).reshape(-1)
    assert tf.size == 1024
    C.memmove(d.tf_rgba, tf.ctypes.data, 4096)
    d.opaque = int(bool(opaque))
    d.ert_alpha = float(ert_alpha)
    d.shadows = int(bool(shadows))
    d.ao_mode = int(ao_mode)
    d.ao_rays = int(ao_rays)
    d.ao_radius = float(ao_radius)
    d.ka = float(ka)
    d.kd = float(kd)
    d.bg[:] = [float(x) for x in bg]
    d.tile_w, d.tile_h = int(tile[0]), int(tile[1])
    d.layout = int(layout)
    d.still = int(bool(still))
    if shadow_level is not None:
        d.shadows = 2
        d.shadow_level = int(shadow_level)
    return d


def lvr_render(ctx: Context, ls: LineSet, lod: Lod | None, view: View, desc: RenderDesc, rgba,
               ao_model=None, counters=None):
    """rgba: float32 (h, w, 4) for the crop (torch CUDA tensor or host array)."""
    _check(ctx.handle, _L.lvr_render(ctx.handle, ls.handle, lod.handle if lod is not None else None,
                                     C.byref(view), C.byref(desc),
                                     ao_model.handle if ao_model is not None else None,
                                     _ptr(rgba), _ptr(counters)))
    return rgba


def lvr_voxelize_static(xyz, attr, curve_offsets, grid: GridDesc, offset, records, keys, stream=None) -> int:
    """Allocation-free voxelisation into caller-owned device tensors.

    For callers that cannot allocate device memory: the library's scratch is
    a static device array (grids up to STATIC_MAX_VOXELS voxels). offset:
    uint32-sized [voxels + 1]; records / keys: 64-bit [capacity]. Returns the
    segment count; raises LVRError(LVR_EOVERFLOW) with .n_segments set when
    the capacity is too small. Calls that overlap on the GPU race.
    """
    nv = int(xyz.shape[0]) if xyz is not None else 0
    nc = int(curve_offsets.shape[0]) - 1
    cap = int(records.shape[0]) if records is not None else 0
    n = _i64(0)
    raw = None
    if stream is not None:
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    dev = getattr(curve_offsets, "device", None)
    if dev is not None and getattr(dev, "type", None) == "cuda":
        import torch   # the call runs on the current device: make it the buffers' device
        with torch.cuda.device(dev):
            rc = _L.lvr_voxelize_static(_ptr(xyz), _ptr(attr), _ptr(curve_offsets), nc, nv, C.byref(grid),
                                        _ptr(offset), _ptr(records), _ptr(keys), cap, C.byref(n), raw)
    else:
        rc = _L.lvr_voxelize_static(_ptr(xyz), _ptr(attr), _ptr(curve_offsets), nc, nv, C.byref(grid),
                                    _ptr(offset), _ptr(records), _ptr(keys), cap, C.byref(n), raw)
    if rc != OK:
        err = LVRError(rc, "lvr_voxelize_static failed")
        err.n_segments = n.value
        raise err
    return n.value


# ---------------------------------------------------------------- learned AO
def lvr_ao_nparams() -> int:
    return int(_L.lvr_ao_nparams())


def lvr_ao_model_create(ctx: Context, params) -> AoModel:
    """params: host float32 [lvr_ao_nparams()]."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.shape != (lvr_ao_nparams(),):
        raise ValueError("params must have lvr_ao_nparams() entries")
    h = _vp()
    _check(ctx.handle, _L.lvr_ao_model_create(ctx.handle, _ptr(p), C.byref(h)))
    return AoModel(ctx, h)


def lvr_ao_model_state(ctx: Context, m: AoModel):
    """Training checkpoint: (params, adam_m, adam_v, step), float32 host arrays."""
    n = lvr_ao_nparams()
    p, mm, vv = (np.empty(n, np.float32) for _ in range(3))
    step = _i64(0)
    _check(ctx.handle, _L.lvr_ao_model_state(ctx.handle, m.handle, _ptr(p), _ptr(mm), _ptr(vv), C.byref(step)))
    return p, mm, vv, step.value


def lvr_ao_model_set_state(ctx: Context, m: AoModel, params, adam_m, adam_v, step: int):
    args = [np.ascontiguousarray(x, np.float32) if isinstance(x, np.ndarray) else x for x in (params, adam_m, adam_v)]
    _check(ctx.handle, _L.lvr_ao_model_set_state(ctx.handle, m.handle, *[_ptr(x) for x in args], int(step)))


def lvr_test_fail_allocation(n: int):
    _L.lvr_test_fail_allocation(int(n))


def lvr_test_live_allocations() -> int:
    return int(_L.lvr_test_live_allocations())


def lvr_free_ao_model(m: AoModel):
    m.free()


AO_NINPUTS = 400


def lvr_ao_infer(ctx: Context, m: AoModel, lod: Lod, voxel, dir_, pos, normal, ao):
    """voxel int32 [n], dir / pos / normal float32 [n, 3], ao float32 [n] (host or device)."""
    n = int(voxel.shape[0])
    _check(ctx.handle, _L.lvr_ao_infer(ctx.handle, m.handle, lod.handle, n, _ptr(voxel), _ptr(dir_), _ptr(pos),
                                       _ptr(normal), _ptr(ao)))
    return ao


def lvr_ao_features(ctx: Context, lod: Lod, voxel, dir_, pos, normal, X):
    """X: device int16/uint16-sized [n, AO_NINPUTS] receiving bfloat16 bit patterns."""
    n = int(voxel.shape[0])
    _check(ctx.handle, _L.lvr_ao_features(ctx.handle, lod.handle, n, _ptr(voxel), _ptr(dir_), _ptr(pos),
                                          _ptr(normal), _ptr(X)))
    return X


def lvr_ao_samples(ctx: Context, ls: LineSet, lod: Lod, view: View, desc: RenderDesc, depth: int, seed: int,
                   voxel, dir_, ao, pos=None, normal=None):
    """Device voxel int32 [h*w], dir float32 [h*w, 3], ao float32 [h*w] (and optional
    pos, normal float32 [h*w, 3]): per pixel the hit of index hash(seed, pixel) mod
    depth with its traced AO (voxel -1: none)."""
    _check(ctx.handle, _L.lvr_ao_samples(ctx.handle, ls.handle, lod.handle, C.byref(view), C.byref(desc),
                                         int(depth), int(seed) & 0xFFFFFFFF, _ptr(voxel), _ptr(dir_), _ptr(ao),
                                         _ptr(pos), _ptr(normal)))


def lvr_ao_judge(ctx: Context, ls: LineSet, lod: Lod, view: View, desc: RenderDesc, m: AoModel,
                 rgba=None) -> dict:
    """Learned vs traced AO over every composited hit of the view (see include/lvr.h)."""
    err = AoError()
    _check(ctx.handle, _L.lvr_ao_judge(ctx.handle, ls.handle, lod.handle, C.byref(view), C.byref(desc),
                                       m.handle, _ptr(rgba), C.byref(err)))
    return err.as_dict()


def lvr_ao_train_step(ctx: Context, m: AoModel, X, y, lr: float = 0.0, grads=None) -> float:
    """One forward/backward (and Adam step if lr > 0) on device X [n, 256] bf16 bits, y [n]."""
    loss = C.c_float(0.0)
    _check(ctx.handle, _L.lvr_ao_train_step(ctx.handle, m.handle, int(X.shape[0]), _ptr(X), _ptr(y),
                                            float(lr), C.byref(loss), _ptr(grads)))
    return loss.value


def lvr_train_ao(ctx: Context, sets, lods, desc: AoTrainDesc):
    """Train a model on traced AO of the given line sets; returns (AoModel, final MSE)."""
    n = len(sets)
    hs = (_vp * n)(*[s.handle for s in sets])
    hl = (_vp * n)(*[l.handle for l in lods])
    h = _vp()
    mse = C.c_float(0.0)
    _check(ctx.handle, _L.lvr_train_ao(ctx.handle, hs, hl, n, C.byref(desc), C.byref(h), C.byref(mse)))
    return AoModel(ctx, h), mse.value


def ao_train_desc(n_samples, epochs, batch, lr, seed, render: RenderDesc, view_size=256, depth=32) -> AoTrainDesc:
    d = AoTrainDesc()
    d.n_samples, d.epochs, d.batch, d.lr, d.seed = int(n_samples), int(epochs), int(batch), float(lr), int(seed)
    d.view_size, d.depth = int(view_size), int(depth)
    d._render = render                       # keep the referenced struct alive
    d.render = C.pointer(render)
    return d


# ---------------------------------------------------------------- record layouts, batches, autotuner
def lvr_lineset_layout(ctx: Context, ls: LineSet, layout: int):
    _check(ctx.handle, _L.lvr_lineset_layout(ctx.handle, ls.handle, int(layout)))


def lvr_lineset_neighbours(ctx: Context, ls: LineSet, radius: float):
    """Camera-at-rest neighbour lists of `ls` for tube radii up to `radius`."""
    _check(ctx.handle, _L.lvr_lineset_neighbours(ctx.handle, ls.handle, float(radius)))


class Batch:
    """lvr_batch: many views in one persistent launch, replayed from a CUDA graph."""

    def __init__(self, ctx: Context, h, keep):
        self.ctx, self.handle, self._keep = ctx, h, keep

    def render(self):
        _check(self.ctx.handle, _L.lvr_batch_render(self.ctx.handle, self.handle))

    def size(self):
        t, r = _i64(0), _i64(0)
        _check(self.ctx.handle, _L.lvr_batch_size(self.handle, C.byref(t), C.byref(r)))
        return t.value, r.value

    def free(self):
        if getattr(self, "handle", None):
            _L.lvr_free_batch(self.handle)
            self.handle = None

    def __del__(self):
        if getattr(self, "ctx", None) is not None and self.ctx.handle:
            self.free()


def _items(entries):
    """entries: (LineSet, Lod | None, View, RenderDesc, AoModel | None, rgba device tensor)."""
    arr = (BatchItem * len(entries))()
    keep = []
    for i, (ls, lod, view, desc, model, rgba) in enumerate(entries):
        arr[i].ls = ls.handle
        arr[i].lod = lod.handle if lod is not None else None
        arr[i].view = view
        arr[i].desc = C.pointer(desc)
        arr[i].ao = model.handle if model is not None else None
        arr[i].rgba = _ptr(rgba)
        keep += [ls, lod, desc, model, rgba]
    return arr, keep


def lvr_batch_create(ctx: Context, entries) -> Batch:
    arr, keep = _items(entries)
    h = _vp()
    _check(ctx.handle, _L.lvr_batch_create(ctx.handle, arr, len(entries), C.byref(h)))
    return Batch(ctx, h, keep)


def lvr_batch_render(ctx: Context, b: Batch):
    b.render()


def lvr_free_batch(b: Batch):
    b.free()


def lvr_autotune(ctx: Context, entries, reps: int = 3) -> dict:
    arr, keep = _items(entries)
    t = Tune()
    _check(ctx.handle, _L.lvr_autotune(ctx.handle, arr, len(entries), int(reps), C.byref(t)))
    return {"tile": (t.tile_w, t.tile_h), "layout": t.layout, "ms": list(t.ms)}


# ---------------------------------------------------------------- spherical per-voxel AO
def lvr_lod_ao_field(ctx: Context, lod: Lod, rays: int = 100, radius: float = 5.0):
    _check(ctx.handle, _L.lvr_lod_ao_field(ctx.handle, lod.handle, int(rays), float(radius)))


def export_ao_field_numpy(ctx: Context, lod: Lod) -> np.ndarray:
    d = lod.info().dims[0]
    out = np.empty(int(d[0]) * int(d[1]) * int(d[2]), np.float32)
    _check(ctx.handle, _L.lvr_export_ao_field(ctx.handle, lod.handle, _ptr(out)))
    return out


# ---------------------------------------------------------------- representative lines
def lvr_lod_rep_lines(ctx: Context, lod: Lod, ls: LineSet):
    _check(ctx.handle, _L.lvr_lod_rep_lines(ctx.handle, lod.handle, ls.handle))


def export_rep_lines_numpy(ctx: Context, lod: Lod, level: int) -> np.ndarray:
    """uint8 [cells][8] of one level (see lvr_export_rep_lines)."""
    d = lod.info().dims[level]
    out = np.empty((int(d[0]) * int(d[1]) * int(d[2]), 8), np.uint8)
    _check(ctx.handle, _L.lvr_export_rep_lines(ctx.handle, lod.handle, int(level), _ptr(out)))
    return out


# ---------------------------------------------------------------- rasterised comparison system
def lvr_raster(ctx: Context, xyz, attr, curve_offsets, grid: GridDesc, view: View, desc: RenderDesc, rgba) -> dict:
    """Per-pixel fragment lists of the input polylines' tubes (opaque: depth
    test); rgba float32 (h, w, 4) for the crop. Returns the fragment stats."""
    nv = int(xyz.shape[0]) if xyz is not None else 0
    nc = int(curve_offsets.shape[0]) - 1
    st = RasterStats()
    _check(ctx.handle, _L.lvr_raster(ctx.handle, _ptr(xyz), _ptr(attr), _ptr(curve_offsets), nc, nv, C.byref(grid),
                                     C.byref(view), C.byref(desc), _ptr(rgba), C.byref(st)))
    return {"fragments": int(st.fragments), "max_per_pixel": int(st.max_per_pixel), "list_bytes": int(st.list_bytes)}
