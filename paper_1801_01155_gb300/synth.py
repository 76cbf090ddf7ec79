"""Seeded synthetic inputs: streamline sets, transfer functions and cameras.

This module only *makes inputs*. It holds none of the rendering method's
arithmetic (no grid transform, no clipping, no quantisation, no ray casting),
so both the CUDA path and the FP64 oracle can take their inputs from here.

The paper's datasets (Tornado, Aneurysm, Turbulence, ECMWF weather; Sec. 6)
are not available, so dense, domain-filling streamlines of a divergence-free
random-Fourier flow stand in for them. The paper describes its data as a few
thousand to a few hundred thousand streamlines of 13 to 410 vertices each,
advected through 3D flows (Sec. 6, dataset list); the configurations below use
the same structure:

  u(x) = sum_m (a_m x k_m/|k_m|) cos(2 pi k_m . x + phi_m)

with integer wave vectors 1 <= |k_m| <= 4, a_m ~ N(0, I3), phi_m ~ U[0, 2pi).
Each term is perpendicular to its own wave vector, so div u = 0. Streamlines
start at uniform seeds in the unit cube and are integrated with classical RK4
in float64 (dt = 1e-3); vertices are stored as float32. The per-vertex
attribute is the local speed |u|, which a transfer function maps to colour and
opacity (Sec. 5.1).

Random draws use numpy's PCG64 ``default_rng(seed)`` in the order: wave
vectors, amplitudes, phases, seed points.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "FourierField",
    "LineSet",
    "fourier_field",
    "make_streamlines",
    "tf_ramp",
    "sigma_lut",
    "orbit_view",
    "CONFIGS",
]


@dataclass
class FourierField:
    k: np.ndarray        # (modes, 3) integer wave vectors
    amp: np.ndarray      # (modes, 3) a_m x k_hat_m
    phi: np.ndarray      # (modes,)
    rng: np.random.Generator

    def velocity(self, x: np.ndarray) -> np.ndarray:
        """u(x) for points x (n, 3), float64."""
        phase = (2.0 * math.pi) * (x @ self.k.T.astype(np.float64)) + self.phi
        return np.cos(phase) @ self.amp


def _wave_vectors(kmin: float, kmax: float) -> np.ndarray:
    r = int(math.ceil(kmax))
    g = np.arange(-r, r + 1)
    kk = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = np.sqrt((kk.astype(np.float64) ** 2).sum(1))
    return kk[(n >= kmin) & (n <= kmax)]


def fourier_field(seed: int, modes: int = 16, kmin: float = 1.0,
                  kmax: float = 4.0) -> FourierField:
    rng = np.random.default_rng(seed)
    cand = _wave_vectors(kmin, kmax)
    k = cand[rng.integers(0, len(cand), size=modes)]
    a = rng.standard_normal((modes, 3))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=modes)
    khat = k / np.linalg.norm(k, axis=1, keepdims=True)
    amp = np.cross(a, khat)
    return FourierField(k=k, amp=amp, phi=phi, rng=rng)


@dataclass
class LineSet:
    """Polylines in world space, laid out as the library's inputs expect."""
    xyz: np.ndarray       # float32 (n_vertices, 3)
    attr: np.ndarray      # float32 (n_vertices,)   per-vertex speed
    offsets: np.ndarray   # int64 (n_curves + 1,)   curve c = vertices [offsets[c], offsets[c+1])
    seed: int

    @property
    def n_curves(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_vertices(self) -> int:
        return int(self.offsets[-1])

    def subset(self, curves) -> "LineSet":
        """Curves selected by index (sorted), re-packed contiguously."""
        curves = np.asarray(curves, dtype=np.int64)
        lens = self.offsets[curves + 1] - self.offsets[curves]
        idx = np.concatenate([np.arange(self.offsets[c], self.offsets[c + 1])
                              for c in curves]) if len(curves) else np.zeros(0, np.int64)
        off = np.zeros(len(curves) + 1, np.int64)
        np.cumsum(lens, out=off[1:])
        return LineSet(self.xyz[idx].copy(), self.attr[idx].copy(), off, self.seed)


def _cache_path(tag: str) -> str | None:
    d = os.environ.get("LVR_SYNTH_CACHE")
    if not d:
        return None
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, tag + ".npz")


def make_streamlines(n_lines: int, n_vertices: int, seed: int,
                     dt: float = 1e-3, modes: int = 16,
                     chunk: int = 65536) -> LineSet:
    """RK4 streamlines through the seeded random-Fourier field.

    Every line has exactly ``n_vertices`` vertices (the seed is vertex 0).
    Lines may leave the unit cube; the voxeliser drops what lies outside
    the grid. If ``LVR_SYNTH_CACHE`` names a directory, results are cached
    there keyed by all arguments.
    """
    tag = f"stream_n{n_lines}_v{n_vertices}_s{seed}_dt{dt:g}_m{modes}"
    path = _cache_path(tag)
    if path and os.path.exists(path):
        z = np.load(path)
        return LineSet(z["xyz"], z["attr"], z["offsets"], seed)

    field = fourier_field(seed, modes)
    seeds = field.rng.random((n_lines, 3))
    xyz = np.empty((n_lines, n_vertices, 3), np.float32)
    attr = np.empty((n_lines, n_vertices), np.float32)
    try:            # vectorised over lines with torch's CPU threads when available
        import torch
        K = torch.from_numpy(field.k.T.astype(np.float64))
        AMP = torch.from_numpy(field.amp)
        PHI = torch.from_numpy(field.phi)
        two_pi = 2.0 * math.pi

        def vel(x):
            return torch.cos(torch.addmm(PHI, x, K, alpha=two_pi)) @ AMP

        for c0 in range(0, n_lines, chunk):
            x = torch.from_numpy(seeds[c0:c0 + chunk].copy())
            for i in range(n_vertices):
                u = vel(x)
                xyz[c0:c0 + chunk, i] = x.numpy()
                attr[c0:c0 + chunk, i] = torch.sqrt((u * u).sum(1)).numpy()
                if i + 1 == n_vertices:
                    break
                k1 = u
                k2 = vel(x + (0.5 * dt) * k1)
                k3 = vel(x + (0.5 * dt) * k2)
                k4 = vel(x + dt * k3)
                x = x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    except ImportError:
        for c0 in range(0, n_lines, chunk):
            x = seeds[c0:c0 + chunk].astype(np.float64)
            for i in range(n_vertices):
                u = field.velocity(x)
                xyz[c0:c0 + chunk, i] = x
                attr[c0:c0 + chunk, i] = np.sqrt((u * u).sum(1))
                if i + 1 == n_vertices:
                    break
                k1 = u
                k2 = field.velocity(x + 0.5 * dt * k1)
                k3 = field.velocity(x + 0.5 * dt * k2)
                k4 = field.velocity(x + dt * k3)
                x = x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    offsets = np.arange(0, (n_lines + 1) * n_vertices, n_vertices, dtype=np.int64)
    ls = LineSet(xyz.reshape(-1, 3), attr.reshape(-1), offsets, seed)
    if path:
        np.savez(path, xyz=ls.xyz, attr=ls.attr, offsets=ls.offsets)
    return ls


def make_streamlines_device(n_lines: int, n_vertices: int, seed: int, device,
                            dt: float = 1e-3, modes: int = 16, chunk: int = 262144):
    """The same RK4 streamlines as make_streamlines, integrated in float64 on
    a torch device (for line sets too large to trace on the host). Returns
    device tensors (xyz float32 [n*v][3], attr float32 [n*v], offsets int64
    [n+1]). Device cos may differ from the host's in the last bits, so the
    vertices can differ from make_streamlines' by rounding."""
    import torch
    field = fourier_field(seed, modes)
    seeds = torch.from_numpy(field.rng.random((n_lines, 3))).to(device)
    K = torch.from_numpy(field.k.T.astype(np.float64)).to(device)
    AMP = torch.from_numpy(field.amp).to(device)
    PHI = torch.from_numpy(field.phi).to(device)
    two_pi = 2.0 * math.pi

    def vel(x):
        return torch.cos(torch.addmm(PHI, x, K, alpha=two_pi)) @ AMP

    xyz = torch.empty((n_lines, n_vertices, 3), dtype=torch.float32, device=device)
    attr = torch.empty((n_lines, n_vertices), dtype=torch.float32, device=device)
    for c0 in range(0, n_lines, chunk):
        x = seeds[c0:c0 + chunk].clone()
        for i in range(n_vertices):
            u = vel(x)
            xyz[c0:c0 + chunk, i] = x.to(torch.float32)
            attr[c0:c0 + chunk, i] = torch.sqrt((u * u).sum(1)).to(torch.float32)
            if i + 1 == n_vertices:
                break
            k1 = u
            k2 = vel(x + (0.5 * dt) * k1)
            k3 = vel(x + (0.5 * dt) * k2)
            k4 = vel(x + dt * k3)
            x = x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    offsets = torch.arange(0, (n_lines + 1) * n_vertices, n_vertices, dtype=torch.int64, device=device)
    return xyz.reshape(-1, 3), attr.reshape(-1), offsets


# ---------------------------------------------------------------- transfer functions
def tf_ramp(alpha_min: float = 1.0, alpha_max: float = 1.0) -> np.ndarray:
    """256-entry RGBA transfer function, float32 (256, 4).

    Colour is a blue -> cyan -> yellow -> red ramp over the attribute byte;
    opacity is linear from alpha_min to alpha_max. Opaque configurations use
    alpha 1 (the renderer ignores alpha in opaque mode anyway).
    """
    s = np.arange(256, dtype=np.float64) / 255.0
    knots = np.array([0.0, 1.0 / 3.0, 2.0 / 3.0, 1.0])
    cols = np.array([[0.10, 0.20, 0.90],
                     [0.10, 0.80, 0.85],
                     [0.95, 0.85, 0.15],
                     [0.90, 0.15, 0.10]])
    rgb = np.stack([np.interp(s, knots, cols[:, c]) for c in range(3)], 1)
    a = alpha_min + (alpha_max - alpha_min) * s
    return np.concatenate([rgb, a[:, None]], 1).astype(np.float32)


def sigma_lut(tf: np.ndarray) -> np.ndarray:
    """Per-attribute-byte opacity sigma used by the density LoD: the TF alpha."""
    return np.ascontiguousarray(tf[:, 3], dtype=np.float32)


# ---------------------------------------------------------------- cameras
def orbit_view(res, width: int, height: int, direction=(1.0, 0.8, 1.3),
               dist_factor: float = 1.8, fovy_deg: float = 40.0,
               light_dir=(-0.3, -1.0, -0.5)) -> dict:
    """Camera looking at the grid centre from ``direction``.

    Positions are in grid (voxel) units: the grid spans [0, res]^3. The
    distance is ``dist_factor`` times the half-diagonal of the grid.
    ``light_dir`` is the direction in which light travels.
    """
    res = np.asarray(res, np.float64)
    c = res / 2.0
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    dist = dist_factor * np.linalg.norm(res) / 2.0
    eye = c + dist * d
    return dict(eye=eye.astype(np.float32), at=c.astype(np.float32),
                up=np.array([0.0, 1.0, 0.0], np.float32), fovy_deg=float(fovy_deg),
                width=int(width), height=int(height),
                light_dir=np.asarray(light_dir, np.float32))


def orbit_views(n: int, res, sizes, seed: int = 5) -> list:
    """n seeded orbit cameras around a grid; sizes cycles through (w, h)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        az = rng.uniform(0.0, 2.0 * math.pi)
        el = rng.uniform(-0.6, 0.9)
        d = (math.cos(el) * math.cos(az), math.sin(el), math.cos(el) * math.sin(az))
        w, h = sizes[i % len(sizes)]
        out.append(orbit_view(res, w, h, direction=d))
    return out


# ---------------------------------------------------------------- workload presets
CONFIGS = {
    # plain method, tiny: 500 x 64, 32^3, r = 0.2 voxel, opaque, 128x128
    "c1": dict(n_lines=500, n_vertices=64, seed=0, res=32, bins=32, radius=0.2,
               opaque=True, width=128, height=128, alpha=(1.0, 1.0),
               shadows=False, ao=False),
    # transparency at scale: 100k x 200, 256^3, r = 0.15, alpha 0.05-0.3, ERT 0.99, 1080p
    "c2": dict(n_lines=100_000, n_vertices=200, seed=1, res=256, bins=32, radius=0.15,
               opaque=False, ert=0.99, width=1920, height=1080, alpha=(0.05, 0.3),
               shadows=False, ao=False),
    # illumination: c1 set + 3-level LoD, shadow + 16 AO rays, transparent, 1080p
    "c3": dict(n_lines=500, n_vertices=64, seed=0, res=32, bins=32, radius=0.2,
               opaque=False, ert=0.99, width=1920, height=1080, alpha=(0.05, 0.3),
               shadows=True, ao=True, ao_rays=16, ao_radius=15.0, levels=3),
}
