"""The oracle's voxel model against the unvoxelised polylines (Secs. 3.1-3.3, 4.1).

The model replaces each polyline, from its first to its last voxel-face
crossing, by face-to-face segments between bin centres (Secs. 3.1, 3.2; the
pieces before the first and after the last crossing end inside a voxel and
are not stored), so its tubes are the tubes of those trimmed polylines moved
by at most the two-way distance delta between the quantised segments and
the trimmed raw polyline. With the
camera at rest (every capsule is found, the image equals a brute force over
all quantised capsules) an opaque frame must therefore cover every ray that
passes within r - delta of the raw polyline and no ray that stays farther
than r + delta from it. delta is measured here on the data, by dense sampling
of both curves, and checked against the bound the quantisation allows.
"""
import numpy as np

from paper_1801_01155_gb300 import synth


def _sample(polyline, step):
    pts = [polyline[:1]]
    for a, b in zip(polyline[:-1], polyline[1:]):
        n = max(1, int(np.ceil(np.linalg.norm(b - a) / step)))
        s = np.arange(1, n + 1)[:, None] / n
        pts.append(a + s * (b - a))
    return np.concatenate(pts)


def _nearest(p, q, chunk=2048):
    """Distance from each point of p to the point set q."""
    out = np.empty(len(p))
    for i in range(0, len(p), chunk):
        d = p[i:i + chunk, None, :] - q[None, :, :]
        out[i:i + chunk] = np.sqrt((d * d).sum(-1)).min(1)
    return out


def test_opaque_frame_within_the_quantisation_of_the_raw_lines(orc):
    res, N, r, step = 16, 32, 0.45, 0.01
    ls = synth.make_streamlines(60, 96, seed=9)
    xyz = ls.xyz.reshape(60, 96, 3)
    keep = np.all((xyz > 0.15) & (xyz < 0.85), axis=(1, 2))
    assert keep.sum() >= 8
    xyz = np.ascontiguousarray(xyz[keep][:12])
    nc = len(xyz)
    offs = np.arange(0, (nc + 1) * 96, 96, dtype=np.int64)
    vs = orc.VoxSet(xyz.reshape(-1, 3), None, offs, orc.make_grid(res, N, scale=float(res)))
    e = vs.export()
    # quantised segments in grid coordinates: voxel + face point of each end
    off = e["offset"].astype(np.int64)
    vox = np.repeat(np.arange(res ** 3), np.diff(off))
    base = np.stack([vox % res, (vox // res) % res, vox // (res * res)], 1).astype(np.float64)
    f = e["fields"].astype(np.int64)

    def face_point(face, u, v):
        ax, side = face >> 1, (face & 1).astype(np.float64)
        cu, cv = (u + 0.5) / N, (v + 0.5) / N
        return np.stack([np.where(ax == 0, side, cu), np.where(ax == 1, side, np.where(ax == 0, cu, cv)),
                         np.where(ax == 2, side, cv)], 1)

    qa = base + face_point(f[:, 0], f[:, 1], f[:, 2])
    qb = base + face_point(f[:, 3], f[:, 4], f[:, 5])
    quant = np.concatenate([_sample(np.stack([a, b]), step) for a, b in zip(qa, qb)])
    raw = []
    for c in xyz:   # each raw polyline between its first and last face crossing
        pts = _sample(c.astype(np.float64) * res, step / 4)
        cell = np.floor(pts).astype(np.int64)
        moved = np.nonzero(np.any(cell[1:] != cell[:-1], axis=1))[0]
        if len(moved):
            raw.append(pts[moved[0]:moved[-1] + 2])
    raw = np.concatenate(raw)
    # two-way distance between the model and the raw lines, plus the sampling error
    delta = max(_nearest(quant, raw).max(), _nearest(raw, quant).max()) + step
    # bin snapping moves an end by at most half a bin diagonal; a chord inside
    # one voxel stays well within the voxel diagonal of the raw curve (Sec. 3.1)
    assert 0.5 * np.sqrt(2.0) / N <= delta < 0.5

    W = H = 64
    cam = synth.orbit_view((res, res, res), W, H)
    view = orc.make_view(cam["eye"], cam["at"], cam["up"], 30.0, W, H, cam["light_dir"])
    pix = orc.pixel_grid(0, 0, W, H)
    rgba, tie, _ = orc.render(vs, None, view, orc.make_rdesc(r, synth.tf_ramp(), opaque=True, still=True), pix)
    covered = rgba[:, 3] > 0.5
    # distance of each primary ray (a half-line from the eye) to the raw polyline
    d_raw = np.empty(len(pix))
    for k, (i, j) in enumerate(pix):
        o, d = orc.primary_ray(view, int(i), int(j))
        o, d = o.astype(np.float64), d.astype(np.float64)
        d /= np.linalg.norm(d)
        w = raw - o
        t = np.maximum(w @ d, 0.0)
        d_raw[k] = np.sqrt(((w - t[:, None] * d) ** 2).sum(1)).min()
    inside, outside = d_raw < r - delta, d_raw > r + delta
    assert covered[inside].all()
    assert not covered[outside].any()
    assert inside.sum() > 200 and outside.sum() > 1000
    # what is left between the two bands is the silhouette seam
    assert (~inside & ~outside).mean() < 0.2
