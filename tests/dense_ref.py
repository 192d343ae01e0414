"""Dense system matrix built by slab clipping of every ray line against every
pixel box (independent of the oracle's plane-crossing traversal), from the
ray definition of ``synth.rays``.  Test helper."""
import numpy as np

from paper_1402_4381_gb300 import synth


def _clip(org, d, lo, hi, t_min):
    """Length of {org + t d : t >= t_min} inside the boxes [lo, hi] (broadcast)."""
    t0 = np.full(np.broadcast(lo[..., 0], hi[..., 0]).shape, t_min, dtype=np.float64)
    t1 = np.full_like(t0, np.inf)
    for k in range(3):
        if d[k] != 0.0:
            a = (lo[..., k] - org[k]) / d[k]
            b = (hi[..., k] - org[k]) / d[k]
            t0 = np.maximum(t0, np.minimum(a, b))
            t1 = np.minimum(t1, np.maximum(a, b))
        else:
            inside = (org[k] >= lo[..., k]) & (org[k] < hi[..., k])  # half-open pixels
            t1 = np.where(inside, t1, -np.inf)
    return np.maximum(t1 - t0, 0.0)


def _pixel_boxes(g):
    nz = g.nz
    dz = g.dz if g.kind == synth.CONE3D_FLAT else 1.0
    xs = (np.arange(g.nx) - g.nx / 2.0) * g.dx + g.offset_x
    ys = (np.arange(g.ny) - g.ny / 2.0) * g.dy + g.offset_y
    zs = (np.arange(nz) - nz / 2.0) * dz + (g.offset_z if g.kind == synth.CONE3D_FLAT else 0.0)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    lo = np.stack([X, Y, Z], -1).reshape(-1, 3)
    if g.kind != synth.CONE3D_FLAT:
        lo[:, 2] = -0.5
    hi = lo + np.array([g.dx, g.dy, dz])
    return lo, hi


def dense_A(g):
    org, dirn = synth.rays(g)
    lo, hi = _pixel_boxes(g)
    nrays = g.nviews * g.nt * g.ns
    A = np.zeros((nrays, lo.shape[0]))
    o2 = org.reshape(-1, 3)
    d2 = dirn.reshape(-1, 3)
    t_min = -np.inf if g.kind == synth.PAR2D else 0.0
    for i in range(nrays):
        A[i] = _clip(o2[i], d2[i], lo, hi, t_min)
    return A


