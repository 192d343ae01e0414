"""Region of interest of the RMS-difference figures (evaluation only).

Sec. V reports convergence as the RMS difference to the converged image over
a "region of interest" that it does not define.  Reading: the scanner's field
of view, i.e. the pixels whose centre projects onto the detector (between the
outer edges of the first and last channel) from every view; for the cone beam
also onto the detector rows from every view of a circular orbit, and for a
helix the heights between the first and last source positions.

This is the one copy used by the benchmark and the warm-start evaluation;
it holds no reconstruction arithmetic.
"""
from __future__ import annotations

import math

import numpy as np

from .synth import CONE3D_FLAT, PAR2D


def roi_mask(geom) -> np.ndarray:
    """Boolean mask [nz][ny][nx] of the field of view of `geom`."""
    ix = (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.dx + geom.offset_x
    iy = (np.arange(geom.ny) - (geom.ny - 1) / 2.0) * geom.dy + geom.offset_y
    Y, X = np.meshgrid(iy, ix, indexing="ij")
    r = np.sqrt(X * X + Y * Y)
    # the two outer cell edges at s = (+-ns/2 + offset_s) ds on the detector;
    # the field of view is the disk inside the nearer edge ray of every view
    half = min(abs(-geom.ns / 2.0 + geom.offset_s), abs(geom.ns / 2.0 + geom.offset_s)) * geom.ds
    if geom.kind == PAR2D:
        R = half
    elif geom.kind == CONE3D_FLAT:
        R = geom.dso * math.sin(math.atan(half / geom.dsd))  # flat panel: edge ray at atan(s / dsd)
    else:
        R = geom.dso * math.sin(half / geom.dsd)  # arc detector: edge ray at s / dsd
    disk = (r <= R)[None]
    if geom.kind != CONE3D_FLAT:
        return disk
    iz = (np.arange(geom.nz) - (geom.nz - 1) / 2.0) * geom.dz + geom.offset_z
    if geom.pitch != 0.0:
        zs = geom.source_z()
        return disk & ((iz >= zs.min()) & (iz <= zs.max()))[:, None, None]
    # largest magnification a voxel at radius r sees over a full orbit: dsd / (dso - r)
    mag = geom.dsd / np.maximum(geom.dso - r, 1e-9)
    return disk & (np.abs(iz)[:, None, None] * mag[None] <= geom.nt * geom.dt / 2.0)
