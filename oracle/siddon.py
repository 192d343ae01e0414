"""ctypes binding of the oracle's FP64 Siddon projector (oracle.c).

Test infrastructure only.  See oracle.c for the reading of the system matrix A
(exact ray/pixel intersection lengths; the paper leaves A unspecified, Sec. IV).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class OgGeom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("offset_x", ctypes.c_double), ("offset_y", ctypes.c_double), ("offset_z", ctypes.c_double),
                ("nviews", ctypes.c_int), ("angle_start", ctypes.c_double), ("angle_span", ctypes.c_double),
                ("ns", ctypes.c_int), ("nt", ctypes.c_int), ("ds", ctypes.c_double), ("dt", ctypes.c_double),
                ("offset_s", ctypes.c_double), ("offset_t", ctypes.c_double),
                ("dso", ctypes.c_double), ("dsd", ctypes.c_double), ("pitch", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        gp = ctypes.POINTER(OgGeom)
        L.oracle_project.argtypes = [gp, dp, ip, ctypes.c_int, dp]
        L.oracle_backproject.argtypes = [gp, dp, ip, ctypes.c_int, dp]
        L.oracle_ray_segments.argtypes = [gp, ctypes.c_int, dp]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_get_threads.argtypes = []
        for f in (L.oracle_project, L.oracle_backproject, L.oracle_ray_segments, L.oracle_set_threads,
                  L.oracle_get_threads):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Host threads of the projector loops (results do not depend on it)."""
    return int(lib().oracle_set_threads(int(n)))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def og(geom) -> OgGeom:
    g = OgGeom()
    for name, _ in OgGeom._fields_:
        setattr(g, name, getattr(geom, name))
    return g


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def project(geom, x, views=None):
    """FP64 forward projection A_views x -> [nv][nt][ns]."""
    if views is None:
        views = np.arange(geom.nviews)
    views = np.ascontiguousarray(views, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    assert x.size == geom.nx * geom.ny * geom.nz
    out = np.zeros((views.size, geom.nt, geom.ns))
    g = og(geom)
    rc = lib().oracle_project(ctypes.byref(g), _dp(x), _ip(views), int(views.size), _dp(out))
    if rc != 0:
        raise ValueError(f"oracle_project failed ({rc})")
    return out


def backproject(geom, sino, views=None):
    """FP64 back-projection A_views^T sino -> image [nz][ny][nx]."""
    if views is None:
        views = np.arange(geom.nviews)
    views = np.ascontiguousarray(views, dtype=np.int32)
    sino = np.ascontiguousarray(sino, dtype=np.float64).reshape(-1)
    assert sino.size == views.size * geom.nt * geom.ns
    out = np.zeros((geom.nz, geom.ny, geom.nx))
    g = og(geom)
    rc = lib().oracle_backproject(ctypes.byref(g), _dp(sino), _ip(views), int(views.size), _dp(out))
    if rc != 0:
        raise ValueError(f"oracle_backproject failed ({rc})")
    return out


def ray_segments(geom, view):
    out = np.zeros((geom.nt, geom.ns, 2, 3))
    g = og(geom)
    rc = lib().oracle_ray_segments(ctypes.byref(g), int(view), _dp(out))
    if rc != 0:
        raise ValueError("oracle_ray_segments failed")
    return out
