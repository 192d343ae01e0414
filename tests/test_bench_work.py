"""The benchmark's own bookkeeping, pinned on the CPU: the closed-form count
of (ray, pixel) intersections that the roofline's work per launch uses,
against the non-zero entries of the dense system matrix built by slab
clipping; and the field-of-view mask of the RMS differences, against a
brute-force check that every view's detector sees each masked pixel."""
import math
import os
import sys

import numpy as np
import pytest

from dense_ref import dense_A
from paper_1402_4381_gb300 import synth, workloads as W

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _generic_fan():
    return synth.Geometry(kind=synth.FAN2D_ARC, nx=9, ny=7, dx=1.1, dy=0.9, nviews=7, angle_start=0.13,
                          angle_span=2 * math.pi, ns=17, ds=1.3, dso=20.0, dsd=35.0, offset_s=0.21)


def _generic_cone(pitch=0.0):
    return synth.Geometry(kind=synth.CONE3D_FLAT, nx=7, ny=6, nz=5, dx=1.1, dy=0.9, dz=0.7, nviews=6,
                          angle_start=0.11, angle_span=2 * math.pi, ns=13, nt=5, ds=1.3, dt=1.1, dso=20.0,
                          dsd=35.0, offset_s=0.21, offset_t=0.13, pitch=pitch)


def _generic_parallel():
    return synth.Geometry(kind=synth.PAR2D, nx=8, ny=10, dx=1.0, dy=0.8, nviews=9, angle_start=0.07,
                          angle_span=math.pi, ns=15, ds=0.9, offset_s=0.17)


@pytest.mark.parametrize("g", [_generic_fan(), _generic_parallel(), _generic_cone(), _generic_cone(pitch=0.7)])
def test_intersection_count_equals_dense_nonzeros(g):
    """Generic positions (no ray through a cell edge or corner, where the
    closed form would count a cell the ray only touches)."""
    A = dense_A(g)
    nnz = int(np.count_nonzero(A > 1e-9))
    assert nnz > 0
    got = bench.intersections_per_subset(g, 1, max_views=g.nviews)
    assert got == nnz


def test_intersection_count_scales_with_subsets():
    g = _generic_fan()
    one = bench.intersections_per_subset(g, 1, max_views=g.nviews)
    assert bench.intersections_per_subset(g, 7, max_views=g.nviews) == pytest.approx(one / 7)
