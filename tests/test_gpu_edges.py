"""Degenerate and extreme cases of the CUDA path against the FP64 oracle:
pure weighted least squares (beta = 0) with pixels that no ray crosses (the
majorizer is 0 there: the pixel keeps its value), a detector much wider than
the image (rays that miss it), and the largest image the 2D ray tables allow
(4096^2) at exactly 45 degrees, where the exact integer part of a row centre,
(2 ia + 1) k / 4096, is at its bound."""
import dataclasses
import math

import numpy as np
import pytest

from gpu_util import COST_RTOL, RMSD_HU_TOL, assert_rel_floor, to_dev, to_host
from oracle import oslalm as O
from oracle import siddon
from paper_1402_4381_gb300 import synth, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_4381_gb300 import build, oslalm
    build.build()
    return oslalm


def test_beta_zero_with_uncovered_pixels(L):
    # a parallel beam whose detector sits 10.5-29.5 mm off the axis: no ray passes
    # within 10 mm of the centre, so the central pixels have D = 0
    g = synth.Geometry(kind=synth.PAR2D, nx=64, ny=64, dx=1.0, dy=1.0, nviews=60, angle_start=0.0,
                       angle_span=2 * math.pi, ns=20, ds=1.0, offset_s=20.0)
    wl = dataclasses.replace(W.c0_parallel(), name="wls_offset", geom=g, fov_radius=25.0, beta=0.0, M=5)
    scan = wl.make_scan()
    y, w = scan["y"], scan["w"]
    x0 = np.full(g.image_shape, 0.01, dtype=np.float32)
    data, _ = O.ct_subset_data(g, y.astype(np.float64), w.astype(np.float64), wl.M, siddon)
    D = data.sqs_denominator(g.image_shape)
    uncovered = D == 0.0
    assert uncovered.sum() > 100
    alg = O.OsLalm(data, D, 0.0, wl.delta, wl.nbr)
    alg.init(x0.astype(np.float64))
    alg.run(2 * wl.M)
    geom = L.Geometry(g)
    prob = L.Problem(geom, to_dev(y), to_dev(w), beta=0.0, delta=wl.delta, nbr=wl.nbr, M=wl.M, rho_mode="replay")
    prob.set_replay([int(h["restart"]) for h in alg.history])
    x = to_dev(x0)
    prob.init(x)
    prob.iterate(x, 2)
    xg = to_host(x)
    assert np.all(np.isfinite(xg))
    np.testing.assert_array_equal(xg[uncovered], np.float32(0.01))
    np.testing.assert_array_equal(alg.x[uncovered], np.float64(np.float32(0.01)))
    assert O.rmsd_hu(xg, alg.x, ~uncovered) <= RMSD_HU_TOL
    assert abs(prob.cost(x) - alg.cost()) <= COST_RTOL * abs(alg.cost())


def test_detector_wider_than_image(L):
    g = synth.Geometry(kind=synth.PAR2D, nx=32, ny=32, dx=1.0, dy=1.0, nviews=12, angle_start=0.2,
                       angle_span=math.pi, ns=96, ds=1.0)
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, size=g.image_shape)
    geom = L.Geometry(g)
    got = to_host(geom.project(to_dev(x)))
    ref = siddon.project(g, x)
    assert (ref == 0).sum() > g.nviews * 20  # rays that miss the image
    assert np.all(got[ref == 0] == 0.0)
    assert_rel_floor(got, ref, what="wide-detector A x")
    r = rng.uniform(0, 1, size=g.sino_shape)
    assert_rel_floor(to_host(geom.backproject(to_dev(r))), siddon.backproject(g, r), what="wide-detector A'r")


def test_largest_image_at_45_degrees(L):
    n = 4096
    g = synth.Geometry(kind=synth.PAR2D, nx=n, ny=n, dx=1.0, dy=1.0, nviews=4, angle_start=math.pi / 4,
                       angle_span=math.pi, ns=5800, ds=1.0, offset_s=0.3)
    rng = np.random.default_rng(9)
    x = rng.uniform(0.0, 0.04, size=g.image_shape).astype(np.float32)
    geom = L.Geometry(g)
    got = to_host(geom.project(to_dev(x)))
    ref = siddon.project(g, x.astype(np.float64))
    assert_rel_floor(got, ref, what="4096^2 A x")
    r = rng.uniform(0.5, 1.5, size=g.sino_shape).astype(np.float32)
    gotb = to_host(geom.backproject(to_dev(r)))
    refb = siddon.backproject(g, r.astype(np.float64))
    assert_rel_floor(gotb, refb, what="4096^2 A'r")
