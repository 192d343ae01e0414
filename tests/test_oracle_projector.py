"""Pins of the oracle's system matrix A (FP64 Siddon, oracle/oracle.c).

The paper does not define A (Sec. IV, Eq. ct_recon); the reading is exact
ray/pixel intersection lengths.  These tests tie the oracle to things it does
not compute itself:
* a dense A built here by clipping every ray line against every pixel box
  (slab clipping, no plane-crossing traversal) from the ray definition in
  ``synth.rays`` -- exact to FP64 rounding;
* closed-form chords (ray through a pixel centre, ray through the image box);
* analytic line integrals of ellipses (error shrinks as pixels shrink);
* the adjoint identity <Ax, r> = <x, A'r>.
"""
import math

import numpy as np
import pytest

from oracle import siddon
from paper_1402_4381_gb300 import synth, workloads as W
from dense_ref import _clip, dense_A


GEOMS = [
    ("parallel", W.tiny_parallel()),
    ("parallel_odd", W.tiny_parallel(n=7, nviews=9, ns=12)),
    ("fan", W.tiny_fan()),
    ("cone", W.tiny_cone()),
    ("helical", W.tiny_helical()),
]


@pytest.mark.parametrize("name,g", GEOMS)
def test_siddon_equals_dense_clipping(name, g, oracle_lib):
    A = dense_A(g)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, size=A.shape[1])
    r = rng.uniform(-1, 1, size=A.shape[0])
    fp = siddon.project(g, x).reshape(-1)
    bp = siddon.backproject(g, r).reshape(-1)
    assert np.abs(A).sum() > 0
    np.testing.assert_allclose(fp, A @ x, rtol=0, atol=1e-11)
    np.testing.assert_allclose(bp, A.T @ r, rtol=0, atol=1e-11)


@pytest.mark.parametrize("name,g", GEOMS)
def test_projection_of_ones_is_box_chord(name, g, oracle_lib):
    """A 1 = length of the ray inside the whole image box (closed form)."""
    org, dirn = synth.rays(g)
    dz = g.dz if g.kind == synth.CONE3D_FLAT else 1.0
    lo = np.array([-g.nx * g.dx / 2, -g.ny * g.dy / 2, -g.nz * dz / 2 if g.kind == 2 else -0.5])
    hi = -lo
    t_min = -np.inf if g.kind == synth.PAR2D else 0.0
    expect = np.array([_clip(o, d, lo, hi, t_min) for o, d in zip(org.reshape(-1, 3), dirn.reshape(-1, 3))])
    got = siddon.project(g, np.ones(g.image_shape)).reshape(-1)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-11)


@pytest.mark.parametrize("theta", [0.0, 0.3, math.pi / 4, 1.1, 2.0, 2.9])
def test_single_pixel_central_chord(theta, oracle_lib):
    """The central ray crosses the centre pixel of an odd grid with chord
    dx / max(|cos|, |sin|)."""
    g = synth.Geometry(kind=synth.PAR2D, nx=7, ny=7, dx=1.3, dy=1.3, nviews=1,
                       angle_start=theta, angle_span=math.pi, ns=3, ds=1.0)
    x = np.zeros(g.image_shape)
    x[0, 3, 3] = 1.0
    p = siddon.project(g, x)
    expect = 1.3 / max(abs(math.cos(theta)), abs(math.sin(theta)))
    assert abs(p[0, 0, 1] - expect) < 1e-12


def test_analytic_ellipse_convergence(oracle_lib):
    """Projections of a pixelised ellipse approach its analytic line integrals
    as the pixels shrink (first order in the pixel size)."""
    ph = [synth.Ellipsoid(3.0, -2.0, 20.0, 12.0, 0.4, 0.02),
          synth.Ellipsoid(-5.0, 4.0, 6.0, 9.0, 1.2, 0.01)]
    errs = []
    for n in (32, 64, 128):
        g = synth.Geometry(kind=synth.FAN2D_ARC, nx=n, ny=n, dx=64.0 / n, dy=64.0 / n, nviews=12,
                           angle_start=0.2, angle_span=2 * math.pi, ns=61, ds=1.5, dso=100.0, dsd=180.0)
        img = synth.pixelize(g, ph, supersample=8)
        p = siddon.project(g, img)
        pa = synth.analytic_sinogram(g, ph)
        errs.append(np.sqrt(np.mean((p - pa) ** 2)) / np.sqrt(np.mean(pa ** 2)))
    assert errs[0] < 0.05
    assert errs[1] < 0.6 * errs[0]
    assert errs[2] < 0.6 * errs[1]


def test_analytic_ellipsoid_cone(oracle_lib):
    """Cone beam: the same first-order convergence to the analytic integrals."""
    ph = [synth.Ellipsoid(1.0, -1.0, 10.0, 7.0, 0.3, 0.02, cz=0.5, c=4.0)]
    errs = []
    for n, nz in ((24, 12), (48, 24), (96, 48)):
        g = synth.Geometry(kind=synth.CONE3D_FLAT, nx=n, ny=n, nz=nz, dx=24.0 / n, dy=24.0 / n,
                           dz=12.0 / nz, nviews=6, angle_start=0.1, angle_span=2 * math.pi,
                           ns=41, nt=21, ds=0.9, dt=0.9, dso=60.0, dsd=100.0)
        img = synth.pixelize(g, ph, supersample=4)
        p = siddon.project(g, img)
        pa = synth.analytic_sinogram(g, ph)
        errs.append(np.sqrt(np.mean((p - pa) ** 2)) / np.sqrt(np.mean(pa ** 2)))
    assert errs[0] < 0.15
    assert errs[1] < 0.6 * errs[0]
    assert errs[2] < 0.6 * errs[1]


@pytest.mark.parametrize("name,g", GEOMS + [("fan32", W.scaled(W.c1_fan(), 32, 24, 40, 4).geom)])
def test_adjoint_identity(name, g, oracle_lib):
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 1, size=g.image_shape)
    r = rng.uniform(0, 1, size=g.sino_shape)
    lhs = float(np.sum(siddon.project(g, x) * r))
    rhs = float(np.sum(x * siddon.backproject(g, r)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_subset_views_projection_matches_full(oracle_lib):
    g = W.tiny_fan()
    x = np.random.default_rng(3).uniform(size=g.image_shape)
    full = siddon.project(g, x)
    views = np.array([5, 1, 6])
    part = siddon.project(g, x, views)
    np.testing.assert_array_equal(part, full[views])


def test_synth_circle_closed_form():
    """The scan simulator's line integrals: a centred disk of radius R seen by
    parallel rays at offset s integrates to 2 mu sqrt(R^2 - s^2)."""
    g = synth.Geometry(kind=synth.PAR2D, nx=8, ny=8, nviews=5, angle_start=0.3,
                       angle_span=math.pi, ns=21, ds=1.0)
    ph = [synth.Ellipsoid(0.0, 0.0, 7.0, 7.0, 0.0, 0.03)]
    p = synth.analytic_sinogram(g, ph)
    s = (np.arange(21) - 10) * 1.0
    expect = 2 * 0.03 * np.sqrt(np.maximum(49 - s ** 2, 0))
    np.testing.assert_allclose(p[:, 0, :], np.broadcast_to(expect, (5, 21)), atol=1e-12)


def test_synth_fan_rays_pass_through_source_and_arc():
    g = W.tiny_fan()
    org, d = synth.rays(g)
    phi = g.view_angles()
    np.testing.assert_allclose(org[:, 0, 0, 0], -g.dso * np.cos(phi), atol=1e-12)
    # central channel (odd ns) points at the isocentre
    c = (g.ns - 1) // 2
    np.testing.assert_allclose(d[:, 0, c, 0], np.cos(phi), atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(d, axis=-1), 1.0, atol=1e-12)


def test_analytic_ellipsoid_helical(oracle_lib):
    """Helical orbit (two turns, pitch 0.7): first-order convergence to the
    analytic integrals of the rising rays."""
    ph = [synth.Ellipsoid(1.0, -1.0, 10.0, 7.0, 0.3, 0.02, cz=0.5, c=4.0)]
    errs = []
    for n, nz in ((24, 12), (48, 24), (96, 48)):
        g = synth.Geometry(kind=synth.CONE3D_FLAT, nx=n, ny=n, nz=nz, dx=24.0 / n, dy=24.0 / n,
                           dz=12.0 / nz, nviews=8, angle_start=0.1, angle_span=4 * math.pi,
                           ns=41, nt=21, ds=0.9, dt=0.9, dso=60.0, dsd=100.0, pitch=0.7)
        img = synth.pixelize(g, ph, supersample=4)
        p = siddon.project(g, img)
        pa = synth.analytic_sinogram(g, ph)
        errs.append(np.sqrt(np.mean((p - pa) ** 2)) / np.sqrt(np.mean(pa ** 2)))
    assert errs[0] < 0.15
    assert errs[1] < 0.6 * errs[0]
    assert errs[2] < 0.6 * errs[1]


def test_helical_source_rises_by_the_table_feed():
    """Source heights: pitch * nt * dt per turn, centred on the angle range."""
    g = W.tiny_helical(nviews=16)
    org, d = synth.rays(g)
    zs = org[:, 0, 0, 2]
    per_view = g.pitch * g.nt * g.dt / 8  # 8 views per turn
    np.testing.assert_allclose(np.diff(zs), per_view, rtol=1e-12)
    assert abs(zs[0] + zs[-1] + per_view) < 1e-12  # symmetric about the middle of the range
    seg = siddon.ray_segments(g, 5)
    np.testing.assert_allclose(seg[:, :, 0, 2], zs[5], atol=1e-12)  # the oracle's own source height
