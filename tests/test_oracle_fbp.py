"""Pins of the oracle's FBP (initial image): on noiseless analytic data of a
uniform ellipse the reconstruction reproduces the attenuation value in the
interior (scaling of the ramp filter, the fan kernel, the distance weights and
the FDK cosine weight), and the whole image is close to the phantom."""
import math

import numpy as np
import pytest

from oracle import fbp
from paper_1402_4381_gb300 import synth, workloads as W

PH = [synth.Ellipsoid(0, 0, 50, 40, 0.2, 0.02), synth.Ellipsoid(10, 5, 10, 8, 0.5, 0.01)]


def _centres(g):
    X, Y = np.meshgrid((np.arange(g.nx) - (g.nx - 1) / 2) * g.dx, (np.arange(g.ny) - (g.ny - 1) / 2) * g.dy)
    return X, Y


@pytest.mark.parametrize("g", [W.c0_parallel().geom, W.scaled(W.c1_fan(), 128, 360, 256, 4).geom])
def test_fbp_reproduces_uniform_region(g):
    x = fbp.fbp(g, synth.analytic_sinogram(g, PH))
    xt = synth.pixelize(g, PH, 4)
    X, Y = _centres(g)
    reg = (X + 20) ** 2 + (Y + 10) ** 2 < 15 ** 2
    assert abs(x[0][reg].mean() - 0.02) < 1e-4
    reg2 = (X - 10) ** 2 + (Y - 5) ** 2 < 5 ** 2
    assert abs(x[0][reg2].mean() - 0.03) < 3e-4
    assert np.sqrt(np.mean((x - xt) ** 2)) < 0.03 * 0.02


def test_fdk_central_slice():
    g = synth.Geometry(kind=2, nx=48, ny=48, nz=8, dx=2.5, dy=2.5, dz=2.5, nviews=120,
                       angle_span=2 * math.pi, ns=96, nt=24, ds=2.5, dt=2.5, dso=300, dsd=500)
    ph = [synth.Ellipsoid(0, 0, 50, 40, 0.2, 0.02, cz=0, c=12)]
    x = fbp.fbp(g, synth.analytic_sinogram(g, ph))
    c = x[3:5, 20:28, 20:28].mean()
    assert abs(c - 0.02) < 2e-4


def test_fbp_rejects_short_fan_scan():
    g = W.tiny_fan()
    g.angle_span = math.pi
    with pytest.raises(ValueError):
        fbp.fbp(g, np.zeros(g.sino_shape))
