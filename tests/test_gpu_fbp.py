"""GPU FBP (initial image) against the FP64 oracle FBP."""
import math

import numpy as np
import pytest

from gpu_util import to_dev, to_host
from oracle import fbp as ofbp
from paper_1402_4381_gb300 import synth, workloads as W

pytestmark = pytest.mark.gpu

PH = [synth.Ellipsoid(0, 0, 50, 40, 0.2, 0.02), synth.Ellipsoid(10, 5, 10, 8, 0.5, 0.01)]


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    from paper_1402_4381_gb300 import build, oslalm
    build.build()
    return oslalm


GEOMS = [
    W.c0_parallel().geom,
    W.scaled(W.c1_fan(), 128, 360, 256, 4).geom,
    W.c1_fan().geom,
    synth.Geometry(kind=2, nx=48, ny=40, nz=6, dx=2.5, dy=2.5, dz=2.5, nviews=60, angle_span=2 * math.pi,
                   ns=96, nt=24, ds=2.5, dt=2.5, dso=300, dsd=500),
]


@pytest.mark.parametrize("g", GEOMS)
def test_fbp_matches_oracle(L, g):
    if g.kind == 2:
        ph = [synth.Ellipsoid(0, 0, 50, 40, 0.2, 0.02, cz=0, c=5)]
    else:
        ph = PH
    p = synth.analytic_sinogram(g, ph).astype(np.float32)
    geom = L.Geometry(g)
    got = to_host(geom.fbp(to_dev(p), clip=False))
    ref = ofbp.fbp(g, p.astype(np.float64))
    err = np.max(np.abs(got - ref))
    assert err <= 3e-4 * np.max(np.abs(ref)), err
    clipped = to_host(geom.fbp(to_dev(p), clip=True))
    assert np.array_equal(clipped, np.maximum(got, 0))
