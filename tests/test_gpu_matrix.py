"""The system matrix held in device memory (oslalm_geom_build_matrix): the
table-driven projector pair and OS-LALM iterations give the same bits as the
evaluating kernels, on parallel and fan geometries of several shapes
(ragged tiles, a view at exactly 45 degrees, mixed ray orientations within
a view), and the matrix is refused for a 3D geometry."""
import math

import numpy as np
import pytest

from gpu_util import to_dev, to_host
from paper_1402_4381_gb300 import synth, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_4381_gb300 import build, oslalm
    build.build()
    return oslalm


def _ragged_fan():
    return synth.Geometry(kind=synth.FAN2D_ARC, nx=37, ny=29, dx=1.7, dy=1.7, nviews=23,
                          angle_start=0.3, angle_span=2 * math.pi, ns=61, ds=1.9, dso=120.0, dsd=200.0)


def _ragged_par():
    return synth.Geometry(kind=synth.PAR2D, nx=45, ny=33, dx=1.1, dy=0.9, nviews=17,
                          angle_start=0.0, angle_span=math.pi, ns=71, ds=0.8, offset_s=0.25)


CASES = [
    ("c0_parallel", W.c0_parallel().geom),  # 180 views over 180 degrees: views at exactly 0, 45, 90, 135
    ("c1_fan_128", W.scaled(W.c1_fan(), 128, 246, 222, 6).geom),
    ("tiny_fan", W.tiny_fan()),
    ("ragged_fan", _ragged_fan()),
    ("ragged_parallel", _ragged_par()),
]


def _pair(L, g):
    plain = L.Geometry(g)
    tab = L.Geometry(g)
    nbytes = tab.build_matrix()
    assert nbytes > 0
    return plain, tab


@pytest.mark.parametrize("name,g", CASES)
def test_projector_pair_from_matrix_is_bit_identical(L, name, g):
    import torch
    plain, tab = _pair(L, g)
    rng = np.random.default_rng(7)
    x = to_dev(rng.uniform(0.0, 0.04, size=g.image_shape))
    r = to_dev(rng.normal(size=(g.nviews, g.nt, g.ns)))
    views = list(rng.permutation(g.nviews)[: max(1, g.nviews // 3)])
    for vv in (None, views):
        a, b = plain.project(x, views=vv), tab.project(x, views=vv)
        assert torch.equal(a, b), f"{name}: forward projections differ"
        rr = r if vv is None else r[: len(views)].contiguous()
        a, b = plain.backproject(rr, views=vv), tab.backproject(rr, views=vv)
        assert torch.equal(a, b), f"{name}: back-projections differ"
        out = torch.ones(g.image_shape, dtype=torch.float32, device="cuda")
        tab.backproject(rr, views=vv, out=out, accumulate=True)
        assert torch.equal(out, a + 1.0) or torch.allclose(out, a + 1.0, rtol=0, atol=1e-6)


@pytest.mark.parametrize("name,g", [CASES[0], CASES[1], CASES[3]])
def test_oslalm_iterations_from_matrix_are_bit_identical(L, name, g):
    import torch
    plain, tab = _pair(L, g)
    rng = np.random.default_rng(11)
    p_true = plain.project(to_dev(synth.pixelize(g, synth.random_ellipse_phantom(3, 0.4 * g.nx * g.dx, 6))))
    counts = rng.poisson(1e4 * np.exp(-to_host(p_true))).clip(min=1)
    y = to_dev(-np.log(counts / 1e4))
    w = to_dev(counts)
    M = 5
    xs = []
    for geom in (plain, tab):
        prob = L.Problem(geom, y, w, beta=2.0 ** 10, delta=1.92e-4, nbr=8, M=M, use_graph=True)
        x = torch.full(g.image_shape, 0.01, dtype=torch.float32, device="cuda")
        prob.init(x)
        prob.iterate(x, 3)
        xs.append((x, prob.cost(x), prob.get_state()))
    assert torch.equal(xs[0][0], xs[1][0])
    assert xs[0][1] == xs[1][1]


def test_matrix_can_be_dropped_and_rebuilt(L):
    import torch
    g = CASES[3][1]
    geom = L.Geometry(g)
    x = to_dev(np.random.default_rng(2).uniform(size=g.image_shape))
    a = geom.project(x)
    n1 = geom.build_matrix()
    b = geom.project(x)
    geom.drop_matrix()
    c = geom.project(x)
    n2 = geom.build_matrix()
    d = geom.project(x)
    assert n1 == n2 and torch.equal(a, b) and torch.equal(a, c) and torch.equal(a, d)


def test_matrix_refused_for_cone_geometry(L):
    geom = L.Geometry(W.tiny_cone())
    with pytest.raises(L.OslalmError, match="2D"):
        geom.build_matrix()
