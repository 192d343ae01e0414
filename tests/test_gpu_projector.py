"""GPU parity of the projector pair (through the C ABI) against the FP64
oracle: per-ray forward projections, per-pixel back-projections, the adjoint
identity, the exact-transpose property, edge cases, and sampled views of the
full-size fan-beam scan."""
import dataclasses
import math

import numpy as np
import pytest

from dense_ref import dense_A
from gpu_util import ADJ_TOL, assert_rel_floor, to_dev, to_host
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


def _ragged_fan():
    return synth.Geometry(kind=synth.FAN2D_ARC, nx=37, ny=29, dx=1.7, dy=1.7, nviews=23,
                          angle_start=0.3, angle_span=2 * math.pi, ns=61, ds=1.9, dso=120.0, dsd=200.0)


def _ragged_par():
    return synth.Geometry(kind=synth.PAR2D, nx=45, ny=33, dx=1.1, dy=0.9, nviews=17,
                          angle_start=0.0, angle_span=math.pi, ns=71, ds=0.8, offset_s=0.25)


CASES = [
    ("c0_parallel", W.c0_parallel().geom),
    ("c1_fan_128", W.scaled(W.c1_fan(), 128, 246, 222, 6).geom),
    ("tiny_parallel", W.tiny_parallel()),
    ("tiny_fan", W.tiny_fan()),
    ("ragged_fan", _ragged_fan()),
    ("ragged_parallel", _ragged_par()),
]


def _image(g, seed):
    rng = np.random.default_rng(seed)
    fov = 0.45 * min(g.nx * g.dx, g.ny * g.dy)
    ph = synth.random_ellipse_phantom(seed, fov, 6)
    img = synth.pixelize(g, ph, supersample=2)
    return img + 0.002 * rng.uniform(size=img.shape)


@pytest.mark.parametrize("name,g", CASES)
def test_forward_projection_matches_oracle(L, name, g):
    x = _image(g, 3)
    geom = L.Geometry(g)
    got = to_host(geom.project(to_dev(x)))
    ref = siddon.project(g, x.astype(np.float32).astype(np.float64))
    assert_rel_floor(got, ref, what=f"{name} A x")


@pytest.mark.parametrize("name,g", CASES)
def test_back_projection_matches_oracle(L, name, g):
    r = np.random.default_rng(4).uniform(0.5, 1.5, size=g.sino_shape)
    geom = L.Geometry(g)
    got = to_host(geom.backproject(to_dev(r)))
    ref = siddon.backproject(g, r.astype(np.float32).astype(np.float64))
    assert_rel_floor(got, ref, what=f"{name} A' r")


@pytest.mark.parametrize("name,g", CASES)
def test_adjoint_identity_gpu(L, name, g):
    rng = np.random.default_rng(5)
    x = to_dev(rng.uniform(0, 1, size=g.image_shape))
    r = to_dev(rng.uniform(0, 1, size=g.sino_shape))
    geom = L.Geometry(g)
    ax = to_host(geom.project(x))
    atr = to_host(geom.backproject(r))
    lhs = float(np.sum(ax * to_host(r)))
    rhs = float(np.sum(to_host(x) * atr))
    assert abs(lhs - rhs) <= ADJ_TOL * abs(lhs)


@pytest.mark.parametrize("g", [W.tiny_fan(), W.tiny_parallel(n=7, nviews=9, ns=12), _ragged_par()])
def test_exact_transpose_and_dense_reference(L, g):
    """Column j of the forward projector (A e_j) equals row j of the
    back-projector (A' e_i over all i) bit for bit, and both match the dense
    clipping reference."""
    import torch
    geom = L.Geometry(g)
    npix, nray = int(np.prod(g.image_shape)), int(np.prod(g.sino_shape))
    Af = np.zeros((nray, npix), dtype=np.float32)
    for j in range(npix):
        e = torch.zeros(g.image_shape, dtype=torch.float32, device="cuda")
        e.view(-1)[j] = 1.0
        Af[:, j] = geom.project(e).cpu().numpy().ravel()
    Ab = np.zeros((nray, npix), dtype=np.float32)
    for i in range(nray):
        e = torch.zeros(g.sino_shape, dtype=torch.float32, device="cuda")
        e.view(-1)[i] = 1.0
        Ab[i, :] = geom.backproject(e).cpu().numpy().ravel()
    assert np.array_equal(Af, Ab)
    Ad = dense_A(g)
    np.testing.assert_allclose(Af, Ad, rtol=0, atol=2e-5 * Ad.max())


def test_empty_view_list_and_accumulate(L):
    import torch
    g = W.tiny_fan()
    geom = L.Geometry(g)
    x = torch.ones(g.image_shape, dtype=torch.float32, device="cuda")
    out = torch.full(g.image_shape, 7.0, device="cuda")
    geom.backproject(torch.zeros((0, 1, g.ns), device="cuda"), views=[], out=out)
    assert float(out.abs().max()) == 0.0
    sino = geom.project(x, views=[2, 5])
    assert sino.shape == (2, 1, g.ns)
    ref = siddon.project(g, np.ones(g.image_shape), [2, 5])
    assert_rel_floor(to_host(sino), ref)
    acc = torch.full(g.image_shape, 1.0, device="cuda")
    geom.backproject(sino, views=[2, 5], out=acc, accumulate=True)
    assert_rel_floor(to_host(acc), 1.0 + siddon.backproject(g, ref, [2, 5]))


def test_bad_arguments_raise(L):
    import torch
    g = W.tiny_fan()
    geom = L.Geometry(g)
    with pytest.raises(ValueError):
        geom.project(torch.ones(3, device="cuda"))
    with pytest.raises(L.OslalmError):
        L._check(L.lib().oslalm_project(geom.handle, None, None, None, -1, None), "project")


def test_full_size_fan_sampled_views(L):
    """Full 512x512, 984-view, 888-channel fan beam: every ray of sampled views
    (including the exact quarter turns) and the back-projection of those views."""
    wl = W.c1_fan()
    g = wl.geom
    ph = wl.make_phantom()
    x = synth.pixelize(g, ph, supersample=2)
    views = [0, 1, 123, 246, 492, 615, 738, 983]
    geom = L.Geometry(g)
    got = to_host(geom.project(to_dev(x), views=views))
    ref = siddon.project(g, x.astype(np.float32).astype(np.float64), views)
    assert_rel_floor(got, ref, what="C1 A x (sampled views)")
    r = np.random.default_rng(9).uniform(0.5, 1.5, size=(len(views), 1, g.ns))
    gotb = to_host(geom.backproject(to_dev(r), views=views))
    refb = siddon.backproject(g, r.astype(np.float32).astype(np.float64), views)
    assert_rel_floor(gotb, refb, what="C1 A' r (sampled views)")
