"""GPU parity of the 3D cone-beam path (flat detector) against the FP64
oracle: forward projections per ray, back-projections per voxel, the adjoint
identity, the exact-transpose property, OS-LALM with the 26-neighbour
regularizer and BF16 weights, and sampled views of the full-size scan."""
import numpy as np
import pytest

from gpu_util import ADJ_TOL, COST_RTOL, RMSD_HU_TOL, assert_rel_floor, to_dev, to_host
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


def small_cone(nx=40, nz=12, nviews=30, ns=56, nt=14, M=5):
    return W.scaled(W.c2_cone(), nx, nviews, ns, M, name_suffix="small", nz=nz, nt=nt)


def small_helical(nx=40, nz=16, nviews=60, ns=56, nt=14, M=5):
    return W.scaled(W.c2_helical(), nx, nviews, ns, M, name_suffix="small", nz=nz, nt=nt)


CASES = [("small", small_cone().geom), ("ragged", small_cone(nx=37, nz=9, nviews=17, ns=45, nt=11).geom),
         ("tiny", W.tiny_cone()), ("helical", small_helical().geom), ("tiny_helical", W.tiny_helical())]


def _volume(g, seed):
    ph = synth.random_ellipse_phantom(seed, 0.4 * g.nx * g.dx, 6, three_d=True, z_half=g.nz * g.dz / 2)
    img = synth.pixelize(g, ph, supersample=2)
    return img + 0.002 * np.random.default_rng(seed).uniform(size=img.shape)


@pytest.mark.parametrize("name,g", CASES)
def test_cone_forward_matches_oracle(L, name, g):
    x = _volume(g, 3)
    geom = L.Geometry(g)
    got = to_host(geom.project(to_dev(x)))
    ref = siddon.project(g, x.astype(np.float32).astype(np.float64))
    assert_rel_floor(got, ref, what=f"cone {name} A x")


@pytest.mark.parametrize("name,g", CASES)
def test_cone_backprojection_matches_oracle(L, name, g):
    r = np.random.default_rng(4).uniform(0.5, 1.5, size=g.sino_shape)
    geom = L.Geometry(g)
    got = to_host(geom.backproject(to_dev(r)))
    ref = siddon.backproject(g, r.astype(np.float32).astype(np.float64))
    assert_rel_floor(got, ref, what=f"cone {name} A' r")


@pytest.mark.parametrize("name,g", CASES)
def test_cone_adjoint(L, name, g):
    rng = np.random.default_rng(5)
    x = to_dev(rng.uniform(0, 1, size=g.image_shape))
    r = to_dev(rng.uniform(0, 1, size=g.sino_shape))
    geom = L.Geometry(g)
    lhs = float(np.sum(to_host(geom.project(x)) * to_host(r)))
    rhs = float(np.sum(to_host(x) * to_host(geom.backproject(r))))
    assert abs(lhs - rhs) <= ADJ_TOL * abs(lhs)


@pytest.mark.parametrize("g", [W.tiny_cone(n=6, nz=3, nviews=5, ns=11, nt=5),
                               W.tiny_helical(n=6, nz=4, nviews=8, ns=11, nt=5)])
def test_cone_exact_transpose(L, g):
    import torch
    geom = L.Geometry(g)
    npix, nray = int(np.prod(g.image_shape)), int(np.prod(g.sino_shape))
    Af = np.zeros((nray, npix), dtype=np.float32)
    for j in range(npix):
        e = torch.zeros(g.image_shape, device="cuda")
        e.view(-1)[j] = 1.0
        Af[:, j] = geom.project(e).cpu().numpy().ravel()
    Ab = np.zeros((nray, npix), dtype=np.float32)
    for i in range(nray):
        e = torch.zeros(g.sino_shape, device="cuda")
        e.view(-1)[i] = 1.0
        Ab[i] = geom.backproject(e).cpu().numpy().ravel()
    assert np.abs(Af).sum() > 0
    assert np.array_equal(Af, Ab)


@pytest.mark.parametrize("orbit", ["circular", "helical"])
def test_cone_oslalm_matches_oracle(L, orbit):
    """26-neighbour hyperbola, BF16 storage of W (the oracle consumes the same
    quantized weights), FP32 D; 2 iterations with the oracle's restarts."""
    from test_gpu_oslalm import quantize_pow2
    wl = small_cone(M=5) if orbit == "circular" else small_helical(M=5)
    g = wl.geom
    scan = wl.make_scan()
    y, w = scan["y"], scan["w"]
    mask = O.roi_mask(g)
    x0 = np.where(mask, 0.01, 0.0).astype(np.float32)
    wq = quantize_pow2(w, "bf16")
    data, _ = O.ct_subset_data(g, y.astype(np.float64), wq, wl.M, siddon)
    D = data.sqs_denominator(g.image_shape)
    alg = O.OsLalm(data, D, wl.beta, wl.delta, 26)
    alg.init(x0.astype(np.float64))
    c0 = alg.cost()
    alg.run(2 * wl.M)
    geom = L.Geometry(g)
    prob = L.Problem(geom, to_dev(y), to_dev(w), beta=wl.beta, delta=wl.delta, nbr=26, M=wl.M,
                     rho_mode="replay", w_dtype="bf16")
    prob.set_replay([int(h["restart"]) for h in alg.history])
    x = to_dev(x0)
    prob.init(x)
    assert_rel_floor(to_host(prob.denominator()), D, what="cone D")
    assert abs(prob.cost(x) - c0) <= COST_RTOL * abs(c0)
    prob.iterate(x, 2)
    assert O.rmsd_hu(to_host(x), alg.x, mask) <= RMSD_HU_TOL
    assert abs(prob.cost(x) - alg.cost()) <= COST_RTOL * abs(alg.cost())


def test_cone_full_size_sampled_view(L):
    """512 x 512 x 128 volume, 888 x 64 flat detector: every ray of one view
    (oracle) and the back-projection of a few detector rows of another."""
    wl = W.c2_cone()
    g = wl.geom
    ph = wl.make_phantom()
    x = synth.pixelize(g, ph, supersample=1).astype(np.float32)
    geom = L.Geometry(g)
    got = to_host(geom.project(to_dev(x), views=[123]))
    ref = siddon.project(g, x.astype(np.float64), [123])
    assert_rel_floor(got, ref, what="C2 A x (view 123)")
    r = np.zeros((1, g.nt, g.ns), dtype=np.float32)
    r[0, [0, 31, 63], :] = np.random.default_rng(1).uniform(0.5, 1.5, size=(3, g.ns))
    gotb = to_host(geom.backproject(to_dev(r), views=[500]))
    refb = siddon.backproject(g, r.astype(np.float64), [500])
    # a single-view, three-row back-projection gives each voxel one or two
    # (ray, voxel) lengths, each carrying ~2^-23 L of FP32 rounding: voxels
    # below 2e-2 of the maximum are compared at 1e-5 x 2e-2 x max absolutely
    assert_rel_floor(gotb, refb, floor=2e-2, what="C2 A' r (view 500)")
