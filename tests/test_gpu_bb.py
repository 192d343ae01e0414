"""GPU parity of the Barzilai-Borwein scaling of the majorizer (supplement
Sec. II-A) through the C ABI: the scale refitted at the end of every
iteration from the subsets' secant pairs, and the images, against the FP64
oracle (2D parallel and fan beam with the oracle's restart decisions
replayed, and a small cone beam), resume, and batches refusing it."""
import numpy as np
import pytest

from gpu_util import COST_RTOL, RMSD_HU_TOL, to_dev, to_host
from oracle import oslalm as O
from oracle import siddon
from paper_1402_4381_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# The scale is a ratio of sums over s_m and y_m, differences of FP32 images
# one iteration apart: each carries ~1e-4 relative rounding on the GPU, so
# the scales agree with the oracle's to about 1e-3.
ALPHA_RTOL = 1e-2


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_4381_gb300 import build, oslalm
    build.build()
    return oslalm


def _oracle(wl, M, x0, replay=None, bb=True):
    scan = wl.make_scan()
    data, _ = O.ct_subset_data(wl.geom, scan["y"].astype(np.float64), scan["w"].astype(np.float64), M, siddon)
    D = data.sqs_denominator(wl.geom.image_shape)
    alg = O.OsLalm(data, D, wl.beta, wl.delta, wl.nbr, bb=bb, replay=replay)
    alg.init(x0.astype(np.float64))
    return alg, scan


def _gpu(L, wl, M, scan, x0, mode="continuation", bb=True):
    geom = L.Geometry(wl.geom)
    prob = L.Problem(geom, to_dev(scan["y"]), to_dev(scan["w"]), beta=wl.beta, delta=wl.delta, nbr=wl.nbr, M=M,
                     rho_mode=mode, bb=bb)
    x = to_dev(x0)
    prob.init(x)
    return geom, prob, x


def _x0(g):
    return np.where(O.roi_mask(g), 0.01, 0.0).astype(np.float32)


@pytest.mark.parametrize("wl,M,iters", [(W.c0_parallel(), 10, 2),
                                        (W.scaled(W.c1_fan(), 96, 120, 111, 6), 6, 3)])
def test_bb_scales_and_images_match_oracle(L, wl, M, iters):
    g = wl.geom
    x0 = _x0(g)
    alg, scan = _oracle(wl, M, x0)
    alg.run(iters * M)
    restarts = [int(h["restart"]) for h in alg.history]
    geom, prob, x = _gpu(L, wl, M, scan, x0, mode="replay")
    prob.set_replay(restarts)
    stats = prob.iterate(x, iters, stats=True)
    a_gpu = np.array([s["alpha"] for s in stats])
    a_ref = np.array([h["alpha"] for h in alg.history])
    assert np.any(a_ref < 1.0)  # the fit is active
    np.testing.assert_allclose(a_gpu, a_ref, rtol=ALPHA_RTOL)
    mask = O.roi_mask(g)
    assert O.rmsd_hu(to_host(x), alg.x, mask) <= RMSD_HU_TOL
    assert abs(prob.cost(x) - alg.cost()) <= COST_RTOL * abs(alg.cost())


def test_bb_cone_matches_oracle(L):
    wl = W.scaled(W.c2_cone(), 40, 30, 56, 5, name_suffix="small", nz=12, nt=14)
    g = wl.geom
    x0 = _x0(g)
    alg, scan = _oracle(wl, 5, x0)
    alg.run(10)
    geom, prob, x = _gpu(L, wl, 5, scan, x0, mode="replay")
    prob.set_replay([int(h["restart"]) for h in alg.history])
    stats = prob.iterate(x, 2, stats=True)
    np.testing.assert_allclose([s["alpha"] for s in stats], [h["alpha"] for h in alg.history], rtol=ALPHA_RTOL)
    assert O.rmsd_hu(to_host(x), alg.x, O.roi_mask(g)) <= RMSD_HU_TOL


def test_bb_resume_keeps_alpha_for_the_next_iteration(L):
    """The scale is part of the saved state, the per-subset secant history is
    not: a resumed run repeats the next iteration bit for bit, then refits."""
    import torch
    wl = W.c0_parallel()
    x0 = _x0(wl.geom)
    scan = wl.make_scan()
    _, p1, x1 = _gpu(L, wl, 10, scan, x0)
    p1.iterate(x1, 2)
    st = p1.get_state()
    assert st["alpha"] != 1.0
    xs = x1.clone()
    p1.iterate(x1, 1)
    _, p2, x2 = _gpu(L, wl, 10, scan, x0)
    p2.set_state(st)
    x2.copy_(xs)
    p2.iterate(x2, 1)
    assert torch.equal(x1, x2)
    assert p2.get_state()["alpha"] == 1.0  # no secant pairs yet after the resume


def test_bb_off_leaves_alpha_at_one(L):
    wl = W.c0_parallel()
    x0 = _x0(wl.geom)
    _, p, x = _gpu(L, wl, 10, wl.make_scan(), x0, bb=False)
    stats = p.iterate(x, 1, stats=True)
    assert all(s["alpha"] == 1.0 for s in stats)


def test_batch_refuses_bb(L):
    wl = W.c0_parallel()
    _, p, _ = _gpu(L, wl, 10, wl.make_scan(), _x0(wl.geom))
    with pytest.raises(L.OslalmError, match="Barzilai"):
        L.Batch([p])
