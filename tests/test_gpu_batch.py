"""Batched OS-LALM (oslalm_batch): several 2D scans of different image
sizes, view counts and numbers of subsets advanced together by persistent
launches.  With the default launch shape every scan is bit-identical to the
same problem iterated alone; other shapes change only summation orders and
agree with the FP64 oracle like the single path; graph replay equals direct
launches; the autotuner restores every scan's image and state."""
import math

import numpy as np
import pytest

from gpu_util import RMSD_HU_TOL, to_dev, to_host
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


def _slices():
    base = W.c1_fan()
    specs = [(64, 96, 4, "fan"), (48, 82, 2, "fan"), (80, 123, 3, "fan"), (32, 41, 1, "fan"), (40, 60, 5, "par")]
    out = []
    for k, (n, nv, M, kind) in enumerate(specs):
        if kind == "par":
            g = synth.Geometry(kind=synth.PAR2D, nx=n, ny=n, dx=3.0, dy=3.0, nviews=nv, angle_start=0.0,
                               angle_span=math.pi, ns=70, ds=2.0)
            wl = W.Workload(f"par{k}", g, "ellipses", 50 + k, 60 + k, 6, 55.0, I0=5e4, sigma=0.0,
                            beta=2.0 ** 10, delta=W.DELTA_10HU, nbr=4, M=M, n_iter=3)
        else:
            wl = W.scaled(base, n, nv, 111, M, name_suffix=f"b{k}")
            wl.phantom, wl.n_ellipses, wl.fov_radius = "ellipses", 6, 200.0
            wl.phantom_seed, wl.noise_seed = 70 + k, 80 + k
            wl.w_dtype = "f16" if k % 2 else "f32"
            wl.d_dtype = "bf16" if k == 2 else "f32"
        scan = wl.make_scan()
        out.append((wl, scan["y"], scan["w"]))
    return out


@pytest.fixture(scope="module")
def slices():
    return _slices()


def _problems(L, slices, mode="continuation", replays=None):
    probs, xs, geoms = [], [], []
    for k, (wl, y, w) in enumerate(slices):
        geom = L.Geometry(wl.geom)
        p = L.Problem(geom, to_dev(y), to_dev(w), beta=wl.beta, delta=wl.delta, nbr=wl.nbr, M=wl.M,
                      rho_mode=mode, w_dtype=wl.w_dtype, d_dtype=wl.d_dtype, use_graph=False)
        if replays is not None:
            p.set_replay(replays[k])
        x = to_dev(np.where(O.roi_mask(wl.geom), 0.01, 0.0).astype(np.float32))
        p.init(x)
        probs.append(p)
        xs.append(x)
        geoms.append(geom)
    return probs, xs, geoms


def test_batch_default_shape_is_bit_identical_to_single(L, slices):
    single, xs1, _g1 = _problems(L, slices)
    for p, x in zip(single, xs1):
        p.iterate(x, 3)
    probs, xs2, _g2 = _problems(L, slices)
    b = L.Batch(probs)
    b.set_shape(0)
    b.iterate(xs2, 2, use_graph=False)
    b.iterate(xs2, 1, use_graph=True)
    for k, (p1, p2) in enumerate(zip(single, probs)):
        assert np.array_equal(to_host(xs1[k]), to_host(xs2[k])), k
        s1, s2 = p1.get_state(), p2.get_state()
        assert np.array_equal(to_host(s1["g"]), to_host(s2["g"])), k
        assert (s1["rho"], s1["l"], s1["j"]) == (s2["rho"], s2["l"], s2["j"]), k


@pytest.mark.parametrize("shape", [1, 2, 3, 4])
def test_batch_other_shapes_match_oracle(L, slices, shape):
    refs, replays = [], []
    for wl, y, w in slices[:3]:
        data, _ = O.ct_subset_data(wl.geom, y.astype(np.float64),
                                   _quant(w, wl.w_dtype), wl.M, siddon)
        D = data.sqs_denominator(wl.geom.image_shape)
        alg = O.OsLalm(data, D, wl.beta, wl.delta, wl.nbr)
        alg.init(np.where(O.roi_mask(wl.geom), 0.01, 0.0))
        alg.run(2 * wl.M)
        refs.append(alg)
        replays.append([int(h["restart"]) for h in alg.history])
    probs, xs, _g = _problems(L, slices[:3], mode="replay", replays=replays)
    b = L.Batch(probs)
    b.set_shape(shape, 2)
    b.iterate(xs, 2)
    for (wl, _, _), alg, x in zip(slices[:3], refs, xs):
        tol = RMSD_HU_TOL if wl.d_dtype == "f32" else 5.0
        assert O.rmsd_hu(to_host(x), alg.x, O.roi_mask(wl.geom)) <= tol


def _quant(w, dtype):
    from test_gpu_oslalm import quantize_pow2
    return quantize_pow2(w, dtype)


def test_batch_graph_equals_direct(L, slices):
    pa, xa, _ga = _problems(L, slices)
    pb, xb, _gb = _problems(L, slices)
    ba, bb = L.Batch(pa), L.Batch(pb)
    ba.set_shape(3)
    bb.set_shape(3)
    ba.iterate(xa, 2, use_graph=True)
    bb.iterate(xb, 2, use_graph=False)
    for k in range(len(slices)):
        assert np.array_equal(to_host(xa[k]), to_host(xb[k])), k


def test_batch_autotune_restores_state(L, slices):
    probs, xs, _g = _problems(L, slices)
    before = [to_host(x) for x in xs]
    states = [p.get_state() for p in probs]
    b = L.Batch(probs)
    ms = b.autotune(xs, probe_iters=1)
    assert len(ms) == len(L.Batch.shapes()) and all(t > 0 for row in ms for t in row)
    shape, bps = b.get_shape()
    assert 0 <= shape < len(ms)
    for k, p in enumerate(probs):
        assert np.array_equal(before[k], to_host(xs[k]))
        s = p.get_state()
        assert np.array_equal(to_host(s["g"]), to_host(states[k]["g"]))
        assert (s["rho"], s["l"], s["j"]) == (states[k]["rho"], states[k]["l"], states[k]["j"])
    b.iterate(xs, 1)


def test_batch_rejects_uninitialised_problem(L, slices):
    wl, y, w = slices[0]
    geom = L.Geometry(wl.geom)
    p = L.Problem(geom, to_dev(y), to_dev(w), beta=wl.beta, delta=wl.delta, nbr=8, M=wl.M)
    with pytest.raises(L.OslalmError) as e:
        L.Batch([p])
    assert e.value.code == -5
