"""GPU parity of the OS-LALM path (through the C ABI) against the FP64 oracle:
the SQS denominator, the cost, whole trajectories with the deterministic
downward continuation (free run and with the oracle's restart decisions
replayed), fixed-rho runs, graph replay, resume, odd/uneven subsets, the
reduced-precision storage form and the full-size fan-beam configuration."""
import math

import numpy as np
import pytest

from gpu_util import COST_RTOL, HU, RMSD_HU_TOL, assert_rel_floor, to_dev, to_host
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


def quantize_pow2(a, dtype):
    """Storage rule of the reduced-precision form: power-of-two scale
    s = 2^k, k minimal with max|a| <= 32768 s, then round a/s to nearest."""
    a = np.asarray(a, dtype=np.float32)
    if dtype == "f32":
        return a.astype(np.float64)
    mx = float(np.max(np.abs(a)))
    s = 1.0
    if mx > 0:
        m, e = np.frexp(np.float32(mx))
        k = int(e) - 16 if m == 0.5 else int(e) - 15
        s = 2.0 ** k
    q = (a / np.float32(s)).astype(np.float32)
    if dtype == "f16":
        q = q.astype(np.float16).astype(np.float64)
    else:  # bf16: round to nearest even on the upper 16 bits
        b = q.view(np.uint32).astype(np.uint64)
        b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
        q = b.astype(np.uint32).view(np.float32).astype(np.float64)
    return q * s


def initial_image(g):
    mask = O.roi_mask(g)
    return np.where(mask, 0.01, 0.0).astype(np.float32)


class Case:
    def __init__(self, wl, M=None, n_scan_views=None):
        self.wl = wl
        self.g = wl.geom
        self.M = M or wl.M
        scan = wl.make_scan()
        self.y = scan["y"]
        self.w = scan["w"]
        self.x0 = initial_image(self.g)
        self.mask = O.roi_mask(self.g)

    def oracle(self, mode="continuation", rho_fixed=1.0, w_dtype="f32", replay=None):
        wq = quantize_pow2(self.w, w_dtype)
        data, _ = O.ct_subset_data(self.g, self.y.astype(np.float64), wq, self.M, siddon)
        D = data.sqs_denominator(self.g.image_shape)
        alg = O.OsLalm(data, D, self.wl.beta, self.wl.delta, self.wl.nbr, rho_mode=mode,
                       rho_fixed=rho_fixed, replay=replay)
        alg.init(self.x0.astype(np.float64))
        return alg

    def gpu(self, L, mode="continuation", rho_fixed=1.0, w_dtype="f32", d_dtype="f32", use_graph=True):
        geom = L.Geometry(self.g)
        prob = L.Problem(geom, to_dev(self.y), to_dev(self.w), beta=self.wl.beta, delta=self.wl.delta,
                         nbr=self.wl.nbr, M=self.M, rho_mode=mode, rho_fixed=rho_fixed, w_dtype=w_dtype,
                         d_dtype=d_dtype, use_graph=use_graph)
        x = to_dev(self.x0)
        prob.init(x)
        return geom, prob, x


def rmsd_hu(a, b, mask):
    return O.rmsd_hu(a, b, mask)


# ---------------------------------------------------------------- C0 (128^2 parallel, M = 10)

@pytest.fixture(scope="module")
def c0():
    return Case(W.c0_parallel())


@pytest.fixture(scope="module")
def c0_oracle_run(c0):
    alg = c0.oracle()
    snaps = {}
    for k in range(1, c0.wl.n_iter + 1):
        alg.run(c0.M)
        if k in (1, 5, c0.wl.n_iter):
            snaps[k] = alg.x.copy()
    return alg, snaps


def test_c0_denominator_and_cost(L, c0):
    _, prob, x = c0.gpu(L)
    alg = c0.oracle()
    assert_rel_floor(to_host(prob.denominator()), alg.D, what="D = A'WA1")
    c_gpu = prob.cost(x)
    c_ref = alg.cost(c0.x0.astype(np.float64))
    assert abs(c_gpu - c_ref) <= COST_RTOL * abs(c_ref)
    # the first subset gradient and the split gradient; zeta = M A'W(Ax - y) is
    # formed from residuals Ax - y that cancel most of Ax, so its FP32 error
    # is ~1e-6 |Ax| / |Ax - y| relative: allow 1e-4 with a 1e-2 floor
    st = prob.get_state()
    assert_rel_floor(to_host(st["zeta"]), alg.zeta, rtol=1e-4, floor=1e-2, what="zeta0")
    assert np.array_equal(to_host(st["zeta"]), to_host(st["g"]))


def test_c0_full_gradient(L, c0):
    """oslalm_gradient = A'W(Ax - y) + grad R(x) (Sec. IV, Eq. ct_recon) against
    the oracle's, at an image with edges (the regularizer is far from inert)."""
    geom = L.Geometry(c0.g)
    beta = 2.0 ** 24
    prob = L.Problem(geom, to_dev(c0.y), to_dev(c0.w), beta=beta, delta=c0.wl.delta, nbr=c0.wl.nbr, M=c0.M)
    scan = c0.wl.make_scan()
    xt = synth.pixelize(c0.g, scan["phantom"], supersample=2).astype(np.float32)
    gr = to_host(prob.gradient(to_dev(xt)))
    data, _ = O.ct_subset_data(c0.g, c0.y.astype(np.float64), c0.w.astype(np.float64), c0.M, siddon)
    ref = sum(data.At_m(data.w[m] * (data.A_m(xt.astype(np.float64), m) - data.y[m]), m) for m in range(c0.M))
    ref = ref + O.reg_grad(xt.astype(np.float64), beta, c0.wl.delta, c0.wl.nbr)
    # the data term is a sum of residuals that cancel most of Ax (FP32 error
    # ~1e-6 |Ax| / |Ax - y|): 1e-4 relative with a 1e-2 floor, as for zeta
    assert_rel_floor(gr, ref, rtol=1e-4, floor=1e-2, what="PWLS gradient")
    assert np.abs(O.reg_grad(xt.astype(np.float64), beta, c0.wl.delta, c0.wl.nbr)).max() > 0.05 * np.abs(ref).max()


def test_c0_continuation_trajectory(L, c0, c0_oracle_run):
    alg, snaps = c0_oracle_run
    ref_restarts = [int(h["restart"]) for h in alg.history]
    # free run
    _, prob, x = c0.gpu(L)
    stats = []
    xs = {}
    for k in range(1, c0.wl.n_iter + 1):
        stats += prob.iterate(x, 1, stats=True)
        if k in snaps:
            xs[k] = to_host(x)
    gpu_restarts = [int(s["restart"]) for s in stats]
    first_diff = next((i for i, (a, b) in enumerate(zip(gpu_restarts, ref_restarts)) if a != b), None)
    # the restart decision is a sign test: a flip is only legitimate where xi is tiny
    xis = np.array([h["xi"] for h in alg.history])
    if first_diff is not None:
        assert abs(xis[first_diff]) < 1e-3 * np.median(np.abs(xis)), (first_diff, xis[first_diff])
        check = [k for k in xs if k * c0.M <= first_diff]
    else:
        check = list(xs)
    assert check, f"the first restart decisions differ at subset-iteration {first_diff}: no free-run snapshot"
    for k in check:
        assert rmsd_hu(xs[k], snaps[k], c0.mask) <= RMSD_HU_TOL, k
    for s, h in zip(stats[: len(check) * c0.M], alg.history):
        assert abs(s["rho_used"] - h["rho_used"]) <= 1e-12
    # replay of the oracle's restart decisions: parity at every snapshot
    _, prob2, x2 = c0.gpu(L, mode="replay")
    prob2.set_replay(ref_restarts)
    done = 0
    for k in sorted(snaps):
        prob2.iterate(x2, k - done)
        done = k
        r = rmsd_hu(to_host(x2), snaps[k], c0.mask)
        assert r <= RMSD_HU_TOL, (k, r)
    c_gpu = prob2.cost(x2)
    c_ref = alg.cost()
    assert abs(c_gpu - c_ref) <= COST_RTOL * abs(c_ref)


@pytest.mark.parametrize("rho", [1.0, 0.2])
def test_c0_fixed_rho(L, c0, rho):
    alg = c0.oracle(mode="fixed", rho_fixed=rho)
    alg.run(5 * c0.M)
    _, prob, x = c0.gpu(L, mode="fixed", rho_fixed=rho)
    prob.iterate(x, 5)
    assert rmsd_hu(to_host(x), alg.x, c0.mask) <= RMSD_HU_TOL
    assert abs(prob.cost(x) - alg.cost()) <= COST_RTOL * abs(alg.cost())


def test_graph_replay_equals_direct_launches(L, c0):
    _, p1, x1 = c0.gpu(L, use_graph=True)
    _, p2, x2 = c0.gpu(L, use_graph=False)
    p1.iterate(x1, 3)
    p2.iterate(x2, 3)
    assert np.array_equal(to_host(x1), to_host(x2))
    s1, s2 = p1.get_state(), p2.get_state()
    assert np.array_equal(to_host(s1["g"]), to_host(s2["g"]))
    assert (s1["rho"], s1["l"], s1["j"]) == (s2["rho"], s2["l"], s2["j"])


def test_resume_is_bit_exact(L, c0):
    import torch
    _, p, x = c0.gpu(L)
    p.iterate(x, 2)
    st = p.get_state()
    x_mid = x.clone()
    p.iterate(x, 3)
    x_a = to_host(x)
    _, q, y = c0.gpu(L)
    y.copy_(x_mid)
    q.set_state(st)
    q.iterate(y, 3)
    assert np.array_equal(x_a, to_host(y))
    torch.cuda.synchronize()


def test_fp16_storage_form_error(L, c0, c0_oracle_run):
    """Reduced-precision storage (W and D in FP16 with power-of-two scales):
    error against the FP64 oracle, reported and bounded."""
    alg, snaps = c0_oracle_run
    k = 5
    _, prob, x = c0.gpu(L, mode="replay", w_dtype="f16", d_dtype="f16")
    prob.set_replay([int(h["restart"]) for h in alg.history])
    prob.iterate(x, k)
    err = rmsd_hu(to_host(x), snaps[k], c0.mask)
    print(f"fp16 W/D storage: RMSD to FP64 oracle after {k} iterations = {err:.4f} HU")
    assert err < 5.0
    # the stored D is the FP16 rounding of the FP32 one
    _, pf, _ = c0.gpu(L)
    d32 = to_host(pf.denominator())
    d16 = to_host(prob.denominator())
    np.testing.assert_allclose(d16, quantize_pow2(d32, "f16"), rtol=2e-3, atol=0)


# ---------------------------------------------------------------- odd / uneven subsets, small fan

def _small_fan(nviews=50, M=7):
    wl = W.scaled(W.c1_fan(), 64, nviews, 96, M, name_suffix="odd")
    return Case(wl)


@pytest.mark.parametrize("nviews,M", [(50, 7), (48, 1), (30, 30), (41, 4)])
def test_uneven_and_odd_subsets(L, nviews, M):
    case = _small_fan(nviews, M)
    alg = case.oracle()
    alg.run(3 * M)
    _, prob, x = case.gpu(L, mode="replay")
    prob.set_replay([int(h["restart"]) for h in alg.history])
    stats = prob.iterate(x, 3, stats=True)
    assert len(stats) == 3 * M
    assert [s["subset"] for s in stats] == [O.bit_reversal_order(M)[(j + 1) % M] for j in range(3 * M)]
    assert rmsd_hu(to_host(x), alg.x, case.mask) <= RMSD_HU_TOL
    for s, h in zip(stats, alg.history):
        assert s["restart"] == h["restart"] and s["l"] == h["l"]
        if abs(h["xi"]) > 1e-6 * max(1.0, max(abs(q["xi"]) for q in alg.history)):
            assert s["xi"] == pytest.approx(h["xi"], rel=2e-3)


def test_errors_are_reported(L, c0):
    import torch
    geom = L.Geometry(c0.g)
    y, w = to_dev(c0.y), to_dev(c0.w)
    with pytest.raises(L.OslalmError):
        L.Problem(geom, y, w, beta=1.0, delta=1e-3, nbr=5, M=10)
    with pytest.raises(L.OslalmError):
        L.Problem(geom, y, w, beta=1.0, delta=1e-3, nbr=8, M=0)
    p = L.Problem(geom, y, w, beta=1.0, delta=1e-3, nbr=8, M=10)
    x = torch.zeros(c0.g.image_shape, device="cuda")
    with pytest.raises(L.OslalmError) as e:
        p.iterate(x, 1)
    assert e.value.code == -5


# ---------------------------------------------------------------- full-size fan beam (bench configuration)

def test_full_size_fan_first_iterations(L):
    """512^2 fan beam, 984 views x 888 channels, M = 24: five full iterations
    (120 subset-iterations, the oracle's restart decisions replayed) in FP32
    storage against the oracle after iterations 1 and 5, then the benchmark's
    FP16-storage form against the same oracle."""
    wl = W.c1_fan()
    case = Case(wl)
    alg = case.oracle(mode="fixed", rho_fixed=1.0)
    D_ref = alg.D
    c_ref0 = alg.cost(case.x0.astype(np.float64))
    alg_c = O.OsLalm(alg.data, D_ref, wl.beta, wl.delta, wl.nbr)
    alg_c.init(case.x0.astype(np.float64))
    snaps = {}
    for k in range(1, 6):
        alg_c.run(wl.M)
        if k in (1, 5):
            snaps[k] = (alg_c.x.copy(), alg_c.cost())
    restarts = [int(h["restart"]) for h in alg_c.history]
    _, prob, x = case.gpu(L, mode="replay")
    assert_rel_floor(to_host(prob.denominator()), D_ref, what="C1 D")
    assert abs(prob.cost(x) - c_ref0) <= COST_RTOL * abs(c_ref0)
    prob.set_replay(restarts)
    _, p16, x16 = case.gpu(L, mode="replay", w_dtype="f16", d_dtype="f16")
    p16.set_replay(restarts)
    done = 0
    for k in (1, 5):
        prob.iterate(x, k - done)
        p16.iterate(x16, k - done)
        done = k
        xr, cr = snaps[k]
        r32 = rmsd_hu(to_host(x), xr, case.mask)
        r16 = rmsd_hu(to_host(x16), xr, case.mask)
        c32 = prob.cost(x)
        print(f"C1 after {k} iterations: RMSD to FP64 oracle {r32:.4f} HU (FP32 storage), {r16:.4f} HU "
              f"(FP16 W and D); cost rel diff {abs(c32 - cr) / abs(cr):.2e}")
        assert r32 <= RMSD_HU_TOL, (k, r32)
        assert abs(c32 - cr) <= COST_RTOL * abs(cr), k
        assert r16 < 2.0, (k, r16)
