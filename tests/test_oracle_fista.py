"""Pins of the oracle's inner solver with n > 1 (the constrained denoising
sub-problem of Eq. os_lalm_iterates with h = R + iota_Omega, Sec. IV-A,
solved by n FISTA steps from the previous image):

* n = 1 is the single projected SQS step of the plain method, bit for bit;
* the momentum weights follow the FISTA recursion of Beck & Teboulle;
* with the fixed curvature (omega = 1, a global majorizer of R's Hessian) the
  iterates obey the FISTA bound
      Phi(u_n) - Phi* <= 2 ||x - v*||_L^2 / (n + 1)^2,  L = rho D + D_R,
  where v* = argmin over v >= 0 of Phi, computed independently by scipy's
  bounded L-BFGS-B;
* with the Huber curvature the inner result approaches the same minimiser
  as n grows;
* one-subset OS-LALM with n = 5 reaches the KKT point of the PWLS problem
  that n = 1 reaches.
"""
import math

import numpy as np
import pytest

from oracle import oslalm as O
from oracle import siddon
from paper_1402_4381_gb300 import workloads as W


def _inner_problem(seed=0, shape=(1, 10, 12), beta=2.0, delta=0.1, rho=0.3):
    rng = np.random.default_rng(seed)
    x = np.maximum(rng.normal(0.5, 0.6, size=shape), 0.0)
    D = rng.uniform(0.5, 3.0, size=shape)
    s = rng.normal(0.0, 1.0, size=shape)
    return x, D, s, beta, delta, rho


def _phi(v, x, D, s, beta, delta, rho, nbr):
    z = x - s / (rho * D)
    return O.reg_value(v, beta, delta, nbr) + 0.5 * rho * float(np.sum(D * (v - z) ** 2))


def _phi_grad(v, x, D, s, beta, delta, rho, nbr):
    return O.reg_grad(v, beta, delta, nbr) + s + rho * D * (v - x)


def _minimiser(x, D, s, beta, delta, rho, nbr):
    from scipy.optimize import minimize
    shp = x.shape
    f = lambda v: _phi(v.reshape(shp), x, D, s, beta, delta, rho, nbr)
    g = lambda v: _phi_grad(v.reshape(shp), x, D, s, beta, delta, rho, nbr).ravel()
    r = minimize(f, x.ravel(), jac=g, method="L-BFGS-B", bounds=[(0.0, None)] * x.size,
                 options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12))
    return r.x.reshape(shp), r.fun


def _alg(D, beta, delta, nbr, n, curvature):
    class _NoData:
        M = 1
    return O.OsLalm(_NoData(), D, beta, delta, nbr, curvature=curvature, n_inner=n)


def test_momentum_weights_follow_fista_recursion():
    g = O.fista_momentum(6)
    assert g[0] == 0.0
    tau = 1.0
    for k in range(6):
        tn = (1 + math.sqrt(1 + 4 * tau * tau)) / 2
        assert tn * tn - tn == pytest.approx(tau * tau, rel=1e-14)  # t_{k+1}^2 - t_{k+1} = t_k^2
        assert g[k] == pytest.approx((tau - 1) / tn, rel=1e-15)
        tau = tn
    assert all(0 <= a < b < 1 for a, b in zip(g[1:], g[2:]))


@pytest.mark.parametrize("curvature", ["huber", "max"])
def test_n1_is_the_single_projected_step(curvature):
    x, D, s, beta, delta, rho = _inner_problem(1)
    alg = _alg(D, beta, delta, 8, 1, curvature)
    u = alg.inner(x, s, rho)
    gR = O.reg_grad(x, beta, delta, 8)
    DR = O.reg_curv(x, beta, delta, 8, curvature)
    assert np.array_equal(u, np.maximum(x - (s + gR) / (rho * D + DR), 0.0))


@pytest.mark.parametrize("nbr", [4, 8])
def test_fixed_curvature_fista_bound(nbr):
    x, D, s, beta, delta, rho = _inner_problem(2)
    vstar, fstar = _minimiser(x, D, s, beta, delta, rho, nbr)
    L = rho * D + O.reg_curv(x, beta, delta, nbr, "max")  # constant: omega = 1
    r2 = float(np.sum(L * (x - vstar) ** 2))
    gaps = []
    for n in (1, 2, 3, 5, 8, 13, 21, 34):
        u = _alg(D, beta, delta, nbr, n, "max").inner(x, s, rho)
        assert np.all(u >= 0.0)
        gap = _phi(u, x, D, s, beta, delta, rho, nbr) - fstar
        assert gap <= 2.0 * r2 / (n + 1) ** 2 + 1e-12
        gaps.append(gap)
    assert gaps[-1] < 1e-2 * gaps[0]


def test_huber_curvature_inner_converges_to_minimiser():
    x, D, s, beta, delta, rho = _inner_problem(3)
    vstar, fstar = _minimiser(x, D, s, beta, delta, rho, 8)
    d = [float(np.max(np.abs(_alg(D, beta, delta, 8, n, "huber").inner(x, s, rho) - vstar)))
         for n in (1, 5, 25, 400)]
    assert d[-1] < 2e-6 * max(1.0, float(np.max(np.abs(vstar))))  # the bounded solver's own accuracy
    assert d[-1] < d[2] < d[1] < d[0]


def test_m1_with_five_inner_steps_reaches_the_kkt_point():
    g = W.tiny_fan(n=8, nviews=16, ns=15)
    rng = np.random.default_rng(4)
    xt = np.zeros(g.image_shape)
    xt[0, 2:6, 2:6] = 1.0
    y = siddon.project(g, xt) + 0.05 * rng.normal(size=g.sino_shape)
    w = rng.uniform(0.5, 1.5, size=g.sino_shape)
    data, _ = O.ct_subset_data(g, y, w, 1, siddon)
    D = data.sqs_denominator(g.image_shape)
    xs = []
    for n in (1, 5):
        alg = O.OsLalm(data, D, beta=0.5, delta=0.1, nbr=8, n_inner=n)
        alg.init(np.full(g.image_shape, 0.5))
        alg.run(1500)
        xs.append(alg.x)
    np.testing.assert_allclose(xs[1], xs[0], atol=1e-6)
    x = xs[1]
    grad = data.At_m(data.w[0] * (data.A_m(x, 0) - data.y[0]), 0) + O.reg_grad(x, 0.5, 0.1, 8)
    scale = np.abs(data.At_m(data.w[0] * data.y[0], 0)).max()
    free = x > 1e-9
    assert np.max(np.abs(grad[free])) < 1e-5 * scale
    assert np.min(grad[~free], initial=0.0) > -1e-5 * scale
