"""Pins of the oracle's OS-LALM (oracle/oslalm.py) against what the paper and
the mathematics fix, each by an argument the oracle does not restate:

* the second-order recurrence of Eq. char_poly_qp on the quadratic toy of
  Eq. quad_problem, and the over-damped rate of Eq. over_damp_rate;
* the continuation penalty rho_l equals the critical damping value of
  Eq. critical_value_qp at mu/L = (pi/(2l+2))^2 (Eq. opt_rho_r_qp);
* the (x, u, d) linearized-AL iterates (Eq. general_lal_iterates with the
  closed-form u-update of Eq. lalm_pls_u) give the same x as the (s, x, g)
  iterates, and u + rho d = y (Eq. u_d_identity);
* rho = 1 reduces to the ordered-subsets SQS algorithm (Sec. III-A);
* the regularizer's gradient (finite differences) and its separable surrogate
  (majorizes, tight for an antisymmetric pair);
* D = diag{A'WA1} majorizes A'WA (Sec. IV-A) on a dense A built by clipping;
* M = 1 convergence to the unique minimiser (Theorem 1 with rho >= rho_min):
  continuation and rho = 1 agree and satisfy the KKT conditions; the rho = 1
  cost is monotone.
"""
import math

import numpy as np
import pytest

from dense_ref import dense_A
from oracle import oslalm as O
from oracle import siddon
from paper_1402_4381_gb300 import workloads as W


# ---------------------------------------------------------------- subsets

def test_bit_reversal_power_of_two():
    assert O.bit_reversal_order(8) == [0, 4, 2, 6, 1, 5, 3, 7]
    assert O.bit_reversal_order(4) == [0, 2, 1, 3]
    assert O.bit_reversal_order(2) == [0, 1]
    assert O.bit_reversal_order(1) == [0]


def test_bit_reversal_non_power_of_two_reading():
    assert O.bit_reversal_order(10) == [0, 8, 4, 2, 6, 1, 9, 5, 3, 7]
    for M in range(1, 65):
        order = O.bit_reversal_order(M)
        assert sorted(order) == list(range(M))


def test_subset_views_partition():
    for nv, M in [(984, 24), (180, 10), (984, 12), (7, 3)]:
        allv = np.concatenate([O.subset_views(nv, M, m) for m in range(M)])
        assert sorted(allv.tolist()) == list(range(nv))
        assert all(np.all(O.subset_views(nv, M, m) % M == m) for m in range(M))


# ---------------------------------------------------------------- continuation

def test_rho_l_is_critical_damping_of_estimated_condition():
    """rho_l = rho_c(q) = 2 sqrt(q (1-q)) with q = mu/L = (pi/(2l+2))^2."""
    for l in range(1, 200):
        q = (math.pi / (2 * l + 2)) ** 2
        rc = 2.0 * math.sqrt(q * (1.0 - q))
        assert abs(O.rho_l(l, 0.0) - rc) < 1e-14


def test_rho_l_shape():
    assert O.rho_l(0) == 1.0
    vals = [O.rho_l(l) for l in range(1, 5000)]
    assert all(0 < v <= 1 for v in vals)
    assert all(a >= b for a, b in zip(vals, vals[1:]))
    # pi/(l+1) drops below rho_min = 1e-3 after l ~ 3141
    assert O.rho_l(4000) == 1e-3
    assert O.rho_l(3000) > 1e-3


# ---------------------------------------------------------------- quadratic toy

def _toy(lams, L, rho, x0, n):
    """Oracle LALM (M=1, h=0, y=0) on A = diag(sqrt(lam)), majorizer L I."""
    A = np.diag(np.sqrt(lams))
    data = O.SubsetData(lambda x, m: A @ x, lambda r, m: A.T @ r,
                        [np.zeros(len(lams))], [np.ones(len(lams))], 1)
    alg = O.OsLalm(data, D=np.full(len(lams), L), beta=0.0, delta=1.0, nbr=4,
                   rho_mode="fixed", rho_fixed=rho, nonneg=False)
    alg.init(np.array(x0, dtype=float))
    xs = [alg.x.copy()]
    for _ in range(n):
        alg.step()
        xs.append(alg.x.copy())
    return np.array(xs)


@pytest.mark.parametrize("rho", [1.0, 0.5, 0.2, 0.05, 0.01])
def test_toy_second_order_recurrence(rho):
    """Each eigen-component obeys (1+rho) x_{k+2} - 2(1-q+rho/2) x_{k+1} + (1-q) x_k = 0."""
    L = 1.0
    lams = np.array([0.001, 0.05, 0.3, 0.5, 0.7, 0.99])
    xs = _toy(lams, L, rho, np.ones(6), 60)
    q = lams / L
    res = (1 + rho) * xs[2:] - 2 * (1 - q + rho / 2) * xs[1:-1] + (1 - q) * xs[:-2]
    scale = np.abs(xs[:-2]) + np.abs(xs[1:-1]) + np.abs(xs[2:]) + 1e-300
    assert np.max(np.abs(res) / scale) < 1e-12


def test_toy_overdamped_rate():
    """rho above the critical value: contraction -> r_o(rho) (Eq. over_damp_rate)."""
    L, lam = 1.0, 0.01
    q = lam / L
    rc = 2 * math.sqrt(q * (1 - q))
    for rho in (0.5, 1.0, 3 * rc):
        xs = _toy(np.array([lam]), L, rho, [1.0], 3000)[:, 0]
        ro = (1 - q + rho / 2 + math.sqrt(rho * rho / 4 - q * (1 - q))) / (1 + rho)
        assert abs(xs[-1] / xs[-2] - ro) < 1e-8


def test_toy_critical_and_underdamped():
    """At rho_c the root is double with modulus r_c (Eq. critical_damp_rate);
    below it the iterates oscillate with cos(psi) of Eq. under_damp_cosine_qp."""
    L, lam = 1.0, 0.02
    q = lam / L
    rc = 2 * math.sqrt(q * (1 - q))
    r_c = math.sqrt((1 - q) / (1 + rc))
    xs = _toy(np.array([lam]), L, rc, [1.0], 4000)[:, 0]
    k = len(xs) - 1
    # x_k ~ (a + b k) r_c^k: the ratio tends to r_c (1 + 1/k)
    assert abs(xs[-1] / xs[-2] / r_c - 1) < 2.0 / k
    rho = rc / 4
    xs = _toy(np.array([lam]), L, rho, [1.0], 400)[:, 0]
    cospsi = (1 - q + rho / 2) / math.sqrt((1 + rho) * (1 - q))
    mod = math.sqrt((1 - q) / (1 + rho))
    # a damped cosine obeys x_{k+1} + mod^2 x_{k-1} = 2 mod cos(psi) x_k
    lhs = xs[2:] + mod * mod * xs[:-2]
    rhs = 2 * mod * cospsi * xs[1:-1]
    assert np.max(np.abs(lhs - rhs)) < 1e-12
    assert np.sum(np.diff(np.sign(xs)) != 0) >= 2  # it really oscillates


# ---------------------------------------------------------------- LALM forms

def _small_problem(seed=0, n=12, m=30):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0, 1, size=(m, n)) * (rng.uniform(size=(m, n)) < 0.6)
    w = rng.uniform(0.5, 2.0, size=m)
    xt = rng.uniform(0, 1, size=n) * (rng.uniform(size=n) < 0.7)
    y = A @ xt + 0.05 * rng.normal(size=m)
    return A, w, y


def test_lalm_xud_form_equals_sxg_form():
    """M = 1, fixed rho, h = R + nonnegativity: the (x,u,d) iterates with the
    W^{1/2} substitution give the same x as the oracle's (s,x,g) iterates."""
    A, w, y = _small_problem()
    n = A.shape[1]
    beta, delta, rho = 0.3, 0.2, 0.25
    D = A.T @ (w * (A @ np.ones(n)))
    img = lambda v: v.reshape(1, 1, n)  # noqa: E731  regularizer on a 1 x n image
    data = O.SubsetData(lambda x, m: A @ x.ravel(), lambda r, m: img(A.T @ r), [y], [w], 1)
    alg = O.OsLalm(data, D=img(D), beta=beta, delta=delta, nbr=4, rho_mode="fixed", rho_fixed=rho)
    x0 = np.full(n, 0.5)
    alg.init(img(x0))
    # (x, u, d) iterates on Ab = W^{1/2} A, yb = W^{1/2} y
    sw = np.sqrt(w)
    Ab, yb = sw[:, None] * A, sw * y
    x = x0.copy()
    u = Ab @ x
    d = (yb - u) / rho
    for k in range(25):
        s = rho * Ab.T @ (Ab @ x - u - d)
        gR = O.reg_grad(img(x), beta, delta, 4).ravel()
        DR = O.reg_curv(img(x), beta, delta, 4).ravel()
        x = np.maximum(x - (s + gR) / (rho * D + DR), 0.0)
        u = rho / (rho + 1) * (Ab @ x - d) + yb / (rho + 1)
        d = d - Ab @ x + u
        np.testing.assert_allclose(u + rho * d, yb, atol=1e-12)
        alg.step()
        np.testing.assert_allclose(alg.x.ravel(), x, rtol=1e-11, atol=1e-13)


def test_rho_one_is_os_sqs():
    """With rho = 1 the split gradient drops out: OS-SQS with M subsets."""
    g = W.tiny_fan(n=8, nviews=12, ns=15)
    rng = np.random.default_rng(2)
    y = rng.uniform(0, 3, size=g.sino_shape)
    w = rng.uniform(10, 100, size=g.sino_shape)
    M = 4
    data, views = O.ct_subset_data(g, y, w, M, siddon)
    D = data.sqs_denominator(g.image_shape)
    beta, delta = 5.0, 0.05
    alg = O.OsLalm(data, D, beta, delta, 8, rho_mode="fixed", rho_fixed=1.0)
    x0 = np.full(g.image_shape, 0.2)
    alg.init(x0)
    x = x0.copy()
    order = O.bit_reversal_order(M)
    for j in range(10):
        m = order[j % M]
        grad = M * siddon.backproject(g, w[views[m]] * (siddon.project(g, x, views[m]) - y[views[m]]), views[m])
        x = np.maximum(x - (grad + O.reg_grad(x, beta, delta, 8)) / (D + O.reg_curv(x, beta, delta, 8)), 0)
        alg.step()
        np.testing.assert_allclose(alg.x, x, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- regularizer

@pytest.mark.parametrize("nbr,shape", [(4, (1, 6, 7)), (8, (1, 6, 7)), (6, (3, 4, 5)), (26, (3, 4, 5))])
def test_regularizer_gradient_finite_difference(nbr, shape):
    rng = np.random.default_rng(nbr)
    delta, beta = 0.01, 3.0
    x = rng.normal(0, 0.02, size=shape)
    g = O.reg_grad(x, beta, delta, nbr)
    h = 1e-7
    for idx in [(0, 1, 1), (0, 0, 0), tuple(s - 1 for s in shape), (shape[0] // 2, 2, 3)]:
        e = np.zeros(shape)
        e[idx] = h
        fd = (O.reg_value(x + e, beta, delta, nbr) - O.reg_value(x - e, beta, delta, nbr)) / (2 * h)
        assert abs(fd - g[idx]) < 1e-6 * max(1.0, abs(g[idx]))


def test_hyperbola_closed_forms():
    d = 0.01
    t = np.array([1e-6, 1e-4, 1.0, 10.0])
    np.testing.assert_allclose(O.psi(t[:2], d), t[:2] ** 2 / 2, rtol=1e-3)
    np.testing.assert_allclose(O.psi(t[2:], d) / (d * np.abs(t[2:])), 1.0, rtol=2e-2)
    tt = np.linspace(-0.05, 0.05, 11)
    fd = (O.psi(tt + 1e-8, d) - O.psi(tt - 1e-8, d)) / 2e-8
    np.testing.assert_allclose(O.dpsi(tt, d), fd, rtol=1e-5, atol=1e-9)
    assert np.all(np.diff(O.omega(np.abs(tt[5:]), d)) <= 0)  # psi'(t)/t non-increasing


@pytest.mark.parametrize("nbr,shape", [(8, (1, 6, 7)), (26, (3, 4, 5))])
def test_regularizer_sqs_majorizes(nbr, shape):
    rng = np.random.default_rng(7)
    delta, beta = 0.01, 2.0
    x = rng.normal(0, 0.02, size=shape)
    gR = O.reg_grad(x, beta, delta, nbr)
    DR = O.reg_curv(x, beta, delta, nbr)
    R0 = O.reg_value(x, beta, delta, nbr)
    for k in range(50):
        z = x + rng.normal(0, 0.03, size=shape)
        surr = R0 + np.sum(gR * (z - x)) + 0.5 * np.sum(DR * (z - x) ** 2)
        assert O.reg_value(z, beta, delta, nbr) <= surr + 1e-12


def test_regularizer_sqs_tight_for_antisymmetric_pair():
    """Two pixels, x = const, z = x + (e, -e): R(z) = beta psi(2e) ~ 2 beta e^2 and
    the separable surrogate gives 1/2 sum D_R e^2 = 2 beta e^2: equality to O(e^4)."""
    beta, delta, e = 1.5, 0.01, 1e-6
    x = np.full((1, 1, 2), 0.3)
    DR = O.reg_curv(x, beta, delta, 4)
    z = x + np.array([e, -e]).reshape(1, 1, 2)
    surr = 0.5 * np.sum(DR * (z - x) ** 2)
    assert abs(O.reg_value(z, beta, delta, 4) / surr - 1) < 1e-6


# ---------------------------------------------------------------- majorizer D

@pytest.mark.parametrize("g", [W.tiny_fan(), W.tiny_parallel(), W.tiny_cone()])
def test_sqs_denominator_majorizes(g):
    A = dense_A(g)
    rng = np.random.default_rng(4)
    w = rng.uniform(1, 5, size=A.shape[0])
    H = A.T @ (w[:, None] * A)
    data, _ = O.ct_subset_data(g, np.zeros(g.sino_shape), w.reshape(g.sino_shape), 3, siddon)
    D = data.sqs_denominator(g.image_shape).ravel()
    np.testing.assert_allclose(D, H.sum(axis=1), rtol=1e-12, atol=1e-12)
    for _ in range(20):
        x = rng.normal(size=A.shape[1])
        assert x @ H @ x <= np.sum(D * x * x) * (1 + 1e-12)


# ---------------------------------------------------------------- convergence

def _tiny_ct(seed=0):
    g = W.tiny_fan(n=8, nviews=16, ns=15)
    rng = np.random.default_rng(seed)
    xt = np.zeros(g.image_shape)
    xt[0, 2:6, 2:6] = 1.0
    xt[0, 3, 3] = 2.0
    y = siddon.project(g, xt) + 0.05 * rng.normal(size=g.sino_shape)
    w = rng.uniform(0.5, 1.5, size=g.sino_shape)
    return g, y, w


def _run(g, y, w, mode, n, M=1, rho=1.0):
    data, _ = O.ct_subset_data(g, y, w, M, siddon)
    D = data.sqs_denominator(g.image_shape)
    alg = O.OsLalm(data, D, beta=0.5, delta=0.1, nbr=8, rho_mode=mode, rho_fixed=rho)
    alg.init(np.full(g.image_shape, 0.5))
    costs = [alg.cost()]
    for _ in range(n):
        alg.step()
        costs.append(alg.cost())
    return alg, np.array(costs), data


@pytest.mark.slow
def test_m1_continuation_and_sqs_reach_kkt_point():
    g, y, w = _tiny_ct()
    a_sqs, c_sqs, data = _run(g, y, w, "fixed", 6000)
    a_c, c_c, _ = _run(g, y, w, "continuation", 1500)
    assert np.all(np.diff(c_sqs) <= 1e-12 * abs(c_sqs[0]))  # monotone for rho = 1
    np.testing.assert_allclose(a_c.x, a_sqs.x, atol=2e-7)
    # KKT of min Psi(x) s.t. x >= 0
    x = a_c.x
    grad = data.At_m(data.w[0] * (data.A_m(x, 0) - data.y[0]), 0) + O.reg_grad(x, 0.5, 0.1, 8)
    scale = np.abs(data.At_m(data.w[0] * data.y[0], 0)).max()
    free = x > 1e-9
    assert np.max(np.abs(grad[free])) < 1e-6 * scale
    assert np.min(grad[~free], initial=0.0) > -1e-6 * scale
    assert np.any(~free)  # the constraint is active somewhere
    # continuation reaches the cost plateau faster than rho = 1
    target = c_sqs[-1] + 1e-6 * abs(c_sqs[-1])
    k_c = int(np.argmax(c_c <= target))
    k_s = int(np.argmax(c_sqs <= target))
    assert 0 < k_c < k_s


def test_continuation_restarts_happen():
    g, y, w = _tiny_ct(1)
    alg, _, _ = _run(g, y, w, "continuation", 200)
    restarts = [h["restart"] for h in alg.history]
    assert any(restarts) and not all(restarts)
    ls = [h["l"] for h in alg.history]
    for h0, h1 in zip(alg.history, alg.history[1:]):
        assert h1["l"] == (0 if h1["restart"] else h0["l"] + 1)
        assert h1["rho_used"] == O.rho_l(h0["l"])
