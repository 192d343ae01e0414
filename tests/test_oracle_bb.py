"""Pins of the oracle's Barzilai-Borwein scaling (supplement Sec. II-A, Eqs.
secant_eq and scale_factor_alpha_k) against what the mathematics fixes:

* on a quadratic data term with one subset, the gradient difference is
  A'WA s exactly, so the oracle's fitted scale must equal s'A'WAs / s'Ds
  computed from the dense matrix (and lie in (0, 1): D majorizes A'WA);
* with M subsets, each subset's gradient difference over one iteration is
  M A_m'W_m A_m s_m exactly, so the scale fitted at the end of an iteration
  must equal sum_m M s_m'A_m'W_m A_m s_m / sum_m s_m'D s_m from the dense
  per-subset matrices and the iterates at which the gradients were taken;
* with rho = 1, no regularizer and no constraint, OS-LALM with BB scaling is
  the textbook diagonally preconditioned Barzilai-Borwein gradient method;
* the constraint alpha <= 1 caps the fit when D does not majorize;
* a fit without positive curvature (s'y <= 0) keeps alpha = 1;
* the scaling changes the path, not the minimiser (M = 1, KKT).

A planted weighting P = I instead of L^-1, a gradient difference from the
wrong pair of iterates, or a missing cap each fail one of these.
"""
import numpy as np
import pytest

from oracle import oslalm as O


def _quadratic(seed=0, m=40, n=12):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0, 1, size=(m, n)) * (rng.uniform(size=(m, n)) < 0.6)
    w = rng.uniform(0.5, 2.0, size=m)
    y = A @ rng.uniform(0, 1, size=n) + 0.05 * rng.normal(size=m)
    return A, w, y


def _data(A, w, y):
    img = lambda v: v.reshape(1, 1, -1)  # noqa: E731
    return O.SubsetData(lambda x, m: A @ x.ravel(), lambda r, m: img(A.T @ r), [y], [w], 1), img


def test_bb_scale_equals_secant_fit_of_the_hessian():
    A, w, y = _quadratic()
    n = A.shape[1]
    H = A.T @ (w[:, None] * A)
    D = A.T @ (w * (A @ np.ones(n)))
    data, img = _data(A, w, y)
    alg = O.OsLalm(data, img(D), beta=0.0, delta=1.0, nbr=4, rho_mode="fixed", rho_fixed=0.5,
                   nonneg=False, bb=True)
    alg.init(img(np.full(n, 0.3)))
    for _ in range(6):
        x0 = alg.x.ravel().copy()
        alg.step()
        s = alg.x.ravel() - x0
        ref = float(s @ H @ s) / float(s @ (D * s))
        assert 0.0 < ref < 1.0
        assert alg.history[-1]["alpha"] == pytest.approx(ref, rel=1e-10)
    # the next x-update used the fitted scale
    assert alg.history[-1]["alpha_used"] == alg.history[-2]["alpha"]


def test_bb_with_rho_one_is_preconditioned_barzilai_borwein_gradient():
    """x_{k+1} = x_k - D^-1 grad l(x_k) / alpha_k, alpha_0 = 1,
    alpha_{k+1} = min(s'y / s'Ds, 1), s = x_{k+1} - x_k, y = grad(x_{k+1}) - grad(x_k)."""
    A, w, y = _quadratic(1)
    n = A.shape[1]
    D = A.T @ (w * (A @ np.ones(n)))
    grad = lambda x: A.T @ (w * (A @ x - y))  # noqa: E731
    data, img = _data(A, w, y)
    alg = O.OsLalm(data, img(D), beta=0.0, delta=1.0, nbr=4, rho_mode="fixed", rho_fixed=1.0,
                   nonneg=False, bb=True)
    x = np.full(n, 0.3)
    alg.init(img(x))
    alpha = 1.0
    for _ in range(8):  # beyond ~10 steps BB's recursion amplifies last-bit differences
        xn = x - grad(x) / (alpha * D)
        s, yk = xn - x, grad(xn) - grad(x)
        alpha = min(float(s @ yk) / float(s @ (D * s)), 1.0)
        x = xn
        alg.step()
        np.testing.assert_allclose(alg.x.ravel(), x, rtol=1e-10, atol=1e-12)


def test_bb_scale_is_capped_at_one():
    A, w, y = _quadratic(2)
    n = A.shape[1]
    H = A.T @ (w[:, None] * A)
    D = 0.05 * (A.T @ (w * (A @ np.ones(n))))  # not a majorizer: the fit exceeds 1
    data, img = _data(A, w, y)
    alg = O.OsLalm(data, img(D), beta=0.0, delta=1.0, nbr=4, rho_mode="fixed", rho_fixed=0.5,
                   nonneg=False, bb=True)
    alg.init(img(np.full(n, 0.3)))
    capped = 0
    for _ in range(8):
        x0 = alg.x.ravel().copy()
        alg.step()
        s = alg.x.ravel() - x0
        ref = float(s @ H @ s) / float(s @ (D * s))
        assert alg.history[-1]["alpha"] == pytest.approx(min(ref, 1.0), rel=1e-10)
        capped += ref > 1.0
    assert capped > 0


def test_bb_without_positive_curvature_keeps_alpha_one():
    A, w, y = _quadratic(3)
    n = A.shape[1]
    D = A.T @ (np.abs(w) * (A @ np.ones(n)))
    data, img = _data(A, -w, y)  # negative weights: y_k = -H s_k, s'y < 0
    alg = O.OsLalm(data, img(D), beta=0.0, delta=1.0, nbr=4, rho_mode="fixed", rho_fixed=0.5,
                   nonneg=False, bb=True)
    alg.init(img(np.full(n, 0.3)))
    for _ in range(4):
        alg.step()
        assert alg.history[-1]["alpha"] == 1.0


def test_bb_changes_the_path_not_the_minimiser():
    A, w, y = _quadratic(4, m=60, n=16)
    n = A.shape[1]
    D = A.T @ (w * (A @ np.ones(n)))
    data, img = _data(A, w, y)
    beta, delta = 0.5, 0.2
    out = []
    for bb in (False, True):
        alg = O.OsLalm(data, img(D), beta=beta, delta=delta, nbr=4, bb=bb)
        alg.init(img(np.full(n, 0.3)))
        alg.run(3000)
        out.append(alg)
    np.testing.assert_allclose(out[1].x, out[0].x, atol=1e-8)
    x = out[1].x
    g = data.At_m(data.w[0] * (data.A_m(x, 0) - data.y[0]), 0) + O.reg_grad(x, beta, delta, 4)
    free = x > 1e-9
    assert np.max(np.abs(g[free])) < 1e-7 * np.abs(data.At_m(data.w[0] * data.y[0], 0)).max()
    assert any(h["alpha_used"] < 1.0 for h in out[1].history)


def test_bb_scale_with_subsets_is_the_per_subset_secant_fit():
    A, w, y = _quadratic(5, m=45, n=12)
    n = A.shape[1]
    M = 3
    rows = [np.arange(m, A.shape[0], M) for m in range(M)]
    img = lambda v: v.reshape(1, 1, -1)  # noqa: E731
    data = O.SubsetData(lambda x, m: A[rows[m]] @ x.ravel(), lambda r, m: img(A[rows[m]].T @ r),
                        [y[r] for r in rows], [w[r] for r in rows], M)
    D = A.T @ (w * (A @ np.ones(n)))
    Hm = [M * A[r].T @ (w[r][:, None] * A[r]) for r in rows]
    alg = O.OsLalm(data, img(D), beta=0.0, delta=1.0, nbr=4, rho_mode="fixed", rho_fixed=0.5, nonneg=False,
                   bb=True)
    alg.init(img(np.full(n, 0.3)))
    at = {alg.order[0]: [alg.x.ravel().copy()]}  # iterates where each subset's gradient was taken
    for k in range(4):
        num = den = 0.0
        for q in range(M):
            alg.step()
            m = alg.order[(alg.j) % M]
            x = alg.x.ravel().copy()
            if m in at:
                sm = x - at[m][-1]
                num += float(sm @ Hm[m] @ sm)
                den += float(sm @ (D * sm))
            at.setdefault(m, []).append(x)
        assert den > 0.0
        assert alg.history[-1]["alpha"] == pytest.approx(min(num / den, 1.0), rel=1e-10)
        assert alg.history[-1]["alpha"] < 1.0
