"""Pins of the FP64 warm-start network reference: parameter count (~2 M),
gradients against central finite differences of the loss, the residual
structure (zero output weights give the identity), and the building blocks'
adjoint pairs (pool / upsample)."""
import numpy as np
import pytest

from oracle import cnn_ref as C


def test_parameter_count_about_two_million():
    p = C.init_params(0)
    assert 1.8e6 < C.n_params(p) < 2.1e6


def test_identity_with_zero_output_weights():
    p = C.init_params(1)
    p["out.w"][:] = 0
    x = np.random.default_rng(2).normal(size=(1, 16, 16))
    y, _ = C.forward(p, x)
    np.testing.assert_allclose(y, x, atol=1e-15)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(2, 8, 8, 3))
    b = rng.normal(size=(2, 4, 4, 3))
    assert abs(np.sum(C.pool(a) * b) - np.sum(a * C.pool_bwd(b))) < 1e-12
    assert abs(np.sum(C.up(b) * a) - np.sum(b * C.up_bwd(a))) < 1e-12


@pytest.mark.parametrize("name", ["e0a.w", "e1b.w", "b3a.b", "d2a.w", "d0b.w", "out.w", "out.b"])
def test_gradients_match_finite_differences(name):
    rng = np.random.default_rng(4)
    p = C.init_params(5)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0, 0.05, size=p[k].shape)
    p["out.w"] = rng.normal(0, 0.3, size=(32,))
    x = rng.normal(size=(1, 16, 16))
    t = rng.normal(size=(1, 16, 16))
    _, g, _ = C.loss_and_grads(p, x, t)
    flat = p[name].reshape(-1)
    idx = rng.choice(flat.size, size=min(4, flat.size), replace=False)
    for i in idx:
        h = 1e-6 * max(1.0, abs(flat[i]))
        old = flat[i]
        flat[i] = old + h
        lp = C.loss_and_grads(p, x, t)[0]
        flat[i] = old - h
        lm = C.loss_and_grads(p, x, t)[0]
        flat[i] = old
        fd = (lp - lm) / (2 * h)
        an = g[name].reshape(-1)[i]
        assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (name, i, fd, an)


def test_bf16_rounding_ties_to_even_and_matches_torch():
    import torch
    ulp = 2.0 ** -7  # BF16 spacing in [1, 2)
    vals = np.array([1 + ulp / 2, 1 + 1.5 * ulp, 1 + 0.49 * ulp, -3.0 - 0.51 * 2 * ulp, 65504.0, 1e-30, 0.0])
    got = C.bf16(vals)
    assert got[0] == 1.0 and got[1] == 1 + 2 * ulp and got[2] == 1.0
    assert got[3] == -3.0 - 2 * ulp  # spacing 2^-6 in [2, 4)
    r = np.random.default_rng(0).normal(0, 10, size=4096)
    ref = torch.as_tensor(r.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(C.bf16(r), ref)


def test_bf16_storage_model_error_stays_below_gpu_bound():
    """The precision floor the GPU gradient check allows (0.25 relative L2)
    holds for the storage model itself, and the identity rounding gives the
    exact reference back."""
    rng = np.random.default_rng(7)
    p = C.init_params(3)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0, 0.05, size=p[k].shape)
    p["out.w"] = rng.normal(0, 0.2, size=(32,))
    x = rng.uniform(0, 2, size=(1, 16, 24))
    t = x + rng.normal(0, 0.3, size=x.shape)
    l0, g0, y0 = C.loss_and_grads(p, x, t)
    li, gi, yi = C.loss_and_grads(p, x, t, q=lambda a: a)
    assert l0 == li and all(np.array_equal(g0[k], gi[k]) for k in g0)
    lq, gq, yq = C.loss_and_grads(p, x, t, q=C.bf16)
    assert np.linalg.norm(yq - y0) <= 5e-2 * np.linalg.norm(y0 - x)
    for k in g0:
        if k != "out.b":
            assert np.linalg.norm(gq[k] - g0[k]) <= 0.25 * np.linalg.norm(g0[k]), k
