"""GPU warm-start network (BF16 tensor-core kernels, FP32 accumulation)
against the FP64 reference: forward output, loss and every parameter
gradient, parameter exchange, and that training lowers the loss.

Tolerance (derived from the arithmetic): activations and weights are rounded
to BF16 (8-bit significand, relative 2^-9) at every layer of a 14-layer
network, so outputs and gradients agree to a few percent in relative L2
norm: 5e-2 for the output correction and 1e-1 for each gradient tensor."""
import numpy as np
import pytest

from oracle import cnn_ref as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_4381_gb300 import build, oslalm
    build.build()
    return oslalm


def _params(seed=3):
    rng = np.random.default_rng(seed)
    p = C.init_params(seed)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0, 0.05, size=p[k].shape)
    p["out.w"] = rng.normal(0, 0.2, size=(32,))
    return p


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_param_exchange_roundtrip(L):
    net = L.WarmStartNet(1, 16, 16, seed=1)
    p = _params()
    flat = L.cnn_flatten(p)
    net.set_params(flat)
    back = net.get_params()
    assert np.array_equal(back, flat)
    assert flat.size == C.n_params(p) == L.WarmStartNet.param_count()


@pytest.mark.parametrize("shape", [(2, 32, 32), (1, 24, 40)])
def test_forward_and_gradients_match_fp64(L, shape):
    import torch
    n, h, w = shape
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 2, size=shape)
    t = x + rng.normal(0, 0.3, size=shape)
    p = _params()
    net = L.WarmStartNet(n, h, w, seed=0)
    net.set_params(L.cnn_flatten(p))
    xd = torch.as_tensor(x.astype(np.float32), device="cuda")
    td = torch.as_tensor(t.astype(np.float32), device="cuda")
    y = net.forward(xd, 1.0).cpu().numpy().astype(np.float64)
    loss_ref, g_ref, y_ref = C.loss_and_grads(p, x.astype(np.float32).astype(np.float64), t.astype(np.float32))
    assert _rel(y - x, y_ref - x) < 5e-2
    loss, g = net.gradients(xd, td, 1.0)
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    gd = L.cnn_unflatten(g)
    for name in g_ref:
        assert _rel(gd[name].astype(np.float64), g_ref[name]) < 1e-1, name


def test_scale_is_applied(L):
    import torch
    net = L.WarmStartNet(1, 16, 16, seed=2)
    x = torch.rand(1, 16, 16, device="cuda") * 0.02
    y1 = net.forward(x, 50.0).clone()
    p = net.get_params()
    net2 = L.WarmStartNet(1, 16, 16, seed=9)
    net2.set_params(p)
    y2 = net2.forward(x * 50.0, 1.0) / 50.0
    np.testing.assert_allclose(y1.cpu().numpy(), y2.cpu().numpy(), rtol=2e-2, atol=2e-4)


def test_training_lowers_loss(L):
    """Learning to remove a fixed pattern from noisy images."""
    import torch
    n, h, w = 4, 32, 32
    g = torch.Generator(device="cuda").manual_seed(0)
    yy, xx = torch.meshgrid(torch.arange(h, device="cuda"), torch.arange(w, device="cuda"), indexing="ij")
    clean = ((xx - 16) ** 2 + (yy - 16) ** 2 < 100).float()[None].repeat(n, 1, 1)
    net = L.WarmStartNet(n, h, w, seed=4)
    losses = []
    for it in range(120):
        noisy = clean + 0.3 * torch.randn(n, h, w, device="cuda", generator=g)
        losses.append(net.train_step(noisy, clean, 1.0, 1e-3))
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10])
