"""FP64 reference of the warm-start network (TEST INFRASTRUCTURE: gradient
checks of the CUDA training kernels).

The paper has no network; the warm-start form maps the FBP image to an
estimate of the converged PWLS image.  Architecture (reading of "4-level
encoder/decoder, 32 base channels, 3x3 convs, ReLU, ~2M params"):

  e0a 1->32, e0b 32->32 | pool | e1a 32->64, e1b 64->64 | pool |
  e2a 64->128, e2b 128->128 | pool | b3a 128->256, b3b 256->256 |
  up, concat e2b -> d2a 384->128, d2b 128->128 | up, concat e1b ->
  d1a 192->64, d1b 64->64 | up, concat e0b -> d0a 96->32, d0b 32->32 |
  out 1x1 32->1, plus the input (residual)

3x3 convolutions with zero padding, bias and ReLU; 2x2 average pooling;
nearest-neighbour 2x upsampling; concatenation puts the upsampled tensor
first and the skip second.  Tensors are NHWC; weights [cout][ky][kx][cin].
Loss: mean squared error over all pixels.
"""
import numpy as np

LAYERS = [  # name, cin, cout
    ("e0a", 1, 32), ("e0b", 32, 32), ("e1a", 32, 64), ("e1b", 64, 64), ("e2a", 64, 128), ("e2b", 128, 128),
    ("b3a", 128, 256), ("b3b", 256, 256), ("d2a", 384, 128), ("d2b", 128, 128), ("d1a", 192, 64),
    ("d1b", 64, 64), ("d0a", 96, 32), ("d0b", 32, 32),
]


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    p = {}
    for name, cin, cout in LAYERS:
        p[name + ".w"] = rng.normal(0, np.sqrt(2.0 / (9 * cin)), size=(cout, 3, 3, cin))
        p[name + ".b"] = np.zeros(cout)
    p["out.w"] = rng.normal(0, 0.01, size=(32,))
    p["out.b"] = np.zeros(1)
    return p


def n_params(p):
    return sum(v.size for v in p.values())


def conv3x3(x, w, b):
    """x [N,H,W,Ci], w [Co,3,3,Ci] -> [N,H,W,Co], zero padding."""
    N, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((N, H, W, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("nhwc,oc->nhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    return out + b


def conv3x3_bwd(x, w, dy):
    """Gradients of conv3x3 w.r.t. x, w and b given dy."""
    N, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("nhwo,nhwc->oc", dy, xp[:, ky:ky + H, kx:kx + W, :])
            dxp[:, ky:ky + H, kx:kx + W, :] += np.einsum("nhwo,oc->nhwc", dy, w[:, ky, kx, :])
    return dxp[:, 1:-1, 1:-1, :], dw, dy.sum(axis=(0, 1, 2))


def pool(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) * 0.25


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(dy):
    N, H, W, C = dy.shape
    return dy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64:
    the storage precision model used to check BF16 training kernels."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    b = a32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(a):
    return a


def forward(p, x, q=None):
    """x [N,H,W] -> prediction [N,H,W] and the activations cache.

    q: optional rounding applied where a reduced-precision implementation
    stores a tensor (input image, conv weights, every activation and pooled
    tensor); the default is exact FP64."""
    q = q or _ident
    c = {"in": q(x[..., None])}

    def cr(name, inp):
        z = conv3x3(inp, q(p[name + ".w"]), p[name + ".b"])
        c[name] = q(np.maximum(z, 0.0))
        return c[name]

    def pl(name, h):
        c[name] = q(pool(h))
        return c[name]

    h = cr("e0b", cr("e0a", c["in"]))
    h = cr("e1b", cr("e1a", pl("p0", h)))
    h = cr("e2b", cr("e2a", pl("p1", h)))
    h = cr("b3b", cr("b3a", pl("p2", h)))
    c["cat2"] = np.concatenate([up(h), c["e2b"]], axis=-1)
    h = cr("d2b", cr("d2a", c["cat2"]))
    c["cat1"] = np.concatenate([up(h), c["e1b"]], axis=-1)
    h = cr("d1b", cr("d1a", c["cat1"]))
    c["cat0"] = np.concatenate([up(h), c["e0b"]], axis=-1)
    h = cr("d0b", cr("d0a", c["cat0"]))
    y = np.einsum("nhwc,c->nhw", h, p["out.w"]) + p["out.b"][0] + x
    return y, c


def loss_and_grads(p, x, target, q=None):
    """Mean squared error, its gradient for every parameter, and the
    prediction.  q as in forward; backward it rounds every stored gradient
    tensor (output-layer gradient, masked conv gradients, data gradients,
    upsampling and pooling gradients)."""
    q = q or _ident
    y, c = forward(p, x, q)
    n = y.size
    loss = float(np.mean((y - target) ** 2))
    dy = 2.0 * (y - target) / n
    g = {"out.w": np.einsum("nhw,nhwc->c", dy, c["d0b"]), "out.b": np.array([dy.sum()])}
    dh = q(dy[..., None] * p["out.w"])

    def crb(name, inp, dout):
        dz = q(dout * (c[name] > 0))
        dx, g[name + ".w"], g[name + ".b"] = conv3x3_bwd(inp, q(p[name + ".w"]), dz)
        return q(dx)

    dcat0 = crb("d0a", c["cat0"], crb("d0b", c["d0a"], dh))
    dh = q(up_bwd(dcat0[..., :64]))
    dskip0 = dcat0[..., 64:]
    dcat1 = crb("d1a", c["cat1"], crb("d1b", c["d1a"], dh))
    dh = q(up_bwd(dcat1[..., :128]))
    dskip1 = dcat1[..., 128:]
    dcat2 = crb("d2a", c["cat2"], crb("d2b", c["d2a"], dh))
    dh = q(up_bwd(dcat2[..., :256]))
    dskip2 = dcat2[..., 256:]
    dh = q(pool_bwd(crb("b3a", c["p2"], crb("b3b", c["b3a"], dh))) + dskip2)
    dh = q(pool_bwd(crb("e2a", c["p1"], crb("e2b", c["e2a"], dh))) + dskip1)
    dh = q(pool_bwd(crb("e1a", c["p0"], crb("e1b", c["e1a"], dh))) + dskip0)
    crb("e0a", c["in"], crb("e0b", c["e0a"], dh))
    return loss, g, y
