"""Pins of the oracle's cost, region of interest and network convolution
against computations that do not restate them:

* the PWLS cost of Sec. IV (Eq. ct_recon), 1/2 (y - Ax)'W(y - Ax) + R(x):
  the data term against the quadratic form of a dense A built by slab
  clipping (tests/dense_ref.py), and the regularizer against closed forms
  on images whose neighbour differences are known (ramps, checkerboards);
* the region of interest of the RMS differences (Sec. V; reading: the
  field of view): a pixel is in it exactly when its centre lies between the
  outer edges of the first and last detector cell from every view, decided
  from the oracle's ray segments alone (no radius formula); both copies of
  the mask (oracle and product) are held to it;
* the 3x3 convolution of the warm-start network: a plain loop over output
  pixels, taps and channels with explicit zero padding, and single-tap
  kernels that shift the image by a known offset.
"""
import math

import numpy as np
import pytest

from dense_ref import dense_A
from oracle import cnn_ref as C
from oracle import oslalm as O
from oracle import siddon
from paper_1402_4381_gb300 import roi, synth, workloads as W


# ---------------------------------------------------------------- PWLS cost

@pytest.mark.parametrize("g", [W.tiny_fan(), W.tiny_parallel(), W.tiny_cone(nz=3)])
@pytest.mark.parametrize("M", [1, 3])
def test_data_cost_is_the_weighted_quadratic_form(g, M):
    """sum over subsets of data_cost == 1/2 (y - Ax)' diag(w) (y - Ax), A dense."""
    A = dense_A(g)
    rng = np.random.default_rng(11 + M)
    x = rng.uniform(0.0, 0.05, size=A.shape[1])
    y = A @ x + rng.normal(0.0, 0.3, size=A.shape[0])
    w = rng.uniform(0.5, 4.0, size=A.shape[0])
    r = y - A @ x
    want = 0.5 * float(r @ (w * r))
    data, _ = O.ct_subset_data(g, y.reshape(g.sino_shape), w.reshape(g.sino_shape), M, siddon)
    got = data.data_cost(x.reshape(g.image_shape))
    assert abs(got - want) <= 1e-12 * abs(want)
    # the same through the algorithm's cost with beta = 0
    alg = O.OsLalm(data, np.ones(g.image_shape), beta=0.0, delta=1.0, nbr=4 if g.kind != 2 else 6)
    assert abs(alg.cost(x.reshape(g.image_shape)) - want) <= 1e-12 * abs(want)


def test_data_cost_of_exact_data_is_zero_and_of_known_residual_is_half_weighted_square():
    g = W.tiny_fan()
    A = dense_A(g)
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 0.05, size=A.shape[1])
    w = rng.uniform(0.5, 4.0, size=A.shape[0])
    data, _ = O.ct_subset_data(g, (A @ x).reshape(g.sino_shape), w.reshape(g.sino_shape), 4, siddon)
    assert data.data_cost(x.reshape(g.image_shape)) <= 1e-24
    e = np.zeros(A.shape[0])
    e[7] = 0.25  # one ray off by 0.25: cost = w_7 * 0.25^2 / 2
    data, _ = O.ct_subset_data(g, (A @ x + e).reshape(g.sino_shape), w.reshape(g.sino_shape), 4, siddon)
    assert abs(data.data_cost(x.reshape(g.image_shape)) - 0.5 * w[7] * 0.0625) <= 1e-14


def _psi(t, d):
    return d * d * (math.sqrt(1.0 + (t / d) ** 2) - 1.0)


def _ramp_pairs(shape, nbr):
    """For x = s * ix (a ramp along x), the pairs with |x_j - x_k| = s and
    their weights: sum over the half neighbourhood of count x weight, only
    offsets with a step along x (the others have difference 0).  Counted
    offset by offset from the neighbourhood's definition."""
    nz, ny, nx = shape
    if nbr in (4, 8):
        offs = [(0, 0, 1), (0, 1, 0)] + ([(0, 1, 1), (0, 1, -1)] if nbr == 8 else [])
    elif nbr == 6:
        offs = [(0, 0, 1), (0, 1, 0), (1, 0, 0)]
    else:
        offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                if (dz, dy, dx) > (0, 0, 0)]
    tot = 0.0
    for dz, dy, dx in offs:
        if dx == 0:
            continue
        count = (nz - abs(dz)) * (ny - abs(dy)) * (nx - abs(dx))
        tot += count / math.sqrt(dz * dz + dy * dy + dx * dx)
    return tot


@pytest.mark.parametrize("nbr,shape", [(4, (1, 5, 7)), (8, (1, 5, 7)), (6, (3, 4, 5)), (26, (3, 4, 5))])
def test_regularizer_value_on_a_ramp(nbr, shape):
    beta, delta, s = 3.0, 0.01, 0.004
    x = s * np.broadcast_to(np.arange(shape[2], dtype=float), shape).copy() + 0.7
    want = beta * _psi(s, delta) * _ramp_pairs(shape, nbr)
    assert abs(O.reg_value(x, beta, delta, nbr) - want) <= 1e-12 * want


def test_regularizer_value_on_a_checkerboard():
    """x = a (-1)^(ix+iy): horizontal and vertical pairs differ by 2a, diagonal
    pairs by 0: R = beta psi(2a) (ny (nx-1) + nx (ny-1)) for 4 and 8 neighbours."""
    ny, nx, a, beta, delta = 6, 9, 0.003, 2.0, 0.01
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = (a * (-1.0) ** (ix + iy))[None]
    want = beta * _psi(2 * a, delta) * (ny * (nx - 1) + nx * (ny - 1))
    for nbr in (4, 8):
        assert abs(O.reg_value(x, beta, delta, nbr) - want) <= 1e-12 * want


def test_cost_adds_data_term_and_regularizer():
    g = W.tiny_fan()
    A = dense_A(g)
    rng = np.random.default_rng(8)
    x = rng.uniform(0.0, 0.05, size=A.shape[1])
    y = A @ x + rng.normal(0.0, 0.3, size=A.shape[0])
    w = rng.uniform(0.5, 4.0, size=A.shape[0])
    data, _ = O.ct_subset_data(g, y.reshape(g.sino_shape), w.reshape(g.sino_shape), 2, siddon)
    beta, delta = 2.0, 0.01
    alg = O.OsLalm(data, np.ones(g.image_shape), beta=beta, delta=delta, nbr=8)
    # ramp image: the regularizer is the closed form above
    xr = 0.004 * np.broadcast_to(np.arange(g.nx, dtype=float), g.image_shape).copy()
    r = y - A @ xr.ravel()
    want = 0.5 * float(r @ (w * r)) + beta * _psi(0.004, delta) * _ramp_pairs(g.image_shape, 8)
    assert abs(alg.cost(xr) - want) <= 1e-12 * want


# ---------------------------------------------------------------- region of interest

def _coverage_margin(g):
    """For every pixel centre: the smallest, over views, signed distance (in
    detector cells) from its detector coordinate to the nearer outer edge of
    the first / last cell; >= 0 when every view sees it.  Decided from the
    oracle's ray segments only: the ray of each cell, interpolated between
    neighbouring cells and extended by half a cell at the two ends.  For the
    cone beam the rows are handled the same way on the detector plane."""
    ix = (np.arange(g.nx) - (g.nx - 1) / 2.0) * g.dx + g.offset_x
    iy = (np.arange(g.ny) - (g.ny - 1) / 2.0) * g.dy + g.offset_y
    iz = (np.arange(g.nz) - (g.nz - 1) / 2.0) * g.dz + g.offset_z if g.kind == synth.CONE3D_FLAT else np.zeros(1)
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
    P = np.stack([X, Y, Z], -1)
    margin = np.full(X.shape, np.inf)

    def edge_margin(coord, cells):
        # cells: coordinate of every cell's ray, monotone; coord: the point's
        d0, d1 = cells[1] - cells[0], cells[-1] - cells[-2]
        lo, hi = cells[0] - 0.5 * d0, cells[-1] + 0.5 * d1
        sgn = 1.0 if d0 > 0 else -1.0
        pitch = abs(d0)
        return np.minimum(sgn * (coord - lo), sgn * (hi - coord)) / pitch

    for v in range(g.nviews):
        seg = siddon.ray_segments(g, v)  # [nt][ns][2][3]
        if g.kind == synth.PAR2D:
            P0, P1 = seg[0, :, 0, :2], seg[0, :, 1, :2]
            u = (P1[0] - P0[0]) / np.linalg.norm(P1[0] - P0[0])
            lat = lambda q: q[..., 0] * u[1] - q[..., 1] * u[0]  # noqa: E731  signed distance across u
            margin = np.minimum(margin, edge_margin(lat(P[..., :2]), lat(P0)))
        elif g.kind == synth.FAN2D_ARC:
            S = seg[0, 0, 0, :2]
            d = seg[0, :, 1, :2] - S
            ref = math.atan2(d[g.ns // 2, 1], d[g.ns // 2, 0])
            ang = lambda q: np.angle(np.exp(1j * (np.arctan2(q[..., 1], q[..., 0]) - ref)))  # noqa: E731
            margin = np.minimum(margin, edge_margin(ang(P[..., :2] - S), ang(d)))
        else:
            S = seg[0, 0, 0]
            cell = seg[:, :, 1, :]  # cell centres on the flat detector [nt][ns][3]
            ea = cell[0, -1] - cell[0, 0]
            ea /= np.linalg.norm(ea)  # lateral axis of the panel
            eb = cell[-1, 0] - cell[0, 0]
            eb /= np.linalg.norm(eb)  # row axis
            n = np.cross(ea, eb)
            dist = float(np.dot(cell[0, 0] - S, n))
            q = P - S
            t = dist / np.sum(q * n, -1)  # the line from the source through P meets the panel at S + t q
            hit = S + t[..., None] * q - cell[0, 0]
            a, b = hit @ ea, hit @ eb
            ca = (cell[0] - cell[0, 0]) @ ea
            cb = (cell[:, 0] - cell[0, 0]) @ eb
            margin = np.minimum(margin, np.minimum(edge_margin(a, ca), edge_margin(b, cb)))
    return margin


def _roi_cases():
    fan = W.scaled(W.c1_fan(), 48, 360, 111, 6).geom
    par = synth.Geometry(kind=synth.PAR2D, nx=40, ny=36, dx=1.0, dy=1.1, nviews=240, angle_start=0.013,
                         angle_span=math.pi, ns=31, ds=1.2)
    cone = W.scaled(W.c2_cone(), 40, 360, 91, 6, nz=12, nt=6).geom
    return [("fan", fan), ("parallel", par), ("cone", cone)]


@pytest.mark.parametrize("name,g", _roi_cases())
@pytest.mark.parametrize("which", ["oracle", "product"])
def test_roi_is_the_region_every_view_covers(name, g, which):
    mask = (O.roi_mask(g) if which == "oracle" else roi.roi_mask(g)).astype(bool)
    margin = _coverage_margin(g)
    assert mask.shape == margin.shape
    assert 0.2 * mask.size < mask.sum() < mask.size  # the boundary lies inside the image
    seen = margin >= 0.0
    # identical except where a finite set of views sees a point a hair beyond
    # the continuous field of view's boundary
    disagree = mask != seen
    assert not np.any(mask & ~seen), f"{name}: masked pixels not seen by every view"
    assert np.all(np.abs(margin[disagree]) < 0.02), f"{name}: field of view too small"


def test_helical_roi_heights_are_the_source_heights():
    g = W.tiny_helical(n=12, nz=10, nviews=40, ns=31)
    zs = np.array([siddon.ray_segments(g, v)[0, 0, 0, 2] for v in range(g.nviews)])
    iz = (np.arange(g.nz) - (g.nz - 1) / 2.0) * g.dz
    inside = (iz >= zs.min()) & (iz <= zs.max())
    for mask in (O.roi_mask(g), roi.roi_mask(g)):
        planes = mask.any(axis=(1, 2))
        np.testing.assert_array_equal(planes, inside)


# ---------------------------------------------------------------- network convolution

def _conv_loops(x, w, b):
    """out[n,h,x,o] = b[o] + sum_{ky,kx,c} w[o,ky,kx,c] x[n, h+ky-1, x+kx-1, c],
    terms outside the image left out (zero padding)."""
    N, H, Wd, Ci = x.shape
    Co = w.shape[0]
    out = np.zeros((N, H, Wd, Co))
    for n in range(N):
        for h in range(H):
            for xx in range(Wd):
                for o in range(Co):
                    acc = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            hh, ww = h + ky - 1, xx + kx - 1
                            if 0 <= hh < H and 0 <= ww < Wd:
                                for c in range(Ci):
                                    acc += w[o, ky, kx, c] * x[n, hh, ww, c]
                    out[n, h, xx, o] = acc
    return out


def test_conv3x3_equals_plain_loops():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 5, 6, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    np.testing.assert_allclose(C.conv3x3(x, w, b), _conv_loops(x, w, b), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("ky,kx", [(0, 2), (2, 0), (1, 0), (0, 1)])
def test_conv3x3_single_tap_shifts(ky, kx):
    """A kernel with only tap (ky, kx) = 1 copies x[h + ky - 1, w + kx - 1]
    (zero where that pixel is outside): correlation, not convolution."""
    rng = np.random.default_rng(ky * 3 + kx)
    x = rng.normal(size=(1, 5, 7, 1))
    w = np.zeros((1, 3, 3, 1))
    w[0, ky, kx, 0] = 1.0
    out = C.conv3x3(x, w, np.zeros(1))[0, :, :, 0]
    for h in range(5):
        for xx in range(7):
            hh, ww = h + ky - 1, xx + kx - 1
            want = x[0, hh, ww, 0] if 0 <= hh < 5 and 0 <= ww < 7 else 0.0
            assert out[h, xx] == want
