"""CPU check of the CUDA path's 2D system model: the library's host-built ray
tables (oslalm_ray_table), with the projector pair's per-(ray, pixel) length
arithmetic re-evaluated here operation by operation in IEEE float32, against
the dense FP64 clipping reference.  No GPU needed."""
import math

import numpy as np
import pytest

from dense_ref import dense_A
from paper_1402_4381_gb300 import synth, workloads as W

F = np.float32


@pytest.fixture(scope="module")
def L():
    from paper_1402_4381_gb300 import build, oslalm
    build.build()
    return oslalm


def decode(packed):
    p = packed.astype(np.int32)
    axis = p & 1
    n0 = (p.astype(np.uint32) << np.uint32(16)).view(np.int32) >> 17
    k = p >> 16
    return axis, n0, k


def _fma32(a, b, c):
    """float32 fused multiply-add (the product of two float32 values is exact
    in float64; one rounding of the sum to float32)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F)


def chords_float32(tab, c, ia, jb):
    """Length of ray c inside pixels (ia, jb) (major, minor indices), with the
    float32 operations of the device code in the same order: the device
    table's derived constants (k / 4096, n0, the row half-width hw, the
    length per unit of minor span lrow / (2 hw)), then the row-centre span
    and the two-pixel split of each row."""
    f0, kl, lrow = F(tab["f0"][c]), F(tab["kappa_lo"][c]), F(tab["lrow"][c])
    axis, n0, k = decode(tab["packed"][c:c + 1])
    n0, k = int(n0[0]), int(k[0])
    kq = F(F(k) * F(2.0 ** -12))
    hw = np.abs(_fma32(F(k), F(2.0 ** -12), F(F(0.5) * kl)))
    lscale = F(float(lrow) / (2.0 * float(hw))) if hw > 0 else F(0)
    ia = np.asarray(ia, np.int64)
    ia2 = (2 * ia + 1).astype(F)
    iah = (ia.astype(F) + F(0.5)).astype(F)
    pq = (ia2 * kq).astype(F)
    q = np.floor(pq)
    fr = (pq - q).astype(F)
    cc = _fma32(iah, kl, (f0 + fr).astype(F))
    lo, hi = (cc - hw).astype(F), (cc + hw).astype(F)
    jl = np.floor(lo)
    jl1 = (jl + F(1)).astype(F)
    j = (F(n0) + q).astype(F) + jl
    with np.errstate(over="ignore", invalid="ignore"):
        part = np.minimum(((jl1 - lo).astype(F) * lscale).astype(F), lrow)
    w0 = np.where(hi > jl1, part, lrow).astype(F)
    w1 = (lrow - w0).astype(F)
    d = np.asarray(jb, np.int64).astype(F) - j
    ch = np.where(d == 0, w0, np.where(d == 1, w1, F(0)))
    return ch.astype(np.float64), int(axis[0])


@pytest.mark.parametrize("g", [W.tiny_fan(), W.tiny_parallel(), W.tiny_parallel(n=7, nviews=9, ns=12),
                               synth.Geometry(kind=0, nx=9, ny=6, dx=1.1, dy=0.9, nviews=8, angle_start=0.0,
                                              angle_span=math.pi, ns=15, ds=0.8, offset_s=0.25)])
def test_float32_chords_match_dense_clipping(L, g):
    A = dense_A(g)
    iy, ix = np.meshgrid(np.arange(g.ny), np.arange(g.nx), indexing="ij")
    ix, iy = ix.ravel(), iy.ravel()
    for v in range(g.nviews):
        tab = L.ray_table(g, v)
        for c in range(g.ns):
            ch, axis = chords_float32(tab, c, iy if decode(tab["packed"][c:c + 1])[0][0] else ix,
                                      ix if decode(tab["packed"][c:c + 1])[0][0] else iy)
            ref = A[v * g.ns + c]
            np.testing.assert_allclose(ch, ref, rtol=0, atol=2e-6 * max(g.dx, g.dy) * 2)


@pytest.mark.parametrize("wl,views", [(W.c0_parallel(), [0, 45, 90, 135]), (W.c1_fan(), [0, 123, 246, 600])])
def test_workload_ray_tables_are_precise(L, wl, views):
    """Full-size tables: every ray's row spans sum to its chord through the
    image box, and positions keep their precision at the far side (quarter
    turns and 45-degree views included)."""
    g = wl.geom
    org, d = synth.rays(g, views)
    lo = np.array([-g.nx * g.dx / 2, -g.ny * g.dy / 2])
    for iv, v in enumerate(views):
        tab = L.ray_table(g, v)
        axis, n0, k = decode(tab["packed"])
        assert np.all(np.abs(k) <= 2048)
        assert np.all((tab["f0"] >= -0.5) & (tab["f0"] < 0.5))
        assert np.all(np.abs(tab["kappa_lo"]) <= 2.0 ** -11)
        for c in range(0, g.ns, 37):
            o, dd = org[iv, 0, c, :2], d[iv, 0, c, :2]
            ia = np.arange(g.ny if axis[c] else g.nx)
            # exact minor coordinate of the ray at the row boundaries (FP64)
            a_mm = lo[axis[c]] + ia * (g.dy if axis[c] else g.dx)
            t = (a_mm - o[axis[c]]) / dd[axis[c]]
            b_mm = o[1 - axis[c]] + t * dd[1 - axis[c]]
            b_idx = (b_mm - lo[1 - axis[c]]) / (g.dx if axis[c] else g.dy)
            nb = g.nx if axis[c] else g.ny
            if tab["lrow"][c] == 0:  # flagged as missing the image: check that it does
                ends = np.concatenate([b_idx, [b_idx[-1] + (b_idx[-1] - b_idx[-2])]])
                assert np.all(ends < 0) or np.all(ends > nb)
                continue
            kap = k[c] / 2048.0 + float(tab["kappa_lo"][c])
            b_tab = n0[c] + float(tab["f0"][c]) + ia * kap
            assert np.max(np.abs(b_tab - b_idx)) < 2e-6
