"""FP64 oracle of the filtered back-projection used for the initial image x0.

TEST INFRASTRUCTURE.  The paper starts every run from an FBP image (Sec. V)
without giving its filter or weights; the reading taken
here is the textbook analytic reconstruction (A. C. Kak and M. Slaney,
Principles of Computerized Tomographic Imaging, ch. 3):

* parallel beam: Ram-Lak ramp filter h[0] = 1/(4 ds^2), h[n odd] =
  -1/(n pi ds)^2, h[n even] = 0; q = ds (p * h); x(r) = (pi/N) sum_v q_v(s(r))
  with s(r) = r . e_v and linear interpolation between channels;
* fan beam, equiangular arc detector over 360 degrees: p'(g) = p(g) dso cos g,
  kernel g[0] = 1/(8 a^2), g[n odd] = -1/(2 pi^2 sin^2(n a)), a = ds/dsd;
  q = a (p' * g); x(r) = (2 pi / N) sum_v q_v(gamma(r)) / L(r)^2 with L the
  source-to-point distance and gamma the point's fan angle;
* cone beam, flat detector (Feldkamp-Davis-Kress): detector coordinates
  scaled to the isocentre (p = s dso/dsd, z = t dso/dsd); p' = p dso /
  sqrt(dso^2 + p^2 + z^2); row-wise Ram-Lak filter with pitch ds dso/dsd;
  x(r) = 1/2 (2 pi / N) sum_v U^-2 q_v(p(r), z(r)), U = (dso + r.u)/dso,
  bilinear interpolation.
Values outside the detector interpolate to zero.  The result is not clipped
(callers clip to the non-negative orthant).
"""
import math

import numpy as np


def ramlak(n_half, d):
    """Ram-Lak taps h[k], k = -n_half..n_half, for sampling pitch d."""
    k = np.arange(-n_half, n_half + 1)
    h = np.zeros(k.size)
    h[k == 0] = 1.0 / (4.0 * d * d)
    odd = (k % 2) != 0
    h[odd] = -1.0 / (np.pi * k[odd] * d) ** 2
    return k, h


def fan_kernel(n_half, a):
    k = np.arange(-n_half, n_half + 1)
    g = np.zeros(k.size)
    g[k == 0] = 1.0 / (8.0 * a * a)
    odd = (k % 2) != 0
    g[odd] = -1.0 / (2.0 * np.pi ** 2 * np.sin(k[odd] * a) ** 2)
    return g


def _filter_rows(rows, taps, scale):
    """rows [..., ns] convolved with centred taps (length 2 ns - 1), times scale."""
    ns = rows.shape[-1]
    out = np.zeros_like(rows)
    flat = rows.reshape(-1, ns)
    of = out.reshape(-1, ns)
    for i in range(flat.shape[0]):
        full = np.convolve(flat[i], taps)  # length 3 ns - 2, centre offset ns - 1
        of[i] = scale * full[ns - 1: 2 * ns - 1]
    return out


def _interp(q, c):
    """Linear interpolation of q at fractional channel c, zero outside [0, ns-1]."""
    ns = q.shape[-1]
    c0 = np.floor(c)
    f = c - c0
    i0 = c0.astype(np.int64)
    v0 = np.where((i0 >= 0) & (i0 < ns), q[np.clip(i0, 0, ns - 1)], 0.0)
    v1 = np.where((i0 + 1 >= 0) & (i0 + 1 < ns), q[np.clip(i0 + 1, 0, ns - 1)], 0.0)
    return (1 - f) * v0 + f * v1


def _view_dirs(g):
    """Beam directions (cos phi_v, sin phi_v), phi_v = pi tau_v, with the
    quarter turns of tau_v taken out exactly."""
    v = np.arange(g.nviews, dtype=np.float64)
    t = g.angle_start / np.pi + v * (g.angle_span / np.pi) / g.nviews
    n = np.floor(2.0 * t + 0.5)
    r = t - 0.5 * n
    c, s = np.cos(np.pi * r), np.sin(np.pi * r)
    q = np.mod(n, 4.0)
    cq = np.where(q == 0, c, np.where(q == 1, -s, np.where(q == 2, -c, s)))
    sq = np.where(q == 0, s, np.where(q == 1, c, np.where(q == 2, -s, -c)))
    return cq, sq


def _pixel_centres(g):
    xs = (np.arange(g.nx) - (g.nx - 1) / 2.0) * g.dx + g.offset_x
    ys = (np.arange(g.ny) - (g.ny - 1) / 2.0) * g.dy + g.offset_y
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    return X, Y


def fbp(g, sino):
    sino = np.asarray(sino, dtype=np.float64).reshape(g.nviews, g.nt, g.ns)
    cu, su = _view_dirs(g)
    c0 = (g.ns - 1) / 2.0 - g.offset_s
    n = g.ns - 1
    if g.kind == 0:
        _, h = ramlak(n, g.ds)
        q = _filter_rows(sino[:, 0, :], h, g.ds)
        X, Y = _pixel_centres(g)
        img = np.zeros((g.ny, g.nx))
        for v in range(g.nviews):
            s = -X * su[v] + Y * cu[v]
            img += _interp(q[v], s / g.ds + c0)
        return (np.pi / g.nviews * img)[None]
    if g.kind == 1:
        if abs(abs(g.angle_span) - 2 * math.pi) > 1e-9:
            raise ValueError("fan-beam FBP needs a full 360-degree scan")
        a = g.ds / g.dsd
        gam = (np.arange(g.ns) - (g.ns - 1) / 2.0 + g.offset_s) * a
        pw = sino[:, 0, :] * g.dso * np.cos(gam)[None]
        q = _filter_rows(pw, fan_kernel(n, a), a)
        X, Y = _pixel_centres(g)
        img = np.zeros((g.ny, g.nx))
        for v in range(g.nviews):
            A = X * cu[v] + Y * su[v] + g.dso
            B = -X * su[v] + Y * cu[v]
            gp = np.arctan2(B, A)
            img += _interp(q[v], gp / a + c0) / (A * A + B * B)
        return (2 * np.pi / g.nviews * img)[None]
    if g.kind == 2:
        if abs(abs(g.angle_span) - 2 * math.pi) > 1e-9:
            raise ValueError("FDK needs a full 360-degree scan")
        mag = g.dso / g.dsd
        dp, dz = g.ds * mag, g.dt * mag
        p = (np.arange(g.ns) - (g.ns - 1) / 2.0 + g.offset_s) * dp
        z = (np.arange(g.nt) - (g.nt - 1) / 2.0 + g.offset_t) * dz
        Z, P = np.meshgrid(z, p, indexing="ij")
        pw = sino * (g.dso / np.sqrt(g.dso ** 2 + P ** 2 + Z ** 2))[None]
        _, h = ramlak(n, dp)
        q = _filter_rows(pw, h, dp)
        X, Y = _pixel_centres(g)
        zc = (np.arange(g.nz) - (g.nz - 1) / 2.0) * g.dz + g.offset_z
        t0 = (g.nt - 1) / 2.0 - g.offset_t
        img = np.zeros((g.nz, g.ny, g.nx))
        for v in range(g.nviews):
            A = X * cu[v] + Y * su[v] + g.dso
            B = -X * su[v] + Y * cu[v]
            U = A / g.dso
            pc = (g.dso * B / A) / dp + c0
            for iz in range(g.nz):
                tc = (g.dso * zc[iz] / A) / dz + t0
                t_lo = np.floor(tc)
                ft = tc - t_lo
                ti = t_lo.astype(np.int64)
                acc = np.zeros_like(A)
                for dt_, wt in ((0, 1 - ft), (1, ft)):
                    tt = ti + dt_
                    ok = (tt >= 0) & (tt < g.nt)
                    rows = q[v][np.clip(tt, 0, g.nt - 1)]  # [ny, nx, ns]
                    cf = np.floor(pc)
                    fc = pc - cf
                    ci = cf.astype(np.int64)
                    v0 = np.where((ci >= 0) & (ci < g.ns), np.take_along_axis(rows, np.clip(ci, 0, g.ns - 1)[..., None], -1)[..., 0], 0.0)
                    v1 = np.where((ci + 1 >= 0) & (ci + 1 < g.ns), np.take_along_axis(rows, np.clip(ci + 1, 0, g.ns - 1)[..., None], -1)[..., 0], 0.0)
                    acc += np.where(ok, wt * ((1 - fc) * v0 + fc * v1), 0.0)
                img[iz] += acc / (U * U)
        return 0.5 * (2 * np.pi / g.nviews) * img
    raise ValueError(g.kind)
