"""Seeded synthetic CT scans: ellipse/ellipsoid phantoms, their analytic line
integrals, Poisson (+Gaussian) counts, the log sinogram y and the statistical
weights W.

This module is the only code shared by the FP64 oracle and the CUDA path. It
holds none of the reconstruction method's arithmetic (no system matrix, no
projector, no optimiser): it simulates a scan from a continuous phantom, so
the data are not produced by either side's discretised model (no inverse
crime).

Scan geometry convention (the same convention both sides implement on their
own):

* view angle ``phi_v = pi * tau_v`` with
  ``tau_v = angle_start/pi + v * (angle_span/pi) / nviews`` (FP64);
  ``(cos phi, sin phi)`` is evaluated by exact quarter-turn reduction of
  ``tau_v``, so views at multiples of 90 degrees are exactly axis-aligned;
  ``u = (cos phi, sin phi)`` is the beam direction (source towards detector),
  ``e = (-sin phi, cos phi)`` is the detector's lateral axis;
* parallel beam: ray ``c`` is the line through ``s_c * e`` along ``u`` with
  ``s_c = (c - (ns-1)/2 + offset_s) * ds``;
* fan beam, arc detector: the source sits at ``-dso * u``; channel ``c`` has
  angle ``gamma_c = (c - (ns-1)/2 + offset_s) * ds / dsd`` and direction
  ``cos(gamma_c) u + sin(gamma_c) e``;
* cone beam, flat detector: source at ``(-dso * u, z_v)``; cell ``(t, c)`` is
  centred at ``(dsd - dso) u + s_c e + (z_v + t_t) z`` with
  ``t_t = (t - (nt-1)/2 + offset_t) * dt``; ``z_v = 0`` for a circular orbit;
  a helical orbit (``pitch > 0``) advances source and detector by
  ``pitch * nt * dt`` per turn (table feed = pitch x detector height at the
  detector, the convention under which a central voxel is covered for
  ``dso / (pitch dsd)`` turns, Sec. IV-B), centred on the scan:
  ``z_v = pitch * nt * dt * (phi_v - phi_mid) / (2 pi)``, ``phi_mid`` the
  middle of the angular range;
* pixels are half-open boxes ``[lo, hi)``: a ray lying exactly on the plane
  between two pixels belongs to the upper one;
* pixel ``(ix, iy, iz)`` is centred at ``((ix - (nx-1)/2) dx + offset_x, ...)``;
  images are stored ``[z][y][x]`` (x fastest), sinograms ``[view][row][channel]``.

The data model follows the PWLS problem of Sec. IV (Eq. ct_recon):
``y_i = -log(c_i / I0)`` with counts ``c_i ~ Poisson(I0 exp(-p_i))`` and
``p_i`` the analytic line integral of the phantom; electronic noise adds
``N(0, sigma^2)``; counts are clamped to at least 1.  Weights: ``w_i = c_i``
without electronic noise, ``w_i = c_i^2 / (c_i + sigma^2)`` with it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

PAR2D = 0
FAN2D_ARC = 1
CONE3D_FLAT = 2

MU_WATER = 0.0192  # /mm, linear attenuation of water (1000 HU)
HU = MU_WATER / 1000.0  # /mm per Hounsfield unit


@dataclasses.dataclass
class Geometry:
    """Scan + image grid description (units: mm and radians)."""

    kind: int
    nx: int
    ny: int
    nz: int = 1
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    offset_x: float = 0.0
    offset_y: float = 0.0
    offset_z: float = 0.0
    nviews: int = 1
    angle_start: float = 0.0
    angle_span: float = math.pi
    ns: int = 1
    nt: int = 1
    ds: float = 1.0
    dt: float = 1.0
    offset_s: float = 0.0  # in units of channels
    offset_t: float = 0.0  # in units of rows
    dso: float = 0.0
    dsd: float = 0.0
    pitch: float = 0.0  # helical cone beam: table feed per turn / (nt dt); 0 = circular orbit

    @property
    def image_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.nviews, self.nt, self.ns)

    def view_turns(self, views=None) -> np.ndarray:
        """tau_v = phi_v / pi (FP64)."""
        v = np.arange(self.nviews, dtype=np.float64) if views is None else np.asarray(views, dtype=np.float64)
        return self.angle_start / np.pi + v * (self.angle_span / np.pi) / self.nviews

    def view_angles(self) -> np.ndarray:
        return np.pi * self.view_turns()

    def source_z(self, views=None) -> np.ndarray:
        """Height of the source (and detector centre) at each view (mm)."""
        v = np.arange(self.nviews, dtype=np.float64) if views is None else np.asarray(views, dtype=np.float64)
        if self.pitch == 0.0:
            return np.zeros_like(v)
        dphi = v * (self.angle_span / self.nviews) - 0.5 * self.angle_span
        return self.pitch * self.nt * self.dt * dphi / (2.0 * np.pi)

    def as_dict(self):
        return dataclasses.asdict(self)


# --------------------------------------------------------------------------
# rays
# --------------------------------------------------------------------------

def cos_sin_pi(t):
    """(cos(pi t), sin(pi t)) with exact quarter-turn reduction (exact 0/+-1
    at multiples of 1/2)."""
    t = np.asarray(t, dtype=np.float64)
    n = np.floor(2.0 * t + 0.5)
    r = t - 0.5 * n
    c, s = np.cos(np.pi * r), np.sin(np.pi * r)
    q = np.mod(n, 4.0)
    cq = np.where(q == 0, c, np.where(q == 1, -s, np.where(q == 2, -c, s)))
    sq = np.where(q == 0, s, np.where(q == 1, c, np.where(q == 2, -s, -c)))
    return cq, sq


def rays(geom: Geometry, views: Sequence[int] | None = None):
    """Return (origin, unit direction) of every ray, FP64, shape [nv, nt, ns, 3].

    For parallel and fan beams the z components are zero and nt == 1.
    """
    if views is None:
        views = np.arange(geom.nviews)
    views = np.asarray(views, dtype=np.int64)
    cu, su = cos_sin_pi(geom.view_turns(views))
    c = np.arange(geom.ns, dtype=np.float64)
    s = (c - (geom.ns - 1) / 2.0 + geom.offset_s) * geom.ds
    nv = views.size
    org = np.zeros((nv, geom.nt, geom.ns, 3))
    dirn = np.zeros((nv, geom.nt, geom.ns, 3))
    if geom.kind == PAR2D:
        # point s*e, direction u
        org[..., 0] = (-su)[:, None, None] * s[None, None, :]
        org[..., 1] = (cu)[:, None, None] * s[None, None, :]
        dirn[..., 0] = cu[:, None, None]
        dirn[..., 1] = su[:, None, None]
    elif geom.kind == FAN2D_ARC:
        gam = s / geom.dsd
        cg, sg = np.cos(gam), np.sin(gam)
        org[..., 0] = (-geom.dso * cu)[:, None, None]
        org[..., 1] = (-geom.dso * su)[:, None, None]
        # cos(g) u + sin(g) e
        dirn[..., 0] = cu[:, None, None] * cg[None, None, :] - su[:, None, None] * sg[None, None, :]
        dirn[..., 1] = su[:, None, None] * cg[None, None, :] + cu[:, None, None] * sg[None, None, :]
    elif geom.kind == CONE3D_FLAT:
        t = (np.arange(geom.nt, dtype=np.float64) - (geom.nt - 1) / 2.0 + geom.offset_t) * geom.dt
        org[..., 0] = (-geom.dso * cu)[:, None, None]
        org[..., 1] = (-geom.dso * su)[:, None, None]
        org[..., 2] = geom.source_z(views)[:, None, None]
        dd = geom.dsd - geom.dso
        px = dd * cu[:, None, None] - su[:, None, None] * s[None, None, :]
        py = dd * su[:, None, None] + cu[:, None, None] * s[None, None, :]
        dx = px - org[..., 0]
        dy = py - org[..., 1]
        dz = np.broadcast_to(t[None, :, None], dx.shape)
        nrm = np.sqrt(dx * dx + dy * dy + dz * dz)
        dirn[..., 0] = dx / nrm
        dirn[..., 1] = dy / nrm
        dirn[..., 2] = dz / nrm
    else:
        raise ValueError(f"unknown geometry kind {geom.kind}")
    return org, dirn


# --------------------------------------------------------------------------
# phantoms
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Ellipsoid:
    """Ellipse (2D, cz/c ignored) or ellipsoid with a rotation about z."""

    cx: float
    cy: float
    a: float
    b: float
    angle: float  # radians, rotation about z
    value: float  # additive attenuation, /mm
    cz: float = 0.0
    c: float = 1e30  # semi-axis along z (infinite: a 2D ellipse / cylinder)


def _to_local(e: Ellipsoid, pts):
    ca, sa = math.cos(e.angle), math.sin(e.angle)
    x = pts[..., 0] - e.cx
    y = pts[..., 1] - e.cy
    z = pts[..., 2] - e.cz
    xl = ca * x + sa * y
    yl = -sa * x + ca * y
    return xl, yl, z


def line_integrals(phantom: Sequence[Ellipsoid], org, dirn) -> np.ndarray:
    """Exact line integral of a sum of uniform ellipsoids along unit-speed lines."""
    out = np.zeros(org.shape[:-1])
    for e in phantom:
        ca, sa = math.cos(e.angle), math.sin(e.angle)
        ox, oy, oz = _to_local(e, org)
        vx = ca * dirn[..., 0] + sa * dirn[..., 1]
        vy = -sa * dirn[..., 0] + ca * dirn[..., 1]
        vz = dirn[..., 2]
        qx, qy, qz = ox / e.a, oy / e.b, oz / e.c
        wx, wy, wz = vx / e.a, vy / e.b, vz / e.c
        A = wx * wx + wy * wy + wz * wz
        B = qx * wx + qy * wy + qz * wz
        C = qx * qx + qy * qy + qz * qz - 1.0
        disc = B * B - A * C
        chord = np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
        out += e.value * chord
    return out


def analytic_sinogram(geom: Geometry, phantom: Sequence[Ellipsoid], views=None) -> np.ndarray:
    org, dirn = rays(geom, views)
    return line_integrals(phantom, org, dirn)


def pixelize(geom: Geometry, phantom: Sequence[Ellipsoid], supersample: int = 4) -> np.ndarray:
    """Mean of the phantom over each pixel (supersample^2 or ^3 sub-samples)."""
    ss = supersample
    off = (np.arange(ss) + 0.5) / ss - 0.5
    xs = ((np.arange(geom.nx) - (geom.nx - 1) / 2.0)[:, None] + off[None, :]).ravel() * geom.dx + geom.offset_x
    ys = ((np.arange(geom.ny) - (geom.ny - 1) / 2.0)[:, None] + off[None, :]).ravel() * geom.dy + geom.offset_y
    if geom.nz > 1 or geom.kind == CONE3D_FLAT:
        zs = ((np.arange(geom.nz) - (geom.nz - 1) / 2.0)[:, None] + off[None, :]).ravel() * geom.dz + geom.offset_z
        ssz = ss
    else:
        zs = np.zeros(1)
        ssz = 1
    img = np.zeros((geom.nz, geom.ny, geom.nx))
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    for iz, z in enumerate(zs):
        acc = np.zeros_like(X)
        for e in phantom:
            ca, sa = math.cos(e.angle), math.sin(e.angle)
            x = X - e.cx
            y = Y - e.cy
            xl = ca * x + sa * y
            yl = -sa * x + ca * y
            zl = z - e.cz
            inside = (xl / e.a) ** 2 + (yl / e.b) ** 2 + (zl / e.c) ** 2 <= 1.0
            acc += e.value * inside
        blk = acc.reshape(geom.ny, ss, geom.nx, ss).mean(axis=(1, 3))
        img[iz // ssz] += blk / ssz
    return img


def _boundary_inside(inner: Ellipsoid, outer: Ellipsoid, margin: float = 0.0) -> bool:
    t = np.linspace(0, 2 * np.pi, 72, endpoint=False)
    ca, sa = math.cos(inner.angle), math.sin(inner.angle)
    px = inner.cx + ca * inner.a * np.cos(t) - sa * inner.b * np.sin(t)
    py = inner.cy + sa * inner.a * np.cos(t) + ca * inner.b * np.sin(t)
    oa, ob = outer.a - margin, outer.b - margin
    co, so = math.cos(outer.angle), math.sin(outer.angle)
    x, y = px - outer.cx, py - outer.cy
    xl, yl = co * x + so * y, -so * x + co * y
    return bool(np.all((xl / oa) ** 2 + (yl / ob) ** 2 <= 1.0))


def _disjoint(e1: Ellipsoid, e2: Ellipsoid, gap: float) -> bool:
    d = math.hypot(e1.cx - e2.cx, e1.cy - e2.cy)
    if d > max(e1.a, e1.b) + max(e2.a, e2.b) + gap:
        return True
    if abs(e1.cz - e2.cz) > e1.c + e2.c + gap:
        return True
    return False


def random_ellipse_phantom(seed: int, fov_radius: float, n: int = 10,
                           vmax: float = 0.04, three_d: bool = False,
                           z_half: float = 0.0) -> List[Ellipsoid]:
    """Body ellipse of water plus n-1 disjoint inner ellipses/ellipsoids whose
    absolute attenuation is uniform in [0, vmax] /mm."""
    rng = np.random.default_rng(seed)
    body = Ellipsoid(cx=0.0, cy=0.0,
                     a=fov_radius * rng.uniform(0.80, 0.92),
                     b=fov_radius * rng.uniform(0.62, 0.80),
                     angle=rng.uniform(-0.2, 0.2), value=MU_WATER,
                     cz=0.0, c=(z_half * 0.9 if three_d else 1e30))
    out = [body]
    tries = 0
    while len(out) < n and tries < 20000:
        tries += 1
        a = fov_radius * rng.uniform(0.05, 0.22)
        b = fov_radius * rng.uniform(0.05, 0.22)
        e = Ellipsoid(cx=rng.uniform(-body.a, body.a), cy=rng.uniform(-body.b, body.b),
                      a=a, b=b, angle=rng.uniform(0, np.pi),
                      value=rng.uniform(0.0, vmax) - MU_WATER)
        if three_d:
            e.c = z_half * rng.uniform(0.15, 0.45)
            e.cz = rng.uniform(-z_half * 0.85 + e.c, z_half * 0.85 - e.c) if z_half * 0.85 > e.c else 0.0
        if not _boundary_inside(e, body, margin=2.0):
            continue
        if all(_disjoint(e, o, 1.0) for o in out[1:]):
            out.append(e)
    return out


def torso_phantom(seed: int, fov_radius: float) -> List[Ellipsoid]:
    """Ellipse torso: water body, bone (0.04 /mm) spine and ribs, and
    soft-tissue ellipses at water x (1 +/- 1%)."""
    rng = np.random.default_rng(seed)
    body = Ellipsoid(0.0, 0.0, a=fov_radius * 0.86, b=fov_radius * 0.62,
                     angle=rng.uniform(-0.05, 0.05), value=MU_WATER)
    out = [body]
    bone = 0.04 - MU_WATER
    # spine
    out.append(Ellipsoid(0.0, -body.b * 0.62, a=fov_radius * 0.08, b=fov_radius * 0.07,
                         angle=0.0, value=bone))
    # ribs near the boundary
    nrib = 8
    for k in range(nrib):
        t = (k + 0.5) / nrib * np.pi + rng.uniform(-0.05, 0.05)
        r = 0.86
        out.append(Ellipsoid(body.a * r * math.cos(t) * 0.97, body.b * r * math.sin(t) * 0.93 - 0.0,
                             a=fov_radius * 0.035, b=fov_radius * 0.02, angle=t, value=bone))
    # soft tissue organs
    tries = 0
    while len(out) < 22 and tries < 5000:
        tries += 1
        e = Ellipsoid(rng.uniform(-body.a * 0.7, body.a * 0.7), rng.uniform(-body.b * 0.55, body.b * 0.65),
                      a=fov_radius * rng.uniform(0.04, 0.18), b=fov_radius * rng.uniform(0.04, 0.14),
                      angle=rng.uniform(0, np.pi),
                      value=MU_WATER * rng.choice([-0.01, 0.01]))
        if not _boundary_inside(e, Ellipsoid(body.cx, body.cy, body.a * 0.78, body.b * 0.72, body.angle, 0.0)):
            continue
        if all(_disjoint(e, o, 1.0) for o in out[1:]):
            out.append(e)
    return out


# --------------------------------------------------------------------------
# counts, log sinogram and weights
# --------------------------------------------------------------------------

def noisy_data(p_true: np.ndarray, I0: float, seed: int, sigma: float = 0.0):
    """Counts, log sinogram y and statistical weights W (all FP64)."""
    rng = np.random.default_rng(seed)
    lam = I0 * np.exp(-p_true)
    counts = rng.poisson(lam).astype(np.float64)
    if sigma > 0:
        counts = counts + rng.normal(0.0, sigma, size=counts.shape)
    counts = np.maximum(counts, 1.0)
    y = np.log(I0 / counts)
    if sigma > 0:
        w = counts * counts / (counts + sigma * sigma)
    else:
        w = counts.copy()
    return counts, y, w


def seeded_uniform(shape, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Generic seeded uniform array (test inputs such as random images)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)
