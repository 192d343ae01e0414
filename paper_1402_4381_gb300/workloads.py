"""Named synthetic workloads (scan geometry, phantom recipe, noise and the
PWLS/OS-LALM parameters).  Pure description: no method arithmetic.

The three single-scan workloads stand in for the paper's proprietary GE
scans (Sec. V): they take the axial GE performance-phantom detector
(888 channels, 64 rows, 984 views, Sec. V-B) and its 24 subsets.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import synth
from .synth import CONE3D_FLAT, FAN2D_ARC, PAR2D, Geometry


@dataclasses.dataclass
class Workload:
    name: str
    geom: Geometry
    phantom: str  # "ellipses" | "torso" | "ellipsoids"
    phantom_seed: int
    noise_seed: int
    n_ellipses: int
    fov_radius: float
    I0: float
    sigma: float
    beta: float
    delta: float  # /mm
    nbr: int  # 4, 8 (2D) or 6, 26 (3D)
    M: int
    n_iter: int
    w_dtype: str = "f32"  # storage of W: f32 | f16 | bf16
    d_dtype: str = "f32"  # storage of the SQS denominator D: f32 | f16 | bf16

    def make_phantom(self):
        if self.phantom == "ellipses":
            return synth.random_ellipse_phantom(self.phantom_seed, self.fov_radius, self.n_ellipses)
        if self.phantom == "torso":
            return synth.torso_phantom(self.phantom_seed, self.fov_radius)
        if self.phantom == "ellipsoids":
            zh = self.geom.nz * self.geom.dz / 2.0
            return synth.random_ellipse_phantom(self.phantom_seed, self.fov_radius, self.n_ellipses,
                                                three_d=True, z_half=zh)
        raise ValueError(self.phantom)

    def make_scan(self, views=None):
        """Return dict(phantom, p_true, counts, y, w) with y, w as float32 arrays."""
        ph = self.make_phantom()
        p = synth.analytic_sinogram(self.geom, ph, views)
        counts, y, w = synth.noisy_data(p, self.I0, self.noise_seed, self.sigma)
        return dict(phantom=ph, p_true=p, counts=counts,
                    y=y.astype(np.float32), w=w.astype(np.float32))


DELTA_10HU = 10.0 * synth.HU  # 1.92e-4 /mm


def c0_parallel() -> Workload:
    """2D parallel beam 128x128, 180 views / 180 deg, 185 bins, M=10."""
    g = Geometry(kind=PAR2D, nx=128, ny=128, dx=1.0, dy=1.0, nviews=180,
                 angle_start=0.0, angle_span=math.pi, ns=185, ds=1.0)
    return Workload("parallel2d_128_v180_b185_M10", g, "ellipses", 1001, 2001, 10, 60.0,
                    I0=1e5, sigma=0.0, beta=2.0 ** 10, delta=DELTA_10HU, nbr=8, M=10, n_iter=20)


def c1_fan() -> Workload:
    """2D fan beam (arc detector) 512x512, 984 views / 360 deg, 888 channels, M=24."""
    g = Geometry(kind=FAN2D_ARC, nx=512, ny=512, dx=0.9766, dy=0.9766, nviews=984,
                 angle_start=0.0, angle_span=2 * math.pi, ns=888, ds=1.0239, dso=541.0, dsd=949.0)
    return Workload("fan2d_512_v984_c888_M24", g, "torso", 1101, 2101, 22, 240.0,
                    I0=1e5, sigma=5.0, beta=2.0 ** 10, delta=DELTA_10HU, nbr=8, M=24, n_iter=50,
                    w_dtype="f16", d_dtype="f16")


def c2_cone() -> Workload:
    """3D circular cone beam, flat detector, 512x512x128, 888x64 cells, 984 views, M=12."""
    g = Geometry(kind=CONE3D_FLAT, nx=512, ny=512, nz=128, dx=0.9766, dy=0.9766, dz=0.625,
                 nviews=984, angle_start=0.0, angle_span=2 * math.pi, ns=888, nt=64,
                 ds=1.0239, dt=1.0963, dso=541.0, dsd=949.0)
    return Workload("cone3d_512x512x128_v984_888x64_M12", g, "ellipsoids", 1201, 2201, 20, 240.0,
                    I0=5e4, sigma=0.0, beta=2.0 ** 10, delta=DELTA_10HU, nbr=26, M=12, n_iter=30,
                    w_dtype="bf16")


def c1_fan_256() -> Workload:
    """The fan-beam scan family at 256^2 pixels, 492 views (M = 12 subsets of
    41 views): one of the batched workload's sizes, and a case small enough
    for detailed kernel profiling."""
    return scaled(c1_fan(), 256, 492, 888, 12, name_suffix="256")


def scaled(w: Workload, nx: int, nviews: int, ns: int, M: int, name_suffix="small",
           nz: int | None = None, nt: int | None = None) -> Workload:
    """Same scan family at a smaller size (same field of view and fan angles)."""
    g = dataclasses.replace(w.geom)
    fov_x = g.nx * g.dx
    g.nx = g.ny = nx
    g.dx = g.dy = fov_x / nx
    det_w = g.ns * g.ds
    g.ns = ns
    g.ds = det_w / ns
    g.nviews = nviews
    if nz is not None:
        zlen = g.nz * g.dz
        g.nz = nz
        g.dz = zlen / nz
    if nt is not None:
        tlen = g.nt * g.dt
        g.nt = nt
        g.dt = tlen / nt
    return dataclasses.replace(w, name=f"{w.name}_{name_suffix}", geom=g, M=M)


def tiny_parallel(n: int = 8, nviews: int = 6, ns: int = 13) -> Geometry:
    return Geometry(kind=PAR2D, nx=n, ny=n, dx=1.0, dy=1.0, nviews=nviews,
                    angle_start=0.1, angle_span=math.pi, ns=ns, ds=1.0)


def tiny_fan(n: int = 8, nviews: int = 8, ns: int = 15) -> Geometry:
    return Geometry(kind=FAN2D_ARC, nx=n, ny=n, dx=1.0, dy=1.0, nviews=nviews,
                    angle_start=0.05, angle_span=2 * math.pi, ns=ns, ds=1.3, dso=20.0, dsd=35.0)


def tiny_cone(n: int = 8, nz: int = 4, nviews: int = 8, ns: int = 15, nt: int = 7) -> Geometry:
    return Geometry(kind=CONE3D_FLAT, nx=n, ny=n, nz=nz, dx=1.0, dy=1.0, dz=0.8, nviews=nviews,
                    angle_start=0.05, angle_span=2 * math.pi, ns=ns, nt=nt, ds=1.3, dt=1.1,
                    dso=20.0, dsd=35.0)


def tiny_helical(n: int = 8, nz: int = 6, nviews: int = 16, ns: int = 15, nt: int = 5, pitch: float = 0.8) -> Geometry:
    """Two turns of a helical cone-beam orbit over a small volume."""
    return Geometry(kind=CONE3D_FLAT, nx=n, ny=n, nz=nz, dx=1.0, dy=1.0, dz=0.8, nviews=nviews,
                    angle_start=0.05, angle_span=4 * math.pi, ns=ns, nt=nt, ds=1.3, dt=1.1,
                    dso=20.0, dsd=35.0, pitch=pitch)


def c2_helical() -> Workload:
    """Helical cone beam with the detector of the cone workload: 512x512x64
    voxels (0.9766^2 x 0.625 mm), 888 x 64 cells, 2 turns of 984 views at pitch
    0.5 (table feed 35 mm per turn), 20 ellipsoids, I0 = 5e4, 26 neighbours,
    M = 36 (Sec. IV-B's helical maximum for s = 24 is 46)."""
    w = c2_cone()
    g = dataclasses.replace(w.geom, nz=64, nviews=2 * 984, angle_span=4 * math.pi, pitch=0.5)
    return dataclasses.replace(w, name="helical_512x512x64_v1968_c888x64_p0.5_M36", geom=g, M=36, n_iter=20)


def c3_batch(n_slices: int = 64, seed: int = 1301, n_iter: int = 30):
    """Batched 2D fan beam: n independent slices, image sizes uniform in
    {256^2, 384^2, 512^2} over a 500 mm field of view, view counts uniform in
    {492, 738, 984}, 888 channels, seeded ellipse phantoms, I0 uniform in
    [2e4, 2e5], M = views / 41 subsets, n_iter iterations."""
    rng = np.random.default_rng(seed)
    base = c1_fan()
    out = []
    for k in range(n_slices):
        n = int(rng.choice([256, 384, 512]))
        nv = int(rng.choice([492, 738, 984]))
        g = dataclasses.replace(base.geom, nx=n, ny=n, dx=500.0 / n, dy=500.0 / n, nviews=nv)
        I0 = float(rng.uniform(2e4, 2e5))
        out.append(dataclasses.replace(base, name=f"batch_slice{k}_{n}_v{nv}", geom=g, phantom="ellipses",
                                       phantom_seed=seed * 1000 + k, noise_seed=seed * 1000 + 500 + k,
                                       n_ellipses=10, I0=I0, sigma=0.0, M=nv // 41, n_iter=n_iter,
                                       w_dtype="f32", d_dtype="f32"))
    return out
