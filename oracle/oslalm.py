"""FP64 oracle of OS-LALM for PWLS X-ray CT reconstruction.

TEST INFRASTRUCTURE: a plain, slow restatement of the method, step by step in
the paper's order and notation, used only to check the CUDA path.

Problem (Sec. IV, Eq. ct_recon):
    x_hat = argmin_{x >= 0}  1/2 ||y - A x||_W^2 + R(x)
with the substitution of Eq. ct_substitution (A <- W^{1/2} A, y <- W^{1/2} y,
h <- R + indicator of the non-negative orthant), so that the data term is
l(x) = 1/2 ||y - Ax||_W^2 and grad l(x) = A' W (A x - y).

OS-LALM (Eq. os_lalm_iterates, Sec. III-A), one "subset-iteration":
    s      = rho * M grad l_m(x) + (1 - rho) g
    x+     = prox_{(rho^-1 t) h}(x - (rho^-1 t) s)        (inner problem)
    g+     = rho/(rho+1) * M grad l_{m+1}(x+) + 1/(rho+1) g
with the diagonal majorizer L_diag = diag{A' W A 1} (Sec. IV-A) in place of
L = 1/t, subsets taken in bit-reversal order (Sec. IV-A) and the
deterministic downward continuation of Eq. rho_l_formula_qp with the restart
indicator of Eq. period_indicator_qp evaluated with subset gradients at every
inner iteration (Sec. III-B).

Readings (the paper is silent or ambiguous):
* inner constrained denoising with n = 1 FISTA step from the warm start x
  (Sec. IV-A; Sec. V finds one inner step enough): one projected gradient step on
  phi(z) = R(z) + <s, z - x> + rho/2 ||z - x||_D^2 with the separable
  majorizer rho D + D_R(x):
      x+ = max(0, x - (s + grad R(x)) / (rho D + D_R(x)));
  a pixel whose majorizer is 0 (no ray crosses it and beta = 0: no
  curvature, no gradient) keeps its value;
* D_R(x) is the Huber-type SQS curvature of the hyperbola potential,
  omega(t) = psi'(t)/t, evaluated at x; the pairwise separable surrogate puts
  2 beta w_jk omega on each pixel of a pair;
* the split gradient starts at g = zeta = M grad l_{sigma(0)}(x0), rho = 1,
  l = 0 (Sec. III-A suggests g0 = grad l(x0));
* all three updates of a subset-iteration use the current rho_l; xi uses the
  old g and the old zeta; l and rho are updated after xi;
* bit-reversal for M not a power of two: bit-reverse 0 .. 2^ceil(log2 M)-1 and
  drop values >= M;
* the subset gradient scale is M (as printed) even when subsets are uneven;
* regularizer R(x) = beta sum_{j<k neighbours} w_jk psi(x_j - x_k) with the
  hyperbola psi(t) = delta^2 (sqrt(1 + (t/delta)^2) - 1), w_jk = 1/(index
  distance), missing neighbours at the border omitted.

Barzilai-Borwein scaling (supplement Sec. II-A, Eqs. secant_eq and
scale_factor_alpha_k), optional: the majorizer L_diag of the x-update becomes
H_k = alpha_k L_diag, with alpha_k the weighted least-squares fit of the secant
equation y_k ~ H_k s_k under P = L_diag^-1 and alpha <= 1:
    alpha* = s'y / s'L_diag s,  alpha = min(alpha*, 1).
Readings: k is the outer iteration (M subset-iterations), and the gradients
are replaced by their subset approximations with the SAME subset one
iteration apart: subset m's gradient zeta_m = M grad l_m is computed once per
iteration, at some iterate x_m; its secant pair over the last iteration is
s_m = x_m^(k) - x_m^(k-1), y_m = zeta_m^(k) - zeta_m^(k-1) (= M A_m'W_m A_m s_m
for the data term, a curvature of the subset that never changes sign; the
gradients of two different subsets would not be).  At the end of iteration k
    alpha = min(sum_m s_m'y_m / sum_m s_m'L_diag s_m, 1)
over the subsets with a pair, and H = alpha L_diag serves the x-updates of
iteration k + 1.  alpha = 1 (the plain majorizer) until the first pairs exist
and whenever the fit has no positive curvature (sum s'y <= 0) or s = 0.
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional, Sequence

import numpy as np

# --------------------------------------------------------------------------
# subsets (Sec. IV-A bit-reversal order, Sec. IV-B uniform view interleave)
# --------------------------------------------------------------------------


def subset_views(nviews: int, M: int, m: int) -> np.ndarray:
    """Views of subset m: every M-th view starting at m (views spread uniformly)."""
    return np.arange(m, nviews, M, dtype=np.int32)


def bit_reversal_order(M: int) -> List[int]:
    """Subset visiting order by bit reversal (reading for M not a power of two:
    reverse the bits of 0..2^b-1, b = ceil(log2 M), keep values < M)."""
    if M <= 0:
        raise ValueError("M must be positive")
    if M == 1:
        return [0]
    b = int(math.ceil(math.log2(M)))
    out = []
    for i in range(1 << b):
        r = 0
        for k in range(b):
            if i & (1 << k):
                r |= 1 << (b - 1 - k)
        if r < M:
            out.append(r)
    return out


# --------------------------------------------------------------------------
# continuation (Sec. III-B, Eq. rho_l_formula_qp)
# --------------------------------------------------------------------------


def rho_l(l: int, rho_min: float = 1e-3) -> float:
    """AL penalty of the deterministic downward continuation at counter l."""
    if l == 0:
        return 1.0
    v = math.pi / (l + 1) * math.sqrt(1.0 - (math.pi / (2 * l + 2)) ** 2)
    return max(v, rho_min)


# --------------------------------------------------------------------------
# edge-preserving hyperbola regularizer (Sec. IV: R edge-preserving)
# --------------------------------------------------------------------------


def psi(t, delta):
    return delta * delta * (np.sqrt(1.0 + (t / delta) ** 2) - 1.0)


def dpsi(t, delta):
    return t / np.sqrt(1.0 + (t / delta) ** 2)


def omega(t, delta):
    """psi'(t)/t: the Huber curvature of the hyperbola."""
    return 1.0 / np.sqrt(1.0 + (t / delta) ** 2)


def neighbour_offsets(nbr: int):
    """Half neighbourhood (each unordered pair once) as ((dz, dy, dx), w_jk)."""
    if nbr == 4:
        offs = [(0, 0, 1), (0, 1, 0)]
    elif nbr == 8:
        offs = [(0, 0, 1), (0, 1, 0), (0, 1, 1), (0, 1, -1)]
    elif nbr == 6:
        offs = [(0, 0, 1), (0, 1, 0), (1, 0, 0)]
    elif nbr == 26:
        offs = []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    o = (dz, dy, dx)
                    if o > (0, 0, 0):  # lexicographically positive half
                        offs.append(o)
    else:
        raise ValueError(f"unsupported neighbourhood {nbr}")
    return [(o, 1.0 / math.sqrt(o[0] ** 2 + o[1] ** 2 + o[2] ** 2)) for o in offs]


def _pair_slices(shape, o):
    """Slices (j, k) such that x[k] is the neighbour x[j + o], both in bounds."""
    sj, sk = [], []
    for n, d in zip(shape, o):
        sj.append(slice(max(0, -d), n - max(0, d)))
        sk.append(slice(max(0, d), n - max(0, -d)))
    return tuple(sj), tuple(sk)


def reg_value(x, beta, delta, nbr):
    x = np.asarray(x, dtype=np.float64)
    tot = 0.0
    for o, w in neighbour_offsets(nbr):
        sj, sk = _pair_slices(x.shape, o)
        tot += beta * w * np.sum(psi(x[sj] - x[sk], delta))
    return float(tot)


def reg_grad(x, beta, delta, nbr):
    x = np.asarray(x, dtype=np.float64)
    g = np.zeros_like(x)
    for o, w in neighbour_offsets(nbr):
        sj, sk = _pair_slices(x.shape, o)
        d = beta * w * dpsi(x[sj] - x[sk], delta)
        g[sj] += d
        g[sk] -= d
    return g


def reg_curv(x, beta, delta, nbr, mode: str = "huber"):
    """Diagonal SQS curvature D_R of R at x ("huber": omega(x_j-x_k); "max": omega=1)."""
    x = np.asarray(x, dtype=np.float64)
    c = np.zeros_like(x)
    for o, w in neighbour_offsets(nbr):
        sj, sk = _pair_slices(x.shape, o)
        if mode == "huber":
            om = omega(x[sj] - x[sk], delta)
        else:
            om = np.ones_like(x[sj])
        d = 2.0 * beta * w * om
        c[sj] += d
        c[sk] += d
    return c


# --------------------------------------------------------------------------
# the PWLS data term on top of a subset projector pair
# --------------------------------------------------------------------------


class SubsetData:
    """y, W split by subsets plus the subset projector pair A_m, A_m'."""

    def __init__(self, A_m: Callable, At_m: Callable, y_sub: Sequence[np.ndarray],
                 w_sub: Sequence[np.ndarray], M: int):
        self.A_m, self.At_m = A_m, At_m
        self.y = [np.asarray(a, dtype=np.float64) for a in y_sub]
        self.w = [np.asarray(a, dtype=np.float64) for a in w_sub]
        self.M = M

    def grad_subset(self, x, m):
        """M grad l_m(x) = M A_m' W_m (A_m x - y_m) (Eq. os_lalm_iterates)."""
        r = self.M * self.w[m] * (self.A_m(x, m) - self.y[m])
        return self.At_m(r, m)

    def data_cost(self, x):
        tot = 0.0
        for m in range(self.M):
            res = self.y[m] - self.A_m(x, m)
            tot += 0.5 * float(np.sum(self.w[m] * res * res))
        return tot

    def sqs_denominator(self, shape):
        """L_diag = A' W A 1 (Sec. IV-A), summed over all subsets."""
        ones = np.ones(shape)
        D = np.zeros(shape)
        for m in range(self.M):
            D += self.At_m(self.w[m] * self.A_m(ones, m), m)
        return D


def ct_subset_data(geom, y, w, M, projector):
    """SubsetData for a CT scan (views interleaved by subset)."""
    views = [subset_views(geom.nviews, M, m) for m in range(M)]
    y = np.asarray(y, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)

    def A_m(x, m):
        return projector.project(geom, x, views[m])

    def At_m(r, m):
        return projector.backproject(geom, r, views[m])

    return SubsetData(A_m, At_m, [y[v] for v in views], [w[v] for v in views], M), views


# --------------------------------------------------------------------------
# OS-LALM
# --------------------------------------------------------------------------


def fista_momentum(n: int):
    """FISTA (Beck & Teboulle 2009) momentum weights gamma_i = (tau_i - 1) /
    tau_{i+1}, tau_0 = 1, tau_{i+1} = (1 + sqrt(1 + 4 tau_i^2)) / 2, for the
    inner steps i = 0..n-1 (gamma_0 = 0)."""
    tau, out = 1.0, []
    for _ in range(n):
        tn = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * tau * tau))
        out.append((tau - 1.0) / tn)
        tau = tn
    return out


class OsLalm:
    """OS-LALM with n inner FISTA steps (n = 1: one projected SQS step),
    fixed rho or downward continuation, optional Barzilai-Borwein scaling of
    the majorizer."""

    def __init__(self, data: SubsetData, D, beta: float, delta: float, nbr: int,
                 order: Optional[Sequence[int]] = None, rho_mode: str = "continuation",
                 rho_fixed: float = 1.0, rho_min: float = 1e-3, curvature: str = "huber",
                 nonneg: bool = True, replay: Optional[Sequence[int]] = None, n_inner: int = 1,
                 bb: bool = False):
        self.data = data
        self.M = data.M
        self.D = np.asarray(D, dtype=np.float64)
        self.beta, self.delta, self.nbr = beta, delta, nbr
        self.order = list(order) if order is not None else bit_reversal_order(self.M)
        self.rho_mode = rho_mode
        self.rho_fixed = rho_fixed
        self.rho_min = rho_min
        self.curvature = curvature
        self.nonneg = nonneg
        self.replay = replay
        self.n_inner = int(n_inner)
        self.bb = bool(bb)
        self.alpha = 1.0
        self._bb_prev = {}  # subset -> (x, zeta) of its last gradient evaluation
        self._bb_sums = [0.0, 0.0]  # sum s'y, sum s'Ds of the current iteration
        self.history = []

    def init(self, x0):
        self.x = np.array(x0, dtype=np.float64)
        self.j = 0  # subset-iterations done
        self.zeta = self.data.grad_subset(self.x, self.order[0])
        self.g = self.zeta.copy()
        self.l = 0
        self.rho = 1.0 if self.rho_mode == "continuation" else self.rho_fixed
        self.alpha = 1.0
        self._bb_prev = {self.order[0]: (self.x.copy(), self.zeta.copy())}
        self._bb_sums = [0.0, 0.0]

    def _reg(self, x):
        if self.beta == 0.0:
            return np.zeros_like(x), np.zeros_like(x)
        return (reg_grad(x, self.beta, self.delta, self.nbr),
                reg_curv(x, self.beta, self.delta, self.nbr, self.curvature))

    def inner(self, x, s, rho):
        """The x-update of Eq. os_lalm_iterates with h = R + iota_Omega (Sec.
        IV-A): the constrained denoising problem
            min_{v in Omega}  Phi(v) = R(v) + (rho/2) ||v - x + D^-1 s / rho||_D^2
        by n FISTA steps from the warm start x.  Step i takes a projected
        separable-quadratic-surrogate step from the extrapolated point v_i
        with the denominators rho D + D_R(v_i):
            u_{i+1} = P_Omega(v_i - grad Phi(v_i) / (rho D + D_R(v_i))),
            grad Phi(v) = grad R(v) + s + rho D (v - x),
            v_{i+1} = u_{i+1} + gamma_i (u_{i+1} - u_i),  u_0 = v_0 = x,
        and returns u_n.  n = 1 is the single projected step
        x - (s + grad R(x)) / (rho D + D_R(x)).  With Barzilai-Borwein
        scaling, H = alpha D takes the place of D."""
        gam = fista_momentum(self.n_inner)
        H = self.alpha * self.D
        u_prev, v = x, x
        for i in range(self.n_inner):
            gR, DR = self._reg(v)
            den = rho * H + DR
            safe = np.where(den > 0.0, den, 1.0)
            if i == 0:
                u = np.where(den > 0.0, x - (s + gR) / safe, x)
            else:
                u = np.where(den > 0.0, v - (gR + s + rho * H * (v - x)) / safe, v)
            if self.nonneg:
                u = np.maximum(u, 0.0)
            v = u + gam[i] * (u - u_prev)
            u_prev = u
        return u_prev

    def step(self):
        rho, x, g, zeta = self.rho, self.x, self.g, self.zeta
        # search direction and the inner constrained denoising (n steps)
        s = rho * zeta + (1.0 - rho) * g
        x_new = self.inner(x, s, rho)
        # next subset gradient and split-gradient update
        m_next = self.order[(self.j + 1) % self.M]
        zeta_new = self.data.grad_subset(x_new, m_next)
        g_new = (rho * zeta_new + g) / (rho + 1.0)
        # restart indicator with subset-gradient approximations
        xi = float(np.sum((g - zeta_new) * (zeta_new - zeta)))
        restart = None
        if self.rho_mode == "continuation":
            if self.replay is not None:
                restart = bool(self.replay[self.j])
            else:
                restart = xi > 0.0
            self.l = 0 if restart else self.l + 1
            self.rho = rho_l(self.l, self.rho_min)
        alpha_used = self.alpha
        if self.bb:  # secant pair of subset m_next over the last iteration
            prev = self._bb_prev.get(m_next)
            if prev is not None:
                sk, yk = x_new - prev[0], zeta_new - prev[1]
                self._bb_sums[0] += float(np.sum(sk * yk))
                self._bb_sums[1] += float(np.sum(self.D * sk * sk))
            self._bb_prev[m_next] = (x_new.copy(), zeta_new.copy())
            if (self.j + 1) % self.M == 0:  # end of an iteration: refit H = alpha D
                num, den = self._bb_sums
                self.alpha = min(num / den, 1.0) if (den > 0.0 and num > 0.0) else 1.0
                self._bb_sums = [0.0, 0.0]
        self.history.append(dict(j=self.j, rho_used=rho, xi=xi, restart=restart, l=self.l,
                                 alpha_used=alpha_used, alpha=self.alpha))
        self.x, self.g, self.zeta = x_new, g_new, zeta_new
        self.j += 1

    def run(self, n_subiters: int):
        for _ in range(n_subiters):
            self.step()
        return self.x

    def cost(self, x=None):
        x = self.x if x is None else x
        return self.data.data_cost(x) + reg_value(x, self.beta, self.delta, self.nbr)


# --------------------------------------------------------------------------
# evaluation (Sec. V: RMS difference in the region of interest, in HU)
# --------------------------------------------------------------------------

HU = 0.0192 / 1000.0


def roi_mask(geom):
    """Pixels inside the scanner's field of view (reading of "region of
    interest"); for the cone beam also voxels that project inside the
    detector rows from every view (circular orbit), or lie between the first
    and last source heights (helix)."""
    ix = (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.dx + geom.offset_x
    iy = (np.arange(geom.ny) - (geom.ny - 1) / 2.0) * geom.dy + geom.offset_y
    Y, X = np.meshgrid(iy, ix, indexing="ij")
    r = np.sqrt(X * X + Y * Y)
    # lateral positions of the outer edges of the first and last detector cell
    s_edge = np.array([-geom.ns / 2.0 + geom.offset_s, geom.ns / 2.0 + geom.offset_s]) * geom.ds
    if geom.kind == 0:  # parallel: the band between the edge rays
        R = float(np.min(np.abs(s_edge)))
    elif geom.kind == 1:  # arc detector: the edge rays leave the source at angle s / dsd
        R = geom.dso * float(np.min(np.sin(np.abs(s_edge) / geom.dsd)))
    else:  # flat detector: at angle atan(s / dsd)
        R = geom.dso * float(np.min(np.sin(np.arctan(np.abs(s_edge) / geom.dsd))))
    m2 = r <= R
    if geom.kind != 2:
        return m2[None]
    iz = (np.arange(geom.nz) - (geom.nz - 1) / 2.0) * geom.dz + geom.offset_z
    if getattr(geom, "pitch", 0.0) != 0.0:  # helix (reading): the cylinder between the first and last source heights
        zs = geom.source_z()
        return m2[None] & ((iz >= zs.min()) & (iz <= zs.max()))[:, None, None]
    tmax = geom.nt * geom.dt / 2.0
    mag = geom.dsd / np.maximum(geom.dso - r, 1e-9)
    return m2[None] & (np.abs(iz)[:, None, None] * mag[None] <= tmax)


def rmsd_hu(x, xref, mask):
    d = (np.asarray(x, dtype=np.float64) - np.asarray(xref, dtype=np.float64))[mask]
    return float(np.sqrt(np.mean(d * d)) / HU)
