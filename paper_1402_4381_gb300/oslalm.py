"""Python binding of liboslalm (include/oslalm.h): argument marshalling only.

Device memory and streams come from PyTorch tensors (``data_ptr()``) and
``torch.cuda.current_stream()``; every computation runs in the library's CUDA
kernels.  There is no fallback: if the library is not built or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

F32, F16, BF16 = 0, 1, 2
_DTYPES = {"f32": F32, "f16": F16, "bf16": BF16}
RHO_CONTINUATION, RHO_FIXED, RHO_REPLAY = 0, 1, 2
_RHO = {"continuation": RHO_CONTINUATION, "fixed": RHO_FIXED, "replay": RHO_REPLAY}
CURV_HUBER, CURV_MAX = 0, 1


class OslalmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liboslalm error {code}: {msg}")
        self.code = code


class GeomDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("offset_x", ctypes.c_double), ("offset_y", ctypes.c_double), ("offset_z", ctypes.c_double),
                ("nviews", ctypes.c_int), ("angle_start", ctypes.c_double), ("angle_span", ctypes.c_double),
                ("ns", ctypes.c_int), ("nt", ctypes.c_int), ("ds", ctypes.c_double), ("dt", ctypes.c_double),
                ("offset_s", ctypes.c_double), ("offset_t", ctypes.c_double),
                ("dso", ctypes.c_double), ("dsd", ctypes.c_double), ("pitch", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("delta", ctypes.c_double), ("nbr", ctypes.c_int), ("M", ctypes.c_int),
                ("rho_min", ctypes.c_double), ("n_inner", ctypes.c_int), ("rho_mode", ctypes.c_int),
                ("rho_fixed", ctypes.c_double), ("curvature", ctypes.c_int), ("w_dtype", ctypes.c_int),
                ("d_dtype", ctypes.c_int), ("use_graph", ctypes.c_int), ("bb", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("xi", ctypes.c_double), ("rho_used", ctypes.c_double), ("l", ctypes.c_int),
                ("restart", ctypes.c_int), ("subset", ctypes.c_int), ("pad", ctypes.c_int), ("alpha", ctypes.c_double)]


_lib = None
_VP = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def lib():
    """Load liboslalm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run __graft_entry__.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(path)
    i, d, ip = ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int)
    sig = {
        "oslalm_last_error": ([], ctypes.c_char_p),
        "oslalm_version": ([], i),
        "oslalm_geom_create": ([ctypes.POINTER(GeomDesc), ctypes.POINTER(_VP)], i),
        "oslalm_geom_destroy": ([_VP], i),
        "oslalm_subset_order": ([i, ip], i),
        "oslalm_subset_views": ([_VP, i, i, ip, ip], i),
        "oslalm_project": ([_VP, _VP, _VP, _VP, i, _VP], i),
        "oslalm_backproject": ([_VP, _VP, _VP, _VP, i, i, _VP], i),
        "oslalm_problem_create": ([_VP, _VP, _VP, ctypes.POINTER(Params), ctypes.POINTER(_VP)], i),
        "oslalm_problem_destroy": ([_VP], i),
        "oslalm_problem_set_data": ([_VP, _VP, _VP, _VP], i),
        "oslalm_init": ([_VP, _VP, _VP], i),
        "oslalm_iterate": ([_VP, _VP, i, ctypes.POINTER(Stats), _VP], i),
        "oslalm_set_replay": ([_VP, ip, i], i),
        "oslalm_cost": ([_VP, _VP, ctypes.POINTER(d), _VP], i),
        "oslalm_get_state": ([_VP, _VP, _VP, ctypes.POINTER(d), _VP], i),
        "oslalm_set_state": ([_VP, _VP, _VP, ctypes.POINTER(d), _VP], i),
        "oslalm_get_denominator": ([_VP, _VP, _VP], i),
        "oslalm_gradient": ([_VP, _VP, _VP, _VP], i),
        "oslalm_rmsd": ([_VP, _VP, _VP, ctypes.c_long, ctypes.POINTER(d), _VP], i),
        "oslalm_profile_iterate": ([_VP, _VP, i, ctypes.POINTER(d), ip, _VP], i),
        "oslalm_fbp": ([_VP, _VP, _VP, i, _VP], i),
        "oslalm_ray_table": ([ctypes.POINTER(GeomDesc), i, _VP, _VP, _VP, _VP], i),
        "oslalm_max_subsets": ([ctypes.POINTER(GeomDesc), d, ctypes.POINTER(d)], i),
        "oslalm_batch_create": ([ctypes.POINTER(_VP), i, ctypes.POINTER(_VP)], i),
        "oslalm_batch_destroy": ([_VP], i),
        "oslalm_batch_iterate": ([_VP, ctypes.POINTER(_VP), i, i, _VP], i),
        "oslalm_batch_autotune": ([_VP, ctypes.POINTER(_VP), i, ctypes.POINTER(d), _VP], i),
        "oslalm_batch_set_shape": ([_VP, i, i], i),
        "oslalm_batch_get_shape": ([_VP, ip, ip], i),
        "oslalm_batch_shape_count": ([], i),
        "oslalm_batch_shape_info": ([i, ip, ip, ip], i),
        "oslalm_cnn_param_count": ([], ctypes.c_long),
        "oslalm_cnn_create": ([i, i, i, ctypes.c_ulonglong, ctypes.POINTER(_VP)], i),
        "oslalm_cnn_destroy": ([_VP], i),
        "oslalm_cnn_get_params": ([_VP, _VP], i),
        "oslalm_cnn_mark_timeout": ([_VP], i),
        "oslalm_cnn_set_tma": ([_VP, ctypes.c_int], i),
        "oslalm_cnn_launch_count": ([], ctypes.c_long),
        "oslalm_cnn_set_params": ([_VP, _VP], i),
        "oslalm_cnn_forward": ([_VP, _VP, _VP, i, ctypes.c_float, _VP], i),
        "oslalm_cnn_gradients": ([_VP, _VP, _VP, i, ctypes.c_float, _VP, ctypes.POINTER(d), _VP], i),
        "oslalm_cnn_train_step": ([_VP, _VP, _VP, i, ctypes.c_float, ctypes.c_float, ctypes.POINTER(d), _VP], i),
        "oslalm_cnn_flops_per_image": ([i, i], d),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc, what):
    if rc != 0:
        msg = lib().oslalm_last_error().decode(errors="replace")
        raise OslalmError(rc, f"{what}: {msg}")


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _VP(s.cuda_stream)


def _ptr(t):
    return _VP(t.data_ptr()) if t is not None else _VP(0)


def _dev_f32(t, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape is not None and t.numel() != int(np.prod(shape)):
        raise ValueError(f"{name} has {t.numel()} elements, expected {int(np.prod(shape))}")
    return t


def geom_desc(geom) -> GeomDesc:
    d = GeomDesc()
    for name, _ in GeomDesc._fields_:
        setattr(d, name, getattr(geom, name))
    return d


def max_subsets(geom, s: float) -> float:
    """Sec. IV-B's largest number of subsets for s views per subset at the
    central voxel (axial or helical orbit; oslalm_max_subsets)."""
    out = ctypes.c_double()
    _check(lib().oslalm_max_subsets(ctypes.byref(geom_desc(geom)), float(s), ctypes.byref(out)), "max_subsets")
    return out.value


def ray_table(geom, view: int):
    """Host copy of the 2D per-ray parameters of one view (no GPU needed):
    dict(f0, kappa_lo, lrow: float32 [ns], packed: int32 [ns])."""
    ns = geom.ns
    f0 = np.zeros(ns, np.float32)
    kl = np.zeros(ns, np.float32)
    lr = np.zeros(ns, np.float32)
    pk = np.zeros(ns, np.int32)
    d = geom_desc(geom)
    _check(lib().oslalm_ray_table(ctypes.byref(d), int(view), f0.ctypes.data, kl.ctypes.data, lr.ctypes.data,
                                  pk.ctypes.data), "ray_table")
    return dict(f0=f0, kappa_lo=kl, lrow=lr, packed=pk)


def subset_order(M: int) -> List[int]:
    arr = (ctypes.c_int * M)()
    _check(lib().oslalm_subset_order(M, arr), "subset_order")
    return list(arr)


class Geometry:
    """Handle of an oslalm_geom built from a ``synth.Geometry`` description."""

    def __init__(self, geom):
        self.desc_py = geom
        d = geom_desc(geom)
        self._h = _VP()
        _check(lib().oslalm_geom_create(ctypes.byref(d), ctypes.byref(self._h)), "geom_create")
        self._views_all = None

    @property
    def handle(self):
        return self._h

    @property
    def image_shape(self):
        return self.desc_py.image_shape

    def sino_shape(self, nv=None):
        g = self.desc_py
        return (g.nviews if nv is None else nv, g.nt, g.ns)

    def views_tensor(self, views=None):
        import torch
        if views is None:
            if self._views_all is None:
                self._views_all = torch.arange(self.desc_py.nviews, dtype=torch.int32, device="cuda")
            return self._views_all
        if isinstance(views, torch.Tensor) and views.is_cuda:
            return views.to(torch.int32).contiguous()
        return torch.as_tensor(np.asarray(views, dtype=np.int32), device="cuda")

    def subset_views(self, M: int, m: int) -> List[int]:
        n = ctypes.c_int()
        arr = (ctypes.c_int * (self.desc_py.nviews // M + 1))()
        _check(lib().oslalm_subset_views(self._h, M, m, arr, ctypes.byref(n)), "subset_views")
        return list(arr[: n.value])

    def project(self, x, views=None, out=None, stream=None):
        import torch
        _dev_f32(x, self.image_shape, "x")
        vt = self.views_tensor(views)
        nv = int(vt.numel())
        if out is None:
            out = torch.empty(self.sino_shape(nv), dtype=torch.float32, device=x.device)
        _dev_f32(out, self.sino_shape(nv), "sino")
        _check(lib().oslalm_project(self._h, _ptr(x), _ptr(out), _ptr(vt), nv, _stream(stream)), "project")
        return out

    def backproject(self, sino, views=None, out=None, accumulate=False, stream=None):
        import torch
        vt = self.views_tensor(views)
        nv = int(vt.numel())
        _dev_f32(sino, self.sino_shape(nv), "sino")
        if out is None:
            out = torch.empty(self.image_shape, dtype=torch.float32, device=sino.device)
        _dev_f32(out, self.image_shape, "x")
        _check(lib().oslalm_backproject(self._h, _ptr(sino), _ptr(out), _ptr(vt), nv, int(accumulate),
                                        _stream(stream)), "backproject")
        return out


    def fbp(self, sino, out=None, clip=True, stream=None):
        """Filtered back-projection of the full sinogram (initial image)."""
        import torch
        _dev_f32(sino, self.sino_shape(), "sino")
        if out is None:
            out = torch.empty(self.image_shape, dtype=torch.float32, device=sino.device)
        _dev_f32(out, self.image_shape, "x")
        _check(lib().oslalm_fbp(self._h, _ptr(sino), _ptr(out), int(bool(clip)), _stream(stream)), "fbp")
        return out

    def close(self):
        if self._h:
            lib().oslalm_geom_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem:
    """PWLS problem + OS-LALM state (oslalm_problem)."""

    def __init__(self, geom: Geometry, y, w, *, beta, delta, nbr, M, rho_min=1e-3, rho_mode="continuation",
                 rho_fixed=1.0, curvature="huber", w_dtype="f32", d_dtype="f32", use_graph=True, n_inner=1,
                 bb=False):
        self.geom = geom
        shape = geom.sino_shape()
        _dev_f32(y, shape, "y")
        _dev_f32(w, shape, "w")
        p = Params()
        p.beta, p.delta, p.nbr, p.M = float(beta), float(delta), int(nbr), int(M)
        p.rho_min, p.n_inner = float(rho_min), int(n_inner)
        p.rho_mode, p.rho_fixed = _RHO[rho_mode], float(rho_fixed)
        p.curvature = CURV_HUBER if curvature == "huber" else CURV_MAX
        p.w_dtype, p.d_dtype = _DTYPES[w_dtype], _DTYPES[d_dtype]
        p.use_graph = int(bool(use_graph))
        p.bb = int(bool(bb))
        self.params = p
        self.M = int(M)
        self._h = _VP()
        _check(lib().oslalm_problem_create(geom.handle, _ptr(y), _ptr(w), ctypes.byref(p), ctypes.byref(self._h)),
               "problem_create")

    def set_data(self, y, w, stream=None):
        shape = self.geom.sino_shape()
        _dev_f32(y, shape, "y")
        _dev_f32(w, shape, "w")
        _check(lib().oslalm_problem_set_data(self._h, _ptr(y), _ptr(w), _stream(stream)), "set_data")

    def init(self, x, stream=None):
        _dev_f32(x, self.geom.image_shape, "x")
        _check(lib().oslalm_init(self._h, _ptr(x), _stream(stream)), "init")

    def iterate(self, x, n_iter=1, stats=False, stream=None):
        _dev_f32(x, self.geom.image_shape, "x")
        buf = None
        if stats:
            buf = (Stats * (n_iter * self.M))()
        _check(lib().oslalm_iterate(self._h, _ptr(x), int(n_iter), buf, _stream(stream)), "iterate")
        if stats:
            return [dict(xi=s.xi, rho_used=s.rho_used, l=s.l, restart=bool(s.restart), subset=s.subset, alpha=s.alpha)
                    for s in buf]
        return None

    def profile_iterate(self, x, n_iter=1, stream=None):
        """Device time (ms) per kernel kind over n_iter iterations, from CUDA
        events around each launch: dict(update, forward, backproject, launches)."""
        _dev_f32(x, self.geom.image_shape, "x")
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_int * 3)()
        _check(lib().oslalm_profile_iterate(self._h, _ptr(x), int(n_iter), ms, cnt, _stream(stream)),
               "profile_iterate")
        return dict(update=ms[0], forward=ms[1], backproject=ms[2], launches=list(cnt))

    def set_replay(self, restarts: Sequence[int]):
        arr = (ctypes.c_int * len(restarts))(*[int(bool(r)) for r in restarts])
        _check(lib().oslalm_set_replay(self._h, arr, len(restarts)), "set_replay")

    def cost(self, x, stream=None) -> float:
        _dev_f32(x, self.geom.image_shape, "x")
        out = ctypes.c_double()
        _check(lib().oslalm_cost(self._h, _ptr(x), ctypes.byref(out), _stream(stream)), "cost")
        return out.value

    def get_state(self, stream=None):
        import torch
        shape = self.geom.image_shape
        g = torch.empty(shape, dtype=torch.float32, device="cuda")
        z = torch.empty(shape, dtype=torch.float32, device="cuda")
        s = (ctypes.c_double * 4)()
        _check(lib().oslalm_get_state(self._h, _ptr(g), _ptr(z), s, _stream(stream)), "get_state")
        return dict(g=g, zeta=z, rho=s[0], l=int(s[1]), j=int(s[2]), alpha=s[3])

    def set_state(self, st, stream=None):
        s = (ctypes.c_double * 4)(st["rho"], st["l"], st["j"], st.get("alpha", 1.0))
        _check(lib().oslalm_set_state(self._h, _ptr(st["g"]), _ptr(st["zeta"]), s, _stream(stream)), "set_state")

    def gradient(self, x, stream=None):
        """A'W(Ax - y) + grad R(x) at x (oslalm_gradient), a new device tensor."""
        import torch
        _dev_f32(x, self.geom.image_shape, "x")
        gr = torch.empty(self.geom.image_shape, dtype=torch.float32, device=x.device)
        _check(lib().oslalm_gradient(self._h, _ptr(x), _ptr(gr), _stream(stream)), "gradient")
        return gr

    def denominator(self, stream=None):
        import torch
        d = torch.empty(self.geom.image_shape, dtype=torch.float32, device="cuda")
        _check(lib().oslalm_get_denominator(self._h, _ptr(d), _stream(stream)), "get_denominator")
        return d

    def close(self):
        if self._h:
            lib().oslalm_problem_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rmsd(x, xref, mask, stream=None) -> float:
    """sqrt(mean over mask of (x - xref)^2), FP64 reduction on the device."""
    import torch
    _dev_f32(x, None, "x")
    _dev_f32(xref, None, "xref")
    if mask.dtype != torch.uint8 or not mask.is_cuda:
        raise ValueError("mask must be a uint8 CUDA tensor")
    out = ctypes.c_double()
    _check(lib().oslalm_rmsd(_ptr(x), _ptr(xref), _ptr(mask), int(x.numel()), ctypes.byref(out), _stream(stream)),
           "rmsd")
    return out.value


class Batch:
    """Several initialised 2D problems advanced together (oslalm_batch)."""

    def __init__(self, problems: Sequence[Problem]):
        self.problems = list(problems)
        arr = (_VP * len(self.problems))(*[p._h for p in self.problems])
        self._h = _VP()
        _check(lib().oslalm_batch_create(arr, len(self.problems), ctypes.byref(self._h)), "batch_create")

    def _xs(self, xs):
        if len(xs) != len(self.problems):
            raise ValueError("one image per problem")
        for x, p in zip(xs, self.problems):
            _dev_f32(x, p.geom.image_shape, "x")
        return (_VP * len(xs))(*[x.data_ptr() for x in xs])

    def iterate(self, xs, n_iter=1, use_graph=True, stream=None):
        _check(lib().oslalm_batch_iterate(self._h, self._xs(xs), int(n_iter), int(bool(use_graph)), _stream(stream)),
               "batch_iterate")

    def autotune(self, xs, probe_iters=1, stream=None):
        n = lib().oslalm_batch_shape_count()
        ms = (ctypes.c_double * (2 * n))()
        _check(lib().oslalm_batch_autotune(self._h, self._xs(xs), int(probe_iters), ms, _stream(stream)),
               "batch_autotune")
        return [list(ms[2 * k: 2 * k + 2]) for k in range(n)]

    def set_shape(self, shape, blocks_per_sm=0):
        _check(lib().oslalm_batch_set_shape(self._h, int(shape), int(blocks_per_sm)), "batch_set_shape")

    def get_shape(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().oslalm_batch_get_shape(self._h, ctypes.byref(a), ctypes.byref(b)), "batch_get_shape")
        return a.value, b.value

    @staticmethod
    def shapes():
        out = []
        for k in range(lib().oslalm_batch_shape_count()):
            tx, ty, ln = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            _check(lib().oslalm_batch_shape_info(k, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(ln)), "shape")
            out.append(dict(tile=(tx.value, ty.value), lanes=ln.value))
        return out

    def close(self):
        if self._h:
            lib().oslalm_batch_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# the exchange layout of the network parameters (matches include/oslalm.h)
CNN_LAYERS = [("e0a", 1, 32), ("e0b", 32, 32), ("e1a", 32, 64), ("e1b", 64, 64), ("e2a", 64, 128),
              ("e2b", 128, 128), ("b3a", 128, 256), ("b3b", 256, 256), ("d2a", 384, 128), ("d2b", 128, 128),
              ("d1a", 192, 64), ("d1b", 64, 64), ("d0a", 96, 32), ("d0b", 32, 32)]


def cnn_flatten(params: dict) -> np.ndarray:
    """dict of arrays (names 'e0a.w' [co,3,3,ci], 'e0a.b', ..., 'out.w', 'out.b') -> flat float32."""
    parts = []
    for name, _, _ in CNN_LAYERS:
        parts += [np.asarray(params[name + ".w"]).ravel(), np.asarray(params[name + ".b"]).ravel()]
    parts += [np.asarray(params["out.w"]).ravel(), np.asarray(params["out.b"]).ravel()]
    return np.concatenate(parts).astype(np.float32)


def cnn_unflatten(flat: np.ndarray) -> dict:
    out, k = {}, 0
    for name, ci, co in CNN_LAYERS:
        n = co * 9 * ci
        out[name + ".w"] = flat[k:k + n].reshape(co, 3, 3, ci)
        k += n
        out[name + ".b"] = flat[k:k + co]
        k += co
    out["out.w"] = flat[k:k + 32]
    out["out.b"] = flat[k + 32:k + 33]
    return out


class WarmStartNet:
    """The warm-start U-Net (oslalm_cnn) for batches of `batch` images."""

    def __init__(self, batch, height, width, seed=0):
        self.batch, self.height, self.width = batch, height, width
        self._h = _VP()
        _check(lib().oslalm_cnn_create(int(batch), int(height), int(width), int(seed), ctypes.byref(self._h)),
               "cnn_create")

    @staticmethod
    def param_count():
        return int(lib().oslalm_cnn_param_count())

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count(), np.float32)
        _check(lib().oslalm_cnn_get_params(self._h, out.ctypes.data), "cnn_get_params")
        return out

    def mark_timeout(self):
        """Set the network's timed-out mark from the host (oslalm_cnn_mark_timeout)."""
        _check(lib().oslalm_cnn_mark_timeout(self._h), "cnn_mark_timeout")

    @staticmethod
    def launch_count() -> int:
        """Kernel launches issued so far by the network functions (oslalm_cnn_launch_count)."""
        return int(lib().oslalm_cnn_launch_count())

    def set_tma(self, enable: bool):
        """Use (default) or bypass the TMA convolution (oslalm_cnn_set_tma)."""
        _check(lib().oslalm_cnn_set_tma(self._h, int(bool(enable))), "cnn_set_tma")

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.param_count()
        _check(lib().oslalm_cnn_set_params(self._h, flat.ctypes.data), "cnn_set_params")

    def forward(self, x, scale, out=None, stream=None):
        import torch
        _dev_f32(x, (self.batch, self.height, self.width), "x")
        if out is None:
            out = torch.empty_like(x)
        _check(lib().oslalm_cnn_forward(self._h, _ptr(x), _ptr(out), self.batch, float(scale), _stream(stream)),
               "cnn_forward")
        return out

    def gradients(self, x, target, scale, stream=None):
        _dev_f32(x, (self.batch, self.height, self.width), "x")
        _dev_f32(target, (self.batch, self.height, self.width), "target")
        g = np.zeros(self.param_count(), np.float32)
        loss = ctypes.c_double()
        _check(lib().oslalm_cnn_gradients(self._h, _ptr(x), _ptr(target), self.batch, float(scale), g.ctypes.data,
                                          ctypes.byref(loss), _stream(stream)), "cnn_gradients")
        return loss.value, g

    def train_step(self, x, target, scale, lr, want_loss=True, stream=None):
        loss = ctypes.c_double()
        _check(lib().oslalm_cnn_train_step(self._h, _ptr(x), _ptr(target), self.batch, float(scale), float(lr),
                                           ctypes.byref(loss) if want_loss else None, _stream(stream)),
               "cnn_train_step")
        return loss.value if want_loss else None

    @staticmethod
    def flops_per_image(height, width):
        return float(lib().oslalm_cnn_flops_per_image(int(height), int(width)))

    def close(self):
        if self._h:
            lib().oslalm_cnn_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
