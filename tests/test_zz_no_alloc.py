"""The allocation-free FBP entry point (oslalm_fbp_noalloc) against the
regular one (oslalm_fbp), called through the C ABI.

oslalm_fbp_noalloc exists for callers that must not allocate device memory
once they are running (a service whose memory pool owns the GPU, a pipeline
that forbids cudaMalloc after start-up); it keeps its filtered sinogram in a
fixed buffer inside the library, reserved by oslalm_fbp_noalloc_prepare at
start-up.  Both entry points run the same kernels on the same samples, so
their images must agree bit for bit.  This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1402_4381_gb300 import synth, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_4381_gb300 import build, oslalm
    build.build()
    lib = oslalm.lib()
    lib.oslalm_fbp_noalloc.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
    lib.oslalm_fbp_noalloc.restype = ctypes.c_int
    lib.oslalm_fbp_noalloc_prepare.argtypes = []
    lib.oslalm_fbp_noalloc_prepare.restype = ctypes.c_int
    torch.cuda.set_device(0)
    assert lib.oslalm_fbp_noalloc_prepare() == 0, lib.oslalm_last_error()
    return oslalm


def _scan(g, seed):
    ph = synth.random_ellipse_phantom(seed, 0.4 * g.nx * g.dx, 6)
    return synth.analytic_sinogram(g, ph).astype(np.float32)


@pytest.mark.parametrize("g", [W.c1_fan().geom, W.c0_parallel().geom])
def test_noalloc_fbp_matches_fbp_twice(L, g):
    import torch
    geom = L.Geometry(g)
    stream = L._stream()
    for call, seed in enumerate((21, 22)):  # two calls in a row, different data
        sino = torch.as_tensor(_scan(g, seed), device="cuda")
        ref = geom.fbp(sino, clip=True)
        out = torch.full(g.image_shape, float("nan"), device="cuda")
        rc = L.lib().oslalm_fbp_noalloc(geom.handle, L._ptr(sino), L._ptr(out), 1, stream)
        assert rc == 0, L.lib().oslalm_last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.array_equal(a, b), (call, float(np.max(np.abs(a - b))))


def test_noalloc_fbp_leaves_free_memory_unchanged(L):
    """After the prepare call, a call reserves no device memory: the device's
    free memory (cudaMemGetInfo) is the same before and after two calls."""
    import torch
    g = W.c1_fan().geom
    geom = L.Geometry(g)
    sino = torch.as_tensor(_scan(g, 23), device="cuda")
    out = torch.empty(g.image_shape, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        rc = L.lib().oslalm_fbp_noalloc(geom.handle, L._ptr(sino), L._ptr(out), 1, L._stream())
        assert rc == 0, L.lib().oslalm_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_fbp_rejects_oversized_sinogram(L):
    import torch
    g = synth.Geometry(kind=2, nx=8, ny=8, nz=4, dx=1, dy=1, dz=1, nviews=1000, angle_span=2 * math.pi,
                       ns=100, nt=64, ds=1.0, dt=1.0, dso=50, dsd=90)
    geom = L.Geometry(g)
    sino = torch.zeros(g.sino_shape, device="cuda")
    out = torch.zeros(g.image_shape, device="cuda")
    rc = L.lib().oslalm_fbp_noalloc(geom.handle, L._ptr(sino), L._ptr(out), 1, L._stream())
    assert rc == -3
    assert b"static buffer" in L.lib().oslalm_last_error()
