"""Helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

# Tolerances (stated in the parity contract): per-ray (and per-pixel)
# |gpu - oracle| <= 1e-5 * max(|oracle|, 1e-3 * max|oracle|); adjoint relative
# gap <= 1e-6; cost relative difference <= 1e-5; image RMSD <= 0.5 HU.
RAY_RTOL = 1e-5
RAY_FLOOR = 1e-3
ADJ_TOL = 1e-6
COST_RTOL = 1e-5
RMSD_HU_TOL = 0.5
HU = 0.0192 / 1000.0


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def assert_rel_floor(got, ref, rtol=RAY_RTOL, floor=RAY_FLOOR, what="values"):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    scale = np.maximum(np.abs(ref), floor * np.max(np.abs(ref)))
    err = np.abs(got - ref)
    bad = err > rtol * scale
    if np.any(bad):
        i = np.unravel_index(np.argmax(err / np.maximum(scale, 1e-300)), ref.shape)
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} outside tolerance; worst at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r} rel {err[i] / scale[i]:.3e}")
    worst = float(np.max(err / np.maximum(scale, 1e-300)))
    # the same without the floor, over the entries not near zero (|ref| above
    # 1e-6 of the largest): how far the floor loosens the per-entry bound
    big = np.abs(ref) > 1e-6 * np.max(np.abs(ref))
    raw = float(np.max(err[big] / np.abs(ref[big]))) if np.any(big) else 0.0
    print(f"{what}: worst relative error {worst:.2e} with the floor, {raw:.2e} without it")
    return worst
