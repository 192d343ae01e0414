"""C-ABI boundary checks that need no GPU: the library loads, exports every
entry point declared in include/*.h, and its host-only logic (subset order and
views, argument validation) behaves as documented."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import oslalm as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(oslalm_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_1402_4381_gb300 import build, oslalm
    build.build()
    return oslalm.lib()


def test_header_declares_entry_points():
    names = _declared()
    for n in ["oslalm_geom_create", "oslalm_subset_order", "oslalm_subset_views", "oslalm_project",
              "oslalm_backproject", "oslalm_iterate", "oslalm_cost", "oslalm_init"]:
        assert n in names


def test_every_declared_symbol_is_exported(L):
    from paper_1402_4381_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(oslalm_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(L, n)


def test_subset_order_matches_oracle(L):
    from paper_1402_4381_gb300 import oslalm
    for M in [1, 2, 3, 8, 10, 12, 24, 41, 64]:
        assert oslalm.subset_order(M) == O.bit_reversal_order(M)


def test_version_and_error_string(L):
    assert L.oslalm_version() >= 100
    assert isinstance(L.oslalm_last_error(), bytes)


def test_geometry_validation_rejects_bad_descriptors(L):
    from paper_1402_4381_gb300 import oslalm
    d = oslalm.GeomDesc()
    d.kind, d.nx, d.ny, d.nz, d.nviews, d.ns, d.nt = 1, 8, 8, 1, 4, 5, 1
    d.dx = d.dy = d.dz = d.ds = d.dt = 1.0
    d.dso, d.dsd = 3.0, 10.0  # image box radius 5.66 mm outside the source circle
    h = ctypes.c_void_p()
    rc = L.oslalm_geom_create(ctypes.byref(d), ctypes.byref(h))
    assert rc == -1 and not h.value
    assert b"source circle" in L.oslalm_last_error()
    d.dso = 20.0
    d.nx = 0
    assert L.oslalm_geom_create(ctypes.byref(d), ctypes.byref(h)) == -1
    d.nx, d.nt = 8, 3  # 2D needs nt = 1
    assert L.oslalm_geom_create(ctypes.byref(d), ctypes.byref(h)) == -1
    assert L.oslalm_geom_create(None, ctypes.byref(h)) == -1


def test_null_handles_are_errors_not_crashes(L):
    from paper_1402_4381_gb300 import oslalm
    assert L.oslalm_iterate(None, None, 1, None, None) == -1
    assert L.oslalm_cost(None, None, None, None) == -1
    assert L.oslalm_project(None, None, None, None, 1, None) == -1
    assert L.oslalm_subset_order(0, None) == -1
    assert L.oslalm_problem_destroy(None) == 0
    assert L.oslalm_geom_destroy(None) == 0
    out = ctypes.c_double()
    assert L.oslalm_rmsd(None, None, None, 0, ctypes.byref(out), None) == -1
    with pytest.raises(oslalm.OslalmError):
        oslalm._check(L.oslalm_subset_order(-3, None), "subset_order")


def test_max_subsets_rule_on_the_papers_scanner():
    """Sec. IV-B with the GE scanner of the paper's experiments (984 views per
    turn, dso 541 mm, dsd 949 mm): axial 984 views / s = 40 -> 24 (the paper
    suggests about 24 for the axial GE performance phantom); helical s = 24:
    pitch 0.5 -> 46 (about 40 for the shoulder), pitch 1.0 -> 23 (about 20 for
    the abdomen), inversely proportional to the pitch."""
    import math
    from paper_1402_4381_gb300 import oslalm, synth
    ax = synth.Geometry(kind=synth.FAN2D_ARC, nx=8, ny=8, nviews=984, angle_span=2 * math.pi, ns=888,
                        ds=1.0239, dso=541.0, dsd=949.0)
    assert math.floor(oslalm.max_subsets(ax, 40)) == 24
    hel = synth.Geometry(kind=synth.CONE3D_FLAT, nx=8, ny=8, nz=4, nviews=7146, angle_span=7146 / 984 * 2 * math.pi,
                         ns=888, nt=32, ds=1.0239, dt=1.0963, dso=541.0, dsd=949.0, pitch=0.5)
    m05 = oslalm.max_subsets(hel, 24)
    assert abs(m05 - 984 * 541.0 / (0.5 * 24 * 949.0)) < 1e-9 and math.floor(m05) == 46
    hel.pitch = 1.0
    assert math.floor(oslalm.max_subsets(hel, 24)) == 23
    assert abs(oslalm.max_subsets(hel, 24) * 2 - m05) < 1e-9


def test_network_creation_validates_sizes_before_any_device_call(L):
    """oslalm_cnn_create rejects sizes its kernels cannot take (not multiples
    of 8; 2^31 pixels or more, the limit of the 32-bit pixel arithmetic of the
    elementwise kernels) before it touches the device, and the network's
    host-only entry points behave on NULL handles."""
    h = ctypes.c_void_p()
    assert L.oslalm_cnn_create(1, 12, 16, 0, ctypes.byref(h)) == -1  # height not a multiple of 8
    assert b"multiples of 8" in L.oslalm_last_error()
    assert L.oslalm_cnn_create(0, 16, 16, 0, ctypes.byref(h)) == -1
    assert L.oslalm_cnn_create(8, 32768, 8192, 0, ctypes.byref(h)) == -1  # exactly 2^31 pixels
    assert b"2^31" in L.oslalm_last_error()
    assert h.value is None
    assert L.oslalm_cnn_create(1, 16, 16, 0, None) == -1
    assert L.oslalm_cnn_set_tma(None, 1) == -1
    assert L.oslalm_cnn_launch_count() >= 0
