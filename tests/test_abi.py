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
