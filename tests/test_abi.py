"""The C-ABI library builds, loads, and exports every entry point of include/fmm.h.

No compute call is made here (no GPU on the build host); only argument checks
that the library performs before touching the device are exercised.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(fmm_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1209_3516_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("fmm_create", "fmm_build", "fmm_evaluate", "fmm_backward", "fmm_destroy",
                     "fmm_last_error_string", "fmm_stats", "fmm_energy", "fmm_evaluate_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_checks_before_any_device_call(lib):
    lib.fmm_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int, ctypes.c_float,
                               ctypes.c_int, ctypes.c_void_p]
    lib.fmm_last_error_string.restype = ctypes.c_char_p
    h = ctypes.c_void_p(1)
    assert lib.fmm_create(ctypes.byref(h), 0, 4, 0.4, 64, None) == -1      # N < 1
    assert h.value is None
    assert b"N must be" in lib.fmm_last_error_string()
    assert lib.fmm_create(ctypes.byref(h), 100, 4, 1.5, 64, None) == -1    # theta out of range
    assert lib.fmm_create(ctypes.byref(h), 100, 4, float("nan"), 64, None) == -1
    assert lib.fmm_create(ctypes.byref(h), 100, 4, 0.4, 0, None) == -1     # ncrit < 1
    assert lib.fmm_create(ctypes.byref(h), 100, 7, 0.4, 64, None) == -2    # P not compiled
    assert lib.fmm_create(None, 100, 4, 0.4, 64, None) == -1
    assert lib.fmm_destroy(None) == 0
    lib.fmm_build.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.fmm_build(None, None) == -1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1209_3516_gb300 import fmm
    monkeypatch.setattr(fmm, "_lib", None)
    monkeypatch.setattr(fmm._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        fmm.load()


def test_product_path_does_not_touch_the_oracle():
    # the package and its kernels never import, link, load or call the oracle
    pkg = os.path.join(ROOT, "paper_1209_3516_gb300")
    forbidden = re.compile(r"import\s+oracle|from\s+oracle|liborc|fmm_oracle|\borc_\w+\(")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not forbidden.search(text), f


def test_backward_argument_checks(lib):
    lib.fmm_backward.argtypes = [ctypes.c_void_p] * 5
    lib.fmm_last_error_string.restype = ctypes.c_char_p
    assert lib.fmm_backward(None, None, None, None, None) == -1
    assert b"null handle" in lib.fmm_last_error_string()


def test_every_entry_point_rejects_null_arguments_before_any_device_call(lib):
    """A null handle or output pointer is an FMM_ERR_ARG (-1) with a message,
    from every entry point, without touching the device."""
    V = ctypes.c_void_p
    lib.fmm_last_error_string.restype = ctypes.c_char_p
    calls = [
        ("fmm_evaluate", (V(), V(), V(), V(), V())),
        ("fmm_evaluate_host", (V(), V(), V(), V(), V())),
        ("fmm_evaluate_batch", (V(), V(), V(), ctypes.c_int(4), V(), V())),
        ("fmm_energy", (V(), V())),
        ("fmm_energy_noalloc", (V(), V(), ctypes.c_int64(10), V(), V())),
        ("fmm_measure_peaks", (V(), V())),
        ("fmm_stats", (V(), V())),
        ("fmm_set_hybrid", (V(), ctypes.c_int64(0))),
        ("fmm_get_norm", (V(), V(), V())),
        ("fmm_get_sorted", (V(), V(), V())),
        ("fmm_get_ncells", (V(), V())),
        ("fmm_get_lists", (V(), V(), V(), V(), V())),
        ("fmm_get_cells", (V(),) + (V(),) * 8),
        ("fmm_multi_build", (V(), V())),
        ("fmm_multi_evaluate", (V(), V(), V(), V())),
        ("fmm_multi_info", (V(), V())),
        ("fmm_multi_set_hybrid", (V(), ctypes.c_int64(0))),
        ("fmm_multi_set_config", (V(), ctypes.c_int(0), ctypes.c_int(-1))),
    ]
    for name, args in calls:
        assert getattr(lib, name)(*args) == -1, name
        assert lib.fmm_last_error_string().startswith(name.encode()), name
    assert lib.fmm_multi_destroy(V()) == 0


def test_multi_and_tuner_argument_checks(lib):
    V = ctypes.c_void_p
    lib.fmm_last_error_string.restype = ctypes.c_char_p
    h = V()
    sizes = (ctypes.c_int64 * 2)(100, 200)
    create = lambda *a: lib.fmm_multi_create(*a)
    f4 = ctypes.c_float
    assert create(ctypes.byref(h), ctypes.c_int(0), sizes, 4, f4(0.4), 64, V()) == -1     # no systems
    assert create(ctypes.byref(h), ctypes.c_int(2), V(), 4, f4(0.4), 64, V()) == -1       # no sizes
    assert create(V(), ctypes.c_int(2), sizes, 4, f4(0.4), 64, V()) == -1                # no handle pointer
    bad = (ctypes.c_int64 * 2)(100, 0)
    assert create(ctypes.byref(h), ctypes.c_int(2), bad, 4, f4(0.4), 64, V()) == -1      # an empty system
    assert create(ctypes.byref(h), ctypes.c_int(2), sizes, 4, f4(1.0), 64, V()) == -1    # theta out of range
    assert create(ctypes.byref(h), ctypes.c_int(2), sizes, 4, f4(0.4), 0, V()) == -1     # ncrit < 1
    assert create(ctypes.byref(h), ctypes.c_int(2), sizes, 7, f4(0.4), 64, V()) == -2    # P not compiled
    assert b"P must be" in lib.fmm_last_error_string()
    best64, best32 = ctypes.c_int64(), ctypes.c_int()
    ms = (ctypes.c_double * 4)()
    cand = (ctypes.c_int64 * 2)(0, 256)
    assert lib.fmm_tune_hybrid(ctypes.c_int64(0), 4, f4(0.4), 64, V(), V(), cand, 2, 1, V(), ctypes.byref(best64),
                               ms) == -1
    ci = (ctypes.c_int * 2)(32, 64)
    assert lib.fmm_tune_ncrit(ctypes.c_int64(0), 4, f4(0.4), V(), V(), ci, 2, 1, V(), ctypes.byref(best32),
                              ms) == -1
