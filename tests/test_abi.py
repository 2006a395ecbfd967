"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/mb.h declares (no compute calls: these run without a GPU)."""
import os
import re
import subprocess

import paper_1602_02170_gb300 as mb
from paper_1602_02170_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "mb.h")).read()
    return sorted(set(re.findall(r"\b(mb_[A-Za-z_0-9]+)\s*\(", text)))


def test_library_builds_and_loads():
    path = B.build()
    assert os.path.exists(path)
    L = mb.load_library()
    assert L.mb_status_string(6) == b"MB_ESINGULAR"
    assert L.mb_status_string(0) == b"MB_OK"


def test_every_declared_symbol_is_exported():
    B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (mb_[A-Za-z_0-9]+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    assert set(mb.EXPORTED_SYMBOLS) == set(declared)


def test_library_targets_sm_103a():
    """Every translation unit and the link are compiled for sm_103a alone."""
    gencodes = [B.NVCC_FLAGS[i + 1] for i, x in enumerate(B.NVCC_FLAGS) if x == "-gencode"]
    assert gencodes == ["arch=compute_103a,code=sm_103a"]
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_null_context_is_rejected_without_gpu():
    L = mb.load_library()
    assert L.mb_context_destroy(None) == 1  # MB_EINVAL
    assert L.mb_mobility_matvec(None, None, None, 0, 1.0, 1.0, 1, 1, None, None) == 1


def test_errors_are_status_codes_without_a_gpu():
    """On a machine without a GPU the library reports errors, never aborts:
    creating a context is MB_ECUDA with a message, and the allocation-free
    matvec checks its arguments on the host (MB_EINVAL) before touching a
    device; N = 0 is a no-op."""
    import ctypes

    import pytest

    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = mb.load_library()
    h = ctypes.c_void_p()
    assert L.mb_context_create(ctypes.byref(h), 0, 0) == 3  # MB_ECUDA
    assert L.mb_last_error(None)
    i64, dbl = ctypes.c_int64, ctypes.c_double
    call = L.mb_mobility_matvec_noalloc
    assert call(None, None, i64(65537), dbl(0.5), dbl(1.0), 1, None, None) == 1
    assert b"MB_NOALLOC_MAX_BLOBS" in L.mb_last_error(None)
    assert call(None, None, i64(-1), dbl(0.5), dbl(1.0), 1, None, None) == 1
    assert call(None, None, i64(10), dbl(0.0), dbl(1.0), 1, None, None) == 1
    assert call(None, None, i64(10), dbl(0.5), dbl(1.0), 1, None, None) == 1
    assert call(None, None, i64(0), dbl(0.5), dbl(1.0), 1, None, None) == 0


def test_binding_declares_every_signature():
    """The Python binding gives every exported entry point its argument types
    (so 64-bit sizes and pointers are never passed as default C ints) and an
    mb_status (int) or documented return type."""
    import ctypes

    L = mb.load_library()
    for name in mb.EXPORTED_SYMBOLS:
        fn = getattr(L, name)
        assert fn.argtypes is not None, name
        assert fn.restype in (ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t), name
