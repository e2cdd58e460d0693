"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without
a GPU and exports every entry point include/tlda.h declares; host argument
checks reject bad input without touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tlda.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tlda_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2511_07809_gb300 import _build, tlda
    path = _build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(tlda.ENTRY_POINTS) == declared


def test_struct_layouts_match_header():
    from paper_2511_07809_gb300 import tlda
    assert ctypes.sizeof(tlda.Params) == 48
    assert tlda.Params.seed.offset == 32 and tlda.Params.alpha0.offset == 8
    assert ctypes.sizeof(tlda.CSR) == 32 and tlda.CSR.indptr.offset == 8


def test_host_argument_checks_without_a_device():
    from paper_2511_07809_gb300 import tlda
    lib = tlda.load()
    p = tlda.Params()
    lib.tlda_default_params(ctypes.byref(p), 10)
    assert (p.k, p.dim, p.alpha0, p.precision, p.same_token_correction, p.max_batch) == \
        (10, 0, 1.0, 0, 1, 8192)
    h = ctypes.c_void_p()
    bad = tlda.Params()
    lib.tlda_default_params(ctypes.byref(bad), 10)
    bad.dim = 5                                     # D < K
    assert lib.tlda_create(ctypes.byref(h), 500, ctypes.byref(bad), None) == tlda.ERR_INVALID
    bad.dim, bad.alpha0 = 0, -1.0                   # alpha0 <= 0
    assert lib.tlda_create(ctypes.byref(h), 500, ctypes.byref(bad), None) == tlda.ERR_INVALID
    bad.alpha0, bad.k = 1.0, 600                    # K padded beyond 512
    assert lib.tlda_create(ctypes.byref(h), 5000, ctypes.byref(bad), None) == tlda.ERR_INVALID
    assert lib.tlda_destroy(None) == tlda.ERR_INVALID
    assert lib.tlda_last_error(None) == b"NULL context"
