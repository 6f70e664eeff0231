"""The C-ABI library builds, loads and exports every symbol include/rlu.h
declares; argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

import paper_1601_04280_gb300 as rg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "rlu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rlu_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    rg.build()
    return rg.load(reload=True)


def test_exports_every_declared_symbol(lib):
    syms = header_symbols()
    assert len(syms) >= 10
    assert sorted(syms) == sorted(rg.C_SYMBOLS)
    for s in syms:
        assert hasattr(lib, s), s


def test_invalid_sizes_rejected_before_any_launch(lib):
    h = ctypes.c_void_p()
    bad = [(0, 10, 1, 1, 1), (100, 100, 5, 4, 10), (100, 100, 5, 10, 8), (8, 100, 2, 9, 20),
           (100, 3, 4, 6, 8), (100, 100, 5, 2000, 4000), (100, 100, 5, 10, 20000), (2**31, 10, 1, 1, 1)]
    for m, n, k, l, l1 in bad:
        assert lib.rlu_create(m, n, k, l, l1, 1, ctypes.byref(h)) == rg.RLU_EINVAL
        assert not h.value
    assert lib.rlu_create(10, 10, 1, 1, 1, 1, None) == rg.RLU_EINVAL
    sz = ctypes.c_size_t()
    assert lib.rlu_workspace_bytes(0, 5, 1, 1, 1, 1, ctypes.byref(sz)) == rg.RLU_EINVAL
    assert lib.rlu_workspace_bytes(8192, 8192, 200, 220, 1600, 1, ctypes.byref(sz)) == rg.RLU_OK
    # Y (m x l f64) and W, B (k x m, k x n, f64-sized) dominate
    assert sz.value > 8 * 8192 * 220 + 2 * 8 * 200 * 8192
    assert lib.rlu_destroy(None) == rg.RLU_OK
    assert lib.rlu_set_precision(None, 1) == rg.RLU_EINVAL
    assert lib.rlu_factor_dense(None, None, 0, 1, None, None, None, None, None) == rg.RLU_EINVAL


def test_strerror(lib):
    for code in (0, 1, 2, 3, 4, 5, 6, 100):
        assert rg.strerror(code)
    assert rg.strerror(12345) == "unknown status"


def test_every_flag_bit_reaches_the_status_word(lib):
    """Each device flag bit gives its own status code, and a set of bits gives
    the most severe one: a timed-out wait (outputs unwritten) before a
    malformed CSR, a non-finite input, and the rank warning.  This is the one
    mapping of the host read-back and of the device-side status writers
    (including the allocation-free sketch)."""
    single = {1: rg.RLU_ETIMEOUT, 2: rg.RLU_ENONFINITE, 4: rg.RLU_WRANK, 8: rg.RLU_EBADCSR}
    for bit, code in single.items():
        assert rg.rlu_debug_status_of_flags(bit) == code
    assert rg.rlu_debug_status_of_flags(0) == rg.RLU_OK
    order = [1, 8, 2, 4]  # most severe first
    for flags in range(1, 16):
        first = next(b for b in order if flags & b)
        assert rg.rlu_debug_status_of_flags(flags) == single[first], flags
