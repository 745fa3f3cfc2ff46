"""The C-ABI library builds, loads and exports every declared entry point;
host-side validation rejects bad inputs before any device work (no GPU)."""
import ctypes

import numpy as np
import pytest

import paper_2004_11571_gb300 as pe
from paper_2004_11571_gb300 import _build


@pytest.fixture(scope="module")
def L():
    _build.build()
    return pe.lib()


def test_exports_every_declared_symbol(L):
    names = pe.declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def _create(L, p, coeffs, exps, variant=0):
    coeffs = np.ascontiguousarray(coeffs, np.uint64)
    exps = np.ascontiguousarray(exps, np.uint32)
    d = pe._Desc(p, exps.shape[1], 4, coeffs.shape[0], coeffs.ctypes.data, exps.ctypes.data, 0, variant)
    h = ctypes.c_void_p()
    return L.poly_eval_create(ctypes.byref(d), ctypes.byref(h)), h


def test_validation_before_device_work(L):
    p = (1 << 61) - 1
    ok_c = [1, 2, 3]
    ok_e = [[1, 0, 2], [0, 1, 3], [0, 0, 1]]
    assert _create(L, p + 1, ok_c, ok_e)[0] == 2                    # even p
    assert _create(L, 1, ok_c, ok_e)[0] == 2                        # p < 3
    assert _create(L, (1 << 62) + 1, ok_c, ok_e)[0] == 2            # above 2^62
    assert _create(L, p, ok_c, ok_e, variant=2)[0] == 2             # FP64 needs p < 2^50
    assert _create(L, p, [1, p, 3], ok_e)[0] == 3                   # coefficient not reduced
    assert _create(L, p, ok_c, [[1, 0, 2], [0, 1, 70000], [0, 0, 1]])[0] == 4   # exponent range
    assert _create(L, p, ok_c, ok_e, variant=9)[0] == 1             # unknown variant
    d = pe._Desc(p, 1, 4, 0, None, None, 0, 0)
    h = ctypes.c_void_p()
    assert L.poly_eval_create(ctypes.byref(d), ctypes.byref(h)) == 1  # n < 2
    assert L.poly_eval_create(None, ctypes.byref(h)) == 1
    assert b"n = 1" in L.poly_eval_last_error() or L.poly_eval_last_error()


def test_binding_raises_without_library(monkeypatch):
    monkeypatch.setattr(pe, "_lib", None)
    monkeypatch.setattr(pe, "LIB_PATH", "/nonexistent/libpolyeval.so")
    with pytest.raises(RuntimeError):
        pe.lib()


def test_validation_of_later_entry_points(L):
    """The interpolation solver, the fast method, multi-prime handles and the
    monomial query check their arguments on the host before any device call."""
    u64 = ctypes.c_uint64
    p = (1 << 61) - 1
    off = np.array([0, 2, 5], np.uint64)
    dummy = ctypes.c_void_p(16)     # never dereferenced: every call below fails validation first
    solve = L.poly_eval_vandermonde_solve
    assert solve(p + 1, 2, off.ctypes.data, dummy, dummy, 5, 2, 1, dummy, None) == 2        # even modulus
    assert solve(p, 2, None, dummy, dummy, 5, 2, 1, dummy, None) == 1                        # off missing
    bad0 = np.array([1, 2, 5], np.uint64)
    assert solve(p, 2, bad0.ctypes.data, dummy, dummy, 5, 2, 1, dummy, None) == 1           # off[0] != 0
    down = np.array([0, 4, 3], np.uint64)
    assert solve(p, 2, down.ctypes.data, dummy, dummy, 5, 2, 1, dummy, None) == 1           # decreasing
    assert solve(p, 2, off.ctypes.data, dummy, dummy, 2, 2, 1, dummy, None) == 1            # rows < 3 terms
    assert solve(p, 2, off.ctypes.data, dummy, dummy, 5, 1, 1, dummy, None) == 1            # lda < G
    assert solve(p, 2, off.ctypes.data, None, dummy, 5, 2, 1, dummy, None) == 1             # z missing
    assert b"device pointers" in L.poly_eval_last_error()
    empty = np.array([0, 0, 0], np.uint64)
    assert solve(p, 2, empty.ctypes.data, None, None, 0, 2, 1, None, None) == 0             # nothing to do
    assert L.poly_eval_run_fast(None, None, 4, 1, dummy, None) == 1
    assert L.poly_eval_monomials(None, None, dummy, None, None) == 1
    h = ctypes.c_void_p()
    assert L.poly_eval_create_like(None, p, dummy, 0, 0, ctypes.byref(h)) == 1
    assert L.poly_eval_create_like(dummy, p, dummy, 0, 0, None) == 1
    ms = (ctypes.c_double * 4)()
    assert L.poly_eval_vandermonde_timing(-1, ms) == 0
    nnz = u64()
    assert L.poly_eval_compact(dummy, 1 << 32, 4, dummy, dummy, dummy, 0, ctypes.byref(nnz), None) == 1


def test_points_must_fit_in_64_bits(L):
    """T <= 2^31 and the last point t0 + T - 1 below 2^64, checked before any
    pointer is looked at (the pointers below are never dereferenced)."""
    p = (1 << 61) - 1
    dummy = ctypes.c_void_p(16)
    na = L.poly_eval_stepb_noalloc
    top = (1 << 64) - 1
    assert na(p, 1, 1, dummy, dummy, dummy, 2, top, dummy, None) == 1          # t0 + 1 wraps
    assert na(p, 1, 1, dummy, dummy, dummy, 2, top - 2, dummy, None) == 1      # t0 + T - 1 fits: the
    assert b"device pointers" in L.poly_eval_last_error()                     # pointer check comes next
    assert na(p, 1, 1, dummy, dummy, dummy, (1 << 31) + 1, 1, dummy, None) == 1
    assert b"2^31" in L.poly_eval_last_error()
    assert na(p, 1, 1, dummy, dummy, dummy, 0, top, dummy, None) == 0         # no points: nothing to do
    assert na(p, 1 << 31, 1 << 31, dummy, dummy, dummy, 1 << 31, 1, dummy, None) == 1   # 2^62 output values
    assert b"2^60" in L.poly_eval_last_error()


def test_batch_queries_validate_their_handle(L):
    k, n = ctypes.c_uint32(7), ctypes.c_uint32(7)
    assert L.poly_eval_batch_launches(None, ctypes.byref(k), ctypes.byref(n)) == 1
    assert b"NULL batch" in L.poly_eval_last_error()
    assert L.poly_eval_batch_launch(None, None) == 1


def test_host_checks_of_query_entry_points(L):
    """Queries reject NULL outputs and out-of-range sizes before any device call."""
    assert L.poly_eval_stepb_noalloc_shape(1000, 64, None) == 1
    sh = (ctypes.c_uint32 * 4)(7, 7, 7, 7)
    assert L.poly_eval_stepb_noalloc_shape(0, 64, sh) == 0 and list(sh) == [0, 0, 0, 0]
    assert L.poly_eval_stepb_noalloc_shape(1 << 40, 64, sh) == 1
    assert L.poly_eval_stepb_noalloc_shape(1000, (1 << 31) + 1, sh) == 1
    assert L.poly_eval_num_sms(None) == 1
    assert L.poly_eval_fp64_pipe_rates(None) == 1
