"""The C-ABI library builds, loads and exports every function include/gbnfft.h
declares; host-only entry points work without a GPU (no compute calls)."""
import ctypes

import pytest

from paper_2001_01583_gb300 import _lib, build as lib_build


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return _lib.load()


def test_every_declared_function_is_exported(lib):
    names = _lib.header_functions()
    assert "nfft_plan_create" in names and "nfft_adjoint" in names and "nfft_forward" in names
    raw = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_status_strings(lib):
    for code in range(0, -9, -1):
        s = lib.nfft_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.nfft_status_string(-99).decode() == "unknown status"
    assert lib.nfft_version() >= 10000


def _params(N, sigma, m, window):
    d = len(N)
    Narr = (ctypes.c_int64 * d)(*N)
    nout = (ctypes.c_int64 * d)()
    taps = ctypes.c_int()
    rc = _lib.load().nfft_plan_params(d, Narr, sigma, m, window, nout, ctypes.byref(taps))
    return rc, tuple(nout), taps.value


def test_plan_params_rule(lib):
    assert _params((64, 64, 64), 2.0, 4, _lib.KAISER_BESSEL) == (0, (128, 128, 128), 8)
    assert _params((256,), 2.0, 6, _lib.GAUSSIAN) == (0, (512,), 14)
    assert _params((100, 64), 1.25, 4, _lib.GAUSSIAN) == (0, (126, 80), 10)
    assert _params((30,), 1.5, 2, _lib.KAISER_BESSEL) == (0, (48,), 4)  # 45 odd, 46 = 2 * 23 -> 48
    assert _params((255,), 2.0, 4, _lib.GAUSSIAN)[0] == _lib.ERR_INVALID_ARG   # odd N
    assert _params((4,), 2.0, 6, _lib.GAUSSIAN)[0] == _lib.ERR_INVALID_ARG     # n = 8 < 2m + 2
    assert _params((16,), 0.5, 2, _lib.GAUSSIAN)[0] == _lib.ERR_INVALID_ARG    # sigma < 1
    assert _params((16,), 2.0, 0, _lib.GAUSSIAN)[0] == _lib.ERR_INVALID_ARG    # m < 1
    assert _params((64,), 2.0, 17, _lib.KAISER_BESSEL)[0] == _lib.ERR_UNSUPPORTED  # 34 taps


def test_plan_params_matches_oracle_rule(lib):
    from oracle import nfft_steps
    for N, sigma, m in [(64, 2.0, 4), (100, 1.25, 4), (30, 1.5, 2), (48, 1.7, 3), (256, 2.0, 12)]:
        rc, n, _ = _params((N,), sigma, m, _lib.KAISER_BESSEL)
        assert rc == 0 and n[0] == nfft_steps.oversampled_size(N, sigma, m)


def test_plan_create_argument_errors_need_no_gpu(lib):
    h = ctypes.c_void_p()
    N = (ctypes.c_int64 * 1)(255)
    assert lib.nfft_plan_create(ctypes.byref(h), 1, N, 10, 2.0, 4, 1, 0, None) == _lib.ERR_INVALID_ARG
    N = (ctypes.c_int64 * 4)(8, 8, 8, 8)
    assert lib.nfft_plan_create(ctypes.byref(h), 4, N, 10, 2.0, 4, 1, 0, None) == _lib.ERR_INVALID_ARG
    N = (ctypes.c_int64 * 1)(16)
    assert lib.nfft_plan_create(ctypes.byref(h), 1, N, 10, 2.0, 4, 7, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.nfft_plan_create(ctypes.byref(h), 1, N, -1, 2.0, 4, 1, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.nfft_plan_create(None, 1, N, 10, 2.0, 4, 1, 0, None) == _lib.ERR_INVALID_ARG
    # null plan handles are rejected, never dereferenced
    assert lib.nfft_set_points(None, None) == _lib.ERR_INVALID_ARG
    assert lib.nfft_adjoint(None, None, None, 1) == _lib.ERR_INVALID_ARG
    assert lib.nfft_forward(None, None, None, 1) == _lib.ERR_INVALID_ARG
    assert lib.nfft_sync(None) == _lib.ERR_INVALID_ARG
    assert lib.nfft_plan_destroy(None) == _lib.OK


def test_batch_total_points_beyond_int32_rejected_without_gpu(lib):
    """Each item may hold up to INT32_MAX points, but the bin sort indexes a
    whole batch with 32-bit integers: two items of 1.2e9 points are refused
    before any device work (so this runs without a GPU)."""
    items = (_lib.BatchItem * 2)()
    for it in items:
        it.d = 3
        for t in range(3):
            it.N[t] = 64
        it.M = 1_200_000_000
        it.sigma = 2.0
        it.m = 4
        it.window = _lib.KAISER_BESSEL
        it.nrhs = 1
    h = ctypes.c_void_p()
    assert lib.nfft_batch_create(ctypes.byref(h), 2, items, _lib.FP32_MIXED, None) == _lib.ERR_UNSUPPORTED
    assert not h.value
