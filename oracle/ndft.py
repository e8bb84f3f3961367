"""Direct NDFT oracle (Eqs. 5 and 6 of the HP-NFFT paper, Section 1).

TEST INFRASTRUCTURE ONLY: a thin ctypes wrapper around the plain-C FP64
direct sums in ndft.c.  Product code never imports this module.

    adjoint  (Eq. 5): fhat(k) = sum_j f(x_j) exp(-2 pi i k.x_j),  k in I_N
    forward  (Eq. 6): f(x_j)  = sum_k fhat(k) exp(+2 pi i k.x_j)

I_N = {k : -N_t/2 <= k_t < N_t/2} (Section 1), stored in C order with each
k_t ascending from -N_t/2.  Points x are M x d, point-major, any finite reals
(both sums are 1-periodic in every x_t because k is integer).
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("oracle_ndft_adjoint", "oracle_ndft_forward"):
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [ctypes.c_int, i64p, ctypes.c_int64, dp, dp, ctypes.c_int64, i64p, dp, ctypes.c_int]
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def threads_used(threads: int = 0) -> int:
    """Number of POSIX threads the oracle runs with for a `threads` request."""
    return _load().oracle_threads(int(threads))


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _prep(x, N):
    N = np.ascontiguousarray(np.atleast_1d(np.asarray(N, dtype=np.int64)))
    d = N.size
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, d))
    return x, N, d


def frequencies(N):
    """The index set I_N per dimension: k_t = -N_t/2, ..., N_t/2 - 1."""
    return [np.arange(-n // 2, n // 2, dtype=np.int64) for n in np.atleast_1d(N)]


def adjoint(x, f, N, ksel=None, threads: int = 0) -> np.ndarray:
    """Eq. 5.  Returns fhat with shape N (C order), or shape (K,) at the K
    frequencies listed in ksel (K x d integers, each inside I_N or not)."""
    x, N, d = _prep(x, N)
    M = x.shape[0]
    f = np.ascontiguousarray(np.asarray(f, dtype=np.complex128).reshape(M))
    fv = f.view(np.float64)
    if ksel is None:
        out = np.zeros(tuple(int(n) for n in N), dtype=np.complex128)
        ks, K = None, 0
    else:
        ks = np.ascontiguousarray(np.asarray(ksel, dtype=np.int64).reshape(-1, d))
        K = ks.shape[0]
        out = np.zeros(K, dtype=np.complex128)
    rc = _load().oracle_ndft_adjoint(d, _ptr(N, ctypes.c_int64), M, _ptr(x, ctypes.c_double),
                                     _ptr(fv, ctypes.c_double), K, _ptr(ks, ctypes.c_int64),
                                     _ptr(out.view(np.float64), ctypes.c_double), int(threads))
    if rc != 0:
        raise RuntimeError("oracle_ndft_adjoint failed: %d" % rc)
    return out


def forward(x, fhat, N, jsel=None, threads: int = 0) -> np.ndarray:
    """Eq. 6.  Returns f(x_j) for all j < M, or for the indices in jsel."""
    x, N, d = _prep(x, N)
    M = x.shape[0]
    h = np.ascontiguousarray(np.asarray(fhat, dtype=np.complex128).reshape(tuple(int(n) for n in N)))
    if jsel is None:
        js, J = None, M
    else:
        js = np.ascontiguousarray(np.asarray(jsel, dtype=np.int64).reshape(-1))
        J = js.size
    out = np.zeros(J, dtype=np.complex128)
    rc = _load().oracle_ndft_forward(d, _ptr(N, ctypes.c_int64), M, _ptr(x, ctypes.c_double),
                                     _ptr(h.view(np.float64), ctypes.c_double), J, _ptr(js, ctypes.c_int64),
                                     _ptr(out.view(np.float64), ctypes.c_double), int(threads))
    if rc != 0:
        raise RuntimeError("oracle_ndft_forward failed: %d" % rc)
    return out


def rel_l2(approx, exact) -> float:
    """Eq. 9 read as ||approx - exact||_2 / ||exact||_2 over the output vector
    the transform produces (k in I_N for the adjoint, j < M for the forward)."""
    a = np.asarray(approx, dtype=np.complex128).ravel()
    e = np.asarray(exact, dtype=np.complex128).ravel()
    den = np.linalg.norm(e)
    return float(np.linalg.norm(a - e) / den) if den > 0 else float(np.linalg.norm(a - e))
