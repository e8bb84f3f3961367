"""The allocation-free Ewald reciprocal-sum entry point.

nfft_ewald_reciprocal_sum_noalloc serves callers that cannot allocate device
memory when they need the sum (a framework's caching allocator owns the GPU
memory, an allocation-free steady-state loop, or no plan at hand).  Its only
scratch is a static device array inside the library.  The GPU tests call it
through the C ABI twice in a row, on different inputs, and check each result
against the plan-based nfft_ewald_reciprocal_sum with the tolerances of the
other reduction tests (1e-13 relative in FP64, 1e-6 in FP32), and against the
oracle's direct n-sum of Eq. 12 on the same input values; one case sits
exactly at the largest accepted size, NFFT_NOALLOC_MAX_MODES (every partial
of the static array in use), and the size just above it is rejected.  This
file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from oracle import ewald
from paper_2001_01583_gb300 import _lib, build as lib_build, inputs

NOALLOC_MAX_MODES = 33554432   # NFFT_NOALLOC_MAX_MODES in include/gbnfft.h


def _noalloc(lib, N, precision, S, L, alpha, out, stream=None):
    Narr = (ctypes.c_int64 * len(N))(*N)
    return lib.nfft_ewald_reciprocal_sum_noalloc(len(N), Narr, precision, ctypes.c_void_p(S), float(L), float(alpha),
                                                 ctypes.c_void_p(out), stream)


def test_noalloc_limit_matches_header():
    import os
    with open(os.path.join(os.path.dirname(__file__), "..", "include", "gbnfft.h")) as fh:
        text = fh.read()
    assert "#define NFFT_NOALLOC_MAX_MODES %d" % NOALLOC_MAX_MODES in text


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib_build.build()
    lib = _lib.load()
    fake = 16  # never dereferenced: the size check comes first
    assert _noalloc(lib, (512, 512, 512), _lib.FP64, fake, 1.0, 1.0, fake) == _lib.ERR_UNSUPPORTED
    assert _noalloc(lib, (1 << 26,), _lib.FP32_MIXED, fake, 1.0, 1.0, fake) == _lib.ERR_UNSUPPORTED
    assert _noalloc(lib, (8192, 4098), _lib.FP32_MIXED, fake, 1.0, 1.0, fake) == _lib.ERR_UNSUPPORTED  # one row over
    assert _noalloc(lib, (15, 16), _lib.FP64, fake, 1.0, 1.0, fake) == _lib.ERR_INVALID_ARG
    assert _noalloc(lib, (16, 16), _lib.FP64, fake, -1.0, 1.0, fake) == _lib.ERR_INVALID_ARG


def _device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_noalloc_matches_plan_reduction_and_oracle(precision, tol):
    torch = _device()
    from paper_2001_01583_gb300 import Plan
    lib = _lib.load()
    prec = _lib.PRECISIONS[precision]
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    N = (40, 36, 32)               # 46080 modes: 6 tiles, the last one ragged
    L, alpha = 11.0, 0.8
    stream = torch.cuda.current_stream()
    with Plan(N, 1, 2.0, 4, "kaiser_bessel", precision) as plan:
        for call, seed in enumerate((5, 6)):     # two calls in a row, different inputs
            S = torch.from_numpy(inputs.complex_normal(N, seed=seed) * (10.0 + call)).to(cdt).cuda()
            ref = plan.ewald_reciprocal_sum(S, L, alpha)
            got = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            rc = _noalloc(lib, N, prec, S.data_ptr(), L, alpha, got.data_ptr(),
                          ctypes.c_void_p(stream.cuda_stream))
            assert rc == _lib.OK
            plan.sync()
            torch.cuda.synchronize()
            assert abs(got.item() - ref.item()) <= tol * abs(ref.item()), (call, got.item(), ref.item())
            # the direct sum of Eq. 12 over the values the GPU read (FP64 arithmetic on both sides)
            want = ewald.reciprocal_sum(S.cpu().numpy().astype(np.complex128), L, alpha)
            assert abs(got.item() - want) <= 1e-12 * abs(want), (call, got.item(), want)


@pytest.mark.gpu
def test_noalloc_at_its_largest_size():
    """|I_N| = NFFT_NOALLOC_MAX_MODES exactly (N = 8192 x 4096, FP32: 256 MB
    of S): all 4096 partials of the static array are written and summed.
    Two calls in a row on different inputs, each against the oracle."""
    torch = _device()
    lib = _lib.load()
    N = (8192, 4096)
    assert N[0] * N[1] == NOALLOC_MAX_MODES
    L, alpha = 1000.0, 2.0         # exp(-pi^2 |n|^2 / (alpha L)^2) decays over the whole of I_N
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((11, 12)):
        S = torch.from_numpy(inputs.complex_normal(N, seed=seed, dtype=np.complex64)).cuda()
        got = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = _noalloc(lib, N, _lib.FP32_MIXED, S.data_ptr(), L, alpha, got.data_ptr(),
                      ctypes.c_void_p(stream.cuda_stream))
        assert rc == _lib.OK
        torch.cuda.synchronize()
        want = ewald.reciprocal_sum(S.cpu().numpy().astype(np.complex128), L, alpha)
        assert abs(got.item() - want) <= 1e-12 * abs(want), (call, got.item(), want)
        del S
