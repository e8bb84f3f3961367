"""The allocation-free Ewald reciprocal-sum entry point.

nfft_ewald_reciprocal_sum_noalloc serves callers that cannot allocate device
memory when they need the sum (a framework's caching allocator owns the GPU
memory, an allocation-free steady-state loop, or no plan at hand).  Its only
scratch is a static device array inside the library.  The GPU test calls it
through the C ABI twice in a row, on different inputs, and checks each result
against the plan-based nfft_ewald_reciprocal_sum with the tolerances of the
other reduction tests (1e-13 relative in FP64, 1e-6 in FP32).  This file is
named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2001_01583_gb300 import _lib, build as lib_build, inputs


def _noalloc(lib, N, precision, S, L, alpha, out, stream=None):
    Narr = (ctypes.c_int64 * len(N))(*N)
    return lib.nfft_ewald_reciprocal_sum_noalloc(len(N), Narr, precision, ctypes.c_void_p(S), float(L), float(alpha),
                                                 ctypes.c_void_p(out), stream)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib_build.build()
    lib = _lib.load()
    fake = 16  # never dereferenced: the size check comes first
    assert _noalloc(lib, (512, 512, 512), _lib.FP64, fake, 1.0, 1.0, fake) == _lib.ERR_UNSUPPORTED
    assert _noalloc(lib, (1 << 26,), _lib.FP32_MIXED, fake, 1.0, 1.0, fake) == _lib.ERR_UNSUPPORTED
    assert _noalloc(lib, (15, 16), _lib.FP64, fake, 1.0, 1.0, fake) == _lib.ERR_INVALID_ARG
    assert _noalloc(lib, (16, 16), _lib.FP64, fake, -1.0, 1.0, fake) == _lib.ERR_INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_noalloc_matches_plan_reduction(precision, tol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_01583_gb300 import Plan
    torch.cuda.set_device(0)
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
