"""GPU parity of the tensor-core spreading kernel (NFFT_OPT_TENSOR_SPREAD).

The kernel computes the spreading step of Section 2 (Fig. 1) as dense MMAs
of TF32 operands split in two (hi + lo, three products), accumulating each
bin's tile in tensor memory.  The bars are those of every FP32 kernel:
element by element against the FP64 gridding oracle, max |gpu - oracle| <=
1e-5 rms and relative l2 <= 1e-6, on uniform and clustered points, for every
window width the kernel is built for, with several right-hand sides, and at
the full size of the 3-D configuration (N = 64^3, M = 10^6).  info() must
report that the tensor-core kernel ran.
"""
import numpy as np
import pytest

from oracle import ndft, nfft_steps as S
from paper_2001_01583_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_ELEM = 1e-5
FP32_L2 = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _elementwise(got, ref, tol):
    got = np.asarray(got).ravel()
    ref = np.asarray(ref).ravel()
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    err = np.max(np.abs(got - ref)) / scale
    assert err <= tol, "elementwise error %.3g > %.3g" % (err, tol)
    return err


def _adjoint_tc(N, x, F, m, window, **opts):
    from paper_2001_01583_gb300 import Plan, _lib
    R = F.shape[0]
    with Plan(N, x.shape[0], 2.0, m, window, "fp32") as p:
        p.set_option(_lib.OPT_TENSOR_SPREAD, 1)
        if R > 1:
            p.set_option(_lib.OPT_RHS_CAPACITY, R)
        for k, v in opts.items():
            p.set_option(getattr(_lib, "OPT_" + k.upper()), v)
        p.set_points(torch.from_numpy(x).cuda())
        a = p.adjoint(torch.from_numpy(F.astype(np.complex64)).cuda())
        p.sync()
        return a.cpu().numpy().astype(np.complex128), p.info()


WIN = {"gaussian": S.GAUSSIAN, "kaiser_bessel": S.KAISER_BESSEL}


@pytest.mark.parametrize("window,m", [("kaiser_bessel", 4), ("kaiser_bessel", 3), ("kaiser_bessel", 2),
                                      ("gaussian", 3), ("gaussian", 2)])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_tensor_spread_against_oracle(window, m, kind):
    N, M = (40, 36, 44), 40000
    if kind == "uniform":
        x = inputs.uniform_points(M, 3, seed=141)
    else:
        x = inputs.clustered_points(M, 3, 6, 0.02, seed=142)
    F = inputs.complex_normal((1, M), seed=143)
    a, info = _adjoint_tc(N, x, F, m, window, sparse_points=-1)
    taps = 2 * m if window == "kaiser_bessel" else 2 * m + 2
    assert info["taps"] == taps and info["tensor_spread"] == 1 and info["spread_block_threads"] == 256
    assert info["bin"] == (12 - taps, 12 - taps, 16)
    sa = S.adjoint(x, F[0].astype(np.complex64).astype(np.complex128), N, 2.0, m, WIN[window])
    e = _elementwise(a[0], sa, FP32_ELEM)
    assert ndft.rel_l2(a[0], sa) <= FP32_L2
    print("%s m=%d %s: max element error / rms %.2e, rel-l2 %.2e" % (window, m, kind, e, ndft.rel_l2(a[0], sa)))


def test_tensor_spread_several_right_hand_sides_and_sparse_split():
    # three right-hand sides; bins below 20 points go to the grid-warp kernel
    N, M, R = (36, 40, 32), 20000, 3
    x = np.concatenate([inputs.clustered_points(M // 2, 3, 4, 0.03, seed=151),
                        inputs.uniform_points(M - M // 2, 3, seed=152)])
    F = inputs.complex_normal((R, M), seed=153)
    a, info = _adjoint_tc(N, x, F, 4, "kaiser_bessel", sparse_points=20)
    assert info["tensor_spread"] == 1
    for r in range(R):
        sa = S.adjoint(x, F[r].astype(np.complex64).astype(np.complex128), N, 2.0, 4, S.KAISER_BESSEL)
        _elementwise(a[r], sa, FP32_ELEM)
        assert ndft.rel_l2(a[r], sa) <= FP32_L2


def test_tensor_spread_bins_must_fit_the_mma():
    from paper_2001_01583_gb300 import Plan, _lib
    with Plan((32, 32, 32), 100, 2.0, 4, "kaiser_bessel", "fp32") as p:
        p.set_option(_lib.OPT_BIN_0, 8)
        p.set_option(_lib.OPT_BIN_1, 8)
        with pytest.raises(_lib.NFFTError) as e:
            p.set_option(_lib.OPT_TENSOR_SPREAD, 1)     # (8 + 7)^2 = 225 > 128 rows
        assert e.value.status == _lib.ERR_UNSUPPORTED


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_tensor_spread_full_size_3d_configuration(kind):
    N, M = (64, 64, 64), 10 ** 6
    if kind == "uniform":
        x = inputs.uniform_points(M, 3, seed=0)
    else:
        x = inputs.clustered_points(M, 3, 32, 0.02, seed=1)
    F = inputs.complex_normal((1, M), seed=7, dtype=np.complex64)
    a, info = _adjoint_tc(N, x, F, 4, "kaiser_bessel")
    assert info["tensor_spread"] == 1
    sa = S.adjoint(x, F[0].astype(np.complex128), N, 2.0, 4, S.KAISER_BESSEL)
    e = _elementwise(a[0], sa, FP32_ELEM)
    assert ndft.rel_l2(a[0], sa) <= FP32_L2
    print("full size %s: max element error / rms %.2e, rel-l2 %.2e" % (kind, e, ndft.rel_l2(a[0], sa)))


# ---- interpolation on the tensor cores (NFFT_OPT_TENSOR_INTERP) -------------
def _forward_tc(N, x, H, m, window, spread=False, **opts):
    from paper_2001_01583_gb300 import Plan, _lib
    R = H.shape[0]
    with Plan(N, x.shape[0], 2.0, m, window, "fp32") as p:
        p.set_option(_lib.OPT_TENSOR_INTERP, 1)
        if spread:
            p.set_option(_lib.OPT_TENSOR_SPREAD, 1)
        if R > 1:
            p.set_option(_lib.OPT_RHS_CAPACITY, R)
        for k, v in opts.items():
            p.set_option(getattr(_lib, "OPT_" + k.upper()), v)
        p.set_points(torch.from_numpy(x).cuda())
        b = p.forward(torch.from_numpy(H.astype(np.complex64)).cuda())
        p.sync()
        return b.cpu().numpy().astype(np.complex128), p.info()


@pytest.mark.parametrize("window,m", [("kaiser_bessel", 4), ("kaiser_bessel", 3), ("kaiser_bessel", 2),
                                      ("gaussian", 3)])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_tensor_interp_against_oracle(window, m, kind):
    N, M = (40, 36, 44), 40000
    if kind == "uniform":
        x = inputs.uniform_points(M, 3, seed=161)
    else:
        x = inputs.clustered_points(M, 3, 6, 0.02, seed=162)
    H = inputs.complex_normal((1,) + N, seed=163)
    b, info = _forward_tc(N, x, H, m, window, sparse_points_interp=-1)
    taps = 2 * m if window == "kaiser_bessel" else 2 * m + 2
    assert info["tensor_interp"] == 1 and info["interp_block_threads"] == 256
    sb = S.forward(x, H[0].astype(np.complex64).astype(np.complex128), N, 2.0, m, WIN[window])
    e = _elementwise(b[0], sb, FP32_ELEM)
    assert ndft.rel_l2(b[0], sb) <= FP32_L2
    print("interp %s m=%d %s: max element error / rms %.2e, rel-l2 %.2e" % (window, m, kind, e, ndft.rel_l2(b[0], sb)))


def test_tensor_interp_several_right_hand_sides_and_both_directions():
    N, M, R = (36, 40, 32), 20000, 3
    x = np.concatenate([inputs.clustered_points(M // 2, 3, 4, 0.03, seed=171),
                        inputs.uniform_points(M - M // 2, 3, seed=172)])
    H = inputs.complex_normal((R,) + N, seed=173)
    b, info = _forward_tc(N, x, H, 4, "kaiser_bessel", spread=True, sparse_points_interp=30)
    assert info["tensor_interp"] == 1 and info["tensor_spread"] == 1
    for r in range(R):
        sb = S.forward(x, H[r].astype(np.complex64).astype(np.complex128), N, 2.0, 4, S.KAISER_BESSEL)
        _elementwise(b[r], sb, FP32_ELEM)
        assert ndft.rel_l2(b[r], sb) <= FP32_L2


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_tensor_interp_full_size_3d_configuration(kind):
    N, M = (64, 64, 64), 10 ** 6
    if kind == "uniform":
        x = inputs.uniform_points(M, 3, seed=0)
    else:
        x = inputs.clustered_points(M, 3, 32, 0.02, seed=1)
    H = inputs.complex_normal((1,) + N, seed=8, dtype=np.complex64)
    b, info = _forward_tc(N, x, H, 4, "kaiser_bessel")
    assert info["tensor_interp"] == 1
    sb = S.forward(x, H[0].astype(np.complex128), N, 2.0, 4, S.KAISER_BESSEL)
    e = _elementwise(b[0], sb, FP32_ELEM)
    assert ndft.rel_l2(b[0], sb) <= FP32_L2
    print("interp full size %s: max element error / rms %.2e, rel-l2 %.2e" % (kind, e, ndft.rel_l2(b[0], sb)))
