"""GPU parity of the pruned 3-D FFT (NFFT_OPT_PRUNED_FFT).

The FFT of Section 2 is separable: a 3-D DFT is the 1-D DFTs along each
dimension in any order.  The pruned form does the transforms along
dimension 0 over the whole grid and the 2-D transforms of dimensions 1, 2
only over the planes that hold I_N (the adjoint's crop reads nothing else;
the forward's padding leaves every other plane zero, and the 2-D DFT of a
zero plane is zero).  So both forms compute the same gridding NFFT: each is
checked element by element against the step-by-step FP64 oracle, and the
two GPU forms against each other.
"""
import numpy as np
import pytest

from oracle import nfft_steps as S
from paper_2001_01583_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_ELEM = 1e-5


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


def _amplification(N, n, m):
    """Per-frequency factor c_0 / c_k of the deconvolution on I_N (C order)
    and its rms."""
    w = [np.abs(v) for v in S.scaling_weights(S.KAISER_BESSEL, m, list(N), list(n))]
    amp = np.ones(())
    for wt in w:
        amp = np.multiply.outer(amp, wt.max() / wt)
    return amp, float(np.sqrt(np.mean(amp ** 2)))


def _run(N, x, F, H, sigma, m, precision, pruned):
    from paper_2001_01583_gb300 import Plan, _lib
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    with Plan(N, x.shape[0], sigma, m, "kaiser_bessel", precision) as p:
        p.set_option(_lib.OPT_PRUNED_FFT, pruned)
        p.set_points(torch.from_numpy(x).cuda())
        a = p.adjoint(torch.from_numpy(F).to(cdt).cuda())
        b = p.forward(torch.from_numpy(H).to(cdt).cuda())
        p.sync()
        return a.cpu().numpy().astype(np.complex128), b.cpu().numpy().astype(np.complex128), p.info()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,sigma", [((16, 12, 20), 2.0), ((20, 16, 16), 1.25), ((8, 24, 10), 1.5)])
def test_pruned_fft_against_oracle_and_full_fft(N, sigma, precision):
    M, m, R = 1500, 3, 2
    x = inputs.uniform_points(M, 3, seed=301)
    F = inputs.complex_normal((R, M), seed=302)
    H = inputs.complex_normal((R,) + N, seed=303)
    a1, b1, i1 = _run(N, x, F, H, sigma, m, precision, 1)
    a0, b0, i0 = _run(N, x, F, H, sigma, m, precision, 0)
    assert i1["pruned_fft"] == 1 and i0["pruned_fft"] == 0
    if precision == "fp64":
        for r in range(R):
            _elementwise(a1[r], S.adjoint(x, F[r], N, sigma, m, S.KAISER_BESSEL), 1e-12)
            _elementwise(b1[r], S.forward(x, H[r], N, sigma, m, S.KAISER_BESSEL), 1e-12)
            _elementwise(a1[r], a0[r], 1e-12)
            _elementwise(b1[r], b0[r], 1e-12)
        return
    # FP32: rounding on the grid reaches the adjoint's output multiplied by
    # the deconvolution factor c_0 / c_k (Section 2), and the forward's input
    # is multiplied by it before the FFT; at sigma < 2 the factor is large at
    # the edge of I_N.  Compare the adjoint with the factor taken out, the
    # forward against the bar times the factor's rms.
    amp, amp_rms = _amplification(N, i1["n"], m)
    for r in range(R):
        sa = S.adjoint(x, F[r], N, sigma, m, S.KAISER_BESSEL)
        scale = np.sqrt(np.mean(np.abs(sa) ** 2))
        for a in (a1[r], a0[r]):
            assert np.max(np.abs(a - sa) / amp) / scale <= FP32_ELEM
        assert np.max(np.abs(a1[r] - a0[r]) / amp) / scale <= FP32_ELEM
        sb = S.forward(x, H[r], N, sigma, m, S.KAISER_BESSEL)
        _elementwise(b1[r], sb, FP32_ELEM * amp_rms)
        _elementwise(b0[r], sb, FP32_ELEM * amp_rms)
        _elementwise(b1[r], b0[r], FP32_ELEM * amp_rms)


def test_pruned_fft_only_where_it_applies():
    """The automatic choice takes the split form for grids beyond the L2
    cache only; forced on, it still needs three dimensions and planes outside
    I_N (sigma = 1 has none); the autotuner keeps one of the two forms."""
    from paper_2001_01583_gb300 import Plan, _lib
    with Plan((16, 16, 16), 100, 2.0, 3, "kaiser_bessel", "fp32") as p:
        assert p.info()["pruned_fft"] == 0          # a 32^3 grid: the 3-D cuFFT
        p.set_option(_lib.OPT_PRUNED_FFT, 1)
        assert p.info()["pruned_fft"] == 1
    with Plan((256, 256, 256), 100, 2.0, 3, "kaiser_bessel", "fp32") as p:
        assert p.info()["pruned_fft"] == 1          # a 512^3 grid, 1 GiB
    with Plan((16, 16), 100, 2.0, 3, "kaiser_bessel", "fp32") as p:
        p.set_option(_lib.OPT_PRUNED_FFT, 1)
        assert p.info()["pruned_fft"] == 0
    with Plan((16, 16, 16), 100, 1.0, 3, "kaiser_bessel", "fp32") as p:
        p.set_option(_lib.OPT_PRUNED_FFT, 1)
        assert p.info()["pruned_fft"] == 0
    x = inputs.uniform_points(20000, 3, seed=304)
    with Plan((64, 64, 64), 20000, 2.0, 3, "kaiser_bessel", "fp32") as p:
        p.set_points(torch.from_numpy(x).cuda())
        p.autotune(reps=2)
        assert p.info()["pruned_fft"] in (0, 1)
        f = torch.from_numpy(inputs.complex_normal(20000, seed=305)).to(torch.complex64).cuda()
        a = p.adjoint(f).cpu().numpy().astype(np.complex128)
        p.sync()
    sa = S.adjoint(x, f.cpu().numpy().astype(np.complex128), (64, 64, 64), 2.0, 3, S.KAISER_BESSEL)
    _elementwise(a, sa, FP32_ELEM)
