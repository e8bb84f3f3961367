"""Host-side parts of the parameter picker (no GPU): features, the rule of
thumb, the validity rule, the cost terms and the cost-model fit, the
fallback of nfft_pick_params without a network."""
import ctypes
import math

import numpy as np
import pytest

from paper_2001_01583_gb300 import _lib, picker


def test_features_of_a_problem():
    f = picker.features(3, (64, 32, 16), 10 ** 6, 0.01, 1e-5)
    assert np.allclose(f, [3, 6, 5, 4, 6, 0.01, -5, math.log10(1e6 / (64 * 32 * 16))])
    f1 = picker.features(1, (1024,), 500, 0.0, 1e-9)
    assert np.allclose(f1, [1, 10, 0, 0, math.log10(500), 0.0, -9, math.log10(500 / 1024)])
    with pytest.raises(RuntimeError):
        picker.features(4, (8, 8, 8), 10, 0.0, 1e-5)
    with pytest.raises(RuntimeError):
        picker.features(2, (8, 8), 10, 0.0, 0.0)


def test_rule_of_thumb():
    # Kaiser-Bessel error estimate exp(-2 pi m sqrt(1 - 1/sigma)) at sigma = 2
    for eps in (1e-3, 1e-5, 1e-8, 1e-10, 1e-14, 1e-30):
        s, m, w = picker.rule_of_thumb(eps)
        want = min(12, max(2, math.ceil(math.log(1 / eps) / (2 * math.pi * math.sqrt(0.5)))))
        assert (s, m, w) == (2.0, want, _lib.KAISER_BESSEL)
    assert picker.rule_of_thumb(1e-5)[1] == 3


def test_pick_without_network_falls_back():
    lib = _lib.load()
    N = (ctypes.c_int64 * 3)(64, 64, 64)
    s, m, w, fb = ctypes.c_double(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.nfft_pick_params(None, 3, N, 10 ** 6, 0.0, 1e-7, _lib.FP32_MIXED, ctypes.byref(s), ctypes.byref(m),
                                ctypes.byref(w), ctypes.byref(fb)) == _lib.OK
    assert (s.value, m.value, w.value, fb.value) == picker.rule_of_thumb(1e-7) + (1,)
    assert lib.nfft_pick_params(None, 3, N, 10 ** 6, 0.0, -1.0, _lib.FP64, ctypes.byref(s), ctypes.byref(m),
                                ctypes.byref(w), ctypes.byref(fb)) == _lib.ERR_INVALID_ARG
    assert lib.nfft_pick_params(None, 3, N, 10 ** 6, 0.0, 1e-7, 7, ctypes.byref(s), ctypes.byref(m), ctypes.byref(w),
                                ctypes.byref(fb)) == _lib.ERR_INVALID_ARG


def test_candidates_and_validity():
    assert len(picker.CANDIDATES) == 66
    assert len(set(picker.CANDIDATES)) == 66
    assert picker.valid((16, 16), 2.0, 12) is True      # ceil(32) >= 26
    assert picker.valid((16, 16), 2.0, 15) is True      # 32 >= 32
    assert picker.valid((16, 16), 2.0, 16) is False
    assert picker.valid((8,), 1.25, 4) is True           # ceil(10) >= 10
    assert picker.valid((8,), 1.25, 5) is False


def test_cost_terms_and_fit():
    t = picker.cost_terms((64, 64, 64), 10 ** 6, 2.0, 4, _lib.KAISER_BESSEL)
    P = 128.0 ** 3
    # 488 points per 8 x 8 x 16 bin: dense
    assert np.allclose(t, [1e6 * 8 ** 3, 0.0, 1e6 * 3 * 8, P * math.log2(P), P, 1e6, 1.0])
    tg = picker.cost_terms((64, 64, 64), 10 ** 6, 2.0, 4, _lib.GAUSSIAN)
    assert tg[0] == 1e6 * 10 ** 3 and tg[2] == 1e6 * 3 * 10
    # 2e4 points: 10 per bin, below 2 * 15 * 15 * 23 / 512 = 20.2: sparse
    ts = picker.cost_terms((64, 64, 64), 20000, 2.0, 4, _lib.KAISER_BESSEL)
    assert ts[0] == 0.0 and ts[1] == 20000 * 8 ** 3
    # the fit recovers a known nonnegative model from exact data
    rng = np.random.default_rng(0)
    coef = np.array([2e-9, 9e-9, 5e-9, 3e-10, 0.0, 1e-7, 0.02])
    rows = [picker.cost_terms((int(n),) * 3, int(M), s, m, w)
            for n, M, s, m, w in zip(rng.choice([16, 32, 64, 128], 60), 10 ** rng.uniform(3, 7, 60),
                                     rng.choice([1.25, 1.5, 2.0], 60), rng.integers(2, 9, 60), rng.integers(0, 2, 60))]
    times = np.array(rows) @ coef
    model = picker.CostModel.fit(rows, times)
    assert np.allclose(np.array(rows) @ model.coef, times, rtol=1e-6)


def test_normalisers_ignore_unlabelled_outputs():
    X = np.array([[1.0, 5.0], [3.0, 5.0]])
    T = np.array([[2.0, 100.0], [4.0, 7.0]])
    W = np.array([[1.0, 0.0], [1.0, 1.0]])
    fm, fs, om, osd = picker.normalisers(X, T, W)
    assert np.allclose(fm, [2.0, 5.0]) and np.allclose(fs, [1.0, 1.0])
    assert np.allclose(om, [3.0, 7.0]) and np.allclose(osd, [1.0, 1.0])


def test_deconvolution_amplification_against_oracle():
    """rms and peak of c_0 / c_k over I_N from the library's host rule agree
    with the oracle's transforms of the windows (its n_t phi_hat)."""
    from oracle import nfft_steps as S
    lib = _lib.load()
    for N, sigma, m, window in [((64,), 2.0, 4, _lib.KAISER_BESSEL), ((36, 30), 1.25, 5, _lib.KAISER_BESSEL),
                                ((32, 28, 24), 1.5, 6, _lib.GAUSSIAN), ((20, 16, 18), 2.0, 12, _lib.GAUSSIAN)]:
        Narr = (ctypes.c_int64 * len(N))(*N)
        rms, peak = ctypes.c_double(), ctypes.c_double()
        assert lib.nfft_deconv_amplification(len(N), Narr, sigma, m, window, ctypes.byref(rms),
                                             ctypes.byref(peak)) == _lib.OK
        n = [S.oversampled_size(v, sigma, m) for v in N]
        r, p = 1.0, 1.0
        for wt in S.scaling_weights(window, m, list(N), n):
            a = np.abs(wt).max() / np.abs(wt)
            r *= np.sqrt(np.mean(a ** 2))
            p *= a.max()
        assert abs(rms.value / r - 1) < 1e-9 and abs(peak.value / p - 1) < 1e-9, (N, rms.value, r, peak.value, p)
