"""Pins of the step-by-step gridding-NFFT oracle.

- window Fourier transforms phihat against numerical quadrature of phi
  (exact for the Gaussian; within the O(exp(-b m)) truncation term for the
  Kaiser-Bessel window, whose I0 formula transforms the untruncated function);
- the approximation error against the direct NDFT (Eq. 9) obeys the
  textbook exponential decay bounds for the Gaussian and Kaiser-Bessel
  windows and shrinks with m;
- the NFFT and its inverse procedure are exact transposes (adjoint identity
  to rounding, independent of the window error);
- the oversampled size rule;
- the B-spline and sinc-power windows (Section 4, Fig. 12): textbook values,
  integral and partition of unity of the cardinal B-spline, both transforms
  against quadrature (the sinc-power one within its truncation tail), the
  error decay against the direct NDFT, exact transposition.
"""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle import ndft, nfft_steps as S
from paper_2001_01583_gb300 import inputs


@pytest.mark.parametrize("window,m,N,n", [(S.GAUSSIAN, 4, 32, 64), (S.GAUSSIAN, 6, 16, 40),
                                          (S.KAISER_BESSEL, 4, 32, 64), (S.KAISER_BESSEL, 3, 20, 30)])
def test_phi_hat_matches_quadrature(window, m, N, n):
    # phihat(k) = int phi(x) exp(-2 pi i k x) dx; phi is even so the cosine part suffices
    lim = m / n if window == S.KAISER_BESSEL else 12.0 * math.sqrt(S.shape_param(window, m, n, N)) / n
    for k in (0, 1, N // 4, N // 2 - 1, -N // 2):
        val, _ = scipy.integrate.quad(lambda x: float(S.phi(window, np.array([n * x]), m, n, N)[0])
                                      * math.cos(2 * math.pi * k * x), -lim, lim, limit=400,
                                      epsabs=1e-15, epsrel=1e-13)
        ref = float(S.phi_hat(window, k, m, n, N))
        if window == S.GAUSSIAN:
            assert abs(val - ref) <= 1e-10 * abs(ref)
        else:
            # the I0 formula is the transform of the untruncated Kaiser-Bessel
            # function; cutting it at |u| = m changes the transform by a
            # amount of order exp(-b m) relative to the peak phihat(0)
            b = S.shape_param(window, m, n, N)
            peak = float(S.phi_hat(window, 0, m, n, N))
            assert abs(val - ref) <= (2.0 * math.exp(-b * m) + 1e-12) * peak


def test_oversampled_size_rule():
    assert S.oversampled_size(64, 2.0, 4) == 128
    assert S.oversampled_size(100, 1.25, 4) == 126      # 125 is odd -> 126 = 2 * 3^2 * 7
    assert S.oversampled_size(256, 1.5, 4) == 384
    with pytest.raises(ValueError):
        S.oversampled_size(4, 2.0, 6)                    # n = 8 < 2m + 2


def _gauss_bound(m, sigma):
    # Steidl (1998): E_inf <= 4 exp(-m pi (1 - 1/(2 sigma - 1)))
    return 4.0 * math.exp(-m * math.pi * (1.0 - 1.0 / (2.0 * sigma - 1.0)))


def _kb_bound(m, sigma):
    # Potts & Steidl: E_inf <= 4 pi (sqrt(m) + m) (1 - 1/sigma)^(1/4) exp(-2 pi m sqrt(1 - 1/sigma))
    s = 1.0 - 1.0 / sigma
    return 4.0 * math.pi * (math.sqrt(m) + m) * s ** 0.25 * math.exp(-2.0 * math.pi * m * math.sqrt(s))


@pytest.mark.parametrize("window,bound", [(S.GAUSSIAN, _gauss_bound), (S.KAISER_BESSEL, _kb_bound)])
def test_error_within_textbook_bound_and_decreasing(window, bound):
    N = (64,)
    M = 400
    x = inputs.uniform_points(M, 1, seed=21)
    f = inputs.complex_normal(M, seed=22)
    exact = ndft.adjoint(x, f, N)
    errs = []
    for m in (2, 3, 4, 5, 6):
        approx = S.adjoint(x, f, N, 2.0, m, window)
        e = ndft.rel_l2(approx, exact)
        assert e < bound(m, 2.0), (m, e)
        errs.append(e)
    assert all(b < a for a, b in zip(errs, errs[1:]))


@pytest.mark.parametrize("d,N", [(1, (32,)), (2, (12, 16)), (3, (8, 8, 6))])
@pytest.mark.parametrize("window", [S.GAUSSIAN, S.KAISER_BESSEL])
def test_nfft_pair_is_exact_transpose(d, N, window):
    M = 120
    x = inputs.uniform_points(M, d, seed=31)
    f = inputs.complex_normal(M, seed=32)
    g = inputs.complex_normal(N, seed=33)
    lhs = np.vdot(S.forward(x, g, N, 2.0, 3, window), f)
    rhs = np.vdot(g, S.adjoint(x, f, N, 2.0, 3, window))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_forward_error_3d_kaiser_bessel():
    N = (16, 16, 16)
    M = 800
    x = inputs.uniform_points(M, 3, seed=41)
    fh = inputs.complex_normal(N, seed=42)
    e = ndft.rel_l2(S.forward(x, fh, N, 2.0, 4, S.KAISER_BESSEL), ndft.forward(x, fh, N))
    assert e < _kb_bound(4, 2.0)
    assert e < 1e-6


def test_points_on_cell_boundaries_and_wrap():
    # a point at x = -1/2 and one at x = +1/2 are the same point (Eq. 5 is
    # 1-periodic); both must give the same NFFT output
    N = (16,)
    f = np.array([1.0 + 0.5j])
    a = S.adjoint(np.array([[-0.5]]), f, N, 2.0, 4, S.KAISER_BESSEL)
    b = S.adjoint(np.array([[0.5]]), f, N, 2.0, 4, S.KAISER_BESSEL)
    assert np.max(np.abs(a - b)) < 1e-14
    exact = ndft.adjoint(np.array([[-0.5]]), f, N)
    assert ndft.rel_l2(a, exact) < 1e-6


def test_reduction_into_the_torus():
    # the coordinate reduction lands in Pi = [-1/2, 1/2) (Section 1) and
    # moves every coordinate by an integer
    x = np.array([[-0.5, 0.5, 0.25], [3.75, -7.125, 12.5], [-0.2500001, 1e-17, -1e-17]])
    n = [16, 16, 16]
    idx, _ = S._taps(x, n, 3, S.KAISER_BESSEL, [8, 8, 8])
    for t in range(3):
        xt = x[:, t] - np.floor(x[:, t] + 0.5)
        assert np.all((xt >= -0.5) & (xt < 0.5))
        assert np.all(np.abs((x[:, t] - xt) - np.round(x[:, t] - xt)) == 0)
        # the first tap is floor(n x) - m, modulo n
        assert np.array_equal(idx[t][:, 0], np.mod(np.floor(n[t] * xt) - 3, n[t]))


@pytest.mark.parametrize("window,m", [(S.KAISER_BESSEL, 4), (S.GAUSSIAN, 6), (S.B_SPLINE, 3), (S.SINC_POWER, 4)])
def test_cell_choice_at_a_boundary_moves_the_result_by_truncation_only(window, m):
    # a point exactly on a cell boundary can be taken as (cell c, offset 0) or
    # (cell c - 1, offset 1): both tap sets place the window at the same
    # position, so the two gridding results differ from each other no more
    # than each differs from the exact sum (the window error)
    N, n = (16,), [32]
    x0 = np.array([[5.0 / 32]])                 # u = 5 exactly
    f = np.array([0.7 - 0.2j])
    a = S.adjoint(x0, f, N, 2.0, m, window)
    # the same point taken as cell 4 at offset 1: every tap one cell lower,
    # weights at the same distances u - l
    idx, w = S._taps(x0, n, m, window, N)
    lo_idx = np.mod(idx[0] - 1, n[0])
    u = 5.0
    lo_w = S.phi(window, u - (np.floor(u) - 1 + np.arange(-m, m + 2)), m, n[0], N[0])
    g = np.zeros(n[0], dtype=np.complex128)
    np.add.at(g, lo_idx[0], f[0] * lo_w)
    ghat = np.fft.fft(g)[np.mod(np.arange(-8, 8), 32)]
    b = ghat / S.scaling_weights(window, m, N, n)[0]
    exact = ndft.adjoint(x0, f, N)
    e_a = ndft.rel_l2(a, exact)
    assert ndft.rel_l2(b, exact) <= 1.5 * max(e_a, 1e-15)
    assert ndft.rel_l2(a, b) <= 2.5 * max(e_a, 1e-15)
    if window in (S.KAISER_BESSEL, S.B_SPLINE, S.SINC_POWER):
        # these windows vanish at |u| = m, so the extra tap of either set is 0
        assert ndft.rel_l2(a, b) < 1e-14


# ---- B-spline and sinc-power windows (Section 4, Fig. 12) ----------------------
def test_cardinal_bspline_textbook_values():
    # the hat function and the cubic B-spline, and the general properties
    assert np.allclose(S.cardinal_bspline(2, np.array([0.0, 0.5, -0.5, 1.0])), [1.0, 0.5, 0.5, 0.0])
    assert np.allclose(S.cardinal_bspline(4, np.array([0.0, 1.0, -1.0, 0.5, 2.0])), [2 / 3, 1 / 6, 1 / 6, 23 / 48, 0.0])
    for order in (2, 5, 8, 13, 24):
        u = np.linspace(-order / 2 - 1, order / 2 + 1, 20001)
        assert abs(np.trapezoid(S.cardinal_bspline(order, u), u) - 1.0) < 1e-6
        shift = 0.3137
        assert abs(S.cardinal_bspline(order, shift + np.arange(-order, order + 1)).sum() - 1.0) < 1e-12
        assert np.allclose(S.cardinal_bspline(order, u), S.cardinal_bspline(order, -u), atol=1e-14)


@pytest.mark.parametrize("m,N,n", [(2, 16, 32), (4, 32, 64), (6, 20, 40), (3, 16, 24)])
def test_bspline_phi_hat_matches_quadrature(m, N, n):
    # compact support |u| < m: the transform is exact, no truncation term
    knots = [(j - m) / n for j in range(2 * m + 1)]
    for k in (0, 1, N // 4, N // 2 - 1, -N // 2):
        val, _ = scipy.integrate.quad(lambda x: float(S.phi(S.B_SPLINE, np.array([n * x]), m, n, N)[0])
                                      * math.cos(2 * math.pi * k * x), -m / n, m / n, points=knots, limit=400,
                                      epsabs=1e-15, epsrel=1e-12)
        assert abs(val - float(S.phi_hat(S.B_SPLINE, k, m, n, N))) <= 1e-10 * float(S.phi_hat(S.B_SPLINE, 0, m, n, N))


@pytest.mark.parametrize("m,N,n", [(3, 16, 32), (5, 32, 64), (4, 20, 40)])
def test_sinc_power_phi_hat_matches_quadrature(m, N, n):
    # phi_hat = M_2m(k / a) is the transform of the untruncated a sinc(pi a x)^(2m);
    # cutting at |u| = m changes it by at most the tail mass
    # 2 a int_{m/n}^inf (pi a x)^(-2m) dx = 2 a (pi a)^(-2m) (m/n)^(1-2m) / (2m - 1)
    a = S.shape_param(S.SINC_POWER, m, n, N)
    tail = 2 * a * (math.pi * a) ** (-2 * m) * (m / n) ** (1 - 2 * m) / (2 * m - 1)
    for k in (0, 1, N // 4, N // 2 - 1, -N // 2):
        val, _ = scipy.integrate.quad(lambda x: float(S.phi(S.SINC_POWER, np.array([n * x]), m, n, N)[0])
                                      * math.cos(2 * math.pi * k * x), -m / n, m / n, limit=400,
                                      epsabs=1e-15, epsrel=1e-12)
        assert abs(val - float(S.phi_hat(S.SINC_POWER, k, m, n, N))) <= tail + 1e-12


@pytest.mark.parametrize("window", [S.B_SPLINE, S.SINC_POWER])
def test_bspline_sinc_power_error_decay(window):
    # the B-spline bound of Steidl: E <= 4 (2 sigma - 1)^(-2m); both windows'
    # errors fall by at least a factor 5 per unit of m at sigma = 2
    N = (64,)
    M = 400
    x = inputs.uniform_points(M, 1, seed=21)
    f = inputs.complex_normal(M, seed=22)
    exact = ndft.adjoint(x, f, N)
    errs = [ndft.rel_l2(S.adjoint(x, f, N, 2.0, m, window), exact) for m in (2, 3, 4, 5, 6)]
    for m, e in zip((2, 3, 4, 5, 6), errs):
        assert e < 4.0 * 3.0 ** (-2 * m), (m, e)
    assert all(b < a / 5 for a, b in zip(errs, errs[1:])), errs


@pytest.mark.parametrize("window", [S.B_SPLINE, S.SINC_POWER])
def test_bspline_sinc_power_pair_is_exact_transpose(window):
    N = (12, 16)
    M = 120
    x = inputs.uniform_points(M, 2, seed=31)
    f = inputs.complex_normal(M, seed=32)
    g = inputs.complex_normal(N, seed=33)
    lhs = np.vdot(S.forward(x, g, N, 2.0, 3, window), f)
    rhs = np.vdot(g, S.adjoint(x, f, N, 2.0, 3, window))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
