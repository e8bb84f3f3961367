"""The gridding NFFT of the HP-NFFT paper, step by step, in numpy FP64.

TEST INFRASTRUCTURE ONLY.  This is the plain, slow restatement of the method
the CUDA library implements, in the order and notation of Section 2:

  NFFT for Eq. 5 (Fig. 1, Algorithm 2):
    1. spreading   g(l)    = sum_j f(x_j) phi~(x_j - l/n),        l in I_n
    2. FFT         ghat(k) = sum_{l in I_n} g(l) exp(-2 pi i k.l/n)
    3. scaling     fhat(k) = ghat(k) / c_k(phi~),                  k in I_N
  inverse NFFT for Eq. 6 (Fig. 2, Algorithm 5):
    1. subdividing ghat(k) = fhat(k) / c_k(phi~) on I_N, 0 on I_n \\ I_N
    2. inverse FFT g(l)    = sum_{k in I_n} ghat(k) exp(+2 pi i k.l/n)
    3. interpolating f(x_j) = sum_l g(l) phi~(x_j - l/n)

The paper names its windows (Gaussian, B-spline, sinc-power, Kaiser-Bessel;
Section 4) but prints no formulas.  The ones here are the standard NFFT
windows, written per dimension in the cell variable u = n x:

  Gaussian       phi(x) = (pi b)^(-1/2) exp(-u^2 / b),   b = 2 sigma m / ((2 sigma - 1) pi)
                 phihat(k) = (1/n) exp(-b (pi k / n)^2)
  Kaiser-Bessel  phi(x) = (1/pi) sinh(b sqrt(m^2 - u^2)) / sqrt(m^2 - u^2)  for |u| < m, else 0,
                 b = pi (2 - 1/sigma);   phihat(k) = (1/n) I0(m sqrt(b^2 - (2 pi k / n)^2))
  B-spline       phi(x) = M_2m(u), the centred cardinal B-spline of order 2m
                 (the 2m-fold convolution of the indicator of [-1/2, 1/2));
                 phihat(k) = (1/n) sinc(pi k / n)^(2m),  sinc(t) = sin(t) / t
  sinc-power     phi(x) = a sinc(pi a x)^(2m),  a = N (2 sigma - 1) / (2m),
                 truncated to |u| < m;  phihat(k) = M_2m(k / a)

with sigma = n_t / N_t of that dimension.  The scaling weight of a
d-dimensional product window is c_k = prod_t n_t phihat_t(k_t): the Poisson
summation sum_{l in I_n} phi~(x - l/n) exp(-2 pi i k l / n)
= n sum_r phihat(k + r n) exp(-2 pi i (k + r n) x), whose r = 0 term is
n phihat(k) exp(-2 pi i k x).

Truncation: every coordinate is first brought into the paper's torus
Pi = [-1/2, 1/2) of Section 1 as x_t - floor(x_t + 1/2); Eq. 5 is 1-periodic
in x because k is an integer vector, so this changes no exact sum.  A point
with u = n x_t, c = floor(u) then reaches the 2m + 2 cells l = c - m, ...,
c + m + 1 of each dimension, taken modulo n (the oversampled grid is
periodic).  The grid array index of cell l is l mod n, so the FFT in step 2 is
numpy's unshifted DFT.  Where u is an integer up to rounding (a point on a
cell boundary), another reduction of x may put it in the neighbouring cell
with offset 1 instead of 0: the same position, a tap set shifted by one cell,
and a result that differs by the window's truncation error at most.
"""
import math

import numpy as np
import scipy.special

GAUSSIAN = 0
KAISER_BESSEL = 1
B_SPLINE = 2
SINC_POWER = 3
WINDOWS = {"gaussian": GAUSSIAN, "kaiser_bessel": KAISER_BESSEL, "b_spline": B_SPLINE, "sinc_power": SINC_POWER}


def cardinal_bspline(order: int, u):
    """Centred cardinal B-spline M_order(u) (support [-order/2, order/2],
    integral 1) through the uniform B-spline N_k(s) = M_k(s - k/2), s in
    [0, k], and its recurrence N_k(s) = (s N_(k-1)(s) + (k - s) N_(k-1)(s - 1))
    / (k - 1) from N_1 = indicator of [0, 1): every step adds nonnegative
    terms, so it loses no digits."""
    s = np.asarray(u, dtype=np.float64) + order / 2.0
    # vals[i] = N_j(s - i), i = 0 .. order - j
    vals = [((s - i >= 0.0) & (s - i < 1.0)).astype(np.float64) for i in range(order)]
    for j in range(2, order + 1):
        vals = [((s - i) * vals[i] + (j - (s - i)) * vals[i + 1]) / (j - 1) for i in range(order - j + 1)]
    return vals[0]


def _sinc(t):
    t = np.asarray(t, dtype=np.float64)
    out = np.ones_like(t)
    nz = t != 0
    out[nz] = np.sin(t[nz]) / t[nz]
    return out


def oversampled_size(N: int, sigma: float, m: int) -> int:
    """n_t: the smallest even integer >= sigma * N_t whose prime factors are
    2, 3, 5 or 7 (the paper fixes sigma = 2 and does not say how to round).
    Raises ValueError when n_t < 2m + 2 or n_t < N_t."""
    target = int(math.ceil(sigma * N - 1e-9))
    n = max(target, 2)
    while True:
        if n % 2 == 0:
            r = n
            for p in (2, 3, 5, 7):
                while r % p == 0:
                    r //= p
            if r == 1:
                break
        n += 1
    if n < 2 * m + 2 or n < N:
        raise ValueError("oversampled size %d too small for N=%d, m=%d" % (n, N, m))
    return n


def shape_param(window: int, m: int, n: int, N: int) -> float:
    sigma = n / N
    if window == GAUSSIAN:
        return 2.0 * sigma * m / ((2.0 * sigma - 1.0) * math.pi)
    if window == KAISER_BESSEL:
        return math.pi * (2.0 - 1.0 / sigma)
    if window == B_SPLINE:
        return 0.0
    if window == SINC_POWER:
        return N * (2.0 * sigma - 1.0) / (2.0 * m)   # a
    raise ValueError("unknown window %r" % window)


def phi(window: int, u, m: int, n: int, N: int):
    """Window phi at x = u / n (u in cells), untruncated except for the
    Kaiser-Bessel and sinc-power support |u| < m (the B-spline's own support
    is |u| < m)."""
    u = np.asarray(u, dtype=np.float64)
    b = shape_param(window, m, n, N)
    if window == GAUSSIAN:
        return np.exp(-(u * u) / b) / math.sqrt(math.pi * b)
    if window == B_SPLINE:
        return cardinal_bspline(2 * m, u)
    if window == SINC_POWER:
        # a sinc(pi a x)^(2m) at x = u / n, truncated to |u| < m
        return np.where(np.abs(u) < m, b * _sinc(math.pi * b * u / n) ** (2 * m), 0.0)
    out = np.zeros_like(u)
    inside = np.abs(u) < m
    r = np.sqrt(m * m - u[inside] ** 2)
    # sinh(b r) / r, with its limit b at r = 0
    with np.errstate(invalid="ignore", divide="ignore"):
        val = np.where(r > 0, np.sinh(b * r) / np.where(r > 0, r, 1.0), b)
    out[inside] = val / math.pi
    return out


def phi_hat(window: int, k, m: int, n: int, N: int):
    """Fourier transform phihat(k) = int phi(x) exp(-2 pi i k x) dx."""
    k = np.asarray(k, dtype=np.float64)
    b = shape_param(window, m, n, N)
    if window == GAUSSIAN:
        return np.exp(-b * (math.pi * k / n) ** 2) / n
    if window == B_SPLINE:
        return _sinc(math.pi * k / n) ** (2 * m) / n
    if window == SINC_POWER:
        return cardinal_bspline(2 * m, k / b)
    arg = b * b - (2.0 * math.pi * k / n) ** 2
    if np.any(arg < 0):
        raise ValueError("Kaiser-Bessel phihat needs |k| <= n b / (2 pi)")
    return scipy.special.i0(m * np.sqrt(arg)) / n


def scaling_weights(window: int, m: int, N, n):
    """Per-dimension c_t(k_t) = n_t phihat_t(k_t), k_t = -N_t/2 .. N_t/2 - 1."""
    return [nt * phi_hat(window, np.arange(-Nt // 2, Nt // 2), m, nt, Nt) for Nt, nt in zip(N, n)]


def _taps(x, n, m, window, N):
    """For each point and dimension: the 2m + 2 grid indices (mod n) a point
    reaches, and the window weights there.  Returns (idx[t], w[t]) with arrays
    of shape (M, 2m + 2)."""
    M, d = x.shape
    idx, wts = [], []
    off = np.arange(-m, m + 2)
    for t in range(d):
        xt = x[:, t] - np.floor(x[:, t] + 0.5)      # into Pi = [-1/2, 1/2) (Section 1)
        u = n[t] * xt                               # cell coordinate; cell l sits at index l mod n
        c = np.floor(u)
        l = c[:, None] + off[None, :]                # cells c - m .. c + m + 1
        idx.append(np.mod(l, n[t]).astype(np.int64))
        wts.append(phi(window, u[:, None] - l, m, n[t], N[t]))
    return idx, wts


def _tap_products(idx, wts, n):
    """Yield (flat grid index, weight) over every tap combination."""
    d = len(idx)
    W = idx[0].shape[1]
    for combo in np.ndindex(*([W] * d)):
        flat = np.zeros(idx[0].shape[0], dtype=np.int64)
        w = np.ones(idx[0].shape[0])
        for t in range(d):
            flat = flat * n[t] + idx[t][:, combo[t]]
            w = w * wts[t][:, combo[t]]
        yield flat, w


def spread(x, f, N, n, m, window):
    """Step 1 of Fig. 1: g(l) on I_n, stored at array index l mod n."""
    x = np.asarray(x, dtype=np.float64).reshape(len(f), len(N))
    f = np.asarray(f, dtype=np.complex128)
    idx, wts = _taps(x, n, m, window, N)
    size = int(np.prod(n))
    gr = np.zeros(size)
    gi = np.zeros(size)
    for flat, w in _tap_products(idx, wts, n):
        gr += np.bincount(flat, weights=f.real * w, minlength=size)
        gi += np.bincount(flat, weights=f.imag * w, minlength=size)
    return (gr + 1j * gi).reshape(tuple(n))


def interpolate(x, g, N, n, m, window):
    """Step 3 of Fig. 2: f(x_j) = sum_l g(l) phi~(x_j - l/n)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, len(N))
    idx, wts = _taps(x, n, m, window, N)
    gf = np.asarray(g).reshape(-1)
    out = np.zeros(x.shape[0], dtype=np.complex128)
    for flat, w in _tap_products(idx, wts, n):
        out += gf[flat] * w
    return out


def _crop_index(N, n):
    """Array indices (mod n_t) of k_t = -N_t/2 .. N_t/2 - 1, per dimension."""
    return [np.mod(np.arange(-Nt // 2, Nt // 2), nt) for Nt, nt in zip(N, n)]


def adjoint(x, f, N, sigma=2.0, m=4, window=KAISER_BESSEL, n=None):
    """Approximate Eq. 5 by spreading, FFT and scaling (Fig. 1)."""
    N = [int(v) for v in np.atleast_1d(N)]
    n = [oversampled_size(Nt, sigma, m) for Nt in N] if n is None else list(n)
    g = spread(x, f, N, n, m, window)
    ghat = np.fft.fftn(g)                                  # exp(-2 pi i k.l/n)
    ghat_N = ghat[np.ix_(*_crop_index(N, n))]
    c = scaling_weights(window, m, N, n)
    ck = c[0]
    for ct in c[1:]:
        ck = np.multiply.outer(ck, ct)
    return ghat_N / ck


def forward(x, fhat, N, sigma=2.0, m=4, window=KAISER_BESSEL, n=None):
    """Approximate Eq. 6 by subdividing, inverse FFT and interpolating (Fig. 2)."""
    N = [int(v) for v in np.atleast_1d(N)]
    n = [oversampled_size(Nt, sigma, m) for Nt in N] if n is None else list(n)
    c = scaling_weights(window, m, N, n)
    ck = c[0]
    for ct in c[1:]:
        ck = np.multiply.outer(ck, ct)
    ghat = np.zeros(tuple(n), dtype=np.complex128)
    ghat[np.ix_(*_crop_index(N, n))] = np.asarray(fhat).reshape(tuple(N)) / ck
    g = np.fft.ifftn(ghat) * float(np.prod(n))            # unnormalised, exp(+2 pi i k.l/n)
    return interpolate(x, g, N, n, m, window)
