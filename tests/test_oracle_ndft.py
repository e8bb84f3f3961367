"""Pins of the direct-NDFT oracle (Eqs. 3-6) to facts other than itself.

- closed form: one point at rational x gives roots of unity exactly;
- special case: points on the equispaced grid x_j = j/N reduce Eq. 5 to the
  DFT of Eq. 3 and Eq. 6 to |I_N| times the inverse DFT of Eq. 4, checked
  against numpy.fft (non-cubic N catches a transposed dimension);
- invariants: adjoint identity <A^H g, f> = <g, A f>, 1-periodicity in x,
  conjugate symmetry for real f, linearity, the subcell split of Eq. 8.
"""
import numpy as np
import pytest

from oracle import ndft
from paper_2001_01583_gb300 import inputs


def _grid_points(N):
    axes = [np.arange(-n // 2, n // 2) / n for n in N]
    g = np.meshgrid(*axes, indexing="ij")
    return np.stack([a.ravel() for a in g], axis=1)


def test_single_point_roots_of_unity():
    # x = (1/4, -3/8): exp(-2 pi i k.x) = (-i)^k0 * exp(+3 pi i k1 / 4)
    N = (6, 8)
    x = np.array([[0.25, -0.375]])
    out = ndft.adjoint(x, np.array([1.0 + 0j]), N)
    s = np.sqrt(0.5)
    eighth = {0: 1, 1: s + s * 1j, 2: 1j, 3: -s + s * 1j, 4: -1, 5: -s - s * 1j, 6: -1j, 7: s - s * 1j}
    quarter = {0: 1, 1: -1j, 2: -1, 3: 1j}
    for a, k0 in enumerate(range(-3, 3)):
        for b, k1 in enumerate(range(-4, 4)):
            expect = quarter[k0 % 4] * eighth[(3 * k1) % 8]
            assert abs(out[a, b] - expect) < 1e-15


def test_single_point_forward_is_conjugate_row():
    # Eq. 6 with fhat = delta_{k = k*} gives exp(+2 pi i k*.x): k* = (1, -2), x = (1/8, 1/4)
    N = (4, 4)
    x = np.array([[0.125, 0.25]])
    fh = np.zeros(N, dtype=complex)
    fh[1 + 2, -2 + 2] = 1.0
    out = ndft.forward(x, fh, N)
    s = np.sqrt(0.5)
    # exp(+2 pi i (1/8 - 1/2)) = exp(-3 pi i / 4)
    assert abs(out[0] - (-s - s * 1j)) < 1e-15


@pytest.mark.parametrize("N", [(16,), (6, 10), (4, 6, 8)])
def test_grid_points_reduce_to_dft(N):
    x = _grid_points(N)
    f = inputs.complex_normal(x.shape[0], seed=3)
    got = ndft.adjoint(x, f, N)
    F = f.reshape(N)
    # Eq. 3 with j, k in I_N: numpy's DFT indexes from 0, hence the shifts
    ref = np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(F)))
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    back = ndft.forward(x, got, N)
    ref_back = np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(got))).ravel() * np.prod(N)
    assert np.max(np.abs(back - ref_back)) < 1e-12 * np.max(np.abs(ref_back))
    assert np.max(np.abs(back / np.prod(N) - f)) < 1e-12


@pytest.mark.parametrize("d,N,M", [(1, (64,), 300), (2, (12, 20), 200), (3, (8, 6, 10), 150)])
def test_adjoint_identity(d, N, M):
    x = inputs.uniform_points(M, d, seed=11)
    f = inputs.complex_normal(M, seed=12)
    g = inputs.complex_normal(N, seed=13)
    lhs = np.vdot(ndft.forward(x, g, N), f)    # <A^H g, f>
    rhs = np.vdot(g, ndft.adjoint(x, f, N))    # <g, A f>
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_periodic_in_x():
    N = (10, 12)
    x = inputs.uniform_points(50, 2, seed=4)
    f = inputs.complex_normal(50, seed=5)
    shift = np.array([3.0, -7.0])
    a = ndft.adjoint(x, f, N)
    b = ndft.adjoint(x + shift, f, N)
    assert np.max(np.abs(a - b)) < 1e-11


def test_conjugate_symmetry_real_f():
    N = (8, 8, 8)
    x = inputs.uniform_points(40, 3, seed=6)
    f = np.random.default_rng(7).standard_normal(40).astype(complex)
    a = ndft.adjoint(x, f, N)
    inner = a[1:, 1:, 1:]                      # k and -k both inside I_N
    assert np.max(np.abs(inner - np.conj(inner[::-1, ::-1, ::-1]))) < 1e-12


def test_linearity_and_subcell_split():
    N = (6, 6, 6)
    x = inputs.uniform_points(90, 3, seed=8)
    f = inputs.complex_normal(90, seed=9)
    g = inputs.complex_normal(90, seed=10)
    whole = ndft.adjoint(x, 2.0 * f - 1j * g, N)
    parts = 2.0 * ndft.adjoint(x, f, N) - 1j * ndft.adjoint(x, g, N)
    assert np.max(np.abs(whole - parts)) < 1e-12 * np.max(np.abs(whole))
    # Eq. 8: the sum of the sub-NDFTs over a partition of the points
    split = np.random.default_rng(1).integers(0, 4, size=90)
    acc = sum(ndft.adjoint(x[split == i], f[split == i], N) for i in range(4))
    assert np.max(np.abs(acc - ndft.adjoint(x, f, N))) < 1e-12 * np.max(np.abs(acc))


def test_sampled_modes_match_full():
    N = (6, 8, 4)
    x = inputs.uniform_points(70, 3, seed=14)
    f = inputs.complex_normal(70, seed=15)
    full = ndft.adjoint(x, f, N)
    idx = [(0, 0, 0), (5, 7, 3), (2, 4, 1), (3, 1, 2)]
    ksel = np.array([[a - 3, b - 4, c - 2] for a, b, c in idx])
    got = ndft.adjoint(x, f, N, ksel=ksel)
    assert np.max(np.abs(got - np.array([full[i] for i in idx]))) < 1e-12
    fh = inputs.complex_normal(N, seed=16)
    allj = ndft.forward(x, fh, N)
    sel = np.array([69, 0, 33])
    assert np.max(np.abs(ndft.forward(x, fh, N, jsel=sel) - allj[sel])) < 1e-13


def test_thread_count_does_not_change_results():
    N = (16, 16)
    x = inputs.uniform_points(500, 2, seed=17)
    f = inputs.complex_normal(500, seed=18)
    a = ndft.adjoint(x, f, N, threads=1)
    b = ndft.adjoint(x, f, N, threads=7)
    assert np.array_equal(a, b)
