"""Direct Ewald sum for the fluorite check of Section 5 (Eqs. 10-12).

TEST INFRASTRUCTURE ONLY.  Plain numpy FP64 sums, no NFFT:

  Eq. 11  U^R = 1/2 sum'_n sum_{i,j} q_i q_j erfc(alpha |r_ij + n L|) / |r_ij + n L|
          (the primed sum omits n = 0 when i = j)
  Eq. 12  U^K = 1/(2 pi L) sum_{n != 0} exp(-pi^2 |n|^2 / (alpha L)^2) / |n|^2 S(n) S(-n)
                - alpha / sqrt(pi) sum_i q_i^2
          S(n) = sum_i q_i exp(-2 pi i n.r_i / L)
  Eq. 10  Madelung = U^E m / (N Z+ Z-),  U^E = U^R + U^K

Forces are the negative gradients of Eqs. 11 and 12 with respect to an ion's
position (the paper names MD as the application but prints no force
formula; these are the derivatives written out):

  F^R_i = q_i sum'_n sum_j q_j (erfc(alpha d)/d + 2 alpha/sqrt(pi) exp(-alpha^2 d^2)) (r_i - r_j + n L) / d^2,
          d = |r_i - r_j + n L|
  F^K_i = (2 q_i / L^2) sum_{n != 0} exp(-pi^2 |n|^2 / (alpha L)^2) / |n|^2  n  Im(S(n) exp(2 pi i n.r_i / L))

(from d|S(n)|^2/dr_i = 2 Re(conj(S(n)) dS(n)/dr_i), dS(n)/dr_i =
-2 pi i q_i n / L exp(-2 pi i n.r_i / L)); the self term does not depend on
the positions.

Lengths are in units of r0, energies in units of q_e^2 / r0 (Gaussian units),
so U^E is negative for an ionic crystal and Z- = -1 makes Eq. 10 positive.
"""
import math

import numpy as np
import scipy.special

from . import ndft


def real_space_energy(r, q, L, alpha, rcut):
    """Eq. 11 with every image within rcut (rcut < L is required so that the
    images |n_t| <= 1 of the minimum-image separation cover the cutoff)."""
    r = np.asarray(r, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    if rcut >= L:
        raise ValueError("rcut must be below the box length")
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], dtype=np.float64) * L
    total = 0.0
    n_ions = r.shape[0]
    chunk = max(1, 4096 * 64 // max(n_ions, 1))
    for i0 in range(0, n_ions, chunk):
        ri = r[i0:i0 + chunk]
        dr = ri[:, None, :] - r[None, :, :]
        dr -= L * np.round(dr / L)                     # minimum image
        qq = q[i0:i0 + chunk, None] * q[None, :]
        for s in shifts:
            dist = np.sqrt(np.sum((dr + s) ** 2, axis=-1))
            mask = (dist > 0) & (dist < rcut)           # the i = j, n = 0 term is omitted
            total += np.sum(qq[mask] * scipy.special.erfc(alpha * dist[mask]) / dist[mask])
    return 0.5 * total


def structure_factor(r, q, L, N):
    """S(n) for n in I_N (C order), via the direct NDFT of Eq. 5 at x = r / L."""
    x = np.asarray(r, dtype=np.float64) / L
    return ndft.adjoint(x, np.asarray(q, dtype=np.complex128), N)


def reciprocal_sum(S, L, alpha):
    """The n != 0 sum of Eq. 12 over the index set S is given on (C order,
    each n_t ascending from -N_t/2), without the self term."""
    S = np.asarray(S)
    axes = [np.arange(-n // 2, n // 2, dtype=np.float64) for n in S.shape]
    n2 = sum(np.meshgrid(*[a * a for a in axes], indexing="ij"))
    w = np.zeros_like(n2)
    nz = n2 > 0
    w[nz] = np.exp(-math.pi ** 2 * n2[nz] / (alpha * L) ** 2) / n2[nz]
    return float(np.sum(w * np.abs(S) ** 2) / (2.0 * math.pi * L))


def self_energy(q, alpha):
    return -alpha / math.sqrt(math.pi) * float(np.sum(np.asarray(q, dtype=np.float64) ** 2))


def reciprocal_energy(r, q, L, alpha, nmax):
    """Eq. 12 with every n in [-nmax, nmax]^3 (plus the self term)."""
    S = structure_factor(r, q, L, (2 * nmax + 2,) * 3)
    return reciprocal_sum(S, L, alpha) + self_energy(q, alpha)


def ewald_energy(r, q, L, alpha, rcut, nmax):
    """U^E = U^R + U^K (Eqs. 11-12)."""
    return real_space_energy(r, q, L, alpha, rcut) + reciprocal_energy(r, q, L, alpha, nmax)


def madelung(U, n_ions, ions_per_formula, z_plus, z_minus):
    """Eq. 10."""
    return U * ions_per_formula / (n_ions * z_plus * z_minus)


def real_space_forces(r, q, L, alpha, rcut):
    """F^R (n x 3): the negative gradient of real_space_energy, every image
    within rcut (rcut < L)."""
    r = np.asarray(r, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    if rcut >= L:
        raise ValueError("rcut must be below the box length")
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], dtype=np.float64) * L
    n_ions = r.shape[0]
    F = np.zeros((n_ions, 3))
    chunk = max(1, 4096 * 64 // max(n_ions, 1))
    for i0 in range(0, n_ions, chunk):
        ri = r[i0:i0 + chunk]
        dr = ri[:, None, :] - r[None, :, :]
        dr -= L * np.round(dr / L)                     # minimum image
        qq = q[i0:i0 + chunk, None] * q[None, :]
        for s in shifts:
            v = dr + s                                  # r_i - r_j + n L
            dist = np.sqrt(np.sum(v ** 2, axis=-1))
            mask = (dist > 0) & (dist < rcut)
            d = np.where(mask, dist, 1.0)
            g = (scipy.special.erfc(alpha * d) / d + 2.0 * alpha / math.sqrt(math.pi) * np.exp(-(alpha * d) ** 2)) \
                / (d * d)
            g = np.where(mask, qq * g, 0.0)
            F[i0:i0 + chunk] += np.sum(g[:, :, None] * v, axis=1)
    return F


def reciprocal_forces(r, q, L, alpha, N):
    """F^K (n x 3) with n over I_N without 0 (each n_t in [-N_t/2, N_t/2)):
    the negative gradient of reciprocal_sum(structure_factor(r, q, L, N), L,
    alpha), the energy under the same truncation.  S by the direct NDFT of
    Eq. 5, the n-sum by the direct NDFT of Eq. 6 of w(n) n_t S(n)."""
    r = np.asarray(r, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    N = tuple(int(v) for v in N)
    x = r / L
    S = ndft.adjoint(x, q.astype(np.complex128), N)
    axes = [np.arange(-n // 2, n // 2, dtype=np.float64) for n in N]
    grids = np.meshgrid(*axes, indexing="ij")
    n2 = sum(g * g for g in grids)
    w = np.zeros_like(n2)
    nz = n2 > 0
    w[nz] = np.exp(-math.pi ** 2 * n2[nz] / (alpha * L) ** 2) / n2[nz]
    F = np.zeros((r.shape[0], 3))
    for t in range(3):
        phase = ndft.forward(x, w * grids[t] * S, N)    # sum_n w n_t S(n) exp(+2 pi i n.x_i)
        F[:, t] = 2.0 * q / (L * L) * phase.imag
    return F
