"""Pins of the Ewald oracle (Section 5, Eqs. 10-12).

- the fluorite Madelung constant the paper prints (Section 5: 2.5194);
- the rock-salt Madelung constant 1.747565 (textbook value, e.g. Kittel,
  Introduction to Solid State Physics), a second crystal through the same code;
- the total energy does not depend on the Ewald parameter alpha (Section 5);
- the structure factor of a perfect lattice has a closed form:
  S(n) = L_c^3 F(n / L_c) if every n_t is a multiple of L_c, else 0, with
  F(h) = sum over the cell basis of q_b exp(-2 pi i h.b).
"""
import math
import os

import numpy as np

from oracle import ewald
from paper_2001_01583_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return float([ln for ln in fh if ln.strip() and not ln.startswith("#")][0])


def _energy(r, q, L, alpha):
    rcut = min(7.0 / alpha, 0.99 * L)
    nmax = int(math.ceil(2.2 * alpha * L))
    return ewald.ewald_energy(r, q, L, alpha, rcut, nmax)


def test_fluorite_madelung_matches_paper():
    r, q, L = inputs.fluorite(2)
    U = _energy(r, q, L, 1.5)
    mad = ewald.madelung(U, len(q), 3, 2, -1)
    assert abs(mad - _golden("madelung_fluorite.txt")) < 5e-5


def test_rock_salt_madelung_textbook():
    r, q, L = inputs.rock_salt(2)
    U = _energy(r, q, L, 1.5)
    assert abs(ewald.madelung(U, len(q), 2, 1, -1) - 1.747564594633) < 1e-9


def test_total_energy_independent_of_alpha():
    r, q, L = inputs.fluorite(2)
    a = _energy(r, q, L, 1.2)
    b = _energy(r, q, L, 1.6)
    assert abs(a - b) < 1e-9 * abs(a)


def test_structure_factor_closed_form():
    Lc = 2
    r, q, L = inputs.fluorite(Lc)
    N = (8, 8, 8)
    S = ewald.structure_factor(r, q, L, N)
    basis_frac = r[:12] / (L / Lc)        # the first cell's 12 ions, in cell units
    qb = q[:12]
    for a, n0 in enumerate(range(-4, 4)):
        for b, n1 in enumerate(range(-4, 4)):
            for c, n2 in enumerate(range(-4, 4)):
                n = np.array([n0, n1, n2])
                if np.all(n % Lc == 0):
                    h = n // Lc
                    F = np.sum(qb * np.exp(-2j * np.pi * (basis_frac @ h)))
                    expect = Lc ** 3 * F
                else:
                    expect = 0.0
                assert abs(S[a, b, c] - expect) < 1e-10


# ---- forces: the negative gradients of Eqs. 11 and 12 -----------------------
def _random_ions(n, L, seed):
    rng = np.random.default_rng(seed)
    r = rng.random((n, 3)) * L
    q = rng.choice([-1.0, 2.0], size=n)
    return r, q - q.mean()   # a neutral box


def _fd_force(energy, r, i, t, h=1e-5):
    rp, rm = r.copy(), r.copy()
    rp[i, t] += h
    rm[i, t] -= h
    return -(energy(rp) - energy(rm)) / (2 * h)


def test_real_space_forces_are_the_energy_gradient():
    # central differences of Eq. 11 itself, component by component: a dropped
    # term, a wrong sign or a wrong power of d fails
    L, alpha, rc = 7.0, 0.9, 3.0
    r, q = _random_ions(24, L, seed=3)
    F = ewald.real_space_forces(r, q, L, alpha, rc)
    for i, t in [(0, 0), (3, 1), (11, 2), (23, 0)]:
        fd = _fd_force(lambda rr: ewald.real_space_energy(rr, q, L, alpha, rc), r, i, t)
        assert abs(F[i, t] - fd) <= 1e-7 * np.abs(F).max(), (i, t, F[i, t], fd)


def test_reciprocal_forces_are_the_energy_gradient():
    L, alpha, N = 7.0, 0.9, (8, 10, 8)
    r, q = _random_ions(20, L, seed=4)
    F = ewald.reciprocal_forces(r, q, L, alpha, N)

    def energy(rr):
        return ewald.reciprocal_sum(ewald.structure_factor(rr, q, L, N), L, alpha)
    for i, t in [(0, 0), (5, 1), (13, 2), (19, 1)]:
        fd = _fd_force(energy, r, i, t)
        assert abs(F[i, t] - fd) <= 1e-7 * np.abs(F).max(), (i, t, F[i, t], fd)


def test_forces_sum_to_zero():
    # Newton's third law for the pair sum; sum_i F^K_i = (2/L^2) sum_n w n
    # Im(S(n) conj(S(n))) = 0 for the reciprocal part
    L, alpha = 8.0, 0.8
    r, q = _random_ions(30, L, seed=5)
    FR = ewald.real_space_forces(r, q, L, alpha, 3.5)
    FK = ewald.reciprocal_forces(r, q, L, alpha, (10, 10, 10))
    assert np.all(np.abs(FR.sum(axis=0)) <= 1e-12 * np.abs(FR).sum())
    assert np.all(np.abs(FK.sum(axis=0)) <= 1e-12 * np.abs(FK).sum())


def test_perfect_fluorite_has_no_net_force_on_any_ion():
    # every ion of the perfect crystal sits on a site whose symmetry leaves no
    # invariant vector, so both parts vanish ion by ion, while a displaced
    # ion is pulled back (a restoring force along the displacement)
    r, q, L = inputs.fluorite(2)
    alpha = 0.9
    FR = ewald.real_space_forces(r, q, L, alpha, 0.49 * L)
    FK = ewald.reciprocal_forces(r, q, L, alpha, (12, 12, 12))
    scale = np.abs(q).max() ** 2 * alpha ** 2
    assert np.abs(FR).max() <= 1e-10 * scale and np.abs(FK).max() <= 1e-10 * scale
    r2 = r.copy()
    r2[0, 0] += 0.05
    F2 = ewald.real_space_forces(r2, q, L, alpha, 0.49 * L) + ewald.reciprocal_forces(r2, q, L, alpha, (12, 12, 12))
    assert F2[0, 0] < 0
