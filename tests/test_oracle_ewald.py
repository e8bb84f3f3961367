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
