"""GPU parity of the Ewald reciprocal energy (Section 5, Eqs. 10-12).

Pins:
  - the reduction alone: S(n) from the oracle's direct NDFT, n-sum of Eq. 12
    on the GPU against the oracle's sum (FP64 rounding level);
  - the fluorite lattice of the paper (32^3 cells, 393216 ions, N = 128^3,
    m = 6): the GPU n-sum against the closed form of a perfect lattice,
    S(n) = L_c^3 F(n / L_c) on n in L_c Z^3 and 0 elsewhere, summed over
    exactly I_N (exact parity, no truncation question);
  - the Madelung constant (Eq. 10): GPU reciprocal energy plus the oracle's
    real-space energy (Eq. 11) against the oracle's direct Ewald sum and the
    value the paper prints (2.5194).
At the paper's alpha in [1.2, 1.8] the reciprocal sum over I_N = 128^3 is not
converged (the Gaussian factor is still large at |n_t| = 64); the Madelung
check therefore uses alpha = 0.6 at L_c = 32 and a converged alpha at L_c = 4.
"""
import math
import os

import numpy as np
import pytest

from oracle import ewald, ndft
from paper_2001_01583_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return float([ln for ln in fh if ln.strip() and not ln.startswith("#")][0])


def _plan(N, M, m, precision):
    from paper_2001_01583_gb300 import Plan
    return Plan(N, M, 2.0, m, "kaiser_bessel", precision)


def _cdt(precision):
    return torch.complex128 if precision == "fp64" else torch.complex64


def _closed_form_sum(Lc, N, L, alpha):
    """n-sum of Eq. 12 for the perfect fluorite lattice over exactly I_N."""
    r, q, _ = inputs.fluorite(1)
    basis = r / (L / Lc)                  # cell-fraction coordinates of the 12 basis ions
    total = 0.0
    rng = [np.arange(-n // 2, n // 2) for n in N]
    for n0 in rng[0][rng[0] % Lc == 0]:
        for n1 in rng[1][rng[1] % Lc == 0]:
            for n2 in rng[2][rng[2] % Lc == 0]:
                n2sum = n0 * n0 + n1 * n1 + n2 * n2
                if n2sum == 0:
                    continue
                h = np.array([n0, n1, n2]) // Lc
                F = np.sum(q * np.exp(-2j * np.pi * (basis @ h)))
                S = Lc ** 3 * F
                total += math.exp(-math.pi ** 2 * n2sum / (alpha * L) ** 2) / n2sum * abs(S) ** 2
    return total / (2 * math.pi * L)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_reciprocal_sum_reduction(precision, tol):
    N = (12, 10, 16)
    M = 300
    x = inputs.uniform_points(M, 3, seed=1)
    q = np.random.default_rng(2).choice([-1.0, 2.0], size=M).astype(np.complex128)
    S = ndft.adjoint(x, q, N)
    L, alpha = 7.5, 0.9
    ref = ewald.reciprocal_sum(S, L, alpha)
    with _plan(N, M, 4, precision) as p:
        a = p.ewald_reciprocal_sum(torch.from_numpy(S).to(_cdt(precision)).cuda(), L, alpha)
        b = p.ewald_reciprocal_sum(torch.from_numpy(S).to(_cdt(precision)).cuda(), L, alpha)
        p.sync()
    assert abs(a.item() - ref) <= tol * abs(ref)
    assert a.item() == b.item()           # deterministic reduction


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-5)])
@pytest.mark.parametrize("alpha", [0.6, 1.5])
def test_fluorite_lattice_closed_form(precision, tol, alpha):
    Lc = 32
    r, q, L = inputs.fluorite(Lc)
    x = inputs.box_points(r, L)
    N = (128, 128, 128)
    ref = _closed_form_sum(Lc, N, L, alpha)
    with _plan(N, len(q), 6, precision) as p:
        p.set_points(torch.from_numpy(x).cuda())
        uk, nsum, self_term = p.ewald_reciprocal(torch.from_numpy(q.astype(np.complex128)).to(_cdt(precision)).cuda(),
                                                 L, alpha)
        p.sync()
    assert abs(nsum - ref) <= tol * abs(ref)
    assert abs(self_term - ewald.self_energy(q, alpha)) <= 1e-12 * abs(self_term)
    assert uk == nsum + self_term


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_madelung_fluorite_4_cells(precision, tol):
    Lc, alpha = 4, 1.0
    r, q, L = inputs.fluorite(Lc)
    N = (48, 48, 48)                         # |n_t| <= 24 covers exp(-pi^2 n^2/(alpha L)^2) > 1e-17
    rcut = 0.99 * L
    ur = ewald.real_space_energy(r, q, L, alpha, rcut)
    direct = ur + ewald.reciprocal_energy(r, q, L, alpha, nmax=24)
    with _plan(N, len(q), 8, precision) as p:
        p.set_points(torch.from_numpy(inputs.box_points(r, L)).cuda())
        uk, _, _ = p.ewald_reciprocal(torch.from_numpy(q.astype(np.complex128)).to(_cdt(precision)).cuda(), L, alpha)
        p.sync()
    mad = ewald.madelung(ur + uk, len(q), 3, 2, -1)
    mad_direct = ewald.madelung(direct, len(q), 3, 2, -1)
    assert abs(mad - mad_direct) <= tol * abs(mad_direct)
    assert abs(mad - _golden("madelung_fluorite.txt")) < 5e-5


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 2e-6)])
def test_madelung_fluorite_32_cells(precision, tol):
    # the paper's system: 32^3 cells, 393216 ions, N = 128^3, m = 6.  The
    # real-space energy per ion of a perfect crystal does not depend on the
    # supercell, so Eq. 11 is taken from the 4-cell crystal (cut-off below its
    # box length, erfc(0.6 * 9.1) ~ 1e-14).
    alpha = 0.6
    r4, q4, L4 = inputs.fluorite(4)
    ur_per_ion = ewald.real_space_energy(r4, q4, L4, alpha, 0.99 * L4) / len(q4)
    r2, q2, L2 = inputs.fluorite(2)
    direct = ewald.madelung(ewald.ewald_energy(r2, q2, L2, 1.5, min(7.0 / 1.5, 0.99 * L2),
                                               int(math.ceil(2.2 * 1.5 * L2))), len(q2), 3, 2, -1)
    r, q, L = inputs.fluorite(32)
    with _plan((128, 128, 128), len(q), 6, precision) as p:
        p.set_points(torch.from_numpy(inputs.box_points(r, L)).cuda())
        uk, _, _ = p.ewald_reciprocal(torch.from_numpy(q.astype(np.complex128)).to(_cdt(precision)).cuda(), L, alpha)
        p.sync()
    mad = ewald.madelung(ur_per_ion * len(q) + uk, len(q), 3, 2, -1)
    assert abs(mad - direct) <= tol * abs(direct)
    assert abs(mad - _golden("madelung_fluorite.txt")) < 5e-5


# ---- Eq. 11 on the GPU (nfft_ewald_real_space) -------------------------------
def _real_space(r, q, L, alpha, rcut):
    from paper_2001_01583_gb300 import ewald_real_space
    return ewald_real_space(torch.from_numpy(np.asarray(r, dtype=np.float64)).cuda(),
                            torch.from_numpy(np.asarray(q, dtype=np.float64)).cuda(), L, alpha, rcut)


def test_real_space_all_pairs_form_against_oracle():
    # L / rcut < 3: every pair and its 27 nearest images, FP64
    r, q, L = inputs.fluorite(4)
    alpha, rcut = 1.0, 0.99 * L
    ref = ewald.real_space_energy(r, q, L, alpha, rcut)
    got = _real_space(r, q, L, alpha, rcut)
    assert abs(got - ref) <= 1e-12 * abs(ref)
    assert _real_space(r, q, L, alpha, rcut) == got           # fixed-order reduction


def test_real_space_cell_list_on_a_supercell():
    # L / rcut >= 3: the cell list (FP32 pair terms).  A perfect crystal has
    # the same real-space energy per ion in any supercell, so the 8-cell
    # crystal's energy is 8 times the 4-cell one's (the cut-offs differ only
    # where erfc(alpha d) / d < 1e-17)
    r4, q4, L4 = inputs.fluorite(4)
    ref = 8 * ewald.real_space_energy(r4, q4, L4, 1.0, 0.99 * L4)
    r8, q8, L8 = inputs.fluorite(8)
    assert L8 / 6.0 >= 3
    got = _real_space(r8, q8, L8, 1.0, 6.0)
    assert abs(got - ref) <= 2e-6 * abs(ref)


def test_real_space_cell_list_random_ions_against_oracle():
    # random ions, coordinates outside [0, L) (reduced mod L), cell list;
    # the bar is relative to the sum of the terms' magnitudes (the oracle with
    # all charges positive), since a random configuration's energy cancels
    rng = np.random.default_rng(11)
    n, L, alpha, rcut = 1500, 20.0, 0.9, 6.5
    r = rng.uniform(0.0, L, size=(n, 3)) + L * rng.integers(-2, 3, size=(n, 3))
    q = rng.choice([-1.0, 1.0, 2.0], size=n)
    ref = ewald.real_space_energy(np.mod(r, L), q, L, alpha, rcut)
    scale = ewald.real_space_energy(np.mod(r, L), np.abs(q), L, alpha, rcut)
    got = _real_space(r, q, L, alpha, rcut)
    assert abs(got - ref) <= 1e-6 * scale


def test_madelung_fluorite_32_cells_all_on_gpu():
    # the paper's system with both parts of the Ewald energy from the GPU:
    # Eq. 11 by the cell list (alpha = 0.6, cut-off 10: erfc(6) ~ 2e-17),
    # Eq. 12 by the adjoint NFFT (N = 128^3, m = 6, FP64), Eq. 10 from both
    alpha = 0.6
    r2, q2, L2 = inputs.fluorite(2)
    direct = ewald.madelung(ewald.ewald_energy(r2, q2, L2, 1.5, min(7.0 / 1.5, 0.99 * L2),
                                               int(math.ceil(2.2 * 1.5 * L2))), len(q2), 3, 2, -1)
    r, q, L = inputs.fluorite(32)
    ur = _real_space(r, q, L, alpha, 10.0)
    with _plan((128, 128, 128), len(q), 6, "fp64") as p:
        p.set_points(torch.from_numpy(inputs.box_points(r, L)).cuda())
        uk, _, _ = p.ewald_reciprocal(torch.from_numpy(q.astype(np.complex128)).cuda(), L, alpha)
        p.sync()
    mad = ewald.madelung(ur + uk, len(q), 3, 2, -1)
    assert abs(mad - direct) <= 2e-6 * abs(direct)
    assert abs(mad - _golden("madelung_fluorite.txt")) < 5e-5


def test_real_space_argument_errors():
    from paper_2001_01583_gb300 import _lib
    r, q, L = inputs.fluorite(1)
    for alpha, rcut in ((0.0, 1.0), (1.0, 0.0), (1.0, L), (1.0, 2 * L)):
        with pytest.raises(_lib.NFFTError) as e:
            _real_space(r, q, L, alpha, rcut)
        assert e.value.status == _lib.ERR_INVALID_ARG
    assert _real_space(np.zeros((0, 3)), np.zeros(0), L, 1.0, 1.0) == 0.0
