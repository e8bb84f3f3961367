"""GPU Ewald forces: the negative gradients of Eqs. 11 and 12 (Section 5).

The reciprocal part runs the adjoint NFFT of the charges, weights w(n) n_t on
I_N and a forward NFFT of three right-hand sides; it is compared ion by ion
with the oracle's direct sums over the same I_N (oracle/ewald.py,
reciprocal_forces, itself pinned by central differences of the oracle's
energy).  The real-space part is compared with the oracle's pair sum in both
of the library's forms (cell list with FP32 pair terms, all pairs in FP64).
The perfect fluorite crystal carries no force on any ion.
"""
import numpy as np
import pytest

from oracle import ewald
from paper_2001_01583_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _random_ions(n, L, seed):
    rng = np.random.default_rng(seed)
    r = rng.random((n, 3)) * L
    q = rng.choice([-1.0, 2.0], size=n)
    return r, q - q.mean()


def _recip_forces(r, q, L, alpha, N, m, precision):
    from paper_2001_01583_gb300 import Plan
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    with Plan(N, len(q), 2.0, m, "kaiser_bessel", precision) as p:
        p.set_points(torch.from_numpy(inputs.box_points(r, L)).cuda())
        F = p.ewald_reciprocal_forces(torch.from_numpy(q.astype(np.complex128)).to(cdt).cuda(), L, alpha)
        p.sync()
        return F.cpu().numpy()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-5)])
def test_reciprocal_forces_against_oracle(precision, tol):
    L, alpha, N = 9.0, 0.7, (24, 20, 16)
    r, q = _random_ions(400, L, seed=21)
    want = ewald.reciprocal_forces(r, q, L, alpha, N)
    got = _recip_forces(r, q, L, alpha, N, 6, precision)
    err = np.abs(got - want).max() / np.abs(want).max()
    print("%s reciprocal forces: max |dF| / max |F| = %.2e" % (precision, err))
    assert err <= tol
    assert np.all(np.abs(got.sum(axis=0)) <= 1e-6 * np.abs(got).sum())


@pytest.mark.parametrize("L,rc,tol", [(14.0, 3.5, 2e-5), (6.0, 2.5, 1e-12)])
def test_real_space_forces_against_oracle(L, rc, tol):
    # L / rc >= 3: the cell list (FP32 pair terms); smaller boxes: all pairs in FP64
    from paper_2001_01583_gb300 import ewald_real_space, ewald_real_space_forces
    alpha = 0.9
    r, q = _random_ions(1500 if L > 10 else 300, L, seed=22)
    want = ewald.real_space_forces(r, q, L, alpha, rc)
    F, e = ewald_real_space_forces(torch.from_numpy(r), torch.from_numpy(q), L, alpha, rc)
    got = F.cpu().numpy()
    err = np.abs(got - want).max() / np.abs(want).max()
    print("real-space forces (L / rc = %.1f): max |dF| / max |F| = %.2e" % (L / rc, err))
    assert err <= tol
    e0 = ewald_real_space(torch.from_numpy(r), torch.from_numpy(q), L, alpha, rc)
    assert abs(e - e0) <= 1e-6 * abs(e0)   # the same pair terms (FP32 in the cell list, contracted alike or not)


def test_perfect_fluorite_forces_vanish_and_a_displaced_ion_is_pulled_back():
    from paper_2001_01583_gb300 import ewald_real_space_forces
    r, q, L = inputs.fluorite(4)
    alpha, N = 0.9, (32, 32, 32)
    FK = _recip_forces(r, q, L, alpha, N, 6, "fp64")
    FR, _ = ewald_real_space_forces(torch.from_numpy(r), torch.from_numpy(q), L, alpha, 0.32 * L)
    scale = 4.0 * alpha ** 2
    assert np.abs(FK).max() <= 1e-8 * scale
    assert np.abs(FR.cpu().numpy()).max() <= 1e-5 * scale
    r2 = r.copy()
    r2[0, 2] += 0.05
    F2 = _recip_forces(r2, q, L, alpha, N, 6, "fp64")[0] + \
        ewald_real_space_forces(torch.from_numpy(r2), torch.from_numpy(q), L, alpha, 0.32 * L)[0].cpu().numpy()[0]
    assert F2[2] < 0
