"""GPU parity at the sizes of the paper's runtime sweeps.

  - Section 4, Fig. 13: NDFT matrices of 58^3, 80^3, 100^3 and 120^3
    nonequispaced points (the paper does not state N; N = 64^3 and 128^3
    here), 3-D, Kaiser-Bessel m = 4, sigma = 2, FP32: the adjoint at 48
    sampled frequencies and the forward at 48 sampled points against the
    direct NDFT (Eqs. 5, 6), relative l2 (Eq. 9) within the 1e-6 target.
  - Section 5, Fig. 16: fluorite crystals of 12 x {45, 56, 64}^3 ions
    (32^3 is in test_gpu_ewald.py), N = 128^3, m = 6: the n-sum of Eq. 12
    against the closed form of a perfect lattice over exactly I_N.
"""
import numpy as np
import pytest

from oracle import ndft
from paper_2001_01583_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("nside", [64, 128])
@pytest.mark.parametrize("side", [58, 80, 100, 120])
def test_fig13_sizes_against_direct_ndft(side, nside):
    from paper_2001_01583_gb300 import Plan
    N, M = (nside,) * 3, side ** 3
    x = inputs.uniform_points(M, 3, seed=1300 + side)
    f = inputs.complex_normal(M, seed=1301 + side, dtype=np.complex64)
    fh = inputs.complex_normal(N, seed=1302 + side, dtype=np.complex64)
    rng = np.random.default_rng(side * nside)
    ks = np.stack([rng.integers(-nside // 2, nside // 2, size=48) for _ in range(3)], axis=1)
    js = rng.choice(M, size=48, replace=False)
    with Plan(N, M, 2.0, 4, "kaiser_bessel", "fp32") as p:
        p.set_points(torch.from_numpy(x).cuda())
        a = p.adjoint(torch.from_numpy(f).cuda())     # N
        b = p.forward(torch.from_numpy(fh).cuda())    # (M,)
        p.sync()
        h = nside // 2
        got_a = a[ks[:, 0] + h, ks[:, 1] + h, ks[:, 2] + h].cpu().numpy()
        got_b = b.cpu().numpy()[js]
    ref_a = ndft.adjoint(x, f.astype(np.complex128), N, ksel=ks)
    ref_b = ndft.forward(x, fh.astype(np.complex128), N, jsel=js)
    assert ndft.rel_l2(got_a, ref_a) <= 1e-6
    assert ndft.rel_l2(got_b, ref_b) <= 1e-6


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-5)])
@pytest.mark.parametrize("lc", [45, 56, 64])
def test_fig16_fluorite_sizes_closed_form(lc, precision, tol):
    from paper_2001_01583_gb300 import Plan
    from test_gpu_ewald import _closed_form_sum
    from oracle import ewald
    alpha = 0.6
    r, q, L = inputs.fluorite(lc)
    x = inputs.box_points(r, L)
    N = (128, 128, 128)
    ref = _closed_form_sum(lc, N, L, alpha)
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    with Plan(N, len(q), 2.0, 6, "kaiser_bessel", precision) as p:
        p.set_points(torch.from_numpy(x).cuda())
        uk, nsum, self_term = p.ewald_reciprocal(torch.from_numpy(q.astype(np.complex128)).to(cdt).cuda(), L, alpha)
        p.sync()
    assert abs(nsum - ref) <= tol * abs(ref)
    assert abs(self_term - ewald.self_energy(q, alpha)) <= 1e-12 * abs(self_term)
