"""GPU parity of batches: many independent transforms in one graph launch.

- heterogeneous items (d = 2 and 3, several N and M, Gaussian and
  Kaiser-Bessel, several right-hand sides) against the step-by-step FP64
  oracle element by element and against the direct NDFT;
- graph replay with new data pointers gives the same results as a fresh call;
- the batch workload at full size: 512 3-D transforms with N drawn from
  {32^3, 64^3} and M log-uniform in [1e3, 1e5], plus one 64^3 point set of
  M = 2e5 with 16 right-hand sides, Kaiser-Bessel m = 4, sigma = 2, FP32,
  against the direct NDFT at sampled frequencies / points of sampled items
  (relative l2 1e-6).
"""
import numpy as np
import pytest

from oracle import ndft, nfft_steps as S
from paper_2001_01583_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_ELEM = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _elementwise(got, ref, tol):
    got = np.asarray(got).ravel()
    ref = np.asarray(ref).ravel()
    err = np.max(np.abs(got - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2))
    assert err <= tol, "elementwise error %.3g > %.3g" % (err, tol)


ITEMS = [
    dict(N=(12, 10, 16), M=1500, window="kaiser_bessel", m=4, nrhs=2),
    dict(N=(16, 16, 16), M=2500, window="kaiser_bessel", m=4, nrhs=1),
    dict(N=(20, 14), M=900, window="gaussian", m=3, nrhs=3),
    dict(N=(12, 10, 16), M=0, window="kaiser_bessel", m=4, nrhs=1),
    dict(N=(8, 8, 8), M=700, window="gaussian", m=2, nrhs=1),
    dict(N=(16, 16, 16), M=4000, window="kaiser_bessel", m=4, nrhs=1),
]
WIN = {"gaussian": S.GAUSSIAN, "kaiser_bessel": S.KAISER_BESSEL}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", FP32_ELEM)])
def test_heterogeneous_batch_against_oracles(precision, tol):
    from paper_2001_01583_gb300 import Batch
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    xs, fs, hs = [], [], []
    for i, it in enumerate(ITEMS):
        d = len(it["N"])
        xs.append(inputs.uniform_points(it["M"], d, seed=100 + i))
        fs.append(inputs.complex_normal((it["nrhs"], it["M"]), seed=200 + i))
        hs.append(inputs.complex_normal((it["nrhs"],) + it["N"], seed=300 + i))
    with Batch(ITEMS, precision) as b:
        b.set_points([torch.from_numpy(x).cuda() for x in xs])
        A = b.adjoint([torch.from_numpy(f).to(cdt).cuda() for f in fs])
        B = b.forward([torch.from_numpy(h).to(cdt).cuda() for h in hs])
        b.sync()
        A = [a.cpu().numpy().astype(np.complex128) for a in A]
        B = [v.cpu().numpy().astype(np.complex128) for v in B]
    for i, it in enumerate(ITEMS):
        for r in range(it["nrhs"]):
            if it["M"] == 0:
                assert np.count_nonzero(A[i][r]) == 0
                continue
            sa = S.adjoint(xs[i], fs[i][r], it["N"], 2.0, it["m"], WIN[it["window"]])
            sb = S.forward(xs[i], hs[i][r], it["N"], 2.0, it["m"], WIN[it["window"]])
            _elementwise(A[i][r], sa, tol)
            _elementwise(B[i][r], sb, tol)
            ea = ndft.rel_l2(sa, ndft.adjoint(xs[i], fs[i][r], it["N"]))
            assert ndft.rel_l2(A[i][r], ndft.adjoint(xs[i], fs[i][r], it["N"])) <= ea * 1.01 + (
                1e-13 if precision == "fp64" else 1e-6)


def test_graph_replay_with_new_pointers():
    from paper_2001_01583_gb300 import Batch
    items = ITEMS[:3]
    xs = [torch.from_numpy(inputs.uniform_points(it["M"], len(it["N"]), seed=10 + i)).cuda()
          for i, it in enumerate(items)]
    f1 = [torch.from_numpy(inputs.complex_normal((it["nrhs"], it["M"]), seed=20 + i, dtype=np.complex64)).cuda()
          for i, it in enumerate(items)]
    f2 = [torch.from_numpy(inputs.complex_normal((it["nrhs"], it["M"]), seed=30 + i, dtype=np.complex64)).cuda()
          for i, it in enumerate(items)]
    with Batch(items, "fp32") as b:
        b.set_points(xs)
        a1 = [a.clone() for a in b.adjoint(f1)]
        a2 = [a.clone() for a in b.adjoint(f2)]
        a1_again = [a.clone() for a in b.adjoint(f1)]
        b.sync()
    with Batch(items, "fp32") as b2:
        b2.set_points(xs)
        fresh = b2.adjoint(f2)
        b2.sync()
    for u, v, w, z in zip(a1, a1_again, a2, fresh):
        assert torch.allclose(u, v, rtol=0, atol=1e-4 * u.abs().max().item())
        assert torch.allclose(w, z, rtol=0, atol=1e-4 * w.abs().max().item())


def test_full_size_batch_workload_sampled():
    from paper_2001_01583_gb300 import Batch
    items = inputs.batch_items(512, N_choices=(32, 64), M_lo=1000, M_hi=100000, d=3, seed=0)
    items = [dict(N=it["N"], M=it["M"], nrhs=1, seed=it["seed"]) for it in items]
    items.append(dict(N=(64, 64, 64), M=200000, nrhs=16, seed=9999))
    xs_np = [inputs.uniform_points(it["M"], 3, seed=it["seed"]) for it in items]
    fs_np = [inputs.complex_normal((it["nrhs"], it["M"]), seed=it["seed"] + 1, dtype=np.complex64) for it in items]
    with Batch([dict(N=it["N"], M=it["M"], nrhs=it["nrhs"]) for it in items], "fp32") as b:
        b.set_points([torch.from_numpy(x).cuda() for x in xs_np])
        A = b.adjoint([torch.from_numpy(f).cuda() for f in fs_np])
        hs = [torch.from_numpy(inputs.complex_normal((it["nrhs"],) + it["N"], seed=it["seed"] + 2,
                                                     dtype=np.complex64)).cuda() for it in items]
        B = b.forward(hs)
        b.sync()
    rng = np.random.default_rng(5)
    check = list(rng.choice(512, size=24, replace=False)) + [512]
    for i in check:
        it = items[i]
        N = it["N"]
        ks = np.stack([rng.integers(-N[0] // 2, N[0] // 2, size=24) for _ in range(3)], axis=1)
        js = rng.integers(0, it["M"], size=24)
        for r in ([0, 7, 15] if it["nrhs"] > 1 else [0]):
            f = fs_np[i][r].astype(np.complex128)
            ref = ndft.adjoint(xs_np[i], f, N, ksel=ks)
            got = A[i][r].cpu().numpy()[ks[:, 0] + N[0] // 2, ks[:, 1] + N[1] // 2, ks[:, 2] + N[2] // 2]
            assert ndft.rel_l2(got, ref) <= 1e-6, (i, r)
            h = hs[i][r].cpu().numpy().astype(np.complex128)
            refb = ndft.forward(xs_np[i], h, N, jsel=js)
            assert ndft.rel_l2(B[i][r].cpu().numpy()[js], refb) <= 1e-6, (i, r)


def test_autotuner_keeps_parity():
    from paper_2001_01583_gb300 import Batch, Plan
    N, M = (16, 16, 16), 30000
    x = inputs.clustered_points(M, 3, 8, 0.03, seed=61)
    f = inputs.complex_normal(M, seed=62)
    fh = inputs.complex_normal(N, seed=63)
    with Plan(N, M, 2.0, 4, "kaiser_bessel", "fp32") as p:
        p.set_points(torch.from_numpy(x).cuda())
        ms = p.autotune(reps=2)
        info = p.info()
        a = p.adjoint(torch.from_numpy(f).to(torch.complex64).cuda())
        b = p.forward(torch.from_numpy(fh).to(torch.complex64).cuda())
        p.sync()
    assert ms > 0.0
    assert info["max_subproblem"] in (256, 1024)
    _elementwise(a.cpu().numpy(), S.adjoint(x, f, N, 2.0, 4, S.KAISER_BESSEL), FP32_ELEM)
    _elementwise(b.cpu().numpy(), S.forward(x, fh, N, 2.0, 4, S.KAISER_BESSEL), FP32_ELEM)
    items = ITEMS[:2]
    xs = [inputs.uniform_points(it["M"], len(it["N"]), seed=70 + i) for i, it in enumerate(items)]
    fs = [inputs.complex_normal((it["nrhs"], it["M"]), seed=80 + i) for i, it in enumerate(items)]
    with Batch(items, "fp64") as bt:
        bt.set_points([torch.from_numpy(v).cuda() for v in xs])
        assert bt.autotune(reps=2) > 0.0
        A = bt.adjoint([torch.from_numpy(v).cuda() for v in fs])
        bt.sync()
    for i, it in enumerate(items):
        for r in range(it["nrhs"]):
            _elementwise(A[i][r].cpu().numpy(), S.adjoint(xs[i], fs[i][r], it["N"], 2.0, it["m"], WIN[it["window"]]),
                         1e-12)
