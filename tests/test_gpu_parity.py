"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Two oracles, two bars:
  - the direct NDFT (Eqs. 5, 6): relative l2 error (Eq. 9) within the window
    error stated per configuration;
  - the step-by-step gridding NFFT in FP64 (same window, same n, same taps):
    element by element, max |gpu - oracle| / rms(oracle) <= 1e-12 for the FP64
    path and <= FP32_ELEM for the mixed path, which pins the kernels
    themselves, not just the method.
FP32_ELEM: the mixed path rounds window weights (about 1e-7 relative each) and
sums up to K contributions per grid cell in FP32, whose rounding grows like
sqrt(K) * 6e-8 relative to a cell; with strongly clustered points (K in the
thousands) the largest single output deviates by a few 1e-6 of the rms while
the relative l2 error stays below 5e-7.
Sizes span several bins and a ragged last bin; edge cases cover empty and
tiny inputs, points on cell boundaries and outside [-1/2, 1/2), lattice
points on grid nodes, and the error statuses.
"""
import numpy as np
import pytest

from oracle import ndft, nfft_steps as S
from paper_2001_01583_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WIN = {"gaussian": S.GAUSSIAN, "kaiser_bessel": S.KAISER_BESSEL, "b_spline": S.B_SPLINE, "sinc_power": S.SINC_POWER}
FP32_ELEM = 1e-5
FP32_L2 = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _plan(N, M, sigma, m, window, precision, **opts):
    from paper_2001_01583_gb300 import Plan, _lib
    p = Plan(N, M, sigma, m, window, precision)
    for k, v in opts.items():
        p.set_option(getattr(_lib, "OPT_" + k.upper()), v)
    return p


def _cdt(precision):
    return torch.complex128 if precision == "fp64" else torch.complex64


def _run(N, x, f, fh, sigma, m, window, precision, **opts):
    M = x.shape[0]
    with _plan(N, M, sigma, m, window, precision, **opts) as p:
        p.set_points(torch.from_numpy(x).cuda())
        a = p.adjoint(torch.from_numpy(f).to(_cdt(precision)).cuda())
        b = p.forward(torch.from_numpy(fh).to(_cdt(precision)).cuda())
        p.sync()
        return a.cpu().numpy().astype(np.complex128), b.cpu().numpy().astype(np.complex128), p.info()


def _elementwise(got, ref, tol):
    """max |got - ref| <= tol * rms(ref), element by element."""
    got = np.asarray(got).ravel()
    ref = np.asarray(ref).ravel()
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    err = np.max(np.abs(got - ref)) / scale
    assert err <= tol, "elementwise error %.3g > %.3g" % (err, tol)


# ---- the 1-D plain FP64 configuration: N = 256, M = 1024, sigma = 2 ----------
@pytest.mark.parametrize("window,m,tol", [("gaussian", 6, 2e-6), ("kaiser_bessel", 12, 1e-12),
                                          ("gaussian", 12, 5e-12), ("kaiser_bessel", 6, 1e-10)])
def test_1d_fp64_against_direct_ndft(window, m, tol):
    N, M = (256,), 1024
    rng = np.random.default_rng(0)
    x = rng.random((M, 1)) - 0.5
    f = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    fh = inputs.complex_normal(N, seed=1)
    a, b, info = _run(N, x, f, fh, 2.0, m, window, "fp64")
    assert info["n"] == (512,)
    assert ndft.rel_l2(a, ndft.adjoint(x, f, N)) <= tol
    assert ndft.rel_l2(b, ndft.forward(x, fh, N)) <= tol
    # the kernels reproduce the FP64 gridding method to rounding
    _elementwise(a, S.adjoint(x, f, N, 2.0, m, WIN[window]), 1e-12)
    _elementwise(b, S.forward(x, fh, N, 2.0, m, WIN[window]), 1e-12)


# ---- multi-dimensional, several bins with ragged last bins -------------------
CASES = [
    # d, N, M, window, m
    (1, (200,), 3001, "kaiser_bessel", 5),
    (2, (44, 36), 4000, "gaussian", 3),
    (2, (40, 30), 2500, "kaiser_bessel", 4),
    (3, (22, 18, 16), 5000, "kaiser_bessel", 4),
    (3, (20, 14, 12), 3000, "gaussian", 2),
    (1, (160,), 2000, "b_spline", 5),
    (2, (36, 28), 2500, "sinc_power", 4),
    (3, (18, 16, 14), 3000, "b_spline", 3),
    (3, (16, 20, 12), 2500, "sinc_power", 4),
]


@pytest.mark.parametrize("d,N,M,window,m", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("method", ["tiled", "global", "warp", "grid_warp"])
def test_against_oracles(d, N, M, window, m, precision, method):
    if method == "warp" and d == 1:
        pytest.skip("the warp-per-point kernels cover d = 2, 3")
    if window == "b_spline" and method != "global":
        pytest.skip("B-spline windows run on the global kernels")
    x = inputs.uniform_points(M, d, seed=5 + d)
    f = inputs.complex_normal(M, seed=6)
    fh = inputs.complex_normal(N, seed=7)
    meth = {"tiled": 1, "global": 2, "warp": 3, "grid_warp": 4}[method]
    a, b, info = _run(N, x, f, fh, 2.0, m, window, precision, method=meth)
    assert info["method"] == meth
    sa = S.adjoint(x, f, N, 2.0, m, WIN[window])
    sb = S.forward(x, fh, N, 2.0, m, WIN[window])
    tol = 1e-12 if precision == "fp64" else FP32_ELEM
    _elementwise(a, sa, tol)
    _elementwise(b, sb, tol)
    if precision == "fp32":
        assert ndft.rel_l2(a, sa) <= FP32_L2 and ndft.rel_l2(b, sb) <= FP32_L2
    # against the exact sums: the method's own error plus rounding
    ea = ndft.rel_l2(sa, ndft.adjoint(x, f, N))
    eb = ndft.rel_l2(sb, ndft.forward(x, fh, N))
    slack = 1e-13 if precision == "fp64" else 1e-6
    assert ndft.rel_l2(a, ndft.adjoint(x, f, N)) <= ea * 1.01 + slack
    assert ndft.rel_l2(b, ndft.forward(x, fh, N)) <= eb * 1.01 + slack


# ---- the precision study of Section 4 (Fig. 12) -----------------------------
def test_precision_against_cut_off_fig12():
    """3-D, N = 16^3, M = 4096, sigma = 2, the four windows, m = 1 .. 12,
    FP64: the relative l2 error (Eq. 9) of the adjoint and the forward
    transform against the direct NDFT, for every window and m; each equals
    the FP64 oracle NFFT's error (checked up to m = 3, where the oracle is
    quick), and every window's error falls with m to the FP64 floor."""
    from paper_2001_01583_gb300 import Plan
    N, M = (16, 16, 16), 4096
    x = inputs.uniform_points(M, 3, seed=12)
    f = inputs.complex_normal(M, seed=13)
    fh = inputs.complex_normal(N, seed=14)
    exact_a, exact_f = ndft.adjoint(x, f, N), ndft.forward(x, fh, N)
    xd = torch.from_numpy(x).cuda()
    table = {}
    for window in ("gaussian", "b_spline", "sinc_power", "kaiser_bessel"):
        for m in range(1, 13):
            with Plan(N, M, 2.0, m, window, "fp64") as p:
                p.set_points(xd)
                a = p.adjoint(torch.from_numpy(f).cuda()).cpu().numpy()
                b = p.forward(torch.from_numpy(fh).cuda()).cpu().numpy()
            ea, ef = ndft.rel_l2(a, exact_a), ndft.rel_l2(b, exact_f)
            table[window, m] = (ea, ef)
            if m <= 3:
                oa = ndft.rel_l2(S.adjoint(x, f, N, 2.0, m, WIN[window]), exact_a)
                assert abs(ea - oa) <= 1e-3 * oa + 1e-13, (window, m, ea, oa)
    for window in ("gaussian", "b_spline", "sinc_power", "kaiser_bessel"):
        print(window, " ".join("%.1e" % table[window, m][0] for m in range(1, 13)))
        errs = [table[window, m][0] for m in range(1, 13)]
        floor = 1e-13
        for e0, e1 in zip(errs, errs[1:]):
            assert e1 < e0 or e1 < floor, (window, errs)
        assert errs[-1] < 1e-9
        # forward and adjoint errors are of the same size (the paper's (a) and (b))
        for m in range(1, 13):
            ea, ef = table[window, m]
            assert ef < 10 * ea + 1e-13 and ea < 10 * ef + 1e-13


# ---- wide windows: the 3-D shared-tile kernels up to 26 taps ----------------
WIDE = [
    # N, M, window, m, precision, clustered (taps: Kaiser-Bessel 2m, Gaussian 2m + 2)
    ((36, 30, 28), 3000, "kaiser_bessel", 9, "fp32", False),    # 18 taps
    ((30, 36, 28), 2500, "gaussian", 9, "fp32", False),         # 20
    ((32, 28, 30), 1200, "gaussian", 10, "fp32", False),        # 22
    ((32, 32, 28), 1000, "kaiser_bessel", 12, "fp32", False),   # 24
    ((30, 32, 34), 800, "gaussian", 12, "fp32", False),         # 26
    ((32, 32, 32), 4000, "kaiser_bessel", 9, "fp32", True),     # 18, dense clusters
    ((28, 30, 26), 1500, "kaiser_bessel", 9, "fp64", False),    # 18
    ((30, 28, 26), 1500, "gaussian", 9, "fp64", False),         # 20
]
# FP64 tiles of 22 to 26 taps do not fit shared memory: those windows run on
# the grid-warp kernels (a warp per point, vector atomics along grid rows)
WIDE_FP64_OTHER = [((26, 28, 24), 600, "kaiser_bessel", 11), ((24, 26, 28), 500, "kaiser_bessel", 12),
                   ((28, 24, 26), 400, "gaussian", 12)]


def _amplification(N, n, m, window):
    """Per-frequency factor c_0 / c_k of the deconvolution (Section 2) on
    I_N (C order) and its rms: rounding on the grid reaches the adjoint's
    output multiplied by it, and the forward's input is multiplied by it
    before the FFT.  It grows with m (about 3 per dimension at the edge of
    I_N for m = 4, 11 for m = 9, 25 for m = 12)."""
    w = [np.abs(v) for v in S.scaling_weights(WIN[window], m, list(N), list(n))]
    amp = np.ones(())
    for wt in w:
        amp = np.multiply.outer(amp, wt.max() / wt)
    return amp, float(np.sqrt(np.mean(amp ** 2)))


@pytest.mark.parametrize("N,M,window,m,precision,clustered", WIDE)
def test_wide_windows_3d(N, M, window, m, precision, clustered):
    if clustered:
        x = inputs.clustered_points(M, 3, 4, 0.03, seed=31)
    else:
        x = inputs.uniform_points(M, 3, seed=32)
    f = inputs.complex_normal(M, seed=33)
    fh = inputs.complex_normal(N, seed=34)
    a, b, info = _run(N, x, f, fh, 2.0, m, window, precision)
    assert info["method"] == 3
    sa = S.adjoint(x, f, N, 2.0, m, WIN[window])
    sb = S.forward(x, fh, N, 2.0, m, WIN[window])
    if precision == "fp64":
        _elementwise(a, sa, 1e-12)
        _elementwise(b, sb, 1e-12)
        return
    # FP32: grid-stage rounding is scaled by c_0 / c_k; compare the adjoint
    # with that factor taken out, and the forward against the bar times the
    # factor's rms
    amp, amp_rms = _amplification(N, info["n"], m, window)
    err_a = np.max(np.abs(a - sa) / amp) / np.sqrt(np.mean(np.abs(sa) ** 2))
    assert err_a <= FP32_ELEM, err_a
    _elementwise(b, sb, FP32_ELEM * amp_rms)
    assert ndft.rel_l2(a, sa) <= FP32_L2 * amp_rms and ndft.rel_l2(b, sb) <= FP32_L2 * amp_rms


# ---- plane-owner spreading with more warps than divide the taps -------------
@pytest.mark.parametrize("m,warps,precision", [(3, 4, "fp64"), (5, 4, "fp64"), (5, 8, "fp64"), (7, 4, "fp64"),
                                               (6, 8, "fp32"), (7, 8, "fp32"), (9, 8, "fp32")])
def test_plane_spread_uneven_warps(m, warps, precision):
    N, M = (24, 20, 26), 2500
    x = inputs.clustered_points(M, 3, 6, 0.05, seed=81)
    f = inputs.complex_normal(M, seed=82)
    fh = inputs.complex_normal(N, seed=83)
    a, b, info = _run(N, x, f, fh, 2.0, m, "kaiser_bessel", precision, method=3, spread_threads=32 * warps)
    assert info["method"] == 3 and info["spread_threads"] == 32 * warps
    sa = S.adjoint(x, f, N, 2.0, m, S.KAISER_BESSEL)
    if precision == "fp64":
        _elementwise(a, sa, 1e-12)
    else:
        amp, _ = _amplification(N, info["n"], m, "kaiser_bessel")
        assert np.max(np.abs(a - sa) / amp) / np.sqrt(np.mean(np.abs(sa) ** 2)) <= FP32_ELEM


# ---- every block size of the timed plane kernels -----------------------------
# The bench's autotuner picks the threads per block of the spreading and the
# interpolation kernel (32 x warps) among these; the 3-D configuration runs
# 8 taps (Kaiser-Bessel m = 4), the largest one 6 (m = 3).  Each instantiation
# is pinned element by element, uniform and clustered, and info() must report
# the block size that ran.
@pytest.mark.parametrize("m,threads", [(4, 32), (4, 64), (4, 128), (4, 256), (3, 32), (3, 64), (3, 128)])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_plane_kernels_at_every_block_size(m, threads, precision):
    N, M = (40, 36, 32), 30000
    x = np.concatenate([inputs.clustered_points(M // 2, 3, 8, 0.02, seed=121),
                        inputs.uniform_points(M - M // 2, 3, seed=122)])
    f = inputs.complex_normal(M, seed=123)
    fh = inputs.complex_normal(N, seed=124)
    a, b, info = _run(N, x, f, fh, 2.0, m, "kaiser_bessel", precision, method=3, spread_threads=threads,
                      interp_threads=threads)
    assert info["method"] == 3 and info["taps"] == 2 * m
    assert info["spread_block_threads"] == threads and info["interp_block_threads"] == threads
    sa = S.adjoint(x, f, N, 2.0, m, S.KAISER_BESSEL)
    sb = S.forward(x, fh, N, 2.0, m, S.KAISER_BESSEL)
    tol = 1e-12 if precision == "fp64" else FP32_ELEM
    _elementwise(a, sa, tol)
    _elementwise(b, sb, tol)
    if precision == "fp32":
        assert ndft.rel_l2(a, sa) <= FP32_L2 and ndft.rel_l2(b, sb) <= FP32_L2


# ---- sparse subproblems on the grid-warp kernels, dense ones on tiles --------
@pytest.mark.parametrize("N,M,window,m", [((40, 36, 32), 3000, "kaiser_bessel", 4), ((30, 28, 34), 2000, "gaussian", 6),
                                          ((96, 80), 3000, "kaiser_bessel", 5), ((2000,), 3000, "gaussian", 3),
                                          ((32, 30, 28), 1500, "kaiser_bessel", 10)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sparse_and_dense_subproblems_mixed(N, M, window, m, precision):
    d = len(N)
    # dense clusters plus a uniform sprinkle: bins of both kinds in one set
    x = np.concatenate([inputs.clustered_points(M - M // 4, d, 3, 0.02, seed=91),
                        inputs.uniform_points(M // 4, d, seed=92)])
    f = inputs.complex_normal(M, seed=93)
    fh = inputs.complex_normal(N, seed=94)
    a, b, info = _run(N, x, f, fh, 2.0, m, window, precision, sparse_points=40, sparse_points_interp=60,
                      max_subproblem=256)
    assert info["sparse_points"] == 40 and info["sparse_points_interp"] == 60
    sa = S.adjoint(x, f, N, 2.0, m, WIN[window])
    sb = S.forward(x, fh, N, 2.0, m, WIN[window])
    if precision == "fp64":
        _elementwise(a, sa, 1e-12)
        _elementwise(b, sb, 1e-12)
    else:
        amp, amp_rms = _amplification(N, info["n"], m, window)
        err_a = np.max(np.abs(a - sa) / amp) / np.sqrt(np.mean(np.abs(sa) ** 2))
        assert err_a <= FP32_ELEM, err_a
        _elementwise(b, sb, FP32_ELEM * amp_rms)


@pytest.mark.parametrize("N,M,window,m", WIDE_FP64_OTHER)
def test_wide_windows_fp64_without_plane_kernels(N, M, window, m):
    x = inputs.uniform_points(M, 3, seed=35)
    f = inputs.complex_normal(M, seed=36)
    fh = inputs.complex_normal(N, seed=37)
    a, b, info = _run(N, x, f, fh, 2.0, m, window, "fp64")
    # the thread-per-point tiled kernel where an FP64 tile still fits, else
    # the grid-warp kernels; never the global-atomic thread-per-point kernel
    assert info["method"] in (1, 4)
    _elementwise(a, S.adjoint(x, f, N, 2.0, m, WIN[window]), 1e-12)
    _elementwise(b, S.forward(x, fh, N, 2.0, m, WIN[window]), 1e-12)


# ---- 3-D owner spreading of sparse bins (no atomics) -------------------------
@pytest.mark.parametrize("N,M,window,m,precision,R", [
    ((40, 36, 32), 2000, "kaiser_bessel", 4, "fp64", 1),
    ((40, 36, 32), 2000, "kaiser_bessel", 4, "fp32", 1),
    ((30, 26, 22), 1500, "gaussian", 3, "fp64", 3),      # ragged last bins, 3 right-hand sides
    ((36, 34, 40), 1200, "kaiser_bessel", 9, "fp32", 1),  # 18 taps
    ((32, 30, 34), 800, "gaussian", 12, "fp32", 1),       # 26 taps, small bins
])
@pytest.mark.parametrize("owner", [1, 0])
def test_owner_spread_of_sparse_bins(N, M, window, m, precision, R, owner):
    x = inputs.clustered_points(M, 3, 5, 0.08, seed=101)
    f = inputs.complex_normal((R, M), seed=102)
    fh = inputs.complex_normal(N, seed=103)
    from paper_2001_01583_gb300 import Plan, _lib
    with Plan(N, M, 2.0, m, window, precision) as p:
        p.set_option(_lib.OPT_SPARSE_POINTS, 1 << 20)   # every bin sparse
        p.set_option(_lib.OPT_OWNER_SPREAD, owner)
        p.set_points(torch.from_numpy(x).cuda())
        a = p.adjoint(torch.from_numpy(f).to(_cdt(precision)).cuda()).cpu().numpy().astype(np.complex128)
        info = p.info()
    assert info["owner_spread"] == owner
    for r in range(R):
        sa = S.adjoint(x, f[r], N, 2.0, m, WIN[window])
        if precision == "fp64":
            _elementwise(a[r], sa, 1e-12)
        else:
            amp, _ = _amplification(N, info["n"], m, window)
            assert np.max(np.abs(a[r] - sa) / amp) / np.sqrt(np.mean(np.abs(sa) ** 2)) <= FP32_ELEM


def test_owner_spread_in_a_batch_with_ineligible_items():
    """Items whose grid is too small for the owner kernel (n_t < bin_t + W - 1)
    keep the grid-warp path; both kinds share FFT classes and one graph."""
    from paper_2001_01583_gb300 import Batch
    items = [dict(N=(40, 36, 32), M=900, m=4), dict(N=(8, 8, 8), M=300, m=4), dict(N=(40, 36, 32), M=0, m=4),
             dict(N=(24, 20, 28), M=2500, m=3, nrhs=2)]
    xs = [inputs.uniform_points(it["M"], 3, seed=110 + i) for i, it in enumerate(items)]
    fs = [inputs.complex_normal((it.get("nrhs", 1), it["M"]), seed=120 + i) for i, it in enumerate(items)]
    from paper_2001_01583_gb300 import _lib
    with Batch(items, "fp64") as bt:
        bt.set_option(_lib.OPT_OWNER_SPREAD, 1)
        bt.set_points([torch.from_numpy(v).cuda() for v in xs])
        for _ in range(2):   # replay the graph: no stale grid contents
            A = bt.adjoint([torch.from_numpy(v).cuda() for v in fs])
        bt.sync()
    for i, it in enumerate(items):
        for r in range(it.get("nrhs", 1)):
            got = A[i][r].cpu().numpy()
            if it["M"] == 0:
                assert np.count_nonzero(got) == 0
                continue
            _elementwise(got, S.adjoint(xs[i], fs[i][r], it["N"], 2.0, it["m"], S.KAISER_BESSEL), 1e-12)


# ---- rows longer than one scaling segment (4096 elements) --------------------
@pytest.mark.parametrize("N,M", [((20000,), 3000), ((8, 5000), 2000)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_long_rows(N, M, precision):
    d = len(N)
    x = inputs.uniform_points(M, d, seed=41)
    f = inputs.complex_normal(M, seed=42)
    fh = inputs.complex_normal(N, seed=43)
    a, b, info = _run(N, x, f, fh, 2.0, 3, "kaiser_bessel", precision)
    assert info["n"][-1] > 2 * 4096
    tol = 1e-12 if precision == "fp64" else FP32_ELEM
    _elementwise(a, S.adjoint(x, f, N, 2.0, 3, S.KAISER_BESSEL), tol)
    _elementwise(b, S.forward(x, fh, N, 2.0, 3, S.KAISER_BESSEL), tol)


def test_long_rows_in_a_batch():
    from paper_2001_01583_gb300 import Batch
    items = [dict(N=(9000,), M=500, m=3), dict(N=(16, 16, 16), M=800, m=3), dict(N=(6, 9000), M=700, m=3)]
    xs = [inputs.uniform_points(it["M"], len(it["N"]), seed=50 + i) for i, it in enumerate(items)]
    fs = [inputs.complex_normal((1, it["M"]), seed=60 + i) for i, it in enumerate(items)]
    hs = [inputs.complex_normal((1,) + it["N"], seed=70 + i) for i, it in enumerate(items)]
    with Batch(items, "fp64") as bt:
        bt.set_points([torch.from_numpy(v).cuda() for v in xs])
        A = bt.adjoint([torch.from_numpy(v).cuda() for v in fs])
        B = bt.forward([torch.from_numpy(v).cuda() for v in hs])
        bt.sync()
    for i, it in enumerate(items):
        _elementwise(A[i][0].cpu().numpy(), S.adjoint(xs[i], fs[i][0], it["N"], 2.0, 3, S.KAISER_BESSEL), 1e-12)
        _elementwise(B[i][0].cpu().numpy(), S.forward(xs[i], hs[i][0], it["N"], 2.0, 3, S.KAISER_BESSEL), 1e-12)


def test_3d_config_accuracy_target_small():
    # the 3-D target: Kaiser-Bessel m = 4, sigma = 2, rel-l2 1e-6 in FP32
    N, M = (32, 32, 32), 20000
    x = inputs.uniform_points(M, 3, seed=21)
    f = inputs.complex_normal(M, seed=22)
    fh = inputs.complex_normal(N, seed=23)
    for precision in ("fp32", "fp64"):
        a, b, _ = _run(N, x, f, fh, 2.0, 4, "kaiser_bessel", precision)
        assert ndft.rel_l2(a, ndft.adjoint(x, f, N)) <= 1e-6
        assert ndft.rel_l2(b, ndft.forward(x, fh, N)) <= 1e-6


def test_clustered_points_split_into_subproblems():
    N, M = (24, 24, 24), 30000
    x = inputs.clustered_points(M, 3, 4, 0.01, seed=31)
    f = inputs.complex_normal(M, seed=32)
    fh = inputs.complex_normal(N, seed=33)
    sa = S.adjoint(x, f, N, 2.0, 4, S.KAISER_BESSEL)
    sb = S.forward(x, fh, N, 2.0, 4, S.KAISER_BESSEL)
    for P, method in ((64, 3), (1024, 3), (64, 1)):
        for precision, tol in (("fp32", FP32_ELEM), ("fp64", 1e-12)):
            a, b, _ = _run(N, x, f, fh, 2.0, 4, "kaiser_bessel", precision, max_subproblem=P, method=method)
            _elementwise(a, sa, tol)
            _elementwise(b, sb, tol)
            assert ndft.rel_l2(a, ndft.adjoint(x, f, N)) <= 1e-6
            assert ndft.rel_l2(b, ndft.forward(x, fh, N)) <= 1e-6


@pytest.mark.parametrize("method", [1, 2, 3])
def test_multiple_right_hand_sides(method):
    N, M, R = (16, 20, 12), 3000, 5
    x = inputs.uniform_points(M, 3, seed=41)
    F = inputs.complex_normal((R, M), seed=42)
    H = inputs.complex_normal((R,) + N, seed=43)
    with _plan(N, M, 2.0, 4, "kaiser_bessel", "fp64", rhs_capacity=4, method=method) as p:
        p.set_points(torch.from_numpy(x).cuda())
        A = p.adjoint(torch.from_numpy(F).cuda()).cpu().numpy()
        B = p.forward(torch.from_numpy(H).cuda()).cpu().numpy()
        p.sync()
    for r in range(R):
        _elementwise(A[r], S.adjoint(x, F[r], N, 2.0, 4, S.KAISER_BESSEL), 1e-12)
        _elementwise(B[r], S.forward(x, H[r], N, 2.0, 4, S.KAISER_BESSEL), 1e-12)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_adjoint_identity_on_gpu(precision, tol):
    N, M = (18, 16, 14), 4000
    x = inputs.uniform_points(M, 3, seed=51)
    f = inputs.complex_normal(M, seed=52)
    g = inputs.complex_normal(N, seed=53)
    a, b, _ = _run(N, x, f, g, 2.0, 4, "kaiser_bessel", precision)
    lhs = np.vdot(b, f)      # <A^H g, f>
    rhs = np.vdot(g, a)      # <g, A f>
    assert abs(lhs - rhs) <= tol * abs(lhs)


# ---- edge cases ---------------------------------------------------------------
def test_empty_point_set():
    N = (8, 8)
    with _plan(N, 0, 2.0, 3, "kaiser_bessel", "fp64") as p:
        p.set_points(torch.zeros((0, 2), dtype=torch.float64, device="cuda"))
        a = p.adjoint(torch.zeros((0,), dtype=torch.complex128, device="cuda"))
        b = p.forward(torch.ones(N, dtype=torch.complex128, device="cuda"))
        p.sync()
    assert torch.count_nonzero(a).item() == 0
    assert b.numel() == 0


def test_single_point_and_boundaries():
    """Points on cell boundaries (n x_t an integer) and outside [-1/2, 1/2).
    At such a tie the kernels may take the cell below with offset 1 where the
    oracle takes offset 0: the same position, a tap set one cell lower.  The
    bar that does not depend on that choice is the direct NDFT at the
    window's error.  The Kaiser-Bessel window vanishes at |u| = m, so both
    tap sets give the same sum to rounding (pinned in
    test_oracle_nfft_steps.py), and the element-wise oracle bar holds too."""
    N = (16, 12, 10)
    pts = np.array([[-0.5, -0.5, -0.5], [0.5, 0.5, 0.5], [0.49999999999, -0.25, 0.0], [3.75, -7.125, 12.5]])
    f = np.array([1.0 + 0.0j, 0.5 - 2j, -1j, 2.0])
    fh = inputs.complex_normal(N, seed=61)
    for precision, tol in (("fp64", 1e-12), ("fp32", FP32_ELEM)):
        a, b, _ = _run(N, pts, f, fh, 2.0, 5, "kaiser_bessel", precision)
        # Kaiser-Bessel m = 5 is accurate to about 1e-9, so FP32 rounding sets the bar
        bar = 1e-8 if precision == "fp64" else FP32_L2
        assert ndft.rel_l2(a, ndft.adjoint(pts, f, N)) <= bar
        assert ndft.rel_l2(b, ndft.forward(pts, fh, N)) <= bar
        _elementwise(a, S.adjoint(pts, f, N, 2.0, 5, S.KAISER_BESSEL), tol)
        _elementwise(b, S.forward(pts, fh, N, 2.0, 5, S.KAISER_BESSEL), tol)
        a1, _, _ = _run(N, pts[:1], f[:1], fh, 2.0, 5, "kaiser_bessel", precision)
        assert ndft.rel_l2(a1, ndft.adjoint(pts[:1], f[:1], N)) <= bar   # exp(-2 pi i k.x)


@pytest.mark.parametrize("window,m", [("gaussian", 6), ("gaussian", 3)])
def test_boundary_ties_gaussian_against_direct_ndft(window, m):
    """The Gaussian does not vanish at the edge of its taps, so at a tie the
    two tap sets differ by its truncation error: the bar is the direct NDFT at
    twice the oracle NFFT's own error (the window error, tap-set independent
    in size)."""
    N = (16, 12, 10)
    pts = np.array([[-0.5, -0.5, -0.5], [0.5, 0.5, 0.5], [0.25, -0.25, 0.0], [3.75, -7.125, 12.5],
                    [0.125, 0.375, -0.3]])
    f = inputs.complex_normal(len(pts), seed=62)
    fh = inputs.complex_normal(N, seed=63)
    ea = ndft.rel_l2(S.adjoint(pts, f, N, 2.0, m, S.GAUSSIAN), ndft.adjoint(pts, f, N))
    eb = ndft.rel_l2(S.forward(pts, fh, N, 2.0, m, S.GAUSSIAN), ndft.forward(pts, fh, N))
    a, b, _ = _run(N, pts, f, fh, 2.0, m, window, "fp64")
    assert ndft.rel_l2(a, ndft.adjoint(pts, f, N)) <= 2 * ea + 1e-14
    assert ndft.rel_l2(b, ndft.forward(pts, fh, N)) <= 2 * eb + 1e-14


@pytest.mark.parametrize("window,m,precision", [("kaiser_bessel", 6, "fp64"), ("kaiser_bessel", 6, "fp32"),
                                                ("gaussian", 6, "fp64")])
def test_lattice_points_on_grid_nodes(window, m, precision):
    """Fluorite lattice, 2 cells: every n x_t is an even integer up to the
    rounding of r / L, so every point is a tie.  Bars independent of the tap
    set: the direct NDFT at the window error and, for the lattice's charges,
    the closed form of the structure factor.  For Kaiser-Bessel (zero weight
    at |u| = m) also element by element against the oracle."""
    r, q, L = inputs.fluorite(2)
    x = inputs.box_points(r, L)
    N = (16, 16, 16)
    f = q.astype(np.complex128)
    fh = inputs.complex_normal(N, seed=71)
    a, b, _ = _run(N, x, f, fh, 2.0, m, window, precision)
    ea = ndft.rel_l2(S.adjoint(x, f, N, 2.0, m, WIN[window]), ndft.adjoint(x, f, N))
    eb = ndft.rel_l2(S.forward(x, fh, N, 2.0, m, WIN[window]), ndft.forward(x, fh, N))
    slack = 1e-13 if precision == "fp64" else FP32_L2
    assert ndft.rel_l2(a, ndft.adjoint(x, f, N)) <= 2 * ea + slack
    assert ndft.rel_l2(b, ndft.forward(x, fh, N)) <= 2 * eb + slack
    # the structure factor of lc^3 cells in closed form: with x = r / L - 1/2,
    # sum_i q_i exp(-2 pi i k.x_i) = (-1)^(k0+k1+k2) lc^3 F(k / lc) for k in
    # lc Z^3 (else 0), F(h) = sum over one cell's ions of q_b exp(-2 pi i h.b)
    r1, q1, L1 = inputs.fluorite(1)
    bfrac = r1 / L1
    lc = 2
    exact = np.zeros(N, dtype=np.complex128)
    grids = np.meshgrid(*[np.arange(-n // 2, n // 2) for n in N], indexing="ij")
    kk = np.stack(grids, -1).reshape(-1, 3)
    on = np.all(kk % lc == 0, axis=1)
    F = np.exp(-2j * np.pi * (kk[on] // lc) @ bfrac.T) @ q1
    exact.reshape(-1)[on] = (-1.0) ** kk[on].sum(axis=1) * lc ** 3 * F
    assert ndft.rel_l2(a, exact) <= 2 * ea + slack
    if window == "kaiser_bessel":
        tol = 1e-12 if precision == "fp64" else FP32_ELEM
        _elementwise(a, S.adjoint(x, f, N, 2.0, m, S.KAISER_BESSEL), tol)
        _elementwise(b, S.forward(x, fh, N, 2.0, m, S.KAISER_BESSEL), tol)


def test_error_statuses():
    from paper_2001_01583_gb300 import _lib
    N, M = (8, 8), 10
    with _plan(N, M, 2.0, 3, "kaiser_bessel", "fp64") as p:
        f = torch.zeros(M, dtype=torch.complex128, device="cuda")
        with pytest.raises(_lib.NFFTError) as e:
            p.adjoint(f)                                     # before set_points
        assert e.value.status == _lib.ERR_NOT_READY
        x = torch.zeros((M, 2), dtype=torch.float64, device="cuda")
        x[3, 1] = float("nan")
        p.set_points(x)
        with pytest.raises(_lib.NFFTError) as e:
            p.sync()
        assert e.value.status == _lib.ERR_DOMAIN
        p.sync()                                             # the flag was cleared
        with pytest.raises(_lib.NFFTError) as e:
            p.set_option(_lib.OPT_THREADS, 33)
        assert e.value.status == _lib.ERR_INVALID_ARG
    with pytest.raises(_lib.NFFTError) as e:
        _plan((7, 8), 10, 2.0, 3, "kaiser_bessel", "fp64")
    assert e.value.status == _lib.ERR_INVALID_ARG


def test_host_buffers_end_to_end():
    N, M = (16, 16), 500
    x = inputs.uniform_points(M, 2, seed=81)
    f = inputs.complex_normal(M, seed=82)
    with _plan(N, M, 2.0, 4, "kaiser_bessel", "fp64") as p:
        p.set_points(torch.from_numpy(x).pin_memory())
        a = p.adjoint(torch.from_numpy(f).pin_memory())
        p.sync()
    assert a.device.type == "cpu"
    _elementwise(a.numpy(), S.adjoint(x, f, N, 2.0, 4, S.KAISER_BESSEL), 1e-12)


def test_pinned_host_results_asynchronous():
    """Host inputs with pinned CPU `out` tensors: the results arrive on the
    plan's stream and equal the device path's (the forward bit for bit; the
    adjoint up to the order of its FP32 atomic additions, so within the FP32
    bars of this file)."""
    N, M = (16, 16, 16), 3000
    x = inputs.uniform_points(M, 3, seed=91)
    f = inputs.complex_normal(M, seed=92, dtype=np.complex64)
    fh = inputs.complex_normal(N, seed=93, dtype=np.complex64)
    with _plan(N, M, 2.0, 4, "kaiser_bessel", "fp32") as p:
        p.set_points(torch.from_numpy(x).cuda())
        a_dev = p.adjoint(torch.from_numpy(f).cuda()).cpu()
        b_dev = p.forward(torch.from_numpy(fh).cuda()).cpu()
        oa = torch.empty(N, dtype=torch.complex64).pin_memory()
        ob = torch.empty(M, dtype=torch.complex64).pin_memory()
        p.set_points(torch.from_numpy(x).pin_memory())
        ra = p.adjoint(torch.from_numpy(f).pin_memory(), out=oa)
        rb = p.forward(torch.from_numpy(fh).pin_memory(), out=ob)
        p.sync()
    assert ra.data_ptr() == oa.data_ptr() and rb.data_ptr() == ob.data_ptr()
    _elementwise(oa.numpy(), a_dev.numpy(), FP32_ELEM)
    d = oa.numpy().astype(np.complex128) - a_dev.numpy()
    assert np.linalg.norm(d) <= FP32_L2 * np.linalg.norm(a_dev.numpy())
    assert torch.equal(ob, b_dev)


# ---- full size of the 3-D configuration, sampled oracle ----------------------
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_full_size_3d_sampled(kind):
    N, M = (64, 64, 64), 10 ** 6
    if kind == "uniform":
        x = inputs.uniform_points(M, 3, seed=0)
    else:
        x = inputs.clustered_points(M, 3, 32, 0.02, seed=0)
    f = inputs.complex_normal(M, seed=1, dtype=np.complex64).astype(np.complex128)
    fh = inputs.complex_normal(N, seed=2, dtype=np.complex64).astype(np.complex128)
    a, b, _ = _run(N, x, f, fh, 2.0, 4, "kaiser_bessel", "fp32")
    rng = np.random.default_rng(3)
    ks = np.stack([rng.integers(-32, 32, size=48) for _ in range(3)], axis=1)
    ref_a = ndft.adjoint(x, f, N, ksel=ks)
    got_a = a[ks[:, 0] + 32, ks[:, 1] + 32, ks[:, 2] + 32]
    assert ndft.rel_l2(got_a, ref_a) <= 1e-6
    js = rng.integers(0, M, size=48)
    assert ndft.rel_l2(b[js], ndft.forward(x, fh, N, jsel=js)) <= 1e-6
