"""Learned choice of the window parameters (sigma, m, window) of the NFFT.

The paper sets the oversampling factor sigma, the cut-off m and the window
(Gaussian or Kaiser-Bessel, Section 2) by hand and measures the resulting
accuracy against m (Section 4, Fig. 12).  This module picks them per problem:
a small network (8 -> 64 -> 64 -> 2K, ReLU) predicts, for each of K candidate
triples, the log10 of the adjoint's relative l2 error divided by the requested
eps and the log10 of the transform's cost.  The library's own kernels train
and evaluate it (nfft_mlp_*: FP16 weights, FP32 accumulation, Adam on FP32
master weights), and nfft_pick_params takes the cheapest candidate predicted
to reach eps with a margin, or the rule of thumb (Kaiser-Bessel, sigma = 2,
m = ceil(ln(1/eps) / (2 pi sqrt(1 - 1/sigma)))) when none qualifies.  For the
FP32 form a candidate must also keep the FP32 rounding floor, which the
scaling step amplifies by c_0 / c_k (large for small sigma and large m),
below eps: floor = kappa * rms(c_0 / c_k), kappa fitted to FP32 runs.

Training data are runs of the plain method itself: FP64 adjoint transforms
(Eq. 5) of random problems with every candidate, each error measured against
an FP64 run with a Kaiser-Bessel window, sigma = 4, m = 12, whose own error
is at the level of FP64 rounding.  Costs come from a linear model of the
transform's work (window taps per point, FFT size) fitted to timed FP32
transforms.  The paper has no such component.

    python -m paper_2001_01583_gb300.picker train --out picker.json
"""
import argparse
import base64
import ctypes
import json
import math
import os
import time

import numpy as np
import torch

from . import _lib, inputs
from .nfft import Batch, Plan, _stream_handle, plan_params

N_FEATURES = 8
HIDDEN = 64
SIGMAS = (1.25, 1.5, 2.0)
CUT_OFFS = tuple(range(2, 13))
WINDOW_SET = (_lib.GAUSSIAN, _lib.KAISER_BESSEL)
CANDIDATES = tuple((s, m, w) for w in WINDOW_SET for s in SIGMAS for m in CUT_OFFS)
REFERENCE = (4.0, 12, _lib.KAISER_BESSEL)
N_CLUSTERS = 64
DEFAULT_CHECKPOINT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "picker_weights.json")


# ---------------------------------------------------------------------------
# the network (C ABI nfft_mlp_*)
# ---------------------------------------------------------------------------
class MLP:
    """n_in -> n_hidden -> n_hidden -> n_out with ReLU, on the GPU.

    Parameters are flattened W1 (n_hidden x n_in), b1, W2, b2, W3
    (n_out x n_hidden), b3, all row-major float32."""

    def __init__(self, n_in=N_FEATURES, n_hidden=HIDDEN, n_out=2 * len(CANDIDATES), seed=0, stream=None):
        self._lib = _lib.load()
        self.n_in, self.n_hidden, self.n_out = int(n_in), int(n_hidden), int(n_out)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _lib.check(self._lib.nfft_mlp_create(ctypes.byref(h), self.n_in, self.n_hidden, self.n_out, int(seed),
                                             _stream_handle(self.stream)), "nfft_mlp_create")
        self._h = h
        n = ctypes.c_int64()
        _lib.check(self._lib.nfft_mlp_num_params(self._h, ctypes.byref(n)), "nfft_mlp_num_params")
        self.num_params = n.value
        self._loss = torch.zeros(1, dtype=torch.float32, device=self.device)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.nfft_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        if flat.size != self.num_params:
            raise ValueError("expected %d parameters, got %d" % (self.num_params, flat.size))
        _lib.check(self._lib.nfft_mlp_set_params(self._h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                   "nfft_mlp_set_params")

    def get_params(self, fp16=False):
        out = np.empty(self.num_params, dtype=np.float32)
        _lib.check(self._lib.nfft_mlp_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                 1 if fp16 else 0), "nfft_mlp_get_params")
        return out

    def _check(self, x, t=None, mask=None):
        tensors = [x] + [v for v in (t, mask) if v is not None]
        for v in tensors:
            if v.device.type != "cuda" or v.dtype != torch.float32 or not v.is_contiguous():
                raise TypeError("expected contiguous float32 CUDA tensors")
        if x.dim() != 2 or x.shape[1] != self.n_in:
            raise ValueError("x must be (B, %d)" % self.n_in)
        for v in tensors[1:]:
            if tuple(v.shape) != (x.shape[0], self.n_out):
                raise ValueError("targets and mask must be (B, %d)" % self.n_out)

    def forward(self, x):
        self._check(x)
        y = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=self.device)
        _lib.check(self._lib.nfft_mlp_forward(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                              int(x.shape[0])), "nfft_mlp_forward")
        return y

    def gradients(self, x, t, mask):
        """(gradient as a float32 CUDA tensor, loss) of the masked loss, no update."""
        self._check(x, t, mask)
        g = torch.empty(self.num_params, dtype=torch.float32, device=self.device)
        loss = ctypes.c_float()
        _lib.check(self._lib.nfft_mlp_gradients(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                                ctypes.c_void_p(mask.data_ptr()), int(x.shape[0]),
                                                ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss)),
                   "nfft_mlp_gradients")
        return g, loss.value

    def train_step(self, x, t, mask, lr):
        """One Adam step; returns the minibatch loss as a 1-element CUDA tensor
        (read it only when needed: reading waits for the device)."""
        self._check(x, t, mask)
        _lib.check(self._lib.nfft_mlp_train_step(self._h, ctypes.c_void_p(x.data_ptr()),
                                                 ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(mask.data_ptr()),
                                                 int(x.shape[0]), float(lr), ctypes.c_void_p(self._loss.data_ptr())),
                   "nfft_mlp_train_step")
        return self._loss


# ---------------------------------------------------------------------------
# host rules (C ABI, no device work)
# ---------------------------------------------------------------------------
def features(d, N, M, cluster_std, eps):
    """The 8 picker features: d, log2 N_0..N_2 (0 if unused), log10 M,
    cluster std (0 = uniform), log10 eps, log10(M / |I_N|)."""
    lib = _lib.load()
    Narr = (ctypes.c_int64 * 3)(*([int(v) for v in N] + [1] * (3 - len(N))))
    out = (ctypes.c_double * N_FEATURES)()
    _lib.check(lib.nfft_picker_features(int(d), Narr, int(M), float(cluster_std), float(eps), out),
               "nfft_picker_features")
    return np.array(out[:], dtype=np.float64)


def rule_of_thumb(eps):
    lib = _lib.load()
    s, m, w = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    _lib.check(lib.nfft_rule_of_thumb(float(eps), ctypes.byref(s), ctypes.byref(m), ctypes.byref(w)),
               "nfft_rule_of_thumb")
    return s.value, m.value, w.value


def amplification(N, sigma, m, window):
    """rms over I_N of c_0 / c_k (the scaling step's amplification of grid
    rounding), from the library's host rule nfft_deconv_amplification."""
    lib = _lib.load()
    Narr = (ctypes.c_int64 * len(N))(*[int(v) for v in N])
    rms = ctypes.c_double()
    _lib.check(lib.nfft_deconv_amplification(len(N), Narr, float(sigma), int(m), int(window), ctypes.byref(rms), None),
               "nfft_deconv_amplification")
    return rms.value


def valid(N, sigma, m):
    """The picker's validity rule for a candidate (as in nfft_pick_params):
    ceil(sigma N_t) >= 2m + 2 in every dimension."""
    return all(math.ceil(sigma * n) >= 2 * m + 2 for n in N)


DEFAULT_BINS = {1: (1024,), 2: (32, 32), 3: (8, 8, 16)}


def cost_terms(N, M, sigma, m, window):
    """Work terms of one adjoint: cell updates M taps^d split by where they
    run (dense bins on shared tiles, sparse bins on grid atomics: at uniform
    density, a bin is sparse below one point per taps^d / 2 tile cells, the
    library's default split), M d taps (window evaluations), P log2 P (FFT
    of P = prod n_t cells), P (grid clear, scaling), M (sort, per-point
    work), 1 (launches)."""
    n, taps = plan_params(N, sigma, m, window)
    P = float(np.prod(n))
    d = len(N)
    bins = [min(b, nt) for b, nt in zip(DEFAULT_BINS[d], n)]
    per_bin = float(M) * float(np.prod(bins)) / P
    tile = float(np.prod([b + taps - 1 for b in bins]))
    sparse = per_bin < 2.0 * tile / taps ** d
    updates = float(M) * taps ** d
    return np.array([0.0 if sparse else updates, updates if sparse else 0.0, float(M) * d * taps,
                     P * math.log2(max(P, 2.0)), P, float(M), 1.0])


class CostModel:
    """Predicted time (ms) of one FP32 adjoint: a nonnegative combination of
    cost_terms fitted to timed runs, minimising relative error."""

    def __init__(self, coef):
        self.coef = np.asarray(coef, dtype=np.float64)

    def __call__(self, N, M, sigma, m, window):
        return float(cost_terms(N, M, sigma, m, window) @ self.coef)

    @classmethod
    def fit(cls, rows, times_ms):
        from scipy.optimize import nnls
        A = np.asarray(rows, dtype=np.float64)
        t = np.asarray(times_ms, dtype=np.float64)
        scale = A.max(axis=0)
        scale[scale == 0] = 1.0
        coef, _ = nnls((A / scale) / t[:, None], np.ones_like(t))
        return cls(coef / scale)


def time_adjoint(N, M, sigma, m, window, x, f, reps=3, precision="fp32"):
    """Median ms of `reps` adjoint calls of one plan after one warm-up call."""
    with Plan(N, M, sigma, m, window, precision) as p:
        p.set_points(x)
        out = p.adjoint(f)
        times = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(p.stream)
            p.adjoint(f, out=out)
            e1.record(p.stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        p.sync()
    return float(np.median(times))


CALIBRATION = [
    # (d, N_t, M): problems timed with a spread of candidates
    (3, 32, 10 ** 4), (3, 32, 10 ** 6), (3, 64, 10 ** 4), (3, 64, 10 ** 5), (3, 64, 10 ** 6), (3, 64, 4 * 10 ** 6),
    (3, 128, 10 ** 5), (3, 128, 2 * 10 ** 6), (3, 256, 10 ** 6), (3, 256, 10 ** 7),
    (2, 512, 10 ** 5), (2, 1024, 10 ** 6), (2, 2048, 10 ** 6), (1, 1 << 16, 10 ** 6), (1, 1 << 20, 10 ** 6),
]
CALIBRATION_CANDIDATES = [(2.0, 2, 1), (2.0, 3, 1), (2.0, 4, 1), (2.0, 6, 1), (2.0, 9, 1), (1.5, 4, 1), (1.5, 7, 1),
                          (1.25, 4, 1), (1.25, 8, 1), (2.0, 4, 0), (1.25, 6, 0)]


def calibrate_cost(reps=3, max_updates=2e10, seed=0, log=None):
    """Times FP32 adjoints of the calibration problems and fits CostModel."""
    rows, times = [], []
    for i, (d, Nt, M) in enumerate(CALIBRATION):
        N = (Nt,) * d
        x = torch.from_numpy(inputs.uniform_points(M, d, seed=seed + i)).cuda()
        f = torch.from_numpy(inputs.complex_normal(M, seed=seed + 1000 + i, dtype=np.complex64)).cuda()
        for (s, m, w) in CALIBRATION_CANDIDATES:
            if not valid(N, s, m):
                continue
            terms = cost_terms(N, M, s, m, w)
            if terms[0] > max_updates:
                continue
            ms = time_adjoint(N, M, s, m, w, x, f, reps=reps)
            rows.append(terms)
            times.append(ms)
            if log:
                log("calibrate d=%d N=%d M=%d sigma=%.2f m=%d w=%d: %.3f ms" % (d, Nt, M, s, m, w, ms))
        del x, f
        torch.cuda.empty_cache()
    model = CostModel.fit(rows, times)
    pred = np.asarray(rows) @ model.coef
    rel = np.abs(pred / np.asarray(times) - 1.0)
    return model, dict(runs=len(times), median_rel_err=float(np.median(rel)), max_rel_err=float(rel.max()))


# ---------------------------------------------------------------------------
# training data: runs of the plain method
# ---------------------------------------------------------------------------
def sample_problems(count, seed, d_choices=(1, 2, 3)):
    """Random problems: d, even N_t (log-uniform per dimension), M
    (log-uniform), cluster std (0 = uniform in half of them)."""
    rng = np.random.default_rng(seed)
    out = []
    lims = {1: (16, 8192), 2: (8, 512), 3: (8, 96)}
    m_hi = {1: 10 ** 5, 2: 10 ** 5, 3: 3 * 10 ** 4}
    for i in range(count):
        d = int(rng.choice(d_choices))
        lo, hi = lims[d]
        N = tuple(int(2 * round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / 2)) for _ in range(d))
        M = int(round(math.exp(rng.uniform(math.log(50), math.log(m_hi[d])))))
        std = 0.0 if rng.random() < 0.5 else float(math.exp(rng.uniform(math.log(0.005), math.log(0.1))))
        out.append(dict(d=d, N=N, M=M, std=std, seed=int(seed * 100003 + i)))
    return out


def problem_points(pb):
    if pb["std"] > 0:
        return inputs.clustered_points(pb["M"], pb["d"], min(N_CLUSTERS, pb["M"]), pb["std"], seed=pb["seed"])
    return inputs.uniform_points(pb["M"], pb["d"], seed=pb["seed"])


def measure_errors(pb, candidates=CANDIDATES, precision="fp64"):
    """Relative l2 error of the adjoint (Eq. 5) of one problem with every
    valid candidate, against the reference parameters; NaN where invalid.
    One batch (one graph launch) runs all candidates."""
    N, M = pb["N"], pb["M"]
    ok = [i for i, (s, m, w) in enumerate(candidates) if valid(N, s, m)]
    items = [dict(N=N, M=M, sigma=candidates[i][0], m=candidates[i][1], window=candidates[i][2]) for i in ok]
    items.append(dict(N=N, M=M, sigma=REFERENCE[0], m=REFERENCE[1], window=REFERENCE[2]))
    cdt = np.complex128 if precision == "fp64" else np.complex64
    x = torch.from_numpy(problem_points(pb)).cuda()
    f = torch.from_numpy(inputs.complex_normal((1, M), seed=pb["seed"] + 7, dtype=cdt)).cuda()
    with Batch(items, precision) as b:
        b.set_points([x] * len(items))
        A = b.adjoint([f] * len(items))
        b.sync()
        ref = A[-1].to(torch.complex128)
        rnorm = torch.linalg.vector_norm(ref).item()
        errs = np.full(len(candidates), np.nan)
        for j, i in enumerate(ok):
            errs[i] = torch.linalg.vector_norm(A[j].to(torch.complex128) - ref).item() / rnorm
    return errs


def measure_errors_fp32(pb, candidates=CANDIDATES):
    """Relative l2 error of the FP32 adjoint of every valid candidate
    against the FP64 reference run; NaN where invalid."""
    N, M = pb["N"], pb["M"]
    ok = [i for i, (s, m, w) in enumerate(candidates) if valid(N, s, m)]
    x = torch.from_numpy(problem_points(pb)).cuda()
    f64 = inputs.complex_normal((1, M), seed=pb["seed"] + 7)
    s, m, w = REFERENCE
    with Plan(N, M, s, m, w, "fp64") as p:
        p.set_points(x)
        ref = p.adjoint(torch.from_numpy(f64[0]).cuda())
        p.sync()
    f = torch.from_numpy(f64.astype(np.complex64)).cuda()
    items = [dict(N=N, M=M, sigma=candidates[i][0], m=candidates[i][1], window=candidates[i][2]) for i in ok]
    errs = np.full(len(candidates), np.nan)
    with Batch(items, "fp32") as b:
        b.set_points([x] * len(items))
        A = b.adjoint([f] * len(items))
        b.sync()
        rnorm = torch.linalg.vector_norm(ref).item()
        for j, i in enumerate(ok):
            errs[i] = torch.linalg.vector_norm(A[j][0].to(torch.complex128) - ref).item() / rnorm
    return errs


def fit_fp32_floor(problems, errors64, errors32, quantile=0.95):
    """FP32 rounding floor per unit of scaling amplification: a high quantile
    of err32 / amplification over runs whose FP64 (window) error is far
    below their FP32 error."""
    ratios = []
    for pb, e64, e32 in zip(problems, errors64, errors32):
        for c, (s, m, w) in enumerate(CANDIDATES):
            if np.isfinite(e32[c]) and np.isfinite(e64[c]) and e64[c] < 0.1 * e32[c]:
                ratios.append(e32[c] / amplification(pb["N"], s, m, w))
    return float(np.quantile(ratios, quantile)), len(ratios)


def generate_runs(problems, log=None):
    """Error table (problems x candidates) from plain-method runs."""
    E = np.full((len(problems), len(CANDIDATES)), np.nan)
    t0 = time.time()
    for p, pb in enumerate(problems):
        E[p] = measure_errors(pb)
        if log and (p + 1) % 25 == 0:
            log("runs: %d problems, %d runs, %.1f s" % (p + 1, int(np.isfinite(E[:p + 1]).sum()), time.time() - t0))
    return E


EPS_RANGE = (1e-10, 1e-3)
ERR_FLOOR = 1e-16


def build_rows(problems, errors, cost_model, eps_per_problem, seed, cost_only=False):
    """Training rows: features of (problem, eps) and targets
    [log10(err_c / eps)]_c ++ [log10(cost_c)]_c with a mask of labelled
    outputs (invalid candidates unlabelled; cost-only rows label costs)."""
    rng = np.random.default_rng(seed)
    K = len(CANDIDATES)
    X, T, W = [], [], []
    for p, pb in enumerate(problems):
        cost = np.full(K, np.nan)
        for c, (s, m, w) in enumerate(CANDIDATES):
            if valid(pb["N"], s, m):
                cost[c] = math.log10(max(cost_model(pb["N"], pb["M"], s, m, w), 1e-6))
        for _ in range(eps_per_problem):
            eps = 10 ** rng.uniform(math.log10(EPS_RANGE[0]), math.log10(EPS_RANGE[1]))
            t = np.zeros(2 * K)
            mask = np.zeros(2 * K)
            if not cost_only:
                e = errors[p]
                fin = np.isfinite(e)
                t[:K][fin] = np.log10(np.maximum(e[fin], ERR_FLOOR) / eps)
                mask[:K][fin] = 1.0
            fin = np.isfinite(cost)
            t[K:][fin] = cost[fin]
            mask[K:][fin] = 1.0
            X.append(features(pb["d"], pb["N"], pb["M"], pb["std"], eps))
            T.append(t)
            W.append(mask)
    return np.array(X), np.array(T), np.array(W)


def sample_cost_problems(count, seed):
    """Problems for cost-only rows, up to the sizes of large transforms
    (no run needed: their labels come from the cost model)."""
    rng = np.random.default_rng(seed)
    lims = {1: (64, 1 << 22), 2: (32, 4096), 3: (16, 512)}
    out = []
    for i in range(count):
        d = int(rng.integers(1, 4))
        lo, hi = lims[d]
        N = tuple(int(2 * round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / 2)) for _ in range(d))
        M = int(round(10 ** rng.uniform(2, 8.3)))
        std = 0.0 if rng.random() < 0.5 else float(math.exp(rng.uniform(math.log(0.005), math.log(0.1))))
        out.append(dict(d=d, N=N, M=M, std=std, seed=i))
    return out


# ---------------------------------------------------------------------------
# the picker
# ---------------------------------------------------------------------------
class Picker:
    """The trained network with its normalisation and candidate table."""

    def __init__(self, mlp, feat_mean, feat_std, out_mean, out_std, err_margin=0.5, meta=None, fp32_floor=0.0):
        self.mlp = mlp
        self.feat_mean = np.asarray(feat_mean, dtype=np.float64)
        self.feat_std = np.asarray(feat_std, dtype=np.float64)
        self.out_mean = np.asarray(out_mean, dtype=np.float64)
        self.out_std = np.asarray(out_std, dtype=np.float64)
        self.meta = dict(meta or {})
        self.fp32_floor = float(fp32_floor)
        self.configure(err_margin)

    def configure(self, err_margin, fp32_floor=None):
        self.err_margin = float(err_margin)
        if fp32_floor is not None:
            self.fp32_floor = float(fp32_floor)
        K = len(CANDIDATES)
        dbl = lambda a: (ctypes.c_double * len(a))(*[float(v) for v in a])
        _lib.check(self.mlp._lib.nfft_picker_configure(
            self.mlp._h, K, dbl([c[0] for c in CANDIDATES]), (ctypes.c_int * K)(*[c[1] for c in CANDIDATES]),
            (ctypes.c_int * K)(*[c[2] for c in CANDIDATES]), dbl(self.feat_mean), dbl(self.feat_std),
            dbl(self.out_mean), dbl(self.out_std), self.err_margin, self.fp32_floor), "nfft_picker_configure")

    def pick(self, N, M, cluster_std, eps, precision="fp32"):
        """(sigma, m, window, used_fallback) for a problem solved in `precision`."""
        N = tuple(int(v) for v in N)
        Narr = (ctypes.c_int64 * 3)(*(list(N) + [1] * (3 - len(N))))
        prec = _lib.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        s, m, w, fb = ctypes.c_double(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(self.mlp._lib.nfft_pick_params(self.mlp._h, len(N), Narr, int(M), float(cluster_std), float(eps),
                                                  prec, ctypes.byref(s), ctypes.byref(m), ctypes.byref(w),
                                                  ctypes.byref(fb)), "nfft_pick_params")
        return s.value, m.value, w.value, bool(fb.value)

    def predict(self, feats):
        """Denormalised network outputs for raw feature rows (B x 8):
        (log10(err / eps), log10(cost)), each B x K."""
        xf = (np.atleast_2d(feats) - self.feat_mean) / self.feat_std
        y = self.mlp.forward(torch.from_numpy(xf.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
        y = y * self.out_std + self.out_mean
        K = len(CANDIDATES)
        return y[:, :K], y[:, K:]

    # -- checkpoint ---------------------------------------------------------------
    def state(self, epoch=None):
        w = self.mlp.get_params()
        return dict(format="gbnfft-picker-1", n_in=self.mlp.n_in, n_hidden=self.mlp.n_hidden, n_out=self.mlp.n_out,
                    candidates=[list(c) for c in CANDIDATES], feat_mean=self.feat_mean.tolist(),
                    feat_std=self.feat_std.tolist(), out_mean=self.out_mean.tolist(), out_std=self.out_std.tolist(),
                    err_margin=self.err_margin, fp32_floor=self.fp32_floor, epoch=epoch,
                    params_f32_b64=base64.b64encode(w.astype("<f4").tobytes()).decode("ascii"), meta=self.meta)

    def save(self, path, epoch=None):
        with open(path, "w") as fh:
            json.dump(self.state(epoch), fh)

    @classmethod
    def load(cls, path, stream=None):
        with open(path) as fh:
            st = json.load(fh)
        if st.get("format") != "gbnfft-picker-1" or [tuple(c) for c in st["candidates"]] != [
                (float(s), int(m), int(w)) for (s, m, w) in CANDIDATES]:
            raise ValueError("%s: not a checkpoint of this picker" % path)
        mlp = MLP(st["n_in"], st["n_hidden"], st["n_out"], stream=stream)
        mlp.set_params(np.frombuffer(base64.b64decode(st["params_f32_b64"]), dtype="<f4"))
        pk = cls(mlp, st["feat_mean"], st["feat_std"], st["out_mean"], st["out_std"], st["err_margin"], st["meta"],
                 st.get("fp32_floor", 0.0))
        pk.epoch = st.get("epoch")
        return pk


def load_default(stream=None):
    """The picker trained by `python -m paper_2001_01583_gb300.picker train`
    and shipped with the package."""
    return Picker.load(DEFAULT_CHECKPOINT, stream=stream)


def normalisers(X, T, mask):
    feat_mean = X.mean(axis=0)
    feat_std = X.std(axis=0)
    feat_std[feat_std < 1e-12] = 1.0
    cnt = np.maximum(mask.sum(axis=0), 1.0)
    out_mean = (T * mask).sum(axis=0) / cnt
    out_std = np.sqrt((((T - out_mean) * mask) ** 2).sum(axis=0) / cnt)
    out_std[out_std < 1e-6] = 1.0
    return feat_mean, feat_std, out_mean, out_std


def train(picker, X, T, mask, epochs=300, batch=512, lr=2e-3, lr_min=5e-5, seed=0, checkpoint=None,
          save_every=50, start_epoch=0, log=None):
    """Adam on the masked loss in normalised units; returns per-epoch mean
    losses.  With `checkpoint`, the state is written every `save_every`
    epochs and at the end (training resumes from such a file via
    Picker.load and start_epoch; the Adam moments restart)."""
    xn = torch.from_numpy(((X - picker.feat_mean) / picker.feat_std).astype(np.float32)).cuda()
    tn = torch.from_numpy(((T - picker.out_mean) / picker.out_std * (mask > 0)).astype(np.float32)).cuda()
    mk = torch.from_numpy(mask.astype(np.float32)).cuda()
    R = xn.shape[0]
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed + start_epoch)
    losses = []
    for ep in range(start_epoch, epochs):
        rate = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * ep / max(epochs, 1)))
        perm = torch.randperm(R, generator=gen).cuda()
        acc = torch.zeros(1, dtype=torch.float32, device=xn.device)
        steps = 0
        for s in range(0, R - batch + 1 if R >= batch else 1, batch):
            idx = perm[s:s + batch]
            xb, tb, mb = xn[idx].contiguous(), tn[idx].contiguous(), mk[idx].contiguous()
            acc += picker.mlp.train_step(xb, tb, mb, rate)
            steps += 1
        losses.append(acc.item() / max(steps, 1))
        if log and (ep + 1) % 25 == 0:
            log("epoch %d: loss %.5f (lr %.2e)" % (ep + 1, losses[-1], rate))
        if checkpoint and (ep + 1) % save_every == 0:
            picker.save(checkpoint, epoch=ep + 1)
    if checkpoint:
        picker.save(checkpoint, epoch=epochs)
    return losses


def choose_margin(picker, problems, errors, eps_list, margins=(0.5, 0.35, 0.25, 0.15, 0.1, 0.05)):
    """Largest margin under which every pick on held-out (problem, eps)
    pairs reaches eps (errors: measured table of those problems)."""
    for mg in margins:
        picker.configure(mg)
        bad = 0
        for p, pb in enumerate(problems):
            for eps in eps_list:
                s, m, w, fb = picker.pick(pb["N"], pb["M"], pb["std"], eps, precision="fp64")
                if fb:
                    continue
                c = CANDIDATES.index((s, m, w))
                if not (errors[p, c] <= eps):
                    bad += 1
        if bad == 0:
            return mg
    return margins[-1]


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the NFFT parameter picker on runs of the plain method")
    ap.add_argument("command", choices=["train"])
    ap.add_argument("--problems", type=int, default=330)
    ap.add_argument("--val-problems", type=int, default=40)
    ap.add_argument("--eps-per-problem", type=int, default=12)
    ap.add_argument("--cost-problems", type=int, default=600)
    ap.add_argument("--fp32-problems", type=int, default=40)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", required=True)
    ap.add_argument("--data-out", default=None, help="optional .npz with the measured error tables")
    args = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)
    torch.cuda.set_device(0)
    t0 = time.time()
    cost_model, cal = calibrate_cost(log=log)
    log("cost model %s, fit %s (%.1f s)" % (cost_model.coef.tolist(), cal, time.time() - t0))
    probs = sample_problems(args.problems, seed=args.seed)
    val = sample_problems(args.val_problems, seed=args.seed + 1000)
    E = generate_runs(probs, log=log)
    Ev = generate_runs(val, log=log)
    n_runs = int(np.isfinite(E).sum())
    log("%d training runs, %d validation runs (%.1f s)" % (n_runs, int(np.isfinite(Ev).sum()), time.time() - t0))
    if args.data_out:
        np.savez_compressed(args.data_out, errors=E, val_errors=Ev,
                            problems=json.dumps(probs), val_problems=json.dumps(val))
    X1, T1, W1 = build_rows(probs, E, cost_model, args.eps_per_problem, seed=args.seed)
    X2, T2, W2 = build_rows(sample_cost_problems(args.cost_problems, args.seed + 7), None, cost_model, 2,
                            seed=args.seed + 8, cost_only=True)
    X, T, W = np.concatenate([X1, X2]), np.concatenate([T1, T2]), np.concatenate([W1, W2])
    fm, fs, om, osd = normalisers(X, T, W)
    mlp = MLP(seed=args.seed)
    meta = dict(runs=n_runs, rows=int(X.shape[0]), cost_coef=cost_model.coef.tolist(), cost_fit=cal,
                epochs=args.epochs, problems=args.problems, seed=args.seed,
                reference=dict(sigma=REFERENCE[0], m=REFERENCE[1], window=REFERENCE[2], precision="fp64"))
    pk = Picker(mlp, fm, fs, om, osd, 0.5, meta)
    losses = train(pk, X, T, W, epochs=args.epochs, seed=args.seed, log=log)
    margin = choose_margin(pk, val, Ev, eps_list=[1e-9, 1e-7, 1e-5, 1e-4, 1e-3])
    sub = probs[:args.fp32_problems]
    E32 = [measure_errors_fp32(pb) for pb in sub]
    floor, n_fit = fit_fp32_floor(sub, E[:len(sub)], E32)
    pk.configure(margin, floor)
    log("fp32 floor %.3g per unit amplification (%d runs)" % (floor, n_fit))
    pk.meta.update(final_loss=losses[-1], first_loss=losses[0], err_margin=margin, fp32_floor=floor,
                   fp32_floor_runs=n_fit, seconds=time.time() - t0)
    pk.save(args.out, epoch=args.epochs)
    log("saved %s: loss %.5f -> %.5f, margin %.2f, %.1f s" % (args.out, losses[0], losses[-1], margin,
                                                            time.time() - t0))


if __name__ == "__main__":
    main()
