"""GPU tests of the learned parameter picker (the network runs in the
library's kernels: FP16 weights, FP32 accumulation).

- forward, loss and gradients against the FP64 oracle network evaluated on
  the same FP16-rounded weights; the FP16 copy is the rounding of the FP32
  master weights;
- the first Adam step moves every weight by lr against the sign of its
  gradient (bias-corrected moments of one step are g and g^2);
- training by the library's kernels on runs of the plain method lowers the
  loss;
- the error labels of those runs agree with the direct NDFT oracle;
- the shipped picker: on held-out problems its choices reach the requested
  eps against the direct NDFT oracle where the rule of thumb misses it in
  some cases, and cost in total no more than the rule of thumb (within 2%:
  these small problems are launch-bound);
- on a grid-dominated problem (N = 256^3, M = 1e6, eps = 1e-5) the FP32
  rounding floor steers the FP32 choice away from the FP64 one, which would
  miss eps in FP32; the FP32 choice reaches eps within 10% of the rule of
  thumb's time;
- applied to N = 256^3, M = 3e7 points in 64 Gaussian clusters of std 0.01,
  FP32, eps = 1e-5: error at sampled frequencies against the oracle <= eps
  and time <= the rule of thumb's.
"""
import math
import time

import numpy as np
import pytest

from oracle import mlp as mlp_ref, ndft
from paper_2001_01583_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_forward_and_gradients_match_oracle():
    from paper_2001_01583_gb300.picker import MLP
    rng = np.random.default_rng(0)
    B, n_in, n_h, n_out = 300, 8, 64, 132          # 3 blocks of 128 samples, ragged tail
    x = rng.standard_normal((B, n_in)).astype(np.float32)
    t = rng.standard_normal((B, n_out)).astype(np.float32)
    mask = (rng.random((B, n_out)) < 0.5).astype(np.float32)
    with MLP(n_in, n_h, n_out, seed=3) as net:
        xd, td, md = (torch.from_numpy(a).cuda() for a in (x, t, mask))
        y = net.forward(xd).cpu().numpy()
        g, loss = net.gradients(xd, td, md)
        g = g.cpu().numpy()
        w16 = net.get_params(fp16=True)
        w32 = net.get_params()
    assert np.array_equal(w16, w32.astype(np.float16).astype(np.float32))
    p = mlp_ref.unflatten(w16.astype(np.float64), n_in, n_h, n_out)
    y_ref, _ = mlp_ref.forward(p, x)
    assert _rel(y, y_ref) <= 1e-5
    loss_ref, g_ref = mlp_ref.loss_and_grads(p, x, t, mask)
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    got = mlp_ref.unflatten(g.astype(np.float64), n_in, n_h, n_out)
    for name in mlp_ref.PARAM_ORDER:
        assert _rel(got[name], g_ref[name]) <= 1e-4, name


def test_first_adam_step():
    from paper_2001_01583_gb300.picker import MLP
    rng = np.random.default_rng(1)
    B = 200
    x = rng.standard_normal((B, 8)).astype(np.float32)
    t = rng.standard_normal((B, 132)).astype(np.float32)
    mask = np.ones((B, 132), dtype=np.float32)
    lr = 1e-3
    with MLP(seed=4) as net:
        xd, td, md = (torch.from_numpy(a).cuda() for a in (x, t, mask))
        g, loss0 = net.gradients(xd, td, md)
        g = g.cpu().numpy()
        before = net.get_params()
        loss_dev = net.train_step(xd, td, md, lr)
        torch.cuda.synchronize()
        assert abs(loss_dev.item() - loss0) <= 1e-6 * loss0
        after = net.get_params()
        w16 = net.get_params(fp16=True)
    expect = before - lr * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(after - expect)) <= 2e-6
    assert np.array_equal(w16, after.astype(np.float16).astype(np.float32))


def test_training_on_plain_method_runs_lowers_loss():
    from paper_2001_01583_gb300 import picker
    probs = picker.sample_problems(16, seed=77, d_choices=(1, 2))
    E = picker.generate_runs(probs)
    assert np.isfinite(E).sum() >= 16 * 40
    cm = picker.CostModel([2e-9, 9e-9, 5e-9, 3e-10, 1e-9, 1e-7, 0.02])
    X, T, W = picker.build_rows(probs, E, cm, 8, seed=3)
    fm, fs, om, osd = picker.normalisers(X, T, W)
    with picker.MLP(seed=2) as net:
        pk = picker.Picker(net, fm, fs, om, osd)
        losses = picker.train(pk, X, T, W, epochs=60, batch=32, lr=3e-3)
    assert losses[-1] < 0.2 * losses[0], losses[::10]


def test_error_labels_agree_with_direct_ndft():
    from paper_2001_01583_gb300 import Plan, picker
    probs = [dict(d=1, N=(96,), M=700, std=0.0, seed=11), dict(d=2, N=(16, 22), M=500, std=0.02, seed=12),
             dict(d=3, N=(8, 10, 12), M=400, std=0.0, seed=13)]
    check = [(2.0, 3, _lib.KAISER_BESSEL), (1.5, 5, _lib.GAUSSIAN), (1.25, 2, _lib.KAISER_BESSEL)]
    for pb in probs:
        errs = picker.measure_errors(pb)
        x = picker.problem_points(pb)
        f = inputs.complex_normal((1, pb["M"]), seed=pb["seed"] + 7)[0]
        exact = ndft.adjoint(x, f, pb["N"])
        xd = torch.from_numpy(x).cuda()
        fd = torch.from_numpy(f).cuda()
        s, m, w = picker.REFERENCE
        with Plan(pb["N"], pb["M"], s, m, w, "fp64") as p:
            p.set_points(xd)
            ref = p.adjoint(fd).cpu().numpy()
        ref_err = ndft.rel_l2(ref, exact)
        assert ref_err <= 1e-13, (pb, ref_err)
        for (s, m, w) in check:
            c = picker.CANDIDATES.index((s, m, w))
            with Plan(pb["N"], pb["M"], s, m, w, "fp64") as p:
                p.set_points(xd)
                true = ndft.rel_l2(p.adjoint(fd).cpu().numpy(), exact)
            assert abs(errs[c] - true) <= 2 * ref_err + 1e-3 * true, (pb, (s, m, w), errs[c], true)


def _held_out(count, seed, budget=2e7):
    from paper_2001_01583_gb300 import picker
    out, k = [], 0
    while len(out) < count:
        pb = picker.sample_problems(1, seed=seed + k)[0]
        k += 1
        if np.prod(pb["N"]) * pb["M"] <= budget:
            out.append(pb)
    return out


def test_picker_reaches_eps_on_held_out_problems():
    """Picks reach eps on every held-out case; the rule of thumb misses some
    (its estimate ignores constant factors), and the picks cost no more
    (within the 2% the cost model resolves on launch-bound problems)."""
    from paper_2001_01583_gb300 import Plan, picker
    pk = picker.load_default()
    cm = picker.CostModel(pk.meta["cost_coef"])
    rows, fails, rule_misses, cost_pick, cost_rule = [], [], 0, 0.0, 0.0
    for pb in _held_out(12, seed=90000):
        x = picker.problem_points(pb)
        f = inputs.complex_normal((1, pb["M"]), seed=pb["seed"] + 7)[0]
        exact = ndft.adjoint(x, f, pb["N"])
        xd = torch.from_numpy(x).cuda()
        fd = torch.from_numpy(f).cuda()

        def err_of(s, m, w):
            with Plan(pb["N"], pb["M"], s, m, w, "fp64") as p:
                p.set_points(xd)
                return ndft.rel_l2(p.adjoint(fd).cpu().numpy(), exact)

        for eps in (1e-9, 1e-7, 1e-4):
            s, m, w, fb = pk.pick(pb["N"], pb["M"], pb["std"], eps, precision="fp64")
            rs, rm, rw = picker.rule_of_thumb(eps)
            err, err_rule = err_of(s, m, w), err_of(rs, rm, rw)
            c_pick, c_rule = cm(pb["N"], pb["M"], s, m, w), cm(pb["N"], pb["M"], rs, rm, rw)
            cost_pick += c_pick
            cost_rule += c_rule
            rule_misses += int(not err_rule <= eps)
            rows.append((pb["N"], pb["M"], pb["std"], eps, (s, m, w, fb), err, err_rule, c_pick / c_rule))
            if not err <= eps:
                fails.append(rows[-1])
    for r in rows:
        print("N=%s M=%d std=%.3f eps=%.0e pick=%s err=%.2e rule err=%.2e cost/rule=%.2f" % r)
    print("rule of thumb misses eps in %d of %d cases; picks in %d; total cost picked / rule %.3f"
          % (rule_misses, len(rows), len(fails), cost_pick / cost_rule))
    assert not fails, fails
    assert rule_misses >= 1
    # these problems are launch-bound: every candidate costs the same within a
    # few percent; the cost gain is tested on a grid-dominated problem below
    assert cost_pick <= cost_rule * 1.02


def _timed_adjoint_sampled(N, M, params, xd, fd, ks, reps=5):
    from paper_2001_01583_gb300 import Plan
    s, m, w = params
    with Plan(N, M, s, m, w, "fp32") as p:
        p.set_points(xd)
        out = p.adjoint(fd)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(p.stream)
            p.adjoint(fd, out=out)
            e1.record(p.stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        h = [n // 2 for n in N]
        got = out[ks[:, 0] + h[0], ks[:, 1] + h[1], ks[:, 2] + h[2]].cpu().numpy()
    return float(np.median(times)), got


def test_picker_fp32_floor_on_grid_dominated_problem():
    """N = 256^3, M = 1e6 (M / |I_N| = 0.06), eps = 1e-5.  The window error
    alone would allow a small oversampling factor with a wide window, but in
    FP32 the scaling step amplifies the grid's rounding by c_0 / c_k: the
    FP64 choice run in FP32 misses eps, the FP32 choice reaches it at no
    more than 10% above the rule of thumb's time."""
    from paper_2001_01583_gb300 import picker
    N, M, eps = (256, 256, 256), 1_000_000, 1e-5
    pk = picker.load_default()
    p32 = pk.pick(N, M, 0.0, eps, precision="fp32")
    p64 = pk.pick(N, M, 0.0, eps, precision="fp64")
    rule = picker.rule_of_thumb(eps)
    assert not p32[3]
    x = inputs.uniform_points(M, 3, seed=4040)
    f = inputs.complex_normal(M, seed=4041, dtype=np.complex64)
    rng = np.random.default_rng(4)
    ks = np.stack([rng.integers(-128, 128, size=48) for _ in range(3)], axis=1)
    ref = ndft.adjoint(x, f.astype(np.complex128), N, ksel=ks)
    xd = torch.from_numpy(x).cuda()
    fd = torch.from_numpy(f).cuda()
    t32, g32 = _timed_adjoint_sampled(N, M, p32[:3], xd, fd, ks)
    t_rule, g_rule = _timed_adjoint_sampled(N, M, rule, xd, fd, ks)
    e32, e_rule = ndft.rel_l2(g32, ref), ndft.rel_l2(g_rule, ref)
    line = "fp32 pick %s: %.3f ms, error %.2e; rule %s: %.3f ms, error %.2e" % (p32, t32, e32, rule, t_rule, e_rule)
    if p64[:3] != p32[:3]:
        t64, g64 = _timed_adjoint_sampled(N, M, p64[:3], xd, fd, ks)
        e64 = ndft.rel_l2(g64, ref)
        line += "; fp64 pick %s run in fp32: %.3f ms, error %.2e" % (p64, t64, e64)
        amp = picker.amplification(N, *p64[:3])
        if pk.fp32_floor * amp > eps:
            assert e64 > eps
    print(line)
    assert e32 <= eps
    assert t32 <= 1.10 * t_rule


def test_picker_on_large_clustered_problem():
    from paper_2001_01583_gb300 import picker
    N, M, std, eps = (256, 256, 256), 30_000_000, 0.01, 1e-5
    pk = picker.load_default()
    picked = pk.pick(N, M, std, eps)
    rule = picker.rule_of_thumb(eps)
    x = inputs.clustered_points(M, 3, 64, std, seed=2024)
    f = inputs.complex_normal(M, seed=2025, dtype=np.complex64)
    rng = np.random.default_rng(3)
    ks = np.stack([rng.integers(-128, 128, size=32) for _ in range(3)], axis=1)
    t0 = time.time()
    ref = ndft.adjoint(x, f.astype(np.complex128), N, ksel=ks)
    t_oracle = time.time() - t0
    xd = torch.from_numpy(x).cuda()
    fd = torch.from_numpy(f).cuda()
    t_pick, got_pick = _timed_adjoint_sampled(N, M, picked[:3], xd, fd, ks)
    t_rule, got_rule = _timed_adjoint_sampled(N, M, rule, xd, fd, ks)
    e_pick, e_rule = ndft.rel_l2(got_pick, ref), ndft.rel_l2(got_rule, ref)
    print("picked %s: %.3f ms (%.3g pts/s), sampled error %.2e" % (picked, t_pick, M / t_pick * 1e3, e_pick))
    print("rule   %s: %.3f ms (%.3g pts/s), sampled error %.2e" % (rule, t_rule, M / t_rule * 1e3, e_rule))
    print("oracle at %d frequencies: %.1f s" % (len(ks), t_oracle))
    assert e_pick <= eps
    assert t_pick <= 1.05 * t_rule
