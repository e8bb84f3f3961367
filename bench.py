"""Throughput benchmark of the GB300 NFFT library.

Workload (one "step", default "picker"): the largest configuration that fits
one GPU, N = 256^3 and M = 3e7 points in 64 Gaussian clusters of std 0.01,
complex64 values, eps = 1e-5, with the window parameters the learned picker
chooses, mixed FP32.  A step runs nfft_set_points (argument reduction + bin
sort), the adjoint NFFT (Eq. 5: spread, FFT, scale) and the forward NFFT
(Eq. 6: subdivide, inverse FFT, interpolate).  Units: a transform of M points
counts M nonuniform points, so a step processes 2 x M points per point set.
The same line reports the relative l2 error (Eq. 9) of the timed outputs at
sampled frequencies and points against the direct NDFT, the rule-of-thumb
parameters and the plain FP64 form of the same workload on the same GPU, the
end-to-end rate with host buffers, and the dominant stage's HBM roofline.

"--workload config" is the 3-D configuration N = 64^3, M = 10^6, Kaiser-Bessel
m = 4, sigma = 2, on two point sets (uniform, and 32 Gaussian clusters of std
0.02).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload picker|config|small|sparse|profile|batch|1d|fluorite|fig13|fig16]
                  [--precision fp32|fp64] [--no-autotune] [--no-cpu-baseline] [--no-fp64-form]
                  [--tensor-spread] [--tensor-interp] [--owner-spread]

"--workload small" (N = 64^3, M = 5e5, uniform only) is the case profiled
with ncu's multi-pass sections.  "--workload fig13" and "fig16" sweep the
sizes of the paper's runtime figures (58^3 ... 120^3 points; fluorite with
12 x {32 ... 64}^3 ions) and list every size in config.sweep.  Prints one JSON
line (rank 0).  Under torchrun every rank runs its own independent copy of the
workload (weak scaling, no collective on the data path); the value is all
ranks' points over the slowest rank's time.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NFFT nonuniform points/s at stated rel-l2 error; % of HBM roofline"
UNIT = "points/s"
SIGMA, MCUT, WINDOW = 2.0, 4, "kaiser_bessel"

DEFAULT_WORKLOAD = "picker"   # the largest configuration that fits one GPU

WORKLOADS = {
    "config": dict(N=(64, 64, 64), M=10 ** 6, sets=("uniform", "clustered"), seeds=dict(x=(0, 1), f=7, fh=8),
                   name="3-D adjoint+forward NFFT, N=64^3, M=10^6, uniform + clustered (32 clusters, std 0.02), "
                        "Kaiser-Bessel m=4, sigma=2, mixed FP32"),
    "batch": dict(N=None, M=None, sets=("batch",),
                  name="batched 3-D adjoint+forward NFFT: 512 transforms, N from {32^3, 64^3}, M log-uniform in "
                       "[1e3, 1e5], plus one 64^3 point set with M=2e5 and 16 right-hand sides; Kaiser-Bessel m=4, "
                       "sigma=2; one CUDA-graph launch per direction"),
    "1d": dict(N=(256,), M=1024, sets=("uniform",), extra=True,
               name="1-D plain FP64 NFFT, N=256, M=1024, Gaussian m=6, sigma=2, adjoint+forward (launch-latency "
                    "bound)"),
    "fluorite": dict(N=(128, 128, 128), M=12 * 32 ** 3, sets=("fluorite",), extra=True,
                     name="Ewald reciprocal energy of fluorite, 32^3 cells (393216 ions), N=128^3, Kaiser-Bessel m=6, "
                          "sigma=2: set_points + adjoint NFFT of the charges + weighted mode sum"),
    "picker": dict(N=(256, 256, 256), M=30_000_000, sets=("clustered64",), picked=True, eps=1e-5,
                   seeds=dict(x=(0,), f=1, fh=2),
                   name="learned parameter picker applied to 3-D N=256^3, M=3x10^7 clustered points (64 Gaussian "
                        "clusters, std 0.01), complex64, eps=1e-5, vs the rule-of-thumb parameters: one step = "
                        "set_points + adjoint + forward NFFT with the picked window parameters, mixed FP32"),
    "profile": dict(N=(128, 128, 128), M=4_000_000, sets=("clustered64",), picked=True, eps=1e-5,
                    seeds=dict(x=(0,), f=1, fh=2),
                    name="scaled-down largest configuration for ncu's multi-pass captures: 3-D N=128^3, M=4x10^6 "
                         "points in 64 Gaussian clusters (std 0.01), eps=1e-5, picked window parameters, mixed FP32"),
    "fig13": dict(N=(128, 128, 128), M=120 ** 3, sets=("uniform",), sweep=True,
                  name="sweep shaped like Fig. 13: 3-D adjoint+forward NFFT of 58^3, 80^3, 100^3 and 120^3 uniform "
                       "points at N=64^3 and 128^3, Kaiser-Bessel m=4, sigma=2, mixed FP32; value at 120^3, N=128^3"),
    "fig16": dict(N=(128, 128, 128), M=12 * 64 ** 3, sets=("fluorite",), sweep=True, lc=64,
                  name="sweep shaped like Fig. 16: Ewald reciprocal energy of fluorite with 12 x {32, 45, 56, 64}^3 "
                       "ions, N=128^3, Kaiser-Bessel m=6, sigma=2, alpha=0.6; value at 12 x 64^3 ions"),
    "sparse": dict(N=(64, 64, 64), M=20000, sets=("uniform",), seeds=dict(x=(0,), f=7, fh=8),
                   name="3-D adjoint+forward NFFT, N=64^3, M=2e4 uniform (about 10 points per bin: the sparse "
                        "grid-warp kernels), Kaiser-Bessel m=4, sigma=2, mixed FP32"),
    "small": dict(N=(64, 64, 64), M=500000, sets=("uniform",), seeds=dict(x=(0,), f=7, fh=8),
                  name="3-D adjoint+forward NFFT, N=64^3, M=5e5, uniform, Kaiser-Bessel m=4, sigma=2, mixed FP32 "
                       "(profiling case: the same grid and bins, half the points, one set)"),
}

# bytes of the shared-memory traffic per cell visit: spread reads and writes
# one complex64 tile cell, interpolation reads one
SMEM_BYTES_PER_CELL = {"spread": 16, "interp": 8}
SMEM_BYTES_PER_CLK_PER_SM = 128   # 32 banks x 4 B


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _oversampled(N_t, sigma):
    """n_t: the smallest even 2,3,5,7-smooth integer >= sigma N_t (the
    library's rule, nfft_plan_params)."""
    n = max(int(np.ceil(sigma * N_t - 1e-9)), 2)
    while True:
        r = n
        for p in (2, 3, 5, 7):
            while r % p == 0:
                r //= p
        if n % 2 == 0 and r == 1:
            return n
        n += 1


def _cells(N, sigma):
    return int(np.prod([_oversampled(n, sigma) for n in N]))


def _stage_hbm_bytes(stage, N, M, sigma=SIGMA, real=4, nrhs=1):
    """Algorithmic HBM bytes of one launch of a stage: each point's d offsets
    and value once per pass, the oversampled grid once per pass, two passes
    per FFT, I_N once per scaling pass.  The sort reads x (8 B per
    coordinate) once and writes the sorted record (d offsets, the cell and
    the point's index).  Index and cell words that the kernels also read
    (perm, packed cell: 8 B per point per pass) are implementation traffic,
    visible in the measured DRAM bytes, not algorithmic."""
    d = len(N)
    NN = int(np.prod(N))
    cells = _cells(N, sigma)
    cz = 2 * real
    rec = d * real
    return {
        "spread": M * (rec + cz * nrhs) + cells * cz * nrhs,
        "interp": M * (rec + cz * nrhs) + cells * cz * nrhs,
        "fft": 2 * cells * cz * nrhs,
        "ifft": 2 * cells * cz * nrhs,
        "deconv": 2 * NN * cz * nrhs,
        "pad": (cells + NN) * cz * nrhs,
        "sort": M * (8 * d + 8 + rec),
    }[stage]


def _transform_bytes(N, M, sigma=SIGMA, nrhs=1, real=4, sort=True, adjoint=True, forward=True, ewald=False):
    """Algorithmic HBM bytes of one transform's stages (the terms of
    _stage_hbm_bytes).  An Ewald adjoint reads its weighted modes once
    instead of writing fhat."""
    NN = int(np.prod(N))
    cz = 2 * real
    st = lambda k: _stage_hbm_bytes(k, N, M, sigma, real, nrhs)   # noqa: E731
    b = 0
    if sort:
        b += st("sort")
    if adjoint:
        b += st("spread") + st("fft") + (NN * cz if ewald else st("deconv"))
    if forward:
        b += st("pad") + st("ifft") + st("interp")
    return b


def _step_roofline(bytes_per_step, ms, note):
    """Whole-step HBM roofline (workloads without per-stage events)."""
    peaks, kind = _peaks()
    achieved = bytes_per_step / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "whole step", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_kind": kind, "traffic": None, "step_hbm_bytes": bytes_per_step,
            "note": note}


def _cpu_baseline(args, wl, rank, world):
    if rank != 0 or world != 1 or args.no_cpu_baseline:
        return None
    v, threads, desc = _oracle_sample(wl)
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# a stage's kernels, from an ncu capture, valid while the kernels' sources
# hash to `sources`; otherwise the traffic is reported null.  Keyed by
# (workload, stage); "scaled" says when a smaller case was captured and its
# bytes scaled by the units processed.
TRAFFIC = {
    # the spreading launch of the largest configuration (N = 256^3, M = 3e7 clustered, 6 taps, autotuned),
    # profiles/launches_largest_3d_n256_m3e7.md
    ("picker", "spread"): {"bytes": 3527202816,
                           "sources": "c81048f3d0ca6b3a5813d50ac739fc51ee0a70e1ac58ed1c01567ad4a6423b23"},
    ("picker", "interp"): {"bytes": 2631691520,
                           "sources": "c81048f3d0ca6b3a5813d50ac739fc51ee0a70e1ac58ed1c01567ad4a6423b23"},
}
TRAFFIC_SOURCES = ("points_planes.cuh", "points_tiled.cuh", "points_gm.cuh", "kernels.h", "common.cuh")


def _sources_hash():
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2001_01583_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic(workload, stage):
    rec = TRAFFIC.get((workload, stage))
    if not rec or rec["sources"] != _sources_hash():
        return None
    return rec["bytes"]


STAGE_KERNELS = {"spread": "k_spread_planes (dense bins) + k_spread_gm (sparse bins), after a grid memset",
                 "interp": "k_interp_groups (dense bins) + k_interp_gm (sparse bins)",
                 "sort": "k_bin_count + k_scan + k_scatter + subproblem kernels",
                 "fft": "cuFFT C2C", "ifft": "cuFFT C2C", "deconv": "k_deconv_crop", "pad": "k_pad_deconv"}


def _roofline(stages, workload, geom, peaks, kind, sms):
    """The dominant stage's algorithmic HBM bytes per launch over its mean
    CUDA-event duration in the timed region, against the measured copy
    bandwidth; the spreading and interpolation stages also against the
    shared-memory pipe (a derived peak) and the FP32 pipe."""
    N, M, sigma, taps, real = geom
    total = {k: v[0] for k, v in stages.items() if v[1] > 0}
    per_launch = {k: v[0] / v[1] for k, v in stages.items() if v[1] > 0}
    dom = max(total, key=total.get)
    t = per_launch[dom] * 1e-3
    alg = _stage_hbm_bytes(dom, N, M, sigma, real)
    achieved = alg / t / 1e9
    r = {"bound": "hbm", "kernel": dom, "kernels": STAGE_KERNELS.get(dom), "achieved": achieved,
         "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
         "peak_kind": "%s (MEASURED_PEAKS.json hbm_gbs)" % kind if kind == "measured" else kind,
         "algorithmic_bytes_per_launch": alg, "launch_ms": per_launch[dom],
         "traffic": _traffic(workload, dom),
         "stage_share": {k: round(v / sum(total.values()), 4) for k, v in total.items()},
         "stage_hbm_frac": {k: round(_stage_hbm_bytes(k, N, M, sigma, real) / (per_launch[k] * 1e-3) / 1e9 /
                                     peaks["hbm_gbs"], 4) for k in per_launch if per_launch[k] > 0},
         "stage_launch_ms": {k: round(v, 5) for k, v in per_launch.items()}}
    for st in ("spread", "interp"):
        if st not in per_launch:
            continue
        ts = per_launch[st] * 1e-3
        visits = M * taps ** len(N)
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = sms * SMEM_BYTES_PER_CLK_PER_SM * mhz * 1e6 / 1e9
        ach = visits * SMEM_BYTES_PER_CELL[st] / ts / 1e9
        # a complex value times a real weight added into a complex cell is two
        # FMAs (4 flops) per update, against 128 FP32 lanes x 2 flops per clock per SM
        r["smem_pipe_" + st] = {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                "peak_kind": "derived: %d SMs x 128 B/clk x %.0f MHz" % (sms, mhz),
                                "cell_updates_per_s": visits / ts,
                                "alu_fp32_frac": visits * 4 / ts / (sms * 128 * 2 * mhz * 1e6)}
    return r


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons, sampled during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _workload_inputs(wl, rank):
    """The seeded synthetic inputs of a plan workload: one point set per
    entry of wl["sets"], the values f (M complex) and fhat (N complex)."""
    from paper_2001_01583_gb300 import inputs
    N, M = wl["N"], wl.get("M")
    sd = wl.get("seeds", dict(x=tuple(range(len(wl["sets"]))), f=7, fh=8))
    gens = {"uniform": lambda s: inputs.uniform_points(M, len(N), seed=s),
            "clustered": lambda s: inputs.clustered_points(M, 3, 32, 0.02, seed=s),
            "clustered64": lambda s: inputs.clustered_points(M, 3, 64, 0.01, seed=s)}
    xs = [gens[name](100 * rank + sd["x"][i]) for i, name in enumerate(wl["sets"])]
    return xs, sd


def _oracle_sample(wl, seconds_target=15.0, xs=None, f=None, fh=None):
    """Time the FP64 direct NDFT (the oracle, as it stands) on the host cores
    for a bounded sample of the workload: the adjoint over all of I_N and the
    forward, both at the first points of the workload's first point set.
    Returns (points/s, threads, text)."""
    from oracle import ndft
    from paper_2001_01583_gb300 import inputs
    # the batch samples its largest item (N = 64^3, M = 1e5)
    N, M = wl["N"] or (64, 64, 64), wl["M"] or 100000
    if xs is not None:
        x = xs[0]
    elif "fluorite" in wl["sets"]:
        r, _, L = inputs.fluorite(wl.get("lc", 32))
        x = inputs.box_points(r, L)
    elif wl.get("seeds"):
        x = _workload_inputs(wl, 0)[0][0]
    else:
        x = inputs.uniform_points(M, len(N), seed=0)
    M = x.shape[0]
    f = inputs.complex_normal(M, seed=1) if f is None else np.asarray(f, dtype=np.complex128)
    fh = inputs.complex_normal(N, seed=2) if fh is None else np.asarray(fh, dtype=np.complex128)
    threads = ndft.threads_used(0)
    m0 = 16
    t0 = time.perf_counter()
    ndft.adjoint(x[:m0], f[:m0], N)
    ndft.forward(x[:m0], fh, N)
    dt = max(time.perf_counter() - t0, 1e-3)
    ms = int(min(M, max(m0, m0 * seconds_target / dt)))
    t0 = time.perf_counter()
    ndft.adjoint(x[:ms], f[:ms], N)
    ndft.forward(x[:ms], fh, N)
    dt = time.perf_counter() - t0
    return 2 * ms / dt, threads, "direct NDFT adjoint (all of I_N = %s) + forward at the first %d of the workload's " \
                                 "points, FP64, %d threads, %.1f s" % ("x".join(map(str, N)), ms, threads, dt)


def _oracle_check(x, f, fh, N, samples):
    """The relative l2 error (Eq. 9) of timed GPU outputs at sampled outputs
    against the direct NDFT (the oracle): samples maps a label to
    (ks, adjoint values at ks, js, forward values at js).  Part of the CPU
    oracle leg, after the timed region."""
    from oracle import ndft
    out = {}
    f64 = np.asarray(f, dtype=np.complex128)
    fh64 = np.asarray(fh, dtype=np.complex128)
    refs = {}
    for label, (ks, ga, js, gb) in samples.items():
        key = (ks.tobytes(), js.tobytes())
        if key not in refs:
            refs[key] = (ndft.adjoint(x, f64, N, ksel=ks), ndft.forward(x, fh64, N, jsel=js))
        ra, rb = refs[key]
        out[label] = {"adjoint": ndft.rel_l2(ga, ra), "forward": ndft.rel_l2(gb, rb)}
    return out


def run_reference(args, wl, rank, world):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return 0
    vals, desc, threads = [], "", 0
    xs = None
    if wl.get("seeds"):
        xs, _ = _workload_inputs(wl, 0)
    for i in range(args.warmup + args.steps):
        v, threads, desc = _oracle_sample(wl, seconds_target=6.0 if i >= args.warmup else 1.0, xs=xs)
        if i >= args.warmup:
            vals.append(v)
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"] + " (oracle: FP64 direct NDFT on a bounded sample of the points)",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_plans(step, plans, stream, dev, steps, warmup, flush, world, profile):
    """W warm-up steps, then K steps bracketed by a barrier and a device
    synchronize, each between CUDA events on the plans' stream (L2 flushed
    between steps, outside the events).  With `profile` the plans record
    per-stage events during the timed steps.  Returns (ms per step, clocks,
    kernels launched, per-stage (ms, launches))."""
    import torch
    import torch.distributed as dist
    from paper_2001_01583_gb300 import _lib
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    for p in plans:
        p.sync()
        p.set_option(_lib.OPT_PROFILE, 1 if profile else 0)
        p.stage_times(reset=True)
    sampler = ClockSampler(dev.index)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = sum(p.info()["kernel_launches"] for p in plans)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.nvtx.range_push("bench_timed")   # lets a profiler select the timed steps' kernels
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(float(i))          # evict L2 between timed steps, outside the step's events
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = sum(p.info()["kernel_launches"] for p in plans) - launches0
    stages = {}
    for p in plans:
        p.sync()
        for k, (ms, n) in p.stage_times(reset=True).items():
            acc = stages.setdefault(k, [0.0, 0])
            acc[0] += ms
            acc[1] += n
        p.set_option(_lib.OPT_PROFILE, 0)
    return float(np.sum([a.elapsed_time(b) for a, b in ev])) / steps, clocks, launches, stages


def run_ours(args, wl, rank, world):
    """The plan workloads (3-D configuration, the largest configuration with
    picked parameters, and the small and sparse profiling cases): every step
    runs set_points, the adjoint and the forward NFFT on each point set."""
    import torch
    import torch.distributed as dist

    from paper_2001_01583_gb300 import Plan, _lib, inputs

    N, M = wl["N"], wl["M"]
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _lib.load()   # fails loudly if the CUDA library was not built
    stream = torch.cuda.Stream(dev)

    # inputs: every rank its own seeds (independent problems)
    xs_host, sd = _workload_inputs(wl, rank)
    ctype = np.complex64 if args.precision == "fp32" else np.complex128
    tctype = torch.complex64 if args.precision == "fp32" else torch.complex128
    f_host = inputs.complex_normal(M, seed=100 * rank + sd["f"], dtype=ctype)
    fh_host = inputs.complex_normal(N, seed=100 * rank + sd["fh"], dtype=ctype)

    # window parameters: the learned picker's for the largest configuration,
    # the stated ones otherwise; the rule of thumb for the plain FP64 form
    params = (SIGMA, MCUT, WINDOW)
    extra = {}
    if wl.get("picked"):
        from paper_2001_01583_gb300 import picker
        pk = picker.load_default(stream=stream)
        s_, m_, w_, fb = pk.pick(N, M, 0.01, wl["eps"], precision=args.precision)
        rs, rm, rw = picker.rule_of_thumb(wl["eps"])
        wname = lambda w: "gaussian" if w == 0 else "kaiser_bessel"   # noqa: E731
        params = (s_, m_, wname(w_))
        rule = (rs, rm, wname(rw))
        pk.mlp.close()
        extra["picked"] = {"sigma": s_, "m": m_, "window": wname(w_), "fallback": fb}
        extra["rule_of_thumb"] = {"sigma": rs, "m": rm, "window": wname(rw)}
        extra["eps"] = wl["eps"]
    else:
        rule = params
    sigma, mcut, window = params

    with torch.cuda.stream(stream):
        xs = [torch.from_numpy(x).to(dev) for x in xs_host]
        f = torch.from_numpy(f_host).to(dev)
        fh = torch.from_numpy(fh_host).to(dev)
        outs_a = [torch.empty((1,) + N, dtype=tctype, device=dev) for _ in xs]
        outs_f = [torch.empty((1, M), dtype=tctype, device=dev) for _ in xs]
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2
    plans = [Plan(N, M, sigma, mcut, window, args.precision, stream=stream) for _ in xs]
    for p in plans:
        if args.tensor_spread:
            p.set_option(_lib.OPT_TENSOR_SPREAD, 1)
        if args.tensor_interp:
            p.set_option(_lib.OPT_TENSOR_INTERP, 1)
    if args.autotune:
        # the library's autotuner, once per point set, outside the timed region
        with torch.cuda.stream(stream):
            for p, x in zip(plans, xs):
                p.set_points(x)
                p.autotune(reps=3)
    info = plans[0].info()
    taps = info["taps"]

    def step():
        for p, x, a, b in zip(plans, xs, outs_a, outs_f):
            p.set_points(x)
            p.adjoint(f, out=a)
            p.forward(fh, out=b)

    ms_per_step, clocks, launches_timed, stages = _time_plans(step, plans, stream, dev, args.steps, args.warmup,
                                                              flush, world, profile=True)

    # sampled outputs of the timed steps, for the relative l2 error against
    # the direct NDFT (computed in the oracle leg below)
    rng = np.random.default_rng(12345)
    nk, nj = (128, 128) if M >= 10 ** 7 else (64, 64)
    ks = np.stack([rng.integers(-n // 2, n // 2, size=nk) for n in N], axis=1)
    js = rng.integers(0, M, size=nj)
    kidx = tuple(torch.from_numpy(ks[:, t] + N[t] // 2).to(dev) for t in range(len(N)))
    jidx = torch.from_numpy(js).to(dev)
    samples = {}
    for name, a, b in zip(wl["sets"], outs_a, outs_f):
        samples[name] = (ks, a[0][kidx].cpu().numpy(), js, b[0][jidx].cpu().numpy())

    # end to end through the public API with host buffers (pinned): inputs
    # copied in and results copied out inside the timed region, every step
    xs_pin = [torch.from_numpy(x).pin_memory() for x in xs_host]
    f_pin = torch.from_numpy(f_host).pin_memory()
    fh_pin = torch.from_numpy(fh_host).pin_memory()
    # results land in pinned host buffers, asynchronously on the plans' stream
    # (the synchronize after each step waits for them)
    oa_pin = [torch.empty((1,) + N, dtype=tctype).pin_memory() for _ in xs]
    of_pin = [torch.empty((1, M), dtype=tctype).pin_memory() for _ in xs]
    h2d = sum(x.numel() * 8 for x in xs_pin) + f_pin.numel() * f_pin.element_size() + \
        fh_pin.numel() * fh_pin.element_size()
    d2h = sum(t.numel() * t.element_size() for t in oa_pin + of_pin)

    def e2e_step():
        for p, x, oa, of in zip(plans, xs_pin, oa_pin, of_pin):
            p.set_points(x)
            p.adjoint(f_pin, out=oa)
            p.forward(fh_pin, out=of)

    with torch.cuda.stream(stream):
        e2e_step()
    for p in plans:
        p.sync()
    torch.cuda.synchronize(dev)
    e_ms = []
    for i in range(max(3, min(args.steps, 5))):
        flush.fill_(float(i))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            e2e_step()
        for p in plans:
            p.sync()
        torch.cuda.synchronize(dev)
        e_ms.append((time.perf_counter() - t0) * 1e3)
    del xs_pin, oa_pin, of_pin
    for p in plans:
        p.close()
    del outs_a, outs_f

    # the other forms of the same workload on the same GPU, timed the same
    # way: the rule-of-thumb parameters in the same precision (when the
    # picker chose others) and the plain FP64 form (rule-of-thumb parameters)
    forms = {}
    form_list = []
    if wl.get("picked") and rule != params:
        form_list.append(("rule_of_thumb_" + args.precision, rule, args.precision))
    if args.precision == "fp32" and not args.no_fp64_form:
        form_list.append(("plain_fp64", rule, "fp64"))
    for label, (fs_, fm_, fw_), prec in form_list:
        cdt = torch.complex64 if prec == "fp32" else torch.complex128
        with torch.cuda.stream(stream):
            fo = f.to(cdt)
            fho = fh.to(cdt)
            oa = [torch.empty((1,) + N, dtype=cdt, device=dev) for _ in xs]
            ob = [torch.empty((1, M), dtype=cdt, device=dev) for _ in xs]
        fplans = [Plan(N, M, fs_, fm_, fw_, prec, stream=stream) for _ in xs]
        if args.autotune:
            with torch.cuda.stream(stream):
                for p, x in zip(fplans, xs):
                    p.set_points(x)
                    p.autotune(reps=2 if prec == "fp64" else 3)

        def fstep(fplans=fplans, fo=fo, fho=fho, oa=oa, ob=ob):
            for p, x, a, b in zip(fplans, xs, oa, ob):
                p.set_points(x)
                p.adjoint(fo, out=a)
                p.forward(fho, out=b)
        fms, _, _, _ = _time_plans(fstep, fplans, stream, dev, max(3, args.steps // 4), 3, flush, world,
                                   profile=False)
        for name, a, b in zip(wl["sets"], oa, ob):
            samples[label + ":" + name] = (ks, a[0][kidx].cpu().numpy(), js, b[0][jidx].cpu().numpy())
        forms[label] = {"sigma": fs_, "m": fm_, "window": fw_, "precision": prec, "ms_per_step": fms,
                        "value": len(xs) * 2 * M * world / (fms * 1e-3)}
        for p in fplans:
            p.close()
        del fo, fho, oa, ob
        torch.cuda.empty_cache()

    points_per_step = len(xs) * 2 * M
    t = torch.tensor([ms_per_step, float(np.median(e_ms))] + [v["ms_per_step"] for v in forms.values()],
                     dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tl = t.tolist()
    ms_max, e2e_max = tl[0], tl[1]
    for k, v in zip(forms, tl[2:]):
        forms[k]["ms_per_step"] = v
        forms[k]["value"] = points_per_step * world / (v * 1e-3)
    value = points_per_step * world / (ms_max * 1e-3)
    e2e_value = points_per_step * world / (e2e_max * 1e-3)

    peaks, kind = _peaks()
    props = torch.cuda.get_device_properties(dev)
    real = 4 if args.precision == "fp32" else 8
    roofline = _roofline(stages, args.workload, (N, M, sigma, taps, real), peaks, kind,
                         props.multi_processor_count)
    hbm_step = len(xs) * _transform_bytes(N, M, sigma, 1, real)
    roofline["step_hbm_bytes"] = hbm_step
    roofline["step_hbm_frac"] = hbm_step / (ms_max * 1e-3) / 1e9 / peaks["hbm_gbs"]

    # the CPU oracle leg (rank 0, one GPU): the timed baseline on a bounded
    # sample, then the relative l2 error of the sampled timed outputs
    cpu, rel = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, threads, desc = _oracle_sample(wl, xs=xs_host, f=f_host, fh=fh_host)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}
        errs = {}
        for i, name in enumerate(wl["sets"]):
            sub = {k: v_ for k, v_ in samples.items() if k == name or k.endswith(":" + name)}
            errs.update(_oracle_check(xs_host[i], f_host, fh_host, N, sub))
        rel = {"value": max(max(e.values()) for k, e in errs.items() if ":" not in k),
               "target": wl.get("eps", 1e-6),
               "per_output": {k: e for k, e in errs.items() if ":" not in k},
               "sample": "direct NDFT (the oracle, FP64) at %d frequencies of I_N (adjoint) and %d points "
                         "(forward), drawn uniformly with seed 12345, per point set, from the last timed step's "
                         "outputs" % (nk, nj)}
        for k, e in errs.items():
            if ":" in k:
                label, _ = k.split(":", 1)
                forms[label].setdefault("rel_l2", {})[k.split(":", 1)[1]] = e

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "rel_l2": rel["value"] if rel else None,
            "config": {"workload": wl["name"], "points_per_step_per_gpu": points_per_step,
                       "precision": args.precision, "sigma": sigma, "m": mcut, "window": window, "taps": taps,
                       "autotuned": bool(args.autotune), "tensor_spread": bool(info.get("tensor_spread")),
                       "tensor_interp": bool(info.get("tensor_interp")),
                       "autotuned_layout": {k: info[k] for k in ("bin", "max_subproblem", "spread_block_threads",
                                                                 "interp_block_threads", "sparse_points",
                                                                 "sparse_points_interp")},
                       "l2": "flushed between timed steps (512 MB write outside the step events); inputs and "
                             "grid larger than L2",
                       "stage_events": "per-stage CUDA events on the plans' stream during the timed steps",
                       "parallelism": "independent replicas x%d" % world},
            "rel_l2_detail": rel,
            "other_forms": forms,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_timed,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks}
    line["config"].update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_batch(args, wl, rank, world):
    """The batch workload: every step is one adjoint and one forward graph
    launch over all 513 items (independent problems per rank)."""
    import torch
    import torch.distributed as dist

    from paper_2001_01583_gb300 import Batch, _lib, inputs

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _lib.load()
    stream = torch.cuda.Stream(dev)
    ctype = np.complex64 if args.precision == "fp32" else np.complex128
    items = inputs.batch_items(512, N_choices=(32, 64), M_lo=1000, M_hi=100000, d=3, seed=100 * rank)
    items = [dict(N=it["N"], M=it["M"], nrhs=1, seed=it["seed"]) for it in items]
    items.append(dict(N=(64, 64, 64), M=200000, nrhs=16, seed=100 * rank + 99))
    with torch.cuda.stream(stream):
        xs = [torch.from_numpy(inputs.uniform_points(it["M"], 3, seed=it["seed"])).to(dev) for it in items]
        fs = [torch.from_numpy(inputs.complex_normal((it["nrhs"], it["M"]), seed=it["seed"] + 1, dtype=ctype)).to(dev)
              for it in items]
        hs = [torch.from_numpy(inputs.complex_normal((it["nrhs"],) + it["N"], seed=it["seed"] + 2,
                                                     dtype=ctype)).to(dev) for it in items]
        outs_a = [torch.empty_like(h) for h in hs]
        outs_f = [torch.empty_like(f) for f in fs]
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    b = Batch([dict(N=it["N"], M=it["M"], nrhs=it["nrhs"]) for it in items], args.precision, stream=stream)
    if args.owner_spread:
        b.set_option(_lib.OPT_OWNER_SPREAD, 1)
    with torch.cuda.stream(stream):
        b.set_points(xs)
        if args.autotune:
            b.autotune(reps=3)
        for _ in range(args.warmup):
            b.adjoint(fs, outs_a)
            b.forward(hs, outs_f)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    sampler.start()
    launches0 = b.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            b.adjoint(fs, outs_a)
            b.forward(hs, outs_f)
            ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    launches_timed = b.kernel_launches() - launches0
    clocks = sampler.stop()
    ms = float(np.sum([x.elapsed_time(y) for x, y in ev])) / args.steps
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = t.item()
    points = 2 * sum(it["M"] * it["nrhs"] for it in items)
    line = {"metric": METRIC, "value": points * world / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": wl["name"], "points_per_step_per_gpu": points, "items": len(items),
                       "precision": args.precision, "autotuned": bool(args.autotune),
                       "owner_spread": bool(args.owner_spread),
                       "l2": "flushed between timed steps (512 MB write outside the step events)"},
            "gpu_launches": launches_timed, "clocks": clocks}
    real = 4 if args.precision == "fp32" else 8
    hbm = sum(_transform_bytes(it["N"], it["M"], SIGMA, it["nrhs"], real, sort=False) for it in items)
    line["roofline"] = _step_roofline(hbm, ms, "one adjoint and one forward per item (points sorted outside the "
                                               "step); per-kernel roofline in the 3-D workloads")
    line["cpu_baseline"] = _cpu_baseline(args, wl, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    return 0


def _timed(step, stream, dev, steps, warmup, flush, plans=()):
    """Device ms per step (CUDA events on the stream, L2 flushed between
    steps outside the events), the clocks seen meanwhile and this library's
    kernels launched by `plans` inside the timed region."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index)
    launches0 = sum(p.info()["kernel_launches"] for p in plans)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    launches = sum(p.info()["kernel_launches"] for p in plans) - launches0
    return float(np.sum([a.elapsed_time(b) for a, b in ev])) / steps, clocks, launches


def run_extra(args, wl, rank, world):
    """The other configurations: 1-D FP64 and the fluorite Ewald energy."""
    import torch
    import torch.distributed as dist

    from paper_2001_01583_gb300 import Plan, _lib, inputs

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _lib.load()
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    N, M = wl["N"], wl["M"]
    extra, points_per_step = {}, 0
    prec = args.precision
    if args.workload == "1d":
        prec = "fp64"
        x = torch.from_numpy(inputs.uniform_points(M, 1, seed=100 * rank)).to(dev)
        f = torch.from_numpy(inputs.complex_normal(M, seed=100 * rank + 1)).to(dev)
        fh = torch.from_numpy(inputs.complex_normal(N, seed=100 * rank + 2)).to(dev)
        plan = Plan(N, M, 2.0, 6, "gaussian", "fp64", stream=stream)
        oa, of = torch.empty((1,) + N, dtype=torch.complex128, device=dev), torch.empty((1, M), dtype=torch.complex128,
                                                                                          device=dev)

        def step():
            plan.set_points(x)
            plan.adjoint(f, out=oa)
            plan.forward(fh, out=of)
        points_per_step = 2 * M
        plans = [plan]
    elif args.workload == "fluorite":
        r, q, L = inputs.fluorite(32)
        xq = torch.from_numpy(inputs.box_points(r, L)).to(dev)
        qd = torch.from_numpy(q.astype(np.complex128 if prec == "fp64" else np.complex64)).to(dev)
        plan = Plan(N, len(q), 2.0, 6, "kaiser_bessel", prec, stream=stream)
        out = {}
        if args.autotune:
            with torch.cuda.stream(stream):
                plan.set_points(xq)
                plan.autotune(reps=3)

        def step():
            plan.set_points(xq)
            out["e"] = plan.ewald_reciprocal(qd, L, 0.6)
        points_per_step = len(q)
        plans = [plan]
    ms, clocks, launches = _timed(step, stream, dev, args.steps, args.warmup, flush, plans=plans[:1])
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = t.item()
    if args.workload == "fluorite":
        # Eq. 11 on the GPU as well (cell list, cut-off 10 r0: erfc(6) ~ 2e-17),
        # timed apart: the whole Madelung constant (Eq. 10) from the GPU
        from paper_2001_01583_gb300 import ewald_real_space
        rd = torch.from_numpy(r).to(dev)
        qr = torch.from_numpy(q.astype(np.float64)).to(dev)
        ewald_real_space(rd, qr, L, 0.6, 10.0, stream=stream)
        rs_ms = []
        for _ in range(max(3, args.steps // 4)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ur = ewald_real_space(rd, qr, L, 0.6, 10.0, stream=stream)
            e1.record(stream)
            e1.synchronize()
            rs_ms.append(e0.elapsed_time(e1))
        madelung = (ur + out["e"][0]) * 3 / (len(q) * 2 * -1)
        extra = {"reciprocal_energy": out["e"], "alpha": 0.6, "L": float(L),
                 "real_space": {"energy": ur, "rcut": 10.0, "ms": float(np.median(rs_ms))},
                 "madelung": madelung}
    cfg = {"workload": wl["name"], "points_per_step_per_gpu": points_per_step, "precision": prec,
           "autotuned": bool(args.autotune) and args.workload == "fluorite",
           "l2": "flushed between timed steps (512 MB write outside the step events)",
           "parallelism": "independent replicas x%d" % world}
    cfg.update(extra)
    line = {"metric": METRIC, "value": points_per_step * world / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
            "data": "synthetic", "config": cfg, "gpu_launches": launches, "clocks": clocks}
    real = 4 if prec == "fp32" else 8
    if args.workload == "fluorite":
        hbm = _transform_bytes(N, points_per_step, SIGMA, 1, real, forward=False, ewald=True)
    else:
        hbm = _transform_bytes(N, M, SIGMA, 1, real)
    line["roofline"] = _step_roofline(hbm, ms, "set_points and the transforms of one step; per-kernel roofline "
                                               "in the 3-D workloads")
    line["cpu_baseline"] = _cpu_baseline(args, wl, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    return 0


def run_sweep(args, wl, rank, world):
    """The single-GPU counterparts of the paper's runtime sweeps (Fig. 13:
    NFFT of 58^3 ... 120^3 points; Fig. 16: fluorite energies of
    12 x {32 ... 64}^3 ions): every size timed like the other workloads,
    one line whose value is the largest size's throughput."""
    import torch
    import torch.distributed as dist

    from paper_2001_01583_gb300 import Plan, _lib, inputs

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _lib.load()
    stream = torch.cuda.Stream(dev)
    prec = args.precision
    ctype = np.complex64 if prec == "fp32" else np.complex128
    real = 4 if prec == "fp32" else 8
    with torch.cuda.stream(stream):
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    steps = max(3, args.steps // 4)
    rows, clocks_all, launches_all = [], [], 0
    if args.workload == "fig13":
        cases = [((n,) * 3, side ** 3) for n in (64, 128) for side in (58, 80, 100, 120)]
    else:
        cases = [((128,) * 3, lc) for lc in (32, 45, 56, 64)]
    for N, size in cases:
        if args.workload == "fig13":
            M = size
            x = torch.from_numpy(inputs.uniform_points(M, 3, seed=100 * rank + size % 97)).to(dev)
            f = torch.from_numpy(inputs.complex_normal(M, seed=100 * rank + 1, dtype=ctype)).to(dev)
            fh = torch.from_numpy(inputs.complex_normal(N, seed=100 * rank + 2, dtype=ctype)).to(dev)
            plan = Plan(N, M, SIGMA, MCUT, WINDOW, prec, stream=stream)
            oa = torch.empty(N, dtype=f.dtype, device=dev)
            of = torch.empty(M, dtype=f.dtype, device=dev)
            if args.autotune:
                with torch.cuda.stream(stream):
                    plan.set_points(x)
                    plan.autotune(reps=3)

            def step():
                plan.set_points(x)
                plan.adjoint(f, out=oa)
                plan.forward(fh, out=of)
            units = 2 * M
            hbm = _transform_bytes(N, M, SIGMA, 1, real)
            row = {"N": N[0], "M": M, "points": "%d^3" % round(M ** (1 / 3))}
        else:
            r, q, L = inputs.fluorite(size)
            M = len(q)
            x = torch.from_numpy(inputs.box_points(r, L)).to(dev)
            qd = torch.from_numpy(q.astype(ctype)).to(dev)
            plan = Plan(N, M, SIGMA, 6, WINDOW, prec, stream=stream)
            out = {}
            if args.autotune:
                with torch.cuda.stream(stream):
                    plan.set_points(x)
                    plan.autotune(reps=3)

            def step():
                plan.set_points(x)
                out["e"] = plan.ewald_reciprocal(qd, L, 0.6)
            units = M
            hbm = _transform_bytes(N, M, SIGMA, 1, real, forward=False, ewald=True)
            row = {"N": N[0], "cells": size, "ions": M}
        ms, clocks, launches = _timed(step, stream, dev, steps, args.warmup, flush, plans=[plan])
        if args.workload == "fig16":
            row["reciprocal_energy"] = out["e"][0]
        row.update(ms_per_step=ms, units_per_s=units / (ms * 1e-3),
                   step_hbm_frac=hbm / (ms * 1e-3) / 1e9 / _peaks()[0]["hbm_gbs"])
        rows.append(row)
        clocks_all.append(clocks)
        launches_all += launches
        plan.close()
        del x
        torch.cuda.empty_cache()
    t = torch.tensor([rows[-1]["ms_per_step"]], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = t.item()
    units = 2 * cases[-1][1] if args.workload == "fig13" else rows[-1]["ions"]
    sm = [c["sm_mhz"] for c in clocks_all if c.get("sm_mhz")]
    clocks = {"sm_mhz": float(np.median(sm)) if sm else None,
              "sm_max_mhz": max((c.get("sm_max_mhz") or 0) for c in clocks_all) or None,
              "reasons": sorted({r_ for c in clocks_all for r_ in c.get("reasons", [])}),
              "samples": sum(c.get("samples", 0) for c in clocks_all)}
    last = cases[-1]
    hbm = _transform_bytes(last[0], last[1], SIGMA, 1, real) if args.workload == "fig13" else \
        _transform_bytes(last[0], rows[-1]["ions"], SIGMA, 1, real, forward=False, ewald=True)
    line = {"metric": METRIC, "value": units * world / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": wl["name"], "precision": prec, "autotuned": bool(args.autotune),
                       "l2": "flushed between timed steps (512 MB write outside the step events)",
                       "parallelism": "independent replicas x%d" % world, "sweep": rows},
            "gpu_launches": launches_all, "clocks": clocks,
            "roofline": _step_roofline(hbm, ms, "largest size of the sweep, whole step; per-kernel roofline in "
                                                "the 3-D workloads"),
            "cpu_baseline": _cpu_baseline(args, wl, rank, world)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--tensor-spread", action="store_true",
                    help="plan workloads: spread the dense bins on the tensor cores (NFFT_OPT_TENSOR_SPREAD)")
    ap.add_argument("--tensor-interp", action="store_true",
                    help="plan workloads: interpolate the dense bins on the tensor cores (NFFT_OPT_TENSOR_INTERP)")
    ap.add_argument("--owner-spread", action="store_true",
                    help="batch workload: spread sparse bins by their cells' owners (NFFT_OPT_OWNER_SPREAD)")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip timing the plain FP64 form of the plan workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the library's autotuner (run by default before timing, outside the timed region)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.workload]
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        if args.workload == "batch":
            return run_batch(args, wl, rank, world)
        if wl.get("sweep"):
            return run_sweep(args, wl, rank, world)
        if wl.get("extra"):
            return run_extra(args, wl, rank, world)
        return run_ours(args, wl, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
