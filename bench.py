"""Throughput benchmark of the GB300 NFFT library.

Workload (one "step"): the 3-D configuration N = 64^3, M = 10^6, Kaiser-Bessel
window m = 4, sigma = 2, mixed FP32 form, on two point sets (uniform, and 32
Gaussian clusters of std 0.02).  For each set a step runs nfft_set_points
(argument reduction + bin sort), the adjoint NFFT (Eq. 5: spread, FFT, scale)
and the forward NFFT (Eq. 6: subdivide, inverse FFT, interpolate).  Units: a
transform of M points counts M nonuniform points, so a step processes
2 sets x 2 transforms x M points.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
independent copy of the workload (weak scaling, no collective on the data
path); the value is all ranks' points over the slowest rank's time.
"""
import argparse
import json
import math
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
N3 = (64, 64, 64)
M = 10 ** 6
SIGMA, MCUT, WINDOW = 2.0, 4, "kaiser_bessel"
WORKLOAD = "3-D adjoint+forward NFFT, N=64^3, M=10^6, uniform + clustered (32 clusters, std 0.02), KB m=4, sigma=2, FP32 mixed"


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
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


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


def _oracle_sample(seconds_target=15.0):
    """Time the FP64 direct NDFT (the oracle, as it stands) on the host cores
    for a bounded sample of the workload's points: adjoint over all of I_N
    and forward at the same points.  Returns (points/s, threads, description)."""
    from oracle import ndft
    from paper_2001_01583_gb300 import inputs
    x = inputs.uniform_points(M, 3, seed=0)
    f = inputs.complex_normal(M, seed=1)
    fh = inputs.complex_normal(N3, seed=2)
    threads = ndft.threads_used(0)
    # calibrate on a small sample, then size the run to about seconds_target
    m0 = 256
    t0 = time.perf_counter()
    ndft.adjoint(x[:m0], f[:m0], N3)
    ndft.forward(x[:m0], fh, N3)
    dt = max(time.perf_counter() - t0, 1e-3)
    ms = int(min(M, max(m0, m0 * seconds_target / dt)))
    t0 = time.perf_counter()
    ndft.adjoint(x[:ms], f[:ms], N3)
    ndft.forward(x[:ms], fh, N3)
    dt = time.perf_counter() - t0
    # two transforms of ms points each
    return 2 * ms / dt, threads, "direct NDFT adjoint (all of I_N = 64^3) + forward at the first %d of the " \
                                 "uniform points, FP64, %d threads, %.1f s" % (ms, threads, dt)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    steps = []
    desc = ""
    threads = 0
    for i in range(args.warmup + args.steps):
        v, threads, desc = _oracle_sample(seconds_target=6.0 if i >= args.warmup else 2.0)
        if i >= args.warmup:
            steps.append(v)
    value = float(np.median(steps))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist

    from paper_2001_01583_gb300 import Plan, _lib, inputs
    from paper_2001_01583_gb300.build import build as build_lib

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(_lib.LIB_PATH):
        build_lib()
    stream = torch.cuda.Stream(dev)

    # inputs: every rank its own seeds (independent problems)
    xs_host = [inputs.uniform_points(M, 3, seed=100 * rank + 0),
               inputs.clustered_points(M, 3, 32, 0.02, seed=100 * rank + 1)]
    f_host = inputs.complex_normal(M, seed=100 * rank + 2, dtype=np.complex64)
    fh_host = inputs.complex_normal(N3, seed=100 * rank + 3, dtype=np.complex64)

    with torch.cuda.stream(stream):
        xs = [torch.from_numpy(x).to(dev) for x in xs_host]
        f = torch.from_numpy(f_host).to(dev)
        fh = torch.from_numpy(fh_host).to(dev)
        outs_a = [torch.empty(N3, dtype=torch.complex64, device=dev) for _ in xs]
        outs_f = [torch.empty(M, dtype=torch.complex64, device=dev) for _ in xs]
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2
    plans = [Plan(N3, M, SIGMA, MCUT, WINDOW, "fp32", stream=stream) for _ in xs]
    for p in plans:
        p.set_option(_lib.OPT_PROFILE, 1)

    def step():
        for p, x, a, b in zip(plans, xs, outs_a, outs_f):
            p.set_points(x)
            p.adjoint(f, out=a.view((1,) + N3))
            p.forward(fh, out=b.view(1, M))

    # warm-up
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    for p in plans:
        p.sync()
        p.stage_times(reset=True)

    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))          # evict L2 between timed steps (outside the step's events)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_per_step = float(np.sum(step_ms)) / args.steps
    stages = {}
    for p in plans:
        for k, (ms, n) in p.stage_times(reset=True).items():
            s = stages.setdefault(k, [0.0, 0])
            s[0] += ms
            s[1] += n
    for p in plans:
        p.sync()

    # end to end through the public API with host buffers (pinned)
    xs_pin = [torch.from_numpy(x).pin_memory() for x in xs_host]
    f_pin = torch.from_numpy(f_host).pin_memory()
    fh_pin = torch.from_numpy(fh_host).pin_memory()
    h2d = sum(x.numel() * 8 for x in xs_pin) + f_pin.numel() * 8 + fh_pin.numel() * 8
    d2h = len(xs) * (int(np.prod(N3)) * 8 + M * 8)
    for p in plans:
        p.set_option(_lib.OPT_PROFILE, 0)

    def e2e_step():
        res = []
        for p, x in zip(plans, xs_pin):
            p.set_points(x)
            res.append(p.adjoint(f_pin))
            res.append(p.forward(fh_pin))
        return res

    with torch.cuda.stream(stream):
        e2e_step()
    torch.cuda.synchronize(dev)
    e_ms = []
    for i in range(max(2, min(args.steps, 5))):
        flush.fill_(float(i))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            e2e_step()
        torch.cuda.synchronize(dev)
        e_ms.append((time.perf_counter() - t0) * 1e3)

    points_per_step = len(xs) * 2 * M
    t = torch.tensor([ms_per_step, float(np.median(e_ms))], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max, e2e_max = t.tolist()
    value = points_per_step * world / (ms_max * 1e-3)
    e2e_value = points_per_step * world / (e2e_max * 1e-3)

    # roofline of the dominant kernel (largest stage share)
    peaks, kind = _peaks()
    per_kernel = {k: v[0] / max(v[1], 1) for k, v in stages.items() if v[1] > 0}
    total = {k: v[0] for k, v in stages.items()}
    dom = max(total, key=total.get)
    cells = 128 ** 3
    bytes_alg = {
        # sorted point records read (4 B perm + 4 B packed cell + 12 B offsets) + gathered f (8 B) + grid flushed (8 B/cell)
        "spread": M * (20 + 8) + cells * 8,
        "interp": M * (20 + 8) + cells * 8,
        "fft": 2 * 2 * cells * 8,
        "ifft": 2 * 2 * cells * 8,
        "deconv": int(np.prod(N3)) * 8 * 2,
        "pad": cells * 8 + int(np.prod(N3)) * 8,
        "sort": M * (24 + 8 + 24 + 20),
    }
    achieved = bytes_alg.get(dom, 0) / (per_kernel[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": dom,
                "peak_kind": kind, "stage_ms_per_launch": {k: round(v, 5) for k, v in per_kernel.items()}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, threads, desc = _oracle_sample()
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}

    launches_per_step = len(xs) * (6 + 2 + 2)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points_per_step_per_gpu": points_per_step,
                       "l2": "flushed between timed steps (512 MB write, outside the step events)",
                       "parallelism": "replicas x%d" % world},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        return run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
