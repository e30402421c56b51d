"""Benchmark: compact 6th-order derivatives of a 512^3 periodic FP64 field.

One step = the whole hot path over one field: the cyclic tridiagonal
derivative (Lele 6th order, alpha = 1/3) along x (contiguous), y and z
(strided), each = stencil + per-partition solve + FP64 interface PCR +
back-substitution (+ refinement), i.e. 3 x 512^3 unknowns.

The headline path is FP32 bulk + FP64-accurate refinement (one sweep), whose
error against the FP64 oracle is <= 1e-12; the plain FP64 path is timed on
the same field and reported beside it.  Inputs (1 GiB) exceed the 129 MB L2,
so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own 512^3 field (independent lines, no
data exchange: weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 512
LINES_PER_DIR = N * N
UNKNOWNS_PER_STEP = 3 * N ** 3
METRIC = "Gunknowns/s (3 x 512^3 cyclic tridiagonal 6th-order derivatives, x/y/z, <=1e-12 rel err)"
CONFIG = {"workload": "512^3 periodic FP64 field, Lele 6th-order cyclic tridiagonal first derivative "
                      "along x, y and z (3 x 262144 systems of n=512)",
          "grid": [N, N, N], "scheme": "alpha=1/3, a=14/9, b=1/9", "segments": "auto",
          "l2": "inputs (1 GiB FP64) larger than L2; no flush"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--size", type=int, default=N,
                    help="grid points per axis (512 = the benchmark workload; smaller for profiling)")
    return ap.parse_args()


# ---------------------------------------------------------------- ranks
def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the process group (identity when not
    initialised).  Used for the step time: the job is as slow as its slowest
    rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput (units/s x 1e-9) when every rank processes
    units_per_rank in ms_max milliseconds (weak scaling)."""
    return world * units_per_rank / (ms_max * 1e-3) / 1e9


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 7 for k in range(4)
                          if r[3 + k].lower() == "active"})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": reasons}


# ---------------------------------------------------------------- oracle (CPU)
def oracle_sample(seconds: float, seed_lines: int = 1024):
    """Time the FP64 oracle on lines of the same workload (n = 512, x/y/z
    lines of a seeded 512^3 field); returns (Gunknowns/s, cores, sample)."""
    import numpy as np
    import oracle
    from paper_2101_02286_gb300 import workloads as W
    rng = np.random.default_rng(W.SEEDS["cube512"])
    lines = rng.uniform(-1.0, 1.0, size=(seed_lines, N))
    h = W.grid_spacing(N)
    oracle.derivative(lines[:8], W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], h)  # warm-up
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.derivative(lines, W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], h)
        done += seed_lines * N
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done / el / 1e9, oracle.num_threads(), \
        "%d solves of %d lines x n=512 (x/y/z lines are identical 1-D systems), %.1f s" % (
            done // (seed_lines * N), seed_lines, el)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2101_02286_gb300 import workloads as W
    rng = np.random.default_rng(W.SEEDS["cube512"])
    sample_lines = 2048
    lines = rng.uniform(-1.0, 1.0, size=(3, sample_lines, N))
    h = W.grid_spacing(N)
    for _ in range(args.warmup):
        for d in range(3):
            oracle.derivative(lines[d], W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], h)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for d in range(3):
            oracle.derivative(lines[d], W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], h)
    el = time.perf_counter() - t0
    unk = 3 * sample_lines * N * args.steps
    val = unk / el / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Gunknowns/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": val, "unit": "Gunknowns/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "per step: x, y and z derivatives of %d seeded lines of n=512 each" % sample_lines},
        "e2e": {"value": val, "unit": "Gunknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------- GPU
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2101_02286_gb300 import workloads as W
    from paper_2101_02286_gb300.solver import Plan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    n = args.size
    f_host, modes = W.noisy_cube(n)  # seeded: U(-1,1) + one plane wave
    f_pin = torch.from_numpy(f_host).pin_memory()
    f = f_pin.to(dev)
    h = W.grid_spacing(n)
    sch = W.LELE6_TRI

    def make(prec):
        return [Plan(f.shape, d, lhs=sch["lhs"], rhs=sch["rhs"], h=h, precision=prec, sweeps=1) for d in range(3)]

    plans = {"fp32_refine": make("fp32_refine"), "fp64": make("fp64")}
    outs = [torch.empty_like(f) for _ in range(3)]

    def step(ps):
        for d in range(3):
            ps[d].solve(f, outs[d], stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(ps, steps, warmup):
        for _ in range(warmup):
            step(ps)
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev_dir = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        ev[0].record(stream)
        for s in range(steps):
            ev_dir[s][0].record(stream)
            for d in range(3):
                ps[d].solve(f, outs[d], stream)
                ev_dir[s][d + 1].record(stream)
        ev[1].record(stream)
        barrier()
        ms = ev[0].elapsed_time(ev[1]) / steps
        per_dir = [sum(ev_dir[s][d].elapsed_time(ev_dir[s][d + 1]) for s in range(steps)) / steps
                   for d in range(3)]
        ms = max_over_ranks(ms, dev)
        return ms, per_dir

    # clocks are sampled (every 100 ms) across all the device-timed work
    sampler = ClockSampler(local)
    with sampler:
        time.sleep(0.3)
        ms_ref, dir_ref = timed(plans["fp32_refine"], args.steps, max(args.warmup, 3))
        ms_64, dir_64 = timed(plans["fp64"], max(3, args.steps // 2), 3)
        for _ in range(max(1, int(0.3 / max(ms_ref * 1e-3, 1e-4)))):  # keep the GPU busy while sampling
            step(plans["fp32_refine"])
        barrier()

    # accuracy of both paths against the FP64 oracle on sampled lines
    err = {}
    if rank == 0:
        import oracle
        rng = np.random.default_rng(7)
        for prec in ("fp32_refine", "fp64"):
            step(plans[prec])
            torch.cuda.synchronize(dev)
            e = 0.0
            for d in range(3):
                ax = 2 - d
                idx = rng.integers(0, n, size=(64, 2))
                fl = np.moveaxis(f_host, ax, -1)[idx[:, 0], idx[:, 1]]
                ref = oracle.derivative(fl, sch["lhs"], sch["rhs"], h)
                got = np.moveaxis(outs[d].cpu().numpy(), ax, -1)[idx[:, 0], idx[:, 1]]
                e = max(e, oracle.rel_err(got, ref))
            err[prec] = e

    # end to end through the public API: pinned host f -> device, 3 solves,
    # results back to pinned host memory, every step
    out_pin = [torch.empty(f.shape, dtype=torch.float64).pin_memory() for _ in range(3)]
    e2e_steps = max(2, args.steps // 4)

    def e2e_step(ps):
        f.copy_(f_pin, non_blocking=True)
        for d in range(3):
            ps[d].solve(f, outs[d], stream)
        for d in range(3):
            out_pin[d].copy_(outs[d], non_blocking=True)

    for _ in range(2):
        e2e_step(plans["fp32_refine"])
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step(plans["fp32_refine"])
    barrier()
    e2e_ms = (time.perf_counter() - t0) / e2e_steps * 1e3
    e2e_ms = max_over_ranks(e2e_ms, dev)

    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except OSError:
            pass
        hbm = peaks.get("hbm_gbs", 6800.0)
        hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
        bytes_per_launch = 16.0 * n ** 3  # read f (FP64), write f' (FP64)
        kdir = max(range(3), key=lambda d: dir_ref[d])
        achieved = bytes_per_launch / (sum(dir_ref) / 3 * 1e-3) / 1e9
        # FP64 path: bound by the FP64 pipe; 15 algorithmic FP64 flops per unknown
        fp64_peak_tflops = 152 * 2 * 2 * 2.07e9 / 1e12
        fp64_flops = 15.0 * n ** 3
        fp64_ach = fp64_flops / (sum(dir_64) / 3 * 1e-3) / 1e12
        clocks = sampler.summary()
        units = 3 * n ** 3
        value = job_throughput(units, world, ms_ref)
        cpu_v, cores, sample = oracle_sample(args.cpu_seconds) if args.cpu_seconds > 0 else (None, None, "skipped")
        rec = {
            "metric": METRIC, "value": value, "unit": "Gunknowns/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_ref, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64-accurate residual via FP32 error-free transforms)",
            "data": "synthetic (seeded U(-1,1) + one plane wave, numpy PCG64 seed 1)",
            "config": dict(CONFIG, grid=[n, n, n], parallelism="replicas" if world > 1 else "single GPU",
                           precision="fp32_refine",
                           sweeps=1, segments=plans["fp32_refine"][0].info()["segments"]),
            "max_rel_err": err.get("fp32_refine"),
            "ms_per_direction": dir_ref,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None, "peak_source": hbm_src,
                         "kernel": "line_kernel<R=1,M=16,refine,K=2>", "slowest_direction": "xyz"[kdir]},
            "fp64_path": {"value": job_throughput(units, world, ms_64), "unit": "Gunknowns/s",
                          "ms_per_step": ms_64, "ms_per_direction": dir_64, "max_rel_err": err.get("fp64"),
                          "segments": plans["fp64"][0].info()["segments"],
                          "roofline": {"bound": "alu", "achieved": fp64_ach, "peak": fp64_peak_tflops,
                                       "unit": "TFLOP/s (FP64)", "frac": fp64_ach / fp64_peak_tflops,
                                       "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"},
                          "hbm_frac": 16.0 * n ** 3 / (sum(dir_64) / 3 * 1e-3) / 1e9 / hbm},
            "speedup_refine_vs_fp64": ms_64 / ms_ref,
            "e2e": {"value": job_throughput(units, world, e2e_ms), "unit": "Gunknowns/s",
                    "h2d_bytes_per_step": 8 * n ** 3, "d2h_bytes_per_step": 3 * 8 * n ** 3,
                    "ms_per_step": e2e_ms},
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
            "cpu_baseline": {"value": cpu_v, "unit": "Gunknowns/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
        }
        print(json.dumps(rec))
    for ps in plans.values():
        for p in ps:
            p.close()
    if world > 1:
        dist.destroy_process_group()


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


if __name__ == "__main__":
    main()
