"""Benchmark: compact 6th-order derivatives of a 512^3 periodic FP64 field.

One step = the whole hot path over one field: the cyclic tridiagonal
derivative (Lele 6th order, alpha = 1/3) along x (contiguous), y and z
(strided), each = stencil + per-partition solve + interface block PCR +
back-substitution (+ refinement), i.e. 3 x 512^3 unknowns.  The partition
count of each direction is picked by the library's autotuner.

The headline path is FP32 bulk + FP64-accurate refinement (one sweep), whose
error against the FP64 oracle is <= 1e-12; the plain FP64 path is timed on
the same field and reported beside it.  Inputs (1 GiB) exceed the 129 MB L2,
so no flush is needed between steps.  The other workloads of the method
(64^3 Fourier field, 32 long pentadiagonal lines, a ragged batch of 48 grids
under a CUDA graph, 256^2 x-lines of 8192, 256^3 acyclic systems, the 256^3
variable-alpha forward and adjoint) are timed after it and reported under "other_workloads", each
with its error against the FP64 oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--size N] [--profile] [--no-configs] [--cpu-seconds S]

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
          "grid": [N, N, N], "scheme": "alpha=1/3, a=14/9, b=1/9", "segments": "autotuned",
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
    ap.add_argument("--profile", action="store_true",
                    help="headline solves only (W + K steps of x, y, z), for profiler captures")
    ap.add_argument("--precision", default="fp32_refine", choices=["fp32_refine", "fp64", "fp32"],
                    help="path run by --profile (the timed headline is always fp32_refine)")
    ap.add_argument("--workload", default="cube", choices=["cube", "long", "var", "batch", "block"],
                    help="what --profile runs: the n^3 field (cube), the 32 x 2^22 pentadiagonal lines "
                         "(long, FP32 right-hand side, refinement with 1 sweep, default segments), the "
                         "256^3 variable-alpha forward + adjoint (var), the ragged batch of 48 grids (batch) or "
                         "256^2 x-lines of 256 points x 2 unknowns with 2 x 2 block entries (block)")
    ap.add_argument("--segments", default="tune",
                    help="partitions per line: 'tune' (autotuner) or a fixed count")
    ap.add_argument("--profile-shape", default=None,
                    help="--profile on a seeded U(-1,1) field of this shape NZ,NY,NX instead of the n^3 cube "
                         "(smaller captures of the same kernels)")
    ap.add_argument("--directions", default="0,1,2",
                    help="--profile: the line directions solved per step (0 = x, 1 = y, 2 = z)")
    ap.add_argument("--batch-mode", default="persistent", choices=["persistent", "per_problem", "auto"],
                    help="--profile --workload batch: how the batch runs (persistent: the one batch_kernel launch)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (64^3 Fourier, long lines, ragged batch, variable alpha)")
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
    lines of a seeded 512^3 field): one untimed warm-up, then the median of
    three timed runs of the same sample (about seconds / 3 each); returns
    (Gunknowns/s, cores, sample)."""
    import numpy as np
    import oracle
    from paper_2101_02286_gb300 import workloads as W
    rng = np.random.default_rng(W.SEEDS["cube512"])
    lines = rng.uniform(-1.0, 1.0, size=(seed_lines, N))
    h = W.grid_spacing(N)
    oracle.derivative(lines, W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], h)  # warm-up (untimed)
    t0 = time.perf_counter()
    oracle.derivative(lines, W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], h)  # sizes the runs (untimed)
    reps = max(1, int(seconds / 3.0 / max(time.perf_counter() - t0, 1e-6)))
    rates = []
    for _ in range(3):
        t1 = time.perf_counter()
        for _ in range(reps):
            oracle.derivative(lines, W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], h)
        rates.append(reps * seed_lines * N / (time.perf_counter() - t1) / 1e9)
    rates.sort()
    return rates[1], oracle.num_threads(), \
        "median of 3 runs (after 1 warm-up) of %d solves of %d lines x n=512 each (x/y/z lines are identical " \
        "1-D systems)" % (reps, seed_lines)


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



def nvtx(torch, label):
    """Push (label) or pop (None) an NVTX range; a no-op where NVTX is absent."""
    try:
        torch.cuda.nvtx.range_push(label) if label else torch.cuda.nvtx.range_pop()
    except (RuntimeError, AttributeError):
        pass


# ---------------------------------------------------------------- traffic record
KERNEL_SOURCES = ("paper_2101_02286_gb300/csrc/cbs_tma.cuh", "paper_2101_02286_gb300/csrc/cbs_tma_launch.cuh",
                  "paper_2101_02286_gb300/csrc/cbs_line.cuh", "paper_2101_02286_gb300/csrc/cbs_internal.h")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record(kernel: str, size: int):
    """DRAM bytes per launch of `kernel` from an ncu capture summarised under
    profiles/ (a line 'traffic-record: kernel=K size=S source=H bytes=B'), or
    None when no record exists or the kernel sources changed since."""
    d = os.path.join(ROOT, "profiles")
    want = kernel_source_hash()
    try:
        names = sorted(os.listdir(d))
    except OSError:
        return None
    for name in names:
        if not name.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(d, name)):
            if not line.startswith("traffic-record:"):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            if kv.get("kernel") == kernel and kv.get("size") == str(size) and kv.get("source") == want:
                return float(kv["bytes"])
    return None


# ---------------------------------------------------------------- other workloads
def time_ms(fn, stream, steps: int, warmup: int = 3) -> float:
    """Average device time of fn() (CUDA events on `stream`, warm-ups first)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _entry(workload, unknowns, ms, bytes_per_unknown, hbm, err, **extra):
    gbs = bytes_per_unknown * unknowns / (ms * 1e-3) / 1e9
    return dict({"workload": workload, "value": unknowns / (ms * 1e-3) / 1e9, "unit": "Gunknowns/s", "ms": ms,
                 "algorithmic_bytes_per_unknown": bytes_per_unknown, "achieved_gbs": gbs, "hbm_frac": gbs / hbm,
                 "max_rel_err": err}, **extra)


def other_configs(dev, stream, steps: int, hbm: float, check: bool) -> list:
    """The other workloads of the method, each timed on `stream` and checked
    against the FP64 oracle (whole output or sampled lines)."""
    import numpy as np
    import torch
    from paper_2101_02286_gb300 import abi
    from paper_2101_02286_gb300 import workloads as W
    from paper_2101_02286_gb300.autograd import variable_plan
    from paper_2101_02286_gb300.solver import Batch, Plan, make_desc
    if check:
        import oracle
    res = []
    rng = np.random.default_rng(17)

    # 64^3 Fourier field, x-derivative, 4 partitions per line, FP64 (fits in L2)
    f64, _ = W.fourier_cube(64, 8)
    sch = W.LELE6_TRI
    h = W.grid_spacing(64)
    pl = Plan(f64.shape, 0, lhs=sch["lhs"], rhs=sch["rhs"], h=h, segments=4, precision="fp64")
    fi = torch.from_numpy(f64).to(dev)
    fo = torch.empty_like(fi)
    ms = time_ms(lambda: pl.solve(fi, fo, stream), stream, max(steps, 20))
    err = oracle.rel_err(fo.cpu().numpy(), oracle.derivative(f64, sch["lhs"], sch["rhs"], h)) if check else None
    res.append(_entry("64^3 sum of 8 plane waves, x-derivative, tri 6th order, p=4, fp64 (L2-resident)",
                      64 ** 3, ms, 16, hbm, err, segments=4))
    pl.close()
    del fi, fo

    # long lines: 32 x 2^22 cyclic pentadiagonal, FP32 right-hand side, FP64 solution
    d = W.long_lines()
    lines, n = d.shape
    di = torch.from_numpy(d.reshape(1, lines, n)).to(dev)
    do = torch.empty((1, lines, n), dtype=torch.float64, device=dev)
    # default segments: 8168 of 514 / 498 rows, a warp per segment and 4
    # segments per CTA (2042 thread blocks per line); p = 1024: the end-row /
    # interface / segment launches (segments of ~4096 rows, a CTA each)
    for prec, sweeps, seg in (("fp32_refine", 1, 0), ("fp32_refine", 2, 1024), ("fp64", 1, 0)):
        pl = Plan((1, lines, n), 0, lhs=W.PENTA10["lhs"], rhs=None, segments=seg, precision=prec,
                  sweeps=sweeps, in_dtype=torch.float32)
        info = pl.info()
        ms = time_ms(lambda: pl.solve(di, do, stream), stream, steps)
        err = None
        if check:
            k = int(rng.integers(0, lines))
            ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.PENTA10["lhs"]), d[k:k + 1].astype(np.float64))
            err = oracle.rel_err(do[0, k:k + 1].cpu().numpy(), ref)
        how = ("%d segments, a warp each, 4 per thread block" % info["segments"] if info["segment_warp"]
               else "%d segments across CTAs" % info["segments"])
        res.append(_entry("32 x 2^22 cyclic penta (1/20,1/2,1,1/2,1/20), N(0,1) rhs stored FP32, FP64 out, "
                          "%s, %s sweeps=%d" % (how, prec, sweeps),
                          lines * n, ms, 12, hbm, err, segments=info["segments"], precision=prec, sampled_lines=1,
                          launches_per_step=abi.cbs_last_launch_count()))
        pl.close()
    del di, do, d

    # ragged batch: 48 grids replayed from a CUDA graph, in the default mode
    # (each problem's own kernels, FP64 problems on a forked stream) and as
    # one persistent launch
    items = W.ragged_batch()
    ins = [torch.from_numpy(it.f).to(dev) for it in items]
    unk = sum(int(np.prod(it.shape_zyx)) for it in items)
    # the persistent launch with the default partitions (the tuner may pick
    # partition sizes that only the per-problem kernels take), then the
    # autotuner on every problem, then the default mode with its choices
    specs = batch_specs(items)
    batches = {"persistent": Batch(specs, mode="persistent")}
    t0 = time.perf_counter()
    for sh, d, kw in specs:
        abi.cbs_autotune(make_desc(sh, d, **kw), 3)
    tune_s = time.perf_counter() - t0
    batches["auto"] = Batch(specs)
    for mode, how in (("auto", "each problem's own kernels (autotuned partitions and tiles), FP64 problems on a "
                               "second stream"),
                      ("persistent", "one persistent launch (default partitions)")):
        b = batches[mode]
        outs = [torch.empty_like(x) for x in ins]
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        b.solve(ins, outs, side)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            b.solve(ins, outs, side)
        launches = abi.cbs_last_launch_count()
        ms = time_ms(g.replay, stream, steps)
        err = None
        if check:
            err = 0.0
            for it, y in zip(items, outs):
                ax = 2 - it.direction
                sc = W.LELE6_TRI if it.scheme == "tri6" else W.PENTA10
                nn = it.shape_zyx[ax]
                fl = np.moveaxis(it.f, ax, -1)
                other = fl.shape[:2]
                idx = [(int(rng.integers(0, other[0])), int(rng.integers(0, other[1]))) for _ in range(4)]
                sel = np.stack([fl[i, j] for i, j in idx])
                ref = oracle.derivative(sel, sc["lhs"], sc["rhs"], W.grid_spacing(nn))
                yl = np.moveaxis(y.cpu().numpy(), ax, -1)
                err = max(err, oracle.rel_err(np.stack([yl[i, j] for i, j in idx]), ref))
        res.append(_entry("ragged batch of 48 grids (sizes from {32..384} per axis, seed 3), mixed tri/penta, "
                          "fp64/fp32_refine, %s, under a CUDA graph" % how, unk, ms, 16, hbm, err,
                          problems=len(items), mode=mode, launches_per_step=launches, sampled_lines=4 * len(items),
                          **({"autotune_s": round(tune_s, 1)} if mode == "auto" else {})))
        b.close()
        del outs, g
    del ins, items

    # the paper's single-GPU workload: 256^2 lines of 8192 along x, y and z
    # (fields 8192 x 256 x 256, 256 x 8192 x 256, 256 x 256 x 8192), cyclic
    # tridiagonal alpha = 1/3, right-hand side given; x: the default (16
    # segments of 513 / 497 rows, a warp each) and p = 7 (2^n - 1),
    # y/z: p = 16 (the default: segments of 513 / 497 rows, a warp each, one
    # segment of 4 adjacent lines per CTA);
    # the three fields share one buffer of random values
    dpx = np.random.default_rng(20).standard_normal(256 * 256 * 8192)
    di = torch.from_numpy(dpx).to(dev)
    do = torch.empty_like(di)
    for direction, prec, p in ((0, "fp32_refine", 0), (0, "fp32_refine", 7), (0, "fp64", 0),
                               (1, "fp32_refine", 16), (1, "fp64", 16), (2, "fp32_refine", 16), (2, "fp64", 16)):
        shape = [(256, 256, 8192), (256, 8192, 256), (8192, 256, 256)][direction]  # (nz, ny, nx)
        pl = Plan(shape, direction, lhs=W.LELE6_TRI["lhs"], rhs=None, precision=prec, segments=p)
        dv, ov = di.view(shape), do.view(shape)
        ms = time_ms(lambda: pl.solve(dv, ov, stream), stream, max(3, steps // 2))
        err = None
        if check:
            ii = rng.integers(0, 256, size=(8, 2))
            src = np.moveaxis(dpx.reshape(shape), 2 - direction, -1)
            got = np.moveaxis(do.cpu().numpy().reshape(shape), 2 - direction, -1)
            lines = np.stack([src[i, j] for i, j in ii])
            ref = oracle.solve_cyclic(oracle.toeplitz_bands(8192, W.LELE6_TRI["lhs"]), lines)
            err = oracle.rel_err(np.stack([got[i, j] for i, j in ii]), ref)
        info = pl.info()
        how = "%d segments per line%s" % (info["segments"], ", a warp each" if info["segment_warp"] else "")
        res.append(_entry("256^2 %s-lines of 8192 (the paper's single-GPU workload), cyclic tridiagonal "
                          "alpha=1/3, right-hand side given, %s, %s" % ("xyz"[direction], how, prec),
                          256 * 256 * 8192, ms, 16, hbm, err, segments=info["segments"], sampled_lines=8))
        pl.close()
    del di, do, dpx

    # acyclic (non-periodic) systems, right-hand side given: 256^3, y lines
    dac = np.random.default_rng(19).standard_normal((256, 256, 256))
    di = torch.from_numpy(dac).to(dev)
    do = torch.empty_like(di)
    for prec in ("fp32_refine", "fp64"):
        pl = Plan(dac.shape, 1, lhs=W.LELE6_TRI["lhs"], rhs=None, precision=prec, cyclic=False)
        ms = time_ms(lambda: pl.solve(di, do, stream), stream, steps)
        err = None
        if check:
            ii = rng.integers(0, 256, size=(32, 2))
            lines = np.stack([dac[i, :, j] for i, j in ii])
            ref = oracle.solve_acyclic(oracle.toeplitz_bands(256, W.LELE6_TRI["lhs"]), lines)
            got = do.cpu().numpy()
            err = oracle.rel_err(np.stack([got[i, :, j] for i, j in ii]), ref)
        res.append(_entry("256^3 acyclic tridiagonal (alpha=1/3, no wrap-around), y lines, right-hand side "
                          "given, %s" % prec, 256 ** 3, ms, 16, hbm, err, segments=pl.info()["segments"],
                          sampled_lines=32))
        pl.close()
    del di, do, dac

    # block-tridiagonal systems with 2 x 2 block entries (Sec. 1), right-hand
    # side given: 2^25 unknowns as 256 x 256 lines of 256 points x 2 unknowns
    # along x, and the same along z
    BLK = (np.array([[0.21, 0.07], [-0.05, 0.18]]), np.array([[1.0, 0.15], [-0.12, 0.9]]),
           np.array([[0.24, -0.06], [0.04, 0.2]]))
    dbk = np.random.default_rng(23).standard_normal(256 * 256 * 512)
    for direction, shape in ((0, (256, 256, 512)), (2, (512, 256, 256))):
        for prec in ("fp64", "fp32"):
            dt = torch.float64 if prec == "fp64" else torch.float32
            di = torch.from_numpy(dbk.reshape(shape)).to(dev, dt)
            do = torch.empty_like(di)
            pl = Plan(shape, direction, blocks=BLK, precision=prec, in_dtype=dt)
            ms = time_ms(lambda: pl.solve(di, do, stream), stream, steps)
            err = None
            if check:
                ii = rng.integers(0, 256, size=(16, 2))
                src = np.moveaxis(di.double().cpu().numpy(), 2 - direction, -1)
                got = np.moveaxis(do.double().cpu().numpy(), 2 - direction, -1)
                lines = np.stack([src[i, j] for i, j in ii])
                ref = oracle.solve_cyclic(oracle.block_tridiagonal_bands(256, *BLK), lines)
                err = oracle.rel_err(np.stack([got[i, j] for i, j in ii]), ref)
            res.append(_entry("256^2 %s-lines of 256 points x 2 unknowns, cyclic block-tridiagonal with 2x2 block "
                              "entries, right-hand side given, %s" % ("xyz"[direction], prec),
                              256 * 256 * 512, ms, 16 if prec == "fp64" else 8, hbm, err,
                              segments=pl.info()["segments"], sampled_lines=16))
            pl.close()
            del di, do
    del dbk

    # staggered schemes of the paper's Taylor-Green runs (App. A.2): 256^3,
    # sixth-order derivative from the nodes to the half points and compact
    # interpolation from the half points to the nodes, along x, y and z
    fs = np.random.default_rng(22).standard_normal((256, 256, 256))
    fi = torch.from_numpy(fs).to(dev)
    outs = [torch.empty_like(fi) for _ in range(3)]
    hs = W.grid_spacing(256)
    for kind, shift, sch in (("staggered", 1, W.STAGGERED6), ("midpoint", 0, W.MIDPOINT6)):
        for prec in ("fp32_refine", "fp64"):
            pls = [Plan(fs.shape, dd, lhs=sch["lhs"], rhs=sch["rhs"], h=hs, precision=prec, stencil=kind,
                        shift=shift) for dd in range(3)]

            def step():
                for dd in range(3):
                    pls[dd].solve(fi, outs[dd], stream)
            ms = time_ms(step, stream, steps)
            err = None
            if check:
                err = 0.0
                for dd in range(3):
                    ax = 2 - dd
                    fl = np.moveaxis(fs, ax, -1)
                    ii = rng.integers(0, 256, size=(8, 2))
                    lines = np.stack([fl[i, j] for i, j in ii])
                    ref = (oracle.staggered_derivative(lines, sch["lhs"], sch["rhs"], hs, shift) if kind == "staggered"
                           else oracle.midpoint_interpolation(lines, sch["lhs"], sch["rhs"], shift))
                    yl = np.moveaxis(outs[dd].cpu().numpy(), ax, -1)
                    err = max(err, oracle.rel_err(np.stack([yl[i, j] for i, j in ii]), ref))
            what = ("staggered 6th-order derivative (alpha=9/62), nodes -> half points" if kind == "staggered"
                    else "compact 6th-order interpolation (alpha=3/10), half points -> nodes")
            res.append(_entry("256^3 %s, x/y/z (3 launches), %s" % (what, prec), 3 * 256 ** 3, ms, 16, hbm, err,
                              segments=pls[0].info()["segments"], sampled_lines=24))
            for pl in pls:
                pl.close()
    del fi, outs, fs

    # variable alpha: 256^3, forward and adjoint, FP64 and FP32 (x lines)
    f, al = W.variable_alpha_cube(256)
    c4 = W.CENTRAL4["rhs"]
    hv = W.grid_spacing(256)
    gseed = np.random.default_rng(18).standard_normal(f.shape)
    for prec, dt, bpu_f, bpu_b in (("fp64", torch.float64, 24, 40), ("fp32", torch.float32, 12, 20)):
        fa, aa, ga = (torch.from_numpy(a).to(dev, dt) for a in (f, al, gseed))
        pl = variable_plan(f.shape, 0, aa, c4, hv, prec, segments="tune")
        x = torch.empty_like(fa)
        gf, gal = torch.empty_like(fa), torch.empty_like(fa)
        ms_f = time_ms(lambda: pl.solve(fa, x, stream), stream, steps)
        ms_b = time_ms(lambda: abi.cbs_solve_transpose(pl.handle, ga.data_ptr(), x.data_ptr(), None, gf.data_ptr(),
                                                       gal.data_ptr(), stream.cuda_stream), stream, steps)
        ef = eb = None
        if check:
            ii = rng.integers(0, 256, size=(32, 2))
            pick = lambda a: np.stack([a[i, j] for i, j in ii])
            src = [pick(a.double().cpu().numpy()) for a in (fa, aa, ga)]
            gfr, gar, _, xr = oracle.adjoint_variable_tri(src[0], src[1], src[2], c4, hv, axis=-1)
            ef = oracle.rel_err(pick(x.double().cpu().numpy()), xr)
            eb = max(oracle.rel_err(pick(gf.double().cpu().numpy()), gfr),
                     oracle.rel_err(pick(gal.double().cpu().numpy()), gar))
        w = "256^3 variable alpha ~ U(0.2,0.4), 4th-order central rhs, x lines, %s" % prec
        res.append(_entry(w + ", forward", 256 ** 3, ms_f, bpu_f, hbm, ef, sampled_lines=32))
        res.append(_entry(w + ", adjoint (grad f and grad alpha)", 256 ** 3, ms_b, bpu_b, hbm, eb, sampled_lines=32))
        pl.close()
    return res

def batch_specs(items):
    """Batch problem descriptions of the ragged-batch workload: 6th-order
    tridiagonal or 10th-order pentadiagonal derivative along each grid's
    direction; pentadiagonal refinement runs two sweeps."""
    from paper_2101_02286_gb300 import workloads as W
    specs = []
    for it in items:
        nn = it.shape_zyx[2 - it.direction]
        sc = W.LELE6_TRI if it.scheme == "tri6" else W.PENTA10
        specs.append((it.shape_zyx, it.direction,
                      dict(lhs=sc["lhs"], rhs=sc["rhs"], h=W.grid_spacing(nn), precision=it.precision,
                           sweeps=2 if (it.scheme == "penta10" and it.precision == "fp32_refine") else 1)))
    return specs


def profile_other(args, dev, stream, rank):
    """--profile for the long-line, variable-alpha, batch or block-entry
    workload: W warm-up and K further solves, nothing timed, for profiler
    captures."""
    import numpy as np
    import torch
    from paper_2101_02286_gb300 import abi
    from paper_2101_02286_gb300 import workloads as W
    from paper_2101_02286_gb300.autograd import variable_plan
    from paper_2101_02286_gb300.solver import Plan
    if args.workload == "long":
        d = W.long_lines()
        lines, n = d.shape
        di = torch.from_numpy(d.reshape(1, lines, n)).to(dev)
        do = torch.empty((1, lines, n), dtype=torch.float64, device=dev)
        prec = args.precision
        pl = Plan((1, lines, n), 0, lhs=W.PENTA10["lhs"], rhs=None, precision=prec, sweeps=1,
                  in_dtype=torch.float32)
        for _ in range(args.warmup + args.steps):
            pl.solve(di, do, stream)
        info = pl.info()
    elif args.workload == "block":
        # 256^2 x-lines of 256 points x 2 unknowns, 2 x 2 block entries
        blk = (np.array([[0.21, 0.07], [-0.05, 0.18]]), np.array([[1.0, 0.15], [-0.12, 0.9]]),
               np.array([[0.24, -0.06], [0.04, 0.2]]))
        shape = (256, 256, 512)
        dt = torch.float64 if args.precision == "fp64" else torch.float32
        di = torch.from_numpy(np.random.default_rng(23).standard_normal(shape)).to(dev, dt)
        do = torch.empty_like(di)
        pl = Plan(shape, 0, blocks=blk, precision="fp64" if dt == torch.float64 else "fp32", in_dtype=dt)
        for _ in range(args.warmup + args.steps):
            pl.solve(di, do, stream)
        info = pl.info()
    elif args.workload == "batch":
        from paper_2101_02286_gb300.solver import Batch
        items = W.ragged_batch()
        b = Batch(batch_specs(items), mode=args.batch_mode)
        ins = [torch.from_numpy(it.f).to(dev) for it in items]
        outs = [torch.empty_like(x) for x in ins]
        for _ in range(args.warmup + args.steps):
            b.solve(ins, outs, stream)
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"profile": True, "workload": "batch", "problems": len(items),
                              "mode": args.batch_mode, "launches_per_step": abi.cbs_last_launch_count()}))
        b.close()
        return
    else:
        f, al = W.variable_alpha_cube(256)
        dt = torch.float64 if args.precision != "fp32" else torch.float32
        fa, aa = (torch.from_numpy(a).to(dev, dt) for a in (f, al))
        pl = variable_plan(f.shape, 0, aa, W.CENTRAL4["rhs"], W.grid_spacing(256),
                           "fp64" if dt == torch.float64 else "fp32")
        x, g, gf, ga = (torch.empty_like(fa) for _ in range(4))
        g.copy_(fa)
        for _ in range(args.warmup + args.steps):  # forward, then adjoint
            pl.solve(fa, x, stream)
            abi.cbs_solve_transpose(pl.handle, g.data_ptr(), x.data_ptr(), None, gf.data_ptr(), ga.data_ptr(),
                                    stream.cuda_stream)
        info = pl.info()
    torch.cuda.synchronize(dev)
    if rank == 0:
        print(json.dumps({"profile": True, "workload": args.workload, "precision": args.precision,
                          "steps": args.steps, "warmup": args.warmup, "segments": info["segments"]}))
    pl.close()


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
    from paper_2101_02286_gb300.solver import Pipe, Plan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    if args.profile and args.workload != "cube":
        profile_other(args, dev, stream, rank)
        return
    n = args.size
    if args.profile and args.profile_shape:
        shape = tuple(int(v) for v in args.profile_shape.split(","))
        f_host = np.random.default_rng(W.SEEDS["cube512"]).uniform(-1.0, 1.0, size=shape)
    else:
        f_host, modes = W.noisy_cube(n)  # seeded: U(-1,1) + one plane wave
    f_pin = torch.from_numpy(f_host).pin_memory()
    f = f_pin.to(dev)
    h = W.grid_spacing(n)
    sch = W.LELE6_TRI
    dirs = [int(v) for v in args.directions.split(",")] if args.profile else [0, 1, 2]

    def make(prec):
        # partition count per direction picked by the library's autotuner
        seg = "tune" if args.segments == "tune" else int(args.segments)
        return {d: Plan(f.shape, d, lhs=sch["lhs"], rhs=sch["rhs"], h=W.grid_spacing(f.shape[2 - d]), precision=prec,
                        sweeps=1, segments=seg) for d in dirs}

    plans = {"fp32_refine": make("fp32_refine")} if not args.profile else {args.precision: make(args.precision)}
    if args.profile:
        outs = [torch.empty_like(f)] * 3  # one output buffer keeps captures small
    else:
        outs = [torch.empty_like(f) for _ in range(3)]

    def step(ps):
        for k, d in enumerate(dirs):
            ps[d].solve(f, outs[k], stream)

    if args.profile:
        # headline solves only: W warm-up steps, then K steps (x, y, z each)
        for _ in range(args.warmup + args.steps):
            step(plans[args.precision])
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"profile": True, "shape": list(f.shape), "directions": dirs, "steps": args.steps,
                              "warmup": args.warmup, "precision": args.precision,
                              "segments": [plans[args.precision][d].info()["segments"] for d in dirs]}))
        return
    plans["fp64"] = make("fp64")
    plans["fp32_refine_i64"] = make("fp32_refine_i64")

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(ps, steps, warmup, label):
        for _ in range(warmup):
            step(ps)
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev_dir = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        nvtx(torch, label)  # lets a profiler select the timed launches
        ev[0].record(stream)
        for s in range(steps):
            ev_dir[s][0].record(stream)
            for d in range(3):
                ps[d].solve(f, outs[d], stream)
                ev_dir[s][d + 1].record(stream)
        ev[1].record(stream)
        nvtx(torch, None)
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
        ms_ref, dir_ref = timed(plans["fp32_refine"], args.steps, max(args.warmup, 3), "headline")
        ms_64, dir_64 = timed(plans["fp64"], max(3, args.steps // 2), 3, "fp64_path")
        ms_i64, dir_i64 = timed(plans["fp32_refine_i64"], max(3, args.steps // 2), 3, "refine_fp64_interface")
        for _ in range(max(1, int(0.3 / max(ms_ref * 1e-3, 1e-4)))):  # keep the GPU busy while sampling
            step(plans["fp32_refine"])
        barrier()

    # accuracy of both paths against the FP64 oracle on sampled lines
    err = {}
    if rank == 0:
        import oracle
        rng = np.random.default_rng(7)
        for prec in ("fp32_refine", "fp64", "fp32_refine_i64"):
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

    # end to end through the C-ABI with host buffers (cbs_pipe_solve): every
    # step uploads the field from pinned host memory, runs the three solves and
    # reads the three results back into pinned host memory, all inside the
    # call; the pipe alternates two sets of device buffers, so step k+1's
    # upload overlaps step k's downloads on the other copy engine.
    out_pin = [torch.empty(f.shape, dtype=torch.float64).pin_memory() for _ in range(3)]
    pipe = Pipe([plans["fp32_refine"][d] for d in range(3)])
    e2e_steps = max(4, args.steps // 2)

    def e2e_run(steps):
        for _ in range(steps):
            pipe.solve(f_pin, out_pin, stream)
        stream.synchronize()

    e2e_run(4)
    # five timed windows; the host link of a shared box shows bursts of
    # contention, so the median window is reported (all five are listed)
    e2e_windows = []
    for _ in range(5):
        barrier()
        t0 = time.perf_counter()
        e2e_run(e2e_steps)
        barrier()
        e2e_windows.append(max_over_ranks((time.perf_counter() - t0) / e2e_steps * 1e3, dev))
    e2e_ms = sorted(e2e_windows)[len(e2e_windows) // 2]
    pipe.close()

    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except OSError:
            pass
        hbm = peaks.get("hbm_gbs", 6800.0)
        hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
        bytes_per_launch = 16.0 * n ** 3  # read f (FP64), write f' (FP64)
        # dominant kernel: the slowest of the three launches of a step (all
        # three run the TMA-fed refinement kernel, with the tile shape the
        # autotuner picked for the direction)
        kdir = max(range(3), key=lambda d: dir_ref[d])
        achieved = bytes_per_launch / (dir_ref[kdir] * 1e-3) / 1e9
        info_ref = [plans["fp32_refine"][d].info() for d in range(3)]
        traffic = traffic_record("refine_tma_%s" % "xyz"[kdir], n)
        per_dir = {"xyz"[d]: {"ms_per_launch": dir_ref[d], "achieved": bytes_per_launch / (dir_ref[d] * 1e-3) / 1e9,
                              "frac": bytes_per_launch / (dir_ref[d] * 1e-3) / 1e9 / hbm,
                              "traffic": traffic_record("refine_tma_%s" % "xyz"[d], n),
                              "kernel": "refine_tma_kernel" if info_ref[d]["tma"] and info_ref[d]["variant"] == 0
                              else "line_kernel_pipe",
                              "tile_lines": info_ref[d]["tile_lines"]} for d in range(3)}
        # FP64 path: bound by the FP64 pipe; 15 algorithmic FP64 flops per
        # unknown against the FP64 fma throughput measured on this device
        from paper_2101_02286_gb300 import abi as _abi
        fp64_peak_tflops = _abi.cbs_probe_fp64_peak()
        fp64_flops = 15.0 * n ** 3
        fp64_ach = fp64_flops / (sum(dir_64) / 3 * 1e-3) / 1e12
        clocks = sampler.summary()
        units = 3 * n ** 3
        value = job_throughput(units, world, ms_ref)
        others = [] if args.no_configs else other_configs(dev, stream, max(5, args.steps // 2), hbm, check=True)
        cpu_v, cores, sample = oracle_sample(args.cpu_seconds) if args.cpu_seconds > 0 else (None, None, "skipped")
        rec = {
            "metric": METRIC, "value": value, "unit": "Gunknowns/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_ref, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64-accurate residual via FP32 error-free transforms)",
            "data": "synthetic (seeded U(-1,1) + one plane wave, numpy PCG64 seed 1)",
            "config": dict(CONFIG, grid=[n, n, n], parallelism="replicas" if world > 1 else "single GPU",
                           precision="fp32_refine", sweeps=1,
                           segments=[plans["fp32_refine"][d].info()["segments"] for d in range(3)]),
            "max_rel_err": err.get("fp32_refine"),
            "ms_per_direction": dir_ref,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "peak_source": hbm_src,
                         "kernel": "refine_tma_kernel (TMA tiles, warp per line, FP32 solves + one "
                                   "FP64-accurate refinement sweep), %s lines" % "xyz"[kdir],
                         "algorithmic_bytes_per_launch": bytes_per_launch, "ms_per_launch": dir_ref[kdir],
                         "slowest_direction": "xyz"[kdir]},
            "roofline_per_direction": per_dir,
            "refine_fp64_interface": {"value": job_throughput(units, world, ms_i64), "unit": "Gunknowns/s",
                                      "ms_per_step": ms_i64, "ms_per_direction": dir_i64,
                                      "max_rel_err": err.get("fp32_refine_i64"),
                                      "note": "same refinement with the interface system of each FP32 "
                                              "solve in FP64"},
            "fp64_path": {"value": job_throughput(units, world, ms_64), "unit": "Gunknowns/s",
                          "ms_per_step": ms_64, "ms_per_direction": dir_64, "max_rel_err": err.get("fp64"),
                          "segments": [plans["fp64"][d].info()["segments"] for d in range(3)],
                          "roofline": {"bound": "alu", "achieved": fp64_ach, "peak": fp64_peak_tflops,
                                       "unit": "TFLOP/s (FP64)", "frac": fp64_ach / fp64_peak_tflops,
                                       "peak_source": "measured: cbs_probe_fp64_peak (register-resident "
                                                      "FP64 fma chains, CUDA events)"},
                          "hbm_frac": 16.0 * n ** 3 / (sum(dir_64) / 3 * 1e-3) / 1e9 / hbm},
            "speedup_refine_vs_fp64": ms_64 / ms_ref,
            "e2e": {"value": job_throughput(units, world, e2e_ms), "unit": "Gunknowns/s",
                    "h2d_bytes_per_step": 8 * n ** 3, "d2h_bytes_per_step": 3 * 8 * n ** 3,
                    "ms_per_step": e2e_ms, "steps": e2e_steps, "window_ms": e2e_windows,
                    "api": "cbs_pipe_solve (C-ABI, pinned host buffers, copies inside the call)",
                    "overlap": "upload, solves and downloads on three streams, two device buffer sets"},
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
            "cpu_baseline": {"value": cpu_v, "unit": "Gunknowns/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "other_workloads": others,
        }
        print(json.dumps(rec))
    for ps in plans.values():
        for p in ps.values():
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
