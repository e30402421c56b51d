"""GPU parity of the ragged batch, in both modes (one persistent launch; each
problem's own launches with the FP64 problems on a forked stream), and its
CUDA-graph capture, against the FP64 oracle problem by problem."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Batch

pytestmark = pytest.mark.gpu
SCH = {"tri6": W.LELE6_TRI, "penta10": W.PENTA10}
MODES = ["persistent", "per_problem"]


def _launches_ok(mode, count):
    n = abi.cbs_last_launch_count()
    return n == 1 if mode == "persistent" else n >= count


def _specs(items):
    specs = []
    for it in items:
        n = it.shape_zyx[2 - it.direction]
        sch = SCH[it.scheme]
        specs.append((it.shape_zyx, it.direction,
                      dict(lhs=sch["lhs"], rhs=sch["rhs"], h=W.grid_spacing(n), precision=it.precision,
                           sweeps=2 if (it.scheme == "penta10" and it.precision == "fp32_refine") else 1)))
    return specs


def _ref(it, f):
    n = it.shape_zyx[2 - it.direction]
    sch = SCH[it.scheme]
    return oracle.derivative(f, sch["lhs"], sch["rhs"], W.grid_spacing(n), axis=2 - it.direction)


@pytest.mark.parametrize("mode", MODES)
def test_ragged_batch_small(cuda, mode):
    items = W.ragged_batch(count=24, seed=123, sizes=(32, 48, 64, 96))
    b = Batch(_specs(items), mode=mode)
    ins = [torch.from_numpy(it.f).cuda() for it in items]
    outs = b.solve(ins)
    assert _launches_ok(mode, len(items))
    torch.cuda.synchronize()
    for it, y in zip(items, outs):
        assert oracle.rel_err(y.cpu().numpy(), _ref(it, it.f)) < 1e-12, it
    b.close()


@pytest.mark.parametrize("mode", MODES)
def test_ragged_batch_cuda_graph(cuda, mode):
    items = W.ragged_batch(count=16, seed=321, sizes=(32, 64, 128))
    b = Batch(_specs(items), mode=mode)
    ins = [torch.from_numpy(it.f).cuda() for it in items]
    outs = [torch.empty_like(x) for x in ins]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.solve(ins, outs, s)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.solve(ins, outs)
    # new data in the same buffers, then replay twice
    rng = np.random.default_rng(5)
    fresh = [rng.uniform(-1, 1, size=it.shape_zyx) for it in items]
    for x, f in zip(ins, fresh):
        x.copy_(torch.from_numpy(f))
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for it, f, y in zip(items, fresh, outs):
        assert oracle.rel_err(y.cpu().numpy(), _ref(it, f)) < 1e-12
    b.close()


def test_batch_of_any_problems_runs_per_problem(cuda):
    # heptadiagonal bands, FP32 input with an FP64 result, block entries and a
    # staggered stencil do not fit the persistent launch: the batch takes
    # them all and runs every problem's own kernels; asking for the
    # persistent launch is refused
    from paper_2101_02286_gb300.solver import Plan
    blk = (np.array([[0.21, 0.07], [-0.05, 0.18]]), np.array([[1.0, 0.15], [-0.12, 0.9]]),
           np.array([[0.24, -0.06], [0.04, 0.2]]))
    specs = [((4, 6, 64), 0, dict(lhs=W.HEPTA12["lhs"])),
             ((4, 64, 6), 1, dict(lhs=(1 / 3,), precision="fp32_refine", in_dtype=torch.float32)),
             ((64, 4, 6), 2, dict(blocks=blk)),
             ((4, 6, 64), 0, dict(lhs=W.STAGGERED6["lhs"], rhs=W.STAGGERED6["rhs"], h=0.1, stencil="staggered")),
             ((4, 4, 64), 0, dict(lhs=(1 / 3,), rhs=(14 / 9, 1 / 9), h=0.1))]
    with pytest.raises(abi.CbsError) as e:
        Batch(specs, mode="persistent")
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED and "batch problem 0" in str(e.value)
    b = Batch(specs)
    rng = np.random.default_rng(8)
    ins = [torch.from_numpy(rng.uniform(-1, 1, size=sh)).cuda().to(kw.get("in_dtype", torch.float64))
           for sh, _, kw in specs]
    outs = [torch.empty(sh, dtype=torch.float64, device="cuda") for sh, _, _ in specs]
    b.solve(ins, outs)
    torch.cuda.synchronize()
    assert abi.cbs_last_launch_count() >= len(specs)
    for (sh, d, kw), x, y in zip(specs, ins, outs):
        pl = Plan(sh, d, **kw)
        ref = pl.solve(x)
        torch.cuda.synchronize()
        assert torch.equal(y, ref), (sh, d)  # the same kernels on the same input
        pl.close()
    b.close()


@pytest.mark.slow
@pytest.mark.parametrize("mode", MODES)
def test_ragged_batch_full_workload_sampled(cuda, mode):
    # the 48-grid ragged batch (sizes up to 384 per axis), sampled lines
    items = W.ragged_batch()
    b = Batch(_specs(items), mode=mode)
    ins = [torch.from_numpy(it.f).cuda() for it in items]
    outs = b.solve(ins)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for it, y in zip(items, outs):
        ax = 2 - it.direction
        fl = np.moveaxis(it.f, ax, -1)
        yl = np.moveaxis(y.cpu().numpy(), ax, -1)
        i0 = rng.integers(0, fl.shape[0], 4)
        i1 = rng.integers(0, fl.shape[1], 4)
        n = fl.shape[-1]
        sch = SCH[it.scheme]
        ref = oracle.derivative(fl[i0, i1], sch["lhs"], sch["rhs"], W.grid_spacing(n))
        assert oracle.rel_err(yl[i0, i1], ref) < 1e-12
    b.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_batch_mixes_long_lines_with_grids(cuda, precision, mode):
    # one persistent launch over on-chip grids (derivatives) and long x-lines
    # (right-hand side given, a warp per segment: 8192 = 16 segments in both
    # sizes, 9 x 513 = 4617: one CTA of 8 segments and one of 1), replayed
    # from a CUDA graph with new data
    items = W.ragged_batch(count=6, seed=77, sizes=(32, 64, 96))
    specs = _specs(items)
    longs = [((1, 5, 8192), W.PENTA10["lhs"]), ((1, 3, 4617), W.LELE6_TRI["lhs"])]
    for shape, lhs in longs:
        specs.append((shape, 0, dict(lhs=lhs, rhs=None, precision=precision, sweeps=1)))
    b = Batch(specs, mode=mode)
    rng = np.random.default_rng(9)
    data = [it.f for it in items] + [rng.standard_normal(shape) for shape, _ in longs]
    ins = [torch.from_numpy(f).cuda() for f in data]
    outs = [torch.empty_like(x) for x in ins]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.solve(ins, outs, s)
    torch.cuda.current_stream().wait_stream(s)
    assert _launches_ok(mode, len(specs))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.solve(ins, outs)
    fresh = [rng.uniform(-1, 1, size=f.shape) for f in data]
    for x, f in zip(ins, fresh):
        x.copy_(torch.from_numpy(f))
    g.replay()
    torch.cuda.synchronize()
    assert abi.cbs_batch_status_poll(b.handle) == abi.CBS_OK
    for it, f, y in zip(items, fresh, outs):
        assert oracle.rel_err(y.cpu().numpy(), _ref(it, f)) < 1e-12
    for (shape, lhs), f, y in zip(longs, fresh[len(items):], outs[len(items):]):
        ref = oracle.solve_cyclic(oracle.toeplitz_bands(shape[2], lhs), f[0])
        assert oracle.rel_err(y.cpu().numpy()[0], ref) < 1e-12
    b.close()


def test_batch_long_lines_off_the_warp_layout_run_per_problem(cuda):
    # long lines whose segments do not hold 32 x 16 rows (and y-lines) are not
    # persistent-launch items; the batch runs their plans' own launches
    from paper_2101_02286_gb300.solver import Plan
    specs = [((1, 2, 1 << 16), 0, dict(lhs=(1 / 3,), rhs=None, segments=16)),
             ((2, 4096, 4), 1, dict(lhs=W.PENTA10["lhs"], rhs=None, precision="fp32_refine"))]
    with pytest.raises(abi.CbsError) as e:
        Batch(specs, mode="persistent")
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED
    b = Batch(specs)
    rng = np.random.default_rng(6)
    data = [rng.standard_normal(sh) for sh, _, _ in specs]
    outs = b.solve([torch.from_numpy(f).cuda() for f in data])
    torch.cuda.synchronize()
    ref0 = oracle.solve_cyclic(oracle.toeplitz_bands(1 << 16, (1 / 3,)), data[0][0])
    assert oracle.rel_err(outs[0].cpu().numpy()[0], ref0) < 1e-12
    ref1 = oracle.solve_cyclic(oracle.toeplitz_bands(4096, W.PENTA10["lhs"]), data[1], axis=1)
    assert oracle.rel_err(outs[1].cpu().numpy(), ref1) < 1e-12
    b.close()


@pytest.mark.parametrize("mode", MODES)
def test_batch_fp32_problems_with_fp64_ones(cuda, mode):
    # FP32 problems (FP32 in and out, no refinement) in the same launch as
    # FP64 and refinement problems; tolerance 2e-5 for the FP32 ones
    items = W.ragged_batch(count=6, seed=91, sizes=(32, 48, 64, 96))
    specs = _specs(items)
    f32 = []
    for k, (shape, direction, scheme) in enumerate([((8, 12, 64), 0, "tri6"), ((16, 96, 8), 1, "penta10"),
                                                    ((48, 8, 8), 2, "tri6")]):
        n = shape[2 - direction]
        sch = SCH[scheme]
        specs.append((shape, direction, dict(lhs=sch["lhs"], rhs=sch["rhs"], h=W.grid_spacing(n), precision="fp32",
                                             in_dtype=torch.float32)))
        f32.append((shape, direction, scheme))
    b = Batch(specs, mode=mode)
    rng = np.random.default_rng(4)
    data = [it.f for it in items] + [rng.uniform(-1, 1, size=sh).astype(np.float32) for sh, _, _ in f32]
    ins = [torch.from_numpy(f).cuda() for f in data]
    outs = b.solve(ins)
    torch.cuda.synchronize()
    assert _launches_ok(mode, len(specs))
    for it, y in zip(items, outs):
        assert oracle.rel_err(y.cpu().numpy(), _ref(it, it.f)) < 1e-12
    for (shape, direction, scheme), f, y in zip(f32, data[len(items):], outs[len(items):]):
        assert y.dtype == torch.float32
        n = shape[2 - direction]
        sch = SCH[scheme]
        ref = oracle.derivative(f.astype(np.float64), sch["lhs"], sch["rhs"], W.grid_spacing(n), axis=2 - direction)
        assert oracle.rel_err(y.double().cpu().numpy(), ref) < 2e-5
    b.close()


def test_batch_modes_agree_and_auto_picks_by_size(cuda):
    # the two modes give the same results element by element up to the
    # kernels' rounding; auto takes per-problem launches from 2^20 unknowns
    # per problem on average, the persistent launch below
    big = [((64, 128, 128), 0, "fp64", "tri6"), ((128, 64, 128), 1, "fp32_refine", "penta10"),
           ((128, 128, 64), 2, "fp64", "penta10")]
    specs = []
    for shape, direction, prec, scheme in big:
        n = shape[2 - direction]
        sch = SCH[scheme]
        specs.append((shape, direction, dict(lhs=sch["lhs"], rhs=sch["rhs"], h=W.grid_spacing(n), precision=prec)))
    rng = np.random.default_rng(12)
    ins = [torch.from_numpy(rng.uniform(-1, 1, size=sh)).cuda() for sh, _, _ in specs]
    got = {}
    for mode in ("persistent", "per_problem", "auto"):
        b = Batch(specs, mode=mode)
        got[mode] = [y.cpu().numpy() for y in b.solve(ins)]
        torch.cuda.synchronize()
        got[mode + "_launches"] = abi.cbs_last_launch_count()
        b.close()
    assert got["persistent_launches"] == 1 and got["per_problem_launches"] >= 3
    assert got["auto_launches"] == got["per_problem_launches"]  # 2^20 unknowns each
    for a, c in zip(got["persistent"], got["per_problem"]):
        assert oracle.rel_err(a, c) < 1e-12
    small = Batch(specs[:1] + [((4, 8, 32), 0, dict(lhs=(1 / 3,), rhs=(14 / 9, 1 / 9), h=0.2))])
    x2 = torch.zeros((4, 8, 32), dtype=torch.float64, device="cuda")
    small.solve([ins[0], x2])
    # (64 * 128 * 128 + 1024) / 2 unknowns on average: below 2^20 -> one launch
    assert abi.cbs_last_launch_count() == 1
    small.close()
    with pytest.raises(ValueError):
        Batch(specs, mode="bogus")
