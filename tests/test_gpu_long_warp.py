"""GPU parity of the warp-per-segment long-line path (x-lines whose segments
hold 32 or 31 inner partitions of 16 rows and whose outer interface system is
decoupled to FP64 rounding) against the FP64 oracle, element by element.

Cases: the paper's 8192-point lines (tri and penta, every precision), line
lengths whose segments are all of one size or of both sizes, a chunk of
segments per CTA that ends mid-line (halo rows from the neighbouring CTA),
the wrap of the cyclic line at both ends, FP32 and FP64 inputs, agreement
with the end-row / interface / segment launches, the allocation-free entry,
and non-finite input reported as CBS_ERR_RANGE.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Plan

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32_refine": 1e-12, "fp32_refine_i64": 1e-12, "fp32": 2e-5}
LHS = {"tri6": W.LELE6_TRI["lhs"], "penta10": W.PENTA10["lhs"]}


def solve(d, lhs, precision="fp32_refine", sweeps=2, in_dtype=torch.float64, variant=0, noalloc=False):
    lines, n = d.shape
    out_dtype = in_dtype if precision == "fp32" else torch.float64
    plan = Plan((1, lines, n), 0, lhs=lhs, rhs=None, precision=precision, sweeps=sweeps, in_dtype=in_dtype,
                out_dtype=out_dtype)
    abi.cbs_plan_set_variant(plan.handle, variant, 0)
    x = torch.from_numpy(d.reshape(1, lines, n)).to("cuda", in_dtype)
    y = torch.empty((1, lines, n), dtype=out_dtype, device="cuda")
    if noalloc:
        abi.cbs_solve_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), 0)
    else:
        plan.solve(x, y)
    torch.cuda.synchronize()
    launches = abi.cbs_last_launch_count()
    info = plan.info()
    st = plan.status()
    plan.close()
    return y.double().cpu().numpy().reshape(lines, n), info, launches, st


def reference(d, lhs):
    return oracle.solve_cyclic(oracle.toeplitz_bands(d.shape[1], lhs), d.astype(np.float64))


@pytest.mark.parametrize("precision", ["fp32_refine", "fp32_refine_i64", "fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["tri6", "penta10"])
def test_paper_lines_8192(cuda, scheme, precision):
    # the paper's 8192-point lines: 16 segments (15 or 14 of 32 x 16 + r rows)
    d = np.random.default_rng(11).standard_normal((40, 8192))
    dt = torch.float32 if precision == "fp32" else torch.float64
    if dt == torch.float32:
        d = d.astype(np.float32).astype(np.float64)
    x, info, launches, st = solve(d, LHS[scheme], precision, in_dtype=dt)
    assert info["kernel"] == 1 and info["segment_warp"] == 1 and info["segments"] == 16
    assert launches == 2 and st == 0
    assert oracle.rel_err(x, reference(d, LHS[scheme])) < TOL[precision]


@pytest.mark.parametrize("n,scheme", [(8208, "tri6"), (4617, "tri6"), (1 << 16, "penta10"), (5140, "penta10"),
                                      (1026, "tri6")])
def test_segment_layouts(cuda, n, scheme):
    # 8208 = 16 x 513: every segment of 32 inner partitions (one launch);
    # 4617 = 9 x 513: one CTA of 8 segments and one of 1 (halo rows across
    # CTAs, the last segment's neighbour wraps to segment 0); 2^16: many CTAs
    # per line, both sizes; 5140 = 10 x 514; 1026 = 2 x 513
    d = np.random.default_rng(n).standard_normal((5, n)).astype(np.float32)
    x, info, _, st = solve(d, LHS[scheme], in_dtype=torch.float32)
    assert info["segment_warp"] == 1 and st == 0
    assert oracle.rel_err(x, reference(d.astype(np.float64), LHS[scheme])) < 1e-12


@pytest.mark.parametrize("scheme", ["tri6", "penta10"])
def test_agrees_with_three_launch_path(cuda, scheme):
    d = np.random.default_rng(5).standard_normal((3, 1 << 15)).astype(np.float32)
    ref = reference(d.astype(np.float64), LHS[scheme])
    x0, i0, _, _ = solve(d, LHS[scheme], in_dtype=torch.float32, variant=0)
    x1, i1, l1, _ = solve(d, LHS[scheme], in_dtype=torch.float32, variant=1)
    assert i0["segment_warp"] == 1 and i1["segment_warp"] == 0 and l1 >= 3
    assert oracle.rel_err(x0, ref) < 1e-12 and oracle.rel_err(x1, ref) < 1e-12


def test_one_sweep_error(cuda):
    # the tridiagonal 8192-point lines with a single refinement sweep
    d = np.random.default_rng(8).standard_normal((16, 8192))
    x, _, _, _ = solve(d, LHS["tri6"], "fp32_refine", sweeps=1)
    assert oracle.rel_err(x, reference(d, LHS["tri6"])) < 1e-12


def test_allocation_free_entry(cuda):
    # the warp path needs no per-solve scratch: any plan size runs
    d = np.random.default_rng(9).standard_normal((4, 1 << 18)).astype(np.float32)
    x, info, launches, st = solve(d, LHS["penta10"], in_dtype=torch.float32, noalloc=True)
    assert info["segment_warp"] == 1 and st == 0 and launches == 2
    assert oracle.rel_err(x, reference(d.astype(np.float64), LHS["penta10"])) < 1e-12


def test_non_finite_reported(cuda):
    d = np.random.default_rng(10).standard_normal((3, 8192))
    d[1, 4000] = np.nan
    x, _, _, st = solve(d, LHS["tri6"])
    assert st == abi.CBS_ERR_RANGE
    ref = reference(d[[0, 2]], LHS["tri6"])
    assert oracle.rel_err(x[[0, 2]], ref) < 1e-12  # the other lines are unaffected


@pytest.mark.slow
def test_config3_full_size_sampled(cuda):
    # 32 lines of 2^22, pentadiagonal, FP32 right-hand side, default segments
    d = W.long_lines()
    lines, n = d.shape
    plan = Plan((1, lines, n), 0, lhs=W.PENTA10["lhs"], rhs=None, precision="fp32_refine", sweeps=2,
                in_dtype=torch.float32)
    assert plan.info()["segment_warp"] == 1
    x = plan.solve(torch.from_numpy(d.reshape(1, lines, n)).cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
    for l in (0, 13, 31):
        ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.PENTA10["lhs"]), d[l:l + 1].astype(np.float64))
        assert oracle.rel_err(x[0, l].cpu().numpy(), ref[0]) < 1e-12


def _yz_field(direction, n, a, b, seed, f32=False):
    shape = [(a, b, n), (a, n, b), (n, a, b)][direction]
    d = np.random.default_rng(seed).standard_normal(shape)
    return d.astype(np.float32).astype(np.float64) if f32 else d


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["tri6", "penta10"])
@pytest.mark.parametrize("direction", [1, 2])
def test_yz_lines_warp_per_segment(cuda, direction, scheme, precision):
    # y/z lines of 8192: a CTA per (segment, group of 4 lines adjacent in x);
    # 7 x 3 lines: groups that end mid-row and a ragged last group
    d = _yz_field(direction, 8192, 3, 7, 40 + direction, f32=precision == "fp32")
    dt = torch.float32 if precision == "fp32" else torch.float64
    lhs = LHS[scheme]
    plan = Plan(d.shape, direction, lhs=lhs, rhs=None, precision=precision, sweeps=1, in_dtype=dt)
    info = plan.info()
    y = plan.solve(torch.from_numpy(d).to("cuda", dt))
    torch.cuda.synchronize()
    st = plan.status()
    plan.close()
    assert info["segment_warp"] == 1 and info["segments"] == 16 and st == 0
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(8192, lhs), d, axis=2 - direction)
    assert oracle.rel_err(y.double().cpu().numpy(), ref) < TOL[precision]


@pytest.mark.parametrize("direction", [1, 2])
def test_yz_agrees_with_three_launch_path(cuda, direction):
    # 2^16-point lines (both segment sizes), FP32 right-hand side, 5 x 2 lines
    d = _yz_field(direction, 1 << 16, 2, 5, 77 + direction, f32=True)
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(1 << 16, LHS["penta10"]), d, axis=2 - direction)
    outs = []
    for variant in (0, 1):
        plan = Plan(d.shape, direction, lhs=LHS["penta10"], rhs=None, precision="fp32_refine", sweeps=2,
                    in_dtype=torch.float32)
        abi.cbs_plan_set_variant(plan.handle, variant, 0)
        assert plan.info()["segment_warp"] == 1 - variant
        y = plan.solve(torch.from_numpy(d).to("cuda", torch.float32))
        torch.cuda.synchronize()
        assert plan.status() == 0
        plan.close()
        outs.append(y.cpu().numpy())
    assert oracle.rel_err(outs[0], ref) < 1e-12 and oracle.rel_err(outs[1], ref) < 1e-12
