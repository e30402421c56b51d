"""GPU parity of the long-line path (segments across CTAs): the
pentadiagonal precision workload and its smaller relatives, against the
FP64 oracle (banded LU + Woodbury)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Plan

pytestmark = pytest.mark.gpu


def _solve(d32, lhs, segments, precision="fp32_refine", sweeps=2, in_dtype=torch.float32):
    lines, n = d32.shape
    plan = Plan((1, lines, n), 0, lhs=lhs, rhs=None, segments=segments, precision=precision, sweeps=sweeps,
                in_dtype=in_dtype)
    x = plan.solve(torch.from_numpy(d32.reshape(1, lines, n)).to("cuda", in_dtype))
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    return x.double().cpu().numpy().reshape(lines, n), info


@pytest.mark.parametrize("lhs", [W.PENTA10["lhs"], W.LELE6_TRI["lhs"]])
@pytest.mark.parametrize("n,p", [(4096, 8), (8192, 16), (3072, 3), (5632, 11), (2048, 1), (16384, 64), (6144, 2)])
def test_long_refine(cuda, lhs, n, p):
    d = np.random.default_rng(n + p).standard_normal((3, n)).astype(np.float32)
    x, info = _solve(d, lhs, p)
    assert info["kernel"] == 1 and info["segments"] == p
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, lhs), d.astype(np.float64))
    assert oracle.rel_err(x, ref) < 1e-12


@pytest.mark.parametrize("precision,tol,sweeps", [("fp64", 1e-12, 1), ("fp32", 2e-5, 1), ("fp32_refine", 1e-12, 1)])
def test_long_precisions(cuda, precision, tol, sweeps):
    n, p = 8192, 8
    d = np.random.default_rng(7).standard_normal((2, n))
    dt = torch.float32 if precision == "fp32" else torch.float64
    x, _ = _solve(d, W.LELE6_TRI["lhs"], p, precision=precision, sweeps=sweeps, in_dtype=dt)
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.LELE6_TRI["lhs"]),
                              d.astype(np.float32).astype(np.float64) if dt == torch.float32 else d)
    assert oracle.rel_err(x, ref) < tol


def test_long_unrefined_fp32_error_scale(cuda):
    # one FP32 solve of the pentadiagonal system stays within 2e-5
    n = 8192
    d = np.random.default_rng(3).standard_normal((2, n)).astype(np.float32)
    x, _ = _solve(d, W.PENTA10["lhs"], 8, precision="fp32", sweeps=1)
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.PENTA10["lhs"]), d.astype(np.float64))
    assert oracle.rel_err(x, ref) < 2e-5


@pytest.mark.slow
def test_long_full_workload_sampled(cuda):
    # 32 lines of 2^22, pentadiagonal, FP32 right-hand side, 1024 segments
    d = W.long_lines()
    lines, n = d.shape
    plan = Plan((1, lines, n), 0, lhs=W.PENTA10["lhs"], rhs=None, segments=1024, precision="fp32_refine",
                sweeps=2, in_dtype=torch.float32)
    x = plan.solve(torch.from_numpy(d.reshape(1, lines, n)).cuda())
    torch.cuda.synchronize()
    plan.close()
    for l in (0, 17, 31):
        ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.PENTA10["lhs"]), d[l:l + 1].astype(np.float64))
        assert oracle.rel_err(x[0, l].cpu().numpy(), ref[0]) < 1e-12


@pytest.mark.parametrize("precision,tol,sweeps,r_lhs", [("fp32_refine", 1e-12, 2, W.PENTA10["lhs"]),
                                                         ("fp64", 1e-12, 1, W.PENTA10["lhs"]),
                                                         ("fp32", 2e-5, 1, W.LELE6_TRI["lhs"])])
def test_long_two_segment_sizes(cuda, precision, tol, sweeps, r_lhs):
    # p segments of 2^16 rows that do not divide n; with n - p r a multiple of 16
    # the segments get 16 K + r or 16 (K - 1) + r rows (whole 16-row inner
    # partitions), both sizes present
    r = len(r_lhs)
    n, p = 1 << 16, (24 if r == 2 else 48)  # n - p r divisible by 16, n by neither p
    d = np.random.default_rng(31).standard_normal((2, n)).astype(np.float32)
    x, info = _solve(d, r_lhs, p, precision=precision, sweeps=sweeps)
    assert info["kernel"] == 1 and info["segments"] == p
    assert info["rows_big"] - info["rows_small"] == 16 and (info["rows_big"] - r) % 16 == 0
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, r_lhs), d.astype(np.float64))
    assert oracle.rel_err(x, ref) < tol


def test_long_refine_fp64_interface(cuda):
    n, p = 1 << 15, 16
    d = np.random.default_rng(77).standard_normal((2, n)).astype(np.float32)
    x, info = _solve(d, W.PENTA10["lhs"], p, precision="fp32_refine_i64", sweeps=2)
    assert info["kernel"] == 1
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.PENTA10["lhs"]), d.astype(np.float64))
    assert oracle.rel_err(x, ref) < 1e-12


@pytest.mark.parametrize("p", [3, 7, 31, 63])
@pytest.mark.parametrize("precision,sweeps", [("fp64", 1), ("fp32_refine", 1)])
def test_long_lines_2n_minus_1_segments(cuda, p, precision, sweeps):
    # the paper's 2^n - 1 partition counts on lines of 8192 (detach / reattach
    # in the segment-level interface system); p does not divide n, so the
    # segments have ceil(n / p) or floor(n / p) rows
    n = 8192
    d = np.random.default_rng(p).standard_normal((3, n))
    x, info = _solve(d, W.LELE6_TRI["lhs"], p, precision=precision, sweeps=sweeps, in_dtype=torch.float64)
    assert info["kernel"] == 1 and info["segments"] == p and info["detach_steps"] > 0
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.LELE6_TRI["lhs"]), d)
    assert oracle.rel_err(x, ref) < 1e-12


@pytest.mark.slow
def test_long_more_lines_than_a_grid_dimension(cuda):
    # 65540 lines (> 65535, the limit of a CUDA grid's y and z extents)
    lines, n, p = 65540, 2048, 2
    d = np.random.default_rng(8).standard_normal((lines, n)).astype(np.float32)
    plan = Plan((1, lines, n), 0, lhs=W.LELE6_TRI["lhs"], rhs=None, segments=p, precision="fp32_refine",
                in_dtype=torch.float32)
    assert plan.info()["kernel"] == 1
    x = plan.solve(torch.from_numpy(d.reshape(1, lines, n)).cuda())
    torch.cuda.synchronize()
    plan.close()
    pick = np.random.default_rng(9).integers(0, lines, size=16)
    pick[0], pick[1] = 0, lines - 1
    got = x[0, pick].cpu().numpy()
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.LELE6_TRI["lhs"]), d[pick].astype(np.float64))
    assert oracle.rel_err(got, ref) < 1e-12
