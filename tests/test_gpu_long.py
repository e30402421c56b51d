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


# ---------------------------------------------------------------- y / z lines
def _solve_dir(f, direction, lhs, segments, precision, sweeps=1, in_dtype=torch.float64):
    plan = Plan(f.shape, direction, lhs=lhs, rhs=None, segments=segments, precision=precision, sweeps=sweeps,
                in_dtype=in_dtype)
    x = plan.solve(torch.from_numpy(np.ascontiguousarray(f)).to("cuda", in_dtype))
    torch.cuda.synchronize()
    info = plan.info()
    assert plan.status() == 0
    plan.close()
    return x.double().cpu().numpy(), info


@pytest.mark.parametrize("direction", [1, 2])
@pytest.mark.parametrize("precision,tol,sweeps", [("fp64", 1e-12, 1), ("fp32", 2e-5, 1), ("fp32_refine", 1e-12, 1),
                                                  ("fp32_refine", 1e-12, 2), ("fp32_refine_i64", 1e-12, 1)])
@pytest.mark.parametrize("lhs,n,p", [(W.LELE6_TRI["lhs"], 2048, 2), (W.LELE6_TRI["lhs"], 2050, 2),
                                     (W.LELE6_TRI["lhs"], 3000, 3), (W.LELE6_TRI["lhs"], 4096, 7),
                                     (W.PENTA10["lhs"], 2048, 2), (W.PENTA10["lhs"], 2052, 2),
                                     (W.PENTA10["lhs"], 3000, 3), (W.PENTA10["lhs"], 1536, 2),
                                     (W.LELE6_TRI["lhs"], 4096, 2), (W.PENTA10["lhs"], 3000, 2),
                                     (W.LELE6_TRI["lhs"], 2048, 4), (W.LELE6_TRI["lhs"], 2052, 4),
                                     (W.PENTA10["lhs"], 2052, 4)])
def test_long_y_z_lines(cuda, direction, precision, tol, sweeps, lhs, n, p):
    # strided lines, a tile of 8 adjacent lines per CTA; line counts that
    # are not a multiple of the tile (12 x 5 and 12 x 3 lines); whole
    # 16-row inner partitions when n - p r is a multiple of 16 (2050 tri,
    # 2052 penta, 2052 / 4 tri), ragged ones otherwise; tiles of 8 lines up
    # to 32 inner partitions (2048 / 4), of 4 up to 64 (2048 / 2), of 2 up to
    # 128 (4096 / 2, 3000 / 2)
    if precision == "fp32_refine" and sweeps == 1 and lhs == W.PENTA10["lhs"]:
        sweeps = 2  # the pentadiagonal system needs the second sweep for 1e-12
    shape = (5, n, 12) if direction == 1 else (n, 3, 12)
    rng = np.random.default_rng(n + 10 * p + direction)
    f = rng.standard_normal(shape)
    dt = torch.float32 if precision == "fp32" else torch.float64
    x, info = _solve_dir(f, direction, lhs, p, precision, sweeps, dt)
    assert info["kernel"] == 1 and info["segments"] == p
    assert info["lines"] == (60 if direction == 1 else 36)
    src = f.astype(np.float32).astype(np.float64) if dt == torch.float32 else f
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, lhs), src, axis=2 - direction)
    assert oracle.rel_err(x, ref) < tol


@pytest.mark.parametrize("direction", [1, 2])
def test_long_y_z_fp32_input(cuda, direction):
    # FP32 right-hand side, FP64 solution (the long-line precision workload's
    # element types) along y and z
    n = 4096
    shape = (3, n, 16) if direction == 1 else (n, 2, 16)
    f = np.random.default_rng(40 + direction).standard_normal(shape).astype(np.float32)
    x, _ = _solve_dir(f, direction, W.PENTA10["lhs"], 4, "fp32_refine", 2, torch.float32)
    ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.PENTA10["lhs"]), f.astype(np.float64), axis=2 - direction)
    assert oracle.rel_err(x, ref) < 1e-12


def test_long_y_z_segment_limit(cuda):
    # y/z segments hold at most 128 inner partitions of 16 rows: one segment
    # of 4096 rows is refused, the default segment count fits
    from paper_2101_02286_gb300 import abi
    f = np.zeros((2, 4096, 8))
    with pytest.raises(abi.CbsError) as e:
        Plan(f.shape, 1, lhs=W.LELE6_TRI["lhs"], rhs=None, segments=1, precision="fp64")
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED
    plan = Plan(f.shape, 1, lhs=W.LELE6_TRI["lhs"], rhs=None, precision="fp64")
    assert plan.info()["kernel"] == 1 and plan.info()["segments"] == 8
    plan.close()


@pytest.mark.slow
@pytest.mark.parametrize("direction", [1, 2])
def test_paper_workload_y_z_sampled(cuda, direction):
    # the paper's workload along y and z: 256^2 lines of 8192, tridiagonal
    # alpha = 1/3, p = 8 and p = 7, checked on sampled lines
    shape = (256, 8192, 256) if direction == 1 else (8192, 256, 256)
    rng = np.random.default_rng(50 + direction)
    f = rng.standard_normal(shape)
    fi = torch.from_numpy(f).cuda()
    lhs = W.LELE6_TRI["lhs"]
    for p in (8, 7):
        plan = Plan(shape, direction, lhs=lhs, rhs=None, segments=p, precision="fp32_refine")
        x = plan.solve(fi)
        torch.cuda.synchronize()
        assert plan.status() == 0
        plan.close()
        xs = x.cpu().numpy()
        del x
        ii = rng.integers(0, 256, size=(8, 2))
        if direction == 1:
            lines = np.stack([f[i, :, j] for i, j in ii])
            got = np.stack([xs[i, :, j] for i, j in ii])
        else:
            lines = np.stack([f[:, i, j] for i, j in ii])
            got = np.stack([xs[:, i, j] for i, j in ii])
        ref = oracle.solve_cyclic(oracle.toeplitz_bands(8192, lhs), lines)
        assert oracle.rel_err(got, ref) < 1e-12, p
