"""GPU parity of the TMA-fed refinement line kernel against the FP64 oracle.

The kernel runs FP32 solves with one refinement sweep on lines of 32
partitions (n = 256 or 512) and rounds the first solution to a per-line grid
before the residual; the tests compare every output element with the oracle
(norm-wise infinity relative error <= 1e-12) on ragged tile counts, all three
directions, both refinement modes, the right-hand-side-given case and the
special paths (zeros, lines of tiny or huge values, values outside the FP32
range), and check that the pipelined kernel (variant 1) agrees as well.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Plan

pytestmark = pytest.mark.gpu

TRI = W.LELE6_TRI


# alpha = 1/3 takes the integer-band residual (A' = 3 A); alpha = 0.3 the
# general one (same sixth-order stencil coefficients: the oracle solves any
# alpha, the kernels do not depend on the scheme being consistent)
LHS = {"int": TRI["lhs"], "gen": (0.3,)}


def solve(f, direction, precision="fp32_refine", rhs=True, variant=0, expect_tma=True, out_offset=0, tile_lines=0,
          lhs="int"):
    n = f.shape[2 - direction]
    plan = Plan(f.shape, direction, lhs=LHS[lhs], rhs=TRI["rhs"] if rhs else None, h=W.grid_spacing(n),
                precision=precision, segments=32)
    info = plan.info()
    assert info["tma"] == (1 if expect_tma else 0), info
    abi.cbs_plan_set_variant(plan.handle, variant, tile_lines)
    x = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    if out_offset:
        buf = torch.empty(f.size + out_offset, dtype=torch.float64, device="cuda")
        y = buf[out_offset:].view(f.shape)
        abi.cbs_solve(plan.handle, x.data_ptr(), y.data_ptr(), 0)
    else:
        y = plan.solve(x)
    torch.cuda.synchronize()
    st = plan.status()
    plan.close()
    return y.cpu().numpy(), st


def reference(f, direction, rhs=True, lhs="int"):
    n = f.shape[2 - direction]
    if rhs:
        return oracle.derivative(f, LHS[lhs], TRI["rhs"], W.grid_spacing(n), axis=2 - direction)
    return oracle.solve_cyclic(oracle.toeplitz_bands(n, LHS[lhs]), f, axis=2 - direction)


def field(direction, n, other, seed):
    """(nz, ny, nx) field with lines of length n along `direction` and a
    ragged number of lines (not a multiple of the 8-line tile)."""
    rng = np.random.default_rng(seed)
    a, b = other
    shape = [(a, b, n), (a, n, b), (n, a, b)][direction]
    return rng.uniform(-1.0, 1.0, size=shape)


@pytest.mark.parametrize("lhs", ["int", "gen"])
@pytest.mark.parametrize("precision", ["fp32_refine", "fp32_refine_i64"])
@pytest.mark.parametrize("n", [512, 256])
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_parity_directions(cuda, direction, n, precision, lhs):
    f = field(direction, n, (5, 14), 100 + direction + n)  # 70 lines: tiles of 4 / 16 and a ragged last one
    got, st = solve(f, direction, precision, lhs=lhs)
    assert st == 0
    assert oracle.rel_err(got, reference(f, direction, lhs=lhs)) < 1e-12


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_parity_many_tiles(cuda, direction):
    # more tiles than resident CTAs, so every CTA reuses both tile buffers
    f = field(direction, 256, (40, 46), 7 + direction)
    got, st = solve(f, direction)
    assert st == 0
    assert oracle.rel_err(got, reference(f, direction)) < 1e-12


@pytest.mark.parametrize("precision", ["fp32_refine", "fp32_refine_i64"])
@pytest.mark.parametrize("tile_lines", [4, 16])
@pytest.mark.parametrize("direction", [1, 2])
def test_tile_shapes(cuda, direction, tile_lines, precision):
    # y/z tiles of 4 lines (two buffers) and of 16 lines (one buffer, two
    # lines per warp); 30 x-positions: a ragged last tile for both shapes
    f = field(direction, 512, (3, 30), 60 + direction + tile_lines)
    got, st = solve(f, direction, precision, tile_lines=tile_lines)
    assert st == 0
    assert oracle.rel_err(got, reference(f, direction)) < 1e-12


@pytest.mark.parametrize("direction", [0, 1])
def test_rhs_given(cuda, direction):
    f = field(direction, 512, (3, 6), 31 + direction)
    got, st = solve(f, direction, rhs=False)
    assert st == 0
    assert oracle.rel_err(got, reference(f, direction, rhs=False)) < 1e-12


@pytest.mark.parametrize("direction", [0, 2])
def test_variants_agree(cuda, direction):
    f = field(direction, 512, (4, 10), 55 + direction)
    ref = reference(f, direction)
    got0, _ = solve(f, direction, variant=0)
    got1, _ = solve(f, direction, variant=1)
    assert oracle.rel_err(got0, ref) < 1e-12
    assert oracle.rel_err(got1, ref) < 1e-12


@pytest.mark.parametrize("lhs", ["int", "gen"])
def test_closed_form_mode(cuda, lhs):
    # a single Fourier mode along x: the scheme's modified wavenumber (Eq. 1)
    # k'h = (a sin kh + (b/2) sin 2kh) / (1 + 2 alpha cos kh), here for the
    # alpha of each residual path
    n, k = 512, 37
    h = W.grid_spacing(n)
    xg = np.arange(n) * h
    f = np.broadcast_to(np.sin(k * xg), (2, 4, n)).copy()
    got, st = solve(f, 0, lhs=lhs)
    assert st == 0
    a, b = TRI["rhs"]
    al = LHS[lhs][0]
    th = k * h
    kp = (a * np.sin(th) + 0.5 * b * np.sin(2 * th)) / (1 + 2 * al * np.cos(th)) / h
    exact = np.broadcast_to(kp * np.cos(k * xg), f.shape)
    assert oracle.rel_err(got, exact) < 1e-12


def test_special_values(cuda):
    # line 0: all zeros; 1: zeros scattered in noise; 2-5: values ~1e-30,
    # 1e30, 1e-100, 1e200 (rescaled by a power of two inside the kernel);
    # 6: a single spike; 7: one value of 1e300 in O(1) noise (the line is
    # rescaled to its spike); 8: values ~2^-50 (inside the range, no
    # rescaling).  Each line is checked against its own scale.
    rng = np.random.default_rng(3)
    f = rng.uniform(-1, 1, size=(1, 12, 512))
    f[0, 0] = 0.0
    f[0, 1, ::7] = 0.0
    f[0, 2] *= 1e-30
    f[0, 3] *= 1e30
    f[0, 4] *= 1e-100
    f[0, 5] *= 1e200
    f[0, 6] = 0.0
    f[0, 6, 100] = 1.0
    f[0, 7, 17] = 1e300
    f[0, 8] *= 2.0 ** -50
    got, st = solve(f, 0)
    assert st == 0
    ref = reference(f, 0)
    assert np.all(got[0, 0] == 0.0)
    for k in range(1, 12):
        assert oracle.rel_err(got[0, k], ref[0, k]) < 1e-12, k


def test_non_finite_input_reports_status(cuda):
    f = np.random.default_rng(4).uniform(-1, 1, size=(1, 3, 512))
    for bad in (np.inf, np.nan):
        f[0, 1, 17] = bad
        got, st = solve(f, 0)
        assert st == abi.CBS_ERR_RANGE
        ref = reference(f, 0)
        for k in (0, 2):  # the other lines are unaffected
            assert oracle.rel_err(got[0, k], ref[0, k]) < 1e-12


def test_unaligned_output_takes_line_kernel(cuda):
    # an output that starts 8 bytes past a 16-byte boundary cannot be a TMA
    # tensor: the pipelined / staged kernels run, with the same accuracy
    f = field(0, 512, (2, 3), 9)
    got, st = solve(f, 0, out_offset=1)
    assert st == 0
    assert oracle.rel_err(got, reference(f, 0)) < 1e-12


def test_transpose_through_tma(cuda):
    # grad_in = S^T A^{-T} g runs the same kernel with negated stencil weights
    rng = np.random.default_rng(12)
    f = rng.uniform(-1, 1, size=(2, 6, 512))
    g = rng.uniform(-1, 1, size=f.shape)
    n = 512
    h = W.grid_spacing(n)
    plan = Plan(f.shape, 0, lhs=TRI["lhs"], rhs=TRI["rhs"], h=h, precision="fp32_refine", segments=32)
    assert plan.info()["tma"] == 1
    gt = torch.from_numpy(g).cuda()
    gin = torch.empty_like(gt)
    lam = torch.empty_like(gt)
    abi.cbs_solve_transpose(plan.handle, gt.data_ptr(), None, lam.data_ptr(), gin.data_ptr(), None, 0)
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
    lam_ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, TRI["lhs"]), g, axis=-1)
    gin_ref = oracle.central_rhs_transpose(lam_ref, TRI["rhs"], h, axis=-1)
    assert oracle.rel_err(lam.cpu().numpy(), lam_ref) < 1e-12
    assert oracle.rel_err(gin.cpu().numpy(), gin_ref) < 1e-12
