"""GPU parity of the staggered schemes (Eq. 2, App. A.2) against the FP64 oracle.

The sixth-order staggered first derivative (alpha = 9/62) and the compact
midpoint interpolation (alpha = 3/10) map a periodic field between a grid and
the grid shifted by half a spacing (shift 0: half points -> nodes; shift 1:
nodes -> half points).  Every case feeds the same seeded input to the CUDA
path and the oracle and compares the whole output (norm-wise infinity
relative error): FP64 and FP32 + refinement <= 1e-12, unrefined FP32 <= 2e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Plan, make_desc

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32_refine": 1e-12, "fp32_refine_i64": 1e-12, "fp32": 2e-5}
KINDS = {"staggered": W.STAGGERED6, "midpoint": W.MIDPOINT6}


def _shape(direction, n, others=(12, 10)):
    shape = [others[0], others[1], others[0]]
    shape[2 - direction] = n
    return tuple(shape)


def oracle_ref(f, kind, lhs, rhs, h, shift, axis):
    if kind == "staggered":
        return oracle.staggered_derivative(f, lhs, rhs, h, shift, axis=axis)
    return oracle.midpoint_interpolation(f, lhs, rhs, shift, axis=axis)


def run(f, direction, kind, shift, precision="fp64", segments=0, sweeps=1, lhs=None, rhs=None):
    n = f.shape[2 - direction]
    sch = KINDS[kind]
    lhs = sch["lhs"] if lhs is None else lhs
    rhs = sch["rhs"] if rhs is None else rhs
    h = W.grid_spacing(n)
    plan = Plan(f.shape, direction, lhs=lhs, rhs=rhs, h=h, segments=segments, precision=precision,
                sweeps=sweeps, stencil=kind, shift=shift)
    y = plan.solve(torch.from_numpy(np.ascontiguousarray(f)).cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    info = plan.info()
    plan.close()
    ref = oracle_ref(f, kind, lhs, rhs, h, shift, 2 - direction)
    return oracle.rel_err(y.double().cpu().numpy(), ref), info


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refine", "fp32_refine_i64"])
@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("kind", ["staggered", "midpoint"])
def test_whole_partitions(cuda, kind, shift, direction, precision):
    # n = 64, p = 4 partitions of 16 rows: the direct (FP64 / FP32) and
    # pipelined (refinement) layouts of every direction
    rng = np.random.default_rng(100 + 10 * direction + shift)
    f = rng.uniform(-1, 1, size=_shape(direction, 64))
    err, info = run(f, direction, kind, shift, precision, segments=4)
    assert info["rows_big"] == 16 and info["count_big"] == 4
    assert err < TOL[precision]


@pytest.mark.parametrize("direction", [1, 2])
@pytest.mark.parametrize("n", [256, 512])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("kind", ["staggered", "midpoint"])
def test_refine_yz_32_partitions(cuda, kind, shift, n, direction):
    # 32 partitions of 8 or 16 rows along y or z: the refinement kernel that
    # holds a line per warp (rows and results through shared memory)
    rng = np.random.default_rng(300 + n + 10 * direction + shift)
    f = rng.uniform(-1, 1, size=_shape(direction, n, others=(20, 11)))
    err, info = run(f, direction, kind, shift, "fp32_refine", segments=32)
    assert info["segments"] == 32 and info["rows_big"] == n // 32
    assert err < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refine"])
@pytest.mark.parametrize("n,p", [(50, 4), (61, 5), (200, 13), (97, 7), (16, 1), (8, 2)])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("kind", ["staggered", "midpoint"])
def test_ragged_partitions(cuda, kind, shift, n, p, precision):
    # partitions of unequal sizes go through the staged tile: the shifted
    # window crosses a ragged partition end, and p = 1 / 2 are the
    # degenerate interface systems
    rng = np.random.default_rng(n * 3 + p + shift)
    f = rng.uniform(-1, 1, size=(3, 5, n))
    err, info = run(f, 0, kind, shift, precision, segments=p)
    assert info["segments"] == p
    assert err < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("direction", [0, 1])
def test_32_row_partitions(cuda, precision, direction):
    # 32-row partitions (FP64 / FP32 kernels only), whole and ragged
    for n, p in ((256, 8), (250, 8)):
        rng = np.random.default_rng(n + direction)
        f = rng.uniform(-1, 1, size=_shape(direction, n, (6, 5)))
        for kind in ("staggered", "midpoint"):
            err, _ = run(f, direction, kind, 1, precision, segments=p)
            assert err < TOL[precision], (n, p, kind)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("kind", ["staggered", "midpoint"])
def test_pentadiagonal_one_term_and_two_sweeps(cuda, kind, precision):
    # the kernels take any Toeplitz band and 1 or 2 terms with the staggered
    # stencils (not only the paper's tridiagonal schemes)
    rng = np.random.default_rng(5)
    for direction in (0, 2):
        f = rng.uniform(-1, 1, size=_shape(direction, 96))
        for lhs, rhs in (((0.3, 0.01), KINDS[kind]["rhs"]), (KINDS[kind]["lhs"], (1.1,))):
            for sweeps in (1, 2) if precision == "fp32_refine" else (1,):
                err, _ = run(f, direction, kind, 0, precision, segments=6, sweeps=sweeps, lhs=lhs, rhs=rhs)
                assert err < 1e-12, (direction, lhs, rhs, sweeps)


def test_fourier_modes_at_half_points(cuda):
    # 64^3, the seeded sum of plane waves: derivative to the half points and
    # interpolation back, against the oracle in every direction
    f, _ = W.fourier_cube(64, 8)
    for direction in (0, 1, 2):
        for kind in ("staggered", "midpoint"):
            err, _ = run(f, direction, kind, 1, "fp32_refine", segments=4)
            assert err < 1e-12, (direction, kind)


@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("kind", ["staggered", "midpoint"])
def test_transpose(cuda, kind, shift):
    # lambda = A^{-T} g and grad_in = S^T lambda (S^T: the other shift's
    # stencil, negated for the derivative)
    rng = np.random.default_rng(21 + shift)
    f = rng.uniform(-1, 1, size=(4, 6, 64))
    g = rng.standard_normal(f.shape)
    sch = KINDS[kind]
    h = W.grid_spacing(64)
    for precision in ("fp64", "fp32_refine"):
        plan = Plan(f.shape, 0, lhs=sch["lhs"], rhs=sch["rhs"], h=h, segments=4, precision=precision,
                    stencil=kind, shift=shift)
        gg = torch.from_numpy(g).cuda()
        lam = torch.empty_like(gg)
        gin = torch.empty_like(gg)
        abi.cbs_solve_transpose(plan.handle, gg.data_ptr(), None, lam.data_ptr(), gin.data_ptr(), None, 0)
        torch.cuda.synchronize()
        assert plan.status() == 0
        plan.close()
        lam_ref = oracle.solve_cyclic(oracle.transpose_bands(oracle.toeplitz_bands(64, sch["lhs"])), g)
        if kind == "staggered":
            gin_ref = oracle.staggered_rhs_transpose(lam_ref, sch["rhs"], h, shift)
        else:
            gin_ref = oracle.midpoint_rhs_transpose(lam_ref, sch["rhs"], shift)
        assert oracle.rel_err(lam.cpu().numpy(), lam_ref) < 1e-12
        assert oracle.rel_err(gin.cpu().numpy(), gin_ref) < 1e-12


def test_round_trip_interpolation_is_near_identity(cuda):
    # nodes -> half points -> nodes with the sixth-order interpolator: a
    # smooth field comes back to within the scheme's truncation error
    n = 64
    xs = np.arange(n) * W.grid_spacing(n)
    f = np.exp(np.sin(xs))[None, None, :].repeat(4, 0).repeat(3, 1)
    sch = W.MIDPOINT6
    up = Plan(f.shape, 0, lhs=sch["lhs"], rhs=sch["rhs"], segments=4, stencil="midpoint", shift=1)
    down = Plan(f.shape, 0, lhs=sch["lhs"], rhs=sch["rhs"], segments=4, stencil="midpoint", shift=0)
    mid = up.solve(torch.from_numpy(f).cuda())
    back = down.solve(mid)
    torch.cuda.synchronize()
    up.close()
    down.close()
    ref = oracle.midpoint_interpolation(oracle.midpoint_interpolation(f, sch["lhs"], sch["rhs"], 1),
                                        sch["lhs"], sch["rhs"], 0)
    assert oracle.rel_err(back.cpu().numpy(), ref) < 1e-12
    assert oracle.rel_err(back.cpu().numpy(), f) < 1e-7  # 2.8e-8 at n = 64


def test_batch_runs_staggered_per_problem(cuda):
    # the persistent batch launch has no staggered stencil: a batch holding
    # one runs every problem's own kernels, and the persistent mode is refused
    from paper_2101_02286_gb300.solver import Batch
    d = make_desc((2, 2, 64), 0, lhs=W.STAGGERED6["lhs"], rhs=W.STAGGERED6["rhs"], h=0.1, stencil="staggered")
    h = abi.cbs_batch_create([d])
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_batch_set_mode(h, abi.CBS_BATCH_PERSISTENT)
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED
    abi.cbs_batch_destroy(h)
    b = Batch([((2, 2, 64), 0, dict(lhs=W.STAGGERED6["lhs"], rhs=W.STAGGERED6["rhs"], h=0.1, stencil="staggered"))])
    f = np.random.default_rng(3).uniform(-1, 1, size=(2, 2, 64))
    (y,) = b.solve([torch.from_numpy(f).cuda()])
    torch.cuda.synchronize()
    ref = oracle.staggered_derivative(f, W.STAGGERED6["lhs"], W.STAGGERED6["rhs"], 0.1, 0, axis=2)
    assert oracle.rel_err(y.cpu().numpy(), ref) < 1e-12
    b.close()
