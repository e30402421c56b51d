"""GPU parity of block-tridiagonal systems with 2 x 2 block entries (Sec. 1).

Lines hold points of two unknowns each (point-major); point m couples to
points m - 1, m, m + 1 through the blocks L, D, U.  The library solves the
flattened banded form (half bandwidth 3, rows periodic with period 2) with the
partition method, partitions made of whole points.  Every case compares the
whole output element by element with the oracle's banded LU + Woodbury solve
of the flattened matrix (pinned against LAPACK on the block matrix assembled
block by block): FP64 <= 1e-12, FP32 <= 2e-5 (norm-wise infinity relative
error).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300.solver import Plan

pytestmark = pytest.mark.gpu

# diagonally dominant, neither symmetric nor diagonal blocks
BLK = (np.array([[0.21, 0.07], [-0.05, 0.18]]), np.array([[1.0, 0.15], [-0.12, 0.9]]),
       np.array([[0.24, -0.06], [0.04, 0.2]]))
# weaker dominance: the point-coupling blocks nearly as large as the diagonal
WEAK = (np.array([[0.4, 0.1], [0.05, 0.35]]), np.array([[1.0, -0.2], [0.1, 1.0]]),
        np.array([[0.38, -0.08], [0.12, 0.36]]))
TOL = {"fp64": 1e-12, "fp32": 2e-5}


def run(f, direction, blocks=BLK, precision="fp64", segments=0, cyclic=True):
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = Plan(f.shape, direction, blocks=blocks, segments=segments, precision=precision, in_dtype=dt,
                cyclic=cyclic)
    y = plan.solve(torch.from_numpy(np.ascontiguousarray(f)).to("cuda", dt))
    torch.cuda.synchronize()
    info = plan.info()
    assert plan.status() == 0
    plan.close()
    return y.double().cpu().numpy(), info


def reference(f, direction, blocks=BLK, cyclic=True):
    ax = 2 - direction
    n = f.shape[ax]
    bands = oracle.block_tridiagonal_bands(n // 2, *blocks)
    if cyclic:
        return oracle.solve_cyclic(bands, f, axis=ax)
    return oracle.solve_acyclic(bands, f, axis=ax)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("n", [64, 96, 100, 256, 512])
def test_block_lines_match_oracle(cuda, direction, n, precision):
    shape = [6, 10, 12]
    shape[2 - direction] = n
    f = np.random.default_rng(n + 10 * direction).uniform(-1, 1, size=tuple(shape))
    if precision == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    y, info = run(f, direction, precision=precision)
    assert info["kernel"] == 0 and info["bandwidth"] == 7
    assert info["rows_big"] % 2 == 0 and info["rows_small"] % 2 == 0  # whole points per partition
    assert oracle.rel_err(y, reference(f, direction)) < TOL[precision]


@pytest.mark.parametrize("segments", [1, 2, 3, 5, 7, 13, 16, 31, 32])
@pytest.mark.parametrize("cyclic", [True, False])
def test_block_partition_counts(cuda, segments, cyclic):
    # 1 to 32 lanes, ragged partitions: 11 s + 3 points over s partitions
    # (11 to 13 points, 22 to 26 rows each; 14 points when s = 1)
    n = 2 * (11 * segments + 3) if segments > 1 else 2 * 14
    f = np.random.default_rng(segments).uniform(-1, 1, size=(3, 5, n))
    y, info = run(f, 0, segments=segments, cyclic=cyclic)
    assert info["segments"] == segments
    assert oracle.rel_err(y, reference(f, 0, cyclic=cyclic)) < 1e-12


@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("cyclic", [True, False])
def test_block_weakly_dominant(cuda, direction, cyclic):
    shape = [8, 8, 8]
    shape[2 - direction] = 128
    f = np.random.default_rng(7).standard_normal(tuple(shape))
    y, _ = run(f, direction, blocks=WEAK, cyclic=cyclic)
    assert oracle.rel_err(y, reference(f, direction, blocks=WEAK, cyclic=cyclic)) < 1e-12


def test_block_decoupled_equals_two_scalar_systems(cuda):
    # diagonal blocks: the two unknowns of every point form two independent
    # tridiagonal systems, each solved against the oracle's Thomas + SM solve
    L, D, U = np.diag([0.2, 0.3]), np.diag([1.0, 1.1]), np.diag([0.25, 0.15])
    f = np.random.default_rng(2).uniform(-1, 1, size=(4, 6, 128))
    y, _ = run(f, 0, blocks=(L, D, U))
    for c in range(2):
        tri = np.zeros((3, 64))
        tri[0], tri[1], tri[2] = L[c, c], D[c, c], U[c, c]
        assert oracle.rel_err(y[..., c::2], oracle.solve_cyclic(tri, f[..., c::2])) < 1e-12


def test_block_plans_reject_what_they_do_not_run(cuda):
    f = torch.zeros((2, 2, 64), dtype=torch.float64, device="cuda")
    plan = Plan(tuple(f.shape), 0, blocks=BLK)
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_solve_transpose(plan.handle, f.data_ptr(), 0, f.data_ptr(), 0, 0, 0)
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED
    plan.close()
    with pytest.raises(abi.CbsError) as e:  # long lines: partitions of more than 32 rows
        Plan((1, 2, 4096), 0, blocks=BLK)
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED
