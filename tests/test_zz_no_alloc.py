"""The allocation-free long-line entry point (cbs_solve_noalloc).

It is meant for callers that cannot allocate device memory while they solve
(under an application-owned allocator, with a fixed memory footprint): it runs the same kernels as cbs_solve on a fixed scratch
array in the library instead of the plan's buffer.  Checked through the
C-ABI against cbs_solve on two calls in a row, plus the size limit.  This
file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Plan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [1, 0])
def test_noalloc_matches_solve_twice(cuda, variant):
    # variant 1: the end-row / interface / segment launches on the fixed
    # scratch; variant 0: a warp per segment (512-row segments), no scratch
    lines, n, p = 4, 8192, 16
    plan = Plan((1, lines, n), 0, lhs=W.PENTA10["lhs"], rhs=None, segments=p, precision="fp32_refine", sweeps=2,
                in_dtype=torch.float32)
    abi.cbs_plan_set_variant(plan.handle, variant, 0)
    assert plan.info()["kernel"] == 1 and plan.info()["segment_warp"] == (1 - variant)
    rng = np.random.default_rng(2024)
    for call in range(2):  # two calls in a row on the shared scratch
        d = rng.standard_normal((1, lines, n)).astype(np.float32)
        x = torch.from_numpy(d).cuda()
        ref = plan.solve(x)
        solve_launches = abi.cbs_last_launch_count()  # 3 or 4 (two segment sizes); 2 for the warp path
        out = torch.full_like(ref, float("nan"))
        abi.cbs_solve_noalloc(plan.handle, x.data_ptr(), out.data_ptr(), 0)
        assert abi.cbs_last_launch_count() == solve_launches >= (3 if variant else 2)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all()
        assert oracle.rel_err(got, want) < 1e-12, call
        exact = oracle.solve_cyclic(oracle.toeplitz_bands(n, W.PENTA10["lhs"]), d[0].astype(np.float64))
        assert oracle.rel_err(got[0], exact) < 1e-12, call
    plan.close()


def test_noalloc_rejects_oversize_and_on_chip_plans(cuda):
    # 64 lines x 2048 segments x 5 r (r = 2) = 1310720 doubles > 524288
    big = Plan((1, 64, 2048 * 64), 0, lhs=W.PENTA10["lhs"], rhs=None, segments=2048, precision="fp32_refine",
               in_dtype=torch.float32)
    x = torch.zeros((1, 64, 2048 * 64), dtype=torch.float32, device="cuda")
    y = torch.zeros((1, 64, 2048 * 64), dtype=torch.float64, device="cuda")
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_solve_noalloc(big.handle, x.data_ptr(), y.data_ptr(), 0)
    assert e.value.status == abi.CBS_ERR_INVALID_ARG and "exceeds" in str(e.value)
    big.close()
    small = Plan((2, 2, 64), 0, lhs=(1 / 3,), rhs=(14 / 9, 1 / 9), h=0.1)
    a = torch.zeros((2, 2, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_solve_noalloc(small.handle, a.data_ptr(), torch.empty_like(a).data_ptr(), 0)
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED
    small.close()


@pytest.mark.parametrize("dims,direction,lhs", [
    ((1, 3, 8191), 0, W.PENTA10["lhs"]),   # 8191 = 16 x 511 + 15: two segment sizes
    ((2, 8191, 4), 1, W.LELE6_TRI["lhs"]),  # y-lines, strided
])
def test_noalloc_ragged_segments(cuda, dims, direction, lhs):
    # the three-launch path on the fixed scratch with segments of two sizes
    # (the last one shorter), FP64 in and out, against the oracle directly
    plan = Plan(dims, direction, lhs=lhs, rhs=None, segments=16, precision="fp64")
    abi.cbs_plan_set_variant(plan.handle, 1, 0)
    assert plan.info()["kernel"] == 1 and plan.info()["segment_warp"] == 0
    rng = np.random.default_rng(77)
    axis = 2 - direction
    n = dims[axis]
    for call in range(2):
        d = rng.standard_normal(dims)
        x = torch.from_numpy(d).cuda()
        out = torch.full_like(x, float("nan"))
        abi.cbs_solve_noalloc(plan.handle, x.data_ptr(), out.data_ptr(), 0)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        exact = oracle.solve_cyclic(oracle.toeplitz_bands(n, lhs), d, axis=axis)
        assert oracle.rel_err(got, exact) < 1e-12, call
    plan.close()
