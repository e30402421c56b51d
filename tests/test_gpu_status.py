"""The device status word (cbs_status_poll): every condition a kernel reports,
made to happen on purpose without faulting the GPU.

  * CBS_ERR_TIMEOUT: a tile wait of the TMA-fed kernel that nothing
    satisfies (cbs_plan_inject_fault: one tile load is not issued and the
    wait limit is 1 ms); the context stays usable.
  * CBS_ERR_SINGULAR: a variable-band line with alpha_i = 1/2 and even n,
    a singular cyclic system (symbol 1 + cos theta = 0 at theta = pi); the
    other lines of the same launch stay correct.
  * CBS_ERR_RANGE: refinement-mode inputs outside the FP32 range in the
    pipelined line kernels and in a batch.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.autograd import variable_plan
from paper_2101_02286_gb300.solver import Batch, Plan

pytestmark = pytest.mark.gpu
TRI = W.LELE6_TRI
C4 = W.CENTRAL4["rhs"]


def test_timeout_injected_and_context_usable(cuda):
    n = 512
    f = np.random.default_rng(1).uniform(-1, 1, size=(4, 24, n))
    h = W.grid_spacing(n)
    plan = Plan(f.shape, 0, lhs=TRI["lhs"], rhs=TRI["rhs"], h=h, precision="fp32_refine", segments=32)
    assert plan.info()["tma"] == 1
    x = torch.from_numpy(f).cuda()
    abi.cbs_plan_inject_fault(plan.handle, 1)
    plan.solve(x)
    torch.cuda.synchronize()
    assert plan.status() == abi.CBS_ERR_TIMEOUT
    assert plan.status() == abi.CBS_OK  # polling clears the word
    abi.cbs_plan_inject_fault(plan.handle, 0)
    y = plan.solve(x)
    torch.cuda.synchronize()
    assert plan.status() == abi.CBS_OK
    assert oracle.rel_err(y.cpu().numpy(), oracle.derivative(f, TRI["lhs"], TRI["rhs"], h, axis=2)) < 1e-12
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_variable_singular_line(cuda, precision):
    n = 64  # even: alpha = 1/2 makes the cyclic line singular
    rng = np.random.default_rng(7)
    f = rng.uniform(-1, 1, size=(2, 5, n))
    al = rng.uniform(0.2, 0.4, size=f.shape)
    al[1, 2, :] = 0.5
    dt = torch.float64 if precision == "fp64" else torch.float32
    aa = torch.from_numpy(al).to("cuda", dt)
    plan = variable_plan(f.shape, 0, aa, C4, W.grid_spacing(n), precision)
    x = plan.solve(torch.from_numpy(f).to("cuda", dt)).double().cpu().numpy()
    torch.cuda.synchronize()
    assert plan.status() == abi.CBS_ERR_SINGULAR
    plan.close()
    good = np.ones(f.shape[:2], dtype=bool)
    good[1, 2] = False
    ref = oracle.derivative_variable_tri(f[good], al[good] if precision == "fp64" else
                                         aa.double().cpu().numpy()[good], C4, W.grid_spacing(n), axis=-1)
    assert oracle.rel_err(x[good], ref) < (1e-12 if precision == "fp64" else 2e-5)


def test_variable_regular_reports_ok(cuda):
    n = 64
    rng = np.random.default_rng(8)
    f = rng.uniform(-1, 1, size=(2, 5, n))
    al = rng.uniform(0.2, 0.4, size=f.shape)
    plan = variable_plan(f.shape, 0, torch.from_numpy(al).cuda(), C4, W.grid_spacing(n), "fp64")
    plan.solve(torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    assert plan.status() == abi.CBS_OK
    plan.close()


@pytest.mark.parametrize("value", [1e300, np.inf, np.nan])
def test_line_kernel_refine_out_of_range(cuda, value):
    # the pipelined / staged line kernels (variant 1) work in the FP32 range
    n = 256
    f = np.random.default_rng(9).uniform(-1, 1, size=(1, 4, n))
    f[0, 2, 30] = value
    plan = Plan(f.shape, 0, lhs=TRI["lhs"], rhs=TRI["rhs"], h=W.grid_spacing(n), precision="fp32_refine")
    abi.cbs_plan_set_variant(plan.handle, 1, 0)
    y = plan.solve(torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    assert plan.status() == abi.CBS_ERR_RANGE
    ref = oracle.derivative(f[:, [0, 1, 3]], TRI["lhs"], TRI["rhs"], W.grid_spacing(n), axis=2)
    assert oracle.rel_err(y.cpu().numpy()[:, [0, 1, 3]], ref) < 1e-12  # the other lines
    plan.close()


def test_batch_status(cuda):
    shapes = [(8, 8, 64), (4, 16, 32)]
    specs = [(sh, 0, dict(lhs=TRI["lhs"], rhs=TRI["rhs"], h=W.grid_spacing(sh[2]), precision="fp32_refine"))
             for sh in shapes]
    b = Batch(specs)
    rng = np.random.default_rng(10)
    ins = [torch.from_numpy(rng.uniform(-1, 1, size=sh)).cuda() for sh in shapes]
    b.solve(ins)
    torch.cuda.synchronize()
    assert abi.cbs_batch_status_poll(b.handle) == abi.CBS_OK
    ins[1][0, 3, 5] = float("inf")
    b.solve(ins)
    torch.cuda.synchronize()
    assert abi.cbs_batch_status_poll(b.handle) == abi.CBS_ERR_RANGE
    assert abi.cbs_batch_status_poll(b.handle) == abi.CBS_OK
    b.close()
