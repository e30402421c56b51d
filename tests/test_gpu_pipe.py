"""Solves from host memory through the C-ABI pipe (cbs_pipe_*): one upload of
the field, every plan's solve, every result downloaded inside the call, with
the device buffers alternating between calls.  Checked element by element
against the device-resident solves and the FP64 oracle on three calls in a
row with new data each time."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Pipe, Plan

pytestmark = pytest.mark.gpu
TRI = W.LELE6_TRI


def _plans(shape, precisions, dtype=torch.float64):
    plans = []
    for d, prec in enumerate(precisions):
        n = shape[2 - d]
        plans.append(Plan(shape, d, lhs=TRI["lhs"], rhs=TRI["rhs"], h=W.grid_spacing(n), precision=prec,
                          in_dtype=dtype))
    return plans


def test_pipe_three_directions_three_calls(cuda):
    shape = (24, 40, 64)
    plans = _plans(shape, ["fp32_refine", "fp64", "fp32_refine"])
    pipe = Pipe(plans)
    f_pin = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    outs = [torch.empty(shape, dtype=torch.float64, pin_memory=True) for _ in plans]
    s = torch.cuda.Stream()
    rng = np.random.default_rng(3)
    for call in range(3):
        f = rng.uniform(-1, 1, size=shape)
        f_pin.copy_(torch.from_numpy(f))
        pipe.solve(f_pin, outs, s)
        assert abi.cbs_last_launch_count() >= 3
        s.synchronize()
        dev = torch.from_numpy(f).cuda()
        for d, (p, y) in enumerate(zip(plans, outs)):
            want = p.solve(dev).cpu().numpy()
            assert oracle.rel_err(y.numpy(), want) < 1e-14, (call, d)
            n = shape[2 - d]
            ref = oracle.derivative(f, TRI["lhs"], TRI["rhs"], W.grid_spacing(n), axis=2 - d)
            assert oracle.rel_err(y.numpy(), ref) < 1e-12, (call, d)
    pipe.close()
    for p in plans:
        p.close()


def test_pipe_fp32_field(cuda):
    shape = (8, 16, 128)
    plans = _plans(shape, ["fp32", "fp32"], dtype=torch.float32)[:1]
    plans.append(Plan(shape, 1, lhs=TRI["lhs"], rhs=TRI["rhs"], h=W.grid_spacing(16), precision="fp32",
                      in_dtype=torch.float32))
    pipe = Pipe(plans)
    f = np.random.default_rng(5).uniform(-1, 1, size=shape).astype(np.float32)
    f_pin = torch.from_numpy(f).pin_memory()
    outs = [torch.empty(shape, dtype=torch.float32, pin_memory=True) for _ in plans]
    pipe.solve(f_pin, outs)
    torch.cuda.synchronize()
    for d, y in enumerate(outs):
        n = shape[2 - d]
        ref = oracle.derivative(f.astype(np.float64), TRI["lhs"], TRI["rhs"], W.grid_spacing(n), axis=2 - d)
        assert oracle.rel_err(y.double().numpy(), ref) < 2e-5
    pipe.close()
    for p in plans:
        p.close()


def test_pipe_rejects_plans_of_different_fields(cuda):
    a = Plan((4, 4, 64), 0, lhs=TRI["lhs"], rhs=TRI["rhs"], h=0.1)
    b = Plan((4, 8, 64), 0, lhs=TRI["lhs"], rhs=TRI["rhs"], h=0.1)
    with pytest.raises(abi.CbsError):
        abi.cbs_pipe_create([a.handle, b.handle])
    a.close()
    b.close()
