"""GPU parity of acyclic derivatives with one-sided boundary closures.

The plan solves the acyclic Toeplitz system with the line kernels and then
corrects the rows near both ends (the Woodbury form of the closure rows, FP64);
the oracle writes out the dense closure matrices row by row and solves them
with LAPACK.  Every case compares the whole output (norm-wise infinity
relative error): FP64 and FP32 + refinement <= 1e-12, FP32 <= 2e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Plan

pytestmark = pytest.mark.gpu

SCHEMES = {"tri6": (W.LELE6_TRI, W.CLOSURE3_4), "penta10": (W.PENTA10, W.CLOSURE3_4_6)}
TOL = {"fp64": 1e-12, "fp32_refine": 1e-12, "fp32_refine_i64": 1e-12, "fp32": 2e-5}


def spacing(n):
    return 1.0 / (n - 1)  # nodes 0, h, .., 1 (both ends on the grid)


def run(f, direction, scheme, precision="fp64", segments=0):
    sch, cl = SCHEMES[scheme]
    n = f.shape[2 - direction]
    dt = torch.float32 if precision == "fp32" else torch.float64
    sweeps = 2 if (scheme == "penta10" and precision.startswith("fp32_refine")) else 1
    plan = Plan(f.shape, direction, lhs=sch["lhs"], rhs=sch["rhs"], h=spacing(n), segments=segments,
                precision=precision, sweeps=sweeps, in_dtype=dt, cyclic=False, closure=cl)
    y = plan.solve(torch.from_numpy(np.ascontiguousarray(f)).to("cuda", dt))
    torch.cuda.synchronize()
    launches = abi.cbs_last_launch_count()
    info = plan.info()
    assert plan.status() == 0
    plan.close()
    return y.double().cpu().numpy(), info, launches


def reference(f, direction, scheme, f32=False):
    sch, cl = SCHEMES[scheme]
    n = f.shape[2 - direction]
    if f32:
        f = f.astype(np.float32).astype(np.float64)
    return oracle.derivative_closure(f, sch["lhs"], sch["rhs"], cl, spacing(n), axis=2 - direction)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine", "fp32_refine_i64", "fp32"])
@pytest.mark.parametrize("scheme", ["tri6", "penta10"])
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_directions_schemes_precisions(cuda, direction, scheme, precision):
    rng = np.random.default_rng(500 + direction)
    shape = [7, 9, 11]
    shape[2 - direction] = 256
    f = rng.uniform(-1, 1, size=tuple(shape))
    got, info, launches = run(f, direction, scheme, precision)
    assert launches == 2  # line kernel + closure correction
    assert oracle.rel_err(got, reference(f, direction, scheme, precision == "fp32")) < TOL[precision]


@pytest.mark.parametrize("scheme", ["tri6", "penta10"])
@pytest.mark.parametrize("n,p,precision", [(64, 4, "fp64"), (97, 7, "fp64"), (250, 31, "fp64"), (512, 32, "fp64"),
                                           (128, 11, "fp32_refine"), (512, 32, "fp32_refine"), (40, 2, "fp64"),
                                           (1024, 32, "fp64")])
def test_segment_counts_and_ragged(cuda, scheme, n, p, precision):
    f = np.random.default_rng(n + 3 * p).uniform(-1, 1, size=(2, 5, n))
    got, info, _ = run(f, 0, scheme, precision, segments=p)
    assert info["segments"] == p
    assert oracle.rel_err(got, reference(f, 0, scheme)) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("direction", [0, 2])
def test_cubic_reproduced(cuda, direction, precision):
    # every closure row is at least third order: a cubic's derivative comes
    # back exactly (to rounding), ends included.  For smooth data the stencil
    # terms w_q f (size |f| / h) cancel to |f'|: the refinement's residual is
    # exact to about 2^-46 of the terms, so its bound is that times the
    # cancellation ratio (sum_q 2 |w_q| max|f| / max|f'|, about 1000 here)
    n = 128
    xg = np.arange(n) * spacing(n)
    c = (0.7, -1.1, 0.4, 2.0)
    line = np.polyval(c, xg)
    shape = [3, 4, 5]
    shape[2 - direction] = n
    f = np.moveaxis(np.broadcast_to(line, tuple(np.moveaxis(np.empty(shape), 2 - direction, -1).shape)),
                    -1, 2 - direction).copy()
    got, _, _ = run(f, direction, "tri6", precision)
    fp = np.polyval(np.polyder(c), xg)
    want = np.moveaxis(np.broadcast_to(fp, np.moveaxis(f, 2 - direction, -1).shape), -1, 2 - direction)
    ratio = sum(2 * abs(cq) / (2 * q * spacing(n)) for q, cq in enumerate(W.LELE6_TRI["rhs"], start=1)) \
        * np.max(np.abs(line)) / np.max(np.abs(fp))
    tol = 1e-12 if precision == "fp64" else max(1e-12, 2.0 ** -46 * ratio * 8)
    assert oracle.rel_err(got, want) < tol


def test_smooth_function_converges(cuda):
    # the error against the exact derivative falls like h^3 on the GPU as well
    errs = []
    for n in (64, 128, 256):
        xg = np.arange(n) * spacing(n)
        f = np.broadcast_to(np.sin(3 * xg) + np.exp(xg), (1, 2, n)).copy()
        got, _, _ = run(f, 0, "tri6", "fp32_refine")
        errs.append(np.max(np.abs(got - (3 * np.cos(3 * xg) + np.exp(xg)))))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.9 < o < 4.0 for o in orders), orders


def test_closure_validation(cuda):
    sch, cl = SCHEMES["penta10"]
    L, R = cl
    with pytest.raises(abi.CbsError):  # two rows cannot hold a three-term stencil
        Plan((1, 2, 64), 0, lhs=sch["lhs"], rhs=sch["rhs"], h=0.1, cyclic=False, closure=(L[:2], R[:2]))
    with pytest.raises(abi.CbsError):  # closures need an acyclic line
        Plan((1, 2, 64), 0, lhs=sch["lhs"], rhs=sch["rhs"], h=0.1, cyclic=True, closure=cl)
    with pytest.raises(abi.CbsError):  # the long-line path has no closures
        Plan((1, 2, 1 << 14), 0, lhs=sch["lhs"], rhs=sch["rhs"], h=0.1, cyclic=False, closure=cl, segments=64)
