"""GPU parity of heptadiagonal (w = 7, r = 3) systems against the FP64 oracle.

The generalised bands of Sec. 2 (Eq. 3-6): the k-system of a w-wide band has
(w - 1) / 2 = 3 interface rows per partition, so the reduced system's blocks
are 3 x 3.  The operator is the 12th-order scheme HEPTA12 (bands 9/16, 9/100,
1/400; a weakly dominant matrix whose symbol falls to 0.05 at kh = pi).  Every
case compares the whole output element by element with the oracle's banded
LU + Woodbury solve (norm-wise infinity relative error): FP64 and FP32 +
refinement <= 1e-12, unrefined FP32 <= 2e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Plan

pytestmark = pytest.mark.gpu

H7 = W.HEPTA12
TOL = {"fp64": 1e-12, "fp32_refine": 1e-12, "fp32_refine_i64": 1e-12, "fp32": 2e-5}


def run(f, direction, precision="fp64", segments=0, rhs=True, cyclic=True, in_dtype=torch.float64):
    n = f.shape[2 - direction]
    sweeps = 2 if precision.startswith("fp32_refine") else 1
    plan = Plan(f.shape, direction, lhs=H7["lhs"], rhs=H7["rhs"] if rhs else None, h=W.grid_spacing(n),
                segments=segments, precision=precision, sweeps=sweeps, in_dtype=in_dtype, cyclic=cyclic)
    y = plan.solve(torch.from_numpy(np.ascontiguousarray(f)).to("cuda", in_dtype))
    torch.cuda.synchronize()
    info = plan.info()
    assert plan.status() == 0
    plan.close()
    return y.double().cpu().numpy(), info


def reference(f, direction, rhs=True, cyclic=True):
    n = f.shape[2 - direction]
    ax = 2 - direction
    if rhs:
        return oracle.derivative(f, H7["lhs"], H7["rhs"], W.grid_spacing(n), axis=ax)
    bands = oracle.toeplitz_bands(n, H7["lhs"])
    return oracle.solve_cyclic(bands, f, axis=ax) if cyclic else oracle.solve_acyclic(bands, f, axis=ax)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refine", "fp32_refine_i64"])
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_directions_precisions(cuda, direction, precision):
    rng = np.random.default_rng(300 + direction)
    shape = [9, 11, 13]
    shape[2 - direction] = 192  # 12 partitions of 16 rows
    f = rng.uniform(-1, 1, size=tuple(shape))
    got, info = run(f, direction, precision)
    assert info["bandwidth"] == 7
    assert oracle.rel_err(got, reference(f, direction)) < TOL[precision]


@pytest.mark.parametrize("n,p,precision", [(48, 2, "fp64"), (64, 4, "fp64"), (97, 7, "fp64"), (192, 32, "fp64"),
                                           (250, 31, "fp64"), (512, 16, "fp64"), (512, 32, "fp64"),
                                           (512, 32, "fp32_refine"), (250, 31, "fp32_refine"),
                                           (192, 32, "fp32_refine_i64"), (384, 24, "fp32")])
def test_segment_counts_and_ragged(cuda, n, p, precision):
    # n = 192, p = 32: the minimum of 2r = 6 rows per partition; 250 / 31 and
    # 97 / 7: ragged partitions; 512 / 16: 32 rows per lane (FP64)
    f = np.random.default_rng(n * 3 + p).uniform(-1, 1, size=(3, 5, n))
    got, info = run(f, 0, precision, segments=p)
    assert info["segments"] == p
    assert oracle.rel_err(got, reference(f, 0)) < TOL[precision]


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_rhs_given_fp32_input(cuda, direction, precision):
    shape = [4, 6, 6]
    shape[2 - direction] = 256
    d = np.random.default_rng(17 + direction).standard_normal(tuple(shape)).astype(np.float32).astype(np.float64)
    got, _ = run(d, direction, precision, rhs=False, in_dtype=torch.float32)
    assert oracle.rel_err(got, reference(d, direction, rhs=False)) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine", "fp32"])
@pytest.mark.parametrize("direction,n,p", [(0, 64, 4), (0, 97, 7), (1, 192, 32), (2, 128, 8)])
def test_acyclic(cuda, precision, direction, n, p):
    shape = [5, 6, 7]
    shape[2 - direction] = n
    d = np.random.default_rng(n + p + direction).standard_normal(tuple(shape))
    got, info = run(d, direction, precision, segments=p, rhs=False, cyclic=False)
    assert info["segments"] == p and info["detach_steps"] == 0
    assert oracle.rel_err(got, reference(d, direction, rhs=False, cyclic=False)) < TOL[precision]


def test_closed_form_mode(cuda):
    # a single Fourier mode: k'h = (a sin kh + (b/2) sin 2kh + (c/3) sin 3kh)
    # / (1 + 2 alpha cos kh + 2 beta cos 2kh + 2 gamma cos 3kh)   (Eq. 3-6)
    n, k = 512, 101
    h = W.grid_spacing(n)
    xg = np.arange(n) * h
    f = np.broadcast_to(np.sin(k * xg), (2, 3, n)).copy()
    got, _ = run(f, 0, "fp32_refine")
    th = k * h
    (al, be, ga), (a, b, c) = H7["lhs"], H7["rhs"]
    kp = (a * np.sin(th) + b / 2 * np.sin(2 * th) + c / 3 * np.sin(3 * th)) / \
        (1 + 2 * al * np.cos(th) + 2 * be * np.cos(2 * th) + 2 * ga * np.cos(3 * th)) / h
    assert oracle.rel_err(got, np.broadcast_to(kp * np.cos(k * xg), f.shape)) < 1e-12


def test_transpose(cuda):
    # grad_in = S^T A^{-T} g for the w = 7 operator (A symmetric circulant)
    rng = np.random.default_rng(23)
    n = 256
    g = rng.uniform(-1, 1, size=(2, 5, n))
    h = W.grid_spacing(n)
    plan = Plan(g.shape, 0, lhs=H7["lhs"], rhs=H7["rhs"], h=h, precision="fp64")
    gt = torch.from_numpy(g).cuda()
    lam = torch.empty_like(gt)
    gin = torch.empty_like(gt)
    abi.cbs_solve_transpose(plan.handle, gt.data_ptr(), None, lam.data_ptr(), gin.data_ptr(), None, 0)
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
    lam_ref = oracle.solve_cyclic(oracle.toeplitz_bands(n, H7["lhs"]), g, axis=-1)
    assert oracle.rel_err(lam.cpu().numpy(), lam_ref) < 1e-12
    assert oracle.rel_err(gin.cpu().numpy(), oracle.central_rhs_transpose(lam_ref, H7["rhs"], h, axis=-1)) < 1e-12


def test_unsupported_paths_rejected(cuda):
    # long lines, staggered stencils and batches stay tri- and pentadiagonal
    with pytest.raises(abi.CbsError):
        Plan((1, 2, 1 << 14), 0, lhs=H7["lhs"], segments=64)
    with pytest.raises(abi.CbsError):
        Plan((1, 2, 64), 0, lhs=H7["lhs"], rhs=(1.0, 0.1), h=0.1, stencil="staggered")
