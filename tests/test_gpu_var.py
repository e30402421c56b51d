"""GPU parity of the variable-alpha solve and the adjoint (differentiation
workload: row-wise alpha_i ~ U(0.2, 0.4), 4th-order central right-hand side)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.autograd import CompactDerivative, VariableCompactDerivative, variable_plan
from paper_2101_02286_gb300.solver import Plan

pytestmark = pytest.mark.gpu
C4 = W.CENTRAL4["rhs"]


def _fields(n, seed, shape=None):
    rng = np.random.default_rng(seed)
    shape = shape or (n, n, n)
    return rng.uniform(-1, 1, size=shape), rng.uniform(0.2, 0.4, size=shape)


@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_variable_forward(cuda, direction, precision, tol):
    f, al = _fields(0, 4 + direction, shape=(24, 40, 64))
    n = f.shape[2 - direction]
    dt = torch.float64 if precision == "fp64" else torch.float32
    fa = torch.from_numpy(f).to("cuda", dt)
    aa = torch.from_numpy(al).to("cuda", dt)
    plan = variable_plan(f.shape, direction, aa, C4, W.grid_spacing(n), precision)
    x = plan.solve(fa).double().cpu().numpy()
    ref = oracle.derivative_variable_tri(f if dt == torch.float64 else fa.double().cpu().numpy(),
                                         al if dt == torch.float64 else aa.double().cpu().numpy(),
                                         C4, W.grid_spacing(n), axis=2 - direction)
    assert oracle.rel_err(x, ref) < tol
    plan.close()


@pytest.mark.parametrize("n,p", [(12, 1), (24, 2), (40, 3), (64, 5), (64, 8), (97, 11), (128, 16), (250, 32)])
def test_variable_segments(cuda, n, p):
    f, al = _fields(0, 40 + p, shape=(2, 3, n))
    plan = variable_plan(f.shape, 0, torch.from_numpy(al).cuda(), C4, W.grid_spacing(n), "fp64", segments=p)
    assert plan.info()["segments"] == p
    x = plan.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    ref = oracle.derivative_variable_tri(f, al, C4, W.grid_spacing(n), axis=2)
    assert oracle.rel_err(x, ref) < 1e-12
    plan.close()


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_variable_adjoint_vs_oracle(cuda, direction):
    f, al = _fields(0, 9, shape=(16, 24, 32))
    g = np.random.default_rng(10).standard_normal(f.shape)
    n = f.shape[2 - direction]
    h = W.grid_spacing(n)
    aa = torch.from_numpy(al).cuda()
    plan = variable_plan(f.shape, direction, aa, C4, h, "fp64")
    fa = torch.from_numpy(f).cuda()
    x = plan.solve(fa)
    ga_, gf_, lam_ = (torch.empty_like(fa) for _ in range(3))
    abi.cbs_solve_transpose(plan.handle, torch.from_numpy(g).cuda().data_ptr(), x.data_ptr(), lam_.data_ptr(),
                            gf_.data_ptr(), ga_.data_ptr(), 0)
    gf, ga, lam, xr = oracle.adjoint_variable_tri(f, al, g, C4, h, axis=2 - direction)
    torch.cuda.synchronize()
    assert oracle.rel_err(x.cpu().numpy(), xr) < 1e-12
    assert oracle.rel_err(lam_.cpu().numpy(), lam) < 1e-12
    assert oracle.rel_err(gf_.cpu().numpy(), gf) < 1e-12
    assert oracle.rel_err(ga_.cpu().numpy(), ga) < 1e-12
    # standalone band gradient agrees with the fused one
    gb = torch.empty_like(fa)
    abi.cbs_band_grad(plan.handle, lam_.data_ptr(), x.data_ptr(), gb.data_ptr(), 0)
    torch.cuda.synchronize()
    assert oracle.rel_err(gb.cpu().numpy(), ga) < 1e-14
    plan.close()


def test_autograd_dense_inverse_n16(cuda):
    n = 16
    f, al = _fields(0, 12, shape=(1, 1, n))
    g = np.random.default_rng(13).standard_normal((1, 1, n))
    fa = torch.from_numpy(f).cuda().requires_grad_()
    aa = torch.from_numpy(al).cuda().requires_grad_()
    plan = variable_plan(f.shape, 0, aa, C4, W.grid_spacing(n), "fp64", segments=2)
    x = VariableCompactDerivative.apply(fa, aa, plan)
    (x * torch.from_numpy(g).cuda()).sum().backward()
    A = oracle.dense_matrix(oracle.variable_alpha_bands(al.reshape(1, n))[0])
    S = np.stack([oracle.central_rhs(np.eye(n)[j], C4, W.grid_spacing(n)) for j in range(n)], axis=1)
    Ai = np.linalg.inv(A)
    xr = Ai @ S @ f.ravel()
    lam = Ai.T @ g.ravel()
    assert oracle.rel_err(fa.grad.cpu().numpy().ravel(), S.T @ lam) < 1e-12
    ga = -lam * (np.roll(xr, 1) + np.roll(xr, -1))
    assert oracle.rel_err(aa.grad.cpu().numpy().ravel(), ga) < 1e-12
    plan.close()


def test_autograd_gradcheck(cuda):
    # central finite differences in FP64 (torch.autograd.gradcheck, eps 1e-6)
    f, al = _fields(0, 14, shape=(2, 3, 16))
    fa = torch.from_numpy(f).cuda().requires_grad_()
    aa = torch.from_numpy(al).cuda().requires_grad_()
    plan = variable_plan(f.shape, 0, aa, C4, W.grid_spacing(16), "fp64")
    assert torch.autograd.gradcheck(lambda a, b: VariableCompactDerivative.apply(a, b, plan), (fa, aa),
                                    eps=1e-6, atol=1e-7, rtol=1e-6)
    plan.close()


def test_toeplitz_adjoint(cuda):
    rng = np.random.default_rng(15)
    f = rng.uniform(-1, 1, size=(4, 8, 64))
    g = rng.standard_normal(f.shape)
    h = W.grid_spacing(64)
    for scheme in (W.LELE6_TRI, W.PENTA10):
        plan = Plan(f.shape, 0, lhs=scheme["lhs"], rhs=scheme["rhs"], h=h)
        fa = torch.from_numpy(f).cuda().requires_grad_()
        x = CompactDerivative.apply(fa, plan)
        (x * torch.from_numpy(g).cuda()).sum().backward()
        lam = oracle.solve_cyclic(oracle.transpose_bands(oracle.toeplitz_bands(64, scheme["lhs"])), g)
        ref = oracle.central_rhs_transpose(lam, scheme["rhs"], h)
        assert oracle.rel_err(fa.grad.cpu().numpy(), ref) < 1e-12
        plan.close()


@pytest.mark.slow
def test_variable_full_size_sampled(cuda):
    # 256^3 forward + backward in the launch configuration of the benchmark,
    # checked on sampled lines
    f, al = W.variable_alpha_cube(256)
    g = np.random.default_rng(99).standard_normal(f.shape)
    h = W.grid_spacing(256)
    fa, aa, gg = (torch.from_numpy(v).cuda() for v in (f, al, g))
    plan = variable_plan(f.shape, 0, aa, C4, h, "fp64")
    x = plan.solve(fa)
    gf_, ga_ = torch.empty_like(fa), torch.empty_like(fa)
    abi.cbs_solve_transpose(plan.handle, gg.data_ptr(), x.data_ptr(), None, gf_.data_ptr(), ga_.data_ptr(), 0)
    torch.cuda.synchronize()
    idx = np.random.default_rng(1).integers(0, 256, size=(32, 2))
    fl, al_, gl = (v[idx[:, 0], idx[:, 1]] for v in (f, al, g))
    gf, ga, lam, xr = oracle.adjoint_variable_tri(fl, al_, gl, C4, h)
    xc, gfc, gac = (v.cpu().numpy()[idx[:, 0], idx[:, 1]] for v in (x, gf_, ga_))
    assert oracle.rel_err(xc, xr) < 1e-12
    assert oracle.rel_err(gfc, gf) < 1e-12
    assert oracle.rel_err(gac, ga) < 1e-12
    plan.close()
