"""torch.autograd bindings of the compact derivative (forward and adjoint
both run in libcbs.so; this module only passes pointers)."""
from __future__ import annotations

import torch

from . import abi
from .solver import Plan


class VariableCompactDerivative(torch.autograd.Function):
    """x = A(alpha)^{-1} S f along one axis, A cyclic tridiagonal with row-wise
    alpha_i.  Backward: lambda = A^{-T} g, grad_f = S^T lambda,
    grad_alpha_i = -lambda_i (x_{i-1} + x_{i+1}), all in one kernel."""

    @staticmethod
    def forward(ctx, f, alpha, plan: Plan):
        f = f.contiguous()
        alpha = alpha.contiguous()
        abi.cbs_plan_set_bands(plan.handle, alpha.data_ptr())
        plan.bands = alpha
        x = plan.solve(f)
        ctx.save_for_backward(alpha, x)
        ctx.plan = plan
        return x

    @staticmethod
    def backward(ctx, g):
        alpha, x = ctx.saved_tensors
        plan = ctx.plan
        g = g.contiguous()
        abi.cbs_plan_set_bands(plan.handle, alpha.data_ptr())
        gf = torch.empty_like(g) if ctx.needs_input_grad[0] else None
        ga = torch.empty_like(alpha) if ctx.needs_input_grad[1] else None
        stream = torch.cuda.current_stream(g.device).cuda_stream
        abi.cbs_solve_transpose(plan.handle, g.data_ptr(), x.data_ptr() if ga is not None else None, None,
                                gf.data_ptr() if gf is not None else None,
                                ga.data_ptr() if ga is not None else None, stream)
        return gf, ga, None


class CompactDerivative(torch.autograd.Function):
    """x = A^{-1} S f with a constant (Toeplitz) cyclic A; backward
    grad_f = S^T A^{-T} g computed by one solve launch."""

    @staticmethod
    def forward(ctx, f, plan: Plan):
        x = plan.solve(f.contiguous())
        ctx.plan = plan
        return x

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous()
        gf = torch.empty(ctx.plan.shape, dtype=ctx.plan.in_dtype, device=g.device)
        stream = torch.cuda.current_stream(g.device).cuda_stream
        abi.cbs_solve_transpose(ctx.plan.handle, g.data_ptr(), None, None, gf.data_ptr(), None, stream)
        return gf, None


def variable_plan(shape_zyx, direction: int, alpha: torch.Tensor, rhs, h: float, precision: str = "fp64",
                  segments: int = 0) -> Plan:
    """Plan for a variable-alpha operator bound to `alpha` (rebindable).  The
    plan keeps a reference to `alpha`: the library reads it at every solve."""
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = Plan(shape_zyx, direction, lhs="variable", bands_ptr=alpha.data_ptr(), rhs=rhs, h=h,
                precision=precision, segments=segments, in_dtype=dt, out_dtype=dt)
    plan.bands = alpha
    return plan
