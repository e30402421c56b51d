"""Torch-facing wrapper over the C-ABI: builds a cbs_desc and passes pointers.

Tensors are (nz, ny, nx) C-contiguous (x fastest), on the current CUDA
device.  Nothing here computes: every step of a solve runs in libcbs.so.
"""
from __future__ import annotations

import torch

from . import abi

_PREC = {"fp64": abi.CBS_FP64, "fp32": abi.CBS_FP32, "fp32_refine": abi.CBS_FP32_REFINE,
         "fp32_refine_i64": abi.CBS_FP32_REFINE_I64}  # refinement, FP64 interface system
_DT = {torch.float64: abi.CBS_DTYPE_F64, torch.float32: abi.CBS_DTYPE_F32}


_STENCIL = {"central": abi.CBS_RHS_CENTRAL, "staggered": abi.CBS_RHS_STAGGERED, "midpoint": abi.CBS_RHS_MIDPOINT}


def make_desc(shape_zyx, direction: int, lhs=(1.0 / 3.0,), rhs=None, h: float = 1.0, segments: int = 0,
              precision: str = "fp64", sweeps: int = 1, in_dtype=torch.float64, out_dtype=None,
              cyclic: bool = True, bands_ptr: int | None = None, stencil: str = "central",
              shift: int = 0, closure=None, blocks=None) -> abi.cbs_desc:
    """Descriptor for lines along `direction` of a (nz, ny, nx) field.

    lhs: (alpha,) tridiagonal, (alpha, beta) pentadiagonal or (alpha, beta,
    gamma) heptadiagonal Toeplitz bands (diagonal 1), or "variable" with bands_ptr pointing at a per-point alpha
    field.  rhs: None (input is b) or the coefficients (c_1, .., c_K) of the
    periodic stencil named by `stencil`: "central" (Eq. 1, spacing h),
    "staggered" (staggered first derivative, App. A.2) or "midpoint" (compact
    interpolation, Eq. 2); the two staggered kinds map half points to nodes
    (shift 0) or nodes to half points (shift 1).  closure: (L, R), two
    equal-shape (rows, width) arrays of one-sided boundary rows for an
    acyclic derivative (row k: sum_j L[k][j] x_j = sum_j R[k][j] f_j / h; the
    right end is their mirror image, see cbs.h).  blocks: (L, D, U), three
    2 x 2 arrays: a block-tridiagonal LHS whose lines hold points of two
    unknowns each, point-major (lhs is then ignored; right-hand side given).
    """
    nz, ny, nx = (int(s) for s in shape_zyx)
    d = abi.cbs_desc()
    d.dims[0], d.dims[1], d.dims[2] = nx, ny, nz
    d.direction = int(direction)
    if blocks is not None:
        import numpy as np
        L, D, U = (np.asarray(a, dtype=np.float64) for a in blocks)
        if not (L.shape == D.shape == U.shape == (2, 2)):
            raise ValueError("blocks: three 2 x 2 arrays (L, D, U)")
        buf = np.ascontiguousarray(np.concatenate([L.ravel(), D.ravel(), U.ravel()]))
        d._blocks_buf = buf  # kept alive with the descriptor
        d.bandwidth = 7
        d.lhs_kind = abi.CBS_LHS_BLOCK
        d.block_size = 2
        d.blocks = buf.ctypes.data
    elif lhs == "variable":
        d.bandwidth = 3
        d.lhs_kind = abi.CBS_LHS_VARIABLE
        d.bands = bands_ptr
    else:
        lhs = tuple(lhs)
        d.bandwidth = 2 * len(lhs) + 1
        d.lhs_kind = abi.CBS_LHS_TOEPLITZ
        d.alpha = float(lhs[0])
        d.beta = float(lhs[1]) if len(lhs) > 1 else 0.0
        d.gamma = float(lhs[2]) if len(lhs) > 2 else 0.0
    d.cyclic = int(bool(cyclic))
    if rhs is None:
        d.rhs_kind = abi.CBS_RHS_NONE
        d.rhs_terms = 0
    else:
        d.rhs_kind = _STENCIL[stencil]
        d.rhs_shift = int(shift)
        d.rhs_terms = len(rhs)
        for q, c in enumerate(rhs):
            d.rhs_coef[q] = float(c)
    d.h = float(h)
    d.segments = int(segments)
    d.precision = _PREC[precision]
    d.refine_sweeps = int(sweeps)
    d.in_dtype = _DT[in_dtype]
    if out_dtype is None:
        out_dtype = torch.float64 if precision != "fp32" else in_dtype
    d.out_dtype = _DT[out_dtype]
    if closure is not None:
        import numpy as np
        L, R = (np.asarray(a, dtype=np.float64) for a in closure)
        if L.ndim != 2 or L.shape != R.shape:
            raise ValueError("closure: two equal-shape (rows, width) arrays")
        buf = np.ascontiguousarray(np.concatenate([L, R], axis=1))
        d._closure_buf = buf  # kept alive with the descriptor
        d.closure_rows, d.closure_width = L.shape
        d.closure = buf.ctypes.data
    return d


class Plan:
    """A pre-factorised solver for one (shape, direction, operator, precision)."""

    def __init__(self, shape_zyx, direction: int, **kw):
        """kw as for make_desc; segments="tune" times every admissible
        partition count and kernel variant first (cbs_autotune) and creates
        the plan from the tuner's record (segments = 0)."""
        self.shape = tuple(int(s) for s in shape_zyx)
        self.direction = int(direction)
        self.in_dtype = kw.get("in_dtype", torch.float64)
        prec = kw.get("precision", "fp64")
        self.out_dtype = kw.get("out_dtype") or (torch.float64 if prec != "fp32" else self.in_dtype)
        tune = kw.get("segments") == "tune"
        if tune:
            kw = dict(kw, segments=0)
        self.desc = make_desc(self.shape, direction, **kw)
        if tune:
            _, self.tuned_ms = abi.cbs_autotune(self.desc)
        self.handle = abi.cbs_plan_create(self.desc)

    def info(self) -> dict:
        return abi.cbs_plan_info_get(self.handle)

    def solve(self, inp: torch.Tensor, out: torch.Tensor | None = None,
              stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        if inp.shape != self.shape or inp.dtype != self.in_dtype or not inp.is_contiguous() or not inp.is_cuda:
            raise ValueError("input must be a contiguous CUDA tensor of shape %s and dtype %s"
                             % (self.shape, self.in_dtype))
        if out is None:
            out = torch.empty(self.shape, dtype=self.out_dtype, device=inp.device)
        elif out.shape != self.shape or out.dtype != self.out_dtype or not out.is_contiguous() \
                or out.device != inp.device:
            raise ValueError("out must be a contiguous tensor of shape %s and dtype %s on the input's device"
                             % (self.shape, self.out_dtype))
        s = stream if stream is not None else torch.cuda.current_stream(inp.device)
        abi.cbs_solve(self.handle, inp.data_ptr(), out.data_ptr(), s.cuda_stream)
        return out

    def status(self) -> int:
        return abi.cbs_status_poll(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            abi.cbs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A ragged batch of independent problems solved together.

    specs: list of (shape_zyx, direction, kwargs for make_desc): any problem
    a Plan takes.  mode: "auto", "persistent" (one launch over a work table
    of line tiles: Toeplitz bands of width 3 or 5, precision "fp64" or
    "fp32_refine" with FP64 input and output or "fp32" with FP32 input and
    output, long x-lines whose plan runs a warp per segment) or
    "per_problem" (each problem's own kernels, FP64 problems on a stream of
    their own).
    """

    MODES = {"auto": abi.CBS_BATCH_AUTO, "persistent": abi.CBS_BATCH_PERSISTENT,
             "per_problem": abi.CBS_BATCH_PER_PROBLEM}

    def __init__(self, specs, mode: str = "auto"):
        if mode not in self.MODES:
            raise ValueError("mode must be one of %s" % sorted(self.MODES))
        self.shapes = [tuple(int(v) for v in sh) for sh, _, _ in specs]
        self.dtypes = [kw.get("in_dtype", torch.float64) for _, _, kw in specs]
        self.out_dtypes = [kw.get("out_dtype") or (torch.float64 if kw.get("precision", "fp64") != "fp32"
                                                   else kw.get("in_dtype", torch.float64)) for _, _, kw in specs]
        descs = [make_desc(sh, d, **kw) for sh, d, kw in specs]
        self.handle = abi.cbs_batch_create(descs)
        try:
            abi.cbs_batch_set_mode(self.handle, self.MODES[mode])
        except abi.CbsError:
            self.close()
            raise

    def solve(self, ins, outs=None, stream: torch.cuda.Stream | None = None):
        if outs is None:
            outs = [torch.empty(sh, dtype=dt, device=x.device) for x, sh, dt in zip(ins, self.shapes, self.out_dtypes)]
        for x, y, sh, dt, dto in zip(ins, outs, self.shapes, self.dtypes, self.out_dtypes):
            if x.shape != sh or y.shape != sh or x.dtype != dt or y.dtype != dto or not x.is_contiguous() \
                    or not y.is_contiguous():
                raise ValueError("batch inputs/outputs must be contiguous tensors of the planned shapes and dtypes")
        s = stream if stream is not None else torch.cuda.current_stream(ins[0].device)
        abi.cbs_batch_solve(self.handle, [x.data_ptr() for x in ins], [y.data_ptr() for y in outs], s.cuda_stream)
        return outs

    def close(self):
        if getattr(self, "handle", None):
            abi.cbs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipe:
    """Plans over one field, solved from host memory (cbs_pipe_*): each
    solve() uploads the field, runs every plan and downloads every result
    inside the call; `stream` then covers the downloads.  Host tensors should
    be pinned (torch.empty(..., pin_memory=True))."""

    def __init__(self, plans):
        self.plans = list(plans)
        self.handle = abi.cbs_pipe_create([p.handle for p in self.plans])

    def solve(self, host_in: torch.Tensor, host_outs, stream: torch.cuda.Stream | None = None):
        for p, y in zip(self.plans, host_outs):
            if y.device.type != "cpu" or y.shape != p.shape or y.dtype != p.out_dtype or not y.is_contiguous():
                raise ValueError("host outputs: contiguous CPU tensors of each plan's shape and output type")
        p0 = self.plans[0]
        if host_in.device.type != "cpu" or host_in.shape != p0.shape or host_in.dtype != p0.in_dtype \
                or not host_in.is_contiguous():
            raise ValueError("host input: a contiguous CPU tensor of the plans' shape and input type")
        s = stream if stream is not None else torch.cuda.current_stream()
        abi.cbs_pipe_solve(self.handle, host_in.data_ptr(), [y.data_ptr() for y in host_outs], s.cuda_stream)
        return host_outs

    def close(self):
        if getattr(self, "handle", None):
            abi.cbs_pipe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
