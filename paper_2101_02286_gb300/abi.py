"""ctypes binding of the C-ABI in include/cbs.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Pointers are
plain integers (device addresses from torch tensors, or host addresses);
every non-zero status raises CbsError with the library's message.  There is
no fallback: if libcbs.so is missing or fails to load, importing this module
raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcbs.so")

# status codes (cbs.h)
CBS_OK, CBS_ERR_INVALID_ARG, CBS_ERR_UNSUPPORTED, CBS_ERR_SINGULAR, CBS_ERR_TIMEOUT, CBS_ERR_CUDA, \
    CBS_ERR_NO_MEMORY, CBS_ERR_RANGE = range(8)
CBS_FP64, CBS_FP32, CBS_FP32_REFINE, CBS_FP32_REFINE_I64 = 0, 1, 2, 3
CBS_DTYPE_F64, CBS_DTYPE_F32 = 0, 1
CBS_LHS_TOEPLITZ, CBS_LHS_VARIABLE, CBS_LHS_BLOCK = 0, 1, 2
CBS_RHS_NONE, CBS_RHS_CENTRAL, CBS_RHS_STAGGERED, CBS_RHS_MIDPOINT = 0, 1, 2, 3
CBS_BATCH_AUTO, CBS_BATCH_PERSISTENT, CBS_BATCH_PER_PROBLEM = 0, 1, 2

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "SINGULAR", 4: "TIMEOUT", 5: "CUDA",
                6: "NO_MEMORY", 7: "RANGE"}

# every entry point declared in include/cbs.h
EXPORTS = ("cbs_plan_create", "cbs_plan_destroy", "cbs_solve", "cbs_solve_transpose", "cbs_band_grad",
           "cbs_status_poll", "cbs_plan_info_get", "cbs_schedule", "cbs_batch_create", "cbs_batch_destroy",
           "cbs_batch_solve", "cbs_batch_status_poll", "cbs_batch_set_mode", "cbs_last_launch_count", "cbs_last_error_string",
           "cbs_version", "cbs_interface_model", "cbs_plan_set_bands", "cbs_solve_noalloc", "cbs_autotune",
           "cbs_plan_set_variant", "cbs_plan_inject_fault", "cbs_probe_fp64_peak", "cbs_pipe_create",
           "cbs_pipe_solve", "cbs_pipe_destroy")


class CbsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class cbs_desc(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int64 * 3),
        ("direction", ctypes.c_int32),
        ("bandwidth", ctypes.c_int32),
        ("cyclic", ctypes.c_int32),
        ("lhs_kind", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("bands", ctypes.c_void_p),
        ("rhs_kind", ctypes.c_int32),
        ("rhs_terms", ctypes.c_int32),
        ("rhs_coef", ctypes.c_double * 3),
        ("h", ctypes.c_double),
        ("segments", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("refine_sweeps", ctypes.c_int32),
        ("in_dtype", ctypes.c_int32),
        ("out_dtype", ctypes.c_int32),
        ("rhs_shift", ctypes.c_int32),
        ("closure_rows", ctypes.c_int32),
        ("closure_width", ctypes.c_int32),
        ("closure", ctypes.c_void_p),
        ("block_size", ctypes.c_int32),
        ("blocks", ctypes.c_void_p),
    ]


class cbs_plan_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("bandwidth", ctypes.c_int32), ("segments", ctypes.c_int32),
        ("rows_big", ctypes.c_int32), ("rows_small", ctypes.c_int32), ("count_big", ctypes.c_int32),
        ("pcr_steps", ctypes.c_int32), ("detach_steps", ctypes.c_int32), ("detached_rows", ctypes.c_int32),
        ("stage_count", ctypes.c_int32), ("kernel", ctypes.c_int32), ("threads_per_line", ctypes.c_int32),
        ("lines", ctypes.c_int64),
        ("message_stages", ctypes.c_int32), ("message_stages_f32", ctypes.c_int32),
        ("inner_message_stages", ctypes.c_int32), ("inner_message_stages_f32", ctypes.c_int32),
        ("variant", ctypes.c_int32), ("tma", ctypes.c_int32), ("tile_lines", ctypes.c_int32),
        ("segment_warp", ctypes.c_int32),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libcbs.so is not built (run __graft_entry__.build() or "
                          "python paper_2101_02286_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "cbs_plan_create": ([P(vp), P(cbs_desc)], st),
        "cbs_plan_destroy": ([vp], st),
        "cbs_solve": ([vp, vp, vp, vp], st),
        "cbs_solve_transpose": ([vp, vp, vp, vp, vp, vp, vp], st),
        "cbs_band_grad": ([vp, vp, vp, vp, vp], st),
        "cbs_status_poll": ([vp, P(i32)], st),
        "cbs_plan_info_get": ([vp, P(cbs_plan_info)], st),
        "cbs_schedule": ([i32, i32, P(i32), i32, P(i32)], st),
        "cbs_batch_create": ([P(vp), P(cbs_desc), i32], st),
        "cbs_batch_destroy": ([vp], st),
        "cbs_batch_solve": ([vp, P(vp), P(vp), vp], st),
        "cbs_batch_status_poll": ([vp, P(i32)], st),
        "cbs_batch_set_mode": ([vp, i32], st),
        "cbs_last_launch_count": ([], i32),
        "cbs_last_error_string": ([], ctypes.c_char_p),
        "cbs_version": ([], i32),
        "cbs_interface_model": ([P(cbs_desc), i32, vp, vp, vp, vp, vp], st),
        "cbs_plan_set_bands": ([vp, vp], st),
        "cbs_solve_noalloc": ([vp, vp, vp, vp], st),
        "cbs_autotune": ([P(cbs_desc), i32, P(i32), P(ctypes.c_double)], st),
        "cbs_plan_set_variant": ([vp, i32, i32], st),
        "cbs_plan_inject_fault": ([vp, i32], st),
        "cbs_probe_fp64_peak": ([P(ctypes.c_double)], st),
        "cbs_pipe_create": ([P(vp), P(vp), i32], st),
        "cbs_pipe_solve": ([vp, vp, P(vp), vp], st),
        "cbs_pipe_destroy": ([vp], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def _check(status: int):
    if status != CBS_OK:
        raise CbsError(status, _lib.cbs_last_error_string().decode())


def cbs_plan_create(desc: cbs_desc) -> int:
    h = ctypes.c_void_p()
    _check(_lib.cbs_plan_create(ctypes.byref(h), ctypes.byref(desc)))
    return h.value


def cbs_autotune(desc: cbs_desc, reps: int = 5) -> tuple[int, float]:
    """Time every admissible partition count; returns (segments, ms per solve)
    and caches the choice for plans created with segments == 0."""
    p = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(_lib.cbs_autotune(ctypes.byref(desc), reps, ctypes.byref(p), ctypes.byref(ms)))
    return p.value, ms.value


def cbs_plan_destroy(plan: int) -> None:
    _check(_lib.cbs_plan_destroy(plan))


def cbs_plan_set_bands(plan: int, bands: int) -> None:
    _check(_lib.cbs_plan_set_bands(plan, bands))


def cbs_plan_set_variant(plan: int, variant: int, tile_lines: int = 0) -> None:
    """variant 0 = automatic (TMA-fed refinement kernel where it qualifies),
    1 = the pipelined / staged line kernels; tile_lines: lines per tile of
    the TMA kernel on y/z lines (4, 8 or 16; 0 = the default, 8)."""
    _check(_lib.cbs_plan_set_variant(plan, variant, tile_lines))


def cbs_plan_inject_fault(plan: int, kind: int) -> None:
    """Test of the device timeout path (1: a tile wait of the TMA kernel
    expires after 1 ms; 0: none)."""
    _check(_lib.cbs_plan_inject_fault(plan, kind))


def cbs_solve(plan: int, inp: int, out: int, stream: int = 0) -> None:
    _check(_lib.cbs_solve(plan, inp, out, stream))


def cbs_solve_noalloc(plan: int, inp: int, out: int, stream: int = 0) -> None:
    """Long-line solve on the library's fixed scratch (no device allocation)."""
    _check(_lib.cbs_solve_noalloc(plan, inp, out, stream))


def cbs_solve_transpose(plan: int, g: int, x: int | None, lam: int | None, grad_in: int | None,
                        grad_bands: int | None, stream: int = 0) -> None:
    _check(_lib.cbs_solve_transpose(plan, g, x, lam, grad_in, grad_bands, stream))


def cbs_band_grad(plan: int, lam: int, x: int, grad_bands: int, stream: int = 0) -> None:
    _check(_lib.cbs_band_grad(plan, lam, x, grad_bands, stream))


def cbs_status_poll(plan: int) -> int:
    v = ctypes.c_int32()
    _check(_lib.cbs_status_poll(plan, ctypes.byref(v)))
    return v.value


def cbs_plan_info_get(plan: int) -> dict:
    info = cbs_plan_info()
    _check(_lib.cbs_plan_info_get(plan, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in cbs_plan_info._fields_}


def cbs_schedule(p: int, cyclic: bool = True) -> list[tuple[int, int, int]]:
    count = ctypes.c_int32()
    _check(_lib.cbs_schedule(p, int(cyclic), None, 0, ctypes.byref(count)))
    buf = (ctypes.c_int32 * (3 * max(count.value, 1)))()
    _check(_lib.cbs_schedule(p, int(cyclic), buf, count.value, ctypes.byref(count)))
    return [(buf[3 * k], buf[3 * k + 1], buf[3 * k + 2]) for k in range(count.value)]


def cbs_interface_model(desc: cbs_desc, p: int, bhat=None):
    """Host-only: (Dhat, Lhat, Uhat) blocks of Eq. 18-20 as numpy (p, r, r)
    arrays, and x~ = A-hat^{-1} b-hat via the plan's stage coefficients when
    bhat (p*r values) is given."""
    import numpy as np
    r = (desc.bandwidth - 1) // 2
    D = np.zeros((p, r, r))
    L = np.zeros((p, r, r))
    U = np.zeros((p, r, r))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    xt = None
    if bhat is not None:
        b = np.ascontiguousarray(bhat, dtype=np.float64).reshape(p * r)
        xt = np.zeros(p * r)
        _check(_lib.cbs_interface_model(ctypes.byref(desc), p, ptr(D), ptr(L), ptr(U), ptr(b), ptr(xt)))
    else:
        _check(_lib.cbs_interface_model(ctypes.byref(desc), p, ptr(D), ptr(L), ptr(U), None, None))
    return D, L, U, xt


def cbs_batch_create(descs: list[cbs_desc]) -> int:
    arr = (cbs_desc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _check(_lib.cbs_batch_create(ctypes.byref(h), arr, len(descs)))
    return h.value


def cbs_pipe_create(plans: list[int]) -> int:
    arr = (ctypes.c_void_p * len(plans))(*plans)
    h = ctypes.c_void_p()
    _check(_lib.cbs_pipe_create(ctypes.byref(h), arr, len(plans)))
    return h.value


def cbs_pipe_solve(pipe: int, host_in: int, host_outs: list[int], stream: int = 0) -> None:
    outs = (ctypes.c_void_p * len(host_outs))(*host_outs)
    _check(_lib.cbs_pipe_solve(pipe, host_in, outs, stream))


def cbs_pipe_destroy(pipe: int) -> None:
    _check(_lib.cbs_pipe_destroy(pipe))


def cbs_batch_destroy(batch: int) -> None:
    _check(_lib.cbs_batch_destroy(batch))


def cbs_batch_solve(batch: int, ins: list[int], outs: list[int], stream: int = 0) -> None:
    n = len(ins)
    a = (ctypes.c_void_p * n)(*ins)
    b = (ctypes.c_void_p * n)(*outs)
    _check(_lib.cbs_batch_solve(batch, a, b, stream))


def cbs_batch_set_mode(batch: int, mode: int) -> None:
    _check(_lib.cbs_batch_set_mode(batch, mode))


def cbs_batch_status_poll(batch: int) -> int:
    v = ctypes.c_int32()
    _check(_lib.cbs_batch_status_poll(batch, ctypes.byref(v)))
    return v.value


def cbs_probe_fp64_peak() -> float:
    """Measured FP64 fma throughput of the current device (TFLOP/s)."""
    v = ctypes.c_double()
    _check(_lib.cbs_probe_fp64_peak(ctypes.byref(v)))
    return v.value


def cbs_last_launch_count() -> int:
    return int(_lib.cbs_last_launch_count())


def cbs_version() -> int:
    return int(_lib.cbs_version())
