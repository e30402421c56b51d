"""GPU parity of the on-chip line kernel against the FP64 oracle.

Every case feeds the same seeded input to both sides and compares the whole
output element by element (norm-wise infinity relative error):
  FP64 and FP32 + refinement: <= 1e-12;  unrefined FP32: <= 2e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300 import workloads as W
from paper_2101_02286_gb300.solver import Plan

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32_refine": 1e-12, "fp32": 2e-5}
SCHEMES = {"tri6": W.LELE6_TRI, "penta10": W.PENTA10}


def gpu_derivative(f, direction, scheme, precision="fp64", segments=0, sweeps=1, in_dtype=torch.float64,
                   rhs=True, out_dtype=None):
    n = f.shape[2 - direction]
    sch = SCHEMES[scheme]
    plan = Plan(f.shape, direction, lhs=sch["lhs"], rhs=sch["rhs"] if rhs else None, h=W.grid_spacing(n),
                segments=segments, precision=precision, sweeps=sweeps, in_dtype=in_dtype, out_dtype=out_dtype)
    x = torch.from_numpy(np.ascontiguousarray(f)).to("cuda", in_dtype)
    y = plan.solve(x)
    torch.cuda.synchronize()
    info = plan.info()
    assert plan.status() == 0
    plan.close()
    return y.double().cpu().numpy(), info


def oracle_derivative(f, direction, scheme, rhs=True):
    sch = SCHEMES[scheme]
    n = f.shape[2 - direction]
    if rhs:
        return oracle.derivative(f, sch["lhs"], sch["rhs"], W.grid_spacing(n), axis=2 - direction)
    return oracle.solve_cyclic(oracle.toeplitz_bands(n, sch["lhs"]), f, axis=2 - direction)


def test_fourier_cube_config(cuda):
    # 64^3, 8 seeded modes, 6th-order tri along x, 4 partitions per line
    f, modes = W.fourier_cube(64, 8)
    got, info = gpu_derivative(f, 0, "tri6", segments=4)
    assert info["segments"] == 4 and info["lines"] == 64 * 64
    ref = oracle_derivative(f, 0, "tri6")
    assert oracle.rel_err(got, ref) < 1e-12


@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("scheme", ["tri6", "penta10"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine", "fp32"])
def test_directions_schemes_precisions(cuda, direction, scheme, precision):
    rng = np.random.default_rng(11 + direction)
    f = rng.uniform(-1, 1, size=(40, 48, 64))  # (nz, ny, nx): ragged-ish line counts
    sweeps = 2 if (scheme == "penta10" and precision == "fp32_refine") else 1
    got, _ = gpu_derivative(f, direction, scheme, precision=precision, sweeps=sweeps)
    ref = oracle_derivative(f, direction, scheme)
    assert oracle.rel_err(got, ref) < TOL[precision]


@pytest.mark.parametrize("scheme", ["tri6", "penta10"])
@pytest.mark.parametrize("n,p", [(64, 1), (64, 2), (64, 3), (64, 5), (61, 4), (97, 7), (96, 11), (100, 13),
                                 (128, 8), (256, 16), (250, 31), (512, 32), (384, 32), (32, 8), (20, 5)])
def test_segment_counts_and_ragged(cuda, scheme, n, p):
    r = len(SCHEMES[scheme]["lhs"])
    if n < 2 * r * p or (n + p - 1) // p > 32:
        pytest.skip("outside the on-chip kernel's partition sizes")
    rng = np.random.default_rng(n * 7 + p)
    f = rng.uniform(-1, 1, size=(3, 5, n))
    got, info = gpu_derivative(f, 0, scheme, segments=p)
    assert info["segments"] == p
    assert oracle.rel_err(got, oracle_derivative(f, 0, scheme)) < 1e-12


@pytest.mark.parametrize("n,p", [(64, 3), (96, 11), (128, 8), (256, 16)])
def test_refine_segment_counts(cuda, n, p):
    rng = np.random.default_rng(n + p)
    f = rng.uniform(-1, 1, size=(2, 9, n))
    if (n + p - 1) // p > 16:
        pytest.skip("refine kernel holds <= 16 rows per lane")
    got, _ = gpu_derivative(f, 0, "tri6", precision="fp32_refine", segments=p)
    assert oracle.rel_err(got, oracle_derivative(f, 0, "tri6")) < 1e-12


@pytest.mark.parametrize("in_dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_rhs_given(cuda, in_dtype, precision):
    # b given directly (no stencil); FP32 input is promoted exactly
    rng = np.random.default_rng(5)
    d = rng.standard_normal(size=(4, 4, 256))
    if in_dtype == torch.float32:
        d = d.astype(np.float32).astype(np.float64)
    got, _ = gpu_derivative(d, 0, "penta10", precision=precision, rhs=False, in_dtype=in_dtype, sweeps=2)
    ref = oracle_derivative(d, 0, "penta10", rhs=False)
    assert oracle.rel_err(got, ref) < 1e-12


def test_minimal_partitions_and_single_line(cuda):
    # n = 2 r p exactly, one line in the field
    f = np.random.default_rng(0).uniform(-1, 1, size=(1, 1, 16))
    got, _ = gpu_derivative(f, 0, "penta10", segments=4)
    assert oracle.rel_err(got, oracle_derivative(f, 0, "penta10")) < 1e-12
    got, _ = gpu_derivative(f, 0, "tri6", segments=8)
    assert oracle.rel_err(got, oracle_derivative(f, 0, "tri6")) < 1e-12


def test_closed_form_mode_512(cuda):
    # the one known plane wave of the 512^3 workload, evaluated on a 512 x 8 x 8 box
    _, modes = W.noisy_cube(8, with_mode=False)
    n = 512
    x = np.arange(n) * W.grid_spacing(n)
    kx = int(modes.k[0, 0])
    f = np.broadcast_to(modes.amp[0] * np.sin(kx * x), (8, 8, n)).copy()
    got, _ = gpu_derivative(f, 0, "tri6", precision="fp32_refine")
    th = 2 * np.pi * kx / n
    kp = (14 / 9 * np.sin(th) + (1 / 18) * np.sin(2 * th)) / (1 + 2 / 3 * np.cos(th)) / W.grid_spacing(n)
    want = modes.amp[0] * kp * np.cos(kx * x)
    assert oracle.rel_err(got[0, 0], want) < 1e-12


def test_invalid_arguments(cuda):
    with pytest.raises(abi.CbsError) as e:
        Plan((1, 1, 8), 0, lhs=(1 / 3,), segments=5)
    assert e.value.status == abi.CBS_ERR_INVALID_ARG
    plan = Plan((1, 1, 64), 0, lhs=(1 / 3,))
    x = torch.zeros((1, 1, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(abi.CbsError):
        abi.cbs_solve(plan.handle, x.data_ptr(), x.data_ptr(), 0)  # aliasing
    with pytest.raises(abi.CbsError):
        abi.cbs_solve(plan.handle, 0, x.data_ptr(), 0)
    plan.close()


def test_autotune_picks_admissible_and_caches(cuda):
    from paper_2101_02286_gb300.solver import make_desc
    shape = (4, 16, 384)
    d = make_desc(shape, 0, lhs=W.LELE6_TRI["lhs"], rhs=W.LELE6_TRI["rhs"], h=W.grid_spacing(384))
    p, ms = abi.cbs_autotune(d, 3)
    assert 1 <= p <= 32 and ms > 0
    # a plan with segments = 0 now uses the cached choice
    plan = Plan(shape, 0, lhs=W.LELE6_TRI["lhs"], rhs=W.LELE6_TRI["rhs"], h=W.grid_spacing(384))
    assert plan.info()["segments"] == p
    f = np.random.default_rng(1).uniform(-1, 1, size=shape)
    y = plan.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    assert oracle.rel_err(y, oracle_derivative(f, 0, "tri6")) < 1e-12
    plan.close()
    tuned = Plan(shape, 0, lhs=W.LELE6_TRI["lhs"], rhs=W.LELE6_TRI["rhs"], h=W.grid_spacing(384), segments="tune")
    assert tuned.info()["segments"] >= 1
    tuned.close()


def test_interface_stages_below_rounding_skip_messages(cuda):
    # 32 partitions of 16 rows: the interface couplings are ~1e-7 of the
    # diagonal blocks and square at every PCR step, so only the first steps
    # exchange values; the rest reduce to local products
    plan = Plan((1, 1, 512), 0, lhs=W.LELE6_TRI["lhs"], segments=32)
    info = plan.info()
    assert info["pcr_steps"] == 5
    assert 1 <= info["message_stages_f32"] <= info["message_stages"] < info["pcr_steps"]
    plan.close()
    # 4096-row segments of a long line decouple completely at the outer level
    long_plan = Plan((1, 2, 1 << 16), 0, lhs=W.PENTA10["lhs"], segments=16)
    li = long_plan.info()
    assert li["kernel"] == 1 and li["message_stages"] == 0 and li["inner_message_stages"] >= 1
    long_plan.close()


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_refine_zeros_and_tiny_values(cuda, direction):
    # whole-size partitions (n = 32 x 16): exact zeros and values far below
    # the FP32 range take the general FP64 -> FP32-pair split
    rng = np.random.default_rng(21 + direction)
    shape = [6, 10, 16]
    shape[2 - direction] = 512
    f = rng.uniform(-1, 1, size=tuple(shape))
    mask = rng.random(f.shape)
    f[mask < 0.1] = 0.0
    f[(mask >= 0.1) & (mask < 0.12)] *= 1e-35
    got, info = gpu_derivative(f, direction, "tri6", precision="fp32_refine", segments=32)
    assert info["rows_big"] == 16
    assert oracle.rel_err(got, oracle_derivative(f, direction, "tri6")) < 1e-12


@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("scheme", ["tri6", "penta10"])
def test_refine_fp64_interface_mode(cuda, direction, scheme):
    # refinement whose correction solves keep the interface system in FP64
    rng = np.random.default_rng(51 + direction)
    shape = [10, 12, 14]
    shape[2 - direction] = 256
    f = rng.uniform(-1, 1, size=tuple(shape))
    sweeps = 2 if scheme == "penta10" else 1
    got, _ = gpu_derivative(f, direction, scheme, precision="fp32_refine_i64", sweeps=sweeps)
    assert oracle.rel_err(got, oracle_derivative(f, direction, scheme)) < 1e-12


def test_pipelined_plans_of_different_widths_in_sequence(cuda):
    # strided y-line plans with 4 and then 32 lanes per line: the second needs
    # more shared memory than the first configured for the same kernel
    for n, p in ((48, 3), (512, 32), (48, 3)):
        f = np.random.default_rng(n).uniform(-1, 1, size=(3, n, 24))
        got, info = gpu_derivative(f, 1, "tri6", precision="fp32_refine", segments=p)
        assert info["rows_big"] == 16
        assert oracle.rel_err(got, oracle_derivative(f, 1, "tri6")) < 1e-12


@pytest.mark.parametrize("direction", [1, 2])
@pytest.mark.parametrize("scheme,n,p,precision,sweeps", [
    ("tri6", 512, 32, "fp32_refine", 1), ("tri6", 256, 32, "fp32_refine", 2), ("penta10", 512, 32, "fp32_refine", 2),
    ("tri6", 384, 24, "fp32_refine", 1), ("penta10", 256, 32, "fp32_refine_i64", 2)])
def test_refine_yz_lines_warp_per_line(cuda, direction, scheme, n, p, precision, sweeps):
    # y/z lines in 32 lanes (n = p x M, p <= 32): rows are copied line-fastest
    # into the slots of the threads that solve them (a warp per line, shuffled
    # messages) and the results leave through the same slots.  13 lines along
    # x leave the second tile of each row ragged, and 2 x 400 tiles are more
    # than the resident CTAs, so CTAs walk several tiles through both halves
    # of their double buffer.
    rng = np.random.default_rng(71 + direction + n)
    shape = [400, 13, 13] if direction == 1 else [13, 400, 13]
    shape[2 - direction] = n
    f = rng.uniform(-1, 1, size=tuple(shape))
    got, info = gpu_derivative(f, direction, scheme, precision=precision, segments=p, sweeps=sweeps)
    assert info["segments"] == p and info["rows_big"] * p == n
    assert oracle.rel_err(got, oracle_derivative(f, direction, scheme)) < 1e-12


@pytest.mark.parametrize("precision,p", [("fp64", 16), ("fp32_refine", 32), ("fp32", 16)])
def test_x_lines_arrays_off_16_byte_boundary(cuda, precision, p):
    # x-lines of whole-size partitions move rows in 16-byte units when both
    # arrays are 16-byte aligned; views that start one element (8 bytes) into
    # their buffers take the staged kernel and give the same results
    rng = np.random.default_rng(81)
    shape = (3, 21, 512)
    f = rng.uniform(-1, 1, size=shape)
    count = int(np.prod(shape))
    h = W.grid_spacing(512)
    plan = Plan(shape, 0, lhs=W.LELE6_TRI["lhs"], rhs=W.LELE6_TRI["rhs"], h=h, segments=p, precision=precision)
    fb = torch.empty(count + 1, dtype=torch.float64, device="cuda")
    ob = torch.full((count + 1,), float("nan"), dtype=torch.float64, device="cuda")
    x, y = fb[1:].view(shape), ob[1:].view(shape)
    assert x.data_ptr() % 16 == 8 and y.data_ptr() % 16 == 8
    x.copy_(torch.from_numpy(f))
    plan.solve(x, y)
    aligned = plan.solve(torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
    got = y.cpu().numpy()
    assert np.isnan(ob[0].item())  # nothing written before the view
    assert oracle.rel_err(got, aligned.cpu().numpy()) < TOL[precision]
    assert oracle.rel_err(got, oracle_derivative(f, 0, "tri6")) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_identity_lhs_gives_explicit_stencil(cuda, precision):
    # alpha = 0: A = I, every coupling block vanishes and x = S f exactly the
    # explicit central difference (a degenerate case of the method)
    rng = np.random.default_rng(61)
    f = rng.uniform(-1, 1, size=(4, 6, 256))
    h = W.grid_spacing(256)
    plan = Plan(f.shape, 0, lhs=(0.0,), rhs=W.LELE6_TRI["rhs"], h=h, precision=precision)
    y = plan.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    info = plan.info()
    plan.close()
    assert info["message_stages"] == 0
    ref = oracle.central_rhs(f, W.LELE6_TRI["rhs"], h, axis=-1)
    assert oracle.rel_err(y, ref) < 1e-12


@pytest.mark.slow
def test_full_512_cube_sampled(cuda):
    # the 512^3 workload in the launch configuration bench.py times
    # (32 partitions of 16 rows, pipelined kernels), 64 sampled lines per
    # direction against the oracle, FP32 + refinement and FP64
    n = 512
    f_host, _ = W.noisy_cube(n)
    f = torch.from_numpy(f_host).cuda()
    out = torch.empty_like(f)
    h = W.grid_spacing(n)
    rng = np.random.default_rng(99)
    for precision in ("fp32_refine", "fp64"):
        for d in range(3):
            plan = Plan(f.shape, d, lhs=W.LELE6_TRI["lhs"], rhs=W.LELE6_TRI["rhs"], h=h, precision=precision,
                        segments=32)
            plan.solve(f, out)
            torch.cuda.synchronize()
            ax = 2 - d
            idx = rng.integers(0, n, size=(64, 2))
            lines = np.moveaxis(f_host, ax, -1)[idx[:, 0], idx[:, 1]]
            ref = oracle.derivative(lines, W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], h)
            got = np.moveaxis(out.cpu().numpy(), ax, -1)[idx[:, 0], idx[:, 1]]
            assert oracle.rel_err(got, ref) < 1e-12, (precision, d)
            plan.close()


@pytest.mark.parametrize("scheme", ["tri6", "penta10"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refine", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("direction,n,p", [(0, 64, 4), (0, 97, 7), (0, 512, 32), (1, 96, 11), (2, 128, 8),
                                           (0, 250, 31), (1, 48, 3), (2, 16, 1)])
def test_acyclic_solves(cuda, scheme, precision, tol, direction, n, p):
    # the acyclic (non-periodic) system of Sec. 3: ceil(log2 p) PCR steps, no
    # wrapped corners; right-hand side given
    lhs = SCHEMES[scheme]["lhs"]
    if n < 2 * len(lhs) * p:
        pytest.skip("n < 2 r p")
    shape = [5, 6, 7]
    shape[2 - direction] = n
    d = np.random.default_rng(n + p + direction).standard_normal(tuple(shape))
    sweeps = 2 if (scheme == "penta10" and precision == "fp32_refine") else 1
    plan = Plan(tuple(shape), direction, lhs=lhs, rhs=None, segments=p, precision=precision, sweeps=sweeps,
                cyclic=False)
    x = plan.solve(torch.from_numpy(d).cuda()).double().cpu().numpy()
    info = plan.info()
    plan.close()
    assert info["segments"] == p and info["detach_steps"] == 0
    ref = oracle.solve_acyclic(oracle.toeplitz_bands(n, lhs), d, axis=2 - direction)
    assert oracle.rel_err(x, ref) < tol
