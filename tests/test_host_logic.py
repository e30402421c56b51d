"""Host logic of the library, no GPU: the interface schedule (Algorithm 1),
its step counts (Sec. 4), the reduced system of Eq. 18-20 against the dense
Schur complement (Sec. 3, Fig. 4) and the pre-factorised stage coefficients
against a dense solve of A-hat."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2101_02286_gb300 import abi
from paper_2101_02286_gb300.solver import make_desc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NAMES = {0: "detach", 1: "pcr", 2: "final", 3: "reattach"}


def test_schedule_p11_matches_paper_example():
    rows = []
    with open(os.path.join(GOLDEN, "schedule_p11_cyclic.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, s, na, _ = line.split()
                rows.append((name, int(s), int(na)))
    got = [(NAMES[t], s, na) for t, s, na in abi.cbs_schedule(11, True)]
    assert got == rows


@pytest.mark.parametrize("p", list(range(1, 130)) + [255, 256, 257, 1023, 1024, 1025, 2047, 2048])
def test_schedule_counts_cyclic(p):
    st = abi.cbs_schedule(p, True)
    pcr = sum(1 for t, _, _ in st if t == 1)
    det = [(s, na) for t, s, na in st if t == 0]
    rea = [(s, na) for t, s, na in st if t == 3]
    fl = int(np.floor(np.log2(p)))
    assert pcr == fl                                   # floor(log2 p) PCR steps
    assert len(det) == bin(p).count("1") - 1           # sum_n (floor(p/2^n) mod 2) - 1
    assert len(rea) == len(det)
    assert sum(s for s, _ in det) == p - 2 ** fl       # rows detached overall
    assert rea == det[::-1]                            # reattach in reverse order
    assert [t for t, _, _ in st].count(2) == 1


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 13, 64, 100])
def test_schedule_counts_acyclic(p):
    st = abi.cbs_schedule(p, False)
    assert sum(1 for t, _, _ in st if t == 1) == (int(np.ceil(np.log2(p))) if p > 1 else 0)
    assert all(t in (1, 2) for t, _, _ in st)


def _cases():
    out = []
    for lhs in [(1 / 3,), (0.45,), (1 / 2, 1 / 20), (0.3, 0.02), (9 / 16, 9 / 100, 1 / 400)]:
        r = len(lhs)
        for n, p in [(16, 1), (16, 2), (17, 3), (24, 4), (33, 5), (40, 7), (64, 11), (64, 16), (96, 13),
                     (128, 32), (130, 31), (192, 32), (200, 31)]:
            if n >= 2 * r * p:
                out.append((lhs, n, p))
    return out


@pytest.mark.parametrize("lhs,n,p", _cases())
@pytest.mark.parametrize("cyclic", [True, False])
def test_reduced_system_matches_schur_complement(lhs, n, p, cyclic):
    r = len(lhs)
    desc = make_desc((1, 1, n), 0, lhs=lhs, cyclic=cyclic)
    D, L, U, _ = abi.cbs_interface_model(desc, p)
    bands = oracle.toeplitz_bands(n, lhs)
    if not cyclic:
        # acyclic: drop the wrapped corner entries
        for k in range(2 * r + 1):
            t = k - r
            for i in range(n):
                if not (0 <= i + t < n):
                    bands[k, i] = 0.0
    Ahat, _, _ = oracle.reduced_system_dense(bands, p)
    # assemble the plan's blocks into a dense p r x p r matrix
    M = np.zeros((p * r, p * r))
    for i in range(p):
        M[i * r:(i + 1) * r, i * r:(i + 1) * r] += D[i]
        im, ip = (i - 1) % p, (i + 1) % p
        M[i * r:(i + 1) * r, im * r:(im + 1) * r] += L[i]
        M[i * r:(i + 1) * r, ip * r:(ip + 1) * r] += U[i]
    assert np.max(np.abs(M - Ahat)) < 1e-13


@pytest.mark.parametrize("lhs,n,p", _cases())
@pytest.mark.parametrize("cyclic", [True, False])
def test_prefactorised_interface_solve(lhs, n, p, cyclic):
    r = len(lhs)
    desc = make_desc((1, 1, n), 0, lhs=lhs, cyclic=cyclic)
    rng = np.random.default_rng(n * 31 + p)
    bhat = rng.standard_normal(p * r)
    D, L, U, xt = abi.cbs_interface_model(desc, p, bhat)
    M = np.zeros((p * r, p * r))
    for i in range(p):
        M[i * r:(i + 1) * r, i * r:(i + 1) * r] += D[i]
        M[i * r:(i + 1) * r, ((i - 1) % p) * r:((i - 1) % p + 1) * r] += L[i]
        M[i * r:(i + 1) * r, ((i + 1) % p) * r:((i + 1) % p + 1) * r] += U[i]
    ref = np.linalg.solve(M, bhat)
    assert oracle.rel_err(xt, ref) < 1e-12


def test_invalid_descriptors_rejected():
    d = make_desc((1, 1, 8), 0, lhs=(1 / 3,))
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_interface_model(d, 5)  # n < 2 r p
    assert e.value.status == abi.CBS_ERR_INVALID_ARG
    d.bandwidth = 9
    with pytest.raises(abi.CbsError):
        abi.cbs_interface_model(d, 2)


def test_singular_interface_reported():
    # alpha = 1/2: A = B[1/2, 1, 1/2] is singular for even n (symbol 1 + cos)
    d = make_desc((1, 1, 16), 0, lhs=(0.5,))
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_interface_model(d, 4, np.ones(4))
    assert e.value.status == abi.CBS_ERR_SINGULAR


def test_plan_create_validates_before_any_device_work():
    # rejected descriptors never reach the device (no GPU needed)
    from paper_2101_02286_gb300.solver import Plan
    cases = [
        (dict(shape=(0, 4, 64)), abi.CBS_ERR_INVALID_ARG),            # empty field
        (dict(shape=(4, 4, 64), precision="fp32_refine", sweeps=3), abi.CBS_ERR_INVALID_ARG),
        (dict(shape=(70000, 2, 64), direction=1), abi.CBS_ERR_UNSUPPORTED),  # y-line grid extent
        (dict(shape=(4, 4, 64), h=0.0), abi.CBS_ERR_INVALID_ARG),     # stencil spacing
        (dict(shape=(4, 4, 8), segments=5), abi.CBS_ERR_INVALID_ARG),  # n < 2 r p
    ]
    for kw, status in cases:
        shape = kw.pop("shape")
        direction = kw.pop("direction", 0)
        h = kw.pop("h", 0.1)
        with pytest.raises(abi.CbsError) as e:
            Plan(shape, direction, lhs=(1 / 3,), rhs=(14 / 9, 1 / 9), h=h, **kw)
        assert e.value.status == status, (shape, kw)
    d = make_desc((4, 4, 64), 0, lhs=(1 / 3,))
    d.precision = 7
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_plan_create(d)
    assert e.value.status == abi.CBS_ERR_INVALID_ARG


def test_closure_descriptors_validated_before_device_work():
    from paper_2101_02286_gb300 import workloads as W
    cl = W.CLOSURE3_4
    tri = W.LELE6_TRI
    d = make_desc((2, 2, 64), 0, lhs=tri["lhs"], rhs=tri["rhs"], h=0.1, cyclic=False)
    with pytest.raises(abi.CbsError) as e:  # an acyclic derivative needs closures
        abi.cbs_plan_create(d)
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED
    d = make_desc((2, 2, 64), 0, lhs=tri["lhs"], rhs=tri["rhs"], h=0.1, cyclic=True, closure=cl)
    with pytest.raises(abi.CbsError) as e:  # closures on a periodic line
        abi.cbs_plan_create(d)
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED
    d = make_desc((2, 2, 64), 0, lhs=tri["lhs"], rhs=tri["rhs"], h=0.1, cyclic=False, closure=cl)
    d.closure = None
    with pytest.raises(abi.CbsError) as e:  # rows without their array
        abi.cbs_plan_create(d)
    assert e.value.status == abi.CBS_ERR_INVALID_ARG
    d = make_desc((2, 2, 64), 0, lhs=tri["lhs"], rhs=tri["rhs"], h=0.1, cyclic=False, closure=cl)
    d.closure_width = 17
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_plan_create(d)
    assert e.value.status == abi.CBS_ERR_INVALID_ARG
    d = make_desc((2, 2, 64), 0, lhs=tri["lhs"], rhs=None, cyclic=False, closure=cl)
    with pytest.raises(abi.CbsError) as e:  # closures belong to a stencil
        abi.cbs_plan_create(d)
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED


def test_staggered_descriptors_validated_before_device_work():
    from paper_2101_02286_gb300 import workloads as W
    from paper_2101_02286_gb300.solver import Plan
    sch = W.STAGGERED6
    cases = [
        (dict(stencil="staggered", shift=2), abi.CBS_ERR_INVALID_ARG),               # shift is 0 or 1
        (dict(stencil="midpoint", rhs=(1.5, 0.1, 0.01)), abi.CBS_ERR_INVALID_ARG),   # 1..2 terms
        (dict(stencil="staggered", h=0.0), abi.CBS_ERR_INVALID_ARG),                 # derivative spacing
        (dict(stencil="staggered", cyclic=False), abi.CBS_ERR_UNSUPPORTED),          # periodic only
        (dict(stencil="midpoint", lhs="variable", bands_ptr=4096), abi.CBS_ERR_UNSUPPORTED),
    ]
    for kw, status in cases:
        kw.setdefault("lhs", sch["lhs"])
        kw.setdefault("rhs", sch["rhs"])
        kw.setdefault("h", 0.1)
        with pytest.raises(abi.CbsError) as e:
            Plan((4, 4, 64), 0, **kw)
        assert e.value.status == status, kw
    d = make_desc((4, 4, 64), 0, lhs=sch["lhs"], rhs=sch["rhs"], h=0.1)
    d.rhs_kind = 4
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_plan_create(d)
    assert e.value.status == abi.CBS_ERR_INVALID_ARG


# ---------------------------------------------------------------- block entries
BLK = (np.array([[0.21, 0.07], [-0.05, 0.18]]), np.array([[1.0, 0.15], [-0.12, 0.9]]),
       np.array([[0.24, -0.06], [0.04, 0.2]]))


@pytest.mark.parametrize("npts,p", [(8, 1), (12, 2), (13, 3), (24, 4), (40, 5), (64, 16), (100, 31), (96, 32)])
@pytest.mark.parametrize("cyclic", [True, False])
def test_block_reduced_system_matches_schur_complement(npts, p, cyclic):
    # the plan's interface system for 2 x 2 block entries (periodic bands of
    # half bandwidth 3, partitions of whole points) against the dense Schur
    # complement of the flattened matrix, and its pre-factorised solve
    n, r = 2 * npts, 3
    desc = make_desc((1, 1, n), 0, blocks=BLK, cyclic=cyclic)
    rng = np.random.default_rng(npts * 7 + p)
    bhat = rng.standard_normal(p * r)
    D, L, U, xt = abi.cbs_interface_model(desc, p, bhat)
    A = oracle.block_dense_matrix(npts, *BLK, cyclic=cyclic)
    bands = np.zeros((7, n))  # the banded form of A (corners dropped when acyclic)
    for i in range(n):
        for k in range(7):
            bands[k, i] = A[i, (i + k - r) % n] if (cyclic or 0 <= i + k - r < n) else 0.0
    Ahat, _, _ = oracle.reduced_system_dense(bands, p, unit=2)
    M = np.zeros((p * r, p * r))
    for i in range(p):
        M[i * r:(i + 1) * r, i * r:(i + 1) * r] += D[i]
        M[i * r:(i + 1) * r, ((i - 1) % p) * r:((i - 1) % p + 1) * r] += L[i]
        M[i * r:(i + 1) * r, ((i + 1) % p) * r:((i + 1) % p + 1) * r] += U[i]
    assert np.max(np.abs(M - Ahat)) < 1e-13
    assert oracle.rel_err(xt, np.linalg.solve(M, bhat)) < 1e-12


def test_block_descriptors_validated():
    from paper_2101_02286_gb300.solver import Plan
    good = dict(blocks=BLK)
    for shape, kw, status in [
            ((1, 1, 63), good, abi.CBS_ERR_INVALID_ARG),                      # odd line length
            ((1, 1, 64), dict(good, precision="fp32_refine"), abi.CBS_ERR_UNSUPPORTED),
            ((1, 1, 64), dict(good, rhs=(14 / 9, 1 / 9)), abi.CBS_ERR_UNSUPPORTED)]:
        with pytest.raises(abi.CbsError) as e:
            Plan(shape, 0, **kw)
        assert e.value.status == status, (shape, kw)
    d = make_desc((1, 1, 64), 0, blocks=BLK)
    d.block_size = 3
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_interface_model(d, 2)
    assert e.value.status == abi.CBS_ERR_UNSUPPORTED
    d = make_desc((1, 1, 64), 0, blocks=BLK)
    d.bandwidth = 5
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_interface_model(d, 2)
    assert e.value.status == abi.CBS_ERR_INVALID_ARG
    d = make_desc((1, 1, 64), 0, blocks=BLK)
    with pytest.raises(abi.CbsError) as e:
        abi.cbs_interface_model(d, 40)  # more partitions than points
    assert e.value.status == abi.CBS_ERR_INVALID_ARG
