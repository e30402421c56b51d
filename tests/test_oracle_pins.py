"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

None of these compares the oracle with itself or with the GPU path:
  * exact Taylor matching (Fractions) of the scheme coefficients;
  * the closed-form modified wavenumber of Eq. 1 on single Fourier modes,
    k'h = (a sin kh + (b/2) sin 2kh + (c/3) sin 3kh) / (1 + 2 alpha cos kh
    + 2 beta cos 2kh), which pins the stencil (signs, indices, 1/(2qh)) and
    the cyclic solve together;
  * dense brute force (numpy LAPACK and the oracle's own pivoting LU) on
    random cyclic banded systems;
  * FFT diagonalisation of circulant systems (any n);
  * the block-LU identity behind the interface system (Sec. 3, Fig. 4);
  * finite differences and an explicit-inverse gradient for the adjoint;
  * the staggered schemes of Eq. 2 / App. A.2: exact Taylor matching, their
    closed-form response to Fourier modes at half-shifted points, sixth-order
    convergence, and the dense transpose of their stencils.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_2101_02286_gb300 import workloads as W


# ---------------------------------------------------------------- scheme order
def _taylor_order(alphas, coefs, kmax=14):
    """Largest P such that the compact scheme
         sum_t A_t f'(t) = sum_q c_q (f(q) - f(-q)) / (2q)      (h = 1)
    is exact for every monomial f = x^k, k <= P (exact rational arithmetic)."""
    A = {0: Fr(1)}
    for q, a in enumerate(alphas, start=1):
        A[q] = A[-q] = Fr(a)
    order = -1
    for k in range(0, kmax + 1):
        lhs = sum(At * (k * Fr(t) ** (k - 1) if k >= 1 else 0) for t, At in A.items())
        rhs = sum(Fr(c) * (Fr(q) ** k - Fr(-q) ** k) / (2 * q) for q, c in enumerate(coefs, start=1))
        if lhs != rhs:
            break
        order = k
    return order


def test_scheme_coefficients_orders():
    f = Fr
    assert _taylor_order([f(1, 3)], [f(14, 9), f(1, 9)]) == 6
    assert _taylor_order([f(1, 2), f(1, 20)], [f(17, 12), f(101, 150), f(1, 100)]) == 10
    assert _taylor_order([], [f(4, 3), f(-1, 3)]) == 4
    assert _taylor_order([f(9, 16), f(9, 100), f(1, 400)], [f(21, 16), f(231, 250), f(147, 2000)]) == 12
    assert W.HEPTA12["lhs"] == (9 / 16, 9 / 100, 1 / 400) and W.HEPTA12["rhs"] == (21 / 16, 231 / 250, 147 / 2000)
    assert _taylor_order([f(9, 16), f(9, 100), f(1, 401)], [f(21, 16), f(231, 250), f(147, 2000)]) < 12
    # the float constants used by the workloads are these rationals
    assert W.LELE6_TRI["lhs"] == (1 / 3,) and W.LELE6_TRI["rhs"] == (14 / 9, 1 / 9)
    assert W.PENTA10["lhs"] == (1 / 2, 1 / 20) and W.PENTA10["rhs"] == (17 / 12, 101 / 150, 1 / 100)
    # a perturbed coefficient loses the order (the check is not vacuous)
    assert _taylor_order([f(1, 3)], [f(14, 9), f(1, 10)]) < 6


# ---------------------------------------------------------------- modified wavenumber
def modified_wavenumber(k, n, lhs, rhs):
    """k' for integer wavenumber k on n points, h = 2 pi / n (derived from Eq. 1)."""
    th = 2 * np.pi * k / n
    num = sum((c / q) * np.sin(q * th) for q, c in enumerate(rhs, start=1))
    den = 1.0 + sum(2 * a * np.cos(q * th) for q, a in enumerate(lhs, start=1))
    return num / den / (2 * np.pi / n)


@pytest.mark.parametrize("scheme", [W.LELE6_TRI, W.PENTA10, W.HEPTA12, {"lhs": (), "rhs": W.CENTRAL4["rhs"]}])
@pytest.mark.parametrize("axis_dir", [0, 1, 2])
def test_closed_form_fourier_cube(scheme, axis_dir):
    # config "64^3, sum of 8 seeded modes": exact answer by linearity
    f, modes = W.fourier_cube(64, 8)
    n = 64
    h = W.grid_spacing(n)
    axis = 2 - axis_dir  # array order (z, y, x)
    lhs = scheme["lhs"]
    got = (oracle.derivative(f, lhs, scheme["rhs"], h, axis=axis) if lhs
           else oracle.central_rhs(f, scheme["rhs"], h, axis=axis))
    x = np.arange(n) * h
    want = np.zeros_like(f)
    for (kx, ky, kz), a in zip(modes.k, modes.amp):
        kd = (kx, ky, kz)[axis_dir]
        phase = kx * x[None, None, :] + ky * x[None, :, None] + kz * x[:, None, None]
        want += a * modified_wavenumber(kd, n, lhs, scheme["rhs"]) * np.cos(phase)
    assert oracle.rel_err(got, want) < 1e-13


def test_closed_form_detects_wrong_sign():
    # planting a sign error in the stencil (oracle input side) breaks the pin
    f, modes = W.fourier_cube(64, 8)
    h = W.grid_spacing(64)
    good = oracle.derivative(f, (1 / 3,), (14 / 9, 1 / 9), h, axis=2)
    bad = oracle.derivative(f, (1 / 3,), (14 / 9, -1 / 9), h, axis=2)
    assert oracle.rel_err(bad, good) > 1e-3


# ---------------------------------------------------------------- brute force
def _random_bands(rng, n, r):
    b = rng.uniform(-1.0, 1.0, size=(2 * r + 1, n))
    b[r] = 2.0 * r + 1.0 + rng.uniform(0.5, 1.5, size=n)  # diagonally dominant
    return b


@pytest.mark.parametrize("r,n", [(r, n) for r in (1, 2, 3) for n in (8, 9, 13, 16, 31, 64) if n >= 4 * r])
def test_cyclic_solve_vs_dense(r, n):
    rng = np.random.default_rng(100 + 7 * n + r)
    bands = _random_bands(rng, n, r)
    d = rng.standard_normal(n)
    A = oracle.dense_matrix(bands)
    ref = np.linalg.solve(A, d)
    ref2 = oracle.dense_solve(A, d)
    assert oracle.rel_err(ref2, ref) < 1e-13
    for method in (["sm", "woodbury"] if r == 1 else ["woodbury"]):
        x = oracle.solve_cyclic(bands, d[None, :], method=method)[0]
        assert oracle.rel_err(x, ref) < 1e-12, method


def test_dense_matrix_layout():
    # bands[k, i] = A[i, (i + k - r) mod n]: check the corners explicitly
    n, r = 6, 2
    b = np.arange(5 * n, dtype=float).reshape(5, n) + 1
    A = oracle.dense_matrix(b)
    assert A[0, n - 2] == b[0, 0] and A[0, n - 1] == b[1, 0] and A[0, 0] == b[2, 0]
    assert A[n - 1, 0] == b[3, n - 1] and A[n - 1, 1] == b[4, n - 1]


def test_per_line_bands_batch():
    rng = np.random.default_rng(5)
    n, lines = 20, 7
    bands = np.stack([_random_bands(rng, n, 1) for _ in range(lines)])
    d = rng.standard_normal((lines, n))
    x = oracle.solve_cyclic(bands, d)
    for l in range(lines):
        assert oracle.rel_err(x[l], np.linalg.solve(oracle.dense_matrix(bands[l]), d[l])) < 1e-12


@pytest.mark.parametrize("lhs", [(1 / 3,), (1 / 2, 1 / 20), (0.45,), (9 / 16, 9 / 100, 1 / 400)])
@pytest.mark.parametrize("n", [512, 1000, 4096])
def test_circulant_fft(lhs, n):
    rng = np.random.default_rng(n)
    d = rng.standard_normal((3, n))
    bands = oracle.toeplitz_bands(n, lhs)
    x = oracle.solve_cyclic(bands, d)
    col = np.zeros(n)
    col[0] = 1.0
    for q, a in enumerate(lhs, start=1):
        col[q] = col[-q] = a
    ref = np.real(np.fft.ifft(np.fft.fft(d, axis=-1) / np.fft.fft(col), axis=-1))
    assert oracle.rel_err(x, ref) < 1e-13
    res = oracle.matvec(bands, x) - d
    assert np.max(np.abs(res)) < 1e-13 * np.max(np.abs(d))


def test_special_cases():
    rng = np.random.default_rng(9)
    d = rng.standard_normal((4, 32))
    # alpha = 0: identity
    assert np.array_equal(oracle.solve_cyclic(oracle.toeplitz_bands(32, (0.0,)), d), d)
    # constant field has zero derivative
    f = np.full((2, 64), 3.25)
    assert np.max(np.abs(oracle.derivative(f, (1 / 3,), (14 / 9, 1 / 9), 0.1))) == 0.0


# ---------------------------------------------------------------- block-LU identity (Sec. 3)
@pytest.mark.parametrize("r,n,p", [(1, 24, 4), (1, 23, 5), (1, 12, 1), (1, 12, 2), (2, 40, 5), (2, 33, 3),
                                   (3, 48, 4), (3, 43, 5)])
def test_schur_complement_identity(r, n, p):
    rng = np.random.default_rng(n * 10 + p)
    bands = _random_bands(rng, n, r)
    b = rng.standard_normal(n)
    Ahat, iface, bulk = oracle.reduced_system_dense(bands, p)
    A = oracle.dense_matrix(bands)
    x = np.linalg.solve(A, b)
    A_IB = A[np.ix_(iface, bulk)]
    A_BB = A[np.ix_(bulk, bulk)]
    bhat = b[iface] - A_IB @ np.linalg.solve(A_BB, b[bulk])
    assert np.allclose(np.linalg.solve(Ahat, bhat), x[iface], rtol=0, atol=1e-12)
    assert Ahat.shape == (p * r, p * r)


def test_partition_convention_fig3():
    # the interface-row convention of the reduced system, against cases worked
    # by hand from Fig. 3 / Eq. 7-8 (interface rows first in each partition)
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "partition_fig3.txt")
    cases = 0
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        head, starts, sizes, iface, bulk = (part.split() for part in line.split("|"))
        n, p, r = (int(v) for v in head)
        got_starts, got_sizes = oracle.partition_bounds(n, p)
        assert got_starts == [int(v) for v in starts] and got_sizes == [int(v) for v in sizes]
        bands = _random_bands(np.random.default_rng(n + p), n, r)
        Ahat, gi, gb = oracle.reduced_system_dense(bands, p)
        assert gi == [int(v) for v in iface] and gb == [int(v) for v in bulk]
        assert Ahat.shape == (p * r, p * r)
        cases += 1
    assert cases == 4


# ---------------------------------------------------------------- adjoint
def test_transpose_bands_is_dense_transpose():
    rng = np.random.default_rng(3)
    for r in (1, 2):
        b = _random_bands(rng, 11, r)
        assert np.allclose(oracle.dense_matrix(oracle.transpose_bands(b)), oracle.dense_matrix(b).T)


def test_stencil_transpose_is_dense_transpose():
    n, coefs, h = 12, (14 / 9, 1 / 9), 0.3
    S = np.stack([oracle.central_rhs(np.eye(n)[j], coefs, h) for j in range(n)], axis=1)
    ST = np.stack([oracle.central_rhs_transpose(np.eye(n)[j], coefs, h) for j in range(n)], axis=1)
    assert np.allclose(ST, S.T, atol=1e-14)


def test_adjoint_dense_inverse_n16():
    rng = np.random.default_rng(4)
    n, coefs, h = 16, W.CENTRAL4["rhs"], W.grid_spacing(16)
    f = rng.uniform(-1, 1, n)
    alpha = rng.uniform(0.2, 0.4, n)
    g = rng.standard_normal(n)
    gf, ga, lam, x = oracle.adjoint_variable_tri(f[None], alpha[None], g[None], coefs, h)
    A = oracle.dense_matrix(oracle.variable_alpha_bands(alpha[None])[0])
    S = np.stack([oracle.central_rhs(np.eye(n)[j], coefs, h) for j in range(n)], axis=1)
    Ainv = np.linalg.inv(A)
    x_ref = Ainv @ S @ f
    lam_ref = Ainv.T @ g
    assert oracle.rel_err(x[0], x_ref) < 1e-13
    assert oracle.rel_err(lam[0], lam_ref) < 1e-13
    assert oracle.rel_err(gf[0], S.T @ lam_ref) < 1e-13
    # dL/dalpha_i = -lam_i (x_{i-1} + x_{i+1}) from dA/dalpha_i = e_i (e_{i-1} + e_{i+1})^T
    ga_ref = np.array([-(lam_ref @ (np.outer(np.eye(n)[i], np.eye(n)[(i - 1) % n] + np.eye(n)[(i + 1) % n]) @ x_ref))
                       for i in range(n)])
    assert oracle.rel_err(ga[0], ga_ref) < 1e-13


def test_adjoint_finite_differences():
    rng = np.random.default_rng(44)
    n, coefs, h = 32, W.CENTRAL4["rhs"], W.grid_spacing(32)
    f = rng.uniform(-1, 1, (2, n))
    alpha = rng.uniform(0.2, 0.4, (2, n))
    g = rng.standard_normal((2, n))
    gf, ga, _, _ = oracle.adjoint_variable_tri(f, alpha, g, coefs, h)

    def loss(ff, aa):
        return float(np.sum(g * oracle.derivative_variable_tri(ff, aa, coefs, h)))

    eps = 1e-6
    for (l, i) in [(0, 0), (1, 7), (0, 31)]:
        e = np.zeros_like(f)
        e[l, i] = eps
        fd_f = (loss(f + e, alpha) - loss(f - e, alpha)) / (2 * eps)
        fd_a = (loss(f, alpha + e) - loss(f, alpha - e)) / (2 * eps)
        assert abs(fd_f - gf[l, i]) < 1e-7 * max(1.0, abs(gf[l, i]))
        assert abs(fd_a - ga[l, i]) < 1e-7 * max(1.0, abs(ga[l, i]))


# ---------------------------------------------------------------- acyclic systems
@pytest.mark.parametrize("lhs", [(1 / 3,), (0.5, 0.05), (9 / 16, 9 / 100, 1 / 400)])
@pytest.mark.parametrize("n", [9, 16, 41])
def test_acyclic_solve_matches_dense_lapack(lhs, n):
    # Sec. 3 acyclic case: no wrapped corners; brute force by LAPACK
    rng = np.random.default_rng(n)
    B = oracle.toeplitz_bands(n, lhs)
    d = rng.standard_normal((3, n))
    A = oracle.acyclic_dense_matrix(B)
    ref = np.linalg.solve(A, d.T).T
    assert oracle.rel_err(oracle.solve_acyclic(B, d), ref) < 1e-14


def test_acyclic_matrix_is_cyclic_without_corners():
    n = 12
    for lhs in [(1 / 3,), (0.5, 0.05), (9 / 16, 9 / 100, 1 / 400)]:
        B = oracle.toeplitz_bands(n, lhs)
        diff = oracle.dense_matrix(B) - oracle.acyclic_dense_matrix(B)
        r = len(lhs)
        nz = np.argwhere(diff != 0)
        # only entries with |i - j| > n - 1 - r (the wrapped corners) differ
        assert len(nz) == r * (r + 1)
        assert all(abs(i - j) >= n - r for i, j in nz)


def test_acyclic_solve_per_line_bands_recovers_known_solution():
    rng = np.random.default_rng(3)
    lines, n = 4, 30
    al = rng.uniform(0.2, 0.4, size=(lines, n))
    bands = oracle.variable_alpha_bands(al)
    x = rng.standard_normal((lines, n))
    d = np.stack([oracle.acyclic_dense_matrix(bands[l]) @ x[l] for l in range(lines)])
    assert oracle.rel_err(oracle.solve_acyclic(bands, d), x) < 1e-13


# ---------------------------------------------------------------- staggered schemes (Eq. 2, App. A.2)
def _staggered_order(alpha, coefs, interp, kmax=12):
    """Largest P such that the staggered scheme (h = 1, output at t = 0, input
    at the half points +-(q - 1/2)) is exact for every monomial x^k, k <= P:
      derivative:    sum_t A_t f'(t) = sum_q c_q (f(q-1/2) - f(1/2-q)) / (2q-1)
      interpolation: sum_t A_t f(t)  = sum_q c_q (f(q-1/2) + f(1/2-q)) / 2."""
    A = {0: Fr(1), 1: Fr(alpha), -1: Fr(alpha)}
    order = -1
    for k in range(0, kmax + 1):
        if interp:
            lhs = sum(At * Fr(t) ** k for t, At in A.items())
        else:
            lhs = sum(At * (k * Fr(t) ** (k - 1) if k >= 1 else 0) for t, At in A.items())
        rhs = Fr(0)
        for q, c in enumerate(coefs, start=1):
            u, d = Fr(2 * q - 1, 2), -Fr(2 * q - 1, 2)
            rhs += Fr(c) * ((u ** k + d ** k) / 2 if interp else (u ** k - d ** k) / (2 * q - 1))
        if lhs != rhs:
            break
        order = k
    return order


def test_staggered_scheme_coefficients_orders():
    f = Fr
    # App. A.2: both printed schemes are sixth order (the derivative is exact
    # through x^6, the interpolation through x^5: error terms h^6 in both)
    assert _staggered_order(f(9, 62), [f(63, 62), f(17, 62)], interp=False) == 6
    assert _staggered_order(f(3, 10), [f(3, 2), f(1, 10)], interp=True) == 5
    assert W.STAGGERED6 == {"lhs": (9 / 62,), "rhs": (63 / 62, 17 / 62)}
    assert W.MIDPOINT6 == {"lhs": (3 / 10,), "rhs": (3 / 2, 1 / 10)}
    # a perturbed coefficient loses the order
    assert _staggered_order(f(9, 62), [f(63, 62), f(17, 63)], interp=False) < 6
    assert _staggered_order(f(3, 10), [f(3, 2), f(1, 11)], interp=True) < 5


def _staggered_modes(rng, lines, n, count=6):
    ks = rng.integers(1, n // 3, size=(lines, count))
    ph = rng.uniform(0, 2 * np.pi, size=(lines, count))
    amp = rng.standard_normal((lines, count))
    return ks, ph, amp


@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("n", [16, 48, 97])
def test_staggered_closed_form_fourier(shift, n):
    # sum of plane waves sampled at the input points; the scheme's exact
    # response at the output points (derived from the definitions):
    #   derivative:    K'(k) = sum_q 2 c_q sin((2q-1) kh/2) / ((2q-1) h) / (1 + 2 alpha cos kh)
    #   interpolation: T(k)  = sum_q c_q cos((2q-1) kh/2) / (1 + 2 alpha cos kh)
    rng = np.random.default_rng(11 + n + shift)
    lines = 5
    h = W.grid_spacing(n)
    ks, ph, amp = _staggered_modes(rng, lines, n)
    j = np.arange(n)
    x_in = (j + (0.5 if shift == 0 else 0.0)) * h
    x_out = (j + (0.0 if shift == 0 else 0.5)) * h
    f = np.zeros((lines, n))
    want_d = np.zeros((lines, n))
    want_i = np.zeros((lines, n))
    (ad,), (cd1, cd2) = W.STAGGERED6["lhs"], W.STAGGERED6["rhs"]
    (ai,), (ci1, ci2) = W.MIDPOINT6["lhs"], W.MIDPOINT6["rhs"]
    for l in range(lines):
        for k, p, a in zip(ks[l], ph[l], amp[l]):
            th = k * h
            f[l] += a * np.sin(k * x_in + p)
            kp = (2 * cd1 * np.sin(th / 2) / h + 2 * cd2 * np.sin(3 * th / 2) / (3 * h)) / (1 + 2 * ad * np.cos(th))
            tt = (ci1 * np.cos(th / 2) + ci2 * np.cos(3 * th / 2)) / (1 + 2 * ai * np.cos(th))
            want_d[l] += a * kp * np.cos(k * x_out + p)
            want_i[l] += a * tt * np.sin(k * x_out + p)
    got_d = oracle.staggered_derivative(f, W.STAGGERED6["lhs"], W.STAGGERED6["rhs"], h, shift)
    got_i = oracle.midpoint_interpolation(f, W.MIDPOINT6["lhs"], W.MIDPOINT6["rhs"], shift)
    assert oracle.rel_err(got_d, want_d) < 1e-13
    assert oracle.rel_err(got_i, want_i) < 1e-13
    # the other shift puts the answer half a cell off: the pin tells them apart
    other = oracle.staggered_derivative(f, W.STAGGERED6["lhs"], W.STAGGERED6["rhs"], h, 1 - shift)
    assert oracle.rel_err(other, want_d) > 1e-3


def test_staggered_sixth_order_convergence():
    # f = exp(sin x) on [0, 2 pi): the error against the exact derivative /
    # midpoint values falls by ~2^6 per doubling of n
    errs_d, errs_i = [], []
    for n in (16, 32, 64):
        h = W.grid_spacing(n)
        xs = (np.arange(n) + 0.5) * h  # staggered input, nodes out (shift 0)
        xn = np.arange(n) * h
        f = np.exp(np.sin(xs))[None, :]
        d = oracle.staggered_derivative(f, W.STAGGERED6["lhs"], W.STAGGERED6["rhs"], h, 0)
        it = oracle.midpoint_interpolation(f, W.MIDPOINT6["lhs"], W.MIDPOINT6["rhs"], 0)
        errs_d.append(np.abs(d[0] - np.cos(xn) * np.exp(np.sin(xn))).max())
        errs_i.append(np.abs(it[0] - np.exp(np.sin(xn))).max())
    for e in (errs_d, errs_i):
        assert e[0] / e[1] > 2 ** 5.5 and e[1] / e[2] > 2 ** 5.5


@pytest.mark.parametrize("shift", [0, 1])
def test_staggered_transpose_is_dense_transpose(shift):
    n, coefs, h = 11, (63 / 62, 17 / 62), 0.3
    I = np.eye(n)
    for fwd, tr, neg in ((lambda v, s: oracle.staggered_rhs(v, coefs, h, s),
                          lambda v, s: oracle.staggered_rhs_transpose(v, coefs, h, s), -1.0),
                         (lambda v, s: oracle.midpoint_rhs(v, coefs, s),
                          lambda v, s: oracle.midpoint_rhs_transpose(v, coefs, s), 1.0)):
        S = np.stack([fwd(I[j], shift) for j in range(n)], axis=1)
        ST = np.stack([tr(I[j], shift) for j in range(n)], axis=1)
        assert np.allclose(ST, S.T, atol=1e-14)
        # S^T is the other shift's stencil, negated for the derivative
        S_other = np.stack([fwd(I[j], 1 - shift) for j in range(n)], axis=1)
        assert np.allclose(ST, neg * S_other, atol=1e-14)


# ---------------------------------------------------------------- boundary closures (acyclic derivative)
def _row_order(L, R, kmax=10):
    """Largest P such that the boundary row sum_j L_j f'(j) = sum_j R_j f(j)
    (h = 1, nodes j = 0, 1, ...) is exact for every monomial x^k, k <= P."""
    order = -1
    for k in range(kmax + 1):
        lhs = sum(Fr(l) * (k * Fr(j) ** (k - 1) if k >= 1 else 0) for j, l in enumerate(L))
        rhs = sum(Fr(r) * Fr(j) ** k for j, r in enumerate(R))
        if lhs != rhs:
            break
        order = k
    return order


def test_closure_rows_taylor_order():
    f = Fr
    third = ([1, 2, 0], [f(-5, 2), 2, f(1, 2)])
    fourth = ([f(1, 4), 1, f(1, 4)], [f(-3, 4), 0, f(3, 4)])
    sixth = ([0, f(1, 3), 1, f(1, 3), 0], [f(-1, 36), f(-7, 9), 0, f(7, 9), f(1, 36)])
    assert _row_order(*third) == 3
    assert _row_order(*fourth) == 4
    assert _row_order(*sixth) == 6
    assert _row_order([1, 2, 0], [f(-5, 2), 2, f(1, 3)]) < 3  # not vacuous
    # the float constants of the workloads are these rationals (rounded)
    def rat(rows):
        return [[Fr(v).limit_denominator(1000) for v in r] for r in rows]
    L, R = W.CLOSURE3_4
    assert rat(L) == [third[0], fourth[0]] and rat(R) == [third[1], fourth[1]]
    L, R = W.CLOSURE3_4_6
    assert rat(L) == [third[0] + [0, 0], fourth[0] + [0, 0], sixth[0]]
    assert rat(R) == [third[1] + [0, 0], fourth[1] + [0, 0], sixth[1]]


def _poly_case(n, deg, L=1.3):
    h = L / (n - 1)
    x = np.arange(n) * h
    c = np.random.default_rng(deg + n).uniform(-1, 1, size=deg + 1)
    f = np.polyval(c, x)
    fp = np.polyval(np.polyder(c), x) if deg > 0 else np.zeros(n)
    return f, fp, h


@pytest.mark.parametrize("scheme,closure", [(W.LELE6_TRI, W.CLOSURE3_4), (W.PENTA10, W.CLOSURE3_4_6)])
@pytest.mark.parametrize("n", [24, 41, 64])
def test_closure_oracle_exact_for_cubics(scheme, closure, n):
    # the lowest-order row (third order) is exact for cubics, every other row
    # for higher degrees, so A_c x = B_c f holds with x = f' exactly: the
    # solve returns the derivative to rounding, on both ends of the line
    for deg in range(4):
        f, fp, h = _poly_case(n, deg)
        x = oracle.derivative_closure(f[None], scheme["lhs"], scheme["rhs"], closure, h)[0]
        assert np.max(np.abs(x - fp)) < 1e-12 * max(1.0, np.max(np.abs(fp))), deg
    f, fp, h = _poly_case(n, 4)  # a quartic is not reproduced (the check is not vacuous)
    x = oracle.derivative_closure(f[None], scheme["lhs"], scheme["rhs"], closure, h)[0]
    assert np.max(np.abs(x - fp)) > 1e-8


def test_closure_mirror_sign_matters():
    # a plausible mistake planted in the oracle's matrices: the right end's
    # RHS rows not negated.  The cubic pin then fails at the right boundary.
    n = 32
    f, fp, h = _poly_case(n, 2)
    A, B = oracle.closure_matrices(n, W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], W.CLOSURE3_4, h)
    B[n - 2:] *= -1.0
    x = np.linalg.solve(A, B @ f)
    assert np.max(np.abs(x[n - 4:] - fp[n - 4:])) > 1e-2


def test_closure_convergence_third_order():
    # smooth non-periodic f: the error falls like h^3 (the third-order row)
    errs = []
    for n in (64, 128, 256):
        h = 1.0 / (n - 1)
        x = np.arange(n) * h
        f = np.sin(3 * x) + np.exp(x)
        got = oracle.derivative_closure(f[None], W.LELE6_TRI["lhs"], W.LELE6_TRI["rhs"], W.CLOSURE3_4, h)[0]
        errs.append(np.max(np.abs(got - (3 * np.cos(3 * x) + np.exp(x)))))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.9 < o < 4.0 for o in orders), orders


# ---------------------------------------------------------------- block entries
# Block-tridiagonal systems with 2 x 2 blocks (Sec. 1: block entries), as the
# banded matrices the oracle's solves take.  Blocks: diagonally dominant,
# neither symmetric nor diagonal, so a transposed block or a swapped L/U
# changes the answer.
BL = np.array([[0.21, 0.07], [-0.05, 0.18]])
BD = np.array([[1.0, 0.15], [-0.12, 0.9]])
BU = np.array([[0.24, -0.06], [0.04, 0.2]])


def test_block_bands_flatten_the_block_matrix():
    # the banded form, expanded, equals the matrix assembled block by block
    # (cyclic and acyclic); half bandwidth 2b - 1 = 3
    for npts in (3, 5, 8):
        bands = oracle.block_tridiagonal_bands(npts, BL, BD, BU)
        assert bands.shape == (7, 2 * npts)
        assert np.array_equal(oracle.dense_matrix(bands), oracle.block_dense_matrix(npts, BL, BD, BU))
        assert np.array_equal(oracle.acyclic_dense_matrix(bands),
                              oracle.block_dense_matrix(npts, BL, BD, BU, cyclic=False))


@pytest.mark.parametrize("npts", [6, 7, 16, 33])  # the oracle's cyclic banded path needs n >= 4r
def test_block_solves_match_lapack(npts):
    rng = np.random.default_rng(npts)
    d = rng.standard_normal((3, 2 * npts))
    bands = oracle.block_tridiagonal_bands(npts, BL, BD, BU)
    for cyclic in (True, False):
        A = oracle.block_dense_matrix(npts, BL, BD, BU, cyclic=cyclic)
        ref = np.linalg.solve(A, d.T).T
        got = oracle.solve_cyclic(bands, d) if cyclic else oracle.solve_acyclic(bands, d)
        assert oracle.rel_err(got, ref) < 1e-13, cyclic


def test_block_diagonal_blocks_decouple():
    # diagonal blocks: the two unknowns of a point never meet, so the system
    # is two independent scalar tridiagonal systems (Thomas + Sherman-Morrison)
    npts = 24
    L, D, U = np.diag([0.2, 0.3]), np.diag([1.0, 1.1]), np.diag([0.25, 0.15])
    rng = np.random.default_rng(3)
    d = rng.standard_normal(2 * npts)
    got = oracle.solve_cyclic(oracle.block_tridiagonal_bands(npts, L, D, U), d)
    for c in range(2):
        tri = np.zeros((3, npts))
        tri[0], tri[1], tri[2] = L[c, c], D[c, c], U[c, c]
        ref = oracle.solve_cyclic(tri, d[c::2])
        assert oracle.rel_err(got[c::2], ref) < 1e-14


def test_block_kronecker_closed_form():
    # L = l K, D = d K, U = u K: A = T (x) K with T = tri(l, d, u) cyclic, so
    # x (points x unknowns) = T^{-1} B K^{-T}
    npts = 20
    K = np.array([[1.0, 0.3], [-0.2, 0.8]])
    l, dd, u = 0.2, 1.0, 0.3
    rng = np.random.default_rng(4)
    B = rng.standard_normal((npts, 2))
    T = np.zeros((npts, npts))
    for m in range(npts):
        T[m, m], T[m, (m - 1) % npts], T[m, (m + 1) % npts] = dd, l, u
    ref = np.linalg.solve(T, B) @ np.linalg.inv(K).T
    got = oracle.solve_cyclic(oracle.block_tridiagonal_bands(npts, l * K, dd * K, u * K), B.ravel())
    assert oracle.rel_err(got.reshape(npts, 2), ref) < 1e-13


def test_block_partition_bounds_keep_points_whole():
    starts, sizes = oracle.partition_bounds(26, 4, unit=2)
    assert sizes == [8, 6, 6, 6] and starts == [0, 8, 14, 20]


def test_woodbury_size_limit_is_reported():
    # n < 4r: the banded Woodbury path refuses with a clear message instead of
    # a misleading pivot error; dense_solve covers such tiny systems
    bands = oracle.toeplitz_bands(8, (0.3, 0.1, 0.02))
    with pytest.raises(ValueError):
        oracle.solve_cyclic(bands, np.ones(8))
    x = oracle.dense_solve(oracle.dense_matrix(bands), np.ones(8))
    assert np.allclose(oracle.dense_matrix(bands) @ x, 1.0)
