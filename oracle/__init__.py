"""FP64 CPU oracle for cyclic compact banded solves -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never imports it, and
it imports nothing from the GPU library: the two share no code.  Inputs reach
both sides from the seeded generators in ``paper_2101_02286_gb300.workloads``,
which hold none of the method's arithmetic.

What the oracle computes is the plain definition of the method's result:

* ``central_rhs``      d = S f, periodic central differences, paper Eq. 1
                       (right-hand side; K-term Lele form).
* ``solve_cyclic``     x = A^{-1} d for cyclic banded A.  Tridiagonal: Thomas +
                       Sherman-Morrison; any half-bandwidth r: banded LU +
                       rank-2r Woodbury (C routines in ``cbs_oracle.c``).
                       The paper's solver is direct (abstract, Sec. 3), so its
                       exact result is this solution.
* ``derivative``       x = A^{-1} S f, the compact first derivative (Eq. 1).
* ``staggered_rhs`` / ``midpoint_rhs``  the right-hand sides of the staggered
                       sixth-order derivative and of the compact midpoint
                       interpolation (Eq. 2, App. A.2), between a grid and the
                       grid shifted by half a spacing; ``staggered_derivative``
                       / ``midpoint_interpolation`` solve with them.
* ``solve_acyclic``    x = B^{-1} d for the non-periodic banded B (Sec. 3,
                       acyclic case): banded LU without pivoting.
* ``closure_matrices`` / ``derivative_closure``  the acyclic first derivative
                       with one-sided boundary rows: the dense matrices A_c,
                       B_c written out row by row (interior rows: Eq. 1; the
                       first and last rows: the given closure rows and their
                       mirror image), x = A_c^{-1} B_c f by a dense solve.  The
                       paper prints no closure; the rows are inputs.
* ``dense_matrix`` / ``acyclic_dense_matrix`` / ``dense_solve``  brute force
                       for tiny n (partial pivoting).
* ``block_tridiagonal_bands`` / ``block_dense_matrix``  block entries (Sec. 1):
                       the block-tridiagonal matrix with b x b blocks as the
                       banded matrix of half bandwidth 2b - 1 that the solves
                       above take, and assembled block by block for dense
                       checks.
* ``adjoint_variable_tri``  gradients of L = <g, x> for x = A(alpha)^{-1} S f:
                       lambda = A^{-T} g, grad_f = S^T lambda,
                       grad_alpha_i = -lambda_i (x_{i-1} + x_{i+1}).  The paper
                       has no adjoint; this is the textbook adjoint of a linear
                       solve.
* ``reduced_system_dense``  the interface system A-hat of Sec. 3 formed as the
                       Schur complement of the permuted matrix P A P^T
                       (Fig. 4 block-LU view), by dense linear algebra.

Every routine is FP64.  Parity is pinned in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cbs_oracle.c")
_LIB = os.path.join(_HERE, "libcbs_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over lines) into oracle/."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L = ctypes.c_long
        lib.orc_central_rhs.argtypes = [dp, dp, L, L, dp, ctypes.c_int, ctypes.c_double]
        lib.orc_central_rhs_transpose.argtypes = [dp, dp, L, L, dp, ctypes.c_int, ctypes.c_double]
        lib.orc_staggered_rhs.argtypes = [dp, dp, L, L, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int]
        lib.orc_staggered_rhs_transpose.argtypes = lib.orc_staggered_rhs.argtypes
        lib.orc_cyclic_tri.argtypes = [dp, L, dp, dp, L, L]
        lib.orc_cyclic_tri.restype = ctypes.c_int
        lib.orc_cyclic_banded.argtypes = [dp, L, dp, dp, L, L, ctypes.c_int]
        lib.orc_cyclic_banded.restype = ctypes.c_int
        lib.orc_acyclic_banded.argtypes = [dp, L, dp, dp, L, L, ctypes.c_int]
        lib.orc_acyclic_banded.restype = ctypes.c_int
        lib.orc_banded_matvec.argtypes = [dp, L, dp, dp, L, L, ctypes.c_int]
        lib.orc_dense_solve.argtypes = [dp, dp, L]
        lib.orc_dense_solve.restype = ctypes.c_int
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the batched C routines use."""
    return int(_load().orc_num_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lines(a: np.ndarray, axis: int):
    """Move `axis` last and return a contiguous (lines, n) FP64 view + restore info."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis, -1)
    shape = a.shape
    return np.ascontiguousarray(a).reshape(-1, shape[-1]), shape


def _unlines(a2: np.ndarray, shape, axis: int) -> np.ndarray:
    return np.moveaxis(a2.reshape(shape), -1, axis)


# ---------------------------------------------------------------- stencils
def central_rhs(f, coefs, h, axis=-1):
    """d_i = sum_k coefs[k-1] (f_{i+k} - f_{i-k}) / (2 k h), periodic (Eq. 1 RHS)."""
    f2, shape = _lines(f, axis)
    c = np.ascontiguousarray(coefs, dtype=np.float64)
    out = np.empty_like(f2)
    _load().orc_central_rhs(_ptr(f2), _ptr(out), f2.shape[0], f2.shape[1], _ptr(c), len(c), float(h))
    return _unlines(out, shape, axis)


def central_rhs_transpose(g, coefs, h, axis=-1):
    """S^T g for the stencil of central_rhs (scatter form)."""
    g2, shape = _lines(g, axis)
    c = np.ascontiguousarray(coefs, dtype=np.float64)
    out = np.empty_like(g2)
    _load().orc_central_rhs_transpose(_ptr(g2), _ptr(out), g2.shape[0], g2.shape[1], _ptr(c), len(c), float(h))
    return _unlines(out, shape, axis)


def _staggered(f, coefs, h, shift, kind, transpose, axis):
    if shift not in (0, 1):
        raise ValueError("shift must be 0 or 1")
    f2, shape = _lines(f, axis)
    c = np.ascontiguousarray(coefs, dtype=np.float64)
    out = np.empty_like(f2)
    fn = _load().orc_staggered_rhs_transpose if transpose else _load().orc_staggered_rhs
    fn(_ptr(f2), _ptr(out), f2.shape[0], f2.shape[1], _ptr(c), len(c), float(h), int(shift), int(kind))
    return _unlines(out, shape, axis)


def staggered_rhs(f, coefs, h, shift=0, axis=-1):
    """Staggered derivative RHS (App. A.2, first scheme), periodic:
    d_i = sum_k coefs[k-1] (f[i+k-1+shift] - f[i-k+shift]) / ((2k-1) h).
    shift = 0: f[j] sits at x_{j+1/2}, d_i at x_i; shift = 1: f[j] at x_j,
    d_i at x_{i+1/2}."""
    return _staggered(f, coefs, h, shift, 0, False, axis)


def midpoint_rhs(f, coefs, shift=0, axis=-1):
    """Compact interpolation RHS (Eq. 2; App. A.2, second scheme), periodic:
    d_i = sum_k coefs[k-1] (f[i+k-1+shift] + f[i-k+shift]) / 2 (points as in
    staggered_rhs)."""
    return _staggered(f, coefs, 1.0, shift, 1, False, axis)


def staggered_rhs_transpose(g, coefs, h, shift=0, axis=-1):
    """S^T g for the stencil of staggered_rhs (scatter form)."""
    return _staggered(g, coefs, h, shift, 0, True, axis)


def midpoint_rhs_transpose(g, coefs, shift=0, axis=-1):
    """S^T g for the stencil of midpoint_rhs (scatter form)."""
    return _staggered(g, coefs, 1.0, shift, 1, True, axis)


# ---------------------------------------------------------------- matrices
def toeplitz_bands(n, lhs):
    """Bands (2r+1, n) of the symmetric cyclic Toeplitz LHS with diagonal 1.

    lhs = (alpha,) gives B[alpha, 1, alpha] (Eq. 1 LHS); lhs = (alpha, beta)
    gives B[beta, alpha, 1, alpha, beta].
    """
    lhs = list(lhs)
    r = len(lhs)
    b = np.zeros((2 * r + 1, n))
    b[r] = 1.0
    for q in range(1, r + 1):
        b[r - q] = lhs[q - 1]
        b[r + q] = lhs[q - 1]
    return b


def block_tridiagonal_bands(npts, L, D, U):
    """Bands (2r+1, n) of a block-tridiagonal matrix with b x b blocks.

    Sec. 1 names block entries (compact schemes for shock capturing couple
    several unknowns per grid point).  A line of npts points with b unknowns
    each, point-major (unknown c of point m is row m b + c), where point m
    couples to points m-1, m, m+1 through L, D, U (the same for every point),
    is a banded matrix: row m b + c holds L[c][j] in column (m-1) b + j, D[c][j]
    in column m b + j and U[c][j] in column (m+1) b + j, i.e. at offsets
    j - c - b, j - c and j - c + b, so its half bandwidth is r = 2b - 1.
    Column indices wrap (cyclic); solve_acyclic drops the wrapped corners.
    """
    L, D, U = (np.asarray(a, dtype=np.float64) for a in (L, D, U))
    b = D.shape[0]
    r = 2 * b - 1
    n = npts * b
    bands = np.zeros((2 * r + 1, n))
    for m in range(npts):
        for c in range(b):
            i = m * b + c
            for j in range(b):
                bands[r + j - c - b, i] += L[c, j]
                bands[r + j - c, i] += D[c, j]
                bands[r + j - c + b, i] += U[c, j]
    return bands


def block_dense_matrix(npts, L, D, U, cyclic=True):
    """Dense (npts b) x (npts b) block-tridiagonal matrix, assembled block by
    block: block (m, m-1) = L, (m, m) = D, (m, m+1) = U; cyclic wraps the
    corner blocks (m = 0 gets L at the last point, the last point U at 0)."""
    L, D, U = (np.asarray(a, dtype=np.float64) for a in (L, D, U))
    b = D.shape[0]
    A = np.zeros((npts * b, npts * b))
    for m in range(npts):
        A[m * b:(m + 1) * b, m * b:(m + 1) * b] += D
        if m > 0 or cyclic:
            mm = (m - 1) % npts
            A[m * b:(m + 1) * b, mm * b:(mm + 1) * b] += L
        if m < npts - 1 or cyclic:
            mp = (m + 1) % npts
            A[m * b:(m + 1) * b, mp * b:(mp + 1) * b] += U
    return A


def variable_alpha_bands(alpha_lines):
    """Row-wise variable tridiagonal bands: A[i,i-1] = A[i,i+1] = alpha_i, A[i,i] = 1.

    alpha_lines: (lines, n).  Returns (lines, 3, n).
    """
    a = np.asarray(alpha_lines, dtype=np.float64)
    return np.stack([a, np.ones_like(a), a], axis=-2)


def transpose_bands(bands):
    """Bands of A^T from bands of A (any r): A^T[i, i+q] = A[i+q, i]."""
    bands = np.asarray(bands, dtype=np.float64)
    w = bands.shape[-2]
    r = (w - 1) // 2
    out = np.empty_like(bands)
    for k in range(w):
        q = k - r  # A^T[i, i+q] = A[i+q, i] lives on diagonal -q of row i+q
        out[..., k, :] = np.roll(bands[..., 2 * r - k, :], -q, axis=-1)
    return out


def dense_matrix(bands):
    """Dense n x n cyclic matrix from one band set (2r+1, n)."""
    bands = np.asarray(bands, dtype=np.float64)
    w, n = bands.shape
    r = (w - 1) // 2
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(w):
            A[i, (i + k - r) % n] += bands[k, i]
    return A


def dense_solve(A, b):
    """Gaussian elimination with partial pivoting (C), for tiny systems."""
    A = np.array(A, dtype=np.float64, order="C")
    x = np.array(b, dtype=np.float64, order="C")
    if _load().orc_dense_solve(_ptr(A), _ptr(x), A.shape[0]):
        raise ArithmeticError("singular dense system")
    return x


# ---------------------------------------------------------------- solves
def solve_cyclic(bands, d, axis=-1, method="auto"):
    """x = A^{-1} d along `axis`.

    bands: (2r+1, n) shared by all lines, or (..., 2r+1, n) with one band set
    per line (leading dims equal to those of d with `axis` moved last).
    method: "sm" (tridiagonal Thomas + Sherman-Morrison), "woodbury" (banded LU
    + rank-2r Woodbury) or "auto" (sm for r = 1).
    """
    d2, shape = _lines(d, axis)
    lines, n = d2.shape
    bands = np.asarray(bands, dtype=np.float64)
    w = bands.shape[-2]
    r = (w - 1) // 2
    if bands.ndim == 2:
        b2 = np.ascontiguousarray(bands)
        stride = 0
    else:
        b2 = np.ascontiguousarray(bands.reshape(lines, w, n))
        stride = w * n
    x = np.empty_like(d2)
    lib = _load()
    if method == "auto":
        method = "sm" if r == 1 else "woodbury"
    if method == "sm":
        assert r == 1
        rc = lib.orc_cyclic_tri(_ptr(b2), stride, _ptr(d2), _ptr(x), lines, n)
    else:
        if n < 4 * r:  # the capacitance form keeps the 2r corner rows apart
            raise ValueError("the banded Woodbury solve needs n >= 4r (n = %d, r = %d); use dense_solve" % (n, r))
        rc = lib.orc_cyclic_banded(_ptr(b2), stride, _ptr(d2), _ptr(x), lines, n, r)
    if rc:
        raise ArithmeticError("zero pivot in the oracle solve")
    return _unlines(x, shape, axis)


def solve_acyclic(bands, d, axis=-1):
    """x = B^{-1} d along `axis` for the acyclic (non-periodic) banded B: the
    band set of ``toeplitz_bands`` (or per line) without the wrapped corner
    entries.  Banded LU without pivoting (``cbs_oracle.c``)."""
    d2, shape = _lines(d, axis)
    lines, n = d2.shape
    bands = np.asarray(bands, dtype=np.float64)
    w = bands.shape[-2]
    r = (w - 1) // 2
    if bands.ndim == 2:
        b2, stride = np.ascontiguousarray(bands), 0
    else:
        b2, stride = np.ascontiguousarray(bands.reshape(lines, w, n)), w * n
    x = np.empty_like(d2)
    if _load().orc_acyclic_banded(_ptr(b2), stride, _ptr(d2), _ptr(x), lines, n, r):
        raise ArithmeticError("zero pivot in the oracle solve")
    return _unlines(x, shape, axis)


def acyclic_dense_matrix(bands):
    """Dense n x n acyclic matrix of one band set (no wrapped corners)."""
    bands = np.asarray(bands, dtype=np.float64)
    w, n = bands.shape
    r = (w - 1) // 2
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(w):
            j = i + k - r
            if 0 <= j < n:
                A[i, j] = bands[k, i]
    return A


def matvec(bands, x, axis=-1):
    """A x along `axis` (bands shared or per line, as in solve_cyclic)."""
    x2, shape = _lines(x, axis)
    lines, n = x2.shape
    bands = np.asarray(bands, dtype=np.float64)
    w = bands.shape[-2]
    r = (w - 1) // 2
    if bands.ndim == 2:
        b2, stride = np.ascontiguousarray(bands), 0
    else:
        b2, stride = np.ascontiguousarray(bands.reshape(lines, w, n)), w * n
    out = np.empty_like(x2)
    _load().orc_banded_matvec(_ptr(b2), stride, _ptr(x2), _ptr(out), lines, n, r)
    return _unlines(out, shape, axis)


def derivative(f, lhs, coefs, h, axis=-1):
    """Compact first derivative along `axis`: x = A^{-1} S f (Eq. 1)."""
    n = np.shape(f)[axis]
    return solve_cyclic(toeplitz_bands(n, lhs), central_rhs(f, coefs, h, axis), axis)


def closure_matrices(n, lhs, coefs, closure, h):
    """Dense (A_c, B_c) of the acyclic compact first derivative A_c x = B_c f.

    Interior rows c <= i < n - c follow Eq. 1: A_c[i, i] = 1, A_c[i, i +- q] =
    lhs[q-1], B_c[i, i +- q] = +- coefs[q-1] / (2 q h).  closure = (L, R), c x W
    arrays: row k < c reads sum_j L[k][j] x_j = sum_j R[k][j] f_j / h, and row
    n-1-k is its mirror image, sum_j L[k][j] x_{n-1-j} = -sum_j R[k][j]
    f_{n-1-j} / h (the derivative of f(-x) is -f'(-x))."""
    L, R = (np.asarray(a, dtype=np.float64) for a in closure)
    c, W = L.shape
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    for i in range(c, n - c):
        A[i, i] = 1.0
        for q, a in enumerate(lhs, start=1):
            A[i, i - q] = A[i, i + q] = a
        for q, cq in enumerate(coefs, start=1):
            B[i, i + q] += cq / (2 * q * h)
            B[i, i - q] -= cq / (2 * q * h)
    for k in range(c):
        for j in range(W):
            A[k, j] = L[k, j]
            B[k, j] = R[k, j] / h
            A[n - 1 - k, n - 1 - j] = L[k, j]
            B[n - 1 - k, n - 1 - j] = -R[k, j] / h
    return A, B


def derivative_closure(f, lhs, coefs, closure, h, axis=-1):
    """Acyclic compact first derivative with boundary closures along `axis`:
    x = A_c^{-1} (B_c f), A_c and B_c from closure_matrices (dense LAPACK solve)."""
    f2, shape = _lines(f, axis)
    A, B = closure_matrices(f2.shape[1], lhs, coefs, closure, h)
    x2 = np.linalg.solve(A, B @ f2.T).T
    return _unlines(np.ascontiguousarray(x2), shape, axis)


def staggered_derivative(f, lhs, coefs, h, shift=0, axis=-1):
    """Staggered compact first derivative: x = A^{-1} S f with S of staggered_rhs."""
    n = np.shape(f)[axis]
    return solve_cyclic(toeplitz_bands(n, lhs), staggered_rhs(f, coefs, h, shift, axis), axis)


def midpoint_interpolation(f, lhs, coefs, shift=0, axis=-1):
    """Compact interpolation to the half-shifted grid: x = A^{-1} S f with S of midpoint_rhs."""
    n = np.shape(f)[axis]
    return solve_cyclic(toeplitz_bands(n, lhs), midpoint_rhs(f, coefs, shift, axis), axis)


def derivative_variable_tri(f, alpha, coefs, h, axis=-1):
    """x = A(alpha)^{-1} S f with row-wise alpha (same shape as f)."""
    a2, shape = _lines(alpha, axis)
    d2, _ = _lines(central_rhs(f, coefs, h, axis), axis)
    x2 = solve_cyclic(variable_alpha_bands(a2), d2, axis=-1)
    return _unlines(x2, shape, axis)


def adjoint_variable_tri(f, alpha, g, coefs, h, axis=-1):
    """Gradients of L = sum(g * x) for x = A(alpha)^{-1} S f.

    Returns (grad_f, grad_alpha, lam, x) with lam = A^{-T} g,
    grad_f = S^T lam and grad_alpha_i = -lam_i (x_{i-1} + x_{i+1}).
    """
    a2, shape = _lines(alpha, axis)
    g2, _ = _lines(g, axis)
    f2, _ = _lines(f, axis)
    bands = variable_alpha_bands(a2)
    d2 = central_rhs(f2, coefs, h, -1)
    x2 = solve_cyclic(bands, d2, -1)
    lam2 = solve_cyclic(transpose_bands(bands), g2, -1)
    gf2 = central_rhs_transpose(lam2, coefs, h, -1)
    ga2 = -lam2 * (np.roll(x2, 1, axis=-1) + np.roll(x2, -1, axis=-1))
    return (_unlines(gf2, shape, axis), _unlines(ga2, shape, axis),
            _unlines(lam2, shape, axis), _unlines(x2, shape, axis))


# ---------------------------------------------------------------- interface system
def partition_bounds(n, p, unit=1):
    """Partition starts/sizes: the first (n/unit) mod p partitions get
    ceil(n/(unit p)) units of `unit` rows (unit = b: whole points of a
    block-entry line)."""
    base, extra = divmod(n // unit, p)
    sizes = [unit * (base + (1 if i < extra else 0)) for i in range(p)]
    starts = np.cumsum([0] + sizes[:-1]).tolist()
    return starts, sizes


def reduced_system_dense(bands, p, unit=1):
    """Interface system A-hat of Sec. 3 as a dense Schur complement.

    The interface unknowns are the first r rows of each partition (Fig. 3);
    the permutation P moves every bulk block D_i first and every interface
    block last (Fig. 4), and block Gaussian elimination leaves
    A-hat = A_II - A_IB A_BB^{-1} A_BI as the trailing block.  Returns the
    (p r) x (p r) matrix and the index lists (interface, bulk).
    """
    A = dense_matrix(bands)
    n = A.shape[0]
    r = (bands.shape[0] - 1) // 2
    starts, sizes = partition_bounds(n, p, unit)
    iface = [s + q for s in starts for q in range(r)]
    bulk = [j for j in range(n) if j not in set(iface)]
    A_II = A[np.ix_(iface, iface)]
    A_IB = A[np.ix_(iface, bulk)]
    A_BI = A[np.ix_(bulk, iface)]
    A_BB = A[np.ix_(bulk, bulk)]
    Ahat = A_II - A_IB @ np.linalg.solve(A_BB, A_BI)
    return Ahat, iface, bulk


# ---------------------------------------------------------------- errors
def rel_err(x, ref):
    """Norm-wise infinity relative error ||x - ref||_inf / ||ref||_inf."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(x - ref)) / (den if den > 0 else 1.0))
