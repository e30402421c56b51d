"""Seeded synthetic inputs for the solver and its oracle (no method arithmetic).

These generators are the only code shared by the GPU path and the CPU oracle:
they produce fields, right-hand sides and operator coefficients, never a
stencil, a solve or an expected value.  All randomness comes from numpy's
PCG64 ``default_rng(seed)``.

Operators (inputs to both sides):
  * LELE6_TRI   -- 6th-order compact first derivative, paper Eq. 1 with
                   alpha = 1/3 (the LHS the paper benchmarks, Sec. 5),
                   a = 14/9, b = 1/9.
  * PENTA10     -- pentadiagonal (beta, alpha) = (1/20, 1/2) with the
                   10th-order right-hand side a = 17/12, b = 101/150, c = 1/100.
  * HEPTA12     -- heptadiagonal (alpha, beta, gamma) = (9/16, 9/100, 1/400)
                   with a = 21/16, b = 231/250, c = 147/2000: the
                   12th-order member of the generalised bands of Sec. 2
                   (w = 7), every coefficient fixed by Taylor matching.
  * CLOSURE3_4  -- one-sided boundary rows for acyclic derivatives (rows
                   k = 0, 1: the third-order one-sided row
                   x_0 + 2 x_1 = (-5/2 f_0 + 2 f_1 + 1/2 f_2) / h and the
                   fourth-order tridiagonal row (1/4, 1, 1/4) with
                   3/4 (f_2 - f_0) / h); CLOSURE3_4_6 adds row 2, the
                   sixth-order tridiagonal scheme, for the pentadiagonal
                   interior.  (L, R): LHS and RHS coefficients per row.
  * CENTRAL4    -- explicit 4th-order central difference (alpha = 0):
                   a = 4/3, b = -1/3 in Lele's form.
  * STAGGERED6  -- 6th-order staggered first derivative (App. A.2):
                   alpha = 9/62, a = 63/62, b = 17/62.
  * MIDPOINT6   -- 6th-order compact midpoint interpolation (Eq. 2, App. A.2):
                   alpha = 3/10, a = 3/2, b = 1/10.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LELE6_TRI = {"lhs": (1.0 / 3.0,), "rhs": (14.0 / 9.0, 1.0 / 9.0)}
PENTA10 = {"lhs": (1.0 / 2.0, 1.0 / 20.0), "rhs": (17.0 / 12.0, 101.0 / 150.0, 1.0 / 100.0)}
HEPTA12 = {"lhs": (9.0 / 16.0, 9.0 / 100.0, 1.0 / 400.0), "rhs": (21.0 / 16.0, 231.0 / 250.0, 147.0 / 2000.0)}
CENTRAL4 = {"rhs": (4.0 / 3.0, -1.0 / 3.0)}
CLOSURE3_4 = ([[1.0, 2.0, 0.0], [0.25, 1.0, 0.25]],
              [[-2.5, 2.0, 0.5], [-0.75, 0.0, 0.75]])
CLOSURE3_4_6 = ([[1.0, 2.0, 0.0, 0.0, 0.0], [0.25, 1.0, 0.25, 0.0, 0.0], [0.0, 1.0 / 3.0, 1.0, 1.0 / 3.0, 0.0]],
                [[-2.5, 2.0, 0.5, 0.0, 0.0], [-0.75, 0.0, 0.75, 0.0, 0.0],
                 [-1.0 / 36.0, -7.0 / 9.0, 0.0, 7.0 / 9.0, 1.0 / 36.0]])
STAGGERED6 = {"lhs": (9.0 / 62.0,), "rhs": (63.0 / 62.0, 17.0 / 62.0)}
MIDPOINT6 = {"lhs": (3.0 / 10.0,), "rhs": (3.0 / 2.0, 1.0 / 10.0)}

SEEDS = {"fourier64": 0, "cube512": 1, "penta_long": 2, "ragged_batch": 3, "variable_alpha": 4}


def grid_spacing(n: int) -> float:
    """Periodic grid on [0, 2 pi): h = 2 pi / n, x_j = j h."""
    return 2.0 * math.pi / n


@dataclass
class Modes:
    """Plane waves f = sum_m amp_m sin(kx_m x + ky_m y + kz_m z)."""
    k: np.ndarray        # (M, 3) integer wavenumbers (kx, ky, kz)
    amp: np.ndarray      # (M,)


def random_modes(rng: np.random.Generator, count: int, kmax: int = 20) -> Modes:
    k = rng.integers(1, kmax + 1, size=(count, 3))
    amp = rng.uniform(-1.0, 1.0, size=count)
    return Modes(k=k, amp=amp)


def plane_waves(shape_zyx, modes: Modes) -> np.ndarray:
    """Evaluate the modes on the periodic grid; array index order (z, y, x)."""
    nz, ny, nx = shape_zyx
    x = np.arange(nx) * grid_spacing(nx)
    y = np.arange(ny) * grid_spacing(ny)
    z = np.arange(nz) * grid_spacing(nz)
    f = np.zeros(shape_zyx)
    for (kx, ky, kz), a in zip(modes.k, modes.amp):
        f += a * np.sin(kx * x[None, None, :] + ky * y[None, :, None] + kz * z[:, None, None])
    return f


def fourier_cube(n: int = 64, count: int = 8, seed: int = SEEDS["fourier64"]):
    """n^3 field that is a sum of `count` seeded plane waves (wavenumbers 1..20)."""
    rng = np.random.default_rng(seed)
    modes = random_modes(rng, count)
    return plane_waves((n, n, n), modes), modes


def noisy_cube(n: int = 512, seed: int = SEEDS["cube512"], with_mode: bool = True):
    """n^3 field, i.i.d. U(-1, 1) plus one seeded plane wave; returns (f, modes)."""
    rng = np.random.default_rng(seed)
    modes = random_modes(rng, 1)
    f = rng.uniform(-1.0, 1.0, size=(n, n, n))
    if with_mode:
        f += plane_waves((n, n, n), modes)
    return f, modes


def mode_only_cube(n: int, modes: Modes) -> np.ndarray:
    return plane_waves((n, n, n), modes)


def long_lines(lines: int = 32, n: int = 1 << 22, seed: int = SEEDS["penta_long"]) -> np.ndarray:
    """Right-hand sides d ~ N(0, 1) drawn in FP64 and stored as FP32, shape (lines, n)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(lines, n)).astype(np.float32)


def variable_alpha_cube(n: int = 256, seed: int = SEEDS["variable_alpha"]):
    """(f, alpha): f ~ U(-1, 1), alpha ~ U(0.2, 0.4) per point, both (n, n, n)."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1.0, 1.0, size=(n, n, n))
    alpha = rng.uniform(0.2, 0.4, size=(n, n, n))
    return f, alpha


@dataclass
class BatchItem:
    shape_zyx: tuple
    direction: int           # 0 = x, 1 = y, 2 = z
    scheme: str              # "tri6" or "penta10"
    precision: str           # "fp64" or "fp32_refine"
    f: np.ndarray = field(repr=False, default=None)


RAGGED_SIZES = (32, 48, 64, 96, 128, 192, 256, 384)


def ragged_batch(count: int = 48, seed: int = SEEDS["ragged_batch"], sizes=RAGGED_SIZES,
                 with_fields: bool = True) -> list[BatchItem]:
    """Ragged set of periodic grids: per-axis sizes, direction, scheme and
    precision drawn by seed; fields U(-1, 1)."""
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(count):
        nx, ny, nz = (int(s) for s in rng.choice(sizes, size=3))
        direction = int(rng.integers(0, 3))
        scheme = "tri6" if rng.integers(0, 2) == 0 else "penta10"
        precision = "fp64" if rng.integers(0, 2) == 0 else "fp32_refine"
        items.append(BatchItem((nz, ny, nx), direction, scheme, precision))
    if with_fields:
        for it in items:
            it.f = rng.uniform(-1.0, 1.0, size=it.shape_zyx)
    return items
