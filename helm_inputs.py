"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

This module holds workload *parameters* and seeded random draws only. It
contains none of the method's arithmetic (no assembly, no operator, no
solver step), so that the oracle and the CUDA path can both read it without
sharing any computation.

Workloads follow the paper's setting (Helmholtz with impedance boundary on
the unit square/cube, Sec. 2) with the discretisations and sizes of the
synthetic test problems used throughout this repository.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

FP64 = 0
MIXED = 1


@dataclass(frozen=True)
class Workload:
    """One Helmholtz solve: -Lap u - k^2 u = f, du/dn - iku = g (Sec. 2, eq. Helmholtz).

    n      : elements per side of the fine mesh (h = 1/n); must be even.
    order  : Lagrange order (1 = P1, 2 = P2) on right triangles / Kuhn tets.
    shift  : the imaginary shift epsilon of the preconditioner operator
             (eq. Helmholtz_shift), i.e. k^2 -> k^2 + i*epsilon.
    rhs    : 'planewave' (f=0, impedance data of exp(ik d.x), d=(cos t, sin t)),
             'gaussian'  (f = exp(-|x-x0|^2/(2 s^2)), s = 2h, x0 = centre, g = 0),
             'random'    (the load vector F itself, N(0,1) + i N(0,1), seeded).
    """
    name: str
    dim: int
    order: int
    n: int
    k: float
    shift: float
    rhs: str
    theta: float = 0.3
    seed: int = 0
    restart: int = 50
    maxit: int = 500
    tol: float = 1e-8
    omega: float = 0.6
    nu: int = 2

    @property
    def h(self) -> float:
        return 1.0 / self.n

    @property
    def dofs_per_side(self) -> int:
        return self.order * self.n + 1

    @property
    def num_dofs(self) -> int:
        return self.dofs_per_side ** self.dim

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def half_k2(k: float) -> float:
    return 0.5 * k * k


# Plain FP64 method, small: 2D P1, h=1/64, k=20, plane wave, restart 50.
SMALL_P1 = Workload("p1_n64_k20_planewave", 2, 1, 64, 20.0, half_k2(20.0), "planewave",
                    restart=50)
# 2D P1, k=200, h=1/512, Gaussian point source, restart 80 (mixed vs FP64).
GAUSS_P1 = Workload("p1_n512_k200_gaussian", 2, 1, 512, 200.0, half_k2(200.0), "gaussian",
                    restart=80)
# 2D P2, k=150, h=1/256, random complex load vector (seed 3).
RANDOM_P2 = Workload("p2_n256_k150_random", 2, 2, 256, 150.0, half_k2(150.0), "random",
                     seed=3, restart=80)
# 3D P1 (Kuhn tetrahedra), k=40, h=1/96, random complex load vector (seed 3).
RANDOM_P1_3D = Workload("p1_3d_n96_k40_random", 3, 1, 96, 40.0, half_k2(40.0), "random",
                        seed=3, restart=80)


def random_load(num_dofs: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) real and imaginary parts, lexicographic DoF order.

    Real parts are drawn first, then imaginary parts, from PCG64(seed).
    """
    g = np.random.Generator(np.random.PCG64(seed))
    re = g.standard_normal(num_dofs)
    im = g.standard_normal(num_dofs)
    return re + 1j * im


def uniform_loads(sizes, seed: int = 0):
    """Load vectors with entries uniform in [-1, 1] (real), one per size, drawn in order from
    PCG64(seed): the right-hand sides of the shift search's sample solves (Sec. 5, data
    generation: f ~ U[-1, 1], g = 0; the draw is taken as the load vector itself)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.uniform(-1.0, 1.0, n).astype(np.complex128) for n in sizes]


def shift_sweep(seed: int = 4, n_pairs: int = 32, n_shifts: int = 16,
                n_min: int = 32, n_max: int = 1024):
    """Batched shift-sample sweep: (k, kh) pairs times a log grid of shifts.

    k ~ U[10, 300], kh ~ U[0.3, 0.8]; n = nearest even integer to k/kh,
    clamped to [n_min, n_max]; shifts on a log grid in [0.05 k^2, 2 k^2].
    Returns a list of Workloads (P1, plane wave, restart 50, cap 500).
    """
    g = np.random.Generator(np.random.PCG64(seed))
    ks = g.uniform(10.0, 300.0, n_pairs)
    khs = g.uniform(0.3, 0.8, n_pairs)
    out = []
    for i in range(n_pairs):
        k = float(ks[i])
        n = int(2 * round(k / khs[i] / 2.0))
        n = min(max(n, n_min), n_max)
        for s in np.geomspace(0.05 * k * k, 2.0 * k * k, n_shifts):
            out.append(Workload(f"sweep_{i}_{len(out)}", 2, 1, n, k, float(s), "planewave",
                                restart=50, maxit=500))
    return out


def poisson_arrivals(seed: int = 5, rate: float = 200.0, count: int = 2000):
    """Arrival times (s) of a Poisson process with the given mean rate."""
    g = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(g.exponential(1.0 / rate, count))


def serving_requests(seed: int = 5, count: int = 2000,
                     grids=(128, 256, 512, 1024), k_range=(20.0, 400.0)):
    """Request parameters of the serving trace: order, n, k (shift chosen by the caller)."""
    g = np.random.Generator(np.random.PCG64(seed + 1000))
    orders = g.integers(1, 3, count)
    ns = g.choice(np.asarray(grids), count)
    ks = g.uniform(k_range[0], k_range[1], count)
    return [(int(orders[i]), int(ns[i]), float(ks[i]), seed + i) for i in range(count)]


# Heterogeneous wavenumber k(x) = k_max * mu(x) with a scaled profile mu: Omega -> [0, 1]
# (Sec. 6). The paper's profiles (wedge, geological cross-sections) are not available; these
# synthetic profiles stand in for them.
WEDGE_VALUES = (1.0, 0.7, 0.45)    # mu above, inside and below the wedge


def wedge_profile(x: np.ndarray) -> np.ndarray:
    """Three-valued wedge: a layer between the lines y = 0.62 + 0.18 (x - 0.5) and
    y = 0.38 - 0.12 (x - 0.5), which close towards x = 0 less than towards x = 1, splits the
    square into an upper, a wedge and a lower region. x: (P, d) points; returns mu (P,)."""
    x = np.asarray(x, dtype=float)
    top = 0.62 + 0.18 * (x[:, 0] - 0.5)
    bot = 0.38 - 0.12 * (x[:, 0] - 0.5)
    y = x[:, 1]
    return np.where(y > top, WEDGE_VALUES[0], np.where(y >= bot, WEDGE_VALUES[1], WEDGE_VALUES[2]))


def cell_profile(x: np.ndarray, cells: int, seed: int) -> np.ndarray:
    """Piecewise-constant mu on a cells^d grid of squares/cubes, values U[0.4, 1] from
    PCG64(seed) in lexicographic cell order (x fastest). x: (P, d) points inside the cells."""
    x = np.asarray(x, dtype=float)
    d = x.shape[1]
    vals = np.random.Generator(np.random.PCG64(seed)).uniform(0.4, 1.0, cells ** d)
    idx = np.minimum((x * cells).astype(np.int64), cells - 1)
    lin = np.zeros(x.shape[0], dtype=np.int64)
    for ax in reversed(range(d)):
        lin = lin * cells + idx[:, ax]
    return vals[lin]
