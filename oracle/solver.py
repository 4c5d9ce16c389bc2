"""Twogrid V-cycle (Algorithm 1) and flexible GMRES (Sec. 4) for the oracle.

TEST INFRASTRUCTURE (see oracle/__init__.py). Plain FP64 (complex128).

Readings of the paper used here (where it is silent or differs from the
workloads; each is listed in the design notes):
  * Smoother: damped Jacobi with D = diag(A_eps) including the boundary term;
    u^0 = 0; post-smoothing uses the same Jacobi sweep (Jacobi is symmetric,
    so S^{-T} of Algorithm 1 changes nothing).
  * Restriction is the plain transpose P^T of the canonical interpolation P
    (Algorithm 1); the coarse matrix is the rediscretisation on the 2h mesh.
  * Coarse solve: a sparse direct LU (library primitive) of the assembled
    coarse matrix, factored once per (k, h, shift) and reused (Sec. 6).
  * FGMRES: x0 = 0, modified Gram-Schmidt, complex Givens rotations, Hermitian
    inner product; a cycle stops when the Givens residual estimate satisfies
    |g_{j+1}| <= tol ||F||; then x is updated and the TRUE residual
    ||F - A0 x|| / ||F|| is checked; a new cycle starts if it is still above
    tol and the iteration cap is not reached. The iteration count is the total
    number of Arnoldi steps (= preconditioner applications).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


def jacobi_sweeps(A, dinv, f, u, omega, nu):
    """nu damped-Jacobi steps u <- u + omega D^{-1} (f - A u) (Algorithm 1, smoothing lines)."""
    for _ in range(nu):
        u = u + omega * dinv * (f - A @ u)
    return u


@dataclass
class TwoGrid:
    """One V(nu, nu)-cycle on A_eps with two levels (Algorithm 1, L = 2)."""
    A_fine: sp.csr_matrix          # A(k, eps) on V_h
    A_coarse: sp.csr_matrix        # A(k, eps) on V_2h (rediscretised)
    P: sp.csr_matrix               # canonical interpolation V_2h -> V_h
    omega: float = 0.6
    nu: int = 2
    coarse_solver: str = "splu"    # 'splu' | 'dense'
    _lu: object = field(default=None, repr=False)
    _dinv: np.ndarray = field(default=None, repr=False)
    _R: sp.csr_matrix = field(default=None, repr=False)

    def __post_init__(self):
        self._dinv = 1.0 / self.A_fine.diagonal()
        self._R = self.P.T.tocsr()
        if self.coarse_solver == "dense":
            self._lu = ("dense", self.A_coarse.toarray())
        else:
            self._lu = ("splu", spla.splu(self.A_coarse.tocsc()))

    def coarse_solve(self, r):
        kind, obj = self._lu
        if kind == "dense":
            return np.linalg.solve(obj, r)
        return obj.solve(r)

    def apply(self, f):
        """u = V-cycle(0, f): presmooth, restrict residual, coarse solve, prolongate, postsmooth."""
        u = np.zeros_like(f)
        u = jacobi_sweeps(self.A_fine, self._dinv, f, u, self.omega, self.nu)
        r_c = self._R @ (f - self.A_fine @ u)
        u_c = self.coarse_solve(r_c)
        u = u + self.P @ u_c
        u = jacobi_sweeps(self.A_fine, self._dinv, f, u, self.omega, self.nu)
        return u


def givens(a, b):
    """Complex Givens rotation (c real, s complex) with [c s; -conj(s) c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0:
        return 0.0, 1.0 + 0.0j, b
    nu = math.hypot(abs(a), abs(b))
    ph = a / abs(a)
    c = abs(a) / nu
    s = ph * np.conj(b) / nu
    return c, s, ph * nu


@dataclass
class FGMRESResult:
    x: np.ndarray
    iters: int
    relres_true: float
    history: list            # Givens residual estimates |g_{j+1}| / ||F|| per iteration
    cycle_true: list         # true relative residual at the end of each cycle
    breakdown: bool = False


def fgmres(A0, F, precond, restart=50, tol=1e-8, maxit=500, record_basis=False):
    """Right-preconditioned flexible GMRES(m) (Saad 1993), x0 = 0.

    Solves A0 P^{-1} (P u) = F with a preconditioner that may change per step
    (Sec. 4). Returns FGMRESResult; with record_basis the last cycle's V, Z and
    Hbar are attached for the Arnoldi-relation pin.
    """
    F = np.asarray(F, dtype=np.complex128)
    nF = np.linalg.norm(F)
    x = np.zeros_like(F)
    if nF == 0.0:
        return FGMRESResult(x, 0, 0.0, [], [0.0])
    total = 0
    history, cycle_true = [], []
    r = F.copy()
    beta = nF
    breakdown = False
    last = None
    while True:
        m = restart
        V = np.zeros((m + 1, F.size), dtype=np.complex128)
        Z = np.zeros((m, F.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        Hraw = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = A0 @ Z[j]
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            Hraw[:, j] = H[:, j]
            happy = H[j + 1, j].real <= 1e-14 * beta
            if not happy:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                          # previous rotations
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            c, s, rr = givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j], H[j + 1, j] = rr, 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            total += 1
            j_end = j + 1
            history.append(abs(g[j + 1]) / nF)
            if happy:
                breakdown = True
                break
            if abs(g[j + 1]) <= tol * nF or total >= maxit:
                break
        y = np.zeros(j_end, dtype=np.complex128)
        for i in range(j_end - 1, -1, -1):             # back substitution
            y[i] = (g[i] - H[i, i + 1:j_end] @ y[i + 1:]) / H[i, i]
        x = x + y @ Z[:j_end]
        r = F - A0 @ x
        rel = np.linalg.norm(r) / nF
        cycle_true.append(rel)
        if record_basis:
            last = (V[:j_end + 1].copy(), Z[:j_end].copy(), Hraw[:j_end + 1, :j_end].copy())
        if rel <= tol or total >= maxit or breakdown:
            break
        beta = np.linalg.norm(r)
    res = FGMRESResult(x, total, rel, history, cycle_true, breakdown)
    if record_basis:
        res.basis = last
    return res


# ----------------------------------------------------------------------------
# One complete problem: mesh, operators, load vector, preconditioner
# ----------------------------------------------------------------------------


@dataclass
class Problem:
    """Assembled FP64 problem for a workload (see helm_inputs.Workload)."""
    wl: object
    mesh: fem.Mesh
    cmesh: fem.Mesh
    K: sp.csr_matrix
    M: sp.csr_matrix
    B: sp.csr_matrix
    A0: sp.csr_matrix
    Aeps: sp.csr_matrix
    Aeps_c: sp.csr_matrix
    P: sp.csr_matrix
    F: np.ndarray

    def twogrid(self, coarse_solver="splu"):
        return TwoGrid(self.Aeps, self.Aeps_c, self.P, self.wl.omega, self.wl.nu, coarse_solver)

    def solve(self, coarse_solver="splu", record_basis=False):
        tg = self.twogrid(coarse_solver)
        return fgmres(self.A0, self.F, tg.apply, self.wl.restart, self.wl.tol, self.wl.maxit,
                      record_basis=record_basis)


def load_vector(wl, mesh, M):
    """Load vector F of the workload's right-hand side kind."""
    if wl.rhs == "planewave":
        return fem.load_planewave(mesh, M, wl.k, wl.theta)
    if wl.rhs == "gaussian":
        return fem.load_gaussian(mesh, M, 2.0 * mesh.h)
    if wl.rhs == "random":
        import helm_inputs
        return helm_inputs.random_load(mesh.num_dofs, wl.seed)
    raise ValueError(wl.rhs)


def build_problem(wl):
    mesh = fem.build_mesh(wl.dim, wl.order, wl.n)
    cmesh = fem.build_mesh(wl.dim, wl.order, wl.n // 2)
    K, M, B = fem.assemble(mesh)
    Kc, Mc, Bc = fem.assemble(cmesh)
    A0 = fem.system_matrix(K, M, B, wl.k, 0.0)
    Aeps = fem.system_matrix(K, M, B, wl.k, wl.shift)
    Aeps_c = fem.system_matrix(Kc, Mc, Bc, wl.k, wl.shift)
    P = fem.prolongation(cmesh, mesh)
    F = load_vector(wl, mesh, M)
    return Problem(wl, mesh, cmesh, K, M, B, A0, Aeps, Aeps_c, P, F)


def build_problem_het(wl, mu, source=None):
    """Problem with the heterogeneous wavenumber k(x) = wl.k * mu(x) (Sec. 6): wl.k is k_max,
    mu maps (P, dim) points to [0, 1] and is taken at each simplex's centroid, on the fine mesh
    and again on the coarse mesh (the coarse operator is rediscretised, Sec. 4). The shift
    wl.shift is one real number for the whole domain (eq. Helmholtz_shift). The load is the
    paper's source f = 2 exp(-1000 |x - s|^2), g = 0 (Sec. 6), s = source (default: centre)."""
    mesh = fem.build_mesh(wl.dim, wl.order, wl.n)
    cmesh = fem.build_mesh(wl.dim, wl.order, wl.n // 2)
    K, Mk, M, B, Bk = fem.assemble_weighted(mesh, wl.k * mu(fem.element_centroids(mesh)))
    Kc, Mkc, Mc, _, Bkc = fem.assemble_weighted(cmesh, wl.k * mu(fem.element_centroids(cmesh)))
    A0 = fem.system_matrix_het(K, Mk, M, Bk, 0.0)
    Aeps = fem.system_matrix_het(K, Mk, M, Bk, wl.shift)
    Aeps_c = fem.system_matrix_het(Kc, Mkc, Mc, Bkc, wl.shift)
    P = fem.prolongation(cmesh, mesh)
    s = np.full(wl.dim, 0.5) if source is None else np.asarray(source, dtype=float)
    f = 2.0 * np.exp(-1000.0 * np.sum((mesh.coords - s) ** 2, axis=1))
    F = fem.load_from_nodal(mesh, M, f)
    return Problem(wl, mesh, cmesh, K, M, B, A0, Aeps, Aeps_c, P, F)


def build_problem_q(wl, mu=None, source=None):
    """Problem on tensor-product Q_p elements (p = wl.order in 1..3, Sec. 2), optionally with the
    heterogeneous wavenumber k(x) = wl.k * mu(x) taken at the element centres (Sec. 6). Loads:
    'planewave' (impedance data of exp(i k d.x); constant k only), 'source' (the paper's
    f = 2 exp(-1000 |x - s|^2), g = 0, s = source or the centre), 'random' (seeded F)."""
    from . import qfem
    mesh = qfem.build_mesh(wl.dim, wl.order, wl.n)
    cmesh = qfem.build_mesh(wl.dim, wl.order, wl.n // 2)
    kf = None if mu is None else wl.k * mu(mesh.centres)
    kc = None if mu is None else wl.k * mu(cmesh.centres)
    K, Mk, M, B, Bk = qfem.assemble(mesh, kf)
    Kc, Mkc, Mc, Bc, Bkc = qfem.assemble(cmesh, kc)
    if mu is None:
        A0 = fem.system_matrix(K, M, B, wl.k, 0.0)
        Aeps = fem.system_matrix(K, M, B, wl.k, wl.shift)
        Aeps_c = fem.system_matrix(Kc, Mc, Bc, wl.k, wl.shift)
    else:
        A0 = fem.system_matrix_het(K, Mk, M, Bk, 0.0)
        Aeps = fem.system_matrix_het(K, Mk, M, Bk, wl.shift)
        Aeps_c = fem.system_matrix_het(Kc, Mkc, Mc, Bkc, wl.shift)
    P = qfem.prolongation(cmesh, mesh)
    if wl.rhs == "planewave":
        assert mu is None
        F = qfem.load_planewave(mesh, M, wl.k, wl.theta)
    elif wl.rhs == "source":
        F = qfem.load_source(mesh, M, np.full(wl.dim, 0.5) if source is None else source)
    elif wl.rhs == "random":
        import helm_inputs
        F = helm_inputs.random_load(mesh.num_dofs, wl.seed)
    else:
        raise ValueError(wl.rhs)
    return Problem(wl, mesh, cmesh, K, M, B, A0, Aeps, Aeps_c, P, F)


# ----------------------------------------------------------------------------
# Sec. 5, data generation: the optimal shift exponent of one problem by a golden-section
# search over sigma in [1, 2] (eps = k^sigma), objective the average convergence rate.
# ----------------------------------------------------------------------------


def shift_rate(k, n, order, sigma, F, maxit=50, omega=0.6, nu=2, dim=2):
    """rho = (r_end / r_0)^(1/end) of FGMRES without restart, stopped at relative residual
    1e-8 or after maxit iterations, right-preconditioned by the twogrid cycle on the shift
    eps = k^sigma; x0 = 0, so r_0 = ||F||, and r_end is the true residual (Sec. 5)."""
    mesh = fem.build_mesh(dim, order, n)
    cmesh = fem.build_mesh(dim, order, n // 2)
    K, M, B = fem.assemble(mesh)
    Kc, Mc, Bc = fem.assemble(cmesh)
    eps = k ** sigma
    tg = TwoGrid(fem.system_matrix(K, M, B, k, eps), fem.system_matrix(Kc, Mc, Bc, k, eps),
                 fem.prolongation(cmesh, mesh), omega, nu)
    r = fgmres(fem.system_matrix(K, M, B, k, 0.0), F, tg.apply, restart=maxit, tol=1e-8, maxit=maxit)
    return r.relres_true ** (1.0 / r.iters) if r.relres_true > 0 else 0.0


def golden_section_min(f, lo, hi, tol):
    """Minimum of a unimodal f on [lo, hi] by golden-section search (Kiefer 1953): the two
    interior points divide the bracket in the golden ratio, the bracket keeps the side of the
    smaller value and reuses the other point, until it is narrower than tol. Returns
    (x, f(x), evaluations) for the better of the two last interior points."""
    r = (math.sqrt(5.0) - 1.0) / 2.0          # 1 / golden ratio
    a, b = lo, hi
    x1, x2 = b - r * (b - a), a + r * (b - a)
    f1, f2 = f(x1), f(x2)
    count = 2
    while b - a > tol:
        if f1 < f2:                            # the minimum lies in [a, x2]
            b, x2, f2 = x2, x1, f1
            x1 = b - r * (b - a)
            f1 = f(x1)
        else:                                  # the minimum lies in [x1, b]
            a, x1, f1 = x1, x2, f2
            x2 = a + r * (b - a)
            f2 = f(x2)
        count += 1
    return (x1, f1, count) if f1 < f2 else (x2, f2, count)


def optimal_shift_exponent(k, n, order, F, tol=1e-2, maxit=50):
    """sigma_hat = argmin over [1, 2] of shift_rate (golden-section search to tol)."""
    return golden_section_min(lambda s: shift_rate(k, n, order, s, F, maxit), 1.0, 2.0, tol)
