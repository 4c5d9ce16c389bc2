"""Pins for the oracle's smoother, twogrid cycle and FGMRES (Sec. 4). CPU only.

Pins: closed forms of the Jacobi and twogrid error propagation written as
dense operators, the exact-preconditioner special case (one iteration), GMRES
minimality against brute-force least squares over an explicit Krylov basis,
the Arnoldi relation, orthonormality, monotone residuals, agreement with a
dense direct solve, and the fitted shift map's printed weights.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import helm_inputs as hi
from oracle import fem, shiftmap, solver

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny(order=1, n=8, k=6.0, shift=18.0, dim=2, rhs="planewave"):
    wl = hi.Workload("tiny", dim, order, n, k, shift, rhs, restart=30, seed=11)
    return solver.build_problem(wl)


def test_jacobi_closed_form():
    """nu damped-Jacobi steps from 0 give u = (I - S^nu) A^{-1} f, S = I - w D^{-1} A."""
    pb = _tiny()
    A = pb.Aeps.toarray()
    f = pb.F
    D = np.diag(np.diag(A))
    S = np.eye(A.shape[0]) - 0.6 * np.linalg.solve(D, A)
    for nu in (1, 2, 3):
        u = solver.jacobi_sweeps(pb.Aeps, 1.0 / np.diag(A), f, np.zeros_like(f), 0.6, nu)
        ref = (np.eye(A.shape[0]) - np.linalg.matrix_power(S, nu)) @ np.linalg.solve(A, f)
        np.testing.assert_allclose(u, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("order,dim", [(1, 2), (2, 2), (1, 3)])
def test_twogrid_error_propagation_closed_form(order, dim):
    """V-cycle(0, f) = (I - T) A^{-1} f with T = S^nu (I - P Ac^{-1} P^T A) S^nu (Sec. 3, T_h^2h)."""
    pb = _tiny(order=order, n=4 if dim == 3 else 8, dim=dim)
    tg = pb.twogrid("dense")
    A = pb.Aeps.toarray()
    Ac = pb.Aeps_c.toarray()
    P = pb.P.toarray()
    N = A.shape[0]
    S = np.eye(N) - tg.omega * np.diag(1.0 / np.diag(A)) @ A
    Snu = np.linalg.matrix_power(S, tg.nu)
    CGC = np.eye(N) - P @ np.linalg.solve(Ac, P.T @ A)
    T = Snu @ CGC @ Snu
    f = pb.F
    ref = (np.eye(N) - T) @ np.linalg.solve(A, f)
    np.testing.assert_allclose(tg.apply(f), ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_coarse_splu_matches_dense():
    pb = _tiny(n=16)
    r = np.random.default_rng(1).standard_normal(pb.Aeps_c.shape[0]) + 0j
    a = pb.twogrid("splu").coarse_solve(r)
    b = np.linalg.solve(pb.Aeps_c.toarray(), r)
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-13)


def test_givens_rotation():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        c, s, r = solver.givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        np.testing.assert_allclose(G @ G.conj().T, np.eye(2), atol=1e-14)
        np.testing.assert_allclose(G @ np.array([a, b]), [r, 0], atol=1e-14)


def test_fgmres_exact_preconditioner_one_iteration():
    pb = _tiny()
    tg = solver.TwoGrid(pb.A0, pb.A0, sp.identity(pb.A0.shape[0], format="csr"),
                        coarse_solver="dense")
    r = solver.fgmres(pb.A0, pb.F, tg.apply, restart=10, tol=1e-10)
    assert r.iters == 1
    assert r.relres_true < 1e-12


def test_gmres_minimality_brute_force():
    """Identity preconditioner: FGMRES == GMRES, whose j-th residual is the minimum of
    ||F - A y|| over the Krylov space K_j(A, F), computed here by dense least squares."""
    pb = _tiny(n=6)
    A = pb.A0.toarray()
    F = pb.F
    r = solver.fgmres(pb.A0, F, lambda v: v, restart=12, tol=1e-14, maxit=12)
    Kry = [F]
    for _ in range(11):
        Kry.append(A @ Kry[-1])
    Kry = np.stack(Kry, axis=1)
    for j in range(1, 12):
        Q, _ = np.linalg.qr(Kry[:, :j])
        y, *_ = np.linalg.lstsq(A @ Q, F, rcond=None)
        best = np.linalg.norm(F - A @ Q @ y) / np.linalg.norm(F)
        assert abs(r.history[j - 1] - best) <= 1e-9 + 1e-6 * best


@pytest.mark.parametrize("order,dim,n", [(1, 2, 8), (2, 2, 8), (1, 3, 4)])
def test_fgmres_matches_dense_direct(order, dim, n):
    pb = _tiny(order=order, dim=dim, n=n, rhs="random")
    r = pb.solve("dense", record_basis=True)
    x_ref = np.linalg.solve(pb.A0.toarray(), pb.F)
    cond = np.linalg.cond(pb.A0.toarray())
    assert r.relres_true <= 1e-8
    assert np.linalg.norm(r.x - x_ref) / np.linalg.norm(x_ref) <= cond * 1e-8
    # monotone Givens residual estimates (GMRES minimality within a cycle)
    h = np.asarray(r.history)
    assert np.all(np.diff(h) <= 1e-12)
    # Arnoldi relation A0 Z_j = V_{j+1} Hbar_j and orthonormal V
    V, Z, Hbar = r.basis
    lhs = (pb.A0 @ Z.T).T
    rhs = Hbar.T @ V
    assert np.abs(lhs - rhs).max() <= 1e-12 * abs(pb.A0).max() * np.abs(Z).max() * Z.shape[1]
    G = V.conj() @ V.T
    # MGS: loss of orthogonality grows like u / relres as the residual falls
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-6


def test_fgmres_restart_monotone_true_residual():
    pb = _tiny(n=16, k=12.0, shift=72.0)
    wl = pb.wl
    tg = pb.twogrid()
    r = solver.fgmres(pb.A0, pb.F, tg.apply, restart=3, tol=1e-8, maxit=200)
    assert r.relres_true <= 1e-8
    assert len(r.cycle_true) > 1
    assert all(b <= a * (1 + 1e-12) for a, b in zip(r.cycle_true, r.cycle_true[1:]))


def test_fgmres_iteration_cap():
    pb = _tiny(n=16, k=12.0, shift=0.0)
    r = solver.fgmres(pb.A0, pb.F, lambda v: v, restart=5, tol=1e-12, maxit=7)
    assert r.iters == 7
    assert r.relres_true > 1e-12


def test_small_p1_workload_converges():
    r = solver.build_problem(hi.SMALL_P1).solve()
    assert r.relres_true <= 1e-8
    assert 15 <= r.iters <= 40


def test_shift_map_weights_are_paper_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_shift_weights.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        p = int(r[0])
        assert tuple(float(x) for x in r[1:]) == shiftmap.PAPER_WEIGHTS[p]


def test_shift_map_properties():
    for p, w in shiftmap.PAPER_WEIGHTS.items():
        kc0, kc1, a0, a1 = w
        for lvl in range(4, 11):
            kc = kc1 * math.exp(kc0 * lvl)
            # at k = k_c the exponent is exactly 1 (beta = 2 - e^0); clamped to [1, 2]
            assert abs(shiftmap.sigma(kc, lvl, w) - 1.0) < 1e-12
            ks = np.linspace(1.0, 4000.0, 200)
            s = [shiftmap.sigma(k, lvl, w) for k in ks]
            assert min(s) >= 1.0 and max(s) <= 2.0
            assert all(b >= a - 1e-15 for a, b in zip(s, s[1:]))     # non-decreasing in k
        assert abs(shiftmap.shift(450.0, 10, w) - 450.0 ** shiftmap.sigma(450.0, 10, w)) < 1e-9
