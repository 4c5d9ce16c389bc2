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


# Values of eq. shiftexp worked out by hand from the columns of Table tab:optweights (Sec. 5):
#   p = 1, l = 10: k_c = 2.5790033 e^{4.5927886} = 2.5790033 * (90.017131 * 1.0972292) = 254.7268
#                  alpha = 1.7580550 e^{-6.2616373} = 1.7580550 * (2.478752e-3 * 0.769765) = 3.35458e-3
#                  k = 450: beta = 2 - e^{-3.35458e-3 * 195.2732} = 2 - e^{-0.655058} = 1.480589
#                  k = k_c + 1/alpha = 254.7268 + 298.1003 = 552.8271: beta = 2 - e^{-1} = 1.632121
#   p = 2, l = 10: k_c = 2.5729975 e^{5.7369269} = 2.5729975 * (298.86740 * 1.0376171) = 797.912
#                  alpha = 1.5966387 e^{-6.6151997} = 1.5966387 * (1.5034392e-3 * 0.8911834) = 2.13925e-3
#                  k = 1100: beta = 2 - e^{-2.13925e-3 * 302.088} = 2 - e^{-0.646242} = 1.475989
#   p = 1, l = 8:  k_c = 2.5790033 e^{3.6742309} = 2.5790033 * (36.598234 * 1.0770554) = 101.660
#                  alpha = 1.7580550 e^{-5.0093098} = 1.7580550 * (6.737947e-3 * 0.990733) = 1.17359e-2
#                  k = 150: beta = 2 - e^{-1.17359e-2 * 48.340} = 2 - e^{-0.567314} = 1.432954
#   p = 1, l = 6:  k_c = 2.5790033 e^{2.7556732} = 2.5790033 * (14.879732 * 1.0572520) = 40.572 > k = 20:
#                  beta < 1, clamped to 1
# Swapping the two weights of k_c(l) or of alpha(l), or a sign, moves them.
SHIFT_MAP_BY_HAND = [   # p, l, k, sigma
    (1, 10, 450.0, 1.480589),
    (1, 10, 552.8271, 1.632121),
    (2, 10, 1100.0, 1.475989),
    (1, 8, 150.0, 1.432954),
    (1, 6, 20.0, 1.0),
]


@pytest.mark.parametrize("p,lvl,k,expected", SHIFT_MAP_BY_HAND)
def test_shift_map_values_worked_by_hand(p, lvl, k, expected):
    assert abs(shiftmap.sigma(k, lvl, shiftmap.PAPER_WEIGHTS[p]) - expected) <= 2e-6


def test_shift_map_pins_catch_swapped_weights():
    """Planted mistakes in the map's weights fail the hand-worked values above."""
    kc0, kc1, a0, a1 = shiftmap.PAPER_WEIGHTS[1]

    def off(w, lvl, k, s):
        try:
            return abs(shiftmap.sigma(k, lvl, w) - s) > 1e-3
        except OverflowError:        # e^{-alpha (k - k_c)} beyond float range: not the value either
            return True
    for bad in ((kc0, kc1, a1, a0), (kc1, kc0, a0, a1), (kc0, kc1, -a0, a1), (-kc0, kc1, a0, a1)):
        assert any(off(bad, lvl, k, s) for p, lvl, k, s in SHIFT_MAP_BY_HAND if p == 1)


def test_golden_section_min_closed_forms():
    """The oracle's golden-section search: minima of closed-form unimodal functions, inside the
    final bracket, with the textbook evaluation count (2 + one per bracket reduction by the
    golden ratio r: the bracket after j reductions is r^j of the start)."""
    r = (math.sqrt(5) - 1) / 2
    for x0, tol in ((1.37, 1e-2), (1.0, 1e-3), (1.9, 1e-4)):
        x, fx, count = solver.golden_section_min(lambda s: (s - x0) ** 2, 1.0, 2.0, tol)
        assert abs(x - x0) <= tol
        assert count == 2 + math.ceil(math.log(tol) / math.log(r))
    x, _, _ = solver.golden_section_min(lambda s: abs(math.sin(3 * s)), 0.5, 1.5, 1e-6)
    assert abs(x - math.pi / 3) <= 1e-6


def test_shift_rate_is_the_average_reduction():
    """rho^iterations equals the true relative residual, and a capped solve has rho < 1."""
    import helm_inputs as hi
    F = hi.uniform_loads([33 * 33], seed=1)[0]
    for sigma in (1.0, 1.6):
        rho = solver.shift_rate(12.0, 32, 1, sigma, F, maxit=50)
        assert 0.0 < rho < 1.0
    rho_cap = solver.shift_rate(12.0, 32, 1, 2.0, F, maxit=5)
    mesh = fem.build_mesh(2, 1, 32)
    cm = fem.build_mesh(2, 1, 16)
    K, M, B = fem.assemble(mesh)
    Kc, Mc, Bc = fem.assemble(cm)
    tg = solver.TwoGrid(fem.system_matrix(K, M, B, 12.0, 144.0), fem.system_matrix(Kc, Mc, Bc, 12.0, 144.0),
                        fem.prolongation(cm, mesh))
    ref = solver.fgmres(fem.system_matrix(K, M, B, 12.0, 0.0), F, tg.apply, restart=5, tol=1e-8, maxit=5)
    assert ref.iters == 5 and abs(rho_cap ** 5 - ref.relres_true) <= 1e-12
