"""Pins of the local Fourier analysis (oracle/lfa.py, Sec. 3).

* Brute force: on a periodic n x n grid the operators are assembled as matrices from element
  matrices (Q1 by tensor products of 1D P1; P1 Kuhn from the oracle's element matrices),
  interpolation is built from its definition (hat functions / barycentric weights) and the
  coarse operator is rediscretised on the coarse periodic grid. Applying them to the Fourier
  modes of the grid gives the hat matrices entry by entry, which must equal the LFA's symbols;
  T_hat must equal the projection of the assembled twogrid operator on the harmonics.
* The formulas Sec. 3 prints for Q1 (symbols of L_h, L_2h, S_h and the transfer columns with
  the factor-of-four reading of the module docstring).
* Invariants: the coarse correction is a projection and the coarse symbol is the Galerkin
  product of the fine one (nested spaces, R = P^T).
* The oracle's damped Jacobi on the bounded P1 problem multiplies a Fourier mode by the
  smoother symbol at nodes farther than nu from the boundary.
* The observations Sec. 3 reports for its figures.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import fem, lfa, solver


# ---------------------------------------------------------------------------- periodic matrices
def _gidx(i, j, n):
    return (i % n) + n * (j % n)


def _q1_element(h):
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    M1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0
    # local nodes (0,0), (1,0), (0,1), (1,1): index a + 2 b = kron(y factor, x factor)
    return np.kron(M1, K1) + np.kron(K1, M1), np.kron(M1, M1), [(0, 0), (1, 0), (0, 1), (1, 1)]


def periodic_matrices(disc, n, h):
    """Stiffness and mass on the periodic n x n grid of spacing h."""
    K = np.zeros((n * n, n * n))
    M = np.zeros((n * n, n * n))
    if disc is lfa.Q1:
        Ke, Me, loc = _q1_element(h)
        elems = [(Ke, Me, loc)]
    else:
        elems = []
        for tri in ([(0, 0), (1, 0), (1, 1)], [(0, 0), (1, 1), (0, 1)]):
            Ke, Me = fem.element_matrices([(a * h, b * h) for a, b in tri], 1)
            elems.append((Ke, Me, tri))
    for i in range(n):
        for j in range(n):
            for Ke, Me, loc in elems:
                g = [_gidx(i + a, j + b, n) for a, b in loc]
                for p in range(len(g)):
                    for q in range(len(g)):
                        K[g[p], g[q]] += Ke[p, q]
                        M[g[p], g[q]] += Me[p, q]
    return K, M


def periodic_interpolation(disc, n):
    """Canonical interpolation from the (n/2)^2 coarse grid (spacing 2h) to the n^2 grid."""
    m = n // 2
    P = np.zeros((n * n, m * m))
    for x in range(n):
        for y in range(n):
            X, Y = x // 2, y // 2
            s, t = (x - 2 * X) / 2.0, (y - 2 * Y) / 2.0
            if disc is lfa.Q1:   # bilinear hat functions
                w = {(0, 0): (1 - s) * (1 - t), (1, 0): s * (1 - t), (0, 1): (1 - s) * t, (1, 1): s * t}
            elif s >= t:         # triangle (0,0), (1,0), (1,1)
                w = {(0, 0): 1 - s, (1, 0): s - t, (1, 1): t}
            else:                # triangle (0,0), (1,1), (0,1)
                w = {(0, 0): 1 - t, (1, 1): s, (0, 1): t - s}
            for (dx, dy), v in w.items():
                if v:
                    P[_gidx(x, y, n), _gidx(X + dx, Y + dy, m)] += v
    return P


def mode(theta, n):
    """phi(theta, x) = exp(i theta . x / h) on the periodic n x n grid."""
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    return np.exp(1j * (theta[0] * i + theta[1] * j)).reshape(-1)


def low_grid_frequencies(n):
    """Frequencies 2 pi j / n of the periodic grid that lie in (-pi/2, pi/2]."""
    return [2 * math.pi * j / n for j in range(-(n // 4) + 1, n // 4 + 1)]


CASES = [
    # disc, n, kh, sigma, omega, nu1, nu2
    (lfa.Q1, 16, 0.5, 1.3, 2.0 / 3.0, 1, 2),
    (lfa.P1_KUHN, 16, 0.6, 1.6, 0.6, 2, 1),
]


def compare_with_periodic_grid(case):
    """Entry-by-entry comparison of every hat matrix with the assembled periodic operators."""
    disc, n, kh, sigma, omega, nu1, nu2 = case
    h = 1.0 / n
    k = kh / h
    lam = lfa.shifted_lambda(k, sigma)
    K, M = periodic_matrices(disc, n, h)
    Kc, Mc = periodic_matrices(disc, n // 2, 2 * h)
    P = periodic_interpolation(disc, n)
    A = K - lam * M
    Ac = Kc - lam * Mc
    S = np.eye(n * n) - omega * (A / np.diag(A)[:, None])
    C = np.eye(n * n) - P @ np.linalg.solve(Ac, P.T @ A)
    T = np.linalg.matrix_power(S, nu2) @ C @ np.linalg.matrix_power(S, nu1)
    assert np.abs(P.T @ A @ P - Ac).max() <= 1e-12 * np.abs(Ac).max()   # Galerkin = rediscretised
    axis = low_grid_frequencies(n)
    for t1 in axis:
        for t2 in axis:
            theta = (t1, t2)
            th = lfa.harmonics(theta)
            Phi = np.stack([mode(t, n) for t in th], axis=1)              # fine harmonics
            phic = mode((2 * t1, 2 * t2), n // 2)                          # coarse mode
            # each harmonic is a mode of the fine grid and the four are orthogonal
            assert np.abs(Phi.conj().T @ Phi - n * n * np.eye(4)).max() <= 1e-9
            for a, t in enumerate(th):
                assert np.allclose(A @ Phi[:, a], lfa.op_symbol(disc, t, lam, h) * Phi[:, a], atol=1e-10)
                assert np.allclose(S @ Phi[:, a], lfa.jacobi_symbol(disc, t, lam, h, omega) * Phi[:, a],
                                   atol=1e-10)
                assert np.allclose(P.T @ Phi[:, a], lfa.restriction_symbol(disc, t) * phic, atol=1e-10)
            assert np.allclose(Ac @ phic, lfa.op_symbol(disc, (2 * t1, 2 * t2), lam, 2 * h) * phic,
                               atol=1e-10)
            Pcol = np.array([lfa.prolongation_symbol(disc, t) for t in th])
            assert np.allclose(P @ phic, Phi @ Pcol, atol=1e-10)
            # T maps the harmonic space into itself; its coefficients are T_hat
            TPhi = T @ Phi
            That = Phi.conj().T @ TPhi / (n * n)
            assert np.abs(TPhi - Phi @ That).max() <= 1e-9
            ref = lfa.twogrid_hat(disc, theta, k, sigma, h, omega, nu1, nu2)
            assert np.abs(That - ref).max() <= 1e-10, theta


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0].name)
def test_hat_matrices_match_periodic_grid(case):
    compare_with_periodic_grid(case)


def _mutations():
    op, tg, pr = lfa.op_symbol, lfa.twogrid_hat, lfa.prolongation_symbol
    return {
        "mass sign": ("op_symbol", lambda st, t, lam, h: op(st, t, -lam, h)),
        "nu1/nu2 swapped": ("twogrid_hat", lambda st, th, k, s, h, w, a, b: tg(st, th, k, s, h, w, b, a)),
        "T_hat transposed": ("twogrid_hat", lambda *a: tg(*a).T),
        "prolongation without 1/4": ("prolongation_symbol", lambda st, t: 4 * pr(st, t)),
    }


@pytest.mark.parametrize("name", list(_mutations()))
def test_planted_mistakes_are_caught(name, monkeypatch):
    """A plausible mistake planted in the LFA fails the periodic-grid comparison."""
    attr, fn = _mutations()[name]
    monkeypatch.setattr(lfa, attr, fn)
    with pytest.raises(AssertionError):
        compare_with_periodic_grid(CASES[0])


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0].name)
def test_rho_loc_is_the_spectral_radius_of_the_periodic_twogrid(case):
    """On the grid's own low frequencies, rho_loc equals the spectral radius of the assembled
    twogrid operator (whose spectrum is the union of the T_hat spectra)."""
    disc, n, kh, sigma, omega, nu1, nu2 = case
    h = 1.0 / n
    k = kh / h
    lam = lfa.shifted_lambda(k, sigma)
    K, M = periodic_matrices(disc, n, h)
    Kc, Mc = periodic_matrices(disc, n // 2, 2 * h)
    P = periodic_interpolation(disc, n)
    A, Ac = K - lam * M, Kc - lam * Mc
    S = np.eye(n * n) - omega * (A / np.diag(A)[:, None])
    T = np.linalg.matrix_power(S, nu2) @ (np.eye(n * n) - P @ np.linalg.solve(Ac, P.T @ A)) \
        @ np.linalg.matrix_power(S, nu1)
    brute = np.sort(np.abs(np.linalg.eigvals(T)))
    axis = low_grid_frequencies(n)
    hat = np.sort(np.concatenate([np.abs(np.linalg.eigvals(
        lfa.twogrid_hat(disc, (t1, t2), k, sigma, h, omega, nu1, nu2))) for t1 in axis for t2 in axis]))
    assert brute.shape == hat.shape
    assert np.abs(brute - hat).max() <= 1e-7
    # the module's sampling of T^low with m = n/2 points per axis is this frequency set
    assert abs(lfa.rho_loc(disc, k, sigma, h, omega, nu1, nu2, m=n // 2) - brute[-1]) <= 1e-7


def test_printed_q1_symbols():
    """Symbols Sec. 3 prints for Q1, and its transfer columns: the printed prolongation column
    is 4 x the interpolation symbol and the printed restriction row 1/4 x that of P^T."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        t1, t2 = rng.uniform(-math.pi / 2, math.pi / 2, 2)
        h = 2.0 ** -rng.integers(4, 9)
        k = rng.uniform(0.1, 0.7) / h
        sigma = rng.uniform(1, 2)
        omega = rng.uniform(0.3, 1.0)
        lam = lfa.shifted_lambda(k, sigma)
        lh2 = lam * h * h
        c1, c2 = math.cos(t1), math.cos(t2)
        Lh = (8 - 2 * c1 - 2 * c2 - 4 * c1 * c2) / 3 - lh2 / 36 * (16 + 8 * c1 + 8 * c2 + 4 * c1 * c2)
        assert abs(lfa.op_symbol(lfa.Q1, (t1, t2), lam, h) - Lh) <= 1e-12
        C1, C2 = math.cos(2 * t1), math.cos(2 * t2)
        L2h = (8 - 2 * C1 - 2 * C2 - 4 * C1 * C2) / 3 - lh2 / 9 * (16 + 8 * C1 + 8 * C2 + 4 * C1 * C2)
        assert abs(lfa.op_symbol(lfa.Q1, (2 * t1, 2 * t2), lam, 2 * h) - L2h) <= 1e-12
        den = 8 / 3 - lh2 * 16 / 36
        S = (1 - omega) + omega * (2 / 3 + lh2 * 8 / 36) / den * (c1 + c2) \
            + omega * (4 / 3 + lh2 * 4 / 36) / den * c1 * c2
        assert abs(lfa.jacobi_symbol(lfa.Q1, (t1, t2), lam, h, omega) - S) <= 1e-12
        printed = [(1 + c1) * (1 + c2), (1 - c1) * (1 - c2), (1 - c1) * (1 + c2), (1 + c1) * (1 - c2)]
        for t, col in zip(lfa.harmonics((t1, t2)), printed):
            assert abs(4 * lfa.prolongation_symbol(lfa.Q1, t) - col) <= 1e-12
            assert abs(lfa.restriction_symbol(lfa.Q1, t) / 4 - col / 4) <= 1e-12   # printed row x 4


@pytest.mark.parametrize("disc", [lfa.Q1, lfa.P1_KUHN], ids=lambda d: d.name)
def test_coarse_correction_is_a_galerkin_projection(disc):
    rng = np.random.default_rng(5)
    for _ in range(20):
        theta = tuple(rng.uniform(-math.pi / 2, math.pi / 2, 2))
        h = 2.0 ** -rng.integers(4, 9)
        k, sigma = rng.uniform(0.1, 0.7) / h, rng.uniform(1, 2)
        lam = lfa.shifted_lambda(k, sigma)
        th = lfa.harmonics(theta)
        Lhat = np.diag([lfa.op_symbol(disc, t, lam, h) for t in th])
        P = np.array([lfa.prolongation_symbol(disc, t) for t in th])
        R = np.array([lfa.restriction_symbol(disc, t) for t in th])
        L2h = lfa.op_symbol(disc, (2 * theta[0], 2 * theta[1]), lam, 2 * h)
        assert abs(R @ Lhat @ P - L2h) <= 1e-12 * max(1.0, abs(L2h))
        Khat = lfa.twogrid_hat(disc, theta, k, sigma, h, 0.6, 0, 0)
        assert np.abs(Khat @ Khat - Khat).max() <= 1e-10
        assert abs(spectral := lfa.spectral_radius(Khat)) - 1.0 <= 1e-10 and spectral >= 1 - 1e-10


def test_oracle_jacobi_multiplies_a_mode_by_the_smoother_symbol():
    """Bounded P1 problem (impedance boundary): with f = A_eps phi the error of nu Jacobi sweeps
    from zero is S^nu (-phi), so u = (1 - S_tilde^nu) phi wherever the sweeps never saw the
    boundary (nodes more than nu steps inside)."""
    n, k, omega = 32, 12.0, 0.6
    eps = 0.5 * k * k
    mesh = fem.build_mesh(2, 1, n)
    K, M, B = fem.assemble(mesh)
    A = fem.system_matrix(K, M, B, k, eps)
    W, h = n + 1, 1.0 / n
    lam = k * k + 1j * eps
    i, j = np.meshgrid(np.arange(W), np.arange(W), indexing="xy")
    i, j = i.reshape(-1), j.reshape(-1)
    for theta in [(0.3, -1.1), (2.0, 0.7), (-2.9, 2.5)]:
        phi = np.exp(1j * (theta[0] * i + theta[1] * j))
        f = A @ phi
        for nu in (1, 2, 3):
            u = solver.jacobi_sweeps(A, 1.0 / A.diagonal(), f, np.zeros_like(f), omega, nu)
            inner = (i > nu) & (i < W - 1 - nu) & (j > nu) & (j < W - 1 - nu)
            expect = (1 - lfa.jacobi_symbol(lfa.P1_KUHN, theta, lam, h, omega) ** nu) * phi
            assert np.abs(u[inner] - expect[inner]).max() <= 1e-12, (theta, nu)
            # and the boundary does change the result (the test is not vacuous)
            assert np.abs(u - expect).max() > 1e-6


def test_paper_observations():
    """Sec. 3 (nu1 = nu2 = 3, omega = 2/3, h = 2^-5, kh = 0.25): rho_loc grows as sigma falls
    from 2 to 1, and the maximum over T^low lies on the axis theta_2 = 0 (every other line
    theta_2 = c, refined the same way, stays below it; also where the method diverges, at
    h = 2^-6, kh = 0.75). sigma_c grows with k at fixed h and shrinks with h at fixed k."""
    omega, nu = 2.0 / 3.0, 3
    lines = [-math.pi / 2 + math.pi * (j + 1) / 16 for j in range(16)]
    for h, kh, sigmas in ((2.0 ** -5, 0.25, (1.0, 1.25, 1.5, 1.75, 2.0)), (2.0 ** -6, 0.75, (1.3, 1.5))):
        k = kh / h
        rho = []
        for sg in sigmas:
            on_axis = lfa.rho_loc(lfa.Q1, k, sg, h, omega, nu, nu, m=32, line=True)
            off = max(lfa.rho_loc(lfa.Q1, k, sg, h, omega, nu, nu, m=32, line=True, theta2=c) for c in lines)
            assert off <= on_axis * (1 + 1e-9), (h, sg)
            rho.append(on_axis)
        assert all(a > b for a, b in zip(rho, rho[1:])), rho
    sc = lambda kk, hh: lfa.sigma_c(lfa.Q1, kk, hh, omega, nu, nu, m=16, steps=16, tol=1e-3)  # noqa: E731
    h = 2.0 ** -6
    assert sc(0.5 / h, h) < sc(0.75 / h, h)
    k = 0.75 / 2.0 ** -6
    assert sc(k, 2.0 ** -7) < sc(k, 2.0 ** -6)


def test_sigma_c_is_the_convergence_threshold():
    h, omega, nu = 2.0 ** -6, 2.0 / 3.0, 3
    k, tol = 0.75 / h, 1e-3
    s = lfa.sigma_c(lfa.Q1, k, h, omega, nu, nu, m=16, steps=16, tol=tol)
    assert 1.0 < s < 2.0
    f = lambda x: lfa.rho_loc(lfa.Q1, k, x, h, omega, nu, nu, m=16, line=True)  # noqa: E731
    assert f(s) < 1.0 <= f(s - 2 * tol)
    # a well-resolved low wavenumber converges for every sigma in [1, 2]
    assert lfa.sigma_c(lfa.Q1, 1.0, h, omega, nu, nu, m=16, steps=4) == 1.0


def test_sigma_c_depends_on_h_not_on_the_smoother():
    """Sec. 3: for kh < 0.75, varying the smoothing steps and the damping barely moves sigma_c,
    while the mesh size at fixed kh moves it markedly."""
    sc = lambda k, h, om, nu: lfa.sigma_c(lfa.Q1, k, h, om, nu, nu, m=32, steps=16, tol=1e-3)  # noqa: E731
    h = 2.0 ** -6
    for kh in (0.5, 0.7):
        vals = [sc(kh / h, h, om, nu) for nu, om in ((2, 0.6), (3, 2.0 / 3.0), (1, 0.8))]
        assert max(vals) - min(vals) <= 0.02, (kh, vals)
    kh = 0.7
    assert sc(kh / 2.0 ** -7, 2.0 ** -7, 2.0 / 3.0, 3) - sc(kh / 2.0 ** -5, 2.0 ** -5, 2.0 / 3.0, 3) >= 0.1
