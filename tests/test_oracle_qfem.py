"""Pins of the tensor-product Q_p oracle (oracle/qfem.py; Sec. 2 elements, Sec. 3 stencils).

* Gauss-Lobatto points and 1D element matrices: textbook closed forms for p = 1, 2; for p = 3
  the matrices against Gauss-Legendre quadrature of the basis evaluated in barycentric form.
* The assembled interior Q1 stencil equals the one Sec. 3 prints (tests/golden/paper_q1_stencil.txt).
* Element-by-element assembly equals the Kronecker form of tensor-product spaces
  (K = K1 (x) M1 + M1 (x) K1, ...), in 2D and 3D.
* Sum rules: |Omega|, |dOmega|, constants in ker K, the energy of a linear function.
* Interpolation from the 2h space reproduces Q_p polynomials; Galerkin = rediscretisation.
* Plane-wave convergence of order p + 1; twogrid-preconditioned FGMRES (V(3,3), omega = 2/3)
  converges, also on the wedge.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import helm_inputs as hi
from oracle import fem, qfem, solver

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gauss_lobatto_points():
    assert np.allclose(qfem.gauss_lobatto_points(1), [0, 1], atol=0)
    assert np.allclose(qfem.gauss_lobatto_points(2), [0, 0.5, 1], atol=1e-15)
    r = math.sqrt(5) / 10
    assert np.allclose(qfem.gauss_lobatto_points(3), [0, 0.5 - r, 0.5 + r, 1], atol=1e-15)


def test_1d_matrices_closed_forms():
    h = 0.3
    K1, M1 = qfem.element_matrices_1d(1, h)
    assert np.allclose(K1, np.array([[1, -1], [-1, 1]]) / h, atol=1e-14)
    assert np.allclose(M1, np.array([[2, 1], [1, 2]]) * h / 6, atol=1e-15)
    K2, M2 = qfem.element_matrices_1d(2, h)
    assert np.allclose(K2, np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3 * h), atol=1e-13)
    assert np.allclose(M2, np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) * h / 30, atol=1e-15)


def _bary_eval(nodes, i, x, deriv=False):
    """Lagrange basis i (or its derivative) at x from the product formula, term by term."""
    others = [j for j in range(len(nodes)) if j != i]
    den = np.prod([nodes[i] - nodes[j] for j in others])
    if not deriv:
        return np.prod([x - nodes[j] for j in others], axis=0) / den
    s = 0.0
    for m in others:
        s = s + np.prod([x - nodes[j] for j in others if j != m], axis=0)
    return s / den


def test_p3_matrices_against_quadrature():
    h = 0.7
    K3, M3 = qfem.element_matrices_1d(3, h)
    nodes = qfem.gauss_lobatto_points(3) * h
    xg, wg = np.polynomial.legendre.leggauss(8)
    x, w = (xg + 1) * h / 2, wg * h / 2
    for i in range(4):
        for j in range(4):
            m = np.sum(w * _bary_eval(nodes, i, x) * _bary_eval(nodes, j, x))
            k = np.sum(w * _bary_eval(nodes, i, x, True) * _bary_eval(nodes, j, x, True))
            assert abs(M3[i, j] - m) <= 1e-14 and abs(K3[i, j] - k) <= 1e-12
    assert np.abs(K3.sum(axis=1)).max() <= 1e-12 and abs(M3.sum() - h) <= 1e-14


def _read_stencils():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_q1_stencil.txt")) if not l.startswith("#")]
    assert rows[0][0] == "stiffness" and rows[4][0] == "mass"
    S = np.array([[float(v) for v in r] for r in rows[1:4]])
    T = np.array([[float(v) for v in r] for r in rows[5:8]])
    return S / 3.0, T / 36.0


def test_q1_interior_stencil_is_the_printed_one():
    S, T = _read_stencils()
    n = 8
    mesh = qfem.build_mesh(2, 1, n)
    K, _, M, _, _ = qfem.assemble(mesh)
    W, h = n + 1, 1.0 / n
    for (i, j) in ((3, 4), (1, 1), (6, 2)):
        row = i + W * j
        k = K[row].toarray().reshape(W, W)[j - 1:j + 2, i - 1:i + 2]   # rows = y, top row printed first
        m = M[row].toarray().reshape(W, W)[j - 1:j + 2, i - 1:i + 2]
        assert np.allclose(k[::-1], S, atol=1e-14)
        assert np.allclose(m[::-1] / (h * h), T, atol=1e-14)


def _global_1d(p, n):
    h = 1.0 / n
    K1, M1 = qfem.element_matrices_1d(p, h)
    W = p * n + 1
    Kg, Mg = np.zeros((W, W)), np.zeros((W, W))
    for c in range(n):
        s = slice(p * c, p * c + p + 1)
        Kg[s, s] += K1
        Mg[s, s] += M1
    return Kg, Mg


@pytest.mark.parametrize("dim,p,n", [(2, 1, 4), (2, 2, 3), (2, 3, 3), (3, 1, 3), (3, 2, 2), (3, 3, 2)])
def test_assembly_equals_kronecker_form(dim, p, n):
    mesh = qfem.build_mesh(dim, p, n)
    K, _, M, B, _ = qfem.assemble(mesh)
    Kg, Mg = _global_1d(p, n)
    W = p * n + 1
    E = np.zeros((W, W))
    E[0, 0] = E[-1, -1] = 1.0
    kr = lambda *ms: ms[0] if len(ms) == 1 else np.kron(kr(*ms[:-1]), ms[-1])  # noqa: E731
    if dim == 2:     # slower axis on the left
        Kr, Mr, Br = kr(Mg, Kg) + kr(Kg, Mg), kr(Mg, Mg), kr(Mg, E) + kr(E, Mg)
    else:
        Kr = kr(Mg, Mg, Kg) + kr(Mg, Kg, Mg) + kr(Kg, Mg, Mg)
        Mr = kr(Mg, Mg, Mg)
        Br = kr(Mg, Mg, E) + kr(Mg, E, Mg) + kr(E, Mg, Mg)
    for A, R in ((K, Kr), (M, Mr), (B, Br)):
        assert np.abs(A.toarray() - R).max() <= 1e-12 * np.abs(R).max()


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_sum_rules(dim, p):
    mesh = qfem.build_mesh(dim, p, 4)
    K, _, M, B, _ = qfem.assemble(mesh)
    one = np.ones(mesh.num_dofs)
    x = mesh.coords[:, 0]
    assert abs(one @ M @ one - 1.0) <= 1e-13
    assert abs(one @ B @ one - 2.0 * dim) <= 1e-13
    assert np.abs(K @ one).max() <= 1e-11
    assert abs(x @ K @ x - 1.0) <= 1e-12             # int |grad x|^2 = |Omega|


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_interpolation_reproduces_polynomials_and_galerkin(dim, p):
    n = 4
    fine, coarse = qfem.build_mesh(dim, p, n), qfem.build_mesh(dim, p, n // 2)
    P = qfem.prolongation(coarse, fine)
    rng = np.random.default_rng(p)
    for _ in range(4):
        e = rng.integers(0, p + 1, dim)                  # degree <= p per variable
        q = lambda X: np.prod(X ** e, axis=1)            # noqa: E731
        assert np.abs(P @ q(coarse.coords) - q(fine.coords)).max() <= 1e-12
    k, eps = 9.0, 30.0
    Kf, _, Mf, Bf, _ = qfem.assemble(fine)
    Kc, _, Mc, Bc, _ = qfem.assemble(coarse)
    Af = fem.system_matrix(Kf, Mf, Bf, k, eps)
    Ac = fem.system_matrix(Kc, Mc, Bc, k, eps)
    assert abs((P.T @ Af @ P).tocsr() - Ac).max() <= 1e-12 * abs(Ac).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_planewave_convergence_order(p):
    k, theta = 8.0, 0.3
    d = np.array([math.cos(theta), math.sin(theta)])
    errs = []
    ns = (4, 8, 16, 32) if p < 3 else (4, 8, 16)
    for n in ns:
        wl = hi.Workload("qpw", 2, p, n, k, 0.0, "planewave")
        pb = solver.build_problem_q(wl)
        x = spla.spsolve(pb.A0.tocsc(), pb.F)
        u = np.exp(1j * k * (pb.mesh.coords @ d))
        e = x - u
        errs.append(math.sqrt(abs(np.vdot(e, pb.M @ e)) / abs(np.vdot(u, pb.M @ u))))
    rate = math.log2(errs[-2] / errs[-1])
    assert rate > p + 1 - 0.25, (p, errs)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_twogrid_fgmres_paper_setting(p):
    wl = hi.Workload("qpw", 2, p, 32, 12.0, 72.0, "planewave", restart=50, omega=2.0 / 3.0, nu=3)
    pb = solver.build_problem_q(wl)
    r = pb.solve()
    assert r.relres_true <= 1e-8 and r.iters < 40
    assert np.linalg.norm(pb.F - pb.A0 @ r.x) <= 1e-8 * np.linalg.norm(pb.F)


def test_wedge_q2():
    kmax = 60.0
    wl = hi.Workload("qw", 2, 2, 64, kmax, kmax ** 1.5, "source", restart=50, omega=2.0 / 3.0, nu=3)
    pb = solver.build_problem_q(wl, hi.wedge_profile, source=(0.5, 0.55))
    r = pb.solve()
    assert r.relres_true <= 1e-8 and r.iters < 80
