"""Pins for the oracle's finite-element layer (Sec. 2). CPU only.

Each test checks the oracle against something other than itself: textbook
element matrices, exact integrals of polynomials the space reproduces,
closed-form stencils, the Galerkin identity of nested spaces, the paper's
printed DoF counts, and the convergence order of the plane-wave
manufactured solution.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- element level

def test_p1_reference_triangle_textbook():
    K, M = fem.element_matrices([[0, 0], [1, 0], [0, 1]], 1)
    K_ref = 0.5 * np.array([[2, -1, -1], [-1, 1, 0], [-1, 0, 1]])
    M_ref = np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) / 24.0
    np.testing.assert_allclose(K, K_ref, atol=1e-15)
    np.testing.assert_allclose(M, M_ref, atol=1e-15)


def test_p2_triangle_mass_textbook():
    # P2 mass on a triangle of area |T|: |T|/180 x {vertex diag 6, vertex-vertex -1,
    # vertex-opposite-midpoint -4, vertex-adjacent-midpoint 0, midpoint diag 32,
    # midpoint-midpoint 16}. Local order: v0 v1 v2 m01 m02 m12.
    area = 0.5
    _, M = fem.element_matrices([[0, 0], [1, 0], [0, 1]], 2)
    ref = np.array([
        [6, -1, -1, 0, 0, -4],
        [-1, 6, -1, 0, -4, 0],
        [-1, -1, 6, -4, 0, 0],
        [0, 0, -4, 32, 16, 16],
        [0, -4, 0, 16, 32, 16],
        [-4, 0, 0, 16, 16, 32]]) * area / 180.0
    np.testing.assert_allclose(M, ref, atol=1e-15)


def test_p1_tet_and_edge_mass_textbook():
    _, M = fem.element_matrices([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], 1)
    np.testing.assert_allclose(M, (np.ones((4, 4)) + np.eye(4)) / 120.0, atol=1e-15)
    B = fem.facet_mass([[0.0, 0.0], [0.0, 0.5]], 1)
    np.testing.assert_allclose(B, 0.5 / 6.0 * np.array([[2, 1], [1, 2]]), atol=1e-15)
    B2 = fem.facet_mass([[0.0, 0.0], [2.0, 0.0]], 2)     # 1D P2 mass: L/30 [4 -1 2; -1 4 2; 2 2 16]
    np.testing.assert_allclose(B2, 2.0 / 30.0 * np.array([[4, -1, 2], [-1, 4, 2], [2, 2, 16]]),
                               atol=1e-15)


# ---------------------------------------------------------------- assembled level

def _interp(mesh, fn):
    return fn(*[mesh.coords[:, a] for a in range(mesh.dim)])


@pytest.mark.parametrize("dim,order,n", [(2, 1, 4), (2, 2, 3), (3, 1, 3)])
def test_assembled_sums(dim, order, n):
    m = fem.build_mesh(dim, order, n)
    K, M, B = fem.assemble(m)
    one = np.ones(m.num_dofs)
    assert np.abs(K @ one).max() < 1e-13          # constants are in the kernel of K
    assert abs(one @ M @ one - 1.0) < 1e-13       # |Omega| = 1
    assert abs(one @ B @ one - 2 * dim) < 1e-13   # |dOmega| = 4 (2D) or 6 (3D)


def test_exact_integrals_p1_2d():
    m = fem.build_mesh(2, 1, 5)
    K, M, B = fem.assemble(m)
    x = _interp(m, lambda x, y: x)
    y = _interp(m, lambda x, y: y)
    assert abs(x @ M @ y - 0.25) < 1e-14           # int xy
    assert abs(x @ K @ x - 1.0) < 1e-13            # int |grad x|^2
    assert abs(x @ K @ y) < 1e-13                  # int grad x . grad y
    assert abs(x @ B @ y - 1.0) < 1e-14            # boundary int xy = 1/2 + 1/2


def test_exact_integrals_p2_2d():
    m = fem.build_mesh(2, 2, 3)
    K, M, B = fem.assemble(m)
    x2 = _interp(m, lambda x, y: x * x)
    xy = _interp(m, lambda x, y: x * y)
    y = _interp(m, lambda x, y: y)
    one = np.ones(m.num_dofs)
    assert abs(x2 @ M @ y - 1.0 / 6.0) < 1e-13     # int x^2 y
    assert abs(x2 @ K @ xy - 0.5) < 1e-13          # int 2x * y
    assert abs(x2 @ B @ one - 5.0 / 3.0) < 1e-13   # 1/3 + 1/3 + 0 + 1
    assert abs(xy @ K @ xy - 2.0 / 3.0) < 1e-13    # int y^2 + x^2


def test_exact_integrals_p1_3d():
    m = fem.build_mesh(3, 1, 3)
    K, M, B = fem.assemble(m)
    u = _interp(m, lambda x, y, z: x + 2 * y + 3 * z)
    x = _interp(m, lambda x, y, z: x)
    y = _interp(m, lambda x, y, z: y)
    one = np.ones(m.num_dofs)
    assert abs(u @ K @ u - 14.0) < 1e-12
    assert abs(x @ M @ y - 0.25) < 1e-13
    assert abs(x @ B @ one - 3.0) < 1e-13


def test_p1_interior_stencils_closed_form():
    # Interior rows on the main-diagonal triangle mesh: K is the 5-point
    # Laplacian [-1,-1,4,-1,-1]; M = h^2/12 [6 centre, 1 at +-x, +-y, +-(1,1)].
    n = 6
    h = 1.0 / n
    m = fem.build_mesh(2, 1, n)
    K, M, _ = fem.assemble(m)
    W = n + 1
    p = 3 + 3 * W
    kr = {(c - p): v for c, v in zip(K[p].indices, K[p].data) if abs(v) > 1e-14}
    mr = {(c - p): v for c, v in zip(M[p].indices, M[p].data) if abs(v) > 1e-14}
    assert set(kr) == {0, 1, -1, W, -W}
    assert abs(kr[0] - 4) < 1e-13 and all(abs(kr[o] + 1) < 1e-13 for o in (1, -1, W, -W))
    assert set(mr) == {0, 1, -1, W, -W, W + 1, -W - 1}
    assert abs(mr[0] - h * h / 2) < 1e-15
    assert all(abs(mr[o] - h * h / 12) < 1e-15 for o in (1, -1, W, -W, W + 1, -W - 1))


def test_dof_counts_match_paper_tables():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_dof_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        p, lvl, d, printed = int(r[0]), int(r[1]), int(r[2]), int(r[3])
        n = 2 ** lvl
        # a P_p simplicial grid has the same DoF lattice as Q_p: (p n + 1)^d complex DoFs
        assert 2 * (p * n + 1) ** d == printed
    # and the oracle's meshes realise that lattice
    for d, p, n in [(2, 1, 8), (2, 2, 4), (3, 1, 4)]:
        assert fem.build_mesh(d, p, n).num_dofs == (p * n + 1) ** d


# ---------------------------------------------------------------- transfers

@pytest.mark.parametrize("dim,order,nc", [(2, 1, 4), (2, 2, 3), (3, 1, 2)])
def test_galerkin_identity_and_reproduction(dim, order, nc):
    cm = fem.build_mesh(dim, order, nc)
    fm = fem.build_mesh(dim, order, 2 * nc)
    P = fem.prolongation(cm, fm)
    Kc, Mc, Bc = fem.assemble(cm)
    Kf, Mf, Bf = fem.assemble(fm)
    for k, eps in [(7.0, 24.5), (3.0, 0.0)]:
        Af = fem.system_matrix(Kf, Mf, Bf, k, eps)
        Ac = fem.system_matrix(Kc, Mc, Bc, k, eps)
        assert abs(P.T @ Af @ P - Ac).max() < 1e-12 * abs(Ac).max()
    # P interpolates exactly every function of the coarse space
    if order == 1:
        fn = lambda *x: 1.0 + sum((a + 2) * xi for a, xi in enumerate(x))
    else:
        fn = lambda x, y: 1 + x - 2 * y + 3 * x * y + x * x - 0.5 * y * y
    uc = _interp(cm, fn)
    uf = _interp(fm, fn)
    assert np.abs(P @ uc - uf).max() < 1e-13
    # rows of P sum to one (partition of unity)
    assert np.abs(P @ np.ones(cm.num_dofs) - 1).max() < 1e-13


# ---------------------------------------------------------------- discretisation

def _planewave_error(dim, order, n, k, theta=0.3):
    m = fem.build_mesh(dim, order, n)
    K, M, B = fem.assemble(m)
    A = fem.system_matrix(K, M, B, k, 0.0)
    F = fem.load_planewave(m, M, k, theta)
    u = spla.spsolve(A.tocsc(), F)
    d = np.zeros(dim)
    d[0], d[1] = math.cos(theta), math.sin(theta)
    ui = fem.plane_wave(m.coords, k, d)
    e = u - ui
    return math.sqrt(abs(np.vdot(e, M @ e)) / abs(np.vdot(ui, M @ ui)))


@pytest.mark.parametrize("dim,order,ns,k,rate", [
    (2, 1, (8, 16, 32, 64), 6.0, 1.85),
    (2, 2, (4, 8, 16, 32), 6.0, 2.7),
    (3, 1, (3, 6, 12), 3.0, 1.7),
])
def test_planewave_convergence_order(dim, order, ns, k, rate):
    """u = exp(ik d.x) solves -Lap u - k^2 u = 0 with g = ik(d.n - 1)u; the FE error
    in the mass norm must shrink like h^(p+1). A wrong sign in the impedance term,
    a wrong normal or a wrong load assembly breaks convergence."""
    errs = [_planewave_error(dim, order, n, k) for n in ns]
    rates = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]
    assert rates[-1] > rate, (errs, rates)
    assert errs[-1] < 0.05


def test_planewave_is_not_solution_with_flipped_boundary_sign():
    # negative control: the opposite impedance sign must not converge to the plane wave
    m = fem.build_mesh(2, 1, 32)
    K, M, B = fem.assemble(m)
    A_bad = (K.astype(complex) - 36.0 * M + 6.0j * B).tocsc()
    F = fem.load_planewave(m, M, 6.0, 0.3)
    u = spla.spsolve(A_bad, F)
    ui = fem.plane_wave(m.coords, 6.0, [math.cos(0.3), math.sin(0.3)])
    e = u - ui
    assert math.sqrt(abs(np.vdot(e, M @ e)) / abs(np.vdot(ui, M @ ui))) > 0.1


# ---------------------------------------------------------------- Gaussian point source

@pytest.mark.parametrize("dim,order,n,sigma,x0", [
    (2, 1, 64, 0.06, (0.5, 0.5)),
    (2, 1, 64, 0.05, (0.42, 0.57)),
    (2, 2, 32, 0.05, (0.45, 0.52)),
    (3, 1, 24, 0.08, (0.5, 0.47, 0.53)),
])
def test_gaussian_load_moments(dim, order, n, sigma, x0):
    """F = M I_h f for f = exp(-|x - x0|^2 / (2 sigma^2)) (the benchmark's point source).

    The basis sums to one, so sum_i F_i = int I_h f, which for a Gaussian well inside the
    domain (tail e^{-(dist to the boundary)^2 / (2 sigma^2)} < 1e-8 here) is the closed form
    (2 pi sigma^2)^{dim/2} up to the interpolation error. Its centroid sum x_i F_i / sum F_i
    is x0 and its second moment sum |x_i - x0|^2 F_i / sum F_i is dim sigma^2 (the variance of
    a normal distribution), both up to O(h^2) (the mass matrix spreads each nodal value over
    neighbouring nodes). A sigma^2 for 2 sigma^2 mistake (factor 2 in the integral and the
    moment) or a shifted centre fails these."""
    mesh = fem.build_mesh(dim, order, n)
    _, M, _ = fem.assemble(mesh)
    F = fem.load_gaussian(mesh, M, sigma, center=np.array(x0))
    assert np.allclose(F.imag, 0.0)
    F = F.real
    total = F.sum()
    assert abs(total / (2 * math.pi * sigma ** 2) ** (dim / 2) - 1.0) <= 1e-3
    x = mesh.coords
    h = 1.0 / n
    np.testing.assert_allclose((x * F[:, None]).sum(0) / total, x0, atol=h * h)
    second = (np.sum((x - np.array(x0)) ** 2, axis=1) * F).sum() / total
    assert abs(second / (dim * sigma ** 2) - 1.0) <= 4 * h * h / sigma ** 2


def test_gaussian_load_centre_and_width_are_the_arguments():
    """The default centre is the domain's centre, and the width enters as exp(-r^2 / (2 s^2))."""
    mesh = fem.build_mesh(2, 1, 32)
    _, M, _ = fem.assemble(mesh)
    a = fem.load_gaussian(mesh, M, 0.07)
    b = fem.load_gaussian(mesh, M, 0.07, center=np.array([0.5, 0.5]))
    np.testing.assert_allclose(a, b, rtol=0, atol=0)
    # f at a DoF r away from the centre relative to the centre's: e^{-r^2 / (2 sigma^2)}
    f = np.linalg.solve(M.toarray(), a.real)
    i0 = np.argmin(np.sum((mesh.coords - 0.5) ** 2, axis=1))
    i1 = np.argmin(np.sum((mesh.coords - [0.5 + 3 / 32, 0.5]) ** 2, axis=1))
    assert abs(f[i1] / f[i0] - math.exp(-(3 / 32) ** 2 / (2 * 0.07 ** 2))) <= 1e-12
