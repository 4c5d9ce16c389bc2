"""Pins of the heterogeneous-wavenumber oracle (k(x) = k_max mu(x), Sec. 2 and Sec. 6).

* A constant profile gives the constant-k system matrix of eq. sys_matrix.
* Closed forms: 1^T M_k 1 = int k^2 and 1^T B_k 1 = int_dOmega k for a profile split at
  x = 1/2 (a mesh line), in 2D P1/P2 and 3D P1.
* Nested spaces: for a profile constant on the coarse cells, P^T A_h P = A_2h (Galerkin equals
  rediscretisation) for the shifted and the unshifted operator.
* Manufactured solution: u = exp(i kappa x) solves -Lap u - k(y)^2 u = f with the impedance
  data of a layered k(y); the discrete solution converges at second order in the mass norm,
  and an operator that ignores the layers (k = k_max everywhere) does not converge.
* The twogrid-preconditioned FGMRES converges on the wedge profile.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import helm_inputs as hi
from oracle import fem, solver


def _split_x(a, b):
    return lambda x: np.where(x[:, 0] < 0.5, a, b)


def test_constant_profile_gives_constant_k_matrix():
    for dim, order, n in ((2, 1, 16), (2, 2, 8), (3, 1, 6)):
        mesh = fem.build_mesh(dim, order, n)
        k, eps = 7.5, 20.0
        K, Mk, M, B, Bk = fem.assemble_weighted(mesh, np.full(mesh.elems.shape[0], k))
        A = fem.system_matrix_het(K, Mk, M, Bk, eps)
        ref = fem.system_matrix(*fem.assemble(mesh), k, eps)
        assert abs(A - ref).max() <= 1e-13 * abs(ref).max()


@pytest.mark.parametrize("dim,order,n", [(2, 1, 16), (2, 2, 8), (3, 1, 6)])
def test_weighted_integrals(dim, order, n):
    a, b, kmax = 0.45, 0.9, 11.0
    mesh = fem.build_mesh(dim, order, n)
    ke = kmax * _split_x(a, b)(fem.element_centroids(mesh))
    _, Mk, _, _, Bk = fem.assemble_weighted(mesh, ke)
    one = np.ones(mesh.num_dofs)
    assert abs(one @ Mk @ one - kmax ** 2 * (a * a + b * b) / 2) <= 1e-12 * kmax ** 2
    # faces x = 0 (value a) and x = 1 (value b), each unit measure; the other 2(dim-1) faces half and half
    boundary = (a + b) + 2 * (dim - 1) * (a + b) / 2
    assert abs(one @ Bk @ one - kmax * boundary) <= 1e-12 * kmax


@pytest.mark.parametrize("dim,order,n", [(2, 1, 16), (2, 2, 8), (3, 1, 8)])
def test_galerkin_identity_for_coarse_cell_profile(dim, order, n):
    mu = lambda x: hi.cell_profile(x, n // 2, seed=9)  # noqa: E731
    wl = hi.Workload("het", dim, order, n, 13.0, 13.0 ** 1.5, "gaussian")
    pb = solver.build_problem_het(wl, mu)
    for A, Ac in ((pb.Aeps, pb.Aeps_c),):
        G = (pb.P.T @ A @ pb.P).tocsr()
        assert abs(G - Ac).max() <= 1e-12 * abs(Ac).max()
    # unshifted operator too (rediscretised on the coarse mesh here)
    cm = pb.cmesh
    K, Mk, M, B, Bk = fem.assemble_weighted(cm, wl.k * mu(fem.element_centroids(cm)))
    A0c = fem.system_matrix_het(K, Mk, M, Bk, 0.0)
    assert abs((pb.P.T @ pb.A0 @ pb.P).tocsr() - A0c).max() <= 1e-12 * abs(A0c).max()


def _layered(x):
    """k(y)/k_max on four layers with interfaces on the lines y = 1/4, 1/2, 3/4."""
    vals = np.array([1.0, 0.6, 0.8, 0.5])
    return vals[np.minimum((x[:, 1] * 4).astype(int), 3)]


def _manufactured_error(n, kmax, kappa, ignore_layers=False):
    mesh = fem.build_mesh(2, 1, n)
    ke = kmax * _layered(fem.element_centroids(mesh))
    K, Mk, M, B, Bk = fem.assemble_weighted(mesh, ke)
    u = np.exp(1j * kappa * mesh.coords[:, 0])
    # f = (kappa^2 - k_e^2) u per element; g = du/dn - i k_F u = i (kappa n_x - k_F) u per facet
    F = kappa ** 2 * (M @ u) - Mk @ u
    F = F + fem.load_from_nodal(mesh, M, np.zeros(mesh.num_dofs),
                                lambda xs, nrm: 1j * kappa * nrm[:, :1] * np.exp(1j * kappa * xs[:, :, 0]))
    F = F - 1j * (Bk @ u)
    if ignore_layers:
        K, Mk, M, B, Bk = fem.assemble_weighted(mesh, np.full(ke.shape, kmax))
    A0 = fem.system_matrix_het(K, Mk, M, Bk, 0.0)
    x = spla.spsolve(A0.tocsc(), F)
    e = x - u
    return math.sqrt(abs(np.vdot(e, M @ e)) / abs(np.vdot(u, M @ u)))


def test_manufactured_layered_solution_converges():
    kmax, kappa = 12.0, 9.0
    errs = [_manufactured_error(n, kmax, kappa) for n in (16, 32, 64, 128)]
    rates = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert rates[-1] > 1.9 and rates[-2] > 1.9, (errs, rates)
    bad = [_manufactured_error(n, kmax, kappa, ignore_layers=True) for n in (32, 128)]
    assert bad[1] > 0.5 * bad[0] and bad[1] > 50 * errs[-1], (bad, errs)


def test_fgmres_converges_on_the_wedge():
    kmax = 60.0
    wl = hi.Workload("wedge", 2, 1, 128, kmax, kmax ** 1.5, "gaussian", restart=50)
    pb = solver.build_problem_het(wl, hi.wedge_profile, source=(0.5, 0.55))
    r = pb.solve()
    assert r.relres_true <= 1e-8 and r.iters < 100
    assert np.linalg.norm(pb.F - pb.A0 @ r.x) <= 1e-8 * np.linalg.norm(pb.F)
    # the wedge profile really has three regions on this mesh
    assert set(np.unique(hi.wedge_profile(fem.element_centroids(pb.mesh)))) == set(hi.WEDGE_VALUES)
