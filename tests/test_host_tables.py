"""Host tables of the matrix-free operators against the oracle's assembled matrices (CPU).

The CUDA kernels apply K, M, B and the interpolation P from per-class tables built on the host
(coefficients read off a small reference mesh, prolongation weights per position class). The
C ABI's inspection entry points return any row of those tables through the kernels' own class
mapping, so every row can be compared with the oracle's assembled CSR matrices (Sec. 2,
eq. discreteproblem; Sec. 4, the interpolation I^(l)) without a GPU.
"""
import ctypes

import numpy as np
import pytest

from oracle import fem
from paper_2104_01439_gb300 import _binding as b

CASES = [(2, 1, 8), (2, 1, 10), (2, 2, 6), (2, 2, 8), (2, 2, 22), (3, 1, 4), (3, 1, 6)]


def _stencil_rows(lib, dim, order, elements, fine_n, level, N):
    R = order
    side = 2 * R + 1
    noff = side ** dim
    K, M, B = ((ctypes.c_double * noff)() for _ in range(3))
    rows = []
    for dof in range(N):
        assert lib.helm_host_stencil_row(dim, order, elements, 1.0 / fine_n, level, dof, K, M, B) == 0
        rows.append((np.array(K[:]), np.array(M[:]), np.array(B[:])))
    return rows, side, noff


def _offsets(dim, side, R, W):
    """Linear lattice offset of every box point (x fastest)."""
    out = []
    for o in range(side ** dim):
        oo, lin, st = o, 0, 1
        for _ in range(dim):
            lin += (oo % side - R) * st
            oo //= side
            st *= W
        out.append(lin)
    return np.array(out)


def _compare_rows(rows, mats, dim, order, W):
    # relative tolerance: 1e-13; 1e-12 for order 3, whose oracle matrices come from monomial-basis
    # polynomial integration pinned to 1e-12 (test_oracle_qfem.test_p3_matrices_against_quadrature)
    tol = 1e-12 if order == 3 else 1e-13
    side = 2 * order + 1
    offs = _offsets(dim, side, order, W)
    for dof, got in enumerate(rows):
        for g, A in zip(got, mats):
            ref = A.getrow(dof)
            dense = dict(zip(ref.indices, ref.data))
            cols = dof + offs
            # every nonzero of the oracle row lies in the box, and the box values agree
            inbox = {c for c, v in zip(cols, g) if v != 0.0}
            assert set(k for k, v in dense.items() if abs(v) > 1e-15) <= set(cols.tolist())
            for c, v in zip(cols, g):
                if v != 0.0:
                    assert c in dense, (dof, c)
                assert abs(v - dense.get(c, 0.0)) <= tol * max(1.0, abs(v)), (dof, c, v, dense.get(c))
            assert inbox <= set(dense)


@pytest.mark.parametrize("dim,order,n", CASES)
def test_stencil_tables_equal_assembled_rows(dim, order, n):
    lib = b.load()
    for level, level_n in ((0, n), (1, n // 2)):   # the coarse level may have an odd n
        mesh = fem.build_mesh(dim, order, level_n)
        K, M, B = fem.assemble(mesh)
        rows, _, _ = _stencil_rows(lib, dim, order, b.HELM_SIMPLICES, n, level, mesh.num_dofs)
        _compare_rows(rows, (K, M, B), dim, order, order * level_n + 1)


@pytest.mark.parametrize("dim,order,n", CASES)
def test_prolongation_weights_equal_interpolation(dim, order, n):
    lib = b.load()
    fine, coarse = fem.build_mesh(dim, order, n), fem.build_mesh(dim, order, n // 2)
    P = fem.prolongation(coarse, fine).tocsr()
    cap = (order + 1) ** dim
    cols = (ctypes.c_int64 * cap)()
    w = (ctypes.c_double * cap)()
    cnt = ctypes.c_int()
    for dof in range(fine.num_dofs):
        assert lib.helm_host_prolongation_row(dim, order, b.HELM_SIMPLICES, 1.0 / n, dof, cols, w,
                                              ctypes.byref(cnt)) == 0
        got = {cols[i]: w[i] for i in range(cnt.value)}
        row = P.getrow(dof)
        ref = {c: v for c, v in zip(row.indices, row.data) if abs(v) > 1e-15}
        assert set(got) == set(ref), dof
        for c in ref:
            assert abs(got[c] - ref[c]) <= 1e-14, (dof, c)


def test_inspection_refuses_bad_arguments():
    lib = b.load()
    K, M, B = ((ctypes.c_double * 9)() for _ in range(3))
    S = b.HELM_SIMPLICES
    assert lib.helm_host_stencil_row(2, 1, S, 1.0 / 8, 0, 81, K, M, B) == -1   # dof out of range
    assert lib.helm_host_stencil_row(2, 1, S, 1.0 / 8, 1, 25, K, M, B) == -1   # (coarse level: 5 x 5)
    assert lib.helm_host_stencil_row(2, 1, S, 1.0 / 8, 1, 24, K, M, B) == 0
    assert lib.helm_host_stencil_row(2, 1, S, 1.0 / 7, 0, 0, K, M, B) == -1    # odd n
    assert lib.helm_host_stencil_row(2, 1, 7, 1.0 / 8, 0, 0, K, M, B) == -1    # unknown family
    assert lib.helm_host_stencil_row(2, 1, S, 1.0 / 8, 2, 0, K, M, B) == -1    # unknown level
    assert lib.helm_host_stencil_row(2, 1, S, 1.0 / 8, 0, -1, K, M, B) == -1


Q_CASES = [(2, 1, 8), (2, 1, 10), (2, 1, 12), (2, 2, 6), (2, 2, 8), (2, 2, 22), (2, 3, 6), (2, 3, 10),
           (3, 1, 4), (3, 1, 6)]


@pytest.mark.parametrize("dim,order,n", Q_CASES)
def test_tensor_tables_equal_assembled_q_rows(dim, order, n):
    """Q_order on squares / cubes (Sec. 2): the tables equal the rows of oracle/qfem.py's
    element-by-element assembly, fine and coarse level, and the transfer weights equal its
    tensor-product interpolation."""
    from oracle import qfem
    lib = b.load()
    for level, level_n in ((0, n), (1, n // 2)):
        mesh = qfem.build_mesh(dim, order, level_n)
        K, _, M, B, _ = qfem.assemble(mesh)
        rows, _, _ = _stencil_rows(lib, dim, order, b.HELM_TENSOR, n, level, mesh.num_dofs)
        _compare_rows(rows, (K, M, B), dim, order, order * level_n + 1)
    fine, coarse = qfem.build_mesh(dim, order, n), qfem.build_mesh(dim, order, n // 2)
    P = qfem.prolongation(coarse, fine).tocsr()
    cap = (order + 1) ** dim
    cols, w, cnt = (ctypes.c_int64 * cap)(), (ctypes.c_double * cap)(), ctypes.c_int()
    for dof in range(fine.num_dofs):
        assert lib.helm_host_prolongation_row(dim, order, b.HELM_TENSOR, 1.0 / n, dof, cols, w,
                                              ctypes.byref(cnt)) == 0
        got = {cols[i]: w[i] for i in range(cnt.value)}
        row = P.getrow(dof)
        ref = {c: v for c, v in zip(row.indices, row.data) if abs(v) > 1e-15}
        assert set(got) == set(ref), dof
        assert all(abs(got[c] - ref[c]) <= 1e-14 for c in ref), dof


def test_q1_stencil_differs_from_p1():
    """The two families really give different operators (Q1 couples all eight neighbours)."""
    lib = b.load()
    K, M, B = ((ctypes.c_double * 9)() for _ in range(3))
    dof = 4 + 9 * 4                                # an interior DoF of the 8 x 8 mesh
    assert lib.helm_host_stencil_row(2, 1, b.HELM_SIMPLICES, 1.0 / 8, 0, dof, K, M, B) == 0
    p1 = np.array(K[:])
    assert lib.helm_host_stencil_row(2, 1, b.HELM_TENSOR, 1.0 / 8, 0, dof, K, M, B) == 0
    q1 = np.array(K[:])
    assert np.count_nonzero(p1) == 5 and np.count_nonzero(q1) == 9
    assert np.allclose(q1 * 3, [-1, -1, -1, -1, 8, -1, -1, -1, -1])


@pytest.mark.parametrize("dim,order,n", [(2, 1, 8), (2, 2, 8), (3, 1, 6)])
def test_tensor_load_vectors_equal_oracle(dim, order, n):
    """Q_order load vectors (Sec. 2, F(v) = int f v + int_dOmega g v): the plane wave's impedance
    data per boundary face and the interpolated Gaussian times the mass matrix."""
    from oracle import qfem
    lib = b.load()
    mesh = qfem.build_mesh(dim, order, n)
    _, _, M, _, _ = qfem.assemble(mesh)
    F = np.empty(mesh.num_dofs, dtype=np.complex128)
    ptr = ctypes.c_void_p(F.ctypes.data)
    k, theta, sigma = 9.0, 0.3, 2.0 / n
    assert lib.helm_load_planewave_e(dim, order, b.HELM_TENSOR, 1.0 / n, k, theta, ptr) == 0
    ref = qfem.load_planewave(mesh, M, k, theta)
    assert np.linalg.norm(F - ref) <= 1e-12 * np.linalg.norm(ref)
    assert lib.helm_load_gaussian_e(dim, order, b.HELM_TENSOR, 1.0 / n, sigma, 0.5, 0.5, 0.5, ptr) == 0
    f = np.exp(-np.sum((mesh.coords - 0.5) ** 2, axis=1) / (2 * sigma * sigma))
    ref = M @ f
    assert np.linalg.norm(F - ref) <= 1e-12 * np.linalg.norm(ref)
    # the simplex family through the same entry point equals the original builder
    G = np.empty_like(F)
    assert lib.helm_load_planewave_e(dim, order, b.HELM_SIMPLICES, 1.0 / n, k, theta, ptr) == 0
    assert lib.helm_load_planewave(dim, order, 1.0 / n, k, theta, ctypes.c_void_p(G.ctypes.data)) == 0
    assert np.array_equal(F, G)
