"""Heterogeneous-wavenumber rows of the product's host setup against the oracle (CPU).

helm_host_het_row returns row `dof` of K, M_k = sum_e k_e^2 M_e, M and B_k = sum_F k_F B_F
(Sec. 2 with k in L^inf; Sec. 6, k(x) = k_max mu(x)) built from one wavenumber per element.
The wavenumbers are a smooth function of the element centroid: the oracle takes it at its own
centroids, and the product's array is filled in the element order the header documents, with
the centroids computed here from that description. So the documented order, the weighting of
every element and the facet owners are all checked against fem.assemble_weighted /
qfem.assemble row by row.
"""
import ctypes
import itertools

import numpy as np
import pytest

from oracle import fem, qfem
from paper_2104_01439_gb300 import _binding as b


def kfun(x):
    return 6.0 + 2.5 * np.sin(7.0 * x[:, 0] + 1.0) * np.cos(5.0 * x[:, 1] - 0.5) + (x[:, 2] if x.shape[1] > 2 else 0.0)


def documented_centroids(dim, n, elements):
    """Centroids in the header's element order: cells x fastest, then the cell's simplices."""
    h = 1.0 / n
    if elements == b.HELM_TENSOR:
        simp_c = [np.full(dim, 0.5)]
    elif dim == 2:
        simp_c = [np.array([2, 1]) / 3.0, np.array([1, 2]) / 3.0]
    else:
        simp_c = []
        for perm in itertools.permutations(range(3)):      # lexicographic axis permutations
            p, verts = [0, 0, 0], [(0, 0, 0)]
            for ax in perm:
                p[ax] += 1
                verts.append(tuple(p))
            simp_c.append(np.mean(np.array(verts, dtype=float), axis=0))
    out = []
    for cell in itertools.product(range(n), repeat=dim):
        c = np.array(cell[::-1], dtype=float)             # product's last index is x: x fastest
        out.extend((c + sc) * h for sc in simp_c)
    return np.array(out)


def _rows_match(lib, dim, order, elements, fine_n, level, k_elem, mats, W):
    side = 2 * order + 1
    noff = side ** dim
    bufs = [(ctypes.c_double * noff)() for _ in range(4)]
    kp = (ctypes.c_double * len(k_elem))(*k_elem)
    offs = []
    for o in range(noff):
        oo, lin, st = o, 0, 1
        for _ in range(dim):
            lin += (oo % side - order) * st
            oo //= side
            st *= W
        offs.append(lin)
    N = W ** dim
    for dof in range(N):
        assert lib.helm_host_het_row(dim, order, elements, 1.0 / fine_n, level, kp, dof, *bufs) == 0
        for buf, A in zip(bufs, mats):
            row = A.getrow(dof)
            ref = dict(zip(row.indices, row.data))
            got = {}
            for o, v in enumerate(buf):
                if v != 0.0:
                    got[dof + offs[o]] = got.get(dof + offs[o], 0.0) + v
            keys = set(got) | {c for c, v in ref.items() if abs(v) > 1e-14}
            for c in keys:
                assert abs(got.get(c, 0.0) - ref.get(c, 0.0)) <= 1e-12 * max(1.0, abs(ref.get(c, 0.0))), (dof, c)


@pytest.mark.parametrize("dim,order,n", [(2, 1, 8), (2, 1, 10), (2, 2, 6), (3, 1, 4)])
def test_simplex_het_rows_equal_oracle(dim, order, n):
    lib = b.load()
    for level, ln in ((0, n), (1, n // 2)):
        mesh = fem.build_mesh(dim, order, ln)
        K, Mk, M, B, Bk = fem.assemble_weighted(mesh, kfun(fem.element_centroids(mesh)))
        k_doc = kfun(documented_centroids(dim, ln, b.HELM_SIMPLICES))
        _rows_match(lib, dim, order, b.HELM_SIMPLICES, n, level, k_doc, (K, Mk, M, Bk), order * ln + 1)


@pytest.mark.parametrize("dim,order,n", [(2, 1, 8), (2, 2, 6), (2, 2, 10), (2, 3, 6), (3, 1, 4)])
def test_tensor_het_rows_equal_oracle(dim, order, n):
    lib = b.load()
    for level, ln in ((0, n), (1, n // 2)):
        mesh = qfem.build_mesh(dim, order, ln)
        K, Mk, M, B, Bk = qfem.assemble(mesh, kfun(mesh.centres))
        k_doc = kfun(documented_centroids(dim, ln, b.HELM_TENSOR))
        _rows_match(lib, dim, order, b.HELM_TENSOR, n, level, k_doc, (K, Mk, M, Bk), order * ln + 1)


def test_constant_k_rows_equal_the_class_tables():
    """With k = 1 everywhere the per-DoF rows are the class tables' rows (M_k = M, B_k = B)."""
    lib = b.load()
    dim, order, n = 2, 2, 8
    N, noff = (order * n + 1) ** dim, (2 * order + 1) ** dim
    ones = (ctypes.c_double * (2 * n * n))(*([1.0] * (2 * n * n)))
    het = [(ctypes.c_double * noff)() for _ in range(4)]
    tab = [(ctypes.c_double * noff)() for _ in range(3)]
    for dof in range(N):
        assert lib.helm_host_het_row(dim, order, b.HELM_SIMPLICES, 1.0 / n, 0, ones, dof, *het) == 0
        assert lib.helm_host_stencil_row(dim, order, b.HELM_SIMPLICES, 1.0 / n, 0, dof, *tab) == 0
        K, Mk, M, Bk = (np.array(x[:]) for x in het)
        Kt, Mt, Bt = (np.array(x[:]) for x in tab)
        assert np.allclose(K, Kt, atol=1e-14) and np.allclose(M, Mt, atol=1e-15)
        assert np.allclose(Mk, Mt, atol=1e-15) and np.allclose(Bk, Bt, atol=1e-15)
