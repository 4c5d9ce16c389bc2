"""Tensor-product Q_p Lagrange elements (p = 1, 2, 3) on the unit square / cube (Sec. 2).

TEST INFRASTRUCTURE (see oracle/__init__.py). FP64, assembled CSR.

The paper discretises with standard Q_p elements on a uniform grid of squares (2D) or cubes
(3D) of side h (Sec. 2). Here:
  * the 1D Lagrange basis of degree p on [0, h] interpolates at the Gauss-Lobatto points
    (endpoints and the roots of P_p'; for p <= 2 these are the equispaced points);
  * 1D element matrices K1 = int phi_i' phi_j', M1 = int phi_i phi_j are integrated exactly
    (polynomial antiderivatives);
  * the element matrices of a square / cube are their tensor products, e.g. in 2D
    K_e = M1 (x) K1 + K1 (x) M1 and M_e = M1 (x) M1 (local index x fastest);
  * boundary facets (edges / squares of the boundary) carry the tensor-product mass of the
    face, B_F = M1 (2D) or M1 (x) M1 (3D);
  * global DoFs are the (p n + 1)^d lattice points, numbered lexicographically, x fastest;
  * assembly is element by element, with an optional wavenumber per element (Sec. 6,
    k(x) = k_max mu(x) taken at the element centre; a boundary facet takes its element's value);
  * the canonical interpolation from the 2h space is the tensor product of the 1D
    interpolation matrices (coarse basis evaluated at the fine points).
"""
import itertools
import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
from numpy.polynomial import Polynomial
from numpy.polynomial import legendre as L


def gauss_lobatto_points(p):
    """Gauss-Lobatto points of degree p on [0, 1]: 0, 1 and the roots of P_p' mapped from [-1, 1]."""
    if p == 1:
        return np.array([0.0, 1.0])
    inner = np.sort(np.real(L.legroots(L.legder([0] * p + [1]))))
    return np.concatenate([[0.0], (inner + 1.0) / 2.0, [1.0]])


def lagrange_1d(p, h=1.0):
    """Lagrange basis polynomials of degree p on [0, h] at the Gauss-Lobatto points."""
    x = gauss_lobatto_points(p) * h
    basis = []
    for i in range(p + 1):
        q = Polynomial([1.0])
        for j in range(p + 1):
            if j != i:
                q = q * Polynomial([-x[j], 1.0]) / (x[i] - x[j])
        basis.append(q)
    return basis, x


def element_matrices_1d(p, h):
    """K1[i, j] = int_0^h phi_i' phi_j', M1[i, j] = int_0^h phi_i phi_j (exact)."""
    basis, _ = lagrange_1d(p, h)
    n = p + 1
    K1 = np.zeros((n, n))
    M1 = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            a = (basis[i].deriv() * basis[j].deriv()).integ()
            b = (basis[i] * basis[j]).integ()
            K1[i, j] = a(h) - a(0.0)
            M1[i, j] = b(h) - b(0.0)
    return K1, M1


def element_matrices(dim, p, h):
    """Stiffness and mass of one square / cube element (local index x fastest)."""
    K1, M1 = element_matrices_1d(p, h)
    if dim == 2:
        return np.kron(M1, K1) + np.kron(K1, M1), np.kron(M1, M1)
    K = np.kron(np.kron(M1, M1), K1) + np.kron(np.kron(M1, K1), M1) + np.kron(np.kron(K1, M1), M1)
    return K, np.kron(np.kron(M1, M1), M1)


@dataclass
class QMesh:
    dim: int
    order: int
    n: int
    coords: np.ndarray      # (N, dim) lattice points, x fastest
    elems: np.ndarray       # (E, (p+1)^dim) DoFs of each element, local index x fastest
    centres: np.ndarray     # (E, dim)
    facets: np.ndarray      # (F, (p+1)^(dim-1)) DoFs of each boundary facet
    facet_elems: np.ndarray  # (F,) owning element
    facet_normals: np.ndarray  # (F, dim)

    @property
    def num_dofs(self):
        return self.coords.shape[0]

    @property
    def h(self):
        return 1.0 / self.n


def build_mesh(dim, p, n):
    """Uniform grid of n^dim squares / cubes of (0,1)^dim with Q_p elements."""
    h = 1.0 / n
    W = p * n + 1
    _, x1 = lagrange_1d(p, h)
    axis = np.concatenate([c * h + x1[:-1] for c in range(n)] + [[1.0]])   # W points
    strides = np.array([W ** a for a in range(dim)], dtype=np.int64)
    idx = np.array(list(itertools.product(range(W), repeat=dim)), dtype=np.int64)[:, ::-1]  # x fastest
    coords = axis[idx]
    loc = np.array(list(itertools.product(range(p + 1), repeat=dim)), dtype=np.int64)[:, ::-1]
    cells = np.array(list(itertools.product(range(n), repeat=dim)), dtype=np.int64)[:, ::-1]
    elems = (p * cells[:, None, :] + loc[None, :, :]) @ strides
    centres = (cells + 0.5) * h
    facets, owners, normals = [], [], []
    floc_all = np.array(list(itertools.product(range(p + 1), repeat=dim - 1)), dtype=np.int64)[:, ::-1]
    for ax in range(dim):
        others = [a for a in range(dim) if a != ax]
        for side in (0, 1):
            sel = np.nonzero(cells[:, ax] == (0 if side == 0 else n - 1))[0]
            fl = np.zeros((floc_all.shape[0], dim), dtype=np.int64)
            fl[:, others] = floc_all
            fl[:, ax] = 0 if side == 0 else p
            facets.append((p * cells[sel][:, None, :] + fl[None, :, :]) @ strides)
            owners.append(sel)
            nrm = np.zeros((sel.shape[0], dim))
            nrm[:, ax] = -1.0 if side == 0 else 1.0
            normals.append(nrm)
    return QMesh(dim, p, n, coords, elems, centres, np.concatenate(facets), np.concatenate(owners),
                 np.concatenate(normals))


def _scatter(N, loc, mat, scale):
    nl = loc.shape[1]
    rows = np.repeat(loc, nl, axis=1).ravel()
    cols = np.tile(loc, (1, nl)).ravel()
    vals = (scale[:, None] * mat.ravel()[None, :]).ravel()
    A = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    A.sum_duplicates()
    A.sort_indices()
    return A


def assemble(mesh, k_elem=None):
    """K, M_k = sum_e k_e^2 M_e, M, B, B_k = sum_F k_F B_F (k_elem None: k = 1)."""
    N, E = mesh.num_dofs, mesh.elems.shape[0]
    ke = np.ones(E) if k_elem is None else np.asarray(k_elem, dtype=float)
    Ke, Me = element_matrices(mesh.dim, mesh.order, mesh.h)
    _, M1 = element_matrices_1d(mesh.order, mesh.h)
    Bf = M1 if mesh.dim == 2 else np.kron(M1, M1)
    one_e, one_f = np.ones(E), np.ones(mesh.facets.shape[0])
    K = _scatter(N, mesh.elems, Ke, one_e)
    M = _scatter(N, mesh.elems, Me, one_e)
    Mk = _scatter(N, mesh.elems, Me, ke ** 2)
    B = _scatter(N, mesh.facets, Bf, one_f)
    Bk = _scatter(N, mesh.facets, Bf, ke[mesh.facet_elems])
    return K, Mk, M, B, Bk


def interpolation_1d(p, n_coarse):
    """(2 p n + 1) x (p n + 1): the coarse 1D basis evaluated at the fine lattice points. A fine
    point on the boundary between two coarse elements gets the same row from either element
    (the coarse functions are continuous there); round-off below 1e-14 is dropped."""
    hc = 1.0 / n_coarse
    basis, _ = lagrange_1d(p, hc)
    _, xf = lagrange_1d(p, hc / 2)
    xfine = np.concatenate([c * hc / 2 + xf[:-1] for c in range(2 * n_coarse)] + [[1.0]])
    P = np.zeros((xfine.shape[0], p * n_coarse + 1))
    for i, x in enumerate(xfine):
        c = min(int(x / hc), n_coarse - 1)
        for a in range(p + 1):
            P[i, p * c + a] = basis[a](x - c * hc)
    P[np.abs(P) < 1e-14] = 0.0
    return P


def prolongation(coarse, fine):
    """Canonical interpolation V_2h -> V_h: tensor product of the 1D interpolations."""
    assert fine.n == 2 * coarse.n and fine.order == coarse.order and fine.dim == coarse.dim
    P1 = sp.csr_matrix(interpolation_1d(fine.order, coarse.n))
    P = P1
    for _ in range(fine.dim - 1):
        P = sp.kron(P1, P).tocsr()     # slower axes on the left (x fastest)
    P.eliminate_zeros()
    return P


def load_planewave(mesh, M, k, theta):
    """Impedance data of u = exp(i k d.x), d = (cos t, sin t[, 0]): f = 0, g = i k (d.n - 1) u,
    interpolated per boundary facet with its own normal."""
    d = np.zeros(mesh.dim)
    d[0], d[1] = math.cos(theta), math.sin(theta)
    _, M1 = element_matrices_1d(mesh.order, mesh.h)
    Bf = M1 if mesh.dim == 2 else np.kron(M1, M1)
    F = np.zeros(mesh.num_dofs, dtype=np.complex128)
    xs = mesh.coords[mesh.facets]                                  # (F, nf, dim)
    g = 1j * k * ((mesh.facet_normals @ d)[:, None] - 1.0) * np.exp(1j * k * (xs @ d))
    np.add.at(F, mesh.facets.ravel(), (g @ Bf.T).ravel())
    return F


def load_source(mesh, M, s, amplitude=2.0, width=1000.0):
    """The paper's source f = 2 exp(-1000 |x - s|^2), g = 0 (Sec. 6), interpolated then M f."""
    f = amplitude * np.exp(-width * np.sum((mesh.coords - np.asarray(s)) ** 2, axis=1))
    return M @ f.astype(np.complex128)
