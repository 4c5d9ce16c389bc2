"""Finite-element assembly for the oracle (Sec. 2: eq. var_form .. eq. sys_matrix).

TEST INFRASTRUCTURE (see oracle/__init__.py). Plain and slow on purpose.

Meshes (the paper uses Q_p quads; the synthetic workloads here use simplices):
  * 2D: unit square, n x n cells, each split along its main diagonal into
    {(i,j),(i+1,j),(i+1,j+1)} and {(i,j),(i+1,j+1),(i,j+1)}. Nested under
    uniform refinement, so V_2h is a subspace of V_h (Sec. 4).
  * 3D: unit cube, Kuhn's six tetrahedra per cube, all sharing the cube's
    (0,0,0)-(1,1,1) diagonal (also nested under refinement).
  * P2 DoFs live on the half-spacing grid, index a + (2n+1) b.
DoFs are numbered lexicographically, x fastest.

Element integrals are exact: every basis function is a polynomial in the
barycentric coordinates and  int_T lam^alpha = d! |T| alpha! / (|alpha|+d)!.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

# ----------------------------------------------------------------------------
# Barycentric polynomials: dict {exponent tuple: coefficient}
# ----------------------------------------------------------------------------


def _poly_mul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0.0) + ca * cb
    return out


def _poly_diff(p, a):
    """d/d lam_a of a barycentric polynomial."""
    out = {}
    for e, c in p.items():
        if e[a] > 0:
            e2 = list(e)
            e2[a] -= 1
            out[tuple(e2)] = out.get(tuple(e2), 0.0) + c * e[a]
    return out


def _poly_integral(p, d, measure):
    """Exact integral over a d-simplex of measure |T| of a barycentric polynomial."""
    s = 0.0
    for e, c in p.items():
        num = math.factorial(d) * math.prod(math.factorial(x) for x in e)
        s += c * num / math.factorial(sum(e) + d)
    return s * measure


def _poly_eval(p, lam):
    return sum(c * math.prod(l ** x for l, x in zip(lam, e)) for e, c in p.items())


def lagrange_basis(d, order):
    """Lagrange basis on a d-simplex in barycentric form.

    Returns (basis polys, node barycentric coords). order 1: lam_i at the
    vertices. order 2: lam_i(2 lam_i - 1) at the vertices, then 4 lam_a lam_b
    at the midpoints of edges (a,b) in itertools.combinations order.
    """
    nv = d + 1
    unit = [tuple(1 if j == i else 0 for j in range(nv)) for i in range(nv)]
    if order == 1:
        basis = [{unit[i]: 1.0} for i in range(nv)]
        nodes = [tuple(float(x) for x in unit[i]) for i in range(nv)]
        return basis, nodes
    if order == 2:
        basis, nodes = [], []
        for i in range(nv):
            two = tuple(2 if j == i else 0 for j in range(nv))
            basis.append({two: 2.0, unit[i]: -1.0})
            nodes.append(tuple(float(x) for x in unit[i]))
        for a, b in itertools.combinations(range(nv), 2):
            e = tuple(1 if j in (a, b) else 0 for j in range(nv))
            basis.append({e: 4.0})
            nodes.append(tuple(0.5 if j in (a, b) else 0.0 for j in range(nv)))
        return basis, nodes
    raise ValueError("order must be 1 or 2")


def simplex_measure(verts):
    """|T| for a simplex given its (d+1) x dim vertex array (dim == d)."""
    v = np.asarray(verts, dtype=float)
    d = v.shape[0] - 1
    if v.shape[1] == d:
        return abs(np.linalg.det(v[1:] - v[0])) / math.factorial(d)
    # lower-dimensional facet embedded in R^dim: sqrt(det(G)) / d!
    J = (v[1:] - v[0]).T
    return math.sqrt(abs(np.linalg.det(J.T @ J))) / math.factorial(d)


def barycentric_gradients(verts):
    """Gradients of the barycentric coordinates of a full-dimensional simplex."""
    v = np.asarray(verts, dtype=float)
    d = v.shape[0] - 1
    T = np.ones((d + 1, d + 1))
    T[1:, :] = v.T
    # lam = T^{-1} [1; x]  ->  grad lam_i = row i of T^{-1}, columns 1..d
    Tinv = np.linalg.inv(T)
    return Tinv[:, 1:]


def element_matrices(verts, order):
    """Stiffness K_e[i,j] = int grad phi_j . grad phi_i and mass M_e[i,j] = int phi_j phi_i."""
    v = np.asarray(verts, dtype=float)
    d = v.shape[0] - 1
    basis, _ = lagrange_basis(d, order)
    meas = simplex_measure(v)
    G = barycentric_gradients(v)          # (d+1) x d
    GG = G @ G.T                          # grad lam_a . grad lam_b
    nb = len(basis)
    dphi = [[_poly_diff(basis[i], a) for a in range(d + 1)] for i in range(nb)]
    K = np.zeros((nb, nb))
    M = np.zeros((nb, nb))
    for i in range(nb):
        for j in range(nb):
            M[i, j] = _poly_integral(_poly_mul(basis[i], basis[j]), d, meas)
            s = 0.0
            for a in range(d + 1):
                for b in range(d + 1):
                    if GG[a, b] != 0.0:
                        s += GG[a, b] * _poly_integral(_poly_mul(dphi[i][a], dphi[j][b]), d, meas)
            K[i, j] = s
    return K, M


def facet_mass(verts, order):
    """Boundary mass int_F phi_j phi_i over a facet (edge in 2D, triangle in 3D)."""
    v = np.asarray(verts, dtype=float)
    d = v.shape[0] - 1
    basis, _ = lagrange_basis(d, order)
    meas = simplex_measure(v)
    nb = len(basis)
    B = np.zeros((nb, nb))
    for i in range(nb):
        for j in range(nb):
            B[i, j] = _poly_integral(_poly_mul(basis[i], basis[j]), d, meas)
    return B


# ----------------------------------------------------------------------------
# Structured simplicial meshes of the unit square / cube
# ----------------------------------------------------------------------------


@dataclass
class Mesh:
    dim: int
    order: int
    n: int                 # cells per side
    coords: np.ndarray     # (N, dim) DoF coordinates
    elems: np.ndarray      # (E, nloc) DoF indices, basis order of lagrange_basis
    elem_verts: np.ndarray  # (E, dim+1) vertex DoF indices
    facets: np.ndarray     # (F, nfloc) boundary facet DoF indices (facet basis order)
    facet_normals: np.ndarray  # (F, dim) outward unit normals
    facet_elems: np.ndarray = None  # (F,) element (simplex) owning each boundary facet

    @property
    def num_dofs(self):
        return self.coords.shape[0]

    @property
    def h(self):
        return 1.0 / self.n


def _simplices_of_cell(dim):
    """Vertex offsets (in cell units) of the simplices of one cell."""
    if dim == 2:
        return [((0, 0), (1, 0), (1, 1)), ((0, 0), (1, 1), (0, 1))]
    out = []
    for perm in itertools.permutations(range(3)):
        p = [0, 0, 0]
        verts = [tuple(p)]
        for ax in perm:
            p[ax] += 1
            verts.append(tuple(p))
        out.append(tuple(verts))
    return out


def _template_local_offsets(dim, order, simp):
    """DoF-grid offsets (units of h/order) of the local DoFs of one cell simplex."""
    basis_nodes = lagrange_basis(dim, order)[1]
    vg = np.asarray(simp, dtype=float) * order
    return np.asarray([[int(round(sum(l * vg[i, ax] for i, l in enumerate(lam))))
                        for ax in range(dim)] for lam in basis_nodes], dtype=np.int64)


def build_mesh(dim, order, n):
    """Structured mesh of (0,1)^dim with n cells per side, Lagrange order 1 or 2.

    Elements are ordered (cell, simplex); cells lexicographic with the first
    axis slowest (itertools.product order).
    """
    if order == 2 and dim == 3:
        raise NotImplementedError("P2 tetrahedra are not part of the workloads")
    q = order
    W = q * n + 1
    h = 1.0 / n
    strides = np.asarray([W ** ax for ax in range(dim)], dtype=np.int64)
    grid = np.stack(np.meshgrid(*([np.arange(W)] * dim), indexing="ij"), axis=-1)
    grid = grid.reshape(-1, dim)
    order_lex = np.argsort(grid @ strides)
    coords = grid[order_lex] * (h / q)

    cells = np.asarray(list(itertools.product(range(n), repeat=dim)), dtype=np.int64)
    templates = _simplices_of_cell(dim)
    S = len(templates)
    nloc = len(lagrange_basis(dim, order)[0])
    elems = np.zeros((cells.shape[0], S, nloc), dtype=np.int64)
    everts = np.zeros((cells.shape[0], S, dim + 1), dtype=np.int64)
    for s, simp in enumerate(templates):
        off = _template_local_offsets(dim, order, simp)
        base = q * cells
        elems[:, s, :] = (base[:, None, :] + off[None, :, :]) @ strides
        voff = np.asarray(simp, dtype=np.int64) * q
        everts[:, s, :] = (base[:, None, :] + voff[None, :, :]) @ strides
    elems = elems.reshape(-1, nloc)
    everts = everts.reshape(-1, dim + 1)

    # Boundary facets: faces of cell simplices lying in a side of the box.
    fnodes = lagrange_basis(dim - 1, order)[1]
    facets, normals, owners = [], [], []
    for s_idx, simp in enumerate(templates):
        sv = np.asarray(simp, dtype=np.int64)
        for face in itertools.combinations(range(dim + 1), dim):
            fv = sv[list(face)]
            floc = np.asarray([[int(round(sum(l * fv[i, ax] * q for i, l in enumerate(lam))))
                                for ax in range(dim)] for lam in fnodes], dtype=np.int64)
            for ax in range(dim):
                for side in (0, 1):
                    if not np.all(fv[:, ax] == side):
                        continue
                    sel = cells[:, ax] == (0 if side == 0 else n - 1)
                    base = q * cells[sel]
                    facets.append((base[:, None, :] + floc[None, :, :]) @ strides)
                    nrm = np.zeros((base.shape[0], dim))
                    nrm[:, ax] = -1.0 if side == 0 else 1.0
                    normals.append(nrm)
                    owners.append(np.nonzero(sel)[0] * S + s_idx)   # elements are (cell, simplex)
    return Mesh(dim, order, n, coords, elems, everts,
                np.concatenate(facets), np.concatenate(normals), np.concatenate(owners))


# ----------------------------------------------------------------------------
# Assembly (Sec. 2): K_ij = a(phi_j, phi_i), M_ij = m(.,.;1,0), B_ij = b(.,.;1)
# ----------------------------------------------------------------------------


def _scatter(N, locs, mats):
    """Sum local matrices mats[g] (nl x nl) into an N x N CSR at DoFs locs[e] of group g."""
    rows, cols, vals = [], [], []
    for loc, mat in zip(locs, mats):
        nl = loc.shape[1]
        rows.append(np.repeat(loc, nl, axis=1).ravel())
        cols.append(np.tile(loc, (1, nl)).ravel())
        vals.append(np.broadcast_to(mat.ravel(), (loc.shape[0], nl * nl)).ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    A.sum_duplicates()
    A.sort_indices()
    return A


def _group_by_shape(mesh, locs, nv):
    """Group simplices (rows of locs) by vertex shape relative to their first vertex."""
    vx = mesh.coords[locs[:, :nv]]
    rel = np.round((vx - vx[:, :1, :]) * mesh.n * 4).astype(np.int64).reshape(locs.shape[0], -1)
    keys, inv = np.unique(rel, axis=0, return_inverse=True)
    return [(np.nonzero(inv.ravel() == g)[0]) for g in range(keys.shape[0])]


def assemble(mesh):
    """Assembled real CSR matrices K (stiffness), M (unit mass), B (unit boundary mass).

    Structured meshes have a handful of distinct simplex shapes (translates);
    each shape's element matrices are integrated once and scattered.
    """
    N = mesh.num_dofs
    groups = _group_by_shape(mesh, mesh.elem_verts, mesh.dim + 1)
    locs, Ks, Ms = [], [], []
    for sel in groups:
        Ke, Me = element_matrices(mesh.coords[mesh.elem_verts[sel[0]]], mesh.order)
        locs.append(mesh.elems[sel])
        Ks.append(Ke)
        Ms.append(Me)
    K = _scatter(N, locs, Ks)
    M = _scatter(N, locs, Ms)
    fgroups = _group_by_shape(mesh, mesh.facets, mesh.dim)
    flocs, Bs = [], []
    for sel in fgroups:
        flocs.append(mesh.facets[sel])
        Bs.append(facet_mass(mesh.coords[mesh.facets[sel[0]][:mesh.dim]], mesh.order))
    B = _scatter(N, flocs, Bs)
    return K, M, B


def system_matrix(K, M, B, k, eps):
    """A(k, eps) = K - (k^2 + i eps) M - i k B  (eq. sys_matrix; the boundary term is unshifted)."""
    return (K.astype(np.complex128) - (k * k + 1j * eps) * M - 1j * k * B).tocsr()


# ----------------------------------------------------------------------------
# Heterogeneous wavenumber (Sec. 2 with k in L^inf; Sec. 6: k(x) = k_max mu(x)).
# The coefficient is element-local: one value per simplex, taken at its centroid.
# ----------------------------------------------------------------------------


def element_centroids(mesh):
    """(E, dim) centroids of the simplices."""
    return mesh.coords[mesh.elem_verts].mean(axis=1)


def _scatter_scaled(N, locs, mats, scales):
    """Sum scales[g][e] * mats[g] into an N x N CSR at DoFs locs[g][e]."""
    rows, cols, vals = [], [], []
    for loc, mat, sc in zip(locs, mats, scales):
        nl = loc.shape[1]
        rows.append(np.repeat(loc, nl, axis=1).ravel())
        cols.append(np.tile(loc, (1, nl)).ravel())
        vals.append((sc[:, None] * mat.ravel()[None, :]).ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    A.sum_duplicates()
    A.sort_indices()
    return A


def assemble_weighted(mesh, k_elem):
    """K, M_k = m(.,.;k,0) = sum_e k_e^2 M_e, M (unit mass), B (unit boundary mass) and
    B_k = b(.,.;k) = sum_F k_F B_F for a wavenumber k_e per simplex; a boundary facet takes its
    owning simplex's value."""
    k_elem = np.asarray(k_elem, dtype=float)
    N = mesh.num_dofs
    K, M, B = assemble(mesh)
    groups = _group_by_shape(mesh, mesh.elem_verts, mesh.dim + 1)
    locs, Ms, sc = [], [], []
    for sel in groups:
        _, Me = element_matrices(mesh.coords[mesh.elem_verts[sel[0]]], mesh.order)
        locs.append(mesh.elems[sel])
        Ms.append(Me)
        sc.append(k_elem[sel] ** 2)
    Mk = _scatter_scaled(N, locs, Ms, sc)
    fgroups = _group_by_shape(mesh, mesh.facets, mesh.dim)
    flocs, Bs, fsc = [], [], []
    for sel in fgroups:
        flocs.append(mesh.facets[sel])
        Bs.append(facet_mass(mesh.coords[mesh.facets[sel[0]][:mesh.dim]], mesh.order))
        fsc.append(k_elem[mesh.facet_elems[sel]])
    Bk = _scatter_scaled(N, flocs, Bs, fsc)
    return K, Mk, M, B, Bk


def system_matrix_het(K, Mk, M, Bk, eps):
    """A(k, eps) = K - M(k, eps) - i B(k) with M(k, eps) = M_k + i eps M (eq. sys_matrix)."""
    return (K.astype(np.complex128) - Mk - 1j * eps * M - 1j * Bk).tocsr()


# ----------------------------------------------------------------------------
# Load vectors F_i = int f conj(phi_i) + int_dOmega g conj(phi_i)  (Sec. 2)
# ----------------------------------------------------------------------------


def load_from_nodal(mesh, M, f_nodal, g_facet_fn=None):
    """F = M I_h f + sum_facets B_F I_F g, with g evaluated per facet (its own normal).

    f is interpolated at the DoFs; g is interpolated on each boundary facet with
    that facet's outward normal, so a corner DoF receives g from each adjacent
    facet separately.
    """
    F = M @ np.asarray(f_nodal, dtype=np.complex128)
    if g_facet_fn is not None:
        for sel in _group_by_shape(mesh, mesh.facets, mesh.dim):
            loc = mesh.facets[sel]
            Be = facet_mass(mesh.coords[loc[0][:mesh.dim]], mesh.order)
            gl = g_facet_fn(mesh.coords[loc], mesh.facet_normals[sel])   # (F, nf)
            np.add.at(F, loc.ravel(), (gl @ Be.T).ravel())
    return F


def plane_wave(x, k, d):
    return np.exp(1j * k * (np.asarray(x) @ np.asarray(d)))


def load_planewave(mesh, M, k, theta):
    """Impedance data of u = exp(i k d.x), d = (cos t, sin t[, 0]): f = 0, g = i k (d.n - 1) u."""
    d = np.zeros(mesh.dim)
    d[0], d[1] = math.cos(theta), math.sin(theta)

    def g(xs, nrm):           # xs: (F, nf, dim), nrm: (F, dim)
        dn = nrm @ d
        return 1j * k * (dn[:, None] - 1.0) * plane_wave(xs, k, d)

    return load_from_nodal(mesh, M, np.zeros(mesh.num_dofs), g)


def load_gaussian(mesh, M, sigma, center=None):
    """Point-like source f = exp(-|x-x0|^2 / (2 sigma^2)), g = 0."""
    x0 = np.full(mesh.dim, 0.5) if center is None else np.asarray(center)
    r2 = np.sum((mesh.coords - x0) ** 2, axis=1)
    return load_from_nodal(mesh, M, np.exp(-r2 / (2.0 * sigma * sigma)))


# ----------------------------------------------------------------------------
# Canonical interpolation V_2h -> V_h (Sec. 4: the matrix I^{(l)}).
# ----------------------------------------------------------------------------


def prolongation(coarse, fine):
    """P[i, J] = coarse basis function J evaluated at fine DoF i (canonical interpolation).

    Fine DoFs are grouped by their position inside the containing coarse cell;
    for each group the containing coarse simplex and its basis values are
    found once from barycentric coordinates.
    """
    assert coarse.dim == fine.dim and coarse.order == fine.order and fine.n == 2 * coarse.n
    dim, order = fine.dim, fine.order
    basis, _ = lagrange_basis(dim, order)
    nc = coarse.n
    S = len(_simplices_of_cell(dim))
    x = fine.coords
    cell = np.minimum(np.floor(x * nc + 1e-9).astype(np.int64), nc - 1)
    xi = np.round((x * nc - cell) * 4 * order).astype(np.int64)   # local position, exact
    lin = np.zeros(x.shape[0], dtype=np.int64)
    for ax in range(dim):
        lin = lin * nc + cell[:, ax]
    keys, inv = np.unique(xi, axis=0, return_inverse=True)
    inv = inv.ravel()
    rows, cols, vals = [], [], []
    for g in range(keys.shape[0]):
        sel = np.nonzero(inv == g)[0]
        ref = sel[0]
        found = False
        for s in range(S):
            e = lin[ref] * S + s
            vx = coarse.coords[coarse.elem_verts[e]]
            T = np.ones((dim + 1, dim + 1))
            T[1:, :] = vx.T
            lam = np.linalg.solve(T, np.concatenate([[1.0], x[ref]]))
            if np.all(lam >= -1e-12):
                es = lin[sel] * S + s
                for j, phi in enumerate(basis):
                    w = _poly_eval(phi, lam)
                    if abs(w) > 1e-14:
                        rows.append(sel)
                        cols.append(coarse.elems[es, j])
                        vals.append(np.full(sel.shape[0], w))
                found = True
                break
        assert found, "fine DoF outside every coarse simplex"
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(fine.num_dofs, coarse.num_dofs))
    P.sum_duplicates()
    return P
