// Host-side setup of the matrix-free operators: per-class stencil
// coefficients of K, M, B (Sec. 2, eq. discreteproblem), prolongation weights
// of the canonical interpolation V_2h -> V_h (Sec. 4), and load vectors, for
// Lagrange P_p on simplices (the solver's elements) and tensor-product Q_p on
// squares / cubes (the paper's); per-DoF rows for a heterogeneous wavenumber
// with one value per element (Sec. 6); host inspection of all of these.
//
// Simplex integrals use Gauss-Legendre quadrature in collapsed (Duffy)
// coordinates on the reference simplex, exact for the polynomial degrees met
// here (<= 4 for the P2 mass matrix); tensor-product elements use exact 1D
// integrals. The stencil of each DoF class is read off a small reference mesh
// that contains every class at least once.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "common.cuh"

namespace helm {
namespace {

// Gauss-Legendre nodes/weights on [0,1] by Newton's method on P_n.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (t * p1 - p0) / (t * t - 1.0);
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);   // = 2/((1-t^2)P'^2) scaled by 1/2
  }
}

// Quadrature on the reference d-simplex: barycentric points, weights summing to 1.
struct Quad {
  std::vector<std::array<double, 4>> lam;
  std::vector<double> w;
};

Quad simplex_quadrature(int d) {
  std::vector<double> x, w;
  gauss_legendre01(4, x, w);
  Quad q;
  if (d == 1) {
    for (int i = 0; i < 4; ++i) {
      q.lam.push_back({1.0 - x[i], x[i], 0.0, 0.0});
      q.w.push_back(w[i]);
    }
  } else if (d == 2) {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        double xi = x[i], eta = x[j] * (1.0 - x[i]);
        q.lam.push_back({1.0 - xi - eta, xi, eta, 0.0});
        q.w.push_back(2.0 * w[i] * w[j] * (1.0 - x[i]));
      }
  } else {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        for (int k = 0; k < 4; ++k) {
          double xi = x[i], eta = x[j] * (1.0 - x[i]), zeta = x[k] * (1.0 - x[i]) * (1.0 - x[j]);
          q.lam.push_back({1.0 - xi - eta - zeta, xi, eta, zeta});
          q.w.push_back(6.0 * w[i] * w[j] * w[k] * (1.0 - x[i]) * (1.0 - x[i]) * (1.0 - x[j]));
        }
  }
  return q;
}

// Lagrange basis on a d-simplex: P1 = lam_i; P2 = vertices lam_i(2lam_i-1) then
// edge midpoints 4 lam_a lam_b over pairs (a<b) in lexicographic pair order.
int nbasis(int d, int order) { return order == 1 ? d + 1 : (d + 1) * (d + 2) / 2; }

void edge_pairs(int d, std::vector<std::pair<int, int>>& e) {
  e.clear();
  for (int a = 0; a <= d; ++a)
    for (int b = a + 1; b <= d; ++b) e.push_back({a, b});
}

double basis_val(int d, int order, int i, const double* lam) {
  if (order == 1) return lam[i];
  if (i <= d) return lam[i] * (2.0 * lam[i] - 1.0);
  std::vector<std::pair<int, int>> e;
  edge_pairs(d, e);
  auto ab = e[i - d - 1];
  return 4.0 * lam[ab.first] * lam[ab.second];
}

// d phi_i / d lam_a
double basis_dlam(int d, int order, int i, int a, const double* lam) {
  if (order == 1) return i == a ? 1.0 : 0.0;
  if (i <= d) return i == a ? 4.0 * lam[i] - 1.0 : 0.0;
  std::vector<std::pair<int, int>> e;
  edge_pairs(d, e);
  auto ab = e[i - d - 1];
  if (a == ab.first) return 4.0 * lam[ab.second];
  if (a == ab.second) return 4.0 * lam[ab.first];
  return 0.0;
}

// Barycentric node coordinates of local DoF i (vertex or edge midpoint).
std::array<double, 4> basis_node(int d, int order, int i) {
  std::array<double, 4> l = {0, 0, 0, 0};
  if (order == 1 || i <= d) {
    l[i] = 1.0;
    return l;
  }
  std::vector<std::pair<int, int>> e;
  edge_pairs(d, e);
  auto ab = e[i - d - 1];
  l[ab.first] = 0.5;
  l[ab.second] = 0.5;
  return l;
}

double det3(const double m[3][3]) {
  return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
         m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
         m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

// Element stiffness/mass on a full-dimensional simplex with vertices v[d+1][d].
void element_km(int d, int order, const double v[4][3], std::vector<double>& K,
                std::vector<double>& M) {
  int nb = nbasis(d, order);
  // Jacobian J = [v1-v0, ..., vd-v0] (columns); grad lam_a for a >= 1 are rows of J^{-1}
  double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int c = 0; c < d; ++c)
    for (int r = 0; r < d; ++r) J[r][c] = v[c + 1][r] - v[0][r];
  double det = d == 2 ? J[0][0] * J[1][1] - J[0][1] * J[1][0] : det3(J);
  double meas = std::fabs(det) / (d == 2 ? 2.0 : 6.0);
  double Ji[3][3] = {{0}};
  if (d == 2) {
    Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
  } else {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
        Ji[r][c] = (J[r1][c1] * J[r2][c2] - J[r1][c2] * J[r2][c1]) / det;
      }
  }
  double G[4][3] = {{0}};   // grad lam_a
  for (int a = 1; a <= d; ++a)
    for (int x = 0; x < d; ++x) G[a][x] = Ji[a - 1][x];
  for (int x = 0; x < d; ++x) {
    double s = 0;
    for (int a = 1; a <= d; ++a) s += G[a][x];
    G[0][x] = -s;
  }
  Quad q = simplex_quadrature(d);
  K.assign(nb * nb, 0.0);
  M.assign(nb * nb, 0.0);
  std::vector<double> phi(nb), grad(nb * 3);
  for (size_t p = 0; p < q.w.size(); ++p) {
    const double* lam = q.lam[p].data();
    for (int i = 0; i < nb; ++i) {
      phi[i] = basis_val(d, order, i, lam);
      for (int x = 0; x < 3; ++x) grad[i * 3 + x] = 0.0;
      for (int a = 0; a <= d; ++a) {
        double da = basis_dlam(d, order, i, a, lam);
        for (int x = 0; x < d; ++x) grad[i * 3 + x] += da * G[a][x];
      }
    }
    double wq = q.w[p] * meas;
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        double gg = 0;
        for (int x = 0; x < d; ++x) gg += grad[i * 3 + x] * grad[j * 3 + x];
        K[i * nb + j] += wq * gg;
        M[i * nb + j] += wq * phi[i] * phi[j];
      }
  }
}

// Mass matrix of a (d-1)-facet with vertices v[d][3] embedded in R^d.
void facet_mass(int d, int order, const double v[4][3], std::vector<double>& B) {
  int fd = d - 1;
  int nb = nbasis(fd, order);
  double meas;
  if (fd == 1) {
    double dx = v[1][0] - v[0][0], dy = v[1][1] - v[0][1];
    meas = std::sqrt(dx * dx + dy * dy);
  } else {
    double a[3], b[3];
    for (int x = 0; x < 3; ++x) { a[x] = v[1][x] - v[0][x]; b[x] = v[2][x] - v[0][x]; }
    double c0 = a[1] * b[2] - a[2] * b[1], c1 = a[2] * b[0] - a[0] * b[2], c2 = a[0] * b[1] - a[1] * b[0];
    meas = 0.5 * std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  }
  Quad q = simplex_quadrature(fd);
  B.assign(nb * nb, 0.0);
  for (size_t p = 0; p < q.w.size(); ++p) {
    const double* lam = q.lam[p].data();
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j)
        B[i * nb + j] += q.w[p] * meas * basis_val(fd, order, i, lam) * basis_val(fd, order, j, lam);
  }
}

// ---------------------------------------------------------------------------
// Structured mesh enumeration: cells of n^d, split into simplices.
// 2D: {(0,0),(1,0),(1,1)} and {(0,0),(1,1),(0,1)}; 3D: Kuhn, one tetrahedron
// per axis permutation along the path (0,0,0) -> ... -> (1,1,1).
// ---------------------------------------------------------------------------
void cell_simplices(int d, std::vector<std::array<std::array<int, 3>, 4>>& out) {
  out.clear();
  if (d == 2) {
    out.push_back({{{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 0, 0}}});
    out.push_back({{{0, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 0}}});
    return;
  }
  int perm[3] = {0, 1, 2};
  std::sort(perm, perm + 3);
  do {
    std::array<std::array<int, 3>, 4> s;
    std::array<int, 3> p = {0, 0, 0};
    s[0] = p;
    for (int k = 0; k < 3; ++k) {
      p[perm[k]] += 1;
      s[k + 1] = p;
    }
    out.push_back(s);
  } while (std::next_permutation(perm, perm + 3));
}

struct SMesh {
  int d, order, n, W;
  double h;
  int elements = HELM_SIMPLICES;   // or HELM_TENSOR: one square / cube element per cell
  int64_t idx(const int* c) const {
    int64_t s = 0;
    for (int ax = d - 1; ax >= 0; --ax) s = s * W + c[ax];
    return s;
  }
};

// Calls fn(local DoF lattice coords [nb][3], vertex coords [d+1][3]) per element.
template <typename Fn> void for_each_element(const SMesh& m, Fn fn) {
  std::vector<std::array<std::array<int, 3>, 4>> simp;
  cell_simplices(m.d, simp);
  int nb = nbasis(m.d, m.order);
  int nc3 = m.d == 3 ? m.n : 1;
  std::vector<std::array<int, 3>> loc(nb);
  double vx[4][3];
  for (int cz = 0; cz < nc3; ++cz)
    for (int cy = 0; cy < m.n; ++cy)
      for (int cx = 0; cx < m.n; ++cx)
        for (auto& s : simp) {
          int cell[3] = {cx, cy, cz};
          for (int i = 0; i < nb; ++i) {
            auto l = basis_node(m.d, m.order, i);
            for (int ax = 0; ax < 3; ++ax) {
              double p = 0;
              for (int a = 0; a <= m.d; ++a) p += l[a] * (cell[ax] + s[a][ax]) * m.order;
              loc[i][ax] = (int)std::lround(p);
            }
          }
          for (int a = 0; a <= m.d; ++a)
            for (int ax = 0; ax < 3; ++ax) vx[a][ax] = (cell[ax] + s[a][ax]) * m.h;
          fn(loc, vx);
        }
}

// Calls fn(facet DoF lattice coords, facet vertex coords [d][3], outward normal[3], owner) per
// boundary facet; owner = the simplex's index in for_each_element's order.
template <typename Fn> void for_each_boundary_facet(const SMesh& m, Fn fn) {
  std::vector<std::array<std::array<int, 3>, 4>> simp;
  cell_simplices(m.d, simp);
  int fd = m.d - 1;
  int nfb = nbasis(fd, m.order);
  int nc3 = m.d == 3 ? m.n : 1;
  std::vector<std::array<int, 3>> loc(nfb);
  double vx[4][3];
  for (int cz = 0; cz < nc3; ++cz)
    for (int cy = 0; cy < m.n; ++cy)
      for (int cx = 0; cx < m.n; ++cx) {
        int cell[3] = {cx, cy, cz};
        bool bnd = false;
        for (int ax = 0; ax < m.d; ++ax) bnd |= (cell[ax] == 0 || cell[ax] == m.n - 1);
        if (!bnd) continue;
        for (size_t si = 0; si < simp.size(); ++si) {
          const auto& s = simp[si];
          const int64_t owner = ((int64_t)(cz * m.n + cy) * m.n + cx) * (int64_t)simp.size() + (int64_t)si;
          // faces: drop one vertex
          for (int drop = 0; drop <= m.d; ++drop) {
            int fv[3][3];
            int c = 0;
            for (int a = 0; a <= m.d; ++a)
              if (a != drop) {
                for (int ax = 0; ax < 3; ++ax) fv[c][ax] = cell[ax] + s[a][ax];
                ++c;
              }
            for (int ax = 0; ax < m.d; ++ax)
              for (int side = 0; side < 2; ++side) {
                int val = side == 0 ? 0 : m.n;
                bool on = true;
                for (int v = 0; v < m.d; ++v) on &= (fv[v][ax] == val);
                if (!on) continue;
                for (int i = 0; i < nfb; ++i) {
                  auto l = basis_node(fd, m.order, i);
                  for (int x = 0; x < 3; ++x) {
                    double p = 0;
                    for (int a = 0; a < m.d; ++a) p += l[a] * fv[a][x] * m.order;
                    loc[i][x] = (int)std::lround(p);
                  }
                }
                for (int a = 0; a < m.d; ++a)
                  for (int x = 0; x < 3; ++x) vx[a][x] = fv[a][x] * m.h;
                double nrm[3] = {0, 0, 0};
                nrm[ax] = side == 0 ? -1.0 : 1.0;
                fn(loc, vx, nrm, owner);
              }
          }
        }
      }
}

// ---------------------------------------------------------------------------
// Tensor-product Q_p elements: 1D Lagrange basis on [0, 1] at the Gauss-Lobatto points (0, 1
// and the roots of P_p'; equispaced for p <= 2, 1/2 -+ sqrt(5)/10 inside for p = 3), 1D element
// matrices on [0, h] integrated exactly by 4-point Gauss-Legendre (degree <= 6 for p <= 3),
// element matrices as tensor products with the local index x fastest (l = sum_ax l_ax (p+1)^ax).
// ---------------------------------------------------------------------------
double gll01(int p, int l) {
  if (p == 3 && (l == 1 || l == 2)) return l == 1 ? 0.5 - std::sqrt(5.0) / 10.0 : 0.5 + std::sqrt(5.0) / 10.0;
  return (double)l / p;
}
double lagrange1(int p, int l, double x) {
  double v = 1.0;
  for (int j = 0; j <= p; ++j)
    if (j != l) v *= (x - gll01(p, j)) / (gll01(p, l) - gll01(p, j));
  return v;
}
double lagrange1_d(int p, int l, double x) {
  double den = 1.0, s = 0.0;
  for (int j = 0; j <= p; ++j)
    if (j != l) den *= gll01(p, l) - gll01(p, j);
  for (int m = 0; m <= p; ++m) {
    if (m == l) continue;
    double t = 1.0;
    for (int j = 0; j <= p; ++j)
      if (j != l && j != m) t *= x - gll01(p, j);
    s += t;
  }
  return s / den;
}
void element_1d(int p, double h, std::vector<double>& K1, std::vector<double>& M1) {
  std::vector<double> x, w;
  gauss_legendre01(4, x, w);
  const int nb = p + 1;
  K1.assign(nb * nb, 0.0);
  M1.assign(nb * nb, 0.0);
  for (size_t q = 0; q < x.size(); ++q)
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        K1[i * nb + j] += w[q] * lagrange1_d(p, i, x[q]) * lagrange1_d(p, j, x[q]) / h;
        M1[i * nb + j] += w[q] * lagrange1(p, i, x[q]) * lagrange1(p, j, x[q]) * h;
      }
}
// local index l -> per-axis indices (x fastest)
void split_local(int l, int nb1, int dims, int* la) {
  for (int ax = 0; ax < dims; ++ax) {
    la[ax] = l % nb1;
    l /= nb1;
  }
}
// tensor-product stiffness / mass of a d-cube and mass of a (d-1)-face
void element_km_tensor(int d, int p, double h, std::vector<double>& K, std::vector<double>& M) {
  std::vector<double> K1, M1;
  element_1d(p, h, K1, M1);
  const int nb1 = p + 1;
  int nb = 1;
  for (int ax = 0; ax < d; ++ax) nb *= nb1;
  K.assign((size_t)nb * nb, 0.0);
  M.assign((size_t)nb * nb, 0.0);
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      int li[3], lj[3];
      split_local(i, nb1, d, li);
      split_local(j, nb1, d, lj);
      double mass = 1.0, stiff = 0.0;
      for (int ax = 0; ax < d; ++ax) {
        double term = K1[li[ax] * nb1 + lj[ax]];
        for (int bx = 0; bx < d; ++bx)
          if (bx != ax) term *= M1[li[bx] * nb1 + lj[bx]];
        stiff += term;
        mass *= M1[li[ax] * nb1 + lj[ax]];
      }
      K[(size_t)i * nb + j] = stiff;
      M[(size_t)i * nb + j] = mass;
    }
}
void face_mass_tensor(int d, int p, double h, std::vector<double>& B) {
  std::vector<double> K1, M1;
  element_1d(p, h, K1, M1);
  const int nb1 = p + 1, fd = d - 1;
  int nb = 1;
  for (int ax = 0; ax < fd; ++ax) nb *= nb1;
  B.assign((size_t)nb * nb, 0.0);
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      int li[3], lj[3];
      split_local(i, nb1, fd, li);
      split_local(j, nb1, fd, lj);
      double v = 1.0;
      for (int ax = 0; ax < fd; ++ax) v *= M1[li[ax] * nb1 + lj[ax]];
      B[(size_t)i * nb + j] = v;
    }
}

// Every element with its matrices: fn(local DoF lattice coords, Ke, Me).
template <typename Fn> void for_each_element_km(const SMesh& m, Fn fn) {
  if (m.elements == HELM_SIMPLICES) {
    std::vector<double> Ke, Me;
    for_each_element(m, [&](const std::vector<std::array<int, 3>>& loc, const double (*vx)[3]) {
      element_km(m.d, m.order, vx, Ke, Me);
      fn(loc, Ke, Me);
    });
    return;
  }
  std::vector<double> Ke, Me;
  element_km_tensor(m.d, m.order, m.h, Ke, Me);
  const int nb1 = m.order + 1;
  int nb = 1;
  for (int ax = 0; ax < m.d; ++ax) nb *= nb1;
  std::vector<std::array<int, 3>> loc(nb);
  const int nc3 = m.d == 3 ? m.n : 1;
  for (int cz = 0; cz < nc3; ++cz)
    for (int cy = 0; cy < m.n; ++cy)
      for (int cx = 0; cx < m.n; ++cx) {
        const int cell[3] = {cx, cy, cz};
        for (int l = 0; l < nb; ++l) {
          int la[3] = {0, 0, 0};
          split_local(l, nb1, m.d, la);
          for (int ax = 0; ax < 3; ++ax) loc[l][ax] = ax < m.d ? cell[ax] * m.order + la[ax] : 0;
        }
        fn(loc, Ke, Me);
      }
}

// Every boundary facet with its mass matrix: fn(facet DoF lattice coords, Be, outward normal,
// owning element in for_each_element_km's order).
template <typename Fn> void for_each_facet_mass(const SMesh& m, Fn fn) {
  if (m.elements == HELM_SIMPLICES) {
    std::vector<double> Be;
    for_each_boundary_facet(m, [&](const std::vector<std::array<int, 3>>& loc, const double (*vx)[3],
                                   const double* nrm, int64_t owner) {
      facet_mass(m.d, m.order, vx, Be);
      fn(loc, Be, nrm, owner);
    });
    return;
  }
  std::vector<double> Be;
  face_mass_tensor(m.d, m.order, m.h, Be);
  const int nb1 = m.order + 1, fd = m.d - 1;
  int nb = 1;
  for (int ax = 0; ax < fd; ++ax) nb *= nb1;
  std::vector<std::array<int, 3>> loc(nb);
  const int nc3 = m.d == 3 ? m.n : 1;
  for (int cz = 0; cz < nc3; ++cz)
    for (int cy = 0; cy < m.n; ++cy)
      for (int cx = 0; cx < m.n; ++cx) {
        const int cell[3] = {cx, cy, cz};
        for (int ax = 0; ax < m.d; ++ax)
          for (int side = 0; side < 2; ++side) {
            if (cell[ax] != (side == 0 ? 0 : m.n - 1)) continue;
            int others[2] = {0, 0}, no = 0;
            for (int bx = 0; bx < m.d; ++bx)
              if (bx != ax) others[no++] = bx;
            for (int l = 0; l < nb; ++l) {
              int la[3] = {0, 0, 0};
              split_local(l, nb1, fd, la);
              for (int bx = 0; bx < 3; ++bx) loc[l][bx] = 0;
              loc[l][ax] = cell[ax] * m.order + (side == 0 ? 0 : m.order);
              for (int k = 0; k < fd; ++k) loc[l][others[k]] = cell[others[k]] * m.order + la[k];
            }
            double nrm[3] = {0, 0, 0};
            nrm[ax] = side == 0 ? -1.0 : 1.0;
            fn(loc, Be, nrm, ((int64_t)cz * m.n + cy) * m.n + cx);
          }
      }
}

// Dense assembly of K, M, B on a small mesh.
void assemble_dense(const SMesh& m, std::vector<double>& K, std::vector<double>& M,
                    std::vector<double>& B) {
  int64_t N = 1;
  for (int ax = 0; ax < m.d; ++ax) N *= m.W;
  K.assign(N * N, 0.0);
  M.assign(N * N, 0.0);
  B.assign(N * N, 0.0);
  for_each_element_km(m, [&](const std::vector<std::array<int, 3>>& loc, const std::vector<double>& Ke,
                             const std::vector<double>& Me) {
    int nb = (int)loc.size();
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        int64_t r = m.idx(loc[i].data()), c = m.idx(loc[j].data());
        K[r * N + c] += Ke[i * nb + j];
        M[r * N + c] += Me[i * nb + j];
      }
  });
  for_each_facet_mass(m, [&](const std::vector<std::array<int, 3>>& loc, const std::vector<double>& Be,
                             const double*, int64_t) {
    int nb = (int)loc.size();
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        int64_t r = m.idx(loc[i].data()), c = m.idx(loc[j].data());
        B[r * N + c] += Be[i * nb + j];
      }
  });
}

// Representative lattice index (on a reference lattice of Wr points) of axis class c.
int class_rep(int c, int Wr, int R, int q) {
  if (c < R) return c;
  if (c >= R + q) return Wr - R + (c - R - q);
  int p = c - R;
  for (int a = R; a < Wr - R; ++a)
    if (a % q == p) return a;
  return -1;
}

void level_stencils(int d, int order, int n, GridDesc& g, std::vector<double>& Ks,
                    std::vector<double>& Ms, std::vector<double>& Bs, int& ncls,
                    int elements = HELM_SIMPLICES) {
  g.dim = d;
  g.R = order;
  g.q = order;
  g.W = order * n + 1;
  g.C1 = 2 * g.R + g.q;
  g.noff = 1;
  g.N = 1;
  for (int ax = 0; ax < d; ++ax) {
    g.noff *= 2 * g.R + 1;
    g.N *= g.W;
  }
  ncls = 1;
  for (int ax = 0; ax < d; ++ax) ncls *= g.C1;
  // reference mesh: smallest n_ref with a full interior period
  int nref = order == 1 ? 2 : 4;
  nref = std::min(nref, n);
  SMesh rm{d, order, nref, order * nref + 1, 1.0 / n, elements};   // same h as the target level
  std::vector<double> K, M, B;
  assemble_dense(rm, K, M, B);
  int64_t Nr = 1;
  for (int ax = 0; ax < d; ++ax) Nr *= rm.W;
  Ks.assign((size_t)ncls * g.noff, 0.0);
  Ms.assign((size_t)ncls * g.noff, 0.0);
  Bs.assign((size_t)ncls * g.noff, 0.0);
  int side = 2 * g.R + 1;
  for (int cls = 0; cls < ncls; ++cls) {
    int cc[3] = {0, 0, 0}, rep[3] = {0, 0, 0};
    int t = cls;
    bool ok = true;
    for (int ax = 0; ax < d; ++ax) {
      cc[ax] = t % g.C1;
      t /= g.C1;
      // a class only exists on the target lattice if it has a member there
      rep[ax] = class_rep(cc[ax], rm.W, g.R, g.q);
      if (rep[ax] < 0) ok = false;
    }
    if (!ok) continue;
    int64_t r = rm.idx(rep);
    for (int o = 0; o < g.noff; ++o) {
      int oo = o, nb[3] = {0, 0, 0};
      bool in = true;
      for (int ax = 0; ax < d; ++ax) {
        int dxx = oo % side - g.R;
        oo /= side;
        nb[ax] = rep[ax] + dxx;
        if (nb[ax] < 0 || nb[ax] >= rm.W) in = false;
      }
      if (!in) continue;
      int64_t c = rm.idx(nb);
      Ks[(size_t)cls * g.noff + o] = K[r * Nr + c];
      Ms[(size_t)cls * g.noff + o] = M[r * Nr + c];
      Bs[(size_t)cls * g.noff + o] = B[r * Nr + c];
    }
  }
}

}  // namespace

int build_tables(int d, int order, int n, HostTables* t, int elements) {
  const bool q3 = elements == HELM_TENSOR && d == 2 && order == 3;   // host tables only
  if (!(d == 2 || d == 3) || !(order == 1 || order == 2 || q3) || (d == 3 && order != 1)) return HELM_EINVAL;
  if (n < 4 || n % 2) return HELM_EINVAL;
  if (elements != HELM_SIMPLICES && elements != HELM_TENSOR) return HELM_EINVAL;
  level_stencils(d, order, n, t->fine, t->Kf, t->Mf, t->Bf, t->ncls_f, elements);
  level_stencils(d, order, n / 2, t->coarse, t->Kc, t->Mc, t->Bc, t->ncls_c, elements);
  // prolongation weights: evaluate coarse basis functions at fine positions
  int q = order;
  t->pf = 2 * q;
  t->npc = 1;
  t->npo = 1;
  for (int ax = 0; ax < d; ++ax) {
    t->npc *= t->pf;
    t->npo *= q + 1;
  }
  t->pw.assign((size_t)t->npc * t->npo, 0.0);
  if (elements == HELM_TENSOR) {
    // Q_p: the coarse basis at fine position class c is the product of 1D Lagrange values at
    // xi_ax = (c_ax / pf) in the coarse cell; coarse local node l is the box offset o = l
    for (int c = 0; c < t->npc; ++c) {
      double xi[3] = {0, 0, 0};
      int tt = c;
      for (int ax = 0; ax < d; ++ax) {
        const int cc = tt % t->pf;   // fine sub-cell cc / q, its local point cc % q
        xi[ax] = (cc / q + gll01(q, cc % q)) / 2.0;
        tt /= t->pf;
      }
      for (int o = 0; o < t->npo; ++o) {
        int la[3] = {0, 0, 0};
        split_local(o, q + 1, d, la);
        double wv = 1.0;
        for (int ax = 0; ax < d; ++ax) wv *= lagrange1(q, la[ax], xi[ax]);
        if (std::fabs(wv) >= 1e-15) t->pw[(size_t)c * t->npo + o] = wv;
      }
    }
    return HELM_OK;
  }
  std::vector<std::array<std::array<int, 3>, 4>> simp;
  cell_simplices(d, simp);
  int nb = nbasis(d, order);
  for (int c = 0; c < t->npc; ++c) {
    double xi[3] = {0, 0, 0};   // position in the coarse cell, [0,1)
    int tt = c;
    for (int ax = 0; ax < d; ++ax) {
      xi[ax] = (double)(tt % t->pf) / t->pf;
      tt /= t->pf;
    }
    bool found = false;
    for (auto& s : simp) {
      // barycentric coords of xi in simplex s (unit cell coords)
      double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, rhs[3] = {0, 0, 0};
      for (int col = 0; col < d; ++col)
        for (int r = 0; r < d; ++r) J[r][col] = s[col + 1][r] - s[0][r];
      for (int r = 0; r < d; ++r) rhs[r] = xi[r] - s[0][r];
      double lam[4] = {0, 0, 0, 0};
      if (d == 2) {
        double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        lam[1] = (rhs[0] * J[1][1] - J[0][1] * rhs[1]) / det;
        lam[2] = (J[0][0] * rhs[1] - rhs[0] * J[1][0]) / det;
      } else {
        double det = det3(J);
        for (int col = 0; col < 3; ++col) {
          double Jc[3][3];
          for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) Jc[r][cc] = cc == col ? rhs[r] : J[r][cc];
          lam[col + 1] = det3(Jc) / det;
        }
      }
      double s0 = 1.0;
      for (int a = 1; a <= d; ++a) s0 -= lam[a];
      lam[0] = s0;
      bool inside = true;
      for (int a = 0; a <= d; ++a) inside &= lam[a] >= -1e-12;
      if (!inside) continue;
      for (int i = 0; i < nb; ++i) {
        double wv = basis_val(d, order, i, lam);
        if (std::fabs(wv) < 1e-15) continue;
        auto l = basis_node(d, order, i);
        int o = 0, mul = 1;
        for (int ax = 0; ax < d; ++ax) {
          double p = 0;
          for (int a = 0; a <= d; ++a) p += l[a] * s[a][ax] * q;
          o += (int)std::lround(p) * mul;
          mul *= q + 1;
        }
        t->pw[(size_t)c * t->npo + o] = wv;
      }
      found = true;
      break;
    }
    if (!found) return HELM_EINVAL;
  }
  return HELM_OK;
}

int64_t num_elements(int d, int n, int elements) {
  int64_t c = 1;
  for (int ax = 0; ax < d; ++ax) c *= n;
  return elements == HELM_TENSOR ? c : c * (d == 2 ? 2 : 6);
}

int build_het_rows(int d, int order, int n, int elements, const double* k_elem, HetRows* out) {
  const bool q3 = elements == HELM_TENSOR && d == 2 && order == 3;
  if (!(d == 2 || d == 3) || !(order == 1 || order == 2 || q3) || (d == 3 && order != 1) || n < 2)
    return HELM_EINVAL;
  if (elements != HELM_SIMPLICES && elements != HELM_TENSOR) return HELM_EINVAL;
  SMesh m{d, order, n, order * n + 1, 1.0 / n, elements};
  GridDesc& g = out->g;
  g.dim = d;
  g.R = order;
  g.q = order;
  g.W = m.W;
  g.C1 = 2 * g.R + g.q;
  g.noff = 1;
  g.N = 1;
  for (int ax = 0; ax < d; ++ax) {
    g.noff *= 2 * g.R + 1;
    g.N *= g.W;
  }
  const size_t total = (size_t)g.N * g.noff;
  out->K.assign(total, 0.0);
  out->Mk.assign(total, 0.0);
  out->M.assign(total, 0.0);
  out->Bk.assign(total, 0.0);
  const int side = 2 * g.R + 1;
  auto box = [&](const std::array<int, 3>& a, const std::array<int, 3>& b) {
    int o = 0, mul = 1;
    for (int ax = 0; ax < d; ++ax) {
      o += (b[ax] - a[ax] + g.R) * mul;
      mul *= side;
    }
    return o;
  };
  int64_t e = 0;
  for_each_element_km(m, [&](const std::vector<std::array<int, 3>>& loc, const std::vector<double>& Ke,
                             const std::vector<double>& Me) {
    const double k2 = k_elem[e] * k_elem[e];
    ++e;
    const int nb = (int)loc.size();
    for (int i = 0; i < nb; ++i) {
      const size_t r = (size_t)m.idx(loc[i].data()) * g.noff;
      for (int j = 0; j < nb; ++j) {
        const size_t c = r + box(loc[i], loc[j]);
        out->K[c] += Ke[i * nb + j];
        out->M[c] += Me[i * nb + j];
        out->Mk[c] += k2 * Me[i * nb + j];
      }
    }
  });
  for_each_facet_mass(m, [&](const std::vector<std::array<int, 3>>& loc, const std::vector<double>& Be,
                             const double*, int64_t owner) {
    const double kf = k_elem[owner];
    const int nb = (int)loc.size();
    for (int i = 0; i < nb; ++i) {
      const size_t r = (size_t)m.idx(loc[i].data()) * g.noff;
      for (int j = 0; j < nb; ++j) out->Bk[r + box(loc[i], loc[j])] += kf * Be[i * nb + j];
    }
  });
  return HELM_OK;
}

// Host inspection of the tables, with the kernels' own class and transfer mapping.
int host_stencil_row(const HostTables& t, int level, int64_t dof, double* K, double* M, double* B) {
  const GridDesc& g = level == 0 ? t.fine : t.coarse;
  const std::vector<double>& Kt = level == 0 ? t.Kf : t.Kc;
  const std::vector<double>& Mt = level == 0 ? t.Mf : t.Mc;
  const std::vector<double>& Bt = level == 0 ? t.Bf : t.Bc;
  if (dof < 0 || dof >= g.N) return HELM_EINVAL;
  int a[3] = {0, 0, 0};
  int64_t r = dof;
  int cls = 0, mul = 1;
  for (int ax = 0; ax < g.dim; ++ax) {
    a[ax] = (int)(r % g.W);
    r /= g.W;
    cls += axis_class(a[ax], g.W, g.R, g.q) * mul;
    mul *= g.C1;
  }
  const int side = 2 * g.R + 1;
  for (int o = 0; o < g.noff; ++o) {
    int oo = o;
    bool in = true;
    for (int ax = 0; ax < g.dim; ++ax) {
      const int b = a[ax] + oo % side - g.R;
      oo /= side;
      in &= b >= 0 && b < g.W;
    }
    const size_t i = (size_t)cls * g.noff + o;
    K[o] = in ? Kt[i] : 0.0;
    M[o] = in ? Mt[i] : 0.0;
    B[o] = in ? Bt[i] : 0.0;
  }
  return HELM_OK;
}

int host_prolongation_row(const HostTables& t, int64_t fine_dof, int64_t* cols, double* w, int* count) {
  const GridDesc &f = t.fine, &c = t.coarse;
  if (fine_dof < 0 || fine_dof >= f.N) return HELM_EINVAL;
  int a[3] = {0, 0, 0}, anc[3] = {0, 0, 0};
  int64_t r = fine_dof;
  int cls = 0, mul = 1;
  for (int ax = 0; ax < f.dim; ++ax) {
    a[ax] = (int)(r % f.W);
    r /= f.W;
    cls += mod_period(a[ax], t.pf) * mul;
    mul *= t.pf;
    anc[ax] = div_period(a[ax], t.pf) * c.q;
  }
  int n = 0;
  for (int o = 0; o < t.npo; ++o) {
    const double wv = t.pw[(size_t)cls * t.npo + o];
    if (wv == 0.0) continue;
    int oo = o;
    int64_t col = 0, st = 1;
    for (int ax = 0; ax < f.dim; ++ax) {
      const int A = anc[ax] + oo % (c.q + 1);
      oo /= c.q + 1;
      if (A < 0 || A >= c.W) return HELM_EINVAL;   // a nonzero weight outside the coarse lattice
      col += (int64_t)A * st;
      st *= c.W;
    }
    cols[n] = col;
    w[n] = wv;
    ++n;
  }
  *count = n;
  return HELM_OK;
}

// Coordinate of lattice index a along an axis: element a / order, local point a % order at the
// element's interpolation node (equispaced for P_p and Q1, Q2; Gauss-Lobatto for Q3).
static double lattice_coord(int a, int order, double h, int elements) {
  if (elements == HELM_TENSOR && order == 3) return (a / 3 + gll01(3, a % 3)) * h;
  return (double)a * h / order;
}

void rhs_planewave(int d, int order, int n, double k, double theta, double2* F, int elements) {
  SMesh m{d, order, n, order * n + 1, 1.0 / n, elements};
  int64_t N = 1;
  for (int ax = 0; ax < d; ++ax) N *= m.W;
  std::memset(F, 0, sizeof(double2) * N);
  double dir[3] = {std::cos(theta), std::sin(theta), 0.0};
  for_each_facet_mass(m, [&](const std::vector<std::array<int, 3>>& loc, const std::vector<double>& Be,
                             const double* nrm, int64_t) {
    int nb = (int)loc.size();
    double dn = dir[0] * nrm[0] + dir[1] * nrm[1] + dir[2] * nrm[2];
    for (int j = 0; j < nb; ++j) {
      double ph = 0;
      for (int ax = 0; ax < d; ++ax) ph += dir[ax] * lattice_coord(loc[j][ax], order, m.h, elements);
      // g = i k (d.n - 1) exp(i k d.x)
      double gr = -k * (dn - 1.0) * std::sin(k * ph), gi = k * (dn - 1.0) * std::cos(k * ph);
      for (int i = 0; i < nb; ++i) {
        int64_t r = m.idx(loc[i].data());
        F[r].x += Be[i * nb + j] * gr;
        F[r].y += Be[i * nb + j] * gi;
      }
    }
  });
}

void rhs_gaussian(int d, int order, int n, double sigma, const double* c, double2* F, int elements) {
  GridDesc g;
  std::vector<double> Ks, Ms, Bs;
  int ncls;
  level_stencils(d, order, n, g, Ks, Ms, Bs, ncls, elements);
  const double he = 1.0 / n;
  int W = g.W, side = 2 * g.R + 1;
  std::vector<double> f(g.N);
  for (int64_t p = 0; p < g.N; ++p) {
    int64_t t = p;
    double r2 = 0;
    for (int ax = 0; ax < d; ++ax) {
      double x = lattice_coord((int)(t % W), order, he, elements) - c[ax];
      t /= W;
      r2 += x * x;
    }
    f[p] = std::exp(-r2 / (2.0 * sigma * sigma));
  }
  for (int64_t p = 0; p < g.N; ++p) {
    int a[3] = {0, 0, 0};
    int64_t t = p;
    int cls = 0, mul = 1;
    for (int ax = 0; ax < d; ++ax) {
      a[ax] = (int)(t % W);
      t /= W;
      cls += axis_class(a[ax], W, g.R, g.q) * mul;
      mul *= g.C1;
    }
    double s = 0;
    for (int o = 0; o < g.noff; ++o) {
      double coef = Ms[(size_t)cls * g.noff + o];
      if (coef == 0.0) continue;
      int oo = o;
      int64_t idx = 0, st = 1;
      for (int ax = 0; ax < d; ++ax) {
        int b = a[ax] + oo % side - g.R;
        oo /= side;
        idx += (int64_t)b * st;
        st *= W;
      }
      s += coef * f[idx];
    }
    F[p] = make_double2(s, 0.0);
  }
}

}  // namespace helm
