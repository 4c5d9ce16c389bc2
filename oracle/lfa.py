"""Local Fourier analysis (LFA) of the twogrid method for the shifted Helmholtz operator (Sec. 3).

TEST INFRASTRUCTURE (see oracle/__init__.py). CPU, complex128, one frequency at a time.

What it computes, for the local operator L_h(sigma) = K - (k^2 + i k^sigma) M on the infinite
uniform grid of spacing h (boundary conditions neglected, Eq. local_operator):
  * the Fourier symbol of a stencil, symbol(S, theta) = sum_kappa s_kappa exp(i theta . kappa)
    (Sec. 3, stencil notation and formal eigenfunctions);
  * the four harmonics theta^alpha of a low frequency theta, in the order
    alpha = (0,0), (1,1), (1,0), (0,1), with theta_i -> theta_i - pi (theta_i >= 0) or
    theta_i + pi (theta_i < 0) on the flipped axes;
  * the 4 x 4 representation of the twogrid error operator on the harmonic space,
    T_hat = S_hat^nu2 K_hat S_hat^nu1, K_hat = I - P_hat L_2h(2 theta)^-1 R_hat L_hat
    (Sec. 3, hat matrices), with diagonal L_hat and S_hat (damped Jacobi), a 4 x 1 prolongation
    column P_hat and a 1 x 4 restriction row R_hat;
  * rho_loc(sigma) = sup of the spectral radius of T_hat over the low frequencies
    T^low = (-pi/2, pi/2]^2, sampled on a uniform grid, or on the line theta_2 = 0 that Sec. 3
    restricts the search to, there with every sampled peak refined (Eq. def_conv);
  * sigma_c = inf{sigma in [1, 2] : rho_loc(sigma) < 1} (Sec. 3, I_conv = [sigma_c, 2]).

Discretisations (stencils of the assembled matrices, h factored out of the mass):
  * Q1 on squares, the paper's analysis (Sec. 3): stiffness (1/3)[-1 -1 -1; -1 8 -1; -1 -1 -1],
    mass (1/36)[1 4 1; 4 16 4; 1 4 1], bilinear interpolation;
  * P1 on Kuhn triangles (cells split along the (0,0)-(1,1) diagonal), the solver's 2D P1
    elements: stiffness 5-point [-1 -1 4 -1 -1] (the diagonal couplings vanish), mass (1/12)
    with 6 on the centre and 1 on the x, y and (1,1) neighbours, linear interpolation along the
    x, y and (1,1) edges.
The coarse operator is the rediscretisation on 2h (in 2D the stiffness stencil is scale-free and
the mass gains a factor 4).

Reading: Sec. 3 prints the prolongation column as (1 +- cos theta_1)(1 +- cos theta_2), four
times the symbol of bilinear interpolation, and the restriction row as a quarter of it, a quarter
of the symbol of P^T. Only the product P_hat R_hat enters T_hat and it equals that of P = the
interpolation and R = P^T, the transfers Algorithm 1 uses, so the symbols are taken as those of
P and P^T.
"""
import cmath
import math

import numpy as np

HARMONICS = ((0, 0), (1, 1), (1, 0), (0, 1))


class Stencils:
    """Stencils of one discretisation: offsets (dx, dy) -> coefficient."""

    def __init__(self, name, stiffness, mass, prolongation):
        self.name = name
        self.stiffness = stiffness
        self.mass = mass                  # per h^2
        self.prolongation = prolongation  # fine offset from a coarse point -> weight


def _square(c, e, k):
    """3 x 3 stencil with centre c, edge neighbours e and corner neighbours k."""
    s = {}
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            n = abs(dx) + abs(dy)
            s[(dx, dy)] = c if n == 0 else e if n == 1 else k
    return s


Q1 = Stencils(
    "Q1",
    stiffness={o: v / 3.0 for o, v in _square(8.0, -1.0, -1.0).items()},
    mass={o: v / 36.0 for o, v in _square(16.0, 4.0, 1.0).items()},
    prolongation={o: v / 4.0 for o, v in _square(4.0, 2.0, 1.0).items()},
)

_P1_NEIGHBOURS = ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1))
P1_KUHN = Stencils(
    "P1-Kuhn",
    stiffness={(0, 0): 4.0, (1, 0): -1.0, (-1, 0): -1.0, (0, 1): -1.0, (0, -1): -1.0},
    mass={(0, 0): 6.0 / 12.0, **{o: 1.0 / 12.0 for o in _P1_NEIGHBOURS}},
    prolongation={(0, 0): 1.0, **{o: 0.5 for o in _P1_NEIGHBOURS}},
)


def symbol(stencil, theta):
    """sum_kappa s_kappa exp(i theta . kappa)."""
    t1, t2 = theta
    return sum(v * cmath.exp(1j * (t1 * dx + t2 * dy)) for (dx, dy), v in stencil.items())


def shifted_lambda(k, sigma):
    """lambda = k^2 + i k^sigma (the shift eps = k^sigma, Sec. 3)."""
    return k * k + 1j * k ** sigma


def op_symbol(st, theta, lam, h):
    """Symbol of L_h = K - lambda M on the grid of spacing h."""
    return symbol(st.stiffness, theta) - lam * h * h * symbol(st.mass, theta)


def jacobi_symbol(st, theta, lam, h, omega):
    """Symbol of S_h = I - omega D_h^-1 L_h, D_h the (constant) diagonal of L_h."""
    d = st.stiffness[(0, 0)] - lam * h * h * st.mass[(0, 0)]
    return 1.0 - omega * op_symbol(st, theta, lam, h) / d


def bar(t):
    return t - math.pi if t >= 0 else t + math.pi


def harmonics(theta):
    """theta^alpha for alpha in HARMONICS."""
    t1, t2 = theta
    return [(bar(t1) if a1 else t1, bar(t2) if a2 else t2) for a1, a2 in HARMONICS]


def prolongation_symbol(st, theta_a):
    """Coefficient of phi_h(theta^alpha) in P phi_2h(2 theta): a quarter of the interpolation
    stencil's sum over the four parity classes of the fine offsets."""
    t1, t2 = theta_a
    return 0.25 * sum(v * cmath.exp(-1j * (t1 * dx + t2 * dy)) for (dx, dy), v in st.prolongation.items())


def restriction_symbol(st, theta_a):
    """R = P^T: R phi_h(theta^alpha) = symbol(P stencil, theta^alpha) phi_2h(2 theta)."""
    return symbol(st.prolongation, theta_a)


def twogrid_hat(st, theta, k, sigma, h, omega, nu1, nu2):
    """T_hat(theta, sigma) = S_hat^nu2 K_hat S_hat^nu1 on the harmonics of theta (Sec. 3)."""
    lam = shifted_lambda(k, sigma)
    th = harmonics(theta)
    L_hat = np.diag([op_symbol(st, t, lam, h) for t in th])
    S_hat = np.diag([jacobi_symbol(st, t, lam, h, omega) for t in th])
    P_hat = np.array([[prolongation_symbol(st, t)] for t in th])          # 4 x 1
    R_hat = np.array([[restriction_symbol(st, t) for t in th]])           # 1 x 4
    L2h = op_symbol(st, (2 * theta[0], 2 * theta[1]), lam, 2 * h)         # 1 x 1
    K_hat = np.eye(4) - P_hat @ R_hat @ L_hat / L2h
    return np.linalg.matrix_power(S_hat, nu2) @ K_hat @ np.linalg.matrix_power(S_hat, nu1)


def spectral_radius(T):
    return float(np.max(np.abs(np.linalg.eigvals(T))))


def low_frequencies(m, line=False, theta2=0.0):
    """Uniform sample of T^low = (-pi/2, pi/2]^2: m points per axis, pi/2 included;
    line=True keeps the line theta_2 = theta2 only."""
    axis = [-math.pi / 2 + math.pi * (j + 1) / m for j in range(m)]
    if line:
        return [(t, theta2) for t in axis]
    return [(t1, t2) for t1 in axis for t2 in axis]


def singular(st, theta, k, sigma, h, tol=1e-12):
    """theta in Lambda: L_h at a harmonic or L_2h at 2 theta (numerically) not invertible."""
    lam = shifted_lambda(k, sigma)
    vals = [op_symbol(st, t, lam, h) for t in harmonics(theta)]
    vals.append(op_symbol(st, (2 * theta[0], 2 * theta[1]), lam, 2 * h))
    return min(abs(v) for v in vals) <= tol


def golden_max(f, a, b, iters=60):
    """Maximum of f on [a, b] by golden-section search (Kiefer 1953): the bracket shrinks by
    1/phi per step around the larger interior value (exact for a unimodal f)."""
    g = (math.sqrt(5.0) - 1.0) / 2.0
    x1, x2 = b - g * (b - a), a + g * (b - a)
    f1, f2 = f(x1), f(x2)
    for _ in range(iters):
        if f1 >= f2:
            b, x2, f2 = x2, x1, f1
            x1 = b - g * (b - a)
            f1 = f(x1)
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + g * (b - a)
            f2 = f(x2)
    return max(f1, f2)


def rho_loc(st, k, sigma, h, omega, nu1, nu2, m=256, line=False, refine=True, theta2=0.0):
    """sup of rho(T_hat) over the low frequencies outside Lambda (Eq. def_conv).

    The spectral radius has sharp peaks near the frequencies where the fine or the coarse symbol
    nearly vanishes (their width shrinks with the shift), so on the line theta_2 = 0 every local
    maximum of the m-point sample is refined by golden-section search inside the bracket of its
    two neighbours (refine=True); theta2 moves the line to theta_2 = theta2. On all of T^low
    (line=False) the m x m sample is returned as it is."""
    pts = low_frequencies(m, line, theta2)
    r = lambda theta: (0.0 if singular(st, theta, k, sigma, h)  # noqa: E731
                       else spectral_radius(twogrid_hat(st, theta, k, sigma, h, omega, nu1, nu2)))
    vals = [r(theta) for theta in pts]
    best = max(vals)
    if line and refine:
        ts = [t for t, _ in pts]
        for i in range(len(ts)):
            left = vals[i - 1] if i > 0 else -1.0
            right = vals[i + 1] if i + 1 < len(ts) else -1.0
            if vals[i] >= left and vals[i] >= right:
                a = ts[i - 1] if i > 0 else -math.pi / 2
                b = ts[i + 1] if i + 1 < len(ts) else math.pi / 2
                best = max(best, golden_max(lambda t: r((t, theta2)), a, b))
    return best


def sigma_c(st, k, h, omega, nu1, nu2, m=256, line=True, steps=32, tol=1e-4):
    """inf{sigma in [1, 2] : rho_loc(sigma) < 1}: the first sigma of a uniform scan of [1, 2]
    (steps intervals) with rho_loc < 1, refined by bisection against its predecessor to tol.
    Returns 1.0 if rho_loc(1) < 1 and nan if no sampled sigma converges."""
    f = lambda s: rho_loc(st, k, s, h, omega, nu1, nu2, m, line)  # noqa: E731
    grid = [1.0 + j / steps for j in range(steps + 1)]
    prev = None
    for s in grid:
        if f(s) < 1.0:
            if prev is None:
                return 1.0
            lo, hi = prev, s
            while hi - lo > tol:
                mid = 0.5 * (lo + hi)
                if f(mid) < 1.0:
                    hi = mid
                else:
                    lo = mid
            return hi
        prev = s
    return float("nan")
