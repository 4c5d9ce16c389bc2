"""Algebraic identities the GPU kernels rely on, checked on small dense models (CPU).

* The coarse solve of the complex64 form runs each half-sweep of the twisted block
  elimination as a segmented recurrence (k_seg_chain phases A and B, k_seg_fixup phase C,
  k_seg_middle): the model below follows the same index logic (paths, segment lengths, segment
  ends, products by block) and must reproduce a dense solve of the block-tridiagonal system.
* The Arnoldi process is lagged classical Gram-Schmidt with reorthogonalisation and lagged
  normalisation (k_dots2, k_coef, k_update2): the model below follows the same state machine
  (column j-1 finished at step j, a final step that only finishes the last column, z_j scaled by
  1/rho_j) and must give the residual history and iteration count of a textbook FGMRES with
  modified Gram-Schmidt.
"""
import numpy as np
import pytest


# ---------------------------------------------------------------- segmented twisted solve

def _make_path(J0, step, n, kmax, kc0):
    k0 = max(1, min(kmax, n))
    ls = (n + k0 - 1) // k0
    return dict(J0=J0, step=step, n=n, Ls=ls, K=(n + ls - 1) // ls, kc0=kc0)


def _seg_end(k, ls, n):
    return min((k + 1) * ls, n) - 1


def _blk(p, q):
    return p["J0"] + p["step"] * q


def _segmented_twisted_solve(D, Lo, Uo, r, kp):
    nb, B = len(D), D[0].shape[0]
    m = nb // 2
    dinv = [None] * nb
    for J in range(m):                                   # top chain
        S = D[J] if J == 0 else D[J] - Lo[J] @ dinv[J - 1] @ Uo[J - 1]
        dinv[J] = np.linalg.inv(S)
    for J in range(nb - 1, m, -1):                       # bottom chain
        S = D[J] if J == nb - 1 else D[J] - Uo[J] @ dinv[J + 1] @ Lo[J + 1]
        dinv[J] = np.linalg.inv(S)
    dinv[m] = np.linalg.inv(D[m] - Lo[m] @ dinv[m - 1] @ Uo[m - 1] - Uo[m] @ dinv[m + 1] @ Lo[m + 1])
    Lm = [None if J == 0 else dinv[J] @ Lo[J] for J in range(nb)]
    Up = [None if J == nb - 1 else dinv[J] @ Uo[J] for J in range(nb)]
    uc = [dinv[J] @ r[J * B:(J + 1) * B] for J in range(nb)]          # pre-pass p = Dinv r
    yb = [np.zeros(B, complex) for _ in range(nb)]
    f = [_make_path(0, 1, m, kp, 0)]
    f.append(_make_path(nb - 1, -1, nb - 1 - m, kp, f[0]["K"]))
    b = [_make_path(m, -1, m + 1, kp, 0)]
    b.append(_make_path(m, 1, nb - m, kp, b[0]["K"]))
    Pf, Pb = [None] * nb, [None] * nb
    for paths, Cs, P in ((f, (Lm, Up), Pf), (b, (Up, Lm), Pb)):
        for pi, p in enumerate(paths):
            for k in range(1, p["K"]):
                for i in range(p["Ls"]):
                    q = k * p["Ls"] + i
                    if q > _seg_end(k, p["Ls"], p["n"]):
                        continue
                    C = Cs[pi][_blk(p, q)]
                    P[_blk(p, q)] = C.copy() if i == 0 else -C @ P[_blk(p, q - 1)]

    def phase_a(inp, out, Cs, paths):
        for pi, p in enumerate(paths):
            for seg in range(p["K"]):
                q0, prev = seg * p["Ls"], None
                for t in range(max(0, min(p["Ls"], p["n"] - q0))):
                    J = _blk(p, q0 + t)
                    v = inp[J].copy() if t == 0 else inp[J] - Cs[pi][J] @ prev
                    out[J], prev = v, v

    def phase_b(z, P, paths):
        for p in paths:
            prev = z[_blk(p, _seg_end(0, p["Ls"], p["n"]))].copy()
            for t in range(p["K"] - 1):
                J = _blk(p, _seg_end(t + 1, p["Ls"], p["n"]))
                z[J] = z[J] - P[J] @ prev
                prev = z[J]

    def phase_c(z, P, paths):
        for p in paths:
            for q in range(p["Ls"], p["n"]):
                k = q // p["Ls"]
                if q == _seg_end(k, p["Ls"], p["n"]):
                    continue
                J = _blk(p, q)
                z[J] = z[J] - P[J] @ z[_blk(p, k * p["Ls"] - 1)]

    phase_a(uc, yb, (Lm, Up), f)
    phase_b(yb, Pf, f)
    phase_c(yb, Pf, f)
    yb[m] = uc[m] - Lm[m] @ yb[m - 1] - Up[m] @ yb[m + 1]
    phase_a(yb, uc, (Up, Lm), b)
    phase_b(uc, Pb, b)
    phase_c(uc, Pb, b)
    return np.concatenate(uc)


@pytest.mark.parametrize("nb,kp", [(16, 2), (17, 2), (19, 4), (33, 4), (40, 3), (64, 8)])
def test_segmented_twisted_solve_equals_direct(nb, kp):
    rng = np.random.default_rng(nb * 10 + kp)
    B = 5
    cplx = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)  # noqa: E731
    D = [np.eye(B) * 4 + 0.3 * cplx(B, B) for _ in range(nb)]
    Lo = [None] + [0.5 * cplx(B, B) for _ in range(1, nb)]
    Uo = [0.5 * cplx(B, B) for _ in range(nb - 1)] + [None]
    A = np.zeros((nb * B, nb * B), complex)
    for J in range(nb):
        A[J * B:(J + 1) * B, J * B:(J + 1) * B] = D[J]
        if J > 0:
            A[J * B:(J + 1) * B, (J - 1) * B:J * B] = Lo[J]
        if J < nb - 1:
            A[J * B:(J + 1) * B, (J + 1) * B:(J + 2) * B] = Uo[J]
    r = cplx(nb * B)
    x = _segmented_twisted_solve(D, Lo, Uo, r, kp)
    xe = np.linalg.solve(A, r)
    assert np.linalg.norm(x - xe) <= 1e-12 * np.linalg.norm(xe)


# ---------------------------------------------------------------- lagged CGS2 FGMRES

def _fgmres_mgs(A, M, F, m, tol, maxit):
    n = len(F)
    x = np.zeros(n, complex)
    nF, tot, hist = np.linalg.norm(F), 0, []
    while True:
        r = F - A @ x
        beta = np.linalg.norm(r)
        if beta / nF <= tol or tot >= maxit:
            return x, tot, hist
        V, Z, H = [r / beta], [], np.zeros((m + 1, m), complex)
        for j in range(m):
            z = M @ V[j]
            w = A @ z
            Z.append(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j])
            tot += 1
            e = np.zeros(j + 2, complex)
            e[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e, rcond=None)[0]
            hist.append(np.linalg.norm(e - H[:j + 2, :j + 1] @ y) / nF)
            if hist[-1] <= tol or tot >= maxit:
                break
        x = x + np.array(Z).T @ y


def _fgmres_lagged(A, M, F, m, tol, maxit, float_first=False, float_second=False, orth=None):
    """The lagged one-sweep CGS2 FGMRES of krylov.cu. float_first: the first pass's projections
    t_i and the second pass's correction sum sum s_i v_i in complex64 arithmetic (the complex64
    form); float_second: the second pass's projections s_i in complex64 too (a negative control).
    orth collects max |V^H V - I| over each cycle's finished basis."""
    c64 = np.complex64

    def dot(a, b, low):
        return complex(np.vdot(a.astype(c64), b.astype(c64))) if low else np.vdot(a, b)
    n = len(F)
    x = np.zeros(n, complex)
    nF, total, hist = np.linalg.norm(F), 0, []
    while True:
        r = F - A @ x
        beta = np.linalg.norm(r)
        if beta / nF <= tol or total >= maxit:
            return x, total, hist
        Vs = np.zeros((m + 1, n), complex)
        Vs[0] = r / beta
        Z = np.zeros((m, n), complex)
        g = np.zeros(m + 1, complex)
        cs, sn = np.zeros(m), np.zeros(m, complex)
        H = np.zeros((m + 1, m), complex)
        zs = np.zeros(m)
        hcol = np.zeros(m + 2, complex)
        j, pre, W = 0, m >= 1 and total + 1 <= maxit, None
        while True:
            if pre:                                      # preconditioner and A0 on slot j
                Z[j] = M @ Vs[j]
                W = A @ Z[j]
            s = np.array([dot(Vs[i], Vs[j], float_second and i < j) for i in range(j + 1)])   # k_dots2
            t = np.array([dot(Vs[i], W, float_first) for i in range(j + 1)]) if pre else None
            rho2 = s[j].real - np.sum(np.abs(s[:j]) ** 2)                      # k_coef
            rho = np.sqrt(rho2) if rho2 > 0 else 0.0
            stop = False
            if j == 0:
                g[0] = beta * rho
            else:                                        # finish column j-1, Givens
                c = j - 1
                hf, hsub = hcol[:j] + s[:j], rho
                u = hf[0]
                for i in range(c):
                    H[i, c] = cs[i] * u + sn[i] * hf[i + 1]
                    u = -np.conj(sn[i]) * u + cs[i] * hf[i + 1]
                aa = abs(u)
                if hsub == 0:
                    cr, sv, rr = 1.0, 0.0, u
                elif aa == 0:
                    cr, sv, rr = 0.0, 1.0, hsub
                else:
                    nu = np.hypot(aa, hsub)
                    cr, sv, rr = aa / nu, (u / aa) * hsub / nu, (u / aa) * nu
                cs[c], sn[c], H[c, c] = cr, sv, rr
                g[c + 1], g[c] = -np.conj(sv) * g[c], cr * g[c]
                total += 1
                hist.append(abs(g[c + 1]) / nF)
                stop = hist[-1] <= tol or not hsub > 1e-14 * beta
            if not pre or not rho > 0 or stop:
                break
            d = np.sum(np.conj(s[:j]) * t[:j])
            hjj = (t[j] - d) / rho / rho                 # the step uses z_j / rho
            hcol[:j], hcol[j], zs[j] = t[:j] / rho, hjj, 1.0 / rho
            corr = (s[:j].astype(c64) @ Vs[:j].astype(c64)).astype(complex) if float_first else s[:j] @ Vs[:j]
            v = (Vs[j] - corr) / rho                     # k_update2
            Vs[j] = v
            W = W / rho - hcol[:j] @ Vs[:j] - hjj * v
            pre = j + 1 < m and total + 2 <= maxit
            j += 1
            Vs[j] = W                                    # unnormalised u_{j+1}
        if orth is not None and j > 0:
            Q = Vs[:j]
            orth.append(np.abs(Q.conj() @ Q.T - np.eye(j)).max())
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j]) * zs[:j] if j > 0 else np.zeros(0)
        x = x + Z[:j].T @ y


@pytest.mark.parametrize("m,maxit", [(20, 500), (7, 500), (1, 40), (20, 13)])
def test_lagged_cgs2_fgmres_matches_mgs_fgmres(m, maxit):
    rng = np.random.default_rng(3)
    n = 120
    A = np.eye(n) * 4 + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    M = np.linalg.inv(A + 0.05 * rng.standard_normal((n, n)))      # inexact preconditioner
    F = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x1, it1, h1 = _fgmres_mgs(A, M, F, m, 1e-10, maxit)
    x2, it2, h2 = _fgmres_lagged(A, M, F, m, 1e-10, maxit)
    assert it1 == it2
    k = min(len(h1), len(h2))
    assert np.allclose(np.log10(h1[:k]), np.log10(h2[:k]), atol=1e-3)
    r1 = np.linalg.norm(F - A @ x1)
    r2 = np.linalg.norm(F - A @ x2)
    assert abs(r1 - r2) <= 1e-6 * np.linalg.norm(F) + 1e-3 * r1


@pytest.mark.parametrize("m", [20, 7])
def test_float_first_pass_keeps_the_basis_orthogonal(m):
    """The complex64 form's Gram-Schmidt: first-pass projections and the second pass's
    correction sum in float, second-pass projections in full precision. The second pass
    removes what the float first pass leaves, so the basis stays orthogonal to ~1e-13, the
    iterations match MGS FGMRES and the Givens estimate equals the true residual. The control
    with the second pass in float too loses orthogonality at the float level."""
    rng = np.random.default_rng(3)
    n = 120
    A = np.eye(n) * 4 + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    M = np.linalg.inv(A + 0.05 * rng.standard_normal((n, n)))
    F = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x1, it1, _ = _fgmres_mgs(A, M, F, m, 1e-10, 500)
    orth = []
    x2, it2, h2 = _fgmres_lagged(A, M, F, m, 1e-10, 500, float_first=True, orth=orth)
    assert abs(it1 - it2) <= 1
    assert max(orth) <= 1e-12
    r2 = np.linalg.norm(F - A @ x2) / np.linalg.norm(F)
    assert r2 <= 1e-10 * 1.01 and abs(h2[-1] - r2) <= 1e-14   # (relative to |F|: the rounding floor)
    assert np.linalg.norm(x2 - x1) <= 1e-8 * np.linalg.norm(x1)
    orth_low = []
    _fgmres_lagged(A, M, F, m, 1e-10, 500, float_first=True, float_second=True, orth=orth_low)
    assert max(orth_low) > 1e-9


def test_segment_products_bounded_on_helmholtz_coarse_operator():
    """On a rediscretised coarse Helmholtz operator (2D P1, 128 x 128 cells, k = 100,
    eps = 0.5 k^2, impedance boundary) with lexicographic line blocks: the segment products of
    the forward sweep (products of the folded couplings Lm = Dinv A_J,J-1 over up to 16 blocks)
    keep spectral norms below one, and a complex64 segmented forward/backward solve is as
    accurate as the complex64 sequential one against a sparse direct solve."""
    import scipy.sparse.linalg as spla
    from oracle import fem
    nc, k = 128, 100.0
    cm = fem.build_mesh(2, 1, nc)
    Kc, Mc, Bc = fem.assemble(cm)
    A = fem.system_matrix(Kc, Mc, Bc, k, 0.5 * k * k).tocsr()
    W = nc + 1
    blk = lambda I, J: A[I * W:(I + 1) * W, J * W:(J + 1) * W].toarray()  # noqa: E731
    assert A[0:W, 2 * W:3 * W].nnz == 0          # block tridiagonal over grid lines
    dinv, Lm, Up = [None] * W, [None] * W, [None] * W
    S = blk(0, 0)
    for J in range(W):                            # single chain (top-down) Schur complements
        if J > 0:
            S = blk(J, J) - blk(J, J - 1) @ (dinv[J - 1] @ blk(J - 1, J))
        dinv[J] = np.linalg.inv(S)
        if J > 0:
            Lm[J] = dinv[J] @ blk(J, J - 1)
        if J < W - 1:
            Up[J] = dinv[J] @ blk(J, J + 1)
    rng = np.random.default_rng(5)
    r = rng.standard_normal(W * W) + 1j * rng.standard_normal(W * W)
    xe = spla.spsolve(A.tocsc(), r)
    c64 = np.complex64

    def sweep(p, C, order, ls):
        n = len(order)
        q = [None] * n
        for t in range(n):                        # phase A: restarted recurrences
            q[t] = p[order[t]] if t % ls == 0 else p[order[t]] - C[order[t]].astype(c64) @ q[t - 1]
        P, norms = {}, []
        for t in range(ls, n):                    # segment products
            C_t = C[order[t]].astype(c64)
            P[t] = C_t if t % ls == 0 else -C_t @ P[t - 1]
            norms.append(np.linalg.norm(P[t], 2))
        y = list(q)
        ends = [min(kk * ls + ls, n) - 1 for kk in range(n // ls + 1) if kk * ls < n]
        for e_prev, e in zip(ends[:-1], ends[1:]):   # phase B: z_e = w_e - P_e z_e(prev)
            y[e] = q[e] - P[e] @ y[e_prev]
        for t in range(ls, n):                    # phase C: z_t = w_t - P_t z_e(k-1)
            if t not in ends:
                y[t] = q[t] - P[t] @ y[(t // ls) * ls - 1]
        out = [None] * n
        for t in range(n):
            out[order[t]] = y[t]
        return out, max(norms)

    p = [(dinv[J].astype(c64) @ r[J * W:(J + 1) * W].astype(c64)) for J in range(W)]
    y, nf = sweep(p, Lm, list(range(W)), 16)
    x, nb = sweep(y, Up, list(range(W - 1, -1, -1)), 16)
    xs = np.concatenate(x)
    ys = [p[0]]
    for J in range(1, W):
        ys.append(p[J] - Lm[J].astype(c64) @ ys[-1])
    xq = [None] * W
    xq[-1] = ys[-1]
    for J in range(W - 2, -1, -1):
        xq[J] = ys[J] - Up[J].astype(c64) @ xq[J + 1]
    xq = np.concatenate(xq)
    err_seg = np.linalg.norm(xs - xe) / np.linalg.norm(xe)
    err_seq = np.linalg.norm(xq - xe) / np.linalg.norm(xe)
    assert nf < 1.0 and nb < 1.0, (nf, nb)
    assert err_seg <= 2.0 * err_seq + 1e-7, (err_seg, err_seq)


def _segment_study(A, W, rows, ls, seed=5):
    """Block-tridiagonal factorisation of A over blocks of `rows` lattice lines, then the
    complex64 segmented forward/backward sweeps (segments of ls blocks) and the sequential ones:
    returns (max product norm forward, backward, relative error segmented, sequential)."""
    import scipy.sparse.linalg as spla
    A = A.tocsr()
    N = A.shape[0]
    Bs = rows * W
    nb = (N + Bs - 1) // Bs
    cut = [(J * Bs, min(N, (J + 1) * Bs)) for J in range(nb)]
    blk = lambda I, J: A[cut[I][0]:cut[I][1], cut[J][0]:cut[J][1]].toarray()  # noqa: E731
    dinv, Lm, Up = [None] * nb, [None] * nb, [None] * nb
    S = blk(0, 0)
    for J in range(nb):
        if J > 0:
            S = blk(J, J) - blk(J, J - 1) @ (dinv[J - 1] @ blk(J - 1, J))
        dinv[J] = np.linalg.inv(S)
        if J > 0:
            Lm[J] = dinv[J] @ blk(J, J - 1)
        if J < nb - 1:
            Up[J] = dinv[J] @ blk(J, J + 1)
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    xe = spla.spsolve(A.tocsc(), r)
    c64 = np.complex64

    def sweep(p, C, order):
        n = len(order)
        q = [p[order[t]] if t % ls == 0 else None for t in range(n)]
        for t in range(n):
            if t % ls:
                q[t] = p[order[t]] - C[order[t]].astype(c64) @ q[t - 1]
        P, norms = {}, [0.0]
        for t in range(ls, n):
            Ct = C[order[t]].astype(c64)
            P[t] = Ct if t % ls == 0 else -Ct @ P[t - 1]
            norms.append(np.linalg.norm(P[t], 2))
        y = list(q)
        ends = [min(kk * ls + ls, n) - 1 for kk in range(n // ls + 1) if kk * ls < n]
        for a, e in zip(ends[:-1], ends[1:]):
            y[e] = q[e] - P[e] @ y[a]
        for t in range(ls, n):
            if t not in ends:
                y[t] = q[t] - P[t] @ y[(t // ls) * ls - 1]
        out = [None] * n
        for t in range(n):
            out[order[t]] = y[t]
        return out, max(norms)

    p = [dinv[J].astype(c64) @ r[cut[J][0]:cut[J][1]].astype(c64) for J in range(nb)]
    y, nf = sweep(p, Lm, list(range(nb)))
    x, nbk = sweep(y, Up, list(range(nb - 1, -1, -1)))
    ys = [p[0]]
    for J in range(1, nb):
        ys.append(p[J] - Lm[J].astype(c64) @ ys[-1])
    xq = [None] * nb
    xq[-1] = ys[-1]
    for J in range(nb - 2, -1, -1):
        xq[J] = ys[J] - Up[J].astype(c64) @ xq[J + 1]
    err = lambda v: np.linalg.norm(np.concatenate(v) - xe) / np.linalg.norm(xe)  # noqa: E731
    return nf, nbk, err(x), err(xq)


@pytest.mark.parametrize("p,nc,k", [(1, 128, 100.0), (2, 64, 100.0)])
def test_segment_products_bounded_on_q_coarse_operators(p, nc, k):
    """The same study on the tensor-product Q1 / Q2 coarse operators (helm_setup_q; blocks of p
    lattice lines): Q1's products stay below one in norm; Q2's single couplings reach about 2, but
    the products do not grow with the segment length; in both the complex64 segmented solve is as
    accurate as the sequential one."""
    from oracle import fem, qfem
    m = qfem.build_mesh(2, p, nc)
    K, _, M, B, _ = qfem.assemble(m)
    A = fem.system_matrix(K, M, B, k, 0.5 * k * k)
    W = p * nc + 1
    nf1, nb1, _, _ = _segment_study(A, W, p, 1)      # segments of one block: the couplings alone
    nf, nbk, err_seg, err_seq = _segment_study(A, W, p, 16)
    if p == 1:
        assert nf < 1.0 and nbk < 1.0, (nf, nbk)
    assert nf <= 1.05 * nf1 and nbk <= 1.05 * nb1, (nf, nf1, nbk, nb1)
    assert err_seg <= 2.0 * err_seq + 1e-7, (err_seg, err_seq)


def test_schur_complements_converge_along_the_chain_for_large_shifts():
    """Premise of reusing converged Schur inverses in the coarse factorisation: the coarse
    operator of the benchmark (2D P1, 256 x 256 cells, k = 200) is block tridiagonal with the same
    blocks on every interior line, so S_J = A - A_J,J-1 S_J-1^-1 A_J-1,J follows one recurrence.
    For eps = k^2 / 2 the inverse stops changing at complex64 level (1e-9 relative) after about
    50 of the 127 blocks of a chain and at FP64 level after about 90; for eps = k it keeps changing
    to the end, so any reuse has to test convergence as it goes."""
    from oracle import fem
    nc, k = 256, 200.0
    cm = fem.build_mesh(2, 1, nc)
    K, M, B = fem.assemble(cm)
    W = nc + 1

    def changes(eps, steps):
        A = fem.system_matrix(K, M, B, k, eps).tocsr()
        blk = lambda I, J: A[I * W:(I + 1) * W, J * W:(J + 1) * W].toarray()  # noqa: E731
        Dprev = np.linalg.inv(blk(0, 0))
        out = []
        for J in range(1, steps + 1):
            D = np.linalg.inv(blk(J, J) - blk(J, J - 1) @ (Dprev @ blk(J - 1, J)))
            out.append(np.linalg.norm(D - Dprev) / np.linalg.norm(D))
            Dprev = D
        return out

    big = changes(0.5 * k * k, 100)
    assert max(big[59:]) < 1e-9 and max(big[94:]) < 1e-14
    small = changes(k, 127)
    assert min(small) > 1e-6


def test_reused_schur_inverses_keep_the_coarse_solve_below_complex64_rounding():
    """Freezing Dinv once consecutive inverses agree to 1e-9 (relative) on the benchmark's coarse
    operator (the last, boundary block still recomputed) needs about a fifth of the inversions of
    the top-down chain and changes the coarse solve by less than complex64 rounding."""
    import scipy.sparse.linalg as spla
    from oracle import fem
    nc, k = 256, 200.0
    cm = fem.build_mesh(2, 1, nc)
    K, M, B = fem.assemble(cm)
    A = fem.system_matrix(K, M, B, k, 0.5 * k * k).tocsr()
    W = nc + 1
    blk = lambda I, J: A[I * W:(I + 1) * W, J * W:(J + 1) * W].toarray()  # noqa: E731

    def factor(tol):
        D, frozen, inversions = [np.linalg.inv(blk(0, 0))], None, 1
        for J in range(1, W):
            if frozen is not None and J < W - 1:
                D.append(frozen)
                continue
            D.append(np.linalg.inv(blk(J, J) - blk(J, J - 1) @ (D[J - 1] @ blk(J - 1, J))))
            inversions += 1
            if tol and J < W - 1 and np.linalg.norm(D[J] - D[J - 1]) / np.linalg.norm(D[J]) < tol:
                frozen = D[J]
        return D, inversions

    def solve(D, r):
        y = [D[0] @ r[:W]]
        for J in range(1, W):
            y.append(D[J] @ (r[J * W:(J + 1) * W] - blk(J, J - 1) @ y[-1]))
        x = [None] * W
        x[-1] = y[-1]
        for J in range(W - 2, -1, -1):
            x[J] = y[J] - D[J] @ (blk(J, J + 1) @ x[J + 1])
        return np.concatenate(x)

    rng = np.random.default_rng(3)
    r = rng.standard_normal(W * W) + 1j * rng.standard_normal(W * W)
    xe = spla.spsolve(A.tocsc(), r)
    Dr, inv_r = factor(1e-9)
    err = np.linalg.norm(solve(Dr, r) - xe) / np.linalg.norm(xe)
    assert inv_r <= 60 and err < 1e-8, (inv_r, err)


def _fgmres_basis_precision(A0, F, M, m, tol, maxit, basis_dtype):
    """FGMRES(m) whose Krylov basis, CGS2 inner products and corrections are held in basis_dtype
    (complex64 or complex128); Givens and least squares in complex128, the true residual in
    complex128 at every cycle end. Returns (iterations, final true relative residual)."""
    N = F.shape[0]
    x = np.zeros(N, complex)
    nF = np.linalg.norm(F)
    total = 0
    while total < maxit:
        r = F - A0 @ x
        beta = np.linalg.norm(r)
        if beta / nF <= tol:
            break
        V = np.zeros((m + 1, N), basis_dtype)
        Z = np.zeros((m, N), complex)
        V[0] = (r / beta).astype(basis_dtype)
        H = np.zeros((m + 1, m), complex)
        g = np.zeros(m + 1, complex)
        g[0] = beta
        cs, sn, jn = np.zeros(m), np.zeros(m, complex), 0
        for j in range(m):
            Z[j] = M(V[j].astype(complex))
            w = (A0 @ Z[j]).astype(basis_dtype)
            h = np.zeros(j + 1, complex)
            for _ in range(2):
                c = V[:j + 1].conj() @ w
                w = w - (c @ V[:j + 1]).astype(basis_dtype)
                h += c
            hn = np.linalg.norm(w.astype(complex))
            H[:j + 1, j], H[j + 1, j] = h, hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            rr = np.hypot(abs(a), abs(bb))
            cs[j] = abs(a) / rr
            sn[j] = (a / abs(a)) * np.conj(bb) / rr if abs(a) > 0 else 1.0
            H[j, j], H[j + 1, j] = cs[j] * a + sn[j] * bb, 0
            g[j + 1], g[j] = -np.conj(sn[j]) * g[j], cs[j] * g[j]
            total, jn = total + 1, j + 1
            if hn > 0:
                V[j + 1] = (w / hn).astype(basis_dtype)
            if abs(g[j + 1]) / nF <= tol or total >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:jn, :jn]), g[:jn])
        x = x + y @ Z[:jn]
    return total, np.linalg.norm(F - A0 @ x) / nF


@pytest.mark.parametrize("n,k", [(128, 50.0), (256, 100.0)])
def test_complex64_krylov_basis_costs_few_iterations(n, k):
    """Premise of a complex64 Gram-Schmidt in the mixed form: on the benchmark's problem class
    (Gaussian source, kh = 0.39, eps = k^2 / 2, FGMRES(80), twogrid preconditioner) a complex64
    basis reaches the 1e-8 true residual with at most ~10% more iterations than a complex128 one
    (46 -> 51 at n = 128, 86 -> 88 at n = 256; at n = 512, the benchmark, both take 163)."""
    import helm_inputs as hi
    from oracle import solver
    pb = solver.build_problem(hi.GAUSS_P1.with_(n=n, k=k, shift=0.5 * k * k))
    tg = pb.twogrid()
    it128, rr128 = _fgmres_basis_precision(pb.A0, pb.F, tg.apply, 80, 1e-8, 500, np.complex128)
    it64, rr64 = _fgmres_basis_precision(pb.A0, pb.F, tg.apply, 80, 1e-8, 500, np.complex64)
    assert rr128 <= 1e-8 and rr64 <= 1e-8
    assert it64 <= 1.12 * it128 + 1, (it128, it64)
