"""GPU parity of every hot-path step against the FP64 CPU oracle (through the C ABI).

Tolerances (derived from the arithmetic):
  * FP64 operator applies: <= 1e-12 relative (a 9..27-term stencil sum in
    complex128 vs CSR SpMV, both ~1e-16 per term).
  * FP64 coarse solve / V-cycle: <= 1e-9 relative (explicit inverses of the
    Schur blocks amplify rounding by the block condition number, ~1e4..1e6).
  * complex64 V-cycle: <= 2e-5 relative (float32 unit roundoff 6e-8 times the
    same conditioning).
  * Solves: true relative residual <= 1e-8 (recomputed here by the oracle's CSR
    A0), FGMRES iterations within +-1 of the oracle (FP64) and within +-3
    (complex64 preconditioner), solution within cond-scaled tolerance.
"""
import numpy as np
import pytest

import helm_inputs as hi
from oracle import fem, solver as osolver
from parity import assert_entrywise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2104_01439_gb300 as pkg  # noqa: E402

_PB = {}


def problem(wl):
    key = (wl.dim, wl.order, wl.n, wl.k, wl.shift, wl.rhs, wl.seed)
    if key not in _PB:
        _PB[key] = osolver.build_problem(wl)
    return _PB[key]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def crand(n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(n) + 1j * g.standard_normal(n)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


CASES = [
    hi.Workload("p1_n8", 2, 1, 8, 6.0, 18.0, "random", seed=1),
    hi.Workload("p1_n36_ragged", 2, 1, 36, 12.0, 72.0, "random", seed=2),
    hi.Workload("p1_n64", 2, 1, 64, 20.0, 200.0, "planewave"),
    hi.Workload("p2_n8", 2, 2, 8, 6.0, 18.0, "random", seed=3),
    hi.Workload("p2_n22_ragged", 2, 2, 22, 10.0, 50.0, "random", seed=4),
    hi.Workload("p1_3d_n6", 3, 1, 6, 4.0, 8.0, "random", seed=5),
]


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_apply_fp64(wl):
    pb = problem(wl)
    s = pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim)
    x = crand(pb.mesh.num_dofs, 7)
    for which, A in ((0, pb.A0), (1, pb.Aeps)):
        y = s.apply(dev(x), which).cpu().numpy()
        assert rel(y, A @ x) <= 1e-12
        assert_entrywise(y, A @ x, pb.mesh.coords, 1e-12, f"A{which} x")
    s.close()


@pytest.mark.parametrize("prec,tol", [(pkg.HELM_FP64, 1e-9), (pkg.HELM_MIXED, 2e-5)])
@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_coarse_solve(wl, prec, tol):
    pb = problem(wl)
    s = pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim, precision=prec)
    r = crand(pb.cmesh.num_dofs, 11)
    uc = s.coarse_solve(dev(r)).cpu().numpy()
    ref = pb.twogrid().coarse_solve(r)
    assert rel(uc, ref) <= tol
    assert_entrywise(uc, ref, pb.cmesh.coords, tol, "coarse solve")
    s.close()


@pytest.mark.parametrize("prec,tol", [(pkg.HELM_FP64, 1e-9), (pkg.HELM_MIXED, 2e-5)])
@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_vcycle(wl, prec, tol):
    pb = problem(wl)
    s = pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim, precision=prec)
    f = crand(pb.mesh.num_dofs, 13)
    u = s.vcycle(dev(f)).cpu().numpy()
    ref = pb.twogrid().apply(f)
    assert rel(u, ref) <= tol
    assert_entrywise(u, ref, pb.mesh.coords, tol, "V-cycle")
    s.close()


@pytest.mark.parametrize("prec,tol", [(pkg.HELM_FP64, 1e-12), (pkg.HELM_MIXED, 2e-6)])
@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_smooth_operator_handle(wl, prec, tol):
    """nu damped-Jacobi sweeps from u = 0 on an operator-only handle against the oracle's
    sweeps (Algorithm 1, smoothing); the handle refuses every call that needs the coarse level."""
    pb = problem(wl)
    s = pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim, precision=prec, operator_only=True)
    f = crand(pb.mesh.num_dofs, 17)
    dinv = 1.0 / pb.Aeps.diagonal()
    for nu in (2, 3, 5):
        u = s.smooth(dev(f), nu).cpu().numpy()
        ref = osolver.jacobi_sweeps(pb.Aeps, dinv, f, np.zeros_like(f), 0.6, nu)
        assert rel(u, ref) <= tol * nu, nu
        assert_entrywise(u, ref, pb.mesh.coords, tol * nu, f"{nu} sweeps")
    x = crand(pb.mesh.num_dofs, 7)
    assert rel(s.apply(dev(x), 1).cpu().numpy(), pb.Aeps @ x) <= 1e-12
    for call in (lambda: s.vcycle(dev(f)), lambda: s.solve(dev(f)), lambda: s.smooth(dev(f), 1),
                 lambda: s.smooth(dev(f), 9)):
        with pytest.raises(pkg.HelmError):
            call()
    s.close()


@pytest.mark.parametrize("wl", [CASES[1], CASES[2], CASES[4], CASES[5]], ids=lambda w: w.name)
def test_rhs_builders(wl):
    pb = problem(wl)
    s = pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim)
    Fp = s.rhs_planewave(0.3).numpy()
    assert rel(Fp, fem.load_planewave(pb.mesh, pb.M, wl.k, 0.3)) <= 1e-12
    Fg = s.rhs_gaussian(2.0 / wl.n).numpy()
    assert rel(Fg, fem.load_gaussian(pb.mesh, pb.M, 2.0 / wl.n)) <= 1e-12
    s.close()


@pytest.mark.parametrize("prec", [pkg.HELM_FP64, pkg.HELM_MIXED])
@pytest.mark.parametrize("wl", [CASES[1], CASES[2], CASES[4], CASES[5]], ids=lambda w: w.name)
def test_solve_parity(wl, prec):
    pb = problem(wl)
    ref = pb.solve()
    s = pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim, restart=wl.restart, maxit=wl.maxit,
                   tol=wl.tol, precision=prec)
    x, res = s.solve(dev(pb.F))
    xh = x.cpu().numpy()
    relres = np.linalg.norm(pb.F - pb.A0 @ xh) / np.linalg.norm(pb.F)
    assert res.status == "converged"
    assert relres <= 1e-8 and abs(relres - res.relres_true) <= 1e-10
    slack = 1 if prec == pkg.HELM_FP64 else 3
    assert abs(res.iters - ref.iters) <= slack, (res.iters, ref.iters)
    assert rel(xh, ref.x) <= 1e-5
    assert_entrywise(xh, ref.x, pb.mesh.coords, 1e-5, "solution")
    s.close()


@pytest.mark.parametrize("prec", [pkg.HELM_FP64, pkg.HELM_MIXED])
def test_batch_and_host_solves_match_single(prec):
    """helm_batch_solve (several handles interleaved on their own streams) and
    helm_solve_host (host buffers, copies inside the call) give what helm_solve gives."""
    wls = [CASES[1], CASES[2], CASES[4]]
    solvers = [pkg.Solver(w.k, w.n, w.order, w.shift, dim=w.dim, restart=w.restart, maxit=w.maxit,
                          tol=w.tol, precision=prec) for w in wls]
    Fs = [dev(problem(w).F) for w in wls]
    singles = [s.solve(F) for s, F in zip(solvers, Fs)]
    xs, results = pkg.batch_solve(solvers, Fs)
    for (x1, r1), x2, r2 in zip(singles, xs, results):
        assert r2.status == "converged" and r2.iters == r1.iters
        a, b = x1.cpu().numpy(), x2.cpu().numpy()
        assert rel(b, a) <= 1e-12
    for s, F, (x1, r1) in zip(solvers, Fs, singles):
        Fh = F.cpu().pin_memory()
        xh = torch.empty_like(Fh).pin_memory()
        r3 = s.solve_host(Fh, xh)
        assert r3.status == "converged" and r3.iters == r1.iters
        assert rel(xh.numpy(), x1.cpu().numpy()) <= 1e-12
    for s in solvers:
        s.close()


_COARSE = {}


def coarse_direct(n, k, shift):
    """The oracle's assembled coarse matrix (2h mesh) and its sparse direct factorisation."""
    key = (n, k, shift)
    if key not in _COARSE:
        import scipy.sparse.linalg as spla
        cm = fem.build_mesh(2, 1, n // 2)
        Kc, Mc, Bc = fem.assemble(cm)
        _COARSE[key] = (cm, spla.splu(fem.system_matrix(Kc, Mc, Bc, k, shift).tocsc()))
    return _COARSE[key]


@pytest.mark.parametrize("prec,tol", [(pkg.HELM_FP64, 1e-9), (pkg.HELM_MIXED, 2e-5)], ids=["fp64", "mixed"])
@pytest.mark.parametrize("n,k,expo", [(64, 20.0, 2.0), (64, 20.0, 1.0), (64, 20.0, 1.5),
                                      (512, 200.0, 2.0), (512, 200.0, 1.0), (512, 200.0, 1.5)],
                         ids=lambda v: str(v))
def test_factor_reuse_coarse_solve(n, k, expo, prec, tol):
    """Coarse factorisation with the reuse of converged Schur inverses (Sec. 6's factor-once
    LU, computed along two block chains): for eps = k^2 / 2 the chains converge and later blocks
    reuse the converged inverse; for eps = k and k^1.5 they do not, and every block is factored.
    Either way the coarse solve matches the oracle's sparse direct solve of its own coarse
    matrix, normwise and entry by entry."""
    shift = 0.5 * k * k if expo == 2.0 else k ** expo
    s = pkg.Solver(k, n, 1, shift, precision=prec)
    cm, lu = coarse_direct(n, k, shift)
    r = crand(cm.num_dofs, 19)
    uc = s.coarse_solve(dev(r)).cpu().numpy()
    ref = lu.solve(r)
    assert rel(uc, ref) <= tol
    assert_entrywise(uc, ref, cm.coords, tol, "coarse solve")
    nb = n // 2 + 1
    assert s.factored_blocks + s.reused_blocks == nb
    if n == 512 and expo == 2.0:
        assert s.reused_blocks >= nb // 3, s.reused_blocks     # the chains converge (large shift)
    if expo == 1.0:
        assert s.reused_blocks == 0                            # no convergence: all factored
    s.close()
