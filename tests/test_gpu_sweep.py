"""Shift sweeps through the request server agree with one-at-a-time solves, and
the golden-section search of Sec. 5 runs batched on the GPU."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2104_01439_gb300 as p
    return p


def test_sweep_matches_single_solves(pkg):
    from paper_2104_01439_gb300 import sweep
    samples = [sweep.Sample(k, n, f * k * k) for k, n in ((15.0, 32), (25.0, 48)) for f in (0.05, 0.5, 2.0)]
    res = sweep.run_sweep(samples, theta=0.3, restart=50, maxit=500, max_active=6)
    for s, r in zip(samples, res):
        slv = pkg.Solver(s.k, s.n, 1, s.shift, restart=50, maxit=500, tol=1e-8, precision=pkg.HELM_MIXED)
        F = slv.rhs_planewave(0.3).cuda()
        _, ra = slv.solve(F)
        slv.close()
        assert r.iters == ra.iters and r.status == ra.status == "converged"
        assert abs(r.relres - ra.relres_true) <= 1e-12
    best = sweep.best_shifts(res)
    assert len(best) == 2
    for b in best:
        grp = [r for r in res if r.sample.k == b.sample.k]
        assert b.iters == min(r.iters for r in grp)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_golden_section_batched(pkg, prec):
    """The batched golden-section search of Sec. 5 (all searches advanced together through the
    request server) against the oracle's one-problem-at-a-time search on the same loads: the
    exponents agree within the search tolerance (a comparison of two nearly equal rates may
    go either way, which moves the final bracket by at most one reduction) and the rates."""
    import helm_inputs as hi
    from oracle import solver as osolver
    from paper_2104_01439_gb300 import sweep
    problems = [(12.0, 32, 1), (20.0, 32, 1)]
    precision = pkg.HELM_FP64 if prec == "fp64" else pkg.HELM_MIXED
    out = sweep.golden_section(problems, tol=1e-2, maxit=50, max_active=4, precision=precision, seed=7)
    loads = hi.uniform_loads([(o * n + 1) ** 2 for _, n, o in problems], seed=7)
    for (k, n, order), F, (s, rho, cnt) in zip(problems, loads, out):
        s_ref, rho_ref, cnt_ref = osolver.optimal_shift_exponent(k, n, order, F, tol=1e-2, maxit=50)
        assert 1.0 <= s <= 2.0 and 0.0 < rho < 1.0
        assert cnt == cnt_ref == 12
        assert abs(s - s_ref) <= 2e-2, (k, s, s_ref)
        assert abs(rho - rho_ref) <= 1e-3 * rho_ref, (k, rho, rho_ref)
