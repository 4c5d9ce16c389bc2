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


def test_golden_section_batched(pkg):
    from paper_2104_01439_gb300 import sweep
    out = sweep.golden_section([(12.0, 32, 1), (20.0, 32, 1)], tol=1e-2, maxit=50, max_active=4)
    for s, rho, n in out:
        assert 1.0 <= s <= 2.0
        assert 0.0 < rho < 1.0
        assert n == 12
