"""Edge cases of the solve through the C ABI: empty (zero) and non-finite load
vectors, the iteration cap, FGMRES(1), an unshifted preconditioner, and
argument validation."""
import numpy as np
import pytest

import helm_inputs as hi
from oracle import solver as osolver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2104_01439_gb300 as pkg  # noqa: E402


@pytest.mark.parametrize("prec", [pkg.HELM_FP64, pkg.HELM_MIXED])
def test_zero_load_gives_zero_solution(prec):
    s = pkg.Solver(10.0, 16, 1, 50.0, precision=prec)
    x, r = s.solve(torch.zeros(s.num_dofs, dtype=torch.complex128, device="cuda"))
    assert r.status == "converged" and r.iters == 0 and r.relres_true == 0.0
    assert torch.count_nonzero(x).item() == 0
    s.close()


def test_nonfinite_load_is_reported():
    s = pkg.Solver(10.0, 16, 1, 50.0, precision=pkg.HELM_MIXED)
    F = torch.ones(s.num_dofs, dtype=torch.complex128, device="cuda")
    F[5] = float("nan")
    _, r = s.solve(F)
    assert r.status == "nonfinite"
    # the handle stays usable
    _, r2 = s.solve(torch.ones(s.num_dofs, dtype=torch.complex128, device="cuda"))
    assert r2.status == "converged"
    s.close()


def test_iteration_cap():
    s = pkg.Solver(20.0, 32, 1, 200.0, restart=50, maxit=5, precision=pkg.HELM_FP64)
    F = torch.from_numpy(hi.random_load(s.num_dofs, 9)).cuda()
    _, r = s.solve(F)
    assert r.status == "maxit" and r.iters == 5 and r.relres_true > 1e-8
    s.close()


def test_restart_one_matches_oracle():
    """FGMRES(1): every iteration is its own cycle (restart logic exercised at each step)."""
    wl = hi.Workload("p1_n16_restart1", 2, 1, 16, 6.0, 18.0, "random", seed=12, restart=1, maxit=400)
    pb = osolver.build_problem(wl)
    ref = pb.solve()
    s = pkg.Solver(wl.k, wl.n, 1, wl.shift, restart=1, maxit=400, tol=1e-8, precision=pkg.HELM_FP64)
    x, r = s.solve(torch.from_numpy(pb.F).cuda())
    assert r.status == "converged"
    assert abs(r.iters - ref.iters) <= 1 and r.cycles == r.iters
    xh = x.cpu().numpy()
    assert np.linalg.norm(pb.F - pb.A0 @ xh) / np.linalg.norm(pb.F) <= 1e-8
    s.close()


def test_unshifted_preconditioner_is_handled():
    """eps = 0: the no-pivot factorisation is not guaranteed to exist; setup either
    succeeds (then the solve converges) or reports a zero pivot."""
    try:
        s = pkg.Solver(8.0, 16, 1, 0.0, precision=pkg.HELM_FP64)
    except pkg.HelmError as e:
        assert "pivot" in str(e)
        return
    F = torch.from_numpy(hi.random_load(s.num_dofs, 2)).cuda()
    _, r = s.solve(F)
    assert r.status in ("converged", "maxit")
    s.close()


@pytest.mark.parametrize("kw", [dict(n=15), dict(n=2), dict(order=3), dict(order=2, dim=3), dict(k=0.0),
                                dict(shift=-1.0), dict(restart=0), dict(nu=0)])
def test_invalid_arguments(kw):
    args = dict(k=10.0, n=16, order=1, shift=50.0, dim=2, restart=50, nu=2)
    args.update(kw)
    with pytest.raises(pkg.HelmError, match="invalid argument"):
        pkg.Solver(args["k"], args["n"], args["order"], args["shift"], dim=args["dim"], restart=args["restart"],
                   nu=args["nu"])
