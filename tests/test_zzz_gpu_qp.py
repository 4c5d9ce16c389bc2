"""GPU parity of the tensor-product Q_p path (helm_setup_q; Sec. 2's Q_p elements) against the
FP64 CPU oracle oracle/qfem.py, through the C ABI.

The kernels are the ones of the simplex path (9/25/27-point class stencils, and 49-point ones
for Q3, the same lattice, block layout and transfers); only the host tables differ, and those
are pinned row by row on the CPU (test_host_tables). Q1-Q3 also run with the paper's own
smoother setting, V(3,3) with omega = 2/3 (Sec. 4, Sec. 7). Tolerances as in test_gpu_parity,
for the same arithmetic: operator applies <= 1e-12, FP64 coarse solve / V-cycle <= 1e-9,
complex64 <= 2e-5, solves to relres 1e-8 with iterations within +-1 (FP64) / +-3 (complex64
preconditioner), all also entry by entry per DoF class.
"""
import numpy as np
import pytest

import helm_inputs as hi
from oracle import qfem, solver as osolver
from parity import assert_entrywise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2104_01439_gb300 as pkg  # noqa: E402

CASES = [
    hi.Workload("q1_n8", 2, 1, 8, 6.0, 18.0, "random", seed=21),
    hi.Workload("q1_n36_ragged", 2, 1, 36, 12.0, 72.0, "random", seed=22),
    hi.Workload("q1_n64", 2, 1, 64, 20.0, 200.0, "planewave"),
    hi.Workload("q2_n8", 2, 2, 8, 6.0, 18.0, "random", seed=23),
    hi.Workload("q2_n22_ragged", 2, 2, 22, 10.0, 50.0, "random", seed=24),
    hi.Workload("q1_3d_n6", 3, 1, 6, 4.0, 8.0, "random", seed=25),
    # Q3 at the Gauss-Lobatto points (49-point stencils, 81 classes, blocks of three lattice lines)
    hi.Workload("q3_n8", 2, 3, 8, 6.0, 18.0, "random", seed=26),
    hi.Workload("q3_n18_ragged", 2, 3, 18, 12.0, 72.0, "random", seed=27),
    hi.Workload("q3_n16", 2, 3, 16, 20.0, 200.0, "planewave"),
]
# The paper's own smoother setting, V(3,3) with omega = 2/3 (Sec. 4, Sec. 7), on Q1, Q2, Q3
V33 = [
    hi.Workload("q1_n64_v33", 2, 1, 64, 20.0, 20.0 ** 1.5, "planewave", omega=2.0 / 3.0, nu=3),
    hi.Workload("q2_n32_v33", 2, 2, 32, 20.0, 20.0 ** 1.5, "planewave", omega=2.0 / 3.0, nu=3),
    hi.Workload("q3_n16_v33", 2, 3, 16, 20.0, 20.0 ** 1.5, "planewave", omega=2.0 / 3.0, nu=3),
]
_PB = {}


def problem(wl):
    if wl.name not in _PB:
        _PB[wl.name] = osolver.build_problem_q(wl)
    return _PB[wl.name]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def crand(n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(n) + 1j * g.standard_normal(n)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def solver_q(wl, **kw):
    return pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim, elements=pkg.HELM_TENSOR, omega=wl.omega,
                      nu=wl.nu, **kw)


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_apply_q(wl):
    pb = problem(wl)
    s = solver_q(wl)
    assert s.num_dofs == pb.mesh.num_dofs
    x = crand(pb.mesh.num_dofs, 7)
    for which, A in ((0, pb.A0), (1, pb.Aeps)):
        y = s.apply(dev(x), which).cpu().numpy()
        assert rel(y, A @ x) <= 1e-12
        assert_entrywise(y, A @ x, pb.mesh.coords, 1e-12, f"A{which} x")
    s.close()


@pytest.mark.parametrize("prec,tol", [(pkg.HELM_FP64, 1e-9), (pkg.HELM_MIXED, 2e-5)])
@pytest.mark.parametrize("wl", CASES + V33, ids=lambda w: w.name)
def test_coarse_solve_and_vcycle_q(wl, prec, tol):
    pb = problem(wl)
    s = solver_q(wl, precision=prec)
    r = crand(pb.cmesh.num_dofs, 11)
    uc, ucr = s.coarse_solve(dev(r)).cpu().numpy(), pb.twogrid().coarse_solve(r)
    assert rel(uc, ucr) <= tol
    assert_entrywise(uc, ucr, pb.cmesh.coords, tol, "coarse solve")
    f = crand(pb.mesh.num_dofs, 13)
    u, ur = s.vcycle(dev(f)).cpu().numpy(), pb.twogrid().apply(f)
    assert rel(u, ur) <= tol
    assert_entrywise(u, ur, pb.mesh.coords, tol, "V-cycle")
    s.close()


@pytest.mark.parametrize("prec", [pkg.HELM_FP64, pkg.HELM_MIXED])
@pytest.mark.parametrize("wl", [CASES[1], CASES[2], CASES[4], CASES[5], CASES[7], CASES[8]] + V33,
                         ids=lambda w: w.name)
def test_solve_parity_q(wl, prec):
    pb = problem(wl)
    ref = pb.solve()
    s = solver_q(wl, restart=wl.restart, maxit=wl.maxit, tol=wl.tol, precision=prec)
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


@pytest.mark.parametrize("wl", [CASES[2], CASES[8]], ids=lambda w: w.name)
def test_rhs_planewave_q(wl):
    """The plane-wave load at the lattice's interpolation nodes (Gauss-Lobatto for Q3)."""
    pb = problem(wl)
    s = solver_q(wl)
    F = s.rhs_planewave(wl.theta).numpy()
    assert rel(F, qfem.load_planewave(pb.mesh, pb.M, wl.k, wl.theta)) <= 1e-12
    s.close()
