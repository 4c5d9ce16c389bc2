"""Full-size checks of the benchmarked and listed workloads (2D P1 n=512, 2D P2
n=256, 3D P1 n=96) and of the whole-grid coarse solve (blocks larger than one
cluster), by properties the oracle computes at any size: the operator apply
against the oracle's assembled CSR matrix, the true residual of the GPU
solution recomputed with the oracle's A0, the coarse residual with the
oracle's assembled coarse matrix, and the iteration count against the
oracle's own full solve (tests/golden/oracle_iterations.json, written by a
script that runs only the oracle). The benchmark's workload is also solved by
the oracle here (about a minute of CPU time) and both GPU forms are compared
with its solution entry by entry."""
import json
import os

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

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_iterations.json")))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def load(wl, s):
    if wl.rhs == "gaussian":
        return s.rhs_gaussian(2.0 / wl.n).numpy()
    return hi.random_load(s.num_dofs, wl.seed)


@pytest.mark.parametrize("wl", [hi.GAUSS_P1, hi.RANDOM_P2,
                                pytest.param(hi.RANDOM_P1_3D, marks=pytest.mark.slow)], ids=lambda w: w.name)
def test_fullsize_solve(wl):
    mesh = fem.build_mesh(wl.dim, wl.order, wl.n)
    K, M, B = fem.assemble(mesh)
    A0 = fem.system_matrix(K, M, B, wl.k, 0.0)
    s = pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim, restart=wl.restart, maxit=wl.maxit, tol=wl.tol,
                   precision=pkg.HELM_MIXED)
    # operator apply at full size
    g = np.random.default_rng(3)
    v = g.standard_normal(s.num_dofs) + 1j * g.standard_normal(s.num_dofs)
    y = s.apply(dev(v), 0).cpu().numpy()
    ref = A0 @ v
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-12
    # the solve: true residual with the oracle's matrix, iterations against the oracle's solve
    F = load(wl, s)
    x, r = s.solve(dev(F))
    xh = x.cpu().numpy()
    relres = np.linalg.norm(F - A0 @ xh) / np.linalg.norm(F)
    assert r.status == "converged" and relres <= 1e-8 and abs(relres - r.relres_true) <= 1e-10
    if wl.name in GOLDEN:
        assert abs(r.iters - GOLDEN[wl.name]["iters"]) <= 3, (r.iters, GOLDEN[wl.name]["iters"])
    s.close()


_ORACLE = {}


def oracle_solve(wl):
    """The oracle's problem and its full FGMRES solve (Sec. 4), once per workload."""
    if wl.name not in _ORACLE:
        pb = osolver.build_problem(wl)
        _ORACLE[wl.name] = (pb, pb.solve())
    return _ORACLE[wl.name]


@pytest.mark.parametrize("prec,slack", [(pkg.HELM_FP64, 1), (pkg.HELM_MIXED, 3)], ids=["fp64", "mixed"])
def test_fullsize_solution_matches_oracle(prec, slack):
    """The benchmark's workload (2D P1, h = 1/512, k = 200) in both forms against the oracle's
    own solve: iterations within +-1 (FP64) / +-3 (complex64 preconditioner), true residual
    <= 1e-8, and the solution within 1e-5 normwise and entry by entry in every DoF class."""
    wl = hi.GAUSS_P1
    pb, ref = oracle_solve(wl)
    assert ref.iters == GOLDEN[wl.name]["iters"]
    s = pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim, restart=wl.restart, maxit=wl.maxit, tol=wl.tol,
                   precision=prec)
    x, r = s.solve(dev(pb.F))
    xh = x.cpu().numpy()
    s.close()
    relres = np.linalg.norm(pb.F - pb.A0 @ xh) / np.linalg.norm(pb.F)
    assert r.status == "converged" and relres <= 1e-8 and abs(relres - r.relres_true) <= 1e-10
    assert abs(r.iters - ref.iters) <= slack, (r.iters, ref.iters)
    assert np.linalg.norm(xh - ref.x) / np.linalg.norm(ref.x) <= 1e-5
    assert_entrywise(xh, ref.x, pb.mesh.coords, 1e-5, "solution")


@pytest.mark.parametrize("prec,tol", [(pkg.HELM_FP64, 1e-10), (pkg.HELM_MIXED, 1e-4)])
def test_grid_coarse_solve_residual(prec, tol):
    """3D P1 n=68: coarse planes of 35^2 = 1225 DoFs exceed one 16-CTA cluster, so the
    coarse solve runs the cooperative whole-grid kernel."""
    n, k = 68, 16.0
    shift = 0.5 * k * k
    cmesh = fem.build_mesh(3, 1, n // 2)
    Kc, Mc, Bc = fem.assemble(cmesh)
    Ac = fem.system_matrix(Kc, Mc, Bc, k, shift)
    s = pkg.Solver(k, n, 1, shift, dim=3, precision=prec)
    assert s.num_coarse_dofs == 35 ** 3
    g = np.random.default_rng(5)
    rc = g.standard_normal(s.num_coarse_dofs) + 1j * g.standard_normal(s.num_coarse_dofs)
    uc = s.coarse_solve(dev(rc)).cpu().numpy()
    assert np.linalg.norm(Ac @ uc - rc) / np.linalg.norm(rc) <= tol
    s.close()
