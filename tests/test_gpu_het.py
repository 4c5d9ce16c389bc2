"""GPU parity of the heterogeneous-wavenumber path (helm_setup_het; Sec. 2 with k in L^inf,
Sec. 6: k(x) = k_max mu(x), one value per element, the coarse operator rediscretised from the
coarse elements' own values) against the oracle's solver.build_problem_het /
solver.build_problem_q with the same profile, through the C ABI.

The wavenumber arrays are filled in the element order helm_host_het_row documents (centroids
computed as in test_host_het); the oracle evaluates the profile at its own elements. Profiles:
the synthetic wedge and a seeded piecewise-constant cell profile (helm_inputs). Tolerances as in
test_gpu_parity: applies <= 1e-12, FP64 coarse solve and V-cycle <= 1e-9, complex64 <= 2e-5,
solves to relres 1e-8 with iterations within +-1 (FP64) / +-3 (complex64 preconditioner) and
the solution within 1e-5, all also entry by entry per DoF class.
"""
import numpy as np
import pytest

import helm_inputs as hi
from oracle import fem, qfem, solver as osolver
from parity import assert_entrywise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2104_01439_gb300 as pkg  # noqa: E402
from test_host_het import documented_centroids  # noqa: E402


def wedge(x):
    return hi.wedge_profile(x)


def cells(x):
    return hi.cell_profile(x, 4, 11)


CASES = [   # name, dim, order, elements, n, k_max, shift, profile
    ("p1_wedge_n64", 2, 1, pkg.HELM_SIMPLICES, 64, 30.0, 0.5 * 30.0 ** 2, wedge),
    ("p1_cells_n36", 2, 1, pkg.HELM_SIMPLICES, 36, 16.0, 16.0 ** 1.5, cells),
    ("p2_cells_n22", 2, 2, pkg.HELM_SIMPLICES, 22, 12.0, 0.5 * 12.0 ** 2, cells),
    ("p1_3d_cells_n8", 3, 1, pkg.HELM_SIMPLICES, 8, 6.0, 0.5 * 6.0 ** 2, cells),
    ("q1_wedge_n32", 2, 1, pkg.HELM_TENSOR, 32, 20.0, 0.5 * 20.0 ** 2, wedge),
]
_PB = {}


def problem(case):
    name, dim, order, elements, n, kmax, shift, mu = case
    if name not in _PB:
        wl = hi.Workload(name, dim, order, n, kmax, shift, "source", restart=50)
        pb = (osolver.build_problem_q(wl, mu) if elements == pkg.HELM_TENSOR
              else osolver.build_problem_het(wl, mu))
        kf = kmax * mu(documented_centroids(dim, n, elements))
        kc = kmax * mu(documented_centroids(dim, n // 2, elements))
        _PB[name] = (wl, pb, kf, kc)
    return _PB[name]


def make(case, **kw):
    wl, pb, kf, kc = problem(case)
    return pkg.Solver(wl.k, wl.n, wl.order, wl.shift, dim=wl.dim, elements=case[3], k_fine=kf, k_coarse=kc,
                      restart=wl.restart, maxit=wl.maxit, tol=wl.tol, **kw)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def crand(n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(n) + 1j * g.standard_normal(n)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_apply_het(case):
    wl, pb, _, _ = problem(case)
    s = make(case)
    assert s.num_dofs == pb.mesh.num_dofs and s.reused_blocks == 0
    x = crand(s.num_dofs, 7)
    for which, A in ((0, pb.A0), (1, pb.Aeps)):
        y = s.apply(dev(x), which).cpu().numpy()
        assert rel(y, A @ x) <= 1e-12
        assert_entrywise(y, A @ x, pb.mesh.coords, 1e-12, f"A{which} x")
    s.close()


@pytest.mark.parametrize("prec,tol", [(pkg.HELM_FP64, 1e-9), (pkg.HELM_MIXED, 2e-5)], ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_coarse_solve_and_vcycle_het(case, prec, tol):
    wl, pb, _, _ = problem(case)
    s = make(case, precision=prec)
    r = crand(s.num_coarse_dofs, 11)
    uc, ucr = s.coarse_solve(dev(r)).cpu().numpy(), pb.twogrid().coarse_solve(r)
    assert rel(uc, ucr) <= tol
    assert_entrywise(uc, ucr, pb.cmesh.coords, tol, "coarse solve")
    f = crand(s.num_dofs, 13)
    u, ur = s.vcycle(dev(f)).cpu().numpy(), pb.twogrid().apply(f)
    assert rel(u, ur) <= tol
    assert_entrywise(u, ur, pb.mesh.coords, tol, "V-cycle")
    s.close()


@pytest.mark.parametrize("prec", [pkg.HELM_FP64, pkg.HELM_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_solve_het(case, prec):
    wl, pb, _, _ = problem(case)
    ref = pb.solve()
    s = make(case, precision=prec)
    F = s.rhs_source().numpy()
    assert rel(F, pb.F) <= 1e-12                      # the paper's source, built by the library
    x, res = s.solve(dev(pb.F))
    xh = x.cpu().numpy()
    relres = np.linalg.norm(pb.F - pb.A0 @ xh) / np.linalg.norm(pb.F)
    assert res.status == "converged" and relres <= 1e-8 and abs(relres - res.relres_true) <= 1e-10
    slack = 1 if prec == pkg.HELM_FP64 else 3
    assert abs(res.iters - ref.iters) <= slack, (res.iters, ref.iters)
    assert rel(xh, ref.x) <= 1e-5
    assert_entrywise(xh, ref.x, pb.mesh.coords, 1e-5, "solution")
    s.close()


def test_het_refuses_bad_input():
    import ctypes
    from paper_2104_01439_gb300 import _binding as b
    lib = b.load()
    n = 8
    ne = 2 * n * n
    kf = (ctypes.c_double * ne)(*([5.0] * ne))
    kc = (ctypes.c_double * (ne // 4))(*([5.0] * (ne // 4)))
    h = ctypes.c_void_p()
    einval = -1
    assert lib.helm_setup_het(b.HELM_SIMPLICES, None, kc, 1.0 / n, 1, 12.5, None, ctypes.byref(h)) == einval
    kf[3] = float("nan")
    assert lib.helm_setup_het(b.HELM_SIMPLICES, kf, kc, 1.0 / n, 1, 12.5, None, ctypes.byref(h)) == einval
    kf[3] = 5.0
    kc[0] = -1.0
    assert lib.helm_setup_het(b.HELM_SIMPLICES, kf, kc, 1.0 / n, 1, 12.5, None, ctypes.byref(h)) == einval
