"""helm_coarse_solve_noalloc: the coarse solve for callers that must not allocate
device memory when they call (fixed memory budget, their own allocator, or no
room for the synchronisation a cudaMalloc may cause). It must give what
helm_coarse_solve gives, call after call, using only the library's fixed 4 MiB
scratch array, and refuse problems that do not fit. Both are also held, entry by
entry, to the oracle's sparse direct solve of its own assembled coarse matrix
(independent of the library's factor). The file's name sorts after every other test
file, so pytest collects it last: a run that stops at the first failure has already run
everything else when it gets here.
"""
import ctypes

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2104_01439_gb300 as pkg  # noqa: E402
from paper_2104_01439_gb300 import _binding  # noqa: E402

HELM_ESCRATCH = -7


def _noalloc(s, rc):
    out = torch.zeros(s.num_coarse_dofs, dtype=torch.complex128, device="cuda")
    code = _binding.load().helm_coarse_solve_noalloc(s.handle, ctypes.c_void_p(rc.data_ptr()),
                                                     ctypes.c_void_p(out.data_ptr()))
    assert code == 0, _binding.load().helm_strerror(code)
    return out


@pytest.mark.parametrize("order,n,k,prec,tol", [
    (1, 36, 12.0, pkg.HELM_FP64, 1e-9),     # ragged coarse blocks (257 -> odd lengths)
    (1, 36, 12.0, pkg.HELM_MIXED, 2e-5),
    (2, 22, 10.0, pkg.HELM_MIXED, 2e-5),    # P2: two lattice lines per block, padded last block
    (1, 512, 200.0, pkg.HELM_FP64, 1e-9),   # the benchmark's coarse grid, near the FP64 limit
])
def test_noalloc_matches_coarse_solve_twice(order, n, k, prec, tol):
    s = pkg.Solver(k, n, order, 0.5 * k * k, precision=prec)
    cmesh = fem.build_mesh(2, order, n // 2)
    Kc, Mc, Bc = fem.assemble(cmesh)
    Ac = fem.system_matrix(Kc, Mc, Bc, k, 0.5 * k * k).tocsc()
    lu = spla.splu(Ac)
    a2 = np.sqrt(spla.norm(Ac, 1) * spla.norm(Ac, np.inf))     # >= ||Ac||_2
    g = np.random.default_rng(17)
    for call in range(2):                   # two calls in a row: no state may leak between calls
        r = g.standard_normal(s.num_coarse_dofs) + 1j * g.standard_normal(s.num_coarse_dofs)
        rc = torch.from_numpy(r).cuda()
        ref = s.coarse_solve(rc).cpu().numpy()
        got = _noalloc(s, rc).cpu().numpy()
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), call
        exact = lu.solve(r)                 # the oracle's coarse matrix, its own direct solve
        for u in (got, ref):
            assert np.max(np.abs(u - exact)) <= tol * np.max(np.abs(exact)), call
            # ||Ac u - r|| = ||Ac (u - exact)|| <= ||Ac|| ||u - exact||
            assert np.linalg.norm(Ac @ u - r) <= tol * a2 * np.linalg.norm(exact), call
    s.close()


def test_noalloc_refuses_problems_beyond_its_scratch():
    # P1 h=1/1024: coarse 513 x 513 -> 2 * 513 * 514 complex64 = 4.2 MB > 4 MiB
    s = pkg.Solver(400.0, 1024, 1, 0.5 * 400.0 ** 2, precision=pkg.HELM_MIXED)
    rc = torch.zeros(s.num_coarse_dofs, dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(rc)
    code = _binding.load().helm_coarse_solve_noalloc(s.handle, ctypes.c_void_p(rc.data_ptr()),
                                                     ctypes.c_void_p(out.data_ptr()))
    assert code == HELM_ESCRATCH
    assert "scratch" in _binding.load().helm_strerror(code).decode()
    s.close()
