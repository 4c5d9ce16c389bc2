"""The GPU smoother against the local Fourier analysis (Sec. 3), independently of the oracle's
sweeps: on the bounded 2D P1 problem, with f = A_eps phi for a Fourier mode phi, nu damped-Jacobi
sweeps from u = 0 (helm_smooth on an operator-only handle) give u = (1 - S~(theta)^nu) phi at
every node more than nu steps from the boundary, S~ the smoother symbol of oracle/lfa.py.

The same check on the CPU with the oracle's sweeps gives 6e-15 (test_oracle_lfa) and 3e-7 with
the sweeps emulated in complex64; the bounds below leave room for the GPU's rounding order.
Only entry points that the other GPU tests validate are used; collected late.
"""
import numpy as np
import pytest

from oracle import fem, lfa

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2104_01439_gb300 as pkg  # noqa: E402


@pytest.mark.parametrize("prec,tol", [(pkg.HELM_FP64, 1e-11), (pkg.HELM_MIXED, 5e-6)])
def test_smoother_multiplies_modes_by_the_lfa_symbol(prec, tol):
    n, k, omega = 32, 12.0, 0.6
    eps = 0.5 * k * k
    mesh = fem.build_mesh(2, 1, n)
    K, M, B = fem.assemble(mesh)
    A = fem.system_matrix(K, M, B, k, eps)
    W, h, lam = n + 1, 1.0 / n, k * k + 1j * eps
    s = pkg.Solver(k, n, 1, eps, omega=omega, precision=prec, operator_only=True)
    i, j = np.meshgrid(np.arange(W), np.arange(W), indexing="xy")
    i, j = i.reshape(-1), j.reshape(-1)
    for theta in [(0.3, -1.1), (2.0, 0.7), (-2.9, 2.5)]:
        phi = np.exp(1j * (theta[0] * i + theta[1] * j))
        f = torch.from_numpy(A @ phi).cuda()
        for nu in (2, 3):
            u = s.smooth(f, nu).cpu().numpy()
            inner = (i > nu) & (i < W - 1 - nu) & (j > nu) & (j < W - 1 - nu)
            expect = (1 - lfa.jacobi_symbol(lfa.P1_KUHN, theta, lam, h, omega) ** nu) * phi
            err = np.abs(u[inner] - expect[inner]).max() / np.abs(expect[inner]).max()
            assert err <= tol, (theta, nu, err)
    s.close()
