"""GB300 (sm_103a) semi matrix-free twogrid-preconditioned FGMRES for Helmholtz.

FGMRES on A0 = A(k,0) right-preconditioned by one twogrid V-cycle on the
complex-shifted operator A(k,eps) (arXiv 2104.01439, Sec. 4), with the hot
path in the CUDA library libhelm.so behind the C ABI of include/helm.h.
"""
from ._binding import (HELM_FP64, HELM_MIXED, HELM_SIMPLICES, HELM_TENSOR, HelmError, Server, Solver,  # noqa: F401
                       SolveResult, TicketInfo, batch_solve, load, load_planewave, make_request, num_dofs,
                       request_bytes)

__all__ = ["HELM_FP64", "HELM_MIXED", "HELM_SIMPLICES", "HELM_TENSOR", "HelmError", "Server", "Solver",
           "SolveResult", "TicketInfo", "batch_solve", "load", "load_planewave", "make_request", "num_dofs",
           "request_bytes"]
