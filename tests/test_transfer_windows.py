"""The restriction kernel's gather window covers the support of every column of P (CPU).

k_restrict forms r_c(A) = sum_a P[a][A] r(a) by visiting, on every axis, the fine indices
lo..hi with cmin = ceil(A / q) - 1, lo = max(0, pf cmin), hi = min(W_f - 1, pf floor(A / q) + pf - 1)
(pf = 2q). That formula is restated here and compared with the true support of column A, read
from the product's own transfer weights (helm_host_prolongation_row), for every coarse point of
2D/3D meshes, simplices and tensor-product elements, orders 1 to 3: a window that missed part of
a column would silently drop contributions to the restricted residual.
"""
import ctypes

import pytest

from paper_2104_01439_gb300 import _binding as b


def window(A, q, Wf):
    pf = 2 * q
    cmin = (A + q - 1) // q - 1
    return max(0, pf * cmin), min(Wf - 1, pf * (A // q) + pf - 1)


@pytest.mark.parametrize("dim,order,elements,n", [
    (2, 1, b.HELM_SIMPLICES, 8), (2, 1, b.HELM_SIMPLICES, 10), (2, 2, b.HELM_SIMPLICES, 8),
    (3, 1, b.HELM_SIMPLICES, 6), (2, 1, b.HELM_TENSOR, 8), (2, 2, b.HELM_TENSOR, 10),
    (2, 3, b.HELM_TENSOR, 6), (2, 3, b.HELM_TENSOR, 8), (3, 1, b.HELM_TENSOR, 4)])
def test_restriction_window_covers_every_column(dim, order, elements, n):
    lib = b.load()
    Wf, Wc = order * n + 1, order * (n // 2) + 1
    cap = (order + 1) ** dim
    cols, w, cnt = (ctypes.c_int64 * cap)(), (ctypes.c_double * cap)(), ctypes.c_int()
    support = {}
    for dof in range(Wf ** dim):
        assert lib.helm_host_prolongation_row(dim, order, elements, 1.0 / n, dof, cols, w, ctypes.byref(cnt)) == 0
        a = [(dof // Wf ** ax) % Wf for ax in range(dim)]
        for i in range(cnt.value):
            support.setdefault(cols[i], []).append(a)
    assert len(support) == Wc ** dim                     # every coarse point has a nonempty column
    for col, fine in support.items():
        A = [(col // Wc ** ax) % Wc for ax in range(dim)]
        for ax in range(dim):
            lo, hi = window(A[ax], order, Wf)
            assert all(lo <= f[ax] <= hi for f in fine), (col, ax, lo, hi)
