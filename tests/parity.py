"""Entry-by-entry comparison of a GPU result with the oracle's, per DoF class.

A normwise bound ||a - b|| / ||b|| lets an error confined to the boundary rows (a few percent of
the DoFs) pass at many times the tolerance. So the parity tests also bound, separately for the
interior DoFs and for each boundary class (DoFs on one side of the square or face of the cube;
on two: the square's corners or the cube's edges; on three: the cube's corners), the largest
entry error relative to the largest entry of the oracle's result.
"""
import numpy as np

CLASS_NAMES = ("interior", "side", "edge/corner", "corner3d")


def dof_classes(coords):
    """Number of domain facets each DoF lies on (0: interior .. dim: corner)."""
    c = np.asarray(coords)
    return (np.isclose(c, 0.0) | np.isclose(c, 1.0)).sum(axis=1)


def classwise_errors(a, b, coords):
    """{class name: max_i |a_i - b_i| / max |b|} over the DoFs of each class present."""
    cls = dof_classes(coords)
    scale = max(np.max(np.abs(b)), 1e-300)
    err = np.abs(np.asarray(a) - np.asarray(b)) / scale
    return {CLASS_NAMES[c]: float(err[cls == c].max()) for c in np.unique(cls)}


def assert_entrywise(a, b, coords, tol, what=""):
    errs = classwise_errors(a, b, coords)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{what}: entry errors above {tol:g} by DoF class: {errs}"
    return errs
