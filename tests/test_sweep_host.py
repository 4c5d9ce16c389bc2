"""Host logic of the shift studies (no GPU): the shift-exponent map against the
paper's printed weights, the golden-section search, the best-shift choice, and
the fit of the map (Sec. 5)."""
import math

import numpy as np
import pytest

from oracle import shiftmap
from paper_2104_01439_gb300 import sweep


@pytest.mark.parametrize("p", [1, 2, 3])
def test_map_matches_paper_weights(p):
    w = shiftmap.PAPER_WEIGHTS[p]
    for k in (5.0, 20.0, 80.0, 300.0):
        for ell in (4, 6.5, 8, 10):
            assert abs(float(sweep.shift_exponent(w, k, ell)) - shiftmap.sigma(k, ell, w)) < 1e-14


def test_golden_search_finds_minimum():
    targets = [1.1, 1.37, 1.92]
    calls = []

    def ev(points):
        calls.append(len(points))
        return [(x - targets[i]) ** 2 + 0.1 for i, x in points]

    res = sweep.golden_search(3, ev, tol=1e-2)
    for (x, f, n), t in zip(res, targets):
        assert abs(x - t) < 1e-2
        # two initial evaluations, then the bracket shrinks by 0.618 per evaluation
        assert n == math.ceil(math.log(1e-2) / math.log((math.sqrt(5) - 1) / 2)) + 2
    assert calls[0] == 6 and all(c <= 3 for c in calls[1:])


def _res(k, n, shift, iters, relres):
    s = sweep.Sample(k, n, shift)
    return sweep.SweepResult(s, iters, "converged", relres, relres ** (1 / iters), 0.0, 0.0)


def test_best_shift_tie_breaks():
    r = [_res(20, 64, 100.0, 30, 1e-9), _res(20, 64, 200.0, 28, 9e-9), _res(20, 64, 400.0, 28, 2e-9),
         _res(20, 64, 800.0, 28, 2e-9), _res(50, 128, 10.0, 40, 5e-9)]
    best = sweep.best_shifts(r)
    assert len(best) == 2
    # fewest iterations (28), then the smaller rho (relres 2e-9), then the smaller shift (400)
    assert best[0].sample.shift == 400.0
    assert best[1].sample.k == 50


def test_fit_recovers_map():
    w = shiftmap.PAPER_WEIGHTS[1]
    g = np.random.Generator(np.random.PCG64(11))
    ell = g.choice(np.arange(4, 11), 300).astype(float)
    h = 2.0 ** -ell
    k = g.uniform(3 / (16 * h), 3 / (4 * h))
    y = sweep.shift_exponent(w, k, ell)
    p, loss = sweep.fit_shift_map(k, ell, y, epochs=20_000, lr=1e-2)
    pred = sweep.shift_exponent(p, k, ell)
    assert np.sqrt(np.mean((pred - y) ** 2)) < 0.05


def test_package_weights_are_the_papers():
    for p in (1, 2, 3):
        assert sweep.PAPER_SHIFT_WEIGHTS[p] == shiftmap.PAPER_WEIGHTS[p]
