"""Shift studies on the GPU: batched shift sweeps, the best-shift table, the
paper's golden-section search for the optimal shift exponent, and the fit of
the shift-exponent map (Sec. 5, data generation and processing).

Every solve runs through the request server (include/helm.h, helm_server_*),
so all samples of a sweep are in flight on the GPU together, admitted by a
device-memory budget. The host side only builds load vectors, groups results
and fits the four coefficients of the map.

Shift convention: eps = k^sigma with the exponent sigma in [1, 2] (Sec. 3 and
Sec. 5), i.e. sigma = log(eps) / log(k).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import _binding as B


@dataclass
class Sample:
    k: float
    n: int
    shift: float
    order: int = 1
    dim: int = 2

    @property
    def ell(self) -> float:
        """Mesh level l = log2(1/h) (real-valued for meshes that are not powers of two)."""
        return math.log2(self.n)

    @property
    def sigma(self) -> float:
        return math.log(self.shift) / math.log(self.k)


@dataclass
class SweepResult:
    sample: Sample
    iters: int
    status: str
    relres: float
    rho: float          # average convergence rate (r_end / r_0)^(1 / end), r_0 = ||F|| (x0 = 0)
    latency_s: float
    setup_ms: float


def run_sweep(samples, theta: float = 0.3, restart: int = 50, maxit: int = 500, tol: float = 1e-8,
              precision: int = B.HELM_MIXED, budget_bytes: int = 64 << 30, max_active: int = 16, loads=None):
    """Solve every sample (plane-wave load vector with direction theta unless `loads` gives
    host load vectors) through one request server; returns a SweepResult per sample."""
    out = [None] * len(samples)
    with B.Server(budget_bytes, max_active) as srv:
        tickets = []
        for i, s in enumerate(samples):
            req = B.make_request(s.k, s.n, s.order, s.shift, dim=s.dim, restart=restart, maxit=maxit, tol=tol,
                                 precision=precision)
            F = loads[i] if loads is not None else B.load_planewave(req, theta)
            tickets.append(srv.submit(req, F))
        for i, t in enumerate(tickets):
            info = srv.wait(t)
            if info.rc != 0:
                raise B.HelmError(f"sample {i} failed with code {info.rc}")
            r = info.result
            rho = r.relres_true ** (1.0 / max(r.iters, 1)) if r.relres_true > 0 else 0.0
            out[i] = SweepResult(samples[i], r.iters, r.status, r.relres_true, rho, info.latency, info.setup_ms)
    return out


def best_shifts(results):
    """Per (k, n, order): the sample with the fewest iterations; ties go to the smaller
    average convergence rate rho, then to the smaller shift."""
    groups = {}
    for r in results:
        key = (r.sample.k, r.sample.n, r.sample.order, r.sample.dim)
        groups.setdefault(key, []).append(r)
    best = []
    for key in sorted(groups):
        g = groups[key]
        best.append(min(g, key=lambda r: (r.iters, r.rho, r.sample.shift)))
    return best


def golden_search(count: int, evaluate, tol: float = 1e-2, lo: float = 1.0, hi: float = 2.0):
    """Golden-section minimisation of `count` independent objectives on [lo, hi] to a bracket
    of width tol, advanced together: evaluate(points) takes a list of (problem index, x)
    and returns the objective values in the same order. Returns (x_hat, f_hat, evaluations)
    per problem."""
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a = [lo] * count
    b = [hi] * count
    c = [hi - g * (hi - lo)] * count
    d = [lo + g * (hi - lo)] * count
    vals = evaluate([(i, c[i]) for i in range(count)] + [(i, d[i]) for i in range(count)])
    fc, fd = list(vals[:count]), list(vals[count:])
    evals = [2] * count
    while True:
        todo = [i for i in range(count) if b[i] - a[i] > tol]
        if not todo:
            break
        pts = []
        for i in todo:
            if fc[i] < fd[i]:            # minimum in [a, d]
                b[i], d[i], fd[i] = d[i], c[i], fc[i]
                c[i] = b[i] - g * (b[i] - a[i])
                pts.append((i, c[i], True))
            else:                        # minimum in [c, b]
                a[i], c[i], fc[i] = c[i], d[i], fd[i]
                d[i] = a[i] + g * (b[i] - a[i])
                pts.append((i, d[i], False))
        vals = evaluate([(i, x) for i, x, _ in pts])
        for (i, _, is_c), v in zip(pts, vals):
            if is_c:
                fc[i] = v
            else:
                fd[i] = v
            evals[i] += 1
    return [((c[i], fc[i]) if fc[i] < fd[i] else (d[i], fd[i])) + (evals[i],) for i in range(count)]


def golden_section(problems, tol: float = 1e-2, maxit: int = 50, precision: int = B.HELM_MIXED,
                   budget_bytes: int = 64 << 30, max_active: int = 16, seed: int = 0):
    """The paper's search for the optimal exponent sigma in [1, 2] of the shift k^sigma
    (Sec. 5, data generation): objective rho = (r_end / r_0)^(1/end) of FGMRES stopped at
    relres 1e-8 or `maxit` iterations (no restart), load vector with entries uniform in
    [-1, 1] and g = 0, golden-section search to a bracket of width tol. All searches advance
    together: every round submits one solve per unfinished search to the request server.

    problems: list of (k, n, order). Returns a list of (sigma_hat, rho_hat, evaluations)."""
    import torch

    import helm_inputs
    loads = [torch.from_numpy(F) for F in
             helm_inputs.uniform_loads([(order * n + 1) ** 2 for k, n, order in problems], seed)]

    def evaluate(points):
        samples = [Sample(problems[i][0], problems[i][1], problems[i][0] ** x, problems[i][2]) for i, x in points]
        res = run_sweep(samples, restart=maxit, maxit=maxit, tol=1e-8, precision=precision,
                        budget_bytes=budget_bytes, max_active=max_active, loads=[loads[i] for i, _ in points])
        return [r.rho for r in res]

    return golden_search(len(problems), evaluate, tol)


# ---------------------------------------------------------------------------- the map

# (kc0, kc1, a0, a1) per element order p as printed in Sec. 5, Table tab:optweights
# (fitted by the paper for its Q_p elements); a default map until a sweep is fitted.
PAPER_SHIFT_WEIGHTS = {
    1: (0.4592788619853418, 2.5790032999702346, -0.6261637288068426, 1.7580549857142198),
    2: (0.5736926870738827, 2.5729974893966001, -0.6615199737374460, 1.5966386518185063),
    3: (0.6305770719029798, 2.4284320222555804, -0.4465407372367102, 0.1287828338493968),
}

def shift_exponent(params, k, ell):
    """Sec. 5, eq. shiftexp: sigma_p(k, l) = min(max(2 - exp(-alpha(l) (k - k_c(l))), 1), 2) with
    k_c(l) = kc1 exp(kc0 l) and alpha(l) = a1 exp(a0 l); params = (kc0, kc1, a0, a1)."""
    kc0, kc1, a0, a1 = params
    k = np.asarray(k, dtype=np.float64)
    ell = np.asarray(ell, dtype=np.float64)
    kc = kc1 * np.exp(kc0 * ell)
    alpha = a1 * np.exp(a0 * ell)
    beta = 2.0 - np.exp(-alpha * (k - kc))
    return np.clip(beta, 1.0, 2.0)


def shift_of(params, k, n):
    """eps = k^sigma for the mesh with n elements per side."""
    return float(k) ** float(shift_exponent(params, k, math.log2(n)))


def fit_shift_map(k, ell, sigma_hat, init=(0.1, 1.0, -0.5, 1.0), epochs: int = 50_000, lr: float = 1e-3):
    """Fit (kc0, kc1, a0, a1) as in Sec. 5: loss = sum_i w_{l_i}^{-2} (sigma_hat_i - sigma(k_i, l_i))^2
    with w_l = (samples at level l) / (all samples), minimised by Adam (learning rate 1e-3,
    initial weights (0.1, 1.0, -0.5, 1.0), 50 000 epochs). The clamp to [1, 2] passes no
    gradient where it is active (as automatic differentiation of min/max does).
    Levels are grouped after rounding l to 1e-9, so real-valued l (non-power-of-two meshes)
    each form their own level."""
    k = np.asarray(k, dtype=np.float64)
    ell = np.asarray(ell, dtype=np.float64)
    y = np.asarray(sigma_hat, dtype=np.float64)
    lv = np.round(ell, 9)
    _, inv, cnt = np.unique(lv, return_inverse=True, return_counts=True)
    w = (cnt / len(lv))[inv]
    wt = w ** -2.0
    p = np.array(init, dtype=np.float64)
    m1 = np.zeros(4)
    m2 = np.zeros(4)
    b1, b2, eps = 0.9, 0.999, 1e-8
    for t in range(1, epochs + 1):
        kc0, kc1, a0, a1 = p
        ekc = np.exp(kc0 * ell)
        ea = np.exp(a0 * ell)
        kc = kc1 * ekc
        alpha = a1 * ea
        e = np.exp(-alpha * (k - kc))
        beta = 2.0 - e
        inside = (beta > 1.0) & (beta < 2.0)
        pred = np.clip(beta, 1.0, 2.0)
        r = pred - y
        gpred = 2.0 * wt * r * inside              # d loss / d beta
        # d beta / d alpha = e (k - kc);  d beta / d kc = -e alpha
        g_alpha = gpred * e * (k - kc)
        g_kc = gpred * (-e * alpha)
        grad = np.array([np.sum(g_kc * kc1 * ekc * ell), np.sum(g_kc * ekc),
                         np.sum(g_alpha * a1 * ea * ell), np.sum(g_alpha * ea)])
        m1 = b1 * m1 + (1 - b1) * grad
        m2 = b2 * m2 + (1 - b2) * grad * grad
        p = p - lr * (m1 / (1 - b1 ** t)) / (np.sqrt(m2 / (1 - b2 ** t)) + eps)
    loss = float(np.sum(wt * (shift_exponent(p, k, ell) - y) ** 2))
    return p, loss
