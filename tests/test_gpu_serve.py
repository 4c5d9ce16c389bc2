"""Request server (helm_server_*): continuous batching of independent solves.

Every request solved in a mix of concurrent requests must give the same
result as the same request solved alone, and admission must respect the
device-memory budget."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import helm_inputs as hi  # noqa: E402

MIX = [  # (k, n, order, shift factor of k^2, dim, precision)
    (20.0, 32, 1, 0.5, 2, "mixed"),
    (30.0, 64, 1, 0.25, 2, "fp64"),
    (15.0, 16, 2, 0.5, 2, "mixed"),
    (25.0, 32, 2, 1.0, 2, "mixed"),
    (10.0, 8, 1, 0.5, 3, "mixed"),
    (40.0, 48, 1, 0.5, 2, "fp64"),
]


def _req(pkg, k, n, order, sf, dim, prec):
    p = pkg.HELM_MIXED if prec == "mixed" else pkg.HELM_FP64
    return pkg.make_request(k, n, order, sf * k * k, dim=dim, restart=30, maxit=300, tol=1e-8, precision=p)


def _load(pkg, req, seed):
    return torch.from_numpy(hi.random_load(pkg.num_dofs(req), seed))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2104_01439_gb300 as p
    return p


def test_mix_equals_alone(pkg):
    reqs = [_req(pkg, *m) for m in MIX]
    Fs = [_load(pkg, r, 100 + i) for i, r in enumerate(reqs)]
    # alone: one solver at a time through the ordinary API
    alone = []
    for (k, n, order, sf, dim, prec), F in zip(MIX, Fs):
        s = pkg.Solver(k, n, order, sf * k * k, dim=dim, restart=30, maxit=300, tol=1e-8,
                       precision=pkg.HELM_MIXED if prec == "mixed" else pkg.HELM_FP64)
        x, r = s.solve(F.cuda())
        alone.append((x.cpu(), r))
        s.close()
    # mixed: all submitted at once, all in flight together
    xs = [torch.empty_like(F) for F in Fs]
    with pkg.Server(budget_bytes=8 << 30, max_active=len(reqs)) as srv:
        tickets = [srv.submit(r, F, x) for r, F, x in zip(reqs, Fs, xs)]
        infos = [srv.wait(t) for t in tickets]
    # every request was admitted before the first one finished (they were in flight together)
    assert max(i.t_admit for i in infos) < min(i.t_done for i in infos)
    for (xa, ra), xm, info in zip(alone, xs, infos):
        assert info.rc == 0
        assert info.result.status == "converged" == ra.status
        assert info.result.iters == ra.iters
        err = (xm - xa).abs().max().item() / xa.abs().max().item()
        assert err <= 1e-12, err


def test_budget_admission(pkg):
    reqs = [_req(pkg, 20.0 + 5 * i, 64, 1, 0.5, 2, "mixed") for i in range(6)]
    need = max(pkg.request_bytes(r) for r in reqs)
    budget = int(2.5 * need)   # at most two requests fit at once
    Fs = [_load(pkg, r, 7 + i) for i, r in enumerate(reqs)]
    with pkg.Server(budget_bytes=budget, max_active=8) as srv:
        tickets = [srv.submit(r, F) for r, F in zip(reqs, Fs)]
        too_big = srv.submit(_req(pkg, 50.0, 512, 1, 0.5, 2, "fp64"), torch.zeros(513 * 513, dtype=torch.complex128))
        infos = [srv.wait(t) for t in tickets]
        big = srv.wait(too_big)
    assert big.rc == -2   # HELM_ENOMEM: can never fit
    for i in infos:
        assert i.rc == 0 and i.result.status == "converged"
        assert i.t_submit <= i.t_admit <= i.t_start <= i.t_done
    # at every admission instant, the bytes of requests in flight stay within the budget
    for a in infos:
        live = sum(b.bytes for b in infos if b.t_admit <= a.t_admit < b.t_done)
        assert live <= budget
    assert max(sum(1 for b in infos if b.t_admit <= a.t_admit < b.t_done) for a in infos) <= 2


def test_estimate_covers_handle(pkg):
    """The server's reservation covers what a handle actually holds."""
    import ctypes
    from paper_2104_01439_gb300 import _binding
    for k, n, order, sf, dim, prec in MIX:
        req = _req(pkg, k, n, order, sf, dim, prec)
        s = pkg.Solver(k, n, order, sf * k * k, dim=dim, restart=30, maxit=300, tol=1e-8,
                       precision=req.opts.precision)
        held = ctypes.c_size_t()
        assert _binding.load().helm_device_bytes(s.handle, ctypes.byref(held)) == 0
        est = pkg.request_bytes(req)
        assert held.value + 2 * 16 * s.num_dofs <= est <= 4 * held.value + (8 << 20), (held.value, est)
        s.close()
