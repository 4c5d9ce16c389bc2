"""Thin ctypes binding of include/helm.h (argument marshalling only).

Every computation happens in libhelm.so's CUDA kernels. Device buffers are
PyTorch complex128 CUDA tensors (interleaved re/im doubles); the library runs
on the CUDA stream given at setup (default: PyTorch's current stream).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhelm.so")

HELM_OK = 0
HELM_SIMPLICES = 0
HELM_TENSOR = 1
HELM_FP64 = 0
HELM_MIXED = 1
STATUS = {0: "converged", 1: "maxit", 2: "breakdown", 3: "nonfinite"}

EXPORTS = [
    "helm_default_opts", "helm_setup", "helm_last_cuda_error", "helm_num_dofs", "helm_num_coarse_dofs", "helm_setup_info",
    "helm_solve", "helm_solve_host", "helm_batch_solve", "helm_destroy", "helm_strerror",
    "helm_rhs_planewave", "helm_rhs_gaussian", "helm_apply", "helm_vcycle", "helm_coarse_solve",
    "helm_last_profile", "helm_set_profiling", "helm_coarse_solve_noalloc",
    "helm_request_bytes", "helm_device_bytes", "helm_server_create", "helm_server_submit", "helm_server_poll",
    "helm_server_wait", "helm_server_drain", "helm_server_destroy", "helm_load_planewave", "helm_load_gaussian",
    "helm_operator_setup", "helm_smooth", "helm_host_stencil_row", "helm_host_prolongation_row",
    "helm_setup_q", "helm_load_planewave_e", "helm_load_gaussian_e", "helm_host_het_row",
    "helm_factor_info", "helm_setup_het", "helm_rhs_source",
]


class HelmOpts(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("omega", ctypes.c_double), ("nu", ctypes.c_int),
                ("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("tol", ctypes.c_double),
                ("precision", ctypes.c_int), ("stream", ctypes.c_void_p)]


class HelmResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("status", ctypes.c_int),
                ("relres_true", ctypes.c_double), ("relres_est", ctypes.c_double),
                ("solve_ms", ctypes.c_float), ("kernels", ctypes.c_int)]


class HelmRequest(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("h", ctypes.c_double), ("order", ctypes.c_int), ("shift", ctypes.c_double),
                ("opts", HelmOpts)]


class HelmTicketInfo(ctypes.Structure):
    _fields_ = [("rc", ctypes.c_int), ("res", HelmResult), ("setup_ms", ctypes.c_float),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("bytes", ctypes.c_size_t)]


class HelmError(RuntimeError):
    pass


_lib = None


def load(path: str = LIB_PATH):
    """Load libhelm.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise HelmError(f"{path} not found: build it with paper_2104_01439_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i, d, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)
    lib.helm_default_opts.argtypes = [ctypes.POINTER(HelmOpts)]
    lib.helm_default_opts.restype = None
    lib.helm_setup.argtypes = [d, d, i, d, ctypes.POINTER(HelmOpts), ctypes.POINTER(vp)]
    lib.helm_num_dofs.argtypes = [vp, i64p]
    lib.helm_num_coarse_dofs.argtypes = [vp, i64p]
    lib.helm_setup_info.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)]
    lib.helm_factor_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.helm_solve.argtypes = [vp, vp, vp, ctypes.POINTER(HelmResult)]
    lib.helm_solve_host.argtypes = [vp, vp, vp, ctypes.POINTER(HelmResult)]
    lib.helm_batch_solve.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(HelmResult)]
    lib.helm_destroy.argtypes = [vp]
    lib.helm_destroy.restype = None
    lib.helm_strerror.argtypes = [i]
    lib.helm_strerror.restype = ctypes.c_char_p
    lib.helm_last_cuda_error.argtypes = []
    lib.helm_last_cuda_error.restype = ctypes.c_char_p
    lib.helm_rhs_planewave.argtypes = [vp, d, vp]
    lib.helm_rhs_gaussian.argtypes = [vp, d, d, d, d, vp]
    lib.helm_apply.argtypes = [vp, i, vp, vp]
    lib.helm_vcycle.argtypes = [vp, vp, vp]
    lib.helm_coarse_solve.argtypes = [vp, vp, vp]
    lib.helm_last_profile.argtypes = [vp, i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(d),
                                      ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.helm_set_profiling.argtypes = [vp, i]
    lib.helm_coarse_solve_noalloc.argtypes = [vp, vp, vp]
    szp = ctypes.POINTER(ctypes.c_size_t)
    lib.helm_request_bytes.argtypes = [ctypes.POINTER(HelmRequest), szp]
    lib.helm_device_bytes.argtypes = [vp, szp]
    lib.helm_server_create.argtypes = [ctypes.c_size_t, i, ctypes.POINTER(vp)]
    lib.helm_server_submit.argtypes = [vp, ctypes.POINTER(HelmRequest), vp, vp, i64p]
    lib.helm_server_poll.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(i), ctypes.POINTER(HelmTicketInfo)]
    lib.helm_server_wait.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(HelmTicketInfo)]
    lib.helm_server_drain.argtypes = [vp]
    lib.helm_server_destroy.argtypes = [vp]
    lib.helm_server_destroy.restype = None
    lib.helm_load_planewave.argtypes = [i, i, d, d, d, vp]
    lib.helm_operator_setup.argtypes = [d, d, i, d, ctypes.POINTER(HelmOpts), ctypes.POINTER(vp)]
    lib.helm_setup_q.argtypes = [d, d, i, d, ctypes.POINTER(HelmOpts), ctypes.POINTER(vp)]
    lib.helm_setup_het.argtypes = [i, ctypes.POINTER(d), ctypes.POINTER(d), d, i, d, ctypes.POINTER(HelmOpts),
                                   ctypes.POINTER(vp)]
    lib.helm_rhs_source.argtypes = [vp, d, d, d, vp]
    lib.helm_load_planewave_e.argtypes = [i, i, i, d, d, d, vp]
    lib.helm_load_gaussian_e.argtypes = [i, i, i, d, d, d, d, d, vp]
    lib.helm_smooth.argtypes = [vp, vp, vp, i]
    lib.helm_load_gaussian.argtypes = [i, i, d, d, d, d, d, vp]
    dp = ctypes.POINTER(ctypes.c_double)
    lib.helm_host_stencil_row.argtypes = [i, i, i, d, i, ctypes.c_int64, dp, dp, dp]
    lib.helm_host_prolongation_row.argtypes = [i, i, i, d, ctypes.c_int64, i64p, dp, ctypes.POINTER(i)]
    lib.helm_host_het_row.argtypes = [i, i, i, d, i, dp, ctypes.c_int64, dp, dp, dp, dp]
    for name in EXPORTS:
        if name not in ("helm_default_opts", "helm_destroy", "helm_strerror", "helm_last_cuda_error",
                        "helm_server_destroy"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def _check(rc: int):
    if rc != HELM_OK:
        lib = load()
        raise HelmError(f"helm error {rc}: {lib.helm_strerror(rc).decode()} "
                        f"(last CUDA error: {lib.helm_last_cuda_error().decode()})")


@dataclass
class SolveResult:
    iters: int
    cycles: int
    status: str
    relres_true: float
    relres_est: float
    solve_ms: float
    kernels: int


def _res(r: HelmResult) -> SolveResult:
    return SolveResult(r.iters, r.cycles, STATUS.get(r.status, str(r.status)), r.relres_true,
                       r.relres_est, r.solve_ms, r.kernels)


def _ptr(t, n=None, device=True):
    """Address of a contiguous complex128 tensor holding at least n values, on the GPU
    (device=True) or in host memory (device=False). The library cannot tell a host address from
    a device one, nor a buffer's length, so a mismatch is refused here instead of reaching a
    kernel or a host copy."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_contiguous():
        raise TypeError("expected a contiguous complex128 tensor")
    if device and not t.is_cuda:
        raise TypeError("expected a CUDA tensor (device buffer)")
    if not device and t.is_cuda:
        raise TypeError("expected a CPU tensor (host buffer)")
    if n is not None and t.numel() < n:
        raise ValueError(f"buffer holds {t.numel()} values, {n} needed")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """A set-up solver for A(k, shift) on the h = 1/n mesh (wraps helm_setup)."""

    def __init__(self, k: float, n: int, order: int = 1, shift: float = 0.0, dim: int = 2,
                 omega: float = 0.6, nu: int = 2, restart: int = 50, maxit: int = 500,
                 tol: float = 1e-8, precision: int = HELM_FP64, stream=None, operator_only: bool = False,
                 elements: int = HELM_SIMPLICES, k_fine=None, k_coarse=None):
        """k_fine / k_coarse (helm_setup_het): one wavenumber per element of the fine and of the
        coarse mesh, in the element order of helm_host_het_row; k is then ignored."""
        import torch
        lib = load()
        o = HelmOpts()
        lib.helm_default_opts(ctypes.byref(o))
        o.dim, o.omega, o.nu, o.restart, o.maxit, o.tol, o.precision = dim, omega, nu, restart, maxit, tol, precision
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o.stream = ctypes.c_void_p(stream.cuda_stream)
        self._h = ctypes.c_void_p()
        self.k, self.n, self.order, self.shift, self.dim, self.precision = k, n, order, shift, dim, precision
        if elements not in (HELM_SIMPLICES, HELM_TENSOR) or (operator_only and elements != HELM_SIMPLICES):
            raise ValueError("elements: HELM_SIMPLICES, or HELM_TENSOR for a full solver handle")
        if k_fine is not None:
            if operator_only or k_coarse is None:
                raise ValueError("a heterogeneous wavenumber needs k_fine and k_coarse and a full solver handle")
            import numpy as np
            kf = np.ascontiguousarray(k_fine, dtype=np.float64)
            kc = np.ascontiguousarray(k_coarse, dtype=np.float64)
            self._k_arrays = (kf, kc)
            dp = ctypes.POINTER(ctypes.c_double)
            _check(lib.helm_setup_het(elements, kf.ctypes.data_as(dp), kc.ctypes.data_as(dp), 1.0 / n, order,
                                      float(shift), ctypes.byref(o), ctypes.byref(self._h)))
        else:
            setup = (lib.helm_operator_setup if operator_only
                     else lib.helm_setup_q if elements == HELM_TENSOR else lib.helm_setup)
            _check(setup(float(k), 1.0 / n, order, float(shift), ctypes.byref(o), ctypes.byref(self._h)))
        nd = ctypes.c_int64()
        _check(lib.helm_num_dofs(self._h, ctypes.byref(nd)))
        self.num_dofs = nd.value
        _check(lib.helm_num_coarse_dofs(self._h, ctypes.byref(nd)))
        self.num_coarse_dofs = nd.value
        ms, nk = ctypes.c_float(), ctypes.c_int()
        _check(lib.helm_setup_info(self._h, ctypes.byref(ms), ctypes.byref(nk)))
        self.setup_ms = ms.value
        self.setup_kernels = nk.value
        self.factored_blocks = self.reused_blocks = 0
        if not operator_only:
            nf, nr = ctypes.c_int(), ctypes.c_int()
            _check(lib.helm_factor_info(self._h, ctypes.byref(nf), ctypes.byref(nr)))
            self.factored_blocks, self.reused_blocks = nf.value, nr.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().helm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, n=None):
        import torch
        return torch.empty(self.num_dofs if n is None else n, dtype=torch.complex128, device="cuda")

    def solve(self, F, x=None) -> tuple:
        x = self._dev() if x is None else x
        r = HelmResult()
        N = self.num_dofs
        _check(load().helm_solve(self._h, _ptr(F, N), _ptr(x, N), ctypes.byref(r)))
        return x, _res(r)

    def solve_host(self, F_host, x_host) -> SolveResult:
        r = HelmResult()
        N = self.num_dofs
        _check(load().helm_solve_host(self._h, _ptr(F_host, N, device=False), _ptr(x_host, N, device=False),
                                      ctypes.byref(r)))
        return _res(r)

    def apply(self, x, which: int = 0, y=None):
        """y = A0 x (which = 0) or A_eps x (which = 1); stream-ordered on the handle's stream."""
        y = self._dev() if y is None else y
        _check(load().helm_apply(self._h, which, _ptr(x, self.num_dofs), _ptr(y, self.num_dofs)))
        return y

    def smooth(self, f, nu: int = 2, u=None):
        """nu damped-Jacobi sweeps on A_eps from u = 0 (helm_smooth); stream-ordered."""
        u = self._dev() if u is None else u
        _check(load().helm_smooth(self._h, _ptr(f, self.num_dofs), _ptr(u, self.num_dofs), int(nu)))
        return u

    def vcycle(self, f):
        u = self._dev()
        _check(load().helm_vcycle(self._h, _ptr(f, self.num_dofs), _ptr(u, self.num_dofs)))
        return u

    def coarse_solve(self, rc):
        uc = self._dev(self.num_coarse_dofs)
        _check(load().helm_coarse_solve(self._h, _ptr(rc, self.num_coarse_dofs), _ptr(uc, self.num_coarse_dofs)))
        return uc

    def rhs_planewave(self, theta: float = 0.3):
        import torch
        F = torch.empty(self.num_dofs, dtype=torch.complex128)
        _check(load().helm_rhs_planewave(self._h, theta, ctypes.c_void_p(F.data_ptr())))
        return F

    def rhs_source(self, center=(0.5, 0.5, 0.5)):
        """The paper's point source f = 2 exp(-1000 |x - s|^2), g = 0 (helm_rhs_source)."""
        import torch
        F = torch.empty(self.num_dofs, dtype=torch.complex128)
        c = list(center) + [0.5] * (3 - len(center))
        _check(load().helm_rhs_source(self._h, c[0], c[1], c[2], ctypes.c_void_p(F.data_ptr())))
        return F

    def rhs_gaussian(self, sigma: float, center=(0.5, 0.5, 0.5)):
        import torch
        F = torch.empty(self.num_dofs, dtype=torch.complex128)
        c = list(center) + [0.5] * (3 - len(center))
        _check(load().helm_rhs_gaussian(self._h, sigma, c[0], c[1], c[2], ctypes.c_void_p(F.data_ptr())))
        return F

    def set_profiling(self, on: bool):
        _check(load().helm_set_profiling(self._h, 1 if on else 0))

    def profile(self) -> dict:
        n = ctypes.c_int()
        names = (ctypes.c_char_p * 16)()
        ms = (ctypes.c_double * 16)()
        calls = (ctypes.c_int * 16)()
        _check(load().helm_last_profile(self._h, 16, names, ms, calls, ctypes.byref(n)))
        return {names[i].decode(): (ms[i], calls[i]) for i in range(n.value)}


def batch_solve(solvers, Fs, xs=None):
    """helm_batch_solve over distinct solvers; returns (xs, results)."""
    n = len(solvers)
    xs = [s._dev() for s in solvers] if xs is None else xs
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    if len(Fs) != n or len(xs) != n:
        raise ValueError("one load vector and one solution buffer per solver")
    fp = (ctypes.c_void_p * n)(*[_ptr(F, s.num_dofs).value for s, F in zip(solvers, Fs)])
    xp = (ctypes.c_void_p * n)(*[_ptr(x, s.num_dofs).value for s, x in zip(solvers, xs)])
    res = (HelmResult * n)()
    _check(load().helm_batch_solve(n, hs, fp, xp, res))
    return xs, [_res(r) for r in res]


# ---------------------------------------------------------------------------- request server

def make_request(k: float, n: int, order: int = 1, shift: float = 0.0, dim: int = 2, omega: float = 0.6,
                 nu: int = 2, restart: int = 50, maxit: int = 500, tol: float = 1e-8,
                 precision: int = HELM_MIXED) -> HelmRequest:
    lib = load()
    o = HelmOpts()
    lib.helm_default_opts(ctypes.byref(o))
    o.dim, o.omega, o.nu, o.restart, o.maxit, o.tol, o.precision = dim, omega, nu, restart, maxit, tol, precision
    return HelmRequest(float(k), 1.0 / n, order, float(shift), o)


def request_bytes(req: HelmRequest) -> int:
    """Peak device bytes the server reserves for one request (host-side estimate)."""
    b = ctypes.c_size_t()
    _check(load().helm_request_bytes(ctypes.byref(req), ctypes.byref(b)))
    return b.value


def num_dofs(req: HelmRequest) -> int:
    n = round(1.0 / req.h)
    return (req.order * n + 1) ** req.opts.dim


@dataclass
class TicketInfo:
    rc: int
    result: SolveResult
    setup_ms: float
    t_submit: float
    t_admit: float
    t_start: float
    t_done: float
    bytes: int

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


def _info(i: HelmTicketInfo) -> TicketInfo:
    return TicketInfo(i.rc, _res(i.res), i.setup_ms, i.t_submit, i.t_admit, i.t_start, i.t_done, i.bytes)


class Server:
    """helm_server_*: admits solve requests by a device-memory budget and overlaps them on the GPU."""

    def __init__(self, budget_bytes: int, max_active: int = 8):
        self._s = ctypes.c_void_p()
        _check(load().helm_server_create(int(budget_bytes), int(max_active), ctypes.byref(self._s)))
        self._keep = {}

    def submit(self, req: HelmRequest, F_host, x_host=None) -> int:
        """F_host: CPU complex128 tensor (copied at once); x_host: CPU complex128 tensor or None."""
        t = ctypes.c_int64()
        N = num_dofs(req)
        xp = _ptr(x_host, N, device=False) if x_host is not None else None
        _check(load().helm_server_submit(self._s, ctypes.byref(req), _ptr(F_host, N, device=False), xp,
                                         ctypes.byref(t)))
        if x_host is not None:
            self._keep[t.value] = x_host   # must outlive the request
        return t.value

    def poll(self, ticket: int):
        done = ctypes.c_int()
        info = HelmTicketInfo()
        _check(load().helm_server_poll(self._s, ticket, ctypes.byref(done), ctypes.byref(info)))
        return _info(info) if done.value else None

    def wait(self, ticket: int) -> TicketInfo:
        info = HelmTicketInfo()
        _check(load().helm_server_wait(self._s, ticket, ctypes.byref(info)))
        self._keep.pop(ticket, None)
        return _info(info)

    def drain(self):
        _check(load().helm_server_drain(self._s))

    def close(self):
        if self._s:
            load().helm_server_destroy(self._s)
            self._s = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_planewave(req: HelmRequest, theta: float = 0.3):
    """Host complex128 load vector of the plane wave exp(i k d.x), d = (cos theta, sin theta)."""
    import torch
    F = torch.empty(num_dofs(req), dtype=torch.complex128)
    _check(load().helm_load_planewave(req.opts.dim, req.order, req.h, req.k, theta, ctypes.c_void_p(F.data_ptr())))
    return F
