"""CPU-side checks of the C ABI library: it builds, loads, and exports every
function declared in include/helm.h; host-only entry points (request sizing, load
vectors) are exercised; no GPU compute call is made."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "helm.h")


def _declared():
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(helm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_api():
    names = _declared()
    for n in ("helm_setup", "helm_solve", "helm_batch_solve", "helm_destroy", "helm_strerror"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    pytest.importorskip("torch")
    from paper_2104_01439_gb300 import _binding, build
    path = build.build()
    assert os.path.exists(path)
    lib = _binding.load(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_binding.EXPORTS) == set(_declared())
    # every entry point has its argument types declared (ctypes would otherwise pass Python
    # floats and ints with default conversions)
    assert not [n for n in _binding.EXPORTS if getattr(lib, n).argtypes is None]
    # pure host functions are safe to call without a GPU
    assert lib.helm_strerror(-4).decode().startswith("zero")
    o = _binding.HelmOpts()
    lib.helm_default_opts(o)
    assert (o.dim, o.nu, o.restart, o.maxit) == (2, 2, 50, 500)
    assert abs(o.omega - 0.6) < 1e-15 and abs(o.tol - 1e-8) < 1e-20


def test_product_path_has_no_cpu_fallback():
    """The package must not import the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2104_01439_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, flags=re.M), f


def test_request_bytes_estimate_is_host_only_and_consistent():
    """helm_request_bytes is pure host arithmetic: monotone in the mesh and the restart
    length, and it counts the dense coarse blocks (nb * B^2 entries) of each form."""
    pytest.importorskip("torch")
    from paper_2104_01439_gb300 import _binding, build
    _binding.load(build.build())
    rb = lambda **kw: _binding.request_bytes(_binding.make_request(100.0, **kw))  # noqa: E731
    small, big = rb(n=64), rb(n=128)
    assert 0 < small < big
    assert rb(n=128, restart=80) > rb(n=128, restart=50)
    # 2D P1 n=512, mixed: five complex64 coarse matrix sets (Dinv, Lm, Up and the two
    # segment-product sets) of 257 blocks of 257 x 258, plus the double-float factor
    # workspace; FP64: three complex128 sets
    blk = 257 * 257 * 258
    assert rb(n=512, restart=80) > 5 * blk * 8 + blk * 16
    assert rb(n=512, restart=80, precision=_binding.HELM_FP64) > 3 * blk * 16
    with pytest.raises(_binding.HelmError):
        rb(n=63)   # 1/h must be even


def test_binding_refuses_wrong_buffers():
    """The library cannot tell host from device addresses or a buffer's length, so the binding
    refuses mismatches before any call: wrong dtype or layout, a host tensor where a device
    buffer is needed (and the reverse), and buffers shorter than the operand."""
    import torch
    from paper_2104_01439_gb300 import _binding as b
    good = torch.zeros(8, dtype=torch.complex128)
    assert b._ptr(good, 8, device=False).value == good.data_ptr()
    assert b._ptr(good, 5, device=False).value == good.data_ptr()    # a longer buffer is fine
    with pytest.raises(TypeError):
        b._ptr(good, 8)                                              # host tensor, device expected
    with pytest.raises(ValueError):
        b._ptr(good, 9, device=False)                                # too short
    with pytest.raises(TypeError):
        b._ptr(torch.zeros(8, dtype=torch.complex64), 8, device=False)
    with pytest.raises(TypeError):
        b._ptr(torch.zeros(8, 2, dtype=torch.complex128).t(), 8, device=False)   # not contiguous
    with pytest.raises(TypeError):
        b._ptr(good.numpy(), 8, device=False)                        # not a tensor


@pytest.mark.parametrize("dim,order,n", [(2, 1, 16), (2, 2, 8), (3, 1, 6)])
def test_host_load_builders_match_the_oracle(dim, order, n):
    """helm_load_planewave / helm_load_gaussian run on the host only, so their parity with the
    oracle's load vectors (Sec. 2, F(v) = int f v + int_dOmega g v) is checked here."""
    import ctypes
    import numpy as np
    from oracle import fem
    from paper_2104_01439_gb300 import _binding as b
    lib = b.load()
    mesh = fem.build_mesh(dim, order, n)
    _, M, _ = fem.assemble(mesh)
    k, theta, sigma = 11.0, 0.3, 2.0 / n
    F = np.empty(mesh.num_dofs, dtype=np.complex128)
    ptr = ctypes.c_void_p(F.ctypes.data)
    assert lib.helm_load_planewave(dim, order, 1.0 / n, k, theta, ptr) == 0
    ref = fem.load_planewave(mesh, M, k, theta)
    assert np.linalg.norm(F - ref) <= 1e-12 * np.linalg.norm(ref)
    assert lib.helm_load_gaussian(dim, order, 1.0 / n, sigma, 0.5, 0.5, 0.5, ptr) == 0
    ref = fem.load_gaussian(mesh, M, sigma)
    assert np.linalg.norm(F - ref) <= 1e-12 * np.linalg.norm(ref)


def test_host_load_builders_refuse_bad_meshes():
    import ctypes
    import numpy as np
    from paper_2104_01439_gb300 import _binding as b
    lib = b.load()
    F = np.zeros(4, dtype=np.complex128)
    ptr = ctypes.c_void_p(F.ctypes.data)
    bad = [(2, 1, 1.0 / 5), (2, 1, 1.0 / 2), (3, 2, 1.0 / 8), (4, 1, 1.0 / 8), (2, 1, 1e-7),
           (2, 1, 1.0 / 65536), (3, 1, 1.0 / 1024), (2, 1, 0.0), (2, 1, -0.25)]
    einval = int(re.search(r"#define HELM_EINVAL \((-?\d+)\)", open(HEADER).read()).group(1))
    for dim, order, h in bad:
        assert lib.helm_load_planewave(dim, order, h, 10.0, 0.3, ptr) == einval, (dim, order, h)
        assert lib.helm_load_gaussian(dim, order, h, 0.1, 0.5, 0.5, 0.5, ptr) == einval, (dim, order, h)
    assert lib.helm_load_planewave(2, 1, 1.0 / 8, 10.0, 0.3, None) == einval
    assert lib.helm_load_planewave(2, 1, 1.0 / 8, 0.0, 0.3, ptr) == einval
    assert np.all(F == 0)


def test_package_names_used_by_gpu_code_exist():
    """The GPU tests, bench.py and smoke() cannot run without a GPU; every attribute of the package
    module they use must exist, so that none of them fails on a missing name at run time."""
    import glob
    import py_compile
    import paper_2104_01439_gb300 as pkg
    files = glob.glob(os.path.join(ROOT, "tests", "test_*.py")) + [
        os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py"),
        os.path.join(ROOT, "paper_2104_01439_gb300", "sweep.py")]
    used = set()
    for f in files:
        py_compile.compile(f, doraise=True)
        used |= set(re.findall(r"\bpkg\.([A-Za-z_][A-Za-z_0-9]*)", open(f).read()))
    assert used and not [n for n in sorted(used) if not hasattr(pkg, n)]
