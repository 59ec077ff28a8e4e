"""The C-ABI library builds, loads and exports every entry point declared in include/*.h (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2203_15461_gb300 import cpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(cpm.LIB_PATH):
        from paper_2203_15461_gb300 import build
        build.build()
    return cpm.load_library()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(cpm_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"cpm_create", "cpm_assemble", "cpm_invert", "cpm_bvec", "cpm_update"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    assert _declared() <= set(cpm._SIGS)


def test_create_rejects_bad_arguments_without_touching_a_gpu(lib):
    p = cpm.cpm_params()
    p.box[:] = [10.0, 10.0, -1.0]
    p.alpha, p.rcut, p.kcut = 0.3, 10.0, 2.0
    h = ctypes.c_void_p()
    assert lib.cpm_create(ctypes.byref(p), None, ctypes.byref(h)) == 1   # CPM_E_ARG
    assert lib.cpm_create(None, None, ctypes.byref(h)) == 1
    lib.cpm_destroy(None)


def test_create_rejects_bad_p3m_parameters_without_touching_a_gpu(lib):
    """P3M order outside 2..7, a mesh axis not a power of two in [8, 512], an xy plane beyond 128 KiB of
    complex values, or the 2D Ewald boundary: CPM_E_ARG before any device is looked up."""
    def params(order, mesh, boundary=1, k_prec=1):
        p = cpm.cpm_params()
        p.box[:] = [20.0, 20.0, 60.0]
        p.alpha, p.rcut, p.kcut = 0.3, 10.0, 2.0
        p.boundary, p.k_prec, p.s_prec = boundary, k_prec, 1
        p.kspace, p.p3m_order = 1, order
        p.p3m_mesh[:] = list(mesh)
        return p
    h = ctypes.c_void_p()
    bad = [params(1, (16, 16, 64)), params(8, (16, 16, 64)), params(5, (12, 16, 64)), params(5, (16, 16, 4)),
           params(5, (16, 16, 1024)), params(5, (256, 128, 64)), params(5, (128, 128, 64), k_prec=0),
           params(5, (16, 16, 64), boundary=3)]
    for p in bad:
        assert lib.cpm_create(ctypes.byref(p), None, ctypes.byref(h)) == 1   # CPM_E_ARG
    q = params(5, (16, 16, 64))
    q.kspace = 2
    assert lib.cpm_create(ctypes.byref(q), None, ctypes.byref(h)) == 1
    # the P3M elastance: only with kspace = P3M, 0 or 1, and its FP64 planes within the limit
    for kspace, flag, mesh in ((0, 1, (16, 16, 64)), (1, 2, (16, 16, 64)), (1, 1, (128, 128, 64))):
        r = params(5, mesh)
        r.kspace, r.p3m_matrix = kspace, flag
        assert lib.cpm_create(ctypes.byref(r), None, ctypes.byref(h)) == 1


def test_no_cpu_fallback_without_a_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    p = cpm.cpm_params()
    p.box[:] = [10.0, 10.0, 10.0]
    p.alpha, p.rcut, p.kcut = 0.3, 10.0, 2.0
    h = ctypes.c_void_p()
    assert lib.cpm_create(ctypes.byref(p), None, ctypes.byref(h)) == 6   # CPM_E_CUDA
    with pytest.raises(cpm.CPMError, match="CPM_E_CUDA"):
        cpm.CPM((10, 10, 10), "slab", 0.3, 10.0, 2.0)


def test_noalloc_binding_refuses_bad_buffers_before_any_launch():
    """cpm_bvec_noalloc receives bare device pointers; the binding checks types, sizes and devices first."""
    torch = pytest.importorskip("torch")
    p = cpm.cpm_params()
    p.box[:] = [10.0, 10.0, 30.0]
    p.alpha, p.rcut, p.kcut, p.boundary = 0.3, 9.0, 2.0, 1
    f64 = torch.float64
    sx, se, b = torch.zeros((4, 3), dtype=f64), torch.ones(4, dtype=f64), torch.zeros(4, dtype=f64)
    x, Q = torch.zeros((2, 3), dtype=f64), torch.zeros(2, dtype=f64)
    with pytest.raises(TypeError, match="float64"):
        cpm.cpm_bvec_noalloc(p, sx.float(), se, x, Q, b)
    with pytest.raises(TypeError, match="float64"):
        cpm.cpm_bvec_noalloc(p, sx, se, x, Q, b.float())
    with pytest.raises(ValueError, match="b_out"):
        cpm.cpm_bvec_noalloc(p, sx, se, x, Q, torch.zeros(3, dtype=f64))
    with pytest.raises(ValueError, match="site_eta"):
        cpm.cpm_bvec_noalloc(p, sx, se[:3], x, Q, b)
    with pytest.raises(ValueError, match="Q"):
        cpm.cpm_bvec_noalloc(p, sx, se, x, Q[:1], b)
    with pytest.raises(ValueError, match="site_xyz"):
        cpm.cpm_bvec_noalloc(p, sx.reshape(-1), se, x, Q, b)
    with pytest.raises(TypeError, match="CUDA"):
        cpm.cpm_bvec_noalloc(p, sx, se, x, Q, b)     # well formed, but host memory
