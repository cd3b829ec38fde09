"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/mpir.h declares.  Host-only entry points (workspace queries,
argument checks) are exercised; nothing here launches GPU work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mpir.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char|long long)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libmpir():
    from paper_2406_16499_gb300 import mpir
    return mpir.lib()


def test_library_exports_every_declared_symbol(libmpir):
    from paper_2406_16499_gb300 import mpir
    names = declared_functions()
    assert "lse_solve" in names and "gls_solve_batched" in names
    for n in names:
        assert hasattr(libmpir, n), "missing export %s" % n
    assert set(names) == set(mpir.exported_symbols())


def test_version_and_defaults(libmpir):
    from paper_2406_16499_gb300 import mpir
    assert b"sm_103a" in libmpir.mpir_version()
    o = mpir.Opts()
    libmpir.mpir_default_opts(ctypes.byref(o))
    assert o.maxit == 40            # Alg. 2 / Alg. 4 default
    assert o.fact == mpir.PREC["fp32"] and o.refine == 0 and o.restart == 30
    assert 0 < o.tol < 1e-13


def test_workspace_queries_and_argument_checks(libmpir):
    from paper_2406_16499_gb300 import mpir
    o = mpir.Opts()
    libmpir.mpir_default_opts(ctypes.byref(o))
    sz = ctypes.c_size_t(0)
    assert libmpir.mpir_lse_workspace_size(200, 100, 20, ctypes.byref(o), ctypes.byref(sz)) == 0
    assert sz.value > 200 * 100 * 4
    assert libmpir.mpir_gls_workspace_size(4096, 1024, 4096, ctypes.byref(o), ctypes.byref(sz)) == 0
    assert sz.value > 4096 * 4096 * 8
    # p <= n <= m + p violated
    assert libmpir.mpir_lse_workspace_size(5, 10, 2, ctypes.byref(o), ctypes.byref(sz)) < 0
    assert libmpir.mpir_lse_workspace_size(10, 5, 6, ctypes.byref(o), ctypes.byref(sz)) < 0
    # m <= n <= m + p violated
    assert libmpir.mpir_gls_workspace_size(5, 6, 2, ctypes.byref(o), ctypes.byref(sz)) < 0
    assert libmpir.mpir_gls_workspace_size(10, 2, 3, ctypes.byref(o), ctypes.byref(sz)) < 0
    # NULL handle is rejected before anything runs
    assert libmpir.lse_solve(None, 4, 3, 1, None, 4, None, 1, None, None, None, None, None, None, None) == -1
    assert libmpir.gls_solve(None, 4, 2, 3, None, 4, None, 4, None, None, None, None, None, None) == -1


def test_library_is_sm103a_only():
    from paper_2406_16499_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_checks_device_and_element_type():
    """The binding hands the C ABI raw device pointers: a host tensor, or one
    whose element type is not the C argument's, is refused before any call
    (a float32 buffer read as doubles would be read past its end)."""
    torch = pytest.importorskip("torch")
    from paper_2406_16499_gb300 import mpir

    class OnDevice:                        # stands in for a CUDA tensor
        is_cuda, device = True, "cuda:0"

        def __init__(self, dtype, n=4):
            self.dtype, self.n = dtype, n

        def numel(self):
            return self.n

        def data_ptr(self):
            return 0x1000

    with pytest.raises(mpir.MpirError):
        mpir.ptr(torch.zeros(4, dtype=torch.float64))            # host memory
    with pytest.raises(mpir.MpirError):
        mpir.ptr(OnDevice(torch.float32))                        # double* argument
    with pytest.raises(mpir.MpirError):
        mpir.ptr(OnDevice(torch.int64), "i32")                   # int* labels
    assert mpir.ptr(OnDevice(torch.float64)) == 0x1000
    assert mpir.ptr(OnDevice(torch.float32), "f32") == 0x1000
    assert mpir.ptr(OnDevice(torch.float64, 0)) is None          # empty -> NULL
    assert mpir.ptr(None) is None
