"""The C ABI library builds, loads without a GPU, and exports every entry point
that include/ap.h declares with the struct layouts the binding mirrors."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(ap_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_17137_gb300 import _capi
    return _capi.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2310_17137_gb300 import _capi
    decl = declared_functions()
    assert len(decl) >= 10
    assert sorted(decl) == sorted(_capi.EXPORTS)
    for name in decl:
        assert hasattr(lib, name), name


def test_struct_layouts_match_binding(lib):
    from paper_2310_17137_gb300 import _capi
    assert lib.ap_sizeof_opts() == ctypes.sizeof(_capi.ap_opts)
    assert lib.ap_sizeof_info() == ctypes.sizeof(_capi.ap_info)
    assert lib.ap_sizeof_hyper() == ctypes.sizeof(_capi.ap_hyper)
    assert lib.ap_sizeof_request() == ctypes.sizeof(_capi.ap_request)
    assert lib.ap_sizeof_request_result() == ctypes.sizeof(_capi.ap_request_result)


def test_defaults_and_status_strings(lib):
    import paper_2310_17137_gb300 as ap
    o = ap.ap_opts_default()
    assert (o.block, o.min_epochs, o.max_epochs, o.tol) == (4096, 11, 1000, 1.0)
    assert o.select == ap.AP_SEL_GS and o.stop == ap.AP_STOP_MEAN_REL and o.precision == ap.AP_FP32
    assert ap.ap_status_str(ap.AP_ERR_NOT_SPD) == "AP_ERR_NOT_SPD"
    assert ap.ap_status_str(99) == "AP_ERR_UNKNOWN"


def test_invalid_arguments_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    from paper_2310_17137_gb300 import _capi
    h = _capi.ap_hyper(0, 2, None, 1.0, 0.1, 0.0)
    o = _capi.ap_opts()
    lib.ap_opts_default(ctypes.byref(o))
    out = ctypes.c_void_p()
    assert lib.ap_create(ctypes.byref(out), None, 10, 2, ctypes.byref(h), ctypes.byref(o)) == _capi.AP_ERR_INVALID_ARG
    assert lib.ap_create(ctypes.byref(out), ctypes.c_void_p(16), 10, 0, ctypes.byref(h), ctypes.byref(o)) == \
        _capi.AP_ERR_INVALID_ARG
    assert lib.ap_solve(None, None, 1, None, None, None) == _capi.AP_ERR_INVALID_ARG
    lib.ap_destroy(None)
    # the cache's FP64 kernel values: unknown kernel, negative count or NULL arrays
    assert lib.ap_phi_fp64_eval(7, None, 1, None) == _capi.AP_ERR_INVALID_ARG
    assert lib.ap_phi_fp64_eval(0, None, -1, None) == _capi.AP_ERR_INVALID_ARG
    assert lib.ap_phi_fp64_eval(0, None, 3, None) == _capi.AP_ERR_INVALID_ARG
    assert lib.ap_phi_fp64_eval(2, None, 0, None) == _capi.AP_OK


def test_package_has_no_cpu_fallback():
    # the product path must not import the oracle
    import paper_2310_17137_gb300 as ap
    src_dir = os.path.dirname(ap.__file__)
    for fn in os.listdir(src_dir):
        if fn.endswith(".py"):
            txt = open(os.path.join(src_dir, fn)).read()
            assert "import oracle" not in txt and "from oracle" not in txt, fn


def test_product_build_has_no_index_checks(lib):
    # the bounds checks exist only in the separately built libap_checked.so
    # (tests/test_gpu_checked.py); the product library answers without a GPU
    import paper_2310_17137_gb300 as ap
    from paper_2310_17137_gb300 import _capi
    if _capi.checked():
        pytest.skip("this process uses the checked build")
    assert ap.ap_bounds_violations() == (-1, "")
    assert ap.ap_bounds_selftest(100) == ap.AP_ERR_UNSUPPORTED


def test_checked_build_compiles_and_exports_the_same_symbols():
    # the bounds-checked variant (AP_CHECKED) is a separate library with the same
    # ABI; it is built here (objects cached under _build_checked/) and loaded next
    # to the product library without a GPU
    import shutil
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_2310_17137_gb300 import _capi
    from paper_2310_17137_gb300 import build as _build
    path = _build.build(checked=True)
    assert path.endswith("libap_checked.so") and path != _build.LIB
    L = ctypes.CDLL(path)
    for name in _capi.EXPORTS:
        assert hasattr(L, name), name
