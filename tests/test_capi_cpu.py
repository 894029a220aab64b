"""The C-ABI library builds, loads and exports every symbol include/cfie.h
declares; host-side argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "cfie.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cfie_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1408_1578_gb300 import build, cfie
    build.build()
    return cfie.load()


def test_header_declares_the_call_sequence():
    names = _declared_functions()
    for required in ["cfie_ctx_create", "cfie_geometry_circle", "cfie_geometry_kite",
                     "cfie_geometry_fourier_star", "cfie_geometry_samples", "cfie_discretise",
                     "cfie_rhs_plane_waves", "cfie_apply", "cfie_gmres_solve", "cfie_last_error",
                     "cfie_op_destroy", "cfie_geom_destroy", "cfie_ctx_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1408_1578_gb300 import cfie
    assert set(_declared_functions()) <= set(cfie.SIGNATURES)


def test_null_arguments_rejected_without_gpu(lib):
    # these checks run before any CUDA call
    from paper_1408_1578_gb300 import cfie
    assert lib.cfie_ctx_create(0, None, None) == cfie.CFIE_EINVAL
    assert lib.cfie_geometry_circle(None, 1.0, None) == cfie.CFIE_EINVAL
    assert lib.cfie_discretise(None, 64, 1.0, 1.0, 0, 0, 0, None) == cfie.CFIE_EINVAL
    assert lib.cfie_apply(None, None, None, 1) == cfie.CFIE_EINVAL
    assert lib.cfie_gmres_solve(None, None, None, 1, 1e-6, 80, 100, None, None) == cfie.CFIE_EINVAL
    assert lib.cfie_op_set_inner_basis(None, 1) == cfie.CFIE_EINVAL
    assert lib.cfie_batch_set_inner_basis(None, 0) == cfie.CFIE_EINVAL
    assert lib.cfie_op_set_variant(None, 1) == cfie.CFIE_EINVAL
    assert lib.cfie_measure_peaks(None, None) == cfie.CFIE_EINVAL
    assert lib.cfie_op_set_residual_variant(None, 1) == cfie.CFIE_EINVAL
    assert lib.cfie_last_error(None) == b"null context"


def test_no_device_is_an_error_not_a_crash(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1408_1578_gb300 import cfie
    h = ctypes.c_void_p()
    assert lib.cfie_ctx_create(0, None, ctypes.byref(h)) == cfie.CFIE_ECUDA


def test_server_needs_a_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1408_1578_gb300 import cfie
    h = ctypes.c_void_p()
    assert lib.cfie_server_create(0, 1 << 30, 2, ctypes.byref(h)) == cfie.CFIE_ECUDA
    assert lib.cfie_server_submit(None, None, None) == cfie.CFIE_EINVAL
    buf = ctypes.create_string_buffer(16)
    assert lib.cfie_server_request_error(None, ctypes.c_longlong(1), buf,
                                         ctypes.c_size_t(16)) == cfie.CFIE_EINVAL


def test_null_handles_documented_behaviour(lib):
    """What include/cfie.h promises for null handles, without a GPU: destroy
    calls ignore them, getters return their empty value, everything that
    returns a status says CFIE_EINVAL."""
    from paper_1408_1578_gb300 import cfie
    for fn in ("cfie_ctx_destroy", "cfie_geom_destroy", "cfie_op_destroy", "cfie_batch_destroy",
               "cfie_server_destroy"):
        getattr(lib, fn)(None)
    assert lib.cfie_op_n(None) == 0 and lib.cfie_batch_length(None) == 0
    stats = cfie.cfie_solve_stats()
    assert lib.cfie_op_last_stats(None, ctypes.byref(stats)) == cfie.CFIE_EINVAL
    assert lib.cfie_batch_last_stats(None, ctypes.byref(stats)) == cfie.CFIE_EINVAL
    counters = cfie.cfie_server_counters()
    assert lib.cfie_server_stats(None, ctypes.byref(counters)) == cfie.CFIE_EINVAL
    assert lib.cfie_server_poll(None, ctypes.c_longlong(1), None, None) == cfie.CFIE_EINVAL
    assert lib.cfie_server_wait_all(None, 1.0) == cfie.CFIE_EINVAL
    assert lib.cfie_server_release(None, ctypes.c_longlong(1)) == cfie.CFIE_EINVAL
    assert isinstance(lib.cfie_server_last_error(None), bytes)
    assert lib.cfie_batch_apply(None, None, None) == cfie.CFIE_EINVAL
    assert lib.cfie_ctx_set_profiling(None, 1) == cfie.CFIE_EINVAL
