"""The C ABI library loads and exports every function include/knn.h declares
(no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "knn.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(knn_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_0804_1448_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("knn_create", "knn_set_reference", "knn_search", "knn_destroy",
                 "knn_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in knn.h but not exported"


def test_host_only_entry_points(lib):
    lib.knn_status_string.restype = ctypes.c_char_p
    assert lib.knn_status_string(0) == b"ok"
    assert lib.knn_status_string(1) == b"invalid argument"
    assert lib.knn_status_string(99) == b"unknown status"
    # knn_create with a NULL output pointer is rejected before any CUDA call
    assert lib.knn_create(None, 0, None) == 1
    # destroy(NULL) is accepted
    assert lib.knn_destroy(None) == 0
    # NULL handle everywhere is KNN_ERR_INVALID
    assert lib.knn_search(None, None, 0, 1, 1, 0, None, None, 1, None) == 1
    assert lib.knn_set_reference(None, None, 1, 1, 0) == 1


def test_every_entry_point_refuses_a_null_handle(lib):
    """Argument checks come before any CUDA call (KNN_ERR_INVALID = 1)."""
    from paper_0804_1448_gb300 import knn
    out = ctypes.c_int64(0)
    stats, info = knn.knn_stats(), knn.knn_batch_info()
    count = ctypes.c_int32(0)
    assert knn.knn_sync(None) == 1
    assert knn.knn_selftest_bounded_wait(None, 10) == 1
    assert knn.knn_set_precision(None, 2) == 1
    assert knn.knn_set_mahalanobis(None, None, 4) == 1
    assert knn.knn_get_stats(None, ctypes.byref(stats)) == 1
    assert knn.knn_set_profiling(None, 1) == 1
    assert knn.knn_get_profile(None, None, None, 0, ctypes.byref(count)) == 1
    assert knn.knn_search_self(None, 4, 0, None, None, None) == 1
    assert knn.knn_create_shared(None, None, None) == 1
    h = knn._H()
    assert knn.knn_create_shared(ctypes.byref(h), None, None) == 1 and not h.value
    assert knn.knn_workspace_size(None, 10, 4, 2, 0, 1, ctypes.byref(out)) == 1
    assert knn.knn_workspace_size(None, 10, 4, 2, 0, 1, None) == 1
    assert knn.knn_reserve(None, 1 << 20) == 1
    assert knn.knn_search_batch(None, None, 0, 0, None) == 1
    assert knn.knn_batch_info_get(None, ctypes.byref(info)) == 1
    w, t, n = (ctypes.c_double * 7)(), (ctypes.c_double * 7)(), (ctypes.c_int64 * 7)()
    assert knn.knn_batch_stage_times(None, w, t, n) == 1
    assert knn.knn_last_error(None) == b""


def test_static_entry_checks_arguments_first(lib):
    """knn_search_static: invalid shapes, metric or pointers are refused, and
    n = 0 is a no-op, all before the device is touched."""
    from paper_0804_1448_gb300 import knn
    buf = (ctypes.c_float * 64)()
    ib = (ctypes.c_int32 * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    q = ctypes.cast(ib, ctypes.c_void_p)
    call = knn.knn_search_static
    assert call(p, 0, p, 1, 4, 1, 0, p, q, None) == 1          # m < 1
    assert call(p, 8, p, -1, 4, 1, 0, p, q, None) == 1         # n < 0
    assert call(p, 8, p, 1, 0, 1, 0, p, q, None) == 1          # d < 1
    assert call(p, 8, p, 1, 4, 9, 0, p, q, None) == 1          # k > m
    assert call(p, 8, p, 1, 4, 1, 3, p, q, None) == 1          # Mahalanobis is not offered
    assert call(None, 8, p, 1, 4, 1, 0, p, q, None) == 1       # no reference set
    assert call(p, 8, None, 1, 4, 1, 0, p, q, None) == 1       # no queries
    assert call(p, 2000, p, 1, 4, 1025, 0, p, q, None) == 7    # k > KNN_K_MAX
    assert call(p, 8, None, 0, 4, 1, 0, None, None, None) == 0  # n = 0: nothing to do


def test_binding_mirrors_the_header():
    from paper_0804_1448_gb300 import knn
    for name in declared_functions():
        assert hasattr(knn, name), f"binding lacks {name}"
