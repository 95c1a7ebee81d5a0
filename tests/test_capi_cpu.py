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


def test_binding_mirrors_the_header():
    from paper_0804_1448_gb300 import knn
    for name in declared_functions():
        assert hasattr(knn, name), f"binding lacks {name}"
