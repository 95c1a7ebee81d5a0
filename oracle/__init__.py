"""Brute-force k-nearest-neighbour oracle (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library never calls it; it shares no code with the CUDA path.

The arithmetic lives in ``knn_oracle.c`` (plain C, FP64, a full sort per
query with ties broken by the smaller index -- Sec. 2.1 of Garcia,
Debreuve and Barlaud, "Fast k Nearest Neighbor Search using GPU").  This
module compiles it with gcc and calls it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

METRICS = {"l2": 0, "l1": 1, "linf": 2}


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile knn_oracle.c into a shared library (gcc, OpenMP, no FMA)."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", f"-DORACLE_MUTANT={int(mutant)}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(mutant: int = 0) -> ctypes.CDLL:
    with _LOCK:
        if mutant in _LIBS:
            return _LIBS[mutant]
        lib = ctypes.CDLL(build(mutant))
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        p = ctypes.c_void_p
        lib.oracle_knn.argtypes = [p, i64, p, i64, i32, i32, i32, p, p, i32]
        lib.oracle_knn.restype = ctypes.c_int
        lib.oracle_knn_subset.argtypes = [p, i64, p, i64, i32, i32, i32, p, i64, p, p, i32]
        lib.oracle_knn_subset.restype = ctypes.c_int
        lib.oracle_key_pairs.argtypes = [p, i64, p, i64, i32, i32, p, p, i64, p]
        lib.oracle_key_pairs.restype = ctypes.c_int
        lib.oracle_knn_mahalanobis.argtypes = [p, i64, p, i64, i32, p, i32, p, p, i32]
        lib.oracle_knn_mahalanobis.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        _LIBS[mutant] = lib
        return lib


def _f32(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("points must be a 2-D array (rows are points)")
    return a


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def max_threads() -> int:
    return int(_lib().oracle_max_threads())


def knn(R, Q, k: int, metric: str = "l2", nthreads: int = 0, mutant: int = 0):
    """k nearest neighbours of every row of Q among the rows of R.

    Returns (dist float64 [n,k], idx int32 [n,k]); row i ascending by
    (distance, index).  Euclidean distances are true (square-rooted)
    distances; the sort compares their squares.
    """
    R, Q = _f32(R), _f32(Q)
    m, d = R.shape
    n = Q.shape[0]
    if Q.shape[1] != d:
        raise ValueError("R and Q differ in dimension")
    dist = np.empty((n, k), dtype=np.float64)
    idx = np.empty((n, k), dtype=np.int32)
    rc = _lib(mutant).oracle_knn(_ptr(R), m, _ptr(Q), n, d, k, METRICS[metric],
                                 _ptr(dist), _ptr(idx), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_knn failed with code {rc}")
    return dist, idx


def knn_subset(R, Q, qsel, k: int, metric: str = "l2", nthreads: int = 0):
    """knn() for the query rows listed in qsel (rows follow qsel's order)."""
    R, Q = _f32(R), _f32(Q)
    m, d = R.shape
    qsel = np.ascontiguousarray(qsel, dtype=np.int64)
    dist = np.empty((len(qsel), k), dtype=np.float64)
    idx = np.empty((len(qsel), k), dtype=np.int32)
    rc = _lib().oracle_knn_subset(_ptr(R), m, _ptr(Q), Q.shape[0], d, k, METRICS[metric],
                                  _ptr(qsel), len(qsel), _ptr(dist), _ptr(idx), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_knn_subset failed with code {rc}")
    return dist, idx


def key_pairs(R, Q, qi, rj, metric: str = "l2"):
    """Raw distance keys (squared for L2) of explicit (query, reference) pairs."""
    R, Q = _f32(R), _f32(Q)
    qi = np.ascontiguousarray(qi, dtype=np.int64)
    rj = np.ascontiguousarray(rj, dtype=np.int64)
    out = np.empty(len(qi), dtype=np.float64)
    rc = _lib().oracle_key_pairs(_ptr(R), R.shape[0], _ptr(Q), Q.shape[0], R.shape[1],
                                 METRICS[metric], _ptr(qi), _ptr(rj), len(qi), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_key_pairs failed with code {rc}")
    return out


def knn_mahalanobis(R, Q, M, k: int, nthreads: int = 0, mutant: int = 0):
    """k nearest neighbours under the Mahalanobis distance sqrt(delta^T M delta)
    (M: d x d symmetric positive definite, the inverse covariance).  Returns
    (dist float64 [n,k], idx int32 [n,k]), ascending by (distance, index)."""
    R, Q = _f32(R), _f32(Q)
    m, d = R.shape
    n = Q.shape[0]
    M = np.ascontiguousarray(M, dtype=np.float64)
    if Q.shape[1] != d or M.shape != (d, d):
        raise ValueError("R, Q and M differ in dimension")
    dist = np.empty((n, k), dtype=np.float64)
    idx = np.empty((n, k), dtype=np.int32)
    rc = _lib(mutant).oracle_knn_mahalanobis(_ptr(R), m, _ptr(Q), n, d, _ptr(M), k,
                                             _ptr(dist), _ptr(idx), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_knn_mahalanobis failed with code {rc}")
    return dist, idx
