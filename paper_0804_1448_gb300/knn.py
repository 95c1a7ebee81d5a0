"""Thin ctypes binding of the C ABI in include/knn.h (same names, argument
marshalling only).

Every step of a search runs in the CUDA library ``libknn_gb300.so``; this
module only converts arguments.  It raises at import if the library has not
been built: there is no CPU fallback.  PyTorch tensors are accepted for device
or pinned host buffers (their data pointers are passed through); numpy arrays
are accepted for host buffers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libknn_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it first (python -m paper_0804_1448_gb300.build). "
        "The library has no CPU fallback.")

_lib = ctypes.CDLL(LIB_PATH)

KNN_L2, KNN_L1 = 0, 1
KNN_FP32, KNN_TF32, KNN_BF16 = 0, 1, 2
KNN_LINF, KNN_MAHALANOBIS = 2, 3
METRICS = {"l2": KNN_L2, "l1": KNN_L1, "linf": KNN_LINF, "mahalanobis": KNN_MAHALANOBIS}
PRECISIONS = {"fp32": KNN_FP32, "tf32": KNN_TF32, "bf16": KNN_BF16}
STATUS = {0: "KNN_OK", 1: "KNN_ERR_INVALID", 2: "KNN_ERR_OOM", 3: "KNN_ERR_CUDA",
          4: "KNN_ERR_TIMEOUT", 5: "KNN_ERR_NOREF", 6: "KNN_ERR_BUSY",
          7: "KNN_ERR_UNSUPPORTED"}
KNN_K_MAX = 1024


class knn_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("rerank_factor", ctypes.c_int32),
                ("workspace_limit", ctypes.c_int64)]


class knn_instance(ctypes.Structure):
    _fields_ = [("R", ctypes.c_void_p), ("m", ctypes.c_int64), ("Q", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("k", ctypes.c_int32),
                ("metric", ctypes.c_int32), ("dist_out", ctypes.c_void_p),
                ("idx_out", ctypes.c_void_p)]


class knn_batch_info(ctypes.Structure):
    _fields_ = [("branches", ctypes.c_int32), ("sm_share", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("graph_nodes", ctypes.c_int64),
                ("tuned", ctypes.c_int32), ("tune_ms", ctypes.c_double),
                ("persistent", ctypes.c_int32), ("items", ctypes.c_int32)]


KNN_BATCH_AUTOTUNE = 1
KNN_BATCH_NO_GRAPH = 2
KNN_BATCH_BRANCHES = 4
# stages of the persistent batch, in the order of knn_batch_stage_times
BATCH_STAGES = ("prepare_r", "prepare_q", "pilot", "threshold", "filter", "finalize", "fallback")


class knn_stats(ctypes.Structure):
    _fields_ = [("searches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("recheck_entries", ctypes.c_int64), ("fallback_queries", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("fallback_short_list", ctypes.c_int64),
                ("fallback_overflow", ctypes.c_int64), ("fallback_wide_cut", ctypes.c_int64),
                ("fallback_uncertified", ctypes.c_int64)]


_H = ctypes.c_void_p
_P = ctypes.c_void_p
_i32, _i64 = ctypes.c_int32, ctypes.c_int64
class knn_plan(ctypes.Structure):
    _fields_ = [("tensor_cores", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("splits", ctypes.c_int32), ("chunk", ctypes.c_int64),
                ("k_blocks", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("whole_tile_stages", ctypes.c_int32), ("raw_staging", ctypes.c_int32),
                ("pilot", ctypes.c_int32), ("pilot_stride", ctypes.c_int32),
                ("pilot_groups", ctypes.c_int32), ("threshold_rank", ctypes.c_int32),
                ("list_capacity", ctypes.c_int32), ("fallback_slots", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_int64), ("small_select", ctypes.c_int32),
                ("pilot_group_size", ctypes.c_int32)]


_SIGS = {
    "knn_options_default": (None, [ctypes.POINTER(knn_options)]),
    "knn_create": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.c_int, ctypes.POINTER(knn_options)]),
    "knn_set_reference": (ctypes.c_int, [_H, _P, _i64, _i32, ctypes.c_int]),
    "knn_search": (ctypes.c_int, [_H, _P, _i64, _i32, _i32, ctypes.c_int, _P, _P,
                                  ctypes.c_int, _P]),
    "knn_sync": (ctypes.c_int, [_H]),
    "knn_selftest_bounded_wait": (ctypes.c_int, [_H, _i32]),
    "knn_selftest_batch_queue": (ctypes.c_int, [_H, _i32]),
    "knn_explain_plan": (ctypes.c_int, [_i64, _i64, _i32, _i32, ctypes.c_int, _i32, _i32, _i32,
                                        ctypes.POINTER(knn_plan)]),
    "knn_set_precision": (ctypes.c_int, [_H, _i32]),
    "knn_set_mahalanobis": (ctypes.c_int, [_H, _P, _i32]),
    "knn_get_stats": (ctypes.c_int, [_H, ctypes.POINTER(knn_stats)]),
    "knn_set_profiling": (ctypes.c_int, [_H, ctypes.c_int]),
    "knn_get_profile": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_char_p), _i32,
                                       ctypes.POINTER(_i32)]),
    "knn_search_static": (ctypes.c_int, [_P, _i64, _P, _i64, _i32, _i32, ctypes.c_int, _P, _P, _P]),
    "knn_create_shared": (ctypes.c_int, [ctypes.POINTER(_H), _H, ctypes.POINTER(knn_options)]),
    "knn_workspace_size": (ctypes.c_int, [_H, _i64, _i32, _i32, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_i64)]),
    "knn_reserve": (ctypes.c_int, [_H, _i64]),
    "knn_search_batch": (ctypes.c_int, [_H, ctypes.POINTER(knn_instance), _i32, _i32, _P]),
    "knn_search_self": (ctypes.c_int, [_H, _i32, ctypes.c_int, _P, _P, _P]),
    "knn_batch_info_get": (ctypes.c_int, [_H, ctypes.POINTER(knn_batch_info)]),
    "knn_batch_stage_times": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)]),
    "knn_destroy": (ctypes.c_int, [_H]),
    "knn_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "knn_last_error": (ctypes.c_char_p, [_H]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

# raw C entry points, same names as include/knn.h
knn_options_default = _lib.knn_options_default
knn_create = _lib.knn_create
knn_set_reference = _lib.knn_set_reference
knn_search = _lib.knn_search
knn_sync = _lib.knn_sync
knn_selftest_bounded_wait = _lib.knn_selftest_bounded_wait
knn_selftest_batch_queue = _lib.knn_selftest_batch_queue
knn_explain_plan = _lib.knn_explain_plan

knn_set_precision = _lib.knn_set_precision
knn_set_mahalanobis = _lib.knn_set_mahalanobis
knn_get_stats = _lib.knn_get_stats
knn_set_profiling = _lib.knn_set_profiling
knn_get_profile = _lib.knn_get_profile
knn_search_static = _lib.knn_search_static
knn_create_shared = _lib.knn_create_shared
knn_workspace_size = _lib.knn_workspace_size
knn_reserve = _lib.knn_reserve
knn_search_batch = _lib.knn_search_batch
knn_search_self = _lib.knn_search_self
knn_batch_info_get = _lib.knn_batch_info_get
knn_batch_stage_times = _lib.knn_batch_stage_times
knn_destroy = _lib.knn_destroy
knn_status_string = _lib.knn_status_string
knn_last_error = _lib.knn_last_error


def explain_plan(n: int, m: int, d: int, k: int, metric: str = "l2", precision: str = "bf16",
                 rerank_factor: int = 4, num_sms: int = 152) -> dict:
    """knn_explain_plan: the plan of a search, as a dict (host only)."""
    p = knn_plan()
    st = knn_explain_plan(n, m, d, k, METRICS[metric], PRECISIONS[precision], rerank_factor,
                          num_sms, ctypes.byref(p))
    if st != 0:
        raise KnnError(st, "knn_explain_plan")
    return {f: getattr(p, f) for f, _ in knn_plan._fields_}


class KnnError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = f"{what}: {STATUS.get(status, status)} ({knn_status_string(status).decode()})"
        if detail:
            msg += f" -- {detail}"
        super().__init__(msg)


def _buf(x):
    """(pointer, is_device, keepalive) of a torch tensor or numpy array."""
    if x is None:
        return None, False, None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data, False, x
    import torch  # only for tensors handed in by the caller
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr(), x.is_cuda, x
    raise TypeError(f"unsupported buffer type {type(x)}")


class Index:
    """One library handle: a resident reference set searched by queries."""

    def __init__(self, device: int = 0, precision: str = "fp32", rerank_factor: int = 4,
                 workspace_limit: int = 0):
        opt = knn_options()
        knn_options_default(ctypes.byref(opt))
        opt.precision = PRECISIONS[precision]
        opt.rerank_factor = rerank_factor
        opt.workspace_limit = workspace_limit
        h = _H()
        st = knn_create(ctypes.byref(h), device, ctypes.byref(opt))
        if st != 0:
            raise KnnError(st, "knn_create")
        self.h = h
        self.device = device
        self.m = 0
        self.d = 0

    @classmethod
    def shared(cls, src: "Index") -> "Index":
        """Another handle on src's reference set (knn_create_shared): its own
        stream, workspace and counters, the reference data shared."""
        ix = cls.__new__(cls)
        h = _H()
        st = knn_create_shared(ctypes.byref(h), src.h, None)
        if st != 0:
            raise KnnError(st, "knn_create_shared")
        ix.h = h
        ix.device = src.device
        ix.m = src.m
        ix.d = src.d
        return ix

    def workspace_size(self, n: int, k: int, metric: str = "l2", io_on_device: bool = True) -> int:
        b = _i64()
        self._check(knn_workspace_size(self.h, n, self.d, k, METRICS[metric], 1 if io_on_device else 0,
                                       ctypes.byref(b)), "knn_workspace_size")
        return int(b.value)

    def reserve(self, nbytes: int):
        self._check(knn_reserve(self.h, int(nbytes)), "knn_reserve")

    def _check(self, st, what):
        if st != 0:
            raise KnnError(st, what, knn_last_error(self.h).decode(errors="replace"))

    def close(self):
        if getattr(self, "h", None):
            knn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_reference(self, R):
        p, dev, keep = _buf(R)
        m, d = R.shape
        self._check(knn_set_reference(self.h, p, m, d, 1 if dev else 0), "knn_set_reference")
        self.m, self.d = int(m), int(d)

    def set_precision(self, precision: str):
        self._check(knn_set_precision(self.h, PRECISIONS[precision]), "knn_set_precision")

    def set_mahalanobis(self, S_inv):
        """Inverse covariance (d x d, symmetric positive definite; host array)
        of metric="mahalanobis"; None forgets it."""
        if S_inv is None:
            self._check(knn_set_mahalanobis(self.h, None, 0), "knn_set_mahalanobis")
            return
        import numpy as np
        M = np.ascontiguousarray(S_inv, dtype=np.float64)
        if M.ndim != 2 or M.shape[0] != M.shape[1]:
            raise ValueError("S_inv must be a square matrix")
        self._check(knn_set_mahalanobis(self.h, M.ctypes.data, M.shape[0]), "knn_set_mahalanobis")

    def search_into(self, Q, k: int, dist_out, idx_out, metric: str = "l2", stream=None):
        """knn_search with caller-provided outputs (device tensors: asynchronous
        on `stream`, a torch.cuda.Stream or raw handle; host: synchronous)."""
        pq, dq, _ = _buf(Q)
        pd, dd, _ = _buf(dist_out)
        pi, di, _ = _buf(idx_out)
        if not (dq == dd == di):
            raise ValueError("Q and the outputs must all be on the device or all on the host")
        n = Q.shape[0]
        d = Q.shape[1] if n > 0 or len(Q.shape) == 2 else self.d
        sp = None
        if stream is not None:
            sp = getattr(stream, "cuda_stream", stream)
            if not sp:
                sp = 1   # torch's default stream is CUDA's legacy stream (cudaStreamLegacy)
        self._check(knn_search(self.h, pq, n, d, k, METRICS[metric], pd, pi,
                               1 if dq else 0, sp), "knn_search")

    def search(self, Q, k: int, metric: str = "l2", stream=None):
        """(dist, idx) for the rows of Q: torch tensors on the device for a
        device tensor Q, numpy arrays for a host array."""
        n = Q.shape[0]
        if isinstance(Q, np.ndarray):
            dist = np.empty((n, k), dtype=np.float32)
            idx = np.empty((n, k), dtype=np.int32)
        else:
            import torch
            dist = torch.empty((n, k), dtype=torch.float32, device=Q.device)
            idx = torch.empty((n, k), dtype=torch.int32, device=Q.device)
        self.search_into(Q, k, dist, idx, metric, stream)
        return dist, idx

    def search_self(self, k: int, metric: str = "l2", stream=None):
        """knn_search_self: for every reference point its k nearest other
        reference points; (dist, idx) device tensors m x k."""
        import torch
        dist = torch.empty((self.m, k), dtype=torch.float32, device=f"cuda:{self.device}")
        idx = torch.empty((self.m, k), dtype=torch.int32, device=f"cuda:{self.device}")
        sp = None
        if stream is not None:
            sp = getattr(stream, "cuda_stream", stream) or 1
        self._check(knn_search_self(self.h, k, METRICS[metric], dist.data_ptr(), idx.data_ptr(), sp),
                    "knn_search_self")
        return dist, idx

    def search_batch(self, instances, flags: int = 0, stream=None):
        """knn_search_batch over a list of dicts with device tensors R, Q,
        dist, idx and ints k (and metric, default l2)."""
        arr = (knn_instance * len(instances))()
        for i, x in enumerate(instances):
            R, Q = x["R"], x["Q"]
            for t in (R, Q, x["dist"], x["idx"]):
                if not (t.is_cuda and t.is_contiguous()):
                    raise ValueError("batch tensors must be contiguous device tensors")
            arr[i] = knn_instance(R.data_ptr(), R.shape[0], Q.data_ptr(), Q.shape[0], R.shape[1],
                                  x["k"], METRICS[x.get("metric", "l2")], x["dist"].data_ptr(),
                                  x["idx"].data_ptr())
        sp = None
        if stream is not None:
            sp = getattr(stream, "cuda_stream", stream) or 1
        self._check(knn_search_batch(self.h, arr, len(instances), flags, sp), "knn_search_batch")

    def batch_info(self) -> dict:
        b = knn_batch_info()
        self._check(knn_batch_info_get(self.h, ctypes.byref(b)), "knn_batch_info_get")
        return {f: getattr(b, f) for f, _ in knn_batch_info._fields_}

    def batch_stage_times(self) -> dict:
        """knn_batch_stage_times: per stage of the last persistent batch run,
        the CTA time its items waited and worked (ms, summed over CTAs) and how
        many ran."""
        w, t, n = (ctypes.c_double * 7)(), (ctypes.c_double * 7)(), (_i64 * 7)()
        self._check(knn_batch_stage_times(self.h, w, t, n), "knn_batch_stage_times")
        return {name: {"wait_ms": w[i], "work_ms": t[i], "items": n[i]}
                for i, name in enumerate(BATCH_STAGES)}

    def sync(self):
        self._check(knn_sync(self.h), "knn_sync")

    def stats(self) -> dict:
        s = knn_stats()
        self._check(knn_get_stats(self.h, ctypes.byref(s)), "knn_get_stats")
        return {f: getattr(s, f) for f, _ in knn_stats._fields_}

    def set_profiling(self, on: bool):
        self._check(knn_set_profiling(self.h, 1 if on else 0), "knn_set_profiling")

    def profile(self) -> dict:
        cap = 16
        ms = (ctypes.c_float * cap)()
        names = (ctypes.c_char_p * cap)()
        cnt = _i32()
        self._check(knn_get_profile(self.h, ms, names, cap, ctypes.byref(cnt)), "knn_get_profile")
        out = {}
        for i in range(min(cnt.value, cap)):
            out[names[i].decode()] = out.get(names[i].decode(), 0.0) + ms[i]
        return out
