"""Thin Python binding of the C ABI in include/rsc.h (ctypes + torch tensors).

Argument marshalling only: every step of the neighbourhood graph runs in the
CUDA library (librsc.so).  torch provides device memory and streams.  The
functions carry the C names; outputs and the workspace are allocated here
with torch and handed to the library as raw device pointers.

If the library has not been built, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "librsc.so")

RSC_OK, RSC_ERR_INVALID_ARG, RSC_ERR_CUDA, RSC_ERR_WORKSPACE, RSC_ERR_TIMEOUT, \
    RSC_ERR_UNSUPPORTED, RSC_ERR_CAPACITY = range(7)
RSC_EUCLIDEAN, RSC_COSINE = 0, 1
RSC_FP32, RSC_BF16, RSC_FP8 = 0, 1, 3

_METRICS = {"euclidean": RSC_EUCLIDEAN, "cosine": RSC_COSINE}
_PRECISIONS = {"fp32": RSC_FP32, "bf16": RSC_BF16, "fp8": RSC_FP8}

_lock = threading.Lock()
_lib = None


class RscError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"rsc status {status}: {message}")
        self.status = status


class rsc_knn_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("db_splits", ctypes.c_int32), ("tc_parts", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("phase_events", ctypes.c_void_p),
                ("locality", ctypes.c_int32), ("prune", ctypes.c_int32), ("stages", ctypes.c_int32)]


class rsc_umap_opts(ctypes.Structure):
    _fields_ = [("a", ctypes.c_float), ("b", ctypes.c_float), ("gamma", ctypes.c_float),
                ("learning_rate", ctypes.c_float), ("negative_sample_rate", ctypes.c_int32),
                ("n_epochs", ctypes.c_int32), ("epoch_first", ctypes.c_int32), ("epoch_last", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p)]


class rsc_nnd_opts(ctypes.Structure):
    _fields_ = [("sample", ctypes.c_int32), ("rev_slots", ctypes.c_int32), ("cand_slots", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("delta", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_void_p)]


class rsc_leiden_opts(ctypes.Structure):
    _fields_ = [("resolution", ctypes.c_double), ("n_iterations", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("stream", ctypes.c_void_p)]


# name -> (restype, argtypes); the full exported surface of include/rsc.h
_vp, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "rsc_version": (ctypes.c_char_p, []),
    "rsc_last_error": (ctypes.c_char_p, []),
    "rsc_workspace_status": (_i32, [_vp, _vp]),
    "rsc_set_wait_budget": (_i32, [_i64]),
    "rsc_knn_workspace_size": (_i32, [_i64, _i32, _i32, _i32, ctypes.POINTER(rsc_knn_opts), ctypes.POINTER(_sz)]),
    "rsc_knn_scan_stats": (_i32, [_i64, _i32, _i32, _i32, ctypes.POINTER(rsc_knn_opts), _vp, _sz,
                                  ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "rsc_knn": (_i32, [_vp, _i64, _i32, _i32, _i32, _vp, _vp, ctypes.POINTER(rsc_knn_opts), _vp, _sz]),
    "rsc_knn_batched_workspace_size": (_i32, [_i64, _i32, _vp, _i32, _i32, _i32, _i32,
                                               ctypes.POINTER(rsc_knn_opts), ctypes.POINTER(_sz)]),
    "rsc_knn_batched": (_i32, [_vp, _i64, _i32, _vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp,
                                ctypes.POINTER(rsc_knn_opts), _vp, _sz]),
    "rsc_knn_batched_scan_stats": (_i32, [_i64, _i32, _vp, _i32, _i32, _i32, _i32, ctypes.POINTER(rsc_knn_opts),
                                           _vp, _sz, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "rsc_connectivities_workspace_size": (_i32, [_i64, _i32, ctypes.POINTER(_sz)]),
    "rsc_connectivities_max_nnz": (_i64, [_i64, _i32]),
    "rsc_connectivities": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rsc_connectivities_nnz": (_i32, [_vp, _vp, _i64, _i32, ctypes.POINTER(_i64), _vp, _sz, _vp]),
    "rsc_connectivities_static": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _i64, _vp, _vp, _vp]),
    "rsc_autotune_workspace_size": (_i32, [_i64, _i32, _i32, _i32, _i32, ctypes.POINTER(_sz)]),
    "rsc_autotune_knn": (_i32, [_vp, _i64, _i32, _i32, _i32, ctypes.POINTER(rsc_knn_opts), _i32, _vp, _vp,
                                 ctypes.POINTER(rsc_knn_opts), ctypes.POINTER(ctypes.c_float), _vp, _sz]),
    "rsc_autotune_knn_batched": (_i32, [_vp, _i64, _i32, _vp, _i32, _i32, _i32, _i32,
                                         ctypes.POINTER(rsc_knn_opts), _i32, _vp, _vp, _vp, _vp,
                                         ctypes.POINTER(rsc_knn_opts), ctypes.POINTER(ctypes.c_float), _vp, _sz]),
    "rsc_autotune_save": (_i32, [ctypes.c_char_p]),
    "rsc_autotune_load": (_i32, [ctypes.c_char_p]),
    "rsc_autotune_clear": (_i32, []),
    "rsc_partitioner_create": (_i32, [_i32, _i32, _i32, _i32, ctypes.c_uint64, ctypes.POINTER(_vp)]),
    "rsc_partitioner_destroy": (_i32, [_vp]),
    "rsc_partitioner_param_count": (_i32, [_vp, ctypes.POINTER(_i64)]),
    "rsc_partitioner_get_params": (_i32, [_vp, _vp]),
    "rsc_partitioner_set_params": (_i32, [_vp, _vp]),
    "rsc_partitioner_loss_grad_workspace_size": (_i32, [_vp, _i32, ctypes.POINTER(_sz)]),
    "rsc_partitioner_loss_grad": (_i32, [_vp, _vp, _vp, _i32, ctypes.POINTER(ctypes.c_float), _vp, _vp, _sz, _vp]),
    "rsc_partitioner_workspace_size": (_i32, [_vp, _i64, _i64, _i32, _i64, _i32, ctypes.POINTER(_sz)]),
    "rsc_partitioner_train": (_i32, [_vp, _vp, _i64, _vp, _i64, _i32, _i32, _i32, _i32, ctypes.c_float,
                                      ctypes.POINTER(ctypes.c_float), _vp, _sz, _vp]),
    "rsc_partitioner_build_index": (_i32, [_vp, _vp, _i64, _vp, _sz, _vp]),
    "rsc_knn_partitioned": (_i32, [_vp, _vp, _i64, _i32, _i32, _i32, _vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "rsc_partitioner_save": (_i32, [_vp, ctypes.c_char_p]),
    "rsc_partitioner_load": (_i32, [ctypes.c_char_p, ctypes.POINTER(_vp)]),
    "rsc_umap_find_ab": (_i32, [ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(ctypes.c_float)]),
    "rsc_umap_workspace_size": (_i32, [_i64, _i64, _i32, ctypes.POINTER(_sz)]),
    "rsc_umap_layout": (_i32, [_vp, _vp, _vp, _i64, _i64, _i32, _vp, ctypes.POINTER(rsc_umap_opts), _vp, _sz]),
    "rsc_edistance_workspace_size": (_i32, [_i64, _i32, _vp, _i32, _vp, _i64, ctypes.POINTER(_sz)]),
    "rsc_edistance": (_i32, [_vp, _i64, _i32, _vp, _vp, _i32, _vp, _i64, _vp, _vp, _vp, _vp, _sz, _vp]),
    "rsc_knn_descent_pairs": (_i32, [_vp, _sz, _vp]),
    "rsc_leiden_last_stats": (_i32, [_vp]),
    "rsc_leiden_workspace_size": (_i32, [_i64, _i64, ctypes.POINTER(_sz)]),
    "rsc_leiden": (_i32, [_vp, _vp, _vp, _i64, _i64, _vp, _vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(rsc_leiden_opts), _vp, _sz]),
    "rsc_knn_descent_workspace_size": (_i32, [_i64, _i32, _i32, ctypes.POINTER(rsc_nnd_opts), ctypes.POINTER(_sz)]),
    "rsc_knn_descent": (_i32, [_vp, _i64, _i32, _i32, _vp, _vp, _vp, _vp, ctypes.POINTER(rsc_nnd_opts), _vp, _sz]),
}


def lib():
    """Load librsc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                                   "(the CUDA library is required; there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int):
    if status != RSC_OK:
        raise RscError(status, lib().rsc_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _workspace(nbytes: int, device, workspace=None):
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError("workspace too small")
        return workspace
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def rsc_version() -> str:
    return lib().rsc_version().decode()


def rsc_set_wait_budget(clocks: int) -> None:
    """Budget (SM clock cycles) of the tensor-core kernels' bounded waits; 0
    restores the default (about 1 s).  For exercising the timeout path."""
    _check(lib().rsc_set_wait_budget(int(clocks)))


def rsc_workspace_status(workspace: torch.Tensor, stream=None) -> int:
    """Status word recorded by kernels in `workspace` (synchronises)."""
    return int(lib().rsc_workspace_status(_ptr(workspace), _stream(stream)))


_LOCALITY = {"auto": 0, "off": 1, "on": 2}


def knn_opts(precision="fp32", candidates=0, db_splits=0, stream=None, phase_events=None,
             locality="auto", prune="auto", stages=0) -> rsc_knn_opts:
    """Option struct; `phase_events` is a ctypes array of 4 raw cudaEvent_t."""
    o = rsc_knn_opts()
    o.locality = _LOCALITY[locality] if isinstance(locality, str) else int(locality)
    o.prune = _LOCALITY[prune] if isinstance(prune, str) else int(prune)
    o.phase_events = ctypes.cast(phase_events, ctypes.c_void_p).value if phase_events is not None else None
    o.precision = _PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.candidates = int(candidates)
    o.db_splits = int(db_splits)
    o.stages = int(stages)
    o.stream = _stream(stream).value
    return o


def rsc_knn_workspace_size(n, d, k, metric="euclidean", precision="fp32", candidates=0, db_splits=0,
                           locality="auto", prune="auto") -> int:
    o = knn_opts(precision, candidates, db_splits, stream=None, locality=locality, prune=prune) \
        if torch.cuda.is_available() else rsc_knn_opts(_PRECISIONS[precision], candidates, db_splits, 0, None, None,
                                                       _LOCALITY[locality], _LOCALITY[prune])
    out = _sz(0)
    _check(lib().rsc_knn_workspace_size(n, d, k, _METRICS.get(metric, metric), ctypes.byref(o), ctypes.byref(out)))
    return int(out.value)


def rsc_knn_scan_stats(n, d, k, workspace, metric="euclidean", precision="fp32", candidates=0, db_splits=0,
                       locality="auto", prune="auto", stream=None):
    """(pairs scanned, pairs total) of the last rsc_knn on `workspace` with these options."""
    o = knn_opts(precision, candidates, db_splits, stream, None, locality, prune)
    a, b = _i64(0), _i64(0)
    _check(lib().rsc_knn_scan_stats(n, d, k, _METRICS.get(metric, metric), ctypes.byref(o), _ptr(workspace),
                                    workspace.numel(), ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def rsc_knn(X: torch.Tensor, k: int, metric="euclidean", precision="fp32", candidates=0, db_splits=0,
            stream=None, workspace=None, out=None, phase_events=None, locality="auto", prune="auto", stages=0,
            tc_parts=0):
    """Exact kNN of every row of X (float32 [n, d] on the GPU).

    Returns (idx int32 [n, k], dist float32 [n, k]) on X's device.
    """
    if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.is_contiguous()):
        raise ValueError("X must be a contiguous float32 [n, d] CUDA tensor")
    n, d = X.shape
    m = _METRICS[metric] if isinstance(metric, str) else int(metric)
    o = knn_opts(precision, candidates, db_splits, stream, phase_events, locality, prune, stages)
    o.tc_parts = int(tc_parts)
    need = _sz(0)
    _check(lib().rsc_knn_workspace_size(n, d, k, m, ctypes.byref(o), ctypes.byref(need)))
    ws = _workspace(need.value, X.device, workspace)
    if out is None:
        idx = torch.empty((n, k), dtype=torch.int32, device=X.device)
        dist = torch.empty((n, k), dtype=torch.float32, device=X.device)
    else:
        idx, dist = out
    _check(lib().rsc_knn(_ptr(X), n, d, k, m, _ptr(idx), _ptr(dist), ctypes.byref(o), _ptr(ws),
                         ws.numel()))
    return idx, dist


def _offsets_host(sample_offsets):
    import numpy as np
    off = np.ascontiguousarray(np.asarray(sample_offsets, dtype=np.int64))
    return off, off.ctypes.data_as(ctypes.c_void_p)


def rsc_knn_batched_workspace_size(n, d, sample_offsets, k_within, k_cross, metric="euclidean",
                                   precision="bf16", locality="auto", prune="auto") -> int:
    off, optr = _offsets_host(sample_offsets)
    o = rsc_knn_opts(_PRECISIONS[precision], 0, 0, 0, None, None, _LOCALITY[locality], _LOCALITY[prune])
    out = _sz(0)
    _check(lib().rsc_knn_batched_workspace_size(n, d, optr, len(off) - 1, k_within, k_cross,
                                                _METRICS.get(metric, metric), ctypes.byref(o), ctypes.byref(out)))
    return int(out.value)


def rsc_knn_batched(X: torch.Tensor, sample_offsets, k_within: int, k_cross: int, metric="euclidean",
                    precision="bf16", stream=None, workspace=None, out=None, locality="auto", prune="auto"):
    """Per-sample kNN and k_cross nearest from every sample (host offsets).

    Returns (idx_within [n, k_within], dist_within, idx_cross [n, S * k_cross], dist_cross).
    """
    if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.is_contiguous()):
        raise ValueError("X must be a contiguous float32 [n, d] CUDA tensor")
    n, d = X.shape
    off, optr = _offsets_host(sample_offsets)
    S = len(off) - 1
    m = _METRICS[metric] if isinstance(metric, str) else int(metric)
    o = knn_opts(precision, 0, 0, stream, locality=locality, prune=prune)
    need = _sz(0)
    _check(lib().rsc_knn_batched_workspace_size(n, d, optr, S, k_within, k_cross, m, ctypes.byref(o),
                                                ctypes.byref(need)))
    ws = _workspace(need.value, X.device, workspace)
    if out is None:
        iw = torch.empty((n, k_within), dtype=torch.int32, device=X.device)
        dw = torch.empty((n, k_within), dtype=torch.float32, device=X.device)
        ix = torch.empty((n, S * k_cross), dtype=torch.int32, device=X.device)
        dx = torch.empty((n, S * k_cross), dtype=torch.float32, device=X.device)
    else:
        iw, dw, ix, dx = out
    _check(lib().rsc_knn_batched(_ptr(X), n, d, optr, S, k_within, k_cross, m, _ptr(iw), _ptr(dw), _ptr(ix),
                                 _ptr(dx), ctypes.byref(o), _ptr(ws), ws.numel()))
    return iw, dw, ix, dx


def rsc_knn_batched_scan_stats(n, d, sample_offsets, k_within, k_cross, workspace, metric="euclidean",
                               precision="bf16", stream=None, locality="auto", prune="auto"):
    """(pairs scanned, pairs total) of the last rsc_knn_batched on `workspace` with these arguments."""
    off, optr = _offsets_host(sample_offsets)
    o = knn_opts(precision, 0, 0, stream, locality=locality, prune=prune)
    a, b = _i64(0), _i64(0)
    _check(lib().rsc_knn_batched_scan_stats(n, d, optr, len(off) - 1, k_within, k_cross,
                                            _METRICS.get(metric, metric), ctypes.byref(o), _ptr(workspace),
                                            workspace.numel(), ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def rsc_connectivities_workspace_size(n: int, k: int) -> int:
    out = _sz(0)
    _check(lib().rsc_connectivities_workspace_size(n, k, ctypes.byref(out)))
    return int(out.value)


def rsc_connectivities_max_nnz(n: int, k: int) -> int:
    return int(lib().rsc_connectivities_max_nnz(n, k))


def rsc_connectivities(idx: torch.Tensor, dist: torch.Tensor, nnz_capacity=None, stream=None,
                       workspace=None, out=None, with_rho_sigma=True):
    """Fuzzy connectivities CSR of a kNN graph.

    Returns (indptr int64 [n+1], indices int32 [cap], data float32 [cap], rho, sigma)
    with the first indptr[n] entries of indices/data valid.
    """
    if not (idx.is_cuda and dist.is_cuda and idx.dtype == torch.int32 and dist.dtype == torch.float32):
        raise ValueError("idx int32 / dist float32 CUDA tensors expected")
    idx, dist = idx.contiguous(), dist.contiguous()
    n, k = idx.shape
    cap = rsc_connectivities_max_nnz(n, k) if nnz_capacity is None else int(nnz_capacity)
    ws = _workspace(rsc_connectivities_workspace_size(n, k), idx.device, workspace)
    if out is None:
        indptr = torch.empty(n + 1, dtype=torch.int64, device=idx.device)
        indices = torch.empty(max(cap, 1), dtype=torch.int32, device=idx.device)
        data = torch.empty(max(cap, 1), dtype=torch.float32, device=idx.device)
        rho = torch.empty(n, dtype=torch.float32, device=idx.device) if with_rho_sigma else None
        sigma = torch.empty(n, dtype=torch.float32, device=idx.device) if with_rho_sigma else None
    else:
        indptr, indices, data, rho, sigma = out
    _check(lib().rsc_connectivities(_ptr(idx), _ptr(dist), n, k, _ptr(indptr), _ptr(indices), _ptr(data), cap,
                                    _ptr(rho), _ptr(sigma), _ptr(ws), ws.numel(), _stream(stream)))
    return indptr, indices, data, rho, sigma


def rsc_connectivities_nnz(idx: torch.Tensor, dist: torch.Tensor, stream=None, workspace=None) -> int:
    n, k = idx.shape
    ws = _workspace(rsc_connectivities_workspace_size(n, k), idx.device, workspace)
    out = _i64(0)
    _check(lib().rsc_connectivities_nnz(_ptr(idx), _ptr(dist), n, k, ctypes.byref(out), _ptr(ws), ws.numel(),
                                        _stream(stream)))
    return int(out.value)


def rsc_connectivities_static(idx: torch.Tensor, dist: torch.Tensor, stream=None, out=None):
    """rsc_connectivities with the library's fixed 32 MiB scratch (no workspace,
    no allocation inside the call; outputs are allocated here unless given).

    Returns (indptr, indices, data, rho, sigma) like rsc_connectivities.
    """
    if not (idx.is_cuda and dist.is_cuda and idx.dtype == torch.int32 and dist.dtype == torch.float32):
        raise ValueError("idx int32 / dist float32 CUDA tensors expected")
    idx, dist = idx.contiguous(), dist.contiguous()
    n, k = idx.shape
    cap = rsc_connectivities_max_nnz(n, k)
    if out is None:
        out = (torch.empty(n + 1, dtype=torch.int64, device=idx.device),
               torch.empty(max(cap, 1), dtype=torch.int32, device=idx.device),
               torch.empty(max(cap, 1), dtype=torch.float32, device=idx.device),
               torch.empty(n, dtype=torch.float32, device=idx.device),
               torch.empty(n, dtype=torch.float32, device=idx.device))
    indptr, indices, data, rho, sigma = out
    _check(lib().rsc_connectivities_static(_ptr(idx), _ptr(dist), n, k, _ptr(indptr), _ptr(indices), _ptr(data),
                                           cap, _ptr(rho), _ptr(sigma), _stream(stream)))
    return indptr, indices, data, rho, sigma


def rsc_autotune_knn(X: torch.Tensor, k: int, metric="euclidean", precision="bf16", trials=2, stream=None):
    """Time rsc_knn's configurations on X, remember the fastest for automatic
    options, and return (chosen option dict, best ms, idx, dist)."""
    n, d = X.shape
    m = _METRICS[metric] if isinstance(metric, str) else int(metric)
    p = _PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    need = _sz(0)
    _check(lib().rsc_autotune_workspace_size(n, d, k, m, p, ctypes.byref(need)))
    ws = _workspace(need.value, X.device)
    idx = torch.empty((n, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((n, k), dtype=torch.float32, device=X.device)
    o = knn_opts(precision, 0, 0, stream)
    best = rsc_knn_opts()
    ms = ctypes.c_float(0)
    _check(lib().rsc_autotune_knn(_ptr(X), n, d, k, m, ctypes.byref(o), trials, _ptr(idx), _ptr(dist),
                                  ctypes.byref(best), ctypes.byref(ms), _ptr(ws), ws.numel()))
    return ({"db_splits": best.db_splits, "candidates": best.candidates, "tc_parts": best.tc_parts,
             "stages": best.stages}, float(ms.value), idx, dist)


def rsc_autotune_knn_batched(X: torch.Tensor, sample_offsets, k_within: int, k_cross: int, metric="euclidean",
                             trials=2, stream=None):
    """Tune rsc_knn_batched's column parts and pipeline stages; returns
    ({"tc_parts", "stages"}, best ms, outputs)."""
    n, d = X.shape
    off, optr = _offsets_host(sample_offsets)
    S = len(off) - 1
    m = _METRICS[metric] if isinstance(metric, str) else int(metric)
    o = knn_opts("bf16", 0, 0, stream)
    need = _sz(0)
    _check(lib().rsc_knn_batched_workspace_size(n, d, optr, S, k_within, k_cross, m, ctypes.byref(o),
                                                ctypes.byref(need)))
    ws = _workspace(need.value, X.device)
    outs = (torch.empty((n, k_within), dtype=torch.int32, device=X.device),
            torch.empty((n, k_within), dtype=torch.float32, device=X.device),
            torch.empty((n, S * k_cross), dtype=torch.int32, device=X.device),
            torch.empty((n, S * k_cross), dtype=torch.float32, device=X.device))
    best = rsc_knn_opts()
    ms = ctypes.c_float(0)
    _check(lib().rsc_autotune_knn_batched(_ptr(X), n, d, optr, S, k_within, k_cross, m, ctypes.byref(o), trials,
                                          *[_ptr(t) for t in outs], ctypes.byref(best), ctypes.byref(ms), _ptr(ws),
                                          ws.numel()))
    return {"tc_parts": int(best.tc_parts), "stages": int(best.stages)}, float(ms.value), outs


def rsc_autotune_save(path: str):
    _check(lib().rsc_autotune_save(path.encode()))


def rsc_autotune_load(path: str):
    _check(lib().rsc_autotune_load(path.encode()))


def rsc_autotune_clear():
    _check(lib().rsc_autotune_clear())


class Partitioner:
    """Owning wrapper of an rsc_partitioner handle (see include/rsc.h)."""

    def __init__(self, d=50, n_parts=1024, hidden=256, bf16_weights=True, seed=0, _handle=None):
        self._h = _vp()
        if _handle is not None:
            self._h = _handle
        else:
            _check(lib().rsc_partitioner_create(d, n_parts, hidden, int(bf16_weights), seed, ctypes.byref(self._h)))
        self.d, self.n_parts, self.hidden = d, n_parts, hidden

    def close(self):
        if self._h:
            lib().rsc_partitioner_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def param_count(self) -> int:
        c = _i64(0)
        _check(lib().rsc_partitioner_param_count(self._h, ctypes.byref(c)))
        return int(c.value)

    def get_params(self):
        import numpy as np
        out = np.empty(self.param_count, dtype=np.float32)
        _check(lib().rsc_partitioner_get_params(self._h, out.ctypes.data_as(_vp)))
        return out

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.param_count
        _check(lib().rsc_partitioner_set_params(self._h, a.ctypes.data_as(_vp)))

    def loss_grad(self, Xb: torch.Tensor, T: torch.Tensor, stream=None):
        B = Xb.shape[0]
        need = _sz(0)
        _check(lib().rsc_partitioner_loss_grad_workspace_size(self._h, B, ctypes.byref(need)))
        ws = _workspace(need.value, Xb.device)
        grad = torch.empty(self.param_count, dtype=torch.float32, device=Xb.device)
        loss = ctypes.c_float(0)
        _check(lib().rsc_partitioner_loss_grad(self._h, _ptr(Xb), _ptr(T), B, ctypes.byref(loss), _ptr(grad),
                                               _ptr(ws), ws.numel(), _stream(stream)))
        return float(loss.value), grad

    def workspace_size(self, n, n_train=0, k=15, n_queries=0, n_probe=8) -> int:
        need = _sz(0)
        _check(lib().rsc_partitioner_workspace_size(self._h, n, n_train, k, n_queries, n_probe, ctypes.byref(need)))
        return int(need.value)

    def train(self, X: torch.Tensor, train_rows: torch.Tensor, k=15, kmeans_iters=10, epochs=10, batch=1024,
              lr=1e-3, stream=None, workspace=None) -> float:
        n = X.shape[0]
        ws = _workspace(self.workspace_size(n, len(train_rows), k, 1, 1), X.device, workspace)
        loss = ctypes.c_float(0)
        _check(lib().rsc_partitioner_train(self._h, _ptr(X), n, _ptr(train_rows), len(train_rows), k, kmeans_iters,
                                           epochs, batch, lr, ctypes.byref(loss), _ptr(ws), ws.numel(),
                                           _stream(stream)))
        return float(loss.value)

    def build_index(self, X: torch.Tensor, stream=None, workspace=None):
        n = X.shape[0]
        ws = _workspace(self.workspace_size(n, 0, 1, 1, 1), X.device, workspace)
        _check(lib().rsc_partitioner_build_index(self._h, _ptr(X), n, _ptr(ws), ws.numel(), _stream(stream)))

    def knn(self, X: torch.Tensor, k=15, n_probe=8, routing="network", query_rows=None, stream=None,
            workspace=None, out=None):
        """kNN of query_rows (int32 CUDA tensor; None = all rows) by probing n_probe parts."""
        n = X.shape[0]
        nq = n if query_rows is None else len(query_rows)
        ws = _workspace(self.workspace_size(n, 0, k, nq, n_probe), X.device, workspace)
        if out is None:
            idx = torch.empty((nq, k), dtype=torch.int32, device=X.device)
            dist = torch.empty((nq, k), dtype=torch.float32, device=X.device)
        else:
            idx, dist = out
        r = {"network": 0, "centroids": 1}[routing]
        _check(lib().rsc_knn_partitioned(self._h, _ptr(X), n, k, n_probe, r, _ptr(query_rows), nq, _ptr(idx),
                                         _ptr(dist), _ptr(ws), ws.numel(), _stream(stream)))
        return idx, dist

    def save(self, path: str):
        _check(lib().rsc_partitioner_save(self._h, path.encode()))

    @classmethod
    def load(cls, path: str):
        h = _vp()
        _check(lib().rsc_partitioner_load(path.encode(), ctypes.byref(h)))
        obj = cls.__new__(cls)
        obj._h = h
        params = _i64(0)
        _check(lib().rsc_partitioner_param_count(h, ctypes.byref(params)))
        obj.d = obj.n_parts = obj.hidden = None
        return obj


def rsc_umap_find_ab(spread: float = 1.0, min_dist: float = 0.5):
    """(a, b) of phi(d) = 1 / (1 + a d^(2b)) fitted to spread / min_dist (host)."""
    a, b = ctypes.c_float(0), ctypes.c_float(0)
    _check(lib().rsc_umap_find_ab(spread, min_dist, ctypes.byref(a), ctypes.byref(b)))
    return float(a.value), float(b.value)


def rsc_umap_workspace_size(n: int, nnz: int, dim: int) -> int:
    out = _sz(0)
    _check(lib().rsc_umap_workspace_size(n, nnz, dim, ctypes.byref(out)))
    return int(out.value)


def umap_opts(a, b, gamma=1.0, learning_rate=1.0, negative_sample_rate=5, n_epochs=200, epoch_first=0,
              epoch_last=0, seed=0, stream=None):
    return rsc_umap_opts(a, b, gamma, learning_rate, negative_sample_rate, n_epochs, epoch_first, epoch_last,
                         seed & (2**64 - 1), _stream(stream))


def rsc_umap_layout(indptr: torch.Tensor, indices: torch.Tensor, data: torch.Tensor, embedding: torch.Tensor,
                    a: float, b: float, gamma=1.0, learning_rate=1.0, negative_sample_rate=5, n_epochs=200,
                    epoch_first=0, epoch_last=0, seed=0, nnz=None, stream=None, workspace=None):
    """Epochs epoch_first..epoch_last (0, 0: all) of the UMAP layout, in place on
    `embedding` (float32 [n, dim] CUDA tensor, the initial positions).  The
    graph is the CSR of rsc_connectivities; nnz defaults to indptr[-1] (read
    from the device, which synchronises: pass it to stay asynchronous)."""
    if not (embedding.is_cuda and embedding.dtype == torch.float32 and embedding.dim() == 2
            and embedding.is_contiguous()):
        raise ValueError("embedding: contiguous float32 [n, dim] CUDA tensor expected")
    if not (indptr.dtype == torch.int64 and indices.dtype == torch.int32 and data.dtype == torch.float32):
        raise ValueError("indptr int64, indices int32, data float32 expected")
    n, dim = embedding.shape
    nnz = int(indptr[n].item()) if nnz is None else int(nnz)
    ws = _workspace(rsc_umap_workspace_size(n, nnz, dim), embedding.device, workspace)
    o = umap_opts(a, b, gamma, learning_rate, negative_sample_rate, n_epochs, epoch_first, epoch_last, seed, stream)
    _check(lib().rsc_umap_layout(_ptr(indptr), _ptr(indices), _ptr(data), n, nnz, dim, _ptr(embedding),
                                 ctypes.byref(o), _ptr(ws), ws.numel()))
    return embedding


def _host_i64(a):
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.int64)


def _host_pairs(pairs):
    import numpy as np
    return None if pairs is None else np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)


def rsc_edistance_workspace_size(n_rows, d, group_offsets, pairs=None) -> int:
    off = _host_i64(group_offsets)
    pr = _host_pairs(pairs)
    out = _sz(0)
    _check(lib().rsc_edistance_workspace_size(n_rows, d, off.ctypes.data, len(off) - 1,
                                              None if pr is None else pr.ctypes.data,
                                              0 if pr is None else len(pr), ctypes.byref(out)))
    return int(out.value)


def rsc_edistance(X: torch.Tensor, group_offsets, cell_index=None, pairs=None, with_mean=True, workspace=None,
                  stream=None):
    """Energy distances of cell groups: returns (sums, mean, E), float64 [G, G]
    CUDA tensors (mean None without with_mean).  group_offsets and pairs are
    host arrays (CSR offsets into cell_index, or into the rows of X)."""
    if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
        raise ValueError("X: float32 [n, d] CUDA tensor expected")
    X = X.contiguous()
    n_rows, d = X.shape
    off = _host_i64(group_offsets)
    G = len(off) - 1
    pr = _host_pairs(pairs)
    if cell_index is not None:
        if not (cell_index.is_cuda and cell_index.dtype == torch.int32):
            raise ValueError("cell_index: int32 CUDA tensor expected")
        cell_index = cell_index.contiguous()
    ws = _workspace(rsc_edistance_workspace_size(n_rows, d, off, pr), X.device, workspace)
    sums = torch.empty((G, G), dtype=torch.float64, device=X.device)
    mean = torch.empty((G, G), dtype=torch.float64, device=X.device) if with_mean else None
    E = torch.empty((G, G), dtype=torch.float64, device=X.device)
    _check(lib().rsc_edistance(_ptr(X), n_rows, d, _ptr(cell_index), off.ctypes.data, G,
                               None if pr is None else pr.ctypes.data, 0 if pr is None else len(pr),
                               _ptr(sums), _ptr(mean), _ptr(E), _ptr(ws), ws.numel(), _stream(stream)))
    return sums, mean, E


def edistance_onesided_pairs(n_groups: int, ref: int):
    """Pairs of the paper's onesided_distances: (ref, b) for every b, and (b, b)."""
    import numpy as np
    pairs = [(min(ref, b), max(ref, b)) for b in range(n_groups)] + [(b, b) for b in range(n_groups)]
    return np.array(pairs, dtype=np.int32)


def nnd_opts(sample=0, rev_slots=0, cand_slots=0, max_iters=0, delta=0.0, seed=0, stream=None) -> rsc_nnd_opts:
    o = rsc_nnd_opts()
    o.sample, o.rev_slots, o.cand_slots, o.max_iters = sample, rev_slots, cand_slots, max_iters
    o.delta, o.seed = float(delta), seed & (2**64 - 1)
    o.stream = _stream(stream) if torch.cuda.is_available() else None
    return o


def rsc_knn_descent_workspace_size(n: int, d: int, k: int, opts: rsc_nnd_opts | None = None) -> int:
    out = _sz(0)
    _check(lib().rsc_knn_descent_workspace_size(n, d, k, ctypes.byref(opts or rsc_nnd_opts()), ctypes.byref(out)))
    return int(out.value)


def rsc_knn_descent(X: torch.Tensor, k: int, sample=0, rev_slots=0, cand_slots=0, max_iters=0, delta=0.0, seed=0,
                    init=None, workspace=None, stream=None, with_changes=False):
    """Approximate kNN by NN-descent: returns (idx int32 [n, k], dist float32
    [n, k]) CUDA tensors, and the int64 [64] change counts with_changes.
    init: int32 [n, k] CUDA tensor of lists to start from (or None)."""
    if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
        raise ValueError("X: float32 [n, d] CUDA tensor expected")
    X = X.contiguous()
    n, d = X.shape
    o = nnd_opts(sample, rev_slots, cand_slots, max_iters, delta, seed, stream)
    ws = _workspace(rsc_knn_descent_workspace_size(n, d, k, o), X.device, workspace)
    idx = torch.empty((n, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((n, k), dtype=torch.float32, device=X.device)
    ch = torch.zeros(64, dtype=torch.int64, device=X.device) if with_changes else None
    if init is not None:
        if not (init.is_cuda and init.dtype == torch.int32 and tuple(init.shape) == (n, k)):
            raise ValueError("init: int32 [n, k] CUDA tensor expected")
        init = init.contiguous()
    _check(lib().rsc_knn_descent(_ptr(X), n, d, k, _ptr(init), _ptr(idx), _ptr(dist), _ptr(ch), ctypes.byref(o),
                                 _ptr(ws), ws.numel()))
    return (idx, dist, ch) if with_changes else (idx, dist)


def rsc_knn_descent_pairs(workspace: torch.Tensor):
    """Pairs joined per iteration by the last call on this workspace (int64 [64], host)."""
    import numpy as np
    out = np.zeros(64, dtype=np.int64)
    _check(lib().rsc_knn_descent_pairs(_ptr(workspace), workspace.numel(), out.ctypes.data))
    return out


def rsc_leiden_workspace_size(n: int, nnz: int) -> int:
    out = _sz(0)
    _check(lib().rsc_leiden_workspace_size(n, nnz, ctypes.byref(out)))
    return int(out.value)


def leiden_opts(resolution=1.0, n_iterations=2, max_levels=32, max_rounds=8, stream=None) -> rsc_leiden_opts:
    o = rsc_leiden_opts()
    o.resolution, o.n_iterations, o.max_levels, o.max_rounds = float(resolution), n_iterations, max_levels, max_rounds
    o.stream = _stream(stream) if torch.cuda.is_available() else None
    return o


def rsc_leiden(indptr: torch.Tensor, indices: torch.Tensor, data: torch.Tensor, resolution=1.0, n_iterations=2,
               max_levels=32, max_rounds=8, init=None, workspace=None, stream=None, nnz=None):
    """Leiden communities of a CSR graph: returns (membership int32 [n] CUDA
    tensor, number of communities, modularity).  nnz defaults to indptr[-1]
    (read back), so rsc_connectivities' capacity-sized outputs can be passed
    as they are."""
    if not (indptr.is_cuda and indptr.dtype == torch.int64 and indices.dtype == torch.int32
            and data.dtype == torch.float32):
        raise ValueError("indptr int64, indices int32, data float32 CUDA tensors expected")
    n = indptr.numel() - 1
    nnz = int(indptr[-1].item()) if nnz is None else int(nnz)
    if nnz > indices.numel() or nnz > data.numel():
        raise ValueError("indices / data shorter than nnz")
    o = leiden_opts(resolution, n_iterations, max_levels, max_rounds, stream)
    ws = _workspace(rsc_leiden_workspace_size(n, nnz), indptr.device, workspace)
    mem = torch.empty(n, dtype=torch.int32, device=indptr.device)
    if init is not None:
        if not (init.is_cuda and init.dtype == torch.int32 and init.numel() == n):
            raise ValueError("init: int32 [n] CUDA tensor expected")
        init = init.contiguous()
    K = _i64(0)
    q = ctypes.c_double(0.0)
    _check(lib().rsc_leiden(_ptr(indptr), _ptr(indices), _ptr(data), n, nnz, _ptr(init), _ptr(mem), ctypes.byref(K),
                            ctypes.byref(q), ctypes.byref(o), _ptr(ws), ws.numel()))
    return mem, int(K.value), float(q.value)


def rsc_leiden_last_stats() -> dict:
    """Work of this thread's last rsc_leiden call."""
    import numpy as np
    out = np.zeros(6, dtype=np.int64)
    _check(lib().rsc_leiden_last_stats(out.ctypes.data))
    return dict(zip(("levels", "move_rounds", "refine_rounds", "entries", "vertices", "launches"), out.tolist()))
