"""Python binding of libmapi.so (include/mapi.h): MAPI on GB300.

Multiplication-avoiding power iteration (Pan et al., arXiv 2110.12065) runs
entirely in the CUDA library; this module only marshals arguments through
ctypes.  Every function has the name of the C entry point it calls.  Device
arrays are torch CUDA tensors (PyTorch provides device memory and streams);
host arrays are numpy.  A non-OK status raises ``MapiError``.

There is no CPU fallback: importing this package without the compiled
library raises ImportError (build it with ``build.build()``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build_mod

__all__ = [
    "MapiError", "load", "mapi_create", "mapi_destroy", "mapi_status_str",
    "mapi_last_error", "mapi_matrix_upload", "mapi_matrix_free",
    "mapi_matrix_info", "mapi_matrix_download", "mapi_iterate", "mapi_mincov",
    "mapi_pca_topk", "mapi_google_matrix", "mapi_pagerank", "mapi_profile",
    "mapi_get_stats", "mapi_iterate_noalloc", "mapi_iterate_batched",
    "mapi_autotune_batched", "mapi_submit", "mapi_poll", "mapi_cancel",
    "mapi_pagerank_sparse", "mapi_iterate_switch", "mapi_minibatch_momentum",
    "mapi_mavp_project", "mapi_image_reconstruct", "mapi_pair_phases", "mapi_debug_stall",
    "mapi_rows_product", "mapi_pair_partial", "mapi_alu_probe", "mapi_pair_cluster_times",
    "mapi_set_batched_rows",
    "KERNEL_CLASSES",
    "OP", "ST", "FLAG_FINAL_L2", "FLAG_RAW_START", "SCALE_AUTO",
    "PCA_MINCOV", "PCA_PAIR", "STATUS",
]

OP = {"min1": 0, "min2": 1, "diamond": 2, "dot": 3}
ST = {"f32": 0, "bf16": 1, "fp8": 2, "i16": 3, "i8": 4}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EBUDGET", 4: "EZERONORM",
          5: "ENONFINITE", 6: "EAGAIN", 7: "ETIMEOUT", 8: "ECANCELLED",
          9: "ECUDA", 10: "ENOTSUP"}
FLAG_FINAL_L2 = 1
FLAG_RAW_START = 2
SCALE_AUTO = -(2 ** 31)
PCA_MINCOV, PCA_PAIR = 0, 1
REQ = {"pca": 0, "pagerank": 1}
_CUDA_STREAM_LEGACY = 1

LIB_PATH = _build_mod.LIB
_lib = None


class MapiError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = "", partial=None):
        self.status = status
        self.name = STATUS.get(status, str(status))
        self.partial = partial
        super().__init__(f"{where}: {self.name} ({detail})")


KERNEL_CLASSES = ("gemv", "pair", "pair_finish", "mincov", "batched")


class _Stats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("timed", C.c_uint64 * 5), ("ms", C.c_double * 5),
                ("bytes", C.c_double * 5), ("terms", C.c_double * 5)]


class _BatchItem(C.Structure):
    _fields_ = [("A", C.c_void_p), ("w0", C.c_void_p), ("w_out", C.c_void_p)]


class _Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("op", C.c_int), ("storage", C.c_int),
                ("max_iters", C.c_int), ("tol_l1", C.c_double),
                ("X", C.c_void_p), ("D", C.c_int), ("N", C.c_int), ("k", C.c_int),
                ("cov_denom", C.c_double), ("indptr", C.c_void_p), ("indices", C.c_void_p),
                ("n", C.c_int), ("alpha", C.c_double), ("w0", C.c_void_p),
                ("out", C.c_void_p), ("user", C.c_void_p)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int * 8), ("last_delta", C.c_double),
                ("queue_ms", C.c_double), ("build_ms", C.c_double), ("run_ms", C.c_double),
                ("latency_ms", C.c_double),
                ("user", C.c_void_p)]


class _Config(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget_bytes", C.c_size_t),
                ("cuda_stream", C.c_void_p), ("max_slots", C.c_int),
                ("tune_cache_path", C.c_char_p)]


def load(path: str | None = None):
    """Load libmapi.so (raises ImportError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libmapi.so not built ({p}); run paper_2110_12065_gb300.build.build()")
    lib = C.CDLL(p)
    i, p_, i64, d, u = C.c_int, C.c_void_p, C.c_int64, C.c_double, C.c_uint
    sigs = {
        "mapi_create": [C.POINTER(_Config), C.POINTER(p_)],
        "mapi_destroy": [p_],
        "mapi_status_str": [i],
        "mapi_last_error": [p_],
        "mapi_matrix_upload": [p_, p_, i, i, i, i, i64, i, i, C.POINTER(p_)],
        "mapi_matrix_free": [p_, p_],
        "mapi_matrix_info": [p_, p_, p_, p_, p_, p_],
        "mapi_matrix_download": [p_, p_, p_, p_],
        "mapi_iterate": [p_, p_, i, i, p_, i64, i, d, u, p_, p_, p_],
        "mapi_mincov": [p_, p_, i, d, p_],
        "mapi_iterate_switch": [p_, p_, i, p_, i, d, i, d, u, p_, p_, p_],
        "mapi_minibatch_momentum": [p_, p_, i, i, p_, i, i, d, i, p_, u, p_],
        "mapi_mavp_project": [p_, i, p_, i64, i, i, p_, i64, i, p_, p_, i64],
        "mapi_image_reconstruct": [p_, p_, i, i, i, i, i, d, p_, p_, p_, p_],
        "mapi_pca_topk": [p_, p_, i, i, i, i, d, d, p_, p_, p_],
        "mapi_google_matrix": [p_, p_, p_, i, d, i, C.POINTER(p_)],
        "mapi_pagerank": [p_, p_, p_, i, d, i, i, p_, i, d, p_, p_, p_],
        "mapi_pagerank_sparse": [p_, p_, p_, i, d, i, p_, i, d, p_, p_, p_],
        "mapi_profile": [p_, i],
        "mapi_pair_phases": [p_, i, p_],
        "mapi_pair_cluster_times": [p_, p_, i, p_],
        "mapi_set_batched_rows": [p_, i, i, i],
        "mapi_rows_product": [p_, p_, i, i, i, p_, p_],
        "mapi_alu_probe": [p_, i, p_],
        "mapi_pair_partial": [p_, p_, i, p_, p_],
        "mapi_debug_stall": [p_, i64],
        "mapi_get_stats": [p_, C.POINTER(_Stats), i],
        "mapi_iterate_noalloc": [p_, i, i64, i, p_, i, d, u, p_, p_, p_, p_],
        "mapi_iterate_batched": [p_, p_, i, i, i, i, d, u, p_, p_, p_],
        "mapi_autotune_batched": [p_, p_, i, i, i, i, p_],
        "mapi_submit": [p_, C.POINTER(_Request), C.POINTER(C.c_uint64)],
        "mapi_poll": [p_, C.c_uint64, C.POINTER(_Result)],
        "mapi_cancel": [p_, C.c_uint64],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.mapi_status_str.restype = C.c_char_p
    lib.mapi_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _check(st: int, where: str, ctx=None, partial=None):
    if st != 0:
        detail = ""
        if ctx is not None:
            detail = (load().mapi_last_error(ctx) or b"").decode(errors="replace")
        raise MapiError(st, where, detail, partial)


def _dptr(t) -> int:
    """Device address of a torch CUDA tensor (checks contiguity and device)."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _torch():
    import torch
    return torch


def mapi_status_str(status: int) -> str:
    return load().mapi_status_str(int(status)).decode()


def mapi_last_error(ctx) -> str:
    return (load().mapi_last_error(ctx) or b"").decode(errors="replace")


def mapi_create(device: int = 0, stream=None, hbm_budget_bytes: int = 0,
                max_slots: int = 0, tune_cache_path: str | None = None):
    """Create a context.  ``stream`` is a torch.cuda.Stream (default: torch's
    current stream, so library work is ordered with the caller's)."""
    lib = load()
    if stream is None:
        stream = _torch().cuda.current_stream(device)
    handle = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    if handle == 0:
        handle = _CUDA_STREAM_LEGACY
    cfg = _Config(int(device), int(hbm_budget_bytes), C.c_void_p(handle), int(max_slots),
                  tune_cache_path.encode() if tune_cache_path else None)
    out = C.c_void_p()
    _check(lib.mapi_create(C.byref(cfg), C.byref(out)), "mapi_create")
    return out


def mapi_destroy(ctx) -> None:
    _check(load().mapi_destroy(ctx), "mapi_destroy")


def mapi_matrix_upload(ctx, src, storage="f32", int_scale_log2: int = SCALE_AUTO):
    """Pack a 2-D FP32 matrix (torch CUDA tensor or numpy host array)."""
    lib = load()
    st = ST[storage] if isinstance(storage, str) else int(storage)
    out = C.c_void_p()
    if isinstance(src, np.ndarray):
        a = np.ascontiguousarray(src, dtype=np.float32)
        rows, cols = a.shape
        r = lib.mapi_matrix_upload(ctx, a.ctypes.data_as(C.c_void_p), 0, 0, rows, cols, cols,
                                   st, int(int_scale_log2), C.byref(out))
    else:
        torch = _torch()
        if src.dtype != torch.float32 or src.dim() != 2:
            raise ValueError("expected a 2-D float32 tensor")
        rows, cols = src.shape
        ld = src.stride(0)
        if src.stride(1) != 1:
            raise ValueError("rows must be contiguous")
        if src.is_cuda:
            r = lib.mapi_matrix_upload(ctx, C.c_void_p(src.data_ptr()), 1, 0, rows, cols, ld, st,
                                       int(int_scale_log2), C.byref(out))
        else:
            r = lib.mapi_matrix_upload(ctx, C.c_void_p(src.data_ptr()), 0, 0, rows, cols, ld, st,
                                       int(int_scale_log2), C.byref(out))
    _check(r, "mapi_matrix_upload", ctx)
    return out


def mapi_matrix_free(ctx, mat) -> None:
    _check(load().mapi_matrix_free(ctx, mat), "mapi_matrix_free", ctx)


def mapi_matrix_info(mat) -> dict:
    rows, cols, stg, q = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    ld = C.c_int64()
    _check(load().mapi_matrix_info(mat, C.byref(rows), C.byref(cols), C.byref(ld),
                                   C.byref(stg), C.byref(q)), "mapi_matrix_info")
    return {"rows": rows.value, "cols": cols.value, "ld": ld.value,
            "storage": stg.value, "int_scale_log2": q.value}


def mapi_matrix_download(ctx, mat):
    """(dequantised values as float64 numpy, FP8 row exponents or None)."""
    info = mapi_matrix_info(mat)
    out = np.empty((info["rows"], info["cols"]), dtype=np.float64)
    ex = np.empty(info["rows"], dtype=np.int32) if info["storage"] == ST["fp8"] else None
    _check(load().mapi_matrix_download(
        ctx, mat, out.ctypes.data_as(C.c_void_p),
        ex.ctypes.data_as(C.c_void_p) if ex is not None else None),
        "mapi_matrix_download", ctx)
    return out, ex


def mapi_iterate(ctx, A, op, w0, max_iters: int, tol_l1: float = 0.0,
                 flags: int = 0, w_out=None):
    """Alg. 1 (or RPI with op='dot') on packed A for the start vectors w0
    (torch CUDA float32, shape (n,) or (nvec, n)).  Returns
    (w_out like w0, iters_done list, last_delta list)."""
    torch = _torch()
    opi = OP[op] if isinstance(op, str) else int(op)
    squeeze = w0.dim() == 1
    w = w0.reshape(1, -1) if squeeze else w0
    if w.dtype != torch.float32:
        raise ValueError("w0 must be float32")
    nvec, n = w.shape
    if w_out is None:
        w_out = torch.empty_like(w)
    it = (C.c_int * nvec)()
    dl = (C.c_double * nvec)()
    st = load().mapi_iterate(ctx, A, opi, nvec, C.c_void_p(_dptr(w)), n, int(max_iters),
                             float(tol_l1), int(flags), C.c_void_p(_dptr(w_out)), it, dl)
    res = (w_out.reshape(-1) if squeeze else w_out, list(it), list(dl))
    _check(st, "mapi_iterate", ctx, partial=res)
    return res


def mapi_iterate_switch(ctx, A, op, w0, mapi_iters: int, rpi_iters: int,
                        mapi_tol: float = 0.0, rpi_tol: float = 0.0, flags: int = 0,
                        w_out=None):
    """MAPI for up to mapi_iters steps, then regular power iteration from its
    iterate.  Returns (w (n,), [iters MAPI, iters RPI], [delta MAPI, delta RPI])."""
    torch = _torch()
    if w_out is None:
        w_out = torch.empty_like(w0)
    opi = OP[op] if isinstance(op, str) else int(op)
    it = (C.c_int * 2)()
    dl = (C.c_double * 2)()
    st = load().mapi_iterate_switch(ctx, A, opi, C.c_void_p(_dptr(w0)), int(mapi_iters),
                                    float(mapi_tol), int(rpi_iters), float(rpi_tol), int(flags),
                                    C.c_void_p(_dptr(w_out)), it, dl)
    res = (w_out, list(it), list(dl))
    _check(st, "mapi_iterate_switch", ctx, partial=res)
    return res


def mapi_minibatch_momentum(ctx, X, batch, beta: float, op, w0, flags: int = 0,
                            w_out=None):
    """Alg. 3 over the sample draws in batch.  X: torch CUDA float32 (N, D);
    batch: torch CUDA int32 (T, s); w0: CUDA float32 (D,).  Returns w_out."""
    torch = _torch()
    if X.dtype != torch.float32 or batch.dtype != torch.int32:
        raise ValueError("X float32, batch int32")
    X = X.contiguous()
    batch = batch.contiguous()
    N, D = X.shape
    T, s = batch.shape
    if w_out is None:
        w_out = torch.empty_like(w0)
    opi = OP[op] if isinstance(op, str) else int(op)
    st = load().mapi_minibatch_momentum(ctx, C.c_void_p(_dptr(X)), int(N), int(D),
                                        C.c_void_p(_dptr(batch)), int(T), int(s), float(beta),
                                        opi, C.c_void_p(_dptr(w0)), int(flags),
                                        C.c_void_p(_dptr(w_out)))
    _check(st, "mapi_minibatch_momentum", ctx, partial=w_out)
    return w_out


def mapi_mavp_project(ctx, op, W, rows_in, add=None, out=None):
    """out_r = (W (+) W^T) in_r + add (Alg. 2 step 8).  W: torch CUDA float32
    (k, D) (row c is component c, i.e. D x k column-major); rows_in: (rows, D);
    add: (D,) or None.  Returns out (rows, D)."""
    torch = _torch()
    W = W.contiguous()
    rows_in = rows_in.contiguous()
    k, D = W.shape
    rows = rows_in.shape[0]
    if out is None:
        out = torch.empty((rows, D), dtype=torch.float32, device=rows_in.device)
    opi = OP[op] if isinstance(op, str) else int(op)
    addp = C.c_void_p(_dptr(add.contiguous())) if add is not None else None
    _check(load().mapi_mavp_project(ctx, opi, C.c_void_p(_dptr(W)), int(D), int(D), int(k),
                                    C.c_void_p(_dptr(rows_in)), int(D), int(rows), addp,
                                    C.c_void_p(_dptr(out)), int(D)),
           "mapi_mavp_project", ctx)
    return out


def mapi_image_reconstruct(ctx, images, k: int, op, iters: int, w0, tol_l1: float = 0.0):
    """Alg. 2 on N images of P pixels (images: torch CUDA float32 (N, P));
    w0: (k, P) raw start vectors.  Returns (W (k, P), recon (N, P), iters)."""
    torch = _torch()
    images = images.contiguous()
    N, P = images.shape
    W = torch.empty((k, P), dtype=torch.float32, device=images.device)
    R = torch.empty((N, P), dtype=torch.float32, device=images.device)
    it = (C.c_int * k)()
    opi = OP[op] if isinstance(op, str) else int(op)
    st = load().mapi_image_reconstruct(ctx, C.c_void_p(_dptr(images)), int(N), int(P), int(k),
                                       opi, int(iters), float(tol_l1),
                                       C.c_void_p(_dptr(w0.contiguous())), C.c_void_p(_dptr(W)),
                                       C.c_void_p(_dptr(R)), it)
    res = (W, R, list(it))
    _check(st, "mapi_image_reconstruct", ctx, partial=res)
    return res


def mapi_mincov(ctx, X, op, denom: float, C_out=None):
    """C = (1/denom) X (+) X^T (Eq. (5)) for packed X (D x N)."""
    torch = _torch()
    D = mapi_matrix_info(X)["rows"]
    if C_out is None:
        C_out = torch.empty((D, D), dtype=torch.float32, device="cuda")
    opi = OP[op] if isinstance(op, str) else int(op)
    _check(load().mapi_mincov(ctx, X, opi, float(denom), C.c_void_p(_dptr(C_out))),
           "mapi_mincov", ctx)
    return C_out


def mapi_pca_topk(ctx, X, k: int, mode, op, iters_per_vec: int, cov_denom: float,
                  w0, tol_l1: float = 0.0, P_out=None):
    """Top-k MAPI principal vectors.  w0: torch CUDA float32 (k, D) (row c is
    start vector c, i.e. D x k column-major).  Returns (P (k, D), iters list)."""
    torch = _torch()
    m = {"mincov": PCA_MINCOV, "pair": PCA_PAIR}[mode] if isinstance(mode, str) else int(mode)
    opi = OP[op] if isinstance(op, str) else int(op)
    if P_out is None:
        P_out = torch.empty_like(w0)
    it = (C.c_int * k)()
    st = load().mapi_pca_topk(ctx, X, int(k), m, opi, int(iters_per_vec), float(tol_l1),
                              float(cov_denom), C.c_void_p(_dptr(w0)),
                              C.c_void_p(_dptr(P_out)), it)
    res = (P_out, list(it))
    _check(st, "mapi_pca_topk", ctx, partial=res)
    return res


def mapi_google_matrix(ctx, indptr, indices, n: int, alpha: float = 0.85,
                       storage="f32"):
    """Pack G = alpha H + (1 - alpha)/n (Eq. (11)) from out-link CSR (torch
    CUDA int32 tensors)."""
    out = C.c_void_p()
    st = ST[storage] if isinstance(storage, str) else int(storage)
    _check(load().mapi_google_matrix(ctx, C.c_void_p(_dptr(indptr)), C.c_void_p(_dptr(indices)),
                                     int(n), float(alpha), st, C.byref(out)),
           "mapi_google_matrix", ctx)
    return out


def mapi_pagerank(ctx, indptr, indices, n: int, w0, max_iters: int,
                  alpha: float = 0.85, storage="f32", op="min1",
                  tol_l1: float = 0.0, rank_out=None):
    """MAPI-PageRank (§3.3).  Returns (rank (n,), iters_done, last_delta)."""
    torch = _torch()
    if rank_out is None:
        rank_out = torch.empty(n, dtype=torch.float32, device="cuda")
    st = ST[storage] if isinstance(storage, str) else int(storage)
    opi = OP[op] if isinstance(op, str) else int(op)
    it, dl = C.c_int(), C.c_double()
    r = load().mapi_pagerank(ctx, C.c_void_p(_dptr(indptr)), C.c_void_p(_dptr(indices)), int(n),
                             float(alpha), st, opi, C.c_void_p(_dptr(w0)), int(max_iters),
                             float(tol_l1), C.c_void_p(_dptr(rank_out)), C.byref(it),
                             C.byref(dl))
    res = (rank_out, it.value, dl.value)
    _check(r, "mapi_pagerank", ctx, partial=res)
    return res


def mapi_pagerank_sparse(ctx, indptr, indices, n: int, w0, max_iters: int,
                         alpha: float = 0.85, op="min1", tol_l1: float = 0.0, rank_out=None):
    """MAPI-PageRank (§3.3) in O(E + n) per step, without forming G.  indptr /
    indices: torch CUDA int32 out-link CSR.  Returns (rank (n,), iters_done,
    last_delta)."""
    torch = _torch()
    if rank_out is None:
        rank_out = torch.empty(n, dtype=torch.float32, device="cuda")
    opi = OP[op] if isinstance(op, str) else int(op)
    it, dl = C.c_int(), C.c_double()
    r = load().mapi_pagerank_sparse(ctx, C.c_void_p(_dptr(indptr)), C.c_void_p(_dptr(indices)),
                                    int(n), float(alpha), opi, C.c_void_p(_dptr(w0)),
                                    int(max_iters), float(tol_l1), C.c_void_p(_dptr(rank_out)),
                                    C.byref(it), C.byref(dl))
    res = (rank_out, it.value, dl.value)
    _check(r, "mapi_pagerank_sparse", ctx, partial=res)
    return res


def mapi_profile(ctx, enable: bool = True) -> None:
    """Time the library's streaming kernels with CUDA events on their stream."""
    _check(load().mapi_profile(ctx, 1 if enable else 0), "mapi_profile", ctx)


def mapi_rows_product(ctx, A, row_begin: int, row_end: int, op, w, y_out=None):
    """y[r] = a_(row_begin + r)^T (+) w for a block of rows of packed A
    (unnormalised; a row shard of Alg. 1 step 3).  w: torch CUDA float32."""
    torch = _torch()
    if y_out is None:
        y_out = torch.empty(max(0, row_end - row_begin), dtype=torch.float32, device=w.device)
    opi = OP[op] if isinstance(op, str) else int(op)
    _check(load().mapi_rows_product(ctx, A, int(row_begin), int(row_end), opi,
                                    C.c_void_p(_dptr(w)), C.c_void_p(_dptr(y_out))),
           "mapi_rows_product", ctx)
    return y_out


def mapi_pair_partial(ctx, X, op, w, y_out=None):
    """Unnormalised pair product of packed X (D x N): y_d = sum_n X_dn (+)
    (x_n^T (+) w), a column shard's partial.  w: torch CUDA float32 (D,)."""
    torch = _torch()
    if y_out is None:
        y_out = torch.empty_like(w)
    opi = OP[op] if isinstance(op, str) else int(op)
    _check(load().mapi_pair_partial(ctx, X, opi, C.c_void_p(_dptr(w)),
                                    C.c_void_p(_dptr(y_out))),
           "mapi_pair_partial", ctx)
    return y_out


PAIR_PHASES = ("steps", "publish_to_start", "start_to_first_arrival", "start_to_last_arrival",
               "last_arrival_to_epilogue", "reduce_rows", "deflate", "norm_stop_publish")


def mapi_pair_phases(ctx, enable: bool = True) -> dict:
    """Pair-step phase stamps since stamping was last switched on (steps,
    then microseconds per step for each phase); then switch it on or off."""
    out = (C.c_double * 8)()
    _check(load().mapi_pair_phases(ctx, 1 if enable else 0, out), "mapi_pair_phases", ctx)
    return {k: float(v) for k, v in zip(PAIR_PHASES, out)}


def mapi_pair_cluster_times(ctx) -> list:
    """Each streaming cluster's loop time per pair step (microseconds) over
    the steps stamped since mapi_pair_phases last switched stamping on."""
    cap = 128
    us = (C.c_double * cap)()
    n = C.c_int()
    _check(load().mapi_pair_cluster_times(ctx, us, cap, C.byref(n)), "mapi_pair_cluster_times",
           ctx)
    return [float(us[c]) for c in range(n.value)]


ALU_MIXES = ("min1_term_f32", "ffma", "fmnmx", "min1_term_bf16", "min1_term_bf16_x4")


def mapi_alu_probe(ctx, mix) -> float:
    """Per-SM, per-clock rate of one instruction mix (see ALU_MIXES)."""
    m = ALU_MIXES.index(mix) if isinstance(mix, str) else int(mix)
    out = C.c_double()
    _check(load().mapi_alu_probe(ctx, m, C.byref(out)), "mapi_alu_probe", ctx)
    return out.value


def mapi_debug_stall(ctx, limit_ns: int) -> None:
    """Failure-detection test hook: later pair steps also wait, bounded by
    limit_ns, on a barrier that nothing arrives at (0 turns it off)."""
    _check(load().mapi_debug_stall(ctx, int(limit_ns)), "mapi_debug_stall", ctx)


def mapi_get_stats(ctx, reset: bool = False) -> dict:
    """Launch count and, per kernel class, timed launches, summed ms,
    algorithmic bytes and terms."""
    st = _Stats()
    _check(load().mapi_get_stats(ctx, C.byref(st), 1 if reset else 0), "mapi_get_stats", ctx)
    out = {"launches": int(st.launches)}
    for i, name in enumerate(KERNEL_CLASSES):
        out[name] = {"launches": int(st.timed[i]), "ms": float(st.ms[i]),
                     "bytes": float(st.bytes[i]), "terms": float(st.terms[i])}
    return out


def mapi_iterate_noalloc(A, op, w0, max_iters: int, tol_l1: float = 0.0, flags: int = 0,
                         w_out=None, stream=None):
    """Alg. 1 on a caller-owned FP32 device matrix without any allocation in
    the library (scratch is a fixed static device array; n <= 8192).  A: torch
    CUDA float32 (n, >= n) with rows 16-byte aligned; w0: (n,).  w_out must be
    preallocated by callers that cannot allocate.  Returns (w_out, iters, delta)."""
    torch = _torch()
    # every size, type and device is checked here, before the library runs:
    # the C side cannot see how long w0 and w_out are, and a short or
    # half-precision w_out would be written past its end
    if A.dim() != 2 or A.stride(1) != 1 or A.dtype != torch.float32:
        raise ValueError("A must be a 2-D float32 tensor with contiguous rows")
    n = A.shape[0]
    if A.shape[1] < n:
        raise ValueError(f"A must hold n = {n} columns, has {A.shape[1]}")
    for name, v in (("w0", w0), ("w_out", w_out)):
        if v is None:
            continue
        if v.dtype != torch.float32 or v.numel() != n or (v.dim() > 1 and not v.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 tensor of {n} elements")
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    dev = A.device
    if dev.index != torch.cuda.current_device():
        raise ValueError("A must be on the current CUDA device")
    for name, v in (("w0", w0), ("w_out", w_out)):
        if v is not None and v.device != dev:
            raise ValueError(f"{name} must be on {dev}, the device of A")
    if w_out is None:
        w_out = torch.empty(n, dtype=torch.float32, device=A.device)
    opi = OP[op] if isinstance(op, str) else int(op)
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    handle = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    it, dl = C.c_int(), C.c_double()
    st = load().mapi_iterate_noalloc(C.c_void_p(A.data_ptr()), n, A.stride(0), opi,
                                     C.c_void_p(_dptr(w0)), int(max_iters), float(tol_l1),
                                     int(flags), C.c_void_p(_dptr(w_out)), C.byref(it),
                                     C.byref(dl), C.c_void_p(handle or None))
    res = (w_out, it.value, dl.value)
    _check(st, "mapi_iterate_noalloc", None, partial=res)
    return res


def _batch_array(items):
    arr = (_BatchItem * len(items))()
    for k, (mat, w0, w_out) in enumerate(items):
        arr[k].A = mat.value if hasattr(mat, "value") else mat
        arr[k].w0 = _dptr(w0)
        arr[k].w_out = _dptr(w_out)
    return arr


def mapi_iterate_batched(ctx, items, op, nvec: int, max_iters: int, tol_l1: float = 0.0,
                         flags: int = 0):
    """Batched Alg. 1.  items: list of (packed matrix, w0, w_out) with w0 / w_out
    torch CUDA float32 of shape (nvec, n).  Returns (iters, last_delta,
    statuses) as (count, nvec) numpy arrays."""
    arr = _batch_array(items)
    n = len(items)
    it = np.zeros((n, nvec), dtype=np.int32)
    dl = np.zeros((n, nvec), dtype=np.float64)
    sts = np.zeros((n, nvec), dtype=np.int32)
    opi = OP[op] if isinstance(op, str) else int(op)
    st = load().mapi_iterate_batched(ctx, arr, n, opi, int(nvec), int(max_iters), float(tol_l1),
                                     int(flags), it.ctypes.data_as(C.c_void_p),
                                     dl.ctypes.data_as(C.c_void_p),
                                     sts.ctypes.data_as(C.c_void_p))
    res = (it, dl, sts)
    _check(st, "mapi_iterate_batched", ctx, partial=res)
    return res


def mapi_autotune_batched(ctx, items, op, nvec: int, iters: int = 2) -> int:
    """Time the batched kernel variants on this batch; returns the chosen
    rows per warp (kept by the context)."""
    arr = _batch_array(items)
    ch = C.c_int()
    opi = OP[op] if isinstance(op, str) else int(op)
    _check(load().mapi_autotune_batched(ctx, arr, len(items), opi, int(nvec), int(iters),
                                        C.byref(ch)), "mapi_autotune_batched", ctx)
    return ch.value


def mapi_set_batched_rows(ctx, storage, nvec: int, rows_per_warp: int) -> None:
    """Pin the batched solve's rows per warp (1, 2, 4, 8) for this context,
    storage ("f32" / "bf16") and vector count, as the autotuner would."""
    st = ST[storage] if isinstance(storage, str) else int(storage)
    _check(load().mapi_set_batched_rows(ctx, st, int(nvec), int(rows_per_warp)),
           "mapi_set_batched_rows", ctx)


# host arrays of each open request (the library reads and writes them until
# the request has finished), keyed by (context, ticket)
_serve_keep = {}


def _ctx_key(ctx):
    return ctx.value if hasattr(ctx, "value") else int(ctx)


def mapi_submit(ctx, kind, w0, op="min1", storage="bf16", max_iters: int = 100,
                tol_l1: float = 0.0, X=None, k: int = 1, cov_denom: float | None = None,
                indptr=None, indices=None, alpha: float = 0.85) -> int:
    """Queue a served request (kind "pca" or "pagerank").  Host numpy inputs:
    PCA X (D x N float32, row-major), w0 (k x D: one start vector per row);
    PageRank indptr / indices (int32 out-link CSR), w0 (n).  Returns the
    ticket; the result comes from mapi_poll."""
    r = _Request()
    r.kind = REQ[kind] if isinstance(kind, str) else int(kind)
    r.op = OP[op] if isinstance(op, str) else int(op)
    r.storage = ST[storage] if isinstance(storage, str) else int(storage)
    r.max_iters = int(max_iters)
    r.tol_l1 = float(tol_l1)
    keep = []
    if r.kind == REQ["pca"]:
        X = np.ascontiguousarray(X, dtype=np.float32)
        D, N = X.shape
        W = np.ascontiguousarray(np.asarray(w0, dtype=np.float32).reshape(k, D))
        out = np.zeros((k, D), dtype=np.float32)
        r.X, r.D, r.N, r.k = X.ctypes.data, D, N, int(k)
        r.cov_denom = float(N if cov_denom is None else cov_denom)
        keep += [X, W]
    else:
        ip = np.ascontiguousarray(indptr, dtype=np.int32)
        ix = np.ascontiguousarray(indices, dtype=np.int32)
        n = ip.shape[0] - 1
        W = np.ascontiguousarray(np.asarray(w0, dtype=np.float32).reshape(n))
        out = np.zeros(n, dtype=np.float32)
        r.indptr, r.indices, r.n, r.alpha = ip.ctypes.data, ix.ctypes.data, n, float(alpha)
        keep += [ip, ix, W]
    r.w0 = W.ctypes.data
    r.out = out.ctypes.data
    t = C.c_uint64()
    _check(load().mapi_submit(ctx, C.byref(r), C.byref(t)), "mapi_submit", ctx)
    _serve_keep[(_ctx_key(ctx), t.value)] = (keep, out)
    return t.value


def mapi_poll(ctx, ticket: int):
    """None while the request is queued or running; afterwards a dict with
    status (int), status_name, iters (per component), last_delta, queue_ms,
    build_ms, run_ms, latency_ms and out (the result array: k x D components, or the
    n-vector of ranks).  Raises MapiError for an unknown ticket."""
    res = _Result()
    st = load().mapi_poll(ctx, C.c_uint64(int(ticket)), C.byref(res))
    if st == 6:  # EAGAIN
        return None
    if st == 1:
        _check(st, "mapi_poll", ctx)
    keep, out = _serve_keep.pop((_ctx_key(ctx), int(ticket)), (None, None))
    return {"status": int(res.status), "status_name": STATUS.get(int(res.status)),
            "iters": list(res.iters), "last_delta": res.last_delta, "queue_ms": res.queue_ms,
            "build_ms": res.build_ms, "run_ms": res.run_ms, "latency_ms": res.latency_ms,
            "out": out}


def mapi_cancel(ctx, ticket: int) -> None:
    """Drop a queued or running request (it then reports ECANCELLED)."""
    _check(load().mapi_cancel(ctx, C.c_uint64(int(ticket))), "mapi_cancel", ctx)
