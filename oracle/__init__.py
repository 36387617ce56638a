"""FP64 CPU oracle for MAPI (arXiv 2110.12065) -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and it imports nothing from them.

The arithmetic lives in ``mapi_oracle.c`` (plain loops, IEEE double,
sequential sums); this module only compiles it with gcc and marshals numpy
arrays through ctypes.  Each wrapper names the passage of the paper it
follows; the C file states the readings of ambiguous points.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

OP_MIN1, OP_MIN2, OP_DIAMOND, OP_DOT = 0, 1, 2, 3
OPS = {"min1": OP_MIN1, "min2": OP_MIN2, "diamond": OP_DIAMOND, "dot": OP_DOT}
FINAL_L2 = 1
RAW_START = 2
OK, EINVAL, EZERONORM, ENONFINITE = 0, 1, 4, 5

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mapi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, OpenMP over rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i, l, p = C.c_double, C.c_int, C.c_long, C.c_void_p
            sig = {
                "or_term": (d, [i, d, d]),
                "or_vecprod": (d, [i, p, p, l]),
                "or_matvec": (None, [i, p, l, l, l, p, p]),
                "or_norm1": (d, [p, l]),
                "or_norm2": (d, [p, l]),
                "or_mapi": (i, [i, p, l, l, p, i, i, d, p, p, p]),
                "or_mincov": (None, [i, p, l, l, l, d, p]),
                "or_mavp_outer": (None, [i, p, l, p]),
                "or_deflate": (None, [i, p, l, p, l, l, p]),
                "or_deflate_vec": (None, [i, p, l, p, l, l]),
                "or_reconstruct": (None, [i, p, l, l, l, p, l, l, p, p, l]),
                "or_pair_step": (None, [i, p, l, l, l, p, d, p]),
                "or_pca_topk": (i, [i, i, p, l, l, l, l, i, d, d, p, l, p, l, p]),
                "or_google_matrix": (None, [l, p, p, d, p]),
                "or_pagerank_sparse": (i, [i, l, p, p, d, i, p, i, d, p, p, p]),
                "or_minibatch_momentum": (i, [i, p, l, l, p, i, i, d, p, i, p]),
                "or_round_bf16": (d, [d]),
                "or_round_e4m3": (d, [d]),
                "or_fp8_row_exponent": (i, [p, l]),
                "or_quant_fp8_rows": (None, [p, l, l, l, p, l, p]),
                "or_quant_bf16": (None, [p, l, l, l, p, l]),
                "or_int_scale": (i, [p, l, l, l, i, p]),
                "or_quant_int": (None, [p, l, l, l, i, p, l]),
                "or_mapi_int": (i, [i, p, l, l, i, p, i, d, p, p, p]),
                "or_set_num_threads": (None, [i]),
                "or_get_max_threads": (i, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _op(op) -> int:
    return OPS[op] if isinstance(op, str) else int(op)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def set_num_threads(n: int) -> None:
    _get().or_set_num_threads(int(n))


def max_threads() -> int:
    return int(_get().or_get_max_threads())


def term(op, a: float, b: float) -> float:
    """One term of min1 Eq. (3), min2 Eq. (4), diamond Eq. (7) or dot."""
    return float(_get().or_term(_op(op), float(a), float(b)))


def vecprod(op, w, x) -> float:
    """w^T (+) x, Eq. (3)/(4)/(7)."""
    w, x = _f64(w), _f64(x)
    assert w.shape == x.shape and w.ndim == 1
    return float(_get().or_vecprod(_op(op), _ptr(w), _ptr(x), w.size))


def matvec(op, A, w) -> np.ndarray:
    """y = A (+) w, rows of A against w (Alg. 1 step 3)."""
    A, w = _f64(A), _f64(w)
    rows, cols = A.shape
    y = np.empty(rows)
    _get().or_matvec(_op(op), _ptr(A), rows, cols, cols, _ptr(w), _ptr(y))
    return y


def mapi(op, A, w0, iters: int, tol: float = 0.0, final_l2: bool = False,
         raw_start: bool = False):
    """Algorithm 1 (MAPI); op='dot' gives regular power iteration, Eq. (1).

    Returns (status, w, iters_done, last_delta)."""
    A, w0 = _f64(A), _f64(w0)
    n = A.shape[0]
    assert A.shape == (n, n) and w0.shape == (n,)
    w = np.empty(n)
    it, dl = C.c_int(0), C.c_double(0.0)
    flags = (FINAL_L2 if final_l2 else 0) | (RAW_START if raw_start else 0)
    st = _get().or_mapi(_op(op), _ptr(A), n, n, _ptr(w0), flags, int(iters),
                        float(tol), _ptr(w), C.byref(it), C.byref(dl))
    return int(st), w, int(it.value), float(dl.value)


def mincov(op, X, denom: float) -> np.ndarray:
    """C = (1/denom) X (+) X^T, Eq. (5) (Alg. 2 step 4 with denom = N - 1)."""
    X = _f64(X)
    D, N = X.shape
    Cm = np.empty((D, D))
    _get().or_mincov(_op(op), _ptr(X), D, N, N, float(denom), _ptr(Cm))
    return Cm


def mavp_outer(op, w) -> np.ndarray:
    """P = w (+) w^T (Alg. 2 steps 6 and 8)."""
    w = _f64(w)
    P = np.empty((w.size, w.size))
    _get().or_mavp_outer(_op(op), _ptr(w), w.size, _ptr(P))
    return P


def deflate(op, Cm, W) -> np.ndarray:
    """C_k = (I - sum_m w_m (+) w_m^T) C (Alg. 2 step 6; §1 sum form)."""
    Cm = _f64(Cm)
    D = Cm.shape[0]
    W = np.asfortranarray(np.asarray(W, dtype=np.float64).reshape(D, -1))
    k = W.shape[1]
    out = np.empty((D, D))
    _get().or_deflate(_op(op), _ptr(Cm), D, _ptr(W), k, D, _ptr(out))
    return out


def deflate_vec(op, y, W) -> np.ndarray:
    """y - sum_m (w_m (+) w_m^T) y."""
    y = _f64(y).copy()
    D = y.size
    W = np.asfortranarray(np.asarray(W, dtype=np.float64).reshape(D, -1))
    _get().or_deflate_vec(_op(op), _ptr(y), D, _ptr(W), W.shape[1], D)
    return y


def pair_step(op, X, w, denom: float) -> np.ndarray:
    """t_n = x_n^T (+) w, y_d = sum_n X_dn (+) t_n / denom (matrix-free PCA step)."""
    X, w = _f64(X), _f64(w)
    D, N = X.shape
    y = np.empty(D)
    _get().or_pair_step(_op(op), _ptr(X), D, N, N, _ptr(w), float(denom), _ptr(y))
    return y


def pca_topk(mode, op, X, k: int, iters: int, denom: float, W0,
             tol: float = 0.0):
    """Top-k MAPI principal vectors; mode 'mincov' (Alg. 2) or 'pair'.

    Returns (status, P (D x k), iters_done (k,))."""
    m = {"mincov": 0, "pair": 1}[mode] if isinstance(mode, str) else int(mode)
    X = _f64(X)
    D, N = X.shape
    W0 = np.asfortranarray(np.asarray(W0, dtype=np.float64).reshape(D, k))
    P = np.zeros((D, k), order="F")
    its = np.zeros(k, dtype=np.int32)
    st = _get().or_pca_topk(m, _op(op), _ptr(X), D, N, N, k, int(iters),
                            float(tol), float(denom), _ptr(W0), D, _ptr(P), D,
                            _ptr(its))
    return int(st), P, its


def reconstruct(op, W, V, m) -> np.ndarray:
    """Alg. 2 step 8 for every column v_i of V (D x N): (W (+) W^T)(v_i - m) + m,
    R_pq = sum_c term(W_pc, W_qc), the product with v_i - m ordinary."""
    V, m = _f64(V), _f64(m)
    D, N = V.shape
    W = np.asfortranarray(np.asarray(W, dtype=np.float64).reshape(D, -1))
    out = np.empty((D, N))
    _get().or_reconstruct(_op(op), _ptr(W), D, W.shape[1], D, _ptr(V), N, N, _ptr(m),
                          _ptr(out), N)
    return out


def image_reconstruct(op, images, k: int, iters: int, W0, tol: float = 0.0):
    """Alg. 2 end to end on N images of P pixels (images: N x P, one image a
    row, i.e. step 1's v_i).  Step 2: V = [v_1 ... v_N] (P x N); step 3: m the
    row mean of V, V - m; step 4: C = (V - m) (+) (V - m)^T / (N - 1); steps
    5-6: k components by MAPI on the deflated C (W0: P x k raw starts); step 8
    for every i.  Returns (status, W (P x k), reconstructions (N x P), iters)."""
    V = np.ascontiguousarray(_f64(images).T)
    P, N = V.shape
    m = V.mean(axis=1)
    X = V - m[:, None]
    st, W, its = pca_topk("mincov", op, X, k, iters, float(N - 1), W0, tol)
    if st != OK:
        return st, W, None, its
    return st, W, reconstruct(op, W, V, m).T.copy(), its


def google_matrix(n: int, indptr, indices, alpha: float = 0.85) -> np.ndarray:
    """G = alpha H + (1 - alpha)/n 1, Eq. (11); dangling columns uniform."""
    ip = np.ascontiguousarray(np.asarray(indptr, dtype=np.int32))
    ix = np.ascontiguousarray(np.asarray(indices, dtype=np.int32))
    G = np.empty((n, n))
    _get().or_google_matrix(n, _ptr(ip), _ptr(ix), float(alpha), _ptr(G))
    return G


def pagerank(op, n: int, indptr, indices, w0, iters: int, alpha: float = 0.85,
             tol: float = 0.0, G=None):
    """MAPI-PageRank (§3.3): Alg. 1 on the Google matrix with a final l2 step."""
    if G is None:
        G = google_matrix(n, indptr, indices, alpha)
    return mapi(op, G, w0, iters, tol=tol, final_l2=True)


def pagerank_sparse(op, n: int, indptr, indices, w0, iters: int, alpha: float = 0.85,
                    tol: float = 0.0, round32: bool = True):
    """MAPI-PageRank (§3.3) on the Google matrix of Eq. (11) without forming
    it; with round32 the entry values are those of an FP32 copy of G.
    Returns (status, w, iters_done, last_delta)."""
    ip = np.ascontiguousarray(np.asarray(indptr, dtype=np.int32))
    ix = np.ascontiguousarray(np.asarray(indices, dtype=np.int32))
    w0 = _f64(w0)
    w = np.empty(n)
    it, dl = C.c_int(0), C.c_double(0.0)
    st = _get().or_pagerank_sparse(_op(op), n, _ptr(ip), _ptr(ix), float(alpha),
                                   1 if round32 else 0, _ptr(w0), int(iters), float(tol),
                                   _ptr(w), C.byref(it), C.byref(dl))
    return st, w, it.value, dl.value


def minibatch_momentum(op, X, batch, beta: float, w0, final_l2: bool = True):
    """Mini-batch MAPI with momentum (Alg. 3).  X: N x D samples (rows);
    batch: T x s sample indices (the draws of step 3).  Returns (status, w)."""
    X = _f64(X)
    N, D = X.shape
    b = np.ascontiguousarray(np.asarray(batch, dtype=np.int32))
    T, s = b.shape
    w0 = _f64(w0)
    w = np.empty(D)
    st = _get().or_minibatch_momentum(_op(op), _ptr(X), N, D, _ptr(b), T, s, float(beta),
                                      _ptr(w0), FINAL_L2 if final_l2 else 0, _ptr(w))
    return st, w


def round_bf16(x) -> np.ndarray:
    f = _get().or_round_bf16
    return np.vectorize(lambda v: f(float(v)), otypes=[np.float64])(np.asarray(x, np.float64))


def round_e4m3(x) -> np.ndarray:
    f = _get().or_round_e4m3
    return np.vectorize(lambda v: f(float(v)), otypes=[np.float64])(np.asarray(x, np.float64))


def quant_bf16(A) -> np.ndarray:
    """Values a bf16 copy of fp32 A holds (round to nearest even)."""
    A = _f32(A)
    rows, cols = A.shape
    out = np.empty((rows, cols))
    _get().or_quant_bf16(_ptr(A), rows, cols, cols, _ptr(out), cols)
    return out


def quant_fp8_rows(A):
    """(dequantised values, row exponents k_i) of the E4M3 copy with scale 2^k_i."""
    A = _f32(A)
    rows, cols = A.shape
    out = np.empty((rows, cols))
    ex = np.empty(rows, dtype=np.int32)
    _get().or_quant_fp8_rows(_ptr(A), rows, cols, cols, _ptr(out), cols, _ptr(ex))
    return out, ex


def int_scale(A, bits: int) -> int:
    """Shared exponent q for int16 (bits=16) or int8 (bits=8) storage."""
    A = _f32(A)
    rows, cols = A.shape
    q = C.c_int(0)
    qmax = 32767 if bits == 16 else 127
    st = _get().or_int_scale(_ptr(A), rows, cols, cols, qmax, C.byref(q))
    if st != OK:
        raise ValueError("matrix entries too large for integer storage")
    return int(q.value)


def quant_int(A, q: int) -> np.ndarray:
    """A_q = RNE(A 2^q) as int64."""
    A = _f32(A)
    rows, cols = A.shape
    out = np.empty((rows, cols), dtype=np.int64)
    _get().or_quant_int(_ptr(A), rows, cols, cols, int(q), _ptr(out), cols)
    return out


def mapi_int(op, Aq, q: int, w0, iters: int, tol: float = 0.0):
    """Alg. 1 in exact integers on integer storage (units of 2^-q).

    Returns (status, w_q (int64), iters_done, last_delta_q)."""
    Aq = np.ascontiguousarray(np.asarray(Aq, dtype=np.int64))
    n = Aq.shape[0]
    w0 = _f32(w0)
    w = np.empty(n, dtype=np.int64)
    it, dl = C.c_int(0), C.c_longlong(0)
    st = _get().or_mapi_int(_op(op), _ptr(Aq), n, n, int(q), _ptr(w0),
                            int(iters), float(tol), _ptr(w), C.byref(it),
                            C.byref(dl))
    return int(st), w, int(it.value), int(dl.value)
