"""ctypes front end of ``numeric.c`` (test infrastructure only; see package doc).

Every function takes numpy arrays (any real dtype; converted to contiguous
fp64, or int32/int64 for indices) and returns fp64 numpy results.  The C file
is compiled on first use with ``gcc -O2 -ffp-contract=off`` (no fast-math, no
contraction) into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "numeric.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile numeric.c into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_dbl = ctypes.c_double

_SIGS = {
    "orc_square": (None, [_D, _D, _i64]),
    "orc_sum_diff": (_dbl, [_D, _D, _i64]),
    "orc_sum_abs_diff": (_dbl, [_D, _D, _i64]),
    "orc_cnd": (_dbl, [_dbl]),
    "orc_bs_call": (None, [_D, _D, _i64, _dbl, _dbl, _dbl, _dbl]),
    "orc_bs_call_scale": (None, [_D, _D, _i64, _dbl, _dbl, _dbl, _dbl]),
    "orc_gauss_weights": (None, [ctypes.c_int, _dbl, _D]),
    "orc_blur": (None, [_D, _D, _i64, _i64, _D, ctypes.c_int]),
    "orc_sobel": (None, [_D, _D, _i64, _i64]),
    "orc_sobel_scale": (None, [_D, _D, _i64, _i64]),
    "orc_minmax": (None, [_D, _i64, _D, _D]),
    "orc_extend": (None, [_D, _dbl, _dbl, _D, _i64]),
    "orc_unsharp": (None, [_D, _D, _dbl, _D, _i64]),
    "orc_combine": (None, [_D, _D, _D, _D, _D, _D, _i64]),
    "orc_scores": (None, [_D, _i64, _i64, _D, _i64, _D, _D]),
    "orc_scores_abs": (None, [_D, _i64, _i64, _D, _i64, _D, _D]),
    "orc_softmax_rows": (None, [_D, _D, _i64, _i64]),
    "orc_argmax_sum": (None, [_D, _D, _i64, _i64, _I32, _D]),
    "orc_spmv_csr": (None, [_i64, _I64, _I32, _D, _D, _D]),
    "orc_spmv_csr_abs": (None, [_i64, _I64, _I32, _D, _D, _D]),
    "orc_l2norm": (_dbl, [_D, _i64]),
    "orc_scale": (None, [_D, _dbl, _D, _i64]),
    "orc_conv3x3_relu_pool": (None, [_D, _i64, _i64, _i64, _i64, _D, _D, _i64, _D]),
    "orc_avgpool": (None, [_D, _i64, _i64, _D]),
    "orc_concat_dense": (None, [_D, _D, _i64, _i64, _D, _D, _i64, _D]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _p(a: np.ndarray):
    if a.dtype == np.float64:
        return a.ctypes.data_as(_D)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_I32)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_I64)
    raise TypeError(a.dtype)


# ---------------------------------------------------------------- VEC
def square(x):
    x = _f64(x)
    out = np.empty_like(x)
    lib().orc_square(_p(x), _p(out), x.size)
    return out


def sum_diff(x, y):
    x, y = _f64(x), _f64(y)
    assert x.size == y.size
    return lib().orc_sum_diff(_p(x), _p(y), x.size)


def sum_abs_diff(x, y):
    x, y = _f64(x), _f64(y)
    return lib().orc_sum_abs_diff(_p(x), _p(y), x.size)


# ---------------------------------------------------------------- B&S
def cnd(x: float) -> float:
    return lib().orc_cnd(float(x))


def bs_call(S, K=60.0, r=0.1, sigma=0.2, T=1.0):
    S = _f64(S)
    C = np.empty_like(S)
    lib().orc_bs_call(_p(S), _p(C), S.size, K, r, sigma, T)
    return C


def bs_call_scale(S, K=60.0, r=0.1, sigma=0.2, T=1.0):
    S = _f64(S)
    A = np.empty_like(S)
    lib().orc_bs_call_scale(_p(S), _p(A), S.size, K, r, sigma, T)
    return A


# ---------------------------------------------------------------- IMG
def gauss_weights(R: int, sigma: float):
    w = np.empty(2 * R + 1, dtype=np.float64)
    lib().orc_gauss_weights(R, sigma, _p(w))
    return w


def blur(img, w):
    img = _f64(img)
    w = _f64(w)
    R = (w.size - 1) // 2
    out = np.empty_like(img)
    lib().orc_blur(_p(img), _p(out), img.shape[0], img.shape[1], _p(w), R)
    return out


def sobel(img):
    img = _f64(img)
    out = np.empty_like(img)
    lib().orc_sobel(_p(img), _p(out), img.shape[0], img.shape[1])
    return out


def sobel_scale(img):
    """Per pixel: sum of |terms| of both Sobel gradients (the condition scale
    of the magnitude)."""
    img = _f64(img)
    out = np.empty_like(img)
    lib().orc_sobel_scale(_p(img), _p(out), img.shape[0], img.shape[1])
    return out


def minmax(x):
    x = _f64(x)
    mn, mx = ctypes.c_double(), ctypes.c_double()
    lib().orc_minmax(_p(x), x.size, ctypes.byref(mn), ctypes.byref(mx))
    return mn.value, mx.value


def extend(x, mn, mx):
    x = _f64(x)
    out = np.empty_like(x)
    lib().orc_extend(_p(x), float(mn), float(mx), _p(out), x.size)
    return out


def unsharp(img, bl, alpha):
    img, bl = _f64(img), _f64(bl)
    out = np.empty_like(img)
    lib().orc_unsharp(_p(img), _p(bl), float(alpha), _p(out), img.size)
    return out


def combine(S, b5, b9, e5, e9):
    S, b5, b9, e5, e9 = (_f64(a) for a in (S, b5, b9, e5, e9))
    out = np.empty_like(S)
    lib().orc_combine(_p(S), _p(b5), _p(b9), _p(e5), _p(e9), _p(out), S.size)
    return out


# ---------------------------------------------------------------- ML
def scores(X, T, bias):
    X, T, bias = _f64(X), _f64(T), _f64(bias)
    rows, feats = X.shape
    classes = T.shape[1]
    S = np.empty((rows, classes), dtype=np.float64)
    lib().orc_scores(_p(X), rows, feats, _p(T), classes, _p(bias), _p(S))
    return S


def scores_abs(X, T, bias):
    X, T, bias = _f64(X), _f64(T), _f64(bias)
    rows, feats = X.shape
    classes = T.shape[1]
    A = np.empty((rows, classes), dtype=np.float64)
    lib().orc_scores_abs(_p(X), rows, feats, _p(T), classes, _p(bias), _p(A))
    return A


def softmax_rows(S):
    S = _f64(S)
    P = np.empty_like(S)
    lib().orc_softmax_rows(_p(S), _p(P), S.shape[0], S.shape[1])
    return P


def argmax_sum(P1, P2):
    P1, P2 = _f64(P1), _f64(P2)
    rows, classes = P1.shape
    labels = np.empty(rows, dtype=np.int32)
    margin = np.empty(rows, dtype=np.float64)
    lib().orc_argmax_sum(_p(P1), _p(P2), rows, classes, _p(labels), _p(margin))
    return labels, margin


# ---------------------------------------------------------------- HITS
def spmv_csr(rowptr, col, val, x):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val, x = _f64(val), _f64(x)
    n = rowptr.size - 1
    y = np.empty(n, dtype=np.float64)
    lib().orc_spmv_csr(n, _p(rowptr), _p(col), _p(val), _p(x), _p(y))
    return y


def spmv_csr_abs(rowptr, col, val, x):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val, x = _f64(val), _f64(x)
    n = rowptr.size - 1
    y = np.empty(n, dtype=np.float64)
    lib().orc_spmv_csr_abs(n, _p(rowptr), _p(col), _p(val), _p(x), _p(y))
    return y


def l2norm(x):
    x = _f64(x)
    return lib().orc_l2norm(_p(x), x.size)


def scale(x, nrm):
    x = _f64(x)
    out = np.empty_like(x)
    lib().orc_scale(_p(x), float(nrm), _p(out), x.size)
    return out


# ---------------------------------------------------------------- DL
def conv3x3_relu_pool(x, wt, bias):
    """x: (n, cin, h, w); wt: (cout, cin, 3, 3); returns (n, cout, h/2, w/2)."""
    x, wt, bias = _f64(x), _f64(wt), _f64(bias)
    n, cin, h, w = x.shape
    cout = wt.shape[0]
    out = np.empty((n, cout, h // 2, w // 2), dtype=np.float64)
    lib().orc_conv3x3_relu_pool(_p(x), n, cin, h, w, _p(wt), _p(bias), cout, _p(out))
    return out


def avgpool(x):
    """x: (n, c, h, w) -> (n, c) means."""
    x = _f64(x)
    n, c, h, w = x.shape
    e = np.empty((n, c), dtype=np.float64)
    lib().orc_avgpool(_p(x), n * c, h * w, _p(e))
    return e


def concat_dense(e1, e2, wd, bias):
    e1, e2, wd, bias = _f64(e1), _f64(e2), _f64(wd), _f64(bias)
    n, c = e1.shape
    classes = wd.shape[1]
    out = np.empty((n, classes), dtype=np.float64)
    lib().orc_concat_dense(_p(e1), _p(e2), n, c, _p(wd), _p(bias), classes, _p(out))
    return out
