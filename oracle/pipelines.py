"""Each benchmark DAG run serially, one launch after the other, in fp64.

Test infrastructure only (see the package doc).  The launch sequences are the
programs of Section IV-B (VEC, B&S, IMG, ML, HITS); every step calls one
routine of ``numeric`` and nothing is fused or reordered.  Every function
returns a dict holding each intermediate array under the name the GPU program
gives it, so that a test can compare node by node.
"""
from __future__ import annotations

import numpy as np

from . import numeric as N

# IMG readings (the paper gives no parameters): 5x5 blur sigma 1, 9x9 blur
# sigma 2, unsharp amount 0.5.
IMG_R5, IMG_SIGMA5 = 2, 1.0
IMG_R9, IMG_SIGMA9 = 4, 2.0
IMG_ALPHA = 0.5

# B&S parameters of the benchmark configuration.
BS_K, BS_R, BS_SIGMA, BS_T = 60.0, 0.1, 0.2, 1.0


def vec(x, y):
    """VEC: K1 x := x*x, K2 y := y*y, K3 z = sum(x - y)."""
    x2 = N.square(x)
    y2 = N.square(y)
    z = N.sum_diff(x2, y2)
    return {"x": x2, "y": y2, "z": z, "z_scale": N.sum_abs_diff(x2, y2)}


def bs(prices, K=BS_K, r=BS_R, sigma=BS_SIGMA, T=BS_T):
    """B&S: one call-price node per input vector, all independent."""
    return {"C%d" % i: N.bs_call(S, K, r, sigma, T) for i, S in enumerate(prices)}


def img(image):
    """IMG: blur5, blur9, sobel x2, minmax x2, extend x2, unsharp, combine."""
    w5 = N.gauss_weights(IMG_R5, IMG_SIGMA5)
    w9 = N.gauss_weights(IMG_R9, IMG_SIGMA9)
    out = {}
    out["b5"] = N.blur(image, w5)
    out["b9"] = N.blur(image, w9)
    out["e5_raw"] = N.sobel(out["b5"])
    out["e9_raw"] = N.sobel(out["b9"])
    out["mm5"] = N.minmax(out["e5_raw"])
    out["mm9"] = N.minmax(out["e9_raw"])
    out["e5"] = N.extend(out["e5_raw"], *out["mm5"]).reshape(image.shape)
    out["e9"] = N.extend(out["e9_raw"], *out["mm9"]).reshape(image.shape)
    out["s"] = N.unsharp(image, out["b5"], IMG_ALPHA)
    out["out"] = N.combine(out["s"], out["b5"], out["b9"], out["e5"], out["e9"])
    return out


def ml(X, nb_table, nb_prior, ridge_w, ridge_b):
    """ML: naive-Bayes and ridge scores, row softmax of each, argmax of sum."""
    out = {}
    out["s1"] = N.scores(X, nb_table, nb_prior)
    out["s2"] = N.scores(X, ridge_w, ridge_b)
    out["s1_scale"] = N.scores_abs(X, nb_table, nb_prior)
    out["s2_scale"] = N.scores_abs(X, ridge_w, ridge_b)
    out["p1"] = N.softmax_rows(out["s1"])
    out["p2"] = N.softmax_rows(out["s2"])
    out["labels"], out["margin"] = N.argmax_sum(out["p1"], out["p2"])
    return out


def hits(csr, csc, iters=5):
    """HITS with simultaneous (Jacobi) updates from h_0 = a_0 = 1:
    a_{k+1} = A^T h_k / ||A^T h_k||, h_{k+1} = A a_k / ||A a_k||
    (a zero norm leaves its vector unscaled).  ``csr`` = (rowptr, col, val)
    of A, ``csc`` = the same of A^T.  Returns every iterate."""
    n = len(csr[0]) - 1
    a = np.ones(n, dtype=np.float64)
    h = np.ones(n, dtype=np.float64)
    out = {"a": [a], "h": [h], "a_raw": [], "h_raw": [], "na": [], "nh": []}
    for _ in range(iters):
        a_raw = N.spmv_csr(csc[0], csc[1], csc[2], h)
        h_raw = N.spmv_csr(csr[0], csr[1], csr[2], a)
        na = N.l2norm(a_raw)
        nh = N.l2norm(h_raw)
        a = N.scale(a_raw, na)
        h = N.scale(h_raw, nh)
        for k, v in (("a_raw", a_raw), ("h_raw", h_raw), ("na", na),
                     ("nh", nh), ("a", a), ("h", h)):
            out[k].append(v)
    return out


def dl(x1, x2, w1, b1, w2, b2, wd, bd):
    """DL: two conv3x3 + ReLU + 2x2 max-pool branches, a global average pool
    of each, the concatenation of the two embeddings and a dense layer."""
    out = {}
    out["p1"] = N.conv3x3_relu_pool(x1, w1, b1)
    out["p2"] = N.conv3x3_relu_pool(x2, w2, b2)
    out["e1"] = N.avgpool(out["p1"])
    out["e2"] = N.avgpool(out["p2"])
    out["logits"] = N.concat_dense(out["e1"], out["e2"], wd, bd)
    return out
