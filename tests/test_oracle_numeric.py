"""Pins of the numeric oracle against things other than itself: library
routines (numpy, scipy), closed forms, limits, a textbook worked example and
brute-force integration.  CPU only."""
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.ndimage
import scipy.signal
import scipy.sparse
import scipy.special

import datagen
from oracle import numeric as N
from oracle import pipelines as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ VEC
def test_square_rounds_to_ieee_single_multiply():
    x, _ = datagen.vec_inputs(4097, seed=11)
    x = np.concatenate([x, np.float32([0.0, -0.0, 1e-20, 3.4e19, -2.5])])
    with np.errstate(over="ignore"):  # 3.4e19^2 overflows to inf on both sides
        got = N.square(x).astype(np.float32)
        want = x * x
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_sum_diff_identities():
    x, y = datagen.vec_inputs(1000, seed=5)
    assert N.sum_diff(x, x) == 0.0
    # x_i = c  ->  sum (c^2 - y_i^2) = n c^2 - sum y_i^2 (exact sums by fsum)
    c = np.float32(0.75)
    out = P.vec(np.full(1000, c, np.float32), y)
    want = 1000 * float(c) ** 2 - math.fsum(float(v) ** 2 for v in y)
    assert abs(out["z"] - want) <= 1e-12 * out["z_scale"]
    # ramp x_i = i, y = 0: sum i^2 = n(n-1)(2n-1)/6
    n = 2000
    out = P.vec(np.arange(n, dtype=np.float32), np.zeros(n, np.float32))
    assert out["z"] == n * (n - 1) * (2 * n - 1) // 6
    # sign: sum(x - y), not sum(y - x)
    assert N.sum_diff(np.float32([2.0]), np.float32([1.0])) == 1.0
    # the condition scale: sum |x - y| (exactly rounded sum by fsum)
    assert N.sum_abs_diff(x, y) == pytest.approx(
        math.fsum(abs(float(a) - float(b)) for a, b in zip(x, y)), rel=1e-14)


# ------------------------------------------------------------------ B&S
def test_cnd_matches_library_ndtr():
    xs = np.linspace(-9, 9, 721)
    got = np.array([N.cnd(v) for v in xs])
    # deep in the left tail the argument -x/sqrt(2) carries a relative
    # rounding of ~1e-16 that erfc amplifies by ~x^2
    np.testing.assert_allclose(got, scipy.special.ndtr(xs), rtol=1e-12, atol=1e-300)


def _load_textbook():
    rows = []
    with open(os.path.join(GOLDEN, "bs_textbook.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def test_bs_textbook_example():
    for S, K, r, s, T, c, dec in _load_textbook():
        got = N.bs_call(np.array([S]), K, r, s, T)[0]
        assert round(got, int(dec)) == pytest.approx(c, abs=1e-12)


@pytest.mark.parametrize("S,K,r,s,T", [(42, 40, 0.1, 0.2, 0.5),
                                        (10, 60, 0.1, 0.2, 1.0),
                                        (99.9, 60, 0.1, 0.2, 1.0),
                                        (60, 60, 0.03, 0.6, 2.0)])
def test_bs_equals_risk_neutral_expectation(S, K, r, s, T):
    """C = exp(-rT) E[max(S_T - K, 0)], S_T lognormal; integrated
    numerically over the standard normal z."""
    def payoff(z):
        ST = S * math.exp((r - 0.5 * s * s) * T + s * math.sqrt(T) * z)
        return max(ST - K, 0.0) * math.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    z0 = (math.log(K / S) - (r - 0.5 * s * s) * T) / (s * math.sqrt(T))
    val, _ = scipy.integrate.quad(payoff, z0, 40.0, epsabs=1e-13, epsrel=1e-13, limit=400)
    want = math.exp(-r * T) * val
    got = N.bs_call(np.array([S]), K, r, s, T)[0]
    assert got == pytest.approx(want, rel=1e-9, abs=1e-11)


def test_bs_forward_at_the_money_closed_form():
    K, r, s, T = 60.0, 0.1, 0.2, 1.0
    S = K * math.exp(-r * T)
    got = N.bs_call(np.array([S]), K, r, s, T)[0]
    assert got == pytest.approx(S * math.erf(s * math.sqrt(T) / (2 * math.sqrt(2))), rel=1e-13)


def test_bs_limits_and_bounds():
    K, r, T = 60.0, 0.1, 1.0
    S = np.linspace(10, 100, 91)
    disc = K * math.exp(-r * T)
    # sigma -> 0: intrinsic value of the forward
    got = N.bs_call(S, K, r, 1e-6, T)
    np.testing.assert_allclose(got, np.maximum(S - disc, 0.0), atol=1e-9)
    C = N.bs_call(S, K, r, 0.2, T)
    assert np.all(C >= np.maximum(S - disc, 0.0) - 1e-12)
    assert np.all(C <= S)
    assert np.all(np.diff(C) > 0)          # increasing in S
    assert np.all(np.diff(C, 2) > -1e-12)  # convex in S


def test_bs_term_scale_limits():
    K, r, T = 60.0, 0.1, 1.0
    disc = K * math.exp(-r * T)
    S = np.array([10.0, 40.0, 59.0, 80.0, 100.0])
    # sigma -> 0: both CDFs are 1 in the money (S + K e^-rT), 0 out of it
    np.testing.assert_allclose(N.bs_call_scale(S, K, r, 1e-6, T),
                               np.where(S > disc, S + disc, 0.0), atol=1e-9)
    C = N.bs_call(S, K, r, 0.2, T)
    A = N.bs_call_scale(S, K, r, 0.2, T)
    assert np.all(A >= np.abs(C)) and np.all(A <= S + disc)


# ------------------------------------------------------------------ IMG
@pytest.mark.parametrize("R,sigma", [(P.IMG_R5, P.IMG_SIGMA5), (P.IMG_R9, P.IMG_SIGMA9)])
def test_gauss_weights_match_scipy_window(R, sigma):
    w = N.gauss_weights(R, sigma)
    ref = scipy.signal.windows.gaussian(2 * R + 1, std=sigma)
    np.testing.assert_allclose(w, ref / ref.sum(), rtol=1e-14)


@pytest.mark.parametrize("shape", [(1, 1), (7, 13), (3, 50), (33, 31)])
@pytest.mark.parametrize("R,sigma", [(2, 1.0), (4, 2.0)])
def test_blur_matches_library_correlate_clamped(shape, R, sigma):
    img = datagen.image(*shape, seed=7)
    w = N.gauss_weights(R, sigma)
    got = N.blur(img, w)
    ref = scipy.ndimage.correlate(img.astype(np.float64), np.outer(w, w), mode="nearest")
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)


def test_blur_impulse_and_constant():
    w = N.gauss_weights(4, 2.0)
    img = np.zeros((21, 21))
    img[10, 10] = 1.0
    got = N.blur(img, w)
    np.testing.assert_allclose(got[6:15, 6:15], np.outer(w, w), rtol=1e-14)
    assert np.all(got[:6] == 0) and np.all(got[:, 15:] == 0)
    const = N.blur(np.full((9, 12), 0.3), w)
    np.testing.assert_allclose(const, 0.3, rtol=1e-14)


@pytest.mark.parametrize("shape", [(1, 1), (5, 9), (40, 33)])
def test_sobel_matches_library_sobel(shape):
    img = datagen.image(*shape, seed=8).astype(np.float64)
    got = N.sobel(img)
    gx = scipy.ndimage.sobel(img, axis=1, mode="nearest")
    gy = scipy.ndimage.sobel(img, axis=0, mode="nearest")
    np.testing.assert_allclose(got, np.hypot(gx, gy), rtol=1e-13, atol=1e-14)


def test_sobel_constant_and_ramp():
    # exact zero for a constant whose multiples are exact; rounding-level
    # otherwise (the nine-term sums cancel in a fixed order)
    assert np.all(N.sobel(np.full((8, 8), 0.75)) == 0.0)
    assert np.all(N.sobel(np.full((8, 8), 0.7)) < 1e-15)
    s = 0.25
    ramp = s * np.tile(np.arange(16.0), (10, 1))  # slope s along columns
    got = N.sobel(ramp)
    np.testing.assert_allclose(got[1:-1, 1:-1], 8 * s, rtol=1e-14)
    # clamped edges see half the difference
    np.testing.assert_allclose(got[1:-1, 0], 4 * s, rtol=1e-14)


@pytest.mark.parametrize("shape", [(1, 1), (6, 11), (31, 40)])
def test_sobel_scale_against_correlation_with_absolute_kernels(shape):
    """The Sobel condition scale is sum |Kx v| + sum |Ky v|: for a signed
    image that is the correlation of |img| with |Kx| plus with |Ky| (clamped
    edges); scipy's correlate gives it independently."""
    img = datagen.image(*shape, seed=18).astype(np.float64) - 0.5
    kx = np.array([[-1.0, 0.0, 1.0], [-2.0, 0.0, 2.0], [-1.0, 0.0, 1.0]])
    a = np.abs(img)
    want = (scipy.ndimage.correlate(a, np.abs(kx), mode="nearest")
            + scipy.ndimage.correlate(a, np.abs(kx.T), mode="nearest"))
    np.testing.assert_allclose(N.sobel_scale(img), want, rtol=1e-14, atol=1e-15)


def test_sobel_scale_closed_forms():
    # constant c: each gradient has terms of total weight 8, so 16 |c|
    np.testing.assert_allclose(N.sobel_scale(np.full((5, 7), -0.75)), 12.0, rtol=1e-15)
    # a single impulse v at an interior pixel: every 3x3 window that holds
    # it sees it once with |Kx| + |Ky| weight (0..4 each); the total over
    # all pixels is sum(|Kx|) + sum(|Ky|) = 16 |v|
    img = np.zeros((9, 9))
    img[4, 4] = 2.5
    sc = N.sobel_scale(img)
    assert sc.sum() == pytest.approx(16 * 2.5, rel=1e-15)
    assert sc[4, 4] == 0.0  # the centre weight of both kernels is 0
    assert sc[4, 3] == pytest.approx(2.5 * (2 + 0), rel=1e-15)
    assert sc[3, 3] == pytest.approx(2.5 * (1 + 1), rel=1e-15)


def test_minmax_extend_unsharp_combine():
    x = datagen.image(13, 17, seed=9).astype(np.float64)
    mn, mx = N.minmax(x)
    assert (mn, mx) == (x.min(), x.max())
    e = N.extend(x, mn, mx)
    assert e.min() == 0.0 and e.max() == 1.0
    np.testing.assert_allclose(e, (x - x.min()) / np.ptp(x), rtol=1e-15)
    assert np.all(N.extend(np.full(5, 2.0), 2.0, 2.0) == 0.0)
    b = datagen.image(13, 17, seed=10).astype(np.float64)
    assert np.array_equal(N.unsharp(x, b, 0.0), x)
    assert np.array_equal(N.unsharp(x, x, 0.5), x)
    np.testing.assert_allclose(N.unsharp(x, b, 0.5), 1.5 * x - 0.5 * b, rtol=1e-15)
    S, b5, b9 = x, b, x * 0.5
    one, zero = np.ones_like(x), np.zeros_like(x)
    assert np.array_equal(N.combine(S, b5, b9, one, zero), S)
    assert np.array_equal(N.combine(S, b5, b9, zero, one), b5)
    assert np.array_equal(N.combine(S, b5, b9, zero, zero), b9)
    half = np.full_like(x, 0.5)
    np.testing.assert_allclose(N.combine(S, b5, b9, half, half),
                               0.5 * S + 0.25 * b5 + 0.25 * b9, rtol=1e-15)


# ------------------------------------------------------------------- ML
def test_scores_match_library_matmul():
    X, T, p, W, b = datagen.ml_inputs(37, feats=64, classes=10, seed=12)
    np.testing.assert_array_equal(N.scores(X, T, p), X.astype(np.float64) @ T + p)
    np.testing.assert_array_equal(N.scores(X, W, b), X.astype(np.float64) @ W + b)
    np.testing.assert_array_equal(N.scores_abs(X, W, b),
                                  np.abs(X.astype(np.float64)) @ np.abs(W) + np.abs(b))


def test_softmax_matches_library():
    S = np.random.default_rng(1).normal(0, 30, size=(50, 10))
    np.testing.assert_allclose(N.softmax_rows(S), scipy.special.softmax(S, axis=1), rtol=1e-13)


def test_argmax_ties_and_margin():
    P1 = np.array([[0.2, 0.5, 0.5], [0.9, 0.05, 0.05], [0.1, 0.1, 0.8]])
    P2 = np.array([[0.3, 0.0, 0.0], [0.0, 0.5, 0.5], [0.2, 0.7, 0.1]])
    labels, margin = N.argmax_sum(P1, P2)
    assert labels.tolist() == [0, 0, 2]
    np.testing.assert_allclose(margin, [0.0, 0.35, 0.1], atol=1e-15)
    labels, _ = N.argmax_sum(np.array([[0.5, 0.5]]), np.array([[0.5, 0.5]]))
    assert labels.tolist() == [0]


def test_ml_dominant_class_labels():
    rows, feats = 20, 32
    X = np.ones((rows, feats), np.int32)
    T = np.zeros((feats, 10), np.float32)
    T[:, 7] = 1.0
    out = P.ml(X, T, np.zeros(10, np.float32), -T, np.zeros(10, np.float32))
    assert np.all(out["labels"] == 7)
    np.testing.assert_allclose(out["p1"].sum(axis=1), 1.0, rtol=1e-15)


# ----------------------------------------------------------------- HITS
def _tiny_graph(n, nnz, seed):
    csr, csc = datagen.hits_graph(n, nnz, seed=seed)
    return csr, csc


def test_spmv_matches_library_sparse():
    (rp, col, val), _ = _tiny_graph(300, 2000, seed=3)
    x = np.random.default_rng(0).random(300)
    A = scipy.sparse.csr_matrix((val.astype(np.float64), col, rp), shape=(300, 300))
    np.testing.assert_allclose(N.spmv_csr(rp, col, val, x), A @ x, rtol=1e-14)
    np.testing.assert_allclose(N.spmv_csr_abs(rp, col, -val, x), A @ x, rtol=1e-14)
    # the benchmark's weights are all 1: general weights, signed, as well
    w = np.random.default_rng(1).normal(size=val.size)
    Aw = scipy.sparse.csr_matrix((w, col, rp), shape=(300, 300))
    np.testing.assert_allclose(N.spmv_csr(rp, col, w, x), Aw @ x, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(N.spmv_csr_abs(rp, col, w, x), abs(Aw) @ x, rtol=1e-12)


def test_l2norm_and_scale():
    x = np.random.default_rng(2).normal(size=1001)
    assert N.l2norm(x) == pytest.approx(np.linalg.norm(x), rel=1e-14)
    np.testing.assert_allclose(N.scale(x, 2.0), x / 2.0, rtol=1e-16)
    z = np.zeros(7)
    assert np.array_equal(N.scale(z, 0.0), z)
    assert np.array_equal(N.scale(x, 0.0), x)


def test_hits_first_iterate_is_degrees():
    csr, csc = _tiny_graph(500, 3000, seed=5)
    out = P.hits(csr, csc, iters=1)
    indeg = np.bincount(csr[1], minlength=500)
    outdeg = np.diff(csr[0])
    assert np.array_equal(out["a_raw"][0], indeg)
    assert np.array_equal(out["h_raw"][0], outdeg)


def test_hits_converges_to_principal_eigenvectors():
    n = 40
    csr, csc = _tiny_graph(n, 300, seed=6)
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(csr[0]))
    A[rows, csr[1]] = 1.0
    out = P.hits(csr, csc, iters=400)
    wa, va = np.linalg.eigh(A.T @ A)
    wh, vh = np.linalg.eigh(A @ A.T)
    assert wa[-1] - wa[-2] > 1e-3 * wa[-1]
    a, h = out["a"][-1], out["h"][-1]
    np.testing.assert_allclose(np.abs(a), np.abs(va[:, -1]), atol=1e-9)
    np.testing.assert_allclose(np.abs(h), np.abs(vh[:, -1]), atol=1e-9)


# ------------------------------------------------------------------- DL
def test_conv_relu_pool_matches_library_correlate():
    (x1, _x2, w1, b1, *_), _ = datagen.dl_inputs(n=2, h=10, w=14, cout=5, seed=1)
    got = N.conv3x3_relu_pool(x1, w1, b1)
    n, cin, h, w = x1.shape
    ref = np.zeros((n, 5, h, w))
    for b in range(n):
        for co in range(5):
            s = np.full((h, w), float(b1[co]))
            for ci in range(cin):
                s += scipy.signal.correlate2d(x1[b, ci].astype(np.float64), w1[co, ci].astype(np.float64),
                                              mode="same", boundary="fill", fillvalue=0.0)
            ref[b, co] = np.maximum(s, 0.0)
    pooled = ref.reshape(n, 5, h // 2, 2, w // 2, 2).max(axis=(3, 5))
    np.testing.assert_allclose(got, pooled, rtol=1e-13, atol=1e-14)


def test_avgpool_and_concat_dense_match_library():
    g = np.random.default_rng(4)
    p = g.random((3, 4, 6, 8))
    np.testing.assert_allclose(N.avgpool(p), p.mean(axis=(2, 3)), rtol=1e-14)
    e1, e2 = g.random((3, 4)), g.random((3, 4))
    wd, bd = g.normal(size=(8, 5)), g.normal(size=5)
    np.testing.assert_allclose(N.concat_dense(e1, e2, wd, bd), np.concatenate([e1, e2], axis=1) @ wd + bd,
                               rtol=1e-13)


def test_bf16_rounding_matches_torch():
    import torch
    a = np.random.default_rng(0).normal(0, 3, 10000).astype(np.float32)
    ours = datagen.to_bf16_bits(a)
    theirs = torch.from_numpy(a).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, theirs)


# ------------------------------------------------------- whole programs
# Each benchmark program composed again from library primitives, so that the
# wiring of the oracle's programs (which intermediate feeds which node) is
# pinned, not only each node.  The inputs of the two branches differ, so a
# crossed wire changes the result.

def _library_conv_pool(x, wt, bias):
    n, cin, h, w = x.shape
    cout = wt.shape[0]
    ref = np.zeros((n, cout, h, w))
    for b in range(n):
        for co in range(cout):
            s = np.full((h, w), float(bias[co]))
            for ci in range(cin):
                s += scipy.signal.correlate2d(x[b, ci].astype(np.float64), wt[co, ci].astype(np.float64),
                                              mode="same", boundary="fill", fillvalue=0.0)
            ref[b, co] = np.maximum(s, 0.0)
    return ref.reshape(n, cout, h // 2, 2, w // 2, 2).max(axis=(3, 5))


def test_img_program_matches_library_composition():
    image = datagen.image(23, 31, seed=21).astype(np.float64)
    out = P.img(image)

    def blur(R, sigma):
        w = scipy.signal.windows.gaussian(2 * R + 1, sigma)
        w /= w.sum()
        return scipy.ndimage.correlate(image, np.outer(w, w), mode="nearest")

    def magnitude(b):
        return np.hypot(scipy.ndimage.sobel(b, axis=0, mode="nearest"), scipy.ndimage.sobel(b, axis=1, mode="nearest"))

    b5, b9 = blur(P.IMG_R5, P.IMG_SIGMA5), blur(P.IMG_R9, P.IMG_SIGMA9)
    e5r, e9r = magnitude(b5), magnitude(b9)
    e5, e9 = (e5r - e5r.min()) / np.ptp(e5r), (e9r - e9r.min()) / np.ptp(e9r)
    s = image + P.IMG_ALPHA * (image - b5)
    final = e5 * s + (1 - e5) * (e9 * b5 + (1 - e9) * b9)
    for key, want in (("b5", b5), ("b9", b9), ("e5_raw", e5r), ("e9_raw", e9r), ("e5", e5), ("e9", e9),
                      ("s", s), ("out", final)):
        np.testing.assert_allclose(np.asarray(out[key]).reshape(image.shape), want, rtol=1e-12, atol=1e-12,
                                   err_msg=key)


def test_ml_program_matches_library_composition():
    X, T, p, W, b = datagen.ml_inputs(41, feats=64, classes=10, seed=22)
    out = P.ml(X, T, p, W, b)
    Xd = X.astype(np.float64)
    s1, s2 = Xd @ T + p, Xd @ W + b
    p1, p2 = scipy.special.softmax(s1, axis=1), scipy.special.softmax(s2, axis=1)
    np.testing.assert_array_equal(out["s1"], s1)
    np.testing.assert_array_equal(out["s2"], s2)
    np.testing.assert_allclose(out["p1"], p1, rtol=1e-13)
    np.testing.assert_allclose(out["p2"], p2, rtol=1e-13)
    assert np.array_equal(out["labels"], np.argmax(p1 + p2, axis=1))


def test_dl_program_matches_library_composition():
    (x1, x2, w1, b1, w2, b2, wd, bd), _ = datagen.dl_inputs(n=2, h=6, w=10, cout=4, classes=3, seed=23)
    out = P.dl(x1, x2, w1, b1, w2, b2, wd, bd)
    p1, p2 = _library_conv_pool(x1, w1, b1), _library_conv_pool(x2, w2, b2)
    e1, e2 = p1.mean(axis=(2, 3)), p2.mean(axis=(2, 3))
    logits = np.concatenate([e1, e2], axis=1) @ wd.astype(np.float64) + bd
    for key, want in (("p1", p1), ("p2", p2), ("e1", e1), ("e2", e2), ("logits", logits)):
        np.testing.assert_allclose(out[key], want, rtol=1e-12, atol=1e-13, err_msg=key)
