"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds input generation only, none of the method's arithmetic: it
is the one piece of code that both the CUDA path's callers and the oracle's
callers use.  Every generator draws from numpy's PCG64 with an explicit seed,
so the same call yields the same bytes on any machine.

Recipes (the paper, Section IV-A, runs every benchmark on random data):

* VEC   x, y ~ U[0, 1) float32.
* B&S   spot prices ~ U[10, 100) float32, one vector per option book.
* IMG   image ~ U[0, 1) float32, row-major rows x cols.
* ML    X ~ U{0..15} int32 (row-major rows x feats); naive-Bayes table =
        log class-conditional probabilities centred over classes and rounded
        to multiples of 1/256 (|k| < 1000), log prior likewise; ridge weights
        ~ N(0, 0.05^2) rounded to multiples of 1/256, intercepts likewise.
        Dyadic tables make every score an exact float32 sum.
* DL    two image batches n x 3 x h x w ~ U[0, 1), conv weights 64 x 3 x 3 x 3
        ~ N(0, 0.3^2) and biases ~ N(0, 0.1^2), dense 128 x 10 ~ N(0, 0.1^2) and
        bias ~ N(0, 0.1^2); images and conv weights rounded to bfloat16 (the
        values are returned as float32 numbers that bfloat16 holds exactly,
        with their bfloat16 bit patterns).
* HITS  directed graph with power-law out-degree (Pareto exponent alpha,
        d = floor(u^(-1/(alpha-1))), capped at n-1), rescaled so the total is
        exactly nnz; destinations uniform, no self-loops, no duplicate edges;
        unit float32 weights; CSR of A and CSR of A^T (the CSC of A).
* HITS batch  `count` such graphs, vertex counts log-uniform on [nmin, nmax],
        `degree` edges per vertex on average (the batched HITS benchmark).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def vec_inputs(n: int, seed: int = 0):
    g = rng(seed)
    x = g.random(n, dtype=np.float32)
    y = g.random(n, dtype=np.float32)
    return x, y


def bs_inputs(n: int, count: int = 10, seed: int = 1, lo=10.0, hi=100.0):
    g = rng(seed)
    return [(lo + (hi - lo) * g.random(n, dtype=np.float64)).astype(np.float32)
            for _ in range(count)]


def image(rows: int, cols: int, seed: int = 2):
    g = rng(seed)
    return g.random((rows, cols), dtype=np.float32)


def _dyadic(a: np.ndarray, limit: int = 999) -> np.ndarray:
    k = np.clip(np.rint(a * 256.0), -limit, limit)
    return (k / 256.0).astype(np.float32)


def ml_inputs(rows: int, feats: int = 1024, classes: int = 10, seed: int = 3):
    """X, naive-Bayes table, log prior, ridge weights, ridge intercepts."""
    g = rng(seed)
    X = g.integers(0, 16, size=(rows, feats), dtype=np.int32)
    # class-conditional feature probabilities and their logs
    p = g.dirichlet(np.full(feats, 2.0), size=classes).T  # feats x classes
    logp = np.log(p)
    logp -= logp.mean(axis=1, keepdims=True)
    nb_table = _dyadic(logp)
    prior = g.dirichlet(np.full(classes, 5.0))
    lp = np.log(prior)
    nb_prior = _dyadic(lp - lp.mean())
    ridge_w = _dyadic(g.normal(0.0, 0.05, size=(feats, classes)))
    ridge_b = _dyadic(g.normal(0.0, 0.5, size=classes))
    return X, nb_table, nb_prior, ridge_w, ridge_b


def power_law_graph(n: int, nnz: int, alpha: float = 2.1, seed: int = 4):
    """(rowptr int64 [n+1], col int32 [nnz]) of a directed graph with n
    vertices and exactly nnz distinct edges (no self-loops), rows sorted."""
    assert n >= 2 and nnz <= n * (n - 1)
    g = rng(seed)
    u = 1.0 - g.random(n)  # (0, 1]
    d = np.floor(u ** (-1.0 / (alpha - 1.0)))
    d = np.minimum(d, n - 1)
    # rescale to the exact total, capped at n - 1 per vertex
    d = np.floor(d * (nnz / d.sum())).astype(np.int64)
    d = np.minimum(d, n - 1)
    deficit = nnz - int(d.sum())
    while deficit > 0:
        room = np.flatnonzero(d < n - 1)
        pick = g.choice(room, size=min(deficit, room.size), replace=False)
        d[pick] += 1
        deficit = nnz - int(d.sum())
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(d, out=rowptr[1:])
    rows = np.repeat(np.arange(n, dtype=np.int64), d)
    # destinations uniform over the other n-1 vertices; duplicates redrawn
    cols = g.integers(0, n - 1, size=nnz, dtype=np.int64)
    cols += cols >= rows
    while True:
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        key_s = key[order]
        dup = np.zeros(nnz, dtype=bool)
        dup[order[1:]] = key_s[1:] == key_s[:-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        c = g.integers(0, n - 1, size=nd, dtype=np.int64)
        c += c >= rows[dup]
        cols[dup] = c
    # sort columns inside each row
    order = np.lexsort((cols, rows))
    cols = cols[order].astype(np.int32)
    return rowptr, cols


def transpose_csr(rowptr: np.ndarray, col: np.ndarray, n_cols: int):
    """CSR of A^T from the CSR of A (stable: sources ascending per row)."""
    n = rowptr.size - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    order = np.lexsort((rows, col.astype(np.int64)))
    t_col = rows[order].astype(np.int32)
    counts = np.bincount(col, minlength=n_cols).astype(np.int64)
    t_rowptr = np.zeros(n_cols + 1, dtype=np.int64)
    np.cumsum(counts, out=t_rowptr[1:])
    return t_rowptr, t_col


def hits_graph(n: int, nnz: int, alpha: float = 2.1, seed: int = 4):
    """CSR of A and of A^T, with unit float32 weights."""
    rowptr, col = power_law_graph(n, nnz, alpha, seed)
    t_rowptr, t_col = transpose_csr(rowptr, col, n)
    val = np.ones(nnz, dtype=np.float32)
    return (rowptr, col, val), (t_rowptr, t_col, val.copy())


def hits_batch(count: int = 64, nmin: int = 10_000, nmax: int = 1_000_000, degree: int = 5,
               alpha: float = 2.1, seed: int = 6):
    """`count` independent graphs for a batched HITS: a list of
    (csr, csc) pairs as hits_graph returns them."""
    g = rng(seed)
    sizes = np.exp(g.uniform(np.log(nmin), np.log(nmax), count)).astype(np.int64)
    sizes = np.maximum(sizes, 2)
    return [hits_graph(int(n), int(min(degree * n, n * (n - 1))), alpha, seed * 1000 + i)
            for i, n in enumerate(sizes)]


def to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns, round to nearest even."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def from_bf16_bits(b: np.ndarray) -> np.ndarray:
    return (b.astype(np.uint32) << 16).view(np.float32)


def dl_inputs(n: int = 16, h: int = 256, w: int = 256, cout: int = 64, classes: int = 10, seed: int = 5):
    """(x1, x2, w1, b1, w2, b2, wd, bd) as float32 (x and w exactly bf16)
    plus the bf16 bit patterns of x1, x2, w1, w2."""
    g = rng(seed)
    q = lambda a: from_bf16_bits(to_bf16_bits(a))
    x1 = q(g.random((n, 3, h, w), dtype=np.float32))
    x2 = q(g.random((n, 3, h, w), dtype=np.float32))
    w1 = q(g.normal(0, 0.3, (cout, 3, 3, 3)).astype(np.float32))
    w2 = q(g.normal(0, 0.3, (cout, 3, 3, 3)).astype(np.float32))
    b1 = g.normal(0, 0.1, cout).astype(np.float32)
    b2 = g.normal(0, 0.1, cout).astype(np.float32)
    wd = g.normal(0, 0.1, (2 * cout, classes)).astype(np.float32)
    bd = g.normal(0, 0.1, classes).astype(np.float32)
    return (x1, x2, w1, b1, w2, b2, wd, bd), {k: to_bf16_bits(v) for k, v in
                                              (("x1", x1), ("x2", x2), ("w1", w1), ("w2", w2))}
