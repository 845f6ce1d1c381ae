"""Seeded input generators: determinism and the structure each recipe fixes."""
import numpy as np
import scipy.sparse

import datagen


def test_seeded_and_ranges():
    x1, y1 = datagen.vec_inputs(1000, seed=0)
    x2, _ = datagen.vec_inputs(1000, seed=0)
    assert np.array_equal(x1, x2) and x1.dtype == np.float32
    assert 0 <= x1.min() and x1.max() < 1 and not np.array_equal(x1, y1)
    S = datagen.bs_inputs(1000, count=3)
    assert len(S) == 3 and all(10 <= s.min() and s.max() < 100 for s in S)


def test_ml_tables_are_dyadic():
    X, T, p, W, b = datagen.ml_inputs(10, feats=64)
    assert X.dtype == np.int32 and X.min() >= 0 and X.max() <= 15
    for t in (T, p, W, b):
        k = t.astype(np.float64) * 256
        assert np.array_equal(k, np.rint(k)) and np.abs(k).max() < 1000


def test_power_law_graph_structure():
    n, nnz = 2000, 15000
    (rp, col, val), (trp, tcol, tval) = datagen.hits_graph(n, nnz, seed=4)
    assert rp[-1] == nnz and col.size == nnz and val.dtype == np.float32
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert not np.any(rows == col)
    key = rows.astype(np.int64) * n + col
    assert np.unique(key).size == nnz
    assert np.all(np.diff(key) > 0)  # sorted rows, sorted columns
    A = scipy.sparse.csr_matrix((val, col, rp), shape=(n, n))
    At = scipy.sparse.csr_matrix((tval, tcol, trp), shape=(n, n))
    assert (A.T != At).nnz == 0
    deg = np.diff(rp)
    assert deg.max() > 20 * deg.mean()  # heavy tail


def test_out_degree_tail_follows_the_stated_exponent():
    """Pareto out-degrees with alpha = 2.1 have a complementary distribution
    falling as k^-(alpha-1): the Hill estimate over the 1000 largest degrees
    recovers alpha - 1 = 1.1 (standard error about 0.035) after the rescaling
    to the exact edge count, which leaves the tail's exponent unchanged."""
    for seed in (4, 5):
        (rp, _col, _val), _ = datagen.hits_graph(200_000, 1_000_000, seed=seed)
        deg = np.sort(np.diff(rp))[::-1].astype(np.float64)
        k = 1000
        hill = 1.0 / np.mean(np.log(deg[:k] / deg[k]))
        assert 0.98 <= hill <= 1.22, (seed, hill)


def test_batch_recipe():
    """Batched HITS: vertex counts log-uniform within the stated range and
    `degree` edges per vertex in every graph."""
    graphs = datagen.hits_batch(count=12, nmin=100, nmax=5000, degree=5, seed=6)
    sizes = [len(csr[0]) - 1 for csr, _ in graphs]
    assert all(100 <= n <= 5000 for n in sizes)
    assert len(set(sizes)) == len(sizes)
    for (rp, col, _), _ in graphs:
        assert rp[-1] == 5 * (len(rp) - 1) == col.size
