"""Batched HITS layout on the CPU: the block-diagonal concatenation of the
graphs against scipy's block_diag, and the batch generator."""
import numpy as np
import scipy.sparse as sp

import datagen
from paper_2012_09646_gb300.workloads import block_diag_csr


def as_scipy(rp, col, val, n):
    return sp.csr_matrix((val, col, rp), shape=(n, n))


def test_block_diag_matches_scipy():
    graphs = datagen.hits_batch(count=7, nmin=2, nmax=400, seed=3)
    # an edgeless graph inside the batch
    graphs.insert(3, ((np.zeros(9, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32)),
                      (np.zeros(9, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))))
    for side in (0, 1):
        mats = [g[side] for g in graphs]
        (rp, col, val), seg = block_diag_csr(mats)
        n = int(seg[-1])
        ref = sp.block_diag([as_scipy(m[0], m[1], m[2], len(m[0]) - 1) for m in mats], format="csr")
        got = as_scipy(rp, col, val, n)
        assert (got != ref).nnz == 0
        assert list(np.diff(seg)) == [len(m[0]) - 1 for m in mats]
        assert np.all(np.diff(rp) >= 0) and rp[-1] == col.size


def test_batch_generator():
    a = datagen.hits_batch(count=6, nmin=100, nmax=5000, degree=4, seed=2)
    b = datagen.hits_batch(count=6, nmin=100, nmax=5000, degree=4, seed=2)
    assert len(a) == 6
    for (csr, csc), (csr2, _) in zip(a, b):
        n = len(csr[0]) - 1
        assert 100 <= n <= 5000
        assert int(csr[0][-1]) == 4 * n == int(csc[0][-1])
        assert np.array_equal(csr[1], csr2[1])
        # csc is the transpose of csr
        A = as_scipy(csr[0], csr[1], csr[2], n)
        AT = as_scipy(csc[0], csc[1], csc[2], n)
        assert (A.T.tocsr() != AT).nnz == 0
