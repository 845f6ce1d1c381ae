"""ML nodes and the ML DAG on the GPU through the C ABI, against the oracle.
Scores: with the dyadic tables of the input recipe every product and partial
sum is an exact float32, so scores must be bit-exact; for general tables,
|got - ref| <= 1e-5 * sum |terms|.  Softmax: 1e-5 relative to max(|p|, 1)
on the GPU's own scores.  Labels: bit-exact, except rows whose oracle top-2
margin is below 4e-5 (twice the summed bound of P1 + P2), which may take
either of the two best labels; their count is reported."""
import numpy as np
import pytest

import datagen
from oracle import numeric as N
from oracle import pipelines as P
from paper_2012_09646_gb300 import gdag as G
from paper_2012_09646_gb300.workloads import MlDag

pytestmark = pytest.mark.gpu
TOL = 1e-5
MARGIN = 4e-5


def run(rows, feats, classes, seed, inputs=None, scores_only=False):
    inp = inputs or datagen.ml_inputs(rows, feats=feats, classes=classes, seed=seed)
    ctx = G.Context()
    d = MlDag(ctx, rows, feats, classes)
    d.load(*inp)
    if scores_only:  # the two score nodes alone (softmax works in place)
        ctx.launch("dense_scores", d.XA, d.T1A, d.b1A, d.S1A, rows, feats, classes)
        ctx.launch("dense_scores", d.XA, d.T2A, d.b2A, d.S2A, rows, feats, classes)
    else:
        d.launch_all()
    ctx.sync()
    return ctx, d, inp


# feats a multiple of 64 up to 1024 runs on the tensor cores, the others on
# CUDA cores
# 19457 and 40001 rows split over 152 CTAs leave each a partial last tile
# (127 or 128 rows; 7 past two full tiles), copied in 8-row boxes.  Up to 10
# classes the table takes the 32-column layout (pieces 10 columns apart), from
# 11 to 16 the 48-column one (16 apart)
@pytest.mark.parametrize("rows,feats,classes", [(1, 32, 10), (7, 64, 3), (100, 1024, 10), (1001, 256, 12),
                                                (333, 96, 1), (64, 32, 16), (129, 1024, 16), (300, 640, 1),
                                                (19457, 1024, 10), (40001, 512, 10), (2049, 1024, 11),
                                                (5000, 1024, 9), (700, 192, 15)])
def test_scores_bit_exact_with_dyadic_tables(rows, feats, classes):
    ctx, d, (X, T1, b1, T2, b2) = run(rows, feats, classes, seed=rows, scores_only=True)
    s1 = d.S1[:rows].cpu().numpy()
    s2 = d.S2[:rows].cpu().numpy()
    assert np.array_equal(s1.astype(np.float64), N.scores(X, T1, b1))
    assert np.array_equal(s2.astype(np.float64), N.scores(X, T2, b2))
    ctx.close()


@pytest.mark.parametrize("classes", [10, 11])
def test_scores_general_tables_within_tolerance(classes):
    rows, feats = 513, 1024
    X, *_ = datagen.ml_inputs(rows, feats=feats, classes=classes, seed=7)
    g = np.random.default_rng(0)
    T = g.normal(0, 1, (feats, classes)).astype(np.float32)
    b = g.normal(0, 1, classes).astype(np.float32)
    ctx, d, _ = run(rows, feats, classes, 0, inputs=(X, T, b, T, b), scores_only=True)
    got = d.S1[:rows].cpu().numpy().astype(np.float64)
    ref = N.scores(X, T, b)
    scale = N.scores_abs(X, T, b)
    assert np.all(np.abs(got - ref) <= TOL * np.maximum(scale, 1.0))
    ctx.close()


@pytest.mark.parametrize("classes", [10, 13])
def test_scores_out_of_bf16_range_rows_fall_back_exactly(classes):
    """Feature values beyond +-256 (not exact in bf16) send their tile (at
    most 128 rows) to the CUDA-core path: those rows meet the tolerance, and
    every row further than a tile from such a row stays bit-exact (dyadic
    tables)."""
    rows, feats = 1000, 1024
    X, T1, b1, T2, b2 = datagen.ml_inputs(rows, feats=feats, classes=classes, seed=11)
    X = X.copy()
    X[5, 17] = 1000
    X[300, 3] = -70000
    X[999, 1023] = 257
    X[640, 0] = -2147483648
    ctx, d, _ = run(rows, feats, classes, 0, inputs=(X, T1, b1, T2, b2), scores_only=True)
    got = d.S1[:rows].cpu().numpy().astype(np.float64)
    ref = N.scores(X, T1, b1)
    scale = N.scores_abs(X, T1, b1)
    assert np.all(np.abs(got - ref) <= TOL * np.maximum(scale, 1.0))
    clean = np.ones(rows, bool)
    for r in (5, 300, 999, 640):
        clean[max(0, r - 127):r + 128] = False
    assert np.array_equal(got[clean], ref[clean])
    ctx.close()


def test_scores_full_size_bit_exact():
    """The benchmark's shape, 100000 x 1024 x 10 (782 tiles over the
    persistent grid, a 32-row last tile): every score bit-exact."""
    rows = 100_000
    ctx, d, (X, T1, b1, T2, b2) = run(rows, 1024, 10, seed=5, scores_only=True)
    assert np.array_equal(d.S1[:rows].cpu().numpy().astype(np.float64), N.scores(X, T1, b1))
    assert np.array_equal(d.S2[:rows].cpu().numpy().astype(np.float64), N.scores(X, T2, b2))
    ctx.close()


@pytest.mark.parametrize("rows", [1, 37, 4097])
def test_softmax_and_labels(rows):
    ctx, d, inp = run(rows, 1024, 10, seed=rows + 1)
    ref = P.ml(*inp)
    p1 = d.S1[:rows].cpu().numpy().astype(np.float64)
    p2 = d.S2[:rows].cpu().numpy().astype(np.float64)
    # softmax of the (exact) scores
    assert np.all(np.abs(p1 - ref["p1"]) <= TOL * np.maximum(np.abs(ref["p1"]), 1.0))
    assert np.all(np.abs(p2 - ref["p2"]) <= TOL * np.maximum(np.abs(ref["p2"]), 1.0))
    np.testing.assert_allclose(p1.sum(axis=1), 1.0, rtol=1e-5)
    labels = d.labels[:rows].cpu().numpy()
    close = ref["margin"] < MARGIN
    assert np.array_equal(labels[~close], ref["labels"][~close])
    top2 = np.argsort(-(ref["p1"] + ref["p2"]), axis=1, kind="stable")[:, :2]
    assert all(labels[i] in top2[i] for i in np.flatnonzero(close))


def test_argmax_ties_lowest_index():
    rows, classes = 3, 4
    with G.Context() as ctx:
        import torch
        p1 = torch.tensor([[0.25, 0.25, 0.5, 0.0], [0.0, 0.0, 0.0, 0.0], [0.1, 0.6, 0.3, 0.0]], device="cuda")
        p2 = torch.tensor([[0.25, 0.25, 0.0, 0.5], [0.0, 0.0, 0.0, 0.0], [0.6, 0.1, 0.3, 0.0]], device="cuda")
        lab = torch.full((rows,), -1, dtype=torch.int32, device="cuda")
        ctx.launch("argmax_combine", ctx.array(p1), ctx.array(p2), ctx.array(lab), rows, classes)
        ctx.sync()
        assert lab.cpu().tolist() == [0, 0, 0]


def test_ml_dag_full_size_host_labels():
    """The benchmark's shape: 100000 x 1024, 10 classes; the host reads the
    labels through the library; every row checked."""
    rows = 100_000
    inp = datagen.ml_inputs(rows, feats=1024, classes=10, seed=3)
    ref = P.ml(*inp)
    with G.Context() as ctx:
        d = MlDag(ctx, rows)
        d.load(*inp)
        d.step()
        labels = d.h_labels[:rows].numpy()
        close = ref["margin"] < MARGIN
        assert np.array_equal(labels[~close], ref["labels"][~close])
        print("near-tie rows:", int(close.sum()))
        st = ctx.stats()
        assert st["streams"] >= 2  # the two score branches ran on two streams
