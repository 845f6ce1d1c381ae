"""The autotuner's per-kernel history (Section III-A keeps an execution
history per kernel): a bounded ring per (kernel, launch shape), medians, the
best shape, and samples taken from a traced context.  CPU only (the fake
backend's trace times every node as zero)."""
from paper_2012_09646_gb300 import autotune as AT
from paper_2012_09646_gb300 import gdag as G


def test_history_is_a_bounded_ring():
    h = AT.History(keep=3)
    for ms in (9.0, 8.0, 1.0, 2.0, 3.0):
        h.add(("k", 256), ms)
    assert list(h.samples[("k", 256)]) == [1.0, 2.0, 3.0]
    assert h.median(("k", 256)) == 2.0
    assert h.median(("k", 512)) is None


def test_best_shape_by_median():
    h = AT.History()
    for ms in (5.0, 1.0, 6.0):      # median 5
        h.add(("k", 128), ms)
    for ms in (3.0, 3.5, 40.0):     # median 3.5, despite one outlier
        h.add(("k", 256), ms)
    h.add(("other", 64), 0.1)
    assert h.best("k") == ("k", 256)
    assert h.best("none") is None


def test_samples_from_a_traced_context():
    ctx = G.Context(backend="fake", trace=True)
    a = ctx.array(dev=0x10000, nbytes=4096)
    b = ctx.array(dev=0x20000, nbytes=4096)
    n1 = ctx.launch("vec_square", a, 1024)
    n2 = ctx.launch("vec_square", b, 1024)
    ctx.launch("vec_square", a, 512)
    h = AT.History()
    h.add_trace(ctx, {n1: ("vec_square", 1024), n2: ("vec_square", 1024)})
    assert list(h.samples) == [("vec_square", 1024)]
    assert list(h.samples[("vec_square", 1024)]) == [0.0, 0.0]
    ctx.close()
