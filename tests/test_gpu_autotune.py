"""Autotuner on the GPU: the tuned launch shape gives the same results as
the default one, the history picks up traced nodes, and the stream-pool and
fusion-threshold searches return measured candidates."""
import numpy as np
import pytest
import torch

import datagen
from paper_2012_09646_gb300 import autotune as AT
from paper_2012_09646_gb300 import gdag as G
from paper_2012_09646_gb300.workloads import BsDag

pytestmark = pytest.mark.gpu


def test_tuned_bs_launch_same_results():
    n = 2_000_003
    p = datagen.bs_inputs(n, count=1, seed=3)[0]
    with G.Context() as ctx:
        S = torch.from_numpy(p).cuda()
        C1 = torch.zeros(n, device="cuda")
        C2 = torch.zeros(n, device="cuda")
        SA, CA1, CA2 = ctx.array(S), ctx.array(C1), ctx.array(C2)
        grid, block, ms = AT.tune_launch(ctx, "bs_call", (SA, CA1, n, 60.0, 0.1, 0.2, 1.0), blocks=(128, 256, 512),
                                         waves=(1, 4))
        assert ms > 0
        ctx.launch("bs_call", SA, CA2, n, 60.0, 0.1, 0.2, 1.0, grid=grid, block=block)
        ctx.launch("bs_call", SA, CA1, n, 60.0, 0.1, 0.2, 1.0)
        ctx.sync()
        assert torch.equal(C1, C2)
        # cached
        assert AT.tune_launch(ctx, "bs_call", (SA, CA1, n, 60.0, 0.1, 0.2, 1.0)) == (grid, block, ms)


def test_history_and_stream_tuning():
    n = 1_000_000
    prices = datagen.bs_inputs(n, count=4, seed=4)
    with G.Context(trace=True) as ctx:
        d = BsDag(ctx, n, count=4, host=False)
        d.load_device(prices)
        first = G.gdag_stats_get(ctx.h).nodes
        d.step_resident()
        ctx.sync()
        h = AT.History()
        h.add_trace(ctx, {first + i: ("bs_call", n) for i in range(4)})
        assert len(h.samples[("bs_call", n)]) == 4 and h.median(("bs_call", n)) > 0
        assert h.best("bs_call") == ("bs_call", n)

    def build(ctx):
        d = BsDag(ctx, n, count=4, host=False)
        d.load_device(prices)
        return d
    best, times = AT.tune_streams(build, lambda d: d.step_resident(), candidates=(1, 4), steps=3)
    assert best in (1, 4) and set(times) == {1, 4}


def test_fusion_threshold_search():
    keep = []

    def member(ctx, n, i):
        S = torch.rand(n, device="cuda") * 90 + 10
        C = torch.empty(n, device="cuda")
        keep.append((S, C))
        return (ctx.array(S), ctx.array(C), n, 60.0, 0.1, 0.2, 1.0)
    sizes = (1 << 12, 1 << 16, 1 << 20)
    thr, times = AT.tune_fusion("bs_call", member, sizes, group=6, reps=3)
    assert set(times) == set(sizes) and all(a > 0 and b > 0 for a, b in times.values())
    assert thr in (0,) + sizes
    assert all(times[n][1] <= times[n][0] for n in sizes if n == thr)
