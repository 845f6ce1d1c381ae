"""Captured DAG shapes replayed as CUDA graphs through the C ABI: the same
results as dynamic scheduling and as the oracle."""
import numpy as np
import pytest
import torch

import datagen
from oracle import pipelines as P
from paper_2012_09646_gb300 import gdag as G
from paper_2012_09646_gb300.workloads import HitsDag, ImgDag, VecDag

pytestmark = pytest.mark.gpu


def test_vec_replay_with_new_inputs_each_time():
    n = 100_003
    with G.Context() as ctx:
        v = VecDag(ctx, n)
        g = ctx.capture(lambda: v.step(read=False))  # host writes copy the views
        for it in range(5):
            x, y = datagen.vec_inputs(n, seed=50 + it)
            v.load(x, y)
            ctx.replay(g)
            ctx.read(v.Z)  # a dynamic read after the replay element
            ref = P.vec(x, y)
            assert abs(float(v.hz[0]) - ref["z"]) <= 1e-5 * ref["z_scale"]
        ctx.drop_graph(g)


def test_img_replay_matches_dynamic():
    rows, cols = 300, 517
    img = torch.from_numpy(datagen.image(rows, cols, seed=8).reshape(-1)).cuda()
    with G.Context() as ctx:
        a = ImgDag(ctx, rows, cols)
        a.img.copy_(img)
        a.launch_all()
        ctx.sync()
        want = a.out.clone()
        b = ImgDag(ctx, rows, cols)
        b.img.copy_(img)
        g = ctx.capture(b.launch_all)
        for _ in range(3):
            ctx.replay(g)
        ctx.sync()
        assert torch.equal(b.out, want)


def test_hits_replay_of_two_iterations():
    n, nnz = 20000, 150000
    csr, csc = datagen.hits_graph(n, nnz, seed=2)
    ref = P.hits(csr, csc, iters=4)
    with G.Context() as ctx:
        d = HitsDag(ctx, csr, csc)
        d.run(iters=0, read=False)
        def two():
            d.iterate("a", "h", "a2", "h2")
            d.iterate("a2", "h2", "a", "h")
        g = ctx.capture(two)
        ctx.replay(g)
        ctx.replay(g)
        ctx.sync()
        a = d.vec["a"][:n].cpu().numpy().astype(np.float64)
        h = d.vec["h"][:n].cpu().numpy().astype(np.float64)
    for got, want in ((a, ref["a"][-1]), (h, ref["h"][-1])):
        assert np.all(np.abs(got - want) <= 1e-5 * np.maximum(np.abs(want), 1.0))
