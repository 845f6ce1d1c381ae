"""Automatic capture of repeated issue sequences (options.auto_graph) on the
GPU, through the C ABI: a DAG step issued again and again is captured once
and replayed, and every step's results must still match the oracle, with new
host inputs each step (a replayed host write copies what the host view holds
when it runs) and bit for bit what the dynamic path computes."""
import numpy as np
import pytest
import torch

import datagen
from oracle import numeric as N
from oracle import pipelines as P
from paper_2012_09646_gb300 import gdag as G
from paper_2012_09646_gb300.workloads import BsDag, ImgDag, VecDag

pytestmark = pytest.mark.gpu
TOL = 1e-5


def nodes_issued(ctx):
    return G.gdag_stats_get(ctx.h).nodes


@pytest.mark.parametrize("threshold", [1, 2, 3])
def test_vec_steps_replayed_with_new_inputs(threshold):
    n = 1_000_000
    with G.Context(auto_graph=threshold) as ctx, G.Context() as dyn:
        v, w = VecDag(ctx, n), VecDag(dyn, n)
        per_step = []
        for step in range(6):
            x, y = datagen.vec_inputs(n, seed=100 + step)
            v.load(x, y)
            w.load(x, y)
            before = nodes_issued(ctx)
            z = v.step()
            per_step.append(nodes_issued(ctx) - before)
            assert z == w.step()  # the same kernels on the same data: the same bits
            want, scale = float(N.sum_diff(x * x, y * y)), float(N.sum_abs_diff(x * x, y * y))
            assert abs(z - want) <= TOL * max(scale, 1.0), (step, z, want)
        # dynamic steps make 6 elements (2 writes, 3 kernels, the read); the
        # capturing step 5 recorded + 1 replay + the read; replays 2
        assert per_step[:threshold - 1] == [6] * (threshold - 1)
        assert per_step[threshold - 1] == 7
        assert per_step[threshold:] == [2] * (6 - threshold)


def test_img_steps_replayed_equal_dynamic_and_oracle():
    rows, cols = 1024, 1024
    with G.Context(auto_graph=2) as ctx, G.Context() as dyn:
        a, b = ImgDag(ctx, rows, cols), ImgDag(dyn, rows, cols)
        for step in range(4):
            img = datagen.image(rows, cols, seed=20 + step)
            a.load(img)
            b.load(img)
            a.step()
            b.step()
            got = a.h_out.numpy().reshape(rows, cols)
            assert np.array_equal(got, b.h_out.numpy().reshape(rows, cols)), step
            ref = P.img(img)["out"]
            err = np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)
            assert err.max() <= TOL, (step, err.max())


def test_bs_resident_kernels_replayed():
    """Ten independent B&S nodes (kernels only, inputs rewritten on the
    device between steps): the replayed graph prices the new inputs."""
    n = 300_001
    with G.Context(auto_graph=2) as ctx:
        d = BsDag(ctx, n, count=10, host=False)
        for step in range(4):
            prices = datagen.bs_inputs(n, count=10, seed=50 + step)
            ctx.sync()
            d.load_device(prices)
            d.step_resident()
            ctx.sync()
            for i in (0, 9):
                got = d.C[i][:n].cpu().numpy().astype(np.float64)
                ref = N.bs_call(prices[i])
                assert (np.abs(got - ref) <= TOL * np.maximum(np.abs(ref), 1.0)).all(), (step, i)


def test_replay_follows_a_moved_array():
    """An array registered again at another address drops the graph: the
    next steps are issued dynamically and captured anew, and compute on the
    new memory."""
    n = 4097
    with G.Context(auto_graph=2) as ctx:
        v = VecDag(ctx, n)
        x, y = datagen.vec_inputs(n, seed=7)
        v.load(x, y)
        z0 = v.step()
        assert v.step() == z0 and v.step() == z0  # captured, replayed
        ctx.sync()
        ctx.unregister(v.Y)
        y2 = torch.zeros(n, dtype=torch.float32, device="cuda")
        v.y = y2
        v.Y = ctx.array(y2, host=v.hy, name="y")
        for _ in range(3):
            assert v.step() == z0  # the host view still holds y
        ctx.sync()
        assert torch.equal(y2.cpu(), torch.from_numpy(y * y))


def test_ml_hits_dl_replayed_equal_dynamic_and_oracle():
    """The other DAGs of the suite with automatic graphs: ML (two score
    nodes, softmaxes, labels), HITS (two alternating iteration sequences,
    each captured at its second issue) and DL (two tensor-core branches):
    every output bit-identical to the dynamic path's, and within tolerance
    of the oracle."""
    from paper_2012_09646_gb300.workloads import DlDag, HitsDag, MlDag
    rows = 4097
    ml_in = datagen.ml_inputs(rows, feats=1024, classes=10, seed=21)
    csr, csc = datagen.hits_graph(20000, 150000, seed=22)
    dl_in, _bits = datagen.dl_inputs(n=2, h=34, w=192, seed=23)
    outs = {}
    for auto in (0, 2):
        with G.Context(auto_graph=auto) as ctx:
            m = MlDag(ctx, rows)
            m.load(*ml_in)
            for _ in range(4):
                m.step()
            ctx.sync()
            h = HitsDag(ctx, csr, csc)
            ka, kh = h.run(iters=5)
            d = DlDag(ctx, 2, 34, 192)
            d.load(*dl_in)
            for _ in range(3):
                d.step()
            ctx.sync()
            assert d.status.tolist() == [0, 0]
            outs[auto] = [m.S1.clone(), m.S2.clone(), m.labels.clone(), h.vec[ka].clone(), h.vec[kh].clone(),
                          d.p1.clone(), d.p2.clone(), d.logits.clone()]
    for a, b in zip(outs[0], outs[2]):
        assert torch.equal(a, b)
    ref = P.ml(*ml_in)
    # the score arrays hold the row softmaxes after a step (in place)
    p1 = outs[2][0][:rows].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(p1 - ref["p1"]) <= TOL * np.maximum(np.abs(ref["p1"]), 1.0))
    hits = P.hits(csr, csc, iters=5)
    for got, want in ((outs[2][3], hits["a"][-1]), (outs[2][4], hits["h"][-1])):
        got = got[:20000].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - want) <= TOL * np.maximum(np.abs(want), 1.0))
