"""Batched HITS on the GPU through the C ABI: the per-segment norm and
scale kernels against the oracle's l2norm and scale on each segment, and a
batch of graphs run as one program (block-diagonal SpMV + segment kernels)
against the oracle's HITS on every graph separately.  Tolerances as for the
single-graph HITS: norms 1e-5 relative (a sum of positive terms), scaled
values 1e-5 * max(|ref|, 1), iterates with the per-step bound accumulated."""
import numpy as np
import pytest
import torch

import datagen
from oracle import numeric as N
from oracle import pipelines as P
from paper_2012_09646_gb300 import gdag as G
from paper_2012_09646_gb300.workloads import HitsBatchDag

pytestmark = pytest.mark.gpu
TOL = 1e-5


# segment lengths: odd sizes and unaligned bounds; segments spanning many
# 4096-element chunks; bounds on chunk boundaries; empty segments inside,
# on a chunk boundary and at the end
SEGMENT_CASES = [
    [0, 1, 5, 255, 256, 257, 1000, 0, 40000, 3, 123457],
    [4096, 4096, 8192, 0, 1, 4095, 0, 12288, 0],
    [0, 0, 0],
    [3, 70001, 2, 1],
]


@pytest.mark.parametrize("lens", SEGMENT_CASES)
def test_segment_kernels(lens):
    g = np.random.default_rng(11)
    seg = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    n = int(seg[-1])
    x = g.standard_normal(max(n, 1)).astype(np.float32)[:n]
    if len(lens) > 4:
        x[seg[3]:seg[4]] = 0.0  # a segment of zeros: norm 0, left unscaled
    G_ = len(lens)
    with G.Context() as ctx:
        xt = torch.as_tensor(x if n else np.zeros(4, np.float32)).cuda()
        st = torch.as_tensor(seg).cuda()
        norms = torch.full((G_,), float("nan"), device="cuda")
        scratch = torch.zeros(G.gdag_scratch_bytes("seg_l2norm", G_), dtype=torch.uint8, device="cuda")
        X, S, NR, SC = ctx.array(xt), ctx.array(st), ctx.array(norms), ctx.array(scratch)
        for _ in range(2):  # the arrival counters are left at zero: a second launch works too
            ctx.launch("seg_l2norm", X, S, NR, SC, G_, n)
        ctx.sync()
        got_n = norms.cpu().numpy().astype(np.float64)
        ctx.launch("seg_scale", X, S, NR, G_, n)
        ctx.sync()
        got_x = xt.cpu().numpy().astype(np.float64)[:n]
    for k in range(G_):
        part = x[seg[k]:seg[k + 1]]
        want = N.l2norm(part) if part.size else 0.0
        assert abs(got_n[k] - want) <= TOL * want + 1e-30, (k, got_n[k], want)
        want_x = N.scale(part, got_n[k]) if part.size else part
        assert np.all(np.abs(got_x[seg[k]:seg[k + 1]] - want_x) <= TOL * np.maximum(np.abs(want_x), 1.0))
    # the per-segment arrival counters (after the G x 32 slice partials) are zero again
    off = G_ * 32 * 8
    assert np.all(scratch.cpu().numpy()[off:off + 4 * G_] == 0)


def batch_cases():
    graphs = datagen.hits_batch(count=12, nmin=2, nmax=3000, seed=4)
    empty = (np.zeros(17, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    graphs.insert(5, (empty, empty))  # no edges: its vectors go to 0 and stay unscaled
    return graphs


@pytest.mark.parametrize("iters", [1, 5])
def test_batched_hits_matches_each_graph(iters):
    graphs = batch_cases()
    with G.Context() as ctx:
        d = HitsBatchDag(ctx, graphs)
        ka, kh = d.run(iters=iters)
        ctx.sync()
        a = d.vec[ka][:d.n].cpu().numpy().astype(np.float64)
        h = d.vec[kh][:d.n].cpu().numpy().astype(np.float64)
    for gi, (csr, csc) in enumerate(graphs):
        ref = P.hits(csr, csc, iters=iters)
        for got, want in ((d.segment(a, gi), ref["a"][-1]), (d.segment(h, gi), ref["h"][-1])):
            assert got.shape == want.shape
            assert np.all(np.abs(got - want) <= TOL * np.maximum(np.abs(want), 1.0)), gi
            nz = want > 0
            assert np.all(np.abs(got[nz] - want[nz]) <= iters * 2 * TOL * want[nz]), gi


@pytest.mark.slow
def test_batched_hits_benchmark_batch_sampled():
    """The benchmark batch (64 graphs, 1e4..1e6 vertices): five iterations,
    with the oracle run on every fourth graph."""
    graphs = datagen.hits_batch(count=64, seed=6)
    with G.Context() as ctx:
        d = HitsBatchDag(ctx, graphs)
        ka, kh = d.run(iters=5)
        ctx.sync()
        a = d.vec[ka][:d.n].cpu().numpy().astype(np.float64)
        h = d.vec[kh][:d.n].cpu().numpy().astype(np.float64)
    for gi in range(0, 64, 4):
        csr, csc = graphs[gi]
        ref = P.hits(csr, csc, iters=5)
        for got, want in ((d.segment(a, gi), ref["a"][-1]), (d.segment(h, gi), ref["h"][-1])):
            assert np.all(np.abs(got - want) <= TOL * np.maximum(np.abs(want), 1.0)), gi


def test_scale_kernels_round_correctly():
    """scale and seg_scale divide with Markstein's correction from RN(1/d):
    every result must equal the correctly rounded fp32 quotient, which numpy
    gives exactly as RN32(RN64(x / d)) (53 >= 2 * 24 + 2)."""
    g = np.random.default_rng(21)
    n = 1 << 20
    mant = g.uniform(1.0, 2.0, n)
    expo = g.integers(-60, 60, n)
    x = (mant * np.exp2(expo)).astype(np.float32)
    x[::7] *= -1.0
    norms = np.array([3.0, 0.1, 7.123456e-3, 1234.5678, 1.0], dtype=np.float32)
    G_ = norms.size
    seg = np.linspace(0, n, G_ + 1).astype(np.int32)
    want = np.empty(n, np.float32)
    for k in range(G_):
        want[seg[k]:seg[k + 1]] = (x[seg[k]:seg[k + 1]].astype(np.float64) / np.float64(norms[k])).astype(np.float32)
    with G.Context() as ctx:
        xt = torch.as_tensor(x).cuda()
        X, S, NR = ctx.array(xt), ctx.array(torch.as_tensor(seg).cuda()), ctx.array(torch.as_tensor(norms).cuda())
        ctx.launch("seg_scale", X, S, NR, G_, n)
        ctx.sync()
        got = xt.cpu().numpy()
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), int((got != want).sum())
        # the single-vector kernel, one norm
        xt2 = torch.as_tensor(x).cuda()
        nt = torch.as_tensor(norms[3:4]).cuda()
        ctx.launch("scale", ctx.array(xt2), ctx.array(nt), n)
        ctx.sync()
        want2 = (x.astype(np.float64) / np.float64(norms[3])).astype(np.float32)
        got2 = xt2.cpu().numpy()
        assert np.array_equal(got2.view(np.uint32), want2.view(np.uint32)), int((got2 != want2).sum())
