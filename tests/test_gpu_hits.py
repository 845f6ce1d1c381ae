"""HITS nodes and the HITS DAG on the GPU through the C ABI, against the
oracle.  SpMV outputs: |got - ref| <= 1e-5 * sum_k |val_k x_col_k| per row
(the reduction reading); with unit weights and x = 1 the sums are integers
below 2^24 and must be bit-exact.  Norm: 1e-5 relative; scale: 1e-5 *
max(|ref|, 1)."""
import numpy as np
import pytest
import torch

import datagen
from oracle import numeric as N
from oracle import pipelines as P
from paper_2012_09646_gb300 import gdag as G
from paper_2012_09646_gb300.workloads import HitsDag

pytestmark = pytest.mark.gpu
TOL = 1e-5


def spmv_gpu(ctx, rowptr, col, val, x):
    n = len(rowptr) - 1
    nnz = int(rowptr[-1])
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()
    rp, cl, vl, xv = t(rowptr, torch.int32), t(col, torch.int32), t(val, torch.float32), t(x, torch.float32)
    y = torch.full((max(n, 1),), float("nan"), device="cuda")
    part = torch.zeros(G.gdag_scratch_bytes("spmv_partition", n + nnz), dtype=torch.uint8, device="cuda")
    carry = torch.zeros(G.gdag_scratch_bytes("spmv_csr", n + nnz), dtype=torch.uint8, device="cuda")
    if cl.numel() == 0:
        cl, vl = torch.zeros(1, dtype=torch.int32, device="cuda"), torch.zeros(1, device="cuda")
    A = ctx.array
    RP, PA = A(rp), A(part)
    ctx.launch("spmv_partition", RP, PA, n, nnz)
    ctx.launch("spmv_csr", RP, A(cl), A(vl), A(xv), PA, A(y), A(carry), n, nnz)
    ctx.sync()
    return y[:n].cpu().numpy().astype(np.float64)


def graph_cases():
    g = np.random.default_rng(5)
    cases = []
    # power-law graphs of several sizes
    for n, nnz, seed in [(2, 1, 1), (50, 300, 2), (1000, 20000, 3), (30000, 250000, 4)]:
        rp, col = datagen.power_law_graph(n, nnz, seed=seed)
        cases.append(("powerlaw_%d" % n, rp, col))
    # one huge row spanning many tiles, empty rows around it
    n = 5000
    deg = np.zeros(n, np.int64)
    deg[1] = 4999
    deg[4000] = 3
    rp = np.concatenate([[0], np.cumsum(deg)])
    col = np.concatenate([np.delete(np.arange(n), 1), [0, 1, 2]]).astype(np.int32)
    cases.append(("huge_row", rp, col))
    # no edges at all, and a single vertex
    cases.append(("empty", np.zeros(101, np.int64), np.zeros(0, np.int32)))
    cases.append(("one_vertex", np.array([0, 0], np.int64), np.zeros(0, np.int32)))
    # rows of every length 0..40 in order
    deg = np.arange(41)
    rp = np.concatenate([[0], np.cumsum(deg)])
    col = g.integers(0, 41, size=int(rp[-1])).astype(np.int32)
    cases.append(("ramp", rp, col))
    return cases


@pytest.mark.parametrize("name,rowptr,col", graph_cases(), ids=[c[0] for c in graph_cases()])
def test_spmv_matches_oracle(name, rowptr, col):
    n = len(rowptr) - 1
    g = np.random.default_rng(len(col))
    val = g.normal(0, 1, len(col)).astype(np.float32)
    x = g.normal(0, 1, n).astype(np.float32)
    with G.Context() as ctx:
        y = spmv_gpu(ctx, rowptr, col, val, x)
        ref = N.spmv_csr(rowptr, col, val, x)
        scale = N.spmv_csr_abs(rowptr, col, val, x)
        assert np.all(np.abs(y - ref) <= TOL * np.maximum(scale, 1e-30)), name
        # unit weights, x = 1: the row lengths, bit-exact
        ones = spmv_gpu(ctx, rowptr, col, np.ones(len(col), np.float32), np.ones(n, np.float32))
        assert np.array_equal(ones, np.diff(rowptr).astype(np.float64)), name
        # deterministic: a second launch gives the same bits
        assert np.array_equal(spmv_gpu(ctx, rowptr, col, val, x), y)


def test_l2norm_and_scale():
    with G.Context() as ctx:
        for n in [1, 5, 4097, 1_000_001]:
            x = np.random.default_rng(n).normal(0, 1, n).astype(np.float32)
            xt = torch.from_numpy(x).cuda()
            nr = torch.zeros(1, device="cuda")
            sc = torch.zeros(G.gdag_scratch_bytes("l2norm", n), dtype=torch.uint8, device="cuda")
            X, NR = ctx.array(xt), ctx.array(nr)
            ctx.launch("l2norm", X, NR, ctx.array(sc), n)
            ctx.launch("scale", X, NR, n)
            ctx.sync()
            want = N.l2norm(x)
            assert abs(float(nr.item()) - want) <= TOL * want
            got = xt.cpu().numpy().astype(np.float64)
            ref = N.scale(x, float(nr.item()))
            assert np.all(np.abs(got - ref) <= TOL * np.maximum(np.abs(ref), 1.0))
        # a zero vector keeps its values (zero norm)
        z = torch.zeros(100, device="cuda")
        nr = torch.zeros(1, device="cuda")
        sc = torch.zeros(G.gdag_scratch_bytes("l2norm", 100), dtype=torch.uint8, device="cuda")
        Z, NR = ctx.array(z), ctx.array(nr)
        ctx.launch("l2norm", Z, NR, ctx.array(sc), 100)
        ctx.launch("scale", Z, NR, 100)
        ctx.sync()
        assert float(nr.item()) == 0.0 and torch.count_nonzero(z).item() == 0


@pytest.mark.parametrize("n,nnz,iters", [(500, 4000, 1), (20000, 150000, 5), (100_000, 500_000, 5)])
@pytest.mark.parametrize("policy", [G.GDAG_POLICY_PARALLEL, G.GDAG_POLICY_SERIAL_SYNC])
def test_hits_dag(n, nnz, iters, policy):
    csr, csc = datagen.hits_graph(n, nnz, seed=n)
    ref = P.hits(csr, csc, iters=iters)
    with G.Context(policy=policy) as ctx:
        d = HitsDag(ctx, csr, csc)
        ka, kh = d.run(iters=iters)
        ctx.sync()
        a = d.vec[ka][:n].cpu().numpy().astype(np.float64)
        h = d.vec[kh][:n].cpu().numpy().astype(np.float64)
    for got, want in ((a, ref["a"][-1]), (h, ref["h"][-1])):
        assert np.all(np.abs(got - want) <= TOL * np.maximum(np.abs(want), 1.0))
        # positive vectors: also relative to each entry, with the per-step
        # bound accumulated over the iterations
        nz = want > 0
        assert np.all(np.abs(got[nz] - want[nz]) <= iters * 2 * TOL * want[nz])


def test_hits_stepwise_from_gpu_iterates():
    """Each iteration checked against the oracle applied to the GPU's own
    previous iterate: the per-node error alone."""
    n, nnz = 30000, 200000
    csr, csc = datagen.hits_graph(n, nnz, seed=9)
    with G.Context() as ctx:
        d = HitsDag(ctx, csr, csc)
        d.run(iters=0, read=False)
        cur, nxt = ("a", "h"), ("a2", "h2")
        for _ in range(3):
            a0 = d.vec[cur[0]][:n].cpu().numpy()
            h0 = d.vec[cur[1]][:n].cpu().numpy()
            d.iterate(cur[0], cur[1], nxt[0], nxt[1])
            ctx.sync()
            a_raw = N.spmv_csr(csc[0], csc[1], csc[2], h0)
            h_raw = N.spmv_csr(csr[0], csr[1], csr[2], a0)
            na, nh = N.l2norm(a_raw), N.l2norm(h_raw)
            assert abs(float(d.norms[0].item()) - na) <= 2 * TOL * na
            assert abs(float(d.norms[1].item()) - nh) <= 2 * TOL * nh
            for k, raw, nr in ((nxt[0], a_raw, na), (nxt[1], h_raw, nh)):
                got = d.vec[k][:n].cpu().numpy().astype(np.float64)
                want = raw / nr
                assert np.all(np.abs(got - want) <= 2 * TOL * np.maximum(want, 1e-30))
            cur, nxt = nxt, cur


@pytest.mark.slow
def test_hits_full_size_properties():
    """1e7 vertices, 5e7 edges, power-law out-degree: the benchmark's graph
    and launch shape.  The unnormalised first iterates are the in- and
    out-degrees (exact integers); rows sampled from the second iterate are
    checked against the oracle's sums over the GPU's first iterate."""
    n, nnz = 10_000_000, 50_000_000
    csr, csc = datagen.hits_graph(n, nnz, seed=4)
    with G.Context() as ctx:
        d = HitsDag(ctx, csr, csc)
        d.run(iters=0, read=False)
        c = ctx
        c.launch("spmv_csr", *d.ATA, d.V["h"], d.PAT, d.V["a2"], d.CAT, n, nnz)
        c.launch("spmv_csr", *d.AA, d.V["a"], d.PA, d.V["h2"], d.CA, n, nnz)
        ctx.sync()
        indeg = np.diff(csc[0]).astype(np.float32)
        outdeg = np.diff(csr[0]).astype(np.float32)
        assert torch.equal(d.vec["a2"][:n].cpu(), torch.from_numpy(indeg))
        assert torch.equal(d.vec["h2"][:n].cpu(), torch.from_numpy(outdeg))
        # second iterate from the GPU's normalised first iterate
        c.launch("l2norm", d.V["a2"], d.NA, d.SA, n)
        c.launch("l2norm", d.V["h2"], d.NH, d.SH, n)
        c.launch("scale", d.V["a2"], d.NA, n)
        c.launch("scale", d.V["h2"], d.NH, n)
        d.iterate("a2", "h2", "a", "h")
        ctx.sync()
        a1 = d.vec["a2"][:n].cpu().numpy().astype(np.float64)
        h1 = d.vec["h2"][:n].cpu().numpy().astype(np.float64)
        h2 = d.vec["h"][:n].cpu().numpy().astype(np.float64)
        nh = float(d.norms[1].item())
        rows = np.concatenate([np.random.default_rng(0).integers(0, n, 2000), [np.argmax(outdeg)]])
        rp, col, val = csr
        # the oracle's SpMV restricted to the sampled rows
        sub_rp = np.concatenate([[0], np.cumsum(np.diff(rp)[rows])])
        sub_col = np.concatenate([col[rp[r]:rp[r + 1]] for r in rows])
        sub_val = np.concatenate([val[rp[r]:rp[r + 1]] for r in rows])
        want = N.spmv_csr(sub_rp, sub_col, sub_val, a1) / nh
        got = h2[rows]
        assert np.all(np.abs(got - want) <= 2 * TOL * np.maximum(np.abs(want), 1e-30))
