"""Serving loop on the GPU: requests of every kind (VEC, B&S, IMG+ML, HITS at
their own scales, and DL) arriving as a Poisson stream on one context.  Each
request's whole result is checked against the oracle run on the same inputs
at the request's size, in the mix and served alone, and the two are the same
bits (the kernels are deterministic), with and without fusing small
same-kind nodes across requests.  A tiny memory budget still serves every
request, in arrival order.

Tolerances are those of the per-DAG tests: fp32 outputs within 1e-5 of the
fp64 oracle (relative to max(|ref|, 1), or to the terms' scale for sums),
labels bit-exact except rows whose top-2 margin is below 4e-5, and the bf16
convolution DAG within 2e-2."""
import numpy as np
import pytest
import torch

import datagen
from oracle import numeric as N
from oracle import pipelines as P
from paper_2012_09646_gb300 import serve as SV

pytestmark = pytest.mark.gpu
TOL = 1e-5
MARGIN = 4e-5
FULL = SV.Full(vec_n=300_000, bs_n=200_000, img_side=512, ml_rows=3000, hits_n=150_000, hits_nnz=750_000,
               dl_n=2, dl_h=32, dl_w=64)
BUCKETS = 4
FUSE_ALL = {"VEC": 1 << 30, "B&S": 1 << 30}


@pytest.fixture(scope="module")
def inputs():
    return SV.Inputs(datagen, full=FULL, hits_buckets=BUCKETS, keep_host=True)


def fresh(reqs):
    return [SV.Request(r.rid, r.kind, r.scale, r.arrival) for r in reqs]


def serve(inputs, reqs, **kw):
    srv = SV.Server(inputs, keep_results=True, **kw)
    srv.warm()
    out = srv.run(reqs)
    srv.close()
    return out


def close(got, ref, scale=1.0):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(got - ref) <= TOL * np.maximum(np.abs(ref), scale)


def check_with_oracle(inputs, r):
    """r's whole result against the oracle at r's size."""
    assert r.error is None, (r.kind, r.error)
    z, res, H = r.size, r.result, inputs.host
    if r.kind == "VEC":
        x, y = H["VEC"]
        ref = P.vec(x[: z["n"]], y[: z["n"]])
        assert abs(float(res["z"][0]) - ref["z"]) <= TOL * max(ref["z_scale"], 1.0)
        assert float(r.resp_view[0]) == float(res["z"][0])
    elif r.kind == "B&S":
        for i, S in enumerate(H["B&S"]):
            got = res["C%d" % i].numpy()
            assert got.size == z["n"]
            assert close(got, N.bs_call(S[: z["n"]])).all(), (i, z)
        assert torch.equal(r.resp_view, res["C0"][: z["resp"] // 4])
    elif r.kind == "IMG+ML":
        img, X, T1, b1, T2, b2 = H["IMG+ML"]
        side, rows = z["side"], z["rows"]
        ref = P.img(img[: side * side].reshape(side, side))
        assert close(res["out"].numpy(), ref["out"].ravel()).all(), z
        assert torch.equal(r.resp_view, res["out"][: z["resp"] // 4])
        m = P.ml(X[:rows], T1, b1, T2, b2)
        lab = res["labels"].numpy()
        sure = m["margin"] >= MARGIN
        assert np.array_equal(lab[sure], m["labels"][sure]), z
    elif r.kind == "HITS":
        csr, csc = H[("HITS", z["bucket"])]
        ref = P.hits(csr, csc, iters=5)
        for got, want in ((res["a"].numpy(), ref["a"][-1]), (res["h"].numpy(), ref["h"][-1])):
            assert close(got, want).all(), z
            nz = want > 0
            assert np.all(np.abs(got[nz] - want[nz]) <= 5 * 2 * TOL * want[nz])
        assert torch.equal(r.resp_view, res["a"][: r.resp_view.numel()])
    else:
        ref = P.dl(*H["DL"])
        got = res["logits"].numpy().reshape(ref["logits"].shape)
        assert np.all(np.abs(got - ref["logits"]) <= 2e-2 * np.maximum(np.abs(ref["logits"]), 0.05))
        for k in ("p1", "p2"):
            g = res[k].float().numpy().reshape(ref[k].shape)
            assert np.all(np.abs(g - ref[k]) <= 2e-2 * np.maximum(np.abs(ref[k]), 0.05)), k


def results_equal(a, b):
    assert a.kind == b.kind and a.size == b.size
    assert torch.equal(a.resp_view, b.resp_view), a.kind
    for k in a.result:
        assert torch.equal(a.result[k], b.result[k]), (a.kind, k)


def alone(inputs, reqs, **kw):
    srv = SV.Server(inputs, keep_results=True, **kw)
    srv.warm()
    out = {}
    for r in fresh(reqs):
        r.arrival = 0.0
        srv.run([r])
        out[r.rid] = r
    srv.close()
    return out


def test_mix_matches_oracle_and_alone(inputs):
    reqs = SV.poisson_requests(20000.0, 60, seed=1)
    assert {r.kind for r in reqs} == set(SV.KINDS)
    mixed = serve(inputs, fresh(reqs))
    # overlap really happened: some request was admitted before an earlier one finished
    assert any(b.admitted < a.done_at for a, b in zip(mixed, mixed[1:]))
    for r in mixed:
        check_with_oracle(inputs, r)
    solo = alone(inputs, reqs)
    for r in mixed:
        results_equal(r, solo[r.rid])
    s = SV.latency_summary(mixed, FULL, BUCKETS)
    assert s["requests"] == 60 and s["failed"] == 0 and s["p99_ms"] >= s["p50_ms"] > 0


def test_every_kind_at_extreme_scales(inputs):
    """The smallest and largest size of every kind (HITS: the first and last
    graph), each against the oracle."""
    reqs = [SV.Request(i, k, s, 0.0) for i, (k, s) in enumerate(
        (k, s) for k in SV.KINDS for s in (SV.SCALE_MIN, 1.0))]
    for r in serve(inputs, reqs):
        check_with_oracle(inputs, r)


def test_fused_mix_matches_oracle_and_alone(inputs):
    """A burst (all arriving at once: one admission pass, fused groups) and a
    Poisson stream, with fusion on, against the oracle and each request
    served alone."""
    burst = [SV.Request(r.rid, r.kind, r.scale, 0.0) for r in SV.poisson_requests(1.0, 30, seed=5)]
    stream = SV.poisson_requests(20000.0, 40, seed=6)
    for reqs in (burst, stream):
        srv = SV.Server(inputs, fuse_max=FUSE_ALL, keep_results=True)
        srv.warm()
        f0 = srv.ctx.stats()["fused_members"]
        mixed = srv.run(fresh(reqs))
        fused = srv.ctx.stats()["fused_members"] - f0
        srv.close()
        if reqs is burst:
            # one admission pass: every VEC/B&S request of a kind that has
            # two or more goes through the fused elements (VEC: 2 squares +
            # 1 reduction per request; B&S: 10 prices per request)
            nv = sum(r.kind == "VEC" for r in reqs)
            nb = sum(r.kind == "B&S" for r in reqs)
            assert nv >= 2 and nb >= 2
            assert fused == 3 * nv + 10 * nb
        solo = alone(inputs, reqs)
        for r in mixed:
            check_with_oracle(inputs, r)
            results_equal(r, solo[r.rid])


def test_window_and_tiny_budget_serve_everything_in_order(inputs):
    reqs = SV.poisson_requests(50000.0, 15, seed=2)
    out = serve(inputs, fresh(reqs), budget_bytes=1)  # one request at a time
    adm = [r.admitted for r in out]
    assert adm == sorted(adm)
    for a, b in zip(out, out[1:]):
        assert b.admitted >= a.done_at  # the next is admitted only after the previous finished
    for r in out:
        check_with_oracle(inputs, r)
    srv = SV.Server(inputs, keep_results=True, window_ms=0.5)
    srv.warm(calibrate=True)
    assert all(a >= 0 and b >= 0 for a, b in srv.cost.values())
    cost = dict(srv.cost)
    out = srv.run(fresh(reqs))
    srv.close()
    for r in out:
        check_with_oracle(inputs, r)
    # two classes (long requests on their own context, short ones on
    # high-priority streams): same results
    split = sorted(a + b for a, b in cost.values())[len(cost) // 2]
    srv = SV.Server(inputs, keep_results=True, window_ms=0.5, split_ms=split)
    srv.warm()
    srv.cost = cost
    out = srv.run(fresh(SV.poisson_requests(50000.0, 30, seed=3)))
    srv.close()
    assert {r.cls for r in out} == {"s", "l"}
    for r in out:
        check_with_oracle(inputs, r)
