"""Serving loop: requests of every kind and several scales arriving as a
Poisson stream on one context give the same response as each request served
alone (the kernels are deterministic, so the bits match), with and without
fusing small same-kind nodes across requests, and a tiny memory budget still
serves every request (FIFO admission)."""
import copy

import numpy as np
import pytest
import torch

import datagen
from paper_2012_09646_gb300 import serve as SV

pytestmark = pytest.mark.gpu

SCALES = [1 / 64, 1 / 16, 1 / 4]
HITS_SMALL = (400_000, 2_000_000)


@pytest.fixture(scope="module")
def inputs():
    return SV.Inputs(datagen, SCALES, hits_full=HITS_SMALL)


def fresh(reqs):
    return [SV.Request(r.rid, r.kind, r.scale, r.arrival) for r in reqs]


def test_mix_equals_alone(inputs):
    reqs = SV.poisson_requests(rate=20000.0, count=48, scales=SCALES, seed=1)
    srv = SV.Server(inputs)
    srv.warm()
    mixed = srv.run(fresh(reqs))
    srv.close()
    assert all(r.done_at is not None for r in mixed)
    # overlap really happened: some request was admitted before an earlier one finished
    assert any(b.admitted < a.done_at for a, b in zip(mixed, mixed[1:]))
    alone_srv = SV.Server(inputs)
    alone_srv.warm()
    for r in fresh(reqs):
        r.arrival = 0.0
        alone_srv.run([r])
        m = mixed[r.rid]
        assert m.kind == r.kind
        assert torch.equal(m.resp_view, r.resp_view), (r.kind, r.scale)
    alone_srv.close()
    s = SV.latency_summary(mixed)
    assert s["requests"] == 48 and s["p99_ms"] >= s["p50_ms"] > 0


def test_tiny_budget_serves_everything_in_order(inputs):
    reqs = SV.poisson_requests(rate=50000.0, count=12, scales=SCALES, seed=2)
    srv = SV.Server(inputs, budget_bytes=1)  # one request at a time
    srv.warm()
    out = srv.run(reqs)
    srv.close()
    adm = [r.admitted for r in out]
    assert adm == sorted(adm)
    for a, b in zip(out, out[1:]):
        assert b.admitted >= a.done_at  # the next is admitted only after the previous finished


def test_vec_response_matches_oracle(inputs):
    from oracle import pipelines as P
    srv = SV.Server(inputs)
    srv.warm(kinds=("VEC",))
    r = SV.Request(0, "VEC", 1 / 4, 0.0)
    srv.run([r])
    d = inputs.data[("VEC", inputs.bucket(1 / 4))]
    ref = P.vec(d["hx"].numpy(), d["hy"].numpy())
    assert abs(float(r.resp_view[0]) - ref["z"]) <= 1e-5 * ref["z_scale"]
    srv.close()


FUSE_ALL = {"VEC": 1 << 30, "B&S": 1 << 30}


def _alone(inputs, reqs):
    srv = SV.Server(inputs)
    srv.warm()
    out = {}
    for r in fresh(reqs):
        r.arrival = 0.0
        srv.run([r])
        out[r.rid] = r
    srv.close()
    return out


def test_fused_mix_equals_alone(inputs):
    """A burst (all arriving at once: one admission pass, fused groups) and a
    Poisson stream, with fusion on, against each request served alone."""
    burst = [SV.Request(r.rid, r.kind, r.scale, 0.0)
             for r in SV.poisson_requests(rate=1.0, count=24, scales=SCALES, seed=5)]
    stream = SV.poisson_requests(rate=20000.0, count=48, scales=SCALES, seed=6)
    for reqs in (burst, stream):
        srv = SV.Server(inputs, fuse_max=FUSE_ALL)
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
        alone = _alone(inputs, reqs)
        for m in mixed:
            assert m.done_at is not None
            assert torch.equal(m.resp_view, alone[m.rid].resp_view), (m.kind, m.scale)
