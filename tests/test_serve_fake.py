"""The serving dispatcher on the recording backend (CPU only): requests of
every kind arrive as a Poisson stream or a burst and are all served;
admission follows arrival order and, under a tiny memory budget, admits one
request at a time; a burst of small VEC and B&S requests is issued as fused
groups (3 members per VEC request, 10 per B&S request).  The fake backend
computes nothing, so this checks the dispatcher's logic, not results (the GPU
tests check those)."""
import datagen
import pytest

from paper_2012_09646_gb300 import serve as SV

SCALES = [1 / 64, 1 / 16]
HITS_SMALL = (20_000, 100_000)


@pytest.fixture(scope="module")
def inputs():
    return SV.Inputs(datagen, SCALES, device="cpu", hits_full=HITS_SMALL)


def server(inputs, **kw):
    srv = SV.Server(inputs, device="cpu", backend="fake", **kw)
    srv.warm()
    return srv


def fresh(reqs):
    return [SV.Request(r.rid, r.kind, r.scale, r.arrival) for r in reqs]


def test_stream_all_served_in_arrival_order(inputs):
    reqs = SV.poisson_requests(rate=50_000.0, count=40, scales=SCALES, seed=3)
    srv = server(inputs)
    out = srv.run(fresh(reqs))
    assert all(r.done_at is not None and r.done_at >= r.arrival for r in out)
    adm = [r.admitted for r in out]
    assert adm == sorted(adm)
    assert {r.kind for r in out} == set(SV.KINDS)
    assert srv.used == 0  # every request's memory was released
    st = srv.ctx.stats()
    assert st["active"] == 0
    srv.close()


def test_tiny_budget_admits_one_at_a_time(inputs):
    reqs = SV.poisson_requests(rate=1e6, count=12, scales=SCALES, seed=4)
    srv = server(inputs, budget_bytes=1)
    out = srv.run(fresh(reqs))
    for a, b in zip(out, out[1:]):
        assert b.admitted >= a.done_at
    srv.close()


def test_burst_issues_fused_groups(inputs):
    burst = [SV.Request(r.rid, r.kind, r.scale, 0.0)
             for r in SV.poisson_requests(rate=1.0, count=30, scales=SCALES, seed=5)]
    nv = sum(r.kind == "VEC" for r in burst)
    nb = sum(r.kind == "B&S" for r in burst)
    assert nv >= 2 and nb >= 2
    srv = server(inputs, fuse_max={"VEC": 1 << 30, "B&S": 1 << 30})
    f0 = srv.ctx.stats()["fused_members"]
    out = srv.run(burst)
    assert all(r.done_at is not None for r in out)
    assert srv.ctx.stats()["fused_members"] - f0 == 3 * nv + 10 * nb
    srv.close()
    # without fusion thresholds nothing is fused
    srv = server(inputs)
    f0 = srv.ctx.stats()["fused_members"]
    srv.run([SV.Request(r.rid, r.kind, r.scale, 0.0) for r in burst])
    assert srv.ctx.stats()["fused_members"] == f0
    srv.close()


def test_fusion_threshold_excludes_large_nodes(inputs):
    """Only nodes at most fuse_max elements are fused: a threshold below the
    smallest bucket fuses nothing."""
    burst = [SV.Request(i, "B&S", SCALES[i % 2], 0.0) for i in range(6)]
    small = inputs.data[("B&S", SCALES[0])]["n"]
    srv = server(inputs, fuse_max={"B&S": small})
    f0 = srv.ctx.stats()["fused_members"]
    srv.run(burst)
    assert srv.ctx.stats()["fused_members"] - f0 == 10 * 3  # the three 1/64 requests
    srv.close()
    srv = server(inputs, fuse_max={"B&S": small - 1})
    f0 = srv.ctx.stats()["fused_members"]
    srv.run([SV.Request(r.rid, r.kind, r.scale, 0.0) for r in burst])
    assert srv.ctx.stats()["fused_members"] == f0
    srv.close()


def _ancestors(edges, sinks):
    par = {}
    for s, d, _a, _k in edges:
        par.setdefault(d, set()).add(s)
    seen, stack = set(), list(sinks)
    while stack:
        v = stack.pop()
        if v not in seen:
            seen.add(v)
            stack.extend(par.get(v, ()))
    return seen


def test_sinks_cover_every_node_of_a_request(inputs):
    """A request is complete when its sinks are: every node it issued is an
    ancestor of (or is) one of them.  For every kind but VEC the response
    prefetch alone does not cover the request (other outputs, the ML branch,
    the last hub update), so the extra sinks are needed."""
    srv = server(inputs, record_log=True)
    for kind in SV.KINDS:
        r = SV.Request(0, kind, SCALES[0], 0.0)
        first = srv._last_node() + 1
        srv.issue(r)
        mine = set(range(first, srv._last_node() + 1))
        edges = srv.ctx.edges()
        assert mine <= _ancestors(edges, r.sinks), kind
        covered_by_prefetch = mine <= _ancestors(edges, r.sinks[-1:])
        assert covered_by_prefetch == (kind == "VEC"), kind
        srv.ctx.sync()
        srv.finish(r, 0.0)
    # fused groups: each member's sink is its prefetch, after the fused nodes
    for kind in ("VEC", "B&S"):
        g = [SV.Request(i, kind, SCALES[i % 2], 0.0) for i in range(4)]
        srv.fuse_max = {kind: 1 << 30}
        first = srv._last_node() + 1
        srv.issue_batch(g)
        mine = set(range(first, srv._last_node() + 1))
        edges = srv.ctx.edges()
        assert all(len(r.sinks) == 1 for r in g)
        assert mine <= set().union(*(_ancestors(edges, r.sinks) for r in g)), kind
        srv.ctx.sync()
        for r in g:
            srv.finish(r, 0.0)
    srv.close()


def test_admission_charges_exactly_what_a_request_allocates(inputs):
    """Admission adds working_bytes(r) to the budget and finish() releases
    it: it must equal the bytes the request allocates, for every kind and
    bucket, alone and in fused groups, so that the budget is never exceeded
    and never held back."""
    srv = server(inputs)
    for s in SCALES:
        for kind in SV.KINDS:
            r = SV.Request(0, kind, s, 0.0)
            srv.issue(r)
            assert r.bytes == srv.working_bytes(r), (kind, s)
            srv.ctx.sync()
            srv.finish(r, 0.0)
    for kind in ("VEC", "B&S"):
        g = [SV.Request(i, kind, SCALES[i % 2], 0.0) for i in range(4)]
        srv.fuse_max = {kind: 1 << 30}
        srv.issue_batch(g)
        assert all(r.bytes == srv.working_bytes(r) for r in g), kind
        srv.ctx.sync()
        for r in g:
            srv.finish(r, 0.0)
    srv.close()


def test_budget_is_exceeded_only_by_a_request_admitted_alone(inputs):
    """Under a budget a few requests wide, the bytes admitted never exceed
    it, except by a single request admitted while nothing else is in flight
    (which must run for the queue to make progress)."""
    reqs = SV.poisson_requests(rate=200_000.0, count=60, scales=SCALES, seed=6)
    srv = server(inputs, budget_bytes=40_000_000)
    seen = []
    issue_batch = srv.issue_batch

    def watched(batch):
        inflight_before = srv.used - sum(r.need for r in batch)
        seen.append((srv.used, inflight_before, len(batch)))
        issue_batch(batch)
    srv.issue_batch = watched
    out = srv.run(fresh(reqs))
    assert all(r.done_at is not None for r in out)
    assert len(seen) > 1
    for used, before, n in seen:
        assert used <= srv.budget or (before == 0 and n == 1), (used, before, n)
    assert srv.used == 0
    srv.close()


def _warm_ops(inputs):
    """Backend operations the server issues before serving (warm-up)."""
    from tests.test_tracker_fake import BACKEND_OPS
    ref = server(inputs, record_log=True)
    n = sum(1 for o in ref.ctx.ops() if o[0] in BACKEND_OPS)
    ref.close()
    return n


def test_a_failed_request_fails_alone(inputs):
    """A backend operation that fails (not sticky) while a request is being
    issued fails that request only: it finishes at once with the error, its
    memory is released, and every other request is served."""
    from paper_2012_09646_gb300 import gdag as G
    w = _warm_ops(inputs)
    reqs = SV.poisson_requests(rate=50_000.0, count=40, scales=SCALES, seed=7)
    for k in (w, w + 37, w + 150, w + 400):
        srv = server(inputs, fake_fail_op=k)
        out = srv.run(fresh(reqs))
        failed = [r for r in out if r.error is not None]
        assert len(failed) == 1, k
        assert failed[0].error.code == G.GDAG_ERR_CUDA
        assert all(r.done_at is not None for r in out)
        assert all(r.resp_view is not None for r in out if r.error is None and r.kind != "VEC")
        assert srv.used == 0 and not srv.ctx.stats()["active"]
        s = SV.latency_summary(out)
        assert s["requests"] == len(out) - 1 and s["failed"] == 1
        srv.close()


def test_a_fused_group_fails_together(inputs):
    from paper_2012_09646_gb300 import gdag as G
    w = _warm_ops(inputs)
    burst = [SV.Request(i, "B&S", SCALES[i % 2], 0.0) for i in range(5)]
    srv = server(inputs, fuse_max={"B&S": 1 << 30}, fake_fail_op=w)  # the group's fused launch
    out = srv.run(burst)
    assert all(r.error is not None and r.error.code == G.GDAG_ERR_CUDA for r in out)
    assert srv.used == 0
    # the server goes on serving
    more = srv.run([SV.Request(9, "VEC", SCALES[0], 0.0)])
    assert more[0].error is None and more[0].done_at is not None
    srv.close()


def test_a_context_losing_failure_stops_the_server(inputs):
    from paper_2012_09646_gb300 import gdag as G
    w = _warm_ops(inputs)
    reqs = SV.poisson_requests(rate=50_000.0, count=20, scales=SCALES, seed=8)
    srv = server(inputs, fake_fail_op=w + 10, fake_fail_sticky=True)
    with pytest.raises(G.GdagError) as e:
        srv.run(fresh(reqs))
    assert e.value.code == G.GDAG_ERR_POISONED
    srv.ctx.close()


def test_a_device_that_stops_completing_times_out(inputs):
    """Nodes that never report complete (the recording backend completes
    them only on a host wait, which the dispatcher never issues): run()
    raises GDAG_ERR_TIMEOUT after the request deadline instead of polling
    forever."""
    import time
    from paper_2012_09646_gb300 import gdag as G
    reqs = SV.poisson_requests(rate=50_000.0, count=5, scales=SCALES, seed=9)
    srv = server(inputs, fake_complete=0, request_timeout_s=0.2)
    t = time.perf_counter()
    with pytest.raises(G.GdagError) as e:
        srv.run(fresh(reqs))
    assert e.value.code == G.GDAG_ERR_TIMEOUT
    assert time.perf_counter() - t < 10
    srv.close()


def test_a_long_serving_run_holds_a_bounded_node_table(inputs):
    """The dispatcher never calls gdag_sync while serving, yet the context
    holds only its active window, not every element of every request
    served: a budget ten requests wide keeps at most ten in flight, and the
    node table and the shared inputs' reader sets stay within twice the
    trim threshold over 4000 requests."""
    n, trim = 4000, 1024
    reqs = [SV.Request(i, "VEC", SCALES[0], 0.0) for i in range(n)]
    srv = server(inputs, trim_nodes=trim)
    srv.budget = 10 * srv.working_bytes(reqs[0])
    peak = [0, 0]
    issue_batch = srv.issue_batch

    def watched(batch):
        issue_batch(batch)
        st = srv.ctx.stats()
        peak[0] = max(peak[0], st["held_nodes"])
        peak[1] = max(peak[1], st["held_readers"])
    srv.issue_batch = watched
    srv.run(reqs)
    st = srv.ctx.stats()
    assert st["nodes"] > 10 * trim  # far more elements than the table keeps
    assert peak[0] <= 2 * trim and peak[1] <= 2 * trim, peak
    assert all(r.error is None for r in reqs)
    srv.close()
