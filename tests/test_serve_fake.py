"""The serving dispatcher on the recording backend (CPU only): requests of
every kind arrive as a Poisson stream or a burst and are all served;
admission follows arrival order and, under a tiny memory budget, admits one
request at a time; a window on the estimated GPU time in flight bounds the
requests in flight; a burst of small VEC and B&S requests is issued as fused
groups (3 members per VEC request, 10 per B&S request).  The fake backend
computes nothing, so this checks the dispatcher's logic, not results (the GPU
tests check those)."""
import datagen
import pytest

from paper_2012_09646_gb300 import serve as SV

SCALES = [1 / 64, 1 / 16]
SMALL = SV.Full(vec_n=4096, bs_n=8192, img_side=64, ml_rows=256, hits_n=20_000, hits_nnz=100_000, dl_n=2, dl_h=8,
                dl_w=64)
BUCKETS = 4


@pytest.fixture(scope="module")
def inputs():
    return SV.Inputs(datagen, full=SMALL, device="cpu", hits_buckets=BUCKETS)


def server(inputs, **kw):
    srv = SV.Server(inputs, device="cpu", backend="fake", **kw)
    srv.warm()
    return srv


def poisson(rate, count, seed):
    return SV.poisson_requests(rate, count, seed=seed)


def request(srv, rid, kind, s):
    """A request with its sizes and a slot, as admission gives it."""
    r = srv._make(kind, s, rid)
    r.slot = srv._take_slot(kind, True)
    return r


def fresh(reqs):
    return [SV.Request(r.rid, r.kind, r.scale, r.arrival) for r in reqs]


def test_stream_all_served_in_arrival_order(inputs):
    reqs = poisson(50_000.0, 60, 3)
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
    reqs = poisson(1e6, 12, 4)
    srv = server(inputs, budget_bytes=1)
    out = srv.run(fresh(reqs))
    for a, b in zip(out, out[1:]):
        assert b.admitted >= a.done_at
    srv.close()


def test_burst_issues_fused_groups(inputs):
    burst = [SV.Request(r.rid, r.kind, r.scale, 0.0) for r in poisson(1.0, 30, 5)]
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
    smallest request fuses nothing."""
    burst = [SV.Request(i, "B&S", SCALES[i % 2], 0.0) for i in range(6)]
    small = SV.sizes(SMALL, "B&S", SCALES[0])["n"]
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


def test_sizes_follow_the_scale():
    """Each request runs its own size: n = round(full * s) for VEC and B&S,
    the image side ~ full * sqrt(s) (a multiple of 8) and the ML rows ~
    full * s for IMG+ML, the smallest HITS graph at least s; DL is fixed."""
    f = SV.Full()
    assert SV.sizes(f, "VEC", 0.5) == {"n": 500_000, "nbytes": 2_000_000}
    assert SV.sizes(f, "B&S", 1 / 64)["n"] == 156_250
    z = SV.sizes(f, "IMG+ML", 0.25)
    assert z["side"] == 2048 and z["rows"] == 25_000 and z["resp"] == SV.RESPONSE_BYTES
    assert SV.sizes(f, "IMG+ML", 1.0)["side"] == 4096
    assert [SV.hits_bucket(s, 16) for s in (1 / 64, 1 / 16, 1 / 16 + 1e-6, 0.5, 1.0)] == [1, 1, 2, 8, 16]
    assert SV.sizes(f, "DL", 0.3) == {}
    # the mean work of U[1/64, 1] requests: about 0.51 for the continuously
    # scaled kinds, about 0.54 for HITS (16 graph scales)
    s = [r.scale for r in SV.poisson_requests(1.0, 20000, seed=1)]
    for kind, want in (("VEC", 0.508), ("B&S", 0.508), ("IMG+ML", 0.508), ("HITS", 0.539)):
        m = sum(SV.work_scale(f, kind, x) for x in s) / len(s)
        assert abs(m - want) < 0.01, (kind, m)


def test_window_bounds_the_requests_in_flight(inputs):
    """With every request estimated at 1 ms, a 3 ms window admits at most
    three at a time (a request is always admitted when nothing is in
    flight)."""
    reqs = fresh(poisson(1e6, 40, 11))
    srv = server(inputs, window_ms=3.0)
    srv.cost = {k: (1.0, 0.0) for k in SV.KINDS}
    peak = [0]
    issue_batch = srv.issue_batch

    def watched(batch):
        issue_batch(batch)
        live = [x for x in reqs if x.admitted is not None and x.done_at is None]
        peak[0] = max(peak[0], len(live))
    srv.issue_batch = watched
    out = srv.run(reqs)
    assert all(r.done_at is not None for r in out)
    assert 1 <= peak[0] <= 3
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
    the last hub update, the DL status copies), so the extra sinks are
    needed."""
    srv = server(inputs, record_log=True)
    for kind in SV.KINDS:
        r = request(srv, 0, kind, SCALES[0])
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
        g = [request(srv, i, kind, SCALES[i % 2]) for i in range(4)]
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


def test_admission_charges_exactly_what_a_slot_holds(inputs):
    """Admission charges slot_bytes(kind) against the budget: it must equal
    the device bytes a slot allocates, for every kind, and every request,
    at any scale, fits its kind's slot."""
    srv = server(inputs)
    for kind in SV.KINDS:
        sl = srv._take_slot(kind, True)
        got = sum(t.numel() * t.element_size() for t in sl.tensors.values())
        assert got == srv.slot_bytes(kind) == sl.nbytes, kind
        srv._return_slot(sl)
    for s in (SV.SCALE_MIN, 0.37, 1.0):
        for kind in SV.SCALED:
            r = request(srv, 0, kind, s)
            srv.issue(r)  # a size beyond the slot would be rejected by the kernels' checks
            srv.ctx.sync()
            srv.finish(r, 0.0)
            assert r.error is None
    assert srv.used == 0
    srv.close()


def test_budget_is_exceeded_only_by_a_request_admitted_alone(inputs):
    """Under a budget a few slots wide, the bytes held (slots in flight plus
    idle slots kept for reuse) never exceed it, except by a single request
    admitted while nothing else is in flight (which must run for the queue
    to make progress); idle slots of other kinds are released for room."""
    reqs = poisson(200_000.0, 80, 6)
    srv = server(inputs)
    srv.budget = 3 * max(srv.slot_bytes(k) for k in SV.KINDS)
    seen = []
    issue_batch = srv.issue_batch

    def watched(batch):
        inflight_before = srv.used - sum(r.need for r in batch)
        seen.append((srv.used + srv.cached, inflight_before, len(batch)))
        issue_batch(batch)
    srv.issue_batch = watched
    out = srv.run(fresh(reqs))
    assert all(r.done_at is not None for r in out)
    assert len(seen) > 1
    for held, before, n in seen:
        assert held <= srv.budget or (before == 0 and n == 1), (held, before, n)
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
    reqs = poisson(50_000.0, 40, 7)
    for k in (w, w + 37, w + 150, w + 400):
        srv = server(inputs, fake_fail_op=k)
        out = srv.run(fresh(reqs))
        failed = [r for r in out if r.error is not None]
        assert len(failed) == 1, k
        assert failed[0].error.code == G.GDAG_ERR_CUDA
        assert all(r.done_at is not None for r in out)
        assert all(r.resp_view is not None for r in out if r.error is None)
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
    reqs = poisson(50_000.0, 20, 8)
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
    reqs = poisson(50_000.0, 5, 9)
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
    srv.budget = 10 * srv.slot_bytes("VEC")
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


def test_long_requests_do_not_hold_up_short_ones(inputs):
    """With split_ms, requests estimated above it form their own class: a
    long request at the head of the queue fills its window without holding
    up the short ones behind it (each class keeps arrival order and its own
    window); with one class the long request holds them up."""
    burst = [SV.Request(0, "HITS", 1.0, 0.0)] + [SV.Request(i, "VEC", SCALES[0], 0.0) for i in range(1, 5)]
    first = {}
    for split in (None, 5.0):
        srv = server(inputs, window_ms=2.0, split_ms=split)
        srv.cost = {k: (1.0, 0.0) for k in SV.KINDS}
        srv.cost["HITS"] = (10.0, 0.0)
        batches = []
        issue_batch = srv.issue_batch

        def watched(batch, batches=batches, issue_batch=issue_batch):
            batches.append([(r.kind, r.cls) for r in batch])
            issue_batch(batch)
        srv.issue_batch = watched
        out = srv.run(fresh(burst))
        assert all(r.done_at is not None and r.error is None for r in out)
        first[split] = batches[0]
        if split is not None:
            assert {r.cls for r in out} == {"s", "l"} and out[0].cls == "l"
            s = SV.latency_summary(out)
            assert set(s["by_class"]) == {"s", "l"}
        srv.close()
    assert first[None] == [("HITS", "s")]
    assert sorted(first[5.0]) == [("HITS", "l"), ("VEC", "s"), ("VEC", "s")]
