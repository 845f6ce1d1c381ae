"""The C++ dependency tracker and stream manager, driven through the C ABI with
the recording fake backend (no GPU), against the brute-force oracle.  CPU
only."""
import random

import pytest

from oracle import dag as D
from paper_2012_09646_gb300 import gdag as G
from tests.test_oracle_dag import CASES, load_cases

MODE_OF = {D.R: G.GDAG_MODE_IN, D.W: G.GDAG_MODE_OUT, D.RW: G.GDAG_MODE_INOUT}
SPEC = G.gdag_argspec(G.GDAG_ARG_ARRAY, G.GDAG_MODE_DEFAULT, 0, 0)


class Program:
    """Feeds a list of oracle elements to a fake-backend context.

    An element {array: mode} becomes a kernel launch over its arrays with
    per-argument mode overrides; ``("write", a)`` and ``("read", a)`` become
    host writes and reads."""

    def __init__(self, n_arrays, **opts):
        opts.setdefault("record_log", True)
        self.ctx = G.Context(backend="fake", **opts)
        self.arrays = [self.ctx.array(dev=0x10000 * (i + 1), nbytes=64, name="a%d" % i) for i in range(n_arrays)]
        self.kern = {}
        for n in range(1, 9):
            self.kern[n] = G.gdag_kernel_register(self.ctx.h, "k%d" % n, None, [SPEC] * n)
        self.elems = []

    def kernel(self, acc):
        items = list(acc.items())
        args = [G.array_arg(self.arrays[a].handle, MODE_OF[m]) for a, m in items]
        node = G.gdag_launch(self.ctx.h, self.kern[len(items)], G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0, args)
        assert node == len(self.elems)
        self.elems.append(dict(acc))
        return node

    def write(self, a):
        self.ctx.write(self.arrays[a], None)
        self.elems.append({a: D.W})

    def read(self, a):
        self.ctx.read(self.arrays[a])
        self.elems.append({a: D.R})

    def prefetch(self, a):
        before = len(self.ctx.nodes())
        self.ctx.prefetch_host(self.arrays[a])
        if len(self.ctx.nodes()) > before:  # no element when the view is current
            self.elems.append({a: D.R})


def edges_of(ctx, names=None):
    return {(s, d, a, k) for s, d, a, k in ctx.edges()}


def run_random(rng, L, n_arrays, **opts):
    p = Program(n_arrays, **opts)
    for _ in range(L):
        r = rng.random()
        if r < 0.12:
            p.write(rng.randrange(n_arrays))
        elif r < 0.22:
            p.read(rng.randrange(n_arrays))
        elif r < 0.28:
            p.prefetch(rng.randrange(n_arrays))
        else:
            k = rng.randint(1, min(4, n_arrays))
            arrs = rng.sample(range(n_arrays), k)
            p.kernel({a: rng.choice([D.R, D.R, D.W, D.RW]) for a in arrs})
    return p


@pytest.mark.parametrize("name", sorted(CASES))
def test_paper_cases_through_tracker(name):
    case = CASES[name]
    names = sorted({a for e in case["elems"] for a in e})
    idx = {a: i for i, a in enumerate(names)}
    p = Program(len(names))
    for e in case["elems"]:
        p.kernel({idx[a]: m for a, m in e.items()})
    want = {(i, j, idx[a], k) for i, j, a, k in case["edges"]}
    assert edges_of(p.ctx) == want


@pytest.mark.parametrize("seed", range(60))
def test_random_programs_match_brute_force(seed):
    rng = random.Random(seed)
    opts = rng.choice([{}, {"max_streams": 2}, {"retire_by_query": True, "fake_complete": True},
                       {"policy": G.GDAG_POLICY_SERIAL_ASYNC}, {"policy": G.GDAG_POLICY_SERIAL_SYNC},
                       {"max_streams": 1}])
    p = run_random(rng, rng.randint(1, 40), rng.randint(1, 6), **opts)
    want = D.expected_edges(p.elems)
    got = edges_of(p.ctx)
    assert got == want
    ops = p.ctx.ops()
    # every edge is ordered by CUDA's stream/event rules plus host waits
    assert D.check_hb(ops, want) == []
    # waits only along true edges, never for a same-stream parent
    assert D.waits_off_edges(ops, want) == []
    # node ids are consecutive in program order
    assert [n[0] for n in p.ctx.nodes()] == list(range(len(p.elems)))


def test_vec_schedule_one_cross_stream_event():
    """Section III-A, VEC example: K1 and K2 on two streams, the join K3 on
    K1's stream with exactly one event wait (on K2); reading z retires all."""
    p = Program(3)
    x, y, z = 0, 1, 2
    k1 = p.kernel({x: D.RW})
    k2 = p.kernel({y: D.RW})
    k3 = p.kernel({x: D.R, y: D.R, z: D.W})
    nodes = {n: s for n, _k, s in p.ctx.nodes()}
    assert nodes[k1] != nodes[k2]
    assert nodes[k3] == nodes[k1]
    waits = [o for o in p.ctx.ops() if o[0] == G.GDAG_OP_WAIT]
    assert len(waits) == 1 and waits[0][3] == k2 and waits[0][1] == nodes[k3]
    p.read(z)
    st = p.ctx.stats()
    assert st["active"] == 0 and st["streams"] == 2


def test_fifo_reuse_and_no_new_stream_when_one_is_empty():
    p = Program(8)
    for a in range(4):
        p.kernel({a: D.W})
    assert p.ctx.stats()["streams"] == 4
    p.ctx.sync()
    before = p.ctx.stats()["streams"]
    used = []
    for a in range(4, 8):
        p.kernel({a: D.W})
        used.append(p.ctx.nodes()[-1][2])
    assert p.ctx.stats()["streams"] == before
    assert used == [0, 1, 2, 3]  # oldest empty first


def test_first_child_on_parent_stream_later_children_elsewhere():
    p = Program(4)
    k0 = p.kernel({0: D.W})
    c1 = p.kernel({0: D.R, 1: D.W})
    c2 = p.kernel({0: D.R, 2: D.W})
    c3 = p.kernel({0: D.R, 3: D.W})
    s = {n: st for n, _k, st in p.ctx.nodes()}
    assert s[c1] == s[k0]
    assert len({s[c1], s[c2], s[c3]}) == 3


def test_stream_cap_falls_back_to_lru():
    p = Program(6, max_streams=3)
    for a in range(6):
        p.kernel({a: D.W})
    assert p.ctx.stats()["streams"] == 3
    s = [st for _n, _k, st in p.ctx.nodes()]
    assert s == [0, 1, 2, 0, 1, 2]


def test_host_write_war_waits_on_gpu_not_host():
    p = Program(2)
    p.kernel({0: D.R, 1: D.W})  # active reader of array 0
    p.write(0)                  # WAR: the copy waits on the GPU
    ops = p.ctx.ops()
    assert not any(o[0] in (G.GDAG_OP_HOST_WAIT, G.GDAG_OP_STREAM_SYNC) for o in ops)
    assert (0, 1, 0, D.WAR) in edges_of(p.ctx)


def test_serial_sync_waits_after_every_op():
    p = Program(3, policy=G.GDAG_POLICY_SERIAL_SYNC)
    p.kernel({0: D.W})
    p.kernel({1: D.W})
    p.kernel({0: D.R, 1: D.R, 2: D.W})
    ops = p.ctx.ops()
    work = [o for o in ops if o[0] == G.GDAG_OP_LAUNCH]
    hw = [o for o in ops if o[0] == G.GDAG_OP_HOST_WAIT]
    assert len(work) == 3 and len(hw) == 3
    assert {o[1] for o in work} == {0}
    assert p.ctx.stats()["active"] == 0


def test_serial_async_one_stream_no_waits():
    p = Program(3, policy=G.GDAG_POLICY_SERIAL_ASYNC)
    p.kernel({0: D.W})
    p.kernel({1: D.W})
    p.kernel({0: D.R, 1: D.R, 2: D.W})
    ops = p.ctx.ops()
    assert not any(o[0] in (G.GDAG_OP_WAIT, G.GDAG_OP_HOST_WAIT) for o in ops)
    assert p.ctx.stats()["streams"] == 1


def test_retire_by_query_drops_waits_on_finished_parents():
    p = Program(3, retire_by_query=True, fake_complete=True)
    p.kernel({0: D.W})
    p.kernel({1: D.W})
    p.kernel({0: D.R, 1: D.R, 2: D.W})
    assert not any(o[0] == G.GDAG_OP_WAIT for o in p.ctx.ops())
    assert len(edges_of(p.ctx)) == 2  # the logical edges stay


def test_validation_errors_leave_no_trace():
    ctx = G.Context(backend="fake", record_log=True)
    a = ctx.array(dev=0x1000, nbytes=400)
    c = ctx.array(dev=0x2000, nbytes=400)
    with pytest.raises(G.GdagError) as e:
        ctx.launch("bs_call", a, c, 101, 60.0, 0.1, 0.2, 1.0)  # n > 100 floats
    assert e.value.code == G.GDAG_ERR_INVALID
    with pytest.raises(G.GdagError):
        ctx.launch("bs_call", a, c, 100)  # wrong argument count
    with pytest.raises(G.GdagError):
        G.gdag_launch(ctx.h, ctx.kernel("bs_call")[0], G.gdag_dim3(0, 0, 0), G.gdag_dim3(0, 0, 0), 0,
                      [G.array_arg(99), G.array_arg(c.handle)] + [G.scalar_arg(1, 8)] + [G.scalar_arg(1.0, 4)] * 4)
    with pytest.raises(G.GdagError):
        G.gdag_launch(ctx.h, ctx.kernel("bs_call")[0], G.gdag_dim3(0, 0, 0), G.gdag_dim3(0, 0, 0), 0,
                      [G.array_arg(a.handle), G.array_arg(c.handle)] + [G.scalar_arg(1, 4)] + [G.scalar_arg(1.0, 4)] * 4)
    with pytest.raises(G.GdagError):
        ctx.write(a, None, off=396, nbytes=8)
    with pytest.raises(G.GdagError):
        ctx.read(a, None, off=401, nbytes=0)
    with pytest.raises(G.GdagError) as e:
        ctx.kernel("no_such_kernel")
    assert e.value.code == G.GDAG_ERR_NOT_FOUND
    assert ctx.nodes() == [] and ctx.edges() == []
    ctx.launch("bs_call", a, c, 100, 60.0, 0.1, 0.2, 1.0)
    assert len(ctx.nodes()) == 1


def test_injected_failure_and_poisoning():
    ctx = G.Context(backend="fake", fake_fail_op=0)
    a = ctx.array(dev=0x1000, nbytes=400)
    with pytest.raises(G.GdagError) as e:
        ctx.launch("vec_square", a, 100)
    assert e.value.code == G.GDAG_ERR_CUDA
    ctx.launch("vec_square", a, 100)  # not sticky: the context goes on
    ctx.close()
    ctx = G.Context(backend="fake", fake_fail_op=1, fake_fail_sticky=True)
    a = ctx.array(dev=0x1000, nbytes=400)
    with pytest.raises(G.GdagError) as e:
        ctx.launch("vec_square", a, 100)  # op 0 launch, op 1 event record
    assert e.value.code == G.GDAG_ERR_POISONED
    with pytest.raises(G.GdagError) as e:
        ctx.launch("vec_square", a, 100)
    assert e.value.code == G.GDAG_ERR_POISONED
    ctx.close()


def test_host_wait_times_out_instead_of_hanging():
    ctx = G.Context(backend="fake", fake_complete=2, timeout_ms=50)
    a = ctx.array(dev=0x1000, nbytes=400)
    ctx.launch("vec_square", a, 100)
    with pytest.raises(G.GdagError) as e:
        ctx.read(a)
    assert e.value.code == G.GDAG_ERR_TIMEOUT
    with pytest.raises(G.GdagError) as e:
        ctx.sync()
    assert e.value.code == G.GDAG_ERR_TIMEOUT


def test_external_call_gets_chosen_stream():
    seen = []
    ctx = G.Context(backend="fake", record_log=True)
    a = ctx.array(dev=0x1000, nbytes=400)
    b = ctx.array(dev=0x2000, nbytes=400)
    ctx.launch("vec_square", a, 100)
    node = ctx.external(lambda s, u: seen.append((s, u)), [(a, G.GDAG_MODE_IN), (b, G.GDAG_MODE_OUT)], user=7)
    # called once, before the call returns, with a stream handle of the pool
    assert len(seen) == 1 and seen[0][0] and seen[0][1] == 7
    assert (0, node, a.handle, G.GDAG_EDGE_RAW) in ctx.edges()
    # the library keeps no reference to the function: many calls hold nothing
    for _ in range(1000):
        ctx.external(lambda s, u: seen.append(s), [(b, G.GDAG_MODE_INOUT)])
    assert len(seen) == 1001


def test_prefetch_then_read_copies_once():
    p = Program(2)
    p.kernel({0: D.R, 1: D.W})
    p.prefetch(1)
    p.read(1)
    ops = p.ctx.ops()
    d2h = [o for o in ops if o[0] == G.GDAG_OP_COPY_D2H]
    assert len(d2h) == 1 and d2h[0][3] == 1          # the prefetch node
    assert [o for o in ops if o[0] == G.GDAG_OP_HOST_WAIT][-1][3] == 1
    assert ops[-1][0] == G.GDAG_OP_HOST_NODE and ops[-1][3] == 2
    # a kernel write after the prefetch makes the read copy again
    p.prefetch(1)
    p.kernel({1: D.W})
    p.read(1)
    assert len([o for o in p.ctx.ops() if o[0] == G.GDAG_OP_COPY_D2H]) == 2
    assert D.check_hb(p.ctx.ops(), D.expected_edges(p.elems)) == []


def test_capture_and_replay_as_one_element():
    p = Program(4)
    # capture a two-branch shape: k0 writes 0, k1 writes 1, k2 reads both, writes 2
    G.gdag_capture_begin(p.ctx.h)
    p.kernel({0: D.W})
    p.kernel({1: D.W})
    p.kernel({0: D.R, 1: D.R, 2: D.W})
    g = G.gdag_capture_end(p.ctx.h)
    n1 = G.gdag_graph_launch(p.ctx.h, g)
    n2 = G.gdag_graph_launch(p.ctx.h, g)
    # the replay element writes 0, 1 and 2 (and reads them): replays chain
    edges = {(s, d) for s, d, _a, _k in p.ctx.edges()}
    assert (n1, n2) in edges
    k = G.gdag_launch(p.ctx.h, p.kern[1], G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0,
                      [G.array_arg(p.arrays[2].handle, G.GDAG_MODE_IN)])
    assert (n2, k) in {(s, d) for s, d, _a, _k in p.ctx.edges()}
    nodes = dict((i, kind) for i, kind, _s in p.ctx.nodes())
    assert nodes[n1] == G.GDAG_NODE_GRAPH
    G.gdag_graph_destroy(p.ctx.h, g)
    with pytest.raises(G.GdagError):
        G.gdag_graph_launch(p.ctx.h, g)


def test_replay_refuses_arrays_registered_again_elsewhere():
    """A graph holds the addresses its arrays had at capture: after one of
    them is unregistered and its handle reused for memory elsewhere, the
    replay is refused; at the same address and size it is allowed."""
    p = Program(2)
    G.gdag_capture_begin(p.ctx.h)
    p.kernel({0: D.R, 1: D.W})
    g = G.gdag_capture_end(p.ctx.h)
    G.gdag_graph_launch(p.ctx.h, g)
    p.ctx.sync()
    dev1 = 0x10000 * 2
    p.ctx.unregister(p.arrays[1])
    with pytest.raises(G.GdagError) as e:
        G.gdag_graph_launch(p.ctx.h, g)
    assert e.value.code == G.GDAG_ERR_INVALID
    b = p.ctx.array(dev=0x90000, nbytes=64)  # takes the freed handle
    assert b.handle == p.arrays[1].handle
    with pytest.raises(G.GdagError) as e:
        G.gdag_graph_launch(p.ctx.h, g)
    assert e.value.code == G.GDAG_ERR_INVALID and "another address" in p.ctx.last_error
    p.ctx.unregister(b)
    c = p.ctx.array(dev=dev1, nbytes=64)  # the captured address again
    assert c.handle == p.arrays[1].handle
    G.gdag_graph_launch(p.ctx.h, g)
    p.ctx.sync()


def test_capture_rejects_host_waits_and_sync_policy():
    p = Program(2)
    G.gdag_capture_begin(p.ctx.h)
    with pytest.raises(G.GdagError) as e:
        p.ctx.read(p.arrays[0])
    assert e.value.code == G.GDAG_ERR_INVALID
    with pytest.raises(G.GdagError):
        G.gdag_capture_begin(p.ctx.h)  # nested
    with pytest.raises(G.GdagError):
        p.ctx.sync()
    g = G.gdag_capture_end(p.ctx.h)
    assert g >= 0
    q = Program(1, policy=G.GDAG_POLICY_SERIAL_SYNC)
    with pytest.raises(G.GdagError):
        G.gdag_capture_begin(q.ctx.h)


def test_node_query_polls_without_blocking():
    p = Program(2, fake_complete=False)
    k = p.kernel({0: D.W})
    assert G.gdag_node_query(p.ctx.h, k) is False  # still running
    q = Program(2, fake_complete=True)
    k = q.kernel({0: D.W})
    assert G.gdag_node_query(q.ctx.h, k) is True
    assert q.ctx.stats()["active"] == 0
    with pytest.raises(G.GdagError):
        G.gdag_node_query(q.ctx.h, 99)


def test_launch_argument_cache_keys_types_and_handles():
    """Repeated launches reuse their marshalled arguments; an int and a float
    of equal value are different scalars (different bits), and a handle
    reused after unregistering resolves to the new array."""
    ctx = G.Context(backend="fake", record_log=True)
    a = ctx.array(dev=0x1000, nbytes=400)
    c = ctx.array(dev=0x2000, nbytes=400)
    ctx.launch("bs_call", a, c, 100, 60.0, 0.1, 0.2, 1.0)
    ctx.launch("bs_call", a, c, 100, 60.0, 0.1, 0.2, 1.0)
    assert len(ctx._prepared) == 1
    ctx.launch("bs_call", a, c, 100, 60, 0.1, 0.2, 1.0)
    assert len(ctx._prepared) == 2
    vals = sorted(p[4][3].value for p in ctx._prepared.values())
    assert vals[0] == 60 and vals[1] == 0x42700000  # int 60 and float 60.0
    ctx.sync()
    ctx.unregister(c)
    c2 = ctx.array(dev=0x3000, nbytes=40)  # may reuse c's handle
    with pytest.raises(G.GdagError):  # n = 100 does not fit the new 10-float array
        ctx.launch("bs_call", a, c2, 100, 60.0, 0.1, 0.2, 1.0)
    assert len(ctx.nodes()) == 3


def test_launch_argument_cache_keeps_the_sign_of_zero_and_numpy_floats():
    """-0.0 == 0.0 in Python, but the two are different arguments: the
    cached marshalling must not hand the bits of one to the other.  numpy
    float scalars are floats, not truncated integers."""
    import numpy as np
    ctx = G.Context(backend="fake")
    a = ctx.array(dev=0x1000, nbytes=400)
    c = ctx.array(dev=0x2000, nbytes=400)

    def r_bits():  # the r argument (index 4) of the latest prepared launch
        return list(ctx._prepared.values())[-1][4][4].value

    ctx.launch("bs_call", a, c, 100, 60.0, 0.0, 0.2, 1.0)
    assert r_bits() == 0
    ctx.launch("bs_call", a, c, 100, 60.0, -0.0, 0.2, 1.0)
    assert r_bits() == 0x80000000 and len(ctx._prepared) == 2
    ctx.launch("bs_call", a, c, 100, 60.0, np.float32(-0.0), 0.2, 1.0)
    assert r_bits() == 0x80000000
    ctx.launch("bs_call", a, c, 100, 60.0, np.float32(0.5), 0.2, 1.0)
    assert r_bits() == 0x3F000000
    ctx.launch("bs_call", a, c, 100, 60.0, np.float32(0.0), 0.2, 1.0)
    assert r_bits() == 0
    assert G._scalar_bits(np.float64(-0.0), 8) == 1 << 63
    assert G._scalar_bits(np.int32(-1), 4) == 0xFFFFFFFF
    assert G._scalar_bits(True, 4) == 1
    # fused members go through the same keys
    buf = bytearray()
    ctx._pack("bs_call", (a, c, 100, 60.0, 0.0, 0.2, 1.0), buf)
    ctx._pack("bs_call", (a, c, 100, 60.0, -0.0, 0.2, 1.0), buf)
    half = len(buf) // 2
    assert bytes(buf[:half]) != bytes(buf[half:])
    ctx.close()


def test_chrome_trace_export(tmp_path):
    import json
    p = Program(3, trace=True, fake_complete=True)
    k0 = p.kernel({0: D.W})
    p.kernel({1: D.W})
    p.kernel({0: D.R, 1: D.R, 2: D.W})
    p.write(0)
    p.ctx.sync()
    out = tmp_path / "trace.json"
    n = p.ctx.chrome_trace(str(out), names={k0: "producer"})
    doc = json.load(open(out))
    assert n == len(doc["traceEvents"]) == 4
    assert {e["cat"] for e in doc["traceEvents"]} == {"kernel", "h2d"}
    assert doc["traceEvents"][0]["name"] == "producer"
    assert all(e["ph"] == "X" and e["dur"] >= 0 for e in doc["traceEvents"])


def test_option_environment_overrides(monkeypatch):
    monkeypatch.setenv("GDAG_MAX_STREAMS", "5")
    monkeypatch.setenv("GDAG_TIMEOUT_MS", "1234")
    monkeypatch.setenv("GDAG_PREFETCH", "not a number")
    monkeypatch.setenv("GDAG_TRIM_NODES", "4096")
    monkeypatch.setenv("GDAG_RECORD_LOG", "2")
    monkeypatch.setenv("GDAG_AUTO_GRAPH", "3")
    o = G.gdag_options_default()
    assert o.max_streams == 5 and o.timeout_ms == 1234 and o.prefetch == 1
    assert o.trim_nodes == 4096 and o.record_log == 2 and o.auto_graph == 3


@pytest.mark.parametrize("fail_op,where", [(4, "wait"), (5, "launch"), (6, "event record")])
def test_failed_element_keeps_its_parents_ordered(fail_op, where):
    """Two readers of x run on two streams; a writer of x, whose wait, launch
    or event record fails, sits between them and a second writer of x.  The
    second writer conflicts with the readers only through the failed one,
    so it must still run after both readers: the failure may not retire
    parents that have not been seen to complete."""
    ctx = G.Context(backend="fake", record_log=True, fake_fail_op=fail_op)
    x = ctx.array(dev=0x1000, nbytes=64)
    k = G.gdag_kernel_register(ctx.h, "k1", None, [SPEC])

    def run(mode):
        return G.gdag_launch(ctx.h, k, G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0,
                             [G.array_arg(x.handle, mode)])

    r1 = run(G.GDAG_MODE_IN)   # ops 0-1: launch, record (stream 0)
    r2 = run(G.GDAG_MODE_IN)   # ops 2-3: launch, record (stream 1)
    with pytest.raises(G.GdagError) as e:
        run(G.GDAG_MODE_OUT)   # op 4 wait on r2, op 5 launch, op 6 record
    assert e.value.code == G.GDAG_ERR_CUDA
    assert "injected failure at op %d" % fail_op in str(e.value)
    w = run(G.GDAG_MODE_OUT)
    assert w == 3
    assert D.check_hb(ctx.ops(), [(r1, w), (r2, w)]) == []
    ctx.sync()
    assert ctx.stats()["active"] == 0
    ctx.close()


BACKEND_OPS = (G.GDAG_OP_RECORD, G.GDAG_OP_WAIT, G.GDAG_OP_LAUNCH, G.GDAG_OP_COPY_H2D, G.GDAG_OP_COPY_D2H,
               G.GDAG_OP_EXTERNAL)


@pytest.mark.parametrize("seed", range(400))
def test_random_programs_with_an_injected_failure_stay_ordered(seed):
    """A random program whose k-th backend op fails (not sticky): the failing
    call raises and the program goes on.  With the failed op taken out of the
    recorded log, every two elements that conflict directly and did not fail
    are still ordered by CUDA's stream/event rules plus host waits, even
    where the nearest edges between them ran through the failed element.
    Without a failure (k beyond the program's ops) this is the plain
    serialisability check over every conflicting pair."""
    rng = random.Random(1000 + seed)
    n_arrays = rng.randint(1, 5)
    opts = rng.choice([{}, {"max_streams": 2}, {"retire_by_query": True, "fake_complete": True},
                       {"policy": G.GDAG_POLICY_SERIAL_ASYNC}, {"policy": G.GDAG_POLICY_SERIAL_SYNC}])
    fail_at = rng.randrange(60)
    p = Program(n_arrays, fake_fail_op=fail_at, **opts)
    failed = []
    for _ in range(rng.randint(1, 30)):
        r = rng.random()
        a = rng.randrange(n_arrays)
        if r < 0.12:
            acc, call = {a: D.W}, lambda: p.ctx.write(p.arrays[a], None)
        elif r < 0.22:
            acc, call = {a: D.R}, lambda: p.ctx.read(p.arrays[a])
        else:
            arrs = rng.sample(range(n_arrays), rng.randint(1, min(4, n_arrays)))
            acc = {b: rng.choice([D.R, D.R, D.W, D.RW]) for b in arrs}
            args = [G.array_arg(p.arrays[b].handle, MODE_OF[m]) for b, m in acc.items()]
            call = lambda: G.gdag_launch(p.ctx.h, p.kern[len(args)], G.gdag_dim3(1, 1, 1),
                                         G.gdag_dim3(32, 1, 1), 0, args)
        try:
            call()
        except G.GdagError as e:
            assert e.code == G.GDAG_ERR_CUDA and "injected failure at op %d" % fail_at in str(e)
            failed.append(len(p.elems))
        p.elems.append(acc)
    assert len(failed) <= 1
    assert [n[0] for n in p.ctx.nodes()] == list(range(len(p.elems)))
    ops = p.ctx.ops()
    backend = [q for q, o in enumerate(ops) if o[0] in BACKEND_OPS]
    if failed:
        del ops[backend[fail_at]]
    pairs = [(i, j) for i, j in D.conflict_pairs(p.elems) if i not in failed and j not in failed]
    assert D.check_hb(ops, pairs) == []
    p.ctx.sync()
    assert p.ctx.stats()["active"] == 0


def test_read_from_the_view_waits_for_the_copy_that_filled_it():
    """A full host write fills the view and starts its copy to the device; a
    host read is then served from the view.  A kernel that next writes the
    array takes its edge from the read alone (the dependency-set rule), so
    the read may not complete before the copy: the host waits for it, and
    the kernel cannot race the copy."""
    p = Program(2)
    p.kernel({1: D.W})          # keeps stream 0 busy
    w = len(p.elems)
    p.write(0)                  # copy on its own stream, still in flight
    r = len(p.elems)
    p.read(0)                   # served from the view
    k = p.kernel({0: D.W})
    edges = {(s, d) for s, d, _a, _k in p.ctx.edges()}
    assert (w, r) in edges and (r, k) in edges and (w, k) not in edges
    ops = p.ctx.ops()
    assert (G.GDAG_OP_HOST_WAIT, ) == tuple(o[0] for o in ops if o[3] == w and o[0] == G.GDAG_OP_HOST_WAIT)
    assert D.check_hb(ops, [(w, k)]) == []


@pytest.mark.parametrize("seed", range(300))
def test_random_programs_of_every_element_kind_are_serialisable(seed):
    """Random programs mixing every kind of element: kernels with mode
    overrides, fused launches, external library calls, full and partial
    host writes, reads and prefetches, replays of a captured graph, with
    syncs, node queries and array re-registrations in between and,
    sometimes, one injected backend failure.  Every two elements that conflict directly, both of which did
    their work, are ordered by CUDA's stream/event rules plus host waits;
    the edge log equals the brute-force edges of the program as issued."""
    rng = random.Random(7000 + seed)
    n_arrays = rng.randint(2, 6)
    opts = rng.choice([{}, {"max_streams": 2}, {"max_streams": 1}, {"prefetch": False}, {"trace": True},
                       {"retire_by_query": True, "fake_complete": True},
                       {"policy": G.GDAG_POLICY_SERIAL_ASYNC}, {"policy": G.GDAG_POLICY_SERIAL_SYNC}])
    # a capture and tracing issue backend ops of their own that the op log
    # leaves out (the fork and join of the capture stream, timing events),
    # so such a program gets no injected failure: the failed op could not be
    # found in the log
    use_capture = rng.random() < 0.5 and opts.get("policy") != G.GDAG_POLICY_SERIAL_SYNC
    inject = not use_capture and not opts.get("trace")
    fail_at = rng.randrange(120) if inject and rng.random() < 0.7 else -1
    p = Program(n_arrays, fake_fail_op=fail_at, **opts)
    for k in range(min(rng.choice([0, 0, 1, 2]), opts.get("max_streams", 16))):  # caller-owned streams
        G.gdag_add_stream(p.ctx.h, 0xC0000 + k)
    arrs = p.arrays    # slot -> registered array (slots are re-registered)
    logical = list(range(n_arrays))   # slot -> logical array id
    handle_of = {i: arrs[i].handle for i in range(n_arrays)}  # logical -> handle
    skip = set()       # elements that did no work (failed, or only captured)
    graph = None
    graph_acc = None
    graph_live = True  # no array of the graph unregistered since its capture

    def n_nodes():
        return G.gdag_stats_get(p.ctx.h).nodes

    def attempt(acc, call, work=True):
        before = n_nodes()
        try:
            call()
        except G.GdagError as e:
            assert e.code == G.GDAG_ERR_CUDA and "injected failure at op %d" % fail_at in str(e)
            work = False
        if n_nodes() > before:  # the call made one element
            assert n_nodes() == before + 1
            if not work:
                skip.add(len(p.elems))
            p.elems.append({logical[b]: m for b, m in acc.items()})

    def random_kernel():
        ks = rng.sample(range(n_arrays), rng.randint(1, min(4, n_arrays)))
        acc = {b: rng.choice([D.R, D.R, D.W, D.RW]) for b in ks}
        args = [G.array_arg(arrs[b].handle, MODE_OF[m]) for b, m in acc.items()]
        return acc, lambda: G.gdag_launch(p.ctx.h, p.kern[len(args)], G.gdag_dim3(1, 1, 1),
                                          G.gdag_dim3(32, 1, 1), 0, args)

    for _ in range(rng.randint(1, 35)):
        r = rng.random()
        a = rng.randrange(n_arrays)
        off = rng.choice([0, 0, 16])
        nb = 64 - off if rng.random() < 0.7 else 16
        if r < 0.10:
            attempt({a: D.W}, lambda: p.ctx.write(arrs[a], None, off, nb))
        elif r < 0.18:
            attempt({a: D.R}, lambda: p.ctx.read(arrs[a], None, off, nb))
        elif r < 0.24:
            attempt({a: D.R}, lambda: p.ctx.prefetch_host(arrs[a], off, nb))
        elif r < 0.30:
            # fused bs_call: members read shared prices, each writes its own output
            outs = rng.sample(range(n_arrays), rng.randint(1, n_arrays - 1))
            ins = [b for b in range(n_arrays) if b not in outs]
            pick = [(rng.choice(ins), o) for o in outs]
            members = [(arrs[i], arrs[o], 16, 60.0, 0.1, 0.2, 1.0) for i, o in pick]
            acc = {}
            for i, o in pick:
                acc[i] = D.R
                acc[o] = D.W
            attempt(acc, lambda: p.ctx.launch_fused("bs_call", members))
        elif r < 0.35:
            ks = rng.sample(range(n_arrays), rng.randint(1, min(3, n_arrays)))
            acc = {b: rng.choice([D.R, D.W, D.RW]) for b in ks}
            attempt(acc, lambda: p.ctx.external(lambda s, u: None, [(arrs[b], MODE_OF[m]) for b, m in acc.items()]))
        elif r < 0.40 and graph is None and use_capture:
            G.gdag_capture_begin(p.ctx.h)
            graph_acc = {}
            try:
                for _ in range(rng.randint(1, 3)):
                    acc, call = random_kernel()
                    call()
                    skip.add(len(p.elems))
                    p.elems.append({logical[b]: m for b, m in acc.items()})
                    for b, m in acc.items():
                        graph_acc[b] = graph_acc.get(b, 0) | m
            finally:
                graph = G.gdag_capture_end(p.ctx.h)
        elif r < 0.48 and graph is not None and graph_live:
            attempt(dict(graph_acc), lambda: G.gdag_graph_launch(p.ctx.h, graph))
        elif r < 0.50:
            # unregister (waits for the array's users) and register a new
            # array, which may take the freed handle: a new logical array
            p.ctx.unregister(arrs[a])
            if graph_acc and a in graph_acc:
                graph_live = False
                with pytest.raises(G.GdagError):
                    G.gdag_graph_launch(p.ctx.h, graph)
            arrs[a] = p.ctx.array(dev=0x1000000 + 0x10000 * len(handle_of), nbytes=64)
            logical[a] = len(handle_of)
            handle_of[logical[a]] = arrs[a].handle
        elif r < 0.52:
            p.ctx.sync()
        elif r < 0.56 and p.elems:
            p.ctx.done(rng.randrange(len(p.elems)))
        else:
            attempt(*random_kernel())
    assert [n[0] for n in p.ctx.nodes()] == list(range(len(p.elems)))
    assert edges_of(p.ctx) == {(i, j, handle_of[a], k) for i, j, a, k in D.expected_edges(p.elems)}
    ops = p.ctx.ops()
    if fail_at >= 0:
        backend = [q for q, o in enumerate(ops) if o[0] in BACKEND_OPS]
        if fail_at < len(backend):
            del ops[backend[fail_at]]
    pairs = [(i, j) for i, j in D.conflict_pairs(p.elems) if i not in skip and j not in skip]
    assert D.check_hb(ops, pairs) == []
    p.ctx.sync()
    assert p.ctx.stats()["active"] == 0
