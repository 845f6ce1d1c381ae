"""Dropping retired elements from the tracker's node table (options.trim_nodes)
and from the arrays' reader sets, driven through the C ABI with the recording
fake backend.  CPU only.

Retired elements are complete and observed, so they cause no waits and pick no
streams.  Dropping them may therefore change nothing the backend sees: the
same random program must issue the same backend operations with and without
trimming, and with the full logs kept its edge log must not change either."""
import random

import pytest

from oracle import dag as D
from paper_2012_09646_gb300 import gdag as G

MODE_OF = {D.R: G.GDAG_MODE_IN, D.W: G.GDAG_MODE_OUT, D.RW: G.GDAG_MODE_INOUT}
SPEC = G.gdag_argspec(G.GDAG_ARG_ARRAY, G.GDAG_MODE_DEFAULT, 0, 0)
NB = 64


def random_script(rng, n_arrays, length):
    """A program as data, so that several contexts can run the same one."""
    out = []
    for _ in range(length):
        r = rng.random()
        a = rng.randrange(n_arrays)
        off = rng.choice([0, 0, 16])
        nb = NB - off if rng.random() < 0.7 else 16
        if r < 0.10:
            out.append(("write", a, off, nb))
        elif r < 0.18:
            out.append(("read", a, off, nb))
        elif r < 0.23:
            out.append(("prefetch", a, off, nb))
        elif r < 0.28 and n_arrays > 1:
            outs = rng.sample(range(n_arrays), rng.randint(1, n_arrays - 1))
            ins = [b for b in range(n_arrays) if b not in outs]
            out.append(("fused", [(rng.choice(ins), o) for o in outs]))
        elif r < 0.32:
            ks = rng.sample(range(n_arrays), rng.randint(1, min(3, n_arrays)))
            out.append(("external", {b: rng.choice([D.R, D.W, D.RW]) for b in ks}))
        elif r < 0.36:
            ks = rng.sample(range(n_arrays), rng.randint(1, min(3, n_arrays)))
            out.append(("capture", [{b: rng.choice([D.R, D.R, D.W, D.RW]) for b in ks}
                                    for _ in range(rng.randint(1, 3))]))
        elif r < 0.42:
            out.append(("replay",))
        elif r < 0.44:
            out.append(("reregister", a))
        elif r < 0.46:
            out.append(("sync",))
        elif r < 0.56:
            out.append(("query", rng.random()))
        else:
            ks = rng.sample(range(n_arrays), rng.randint(1, min(4, n_arrays)))
            out.append(("kernel", {b: rng.choice([D.R, D.R, D.W, D.RW]) for b in ks}))
    return out


def run_script(script, n_arrays, **opts):
    """Run `script` on a fresh fake-backend context; returns the context and
    one outcome per step (None, or the error code a step raised)."""
    ctx = G.Context(backend="fake", **opts)
    arrs = [ctx.array(dev=0x10000 * (i + 1), nbytes=NB) for i in range(n_arrays)]
    kern = {n: G.gdag_kernel_register(ctx.h, "k%d" % n, None, [SPEC] * n) for n in range(1, 9)}
    graphs = []
    fresh = [0x4000000]

    def launch(acc):
        args = [G.array_arg(arrs[b].handle, MODE_OF[m]) for b, m in acc.items()]
        G.gdag_launch(ctx.h, kern[len(args)], G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0, args)

    outcome = []
    for step in script:
        kind = step[0]
        try:
            if kind == "write":
                ctx.write(arrs[step[1]], None, step[2], step[3])
            elif kind == "read":
                ctx.read(arrs[step[1]], None, step[2], step[3])
            elif kind == "prefetch":
                ctx.prefetch_host(arrs[step[1]], step[2], step[3])
            elif kind == "fused":
                ctx.launch_fused("bs_call", [(arrs[i], arrs[o], 16, 60.0, 0.1, 0.2, 1.0) for i, o in step[1]])
            elif kind == "external":
                ctx.external(lambda s, u: None, [(arrs[b], MODE_OF[m]) for b, m in step[1].items()])
            elif kind == "capture":
                if opts.get("policy") == G.GDAG_POLICY_SERIAL_SYNC:
                    outcome.append("skip")
                    continue
                G.gdag_capture_begin(ctx.h)
                try:
                    for acc in step[1]:
                        launch(acc)
                finally:
                    graphs.append(G.gdag_capture_end(ctx.h))
            elif kind == "replay":
                if not graphs:
                    outcome.append("skip")
                    continue
                G.gdag_graph_launch(ctx.h, graphs[-1])
            elif kind == "reregister":
                ctx.unregister(arrs[step[1]])
                fresh[0] += 0x10000
                arrs[step[1]] = ctx.array(dev=fresh[0], nbytes=NB)
            elif kind == "sync":
                ctx.sync()
            elif kind == "query":
                n = ctx.stats()["nodes"]
                if n:
                    ctx.done(int(step[1] * n))
            else:
                launch(step[1])
            outcome.append(None)
        except G.GdagError as e:
            outcome.append(e.code)
    return ctx, outcome


@pytest.mark.parametrize("seed", range(120))
def test_trimming_changes_no_backend_operation(seed):
    rng = random.Random(9100 + seed)
    n_arrays = rng.randint(1, 6)
    opts = rng.choice([{}, {"max_streams": 2}, {"max_streams": 1}, {"prefetch": False},
                       {"retire_by_query": True, "fake_complete": True},
                       {"retire_by_query": True, "fake_complete": True, "max_streams": 3},
                       {"policy": G.GDAG_POLICY_SERIAL_ASYNC}, {"policy": G.GDAG_POLICY_SERIAL_SYNC}])
    if rng.random() < 0.3:
        opts["fake_fail_op"] = rng.randrange(200)
    trim = rng.choice([1, 2, 3, 8, 32])
    script = random_script(rng, n_arrays, rng.randint(50, 250))

    ref, out_ref = run_script(script, n_arrays, record_log=1, **opts)           # nothing dropped
    full, out_full = run_script(script, n_arrays, record_log=1, trim_nodes=trim, **opts)
    lean, out_lean = run_script(script, n_arrays, record_log=2, trim_nodes=trim, **opts)

    assert out_full == out_ref and out_lean == out_ref
    ops = ref.ops()
    assert full.ops() == ops
    assert lean.ops() == ops
    # the full logs survive a trimmed node table unchanged
    assert set(full.edges()) == set(ref.edges())
    assert full.nodes() == ref.nodes()
    keys = ("nodes", "waits", "launches", "copies", "host_waits", "streams", "active", "fused_members")
    s_ref, s_full, s_lean = ref.stats(), full.stats(), lean.stats()
    assert all(s_full[k] == s_ref[k] and s_lean[k] == s_ref[k] for k in keys)
    assert s_full["edges"] == s_ref["edges"]
    # reader sets: kept whole with the full logs, pruned with the op log only
    assert s_full["held_readers"] == s_ref["held_readers"]
    assert s_lean["held_readers"] <= s_ref["held_readers"]
    for c in (ref, full, lean):
        c.sync()
    # after a sync every element is retired: the op-log-only context drops
    # them all, and its running reader count returns to exactly zero
    assert lean.stats()["held_nodes"] == 0 and lean.stats()["held_readers"] == 0
    assert full.stats()["held_nodes"] == 0
    for c in (ref, full, lean):
        c.close()


def test_long_program_holds_its_active_window_only():
    """A serving-like program that never calls gdag_sync: each request writes
    its input, runs one kernel that also reads a shared resident table, and
    reads its output, which retires the request.  The node table and the
    shared table's reader set stay bounded instead of growing with every
    request."""
    trim = 256
    ctx = G.Context(backend="fake", trim_nodes=trim)
    k = G.gdag_kernel_register(ctx.h, "req", None, [SPEC] * 3)
    table = ctx.array(dev=0x100000, nbytes=NB)
    slots = [(ctx.array(dev=0x200000 + 0x1000 * i, nbytes=NB), ctx.array(dev=0x300000 + 0x1000 * i, nbytes=NB))
             for i in range(8)]
    peak_nodes = peak_readers = 0
    requests = 20000
    for i in range(requests):
        x, y = slots[i % len(slots)]
        ctx.write(x, None)
        G.gdag_launch(ctx.h, k, G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0,
                      [G.array_arg(table.handle, G.GDAG_MODE_IN), G.array_arg(x.handle, G.GDAG_MODE_IN),
                       G.array_arg(y.handle, G.GDAG_MODE_OUT)])
        ctx.read(y)
        if i % 97 == 0:
            s = ctx.stats()
            peak_nodes = max(peak_nodes, s["held_nodes"])
            peak_readers = max(peak_readers, s["held_readers"])
    s = ctx.stats()
    assert s["nodes"] == 3 * requests
    assert s["active"] == 0
    assert peak_nodes <= 2 * trim
    assert peak_readers <= 2 * trim
    ctx.close()


def test_edge_log_keeps_every_reader():
    """With the full logs kept, a writer after many readers still gets an
    edge from every one of them, dropped from the node table or not."""
    for level, kept in ((1, 50), (0, 0)):
        ctx = G.Context(backend="fake", record_log=level, trim_nodes=4)
        k1 = G.gdag_kernel_register(ctx.h, "k1", None, [SPEC])
        a = ctx.array(dev=0x10000, nbytes=NB)
        readers = 50
        for _ in range(readers):
            G.gdag_launch(ctx.h, k1, G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0,
                          [G.array_arg(a.handle, G.GDAG_MODE_IN)])
        # readers of one array never wait for each other: all still active
        assert ctx.stats()["held_nodes"] == readers
        ctx.sync()  # retires them all; the node table empties
        assert ctx.stats()["held_nodes"] == 0
        assert ctx.stats()["held_readers"] == kept
        w = G.gdag_launch(ctx.h, k1, G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0,
                          [G.array_arg(a.handle, G.GDAG_MODE_OUT)])
        assert w == readers
        if level == 1:
            assert {(s, d, k) for s, d, _, k in ctx.edges()} == {(r, w, G.GDAG_EDGE_WAR) for r in range(readers)}
        ctx.close()


def test_dropped_elements_read_as_complete():
    ctx = G.Context(backend="fake", trim_nodes=2)
    k1 = G.gdag_kernel_register(ctx.h, "k1", None, [SPEC])
    a = ctx.array(dev=0x10000, nbytes=NB)
    first = G.gdag_launch(ctx.h, k1, G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0,
                          [G.array_arg(a.handle, G.GDAG_MODE_INOUT)])
    ctx.read(a)  # a host wait: retires the launch
    for _ in range(8):
        G.gdag_launch(ctx.h, k1, G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0,
                      [G.array_arg(a.handle, G.GDAG_MODE_INOUT)])
    assert ctx.stats()["held_nodes"] < ctx.stats()["nodes"]
    assert ctx.done(first)
    with pytest.raises(G.GdagError):
        ctx.done(ctx.stats()["nodes"])  # not issued yet
    ctx.sync()
    ctx.close()


def test_log_levels_and_option_checks():
    lean = G.Context(backend="fake", record_log=2)
    k1 = G.gdag_kernel_register(lean.h, "k1", None, [SPEC])
    a = lean.array(dev=0x10000, nbytes=NB)
    G.gdag_launch(lean.h, k1, G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0,
                  [G.array_arg(a.handle, G.GDAG_MODE_INOUT)])
    assert [o[0] for o in lean.ops()] == [G.GDAG_OP_LAUNCH, G.GDAG_OP_RECORD]
    for export in (lean.edges, lean.nodes):
        with pytest.raises(G.GdagError) as e:
            export()
        assert e.value.code == G.GDAG_ERR_INVALID
    lean.close()
    for bad in ({"record_log": 3}, {"record_log": -1}, {"trim_nodes": -1}):
        with pytest.raises(G.GdagError) as e:
            G.Context(backend="fake", **bad)
        assert e.value.code == G.GDAG_ERR_INVALID
