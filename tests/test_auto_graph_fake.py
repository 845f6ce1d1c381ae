"""Automatic capture of repeated gdag_issue sequences (options.auto_graph) on
the recording backend (CPU only).  A sequence issued auto_graph times is
captured into a graph and replayed from then on as one element whose
accesses are the union of the sequence's; the edge log must then be the
brute-force rule applied to the elements the library actually made (the
captured elements, which run nothing, and each replay element)."""
import random

import pytest

from oracle import dag as D
from paper_2012_09646_gb300 import gdag as G
from tests.test_issue_fake import ARR, I64, MODE_OF, kernel_args


def make_ctx(n_arrays, **opts):
    opts.setdefault("record_log", True)
    ctx = G.Context(backend="fake", **opts)
    arrays = [ctx.array(dev=0x10000 * (i + 1), nbytes=64, name="a%d" % i) for i in range(n_arrays)]
    kern = {n: "k%d" % n for n in range(1, 6)}
    for n, name in kern.items():
        kid = G.gdag_kernel_register(ctx.h, name, None, [ARR] * n + [I64])
        ctx._kernels[name] = (kid, G.gdag_kernel_signature(ctx.h, kid))
    return ctx, arrays, kern


def record(ctx, arrays, kern, seq, value=None):
    """A Program of seq: ("write", a) or ("kernel", [(a, mode)], scalar);
    the scalar is a Param "v" when value is given."""
    p = ctx.program()
    for e in seq:
        if e[0] == "write":
            p.write(arrays[e[1]])
        elif e[0] == "prefetch":
            p.prefetch_host(arrays[e[1]])
        else:
            p.launch(kern[len(e[1])], *kernel_args(arrays, e[1]), G.Param("v") if value is not None else e[2],
                     grid=(1, 1, 1), block=(32, 1, 1))
    return p


def accesses(seq):
    out = []
    for e in seq:
        if e[0] == "write":
            out.append({e[1]: D.W})
        elif e[0] == "prefetch":
            out.append({e[1]: D.R})
        else:
            acc = {}
            for a, m in e[1]:
                acc[a] = acc.get(a, 0) | m
            out.append(acc)
    return out


def union(accs):
    u = {}
    for acc in accs:
        for a, m in acc.items():
            u[a] = u.get(a, 0) | m
    return u


def kinds(ctx):
    return {i: k for i, k, _s in ctx.nodes()}


SEQ = [("write", 0), ("kernel", [(0, D.R), (1, D.W)], 3), ("kernel", [(1, D.R), (2, D.RW)], 4)]


def test_repeated_sequence_is_captured_then_replayed():
    ctx, arrays, kern = make_ctx(3, auto_graph=2)
    p = record(ctx, arrays, kern, SEQ)
    first = p.issue()
    assert first == [0, 1, 2]  # dynamic: one node per element
    second = p.issue()  # captured (nodes 3..5 record, run nothing), then replayed
    assert second == [6, 6, 6]
    k = kinds(ctx)
    assert k[6] == G.GDAG_NODE_GRAPH
    assert p.issue() == [7, 7, 7] and p.issue() == [8, 8, 8]
    assert kinds(ctx)[8] == G.GDAG_NODE_GRAPH
    # consecutive replays write the same arrays: they chain
    edges = {(s, d) for s, d, _a, _k in ctx.edges()}
    assert (6, 7) in edges and (7, 8) in edges
    # a later host read of an array the sequence writes waits for the replay
    ctx.read(arrays[2])
    assert (8, 9) in {(s, d) for s, d, _a, _k in ctx.edges()}
    ctx.close()


def test_threshold_one_captures_on_first_issue_and_zero_never():
    ctx, arrays, kern = make_ctx(3, auto_graph=1)
    p = record(ctx, arrays, kern, SEQ)
    assert p.issue() == [3, 3, 3]
    ctx.close()
    ctx, arrays, kern = make_ctx(3)  # auto_graph = 0
    p = record(ctx, arrays, kern, SEQ)
    for i in range(4):
        assert p.issue() == [3 * i, 3 * i + 1, 3 * i + 2]
    ctx.close()


def test_other_scalar_values_are_other_sequences():
    ctx, arrays, kern = make_ctx(3, auto_graph=2)
    p = record(ctx, arrays, kern, SEQ, value=True)
    assert p.issue(v=1) == [0, 1, 2]
    assert p.issue(v=2) == [3, 4, 5]  # another key: dynamic
    assert p.issue(v=1) == [9, 9, 9]  # the key of v=1 seen twice: captured (6..8), replayed
    assert p.issue(v=2) == [13, 13, 13]
    assert p.issue(v=1) == [14, 14, 14]
    ctx.close()


@pytest.mark.parametrize("opts", [{"policy": G.GDAG_POLICY_SERIAL_SYNC}, {"trace": True}])
def test_never_captured_under_serial_sync_or_tracing(opts):
    ctx, arrays, kern = make_ctx(3, auto_graph=1, **opts)
    p = record(ctx, arrays, kern, SEQ)
    for i in range(3):
        assert p.issue() == [3 * i, 3 * i + 1, 3 * i + 2]
    assert G.GDAG_NODE_GRAPH not in kinds(ctx).values()
    ctx.close()


def test_sequence_with_a_prefetch_is_never_captured():
    ctx, arrays, kern = make_ctx(3, auto_graph=1)
    p = record(ctx, arrays, kern, SEQ + [("prefetch", 2)])
    for _ in range(3):
        p.issue()
    assert G.GDAG_NODE_GRAPH not in kinds(ctx).values()
    ctx.close()


def test_moved_array_drops_the_graph_and_starts_over():
    ctx, arrays, kern = make_ctx(3, auto_graph=2)
    p = record(ctx, arrays, kern, SEQ)
    p.issue()
    assert p.issue() == [6, 6, 6]
    ctx.sync()
    ctx.unregister(arrays[1])
    b = ctx.array(dev=0x90000, nbytes=64)  # same handle, another address
    assert b.handle == arrays[1].handle
    # the stale graph is dropped: dynamic again, then captured anew
    assert p.issue() == [7, 8, 9]
    assert p.issue() == [13, 13, 13]
    assert kinds(ctx)[13] == G.GDAG_NODE_GRAPH
    ctx.close()


def test_least_recently_used_sequence_leaves_beyond_the_cap():
    ctx, arrays, kern = make_ctx(3, auto_graph=1)
    p = record(ctx, arrays, kern, SEQ, value=True)
    cap = G.GDAG_AUTO_GRAPH_SEQS
    nxt = 0
    for v in range(cap):  # every key captured at once: 3 recorded nodes + 1 replay
        assert p.issue(v=v) == [nxt + 3] * 3
        nxt += 4
    assert p.issue(v=0) == [nxt] * 3  # key 0 replayed: now the most recent
    nxt += 1
    assert p.issue(v=cap) == [nxt + 3] * 3  # a new key drops key 1 (least recent)
    nxt += 4
    assert p.issue(v=0) == [nxt] * 3  # still cached
    nxt += 1
    assert p.issue(v=1) == [nxt + 3] * 3  # captured again
    ctx.close()


@pytest.mark.parametrize("seed", range(30))
def test_edges_follow_the_rule_over_the_elements_made(seed):
    """Random interleavings of a few sequences (each issued several times),
    single host writes and reads: the edge log equals the brute-force edge
    set over the library's elements: each dynamic element, each captured
    element, and each replay with the union of its sequence's accesses."""
    rng = random.Random(seed)
    n_arrays = rng.randint(2, 5)
    ctx, arrays, kern = make_ctx(n_arrays, auto_graph=rng.randint(1, 3),
                                 max_streams=rng.choice([2, 16]))
    seqs = []
    for _ in range(rng.randint(1, 3)):
        seq = []
        for _ in range(rng.randint(1, 5)):
            if rng.random() < 0.2:
                seq.append(("write", rng.randrange(n_arrays)))
            else:
                k = rng.randint(1, min(4, n_arrays))
                seq.append(("kernel", [(a, rng.choice([D.R, D.W, D.RW])) for a in rng.sample(range(n_arrays), k)],
                            rng.randrange(5)))
        seqs.append((record(ctx, arrays, kern, seq), accesses(seq)))
    elems = []
    for _ in range(rng.randint(5, 25)):
        r = rng.random()
        if r < 0.15:
            a = rng.randrange(n_arrays)
            ctx.read(arrays[a])
            elems.append({a: D.R})
        elif r < 0.25:
            a = rng.randrange(n_arrays)
            ctx.write(arrays[a], None)
            elems.append({a: D.W})
        else:
            p, acc = rng.choice(seqs)
            before = len(elems)
            nodes = p.issue()
            made = max(nodes) + 1 - before
            if made == len(acc):            # dynamic
                assert nodes == list(range(before, before + len(acc)))
                elems += acc
            elif made == 1:                 # replay
                assert nodes == [before] * len(acc)
                elems.append(union(acc))
            else:                           # captured, then replayed
                assert made == len(acc) + 1 and nodes == [before + len(acc)] * len(acc)
                elems += acc
                elems.append(union(acc))
    assert len(ctx.nodes()) == len(elems)
    assert set(ctx.edges()) == D.expected_edges(elems)
    ctx.close()
