"""Pins of the brute-force dependency oracle: the paper's worked cases
(Section III-A, Fig. 3 and the VEC example) and the textbook serialisability
condition (the closure of the edge set equals the closure of all conflicting
pairs).  CPU only."""
import os
import random

import pytest

from oracle import dag as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
_MODES = {"R": D.R, "W": D.W, "RW": D.RW}
_KINDS = {"RAW": D.RAW, "WAR": D.WAR, "WAW": D.WAW}


def load_cases(name="fig3_read_only_rules.txt"):
    cases, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"elems": [], "edges": set()}
                cases[tok[1]] = cur
            elif tok[0] == "edge":
                cur["edges"].add((int(tok[1]), int(tok[2]), tok[3], _KINDS[tok[4]]))
            elif tok[0] == "end":
                cur = None
            else:
                cur["elems"].append({a: _MODES[m] for a, m in (t.split(":") for t in tok[1:])})
    return cases


CASES = load_cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_paper_worked_cases(name):
    c = CASES[name]
    assert D.expected_edges(c["elems"]) == c["edges"]


def random_program(rng, L, n_arrays):
    elems = []
    for _ in range(L):
        k = rng.randint(1, min(4, n_arrays))
        arrs = rng.sample(range(n_arrays), k)
        elems.append({a: rng.choice([D.R, D.W, D.RW, D.R]) for a in arrs})
    return elems


def test_closure_equals_full_conflict_closure():
    rng = random.Random(0)
    for _ in range(300):
        L = rng.randint(1, 25)
        elems = random_program(rng, L, rng.randint(1, 5))
        e = D.expected_edges(elems)
        pairs = {(i, j) for i, j, _a, _k in e}
        conf = D.conflict_pairs(elems)
        assert pairs <= conf
        assert D.closure(pairs, L) == D.closure(conf, L)


def test_dropping_any_edge_breaks_closure():
    """Every edge is needed: removing it loses some conflict ordering unless
    another path already implies it (then the closure is unchanged)."""
    rng = random.Random(1)
    for _ in range(100):
        L = rng.randint(2, 15)
        elems = random_program(rng, L, 3)
        e = D.expected_edges(elems)
        pairs = {(i, j) for i, j, _a, _k in e}
        conf_cl = D.closure(D.conflict_pairs(elems), L)
        for p in pairs:
            rest = pairs - {p}
            if p not in D.closure(rest, L):
                assert D.closure(rest, L) != conf_cl


def test_happens_before_rules():
    L, C, H, REC, WT, HW = D.OP_LAUNCH, D.OP_COPY_H2D, D.OP_HOST_NODE, D.OP_RECORD, D.OP_WAIT, D.OP_HOST_WAIT
    ops = [
        (C, 0, -1, 0),    # 0: node 0 on stream 0
        (REC, 0, 5, 0),   # 1
        (L, 1, -1, 1),    # 2: node 1 on stream 1 (unordered with node 0)
        (REC, 1, 6, 1),   # 3
        (WT, 1, 5, -1),   # 4: stream 1 waits node 0
        (L, 1, -1, 2),    # 5: node 2 after nodes 0 and 1
        (HW, -1, 6, -1),  # 6: host waits node 1
        (H, -1, -1, 3),   # 7: host node 3
        (L, 0, -1, 4),    # 8: node 4 on stream 0
    ]
    anc = D.happens_before(ops)
    hb = lambda p, q: bool((anc[q] >> p) & 1)
    assert not hb(0, 2) and not hb(2, 0)
    assert hb(0, 5) and hb(2, 5)
    assert hb(2, 7) and not hb(0, 7)
    assert hb(2, 8) and hb(7, 8) and hb(0, 8)
    assert not hb(5, 8)
    assert D.check_hb(ops, {(0, 2), (1, 2), (1, 3), (3, 4)}) == []
    assert D.check_hb(ops, {(2, 4)}) == [(2, 4)]
    assert D.waits_off_edges(ops, {(0, 2), (1, 2)}) == []
    assert D.waits_off_edges(ops, {(1, 2)}) == [(0, 2, 5)]


def test_hazard_labels_follow_the_textbook_classes():
    """Between a writer and the next element that writes the same array, the
    edge is a true (read-after-write) dependence when that element also
    reads the array, and an output (write-after-write) dependence when it
    only overwrites it; a reader after readers of a written value gives
    anti (write-after-read) dependences."""
    X = "X"
    assert D.expected_edges([{X: D.W}, {X: D.RW}]) == {(0, 1, X, D.RAW)}
    assert D.expected_edges([{X: D.RW}, {X: D.RW}]) == {(0, 1, X, D.RAW)}
    assert D.expected_edges([{X: D.W}, {X: D.W}]) == {(0, 1, X, D.WAW)}
    assert D.expected_edges([{X: D.RW}, {X: D.W}]) == {(0, 1, X, D.WAW)}
    assert D.expected_edges([{X: D.W}, {X: D.R}, {X: D.RW}]) == {(0, 1, X, D.RAW), (1, 2, X, D.WAR)}


def test_stream_sync_and_same_stream_waits():
    """A STREAM_SYNC orders everything issued on its stream before what the
    host issues next; a WAIT whose recorded parent runs on the waiting
    stream is not a cross-stream wait along an edge."""
    L, REC, WT, SS, H = D.OP_LAUNCH, D.OP_RECORD, D.OP_WAIT, D.OP_STREAM_SYNC, D.OP_HOST_NODE
    ops = [
        (L, 0, -1, 0),    # 0: node 0 on stream 0
        (L, 1, -1, 1),    # 1: node 1 on stream 1
        (SS, 0, -1, -1),  # 2: host syncs stream 0
        (H, -1, -1, 2),   # 3: host node 2
        (L, 2, -1, 3),    # 4: node 3 on stream 2
    ]
    anc = D.happens_before(ops)
    hb = lambda p, q: bool((anc[q] >> p) & 1)
    assert hb(0, 3) and hb(0, 4) and hb(2, 4)
    assert not hb(1, 3) and not hb(1, 4)
    assert D.check_hb(ops, {(0, 2), (0, 3)}) == []
    assert D.check_hb(ops, {(1, 3)}) == [(1, 3)]
    same = [(L, 0, -1, 0), (REC, 0, 5, 0), (WT, 0, 5, -1), (L, 0, -1, 1)]
    assert D.waits_off_edges(same, {(0, 1)}) == [(0, 1, 5)]
    cross = [(L, 0, -1, 0), (REC, 0, 5, 0), (WT, 1, 5, -1), (L, 1, -1, 1)]
    assert D.waits_off_edges(cross, {(0, 1)}) == []
