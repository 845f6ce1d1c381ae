"""Brute-force dependency oracle (test infrastructure only; see package doc).

A program is a list of elements e_0 .. e_{L-1} (kernels, host writes, host
reads, library calls).  Each element is a dict ``{array_id: mode}`` with
``mode`` a bit set: ``R`` (read) and/or ``W`` (write).

Section III-A (dependency sets and the read-only rules of Fig. 3) in pairwise
form: for i < j both touching array a, with at least one of them writing a,
the edge (i, j, a) exists iff

* i writes a, j only reads a, and no k in (i, j) writes a            -> RAW
* i writes a, j writes a, and no k in (i, j) touches a at all        -> RAW if
  j also reads a, else WAW
* i only reads a, j writes a, and no k in (i, j) writes a            -> WAR

(a later writer depends on every reader since the previous writer, not on the
writer; a reader depends on the last writer only).  Every test of the edge
rule below scans the elements strictly between i and j; nothing is cached.
"""
from __future__ import annotations

R = 1
W = 2
RW = 3

RAW, WAR, WAW = 0, 1, 2
KIND_NAMES = {RAW: "RAW", WAR: "WAR", WAW: "WAW"}


def expected_edges(elems):
    """Set of (i, j, array, kind) for the program ``elems``."""
    edges = set()
    L = len(elems)
    for j in range(L):
        for a, mj in elems[j].items():
            for i in range(j):
                mi = elems[i].get(a)
                if mi is None:
                    continue
                between = [elems[k].get(a, 0) for k in range(i + 1, j)]
                if mi & W and mj == R:
                    if not any(m & W for m in between):
                        edges.add((i, j, a, RAW))
                elif mi & W and mj & W:
                    if not any(m != 0 for m in between):
                        edges.add((i, j, a, RAW if mj & R else WAW))
                elif mi == R and mj & W:
                    if not any(m & W for m in between):
                        edges.add((i, j, a, WAR))
    return edges


def conflict_pairs(elems):
    """Every (i, j), i < j, touching a common array with at least one write:
    the textbook serialisability constraints."""
    pairs = set()
    L = len(elems)
    for j in range(L):
        for i in range(j):
            for a, mj in elems[j].items():
                mi = elems[i].get(a)
                if mi is not None and ((mi | mj) & W):
                    pairs.add((i, j))
                    break
    return pairs


def closure(pairs, L):
    """Transitive closure of a set of (i, j) pairs, i < j, over L nodes."""
    succ = [set() for _ in range(L)]
    for i, j in pairs:
        succ[i].add(j)
    reach = [set() for _ in range(L)]
    for i in range(L - 1, -1, -1):
        r = set()
        for j in succ[i]:
            r.add(j)
            r |= reach[j]
        reach[i] = r
    return {(i, j) for i in range(L) for j in reach[i]}


# ----------------------------------------------------------------------------
# Happens-before replay of recorded runtime operations.
#
# Op types (numbering of the C ABI's gdag_op.type):
OP_LAUNCH, OP_COPY_H2D, OP_COPY_D2H, OP_EXTERNAL = 0, 1, 2, 3
OP_RECORD, OP_WAIT = 4, 5
OP_HOST_WAIT, OP_STREAM_SYNC, OP_HOST_NODE, OP_QUERY_DONE = 6, 7, 8, 9
WORK_OPS = (OP_LAUNCH, OP_COPY_H2D, OP_COPY_D2H, OP_EXTERNAL)


def happens_before(ops):
    """Ancestor bitsets of every op, from CUDA's ordering rules only:

    * ops on one stream run in issue order;
    * a WAIT on event e orders everything up to the latest RECORD of e issued
      before the WAIT ahead of everything after the WAIT on its stream;
    * a HOST_WAIT on e (or a STREAM_SYNC of s) returns only after the latest
      RECORD of e (the last op on s) completed; the host issues everything
      after it later, and host-only elements (HOST_NODE) run at issue time;
    * a QUERY_DONE on e is a non-blocking query that found the latest RECORD
      of e complete: for ordering it is a host wait that did not block.

    ``ops`` is a list of tuples (type, stream, event, node) in issue order.
    Returns ``anc`` with bit p of anc[q] set iff op p happens before op q."""
    anc = [0] * len(ops)
    last_on_stream = {}
    last_record = {}
    host_frontier = None
    for q, (t, s, e, _node) in enumerate(ops):
        preds = []
        if host_frontier is not None:
            preds.append(host_frontier)
        if t in WORK_OPS or t in (OP_RECORD, OP_WAIT):
            if s in last_on_stream:
                preds.append(last_on_stream[s])
            if t == OP_WAIT and e in last_record:
                preds.append(last_record[e])
        elif t in (OP_HOST_WAIT, OP_QUERY_DONE):
            if e in last_record:
                preds.append(last_record[e])
        elif t == OP_STREAM_SYNC:
            if s in last_on_stream:
                preds.append(last_on_stream[s])
        a = 0
        for p in preds:
            a |= anc[p] | (1 << p)
        anc[q] = a
        if t in WORK_OPS or t in (OP_RECORD, OP_WAIT):
            last_on_stream[s] = q
        if t == OP_RECORD:
            last_record[e] = q
        if t in (OP_HOST_WAIT, OP_STREAM_SYNC, OP_HOST_NODE, OP_QUERY_DONE):
            host_frontier = q
    return anc


def node_ops(ops):
    """node id -> index of the op that performs that node's work."""
    out = {}
    for q, (t, _s, _e, node) in enumerate(ops):
        if (t in WORK_OPS or t == OP_HOST_NODE) and node >= 0:
            out[node] = q
    return out


def check_hb(ops, edges):
    """Edges (i, j, ...) whose work ops are not ordered i before j.

    A host write fills the array's host view on the host when it is issued
    (its COPY_H2D then moves the view to the device), so a host read served
    from the view (a HOST_NODE) is ordered after an earlier host write by
    program order alone."""
    anc = happens_before(ops)
    where = node_ops(ops)
    bad = []
    for e in edges:
        i, j = e[0], e[1]
        if i not in where or j not in where:
            bad.append(e)
            continue
        if ops[where[i]][0] == OP_COPY_H2D and ops[where[j]][0] == OP_HOST_NODE and where[i] < where[j]:
            continue
        if not (anc[where[j]] >> where[i]) & 1:
            bad.append(e)
    return bad


def waits_off_edges(ops, edges):
    """WAITs that do not follow a true edge.

    Every WAIT issued on stream s is attributed to the next work op issued on
    s; the waited-on node (the node whose RECORD the WAIT matches) must be a
    parent of that op's node in ``edges``, and must run on another stream."""
    parents = {}
    for e in edges:
        parents.setdefault(e[1], set()).add(e[0])
    rec_node, rec_stream = {}, {}
    pending = {}
    bad = []
    for t, s, e, node in ops:
        if t == OP_RECORD:
            rec_node[e] = node
            rec_stream[e] = s
        elif t == OP_WAIT:
            pending.setdefault(s, []).append((rec_node.get(e), rec_stream.get(e), e))
        elif t in WORK_OPS:
            for pnode, pstream, ev in pending.pop(s, []):
                if pnode is None or pnode not in parents.get(node, ()) or pstream == s:
                    bad.append((pnode, node, ev))
    for s, lst in pending.items():
        for pnode, _pstream, ev in lst:
            bad.append((pnode, None, ev))
    return bad
