"""Evaluation quantities of Sections IV-E and IV-F, computed from what the
library records.

critical_path
    The contention-free bound of Section IV-E: the longest path through the
    DAG when every node takes the time it takes alone on the GPU.
overlap_metrics
    The overlaps of Section IV-F over an execution timeline: CT (share of
    computation time that overlaps any transfer), TC (share of transfer time
    that overlaps any computation), CC (share of computation time that
    overlaps other computation) and TOT (share of all time, computation and
    transfer, that overlaps anything else).  Each element's overlapped time is
    counted once however many others it overlaps (the union of the overlap
    intervals), then summed over elements and divided by their total time.
"""
from __future__ import annotations


def critical_path(weights, edges):
    """Longest path weight; ``weights[i]`` per node, ``edges`` (i, j, ...)
    with i < j (program order is a topological order)."""
    n = len(weights)
    preds = [[] for _ in range(n)]
    for e in edges:
        preds[e[1]].append(e[0])
    finish = [0.0] * n
    for j in range(n):
        start = max((finish[i] for i in preds[j]), default=0.0)
        finish[j] = start + weights[j]
    return max(finish, default=0.0)


def _union(intervals):
    out = []
    for a, b in sorted(intervals):
        if b <= a:
            continue
        if out and a <= out[-1][1]:
            out[-1][1] = max(out[-1][1], b)
        else:
            out.append([a, b])
    return out


def _covered(interval, union):
    """Length of ``interval`` covered by a sorted disjoint union."""
    a, b = interval
    s = 0.0
    for u, v in union:
        lo, hi = max(a, u), min(b, v)
        if hi > lo:
            s += hi - lo
    return s


def _share(elems, others_of):
    total = sum(b - a for a, b in elems)
    if total <= 0:
        return 0.0
    return sum(_covered(e, _union(others_of(k))) for k, e in enumerate(elems)) / total


def overlap_metrics(compute, transfer):
    """``compute`` and ``transfer``: lists of (start, end).  Returns a dict
    with CT, TC, CC and TOT as fractions in [0, 1]."""
    compute = [tuple(x) for x in compute]
    transfer = [tuple(x) for x in transfer]
    allel = compute + transfer
    return {
        "CT": _share(compute, lambda k: transfer),
        "TC": _share(transfer, lambda k: compute),
        "CC": _share(compute, lambda k: compute[:k] + compute[k + 1:]),
        "TOT": _share(allel, lambda k: allel[:k] + allel[k + 1:]),
    }
