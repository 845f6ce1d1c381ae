"""Brute-force counterparts of the evaluation quantities (test
infrastructure only; see the package doc).

Overlaps (Section IV-F) on integer timelines: every unit time step of every
element is inspected and counted as overlapped if any other element of the
relevant class is running during that step.  Longest path (Section IV-E) by
enumerating every path of a small DAG."""
from __future__ import annotations


def overlaps_bruteforce(compute, transfer):
    def share(elems, other_sets):
        tot = 0
        hit = 0
        for k, (a, b) in enumerate(elems):
            for t in range(a, b):
                tot += 1
                if any(u <= t < v for (u, v) in other_sets(k)):
                    hit += 1
        return hit / tot if tot else 0.0

    allel = list(compute) + list(transfer)
    return {
        "CT": share(compute, lambda k: transfer),
        "TC": share(transfer, lambda k: compute),
        "CC": share(compute, lambda k: [c for i, c in enumerate(compute) if i != k]),
        "TOT": share(allel, lambda k: [c for i, c in enumerate(allel) if i != k]),
    }


def longest_path_bruteforce(weights, edges):
    succ = {}
    for e in edges:
        succ.setdefault(e[0], []).append(e[1])
    best = 0.0

    def walk(v, acc):
        nonlocal best
        acc += weights[v]
        best = max(best, acc)
        for w in succ.get(v, []):
            walk(w, acc)

    for v in range(len(weights)):
        walk(v, 0.0)
    return best
