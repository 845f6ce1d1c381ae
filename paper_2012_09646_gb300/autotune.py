"""Per-kernel history and an autotuner built on it.

Section III-A keeps each kernel's execution history so that later scheduling
can use it; Section VI names block-size selection from previous executions as
the next step.  This module does both on top of the library's own timing
(``options.trace``):

``History``
    durations of every traced node, grouped by kernel name and launch shape.
``tune_launch``
    for a kernel that takes an explicit launch shape (the streaming and
    grid-stride kernels), time each candidate block size on the caller's own
    arguments and keep the fastest; the choice is cached per (kernel, sizes).
``tune_streams``
    for a DAG program, time its makespan under each stream-pool size and
    return the best (the pool size trades concurrency against contention).
``tune_fusion``
    for a kernel with a fused form, time a group of same-kind launches issued
    one by one (each its own DAG element, spread over streams) against one
    fused element, per member size; the largest size at which fusing is no
    slower is the fusion threshold the serving loop uses.
"""
from __future__ import annotations

import collections
import statistics

import torch

from . import gdag as G

_CACHE = {}


class History:
    """Durations (ms) per (kernel name, launch shape) from traced contexts,
    the most recent ``keep`` per key (a ring: a long-running process holds
    a bounded history, and old samples age out as conditions change)."""

    def __init__(self, keep=256):
        self.samples = collections.defaultdict(lambda: collections.deque(maxlen=keep))

    def add(self, key, ms):
        self.samples[key].append(ms)

    def add_trace(self, ctx, names):
        """``names``: node id -> (kernel name, shape key) for the nodes of
        interest; trace records of other nodes are ignored."""
        for node, _kind, _stream, t0, t1 in ctx.trace():
            if node in names:
                self.add(names[node], t1 - t0)

    def median(self, key):
        s = self.samples.get(key)
        return statistics.median(s) if s else None

    def best(self, name):
        """Shape key of kernel ``name`` with the lowest median duration."""
        keys = [k for k in self.samples if k[0] == name]
        return min(keys, key=self.median) if keys else None


def _key(name, args):
    return (name,) + tuple(getattr(a, "nbytes", a) if hasattr(a, "handle") else a for a in args)


def tune_launch(ctx, name, args, blocks=(128, 256, 512, 1024), waves=(1, 2, 4, 8), reps=5, device="cuda"):
    """Time `name(*args)` for each block size and grid (waves x SMs) and
    return (grid, block) of the fastest; cached per kernel and sizes.  Only
    for kernels whose launch shape is free (grid-stride kernels); shapes the
    kernel rejects are skipped."""
    key = _key(name, args)
    if key in _CACHE:
        return _CACHE[key]
    sms = torch.cuda.get_device_properties(torch.device(device)).multi_processor_count
    st = torch.cuda.Stream()
    best = None
    for b in blocks:
        for w in waves:
            g = sms * w * max(1, 1024 // b)
            try:  # a kernel may reject a launch shape (e.g. a block larger than it supports)
                ctx.launch_raw(name, *args, stream=st.cuda_stream, grid=(g, 1, 1), block=(b, 1, 1))
            except G.GdagError:
                continue
            ctx.launch_raw(name, *args, stream=st.cuda_stream, grid=(g, 1, 1), block=(b, 1, 1))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                ctx.launch_raw(name, *args, stream=st.cuda_stream, grid=(g, 1, 1), block=(b, 1, 1))
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            if best is None or ms < best[0]:
                best = (ms, (g, 1, 1), (b, 1, 1))
    _CACHE[key] = (best[1], best[2], best[0])
    return _CACHE[key]


def tune_streams(build, step, candidates=(1, 2, 4, 8, 16, 32), steps=10, policy=G.GDAG_POLICY_PARALLEL):
    """``build(ctx)`` -> program object, ``step(obj)`` issues one DAG.  Returns
    (best max_streams, {max_streams: ms per DAG})."""
    out = {}
    s0 = torch.cuda.Stream()
    for m in candidates:
        ctx = G.Context(policy=policy, max_streams=m)
        obj = build(ctx)
        for _ in range(2):
            step(obj)
        ctx.sync()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s0)
        ctx.fork(s0.cuda_stream)
        for _ in range(steps):
            step(obj)
        ctx.wait_all(s0.cuda_stream)
        e1.record(s0)
        torch.cuda.synchronize()
        out[m] = e0.elapsed_time(e1) / steps
        ctx.sync()
        ctx.close()
        del obj
    return min(out, key=out.get), out


def tune_fusion(name, make_member, sizes, group=8, reps=5, max_streams=16):
    """``make_member(ctx, n, i)`` -> the argument tuple of member i of size n
    (arrays registered on ctx; members must not conflict).  For each n in
    ``sizes``: ms per group of ``group`` members issued as separate elements
    (PARALLEL) and as one fused element.  Returns (threshold, {n: (separate
    ms, fused ms)}), threshold = the largest n at which the fused group is no
    slower (0 if none)."""
    out = {}
    s0 = torch.cuda.Stream()
    for n in sizes:
        ms = []
        for fused in (False, True):
            ctx = G.Context(max_streams=max_streams)
            members = [make_member(ctx, n, i) for i in range(group)]

            def issue():
                if fused:
                    ctx.launch_fused(name, members)
                else:
                    for m in members:
                        ctx.launch(name, *m)
            for _ in range(2):
                issue()
            ctx.sync()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s0)
            ctx.fork(s0.cuda_stream)
            for _ in range(reps):
                issue()
            ctx.wait_all(s0.cuda_stream)
            e1.record(s0)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1) / reps)
            ctx.sync()
            ctx.close()
        out[n] = tuple(ms)
    ok = [n for n, (sep, fu) in out.items() if fu <= sep]
    return (max(ok) if ok else 0), out
