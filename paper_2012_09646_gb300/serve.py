"""Serving loop over the run-time DAG scheduler.

Requests are DAG programs (VEC, B&S, IMG+ML, HITS) scaled by a factor s, and
they arrive as a Poisson stream.  One dispatcher thread does four things:

* admits queued requests in arrival order while their working set fits the
  HBM budget (continuous batching: a request admitted while others run simply
  adds nodes to the same context; independent requests share no arrays, so
  the scheduler puts them on separate streams and they overlap on the GPU);
* issues each admitted request's elements without blocking, ending with a
  device-to-host prefetch of the response;
* polls in-flight requests with a non-blocking node query, reads the response
  of each one that finished (served from the prefetched host view), and
  releases its memory;
* records each request's latency, from its arrival time to the moment all
  of its work has completed and its response is on the host.  A request is
  complete when its sinks are: the response prefetch plus every node of the
  request that is not an ancestor of it (the other nine B&S outputs, the ML
  branch beside the image, the last hub update of HITS).

Requests admitted in the same dispatcher pass are issued together.  With
fusion on, the small same-kind nodes of a VEC or B&S group (at most
``fuse_max[kind]`` elements each) become one fused element per node kind
(``gdag_launch_fused``: one persistent launch for the whole group), so a
burst of small requests costs a few launches instead of a few per request.
Each member's result is bit-identical to its unfused launch.

Inputs that a request only reads (price books, images, feature matrices,
graphs) are resident per scale bucket and shared by every request of that
bucket.  A response is the head of the request's result (at most
``RESPONSE_BYTES``); the rest of the result stays on the device.
"""
from __future__ import annotations

import collections
import math
import time

import numpy as np
import torch

from . import gdag as G
from . import workloads as W

KINDS = ("VEC", "B&S", "IMG+ML", "HITS")
RESPONSE_BYTES = 64 * 1024
F32 = torch.float32


class Inputs:
    """Read-only inputs per (kind, bucket), generated once and resident."""

    def __init__(self, datagen, scales, kinds=KINDS, device="cuda", hits_full=(10_000_000, 50_000_000),
                 full=None):
        """``full``: already generated full-scale inputs to reuse for s = 1
        (keys "bs", "img", "ml", "hits" as the benchmark builds them).
        ``device="cpu"`` keeps everything in ordinary host memory (for
        driving the dispatcher on the recording backend, which computes
        nothing)."""
        self.scales = scales
        pin = (lambda t: t.pin_memory()) if device != "cpu" else (lambda t: t)
        self.data = {}
        full = full or {}
        for s in scales:
            if s == 1.0 and full:
                self._from_full(full, kinds, device, pin)
                continue
            if "VEC" in kinds:
                n = max(1, int(1_000_000 * s))
                x, y = datagen.vec_inputs(n, seed=10)
                hx = pin(torch.from_numpy(x))
                hy = pin(torch.from_numpy(y))
                self.data[("VEC", s)] = {"n": n, "hx": hx, "hy": hy}
            if "B&S" in kinds:
                n = max(4, int(10_000_000 * s))
                S = [torch.from_numpy(p).to(device) for p in datagen.bs_inputs(n, count=10, seed=11)]
                self.data[("B&S", s)] = {"n": n, "S": S}
            if "IMG+ML" in kinds:
                side = max(8, int(4096 * math.sqrt(s)) // 8 * 8)
                img = torch.from_numpy(datagen.image(side, side, seed=12).reshape(-1)).to(device)
                rows = max(1, int(100_000 * s))
                X, T1, b1, T2, b2 = datagen.ml_inputs(rows, feats=1024, classes=10, seed=13)
                t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
                self.data[("IMG+ML", s)] = {"side": side, "img": img, "rows": rows, "X": t(X), "T1": t(T1),
                                            "b1": t(b1), "T2": t(T2), "b2": t(b2)}
            if "HITS" in kinds:
                n = max(64, int(hits_full[0] * s))
                nnz = max(64, int(hits_full[1] * s))
                csr, csc = datagen.hits_graph(n, nnz, seed=14)
                i32 = torch.int32
                d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dt).to(device)
                self.data[("HITS", s)] = {"n": n, "nnz": nnz,
                                          "A": (d(csr[0], i32), d(csr[1], i32), d(csr[2], F32)),
                                          "AT": (d(csc[0], i32), d(csc[1], i32), d(csc[2], F32))}

    def _from_full(self, full, kinds, device, pin):
        import datagen
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        if "VEC" in kinds:
            x, y = datagen.vec_inputs(1_000_000, seed=10)
            self.data[("VEC", 1.0)] = {"n": 1_000_000, "hx": pin(torch.from_numpy(x)),
                                       "hy": pin(torch.from_numpy(y))}
        if "B&S" in kinds:
            self.data[("B&S", 1.0)] = {"n": full["bs"][0].size, "S": [t(p) for p in full["bs"]]}
        if "IMG+ML" in kinds:
            X, T1, b1, T2, b2 = full["ml"]
            self.data[("IMG+ML", 1.0)] = {"side": 4096, "img": full["img"].to(device), "rows": X.shape[0],
                                          "X": t(X), "T1": t(T1), "b1": t(b1), "T2": t(T2), "b2": t(b2)}
        if "HITS" in kinds:
            csr, csc = full["hits"]
            i32 = torch.int32
            d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dt).to(device)
            self.data[("HITS", 1.0)] = {"n": len(csr[0]) - 1, "nnz": int(csr[0][-1]),
                                        "A": (d(csr[0], i32), d(csr[1], i32), d(csr[2], F32)),
                                        "AT": (d(csc[0], i32), d(csc[1], i32), d(csc[2], F32))}

    def bucket(self, s):
        for b in self.scales:
            if s <= b * (1 + 1e-12):
                return b
        return self.scales[-1]


class Request:
    """One DAG submission.  ``done_at`` is set when it completes or fails;
    ``error`` is then None or the GdagError that failed it."""

    __slots__ = ("rid", "kind", "scale", "arrival", "admitted", "done_at", "bytes", "sinks", "tensors", "arrays",
                 "resp", "resp_view", "slot", "scratch", "need", "error")

    def __init__(self, rid, kind, scale, arrival):
        self.rid, self.kind, self.scale, self.arrival = rid, kind, scale, arrival
        self.admitted = self.done_at = None
        self.bytes = 0
        self.sinks = []
        self.tensors, self.arrays = [], []
        self.resp = None
        self.resp_view = None
        self.slot = None
        self.scratch = []
        self.need = 0
        self.error = None


class Server:
    """One gdag context shared by every request."""

    def __init__(self, inputs, budget_bytes=40 << 30, max_streams=32, device="cuda", fuse_max=None, backend="cuda",
                 record_log=False, fake_fail_op=-1, fake_fail_sticky=False, fake_complete=None,
                 request_timeout_s=120.0, trim_nodes=0):
        """``fuse_max``: {kind: largest node size (elements) that is fused
        across requests}; None or {} turns fusion off.  ``backend="fake"``
        (with ``device="cpu"``) runs the dispatcher on the recording backend:
        admission, batching and bookkeeping without a GPU (every node
        reports complete when queried; nothing is computed), and
        ``fake_fail_op`` / ``fake_fail_sticky`` / ``fake_complete`` inject
        a failure or a device that never completes there.
        ``request_timeout_s``: a request still incomplete this long after
        its admission means the device has stopped making progress; run()
        then raises GDAG_ERR_TIMEOUT instead of polling forever (None: no
        limit).  ``trim_nodes``: the context's node-table threshold for
        dropping retired elements (0: the library default)."""
        self.inp = inputs
        self.fuse_max = dict(fuse_max or {})
        self.budget = budget_bytes
        self.used = 0
        self.device = device
        self.ctx = G.Context(max_streams=max_streams, retire_by_query=True, backend=backend,
                             fake_complete=(backend == "fake") if fake_complete is None else fake_complete,
                             record_log=record_log, fake_fail_op=fake_fail_op, fake_fail_sticky=fake_fail_sticky,
                             trim_nodes=trim_nodes)
        self.request_timeout_s = request_timeout_s
        self.shared = {}
        self._slots = []  # pinned response buffers, reused
        self._scratch_pool = {}
        self._need = {}  # (kind, bucket) -> working bytes
        self.partitions = {}

    # ---------------------------------------------------------- helpers
    def _arr(self, r, t, host=None, name=None):
        r.tensors.append(t)
        a = self.ctx.array(t, host=host, name=name)
        r.arrays.append(a)
        r.bytes += t.numel() * t.element_size()
        return a

    def _shared(self, key, t):
        """Register a resident read-only input once."""
        k = (key, t.data_ptr())
        if k not in self.shared:
            self.shared[k] = self.ctx.array(t)
        return self.shared[k]

    def _zeroed(self, r, nbytes):
        """Reduction scratch from a pool: zeroed once when created (the
        kernels leave their arrival counters at zero), so serving issues no
        fill kernels that would order behind in-flight requests."""
        pool = self._scratch_pool.setdefault(nbytes, [])
        if pool:
            t, a = pool.pop()
        else:
            t = torch.zeros(nbytes, dtype=torch.uint8, device=self.device)
            a = self.ctx.array(t)
        r.scratch.append((nbytes, t, a))
        r.bytes += nbytes
        return a

    def _slot(self):
        if self._slots:
            return self._slots.pop()
        return torch.empty(RESPONSE_BYTES // 4, dtype=F32, pin_memory=self.device != "cpu")

    def working_bytes(self, r):
        """Bytes of the private arrays and scratch a request will allocate
        (exactly what issue() adds up in r.bytes), per kind and bucket."""
        key = (r.kind, self.inp.bucket(r.scale))
        got = self._need.get(key)
        if got is None:
            d = self.inp.data[key]
            S = G.gdag_scratch_bytes
            if r.kind == "VEC":
                n = d["n"]
                got = 2 * 4 * n + 4 + S("vec_reduce_diff", n)           # x, y, z, scratch
            elif r.kind == "B&S":
                got = 10 * 4 * d["n"]                                  # ten price outputs
            elif r.kind == "IMG+ML":
                n, rows = d["side"] ** 2, d["rows"]
                got = (6 * 4 * n + 2 * 8 + 2 * S("minmax", n)          # five images, output, min/max pairs
                       + 2 * 4 * rows * 10 + 4 * rows)                 # two score tables, labels
            else:
                n, nnz = d["n"], d["nnz"]
                got = (4 * 4 * n + 2 * 4 + 2 * S("l2norm", n)          # ping-pong vectors, norms
                       + 2 * S("spmv_csr", n + nnz))                   # carries
            self._need[key] = got
        return got

    # ----------------------------------------------------------- issue
    def issue(self, r):
        """Issue every element of request r (never blocks)."""
        c = self.ctx
        b = self.inp.bucket(r.scale)
        d = self.inp.data[(r.kind, b)]
        dev = self.device
        r.slot = self._slot()
        tails = []  # nodes of r that are not ancestors of its response prefetch
        if r.kind == "VEC":
            n = d["n"]
            X = self._arr(r, torch.empty(n, dtype=F32, device=dev), host=d["hx"])
            Y = self._arr(r, torch.empty(n, dtype=F32, device=dev), host=d["hy"])
            Z = self._arr(r, torch.empty(1, dtype=F32, device=dev), host=r.slot)
            S = self._zeroed(r, G.gdag_scratch_bytes("vec_reduce_diff", n))
            c.write(X, None, 0, 4 * n)
            c.write(Y, None, 0, 4 * n)
            c.launch("vec_square", X, n)
            c.launch("vec_square", Y, n)
            c.launch("vec_reduce_diff", X, Y, Z, S, n)
            r.resp = (Z, 4)
        elif r.kind == "B&S":
            n = d["n"]
            outs = []
            for i, St in enumerate(d["S"]):
                Sa = self._shared(("bs", b, i), St)
                Ca = self._arr(r, torch.empty(n, dtype=F32, device=dev), host=r.slot if i == 0 else None)
                k = c.launch("bs_call", Sa, Ca, n, 60.0, 0.1, 0.2, 1.0)
                if i:
                    tails.append(k)
                outs.append(Ca)
            r.resp = (outs[0], min(4 * n, RESPONSE_BYTES))
        elif r.kind == "IMG+ML":
            side, rows = d["side"], d["rows"]
            n = side * side
            IMG = self._shared(("img", b), d["img"])
            t = lambda: torch.empty(n, dtype=F32, device=dev)
            B5, B9, E5, E9, Sh = (self._arr(r, t()) for _ in range(5))
            OUT = self._arr(r, t(), host=r.slot)
            MM5 = self._arr(r, torch.empty(2, dtype=F32, device=dev))
            MM9 = self._arr(r, torch.empty(2, dtype=F32, device=dev))
            SC5 = self._zeroed(r, G.gdag_scratch_bytes("minmax", n))
            SC9 = self._zeroed(r, G.gdag_scratch_bytes("minmax", n))
            w5, w9 = self._weights()
            c.launch("gauss_blur", IMG, B5, w5, side, side, 2)
            c.launch("gauss_blur", IMG, B9, w9, side, side, 4)
            c.launch("sobel", B5, E5, side, side)
            c.launch("sobel", B9, E9, side, side)
            c.launch("minmax", E5, MM5, SC5, n)
            c.launch("minmax", E9, MM9, SC9, n)
            c.launch("extend", E5, MM5, n)
            c.launch("extend", E9, MM9, n)
            c.launch("unsharp", IMG, B5, Sh, 0.5, n)
            c.launch("combine", Sh, B5, B9, E5, E9, OUT, n)
            XA = self._shared(("X", b), d["X"])
            T1, B1 = self._shared(("T1", b), d["T1"]), self._shared(("b1", b), d["b1"])
            T2, B2 = self._shared(("T2", b), d["T2"]), self._shared(("b2", b), d["b2"])
            S1 = self._arr(r, torch.empty(rows * 10, dtype=F32, device=dev))
            S2 = self._arr(r, torch.empty(rows * 10, dtype=F32, device=dev))
            LAB = self._arr(r, torch.empty(rows, dtype=torch.int32, device=dev))
            c.launch("dense_scores", XA, T1, B1, S1, rows, 1024, 10)
            c.launch("dense_scores", XA, T2, B2, S2, rows, 1024, 10)
            c.launch("row_softmax", S1, rows, 10)
            c.launch("row_softmax", S2, rows, 10)
            tails.append(c.launch("argmax_combine", S1, S2, LAB, rows, 10))
            # the response: the head of the combined image (the labels stay
            # on the device)
            r.resp = (OUT, min(4 * n, RESPONSE_BYTES))
        else:
            n, nnz = d["n"], d["nnz"]
            A = [self._shared(("A", b, i), t) for i, t in enumerate(d["A"])]
            AT = [self._shared(("AT", b, i), t) for i, t in enumerate(d["AT"])]
            PA, PAT = self._partitions(b, A, AT, n, nnz)
            v = {k: self._arr(r, torch.empty(n, dtype=F32, device=dev), host=r.slot if k == "a2" else None)
                 for k in ("a", "h", "a2", "h2")}
            NA = self._arr(r, torch.empty(1, dtype=F32, device=dev))
            NH = self._arr(r, torch.empty(1, dtype=F32, device=dev))
            SA = self._zeroed(r, G.gdag_scratch_bytes("l2norm", n))
            SH = self._zeroed(r, G.gdag_scratch_bytes("l2norm", n))
            cb = G.gdag_scratch_bytes("spmv_csr", n + nnz)
            CA = self._arr(r, torch.empty(cb, dtype=torch.uint8, device=dev))  # fully written before read
            CAT = self._arr(r, torch.empty(cb, dtype=torch.uint8, device=dev))
            ones = self._ones(n)  # a_0 = h_0 = 1: a shared, read-only vector
            cur = (ones, ones)
            bufs = [(v["a2"], v["h2"]), (v["a"], v["h"])]
            for it in range(5):
                a_in, h_in = cur
                a_out, h_out = bufs[it % 2]
                c.launch("spmv_csr", *AT, h_in, PAT, a_out, CAT, n, nnz)
                c.launch("spmv_csr", *A, a_in, PA, h_out, CA, n, nnz)
                c.launch("l2norm", a_out, NA, SA, n)
                c.launch("l2norm", h_out, NH, SH, n)
                c.launch("scale", a_out, NA, n)
                k = c.launch("scale", h_out, NH, n)
                cur = (a_out, h_out)
            tails.append(k)  # the last hub update
            # 5 iterations end in the first buffer pair (a2, h2)
            r.resp = (v["a2"], min(4 * n, RESPONSE_BYTES))
        self._finish_issue(r, tails)

    def _fusable(self, r):
        lim = self.fuse_max.get(r.kind)
        if lim is None or r.kind not in ("VEC", "B&S"):
            return False
        return self.inp.data[(r.kind, self.inp.bucket(r.scale))]["n"] <= lim

    def issue_batch(self, rs):
        """Issue the requests admitted in one pass: fusable VEC and B&S
        requests as fused groups (when two or more share a kind), the rest
        one by one.  A call that fails fails the requests it was issuing
        (all members of a fused group) and no others."""
        groups = {"VEC": [], "B&S": []}
        for r in rs:
            if self._fusable(r):
                groups[r.kind].append(r)
            else:
                self._guarded([r], self.issue, r)
        for kind, g in groups.items():
            if len(g) == 1:
                self._guarded(g, self.issue, g[0])
            elif g:
                self._guarded(g, self._issue_vec_group if kind == "VEC" else self._issue_bs_group, g)

    def _guarded(self, rs, fn, arg):
        """fn(arg); on a library error the requests `rs` fail: they get no
        sinks, so the dispatcher finishes them at once (finish() releases
        what they hold).  An error that poisoned the context is raised:
        nothing further can run on it."""
        try:
            fn(arg)
        except G.GdagError as e:
            if e.code == G.GDAG_ERR_POISONED:
                raise
            for r in rs:
                r.error = e
                r.sinks = []

    def _issue_vec_group(self, g):
        c = self.ctx
        sq, red = [], []
        for r in g:
            d = self.inp.data[("VEC", self.inp.bucket(r.scale))]
            n = d["n"]
            r.slot = self._slot()
            X = self._arr(r, torch.empty(n, dtype=F32, device=self.device), host=d["hx"])
            Y = self._arr(r, torch.empty(n, dtype=F32, device=self.device), host=d["hy"])
            Z = self._arr(r, torch.empty(1, dtype=F32, device=self.device), host=r.slot)
            S = self._zeroed(r, G.gdag_scratch_bytes("vec_reduce_diff", n))
            c.write(X, None, 0, 4 * n)
            c.write(Y, None, 0, 4 * n)
            sq += [(X, n), (Y, n)]
            red.append((X, Y, Z, S, n))
            r.resp = (Z, 4)
        c.launch_fused("vec_square", sq)
        c.launch_fused("vec_reduce_diff", red)
        for r in g:
            self._finish_issue(r)

    def _issue_bs_group(self, g):
        members = []
        for r in g:
            b = self.inp.bucket(r.scale)
            d = self.inp.data[("B&S", b)]
            n = d["n"]
            r.slot = self._slot()
            outs = []
            for i, St in enumerate(d["S"]):
                Sa = self._shared(("bs", b, i), St)
                Ca = self._arr(r, torch.empty(n, dtype=F32, device=self.device), host=r.slot if i == 0 else None)
                members.append((Sa, Ca, n, 60.0, 0.1, 0.2, 1.0))
                outs.append(Ca)
            r.resp = (outs[0], min(4 * n, RESPONSE_BYTES))
        self.ctx.launch_fused("bs_call", members)
        for r in g:
            self._finish_issue(r)

    def _finish_issue(self, r, tails=()):
        """Issue r's response prefetch and set its sinks (in a fused group
        every member's nodes are ancestors of its prefetch)."""
        arr, nb = r.resp
        self.ctx.prefetch_host(arr, 0, nb)
        r.sinks = list(tails) + [self._last_node()]

    def _last_node(self):
        return G.gdag_stats_get(self.ctx.h).nodes - 1

    def _weights(self):
        if "w" not in self.shared:
            w5 = W.gaussian_weights(2, 1.0).to(self.device)
            w9 = W.gaussian_weights(4, 2.0).to(self.device)
            self.shared["w_t"] = (w5, w9)
            self.shared["w"] = (self.ctx.array(w5), self.ctx.array(w9))
        return self.shared["w"]

    def _ones(self, n):
        key = ("ones", n)
        if key not in self.shared:
            t = torch.ones(n, dtype=F32, device=self.device)
            self.shared[key + ("t",)] = t
            self.shared[key] = self.ctx.array(t)
        return self.shared[key]

    def _partitions(self, b, A, AT, n, nnz):
        if b not in self.partitions:
            pb = G.gdag_scratch_bytes("spmv_partition", n + nnz)
            pa = torch.zeros(pb, dtype=torch.uint8, device=self.device)
            pat = torch.zeros(pb, dtype=torch.uint8, device=self.device)
            PA, PAT = self.ctx.array(pa), self.ctx.array(pat)
            self.ctx.launch("spmv_partition", A[0], PA, n, nnz)
            self.ctx.launch("spmv_partition", AT[0], PAT, n, nnz)
            self.partitions[b] = (PA, PAT, pa, pat)
        return self.partitions[b][:2]

    # ------------------------------------------------------------ finish
    def finish(self, r, now):
        if r.error is None:
            arr, nb = r.resp
            self.ctx.read(arr, None, 0, nb)  # served from the completed prefetch
            r.resp_view = r.slot[: nb // 4].clone() if nb >= 4 else None
        r.done_at = now
        # unregistering waits for the request's elements that use an array,
        # also those a failed request had issued before its error
        for a in r.arrays:
            self.ctx.unregister(a)
        r.arrays.clear()
        r.tensors.clear()
        for nbytes, t, a in r.scratch:
            if r.error is None:
                self._scratch_pool[nbytes].append((t, a))
            else:  # a failed reduction may have left its counter nonzero
                self.ctx.unregister(a)
        r.scratch.clear()
        if r.slot is not None:
            self._slots.append(r.slot)
        r.slot = None
        self.used -= r.need

    def warm(self, kinds=KINDS):
        """Build the per-bucket shared state (partitions, weights) once."""
        for s in self.inp.scales:
            for k in kinds:
                if (k, s) in self.inp.data:
                    r = Request(-1, k, s, 0.0)
                    self.issue(r)
                    self.ctx.sync()
                    self.finish(r, 0.0)

    def run(self, requests, clock=time.perf_counter, spin=True):
        """Serve a list of requests (sorted by arrival, seconds from start)."""
        pending = collections.deque()
        inflight = []
        i = 0
        t0 = clock()
        done = 0
        while done < len(requests):
            now = clock() - t0
            while i < len(requests) and requests[i].arrival <= now:
                pending.append(requests[i])
                i += 1
            batch = []
            while pending:
                r = pending[0]
                need = self.working_bytes(r)
                if (inflight or batch) and self.used + need > self.budget:
                    break
                pending.popleft()
                r.admitted = now
                r.need = need  # released on completion: the same figure
                self.used += need
                batch.append(r)
            if batch:
                self.issue_batch(batch)
                inflight.extend(batch)
            still = []
            for r in inflight:
                while r.sinks and self.ctx.done(r.sinks[-1]):
                    r.sinks.pop()
                if not r.sinks:
                    self.finish(r, clock() - t0)
                    done += 1
                else:
                    still.append(r)
            inflight = still
            if inflight and self.request_timeout_s is not None:
                late = clock() - t0 - self.request_timeout_s
                for r in inflight:
                    if r.admitted < late:
                        raise G.GdagError(G.GDAG_ERR_TIMEOUT, "request %d (%s) incomplete %.1f s after admission"
                                          % (r.rid, r.kind, self.request_timeout_s))
            if not inflight and not pending and i < len(requests):
                # idle until the next arrival
                wait = requests[i].arrival - (clock() - t0)
                if wait > 0 and not spin:
                    time.sleep(wait)
        return requests

    def close(self):
        self.ctx.sync()
        self.ctx.close()


def poisson_requests(rate, count, scales, seed=0, kinds=KINDS):
    """Arrival times of a Poisson stream of `rate` req/s; kinds uniform;
    scale s ~ U[1/64, 1]."""
    g = np.random.default_rng(seed)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    out = []
    for k in range(count):
        kind = kinds[int(g.integers(0, len(kinds)))]
        s = float(g.uniform(1.0 / 64, 1.0))
        out.append(Request(k, kind, s, float(t[k])))
    return out


def latency_summary(reqs):
    failed = sum(r.error is not None for r in reqs)
    reqs = [r for r in reqs if r.error is None]
    lat = np.array([(r.done_at - r.arrival) * 1e3 for r in reqs])
    span = max(r.done_at for r in reqs) - min(r.arrival for r in reqs)
    by = {}
    for k in sorted({r.kind for r in reqs}):
        l = np.array([(r.done_at - r.arrival) * 1e3 for r in reqs if r.kind == k])
        by[k] = {"n": int(l.size), "p50_ms": float(np.percentile(l, 50)), "p99_ms": float(np.percentile(l, 99))}
    return {"requests": len(reqs), "failed": failed,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "throughput_req_s": len(reqs) / span, "by_kind": by}
