"""Serving loop over the run-time DAG scheduler.

Requests are DAG programs of five kinds: VEC, B&S, IMG+ML and HITS, each
scaled by its own factor s ~ U[1/64, 1], and the DL convolution DAG at its
stated batch of 16 images.  They arrive as a Poisson stream, and one
dispatcher thread does four things:

* admits queued requests in arrival order while (1) a slot of the request's
  kind is free, or a new one fits the HBM budget (idle slots of other kinds
  are released to make room), and (2) the estimated GPU time of the
  admitted, unfinished requests stays within ``window_ms``.  This is
  continuous batching: an admitted request adds its elements to a shared
  context, and requests share no written array, so the scheduler puts them
  on separate streams and they overlap on the GPU.  The window keeps the
  device queue short, so that a request is not queued behind every request
  admitted before it.  With ``split_ms`` the requests form two classes by
  their estimated GPU time, each with its own queue (arrival order within
  the class), its own window and its own context; the short class's
  context runs on high-priority CUDA streams, so short requests neither
  wait behind a long one on the host nor behind its kernels on the GPU;
* issues each admitted request's whole program with one ``gdag_issue`` call
  (a recorded :class:`~.gdag.Program` whose sizes are bound per request),
  ending with a device-to-host prefetch of the response.  Requests admitted
  in the same pass are issued together, and with fusion on the small VEC and
  B&S nodes of such a group become one fused element per node kind
  (``gdag_launch_fused``: one persistent launch for the group);
* polls the sinks of every in-flight request with one ``gdag_nodes_query``
  call, reads the response of each finished request (served from the
  prefetched host view) and returns its slot to the pool;
* records each request's latency, from its arrival until all of its work has
  completed and its response is on the host.  It is split into queue wait
  (arrival to admission), host issue, and issue to completion.

A slot holds the private device arrays of one request of a kind at the
kind's full size, registered once with the context.  A request uses the
prefix its size needs.  Reusing a slot adds logical edges from the slot's
previous request, which has completed, so they cost no wait.

Inputs that a request only reads are resident and shared.  They are VEC's
pinned host vectors, B&S's ten price vectors, the IMG image and the ML
feature matrix (a request of scale s reads their first elements), the DL
batch, and HITS graphs at ``hits_buckets`` scales k/B (a request takes the
smallest one at least s).  The response is the head of the request's main
result, at most ``RESPONSE_BYTES``: the scalar z, the first price vector,
the combined image, the final authority vector, the logits.  The rest stays
on the device; with ``keep_results`` the whole result is copied out as well
(for tests).
"""
from __future__ import annotations

import collections
import gc
import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import gdag as G
from . import workloads as W

KINDS = ("VEC", "B&S", "IMG+ML", "HITS", "DL")
SCALED = ("VEC", "B&S", "IMG+ML", "HITS")
RESPONSE_BYTES = 64 * 1024
F32 = torch.float32
BS_PARAMS = (60.0, 0.1, 0.2, 1.0)
IMG_R5, IMG_SIGMA5, IMG_R9, IMG_SIGMA9, IMG_ALPHA = 2, 1.0, 4, 2.0, 0.5
SCALE_MIN = 1.0 / 64


@dataclass(frozen=True)
class Full:
    """The full size of each kind (scale 1), as configured."""
    vec_n: int = 1_000_000
    bs_n: int = 10_000_000
    bs_count: int = 10
    img_side: int = 4096
    ml_rows: int = 100_000
    ml_feats: int = 1024
    ml_classes: int = 10
    hits_n: int = 10_000_000
    hits_nnz: int = 50_000_000
    dl_n: int = 16
    dl_h: int = 256
    dl_w: int = 256


def hits_bucket(s, buckets):
    """Index k (1..buckets) of the smallest HITS graph scale k/buckets >= s."""
    return min(buckets, max(1, math.ceil(s * buckets - 1e-9)))


def sizes(full, kind, s, buckets=16):
    """The per-request sizes of a request of `kind` at scale s."""
    if kind == "VEC":
        n = max(1, min(full.vec_n, round(full.vec_n * s)))
        return {"n": n, "nbytes": 4 * n}
    if kind == "B&S":
        n = max(1, min(full.bs_n, round(full.bs_n * s)))
        return {"n": n, "resp": min(4 * n, RESPONSE_BYTES)}
    if kind == "IMG+ML":
        side = min(full.img_side, max(8, int(round(full.img_side * math.sqrt(s) / 8.0)) * 8))
        rows = max(1, min(full.ml_rows, round(full.ml_rows * s)))
        return {"side": side, "npx": side * side, "rows": rows, "resp": min(4 * side * side, RESPONSE_BYTES)}
    if kind == "HITS":
        return {"bucket": hits_bucket(s, buckets)}
    return {}


def work_scale(full, kind, s, buckets=16):
    """The fraction of the kind's full-size work a request of scale s does."""
    if kind == "VEC":
        return sizes(full, kind, s)["n"] / full.vec_n
    if kind == "B&S":
        return sizes(full, kind, s)["n"] / full.bs_n
    if kind == "IMG+ML":
        z = sizes(full, kind, s)
        return 0.5 * z["npx"] / full.img_side ** 2 + 0.5 * z["rows"] / full.ml_rows
    if kind == "HITS":
        return hits_bucket(s, buckets) / buckets
    return 1.0


def _hits_graph(args):
    import datagen
    n, nnz, seed = args
    return datagen.hits_graph(n, nnz, seed=seed)


class Inputs:
    """Read-only inputs, generated once and resident, shared by every
    request.  ``device="cpu"`` keeps everything in ordinary host memory (for
    driving the dispatcher on the recording backend, which computes
    nothing).  ``full_data``: already generated full-size inputs to reuse
    (keys "bs", "img", "ml", "hits", "dl" as the benchmark builds them).
    ``workers``: processes generating the HITS graphs in parallel (spawned,
    so safe once CUDA is initialised).  ``keep_host``: keep numpy copies of
    every input (for oracle checks)."""

    def __init__(self, datagen, full=Full(), kinds=KINDS, device="cuda", hits_buckets=16, full_data=None,
                 workers=0, keep_host=False):
        self.full, self.kinds, self.device, self.hits_buckets = full, tuple(kinds), device, hits_buckets
        pin = (lambda t: t.pin_memory()) if device != "cpu" else (lambda t: t)
        dev = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        fd = full_data or {}
        self.host = {} if keep_host else None
        self.data = {}
        if "VEC" in kinds:
            x, y = datagen.vec_inputs(full.vec_n, seed=10)
            self.data["VEC"] = {"hx": pin(torch.from_numpy(x)), "hy": pin(torch.from_numpy(y))}
            self._keep("VEC", (x, y))
        if "B&S" in kinds:
            ps = fd.get("bs") or datagen.bs_inputs(full.bs_n, count=full.bs_count, seed=11)
            self.data["B&S"] = {"S": [dev(p) for p in ps]}
            self._keep("B&S", ps)
        if "IMG+ML" in kinds:
            img = fd.get("img")
            if img is None:
                img = datagen.image(full.img_side, full.img_side, seed=12)
            elif torch.is_tensor(img):
                img = img.cpu().numpy()
            ml = fd.get("ml") or datagen.ml_inputs(full.ml_rows, feats=full.ml_feats, classes=full.ml_classes,
                                                   seed=13)
            X, T1, b1, T2, b2 = ml
            self.data["IMG+ML"] = {"img": dev(np.ravel(img)), "X": dev(X), "T1": dev(T1), "b1": dev(b1),
                                   "T2": dev(T2), "b2": dev(b2),
                                   "w5": W.gaussian_weights(IMG_R5, IMG_SIGMA5).to(device),
                                   "w9": W.gaussian_weights(IMG_R9, IMG_SIGMA9).to(device)}
            self._keep("IMG+ML", (np.ravel(img), X, T1, b1, T2, b2))
        if "HITS" in kinds:
            B = hits_buckets
            jobs = [(max(64, round(full.hits_n * k / B)), max(64, round(full.hits_nnz * k / B)), 1400 + k)
                    for k in range(1, B + 1)]
            graphs = {}
            if fd.get("hits") is not None:
                graphs[B] = fd["hits"]
            todo = [k for k in range(1, B + 1) if k not in graphs]
            if workers > 1 and len(todo) > 1:
                import multiprocessing as mp
                with mp.get_context("spawn").Pool(min(workers, len(todo))) as pool:
                    for k, g in zip(todo, pool.map(_hits_graph, [jobs[k - 1] for k in todo])):
                        graphs[k] = g
            else:
                for k in todo:
                    graphs[k] = _hits_graph(jobs[k - 1])
            i32 = torch.int32
            self.data["HITS"] = {}
            nmax = 0
            for k in range(1, B + 1):
                csr, csc = graphs[k]
                n = len(csr[0]) - 1
                nmax = max(nmax, n)
                self.data["HITS"][k] = {"n": n, "nnz": int(csr[0][-1]),
                                        "A": (dev(csr[0], i32), dev(csr[1], i32), dev(csr[2], F32)),
                                        "AT": (dev(csc[0], i32), dev(csc[1], i32), dev(csc[2], F32))}
                self._keep(("HITS", k), (csr, csc))
            self.data["HITS_ones"] = torch.ones(nmax, dtype=F32, device=device)
        if "DL" in kinds:
            dl = fd.get("dl") or datagen.dl_inputs(n=full.dl_n, h=full.dl_h, w=full.dl_w, seed=15)[0]
            x1, x2, w1, b1, w2, b2, wd, bd = dl
            bf = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16).to(device)
            self.data["DL"] = {"x1": bf(x1), "x2": bf(x2), "w1": bf(w1), "w2": bf(w2), "b1": dev(b1),
                               "b2": dev(b2), "wd": dev(wd), "bd": dev(bd)}
            self._keep("DL", dl)

    def _keep(self, key, value):
        if self.host is not None:
            self.host[key] = value


class Request:
    """One DAG submission.  ``done_at`` is set when it completes or fails;
    ``error`` is then None or the GdagError that failed it.  Times are in
    seconds from the start of the run."""

    __slots__ = ("rid", "kind", "scale", "arrival", "admitted", "issued", "done_at", "sinks", "slot", "need",
                 "est", "size", "resp", "resp_view", "result", "error", "cls")

    def __init__(self, rid, kind, scale, arrival):
        self.rid, self.kind, self.scale, self.arrival = rid, kind, scale, arrival
        self.admitted = self.issued = self.done_at = None
        self.sinks = []
        self.slot = None
        self.need = 0
        self.est = 0.0
        self.size = None
        self.resp = None
        self.resp_view = None
        self.result = None
        self.error = None
        self.cls = "s"


class Slot:
    """The private arrays of one request of a kind, at full size."""

    __slots__ = ("kind", "cls", "ctx", "tensors", "A", "host", "nbytes", "programs", "tainted")

    def __init__(self, kind, cls, ctx):
        self.kind, self.cls, self.ctx = kind, cls, ctx
        self.tensors = {}
        self.A = {}
        self.host = None  # pinned response buffer (host view of the response arrays)
        self.nbytes = 0
        self.programs = {}
        self.tainted = False


class Server:
    """One gdag context shared by every request."""

    def __init__(self, inputs, budget_bytes=40 << 30, max_streams=32, device="cuda", fuse_max=None,
                 backend="cuda", record_log=False, fake_fail_op=-1, fake_fail_sticky=False, fake_complete=None,
                 request_timeout_s=120.0, trim_nodes=0, window_ms=None, keep_results=False, split_ms=None,
                 short_priority=-5, long_window_ms=None):
        """``fuse_max``: {kind: largest node size (elements) that is fused
        across requests}; None or {} turns fusion off.  ``window_ms``: the
        largest estimated GPU time of admitted, unfinished requests (None:
        memory alone limits admission); the estimates come from
        :meth:`calibrate`.  ``backend="fake"`` (with ``device="cpu"``) runs
        the dispatcher on the recording backend: admission, batching and
        bookkeeping without a GPU (every node reports complete when queried;
        nothing is computed), and ``fake_fail_op`` / ``fake_fail_sticky`` /
        ``fake_complete`` inject a failure or a device that never completes
        there.  ``request_timeout_s``: a request still incomplete this long
        after its admission means the device has stopped making progress;
        run() then raises GDAG_ERR_TIMEOUT instead of polling forever (None:
        no limit).  ``trim_nodes``: the context's node-table threshold for
        dropping retired elements (0: the library default).
        ``keep_results``: copy every request's whole result to the host when
        it completes (``request.result``).  ``split_ms``: requests estimated
        above it form the long class (its own queue, window and context);
        the short class's context creates its streams at CUDA priority
        ``short_priority`` (None: one class); ``long_window_ms`` is the long
        class's window (default: ``window_ms``)."""
        self.inp = inputs
        self.full = inputs.full
        self.fuse_max = dict(fuse_max or {})
        self.budget = budget_bytes
        self.used = 0     # bytes of the slots held by admitted, unfinished requests
        self.cached = 0   # bytes of idle slots in the pools
        self.device = device
        self.window_ms = window_ms
        self.windows = {"s": window_ms, "l": window_ms if long_window_ms is None else long_window_ms}
        self.keep_results = keep_results
        self.split_ms = split_ms

        def context(priority):
            return G.Context(max_streams=max_streams, retire_by_query=True, backend=backend,
                             fake_complete=(backend == "fake") if fake_complete is None else fake_complete,
                             record_log=record_log, fake_fail_op=fake_fail_op, fake_fail_sticky=fake_fail_sticky,
                             trim_nodes=trim_nodes, stream_priority=priority)
        # class "s" (short; the only class without split_ms) and "l" (long)
        self.ctxs = {"s": context(short_priority if split_ms is not None else 0)}
        if split_ms is not None:
            self.ctxs["l"] = context(0)
        self.ctx = self.ctxs["s"]
        self.request_timeout_s = request_timeout_s
        self.shared = {}
        self.pools = {(k, c): [] for k in KINDS for c in self.ctxs}
        self.cost = {k: (1.0, 0.0) for k in KINDS}   # est ms = a + b * work scale
        self._partitions = {}
        self._slot_bytes = {}

    # ------------------------------------------------------------ shared
    def _shared(self, ctx, key, t):
        """Register a resident read-only input once per context."""
        k = (id(ctx), key)
        if k not in self.shared:
            self.shared[k] = ctx.array(t)
        return self.shared[k]

    def _hits_shared(self, ctx, k):
        """Arrays of HITS graph k in a context: the CSR of A and A^T, their
        merge-path partitions (computed once per context, by a DAG element
        that later requests read), and the all-ones start vector."""
        g = self.inp.data["HITS"][k]
        A = [self._shared(ctx, ("A", k, i), t) for i, t in enumerate(g["A"])]
        AT = [self._shared(ctx, ("AT", k, i), t) for i, t in enumerate(g["AT"])]
        pk = (id(ctx), k)
        if pk not in self._partitions:
            n, nnz = g["n"], g["nnz"]
            pb = G.gdag_scratch_bytes("spmv_partition", n + nnz)
            pa = torch.zeros(pb, dtype=torch.uint8, device=self.device)
            pat = torch.zeros(pb, dtype=torch.uint8, device=self.device)
            PA, PAT = ctx.array(pa), ctx.array(pat)
            ctx.launch("spmv_partition", A[0], PA, n, nnz)
            ctx.launch("spmv_partition", AT[0], PAT, n, nnz)
            self._partitions[pk] = (PA, PAT, pa, pat)
        ones = self._shared(ctx, "ones", self.inp.data["HITS_ones"])
        return A, AT, self._partitions[pk][0], self._partitions[pk][1], ones

    # ------------------------------------------------------------- slots
    def slot_bytes(self, kind):
        """Device bytes of one slot of `kind` (what admission charges)."""
        got = self._slot_bytes.get(kind)
        if got is None:
            got = sum(n * e for n, e in self._slot_layout(kind).values())
            self._slot_bytes[kind] = got
        return got

    def _slot_layout(self, kind):
        """{array name: (elements, element bytes)} of a slot."""
        f, S = self.full, G.gdag_scratch_bytes
        if kind == "VEC":
            return {"x": (f.vec_n, 4), "y": (f.vec_n, 4), "z": (1, 4),
                    "s": (S("vec_reduce_diff", f.vec_n), 1)}
        if kind == "B&S":
            return {"C%d" % i: (f.bs_n, 4) for i in range(f.bs_count)}
        if kind == "IMG+ML":
            npx = f.img_side ** 2
            lay = {nm: (npx, 4) for nm in ("b5", "b9", "e5", "e9", "sh", "out")}
            lay.update({"mm5": (2, 4), "mm9": (2, 4), "sc5": (S("minmax", npx), 1), "sc9": (S("minmax", npx), 1),
                        "s1": (f.ml_rows * f.ml_classes, 4), "s2": (f.ml_rows * f.ml_classes, 4),
                        "lab": (f.ml_rows, 4)})
            return lay
        if kind == "HITS":
            n, nnz = self._hits_max()
            lay = {nm: (n, 4) for nm in ("a", "h", "a2", "h2")}
            lay.update({"na": (1, 4), "nh": (1, 4), "sa": (S("l2norm", n), 1), "sh": (S("l2norm", n), 1),
                        "ca": (S("spmv_csr", n + nnz), 1), "cat": (S("spmv_csr", n + nnz), 1)})
            return lay
        n, h, w = f.dl_n, f.dl_h, f.dl_w
        pooled = n * 64 * (h // 2) * (w // 2)
        return {"p1": (pooled, 2), "p2": (pooled, 2), "e1": (n * 64, 4), "e2": (n * 64, 4),
                "logits": (n * 10, 4), "st1": (1, 4), "st2": (1, 4)}

    def _hits_max(self):
        gs = self.inp.data["HITS"].values()
        return max(g["n"] for g in gs), max(g["nnz"] for g in gs)

    def _new_slot(self, kind, cls):
        sl = Slot(kind, cls, self.ctxs[cls])
        dtypes = {1: torch.uint8, 2: torch.bfloat16, 4: F32}
        pin = self.device != "cpu"
        sl.host = torch.zeros(RESPONSE_BYTES // 4, dtype=F32, pin_memory=pin)
        # the arrays whose head is prefetched to the host: the response
        # buffer is their host view (the server only touches that head)
        resp = {"VEC": "z", "B&S": "C0", "IMG+ML": "out", "HITS": "a2", "DL": "logits"}[kind]
        for nm, (n, eb) in self._slot_layout(kind).items():
            dt = torch.int32 if nm == "lab" else dtypes[eb]
            zero = nm in ("s", "sc5", "sc9", "sa", "sh", "st1", "st2")  # scratch counters and status start at 0
            t = (torch.zeros if zero else torch.empty)(n, dtype=dt, device=self.device)
            sl.tensors[nm] = t
            host = None
            if nm == resp:
                host = sl.host
            elif kind == "VEC" and nm in ("x", "y"):
                host = self.inp.data["VEC"]["h" + nm]
            elif kind == "DL" and nm in ("st1", "st2"):
                # the status words after the logits in the response buffer
                host = sl.host[self.full.dl_n * 10 + (nm == "st2"):].data_ptr()
            sl.A[nm] = sl.ctx.array(t, host=host)
        sl.nbytes = self.slot_bytes(kind)
        return sl

    def _drop_slot(self, sl):
        """Unregister a slot's arrays (waits for their users) and free it."""
        for a in sl.A.values():
            sl.ctx.unregister(a)
        sl.A.clear()
        sl.tensors.clear()
        sl.programs.clear()

    def _take_slot(self, kind, alone, cls="s"):
        """A slot for a new request of class cls, or None if the budget has
        no room (an idle slot of another kind or class is released first
        when that makes room; a request admitted while nothing else is in
        flight always gets one)."""
        pool = self.pools[(kind, cls)]
        if pool:
            sl = pool.pop()
            self.cached -= sl.nbytes
            self.used += sl.nbytes
            return sl
        nb = self.slot_bytes(kind)
        while self.used + self.cached + nb > self.budget and self.cached:
            other = max((k for k in self.pools if self.pools[k]), key=lambda k: self.slot_bytes(k[0]))
            victim = self.pools[other].pop()
            self.cached -= victim.nbytes
            self._drop_slot(victim)
        if self.used + self.cached + nb > self.budget and not alone:
            return None
        sl = self._new_slot(kind, cls)
        self.used += sl.nbytes
        return sl

    def _return_slot(self, sl):
        self.used -= sl.nbytes
        if sl.tainted:  # a failed request may have left a counter or status nonzero
            self._drop_slot(sl)
        else:
            self.pools[(sl.kind, sl.cls)].append(sl)
            self.cached += sl.nbytes

    # ----------------------------------------------------------- programs
    def _program(self, sl, r):
        """The recorded program of request r on slot sl (recorded on first
        use; sizes are parameters) and its sink elements: the elements of
        the request that are not ancestors of its last one."""
        key = ("HITS", r.size["bucket"]) if r.kind == "HITS" else r.kind
        got = sl.programs.get(key)
        if got is not None:
            return got
        c, A, P = sl.ctx, sl.A, G.Param
        sh = lambda key, t: self._shared(c, key, t)
        p = c.program()
        tails = []
        if r.kind == "VEC":
            p.write(A["x"], 0, P("nbytes"))
            p.write(A["y"], 0, P("nbytes"))
            p.launch("vec_square", A["x"], P("n"))
            p.launch("vec_square", A["y"], P("n"))
            p.launch("vec_reduce_diff", A["x"], A["y"], A["z"], A["s"], P("n"))
            p.prefetch_host(A["z"], 0, 4)
        elif r.kind == "B&S":
            for i, St in enumerate(self.inp.data["B&S"]["S"]):
                k = p.launch("bs_call", sh(("bs", i), St), A["C%d" % i], P("n"), *BS_PARAMS)
                if i:
                    tails.append(k)
            p.prefetch_host(A["C0"], 0, P("resp"))
        elif r.kind == "IMG+ML":
            d = self.inp.data["IMG+ML"]
            IMG = sh("img", d["img"])
            w5, w9 = sh("w5", d["w5"]), sh("w9", d["w9"])
            side, npx = P("side"), P("npx")
            p.launch("gauss_blur", IMG, A["b5"], w5, side, side, IMG_R5)
            p.launch("gauss_blur", IMG, A["b9"], w9, side, side, IMG_R9)
            p.launch("sobel", A["b5"], A["e5"], side, side)
            p.launch("sobel", A["b9"], A["e9"], side, side)
            p.launch("minmax", A["e5"], A["mm5"], A["sc5"], npx)
            p.launch("minmax", A["e9"], A["mm9"], A["sc9"], npx)
            p.launch("extend", A["e5"], A["mm5"], npx)
            p.launch("extend", A["e9"], A["mm9"], npx)
            p.launch("unsharp", IMG, A["b5"], A["sh"], IMG_ALPHA, npx)
            p.launch("combine", A["sh"], A["b5"], A["b9"], A["e5"], A["e9"], A["out"], npx)
            X = sh("X", d["X"])
            f, k_ = self.full.ml_feats, self.full.ml_classes
            rows = P("rows")
            p.launch("dense_scores", X, sh("T1", d["T1"]), sh("b1", d["b1"]), A["s1"], rows, f, k_)
            p.launch("dense_scores", X, sh("T2", d["T2"]), sh("b2", d["b2"]), A["s2"], rows, f, k_)
            p.launch("row_softmax", A["s1"], rows, k_)
            p.launch("row_softmax", A["s2"], rows, k_)
            tails.append(p.launch("argmax_combine", A["s1"], A["s2"], A["lab"], rows, k_))
            p.prefetch_host(A["out"], 0, P("resp"))
        elif r.kind == "HITS":
            k = r.size["bucket"]
            g = self.inp.data["HITS"][k]
            n, nnz = g["n"], g["nnz"]
            GA, GAT, PA, PAT, ones = self._hits_shared(c, k)
            cur = (ones, ones)
            bufs = [(A["a2"], A["h2"]), (A["a"], A["h"])]
            for it in range(5):
                a_in, h_in = cur
                a_out, h_out = bufs[it % 2]
                p.launch("spmv_csr", *GAT, h_in, PAT, a_out, A["cat"], n, nnz)
                p.launch("spmv_csr", *GA, a_in, PA, h_out, A["ca"], n, nnz)
                p.launch("l2norm", a_out, A["na"], A["sa"], n)
                p.launch("l2norm", h_out, A["nh"], A["sh"], n)
                p.launch("scale", a_out, A["na"], n)
                last = p.launch("scale", h_out, A["nh"], n)
                cur = (a_out, h_out)
            tails.append(last)  # the last hub update
            # five iterations end in the first buffer pair (a2, h2)
            p.prefetch_host(A["a2"], 0, min(4 * n, RESPONSE_BYTES))
        else:
            d = self.inp.data["DL"]
            n, h, w = self.full.dl_n, self.full.dl_h, self.full.dl_w
            S = lambda nm: sh(("dl", nm), d[nm])
            p.launch("conv3x3_relu_pool", S("x1"), S("w1"), S("b1"), A["p1"], A["st1"], n, h, w)
            p.launch("conv3x3_relu_pool", S("x2"), S("w2"), S("b2"), A["p2"], A["st2"], n, h, w)
            p.launch("avgpool_global", A["p1"], A["e1"], n * 64, (h // 2) * (w // 2))
            p.launch("avgpool_global", A["p2"], A["e2"], n * 64, (h // 2) * (w // 2))
            p.launch("concat_dense", A["e1"], A["e2"], S("wd"), S("bd"), A["logits"], n, 64, 10)
            tails.append(p.prefetch_host(A["st1"], 0, 4))
            tails.append(p.prefetch_host(A["st2"], 0, 4))
            p.prefetch_host(A["logits"], 0, 4 * n * 10)
        params = {"VEC": ("n", "nbytes"), "B&S": ("n", "resp"), "IMG+ML": ("side", "npx", "rows", "resp")}
        got = (p, tails, params.get(r.kind, ()))
        sl.programs[key] = got
        return got

    def _resp_bytes(self, r):
        """Bytes of r's response: its result's head, as prefetched."""
        if r.kind == "VEC":
            return 4
        if r.kind == "HITS":
            return min(4 * self.inp.data["HITS"][r.size["bucket"]]["n"], RESPONSE_BYTES)
        if r.kind == "DL":
            return 4 * self.full.dl_n * 10 + 8  # the logits and the two status words
        return r.size["resp"]

    # ----------------------------------------------------------- issue
    def issue(self, r):
        """Issue every element of request r with one call (never blocks)."""
        p, tails, names = self._program(r.slot, r)
        nodes = p.issue(**{k: r.size[k] for k in names})
        # a prefetch of a view that is already current makes no node (-1)
        r.sinks = [n for n in [nodes[i] for i in tails] + [nodes[-1]] if n >= 0]

    def _fusable(self, r):
        lim = self.fuse_max.get(r.kind)
        return lim is not None and r.kind in ("VEC", "B&S") and r.size["n"] <= lim

    def issue_batch(self, rs):
        """Issue the requests admitted in one pass: fusable VEC and B&S
        requests as fused groups (when two or more share a kind), the rest
        one by one.  A call that fails fails the requests it was issuing
        (all members of a fused group) and no others."""
        groups = {}
        for r in rs:
            if self._fusable(r):
                groups.setdefault((r.kind, r.cls), []).append(r)
            else:
                self._guarded([r], self.issue, r)
        for g in groups.values():
            if len(g) == 1:
                self._guarded(g, self.issue, g[0])
            elif g:
                self._guarded(g, self._issue_group, g)

    def _guarded(self, rs, fn, arg):
        """fn(arg); on a library error the requests `rs` fail.  Their sinks
        become whatever elements had been issued, so each finishes once that
        work has completed, and their slots are not reused.  An error that
        poisoned the context is raised: nothing further can run on it."""
        try:
            fn(arg)
        except G.GdagError as e:
            if e.code == G.GDAG_ERR_POISONED:
                raise
            done = [n for n in getattr(e, "nodes", []) if n >= 0]
            for r in rs:
                r.error = e
                r.sinks = list(done)
                r.slot.tainted = True

    def _issue_group(self, g):
        """One program for a group of fusable requests of one kind and
        class: the copies, one fused element per node kind, and one prefetch
        per request (each request's sink; the fused elements are its
        ancestors)."""
        c = g[0].slot.ctx
        p = c.program()
        pref = []
        if g[0].kind == "VEC":
            sq, red = [], []
            for r in g:
                A, n = r.slot.A, r.size["n"]
                p.write(A["x"], 0, 4 * n)
                p.write(A["y"], 0, 4 * n)
                sq += [(A["x"], n), (A["y"], n)]
                red.append((A["x"], A["y"], A["z"], A["s"], n))
            p.launch_fused("vec_square", sq)
            p.launch_fused("vec_reduce_diff", red)
            for r in g:
                pref.append(p.prefetch_host(r.slot.A["z"], 0, 4))
        else:
            members = []
            for r in g:
                A, n = r.slot.A, r.size["n"]
                for i, St in enumerate(self.inp.data["B&S"]["S"]):
                    members.append((self._shared(c, ("bs", i), St), A["C%d" % i], n) + BS_PARAMS)
            p.launch_fused("bs_call", members)
            for r in g:
                pref.append(p.prefetch_host(r.slot.A["C0"], 0, r.size["resp"]))
        nodes = p.issue()
        for r, i in zip(g, pref):
            r.sinks = [nodes[i]] if nodes[i] >= 0 else []

    def _last_node(self):
        return G.gdag_stats_get(self.ctx.h).nodes - 1

    # ------------------------------------------------------------ finish
    def finish(self, r, now):
        sl = r.slot
        if r.error is None:
            nb = self._resp_bytes(r)
            arr = sl.A[{"VEC": "z", "B&S": "C0", "IMG+ML": "out", "HITS": "a2", "DL": "logits"}[r.kind]]
            if r.kind == "DL":
                # logits and the two status words, each from its own prefetch
                sl.ctx.read(arr, None, 0, nb - 8)
                sl.ctx.read(sl.A["st1"], None, 0, 4)
                sl.ctx.read(sl.A["st2"], None, 0, 4)
                st = sl.host[self.full.dl_n * 10:self.full.dl_n * 10 + 2].view(torch.int32)
                if int(st[0]) or int(st[1]):
                    r.error = G.GdagError(G.GDAG_ERR_TIMEOUT, "convolution status %d %d" % (int(st[0]), int(st[1])))
                    sl.tainted = True
            else:
                sl.ctx.read(arr, None, 0, nb)  # served from the completed prefetch
            r.resp_view = sl.host[: nb // 4].clone()
            if self.keep_results and r.error is None:
                r.result = self._result(r)
        r.done_at = now
        self._return_slot(sl)
        r.slot = None

    def _result(self, r):
        """The request's whole result, copied from the device (its work has
        completed)."""
        T, z = r.slot.tensors, r.size
        if r.kind == "VEC":
            return {"z": T["z"].cpu().clone()}
        if r.kind == "B&S":
            return {"C%d" % i: T["C%d" % i][: z["n"]].cpu() for i in range(self.full.bs_count)}
        if r.kind == "IMG+ML":
            return {"out": T["out"][: z["npx"]].cpu(), "labels": T["lab"][: z["rows"]].cpu(),
                    "e5": T["e5"][: z["npx"]].cpu(), "e9": T["e9"][: z["npx"]].cpu()}
        if r.kind == "HITS":
            n = self.inp.data["HITS"][z["bucket"]]["n"]
            return {"a": T["a2"][:n].cpu(), "h": T["h2"][:n].cpu()}
        return {"logits": T["logits"].cpu().clone(), "p1": T["p1"].cpu(), "p2": T["p2"].cpu()}

    # ------------------------------------------------------------- warm
    def estimate(self, r):
        a, b = self.cost[r.kind]
        return a + b * work_scale(self.full, r.kind, r.scale, self.inp.hits_buckets)

    def warm(self, kinds=None, calibrate=False):
        """Record each kind's program, build the shared state (HITS
        partitions, resident inputs' registrations) and, with
        ``calibrate``, fit each kind's GPU-time model.  Then freeze the
        objects that live for the whole run out of the garbage collector's
        scans, so its collections during serving stay short."""
        kinds = [k for k in (kinds or KINDS) if k in self.inp.kinds]
        for k in kinds:
            scales = [SCALE_MIN, 1.0] if k in SCALED else [1.0]
            for s in scales:
                for cls in self.ctxs:
                    r = self._make(k, s)
                    r.cls = cls
                    self._run_alone(r)
        if calibrate:
            self.calibrate(kinds)
        gc.collect()
        gc.freeze()

    def _make(self, kind, s, rid=-1):
        r = Request(rid, kind, s, 0.0)
        r.size = sizes(self.full, kind, s, self.inp.hits_buckets)
        return r

    def _run_alone(self, r):
        r.slot = self._take_slot(r.kind, True, r.cls)
        self.issue(r)
        r.slot.ctx.sync()
        self.finish(r, 0.0)

    def calibrate(self, kinds=None, reps=3):
        """GPU time of each kind alone (issue to completion, median of
        `reps`) at two work scales, fitted as a + b * scale ms."""
        for k in kinds or KINDS:
            if k not in self.inp.kinds:
                continue
            pts = []
            for s in ([1.0 / 16, 1.0] if k in SCALED else [1.0]):
                ts = []
                for _ in range(reps):
                    r = self._make(k, s)
                    r.slot = self._take_slot(k, True)
                    t0 = time.perf_counter()
                    self.issue(r)
                    r.slot.ctx.sync()
                    ts.append((time.perf_counter() - t0) * 1e3)
                    self.finish(r, 0.0)
                pts.append((work_scale(self.full, k, s, self.inp.hits_buckets), float(np.median(ts))))
            if len(pts) == 2:
                (x0, y0), (x1, y1) = pts
                b = max(0.0, (y1 - y0) / (x1 - x0))
                self.cost[k] = (max(0.0, y0 - b * x0), b)
            else:
                self.cost[k] = (pts[0][1], 0.0)
        return dict(self.cost)

    # -------------------------------------------------------------- run
    def classify(self, r):
        """The request's class: "l" (long) if its estimate is above
        split_ms, else "s"."""
        return "l" if self.split_ms is not None and r.est > self.split_ms else "s"

    def run(self, requests, clock=time.perf_counter, spin=True):
        """Serve a list of requests (sorted by arrival, seconds from start)."""
        pending = {c: collections.deque() for c in self.ctxs}
        inflight = []
        i = 0
        t0 = clock()
        done = 0
        est_inflight = {c: 0.0 for c in self.ctxs}
        n_inflight = {c: 0 for c in self.ctxs}
        total = len(requests)
        full, B = self.full, self.inp.hits_buckets
        while done < total:
            now = clock() - t0
            while i < total and requests[i].arrival <= now:
                r = requests[i]
                r.size = sizes(full, r.kind, r.scale, B)
                r.est = self.estimate(r)
                r.cls = self.classify(r)
                pending[r.cls].append(r)
                i += 1
            batch = []
            for c, q in pending.items():
                # arrival order within the class; a class whose head cannot
                # be admitted does not hold up the other class
                while q:
                    r = q[0]
                    busy = n_inflight[c] > 0
                    w = self.windows[c]
                    if busy and w is not None and est_inflight[c] + r.est > w:
                        break
                    sl = self._take_slot(r.kind, not (inflight or batch), c)
                    if sl is None:
                        break
                    q.popleft()
                    r.slot, r.need, r.admitted = sl, sl.nbytes, now
                    est_inflight[c] += r.est
                    n_inflight[c] += 1
                    batch.append(r)
            if batch:
                self.issue_batch(batch)
                t = clock() - t0
                for r in batch:
                    r.issued = t
                inflight.extend(batch)
            if inflight:
                flags = {}
                for c, ctx in self.ctxs.items():
                    flat = [n for r in inflight if r.cls == c for n in r.sinks]
                    flags[c] = iter(ctx.done_many(flat) if flat else [])
                still = []
                for r in inflight:
                    f = flags[r.cls]
                    ok = all([next(f) for _ in r.sinks])
                    if ok:
                        est_inflight[r.cls] -= r.est
                        n_inflight[r.cls] -= 1
                        if not n_inflight[r.cls]:
                            est_inflight[r.cls] = 0.0  # no drift from rounding
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
            if not inflight and not any(pending.values()) and i < total:
                # idle until the next arrival
                wait = requests[i].arrival - (clock() - t0)
                if wait > 0 and not spin:
                    time.sleep(wait)
        return requests

    def close(self):
        for ctx in self.ctxs.values():
            ctx.sync()
            ctx.close()


def poisson_requests(rate, count, seed=0, kinds=KINDS):
    """Arrival times of a Poisson stream of `rate` req/s; kinds uniform;
    scale s ~ U[1/64, 1] (DL requests ignore it: their batch is fixed)."""
    g = np.random.default_rng(seed)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    out = []
    for k in range(count):
        kind = kinds[int(g.integers(0, len(kinds)))]
        s = float(g.uniform(SCALE_MIN, 1.0))
        out.append(Request(k, kind, s, float(t[k])))
    return out


def latency_summary(reqs, full=Full(), buckets=16):
    """p50/p99 latency overall and per kind, with the split of each
    request's latency into queue wait, host issue and issue to completion,
    the achieved throughput, and the mean work per request (as a fraction of
    each kind's full size)."""
    failed = sum(r.error is not None for r in reqs)
    ok = [r for r in reqs if r.error is None]
    pct = lambda a, p: float(np.percentile(a, p)) if len(a) else float("nan")

    def stats(rs):
        lat = np.array([(r.done_at - r.arrival) * 1e3 for r in rs])
        q = np.array([(r.admitted - r.arrival) * 1e3 for r in rs])
        iss = np.array([(r.issued - r.admitted) * 1e3 for r in rs if r.issued is not None])
        dev = np.array([(r.done_at - r.issued) * 1e3 for r in rs if r.issued is not None])
        return {"n": len(rs), "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": float(lat.mean()),
                "queue_p50_ms": pct(q, 50), "queue_p99_ms": pct(q, 99),
                "issue_p50_ms": pct(iss, 50), "issue_p99_ms": pct(iss, 99),
                "device_p50_ms": pct(dev, 50), "device_p99_ms": pct(dev, 99)}
    out = stats(ok)
    span = max(r.done_at for r in ok) - min(r.arrival for r in ok)
    out.update({"requests": len(ok), "failed": failed, "throughput_req_s": len(ok) / span,
                "mean_work_scale": float(np.mean([work_scale(full, r.kind, r.scale, buckets) for r in ok])),
                "by_kind": {k: stats([r for r in ok if r.kind == k]) for k in sorted({r.kind for r in ok})},
                "by_class": {c: stats([r for r in ok if r.cls == c]) for c in sorted({r.cls for r in ok})}})
    return out
