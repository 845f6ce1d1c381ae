"""Benchmark: DAG makespan of the B&S program (10 independent Black-Scholes
nodes over 10 x 1e7 float32 prices) under the run-time DAG scheduler, beside
serial single-stream execution, a hand-built CUDA Graph of the same DAG, the
critical-path bound from the solo node times, and the CPU oracle; then the
same comparison for every other DAG of the suite (VEC, IMG, ML, HITS at their
configured sizes) under ``dags``.

One JSON line on rank 0.  ``value`` = DAGs per second with the inputs already
resident in HBM; ``e2e`` = the same metric through the public API with the
host writing every input and reading every result each step (pinned host
buffers, copies inside the timed region), with the copy/compute overlaps of
one traced step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# one hardware work queue per scheduler stream (see paper_2012_09646_gb300/gdag.py);
# set before anything creates the CUDA context
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

N_OPTS = 10_000_000
N_VEC = 10
BS_PARAMS = (60.0, 0.1, 0.2, 1.0)
BYTES_PER_OPTION = 8  # 4 read + 4 written
METRIC = "DAG makespan speedup vs serial stream; kernel HBM GB/s; serve p50/p99 latency"
UNIT = "DAG/s"
# DRAM bytes (read + write) of one bs_call launch from one ncu capture
# (profiles/bs_call_bs_10x1e7.md), valid only for the kernel source it was
# taken on: a changed k_bs.cu reports null.
BS_CALL_TRAFFIC = {"bytes": 41681408,
                   "sha256": "cf6b97c658f7616b8b7d3d16bce2da5f334d37a24836df2da907060d0e27e7ed",
                   "note": "one launch captured alone: its 40 MB output is still in L2 when the kernel ends"}
WORKLOAD = "B&S: 10 independent Black-Scholes call nodes, 10 x 1e7 float32 spot prices U[10,100), K=60 r=0.1 sigma=0.2 T=1"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--dags", default="all", choices=["all", "bs"],
                    help="also measure the VEC, IMG, ML and HITS DAGs (rank 0)")
    ap.add_argument("--profile", default=None, choices=["bs", "vec", "img", "ml", "hits", "dl", "hits_batch", "bs_fused"],
                    help="run only --steps steps of one DAG through the library (a small, "
                         "single-context command for ncu captures); prints nothing")
    ap.add_argument("--img-size", type=int, default=4096)
    ap.add_argument("--vec-n", type=int, default=1_000_000, help="VEC length for --profile vec")
    ap.add_argument("--serve", type=int, default=1, help="run the serving benchmark (with --dags all)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="seconds of Poisson arrivals per rate")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """SM clock, power and clock-event reasons sampled every 100 ms on a
    thread through NVML's read-only queries (nvidia-smi's output is block
    buffered through a pipe).  Nothing is ever set."""

    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap"}

    def __init__(self, index, uuid=None):
        self.index, self.uuid = index, uuid
        self.samples = []
        self.stop = threading.Event()
        self.t = None
        self.err = None

    def _open(self):
        import ctypes
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        ok = False
        if self.uuid:
            ok = nv.nvmlDeviceGetHandleByUUID(self.uuid.encode(), ctypes.byref(h)) == 0
        if not ok and nv.nvmlDeviceGetHandleByIndex_v2(self.index, ctypes.byref(h)) != 0:
            raise OSError("no NVML handle")
        return nv, h

    def _run(self):
        import ctypes
        try:
            nv, h = self._open()
        except OSError as e:
            self.err = str(e)
            return
        clk, mx, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        while not self.stop.is_set():
            a = nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk))      # NVML_CLOCK_SM
            b = nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
            c = nv.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw))
            d = reasons_fn(h, ctypes.byref(rs))
            if a == 0 and b == 0:
                self.samples.append((clk.value, mx.value, pw.value / 1e3 if c == 0 else None,
                                     rs.value if d == 0 else 0))
            self.stop.wait(0.1)
        nv.nvmlShutdown()

    def __enter__(self):
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()
        t_end = time.time() + 3.0
        while not self.samples and self.err is None and time.time() < t_end:
            time.sleep(0.01)
        return self

    def __exit__(self, *exc):
        self.stop.set()
        if self.t:
            self.t.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled: %s" % self.err], "samples": 0}
        reasons = set()
        for _c, _m, _p, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        sm = [c for c, _m, _p, _r in self.samples]
        pw = [p for _c, _m, p, _r in self.samples if p is not None]
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm),
                "sm_max_mhz": max(m for _c, m, _p, _r in self.samples), "reasons": sorted(reasons),
                "power_w_max": max(pw) if pw else None, "samples": len(sm)}


def bs_call_traffic():
    import hashlib
    with open(os.path.join(ROOT, "paper_2012_09646_gb300", "csrc", "k_bs.cu"), "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()
    return BS_CALL_TRAFFIC["bytes"] if h == BS_CALL_TRAFFIC["sha256"] else None


def time_launches(torch, issue, reps):
    """Device ms per call of ``issue(stream_handle)`` (which enqueues one
    kernel on that stream), with the host taken out of the measurement: the
    calls are captured once into a CUDA graph, and the graph's replay is timed
    with CUDA events on its stream (launching from Python one by one would
    time the host's enqueue rate for any kernel shorter than it)."""
    s = torch.cuda.Stream()
    for _ in range(2):
        issue(s.cuda_stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(reps):
            issue(s.cuda_stream)
    with torch.cuda.stream(s):
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.replay()
        e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del g
    return ms


_FLUSH = []


def time_cold(torch, issue, reps):
    """Device ms of one call of ``issue(stream_handle)`` with a cold L2: each
    of `reps` launches follows a read of a 512 MB buffer (four times the
    L2), which leaves L2 holding clean lines of that buffer, and is timed
    alone with CUDA events on its stream (the host enqueues the launch
    while the flush runs); the median is returned."""
    if not _FLUSH:
        _FLUSH.append((torch.empty(128 << 20, dtype=torch.float32, device="cuda").fill_(1.0),
                       torch.empty((), dtype=torch.float32, device="cuda")))
    buf, acc = _FLUSH[0]
    s = torch.cuda.Stream()
    issue(s.cuda_stream)
    torch.cuda.synchronize()
    ev = []
    with torch.cuda.stream(s):
        for _ in range(reps):
            torch.sum(buf, dim=0, out=acc)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            issue(s.cuda_stream)
            e1.record(s)
            ev.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------- reference arm
def cpu_oracle_rate(seconds, n_per_vec=1_000_000):
    """The oracle, as it stands, over bounded samples of the workload: each
    sample prices n_per_vec options of every one of the 10 vectors.  Returns
    (DAG/s extrapolated, samples done, wall seconds)."""
    import datagen
    from oracle import numeric as N
    prices = datagen.bs_inputs(n_per_vec, count=N_VEC, seed=1)
    K, r, s, T = BS_PARAMS
    N.bs_call(prices[0][:10], K, r, s, T)  # load
    done, t0 = 0, time.perf_counter()
    while True:
        for p in prices:
            N.bs_call(p, K, r, s, T)
        done += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    frac = done * n_per_vec / N_OPTS  # DAGs' worth of work
    return frac / el, done, el


def _cpu_oracle_worker(seconds, n_per_vec, seed):
    """One process of the all-cores baseline: the oracle, as it stands,
    pricing its own 10 x n_per_vec options repeatedly for `seconds`."""
    import datagen
    from oracle import numeric as N
    prices = datagen.bs_inputs(n_per_vec, count=N_VEC, seed=seed)
    K, r, s, T = BS_PARAMS
    N.bs_call(prices[0][:10], K, r, s, T)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for q in prices:
            N.bs_call(q, K, r, s, T)
        done += 1
    return done * n_per_vec * N_VEC, time.perf_counter() - t0


def cpu_oracle_rate_all_cores(seconds, n_per_vec=250_000):
    """The same oracle on every host core at once: one spawned process per
    core (the options are independent, so this is the oracle run in
    parallel, not changed).  Returns (DAG/s, processes, wall seconds)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_cpu_oracle_worker, [(seconds, n_per_vec, 100 + i) for i in range(cores)])
    options = sum(o for o, _ in res)
    wall = max(t for _, t in res)
    return options / (N_OPTS * N_VEC) / wall, cores, wall


_REF_SHARDS = {}


def _ref_price_shard(i, n_shard):
    """Reference-arm worker: price shard i of a whole DAG (the ten vectors'
    options i*n_shard .. (i+1)*n_shard, drawn like the workload's) with the
    fp64 C oracle as it stands.  The shard's prices are generated on first
    use and kept, so a timed step is pricing only."""
    from oracle import numeric as N
    if i not in _REF_SHARDS:
        import datagen
        _REF_SHARDS[i] = datagen.bs_inputs(n_shard, count=N_VEC, seed=1000 + i)
    K, r, s, T = BS_PARAMS
    for p in _REF_SHARDS[i]:
        N.bs_call(p, K, r, s, T)
    return len(_REF_SHARDS[i]) * n_shard


def run_reference(args, rank):
    """The base contract's reference arm: the CPU oracle, as it stands, on
    the host cores.  Each step prices one whole B&S DAG (10 x 1e7 options),
    its options split into one shard per core and priced by one spawned
    process per core (the options are independent, so the oracle runs
    unchanged, in parallel)."""
    from paper_2012_09646_gb300 import replicas as RP
    if not RP.reports(rank):
        return
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    shards = cores
    n_shard = -(-N_OPTS // shards)
    with mp.get_context("spawn").Pool(cores) as pool:
        jobs = [(i, n_shard) for i in range(shards)]
        for _ in range(max(1, args.warmup)):
            pool.starmap(_ref_price_shard, jobs)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            done = sum(pool.starmap(_ref_price_shard, jobs))
            times.append(time.perf_counter() - t0)
    frac = done / (N_OPTS * N_VEC)  # >= 1: shards round up
    ms_dag = statistics.mean(times) / frac * 1e3
    value = 1e3 / ms_dag
    sample = ("each step prices one whole DAG (10 x %d options, in %d shards of %d options per vector) with "
              "the fp64 C oracle, one spawned process per host core" % (N_OPTS, shards, n_shard))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_dag, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "parallelism": "%d host processes" % cores},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- our arm
class Recorder:
    """Forwards every call to a Context and records the program's elements in
    issue order (kernel launches with their arguments, host writes, reads and
    prefetches), so that each node can be re-run alone for its solo time."""

    def __init__(self, ctx):
        self.ctx = ctx
        self.log = []

    def launch(self, name, *args, **kw):
        self.log.append(("k", name, args))
        return self.ctx.launch(name, *args, **kw)

    def write(self, a, src=None, off=0, nbytes=None):
        self.log.append(("h2d", a, a.nbytes - off if nbytes is None else nbytes))
        return self.ctx.write(a, src, off, nbytes)

    def read(self, a, dst=None, off=0, nbytes=None):
        self.log.append(("d2h", a, a.nbytes - off if nbytes is None else nbytes))
        return self.ctx.read(a, dst, off, nbytes)

    def prefetch_host(self, a, off=0, nbytes=None):
        self.log.append(("d2h", a, a.nbytes - off if nbytes is None else nbytes))
        return self.ctx.prefetch_host(a, off, nbytes)

    def program(self):
        return _RecordedProgram(self)

    def __getattr__(self, k):
        return getattr(self.ctx, k)


class _RecordedProgram:
    """A Program whose elements the Recorder logs at every issue."""

    def __init__(self, rec):
        self.rec, self.p, self.elems = rec, rec.ctx.program(), []

    def __len__(self):
        return len(self.p)

    def launch(self, name, *args, **kw):
        self.elems.append(("k", name, args))
        return self.p.launch(name, *args, **kw)

    def write(self, a, off=0, nbytes=None):
        self.elems.append(("h2d", a, a.nbytes - off if nbytes is None else nbytes))
        return self.p.write(a, off, nbytes)

    def prefetch_host(self, a, off=0, nbytes=None):
        self.elems.append(("d2h", a, a.nbytes - off if nbytes is None else nbytes))
        return self.p.prefetch_host(a, off, nbytes)

    def issue(self, **values):
        self.rec.log.extend(self.elems)
        return self.p.issue(**values)


def alg_bytes(name, a):
    """Algorithmic HBM bytes of one node: every input read once, every output
    written once (the per-unit figures of the design's roofline table)."""
    if name in ("vec_square", "bs_call"):
        n = a[1] if name == "vec_square" else a[2]
        return 8 * n
    if name == "vec_reduce_diff":
        return 8 * a[4]
    if name in ("gauss_blur", "sobel"):
        r, c = (a[3], a[4]) if name == "gauss_blur" else (a[2], a[3])
        return 8 * r * c
    if name == "minmax":
        return 4 * a[3]
    if name in ("extend", "scale"):
        return 8 * a[2]
    if name == "unsharp":
        return 12 * a[4]
    if name == "combine":
        return 24 * a[6]
    if name == "dense_scores":
        rows, feats, classes = a[4], a[5], a[6]
        return 4 * rows * feats + 4 * rows * classes + 4 * feats * classes
    if name == "row_softmax":
        return 8 * a[1] * a[2]
    if name == "argmax_combine":
        return 8 * a[3] * a[4] + 4 * a[3]
    if name == "spmv_csr":
        n, nnz = a[7], a[8]
        return 4 * (n + 1) + 8 * nnz + 4 * n + 4 * n
    if name == "l2norm":
        return 4 * a[3]
    if name == "seg_l2norm":
        return 4 * a[5] + 4 * (a[4] + 1) + 4 * a[4]
    if name == "seg_scale":
        return 8 * a[4] + 4 * (a[3] + 1) + 4 * a[3]
    if name == "conv3x3_relu_pool":
        n, h, w = a[5], a[6], a[7]
        return 2 * 3 * n * h * w + 2 * 64 * n * (h // 2) * (w // 2) + 64 * 27 * 2 + 64 * 4
    if name == "avgpool_global":
        return 2 * a[2] * a[3] + 4 * a[2]
    return 0


class Spec:
    """One benchmark DAG: build(ctx) -> program object; step(obj) issues one
    DAG through the library; hand(obj, ctx, H) issues the same DAG by hand on
    explicit streams (the CUDA Graph baseline); host_sync: whether each step
    ends with the host reading a result.  capture_step / after_replay: the
    part of a step that can be recorded as a graph, and what follows each
    replay (the host read)."""
    name = ""
    host_sync = False

    def __init__(self, G, W, data):
        self.G, self.W, self.data = G, W, data

    def capture_step(self, obj):
        self.step(obj)

    def after_replay(self, ctx, obj):
        pass


class BsSpec(Spec):
    name = "B&S"

    def build(self, ctx, batched=True):
        d = self.W.BsDag(ctx, N_OPTS, count=N_VEC, host=False, batched=batched)
        d.load_device(self.data["bs"])
        return d

    def step(self, d):
        d.step_resident()

    def hand(self, d, ctx, H):
        K, r, s, T = BS_PARAMS
        for i in range(N_VEC):
            H.k(i, "bs_call", d.SA[i], d.CA[i], N_OPTS, K, r, s, T)


class VecSpec(Spec):
    name = "VEC"
    host_sync = True

    def build(self, ctx, batched=True):
        d = self.W.VecDag(ctx, 1_000_000, batched=batched)
        d.load(*self.data["vec"])
        return d

    def step(self, d):
        d.step(read=True)

    def capture_step(self, d):
        d.step(read=False)

    def after_replay(self, ctx, d):
        ctx.read(d.Z)

    def hand(self, d, ctx, H):
        n = d.n
        H.copy(0, d.x, d.hx)
        H.k(0, "vec_square", d.X, n)
        H.copy(1, d.y, d.hy)
        H.k(1, "vec_square", d.Y, n)
        H.dep(0, 1)
        H.k(0, "vec_reduce_diff", d.X, d.Y, d.Z, d.S, n)
        H.copy(0, d.hz, d.z)


class ImgSpec(Spec):
    name = "IMG"

    def build(self, ctx, batched=True):
        d = self.W.ImgDag(ctx, 4096, 4096, batched=batched)
        d.img.copy_(self.data["img"])
        return d

    def step(self, d):
        d.launch_all()

    def hand(self, d, ctx, H):
        n, R, C = d.n, d.rows, d.cols
        H.k(0, "gauss_blur", d.IMG, d.B5, d.W5, R, C, d.R5)
        H.k(1, "gauss_blur", d.IMG, d.B9, d.W9, R, C, d.R9)
        H.dep(2, 0)
        H.k(2, "unsharp", d.IMG, d.B5, d.S, d.ALPHA, n)
        H.k(0, "sobel", d.B5, d.E5, R, C)
        H.k(1, "sobel", d.B9, d.E9, R, C)
        H.k(0, "minmax", d.E5, d.MM5, d.SC5, n)
        H.k(1, "minmax", d.E9, d.MM9, d.SC9, n)
        H.k(0, "extend", d.E5, d.MM5, n)
        H.k(1, "extend", d.E9, d.MM9, n)
        H.dep(0, 1)
        H.dep(0, 2)
        H.k(0, "combine", d.S, d.B5, d.B9, d.E5, d.E9, d.OUT, n)


class MlSpec(Spec):
    name = "ML"

    def build(self, ctx, batched=True):
        d = self.W.MlDag(ctx, 100_000, batched=batched)
        d.load(*self.data["ml"])
        return d

    def step(self, d):
        d.launch_all()

    def hand(self, d, ctx, H):
        r, f, k = d.rows, d.feats, d.classes
        H.k(0, "dense_scores", d.XA, d.T1A, d.b1A, d.S1A, r, f, k)
        H.k(1, "dense_scores", d.XA, d.T2A, d.b2A, d.S2A, r, f, k)
        H.k(0, "row_softmax", d.S1A, r, k)
        H.k(1, "row_softmax", d.S2A, r, k)
        H.dep(0, 1)
        H.k(0, "argmax_combine", d.S1A, d.S2A, d.LA, r, k)


class HitsSpec(Spec):
    name = "HITS"
    ITERS = 5

    def build(self, ctx, batched=True):
        csr, csc = self.data["hits"]
        d = self.W.HitsDag(ctx, csr, csc, batched=batched)
        d.run(iters=0, read=False)  # a = h = 1
        return d

    def step(self, d):
        cur, nxt = ("a", "h"), ("a2", "h2")
        for _ in range(self.ITERS):
            d.iterate(cur[0], cur[1], nxt[0], nxt[1])
            cur, nxt = nxt, cur

    def hand(self, d, ctx, H):
        n, nnz = d.n, d.nnz
        cur, nxt = ("a", "h"), ("a2", "h2")
        for it in range(self.ITERS):
            if it:
                H.dep(0, 1)  # s0 reads the hub vector s1 finished, and overwrites s1's input
                H.dep(1, 0)
            H.k(0, "spmv_csr", *d.ATA, d.V[cur[1]], d.PAT, d.V[nxt[0]], d.CAT, n, nnz)
            H.k(1, "spmv_csr", *d.AA, d.V[cur[0]], d.PA, d.V[nxt[1]], d.CA, n, nnz)
            H.k(0, "l2norm", d.V[nxt[0]], d.NA, d.SA, n)
            H.k(1, "l2norm", d.V[nxt[1]], d.NH, d.SH, n)
            H.k(0, "scale", d.V[nxt[0]], d.NA, n)
            H.k(1, "scale", d.V[nxt[1]], d.NH, n)
            cur, nxt = nxt, cur
        H.dep(0, 1)


class HitsBatchSpec(HitsSpec):
    """HITS over 64 independent graphs (1e4..1e6 vertices) as one program:
    block-diagonal SpMV and per-graph segment kernels, six launches per
    iteration for the whole batch."""
    name = "HITS-batch"

    def build(self, ctx, batched=True):
        d = self.W.HitsBatchDag(ctx, self.data["hits_batch"], batched=batched)
        d.run(iters=0, read=False)
        return d

    def hand(self, d, ctx, H):
        n, nnz, G_ = d.n, d.nnz, d.G
        cur, nxt = ("a", "h"), ("a2", "h2")
        for it in range(self.ITERS):
            if it:
                H.dep(0, 1)
                H.dep(1, 0)
            H.k(0, "spmv_csr", *d.ATA, d.V[cur[1]], d.PAT, d.V[nxt[0]], d.CAT, n, nnz)
            H.k(1, "spmv_csr", *d.AA, d.V[cur[0]], d.PA, d.V[nxt[1]], d.CA, n, nnz)
            H.k(0, "seg_l2norm", d.V[nxt[0]], d.SEG, d.NAS, d.SAS, G_, n)
            H.k(1, "seg_l2norm", d.V[nxt[1]], d.SEG, d.NHS, d.SHS, G_, n)
            H.k(0, "seg_scale", d.V[nxt[0]], d.SEG, d.NAS, G_, n)
            H.k(1, "seg_scale", d.V[nxt[1]], d.SEG, d.NHS, G_, n)
            cur, nxt = nxt, cur
        H.dep(0, 1)


def measure_hits_separate(torch, G, W, graphs, steps, iters=5):
    """The unfused form of the HITS batch: one HITS program per graph, all
    issued into one PARALLEL context (the scheduler spreads the independent
    programs over its streams).  ms per step of `iters` iterations on every
    graph."""
    ctx = G.Context()
    dags = [W.HitsDag(ctx, csr, csc) for csr, csc in graphs]
    for d in dags:
        d.run(iters=0, read=False)

    def step():
        for d in dags:
            cur, nxt = ("a", "h"), ("a2", "h2")
            for _ in range(iters):
                d.iterate(cur[0], cur[1], nxt[0], nxt[1])
                cur, nxt = nxt, cur

    for _ in range(2):
        step()
    ctx.sync()
    torch.cuda.synchronize()
    s0 = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(s0)
    ctx.fork(s0.cuda_stream)
    for _ in range(steps):
        step()
    ctx.wait_all(s0.cuda_stream)
    e1.record(s0)
    host_ms = (time.perf_counter() - t0) * 1e3 / steps
    torch.cuda.synchronize()
    out = {"makespan_ms": e0.elapsed_time(e1) / steps, "host_issue_ms": host_ms,
           "launches_per_step": len(dags) * iters * 6, "streams": ctx.stats()["streams"]}
    ctx.close()
    return out


class DlSpec(Spec):
    name = "DL"

    def build(self, ctx, batched=True):
        d = self.W.DlDag(ctx, batched=batched)
        d.load(*self.data["dl"])
        return d

    def step(self, d):
        d.launch_all()

    def hand(self, d, ctx, H):
        n, h, w = d.n, d.h, d.w
        H.k(0, "conv3x3_relu_pool", d.X1, d.W1, d.B1, d.P1, d.ST1, n, h, w)
        H.k(1, "conv3x3_relu_pool", d.X2, d.W2, d.B2, d.P2, d.ST2, n, h, w)
        H.k(0, "avgpool_global", d.P1, d.E1, n * 64, (h // 2) * (w // 2))
        H.k(1, "avgpool_global", d.P2, d.E2, n * 64, (h // 2) * (w // 2))
        H.dep(0, 1)
        H.k(0, "concat_dense", d.E1, d.E2, d.WD, d.BD, d.LOG, n, 64, d.classes)


class Hand:
    """Explicit multi-stream schedule for stream capture: every stream forks
    from the capture stream and joins back into it."""

    def __init__(self, torch, ctx, nstreams, cap):
        self.torch, self.ctx, self.cap = torch, ctx, cap
        self.s = [torch.cuda.Stream() for _ in range(nstreams)]
        fork = torch.cuda.Event()
        fork.record(cap)
        for st in self.s:
            st.wait_event(fork)

    def k(self, i, name, *args):
        self.ctx.launch_raw(name, *args, stream=self.s[i].cuda_stream)

    def copy(self, i, dst, src):
        with self.torch.cuda.stream(self.s[i]):
            dst.copy_(src, non_blocking=True)

    def dep(self, to, frm):
        ev = self.torch.cuda.Event()
        ev.record(self.s[frm])
        self.s[to].wait_event(ev)

    def join(self):
        for st in self.s:
            ev = self.torch.cuda.Event()
            ev.record(st)
            self.cap.wait_event(ev)


def make_data(datagen, which):
    import numpy as np
    import torch
    data = {}
    if "bs" in which:
        data["bs"] = datagen.bs_inputs(N_OPTS, count=N_VEC, seed=1)
    if "vec" in which:
        data["vec"] = datagen.vec_inputs(1_000_000, seed=0)
    if "img" in which:
        data["img"] = torch.from_numpy(datagen.image(4096, 4096, seed=2).reshape(-1)).cuda()
    if "ml" in which:
        data["ml"] = datagen.ml_inputs(100_000, feats=1024, classes=10, seed=3)
    if "hits" in which:
        data["hits"] = datagen.hits_graph(10_000_000, 50_000_000, seed=4)
    if "dl" in which:
        data["dl"] = datagen.dl_inputs(n=16, h=256, w=256, seed=5)[0]
    if "hits_batch" in which:
        data["hits_batch"] = datagen.hits_batch(count=64, nmin=10_000, nmax=1_000_000, seed=6)
    return data


def measure_dag(torch, G, spec, steps, peak_gbs, link):
    """Makespan per DAG under each policy and as a hand-built CUDA Graph,
    the critical-path and resource bounds."""
    import numpy as np
    s0 = torch.cuda.Stream()
    out = {}
    # a timed region of at least about 50 ms for every variant: small DAGs
    # (VEC, DL) take hundreds of steps, so that no single slow step (an OS
    # or allocator hiccup on the host) moves their mean
    cal = G.Context()
    cobj = spec.build(cal)
    for _ in range(5):
        spec.step(cobj)
    cal.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        spec.step(cobj)
    cal.sync()
    est_ms = (time.perf_counter() - t0) * 1e3 / 5
    cal.close()
    del cobj
    steps = max(steps, min(2000, int(50.0 / max(est_ms, 1e-3))))

    elements_per_step = {}

    def timed_ctx(policy, batched=True, auto_graph=0, label=None):
        ctx = G.Context(policy=policy, auto_graph=auto_graph)
        obj = spec.build(ctx, batched=batched)
        # warm-up: at least 10 steps and 20 ms, so that the context's stream
        # and event pools have reached their steady size
        t0, k = time.perf_counter(), 0
        while k < 10 or time.perf_counter() - t0 < 0.02:
            spec.step(obj)
            k += 1
        ctx.sync()
        torch.cuda.synchronize()
        nodes0 = G.gdag_stats_get(ctx.h).nodes
        if policy == G.GDAG_POLICY_SERIAL_SYNC or spec.host_sync:
            # a step that ends with a host read is complete when it returns:
            # timed on the host, like the hand-built graph's replay + sync
            t0 = time.perf_counter()
            for _ in range(steps):
                spec.step(obj)
            ctx.sync()
            ms = (time.perf_counter() - t0) * 1e3 / steps
        else:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s0)
            ctx.fork(s0.cuda_stream)
            for _ in range(steps):
                spec.step(obj)
            ctx.wait_all(s0.cuda_stream)
            e1.record(s0)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
        if label:
            elements_per_step[label] = (G.gdag_stats_get(ctx.h).nodes - nodes0) / steps
        ctx.sync()
        return ctx, obj, ms

    # the dynamic path as a program issues it one call per element (the
    # paper's form), then batched: each step's non-blocking elements in one
    # gdag_issue call (same DAG, streams and waits)
    c1, o1, out["parallel_single_calls"] = timed_ctx(G.GDAG_POLICY_PARALLEL, batched=False)
    c1.close()
    del o1
    # the same steps with the library's automatic capture of repeated
    # sequences: after two issues a step's sequence replays as one graph
    ca, oa, out["parallel_auto_graph"] = timed_ctx(G.GDAG_POLICY_PARALLEL, auto_graph=2, label="auto_graph")
    ca.close()
    del oa
    ctx, obj, out["parallel"] = timed_ctx(G.GDAG_POLICY_PARALLEL, label="parallel")
    streams_used = ctx.stats()["streams"]

    def single_runs(c, o, policy, runs=30):
        """Makespan of single DAG executions (the paper's form: each run from
        its first operation to the end of its last, with the GPU idle before
        it), p10 / p50 / p90 over `runs` runs."""
        ms = []
        for _ in range(runs):
            c.sync()
            torch.cuda.synchronize()
            if policy == G.GDAG_POLICY_SERIAL_SYNC:
                t0 = time.perf_counter()
                spec.step(o)
                c.sync()
                ms.append((time.perf_counter() - t0) * 1e3)
            else:
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(s0)
                c.fork(s0.cuda_stream)
                spec.step(o)
                c.wait_all(s0.cuda_stream)
                a1.record(s0)
                torch.cuda.synchronize()
                ms.append(a0.elapsed_time(a1))
        q = np.percentile(np.array(ms), [10, 50, 90])
        return {"runs": runs, "p10": float(q[0]), "p50": float(q[1]), "p90": float(q[2])}
    single = {"parallel": single_runs(ctx, obj, G.GDAG_POLICY_PARALLEL)}
    # the same DAG captured once by the library and replayed as one element
    gid = ctx.capture(lambda: spec.capture_step(obj))
    for _ in range(3):
        ctx.replay(gid)
        spec.after_replay(ctx, obj)
    ctx.sync()
    torch.cuda.synchronize()
    if spec.host_sync:
        t0 = time.perf_counter()
        for _ in range(steps):
            ctx.replay(gid)
            spec.after_replay(ctx, obj)
        ctx.sync()
        out["library_graph"] = (time.perf_counter() - t0) * 1e3 / steps
    else:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s0)
        ctx.fork(s0.cuda_stream)
        for _ in range(steps):
            ctx.replay(gid)
            spec.after_replay(ctx, obj)
        ctx.wait_all(s0.cuda_stream)
        e1.record(s0)
        torch.cuda.synchronize()
        out["library_graph"] = e0.elapsed_time(e1) / steps
    ctx.drop_graph(gid)
    c2, o2, out["serial_async_one_stream"] = timed_ctx(G.GDAG_POLICY_SERIAL_ASYNC)
    c2.close()
    del o2
    c3, o3, out["serial_sync"] = timed_ctx(G.GDAG_POLICY_SERIAL_SYNC)
    single["serial_sync"] = single_runs(c3, o3, G.GDAG_POLICY_SERIAL_SYNC)
    single["speedup_p50"] = single["serial_sync"]["p50"] / single["parallel"]["p50"]
    c3.close()
    del o3

    # hand-built CUDA Graph of the same DAG
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=cap):
        H = Hand(torch, ctx, 10 if spec.name == "B&S" else 3, cap)
        spec.hand(obj, ctx, H)
        H.join()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if spec.host_sync:
        t0 = time.perf_counter()
        for _ in range(steps):
            g.replay()
            torch.cuda.synchronize()  # the host reads the result each step
        out["hand_cuda_graph"] = (time.perf_counter() - t0) * 1e3 / steps
    else:
        e0.record(cur)
        for _ in range(steps):
            g.replay()
        e1.record(cur)
        torch.cuda.synchronize()
        out["hand_cuda_graph"] = e0.elapsed_time(e1) / steps
    del g

    # critical path from solo node times along the library's own edges
    lctx = G.Context(record_log=True)
    rec = Recorder(lctx)
    lobj = spec.build(rec)
    lctx.sync()
    first = len(rec.log)
    spec.step(lobj)
    lctx.sync()
    elems = rec.log
    solo_cache = {}

    def solo(e):
        kind = e[0]
        if kind == "k":
            key = (e[1],) + tuple(getattr(x, "handle", x) for x in e[2])
            if key not in solo_cache:
                solo_cache[key] = time_cold(torch, lambda sh: lctx.launch_raw(e[1], *e[2], stream=sh), 5)
            return solo_cache[key]
        nb = e[2]
        return nb / (link[kind] * 1e9) * 1e3
    weights = [solo(e) if i >= first else 0.0 for i, e in enumerate(elems)]
    edges = [(s, d) for s, d, _a, _k in lctx.edges()]
    from paper_2012_09646_gb300.analysis import critical_path
    cp = critical_path(weights, edges)
    hbm = sum(alg_bytes(e[1], [getattr(x, "handle", x) for x in e[2]]) for e in elems[first:] if e[0] == "k")
    h2d = sum(e[2] for e in elems[first:] if e[0] == "h2d")
    d2h = sum(e[2] for e in elems[first:] if e[0] == "d2h")
    res = max(cp, hbm / (peak_gbs * 1e9) * 1e3, h2d / (link["h2d"] * 1e9) * 1e3, d2h / (link["d2h"] * 1e9) * 1e3)
    out["critical_path_bound"] = cp
    out["resource_bound"] = res
    out["sum_solo"] = sum(weights)
    per_kernel = {}
    for i, e in enumerate(elems):
        if i < first or e[0] != "k":
            continue
        k = per_kernel.setdefault(e[1], {"launches": 0, "solo_ms": 0.0, "alg_bytes": 0})
        k["launches"] += 1
        k["solo_ms"] += weights[i]
        k["alg_bytes"] += alg_bytes(e[1], [getattr(x, "handle", x) for x in e[2]])
    for k in per_kernel.values():
        k["alg_gbs"] = k["alg_bytes"] / (k["solo_ms"] * 1e-3) / 1e9 if k["solo_ms"] > 0 else None
        k["frac_of_hbm_peak"] = k["alg_gbs"] / peak_gbs if k["alg_gbs"] else None
    lctx.close()
    ctx.close()
    kern = sum(1 for e in elems[first:] if e[0] == "k")
    # copy/compute overlap of one traced step (Section IV-F): CT, TC, CC, TOT
    from paper_2012_09646_gb300 import analysis
    tctx = G.Context(trace=True)
    tobj = spec.build(tctx)
    for _ in range(2):  # warm: the traced step is a steady-state one
        spec.step(tobj)
    tctx.sync()
    t_first = G.gdag_stats_get(tctx.h).nodes
    spec.step(tobj)
    tctx.sync()
    tr = [t for t in tctx.trace() if t[0] >= t_first]
    comp = [(t[3], t[4]) for t in tr if t[1] in (G.GDAG_NODE_KERNEL, G.GDAG_NODE_GRAPH, G.GDAG_NODE_EXTERNAL)]
    tran = [(t[3], t[4]) for t in tr if t[1] in (G.GDAG_NODE_HOST_WRITE, G.GDAG_NODE_HOST_READ,
                                                  G.GDAG_NODE_HOST_PREFETCH) and t[4] > t[3]]
    overlap = analysis.overlap_metrics(comp, tran)
    tctx.close()
    del tobj
    return {
        "makespan_ms": out, "steps_timed": steps, "nodes": len(elems) - first, "kernels": kern,
        "streams": streams_used,
        "algorithmic_hbm_bytes": hbm, "h2d_bytes": h2d, "d2h_bytes": d2h,
        "speedup_vs_serial_async": out["serial_async_one_stream"] / out["parallel"],
        "speedup_vs_serial_sync": out["serial_sync"] / out["parallel"],
        "vs_hand_cuda_graph": out["hand_cuda_graph"] / out["parallel"],
        "library_graph_vs_hand_cuda_graph": out["hand_cuda_graph"] / out["library_graph"],
        "single_calls_vs_hand_cuda_graph": out["hand_cuda_graph"] / out["parallel_single_calls"],
        "auto_graph_vs_hand_cuda_graph": out["hand_cuda_graph"] / out["parallel_auto_graph"],
        "elements_per_step": elements_per_step,
        "frac_of_cp_bound": cp / out["parallel"], "frac_of_resource_bound": res / out["parallel"],
        "launches_per_step": kern, "per_kernel_solo": per_kernel,
        "makespan_single_run_ms": single, "overlap": overlap,
    }


def run_serving(args, torch, datagen, data):
    """The serving loop (Section III-B's non-blocking completion, run as a
    request server): Poisson arrivals of the five request kinds at their
    drawn scales, on one context.  Fusion thresholds come from the
    autotuner, the per-kind GPU-time model from a calibration pass; the
    admission window is picked by p99 at the configured rate."""
    from paper_2012_09646_gb300 import autotune as AT
    from paper_2012_09646_gb300 import serve as SV
    rate0 = 2000.0
    t0 = time.perf_counter()
    inputs = SV.Inputs(datagen, full_data=data, workers=max(1, min(15, (os.cpu_count() or 2) - 1)))
    out = {"kinds": list(SV.KINDS), "scale": "U[1/64, 1] per request (DL: batch 16, unscaled)",
           "hits_graph_scales": inputs.hits_buckets, "budget_gb": 40, "response_bytes_max": SV.RESPONSE_BYTES,
           "inputs_s": time.perf_counter() - t0, "runs": []}
    keep = []

    def bs_member(ctx_, n, i):
        St, Ct = torch.rand(n, device="cuda") * 90 + 10, torch.empty(n, device="cuda")
        keep.append((St, Ct))
        return (ctx_.array(St), ctx_.array(Ct), n, 60.0, 0.1, 0.2, 1.0)

    def sq_member(ctx_, n, i):
        Xt = torch.rand(n, device="cuda")
        keep.append(Xt)
        return (ctx_.array(Xt), n)
    fr = (1 / 64, 1 / 8, 1 / 4, 1 / 2, 1.0)
    thr_bs, t_bs = AT.tune_fusion("bs_call", bs_member, [int(1e7 * s) for s in fr], group=10, reps=5)
    thr_sq, t_sq = AT.tune_fusion("vec_square", sq_member, [int(1e6 * s) for s in fr], group=8, reps=5)
    del keep
    fuse_max = {"B&S": thr_bs, "VEC": thr_sq}
    out["fusion"] = {"fuse_max_elems": fuse_max,
                     "bs_call_group10_ms": {str(n): {"separate": a, "fused": b} for n, (a, b) in t_bs.items()},
                     "vec_square_group8_ms": {str(n): {"separate": a, "fused": b} for n, (a, b) in t_sq.items()}}
    cost = None

    def one(rate, window, fm, split=None, seed=7, long_window=None):
        nonlocal cost
        srv = SV.Server(inputs, fuse_max=fm, max_streams=32, window_ms=window, split_ms=split,
                        long_window_ms=long_window)
        srv.warm(calibrate=cost is None)
        if cost is None:
            cost = dict(srv.cost)
        srv.cost = dict(cost)
        f0 = sum(c.stats()["fused_members"] for c in srv.ctxs.values())
        reqs = SV.poisson_requests(rate, int(rate * args.serve_seconds), seed=seed)
        srv.run(reqs)
        fused = sum(c.stats()["fused_members"] for c in srv.ctxs.values()) - f0
        srv.close()
        return dict(SV.latency_summary(reqs), offered_req_s=rate, window_ms=window, split_ms=split,
                    long_window_ms=long_window if long_window is not None else window, fusion=bool(fm),
                    fused_members=fused)
    # the admission window (estimated GPU ms in flight) and the class split
    # (requests estimated above split_ms form the long class, short ones run
    # on high-priority streams): among the settings that keep up with the
    # configured rate, those whose p99 is within 15% of the best p99 (one
    # short sweep run's noise), and of those the lowest p50
    sweep = {}
    for w, split, lw in ((1.0, None, None), (2.0, None, None), (4.0, None, None), (1.0, 0.5, 2.0), (2.0, 0.5, 2.0),
                         (1.0, 0.5, 4.0), (2.0, 0.5, 4.0)):
        q = one(rate0, w, fuse_max, split, seed=8, long_window=lw)
        sweep[(w, split, lw)] = {k: q[k] for k in ("p50_ms", "p99_ms", "throughput_req_s")}
    keeps_up = [k for k in sweep if sweep[k]["throughput_req_s"] >= 0.97 * rate0] or list(sweep)
    p99_best = min(sweep[k]["p99_ms"] for k in keeps_up)
    near = [k for k in keeps_up if sweep[k]["p99_ms"] <= 1.15 * p99_best]
    best_w, best_split, best_lw = min(near, key=lambda k: sweep[k]["p50_ms"])
    out["cost_model_ms"] = {k: {"a": a, "b": b} for k, (a, b) in cost.items()}
    out["sweep_2000_req_s"] = {"window %s split %s long window %s" % k: v for k, v in sweep.items()}
    out["window_ms"] = best_w
    out["split_ms"] = best_split
    out["long_window_ms"] = best_lw
    out["max_streams"] = 32
    # the configured rate (the headline), without fusion, at half the rate,
    # and without a window or classes (admission by memory alone)
    for rate, w, fm, split, lw in ((rate0, best_w, fuse_max, best_split, best_lw),
                                   (rate0, best_w, None, best_split, best_lw),
                                   (1000.0, best_w, fuse_max, best_split, best_lw),
                                   (rate0, None, fuse_max, None, None)):
        out["runs"].append(one(rate, w, fm, split, long_window=lw))
    del inputs
    return out


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import datagen
    from paper_2012_09646_gb300 import analysis
    from paper_2012_09646_gb300 import gdag as G
    from paper_2012_09646_gb300 import workloads as W
    from paper_2012_09646_gb300 import replicas as RP

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist:
            dist.barrier()

    which = ["bs"] + (["vec", "img", "ml", "hits", "dl", "hits_batch"] if args.dags == "all" and rank == 0 else [])
    data = make_data(datagen, which)
    prices = data["bs"]
    s0 = torch.cuda.Stream()
    K, r, sg, T = BS_PARAMS
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    # ---- headline: B&S under the PARALLEL policy, inputs resident in HBM
    ctx = G.Context(device=local_rank, policy=G.GDAG_POLICY_PARALLEL)
    dag = W.BsDag(ctx, N_OPTS, count=N_VEC, host=False)
    dag.load_device(prices)
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(local_rank, uuid)
    clocks.__enter__()
    for _ in range(args.warmup):
        dag.step_resident()
    ctx.sync()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s0)
    ctx.fork(s0.cuda_stream)
    for _ in range(args.steps):
        dag.step_resident()
    ctx.wait_all(s0.cuda_stream)
    e1.record(s0)
    torch.cuda.synchronize()
    ms_par = e0.elapsed_time(e1) / args.steps
    ctx.sync()
    barrier()
    ms_all = RP.job_time_ms(dist, ms_par, device=dev)

    out = None
    if RP.reports(rank):
        nsteps_other = max(5, args.steps // 2)
        # ---- the dominant kernel alone: bs_call, 20 launches back to back
        # (one per price vector in turn: 800 MB cycled, more than L2),
        # replayed from a CUDA graph so that the host's launch rate is not
        # what is timed
        reps = 20
        turn = [0]

        def one_bs(sh):
            i = turn[0] % N_VEC
            turn[0] += 1
            ctx.launch_raw("bs_call", dag.SA[i], dag.CA[i], N_OPTS, K, r, sg, T, stream=sh)
        ms_solo = time_launches(torch, one_bs, reps)
        bytes_launch = BYTES_PER_OPTION * N_OPTS
        achieved = bytes_launch / (ms_solo * 1e-3) / 1e9
        # the floor of one launch moving this many bytes: the same 40 MB in
        # and 40 MB out through PyTorch's elementwise kernel (a plain copy),
        # replayed the same way (a launch this short pays its ramp and tail)
        turn_c = [0]

        def one_copy(sh):
            i = turn_c[0] % N_VEC
            turn_c[0] += 1
            torch.mul(dag.S[i], 1.0, out=dag.C[i])
        ms_copy = time_launches(torch, one_copy, reps)

        # ---- host link bandwidths (copy engines), for the transfer bounds
        link = {}
        hb = torch.empty(N_OPTS, dtype=torch.float32, pin_memory=True)
        db = torch.empty(N_OPTS, dtype=torch.float32, device=dev)
        for kind, (dst, src) in (("h2d", (db, hb)), ("d2h", (hb, db))):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            link[kind] = 3 * 4 * N_OPTS / (time.perf_counter() - t0) / 1e9
        del hb, db
        # both directions at once, as in the e2e step but with nothing else
        # to do: N_VEC vectors in on one stream while N_VEC vectors go out
        # on another
        hb_in = torch.empty(N_VEC * N_OPTS, dtype=torch.float32, pin_memory=True)
        hb_out = torch.empty(N_VEC * N_OPTS, dtype=torch.float32, pin_memory=True)
        db_in = torch.empty(N_VEC * N_OPTS, dtype=torch.float32, device=dev)
        db_out = torch.zeros(N_VEC * N_OPTS, dtype=torch.float32, device=dev)
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        duplex_ms = []
        for rep in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(s_in):
                db_in.copy_(hb_in, non_blocking=True)
            with torch.cuda.stream(s_out):
                hb_out.copy_(db_out, non_blocking=True)
            torch.cuda.synchronize()
            if rep:
                duplex_ms.append((time.perf_counter() - t0) * 1e3)
        link["duplex_ms"] = statistics.median(duplex_ms)
        link["duplex_gbs"] = 2 * N_VEC * 4 * N_OPTS / (link["duplex_ms"] * 1e-3) / 1e9
        del hb_in, hb_out, db_in, db_out

        # ---- every DAG of the suite: policies, hand-built CUDA Graph, bounds
        specs = [BsSpec(G, W, data)]
        if args.dags == "all":
            specs += [VecSpec(G, W, data), ImgSpec(G, W, data), MlSpec(G, W, data), HitsSpec(G, W, data),
                      DlSpec(G, W, data), HitsBatchSpec(G, W, data)]
        dags = {}
        for sp in specs:
            dags[sp.name] = measure_dag(torch, G, sp, nsteps_other, hbm, link)
        if "HITS" in dags:
            # the SpMV's own ceiling: random 4-byte reads of a vector that
            # fits in L2 move a 32-byte sector each, so any SpMV of this graph
            # is bounded by the time of a plain gather of nnz values from an
            # n-vector (timed here with PyTorch's index_select as an
            # independent yardstick, like the copy and GEMM peaks)
            n_h = len(data["hits"][0][0]) - 1
            nnz_h = int(data["hits"][0][0][-1])
            xg = torch.rand(n_h, device=dev)
            ig = torch.randint(0, n_h, (nnz_h,), device=dev, dtype=torch.int64)
            yg = torch.empty(nnz_h, device=dev)
            ms_g = time_launches(torch, lambda sh: torch.index_select(xg, 0, ig, out=yg), 5)
            del xg, ig, yg
            hd = dags["HITS"]
            pk = hd["per_kernel_solo"]["spmv_csr"]
            per_spmv = pk["solo_ms"] / pk["launches"]
            # a resource bound that knows the gathers: the SpMVs share one
            # gather path, so their gather times add up; the other kernels are
            # bounded by their HBM bytes
            other_bytes = hd["algorithmic_hbm_bytes"] - pk["alg_bytes"]
            res_g = max(hd["makespan_ms"]["resource_bound"],
                        pk["launches"] * ms_g + other_bytes / (hbm * 1e9) * 1e3)
            hd["gather_bound"] = {
                "what": "torch.index_select of %d random float32 from a %d-vector (index int64)" % (nnz_h, n_h),
                "ms": ms_g, "spmv_ms": per_spmv, "spmv_frac_of_gather_bound": ms_g / per_spmv,
                "resource_bound_with_gathers_ms": res_g,
                "frac_of_resource_bound_with_gathers": res_g / hd["makespan_ms"]["parallel"]}
        if "HITS-batch" in dags:
            hb = data["hits_batch"]
            sep = measure_hits_separate(torch, G, W, hb, max(2, nsteps_other // 4))
            fused = dags["HITS-batch"]
            fused["graphs"] = len(hb)
            fused["vertices"] = int(sum(len(g[0][0]) - 1 for g in hb))
            fused["edges"] = int(sum(int(g[0][0][-1]) for g in hb))
            fused["separate_programs"] = sep
            fused["speedup_vs_separate_programs"] = sep["makespan_ms"] / fused["makespan_ms"]["parallel"]
        bsm = dags["B&S"]["makespan_ms"]

        # ---- serving: Poisson streams of DAG requests on one context
        serve_out = None
        if args.dags == "all" and args.serve:
            serve_out = run_serving(args, torch, datagen, data)

        # ---- e2e through the public API with host buffers: each vector's
        # copy-price-copy chain whole, and in ranges (independent chains
        # whose copies overlap on both link directions); the fastest is the
        # e2e figure
        n_e2e = max(5, args.steps // 5)
        e2e_by_chunks = {}
        best = None
        for chunks in (1, 4):
            ctx2 = G.Context(device=local_rank, policy=G.GDAG_POLICY_PARALLEL)
            d2 = W.BsDag(ctx2, N_OPTS, count=N_VEC, host=True, chunks=chunks)
            d2.load_host(prices)
            for _ in range(2):
                d2.step_e2e()
            ctx2.sync()
            # each step ends with its host reads (the step's results are on
            # the host), so per-step host times are complete; the median of
            # them is the step time (a shared host link can stall a single step)
            torch.cuda.synchronize()
            step_ms = []
            for _ in range(n_e2e):
                t0 = time.perf_counter()
                d2.step_e2e()
                step_ms.append((time.perf_counter() - t0) * 1e3)
            med = statistics.median(step_ms)
            e2e_by_chunks[chunks] = {"ms_per_step": med, "min_max": [min(step_ms), max(step_ms)]}
            ctx2.sync()
            if best is None or med < best[1]:
                if best is not None:
                    best[2].close()
                best = (chunks, med, ctx2, d2, step_ms)
            else:
                ctx2.close()
        e2e_chunks, ms_e2e, ctx2, d2, step_ms = best
        from oracle import numeric as N
        idx = np.arange(0, N_OPTS, 997)
        ref = N.bs_call(prices[3][idx], K, r, sg, T)
        got = d2.hC[3].numpy()[idx].astype(np.float64)
        e2e_err = float((np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)).max())
        ctx2.close()
        # one traced e2e step: copy/compute overlap (Section IV-F)
        ctx3 = G.Context(device=local_rank, trace=True)
        d3 = W.BsDag(ctx3, N_OPTS, count=N_VEC, host=True, chunks=e2e_chunks)
        d3.load_host(prices)
        d3.step_e2e()
        ctx3.sync()
        tr = ctx3.trace()
        comp = [(t[3], t[4]) for t in tr if t[1] == G.GDAG_NODE_KERNEL]
        tran = [(t[3], t[4]) for t in tr if t[1] != G.GDAG_NODE_KERNEL]
        overlap = analysis.overlap_metrics(comp, tran)
        ctx3.close()
        clocks.__exit__(None, None, None)

        # ---- CPU oracle baseline (bounded samples): one thread in program
        # order, then every host core at once
        cpu_val, cpu_samples, cpu_s = cpu_oracle_rate(args.cpu_seconds)
        cpu_all, cpu_cores, cpu_all_s = cpu_oracle_rate_all_cores(max(1.0, args.cpu_seconds / 2))

        value = RP.job_value(world, 1, ms_all)  # one DAG per rank per step
        gpu_launches = args.steps * N_VEC
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "policy": "PARALLEL (run-time DAG, multi-stream)",
                       "l2": "inputs larger than L2 (800 MB touched per step)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "makespan_ms": dict(bsm, parallel_headline=ms_par),
            "speedup_vs_serial_async": bsm["serial_async_one_stream"] / ms_par,
            "speedup_vs_serial_sync": bsm["serial_sync"] / ms_par,
            "vs_hand_cuda_graph": bsm["hand_cuda_graph"] / ms_par,
            "frac_of_cp_bound": bsm["critical_path_bound"] / ms_par,
            "frac_of_resource_bound": bsm["resource_bound"] / ms_par,
            "roofline": {"kernel": "bs_call", "bound": "hbm", "achieved": achieved, "peak": hbm,
                         "peak_source": peak_src + " hbm_gbs (burst; kernel timed alone)", "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": bs_call_traffic(),
                         "traffic_note": BS_CALL_TRAFFIC["note"],
                         "algorithmic_bytes_per_launch": bytes_launch, "launch_ms": ms_solo,
                         "copy_same_bytes_ms": ms_copy, "copy_same_bytes_frac": bytes_launch / (ms_copy * 1e-3) / 1e9 / hbm,
                         "frac_of_copy_same_bytes": ms_copy / ms_solo},
            "e2e": {"value": 1e3 / ms_e2e, "unit": UNIT, "ms_per_step": ms_e2e,
                    "ms_per_step_min_max": [min(step_ms), max(step_ms)], "steps_timed": n_e2e,
                    "chains_per_vector": e2e_chunks, "ms_per_step_by_chains_per_vector": e2e_by_chunks,
                    "h2d_bytes_per_step": N_VEC * 4 * N_OPTS, "d2h_bytes_per_step": N_VEC * 4 * N_OPTS,
                    "max_rel_err_sampled": e2e_err, "overlap": overlap,
                    "link_gbs": {k: v for k, v in link.items() if k != "duplex_ms"},
                    "link_bound_ms": max(N_VEC * 4 * N_OPTS / (link["h2d"] * 1e9),
                                         N_VEC * 4 * N_OPTS / (link["d2h"] * 1e9)) * 1e3,
                    "duplex_copy_ms": link["duplex_ms"],
                    "frac_of_duplex_copy": link["duplex_ms"] / ms_e2e},
            "dags": dags,
            "serve": serve_out,
            "cpu_baseline": {"value": cpu_val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d samples of 10 x 1e6 options (fp64 C oracle, one thread) in %.1f s; "
                                       "scaled to whole DAGs" % (cpu_samples, cpu_s)},
            "cpu_baseline_all_cores": {"value": cpu_all, "unit": UNIT, "cores": cpu_cores, "kind": "oracle",
                                       "sample": "%d processes, each pricing 10 x 2.5e5 options repeatedly with the "
                                                 "fp64 C oracle for %.1f s; scaled to whole DAGs"
                                                 % (cpu_cores, cpu_all_s)},
            "gpu_launches": gpu_launches,
            "clocks": dict(clocks.summary(), window="warm-up through the last GPU measurement"),
        }
        out["summary"] = compact_summary(out)
    clocks.__exit__(None, None, None)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)
        print_summary(out)


def compact_summary(out):
    """The bench line's headline results in a few hundred characters, placed
    last on the line so that a reader who keeps only the line's end still has
    them: per DAG the PARALLEL makespan (ms) and its speedups over
    SERIAL_SYNC and over the hand-built CUDA Graph, the automatically
    captured and replayed steps against that graph, with the fractions of the
    critical-path and resource bounds; per served rate the p50 / p99 latency
    (ms) and the served rate, with and without fusion and the admission
    window; the kernels' cold solo fractions of HBM."""
    r3 = lambda v: None if v is None else round(float(v), 3)
    dags = {}
    for name, d in (out.get("dags") or {}).items():
        dags[name] = [r3(d["makespan_ms"]["parallel"]), r3(d["speedup_vs_serial_sync"]),
                      r3(d["vs_hand_cuda_graph"]), r3(d.get("auto_graph_vs_hand_cuda_graph")),
                      r3(d["frac_of_cp_bound"]), r3(d["frac_of_resource_bound"])]
    kern = {}
    for d in (out.get("dags") or {}).values():
        for k, v in d.get("per_kernel_solo", {}).items():
            if v.get("frac_of_hbm_peak") is not None:
                kern[k] = max(kern.get(k, 0.0), round(v["frac_of_hbm_peak"], 2))
    serve = []
    for rr in ((out.get("serve") or {}).get("runs") or []):
        serve.append([rr["offered_req_s"], int(rr["fusion"]), int(rr.get("window_ms") is not None),
                      r3(rr["throughput_req_s"]), r3(rr["p50_ms"]), r3(rr["p99_ms"])])
    return {"dag_cols": ["parallel_ms", "vs_serial_sync", "vs_hand_graph", "auto_graph_vs_hand_graph", "of_cp_bound",
                         "of_resource_bound"],
            "dags": dags, "serve_cols": ["offered_req_s", "fusion", "admission_window", "served_req_s", "p50_ms", "p99_ms"],
            "serve": serve, "kernel_cold_frac_of_hbm": kern,
            "bs_call_frac": r3(out["roofline"]["frac"]), "e2e_ms": r3(out["e2e"]["ms_per_step"])}


def print_summary(out):
    """A short human-readable digest of the bench line on stderr."""
    w = sys.stderr.write
    e2e = out["e2e"]
    w("summary: %s %.0f %s resident (%.3f ms/step), e2e %.1f %s (%.3f ms/step, %s of a duplex copy); "
      "%s %.3f of HBM peak\n" % (
        out["config"]["workload"].split(":")[0], out["value"], out["unit"], out["ms_per_step"], e2e["value"],
        out["unit"], e2e.get("ms_per_step", 0.0),
        "%.2f" % e2e["frac_of_duplex_copy"] if "frac_of_duplex_copy" in e2e else "n/a",
        out["roofline"]["kernel"], out["roofline"]["frac"]))
    w("%-11s %8s %8s %8s %8s %8s %8s %8s\n" % ("DAG", "par_ms", "vsSYNC", "vsGraph", "1call/G", "auto/G", "ofCP",
                                                "ofRes"))
    for name, d in (out.get("dags") or {}).items():
        m = d["makespan_ms"]
        w("%-11s %8.3f %8.2f %8.2f %8.2f %8.2f %8.2f %8.2f\n" % (
            name, m["parallel"], d["speedup_vs_serial_sync"], d["vs_hand_cuda_graph"],
            d["single_calls_vs_hand_cuda_graph"], d["auto_graph_vs_hand_cuda_graph"], d["frac_of_cp_bound"],
            d["frac_of_resource_bound"]))
    sv = out.get("serve")
    if sv:
        for r in sv["runs"]:
            w("serve %5.0f req/s window %s/%s split %s fusion %d: served %.0f req/s p50 %.2f ms p99 %.2f ms "
              "(queue p99 %.2f, device p99 %.2f)\n" % (
                  r["offered_req_s"], r["window_ms"], r["long_window_ms"], r["split_ms"], r["fusion"],
                  r["throughput_req_s"], r["p50_ms"], r["p99_ms"], r["queue_p99_ms"], r["device_p99_ms"]))
            for c, v in sorted(r.get("by_class", {}).items()):
                w("      class %s: %d requests p50 %.2f ms p99 %.2f ms\n" % (c, v["n"], v["p50_ms"], v["p99_ms"]))
    sys.stderr.flush()


def run_profile(args):
    """One DAG, one PARALLEL context, warm-up plus --steps steps, nothing
    else on the device (a few GB at most)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import datagen
    from paper_2012_09646_gb300 import gdag as G
    from paper_2012_09646_gb300 import workloads as W
    torch.cuda.set_device(0)
    ctx = G.Context()
    if args.profile == "bs":
        d = W.BsDag(ctx, N_OPTS, count=N_VEC, host=False)
        d.load_device(datagen.bs_inputs(N_OPTS, count=N_VEC, seed=1))
        step = d.step_resident
    elif args.profile == "bs_fused":
        # a serving burst: eight B&S requests of 1/4 scale (10 nodes of
        # 2.5e6 options each) as one fused element of 80 members
        n = N_OPTS // 4
        reqs = [W.BsDag(ctx, n, count=N_VEC, host=False) for _ in range(8)]
        prices = datagen.bs_inputs(n, count=N_VEC, seed=1)
        for d in reqs:
            d.load_device(prices)
        K, r, sg, T = BS_PARAMS
        members = [(Sa, Ca, n, K, r, sg, T) for d in reqs for Sa, Ca in zip(d.SA, d.CA)]
        step = lambda: ctx.launch_fused("bs_call", members)
    elif args.profile == "vec":
        d = W.VecDag(ctx, args.vec_n)
        d.load(*datagen.vec_inputs(args.vec_n, seed=0))
        step = d.step
    elif args.profile == "img":
        n = args.img_size
        d = W.ImgDag(ctx, n, n)
        d.img.copy_(torch.from_numpy(datagen.image(n, n, seed=2).reshape(-1)).cuda())
        step = d.launch_all
    elif args.profile == "ml":
        d = W.MlDag(ctx, 100_000)
        d.load(*datagen.ml_inputs(100_000, feats=1024, classes=10, seed=3))
        step = d.launch_all
    elif args.profile == "hits_batch":
        d = W.HitsBatchDag(ctx, datagen.hits_batch(count=64, nmin=10_000, nmax=1_000_000, seed=6))
        d.run(iters=0, read=False)
        spec = HitsBatchSpec(G, W, {})
        step = lambda: spec.step(d)
    elif args.profile == "dl":
        d = W.DlDag(ctx)
        d.load(*datagen.dl_inputs(n=16, h=256, w=256, seed=5)[0])
        step = d.launch_all
    else:
        d = W.HitsDag(ctx, *datagen.hits_graph(10_000_000, 50_000_000, seed=4))
        d.run(iters=0, read=False)
        spec = HitsSpec(G, W, {})
        step = lambda: spec.step(d)
    for _ in range(args.warmup + args.steps):
        step()
    ctx.sync()
    torch.cuda.synchronize()
    ctx.close()


def main():
    args = parse()
    if args.profile:
        run_profile(args)
        return
    from paper_2012_09646_gb300 import replicas as RP
    rank, world, local_rank = RP.rank_env()
    # timed numbers follow at least three untimed warm-up steps; the JSON
    # line reports the count actually run
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
