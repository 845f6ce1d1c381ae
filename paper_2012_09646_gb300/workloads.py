"""The benchmark programs of Section IV-B as plain launch sequences.

Each class owns its device arrays (torch tensors, the only use of PyTorch:
device memory) and pinned host views, registers them with a
:class:`~paper_2012_09646_gb300.gdag.Context`, and issues one DAG iteration
per ``step`` call exactly as a user program would: host writes, kernel
launches with per-argument access modes, host reads.  The dependency DAG,
streams, events and copies are entirely the library's.

With ``batched=True`` (the default) the non-blocking elements of a step are
recorded once as a :class:`~paper_2012_09646_gb300.gdag.Program` and issued
with one ``gdag_issue`` call per step; the library infers, places and
issues each element exactly as one call per element would (``batched=False``),
but the host's per-element cost leaves the critical path of short DAGs.
"""
from __future__ import annotations

import torch

from . import gdag as G

F32 = torch.float32


def _pinned(shape, dtype):
    return torch.empty(shape, dtype=dtype, pin_memory=True)


class _Calls:
    """The Program recording interface, one library call per element."""

    def __init__(self, ctx):
        self.ctx = ctx

    def launch(self, name, *args, **kw):
        return self.ctx.launch(name, *args, **kw)

    def write(self, a, off=0, nbytes=None):
        return self.ctx.write(a, None, off, nbytes)

    def prefetch_host(self, a, off=0, nbytes=None):
        return self.ctx.prefetch_host(a, off, nbytes)


class _Issuer:
    """Issues a DAG's recorded element sequences: one Program per sequence
    (recorded on first use) when batched, else one call per element."""

    def _init_issuer(self, ctx, batched):
        self._batched = batched
        self._progs = {}

    def _run(self, key, record):
        """record(c) issues the sequence on c, which has the Program
        recording interface (launch, write from the view, prefetch_host)."""
        if not self._batched:
            record(_Calls(self.ctx))
            return
        p = self._progs.get(key)
        if p is None:
            p = self.ctx.program()
            record(p)
            self._progs[key] = p
        p.issue()


def _scratch(ctx, kernel, n, device):
    nbytes = G.gdag_scratch_bytes(kernel, n)
    t = torch.zeros(nbytes, dtype=torch.uint8, device=device)
    return t, ctx.array(t, name=kernel + "_scratch")


class VecDag(_Issuer):
    """VEC: host writes x and y; K1 x := x*x; K2 y := y*y; K3 z = sum(x - y);
    host reads z."""

    def __init__(self, ctx, n, device="cuda", batched=True):
        self.ctx, self.n = ctx, n
        self._init_issuer(ctx, batched)
        self.x = torch.zeros(max(n, 1), dtype=F32, device=device)
        self.y = torch.zeros(max(n, 1), dtype=F32, device=device)
        self.z = torch.zeros(1, dtype=F32, device=device)
        self.hx, self.hy, self.hz = _pinned(max(n, 1), F32), _pinned(max(n, 1), F32), _pinned(1, F32)
        # the result is read through a numpy view of the pinned scalar: a
        # torch element access costs the host several microseconds, which a
        # host-synchronised step of this size would pay on its critical path
        self._hz_np = self.hz.numpy()
        self.X = ctx.array(self.x, host=self.hx, name="x")
        self.Y = ctx.array(self.y, host=self.hy, name="y")
        self.Z = ctx.array(self.z, host=self.hz, name="z")
        self._s, self.S = _scratch(ctx, "vec_reduce_diff", n, device)

    def load(self, x, y):
        """Put new inputs into the pinned host views (host-side, untimed)."""
        self.hx[: self.n].copy_(torch.as_tensor(x))
        self.hy[: self.n].copy_(torch.as_tensor(y))

    def _elements(self, c):
        n = self.n
        c.write(self.X, 0, 4 * n)
        c.write(self.Y, 0, 4 * n)
        c.launch("vec_square", self.X, n)
        c.launch("vec_square", self.Y, n)
        c.launch("vec_reduce_diff", self.X, self.Y, self.Z, self.S, n)

    def step(self, read=True):
        self._run("step", self._elements)
        if read:
            self.ctx.read(self.Z)
            return float(self._hz_np[0])
        return None


class BsDag(_Issuer):
    """B&S: `count` independent call-price nodes.  With ``host_inputs`` each
    step rewrites every price vector from the host (copy nodes overlapping
    the other chains' kernels) and reads every result back."""

    def __init__(self, ctx, n, count=10, K=60.0, r=0.1, sigma=0.2, T=1.0, device="cuda", host=True,
                 batched=True, chunks=1):
        """``chunks`` > 1 (with ``host``): each vector's copy-price-copy
        chain of step_e2e is issued as `chunks` independent chains over
        consecutive ranges of the vector (each range registered as its own
        array over the same memory), so the copies of different ranges
        overlap on both directions of the host link with a short fill and
        drain; the prices are the same.  The range arrays share memory with
        the whole-vector arrays (S, C), which the library tracks as other
        arrays: a program that mixes step_e2e with the whole-vector steps
        must order them itself (e.g. a sync between them)."""
        self.ctx, self.n, self.count = ctx, n, count
        self._init_issuer(ctx, batched)
        self.params = (float(K), float(r), float(sigma), float(T))
        self.S = [torch.zeros(max(n, 1), dtype=F32, device=device) for _ in range(count)]
        self.C = [torch.zeros(max(n, 1), dtype=F32, device=device) for _ in range(count)]
        self.hS = [_pinned(max(n, 1), F32) for _ in range(count)] if host else [None] * count
        self.hC = [_pinned(max(n, 1), F32) for _ in range(count)] if host else [None] * count
        self.SA = [ctx.array(t, host=h, name="S%d" % i) for i, (t, h) in enumerate(zip(self.S, self.hS))]
        self.CA = [ctx.array(t, host=h, name="C%d" % i) for i, (t, h) in enumerate(zip(self.C, self.hC))]
        self.chunks = max(1, chunks) if host else 1
        self.parts = []  # per vector: [(lo, hi, S range array, C range array)]
        if self.chunks > 1:
            # a multiple of 4 floats, so every range is 16-byte aligned
            step = max(4, ((n + self.chunks - 1) // self.chunks + 3) // 4 * 4)
            for i in range(count):
                rs = []
                for lo in range(0, n, step):
                    hi = min(n, lo + step)
                    nb = 4 * (hi - lo)
                    sa = ctx.array(dev=self.S[i].data_ptr() + 4 * lo, nbytes=nb, host=self.hS[i].data_ptr() + 4 * lo,
                                   name="S%d[%d:%d]" % (i, lo, hi))
                    ca = ctx.array(dev=self.C[i].data_ptr() + 4 * lo, nbytes=nb, host=self.hC[i].data_ptr() + 4 * lo,
                                   name="C%d[%d:%d]" % (i, lo, hi))
                    rs.append((lo, hi, sa, ca))
                self.parts.append(rs)

    def load_host(self, prices):
        for h, p in zip(self.hS, prices):
            h[: self.n].copy_(torch.as_tensor(p))

    def load_device(self, prices):
        for d, p in zip(self.S, prices):
            d[: self.n].copy_(torch.as_tensor(p).to(d.device))
        torch.cuda.synchronize()

    def _kernels(self, c):
        K, r, s, T = self.params
        for Sa, Ca in zip(self.SA, self.CA):
            c.launch("bs_call", Sa, Ca, self.n, K, r, s, T)

    def launch_all(self):
        self._run("kernels", self._kernels)

    def step_resident(self):
        """Kernels only (inputs already in HBM); no host access."""
        self.launch_all()

    def _chains(self, c, prefetch):
        nb = 4 * self.n
        K, r, s, T = self.params
        for Sa, Ca in zip(self.SA, self.CA):
            c.write(Sa, 0, nb)
            c.launch("bs_call", Sa, Ca, self.n, K, r, s, T)
            if prefetch:
                c.prefetch_host(Ca, 0, nb)

    def _range_chains(self, c, prefetch):
        K, r, s, T = self.params
        for rs in self.parts:
            for lo, hi, sa, ca in rs:
                c.write(sa, 0, 4 * (hi - lo))
                c.launch("bs_call", sa, ca, hi - lo, K, r, s, T)
                if prefetch:
                    c.prefetch_host(ca, 0, 4 * (hi - lo))

    def step_e2e(self, prefetch=True):
        """Host write of every price vector, all kernels, host read of every
        result (the paper's streaming form of the benchmark).  With
        ``prefetch`` each result's copy to the host is started right after its
        kernel, so it overlaps the other chains' input copies."""
        if self.chunks > 1:
            self._run(("e2e_ranges", prefetch), lambda c: self._range_chains(c, prefetch))
            for rs in self.parts:
                for lo, hi, sa, ca in rs:
                    self.ctx.read(ca, None, 0, 4 * (hi - lo))
            return
        self._run(("e2e", prefetch), lambda c: self._chains(c, prefetch))
        for Ca in self.CA:
            self.ctx.read(Ca, None, 0, 4 * self.n)


def gaussian_weights(radius, sigma):
    """Normalised Gaussian taps exp(-k^2 / (2 sigma^2)), k = -radius..radius,
    as float32 (filter parameters of the blur nodes)."""
    import math
    w = [math.exp(-(k * k) / (2.0 * sigma * sigma)) for k in range(-radius, radius + 1)]
    s = sum(w)
    return torch.tensor([v / s for v in w], dtype=F32)


class ImgDag(_Issuer):
    """IMG: blur5 and blur9 of the image, Sobel of each, min/max of each,
    contrast stretch of each edge map, unsharp mask of the image with blur5,
    and the final combination (10 kernels).  The host writes the image and
    reads the result each step."""

    R5, SIGMA5, R9, SIGMA9, ALPHA = 2, 1.0, 4, 2.0, 0.5

    def __init__(self, ctx, rows, cols, device="cuda", batched=True):
        self.ctx, self.rows, self.cols = ctx, rows, cols
        self._init_issuer(ctx, batched)
        n = rows * cols
        self.n = n
        t = lambda: torch.zeros(n, dtype=F32, device=device)
        self.img, self.b5, self.b9, self.e5, self.e9, self.s, self.out = (t() for _ in range(7))
        self.mm5 = torch.zeros(2, dtype=F32, device=device)
        self.mm9 = torch.zeros(2, dtype=F32, device=device)
        self.w5 = gaussian_weights(self.R5, self.SIGMA5).to(device)
        self.w9 = gaussian_weights(self.R9, self.SIGMA9).to(device)
        self.h_img, self.h_out = _pinned(n, F32), _pinned(n, F32)
        A = ctx.array
        self.IMG = A(self.img, host=self.h_img, name="img")
        self.OUT = A(self.out, host=self.h_out, name="out")
        self.B5, self.B9, self.E5, self.E9, self.S = (A(x, name=nm) for x, nm in (
            (self.b5, "b5"), (self.b9, "b9"), (self.e5, "e5"), (self.e9, "e9"), (self.s, "s")))
        self.MM5, self.MM9 = A(self.mm5, name="mm5"), A(self.mm9, name="mm9")
        self.W5, self.W9 = A(self.w5, name="w5"), A(self.w9, name="w9")
        self._s5, self.SC5 = _scratch(ctx, "minmax", n, device)
        self._s9, self.SC9 = _scratch(ctx, "minmax", n, device)

    def load(self, image):
        self.h_img.copy_(torch.as_tensor(image).reshape(-1))

    def _kernels(self, c):
        n, rows, cols = self.n, self.rows, self.cols
        c.launch("gauss_blur", self.IMG, self.B5, self.W5, rows, cols, self.R5)
        c.launch("gauss_blur", self.IMG, self.B9, self.W9, rows, cols, self.R9)
        c.launch("sobel", self.B5, self.E5, rows, cols)
        c.launch("sobel", self.B9, self.E9, rows, cols)
        c.launch("minmax", self.E5, self.MM5, self.SC5, n)
        c.launch("minmax", self.E9, self.MM9, self.SC9, n)
        c.launch("extend", self.E5, self.MM5, n)
        c.launch("extend", self.E9, self.MM9, n)
        c.launch("unsharp", self.IMG, self.B5, self.S, self.ALPHA, n)
        c.launch("combine", self.S, self.B5, self.B9, self.E5, self.E9, self.OUT, n)

    def launch_all(self):
        self._run("kernels", self._kernels)

    def step(self, read=True):
        def elements(c):
            c.write(self.IMG, 0, self.IMG.nbytes)
            self._kernels(c)
        self._run("step", elements)
        if read:
            self.ctx.read(self.OUT)


class MlDag(_Issuer):
    """ML: naive-Bayes scores and ridge scores of the same X (both read-only
    users of X, so they run concurrently), a softmax of each, and the argmax
    of their sum as int32 labels.  X and the tables are resident; the host
    reads the labels each step."""

    def __init__(self, ctx, rows, feats=1024, classes=10, device="cuda", batched=True):
        self.ctx, self.rows, self.feats, self.classes = ctx, rows, feats, classes
        self._init_issuer(ctx, batched)
        self.X = torch.zeros((max(rows, 1), feats), dtype=torch.int32, device=device)
        self.T1 = torch.zeros((feats, classes), dtype=F32, device=device)
        self.b1 = torch.zeros(classes, dtype=F32, device=device)
        self.T2 = torch.zeros((feats, classes), dtype=F32, device=device)
        self.b2 = torch.zeros(classes, dtype=F32, device=device)
        self.S1 = torch.zeros((max(rows, 1), classes), dtype=F32, device=device)
        self.S2 = torch.zeros((max(rows, 1), classes), dtype=F32, device=device)
        self.labels = torch.zeros(max(rows, 1), dtype=torch.int32, device=device)
        self.h_labels = _pinned(max(rows, 1), torch.int32)
        A = ctx.array
        self.XA, self.T1A, self.b1A = A(self.X, name="X"), A(self.T1, name="nb_table"), A(self.b1, name="nb_prior")
        self.T2A, self.b2A = A(self.T2, name="ridge_w"), A(self.b2, name="ridge_b")
        self.S1A, self.S2A = A(self.S1, name="s1"), A(self.S2, name="s2")
        self.LA = A(self.labels, host=self.h_labels, name="labels")

    def load(self, X, nb_table, nb_prior, ridge_w, ridge_b):
        """Device-resident inputs (set once, outside the timed region)."""
        self.X[: self.rows].copy_(torch.as_tensor(X))
        self.T1.copy_(torch.as_tensor(nb_table))
        self.b1.copy_(torch.as_tensor(nb_prior))
        self.T2.copy_(torch.as_tensor(ridge_w))
        self.b2.copy_(torch.as_tensor(ridge_b))
        torch.cuda.synchronize()

    def _kernels(self, c):
        r, f, k = self.rows, self.feats, self.classes
        c.launch("dense_scores", self.XA, self.T1A, self.b1A, self.S1A, r, f, k)
        c.launch("dense_scores", self.XA, self.T2A, self.b2A, self.S2A, r, f, k)
        c.launch("row_softmax", self.S1A, r, k)
        c.launch("row_softmax", self.S2A, r, k)
        c.launch("argmax_combine", self.S1A, self.S2A, self.LA, r, k)

    def launch_all(self):
        self._run("kernels", self._kernels)

    def step(self, read=True):
        self.launch_all()
        if read:
            self.ctx.read(self.LA, None, 0, 4 * self.rows)


class HitsDag(_Issuer):
    """HITS: per iteration a' = A^T h and h' = A a (two SpMVs that read the
    previous iterate, so they run concurrently), the L2 norm of each and the
    scaling by it; ping-pong buffers.  The graph (CSR of A and of A^T, int32
    indices, float32 weights) is resident; the merge-path partition of each
    matrix is computed once by a spmv_partition node.  The host writes
    a = h = 1 and reads both final vectors."""

    def __init__(self, ctx, csr, csc, device="cuda", batched=True):
        self.ctx = ctx
        self._init_issuer(ctx, batched)
        rp, col, val = csr
        trp, tcol, tval = csc
        self.n = n = len(rp) - 1
        self.nnz = nnz = int(rp[-1])
        i32 = torch.int32
        dev = lambda a, dt: torch.as_tensor(a).to(dtype=dt).to(device)
        self.A = (dev(rp, i32), dev(col, i32), dev(val, F32))
        self.AT = (dev(trp, i32), dev(tcol, i32), dev(tval, F32))
        A = ctx.array
        self.AA = [A(t, name=nm) for t, nm in zip(self.A, ("rowptr", "col", "val"))]
        self.ATA = [A(t, name=nm) for t, nm in zip(self.AT, ("t_rowptr", "t_col", "t_val"))]
        pb = G.gdag_scratch_bytes("spmv_partition", n + nnz)
        cb = G.gdag_scratch_bytes("spmv_csr", n + nnz)
        self._pA = torch.zeros(pb, dtype=torch.uint8, device=device)
        self._pAT = torch.zeros(pb, dtype=torch.uint8, device=device)
        self._cA = torch.zeros(cb, dtype=torch.uint8, device=device)
        self._cAT = torch.zeros(cb, dtype=torch.uint8, device=device)
        self.PA, self.PAT = A(self._pA, name="part_A"), A(self._pAT, name="part_AT")
        self.CA, self.CAT = A(self._cA, name="carry_A"), A(self._cAT, name="carry_AT")
        v = lambda: torch.zeros(max(n, 1), dtype=F32, device=device)
        self.vec = {"a": v(), "h": v(), "a2": v(), "h2": v()}
        self.h_a, self.h_h = _pinned(max(n, 1), F32), _pinned(max(n, 1), F32)
        self.V = {k: A(t, host=self.h_a if k == "a" else (self.h_h if k == "h" else None), name=k)
                  for k, t in self.vec.items()}
        self.norms = torch.zeros(2, dtype=F32, device=device)
        self.NA = A(self.norms[0:1], name="norm_a")
        self.NH = A(self.norms[1:2], name="norm_h")
        self._sa, self.SA = _scratch(ctx, "l2norm", n, device)
        self._sh, self.SH = _scratch(ctx, "l2norm", n, device)
        ctx.launch("spmv_partition", self.AA[0], self.PA, n, nnz)
        ctx.launch("spmv_partition", self.ATA[0], self.PAT, n, nnz)

    def _iteration(self, c, a, h, a_next, h_next):
        n, nnz = self.n, self.nnz
        c.launch("spmv_csr", *self.ATA, self.V[h], self.PAT, self.V[a_next], self.CAT, n, nnz)
        c.launch("spmv_csr", *self.AA, self.V[a], self.PA, self.V[h_next], self.CA, n, nnz)
        c.launch("l2norm", self.V[a_next], self.NA, self.SA, n)
        c.launch("l2norm", self.V[h_next], self.NH, self.SH, n)
        c.launch("scale", self.V[a_next], self.NA, n)
        c.launch("scale", self.V[h_next], self.NH, n)

    def iterate(self, a, h, a_next, h_next):
        self._run(("it", a, h, a_next, h_next), lambda c: self._iteration(c, a, h, a_next, h_next))

    def run(self, iters=5, read=True):
        """Host writes a = h = 1, then `iters` iterations; returns the names
        of the buffers holding the final (a, h)."""
        self.h_a.fill_(1.0)
        self.h_h.fill_(1.0)
        self.ctx.write(self.V["a"], None, 0, 4 * self.n)
        self.ctx.write(self.V["h"], None, 0, 4 * self.n)
        cur, nxt = ("a", "h"), ("a2", "h2")
        for _ in range(iters):
            self.iterate(cur[0], cur[1], nxt[0], nxt[1])
            cur, nxt = nxt, cur
        if read:
            for k in cur:
                self.ctx.read(self.V[k], None, 0, 4 * self.n)
        return cur


def block_diag_csr(mats):
    """Block-diagonal concatenation of square CSR matrices given as
    (rowptr, col, val): returns the combined (rowptr, col, val) and the
    segment starts (the first vertex of each matrix, plus the total).  This
    is input layout only (index offsets), done once when a batch is built."""
    import numpy as np
    rps, cols, vals, seg = [], [], [], [0]
    nv, ne = 0, 0
    for rp, col, val in mats:
        rp = np.asarray(rp, dtype=np.int64)
        rps.append(rp[:-1] + ne)
        cols.append(np.asarray(col, dtype=np.int64) + nv)
        vals.append(np.asarray(val, dtype=np.float32))
        nv += rp.size - 1
        ne += int(rp[-1])
        seg.append(nv)
    if nv + ne >= 2 ** 31:
        raise ValueError("batch too large for int32 indexing")
    rowptr = np.concatenate(rps + [np.array([ne], dtype=np.int64)])
    return (rowptr, np.concatenate(cols), np.concatenate(vals)), np.asarray(seg, dtype=np.int64)


class HitsBatchDag(HitsDag):
    """HITS over a batch of independent graphs in one program: the graphs are
    stored block-diagonally, so each SpMV covers every graph, and the norms
    and scaling are per-graph segment kernels -- six launches per iteration
    for the whole batch (the fused form of one HITS program per graph)."""

    def __init__(self, ctx, graphs, device="cuda", batched=True):
        csr, seg = block_diag_csr([g[0] for g in graphs])
        csc, seg_t = block_diag_csr([g[1] for g in graphs])
        assert (seg == seg_t).all()
        super().__init__(ctx, csr, csc, device=device, batched=batched)
        self.G = G_ = len(graphs)
        self.seg_host = seg
        self.seg = torch.as_tensor(seg).to(dtype=torch.int32).to(device)
        self.SEG = ctx.array(self.seg, name="seg")
        self.seg_norms = torch.zeros((2, max(G_, 1)), dtype=F32, device=device)
        self.NAS = ctx.array(self.seg_norms[0], name="norms_a")
        self.NHS = ctx.array(self.seg_norms[1], name="norms_h")
        self._sas, self.SAS = _scratch(ctx, "seg_l2norm", G_, device)
        self._shs, self.SHS = _scratch(ctx, "seg_l2norm", G_, device)
        torch.cuda.synchronize()

    def _iteration(self, c, a, h, a_next, h_next):
        n, nnz, G_ = self.n, self.nnz, self.G
        c.launch("spmv_csr", *self.ATA, self.V[h], self.PAT, self.V[a_next], self.CAT, n, nnz)
        c.launch("spmv_csr", *self.AA, self.V[a], self.PA, self.V[h_next], self.CA, n, nnz)
        c.launch("seg_l2norm", self.V[a_next], self.SEG, self.NAS, self.SAS, G_, n)
        c.launch("seg_l2norm", self.V[h_next], self.SEG, self.NHS, self.SHS, G_, n)
        c.launch("seg_scale", self.V[a_next], self.SEG, self.NAS, G_, n)
        c.launch("seg_scale", self.V[h_next], self.SEG, self.NHS, G_, n)

    def segment(self, vec, g):
        return vec[int(self.seg_host[g]):int(self.seg_host[g + 1])]


class DlDag(_Issuer):
    """DL: two convolution branches (conv3x3 + bias + ReLU + 2x2 max-pool on
    the tensor cores), a global average pool of each, and a dense layer over
    the concatenated embeddings.  bf16 NCHW activations, fp32 embeddings and
    logits; inputs resident, the host reads the logits."""

    def __init__(self, ctx, n=16, h=256, w=256, classes=10, device="cuda", batched=True):
        self.ctx, self.n, self.h, self.w, self.classes = ctx, n, h, w, classes
        self._init_issuer(ctx, batched)
        bf = torch.bfloat16
        self.x1 = torch.zeros((n, 3, h, w), dtype=bf, device=device)
        self.x2 = torch.zeros((n, 3, h, w), dtype=bf, device=device)
        self.w1 = torch.zeros((64, 3, 3, 3), dtype=bf, device=device)
        self.w2 = torch.zeros((64, 3, 3, 3), dtype=bf, device=device)
        self.b1 = torch.zeros(64, dtype=F32, device=device)
        self.b2 = torch.zeros(64, dtype=F32, device=device)
        self.p1 = torch.zeros((n, 64, h // 2, w // 2), dtype=bf, device=device)
        self.p2 = torch.zeros((n, 64, h // 2, w // 2), dtype=bf, device=device)
        self.e1 = torch.zeros((n, 64), dtype=F32, device=device)
        self.e2 = torch.zeros((n, 64), dtype=F32, device=device)
        self.wd = torch.zeros((128, classes), dtype=F32, device=device)
        self.bd = torch.zeros(classes, dtype=F32, device=device)
        self.logits = torch.zeros((n, classes), dtype=F32, device=device)
        # one status word per branch: a shared one would order the two
        # branches (both write it)
        self.status = torch.zeros(2, dtype=torch.int32, device=device)
        self.h_logits = _pinned((n, classes), F32)
        A = ctx.array
        self.X1, self.X2, self.W1, self.W2 = A(self.x1), A(self.x2), A(self.w1), A(self.w2)
        self.B1, self.B2, self.P1, self.P2 = A(self.b1), A(self.b2), A(self.p1), A(self.p2)
        self.E1, self.E2, self.WD, self.BD = A(self.e1), A(self.e2), A(self.wd), A(self.bd)
        self.LOG = A(self.logits, host=self.h_logits)
        self.ST1, self.ST2 = A(self.status[0:1]), A(self.status[1:2])
        torch.cuda.synchronize()

    def load(self, x1, x2, w1, b1, w2, b2, wd, bd):
        """float32 inputs whose x and w values bfloat16 holds exactly."""
        for dst, src in ((self.x1, x1), (self.x2, x2), (self.w1, w1), (self.w2, w2)):
            dst.copy_(torch.as_tensor(src).to(torch.bfloat16))
        for dst, src in ((self.b1, b1), (self.b2, b2), (self.wd, wd), (self.bd, bd)):
            dst.copy_(torch.as_tensor(src))
        torch.cuda.synchronize()

    def _kernels(self, c):
        n, h, w = self.n, self.h, self.w
        c.launch("conv3x3_relu_pool", self.X1, self.W1, self.B1, self.P1, self.ST1, n, h, w)
        c.launch("conv3x3_relu_pool", self.X2, self.W2, self.B2, self.P2, self.ST2, n, h, w)
        c.launch("avgpool_global", self.P1, self.E1, n * 64, (h // 2) * (w // 2))
        c.launch("avgpool_global", self.P2, self.E2, n * 64, (h // 2) * (w // 2))
        c.launch("concat_dense", self.E1, self.E2, self.WD, self.BD, self.LOG, n, 64, self.classes)

    def launch_all(self):
        self._run("kernels", self._kernels)

    def step(self, read=True):
        self.launch_all()
        if read:
            self.ctx.read(self.LOG)
