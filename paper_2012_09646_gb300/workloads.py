"""The benchmark programs of Section IV-B as plain launch sequences.

Each class owns its device arrays (torch tensors, the only use of PyTorch:
device memory) and pinned host views, registers them with a
:class:`~paper_2012_09646_gb300.gdag.Context`, and issues one DAG iteration
per ``step`` call exactly as a user program would: host writes, kernel
launches with per-argument access modes, host reads.  The dependency DAG,
streams, events and copies are entirely the library's.
"""
from __future__ import annotations

import torch

from . import gdag as G

F32 = torch.float32


def _pinned(shape, dtype):
    return torch.empty(shape, dtype=dtype, pin_memory=True)


def _scratch(ctx, kernel, n, device):
    nbytes = G.gdag_scratch_bytes(kernel, n)
    t = torch.zeros(nbytes, dtype=torch.uint8, device=device)
    return t, ctx.array(t, name=kernel + "_scratch")


class VecDag:
    """VEC: host writes x and y; K1 x := x*x; K2 y := y*y; K3 z = sum(x - y);
    host reads z."""

    def __init__(self, ctx, n, device="cuda"):
        self.ctx, self.n = ctx, n
        self.x = torch.zeros(max(n, 1), dtype=F32, device=device)
        self.y = torch.zeros(max(n, 1), dtype=F32, device=device)
        self.z = torch.zeros(1, dtype=F32, device=device)
        self.hx, self.hy, self.hz = _pinned(max(n, 1), F32), _pinned(max(n, 1), F32), _pinned(1, F32)
        self.X = ctx.array(self.x, host=self.hx, name="x")
        self.Y = ctx.array(self.y, host=self.hy, name="y")
        self.Z = ctx.array(self.z, host=self.hz, name="z")
        self._s, self.S = _scratch(ctx, "vec_reduce_diff", n, device)

    def load(self, x, y):
        """Put new inputs into the pinned host views (host-side, untimed)."""
        self.hx[: self.n].copy_(torch.as_tensor(x))
        self.hy[: self.n].copy_(torch.as_tensor(y))

    def step(self, read=True):
        c, n = self.ctx, self.n
        c.write(self.X, None, 0, 4 * n)
        c.write(self.Y, None, 0, 4 * n)
        c.launch("vec_square", self.X, n)
        c.launch("vec_square", self.Y, n)
        c.launch("vec_reduce_diff", self.X, self.Y, self.Z, self.S, n)
        if read:
            c.read(self.Z)
            return float(self.hz[0])
        return None


class BsDag:
    """B&S: `count` independent call-price nodes.  With ``host_inputs`` each
    step rewrites every price vector from the host (copy nodes overlapping
    the other chains' kernels) and reads every result back."""

    def __init__(self, ctx, n, count=10, K=60.0, r=0.1, sigma=0.2, T=1.0, device="cuda", host=True):
        self.ctx, self.n, self.count = ctx, n, count
        self.params = (float(K), float(r), float(sigma), float(T))
        self.S = [torch.zeros(max(n, 1), dtype=F32, device=device) for _ in range(count)]
        self.C = [torch.zeros(max(n, 1), dtype=F32, device=device) for _ in range(count)]
        self.hS = [_pinned(max(n, 1), F32) for _ in range(count)] if host else [None] * count
        self.hC = [_pinned(max(n, 1), F32) for _ in range(count)] if host else [None] * count
        self.SA = [ctx.array(t, host=h, name="S%d" % i) for i, (t, h) in enumerate(zip(self.S, self.hS))]
        self.CA = [ctx.array(t, host=h, name="C%d" % i) for i, (t, h) in enumerate(zip(self.C, self.hC))]

    def load_host(self, prices):
        for h, p in zip(self.hS, prices):
            h[: self.n].copy_(torch.as_tensor(p))

    def load_device(self, prices):
        for d, p in zip(self.S, prices):
            d[: self.n].copy_(torch.as_tensor(p).to(d.device))
        torch.cuda.synchronize()

    def launch_all(self):
        K, r, s, T = self.params
        for Sa, Ca in zip(self.SA, self.CA):
            self.ctx.launch("bs_call", Sa, Ca, self.n, K, r, s, T)

    def step_resident(self):
        """Kernels only (inputs already in HBM); no host access."""
        self.launch_all()

    def step_e2e(self):
        """Host write of every price vector, all kernels, host read of every
        result (the paper's streaming form of the benchmark)."""
        c, nb = self.ctx, 4 * self.n
        K, r, s, T = self.params
        for Sa, Ca in zip(self.SA, self.CA):
            c.write(Sa, None, 0, nb)
            c.launch("bs_call", Sa, Ca, self.n, K, r, s, T)
        for Ca in self.CA:
            c.read(Ca, None, 0, nb)
