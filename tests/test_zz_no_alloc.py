"""The allocation-free reduction entry point, for callers that cannot call
cudaMalloc (plug-ins whose host application owns device memory, budgeted
allocators, latency-critical loops).  It is called through the C ABI and must
give what the regular "vec_reduce_diff" launch gives, on two calls in a row
with different inputs (the shared static scratch keeps the previous call's
contents), and what the fp64 oracle gives within the reduction tolerance.
Kept in a file pytest collects last."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import datagen
from oracle import numeric as O
from paper_2012_09646_gb300 import gdag as G

pytestmark = pytest.mark.gpu
TOL = 1e-5
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def regular_launch(dx, dy, n):
    """The existing entry point: a context launch with caller scratch."""
    with G.Context() as ctx:
        z = torch.zeros(1, dtype=torch.float32, device="cuda")
        s = torch.zeros(G.gdag_scratch_bytes("vec_reduce_diff", n), dtype=torch.uint8, device="cuda")
        ctx.launch("vec_reduce_diff", ctx.array(dx), ctx.array(dy), ctx.array(z), ctx.array(s), n)
        ctx.sync()
        return float(z.item())


def check_against_oracle(x, y, got):
    want = float(O.sum_diff(x, y))
    scale = float(O.sum_abs_diff(x, y))
    assert abs(got - want) <= TOL * max(scale, 1.0), (len(x), got, want)


def test_noalloc_matches_regular_entry_twice():
    cases = [(1_000_003, 31), (4097, 32)]
    stream = torch.cuda.current_stream().cuda_stream
    for n, seed in cases:
        x, y = datagen.vec_inputs(n, seed=seed)
        dx = torch.from_numpy(x).cuda()
        dy = torch.from_numpy(y).cuda()
        want = regular_launch(dx, dy, n)
        scale = float(np.abs(x.astype(np.float64) - y).sum())
        z = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        G.gdag_vec_reduce_diff_noalloc(dx.data_ptr(), dy.data_ptr(), z.data_ptr(), n, stream)
        torch.cuda.synchronize()
        got = float(z.item())
        assert abs(got - want) <= TOL * max(scale, 1.0), (n, got, want)
        check_against_oracle(x, y, got)


def test_noalloc_allocates_nothing():
    """Once the inputs exist, repeated calls leave both torch's allocator and
    the device's free memory unchanged."""
    n = 2_000_000
    x, y = datagen.vec_inputs(n, seed=33)
    dx = torch.from_numpy(x).cuda()
    dy = torch.from_numpy(y).cuda()
    z = torch.zeros(1, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    G.gdag_vec_reduce_diff_noalloc(dx.data_ptr(), dy.data_ptr(), z.data_ptr(), n, s.cuda_stream)
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(50):
        G.gdag_vec_reduce_diff_noalloc(dx.data_ptr(), dy.data_ptr(), z.data_ptr(), n, s.cuda_stream)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == torch_before
    assert torch.cuda.mem_get_info()[0] == free_before
    check_against_oracle(x, y, float(z.item()))


# Run in a fresh process, so that this is the first call of the entry point on
# the device and it goes to a non-blocking stream (as torch side streams are).
_FIRST_CALL = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import datagen
from paper_2012_09646_gb300 import gdag as G
out = []
s = torch.cuda.Stream()  # cudaStreamNonBlocking
for n, seed in ((3_000_001, 41), (777, 42)):
    x, y = datagen.vec_inputs(n, seed=seed)
    with torch.cuda.stream(s):
        dx = torch.from_numpy(x).to("cuda", non_blocking=False)
        dy = torch.from_numpy(y).to("cuda", non_blocking=False)
        z = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    s.synchronize()
    G.gdag_vec_reduce_diff_noalloc(dx.data_ptr(), dy.data_ptr(), z.data_ptr(), n, s.cuda_stream)
    s.synchronize()
    out.append(repr(float(z.item())))
print(" ".join(out))
"""


def test_noalloc_first_call_on_a_non_blocking_stream():
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL, ROOT], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    got = [float(v) for v in r.stdout.split()[-2:]]
    for (n, seed), g in zip(((3_000_001, 41), (777, 42)), got):
        x, y = datagen.vec_inputs(n, seed=seed)
        check_against_oracle(x, y, g)


def test_noalloc_rejects_bad_requests_without_launching():
    z = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(G.GdagError) as e:
        G.gdag_vec_reduce_diff_noalloc(z.data_ptr(), z.data_ptr(), z.data_ptr(), -1, None)
    assert e.value.code == G.GDAG_ERR_INVALID
    with pytest.raises(G.GdagError) as e:
        G.gdag_vec_reduce_diff_noalloc(z.data_ptr(), z.data_ptr(), None, 1, None)
    assert e.value.code == G.GDAG_ERR_INVALID
