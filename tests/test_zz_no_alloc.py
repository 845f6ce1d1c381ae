"""The allocation-free reduction entry point, for callers that cannot call
cudaMalloc (plug-ins whose host application owns device memory, budgeted
allocators, latency-critical loops).  It is called through the C ABI and must
give what the regular "vec_reduce_diff" launch gives, on two calls in a row
with different inputs (the shared static scratch keeps the previous call's
contents).  Kept in a file pytest collects last."""
import numpy as np
import pytest
import torch

import datagen
from paper_2012_09646_gb300 import gdag as G

pytestmark = pytest.mark.gpu
TOL = 1e-5


def regular_launch(dx, dy, n):
    """The existing entry point: a context launch with caller scratch."""
    with G.Context() as ctx:
        z = torch.zeros(1, dtype=torch.float32, device="cuda")
        s = torch.zeros(G.gdag_scratch_bytes("vec_reduce_diff", n), dtype=torch.uint8, device="cuda")
        ctx.launch("vec_reduce_diff", ctx.array(dx), ctx.array(dy), ctx.array(z), ctx.array(s), n)
        ctx.sync()
        return float(z.item())


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


def test_noalloc_rejects_bad_requests_without_launching():
    z = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(G.GdagError) as e:
        G.gdag_vec_reduce_diff_noalloc(z.data_ptr(), z.data_ptr(), z.data_ptr(), -1, None)
    assert e.value.code == G.GDAG_ERR_INVALID
    with pytest.raises(G.GdagError) as e:
        G.gdag_vec_reduce_diff_noalloc(z.data_ptr(), z.data_ptr(), None, 1, None)
    assert e.value.code == G.GDAG_ERR_INVALID
