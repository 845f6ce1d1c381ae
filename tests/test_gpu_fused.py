"""Fused launches on the GPU through the C ABI: each member of a
gdag_launch_fused element gives exactly (bit for bit) what its own
gdag_launch gives, for members of mixed sizes (empty, a ragged scalar tail,
one element, several chunks, a reduction with its full 912-block partition),
unaligned members, and more members than one kernel table holds; prices and
sums also meet the oracle's tolerance (1e-5 relative; for the sums, relative
to the sum of |terms|)."""
import numpy as np
import pytest
import torch

import datagen
from oracle import pipelines as P
from paper_2012_09646_gb300 import gdag as G

pytestmark = pytest.mark.gpu
TOL = 1e-5
SIZES = [0, 1, 3, 4, 1023, 4096, 4097, 65_539, 1_000_003, 5_000_000]


def _bs_args(S, C, n):
    return (S, C, n, 60.0, 0.1, 0.2, 1.0)


def test_fused_bs_call_equals_plain_launches_and_oracle():
    with G.Context() as ctx:
        members, plain, keep = [], [], []
        for i, n in enumerate(SIZES):
            p = torch.from_numpy(datagen.bs_inputs(max(n, 1), count=1, seed=40 + i)[0]).cuda()
            Cf = torch.full((max(n, 1),), -1.0, device="cuda")
            Cp = torch.full((max(n, 1),), -2.0, device="cuda")
            S_a, Cf_a, Cp_a = ctx.array(p), ctx.array(Cf), ctx.array(Cp)
            members.append(_bs_args(S_a, Cf_a, n))
            plain.append(_bs_args(S_a, Cp_a, n))
            keep.append((n, p, Cf, Cp))
        ctx.launch_fused("bs_call", members)
        for args in plain:
            ctx.launch("bs_call", *args)
        ctx.sync()
        for n, p, Cf, Cp in keep:
            if n == 0:
                assert Cf[0].item() == -1.0  # nothing written
                continue
            got = Cf[:n].cpu().numpy()
            assert np.array_equal(got, Cp[:n].cpu().numpy())
            idx = np.unique(np.linspace(0, n - 1, min(n, 2000)).astype(np.int64))
            want = P.bs([p[:n].cpu().numpy()[idx]])["C0"]
            err = np.abs(got[idx] - want) / np.maximum(np.abs(want), 1.0)
            assert err.max() <= TOL


def test_fused_bs_unaligned_member_and_mixed_parameters():
    n = 10_001
    with G.Context() as ctx:
        base = torch.zeros(n + 1, device="cuda")
        p = torch.from_numpy(datagen.bs_inputs(n, count=1, seed=5)[0]).cuda()
        base[1:].copy_(p)
        S_u = ctx.array(dev=base.data_ptr() + 4, nbytes=4 * n)  # 4-byte aligned only
        S_a = ctx.array(p)
        outs = [torch.empty(n, device="cuda") for _ in range(4)]
        O = [ctx.array(o) for o in outs]
        params = [(60.0, 0.1, 0.2, 1.0), (75.0, 0.03, 0.35, 0.5)]
        ctx.launch_fused("bs_call", [(S_u, O[0], n) + params[0], (S_a, O[1], n) + params[1]])
        ctx.launch("bs_call", S_a, O[2], n, *params[0])
        ctx.launch("bs_call", S_a, O[3], n, *params[1])
        ctx.sync()
        assert torch.equal(outs[0], outs[2])
        assert torch.equal(outs[1], outs[3])


def test_fused_vec_square_exact():
    with G.Context() as ctx:
        xs, arrays, keep = [], [], []
        for i, n in enumerate(SIZES):
            x = datagen.vec_inputs(max(n, 1), seed=60 + i)[0][:n]
            t = torch.from_numpy(x.copy()).cuda() if n else torch.zeros(1, device="cuda")
            arrays.append((ctx.array(t), n))
            keep.append((x, t, n))
        # an unaligned member too
        base = torch.zeros(5001, device="cuda")
        xu = datagen.vec_inputs(5000, seed=7)[0]
        base[1:].copy_(torch.from_numpy(xu))
        arrays.append((ctx.array(dev=base.data_ptr() + 4, nbytes=20000), 5000))
        ctx.launch_fused("vec_square", arrays)
        ctx.sync()
        for x, t, n in keep:
            assert np.array_equal(t[:n].cpu().numpy(), x * x)
            if n == 0:
                assert t[0].item() == 0.0
        assert np.array_equal(base[1:].cpu().numpy(), xu * xu)


def test_fused_vec_reduce_diff_bit_identical_to_plain():
    sb = G.gdag_scratch_bytes("vec_reduce_diff", 1)
    with G.Context() as ctx:
        members, plain, keep = [], [], []
        for i, n in enumerate(SIZES):
            x, y = datagen.vec_inputs(max(n, 1), seed=80 + i)
            x, y = x[:n], y[:n]
            tx = torch.from_numpy(x.copy()).cuda() if n else torch.zeros(1, device="cuda")
            ty = torch.from_numpy(y.copy()).cuda() if n else torch.zeros(1, device="cuda")
            zf = torch.full((1,), -7.0, device="cuda")
            zp = torch.full((1,), -9.0, device="cuda")
            sf = torch.zeros(sb, dtype=torch.uint8, device="cuda")
            sp = torch.zeros(sb, dtype=torch.uint8, device="cuda")
            X, Y = ctx.array(tx), ctx.array(ty)
            members.append((X, Y, ctx.array(zf), ctx.array(sf), n))
            plain.append((X, Y, ctx.array(zp), ctx.array(sp), n))
            keep.append((x, y, zf, zp, sf, n))
        for rep in range(2):  # the arrival counters come back to zero
            ctx.launch_fused("vec_reduce_diff", members)
            for args in plain:
                ctx.launch("vec_reduce_diff", *args)
            ctx.sync()
            for x, y, zf, zp, sf, n in keep:
                assert zf.item() == zp.item()
                d = x.astype(np.float64) - y.astype(np.float64)
                assert abs(zf.item() - d.sum()) <= TOL * max(np.abs(d).sum(), 1.0)
                assert int(sf[-16:].view(torch.int32)[0].item()) == 0


def test_fused_more_members_than_one_table():
    """300 small members (one element, three persistent launches)."""
    n_members = 2 * G.GDAG_FUSED_TABLE + 44
    with G.Context() as ctx:
        rng = np.random.default_rng(3)
        sizes = rng.integers(0, 3000, size=n_members)
        data = [rng.random(int(n), dtype=np.float32) for n in sizes]
        ts = [torch.from_numpy(d).cuda() if d.size else torch.zeros(1, device="cuda") for d in data]
        before = ctx.stats()["launches"]
        node = ctx.launch_fused("vec_square", [(ctx.array(t), int(n)) for t, n in zip(ts, sizes)])
        ctx.sync()
        assert ctx.stats()["launches"] == before + 1 and ctx.stats()["fused_members"] == n_members
        assert node == ctx.stats()["nodes"] - 1
        for d, t in zip(data, ts):
            assert np.array_equal(t[: d.size].cpu().numpy(), d * d)
