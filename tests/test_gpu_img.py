"""IMG nodes and the IMG DAG on the GPU through the C ABI, against the
oracle: node by node (each node fed the GPU's own upstream output, so that
only that node's error is measured) and end to end.  Tolerance: |got - ref|
<= 1e-5 * max(|ref|, 1); min/max bit-exact."""
import numpy as np
import pytest
import torch

import datagen
from oracle import numeric as N
from oracle import pipelines as P
from paper_2012_09646_gb300 import gdag as G
from paper_2012_09646_gb300.workloads import ImgDag

pytestmark = pytest.mark.gpu
TOL = 1e-5


def check(got, ref, scale=1.0, what=""):
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    if np.ndim(scale):
        scale = np.asarray(scale, np.float64).ravel()
    err = np.abs(got - ref) / np.maximum(np.abs(ref), scale)
    assert err.max() <= TOL, (what, err.max(), int(err.argmax()))


def host(t, shape):
    return t.cpu().numpy().reshape(shape).astype(np.float64)


# (1500, 4100) and (1300, 3001): more tiles than the persistent stencil grid
# holds, so each block walks several tiles (interior tiles double-buffered by
# cp.async, border and unaligned-row tiles staged with clamping); 4096 x 4096
# is the benchmark's size and launch shape, compared pixel by pixel
@pytest.mark.parametrize("shape", [(1, 1), (7, 13), (33, 65), (100, 257), (512, 512), (1500, 4100), (1300, 3001),
                                   (4096, 4096)])
def test_img_nodes_stepwise(shape):
    rows, cols = shape
    img = datagen.image(rows, cols, seed=rows * 1000 + cols)
    with G.Context() as ctx:
        d = ImgDag(ctx, rows, cols)
        d.load(img)
        d.step()
        ctx.sync()
        b5, b9 = host(d.b5, shape), host(d.b9, shape)
        check(b5, N.blur(img, N.gauss_weights(2, 1.0)), what="blur5")
        check(b9, N.blur(img, N.gauss_weights(4, 2.0)), what="blur9")
        e5, e9 = host(d.e5, shape), host(d.e9, shape)
        mm5, mm9 = d.mm5.cpu().numpy(), d.mm9.cpu().numpy()
        # extend ran in place: recompute the raw Sobel output of the GPU's
        # own blurs on the GPU (so that min/max and extend can be checked
        # exactly on the GPU's values)
        d2 = ImgDag(ctx, rows, cols)
        for b, E, MM, SC, e_t, mm_t, mm_dag, e_dag, tag in (
                (b5, d2.E5, d2.MM5, d2.SC5, d2.e5, d2.mm5, mm5, e5, "5"),
                (b9, d2.E9, d2.MM9, d2.SC9, d2.e9, d2.mm9, mm9, e9, "9")):
            d2.img.copy_(torch.from_numpy(b.astype(np.float32).ravel()))
            ctx.launch("sobel", d2.IMG, E, rows, cols)
            ctx.launch("minmax", E, MM, SC, rows * cols)
            ctx.sync()
            g_raw = host(e_t, shape)
            # the magnitude sqrt(gx^2 + gy^2) of sums of terms of both signs:
            # the scale of the relative bound is each pixel's sum of |terms|
            check(g_raw, N.sobel(b), scale=N.sobel_scale(b), what="sobel" + tag)
            assert tuple(mm_t.cpu().numpy()) == (np.float32(g_raw.min()), np.float32(g_raw.max())), tag
            assert tuple(mm_dag) == tuple(mm_t.cpu().numpy()), tag
            # extend of the GPU's raw edges with the GPU's min/max
            check(e_dag, N.extend(g_raw, *mm_dag.astype(np.float64)), what="extend" + tag)
        s = host(d.s, shape)
        check(s, N.unsharp(img, b5, 0.5), what="unsharp")
        out = host(d.out, shape)
        check(out, N.combine(s, b5, b9, e5, e9), what="combine")
        check(d.h_out.numpy().reshape(shape), out, what="host read")


# one float; a ragged tail; one chunk and a bit; 2^25 + 7 floats (4097 chunks
# of 8192 floats, more than the 4096 blocks, so a block takes two); 4e7
# floats; a start 12 bytes past a 16-byte boundary (the scalar path)
@pytest.mark.parametrize("n,off", [(1, 0), (3, 0), (8193, 0), ((1 << 25) + 7, 0), (40_000_003, 0), (1_000_001, 3)])
def test_minmax_sizes_and_alignment(n, off):
    """minmax alone, bit-exact against the oracle's min and max, with the
    extremes placed in the ragged tail and in a middle chunk."""
    rng = np.random.default_rng(n + off)
    x = (rng.standard_normal(n + off) * 100.0).astype(np.float32)
    x[off + n // 2] = 3.0e30
    x[off + n - 1] = -3.0e30
    mn, mx = N.minmax(x[off:].astype(np.float64))
    with G.Context() as ctx:
        buf = torch.from_numpy(x).cuda()
        mm = torch.full((2,), 7.0, device="cuda")
        sc = torch.zeros(G.gdag_scratch_bytes("minmax", n), dtype=torch.uint8, device="cuda")
        X = ctx.array(dev=buf.data_ptr() + 4 * off, nbytes=4 * n)
        ctx.launch("minmax", X, ctx.array(mm), ctx.array(sc), n)
        ctx.sync()
        got = mm.cpu().numpy()
    assert (got[0], got[1]) == (np.float32(mn), np.float32(mx)), (got, mn, mx)


@pytest.mark.parametrize("shape,policy", [(sh, p) for sh in ((64, 64), (129, 300), (1024, 1024))
                                          for p in (G.GDAG_POLICY_PARALLEL, G.GDAG_POLICY_SERIAL_SYNC)]
                         + [((4096, 4096), G.GDAG_POLICY_PARALLEL)])
def test_img_dag_end_to_end(shape, policy):
    rows, cols = shape
    img = datagen.image(rows, cols, seed=2)
    ref = P.img(img)
    with G.Context(policy=policy) as ctx:
        d = ImgDag(ctx, rows, cols)
        d.load(img)
        d.step()
        got = d.h_out.numpy().reshape(shape)
        err = np.abs(got - ref["out"]) / np.maximum(np.abs(ref["out"]), 1.0)
        assert err.max() <= TOL, err.max()
        ctx.sync()


def test_img_constant_and_ramp_images():
    rows, cols = 40, 70
    with G.Context() as ctx:
        d = ImgDag(ctx, rows, cols)
        d.load(np.full((rows, cols), 0.75, np.float32))
        d.step()
        ctx.sync()
        assert np.all(d.e5.cpu().numpy() == 0)  # flat edges -> extend maps to 0
        np.testing.assert_allclose(d.b5.cpu().numpy(), 0.75, rtol=1e-6)
        ramp = np.tile(np.arange(cols, dtype=np.float32) * 0.25, (rows, 1))
        d.load(ramp)
        d.step()
        ctx.sync()
        # interior of the Sobel of a blurred ramp: the blur keeps the slope
        # away from the edges, so the raw magnitude there is 8 * 0.25
        ctx.launch("sobel", d.IMG, d.E9, rows, cols)
        ctx.sync()
        e = d.e9.cpu().numpy().reshape(rows, cols)
        np.testing.assert_allclose(e[1:-1, 1:-1], 2.0, rtol=1e-6)
