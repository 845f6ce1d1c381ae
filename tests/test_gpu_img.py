"""IMG nodes and the IMG DAG on the GPU through the C ABI, against the
oracle: node by node (each node fed the GPU's own upstream output, so that
only that node's error is measured) and end to end.  Tolerance: |got - ref|
<= 1e-5 * max(|ref|, 1); min/max bit-exact."""
import numpy as np
import pytest

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
    err = np.abs(got - ref) / np.maximum(np.abs(ref), scale)
    assert err.max() <= TOL, (what, err.max(), int(err.argmax()))


def host(t, shape):
    return t.cpu().numpy().reshape(shape).astype(np.float64)


# (1500, 4100) and (1300, 3001): more tiles than the persistent stencil grid
# holds, so each block walks several tiles (interior tiles double-buffered by
# cp.async, border and unaligned-row tiles staged with clamping)
@pytest.mark.parametrize("shape", [(1, 1), (7, 13), (33, 65), (100, 257), (512, 512), (1500, 4100), (1300, 3001)])
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
        # sobel of the GPU's blur; the magnitude is a sqrt of a sum of squares
        # of differences: scale = the gradient terms' size (|b| * 8)
        e5, e9 = host(d.e5, shape), host(d.e9, shape)
        mm5, mm9 = d.mm5.cpu().numpy(), d.mm9.cpu().numpy()
        # extend ran in place: recover the raw Sobel output from a fresh run
        raw5 = N.sobel(b5)
        raw9 = N.sobel(b9)
        # min/max of the GPU's own raw edges are exact: recompute raw on GPU
        d2 = ImgDag(ctx, rows, cols)
        d2.img.copy_(d.b5)
        ctx.launch("sobel", d2.IMG, d2.E5, rows, cols)
        ctx.launch("minmax", d2.E5, d2.MM5, d2.SC5, rows * cols)
        ctx.sync()
        g_raw5 = host(d2.e5, shape)
        check(g_raw5, raw5, scale=8 * max(np.abs(b5).max(), 1e-30), what="sobel5")
        assert tuple(d2.mm5.cpu().numpy()) == (np.float32(g_raw5.min()), np.float32(g_raw5.max()))
        assert tuple(mm5) == tuple(d2.mm5.cpu().numpy())
        # extend of the GPU's raw edges with the GPU's min/max
        check(e5, N.extend(g_raw5, *mm5.astype(np.float64)), what="extend5")
        s = host(d.s, shape)
        check(s, N.unsharp(img, b5, 0.5), what="unsharp")
        out = host(d.out, shape)
        check(out, N.combine(s, b5, b9, e5, e9), what="combine")
        check(d.h_out.numpy().reshape(shape), out, what="host read")


@pytest.mark.parametrize("shape", [(64, 64), (129, 300), (1024, 1024)])
@pytest.mark.parametrize("policy", [G.GDAG_POLICY_PARALLEL, G.GDAG_POLICY_SERIAL_SYNC])
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


@pytest.mark.slow
def test_img_full_size_sampled():
    """4096 x 4096, the benchmark's launch shape; sampled pixels of every
    node against the oracle evaluated at those pixels only."""
    rows = cols = 4096
    img = datagen.image(rows, cols, seed=2)
    rng = np.random.default_rng(1)
    ys = np.concatenate([rng.integers(0, rows, 2000), [0, rows - 1, 0, rows - 1]])
    xs = np.concatenate([rng.integers(0, cols, 2000), [0, 0, cols - 1, cols - 1]])
    with G.Context() as ctx:
        d = ImgDag(ctx, rows, cols)
        d.load(img)
        d.step()
        ctx.sync()
        b5 = host(d.b5, (rows, cols))
        b9 = host(d.b9, (rows, cols))
        w5, w9 = N.gauss_weights(2, 1.0), N.gauss_weights(4, 2.0)
        for y, x in zip(ys, xs):
            for b, w, R in ((b5, w5, 2), (b9, w9, 4)):
                ys_ = np.clip(np.arange(y - R, y + R + 1), 0, rows - 1)
                xs_ = np.clip(np.arange(x - R, x + R + 1), 0, cols - 1)
                want = float(np.outer(w, w).ravel() @ img[np.ix_(ys_, xs_)].astype(np.float64).ravel())
                assert abs(b[y, x] - want) <= TOL * max(abs(want), 1.0)
        # whole-image exact properties at full size
        mm5 = d.mm5.cpu().numpy()
        e5 = d.e5.cpu().numpy()
        assert e5.min() == 0.0 and e5.max() == 1.0 and mm5[1] > mm5[0]
        s = host(d.s, (rows, cols))
        i = ys * cols + xs
        np.testing.assert_allclose(s.ravel()[i], N.unsharp(img.ravel()[i], b5.ravel()[i], 0.5), rtol=1e-6, atol=1e-6)
