"""Every built-in kernel's launch contract as include/gdag.h documents it:
argument modes, and the bytes each array must hold for given sizes.  On the
recording fake backend (validation runs before anything is queued), a launch
with every array exactly as large as documented is accepted, and one with any
single array a byte smaller is rejected with INVALID and leaves no element.
Scratch, partition and carry buffers are documented as "the size
gdag_scratch_bytes gives", which may hold slack (the SpMV carry buffer has 16
bytes), so for those half the size must be rejected.  CPU only."""
import pytest

from paper_2012_09646_gb300 import gdag as G

IN, OUT, INOUT = G.GDAG_MODE_IN, G.GDAG_MODE_OUT, G.GDAG_MODE_INOUT
S = G.gdag_scratch_bytes


def A(mode, nbytes, exact=True):
    return ("array", mode, nbytes, exact)


def SC(mode, kernel, n):
    """A buffer sized by gdag_scratch_bytes (an upper bound)."""
    return A(mode, S(kernel, n), exact=False)


def V(value):
    return ("scalar", value)


def contracts():
    """name -> argument list, at small sizes with ragged tails."""
    n = 1003
    rows, cols, R = 37, 53, 4
    mr, feats, classes = 129, 64, 10
    hn, hnnz = 100, 20017  # several merge-path tiles
    g, gn = 7, 1000
    bn, bh, bw = 2, 6, 16
    planes, hw = 12, 49
    cn, cc, ccl = 3, 64, 10
    return {
        "vec_square": [A(INOUT, 4 * n), V(n)],
        "vec_reduce_diff": [A(IN, 4 * n), A(IN, 4 * n), A(OUT, 4), SC(INOUT, "vec_reduce_diff", n), V(n)],
        "bs_call": [A(IN, 4 * n), A(OUT, 4 * n), V(n), V(60.0), V(0.1), V(0.2), V(1.0)],
        "gauss_blur": [A(IN, 4 * rows * cols), A(OUT, 4 * rows * cols), A(IN, 4 * (2 * R + 1)),
                       V(rows), V(cols), V(R)],
        "sobel": [A(IN, 4 * rows * cols), A(OUT, 4 * rows * cols), V(rows), V(cols)],
        "minmax": [A(IN, 4 * n), A(OUT, 8), SC(INOUT, "minmax", n), V(n)],
        "extend": [A(INOUT, 4 * n), A(IN, 8), V(n)],
        "unsharp": [A(IN, 4 * n), A(IN, 4 * n), A(OUT, 4 * n), V(0.5), V(n)],
        "combine": [A(IN, 4 * n)] * 5 + [A(OUT, 4 * n), V(n)],
        "dense_scores": [A(IN, 4 * mr * feats), A(IN, 4 * feats * classes), A(IN, 4 * classes),
                         A(OUT, 4 * mr * classes), V(mr), V(feats), V(classes)],
        "row_softmax": [A(INOUT, 4 * mr * classes), V(mr), V(classes)],
        "argmax_combine": [A(IN, 4 * mr * classes), A(IN, 4 * mr * classes), A(OUT, 4 * mr), V(mr), V(classes)],
        "spmv_partition": [A(IN, 4 * (hn + 1)), SC(OUT, "spmv_partition", hn + hnnz), V(hn), V(hnnz)],
        "spmv_csr": [A(IN, 4 * (hn + 1)), A(IN, 4 * hnnz), A(IN, 4 * hnnz), A(IN, 4 * hn),
                     SC(IN, "spmv_partition", hn + hnnz), A(OUT, 4 * hn), SC(INOUT, "spmv_csr", hn + hnnz),
                     V(hn), V(hnnz)],
        "l2norm": [A(IN, 4 * n), A(OUT, 4), SC(INOUT, "l2norm", n), V(n)],
        "scale": [A(INOUT, 4 * n), A(IN, 4), V(n)],
        "seg_l2norm": [A(IN, 4 * gn), A(IN, 4 * (g + 1)), A(OUT, 4 * g), SC(INOUT, "seg_l2norm", g), V(g), V(gn)],
        "seg_scale": [A(INOUT, 4 * gn), A(IN, 4 * (g + 1)), A(IN, 4 * g), V(g), V(gn)],
        "conv3x3_relu_pool": [A(IN, 2 * bn * 3 * bh * bw), A(IN, 2 * 64 * 27), A(IN, 4 * 64),
                              A(OUT, 2 * bn * 64 * (bh // 2) * (bw // 2)), A(INOUT, 4), V(bn), V(bh), V(bw)],
        "avgpool_global": [A(IN, 2 * planes * hw), A(OUT, 4 * planes), V(planes), V(hw)],
        "concat_dense": [A(IN, 4 * cn * cc), A(IN, 4 * cn * cc), A(IN, 4 * 2 * cc * ccl), A(IN, 4 * ccl),
                         A(OUT, 4 * cn * ccl), V(cn), V(cc), V(ccl)],
    }


# the built-in kernels, listed here so that collecting these tests loads no
# library (the table itself asks the library for scratch sizes)
NAMES = ["argmax_combine", "avgpool_global", "bs_call", "combine", "concat_dense", "conv3x3_relu_pool",
         "dense_scores", "extend", "gauss_blur", "l2norm", "minmax", "row_softmax", "scale", "seg_l2norm",
         "seg_scale", "sobel", "spmv_csr", "spmv_partition", "unsharp", "vec_reduce_diff", "vec_square"]


def issue(ctx, name, args, shrink=None):
    """Register each array at its documented size (for argument `shrink`,
    one byte less, or half for a gdag_scratch_bytes size) at a 256-byte
    aligned address, and launch."""
    vals = []
    for i, a in enumerate(args):
        if a[0] == "array":
            nb = a[2] if i != shrink else (a[2] - 1 if a[3] else a[2] // 2)
            vals.append(ctx.array(dev=0x10000000 * (i + 1), nbytes=nb))
        else:
            vals.append(a[1])
    return ctx.launch(name, *vals)


@pytest.mark.parametrize("name", NAMES)
def test_documented_modes(name):
    ctx = G.Context(backend="fake")
    _, spec = ctx.kernel(name)
    args = contracts()[name]
    assert len(spec) == len(args)
    for sp, a in zip(spec, args):
        if a[0] == "array":
            assert sp.kind == G.GDAG_ARG_ARRAY and sp.mode == a[1]
        else:
            assert sp.kind == G.GDAG_ARG_SCALAR
    ctx.close()


@pytest.mark.parametrize("name", NAMES)
def test_documented_sizes_are_exactly_enough(name):
    args = contracts()[name]
    ctx = G.Context(backend="fake", record_log=True)
    issue(ctx, name, args)
    assert len(ctx.nodes()) == 1
    ctx.close()
    for i, a in enumerate(args):
        if a[0] != "array" or a[2] == 0:
            continue
        ctx = G.Context(backend="fake", record_log=True)
        with pytest.raises(G.GdagError) as e:
            issue(ctx, name, args, shrink=i)
        assert e.value.code == G.GDAG_ERR_INVALID, (name, i)
        assert ctx.nodes() == [] and ctx.edges() == []
        ctx.close()


def test_every_builtin_kernel_has_a_contract():
    """The table above covers the whole built-in kernel table."""
    assert sorted(contracts()) == NAMES
    ctx = G.Context(backend="fake")
    for name in contracts():
        ctx.kernel(name)
    # a name outside the table is not built in
    with pytest.raises(G.GdagError) as e:
        ctx.kernel("vec_cube")
    assert e.value.code == G.GDAG_ERR_NOT_FOUND
    ctx.close()


BIG = 1 << 26  # every array large enough that only the rule under test can fail

# (kernel, scalars, accepted?, launch shape or None, {array index: address offset})
LIMITS = [
    ("gauss_blur", (37, 53, 8), True, None, {}),
    ("gauss_blur", (37, 53, 0), False, None, {}),
    ("gauss_blur", (37, 53, 9), False, None, {}),
    ("gauss_blur", (0, 53, 2), False, None, {}),
    ("sobel", (37, 0), False, None, {}),
    ("minmax", (1,), True, None, {}),
    ("minmax", (0,), False, None, {}),
    ("dense_scores", (1, 64, 16), True, None, {}),
    ("dense_scores", (1, 48, 10), False, None, {}),
    ("dense_scores", (1, 0, 10), False, None, {}),
    ("dense_scores", (1, 64, 0), False, None, {}),
    ("dense_scores", (1, 64, 17), False, None, {}),
    ("dense_scores", (1, 3168, 16), True, None, {}),   # 3168 * 4 <= 12796
    ("dense_scores", (1, 3200, 16), False, None, {}),  # 3200 * 4 > 12796
    ("dense_scores", (1, 4256, 12), True, None, {}),   # 4256 * 3 <= 12796
    ("dense_scores", (1, 4288, 12), False, None, {}),
    ("dense_scores", (1, 64, 10), False, None, {0: 4}),  # X not 16-byte aligned
    ("dense_scores", (-1, 64, 10), False, None, {}),
    ("row_softmax", (5, 32), True, None, {}),
    ("row_softmax", (5, 33), False, None, {}),
    ("row_softmax", (5, 0), False, None, {}),
    ("argmax_combine", (5, 0), False, None, {}),
    ("conv3x3_relu_pool", (1, 2, 8), True, None, {}),
    ("conv3x3_relu_pool", (0, 2, 8), False, None, {}),
    ("conv3x3_relu_pool", (1, 5, 8), False, None, {}),
    ("conv3x3_relu_pool", (1, 0, 8), False, None, {}),
    ("conv3x3_relu_pool", (1, 2, 12), False, None, {}),
    ("conv3x3_relu_pool", (1, 2, 8), False, None, {0: 8}),  # x not 16-byte aligned
    ("conv3x3_relu_pool", (1, 2, 8), False, None, {3: 8}),  # out not 16-byte aligned
    ("avgpool_global", (0, 4), False, None, {}),
    ("avgpool_global", (4, 0), False, None, {}),
    ("concat_dense", (0, 4, 2), False, None, {}),
    ("concat_dense", (1, 0, 2), False, None, {}),
    ("concat_dense", (1, 4, 0), False, None, {}),
    ("seg_l2norm", (65535, 100), True, None, {}),
    ("seg_l2norm", (65536, 100), False, None, {}),
    ("seg_l2norm", (4, 100), False, None, {0: 4}),  # x not 16-byte aligned
    ("seg_scale", (65536, 100), False, None, {}),
    ("seg_scale", (4, 100), False, None, {0: 4}),
    ("bs_call", (100, 60.0, 0.1, 0.2, 1.0), True, ((4, 1, 1), (256, 1, 1)), {}),
    ("bs_call", (100, 60.0, 0.1, 0.2, 1.0), False, ((4, 1, 1), (512, 1, 1)), {}),
    ("bs_call", (100, 0.0, 0.1, 0.2, 1.0), False, None, {}),
    ("bs_call", (100, 60.0, 0.1, 0.0, 1.0), False, None, {}),
    ("bs_call", (100, 60.0, 0.1, 0.2, 0.0), False, None, {}),
    ("bs_call", (100, float("nan"), 0.1, 0.2, 1.0), False, None, {}),
    ("vec_reduce_diff", (100,), True, ((1024, 1, 1), (256, 1, 1)), {}),
    ("vec_reduce_diff", (100,), False, ((1025, 1, 1), (256, 1, 1)), {}),
    ("vec_reduce_diff", (100,), False, ((8, 1, 1), (128, 1, 1)), {}),
    ("spmv_partition", (-1, 10), False, None, {}),
    ("spmv_csr", (10, -1), False, None, {}),
] + [(k, s, False, None, {}) for k, s in [
    ("vec_square", (-1,)), ("vec_reduce_diff", (-1,)), ("bs_call", (-1, 60.0, 0.1, 0.2, 1.0)),
    ("extend", (-1,)), ("unsharp", (0.5, -1)), ("combine", (-1,)), ("l2norm", (-1,)), ("scale", (-1,)),
    ("row_softmax", (-1, 10)), ("argmax_combine", (-1, 10))]]


@pytest.mark.parametrize("case", LIMITS, ids=lambda c: "%s%s%s" % (c[0], c[1], "-ok" if c[2] else ""))
def test_documented_limits(case):
    name, scalars, ok, shape, shift = case
    ctx = G.Context(backend="fake", record_log=True)
    _, spec = ctx.kernel(name)
    vals, it = [], iter(scalars)
    for i, sp in enumerate(spec):
        if sp.kind == G.GDAG_ARG_ARRAY:
            vals.append(ctx.array(dev=0x100000000 * (i + 1) + shift.get(i, 0), nbytes=BIG))
        else:
            vals.append(next(it))
    grid, block = shape if shape else (None, None)
    if ok:
        ctx.launch(name, *vals, grid=grid, block=block)
        assert len(ctx.nodes()) == 1
    else:
        with pytest.raises(G.GdagError) as e:
            ctx.launch(name, *vals, grid=grid, block=block)
        assert e.value.code == G.GDAG_ERR_INVALID
        assert ctx.nodes() == []
    ctx.close()
