"""Batched issue (gdag_issue through gdag.Program) and the batched completion
query (gdag_nodes_query) on the recording backend (CPU only).  A program
issued in batches must give exactly what the same elements issued one call
at a time give: the same edge log, element log and backend operation log,
so the DAG, the streams and the waits are the single calls'."""
import random

import pytest

from oracle import dag as D
from paper_2012_09646_gb300 import gdag as G

MODE_OF = {D.R: G.GDAG_MODE_IN, D.W: G.GDAG_MODE_OUT, D.RW: G.GDAG_MODE_INOUT}
ARR = G.gdag_argspec(G.GDAG_ARG_ARRAY, G.GDAG_MODE_DEFAULT, 0, 0)
I64 = G.gdag_argspec(G.GDAG_ARG_SCALAR, 0, 8, 0)


def make_ctx(n_arrays, **opts):
    opts.setdefault("record_log", True)
    ctx = G.Context(backend="fake", **opts)
    arrays = [ctx.array(dev=0x10000 * (i + 1), nbytes=64, name="a%d" % i) for i in range(n_arrays)]
    kern = {n: "k%d" % n for n in range(1, 6)}
    for n, name in kern.items():
        kid = G.gdag_kernel_register(ctx.h, name, None, [ARR] * n + [I64])
        ctx._kernels[name] = (kid, G.gdag_kernel_signature(ctx.h, kid))
    return ctx, arrays, kern


def random_elements(rng, L, n_arrays):
    """Non-blocking elements (launches, writes, prefetches), with host reads
    (blocking, issued as single calls) in between."""
    out = []
    for _ in range(L):
        r = rng.random()
        if r < 0.15:
            out.append(("write", rng.randrange(n_arrays)))
        elif r < 0.25:
            out.append(("prefetch", rng.randrange(n_arrays)))
        elif r < 0.32:
            out.append(("read", rng.randrange(n_arrays)))
        else:
            k = rng.randint(1, min(5, n_arrays))
            arrs = rng.sample(range(n_arrays), k)
            out.append(("kernel", [(a, rng.choice([D.R, D.R, D.W, D.RW])) for a in arrs], rng.randrange(100)))
    return out


def kernel_args(arrays, acc):
    return [G.Mode(arrays[a], MODE_OF[m]) for a, m in acc]


def issue_singly(ctx, arrays, kern, elems):
    for e in elems:
        if e[0] == "write":
            ctx.write(arrays[e[1]], None)
        elif e[0] == "prefetch":
            ctx.prefetch_host(arrays[e[1]])
        elif e[0] == "read":
            ctx.read(arrays[e[1]])
        else:
            ctx.launch(kern[len(e[1])], *kernel_args(arrays, e[1]), e[2], grid=(1, 1, 1), block=(32, 1, 1))


def issue_batched(ctx, arrays, kern, elems, rng):
    prog = None
    n_param = 0
    values = {}

    def flush():
        nonlocal prog, values
        if prog is not None and len(prog):
            prog.issue(**values)
        prog, values = ctx.program(), {}

    flush()
    for e in elems:
        if e[0] == "read":
            flush()
            ctx.read(arrays[e[1]])
        elif e[0] == "write":
            prog.write(arrays[e[1]])
        elif e[0] == "prefetch":
            prog.prefetch_host(arrays[e[1]])
        else:
            # some scalars bound at issue time, the rest recorded
            if rng.random() < 0.5:
                name = "p%d" % n_param
                n_param += 1
                values[name] = e[2]
                scal = G.Param(name)
            else:
                scal = e[2]
            prog.launch(kern[len(e[1])], *kernel_args(arrays, e[1]), scal, grid=(1, 1, 1), block=(32, 1, 1))
        if rng.random() < 0.1:
            flush()
    flush()


@pytest.mark.parametrize("seed", range(40))
def test_batched_issue_equals_single_calls(seed):
    rng = random.Random(seed)
    opts = rng.choice([{}, {"max_streams": 2}, {"retire_by_query": True, "fake_complete": True},
                       {"policy": G.GDAG_POLICY_SERIAL_ASYNC}, {"policy": G.GDAG_POLICY_SERIAL_SYNC},
                       {"prefetch": False}])
    n_arrays = rng.randint(1, 6)
    elems = random_elements(rng, rng.randint(1, 60), n_arrays)
    a_ctx, a_arr, kern = make_ctx(n_arrays, **opts)
    issue_singly(a_ctx, a_arr, kern, elems)
    b_ctx, b_arr, _ = make_ctx(n_arrays, **opts)
    issue_batched(b_ctx, b_arr, kern, elems, random.Random(seed + 1000))
    assert a_ctx.edges() == b_ctx.edges()
    assert a_ctx.nodes() == b_ctx.nodes()
    assert a_ctx.ops() == b_ctx.ops()
    a_ctx.close()
    b_ctx.close()


def test_issue_returns_each_elements_node():
    ctx, arrays, kern = make_ctx(3)
    p = ctx.program()
    p.write(arrays[0])
    p.launch(kern[2], G.Mode(arrays[0], G.GDAG_MODE_IN), G.Mode(arrays[1], G.GDAG_MODE_OUT), 5,
             grid=(1, 1, 1), block=(32, 1, 1))
    p.prefetch_host(arrays[1])
    p.prefetch_host(arrays[2])  # never written from the host: its view is not current, so a copy node
    nodes = p.issue()
    assert nodes[:3] == [0, 1, 2]
    # a second issue of the same recording continues the numbering
    ctx.read(arrays[1])
    nodes2 = p.issue()
    assert min(n for n in nodes2 if n >= 0) > max(nodes)
    ctx.close()


def test_prefetch_of_a_current_view_makes_no_node():
    ctx, arrays, _ = make_ctx(1)
    ctx.write(arrays[0], None)  # a full host write: the view holds the data
    p = ctx.program()
    p.prefetch_host(arrays[0])
    assert p.issue() == [-1]
    ctx.close()


def test_params_are_bound_per_issue_and_checked():
    """A size bound at issue time is validated like a single call's: the
    built-in vec_square rejects n beyond its array."""
    ctx = G.Context(backend="fake")
    x = ctx.array(dev=0x10000, nbytes=4 * 100)
    p = ctx.program()
    p.write(x, 0, G.Param("nbytes"))
    p.launch("vec_square", x, G.Param("n"))
    assert p.params() == ["n", "nbytes"]
    nodes = p.issue(n=100, nbytes=400)
    assert nodes == [0, 1]
    with pytest.raises(G.GdagError) as e:
        p.issue(n=101, nbytes=400)
    assert e.value.code == G.GDAG_ERR_INVALID and e.value.issued == 1
    assert e.value.nodes[0] >= 0 and e.value.nodes[1] == -1
    with pytest.raises(G.GdagError) as e:
        p.issue(n=10, nbytes=404)  # a write past the array
    assert e.value.code == G.GDAG_ERR_INVALID and e.value.issued == 0
    with pytest.raises(G.GdagError) as e:
        p.issue(n=10)  # a parameter left unbound
    assert e.value.code == G.GDAG_ERR_INVALID
    ctx.close()


def test_failure_stops_the_batch_at_the_failing_element():
    """An injected backend failure in element i: the elements before it stay
    issued, element i has its node (retired, as a failed single call's), and
    the ones after it are not issued."""
    # every backend operation of the three elements in turn (copy, launches
    # and their event records)
    for fail in range(0, 6):
        ctx, arrays, kern = make_ctx(2, fake_fail_op=fail)
        p = ctx.program()
        p.write(arrays[0])
        p.launch(kern[2], G.Mode(arrays[0], G.GDAG_MODE_IN), G.Mode(arrays[1], G.GDAG_MODE_OUT), 1,
                 grid=(1, 1, 1), block=(32, 1, 1))
        p.launch(kern[1], G.Mode(arrays[1], G.GDAG_MODE_INOUT), 2, grid=(1, 1, 1), block=(32, 1, 1))
        try:
            nodes = p.issue()
            issued, err = 3, None
        except G.GdagError as e:
            nodes, issued, err = e.nodes, e.issued, e
        if err is None:
            assert nodes == [0, 1, 2], fail
        else:
            assert err.code == G.GDAG_ERR_CUDA
            assert nodes[:issued + 1] == list(range(issued + 1))
            assert all(n == -1 for n in nodes[issued + 1:])
            # the context goes on: later elements are ordered after the failed one's parents
            ctx.sync()
        ctx.close()


def test_bad_element_type_and_argument_range():
    ctx, arrays, kern = make_ctx(1)
    elems = (G.gdag_elem * 1)()
    elems[0].type = 9
    args = (G.gdag_arg * 1)()
    with pytest.raises(G.GdagError) as e:
        G.gdag_issue(ctx.h, elems, args)
    assert e.value.code == G.GDAG_ERR_INVALID and e.value.issued == 0
    elems[0].type = G.GDAG_ELEM_LAUNCH
    elems[0].kernel = ctx.kernel(kern[1])[0]
    elems[0].nargs = 2
    elems[0].arg0 = 0  # two arguments, one given
    elems[0].grid = G.gdag_dim3(1, 1, 1)
    elems[0].block = G.gdag_dim3(32, 1, 1)
    with pytest.raises(G.GdagError) as e:
        G.gdag_issue(ctx.h, elems, args)
    assert e.value.code == G.GDAG_ERR_INVALID
    assert ctx.stats()["nodes"] == 0
    ctx.close()


def test_nodes_query_matches_node_query():
    ctx, arrays, kern = make_ctx(2, fake_complete=False)
    p = ctx.program()
    p.launch(kern[1], G.Mode(arrays[0], G.GDAG_MODE_INOUT), 1, grid=(1, 1, 1), block=(32, 1, 1))
    p.launch(kern[1], G.Mode(arrays[1], G.GDAG_MODE_INOUT), 1, grid=(1, 1, 1), block=(32, 1, 1))
    nodes = p.issue()
    assert list(ctx.done_many(nodes)) == [0, 0] == [int(ctx.done(n)) for n in nodes]
    ctx.read(arrays[0])  # a host wait completes node 0 (and retires it)
    assert list(ctx.done_many(nodes)) == [1, 0]
    with pytest.raises(G.GdagError):
        ctx.done_many([0, 99])
    ctx.close()
