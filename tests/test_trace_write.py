"""gdag_trace_write: the library writes a traced context's node timings as a
Chrome trace file (CPU only, on the recording backend, whose timings are
zero): one event per node, kernels named after their kernel, copies after
their kind, one track per pool stream."""
import json

from paper_2012_09646_gb300 import gdag as G

ARR = G.gdag_argspec(G.GDAG_ARG_ARRAY, G.GDAG_MODE_INOUT, 0, 0)


def test_trace_file_lists_every_node(tmp_path):
    with G.Context(backend="fake", trace=True, fake_complete=True) as ctx:
        k = G.gdag_kernel_register(ctx.h, 'my "kernel"', None, [ARR])
        ctx._kernels["mine"] = (k, G.gdag_kernel_signature(ctx.h, k))
        a, b = ctx.array(dev=0x1000, nbytes=64), ctx.array(dev=0x2000, nbytes=64)
        ctx.write(a, None)
        ctx.launch("mine", a, grid=(1, 1, 1), block=(32, 1, 1))
        ctx.launch("mine", b, grid=(1, 1, 1), block=(32, 1, 1))
        ctx.prefetch_host(a)
        ctx.read(a)
        path = tmp_path / "trace.json"
        ctx.trace_write(str(path))
        want = ctx.trace()
    doc = json.loads(path.read_text())
    ev = doc["traceEvents"]
    assert [e["args"]["node"] for e in ev] == [t[0] for t in want]
    names = [e["name"] for e in ev]
    assert names[:4] == ["h2d", 'my "kernel"', 'my "kernel"', "d2h"]
    assert all(e["ph"] == "X" and e["dur"] >= 0 for e in ev)
    assert {e["tid"] for e in ev if e["cat"] == "kernel"} <= {"stream %d" % s for s in range(16)}


def test_trace_write_needs_tracing(tmp_path):
    import pytest
    with G.Context(backend="fake") as ctx:
        with pytest.raises(G.GdagError) as e:
            ctx.trace_write(str(tmp_path / "t.json"))
        assert e.value.code == G.GDAG_ERR_INVALID
