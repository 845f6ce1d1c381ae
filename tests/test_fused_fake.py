"""Fused launches (gdag_launch_fused) in the dependency tracker, driven through
the C ABI with the recording fake backend (no GPU): a fused element's edges
are those of one element whose accesses are the union of its members', as the
brute-force oracle computes them; invalid member sets are rejected before
anything is recorded.  CPU only."""
import random

import pytest

from oracle import dag as D
from paper_2012_09646_gb300 import gdag as G

N = 4096  # floats per fake array


class FusedProgram:
    """Random programs of built-in VEC/B&S launches on fake device arrays,
    some issued one by one and some fused, mirrored as oracle elements."""

    def __init__(self, n_arrays, n_scratch, **opts):
        opts.setdefault("record_log", True)
        self.ctx = G.Context(backend="fake", **opts)
        self.arrays = [self.ctx.array(dev=0x100000 * (i + 1), nbytes=4 * N) for i in range(n_arrays)]
        sb = G.gdag_scratch_bytes("vec_reduce_diff", N)
        self.scratch = [self.ctx.array(dev=0x10000000 + 0x100000 * i, nbytes=sb) for i in range(n_scratch)]
        self.elems = []

    def member(self, rng, kind, used_w, used):
        """Arguments and oracle accesses of one member whose written arrays
        avoid every array already used in this element (and whose read arrays
        avoid those already written)."""
        free = [i for i in range(len(self.arrays)) if i not in used]
        readable = [i for i in range(len(self.arrays)) if i not in used_w]
        if kind == "vec_square":
            if not free:
                return None
            a = rng.choice(free)
            return (self.arrays[a], N), {a: D.RW}
        if kind == "bs_call":
            if not free or not readable:
                return None
            c = rng.choice(free)
            s = rng.choice([i for i in readable if i != c] or [None])
            if s is None:
                return None
            return (self.arrays[s], self.arrays[c], N, 60.0, 0.1, 0.2, 1.0), {s: D.R, c: D.W}
        # vec_reduce_diff: x, y read, z written, scratch read and written
        sfree = [j for j in range(len(self.scratch)) if ("s", j) not in used]
        if len(free) < 1 or len(readable) < 2 or not sfree:
            return None
        z = rng.choice(free)
        xs = [i for i in readable if i != z]
        if len(xs) < 2:
            return None
        x, y = rng.sample(xs, 2)
        j = rng.choice(sfree)
        return ((self.arrays[x], self.arrays[y], self.arrays[z], self.scratch[j], N),
                {x: D.R, y: D.R, z: D.W, ("s", j): D.RW})

    def issue(self, rng, kind, count):
        members, acc = [], {}
        used, used_w = set(), set()
        for _ in range(count):
            m = self.member(rng, kind, used_w, used)
            if m is None:
                break
            args, a = m
            members.append(args)
            for k, mode in a.items():
                acc[k] = acc.get(k, 0) | mode
                used.add(k)
                if mode & D.W:
                    used_w.add(k)
        if not members:
            return None
        if len(members) == 1 and rng.random() < 0.5:
            node = self.ctx.launch(kind, *members[0])
        else:
            node = self.ctx.launch_fused(kind, members)
        assert node == len(self.elems)
        self.elems.append(acc)
        return node

    def oracle_elems(self):
        """Element maps with scratch arrays renamed past the data arrays."""
        n = len(self.arrays)
        return [{(n + k[1] if isinstance(k, tuple) else k): m for k, m in e.items()} for e in self.elems]

    def handle_map(self):
        n = len(self.arrays)
        m = {a.handle: i for i, a in enumerate(self.arrays)}
        m.update({s.handle: n + j for j, s in enumerate(self.scratch)})
        return m


@pytest.mark.parametrize("seed", range(40))
def test_random_fused_programs_match_brute_force(seed):
    rng = random.Random(seed)
    opts = rng.choice([{}, {"max_streams": 2}, {"retire_by_query": True, "fake_complete": True},
                       {"policy": G.GDAG_POLICY_SERIAL_ASYNC}, {"max_streams": 1}])
    p = FusedProgram(rng.randint(3, 10), rng.randint(1, 4), **opts)
    for _ in range(rng.randint(1, 30)):
        p.issue(rng, rng.choice(["vec_square", "bs_call", "vec_reduce_diff"]), rng.randint(1, 5))
    hm = p.handle_map()
    got = {(s, d, hm[a], k) for s, d, a, k in p.ctx.edges()}
    want = D.expected_edges(p.oracle_elems())
    assert got == want
    ops = p.ctx.ops()
    assert D.check_hb(ops, want) == []
    assert D.waits_off_edges(ops, want) == []
    # one launch op per element, fused or not
    launches = [o for o in ops if o[0] == G.GDAG_OP_LAUNCH]
    assert len(launches) == len(p.elems)


def test_fused_element_takes_every_members_edges():
    """Three producers on three streams, then one fused consumer of all three:
    it waits on each producer (RAW on each array) and is one node."""
    ctx = G.Context(backend="fake", record_log=True)
    a = [ctx.array(dev=0x100000 * (i + 1), nbytes=4 * N) for i in range(6)]
    p = [ctx.launch("vec_square", a[i], N) for i in range(3)]
    node = ctx.launch_fused("bs_call", [(a[i], a[3 + i], N, 60.0, 0.1, 0.2, 1.0) for i in range(3)])
    edges = set(ctx.edges())
    for i in range(3):
        assert (p[i], node, a[i].handle, G.GDAG_EDGE_RAW) in edges
    assert len(ctx.nodes()) == 4
    st = ctx.stats()
    assert st["fused_members"] == 3 and st["launches"] == 4
    waits = [o for o in ctx.ops() if o[0] == G.GDAG_OP_WAIT and o[3] in p]
    assert len(waits) == 2  # the fused node sits on one producer's stream


def test_fused_rejects_conflicting_members_and_kernels_without_a_fused_form():
    ctx = G.Context(backend="fake", record_log=True)
    a = [ctx.array(dev=0x100000 * (i + 1), nbytes=4 * N) for i in range(4)]
    bs = lambda s, c: (s, c, N, 60.0, 0.1, 0.2, 1.0)
    with pytest.raises(G.GdagError) as e:  # the same output twice
        ctx.launch_fused("bs_call", [bs(a[0], a[1]), bs(a[2], a[1])])
    assert e.value.code == G.GDAG_ERR_INVALID
    with pytest.raises(G.GdagError):  # one member reads what another writes
        ctx.launch_fused("bs_call", [bs(a[0], a[1]), bs(a[1], a[2])])
    with pytest.raises(G.GdagError):  # the same in-place array twice
        ctx.launch_fused("vec_square", [(a[0], N), (a[0], N)])
    with pytest.raises(G.GdagError):  # a member gdag_launch would reject (n too large)
        ctx.launch_fused("vec_square", [(a[0], N), (a[1], N + 1)])
    with pytest.raises(G.GdagError) as e:  # no fused form
        ctx.launch_fused("scale", [(a[0], a[1], N)])
    assert e.value.code == G.GDAG_ERR_INVALID
    with pytest.raises(G.GdagError):
        ctx.launch_fused("vec_square", [])
    # two readers of one input are fine
    ctx.launch_fused("bs_call", [bs(a[0], a[1]), bs(a[0], a[2])])
    assert len(ctx.nodes()) == 1
    assert ctx.stats()["fused_members"] == 2


def test_fused_count_limits():
    ctx = G.Context(backend="fake")
    kid = ctx.kernel("vec_square")[0]
    with pytest.raises(G.GdagError):
        G.gdag_launch_fused(ctx.h, kid, [], 2, 0)
    arrays = [ctx.array(dev=0x1000 * (i + 1), nbytes=16) for i in range(G.GDAG_FUSED_MAX + 1)]
    args = []
    for x in arrays:
        args += [G.array_arg(x.handle), G.scalar_arg(4, 8)]
    with pytest.raises(G.GdagError):
        G.gdag_launch_fused(ctx.h, kid, args, 2, G.GDAG_FUSED_MAX + 1)
    # more members than one kernel table holds: still one element
    n = G.GDAG_FUSED_TABLE * 2 + 3
    G.gdag_launch_fused(ctx.h, kid, args[: 2 * n], 2, n)
    st = ctx.stats()
    assert st["nodes"] == 1 and st["fused_members"] == n
