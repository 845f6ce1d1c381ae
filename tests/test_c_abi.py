"""The boundary as a C program sees it: include/gdag.h compiles as strict C99
and as C++17 with warnings as errors, every struct has the size and field
offsets the ctypes binding assumes, and a C program drives a context on the
recording fake backend through the library.  CPU only (needs gcc)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2012_09646_gb300 import build as B
from paper_2012_09646_gb300 import gdag as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
STRUCTS = [G.gdag_dim3, G.gdag_options, G.gdag_arg, G.gdag_argspec, G.gdag_edge, G.gdag_node_info, G.gdag_op,
           G.gdag_trace_rec, G.gdag_stats, G.gdag_elem]

PROGRAM = r"""
#include "gdag.h"
#include <stddef.h>
#include <stdio.h>

#define CHECK(x) do { int rc_ = (x); if (rc_) { printf("fail %s %d\n", #x, rc_); return 1; } } while (0)

int main(void)
{
@LAYOUT@
    gdag_options o;
    gdag_options_default(&o);
    o.backend = GDAG_BACKEND_FAKE;
    o.record_log = 1;
    gdag_ctx *c = NULL;
    CHECK(gdag_create(&c, &o));
    gdag_array x, y;
    CHECK(gdag_array_register(c, (void *)0x100000, 4000, NULL, &x));
    CHECK(gdag_array_register(c, (void *)0x200000, 4000, NULL, &y));
    gdag_kernel k;
    CHECK(gdag_kernel_lookup(c, "vec_square", &k));
    gdag_arg args[2];
    args[0].kind = GDAG_ARG_ARRAY; args[0].mode = GDAG_MODE_SIGNATURE; args[0].array = x;
    args[0].size = 0; args[0].value = 0;
    args[1].kind = GDAG_ARG_SCALAR; args[1].mode = 0; args[1].array = 0; args[1].size = 8; args[1].value = 1000;
    gdag_dim3 auto_shape = {0, 0, 0};
    int64_t n1 = -1, n2 = -1, n3 = -1;
    CHECK(gdag_launch(c, k, auto_shape, auto_shape, 0, args, 2, &n1));
    args[0].array = y;
    CHECK(gdag_launch(c, k, auto_shape, auto_shape, 0, args, 2, &n2));
    args[0].array = x;
    args[0].mode = GDAG_MODE_IN;  /* a read of x after its writer: RAW */
    CHECK(gdag_launch(c, k, auto_shape, auto_shape, 0, args, 2, &n3));
    int bad = gdag_kernel_lookup(c, "no_such_kernel", &k);
    CHECK(gdag_sync(c));
    gdag_stats st;
    CHECK(gdag_stats_get(c, &st));
    gdag_edge e[8];
    size_t ne = 0;
    CHECK(gdag_dag_export(c, e, 8, &ne));
    printf("nodes %lld %lld %lld %lld\n", (long long)st.nodes, (long long)n1, (long long)n2, (long long)n3);
    printf("streams %d active %d\n", st.streams, st.active);
    printf("edges %zu\n", ne);
    for (size_t i = 0; i < ne && i < 8; ++i)
        printf("edge %lld %lld %d\n", (long long)e[i].src, (long long)e[i].dst, e[i].kind);
    printf("lookup %d\n", bad);
    gdag_destroy(c);
    return 0;
}
"""


def layout_lines():
    out = []
    for T in STRUCTS:
        name = T.__name__
        out.append('    printf("size %s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in T._fields_:
            out.append('    printf("field %s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    return "\n".join(out)


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    lib = B.build()
    d = tmp_path_factory.mktemp("cabi")
    src = d / "probe.c"
    src.write_text(PROGRAM.replace("@LAYOUT@", layout_lines()))
    exe = d / "probe"
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", INCLUDE, str(src),
           "-L", libdir, "-lgdag", "-Wl,-rpath," + libdir, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout.splitlines()


def test_header_compiles_as_cxx(tmp_path):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    src = tmp_path / "h.cpp"
    src.write_text('#include "gdag.h"\nint main() { gdag_options o; gdag_options_default(&o); return o.policy; }\n')
    r = subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", INCLUDE, "-c",
                        str(src), "-o", str(tmp_path / "h.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_struct_layouts_match_the_binding(program):
    sizes = {l.split()[1]: int(l.split()[2]) for l in program if l.startswith("size ")}
    fields = {(l.split()[1], l.split()[2]): int(l.split()[3]) for l in program if l.startswith("field ")}
    for T in STRUCTS:
        assert sizes[T.__name__] == ctypes.sizeof(T), T.__name__
        for f, _ in T._fields_:
            assert fields[(T.__name__, f)] == getattr(T, f).offset, (T.__name__, f)


def test_c_program_drives_a_context(program):
    lines = [l for l in program if not l.startswith(("size ", "field "))]
    assert lines[0] == "nodes 3 0 1 2"
    assert lines[1] == "streams 2 active 0"  # two independent squares, then the reader on x's stream
    assert lines[2] == "edges 1"
    assert lines[3] == "edge 0 2 %d" % G.GDAG_EDGE_RAW
    assert lines[4] == "lookup %d" % G.GDAG_ERR_NOT_FOUND
