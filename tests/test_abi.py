"""The C-ABI library loads and exports every function include/gdag.h
declares (no compute calls: CPU only)."""
import ctypes
import os
import re

from paper_2012_09646_gb300 import build as B
from paper_2012_09646_gb300 import gdag as G

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gdag.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gdag_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    B.build()
    lib = ctypes.CDLL(G.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []
    # and the binding covers all of them
    assert sorted(G.SIGNATURES) == names


def test_builtin_kernel_table():
    ctx = G.Context(backend="fake")
    for name, nargs in [("vec_square", 2), ("vec_reduce_diff", 5), ("bs_call", 7)]:
        kid, spec = ctx.kernel(name)
        assert len(spec) == nargs
    ctx.close()


def test_scratch_sizes():
    assert G.gdag_scratch_bytes("vec_reduce_diff", 10) >= 8 * 1024 + 4
    assert G.gdag_scratch_bytes("bs_call", 10) == 0


def test_binding_constants_match_the_header():
    """Every integer #define of gdag.h that the binding mirrors has the
    header's value (the ctypes binding cannot include the header)."""
    hdr = open(HEADER).read()
    seen = 0
    for name, val in re.findall(r"^#define (GDAG_\w+)\s+(-?\d+)\b", hdr, flags=re.M):
        if hasattr(G, name):
            assert getattr(G, name) == int(val), name
            seen += 1
    assert seen >= 40 and G.GDAG_AUTO_GRAPH_SEQS == 64
