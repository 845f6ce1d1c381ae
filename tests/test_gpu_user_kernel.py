"""A user kernel registered with gdag_kernel_register (Section III-D: the
programmer's own kernels, with each argument annotated as read-only or
modified) and launched through the CUDA backend as a DAG element.  The
kernel is compiled here into its own shared library (nvcc, sm_103a, the
shared CUDA runtime, as the library uses), so it is a __global__ function
the library did not build.  Checked against a numpy fp64 oracle, and its
edges against the built-in kernels around it."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from paper_2012_09646_gb300 import gdag as G

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def axpy_handle(tmp_path_factory):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("user") / "libaxpy.so")
    subprocess.run([nvcc, "-shared", "-Xcompiler", "-fPIC", "-gencode=arch=compute_103a,code=sm_103a",
                    "-cudart", "shared", "-O2", os.path.join(HERE, "user_kernels", "axpy.cu"), "-o", out],
                   check=True, capture_output=True, text=True)
    lib = ctypes.CDLL(out)
    lib.user_axpy_handle.restype = ctypes.c_void_p
    return lib, lib.user_axpy_handle()


def spec(kind, mode=G.GDAG_MODE_DEFAULT, size=0):
    return G.gdag_argspec(kind, mode, size, 0)


def test_user_kernel_runs_as_a_dag_element(axpy_handle):
    _lib, fn = axpy_handle
    n = 1_000_003
    g = np.random.default_rng(4)
    x = g.random(n, dtype=np.float32)
    y = g.random(n, dtype=np.float32)
    a = np.float32(1.75)
    with G.Context(record_log=True) as ctx:
        k = G.gdag_kernel_register(ctx.h, "user_axpy", fn, [
            spec(G.GDAG_ARG_ARRAY, G.GDAG_MODE_IN), spec(G.GDAG_ARG_ARRAY, G.GDAG_MODE_INOUT),
            spec(G.GDAG_ARG_SCALAR, size=4), spec(G.GDAG_ARG_SCALAR, size=8)])
        ctx._kernels["user_axpy"] = (k, G.gdag_kernel_signature(ctx.h, k))
        dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        X, Y = ctx.array(dx), ctx.array(dy)
        # x := x*x (built in), y := a x + y (user), y := y*y (built in)
        k0 = ctx.launch("vec_square", X, n)
        k1 = ctx.launch("user_axpy", X, Y, float(a), n, grid=(4 * 152, 1, 1), block=(256, 1, 1))
        k2 = ctx.launch("vec_square", Y, n)
        ctx.sync()
        got = dy.cpu().numpy().astype(np.float64)
        edges = {(s, d) for s, d, _a, _k in ctx.edges()}
    assert (k0, k1) in edges and (k1, k2) in edges
    x2 = x.astype(np.float64) ** 2
    want = (np.float64(a) * x2 + y) ** 2
    # fp32 steps (a multiply-add and two squares): a few units in the last place
    assert np.all(np.abs(got - want) <= 1e-6 * np.maximum(np.abs(want), 1.0))


def test_user_kernel_signature_checks(axpy_handle):
    _lib, fn = axpy_handle
    with G.Context() as ctx:
        k = G.gdag_kernel_register(ctx.h, "user_axpy", fn, [
            spec(G.GDAG_ARG_ARRAY, G.GDAG_MODE_IN), spec(G.GDAG_ARG_ARRAY, G.GDAG_MODE_INOUT),
            spec(G.GDAG_ARG_SCALAR, size=4), spec(G.GDAG_ARG_SCALAR, size=8)])
        t = torch.zeros(8, device="cuda")
        A = ctx.array(t)
        # a user kernel needs an explicit launch shape
        with pytest.raises(G.GdagError) as e:
            G.gdag_launch(ctx.h, k, G.gdag_dim3(0, 0, 0), G.gdag_dim3(0, 0, 0), 0,
                          [G.array_arg(A.handle), G.array_arg(A.handle), G.scalar_arg(1.0, 4), G.scalar_arg(8, 8)])
        assert e.value.code == G.GDAG_ERR_INVALID
        # a scalar of the wrong size
        with pytest.raises(G.GdagError) as e:
            G.gdag_launch(ctx.h, k, G.gdag_dim3(1, 1, 1), G.gdag_dim3(32, 1, 1), 0,
                          [G.array_arg(A.handle), G.array_arg(A.handle), G.scalar_arg(1.0, 8), G.scalar_arg(8, 8)])
        assert e.value.code == G.GDAG_ERR_INVALID
