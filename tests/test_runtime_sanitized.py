"""The C++ runtime under AddressSanitizer and UndefinedBehaviorSanitizer.

The library's host code (tracker, stream manager, fake backend, argument
validation) is rebuilt with both sanitizers into a temporary directory, and a
plain-C driver (tests/c/random_programs.c) runs hundreds of random programs
of every element kind through the C ABI on the recording fake backend: small
node-table trim thresholds, every log level, captures and replays, fused
launches, re-registration and injected failures.  Any invalid access, leak or
undefined behaviour aborts the driver.  CPU only (needs nvcc and gcc)."""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2012_09646_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DRIVER = os.path.join(ROOT, "tests", "c", "random_programs.c")
SAN = "-fsanitize=address,-fsanitize=undefined,-fno-omit-frame-pointer,-fno-sanitize-recover=all"


def _compile(src, out):
    cmd = [B.nvcc(), "-std=c++17", "-O1", "-g", "-Xcompiler", "-fPIC," + SAN, "-I", B.INCLUDE, "-I", B.CSRC,
           "-c", src, "-o", out]
    if src.endswith(".cu"):
        cmd[1:1] = [B.ARCH, "--expt-relaxed-constexpr"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if not shutil.which("gcc") or not os.path.exists(B.nvcc()):
        pytest.skip("needs nvcc and gcc")
    d = tmp_path_factory.mktemp("san")
    srcs = B.sources()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        objs = list(ex.map(lambda s: _compile(s, str(d / (os.path.basename(s) + ".o"))), srcs))
    lib = str(d / "libgdag_san.so")
    r = subprocess.run([B.nvcc(), "-shared", B.ARCH, "-cudart", "shared", "-Xcompiler", SAN, "-o", lib] + objs,
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    exe = str(d / "random_programs")
    r = subprocess.run(["gcc", "-std=c99", "-O1", "-g", "-Wall", "-Wextra", "-Werror",
                        "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
                        "-I", B.INCLUDE, DRIVER, "-L", str(d), "-lgdag_san", "-Wl,-rpath," + str(d), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("seed", range(4))
def test_random_programs_are_clean_under_sanitizers(driver, seed):
    env = dict(os.environ,
               ASAN_OPTIONS="detect_leaks=1:halt_on_error=1:protect_shadow_gap=0:abort_on_error=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([driver, "150", "300", str(seed)], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    assert r.stdout.startswith("ok 150 programs"), r.stdout
    assert "runtime error" not in r.stderr and "Sanitizer" not in r.stderr, r.stderr[-4000:]
