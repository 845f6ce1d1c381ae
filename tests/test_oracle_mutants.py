"""The oracle's pins catch plausible mistakes.

Each mutant below is one plausible slip planted in a copy of the oracle: a
dropped term, a flipped sign, a transposed index, a wrong bound or label.
The pins (the oracle's own tests against closed forms, worked examples,
library special cases and brute force) run against the mutated copy in a
separate pytest process, and at least one of them must fail.  An unmutated
copy must pass, so a failure is the mutant's doing.  CPU only; mistakes are
planted in the oracle only, never in the product."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_numeric.py", "tests/test_oracle_dag.py", "tests/test_analysis.py"]

# (file in oracle/, text, replacement): the first occurrence is replaced
MUTANTS = [
    # VEC
    ("numeric.c", "out[i] = x[i] * x[i];", "out[i] = x[i] + x[i];"),
    ("numeric.c", "s += x[i] - y[i];", "s += y[i] - x[i];"),
    ("numeric.c", "s += fabs(x[i] - y[i]);", "s += x[i] - y[i];"),
    # B&S
    ("numeric.c", "return 0.5 * erfc(-x / sqrt(2.0));", "return 0.5 * erfc(x / sqrt(2.0));"),
    ("numeric.c", "return 0.5 * erfc(-x / sqrt(2.0));", "return 0.5 * erfc(-x / 2.0);"),
    ("numeric.c", "(r + 0.5 * sigma * sigma) * T)", "(r + sigma * sigma) * T)"),
    ("numeric.c", "double d2 = d1 - sigma * sqrt(T);", "double d2 = d1 + sigma * sqrt(T);"),
    ("numeric.c", "C[i] = S[i] * orc_cnd(d1) - K * exp(-r * T) * orc_cnd(d2);",
     "C[i] = S[i] * orc_cnd(d1) - K * exp(r * T) * orc_cnd(d2);"),
    ("numeric.c", "C[i] = S[i] * orc_cnd(d1) - K * exp(-r * T) * orc_cnd(d2);",
     "C[i] = S[i] * orc_cnd(d2) - K * exp(-r * T) * orc_cnd(d1);"),
    ("numeric.c", "A[i] = S[i] * orc_cnd(d1) + K * exp(-r * T) * orc_cnd(d2);",
     "A[i] = S[i] * orc_cnd(d1) - K * exp(-r * T) * orc_cnd(d2);"),
    # IMG
    ("numeric.c", "(2.0 * sigma * sigma)", "(sigma * sigma)"),
    ("numeric.c", "w[k] /= s;", "w[k] /= 1.0;"),
    ("numeric.c", "int64_t rr = clampi(r + i, 0, rows - 1);", "int64_t rr = clampi(r + i, 0, cols - 1);"),
    ("numeric.c", "s += w[i + R] * w[j + R] * img[rr * cols + cc];", "s += w[i + R] * img[rr * cols + cc];"),
    ("numeric.c", "gy += Kx[j + 1][i + 1] * v;", "gy += Kx[i + 1][j + 1] * v;"),
    ("numeric.c", "out[r * cols + c] = sqrt(gx * gx + gy * gy);", "out[r * cols + c] = gx * gx + gy * gy;"),
    ("numeric.c", "sy += fabs(Kx[j + 1][i + 1] * v);", "sy += fabs(Kx[i + 1][j + 1] * v);"),
    ("numeric.c", "out[r * cols + c] = sx + sy;", "out[r * cols + c] = sx;"),
    ("numeric.c", "if (x[i] > hi) hi = x[i];", "if (x[i] < hi) hi = x[i];"),
    ("numeric.c", "(in[i] - mn) / (mx - mn)", "(in[i] - mn) / mx"),
    ("numeric.c", "(in[i] - mn) / (mx - mn) : 0.0;", "(in[i] - mn) / (mx - mn) : in[i];"),
    ("numeric.c", "img[i] + alpha * (img[i] - blur[i])", "img[i] - alpha * (img[i] - blur[i])"),
    ("numeric.c", "(e9[i] * b5[i] + (1.0 - e9[i]) * b9[i])", "(e9[i] * b9[i] + (1.0 - e9[i]) * b5[i])"),
    # ML
    ("numeric.c", "s += X[i * feats + f] * T[f * classes + c];", "s += X[i * feats + f] * T[c * feats + f];"),
    ("numeric.c", "double s = bias[c];", "double s = 0.0;"),
    ("numeric.c", "s += fabs(X[i * feats + f] * T[f * classes + c]);", "s += X[i * feats + f] * T[f * classes + c];"),
    ("numeric.c", "P[i * classes + c] = exp(S[i * classes + c] - m) / z;", "P[i * classes + c] = exp(S[i * classes + c] - m);"),
    ("numeric.c", "if (v > bv) {", "if (v >= bv) {"),
    ("numeric.c", "margin[i] = (classes > 1) ? bv - second : INFINITY;", "margin[i] = (classes > 1) ? bv : INFINITY;"),
    # HITS
    ("numeric.c", "s += val[k] * x[col[k]];", "s += x[col[k]];"),
    ("numeric.c", "for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)",
     "for (int64_t k = rowptr[i]; k + 1 < rowptr[i + 1]; ++k)"),
    ("numeric.c", "s += fabs(val[k] * x[col[k]]);", "s += val[k] * x[col[k]];"),
    ("numeric.c", "return sqrt(s);", "return s;"),
    ("numeric.c", "out[i] = (nrm > 0.0) ? x[i] / nrm : x[i];", "out[i] = (nrm > 0.0) ? x[i] * nrm : x[i];"),
    ("numeric.c", "out[i] = (nrm > 0.0) ? x[i] / nrm : x[i];", "out[i] = (nrm > 0.0) ? x[i] / nrm : 0.0;"),
    # DL
    ("numeric.c", "double s = bias[co];", "double s = 0.0;"),
    ("numeric.c", "const double r = s > 0.0 ? s : 0.0;", "const double r = s;"),
    ("numeric.c", "wt[((co * cin + ci) * 3 + (dy + 1)) * 3 + (dx + 1)]",
     "wt[((co * cin + ci) * 3 + (dx + 1)) * 3 + (dy + 1)]"),
    ("numeric.c", "if (r > best) best = r;", "best = r;"),
    ("numeric.c", "e[p] = s / (double)hw;", "e[p] = s / (double)(hw + 1);"),
    ("numeric.c", "s += e2[b * c + i] * wd[(c + i) * classes + j];", "s += e2[b * c + i] * wd[i * classes + j];"),
    # dependency rule (Section III-A, Fig. 3)
    ("dag.py", "if mi & W and mj == R:\n                    if not any(m & W for m in between):",
     "if mi & W and mj == R:\n                    if not any(m != 0 for m in between):"),
    ("dag.py", "if not any(m != 0 for m in between):", "if not any(m & W for m in between):"),
    ("dag.py", "edges.add((i, j, a, WAR))", "edges.add((i, j, a, WAW))"),
    ("dag.py", "RAW if mj & R else WAW", "WAW"),
    ("dag.py", "if mi is not None and ((mi | mj) & W):", "if mi is not None and ((mi & mj) & W):"),
    ("dag.py", "            r |= reach[j]\n", ""),
    # happens-before replay
    ("dag.py", "            if t == OP_WAIT and e in last_record:\n                preds.append(last_record[e])",
     "            if t == OP_WAIT and e in last_record:\n                pass"),
    ("dag.py", "        elif t == OP_STREAM_SYNC:\n            if s in last_on_stream:\n                preds.append(last_on_stream[s])",
     "        elif t == OP_STREAM_SYNC:\n            pass"),
    ("dag.py", "if t in (OP_HOST_WAIT, OP_STREAM_SYNC, OP_HOST_NODE, OP_QUERY_DONE):\n            host_frontier = q",
     "if t in (OP_HOST_WAIT, OP_STREAM_SYNC):\n            host_frontier = q"),
    ("dag.py", "if pnode is None or pnode not in parents.get(node, ()) or pstream == s:",
     "if pnode is None or pnode not in parents.get(node, ()):"),
    # the benchmark programs composed from the nodes
    ("pipelines.py", "z = N.sum_diff(x2, y2)", "z = N.sum_diff(x, y)"),
    ("pipelines.py", 'out["e9_raw"] = N.sobel(out["b9"])', 'out["e9_raw"] = N.sobel(out["b5"])'),
    ("pipelines.py", 'out["e5"] = N.extend(out["e5_raw"], *out["mm5"])', 'out["e5"] = N.extend(out["e5_raw"], *out["mm9"])'),
    ("pipelines.py", 'out["s"] = N.unsharp(image, out["b5"], IMG_ALPHA)', 'out["s"] = N.unsharp(image, out["b9"], IMG_ALPHA)'),
    ("pipelines.py", 'out["out"] = N.combine(out["s"], out["b5"], out["b9"], out["e5"], out["e9"])',
     'out["out"] = N.combine(out["s"], out["b5"], out["b9"], out["e9"], out["e5"])'),
    ("pipelines.py", 'out["s2"] = N.scores(X, ridge_w, ridge_b)', 'out["s2"] = N.scores(X, ridge_w, nb_prior)'),
    ("pipelines.py", 'out["p2"] = N.softmax_rows(out["s2"])', 'out["p2"] = N.softmax_rows(out["s1"])'),
    ("pipelines.py", "a_raw = N.spmv_csr(csc[0], csc[1], csc[2], h)", "a_raw = N.spmv_csr(csr[0], csr[1], csr[2], h)"),
    ("pipelines.py", "h_raw = N.spmv_csr(csr[0], csr[1], csr[2], a)", "h_raw = N.spmv_csr(csr[0], csr[1], csr[2], h)"),
    ("pipelines.py", "a = N.scale(a_raw, na)", "a = N.scale(a_raw, nh)"),
    ("pipelines.py", 'out["p2"] = N.conv3x3_relu_pool(x2, w2, b2)', 'out["p2"] = N.conv3x3_relu_pool(x2, w1, b2)'),
    ("pipelines.py", 'out["e2"] = N.avgpool(out["p2"])', 'out["e2"] = N.avgpool(out["p1"])'),
    ("pipelines.py", 'out["logits"] = N.concat_dense(out["e1"], out["e2"], wd, bd)',
     'out["logits"] = N.concat_dense(out["e2"], out["e1"], wd, bd)'),
    # overlap metrics and the longest path (Sections IV-E, IV-F)
    ("overlap.py", "if any(u <= t < v for (u, v) in other_sets(k)):", "if any(u < t < v for (u, v) in other_sets(k)):"),
    ("overlap.py", "\"CC\": share(compute, lambda k: [c for i, c in enumerate(compute) if i != k]),",
     "\"CC\": share(compute, lambda k: compute),"),
    ("overlap.py", "        acc += weights[v]\n", ""),
]


def run_pins(tmp, mutant):
    """Copy oracle/ under tmp, apply `mutant` (None: unmutated), run the
    pins against the copy; returns (return code, output tail)."""
    dst = os.path.join(tmp, "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), dst, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    if mutant is not None:
        fname, old, new = mutant
        path = os.path.join(dst, fname)
        text = open(path).read()
        assert old in text, mutant
        open(path, "w").write(text.replace(old, new, 1))
    env = dict(os.environ, ORACLE_UNDER_TEST=tmp, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    built = os.path.exists(os.path.join(dst, "_build", "liboracle.so"))
    return r.returncode, (r.stdout + r.stderr)[-2000:], built


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    jobs = [None] + MUTANTS
    dirs = [str(tmp_path_factory.mktemp("m%d" % i)) for i in range(len(jobs))]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(run_pins, dirs, jobs))
    return dict(zip(range(len(jobs)), res))


def test_unmutated_copy_passes(outcomes):
    rc, out, built = outcomes[0]
    assert rc == 0, out
    assert built  # the pins ran the copy's own C oracle, not the repository's


@pytest.mark.parametrize("k", range(1, len(MUTANTS) + 1))
def test_mutant_is_caught(outcomes, k):
    rc, out, _ = outcomes[k]
    # 1: a pin failed (not a crash, a collection error or a usage error)
    assert rc == 1 and " failed" in out, (MUTANTS[k - 1], rc, out)
