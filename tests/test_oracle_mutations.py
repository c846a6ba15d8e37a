"""The pins catch plausible mistakes in the oracle: each case copies the oracle
package, plants one error in its C source (on the CPU, in the copy only), and
runs the pin suite against the copy, which must fail.  An unmodified copy must
pass, so a failure means the planted error, not the harness."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, text in scpl_oracle.c, planted replacement); names ending in "(py)" plant
# the error in the wrapper module __init__.py instead
MUTATIONS = [
    ("luma weights swapped",
     "return (77 * (int)px[0] + 150 * (int)px[1] + 29 * (int)px[2] + 128) >> 8;",
     "return (29 * (int)px[0] + 150 * (int)px[1] + 77 * (int)px[2] + 128) >> 8;"),
    ("Sobel centre weight 1",
     "int gx = (y[0][2] + 2 * y[1][2] + y[2][2]) - (y[0][0] + 2 * y[1][0] + y[2][0]);",
     "int gx = (y[0][2] + y[1][2] + y[2][2]) - (y[0][0] + y[1][0] + y[2][0]);"),
    ("first frame has motion", "D[p] = 0;", "D[p] = 7;"),
    ("DP ties to the highest column",
     "if (best_j < 0 || up[jj] < up[best_j]) best_j = jj;",
     "if (best_j < 0 || up[jj] <= up[best_j]) best_j = jj;"),
    ("selection ties to the highest column",
     "return a->ce < b->ce || (a->ce == b->ce && a->col < b->col);",
     "return a->ce < b->ce || (a->ce == b->ce && a->col > b->col);"),
    ("backtrack mirrored",
     "path[i - 1] = path[i] + (int)dir[(long)i * W + path[i]] - 1;",
     "path[i - 1] = path[i] - (int)dir[(long)i * W + path[i]] + 1;"),
    ("sqrt(n) for sqrt(n-1)", "thr = thr * sqrt((double)(n - 1));",
     "thr = thr * sqrt((double)n);"),
    ("no t_max cap", "if (n == t_max) {", "if (n == t_max + 1) {"),
    ("motion of the first frame only",
     "E[p] += wg * G[p] + wm * (int)dm[(long)t * hw + p];",
     "E[p] += wg * G[p] + wm * (int)dm[p];"),
    ("forward diagonal terms swapped",
     "if (jj == j - 1) c += (int64_t)wf * A[p];\n                if (jj == j + 1) c += (int64_t)wf * B[p];",
     "if (jj == j - 1) c += (int64_t)wf * B[p];\n                if (jj == j + 1) c += (int64_t)wf * A[p];"),
    ("forward row term clamped at the border",
     "CU[p] = (j > 0 && j < W - 1) ? abs((int)r[j + 1] - (int)r[j - 1]) : 0;",
     "CU[p] = abs((int)r[j + 1 < W ? j + 1 : j] - (int)r[j > 0 ? j - 1 : 0]);"),
    ("forward diagonal term from the wrong column",
     "A[p] = (u && j >= 1) ? abs((int)u[j] - (int)r[j - 1]) : 0;",
     "A[p] = (u && j >= 1) ? abs((int)u[j - 1] - (int)r[j - 1]) : 0;"),
    ("label of the previous row's column",
     "CE[p] = (int64_t)E[p] + up[best_j];\n            L[p] = L[(long)(i - 1) * W + best_j];",
     "CE[p] = (int64_t)E[p] + up[best_j];\n            L[p] = best_j;"),
    ("no cap on k", "int cap = k < W - target ? k : W - target;", "int cap = k;"),
    ("flush starts after the crossing frame", "            start = f;",
     "            start = f + 1;"),
    ("maxval kept across a flush", "M = maxval_mode == 1 ? maxval_theory : emax;",
     "M = maxval_mode == 1 ? maxval_theory : M1;"),
    ("spread scaled by 128, not 256",
     "int64_t Q = (int64_t)n1 * a2 - a1 * a1;\n            A += (int64_t)isqrt_floor((uint64_t)Q << 16);",
     "int64_t Q = (int64_t)n1 * a2 - a1 * a1;\n            A += (int64_t)isqrt_floor((uint64_t)Q << 14);"),
    ("first child per parent instead of the least",
     "if (best[a].col < 0 || cand_less(&c, &best[a])) best[a] = c;",
     "if (best[a].col < 0) best[a] = c;"),
    ("seams recorded at the current column",
     "if (seams) seams[(long)(removed + s) * H + i] = (int16_t)orig[p];",
     "if (seams) seams[(long)(removed + s) * H + i] = (int16_t)path[i];"),
    ("every buffer carved from the clip's first frames",
     "int it = orc_carve_buffer(frames + 3 * (long)t0 * hw, D + (long)t0 * hw, tb, H, W0, target,",
     "int it = orc_carve_buffer(frames, D + (long)t0 * hw, tb, H, W0, target,"),
    ("one-sided frame difference", "D[(long)t * hw + p] = (uint8_t)abs(a - b);",
     "D[(long)t * hw + p] = (uint8_t)(a > b ? a - b : 0);"),
    ("insertion mean rounds down (py)", "out[t0:t1, i] = ((a + c + 1) >> 1).astype(np.uint8)",
     "out[t0:t1, i] = ((a + c) >> 1).astype(np.uint8)"),
    ("inserted pixel blends with the left neighbour (py)",
     "right.append(min(x + 1, W - 1))", "right.append(max(x - 1, 0))"),
    ("blend of one frame fewer (py)", "num += mag(Y[t:t + window].sum(axis=0))",
     "num += mag(Y[t:t + window - 1].sum(axis=0))"),
]


def _copy(tmp_path, name, old=None, new=None) -> str:
    dst = os.path.join(str(tmp_path), "oracle_copy")
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("*.so", "*.tmp*", "__pycache__"))
    if old is not None:
        src = os.path.join(dst, "__init__.py" if name.endswith("(py)") else "scpl_oracle.c")
        with open(src) as fh:
            text = fh.read()
        assert text.count(old) == 1, f"mutation target not unique: {old[:40]}"
        with open(src, "w") as fh:
            fh.write(text.replace(old, new))
    return dst


def _run_pins(path: str) -> subprocess.CompletedProcess:
    env = dict(os.environ, SCPL_ORACLE_DIR=path)
    return subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p",
                           "no:cacheprovider"], capture_output=True, text=True, env=env,
                          cwd=ROOT, timeout=300)


def test_unmodified_copy_passes(tmp_path):
    r = _run_pins(_copy(tmp_path, "oracle_copy"))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_error_fails_a_pin(tmp_path, name, old, new):
    r = _run_pins(_copy(tmp_path, name, old, new))
    assert r.returncode == 1, (name, r.returncode, r.stdout[-2000:])
    assert "failed" in r.stdout
