"""Planted-mistake check of the oracle's pins (a collected CPU test).

For each entry of MISTAKES a scratch copy of oracle/, tests/ and the
package's Python sources gets one plausible mistake planted in its copy of
the oracle (a flipped sign, a swapped operand or weight, a dropped factor, a
wrong index or tie order), and the oracle's pin tests run there; the mistake
counts as caught when that run fails.  Every mistake must be caught by all
pins, and also with the two tests that compare the oracle with a numpy
restatement of its own formula left out (closed forms, invariants and
hand-worked values alone).  The plantings run in parallel, each in its own
scratch directory; the repository itself is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_filter.py", "tests/test_oracle_backproject.py", "tests/test_oracle_offset.py",
        "tests/test_oracle_preprocess.py", "tests/test_oracle_sap.py", "tests/test_golden.py",
        "tests/test_phantoms.py"]

C = "oracle/fbp_oracle.c"
PY = "oracle/__init__.py"
SAP = "oracle/sap.py"
MISTAKES = [
    ("ramlak odd-tap sign", C, [("return -1.0 / (ORACLE_PI * ORACLE_PI * (double)n * (double)n * t2);",
                                 "return 1.0 / (ORACLE_PI * ORACLE_PI * (double)n * (double)n * t2);")]),
    ("ramlak h(0) = 1/(2 tau^2)", C, [("if (n == 0) return 1.0 / (4.0 * t2);", "if (n == 0) return 1.0 / (2.0 * t2);")]),
    ("ramlak even taps not zero", C, [("if ((n % 2) == 0) return 0.0;",
                                       "if ((n % 2) == 0) return -1.0 / (ORACLE_PI * ORACLE_PI * (double)n * (double)n * t2);")]),
    ("shepp-logan 4n^2+1", C, [("(4.0 * (double)n * (double)n - 1.0));", "(4.0 * (double)n * (double)n + 1.0));")]),
    ("filter drops tau", C, [("qk[j] = tau * s;", "qk[j] = s;")]),
    ("fft twiddle sign", C, [("double wr = cos(ang), wi = sin(ang);", "double wr = cos(ang), wi = -sin(ang);")]),
    ("interp weights swapped", C, [("return (1.0 - w) * qt(qk, D, j) + w * qt(qk, D, j + 1);",
                                    "return w * qt(qk, D, j) + (1.0 - w) * qt(qk, D, j + 1);")]),
    ("clamp instead of zero outside", C, [("return (j >= 0 && j < D) ? qk[j] : 0.0;",
                                           "return qk[j < 0 ? 0 : (j >= D ? D - 1 : j)];")]),
    ("pixel centre c - N/2", C, [("double X = (double)c - 0.5 * (double)(g->n - 1);",
                                  "double X = (double)c - 0.5 * (double)(g->n);")]),
    ("cos/sin swapped", C, [("return alpha * (X * ck + Y * sk) + g->det_center;",
                             "return alpha * (X * sk + Y * ck) + g->det_center;")]),
    ("detector centre sign", C, [("return alpha * (X * ck + Y * sk) + g->det_center;",
                                  "return alpha * (X * ck + Y * sk) - g->det_center;")]),
    ("Y term sign", C, [("return alpha * (X * ck + Y * sk) + g->det_center;",
                         "return alpha * (X * ck - Y * sk) + g->det_center;")]),
    ("alpha dropped", C, [("return alpha * (X * ck + Y * sk) + g->det_center;",
                           "return (X * ck + Y * sk) + g->det_center;")]),
    ("angles offset by half a step", C, [("double th = g->angle_start + (double)k * g->angle_step;",
                                          "double th = g->angle_start + ((double)k + 0.5) * g->angle_step;")]),
    ("backprojection output transposed", C, [("f[(size_t)r * N + c] = scale * acc;", "f[(size_t)c * N + r] = scale * acc;")]),
    ("forward weights swapped", C, [("if (j >= 0 && j < D) pk[j] += (1.0 - w) * v;", "if (j >= 0 && j < D) pk[j] += w * v;"),
                                    ("if (j + 1 >= 0 && j + 1 < D) pk[j + 1] += w * v;",
                                     "if (j + 1 >= 0 && j + 1 < D) pk[j + 1] += (1.0 - w) * v;")]),
    ("forward drops the second bin", C, [("if (j + 1 >= 0 && j + 1 < D) pk[j + 1] += w * v;", "(void)0;")]),
    ("fbp scale 1 instead of dtheta", C, [("rc = oracle_backproject(q, g, g->angle_step, f);",
                                           "rc = oracle_backproject(q, g, 1.0, f);")]),
    ("beer-lambert sign", PY, [("return float(mu_scale) * -np.log(I / _f64(I0))", "return float(mu_scale) * np.log(I / _f64(I0))")]),
    ("gaussian radius floor(4 sigma)", PY, [("r = int(4.0 * sigma + 0.5)", "r = int(4.0 * sigma)")]),
    ("gaussian not normalised", PY, [("return w / w.sum()", "return w")]),
    ("blur index sign", PY, [("y[..., lo:hi] += w[i] * p[..., lo - k:hi - k]", "y[..., lo:hi] += w[i] * p[..., lo - k:hi - k][..., ::-1]")]),
    ("HU factor 100", PY, [("return 1000.0 * (_f64(mu) - mu_water) / (mu_water - mu_air)",
                            "return 100.0 * (_f64(mu) - mu_water) / (mu_water - mu_air)")]),
    ("HU window 65536", PY, [("x = (hu(mu, mu_water, mu_air) - hu_min) / (hu_max - hu_min) * 65535.0",
                              "x = (hu(mu, mu_water, mu_air) - hu_min) / (hu_max - hu_min) * 65536.0")]),
    ("offset weight 1 - sin", PY, [("w[mid] = np.sin(0.25 * np.pi * (1.0 + t[mid] / overlap)) ** 2",
                                    "w[mid] = np.cos(0.25 * np.pi * (1.0 + t[mid] / overlap)) ** 2")]),
    ("offset weight 1/2 below the overlap", PY, [("w = np.where(t > overlap, 1.0, 0.0)", "w = np.where(t > overlap, 1.0, 0.5)")]),
    ("smoothing weights 1-2-3-2-1", SAP, [("BINOMIAL5 = (1, 4, 6, 4, 1)", "BINOMIAL5 = (1, 2, 3, 2, 1)")]),
    ("sobel gx centre weight 1", SAP, [("gx = (at(-1, 1) + 2 * at(0, 1) + at(1, 1)) - (at(-1, -1) + 2 * at(0, -1) + at(1, -1))",
                                       "gx = (at(-1, 1) + at(0, 1) + at(1, 1)) - (at(-1, -1) + at(0, -1) + at(1, -1))")]),
    ("sobel gx/gy swapped", SAP, [("return gx, gy\n", "return gy, gx\n")]),
    ("tangent sectors swapped", SAP, [("horiz = ay * 32768 <= TAN22_Q15 * ax", "horiz = ay * 32768 <= TAN67_Q15 * ax")]),
    ("diagonal sector sign", SAP, [("diag = ~horiz & ~vert & ((gx > 0) == (gy > 0))", "diag = ~horiz & ~vert & ((gx > 0) != (gy > 0))")]),
    ("suppression >= on both sides", SAP, [("keep = (m > lo) & (m > prev) & (m >= nxt)", "keep = (m > lo) & (m >= prev) & (m >= nxt)")]),
    ("hysteresis 4-connected", SAP, [("structure=np.ones((3, 3), dtype=int)", "structure=None")]),
    ("morton x in odd bits", SAP, [("code |= ((x >> b) & 1) << (2 * b) | ((y >> b) & 1) << (2 * b + 1)",
                                    "code |= ((y >> b) & 1) << (2 * b) | ((x >> b) & 1) << (2 * b + 1)")]),
    ("variance key sign", SAP, [("return float(np.float64(s2) - t)", "return float(t - np.float64(s2))")]),
    ("deeper node first on ties", SAP, [("return (-v, -key2, level, morton(x0 // P, y0 // P)), (x0, y0, s, key2)",
                                         "return (-v, -key2, -level, morton(x0 // P, y0 // P)), (x0, y0, s, key2)")]),
    ("patch mean divides by f", SAP, [("out[i] = (sums / np.float64(f * f)).astype(np.float32)",
                                       "out[i] = (sums / np.float64(f)).astype(np.float32)")]),
    ("patch blocks transposed", SAP, [("sums = blk.sum(axis=(1, 3)).astype(np.float64)",
                                       "sums = blk.sum(axis=(1, 3)).T.astype(np.float64)")]),
    ("pack2 bit order reversed", SAP, [("return (q[..., 0] | (q[..., 1] << 2) | (q[..., 2] << 4) | (q[..., 3] << 6)).astype(np.uint8)",
                                        "return (q[..., 3] | (q[..., 2] << 2) | (q[..., 1] << 4) | (q[..., 0] << 6)).astype(np.uint8)")]),
]


NUMPY_RESTATEMENTS = "not numpy_interp and not numpy_linear_convolution"


def fresh_copy(copy):
    if os.path.exists(copy):
        shutil.rmtree(copy)
    os.makedirs(copy)
    ign = shutil.ignore_patterns("*.so", "_build", "__pycache__", "*.o", ".pytest_cache")
    for d in ("oracle", "tests", "paper_2505_13955_gb300"):
        shutil.copytree(os.path.join(REPO, d), os.path.join(copy, d), ignore=ign)
    shutil.copy(os.path.join(REPO, "pytest.ini"), copy)


# the two pins that reconstruct whole phantoms with the oracle take most of
# the time: they run only when the others have not caught the mistake
SLOW = "shepp_logan_fbp_approaches_analytic_phantom or random_ellipses_fbp_close_to_phantom"


def run_pins(copy, k_expr, threads):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    for phase in (f"not ({SLOW})", SLOW):
        k = f"({phase}) and ({k_expr})" if k_expr else phase
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                            "-k", k, *PINS], cwd=copy, capture_output=True, text=True, timeout=900, env=env)
        failed = [l.split(" ")[1] for l in r.stdout.splitlines() if l.startswith("FAILED")]
        if r.returncode != 0:
            return r.returncode, failed
    return 0, []


def plant_and_run(root, index, k_expr, threads=1):
    """Plant MISTAKES[index] (index -1: none) in a fresh copy under root and
    run the pins: (return code, first failing test)."""
    copy = os.path.join(root, f"copy{index}")
    fresh_copy(copy)
    if index >= 0:
        name, f, reps = MISTAKES[index]
        path = os.path.join(copy, f)
        s = open(path).read()
        for a, b in reps:
            assert a in s, f"{name}: the line to change is not in {f}"
            s = s.replace(a, b, 1)
        with open(path, "w") as fh:
            fh.write(s)
    rc, failed = run_pins(copy, k_expr, threads)
    shutil.rmtree(copy, ignore_errors=True)
    return rc, failed[:1]


@pytest.mark.slow
def test_every_planted_mistake_is_caught(tmp_path):
    """All pins, and the pins without the two numpy restatements, each catch
    every planted mistake (both sets run in one pool of scratch copies)."""
    import concurrent.futures as cf
    cores = os.cpu_count() or 2
    sets = {"all pins": None, "without numpy restatements": NUMPY_RESTATEMENTS}
    for label, k in sets.items():
        rc, failed = plant_and_run(str(tmp_path / "base"), -1, k, threads=cores)
        assert rc == 0, f"{label}: the unmodified pins fail in the scratch copy: {failed}"
    with cf.ThreadPoolExecutor(max_workers=max(2, min(16, cores))) as ex:
        futs = {(label, i): ex.submit(plant_and_run, str(tmp_path / f"set{j}"), i, k)
                for j, (label, k) in enumerate(sets.items()) for i in range(len(MISTAKES))}
        missed = [(label, MISTAKES[i][0]) for (label, i), f in futs.items() if f.result()[0] == 0]
    assert not missed, f"planted mistakes the pins did not catch: {missed}"
