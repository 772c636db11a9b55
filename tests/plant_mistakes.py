"""Planted-mistake check of the oracle's pins (run by hand, not collected by
pytest):

    python tests/plant_mistakes.py [--scratch DIR] [--k EXPR] [NAME ...]

For each entry of MISTAKES it copies oracle/, tests/ and the package's
Python sources into a scratch directory, plants one plausible mistake in the
copy of the oracle (a flipped sign, a swapped operand or weight, a dropped
factor, a wrong index or tie order), and runs the oracle's pin tests there.
A mistake counts as caught when that run fails.  `--k` passes a pytest -k
expression, e.g. to leave out the tests that compare the oracle with a
numpy restatement of its own formula and keep only closed forms,
invariants and hand-worked values.  The repository itself is never
modified."""
import argparse
import json
import os
import shutil
import subprocess
import sys
import tempfile
import time

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COPY = None
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


def fresh_copy():
    if os.path.exists(COPY):
        shutil.rmtree(COPY)
    os.makedirs(COPY)
    ign = shutil.ignore_patterns("*.so", "_build", "__pycache__", "*.o")
    for d in ("oracle", "tests", "paper_2505_13955_gb300"):
        shutil.copytree(os.path.join(REPO, d), os.path.join(COPY, d), ignore=ign)
    shutil.copy(os.path.join(REPO, "pytest.ini"), COPY)


def run():
    extra = ["-k", K_EXPR] if K_EXPR else []
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *extra, *PINS],
                       cwd=COPY, capture_output=True, text=True, timeout=900)
    tail = (r.stdout.strip().splitlines() or [""])[-1]
    failed = [l.split(" ")[1] for l in r.stdout.splitlines() if l.startswith("FAILED")]
    return r.returncode, tail, failed


K_EXPR = None


def main():
    global COPY, K_EXPR
    ap = argparse.ArgumentParser()
    ap.add_argument("--scratch", default=None, help="scratch directory (default: a new temporary one)")
    ap.add_argument("--k", default=None, help="pytest -k expression for the pin run")
    ap.add_argument("names", nargs="*", help="run only these entries of MISTAKES")
    args = ap.parse_args()
    COPY = os.path.join(args.scratch or tempfile.mkdtemp(prefix="plant_mistakes_"), "copy")
    K_EXPR = args.k
    fresh_copy()
    rc, tail, _ = run()
    print("baseline:", rc, tail, flush=True)
    if rc != 0:
        sys.exit("the unmodified pins fail in the scratch copy")
    results = []
    for name, f, reps in MISTAKES:
        if args.names and name not in args.names:
            continue
        fresh_copy()
        path = os.path.join(COPY, f)
        s = open(path).read()
        for a, b in reps:
            if a not in s:
                sys.exit(f"{name}: the line to change is not in {f}")
            s = s.replace(a, b, 1)
        with open(path, "w") as fh:
            fh.write(s)
        t0 = time.time()
        rc, tail, failed = run()
        caught = rc != 0
        results.append({"mistake": name, "file": f, "caught": caught, "by": failed[:1],
                        "s": round(time.time() - t0, 1)})
        print(("CAUGHT " if caught else "MISSED ") + name, failed[:1], flush=True)
    shutil.rmtree(COPY, ignore_errors=True)
    print(sum(r["caught"] for r in results), "of", len(results), "caught")
    print(json.dumps(results))
    sys.exit(0 if all(r["caught"] for r in results) else 1)


if __name__ == "__main__":
    main()
