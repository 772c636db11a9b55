"""The oracle against the hand-worked examples in tests/golden/ (each file
states its derivation and the passage it follows): ramp filtering of a
three-bin row, backprojection and forward projection on a 2 x 2 image, and
the Eq. (1) quadtree on an 8 x 8 slice."""
import os

import numpy as np
import pytest

import oracle
from oracle import sap

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def records(name):
    """Data lines of a fixture as (first word, remaining words)."""
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                words = line.split()
                out.append((words[0], words[1:]))
    return out


def triples(words):
    return [tuple(int(v) for v in w.split(",")) for w in words]


@pytest.mark.parametrize("filter_fn", [oracle.filter_direct, oracle.filter_fft])
def test_three_bin_filter(filter_fn):
    kinds = {"ramlak": oracle.RAMLAK, "shepp_logan": oracle.SHEPP_LOGAN}
    inputs = {"impulse": [0.0, 1.0, 0.0], "ones": [1.0, 1.0, 1.0]}
    rows = [r for r in records("filter_3bin.txt")]
    assert len(rows) == 4
    for kind, rest in rows:
        p = np.array([inputs[rest[0]]])
        want = np.array([float(v) for v in rest[1:]])
        got = filter_fn(p, kinds[kind])[0]
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15)


def test_two_by_two_backprojection_and_forward_projection():
    rec = dict(records("projector_2x2.txt"))
    g = oracle.Geometry(2, 2, 2)
    q = np.array([float(v) for v in rec["bp_input"]]).reshape(2, 2)      # [K][D]
    f = oracle.backproject(q, g)
    np.testing.assert_allclose(f.ravel(), [float(v) for v in rec["bp_output"]], rtol=1e-14)
    img = np.array([float(v) for v in rec["fwd_input"]]).reshape(2, 2)   # [N][N]
    p = oracle.forward(img, g)
    np.testing.assert_allclose(p.ravel(), [float(v) for v in rec["fwd_output"]], rtol=1e-14, atol=1e-14)


def test_eight_by_eight_quadtree():
    rec = dict(records("sap_quadtree_8x8.txt"))
    img = np.zeros((8, 8), dtype=np.uint16)
    edges = np.zeros((8, 8), dtype=np.uint8)
    for r, c in (tuple(int(v) for v in w.split(",")) for w in rec["edges_row_col"]):
        edges[r, c] = 1
    leaves, splits = sap.quadtree(img, edges, 2, 7)
    assert splits == triples(rec["length7_splits"])
    assert leaves == triples(rec["length7_leaves"])
    _, splits = sap.quadtree(img, edges, 2, 10)
    assert splits[2] == triples(rec["length10_third_split"])[0]
