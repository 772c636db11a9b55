"""Pins for the SAP oracle (Sec. V-B(c), Eq. (1); Sec. V-C(a) 2-bit masks):
hand-derived edges of step images, the hysteresis rule on constructed
chains, a hand-worked quadtree, the greedy split order's equivalence with a
top-M selection and its invariants, patch means, depatching and the 2-bit
layout."""
import numpy as np
import pytest

from oracle import sap


def test_tangent_constants():
    assert sap.TAN22_Q15 == 13573 and sap.TAN67_Q15 == 79109


def test_smoothing_is_the_binomial_filter_with_replicated_borders():
    rng = np.random.default_rng(0)
    img = rng.integers(0, 65536, (9, 11))
    s = sap.smooth(img)
    # brute force: sum over the 5 x 5 outer product of (1 4 6 4 1), indices clamped
    w = np.array(sap.BINOMIAL5)
    for r in range(9):
        for c in range(11):
            acc = 0
            for i in range(5):
                for j in range(5):
                    acc += w[i] * w[j] * int(img[min(max(r + i - 2, 0), 8), min(max(c + j - 2, 0), 10)])
            assert s[r, c] == acc
    assert sap.smooth(np.full((4, 4), 7)).tolist() == np.full((4, 4), 7 * 256).tolist()


def test_vertical_step_gives_one_column_of_edges():
    """I = a left of column c0, b from c0 on: the smoothed gradient is
    symmetric about c0 - 1/2, so the non-maximum test (strictly above the
    left neighbour, not below the right one) keeps column c0 - 1 only."""
    img = np.full((24, 32), 1000, dtype=np.uint16)
    img[:, 13:] = 5000
    e = sap.canny(img, lo=1000, hi=200000)
    assert set(zip(*np.nonzero(e))) == {(r, 12) for r in range(24)}
    # the mirrored step (b on the left) puts the edge at the same column
    e2 = sap.canny(img[:, ::-1].copy(), lo=1000, hi=200000)
    assert set(zip(*np.nonzero(e2))) == {(r, 31 - 13) for r in range(24)}


def test_horizontal_step_and_threshold_band():
    img = np.full((20, 16), 200, dtype=np.uint16)
    img[7:, :] = 600
    gx, gy = sap.sobel(sap.smooth(img))
    peak = int((np.abs(gx) + np.abs(gy)).max())
    assert set(zip(*np.nonzero(sap.canny(img, 0, peak - 1)))) == {(6, c) for c in range(16)}
    # peak magnitude not above hi: weak only, and no strong pixel keeps it
    assert sap.canny(img, 0, peak).sum() == 0
    assert sap.canny(img, peak, peak + 1).sum() == 0     # not above lo


def test_diagonal_step_keeps_the_two_pixels_beside_the_boundary():
    """Step along c = r + 1/2: gx = -gy, so the 45-degree test compares each
    pixel with the pixels two diagonals away, (r - 1, c + 1) and (r + 1, c - 1).
    The magnitude depends on c - r only and peaks at c - r = 0 and 1 (equal by
    symmetry), so both pixels beside the boundary survive, and nothing else."""
    n = 32
    r, c = np.mgrid[0:n, 0:n]
    img = np.where(c > r, 9000, 1000).astype(np.uint16)
    gx, gy = sap.sobel(sap.smooth(img))
    m = np.abs(gx) + np.abs(gy)
    assert np.all(gx[3:-3, 3:-3] == -gy[3:-3, 3:-3])
    peak = int(m[10, 10])
    assert peak == int(m[10, 11]) and peak > int(m[10, 9])
    e = sap.canny(img, lo=1000, hi=peak - 1)
    for i in range(3, n - 3):
        assert np.nonzero(e[i])[0].tolist() == [i, i + 1]
    assert sap.canny(img, lo=1000, hi=peak).sum() == 0      # no strong pixel


def test_hysteresis_keeps_weak_chains_touching_a_strong_pixel():
    cls = np.zeros((10, 12), dtype=np.uint8)
    cls[2, 1] = 2                       # strong
    cls[3, 2] = cls[4, 3] = cls[4, 4] = cls[5, 5] = 1   # weak chain, 8-connected to it
    cls[8, 8] = cls[8, 9] = 1           # isolated weak pair
    cls[0, 10] = 2                      # lone strong
    e = sap.hysteresis(cls)
    assert set(zip(*np.nonzero(e))) == {(2, 1), (3, 2), (4, 3), (4, 4), (5, 5), (0, 10)}


def nms_loops(gx, gy, lo, hi):
    """Brute force: the suppression rule pixel by pixel."""
    m = np.abs(gx) + np.abs(gy)
    n0, n1 = m.shape
    out = np.zeros((n0, n1), dtype=np.uint8)
    for r in range(n0):
        for c in range(n1):
            if m[r, c] <= lo:
                continue
            ax, ay = abs(int(gx[r, c])), abs(int(gy[r, c]))
            if ay * 32768 <= 13573 * ax:
                d = (0, 1)
            elif ay * 32768 >= 79109 * ax:
                d = (1, 0)
            elif (gx[r, c] > 0) == (gy[r, c] > 0):
                d = (1, 1)
            else:
                d = (1, -1)
            mag = [m[rr, cc] if 0 <= rr < n0 and 0 <= cc < n1 else 0
                   for rr, cc in ((r - d[0], c - d[1]), (r + d[0], c + d[1]))]
            if m[r, c] > mag[0] and m[r, c] >= mag[1]:
                out[r, c] = 2 if m[r, c] > hi else 1
    return out


def hysteresis_bfs(cls):
    """Brute force: grow from every strong pixel through weak 8-neighbours."""
    n0, n1 = cls.shape
    edge = np.zeros((n0, n1), dtype=np.uint8)
    stack = [(int(r), int(c)) for r, c in zip(*np.nonzero(cls == 2))]
    for r, c in stack:
        edge[r, c] = 1
    while stack:
        r, c = stack.pop()
        for dr in (-1, 0, 1):
            for dc in (-1, 0, 1):
                rr, cc = r + dr, c + dc
                if 0 <= rr < n0 and 0 <= cc < n1 and not edge[rr, cc] and cls[rr, cc] == 1:
                    edge[rr, cc] = 1
                    stack.append((rr, cc))
    return edge


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_vectorised_suppression_and_labelling_equal_brute_force(seed):
    img = random_slice(48, seed)
    gx, gy = sap.sobel(sap.smooth(img))
    m = np.abs(gx) + np.abs(gy)
    lo, hi = int(np.percentile(m, 60)), int(np.percentile(m, 90))
    cls = sap.nms_classes(gx, gy, lo, hi)
    np.testing.assert_array_equal(cls, nms_loops(gx, gy, lo, hi))
    np.testing.assert_array_equal(sap.hysteresis(cls), hysteresis_bfs(cls))
    e = sap.hysteresis(cls)
    assert np.all(e[cls == 2] == 1) and np.all(e[cls == 0] == 0) and (cls == 2).sum() > 0


def test_morton_interleave():
    assert [sap.morton(x, y) for x, y in [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (3, 5)]] == [0, 1, 2, 3, 4, 39]


def test_hand_worked_quadtree():
    """8 x 8 slice, P = 2, edges only in the top-left 4 x 4 quadrant and most
    of them in its top-right 2 x 2 child: length 7 splits the root, then that
    quadrant; length 10 then splits by variance (the edges sit in leaves of
    side P, which cannot split)."""
    img = np.zeros((8, 8), dtype=np.uint16)
    edges = np.zeros((8, 8), dtype=np.uint8)
    edges[0:2, 2:4] = 1
    edges[3, 0] = 1
    leaves, splits = sap.quadtree(img, edges, 2, 7)
    assert splits == [(0, 0, 8), (0, 0, 4)]
    assert leaves == [(0, 0, 2), (2, 0, 2), (0, 2, 2), (2, 2, 2), (4, 0, 4), (0, 4, 4), (4, 4, 4)]
    # length 10: every remaining node with edges is a 2 x 2 leaf (not splittable),
    # so the next split goes by variance among the 4 x 4 leaves; with a constant
    # slice all keys tie and the smallest Morton code goes first
    leaves, splits = sap.quadtree(img, edges, 2, 10)
    assert splits[2] == (4, 0, 4)
    img2 = img.copy()
    img2[6, 5] = 50                      # variance only in the bottom-right quadrant
    _, splits = sap.quadtree(img2, edges, 2, 10)
    assert splits[2] == (4, 4, 4)


def test_ties_go_to_the_shallower_node_then_the_smaller_morton_code():
    """16 x 16 constant slice, no edges, P = 2: every V and variance key
    ties.  Split 1 takes the root; split 2 the level-1 node with the smallest
    Morton code, (0, 0, 8); split 3 must take another level-1 node, (8, 0, 8),
    not one of the level-2 children (0, 0, 4) ... just created."""
    img = np.full((16, 16), 1234, dtype=np.uint16)
    edges = np.zeros((16, 16), dtype=np.uint8)
    leaves, splits = sap.quadtree(img, edges, 2, 10)
    assert splits == [(0, 0, 16), (0, 0, 8), (8, 0, 8)]
    assert leaves == [(0, 0, 4), (4, 0, 4), (0, 4, 4), (4, 4, 4),
                      (8, 0, 4), (12, 0, 4), (8, 4, 4), (12, 4, 4), (0, 8, 8), (8, 8, 8)]


def random_slice(n, seed):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 3000, (n, n)).astype(np.uint16)
    yy, xx = np.mgrid[0:n, 0:n]
    for _ in range(6):
        cx, cy, rad = rng.uniform(0, n, 2).tolist() + [rng.uniform(n / 10, n / 3)]
        img[(xx - cx) ** 2 + (yy - cy) ** 2 < rad ** 2] += np.uint16(rng.integers(5000, 20000))
    return img


@pytest.mark.parametrize("n,P,length,seed", [(32, 4, 40, 1), (64, 4, 100, 2), (64, 8, 40, 3), (32, 2, 256, 4)])
def test_quadtree_is_the_top_m_nodes_and_tiles_the_slice(n, P, length, seed):
    img = random_slice(n, seed)
    edges = sap.canny(img, 4000, 12000)
    leaves, splits = sap.quadtree(img, edges, P, length)
    assert len(leaves) == length and len(splits) == (length - 1) // 3
    # the leaves tile the slice exactly once, and are sorted in Z-order
    cover = np.zeros((n, n), dtype=int)
    for x0, y0, s in leaves:
        assert s >= P and x0 % s == 0 and y0 % s == 0
        cover[y0:y0 + s, x0:x0 + s] += 1
    assert np.all(cover == 1)
    codes = [sap.morton(x // P, y // P) for x, y, _ in leaves]
    assert codes == sorted(codes)

    # brute force: the split set is the top-M of all splittable nodes by
    # (V, SSD key with its ancestors' minimum, shallower, smaller Morton)
    keys = {}

    def walk(x0, y0, s, parent_key, level):
        v, s1, s2, cnt = sap.node_stats(img, edges, x0, y0, s)
        k2 = min(sap.ssd_key(s1, s2, cnt), parent_key)
        if s > P:
            keys[(x0, y0, s)] = (v, k2, -level, -sap.morton(x0 // P, y0 // P))
            h = s // 2
            for dy in (0, h):
                for dx in (0, h):
                    walk(x0 + dx, y0 + dy, h, k2, level + 1)

    walk(0, 0, n, float("inf"), 0)
    top = sorted(keys, key=lambda k: keys[k], reverse=True)[:len(splits)]
    assert set(top) == set(splits)
    # split keys never increase along the greedy order
    ks = [keys[s] for s in splits]
    assert all(a >= b for a, b in zip(ks, ks[1:]))


def test_quadtree_argument_checks():
    img = np.zeros((16, 16), dtype=np.uint16)
    e = np.zeros_like(img, dtype=np.uint8)
    with pytest.raises(ValueError):
        sap.quadtree(img, e, 4, 9)          # not 1 mod 3
    with pytest.raises(ValueError):
        sap.quadtree(img, e, 4, 19)         # more than 16 patches
    with pytest.raises(ValueError):
        sap.quadtree(img[:, :12], e[:, :12], 4, 4)
    leaves, splits = sap.quadtree(img, e, 4, 16)
    assert len(leaves) == 16 and all(s == 4 for _, _, s in leaves)
    leaves, splits = sap.quadtree(img, e, 4, 1)
    assert leaves == [(0, 0, 16)] and splits == []


def test_ssd_key_is_the_sum_of_squared_deviations():
    rng = np.random.default_rng(5)
    x = rng.integers(0, 65536, 64).astype(np.int64)
    exact = float(((x - x.mean()) ** 2).sum())
    assert sap.ssd_key(int(x.sum()), int((x * x).sum()), 64) == pytest.approx(exact, rel=1e-12)
    assert sap.ssd_key(7 * 64, 49 * 64, 64) == 0.0


def test_patches_are_block_means():
    img = random_slice(32, 6)
    leaves = [(0, 0, 16), (16, 0, 8), (24, 0, 8), (16, 8, 8), (24, 8, 8), (0, 16, 16), (16, 16, 16)]
    p = sap.extract_patches(img, leaves, 8)
    assert p.dtype == np.float32 and p.shape == (7, 8, 8)
    np.testing.assert_array_equal(p[1], img[0:8, 16:24].astype(np.float32))     # side P: the pixels
    ref = img[0:16, 0:16].astype(np.float64).reshape(8, 2, 8, 2).mean(axis=(1, 3))
    np.testing.assert_allclose(p[0], ref, rtol=2 ** -24)


def test_depatch_inverts_patching_of_leaf_aligned_masks():
    n, P = 32, 4
    img = random_slice(n, 7)
    leaves, _ = sap.quadtree(img, sap.canny(img, 4000, 12000), P, 22)
    rng = np.random.default_rng(8)
    cls = rng.integers(0, 4, len(leaves))
    mask = np.zeros((n, n), dtype=np.uint8)
    for (x0, y0, s), k in zip(leaves, cls):
        mask[y0:y0 + s, x0:x0 + s] = k
    patches = sap.extract_patches(mask, leaves, P)
    np.testing.assert_array_equal(sap.depatch(patches.astype(np.uint8), leaves, n, P), mask)


def test_two_bit_layout_and_round_trip():
    assert sap.pack2(np.array([[1, 2, 3, 0]])).tolist() == [[0x39]]
    rng = np.random.default_rng(9)
    m = rng.integers(0, 4, (6, 40)).astype(np.uint8)
    p = sap.pack2(m)
    assert p.shape == (6, 10) and p.nbytes * 16 == m.size * 4      # 1/16 of int32 storage
    np.testing.assert_array_equal(sap.unpack2(p), m)
    with pytest.raises(ValueError):
        sap.pack2(np.array([[4, 0, 0, 0]]))
