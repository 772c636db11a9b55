"""Plain CPU oracle for symmetric adaptive patching (SAP) of a reconstructed
slice and the 2-bit masks -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  It shares no code with the CUDA library.

The paper's AI stage (Sec. V-B(c), "Symmetric Adaptive Patching") turns a
slice into a short sequence of patches before the segmentation model:

  (1) edge detection by Canny's method;
  (2) a quadtree built by repeatedly splitting the leaf whose edge image
      has the largest sum (Eq. 1: split argmax_i V(L_n[i]) into s = 2^d = 4
      children until the leaf count reaches the target), then splitting by
      pixel-intensity variance so that every slice gives the same sequence
      length, and ordering the patches along a Z-order curve;
  (3) depatching: mask patches are scaled back onto the slice through the
      stored quadtree.
The fused pipeline stores 4-class masks as 2 bits per pixel (Sec. V-C(a)).

The paper fixes none of the numbers or tie rules; the readings here are:

* input: the slice's uint16 codes (the stage-4 output of the reconstruction);
* Canny in integer arithmetic: a 5-tap binomial smoothing (1 4 6 4 1) along
  each axis, 3x3 Sobel gradients, L1 magnitude M = |gx| + |gy|, borders
  replicated; non-maximum suppression along the gradient direction quantised
  to 0, 45, 90 or 135 degrees (the sector tests compare |gy| 2^15 with
  round(tan(22.5 deg) 2^15) |gx| and round(tan(67.5 deg) 2^15) |gx|); a
  pixel survives if its M is above the previous neighbour's and not below
  the next one's (outside the slice M = 0); strong if M > hi, weak if
  lo < M <= hi; the edges are the strong pixels and the weak pixels
  8-connected to them through weak pixels;
* V(node) = number of edge pixels in the node;
* the variance criterion: the node's sum of squared deviations
  SSD = sum x^2 - (sum x)^2 / n, evaluated in IEEE double as
  d(S2) - d(S1) * d(S1) / d(n) with each operation rounded once (sums are
  exact integers); SSD never grows from a node to its children, and the key
  used is min(SSD, the parent's key) so that rounding cannot break that;
* a leaf may be split while its side exceeds the patch size P; the next
  split takes the splittable leaf with the largest (V, SSD key), ties broken
  by the shallower level and then the smaller Morton code; splitting stops
  when the leaf count reaches the target length, which must be 1 mod 3;
* the sequence is the leaves in Z-order (Morton code of the top-left corner,
  x in the even bits); each leaf of side s = P 2^j becomes a P x P patch of
  the means of its 2^j x 2^j blocks, rounded to float32 from
  d(block sum) / d(block size);
* depatching writes patch value [r][c] to the leaf's pixels
  [y0 + r 2^j + a][x0 + c 2^j + b]; the 2-bit mask stores pixel 4k + i of a
  row in bits 2i..2i+1 of byte k.
"""
from __future__ import annotations

import heapq

import numpy as np

TAN22_Q15 = int(round(np.tan(np.pi / 8) * 32768))        # 13573
TAN67_Q15 = int(round(np.tan(3 * np.pi / 8) * 32768))    # 79109
BINOMIAL5 = (1, 4, 6, 4, 1)


# ---------------------------------------------------------------------------
# (1) Canny edges
# ---------------------------------------------------------------------------
def smooth(img) -> np.ndarray:
    """Binomial 5-tap smoothing along x then y, borders replicated; the
    result is the exact integer sum (scale 256)."""
    a = np.asarray(img, dtype=np.int64)
    n0, n1 = a.shape
    p = np.pad(a, ((0, 0), (2, 2)), mode="edge")
    h = sum(w * p[:, i:i + n1] for i, w in enumerate(BINOMIAL5))
    p = np.pad(h, ((2, 2), (0, 0)), mode="edge")
    return sum(w * p[i:i + n0, :] for i, w in enumerate(BINOMIAL5))


def sobel(s):
    """(gx, gy) of the 3x3 Sobel operator, borders replicated; gx grows with
    the column index, gy with the row index."""
    p = np.pad(np.asarray(s, dtype=np.int64), 1, mode="edge")
    n0, n1 = s.shape

    def at(dr, dc):
        return p[1 + dr:1 + dr + n0, 1 + dc:1 + dc + n1]

    gx = (at(-1, 1) + 2 * at(0, 1) + at(1, 1)) - (at(-1, -1) + 2 * at(0, -1) + at(1, -1))
    gy = (at(1, -1) + 2 * at(1, 0) + at(1, 1)) - (at(-1, -1) + 2 * at(-1, 0) + at(-1, 1))
    return gx, gy


def nms_classes(gx, gy, lo: int, hi: int) -> np.ndarray:
    """Non-maximum suppression and double threshold: 0 none, 1 weak, 2 strong.
    The gradient direction is quantised by integer comparisons; the pixel is
    compared with its two neighbours along it (M = 0 outside the slice)."""
    gx = np.asarray(gx, dtype=np.int64)
    gy = np.asarray(gy, dtype=np.int64)
    m = np.abs(gx) + np.abs(gy)
    n0, n1 = m.shape
    mp = np.pad(m, 1, mode="constant")          # M = 0 outside the slice

    def shifted(dr, dc):                         # M at (r + dr, c + dc)
        return mp[1 + dr:1 + dr + n0, 1 + dc:1 + dc + n1]

    ax, ay = np.abs(gx), np.abs(gy)
    horiz = ay * 32768 <= TAN22_Q15 * ax
    vert = ~horiz & (ay * 32768 >= TAN67_Q15 * ax)
    diag = ~horiz & ~vert & ((gx > 0) == (gy > 0))     # along (+r, +c)
    anti = ~horiz & ~vert & ~diag                     # along (+r, -c)
    prev = np.select([horiz, vert, diag, anti], [shifted(0, -1), shifted(-1, 0), shifted(-1, -1), shifted(-1, 1)])
    nxt = np.select([horiz, vert, diag, anti], [shifted(0, 1), shifted(1, 0), shifted(1, 1), shifted(1, -1)])
    keep = (m > lo) & (m > prev) & (m >= nxt)
    out = np.zeros((n0, n1), dtype=np.uint8)
    out[keep & (m <= hi)] = 1
    out[keep & (m > hi)] = 2
    return out


def hysteresis(cls) -> np.ndarray:
    """Edges: the 8-connected components of the candidate (weak or strong)
    pixels that hold a strong pixel.  The labelling is scipy's."""
    from scipy import ndimage
    cls = np.asarray(cls)
    lab, count = ndimage.label(cls > 0, structure=np.ones((3, 3), dtype=int))
    strong = np.zeros(count + 1, dtype=bool)
    strong[np.unique(lab[cls == 2])] = True
    strong[0] = False
    return strong[lab].astype(np.uint8)


def canny(img, lo: int, hi: int) -> np.ndarray:
    """Edge map (uint8, 1 on edges) of a uint16 slice."""
    gx, gy = sobel(smooth(img))
    return hysteresis(nms_classes(gx, gy, lo, hi))


# ---------------------------------------------------------------------------
# (2) Adaptive quadtree, Eq. (1), and the Z-order sequence
# ---------------------------------------------------------------------------
def morton(x: int, y: int) -> int:
    """Interleave x (even bits) and y (odd bits)."""
    code = 0
    for b in range(32):
        code |= ((x >> b) & 1) << (2 * b) | ((y >> b) & 1) << (2 * b + 1)
    return code


def ssd_key(s1: int, s2: int, n: int) -> float:
    """d(S2) - d(S1) * d(S1) / d(n), each operation rounded once in IEEE double."""
    a = np.float64(s1)
    t = (a * a) / np.float64(n)
    return float(np.float64(s2) - t)


def node_stats(img, edges, x0: int, y0: int, s: int):
    """(V, S1, S2, n) of the s x s node at (x0, y0): edge count, sum and sum of
    squares of the codes, pixel count (exact integers)."""
    blk = np.asarray(img[y0:y0 + s, x0:x0 + s], dtype=np.int64)
    v = int(np.asarray(edges[y0:y0 + s, x0:x0 + s], dtype=np.int64).sum())
    return v, int(blk.sum()), int((blk * blk).sum()), s * s


def quadtree(img, edges, P: int, length: int):
    """Greedy adaptive quadtree: returns (leaves, splits), leaves as (x0, y0, s)
    in Z-order, splits as the list of split nodes (x0, y0, s) in split order."""
    n = img.shape[0]
    if img.shape != (n, n) or n & (n - 1) or n < P or P < 1 or P & (P - 1):
        raise ValueError("the slice must be square with a power-of-two side >= P (a power of two)")
    if length < 1 or (length - 1) % 3:
        raise ValueError("the sequence length must be 1 mod 3")
    max_leaves = (n // P) ** 2
    if length > max_leaves:
        raise ValueError("sequence longer than the number of P x P patches")

    def entry(x0, y0, s, parent_key):
        v, s1, s2, cnt = node_stats(img, edges, x0, y0, s)
        key2 = min(ssd_key(s1, s2, cnt), parent_key)
        level = (n // s).bit_length() - 1
        # heapq pops the smallest: negate the "largest first" keys
        return (-v, -key2, level, morton(x0 // P, y0 // P)), (x0, y0, s, key2)

    heap = []
    final = []                       # leaves that cannot be split (side == P)
    k, node = entry(0, 0, n, float("inf"))
    (heap if n > P else final).append((k, node))
    heapq.heapify(heap)
    splits = []
    count = 1
    while count < length:
        _, (x0, y0, s, key2) = heapq.heappop(heap)
        splits.append((x0, y0, s))
        h = s // 2
        for dy in (0, h):
            for dx in (0, h):
                k, node = entry(x0 + dx, y0 + dy, h, key2)
                if h > P:
                    heapq.heappush(heap, (k, node))
                else:
                    final.append((k, node))
        count += 3
    leaves = [(nd[0], nd[1], nd[2]) for _, nd in heap] + [(nd[0], nd[1], nd[2]) for _, nd in final]
    leaves.sort(key=lambda t: morton(t[0] // P, t[1] // P))
    return leaves, splits


def extract_patches(img, leaves, P: int) -> np.ndarray:
    """Each leaf of side s = P 2^j as a P x P patch of its 2^j x 2^j block means."""
    out = np.empty((len(leaves), P, P), dtype=np.float32)
    for i, (x0, y0, s) in enumerate(leaves):
        f = s // P
        blk = np.asarray(img[y0:y0 + s, x0:x0 + s], dtype=np.int64).reshape(P, f, P, f)
        sums = blk.sum(axis=(1, 3)).astype(np.float64)
        out[i] = (sums / np.float64(f * f)).astype(np.float32)
    return out


# ---------------------------------------------------------------------------
# (3) Depatching and the 2-bit mask
# ---------------------------------------------------------------------------
def depatch(patches, leaves, n: int, P: int) -> np.ndarray:
    """Mask [n][n] from per-leaf P x P mask patches (nearest upscaling)."""
    patches = np.asarray(patches)
    out = np.zeros((n, n), dtype=patches.dtype)
    for i, (x0, y0, s) in enumerate(leaves):
        f = s // P
        out[y0:y0 + s, x0:x0 + s] = np.repeat(np.repeat(patches[i], f, axis=0), f, axis=1)
    return out


def pack2(mask) -> np.ndarray:
    """4-class mask [rows][cols] (values 0..3, cols a multiple of 4) to bytes
    [rows][cols / 4]: pixel 4k + i in bits 2i..2i+1 of byte k."""
    m = np.asarray(mask, dtype=np.uint8)
    if m.shape[-1] % 4 or np.any(m > 3):
        raise ValueError("columns must be a multiple of 4 and classes in 0..3")
    q = m.reshape(m.shape[:-1] + (m.shape[-1] // 4, 4))
    return (q[..., 0] | (q[..., 1] << 2) | (q[..., 2] << 4) | (q[..., 3] << 6)).astype(np.uint8)


def unpack2(packed) -> np.ndarray:
    b = np.asarray(packed, dtype=np.uint8)
    out = np.stack([(b >> (2 * i)) & 3 for i in range(4)], axis=-1)
    return out.reshape(b.shape[:-1] + (b.shape[-1] * 4,))
