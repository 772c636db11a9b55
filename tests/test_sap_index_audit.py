"""CPU replays of the index arithmetic of the patching kernels (csrc/sap.cu)
and the streamed filter's staging (csrc/filter.cu): every shared-memory
read lands inside the region the previous stage wrote, every global access
stays inside its buffer.  No GPU is needed; the constants are the kernels'."""
import itertools

import numpy as np
import pytest

TILE, HALO, SPAN = 32, 4, 40
STRIDES = {"IN": 68, "HH": 68, "SS": 66, "MM": 64}


def clamp(v, hi):
    return 0 if v < 0 else hi if v > hi else v


def canny_tile_accesses(n, bx, by, clamped):
    """Replay canny_tile for one block: returns {array: (writes, reads)} as
    sets of (row, col) staged indices, and the global pixels written."""
    nm = n - 1
    oy, ox = by * TILE - HALO, bx * TILE - HALO
    cl = (lambda v: clamp(v, nm)) if clamped else (lambda v: v)
    iy = lambda y: cl(y) - oy
    ix = lambda x: cl(x) - ox
    acc = {k: (set(), set()) for k in ("IN", "HH", "SS", "GX", "GY", "MM")}
    glob = set()
    for r, c in itertools.product(range(SPAN), range(SPAN)):       # staging
        acc["IN"][0].add((r, c))
        y, x = (clamp(oy + r, nm), clamp(ox + c, nm)) if clamped else (oy + r, ox + c)
        assert 0 <= y < n and 0 <= x < n
    for r, c in itertools.product(range(SPAN), range(2, SPAN - 2)):  # horizontal
        x = cl(ox + c)
        for k in range(-2, 3):
            acc["IN"][1].add((r, ix(x + k)))
        acc["HH"][0].add((r, c))
    for r, c in itertools.product(range(2, SPAN - 2), repeat=2):       # vertical
        y = cl(oy + r)
        for k in range(-2, 3):
            acc["HH"][1].add((iy(y + k), c))
        acc["SS"][0].add((r, c))
    for r, c in itertools.product(range(3, SPAN - 3), repeat=2):       # Sobel
        y, x = cl(oy + r), cl(ox + c)
        for dy, dx in itertools.product((-1, 0, 1), repeat=2):
            acc["SS"][1].add((iy(y + dy), ix(x + dx)))
        for k in ("GX", "GY", "MM"):
            acc[k][0].add((r, c))
    for r, c in itertools.product(range(HALO, HALO + TILE), repeat=2):   # suppression
        y, x = oy + r, ox + c
        if y >= n or x >= n:
            continue
        glob.add((y, x))
        acc["GX"][1].add((r, c))
        acc["GY"][1].add((r, c))
        acc["MM"][1].add((r, c))
        for dy, dx in ((0, 1), (1, 0), (1, 1), (1, -1)):
            for sgn in (-1, 1):
                py, px = y + sgn * dy, x + sgn * dx
                if 0 <= py < n and 0 <= px < n:
                    acc["MM"][1].add((r + sgn * dy, c + sgn * dx))
    return acc, glob


@pytest.mark.parametrize("n", [16, 32, 64, 128])
def test_canny_staging_reads_only_what_was_written(n):
    tiles = (n + TILE - 1) // TILE
    seen = set()
    for by, bx in itertools.product(range(tiles), repeat=2):
        oy, ox = by * TILE - HALO, bx * TILE - HALO
        interior = oy >= 0 and ox >= 0 and oy + SPAN <= n and ox + SPAN <= n
        for clamped in ([False, True] if interior else [True]):
            acc, glob = canny_tile_accesses(n, bx, by, clamped)
            for name, (w, r) in acc.items():
                assert r <= w, f"{name} read outside its written region (n={n}, tile {bx},{by})"
                stride = STRIDES.get({"GX": "IN", "GY": "HH"}.get(name, name))
                assert all(0 <= a < SPAN and 0 <= b < stride for a, b in w)
            seen |= glob
    assert seen == set(itertools.product(range(n), repeat=2))     # every pixel classified once per tile


def test_canny_shared_memory_size_and_vector_alignment():
    words = SPAN * sum(STRIDES.values())
    assert words * 4 == 42560 and words * 4 <= 48 * 1024
    # the interior staging stores 16-byte vectors into IN at column 4 c4 of each row
    assert (STRIDES["IN"] * 4) % 16 == 0
    # interior tiles load 8 bytes at ox = 32 bx - 4 codes: 2 (32 bx - 4) bytes
    assert all((2 * (32 * bx - 4)) % 8 == 0 for bx in range(1, 300))


def test_canny_strides_are_conflict_free_for_their_readers():
    """A warp's 32 consecutive linear indices over a region W wide, stored
    with row stride S, touch 32 distinct banks when S = W (mod 32)."""
    for name, width in (("IN", 36), ("HH", 36), ("SS", 34), ("MM", 32)):
        s = STRIDES[name]
        for start in range(0, 4 * width):
            banks = {((i // width) * s + i % width) % 32 for i in range(start, start + 32)}
            assert len(banks) == 32, (name, start)


def level_base(l):
    return (4 ** l - 1) // 3


@pytest.mark.parametrize("n,P", [(16, 4), (64, 8), (256, 16), (8192, 16), (16384, 4), (512, 64)])
def test_tree_indices_stay_inside_the_node_arrays(n, P):
    L = int(np.log2(n // P))
    T, Ns = level_base(L + 1), level_base(L)
    for l in range(L + 1):
        count = 4 ** l
        lo, hi = level_base(l), level_base(l) + count - 1
        assert hi < T
        if l < L:
            assert hi < Ns                                     # keys and split flags
            assert level_base(l + 1) + 4 * (count - 1) + 3 < T  # children
        if l > 0:
            assert level_base(l - 1) + (count - 1) // 4 < Ns   # parent key / split flag
    # keys: V < 2^29 fits above bit 35 of the high word, the Morton code of a
    # corner in units of P below bit 31 of the low word, the level in 4 bits
    assert n * n < 2 ** 29 and (n // P) ** 2 <= 2 ** 31 and L < 16


@pytest.mark.parametrize("n,P", [(64, 4), (64, 16), (1024, 8), (8192, 16)])
def test_depatch_rows_and_words_stay_inside_leaf_and_mask(n, P):
    """Replay depatch_pack_kernel's (row phase, item) walk for every leaf
    side: rows by + 4 i < s, words or bytes inside the leaf's packed span."""
    phases = 4
    for s in [P * 2 ** j for j in range(int(np.log2(n // P)) + 1)]:
        f = s // P
        lf = int(np.log2(f))
        x0 = y0 = n - s                                        # the last aligned leaf
        for by in range(phases):
            if by >= s:
                continue
            rows = (s - by + phases - 1) // phases
            ys = [by + phases * i for i in range(rows)]
            assert all(y < s for y in ys) and (ys[-1] + phases >= s)
            if s >= 16:
                wpr = s >> 4
                for w in (0, wpr - 1):
                    assert (16 * w + 15) >> lf < P            # patch column
                    off = x0 // 4 + 4 * w
                    assert off % 4 == 0 and off + 4 <= n // 4
            else:
                bpr = s // 4
                for k in (0, bpr - 1):
                    assert (4 * k + 3) >> lf < P and x0 // 4 + k < n // 4
            assert (ys[-1] >> lf) < P and y0 + ys[-1] < n


@pytest.mark.parametrize("D", [4, 8, 2048, 2052, 4096, 4100, 8188, 8192])
def test_streamed_filter_staging_fits(D):
    """The streamed filter runs where the transform length L is 8192 or
    16384 (one pair per block); two rows of D floats must fit in the L-float
    staging buffer, and every bulk copy is a multiple of 16 bytes from a
    16-byte aligned row."""
    L = max(512, 1 << int(np.ceil(np.log2(2 * D - 1)))) if D > 1 else 512
    if L not in (8192, 16384) or D % 4:
        return
    assert 2 * D <= L
    assert (D * 4) % 16 == 0 and (2 * D * 4) % 16 == 0
    assert 2 * D * 4 < 2 ** 20                                 # mbarrier transaction count
    assert L * 8 + L * 4 <= 227 * 1024                         # transform + staging buffers
