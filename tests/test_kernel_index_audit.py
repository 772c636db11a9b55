"""CPU audit of the kernels' index arithmetic (no GPU needed).

Replays, in numpy float32, the backprojection kernel's per-pixel coordinate
path (bp_tile.cuh) for every tile and angle of several geometries, and checks
that every interpolation index i = rne(u') lies inside the staged window
[-H, H] that the host sizes with bp_window_half().  Also checks the shared
memory index ranges of the FFT filter kernel's two layouts and the
batched-filter buffer bound, and the forward projector's candidate count.
"""
import math

import numpy as np
import pytest

F = np.float32


def window_half(alpha, tw, th):
    # restates runtime.cu:bp_window_half
    hx, hy = 0.5 * (tw - 1), 0.5 * (th - 1)
    return int(math.ceil(alpha * math.sqrt(hx * hx + hy * hy))) + 2


SHAPES = [  # (TXT, TYT, PX, PY) of the compiled variants (backproject.cu)
    (16, 16, 4, 4), (16, 16, 4, 2), (16, 16, 2, 4), (32, 8, 2, 8)]


def max_index(N, K, alpha, det_center, shape, angle_start=0.0, angle_step=None,
              tiles=None):
    TXT, TYT, PX, PY = shape
    TW, TH = TXT * PX, TYT * PY
    if angle_step is None:
        angle_step = math.pi / K
    H = window_half(alpha, TW, TH)
    tx = np.arange(TXT)
    ty = np.arange(TYT)
    dxt = (tx.astype(F) - F(0.5 * (TW - 1)))
    dyt = (ty.astype(F) - F(0.5 * (TH - 1)))
    ntx, nty = -(-N // TW), -(-N // TH)
    if tiles is None:
        tiles = [(a, b) for a in range(ntx) for b in range(nty)]
    worst = 0
    k = np.arange(K)
    th = angle_start + k * angle_step
    c = alpha * np.cos(th)
    s = alpha * np.sin(th)
    for (bx, by) in tiles:
        x0, y0 = bx * TW, by * TH
        Xc = x0 + 0.5 * (TW - 1) - 0.5 * (N - 1)
        Yc = y0 + 0.5 * (TH - 1) - 0.5 * (N - 1)
        uc = c * Xc + s * Yc + det_center
        jc = np.floor(uc)
        fc = (uc - jc - 0.5).astype(F)
        cx, sy = c.astype(F), s.astype(F)
        # u0[k, ty, tx] = fc + dxt*cx + dyt*sy
        u0 = (fc[:, None, None] + dxt[None, None, :] * cx[:, None, None]
              + dyt[None, :, None] * sy[:, None, None]).astype(F)
        stx, sty = (F(TXT) * cx).astype(F), (F(TYT) * sy).astype(F)
        for iy in range(PY):
            ur = (u0 + F(iy) * sty[:, None, None]).astype(F)
            for ix in range(PX):
                u = (ur + F(ix) * stx[:, None, None]).astype(F)
                i = np.rint(u)  # round half to even, as the magic-number add does
                worst = max(worst, int(np.max(np.abs(i))))
    return worst, H


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("N,K,alpha,dc", [
    (64, 90, 1.0, None), (100, 37, 1.0, 49.5), (257, 180, 1.0, None),
    (96, 64, 2.5, None), (96, 64, 0.125, 10.0), (130, 50, 0.7, 70.3)])
def test_backprojection_indices_stay_in_window(shape, N, K, alpha, dc):
    D = N
    worst, H = max_index(N, K, alpha, 0.5 * (D - 1) if dc is None else dc, shape)
    assert worst <= H


@pytest.mark.parametrize("shape", SHAPES[:1])
def test_backprojection_indices_n8192_sampled_tiles(shape):
    N, K = 8192, 4096
    TW = shape[0] * shape[2]
    nt = N // TW
    tiles = [(0, 0), (nt - 1, nt - 1), (0, nt - 1), (nt // 2, nt // 2), (17, 93), (nt - 1, 0)]
    worst, H = max_index(N, K, 1.0, 0.5 * (N - 1), shape, tiles=tiles)
    assert worst <= H


def test_magic_number_rounding_reads_index_from_bits():
    # t = u + 1.5*2^23 has unit ulp for |u| < 2^22; its bits are 0x4B400000 + rne(u)
    u = np.array([-300.5, -2.5, -1.5, -0.5, -0.49, 0.0, 0.5, 1.5, 2.49999, 47.3], dtype=F)
    t = (u + F(12582912.0)).astype(F)
    idx = t.view(np.uint32).astype(np.int64) - 0x4B400000
    np.testing.assert_array_equal(idx, np.rint(u).astype(np.int64))


@pytest.mark.parametrize("N1", [1, 2, 4, 8, 16, 32])
def test_filter_shared_layouts_fit_buffer(N1):
    L = 512 * N1
    size = L + 32
    logN1 = int(math.log2(N1))
    padsh = 4 + logN1
    n = np.arange(L)
    pos = n + (n >> padsh)
    assert pos.max() < size
    # step-1 reads: stride 16*N1 + 1 across lanes -> distinct banks per half-warp
    for n1 in range(N1):
        for r in range(16):
            lanes = np.arange(16)
            nn = n1 + N1 * (16 * lanes + r)
            p = nn + (nn >> padsh)
            assert len(set((2 * p) % 32)) == 16
    P = 512 + (1 if N1 >= 16 else 16 // N1)
    assert N1 * P <= size
    # transposed layout: T(n1, k2) = n1*P + k2 for k2 < 512
    assert (N1 - 1) * P + 511 < size
    # step-2 read pattern of a half-warp: n1 = lane & (N1-1), G from lane >> logN1
    for w in range(N1):
        lanes = np.arange(16)
        n1 = lanes & (N1 - 1)
        sg = lanes >> logN1
        G = w * (32 >> logN1) + sg
        p = n1 * P + G
        assert len(set((2 * p) % 32)) == 16
    # H index in step 2: 32 r + G + 512 k1 < L
    assert 32 * 15 + 31 + 512 * (N1 - 1) < L
    # batched filter: (32 / N1) groups of (L + 32) float2 fit the fixed buffer
    assert (32 // N1) * size <= 16384 + 1024


@pytest.mark.parametrize("alpha", [0.125, 0.5, 0.7, 1.0, 2.5])
def test_forward_candidate_count_bound(alpha):
    # candidates per line: ceil(2 / g), g = alpha * max(|cos|, |sin|) >= alpha / sqrt(2)
    th = np.linspace(0, np.pi, 10001)
    g = alpha * np.maximum(np.abs(np.cos(th)), np.abs(np.sin(th)))
    nc = np.ceil(2.0 / g)
    bound = math.ceil(2.0 * 1.4142135623730951 / alpha)
    assert nc.max() <= bound
    assert bound <= 24


ORBIT_SHAPES = [(16, 8, 2, 4), (16, 16, 4, 4)]   # (TXT, TYT, PX, PY), square tiles


def orbit_max_index(N, K, D, alpha, shape, tiles=None):
    """Replay of bp_orbit.cuh's coordinate path for both windows of every
    angle pair: u1 = f1 + dx c + dy s, u2 = f2 - dx s + dy c."""
    TXT, TYT, PX, PY = shape
    TILE = TXT * PX
    H = window_half(alpha, TILE, TILE)
    m = 0.5 * (N - 1)
    cd = 0.5 * (D - 1)
    dxt = np.arange(TXT).astype(F) - F(0.5 * (TILE - 1))
    dyt = np.arange(TYT).astype(F) - F(0.5 * (TILE - 1))
    half = N // TILE // 2
    if tiles is None:
        tiles = [(a, b) for a in range(half) for b in range(half)]
    th = np.arange(K // 2) * (math.pi / K)
    c = alpha * np.cos(th)
    s = alpha * np.sin(th)
    worst = 0
    for (ox, oy) in tiles:
        Xc = ox * TILE + 0.5 * (TILE - 1) - m
        Yc = oy * TILE + 0.5 * (TILE - 1) - m
        for (A, B, Ctr) in ((c, s, c * Xc + s * Yc + cd), (-s, c, -s * Xc + c * Yc + cd)):
            f = (Ctr - np.floor(Ctr) - 0.5).astype(F)
            A32, B32 = A.astype(F), B.astype(F)
            u0 = (f[:, None, None] + dxt[None, None, :] * A32[:, None, None]
                  + dyt[None, :, None] * B32[:, None, None]).astype(F)
            for iy in range(PY):
                ur = (u0 + F(iy) * (F(TYT) * B32)[:, None, None]).astype(F)
                for ix in range(PX):
                    u = (ur + F(ix) * (F(TXT) * A32)[:, None, None]).astype(F)
                    worst = max(worst, int(np.max(np.abs(np.rint(u)))))
    return worst, H


@pytest.mark.parametrize("shape", ORBIT_SHAPES)
@pytest.mark.parametrize("N,D,K,alpha", [(128, 128, 90, 1.0), (256, 230, 70, 0.9),
                                         (256, 300, 64, 2.5), (128, 40, 36, 0.125)])
def test_orbit_indices_stay_in_window(shape, N, D, K, alpha):
    if N % (2 * shape[0] * shape[2]):
        pytest.skip("geometry not eligible for this tile")
    worst, H = orbit_max_index(N, K, D, alpha, shape)
    assert worst <= H


def test_orbit_indices_n8192_sampled_tiles():
    N, K = 8192, 4096
    half = N // 32 // 2
    tiles = [(0, 0), (half - 1, half - 1), (0, half - 1), (half - 1, 0), (37, 101)]
    worst, H = orbit_max_index(N, K, N, 1.0, ORBIT_SHAPES[0], tiles=tiles)
    assert worst <= H


def test_orbit_smem_and_rotation_maps():
    # staged bytes per block fit the 200 KB budget for the compiled shapes
    for TILE, KT, EB in ((32, 16, 32), (32, 32, 16), (32, 8, 32), (64, 8, 32)):
        for alpha in (0.125, 1.0, 2.5):
            W = 2 * window_half(alpha, TILE, TILE) + 1
            assert KT * 32 + KT * 2 * W * EB <= 200 * 1024 or alpha > 2.0
    # the four stores of an orbit cover every pixel exactly once
    N, TILE = 64, 8
    hits = np.zeros((N, N), dtype=int)
    for oy in range(N // TILE // 2):
        for ox in range(N // TILE // 2):
            for a in range(TILE):
                for b in range(TILE):
                    r, c = oy * TILE + a, ox * TILE + b
                    for (rr, cc) in ((r, c), (c, N - 1 - r), (N - 1 - r, N - 1 - c), (N - 1 - c, r)):
                        hits[rr, cc] += 1
    assert np.all(hits == 1)


# ---------------------------------------------------------------------------
# Forward projector (forward.cu, fwd_strip_kernel): strip bounds
# ---------------------------------------------------------------------------
def fwd_pitch(alpha, ncmax):
    # restates forward.cu:fwd_span_pitch
    span = 127.0 * 1.4142135623730951 / alpha + 31.0 + ncmax + 5.0
    return int(math.ceil(span)) | 1


def fwd_walk(c, s, alpha, N, det_center, j, ncmax):
    walk_rows = abs(c) >= abs(s)
    cp = alpha * (c if walk_rows else s)
    cq = alpha * (s if walk_rows else c)
    g = abs(cp)
    h = 1.0 / g
    nc = min(ncmax, math.ceil(2.0 * h))
    m = 0.5 * (N - 1)
    slope = cq / cp
    B = (j - det_center + cq * m) / cp + m - h
    return walk_rows, g, nc, slope, B


def fwd_lines(slope, B, nc, N):
    lo, hi = 0.0, float(N - 1)
    if slope > 0:
        lo = max(lo, math.floor((B - N) / slope) - 1.0)
        hi = min(hi, math.ceil((B + nc + 1) / slope) + 1.0)
    elif slope < 0:
        lo = max(lo, math.floor((B + nc + 1) / slope) - 1.0)
        hi = min(hi, math.ceil((B - N) / slope) + 1.0)
    elif not (-nc - 1.0 < B < N):
        hi = -1.0
    return int(min(lo, N)), int(max(hi, -1.0))


def fwd_strip_audit(N, D, K, alpha, det_center, ks):
    ncmax = math.ceil(2.0 * 1.4142135623730951 / alpha)
    NCT = 4 if ncmax <= 4 else 24
    P = fwd_pitch(alpha, NCT)
    two32 = 4294967296.0
    for k in ks:
        th = k * math.pi / K
        c, s = math.cos(th), math.sin(th)
        for j0 in range(0, D, 128):
            jl = min(j0 + 127, D - 1)
            _, _, nca, sl_a, Ba = fwd_walk(c, s, alpha, N, det_center, j0, NCT)
            _, _, ncb, sl_b, Bb = fwd_walk(c, s, alpha, N, det_center, jl, NCT)
            if sl_a != 0.0:
                a0, a1 = fwd_lines(sl_a, Ba, nca, N)
                b0, b1 = fwd_lines(sl_b, Bb, ncb, N)
                blo, bhi = max(0, min(a0, b0)), min(N - 1, max(a1, b1))
            else:
                blo, bhi = 0, N - 1
            if blo > bhi:
                continue
            # block setup (thread 0): end bins' fixed-point positions at line blo
            SL = int(round(sl_a * two32))
            XMa = int(round((Ba - sl_a * blo) * two32))
            XMb = int(round((Bb - sl_b * blo) * two32))
            # every bin of the block (padding threads walk like the last bin)
            m = 0.5 * (N - 1)
            walk_rows = abs(c) >= abs(s)
            cp = alpha * (c if walk_rows else s)
            cq = alpha * (s if walk_rows else c)
            inv_cp = 1.0 / cp
            h = 1.0 / abs(cp)
            jw = np.minimum(np.arange(j0, j0 + 128), D - 1).astype(np.float64)
            Bj = (jw - det_center + cq * m) * inv_cp + m - h
            XM0 = np.array([int(round((b - sl_a * blo) * two32)) for b in Bj], dtype=np.int64)
            nc = nca
            for wc in range(blo, bhi + 1, 32):
                d0, d1 = (wc - blo) * SL, (wc + 31 - blo) * SL
                cs_ = [(XMa - d0) >> 32, (XMa - d1) >> 32, (XMb - d0) >> 32, (XMb - d1) >> 32]
                s_lo = min(cs_)
                s_hi = max(cs_) + NCT + 1
                span = s_hi - s_lo + 1
                assert span <= P - 1, (k, j0, wc, span, P)
                lines = np.arange(wc, min(wc + 32, bhi + 1))
                XM = XM0[None, :] - (lines - blo)[:, None] * np.int64(SL)
                start = (XM >> 32) + 1
                first = start - s_lo
                last = first + nc - 1
                assert first.min() >= 0, (k, j0, wc, first.min())
                assert last.max() <= span - 1, (k, j0, wc, last.max(), span)


@pytest.mark.parametrize("N,D,K,alpha,dc", [
    (64, 64, 36, 1.0, None), (130, 150, 40, 1.0, 70.25), (100, 90, 24, 1.3, None),
    (96, 300, 16, 2.4, None), (150, 40, 24, 0.25, 25.0), (128, 128, 20, 0.5, None),
    (64, 64, 8, 1.0, None)])
def test_forward_strip_reads_stay_in_staged_strip(N, D, K, alpha, dc):
    dc = 0.5 * (D - 1) if dc is None else dc
    fwd_strip_audit(N, D, K, alpha, dc, range(K))


def test_forward_strip_n1024_and_n8192_sampled_angles():
    for N, K in ((1024, 1800), (8192, 4096)):
        ks = [0, 1, K // 4 - 1, K // 4, K // 2 - 1, K // 2, K // 2 + 1, 3 * K // 4, K - 1, 777 % K]
        fwd_strip_audit(N, N, K, 1.0, 0.5 * (N - 1), ks)
