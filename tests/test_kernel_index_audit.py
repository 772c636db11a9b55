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
