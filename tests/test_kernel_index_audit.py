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


# ---------------------------------------------------------------------------
# Filter (filter.cu): transform shapes, buffer indices, and a replay of the
# three-step factorisation and of the in-register radix-2 DFT
# ---------------------------------------------------------------------------
FFT_SHAPES = {512: (4, 4), 1024: (8, 4), 2048: (8, 8), 4096: (16, 8), 8192: (16, 16), 16384: (32, 16)}


def group_threads(L):
    return 128 if L in (512, 1024) else 256 if L in (2048, 4096) else 512


@pytest.mark.parametrize("L", sorted(FFT_SHAPES))
def test_filter_shapes_and_indices(L):
    R, VPL = FFT_SHAPES[L]
    C = 32 * VPL
    assert C == group_threads(L) and R * C == L and 512 % C == 0
    NWG = C // 32
    assert R % NWG == 0                               # whole rows per warp in step 2
    t, k1 = np.meshgrid(np.arange(C), np.arange(R))
    assert (k1 * C + t).max() == L - 1                # buffer S[k1][t]
    assert (t * k1).max() < L                         # W_L^{t k1} index
    lane, kr = np.meshgrid(np.arange(32), np.arange(VPL))
    assert (lane * kr * R).max() < L                  # W_C^{l kr} index
    kl = np.arange(32)
    k = k1[:, :1, None] + R * (np.arange(VPL)[None, :, None] + VPL * kl[None, None, :])
    assert sorted(k.ravel().tolist()) == list(range(L))   # G index covers the spectrum once
    # batched kernel: (512 / C) pairs x L float2 grows with L, so the longest
    # item's size bounds every block; 4 reduction floats per warp
    sizes = [(512 // group_threads(x)) * x for x in sorted(FFT_SHAPES)]
    assert sizes == sorted(sizes)
    assert (512 // C) * 4 * NWG == 64


def brev_bits(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def step2_shape(L):
    """Step 2's pass-B shape: RB = min(R, 16) values per lane, NRD = R / RB
    rounds, SL = 32 / RB lanes per 32-point transform."""
    R, VPL = FFT_SHAPES[L]
    RB = min(R, 16)
    return R, VPL, RB, R // RB, 32 // RB


def swz_key(R, c):
    # restates filter_impl.cuh:swz_key
    return c if R >= 16 else c * (16 // R)


def g_entry_k(L, o):
    """runtime.cu:diff_spectrum_kernel's order: spectrum index k of entry o."""
    R, VPL, RB, NRD, SL = step2_shape(L)
    j, m, rd, w = o & 31, (o >> 5) % RB, (o // (32 * RB)) % NRD, o // (32 * R)
    c, s = rd * RB + j % RB, j // RB
    k1, kr = w * (R // VPL) + c // VPL, c % VPL
    q = brev_bits(s, SL.bit_length() - 1)
    return k1 + R * (kr + VPL * (m + RB * q))


@pytest.mark.parametrize("L", sorted(FFT_SHAPES))
def test_filter_table_layouts(L):
    """runtime.cu writes G entry o = ((w NRD + rd) RB + m) 32 + j at
    k = k1 + R (kr + VPL (m + RB brev(s))); every spectrum index once.  The
    twiddle plan has L + C + 32 entries: W_L^{t k1} at k1 C + t, W_C^{l kr}
    at L + 32 kr + l, W_32^m at L + C + m."""
    R, VPL = FFT_SHAPES[L]
    C = 32 * VPL
    k = [g_entry_k(L, o) for o in range(L)]
    assert sorted(k) == list(range(L))
    # twiddle plan: the kernel's reads stay in their sections
    t, kk = np.meshgrid(np.arange(C), np.arange(R))
    assert (kk * C + t).max() < L
    lane, r = np.meshgrid(np.arange(32), np.arange(VPL))
    assert (L + 32 * r + lane).min() >= L and (L + 32 * r + lane).max() < L + C
    for h in (1, 2, 4, 8, 16):
        idx = (np.arange(32) & (h - 1)) * (16 // h)
        assert idx.max() < 32 and np.array_equal(idx * 2 * h // 32, np.arange(32) & (h - 1))


@pytest.mark.parametrize("L", sorted(FFT_SHAPES))
def test_filter_step2_exchange_is_conflict_free(L):
    """The swizzled exchange inside step 2: each 32-entry run (row, kr) is
    a permutation (pass A writes), pass B's reads cover every entry of the
    warp's rows once, and each half-warp's 8-byte accesses fall in 16
    different bank pairs, for pass A and for every read of pass B."""
    R, VPL, RB, NRD, SL = step2_shape(L)
    C, RPW = 32 * VPL, R // VPL
    lane = np.arange(32)
    seen = np.zeros(RPW * C, int)
    for rr in range(RPW):
        for kr in range(VPL):
            e = rr * C + 32 * kr + (lane ^ swz_key(R, rr * VPL + kr))
            assert sorted((e - rr * C - 32 * kr).tolist()) == list(range(32))
            for half in (lane[:16], lane[16:]):
                assert len(set((e[half] % 16).tolist())) == 16
    for rd in range(NRD):
        c = rd * RB + (lane & (RB - 1))
        s = lane // RB
        key = np.array([swz_key(R, int(x)) for x in c])
        for i in range(RB):
            e = (c // VPL) * C + 32 * (c % VPL) + ((s + SL * i) ^ key)
            seen[e] += 1
            for half in (slice(0, 16), slice(16, 32)):
                assert len(set((e[half] % 16).tolist())) == 16
    assert (seen == 1).all()


def dft_reg_replay(v, inv):
    """The kernel's in-register DFT: compile-time bit reversal, then radix-2
    DIT with twiddle W_32^j, j = m*16/h at half-size h: none for m = 0, a
    swap for j = 8, else the six-FMA form a +- f (tx + i ty) with the
    larger of |wc|, |ws| factored out."""
    M = len(v)
    bits = M.bit_length() - 1
    v = v.copy()
    rev = [int(format(i, f"0{bits}b")[::-1], 2) if bits else 0 for i in range(M)]
    v = v[rev]
    h = 1
    while h < M:
        for blk in range(0, M, 2 * h):
            for m in range(h):
                a, b = v[blk + m], v[blk + m + h]
                j = m * (16 // h)
                if m == 0 or j == 8:
                    if j == 8:
                        b = complex(-b.imag, b.real) if inv else complex(b.imag, -b.real)
                    v[blk + m + h], v[blk + m] = a - b, a + b
                    continue
                wc, ws = math.cos(2 * math.pi * j / 32), -math.sin(2 * math.pi * j / 32)
                if inv:
                    ws = -ws
                if abs(wc) >= abs(ws):
                    r, f = ws / wc, wc
                    t = complex(b.real - r * b.imag, b.imag + r * b.real)
                else:
                    r, f = wc / ws, ws
                    t = complex(r * b.real - b.imag, r * b.imag + b.real)
                v[blk + m + h], v[blk + m] = a - f * t, a + f * t
        h *= 2
    return v


@pytest.mark.parametrize("M", [4, 8, 16, 32])
def test_filter_register_dft_replay(M):
    rng = np.random.default_rng(M)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    np.testing.assert_allclose(dft_reg_replay(x, False), np.fft.fft(x), atol=1e-12)
    np.testing.assert_allclose(dft_reg_replay(x, True), np.fft.ifft(x) * M, atol=1e-12)


def lane_dif_replay(x, s, R, w):
    """filter_impl.cuh:lane_dif_s on all 32 lanes at once: x[lane] holds one
    value; radix-2 DIF over s = lane / R (natural in, bit-reversed out)."""
    SL = 32 // R
    h = SL // 2
    while h >= 1:
        o = x[np.arange(32) ^ (R * h)]
        hi = (s & h) != 0
        y = np.where(hi, -x, x) + o
        tw = np.where(hi, w((s & (h - 1)) * (16 // h)), 1.0) if h > 1 else 1.0
        x = y * tw
        h //= 2
    return x


def lane_dit_inv_replay(x, s, R, w):
    SL = 32 // R
    h = 1
    while h < SL:
        hi = (s & h) != 0
        tw = np.where(hi, np.conj(w((s & (h - 1)) * (16 // h))), 1.0) if h > 1 else 1.0
        y = x * tw
        o = y[np.arange(32) ^ (R * h)]
        x = np.where(hi, -y, y) + o
        h *= 2
    return x


@pytest.mark.parametrize("L", sorted(FFT_SHAPES))
def test_filter_three_step_factorisation_replay(L):
    """Step 1 (R-point DFT over n1, W_L^{t k1}); step 2 per warp as the
    kernel runs it: pass A (VPL-point over r, W_C^{l kr}, swizzled writes),
    pass B per round (swizzled reads l = s + SL i, RB-point over i,
    W_32^{s m}, the lane transform over s, times G in the table's order, and
    the inverses), pass C; step 3 (W_L^{-t k1}, inverse R-point): equals the
    circular convolution IFFT(FFT(z) G) * L."""
    R, VPL, RB, NRD, SL = step2_shape(L)
    C, RPW = 32 * VPL, R // VPL
    rng = np.random.default_rng(L)
    z = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    Gk = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    Gt = np.array([Gk[g_entry_k(L, o)] for o in range(L)])      # the table as stored
    W = lambda m: np.exp(-2j * np.pi * m / L)
    w32 = lambda m: np.exp(-2j * np.pi * (np.asarray(m) & 31) / 32)
    tk = np.outer(np.arange(R), np.arange(C))
    S = (np.fft.fft(z.reshape(R, C), axis=0) * W(tk)).reshape(-1)
    lane = np.arange(32)
    for gw in range(VPL):                        # NWG = VPL warps per group
        for rr in range(RPW):                    # pass A
            k1 = gw * RPW + rr
            u = np.fft.fft(S[k1 * C + lane[None, :] + 32 * np.arange(VPL)[:, None]], axis=0)
            u = u * np.exp(-2j * np.pi * np.outer(np.arange(VPL), lane) / C)
            for kr in range(VPL):
                S[k1 * C + 32 * kr + (lane ^ swz_key(R, rr * VPL + kr))] = u[kr]
        for rd in range(NRD):                    # pass B
            c = rd * RB + (lane & (RB - 1))
            s = lane // RB
            base = (gw * RPW + c // VPL) * C + 32 * (c % VPL)
            key = np.array([swz_key(R, int(x)) for x in c])
            idx = base[None, :] + ((s[None, :] + SL * np.arange(RB)[:, None]) ^ key[None, :])
            x = np.fft.fft(S[idx], axis=0)                        # i -> m
            x = x * w32(s[None, :] * np.arange(RB)[:, None])
            x = np.array([lane_dif_replay(x[m], s, RB, w32) for m in range(RB)])
            g = Gt[((gw * NRD + rd) * RB + np.arange(RB))[:, None] * 32 + lane[None, :]]
            x = x * g
            x = np.array([lane_dit_inv_replay(x[m], s, RB, w32) for m in range(RB)])
            x = x * np.conj(w32(s[None, :] * np.arange(RB)[:, None]))
            S[idx] = np.fft.ifft(x, axis=0) * RB                  # m -> i
        for rr in range(RPW):                    # pass C
            k1 = gw * RPW + rr
            u = np.array([S[k1 * C + 32 * kr + (lane ^ swz_key(R, rr * VPL + kr))] for kr in range(VPL)])
            u = u * np.exp(2j * np.pi * np.outer(np.arange(VPL), lane) / C)
            S[k1 * C + lane[None, :] + 32 * np.arange(VPL)[:, None]] = np.fft.ifft(u, axis=0) * VPL
    out = (np.fft.ifft(S.reshape(R, C) * np.conj(W(tk)), axis=0) * R).reshape(-1)
    ref = np.fft.ifft(np.fft.fft(z) * Gk) * L
    np.testing.assert_allclose(out, ref, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("alpha", [0.125, 0.5, 0.7, 1.0, 2.5])
def test_forward_candidate_count_bound(alpha):
    # candidates per line: ceil(2 / g), g = alpha * max(|cos|, |sin|) >= alpha / sqrt(2)
    th = np.linspace(0, np.pi, 10001)
    g = alpha * np.maximum(np.abs(np.cos(th)), np.abs(np.sin(th)))
    nc = np.ceil(2.0 / g)
    bound = math.ceil(2.0 * 1.4142135623730951 / alpha)
    assert nc.max() <= bound
    assert bound <= 24


ORBIT_SHAPES = [(16, 8, 2, 4), (16, 16, 4, 4), (8, 8, 2, 2)]   # (TXT, TYT, PX, PY), square tiles


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


# ---------------------------------------------------------------------------
# Forward projector, tile-owned form (forward.cu, fwd_tile_kernel): a replay
# of its fixed-point walk, checked for int32 range, padded-tile indices and
# coverage (the replayed projection equals the oracle's).
# ---------------------------------------------------------------------------
FT, FPAD, FBIAS, FFRAC = 64, 3, 4, 23


def fwd_tile_replay(img, K, D, alpha, det_center, bpw):
    """Returns (projection [K][D], min P, max P, max padded index) of the
    kernel's arithmetic on image img (N x N)."""
    N = img.shape[0]
    LS = 32 // bpw
    m = 0.5 * (N - 1)
    tiles_x = -(-N // FT)
    th = np.arange(K) * (math.pi / K)
    out = np.zeros((K, D))
    pmin, pmax, imax = 0, 0, 0
    two32 = 4294967296.0
    pad = np.zeros((FT + 2 * FPAD, FT + 2 * FPAD))
    for ty in range(tiles_x):
        for tx in range(tiles_x):
            r0, c0 = ty * FT, tx * FT
            pad[:] = 0.0
            blk = img[r0:r0 + FT, c0:c0 + FT]
            pad[FPAD:FPAD + blk.shape[0], FPAD:FPAD + blk.shape[1]] = blk
            for k in range(K):
                cs, sn = math.cos(th[k]), math.sin(th[k])
                ax, ay = alpha * cs, alpha * sn
                ua = ax * (c0 - m) + ay * (r0 - m) + det_center
                dx, dy = ax * (FT - 1), ay * (FT - 1)
                umin = ua + min(0.0, dx) + min(0.0, dy)
                umax = ua + max(0.0, dx) + max(0.0, dy)
                jbase = math.floor(umin)
                W = math.floor(umax) + 2 - jbase
                rows = abs(cs) >= abs(sn)
                cp, cq = (ax, ay) if rows else (ay, ax)
                s0, l0 = (c0, r0) if rows else (r0, c0)
                P0 = (jbase - det_center - cq * (l0 - m)) / cp - s0 + m - 1.0 / abs(cp)
                BJ, SL = 1.0 / cp, cq / cp
                P0i = int(np.rint((P0 + FBIAS) * two32))
                BJi = int(np.rint(BJ * two32))
                SLi = int(np.rint(SL * two32))
                g = np.float32(abs(cp))
                p0f, bjf, slf = np.float32(P0), np.float32(BJ), np.float32(SL)
                dP = (LS * SLi + (1 << (31 - FFRAC))) >> (32 - FFRAC)
                for q in range(-(-W // bpw)):
                    bA, bB = q * bpw, min(q * bpw + bpw - 1, W - 1)
                    PA = np.float32(np.float32(bA) * bjf + p0f)
                    PB = np.float32(np.float32(bB) * bjf + p0f)
                    Pl, Ph = np.float32(min(PA, PB) - 0.01), np.float32(max(PA, PB) + 0.01)
                    lo_f, hi_f = 0.0, float(FT - 1)
                    if slf > 0:
                        hi_f = min(hi_f, float(np.float32((Ph + 3) / slf)))
                        lo_f = max(lo_f, float(np.float32((Pl - (FT - 1)) / slf)))
                    elif slf < 0:
                        lo_f = max(lo_f, float(np.float32((Ph + 3) / slf)))
                        hi_f = min(hi_f, float(np.float32((Pl - (FT - 1)) / slf)))
                    elif not (Ph >= -3 and Pl < FT - 1):
                        hi_f = -1.0
                    lo = max(0, math.floor(min(lo_f, FT)) - 1)
                    hi = min(FT - 1, math.floor(max(hi_f, -1.0)) + 1)
                    for bl in range(bpw):
                        b = bA + bl
                        Pb = P0i + b * BJi
                        acc = 0.0
                        for lsub in range(LS):
                            l = lo + lsub
                            if l > hi:
                                continue
                            P = (Pb - l * SLi) >> (32 - FFRAC)
                            while l <= hi:
                                pmin, pmax = min(pmin, P), max(pmax, P)
                                st = P >> FFRAC
                                c = st if 0 <= st <= FT + FPAD else FT + FPAD
                                imax = max(imax, c + 2)
                                F = 1.0 + (P & 0x7FFFFF) / 8388608.0
                                e = float(g) * (2.0 - F)
                                w = (e, 1.0 - abs(e + float(g) - 1.0), max(0.0, 2.0 - 2.0 * float(g) - e))
                                for i in range(3):
                                    v = pad[l + FPAD, c + i] if rows else pad[c + i, l + FPAD]
                                    acc += w[i] * v
                                P -= dP
                                l += LS
                        j = jbase + b
                        if b < W and 0 <= j < D:
                            out[k, j] += acc
    return out, pmin, pmax, imax


@pytest.mark.parametrize("bpw", [8, 32])
@pytest.mark.parametrize("N,D,K,alpha", [(64, 64, 12, 1.0), (100, 110, 10, 0.95), (130, 128, 8, 1.0)])
def test_forward_tile_replay_matches_oracle(bpw, N, D, K, alpha):
    import oracle
    rng = np.random.default_rng(N + K)
    img = rng.standard_normal((N, N))
    dc = 0.5 * (D - 1)
    out, pmin, pmax, imax = fwd_tile_replay(img, K, D, alpha, dc, bpw)
    assert -(1 << 31) <= pmin and pmax < (1 << 31)
    assert -256 * (1 << FFRAC) < pmin and pmax < 256 * (1 << FFRAC)   # 9.23 with the bias
    assert imax <= FT + 2 * FPAD - 1
    g = oracle.Geometry(K, D, N, pixel_size=alpha)
    ref = oracle.forward(img, g)
    assert np.max(np.abs(out - ref)) <= 1e-5 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# Fused pre-processing (filter.cu, blur_diff): the first difference of the
# blurred, truncated row as one (2r+2)-tap filter plus the two end cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("sigma", [0.0, 0.6, 1.0, 2.5, 3.875])
@pytest.mark.parametrize("D", [1, 2, 7, 64, 301])
def test_blur_difference_replay(sigma, D):
    import oracle
    rng = np.random.default_rng(D)
    p = rng.standard_normal(D)
    w = oracle.gaussian_taps(sigma)
    r = (len(w) - 1) // 2
    assert r <= 16                                   # kMaxBlurRadius = kPrePad
    c = np.append(w, 0.0) - np.insert(w, 0, 0.0)     # c_m = w_m - w_{m-1}, m in [-r, r+1]
    pad = np.zeros(D + 32)
    pad[16:16 + D] = p

    def blur_at(n):
        return sum(w[k + r] * pad[16 + n - k] for k in range(-r, r + 1))

    d = np.zeros(D + 1)
    for n in range(D + 1):
        if n == 0:
            d[n] = blur_at(0)
        elif n == D:
            d[n] = -blur_at(D - 1)
        else:
            d[n] = sum(c[m + r] * pad[16 + n - m] for m in range(-r, r + 2))
    pb = oracle.gaussian_blur(p, sigma)
    ref = np.diff(np.concatenate([[0.0], pb, [0.0]]))
    np.testing.assert_allclose(d, ref, atol=1e-12)


@pytest.mark.parametrize("NS,threads,blocks", [(1, 256, 4), (2, 256, 4), (4, 384, 2)])
def test_forward_tile_shared_memory_allows_its_blocks_per_sm(NS, threads, blocks):
    """fwd_tile_kernel's dynamic shared memory -- the padded 70 x 71 tile of
    NS-slice vectors plus one 64-byte walk record per thread -- fits one
    block (227 KB) and the blocks per SM its launch bounds ask for (228 KB
    per SM, 1 KB reserved per block)."""
    side, pitch = 70, 71
    tile = (side * pitch * 4 * NS + 63) // 64 * 64
    smem = tile + threads * 64
    assert smem <= 227 * 1024
    assert blocks * (smem + 1024) <= 228 * 1024
    assert threads % 32 == 0


# Staged backprojection (bp_staged.cu): the shapes of kStagedShapes32 and
# kStagedShapes16 as (TXT, TYT, PX, PY, KT, NS, blocks per SM), and the
# shared-memory layout of bp_staged_kernel restated from its offsets.
STAGED_F32 = [(16, 8, 2, 4, 4, 2, 6), (16, 8, 2, 4, 4, 3, 5), (16, 8, 2, 4, 8, 2, 3), (16, 16, 4, 4, 8, 2, 2)]
# (shapes 2 and 3 of the 16-bit list are compiled with registers for four
# blocks per SM, but their stage buffers allow two and three: None, no
# occupancy is stated for them)
STAGED_16 = [(16, 16, 4, 4, 8, 3, 2), (16, 16, 4, 4, 16, 2, 2), (16, 8, 2, 4, 16, 3, None),
             (16, 8, 2, 4, 8, 4, None), (16, 8, 2, 4, 8, 3, 5), (16, 8, 2, 4, 8, 2, 6)]


def staged_smem_bytes(KT, NS, halves, Wp):
    params = (NS * KT * 16 + 127) // 128 * 128
    return 128 + 128 + params + NS * halves * 2 * KT * Wp * 16


@pytest.mark.parametrize("halves,shape", [(2, s) for s in STAGED_F32] + [(1, s) for s in STAGED_16])
@pytest.mark.parametrize("alpha", [0.125, 0.9, 1.0, 2.5])
@pytest.mark.parametrize("raw_offset", [0, 16, 48, 112])
def test_staged_shared_layout_fits_and_aligns(halves, shape, alpha, raw_offset):
    """Every address the staged kernel forms -- mbarriers, counters, pair
    parameters, and each bulk-copy destination of every window of every
    stage buffer -- lies inside the dynamic allocation the host requests
    (whatever 16-byte-aligned offset the allocation starts at), every copy
    destination is 128-byte aligned, every box is at most 256 entries, and
    the shapes with a stated occupancy fit that many blocks in the SM's
    shared memory when the window is the orbit's at unit pixel/bin ratio."""
    TXT, TYT, PX, PY, KT, NS, minb = shape
    tile = TXT * PX
    H = window_half(alpha, tile, tile)
    W = 2 * H + 1
    if W > 256:
        pytest.skip("refused on the host: window wider than one bulk copy")
    Wp = (W + 7) // 8 * 8
    size = staged_smem_bytes(KT, NS, halves, Wp)
    raw = 1 << 20 | raw_offset                         # shared address of the dynamic buffer
    base = (raw + 127) & ~127
    end = raw + size
    assert base + 8 * NS <= base + 12 * NS <= base + 16 * NS <= base + 128      # mbarriers, done, issued
    assert base + 128 + NS * KT * 16 <= base + 128 + (NS * KT * 16 + 127) // 128 * 128
    tab0 = base + 128 + (NS * KT * 16 + 127) // 128 * 128
    half_bytes = 2 * KT * Wp * 16
    stage_bytes = halves * half_bytes
    for b in range(NS):
        for lane in range(KT):
            for h in range(halves):
                for win in range(2):
                    dst = tab0 + b * stage_bytes + h * half_bytes + 2 * lane * Wp * 16 + win * Wp * 16
                    assert dst % 128 == 0
                    assert raw <= dst and dst + W * 16 <= end
    # the expected transaction bytes of a full stage fit an mbarrier's count
    assert KT * 2 * W * 16 * halves < (1 << 20)
    if alpha == 1.0 and minb is not None:
        assert minb * (size + 1024) <= 228 * 1024, f"{minb} blocks of {size} bytes"


# Staged ragged batches (bp_staged_batch.cu): every window copy of every
# orbit unit stays inside its item's padded table, for the ragged workload's
# sizes and for pixel/bin ratios and detector widths that push the corner
# windows far past the detector; FP32 rows run 32 x 32 tiles (4 pairs per
# stage, two 16-byte halves, six blocks per SM), 16-bit rows 64 x 64 tiles
# (16 pairs per stage, two blocks per SM).
BATCH_GEOMS = [(True, 720, 512, 512, 1.0), (True, 1800, 1024, 1024, 1.0), (True, 3600, 4096, 4096, 1.0),
               (True, 100, 80, 128, 1.3), (True, 72, 200, 128, 0.7), (True, 36, 33, 64, 1.45),
               (True, 180, 256, 192, 1.0), (True, 360, 700, 1024, 1.5), (True, 64, 2, 256, 0.05),
               (False, 720, 512, 512, 1.0), (False, 3600, 4096, 4096, 1.0), (False, 100, 80, 256, 1.05),
               (False, 72, 200, 128, 0.7), (False, 36, 40, 128, 1.08), (False, 180, 300, 256, 1.0),
               (False, 64, 2, 256, 0.05)]


@pytest.mark.parametrize("f32,K,D,N,alpha", BATCH_GEOMS)
def test_staged_batch_windows_inside_padded_tables(f32, K, D, N, alpha):
    """The first entry e of each window (floor(v) - H + 1 + P_lo, with v the
    tile centre's detector coordinate formed in FP64 as the kernel forms it)
    satisfies 0 <= e <= Ep - W for both windows of every angle pair and every
    orbit base tile; the copies' sources and sizes are 16-byte multiples and
    the stage buffers hold the window pitch at the occupancy the launch
    asks for."""
    from batch_layout import staged_item_geom
    geom = staged_item_geom(K, D, N, alpha, f32=f32)
    assert geom is not None
    H, W, Wp, P_lo, Ep = geom
    T = 32 if f32 else 64
    c_d = 0.5 * (D - 1)
    m = 0.5 * (N - 1)
    t = np.arange(0, N // 2, T, dtype=np.float64) + 0.5 * (T - 1) - m     # base tile centres (one axis)
    Xc, Yc = np.meshgrid(t, t)
    Xc, Yc = Xc.ravel(), Yc.ravel()
    th = np.arange(K // 2) * (np.pi / K)
    worst_lo, worst_hi = 1 << 30, -(1 << 30)
    for k in range(K // 2):
        c, s = alpha * np.cos(th[k]), alpha * np.sin(th[k])
        v1 = c * Xc + (s * Yc + c_d)
        v2 = -s * Xc + (c * Yc + c_d)
        for v in (v1, v2):
            e = np.floor(v).astype(np.int64) - H + 1 + P_lo
            worst_lo = min(worst_lo, int(e.min()))
            worst_hi = max(worst_hi, int(e.max()))
    assert worst_lo >= 0 and worst_hi <= Ep - W, (worst_lo, worst_hi, Ep - W)
    # at least one entry of margin on the side the geometry reaches
    assert worst_lo >= 1 or worst_hi <= Ep - W - 1
    # every real segment [-1, D-1] is in the padded row
    assert P_lo + D + 1 <= Ep
    # copies: W entries of 16 bytes from 16-byte entries; shared layout
    assert Wp % 8 == 0 and W <= Wp <= (72 if f32 else 104)
    KT, halves, blocks = (4, 2, 6) if f32 else (16, 1, 2)
    size = staged_smem_bytes(KT, 2, halves, Wp)
    assert KT * 2 * W * 16 * halves < (1 << 20)
    if f32 and alpha > 1.0:
        blocks = 5
    assert blocks * (size + 1024) <= 228 * 1024, (blocks, size)
