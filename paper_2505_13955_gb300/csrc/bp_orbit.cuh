// bp_orbit.cuh -- K2 for the standard geometry, using the square image's
// 90-degree symmetry: one detector-coordinate evaluation feeds four updates.
//
// Geometry condition: angle step pi/K with K even (so th_{k+K/2} = th_k +
// pi/2), detector centre c_d = (D-1)/2, and N a multiple of 2*TILE (tiles
// rotate onto tiles).  With U(p, th) = alpha (X cos th + Y sin th) the
// centred coordinate of pixel p = (X, Y) and R the rotation (X, Y) -> (-Y, X)
// (pixel [r][c] -> [c][N-1-r]), for th' = th + pi/2:
//     U1 = U(p, th)  is also U(Rp, th'), and -U1 = U(R^2 p, th) = U(R^3 p, th')
//     U2 = U(p, th') is also U(R^3 p, th), and -U2 = U(Rp, th) = U(R^2 p, th')
// A negated coordinate reads the mirrored row q~[j] = q[D-1-j] at +U (the
// interpolant commutes with the reflection u -> D-1-u).  So a block owns the
// orbit {T, RT, R^2 T, R^3 T} of one tile, loops over the K/2 angle pairs
// (th, th'), and stages, per pair and per window (W1 around U1 of the tile
// centre, W2 around U2), the four rows {th, th', th~, th'~} interleaved at
// each index.  A thread evaluates u1 and u2 for each of its pixels and reads
// all four rows of each window with one load:
//     W1 at u1 -> p@th, Rp@th', R^2p@th (mirror), R^3p@th' (mirror)
//     W2 at u2 -> p@th', R^3p@th, Rp@th (mirror), R^2p@th' (mirror)
//
// Table entries (see bp_tile.cuh for the split FP64/FP32 coordinate):
//   FP32 rows: per row (a_i, d_i), Q = a_i + u' d_i        -> 32 B per index,
//     kept as two 16-byte arrays (rows th, th' | mirrored rows) so that each
//     16-byte load strides like the 16-bit table (no 4-entry bank aliasing)
//   16-bit rows: per row (q'_i, d_i) in the row's 16-bit type, with
//     q'_i = q_i + d_i / 2 the segment midpoint, Q = q'_i + (u' - i) d_i,
//     the product and sum taken by mixed-precision FMA/ADD into FP32
//                                                            -> 16 B per index
// so 16-bit staging moves 4 B per update out of shared memory instead of 8.
// 16-bit rows are staged as q * s_k / S, S = max_k s_k of the slice (no
// overflow in FP16), and S is applied once to the final sum.
#pragma once

#include "bp_tile.cuh"

namespace fbp {

struct BpOrbitJob {
    const void *filt;          // this slice's [K][D] rows
    const float *row_scale;    // this slice's [K] scales, or null
    float *out;                // this slice's [N][N]
    unsigned short *out16;     // or, when set, this slice's [N][N] uint16 codes (bp_tile.cuh)
    float hu_a, hu_b;
    const double2 *cs;         // [K] (only k < K/2 is read)
    int K, D, N;
    double alpha, det_center;
    float scale;
    int accumulate;
    int H, W;
    int x0, y0;                // origin of the orbit's representative tile (top-left quadrant)
    int kb, ke;                // angle pairs [kb, ke) of this block (0, K/2 unless split)
    unsigned *status;
};

template <typename T> struct OrbitEntry;
template <> struct OrbitEntry<float> { static constexpr int bytes = 32; };   // 2 arrays x 16 B
template <> struct OrbitEntry<__half> { static constexpr int bytes = 16; };
template <> struct OrbitEntry<__nv_bfloat16> { static constexpr int bytes = 16; };

template <int KT, typename T>
__host__ __device__ constexpr size_t bp_orbit_smem_size(int W)
{
    // [KT] x (float4 coords + uint4 addresses/window starts) + [KT][2][W] entries
    return (size_t)KT * 32 + (size_t)KT * 2 * W * OrbitEntry<T>::bytes;
}

__device__ __forceinline__ float4 lds_f4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint4 lds_u4(uint32_t addr)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}

// 16-bit helpers: pack (lo, hi) rounded to nearest even; fraction to 16 bits;
// acc + lo + fr * hi with the products and sums in FP32.
template <typename T> __device__ __forceinline__ uint32_t pack16(float lo, float hi);
template <> __device__ __forceinline__ uint32_t pack16<__half>(float lo, float hi)
{
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}
template <> __device__ __forceinline__ uint32_t pack16<__nv_bfloat16>(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

template <typename T> __device__ __forceinline__ unsigned short frac16(float x);
template <> __device__ __forceinline__ unsigned short frac16<__half>(float x)
{
    unsigned short h;
    asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}
template <> __device__ __forceinline__ unsigned short frac16<__nv_bfloat16>(float x)
{
    unsigned short h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}

template <typename T> __device__ __forceinline__ void mac16(float &acc, unsigned short fr, uint32_t e);
template <> __device__ __forceinline__ void mac16<__half>(float &acc, unsigned short fr, uint32_t e)
{
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "fma.rn.f32.f16 %0, %1, hi, %0;\n\tadd.rn.f32.f16 %0, lo, %0;\n\t}"
        : "+f"(acc) : "h"(fr), "r"(e));
}
template <> __device__ __forceinline__ void mac16<__nv_bfloat16>(float &acc, unsigned short fr, uint32_t e)
{
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "fma.rn.f32.bf16 %0, %1, hi, %0;\n\tadd.rn.f32.bf16 %0, lo, %0;\n\t}"
        : "+f"(acc) : "h"(fr), "r"(e));
}

// Midpoint and slope of the segment (v0, v1) of a 16-bit row scaled by sc,
// each operation rounded once (no contraction), so that the staged entries
// are the same wherever they are formed (in the block, or by the
// pre-staging pass of bp_staged.cu).
__device__ __forceinline__ void orbit_mid_slope(float v0, float v1, float sc, float &mid, float &slp)
{
    const float x0 = __fmul_rn(v0, sc), x1 = __fmul_rn(v1, sc);
    mid = __fmul_rn(0.5f, __fadd_rn(x0, x1));
    slp = __fsub_rn(x1, x0);
}

// Packed FP32 pairs (two windows' coordinates at once) and packed 16-bit
// interpolation (two rows at once), for the PACKED 16-bit variant.
__device__ __forceinline__ unsigned long long pk2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long p, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long fsub2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// (x, x) rounded to the 16-bit type and packed
template <typename T> __device__ __forceinline__ uint32_t splat16(float x);
template <> __device__ __forceinline__ uint32_t splat16<__half>(float x)
{
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %1;" : "=r"(r) : "f"(x));
    return r;
}
template <> __device__ __forceinline__ uint32_t splat16<__nv_bfloat16>(float x)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %1;" : "=r"(r) : "f"(x));
    return r;
}
// a * b + c on packed pairs of the 16-bit type
template <typename T> __device__ __forceinline__ uint32_t hfma2(uint32_t a, uint32_t b, uint32_t c);
template <> __device__ __forceinline__ uint32_t hfma2<__half>(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
template <> __device__ __forceinline__ uint32_t hfma2<__nv_bfloat16>(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// lo_acc += low half of v, hi_acc += high half, in FP32
template <typename T> __device__ __forceinline__ void add2to32(float &lo_acc, float &hi_acc, uint32_t v);
template <> __device__ __forceinline__ void add2to32<__half>(float &lo_acc, float &hi_acc, uint32_t v)
{
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "add.rn.f32.f16 %0, lo, %0;\n\tadd.rn.f32.f16 %1, hi, %1;\n\t}"
        : "+f"(lo_acc), "+f"(hi_acc) : "r"(v));
}
template <> __device__ __forceinline__ void add2to32<__nv_bfloat16>(float &lo_acc, float &hi_acc, uint32_t v)
{
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "add.rn.f32.bf16 %0, lo, %0;\n\tadd.rn.f32.bf16 %1, hi, %1;\n\t}"
        : "+f"(lo_acc), "+f"(hi_acc) : "r"(v));
}

// One angle pair of an orbit block: accumulate the updates of every pixel
// the thread owns from the pair's two staged windows (cb1, cb2: their shared
// addresses biased for the rounded index, see bp_orbit; tab_b: FP32 rows'
// offset of the mirrored-row array).  The block-staged kernel below and the
// bulk-copy-fed kernel (bp_staged.cu) both run it.
template <int TXT, int TYT, int PX, int PY, typename T, bool CHECKED, bool PACKED>
__device__ __forceinline__ void orbit_pair(float (&acc)[4][PY][PX], const float4 pv, const uint32_t cb1,
                                           const uint32_t cb2, const uint32_t tab_b, const float dxt,
                                           const float dyt, const int H, unsigned *status)
{
    constexpr bool F32 = sizeof(T) == 4;
    if constexpr (PACKED) {
        const unsigned long long Mp = pk2(kRoundMagic, kRoundMagic);
        const unsigned long long nMp = pk2(-kRoundMagic, -kRoundMagic);
        {
            const float c = pv.x, s = pv.y;
            // (u1, u2) of the thread's first pixel, and per-row / per-column steps
            const unsigned long long u0 = pk2(fmaf(dxt, c, fmaf(dyt, s, pv.z)),
                                              fmaf(dxt, -s, fmaf(dyt, c, pv.w)));
            const unsigned long long sx = pk2((float)TXT * c, -(float)TXT * s);
            const unsigned long long sy = pk2((float)TYT * s, (float)TYT * c);
#pragma unroll
            for (int iy = 0; iy < PY; ++iy) {
                const unsigned long long r = iy == 0 ? u0 : ffma2(pk2((float)iy, (float)iy), sy, u0);
#pragma unroll
                for (int ix = 0; ix < PX; ++ix) {
                    const unsigned long long u = ix == 0 ? r : ffma2(pk2((float)ix, (float)ix), sx, r);
                    const unsigned long long t = fadd2(u, Mp);
                    const unsigned long long fr = fsub2(u, fadd2(t, nMp));
                    float t1, t2, f1, f2;
                    upk2(t, t1, t2);
                    upk2(fr, f1, f2);
                    uint32_t tb1 = __float_as_uint(t1), tb2 = __float_as_uint(t2);
                    if (CHECKED) {
                        const int i1 = (int)(tb1 - kRoundMagicBits), i2 = (int)(tb2 - kRoundMagicBits);
                        if (i1 < -H || i1 > H || i2 < -H || i2 > H) {
                            atomicCAS(status, 0u, (unsigned)FAULT_TABLE_INDEX);
                            tb1 = tb2 = kRoundMagicBits;
                        }
                    }
                    const uint4 e1 = lds_u4(cb1 + (tb1 << 4));
                    const uint4 e2 = lds_u4(cb2 + (tb2 << 4));
                    const uint32_t h1 = splat16<T>(f1), h2 = splat16<T>(f2);
                    // W1: th -> p, th' -> Rp, th~ -> R^2 p, th'~ -> R^3 p
                    add2to32<T>(acc[0][iy][ix], acc[1][iy][ix], hfma2<T>(h1, e1.y, e1.x));
                    add2to32<T>(acc[2][iy][ix], acc[3][iy][ix], hfma2<T>(h1, e1.w, e1.z));
                    // W2: th -> R^3 p, th' -> p, th~ -> Rp, th'~ -> R^2 p
                    add2to32<T>(acc[3][iy][ix], acc[0][iy][ix], hfma2<T>(h2, e2.y, e2.x));
                    add2to32<T>(acc[1][iy][ix], acc[2][iy][ix], hfma2<T>(h2, e2.w, e2.z));
                }
            }
        }
    } else {
        {
            const float c = pv.x, s = pv.y;
            const float u10 = fmaf(dxt, c, fmaf(dyt, s, pv.z));
            const float u20 = fmaf(dxt, -s, fmaf(dyt, c, pv.w));
            const float s1x = (float)TXT * c, s1y = (float)TYT * s;
            const float s2x = -(float)TXT * s, s2y = (float)TYT * c;
#pragma unroll
            for (int iy = 0; iy < PY; ++iy) {
                const float r1 = iy == 0 ? u10 : fmaf((float)iy, s1y, u10);
                const float r2 = iy == 0 ? u20 : fmaf((float)iy, s2y, u20);
#pragma unroll
                for (int ix = 0; ix < PX; ++ix) {
#pragma unroll
                    for (int win = 0; win < 2; ++win) {
                        const float u = win == 0 ? (ix == 0 ? r1 : fmaf((float)ix, s1x, r1))
                                                 : (ix == 0 ? r2 : fmaf((float)ix, s2x, r2));
                        const float t = __fadd_rn(u, kRoundMagic);
                        uint32_t tb = __float_as_uint(t);
                        if (CHECKED) {
                            const int i = (int)(tb - kRoundMagicBits);
                            if (i < -H || i > H) {
                                atomicCAS(status, 0u, (unsigned)FAULT_TABLE_INDEX);
                                tb = kRoundMagicBits;
                            }
                        }
                        const uint32_t cb = win == 0 ? cb1 : cb2;
                        // orbit members fed by rows (th, th', th~, th'~)
                        const int m0 = win == 0 ? 0 : 3, m1 = win == 0 ? 1 : 0;
                        const int m2 = win == 0 ? 2 : 1, m3 = win == 0 ? 3 : 2;
                        if constexpr (F32) {
                            const uint32_t e = cb + (tb << 4);
                            const float4 e0 = lds_f4(e), e1 = lds_f4(e + tab_b);
                            acc[m0][iy][ix] += fmaf(u, e0.y, e0.x);
                            acc[m1][iy][ix] += fmaf(u, e0.w, e0.z);
                            acc[m2][iy][ix] += fmaf(u, e1.y, e1.x);
                            acc[m3][iy][ix] += fmaf(u, e1.w, e1.z);
                        } else {
                            const uint4 e = lds_u4(cb + (tb << 4));
                            const float fr = u - (t - kRoundMagic);
                            const unsigned short f16 = frac16<T>(fr);
                            mac16<T>(acc[m0][iy][ix], f16, e.x);
                            mac16<T>(acc[m1][iy][ix], f16, e.y);
                            mac16<T>(acc[m2][iy][ix], f16, e.z);
                            mac16<T>(acc[m3][iy][ix], f16, e.w);
                        }
                    }
                }
            }
        }
    }
}

// The four orbit members' pixels of the thread (its first pixel at column
// c0, row r0 of the representative tile): p -> [r][c], Rp -> [c][N-1-r],
// R^2p -> [N-1-r][N-1-c], R^3p -> [N-1-c][r], each value times `gain`.
template <int TXT, int TYT, int PX, int PY>
__device__ __forceinline__ void orbit_store(const float (&acc)[4][PY][PX], float *out, unsigned short *out16,
                                            float hu_a, float hu_b, int accumulate, int N, int c0, int r0,
                                            float gain)
{
#pragma unroll
    for (int iy = 0; iy < PY; ++iy) {
        const int r = r0 + TYT * iy;
#pragma unroll
        for (int ix = 0; ix < PX; ++ix) {
            const int c = c0 + TXT * ix;
            const size_t o0 = (size_t)r * N + c;
            const size_t o1 = (size_t)c * N + (N - 1 - r);
            const size_t o2 = (size_t)(N - 1 - r) * N + (N - 1 - c);
            const size_t o3 = (size_t)(N - 1 - c) * N + r;
            const size_t os[4] = {o0, o1, o2, o3};
#pragma unroll
            for (int o = 0; o < 4; ++o)
                store_pixel(out, out16, hu_a, hu_b, accumulate, os[o], acc[o][iy][ix] * gain);
        }
    }
}

// PACKED (16-bit rows only): entries hold (q'_th, q'_th'), (d_th, d_th'),
// and the same for the mirrored rows, so one packed FMA interpolates two
// rows (the interpolated value is rounded once to the 16-bit type before the
// FP32 accumulation), and both windows' coordinates are formed with packed
// FP32 pair instructions.
//
// SPLIT: the block is one of the P blocks of a thread-block cluster that
// share the orbit, each summing the angle pairs [kb, ke) of its part.  The
// partial sums go to each block's shared memory; after a cluster barrier the
// block of rank r adds, for the entries e = r, r + P, ... of every thread,
// the P partial sums in rank order (distributed shared memory reads) and
// stores the pixel; a second cluster barrier keeps every block's shared
// memory alive until the others have read it.  The sum is deterministic and
// does not depend on the number of slices in the launch.
template <int TXT, int TYT, int PX, int PY>
__host__ __device__ constexpr size_t bp_orbit_split_bytes()
{
    return (size_t)4 * PY * PX * TXT * TYT * sizeof(float);
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The cluster's reduction of one orbit's partial sums (SPLIT launches of the
// orbit and staged kernels): every thread's accumulators go to `scratch`
// (this block's shared memory, bp_orbit_split_bytes, free of every other
// use), then the block of rank r adds, for entries r, r + P, ... of every
// thread, the P partial sums in rank order and stores the pixel times `gain`
// (unless `store` is false: a block that has recorded a fault).  Both
// cluster barriers are reached by every thread of every block.
template <int TXT, int TYT, int PX, int PY>
__device__ __forceinline__ void orbit_split_store(const float (&acc)[4][PY][PX], unsigned char *scratch, bool store,
                                                  float *out, unsigned short *out16, float hu_a, float hu_b,
                                                  int accumulate, int N, int c0, int r0, float gain)
{
    constexpr int NT = TXT * TYT, E = 4 * PY * PX;
    const int tid = threadIdx.x;
    float *mine = reinterpret_cast<float *>(scratch); // [E][NT]
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int iy = 0; iy < PY; ++iy)
#pragma unroll
            for (int ix = 0; ix < PX; ++ix) mine[((o * PY + iy) * PX + ix) * NT + tid] = acc[o][iy][ix];
    cluster_sync_all();
    uint32_t rank, parts;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(parts));
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(mine) + 4u * (uint32_t)tid;
    for (int e = (int)rank; e < E; e += (int)parts) {
        float v = 0.f;
        for (uint32_t p = 0; p < parts; ++p) {
            uint32_t ra;
            float x;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(base + 4u * (uint32_t)(e * NT)), "r"(p));
            asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(x) : "r"(ra) : "memory");
            v += x;
        }
        // entry e = (o, iy, ix): the member's pixel, as orbit_store places it
        const int ix = e % PX, iy = (e / PX) % PY, o = e / (PX * PY);
        const int r = r0 + TYT * iy, c = c0 + TXT * ix;
        const size_t idx = o == 0 ? (size_t)r * N + c
                         : o == 1 ? (size_t)c * N + (N - 1 - r)
                         : o == 2 ? (size_t)(N - 1 - r) * N + (N - 1 - c)
                                  : (size_t)(N - 1 - c) * N + r;
        if (store) store_pixel(out, out16, hu_a, hu_b, accumulate, idx, v * gain);
    }
    cluster_sync_all();
}

template <int TILE, int TXT, int TYT, int PX, int PY, int KT, typename T, bool CHECKED,
          bool PACKED = false, bool SPLIT = false>
__device__ __forceinline__ void bp_orbit(const BpOrbitJob &j, unsigned char *smem)
{
    constexpr int NT = TXT * TYT;
    constexpr int WX = TXT / 8;
    constexpr bool F32 = sizeof(T) == 4;
    static_assert(!(PACKED && F32), "packed interpolation is for 16-bit rows");
    constexpr int EB = 16;                                          // index stride of each array
    static_assert(TXT * PX == TILE && TYT * PY == TILE, "square tile");
    static_assert(TXT % 8 == 0 && TYT % 4 == 0 && (TXT / 8) * (TYT / 4) * 32 == NT, "warp layout");

    float4 *prm = reinterpret_cast<float4 *>(smem);                 // cos, sin, f1, f2
    uint4 *adr = reinterpret_cast<uint4 *>(smem + KT * 16);         // cb1, cb2, jlo1, jlo2
    unsigned char *tab = smem + KT * 32;
    const uint32_t tab_s = (uint32_t)__cvta_generic_to_shared(tab);
    const uint32_t tab_b = (uint32_t)(KT * 2 * j.W * EB);          // FP32: offset of the mirrored-row array

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tx = (warp % WX) * 8 + (lane & 7);
    const int ty = (warp / WX) * 4 + (lane >> 3);
    const int N = j.N, D = j.D, K = j.K, K2 = j.K / 2;
    const double m = 0.5 * (N - 1);
    const double Xc = (double)j.x0 + 0.5 * (TILE - 1) - m;
    const double Yc = (double)j.y0 + 0.5 * (TILE - 1) - m;
    const float dxt = (float)tx - 0.5f * (TILE - 1);
    const float dyt = (float)ty - 0.5f * (TILE - 1);
    const T *q = static_cast<const T *>(j.filt);
    const int H = j.H, W = j.W;

    // 16-bit rows: slice-wide scale S = max_k s_k
    float S = 1.f;
    if constexpr (!F32) {
        __shared__ float s_red[NT / 32];
        float mx = 0.f;
        for (int k = tid; k < K; k += NT) mx = fmaxf(mx, __ldg(j.row_scale + k));
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_red[warp] = mx;
        __syncthreads();
        mx = 0.f;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) mx = fmaxf(mx, s_red[w]);
        S = mx > 0.f ? mx : 1.f;
    }
    const float invS = __frcp_rn(S);

    float acc[4][PY][PX];
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int iy = 0; iy < PY; ++iy)
#pragma unroll
            for (int ix = 0; ix < PX; ++ix) acc[o][iy][ix] = 0.f;

    for (int k0 = j.kb; k0 < j.ke; k0 += KT) {
        const int na = min(KT, j.ke - k0);
        __syncthreads();
        if (tid < KT) {
            float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
            int jl1 = 0, jl2 = 0;
            if (tid < na) {
                const double2 cs = j.cs[k0 + tid];
                const double c = j.alpha * cs.x, s = j.alpha * cs.y;
                const double v1 = fma(c, Xc, fma(s, Yc, j.det_center));
                const double v2 = fma(-s, Xc, fma(c, Yc, j.det_center));
                const double jc1 = floor(v1), jc2 = floor(v2);
                pv.x = (float)c;
                pv.y = (float)s;
                pv.z = (float)(v1 - jc1 - 0.5);
                pv.w = (float)(v2 - jc2 - 0.5);
                jl1 = (int)jc1 - H;
                jl2 = (int)jc2 - H;
            }
            const uint32_t cb1 = tab_s + (uint32_t)EB * (uint32_t)((2 * tid) * W + H) - (uint32_t)EB * kRoundMagicBits;
            const uint32_t cb2 = tab_s + (uint32_t)EB * (uint32_t)((2 * tid + 1) * W + H) - (uint32_t)EB * kRoundMagicBits;
            prm[tid] = pv;
            adr[tid] = make_uint4(cb1, cb2, (uint32_t)jl1, (uint32_t)jl2);
        }
        __syncthreads();
        // stage both windows of every pair: rows th, th', mirrored th, mirrored th'
        for (int aw = warp; aw < 2 * KT; aw += NT / 32) {
            const int a = aw >> 1, win = aw & 1;
            const bool valid = a < na;
            const uint4 ad = adr[a];
            const int jl = (int)(win ? ad.w : ad.z);
            const int k = k0 + (valid ? a : 0);
            const T *r0 = q + (size_t)k * D;
            const T *r1 = q + (size_t)(k + K2) * D;
            float sc0 = 1.f, sc1 = 1.f;
            if constexpr (!F32) {
                sc0 = valid ? __fmul_rn(__ldg(j.row_scale + k), invS) : 0.f;
                sc1 = valid ? __fmul_rn(__ldg(j.row_scale + k + K2), invS) : 0.f;
            }
            unsigned char *dst = tab + (size_t)aw * W * EB;
            for (int i = lane; i < W; i += 32) {
                const int jj = jl + i;               // direct bins jj, jj+1
                const int mj = D - 1 - jj;           // mirrored: q~[jj] = q[mj], q~[jj+1] = q[mj-1]
                float v[8];
                v[0] = (valid && (unsigned)jj < (unsigned)D) ? load_q<T>(r0 + jj) : 0.f;
                v[1] = (valid && (unsigned)(jj + 1) < (unsigned)D) ? load_q<T>(r0 + jj + 1) : 0.f;
                v[2] = (valid && (unsigned)jj < (unsigned)D) ? load_q<T>(r1 + jj) : 0.f;
                v[3] = (valid && (unsigned)(jj + 1) < (unsigned)D) ? load_q<T>(r1 + jj + 1) : 0.f;
                v[4] = (valid && (unsigned)mj < (unsigned)D) ? load_q<T>(r0 + mj) : 0.f;
                v[5] = (valid && (unsigned)(mj - 1) < (unsigned)D) ? load_q<T>(r0 + mj - 1) : 0.f;
                v[6] = (valid && (unsigned)mj < (unsigned)D) ? load_q<T>(r1 + mj) : 0.f;
                v[7] = (valid && (unsigned)(mj - 1) < (unsigned)D) ? load_q<T>(r1 + mj - 1) : 0.f;
                if constexpr (F32) {
                    const float il = (float)(i - H);
                    float4 e0, e1;
                    float d;
                    d = v[1] - v[0]; e0.x = fmaf(0.5f - il, d, v[0]); e0.y = d;
                    d = v[3] - v[2]; e0.z = fmaf(0.5f - il, d, v[2]); e0.w = d;
                    d = v[5] - v[4]; e1.x = fmaf(0.5f - il, d, v[4]); e1.y = d;
                    d = v[7] - v[6]; e1.z = fmaf(0.5f - il, d, v[6]); e1.w = d;
                    reinterpret_cast<float4 *>(dst)[i] = e0;
                    reinterpret_cast<float4 *>(dst + tab_b)[i] = e1;
                } else {
                    // midpoints and slopes of the four rows (scaled by s_k / S)
                    float mid[4], slp[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) orbit_mid_slope(v[2 * r], v[2 * r + 1], (r & 1) ? sc1 : sc0,
                                                                mid[r], slp[r]);
                    uint4 e;
                    if constexpr (PACKED) {
                        e.x = pack16<T>(mid[0], mid[1]);
                        e.y = pack16<T>(slp[0], slp[1]);
                        e.z = pack16<T>(mid[2], mid[3]);
                        e.w = pack16<T>(slp[2], slp[3]);
                    } else {
                        e.x = pack16<T>(mid[0], slp[0]);
                        e.y = pack16<T>(mid[1], slp[1]);
                        e.z = pack16<T>(mid[2], slp[2]);
                        e.w = pack16<T>(mid[3], slp[3]);
                    }
                    reinterpret_cast<uint4 *>(dst)[i] = e;
                }
            }
        }
        __syncthreads();
        for (int a = 0; a < na; ++a) {
            const uint4 ad = adr[a];
            orbit_pair<TXT, TYT, PX, PY, T, CHECKED, PACKED>(acc, prm[a], ad.x, ad.y, tab_b, dxt, dyt, H,
                                                               j.status);
        }
    }

    if constexpr (!SPLIT) {
        orbit_store<TXT, TYT, PX, PY>(acc, j.out, j.out16, j.hu_a, j.hu_b, j.accumulate, N, j.x0 + tx,
                                      j.y0 + ty, j.scale * S);
    } else {
        __syncthreads();                               // the staging buffers are free
        orbit_split_store<TXT, TYT, PX, PY>(acc, smem, true, j.out, j.out16, j.hu_a, j.hu_b, j.accumulate, N,
                                            j.x0 + tx, j.y0 + ty, j.scale * S);
    }
}

}  // namespace fbp
