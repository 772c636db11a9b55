// bp_staged.cuh -- device code shared by the staged backprojection
// kernels (bp_staged.cu: one geometry per launch, windows moved by
// bulk-tensor copies; bp_staged_batch.cu: ragged batches, windows moved by
// plain bulk copies from padded tables): the table entries, the FP32
// per-pair arithmetic, the capped mbarrier wait and the shared-memory layout.
#pragma once

#include "bp_orbit.cuh"

namespace fbp {

constexpr long long kStagedWaitCap = 1LL << 22;   // polls of one wait (well under a second)

// The 16-byte entry of angle pair (r0 = row th, r1 = row th + pi/2) for
// detector segment jj (bins jj, jj + 1; the mirrored rows read bins D-1-jj,
// D-2-jj; bins outside [0, D) read as zero): midpoints and slopes of the
// four rows scaled by sc0 (rows of th) and sc1 (rows of th + pi/2), rounded
// to T, in the orbit kernel's packing.
template <typename T, bool PACKED>
__device__ __forceinline__ uint4 orbit_entry16(const T *r0, const T *r1, int D, int jj, float sc0, float sc1)
{
    const int mj = D - 1 - jj;
    float v[8];
    v[0] = (unsigned)jj < (unsigned)D ? load_q<T>(r0 + jj) : 0.f;
    v[1] = (unsigned)(jj + 1) < (unsigned)D ? load_q<T>(r0 + jj + 1) : 0.f;
    v[2] = (unsigned)jj < (unsigned)D ? load_q<T>(r1 + jj) : 0.f;
    v[3] = (unsigned)(jj + 1) < (unsigned)D ? load_q<T>(r1 + jj + 1) : 0.f;
    v[4] = (unsigned)mj < (unsigned)D ? load_q<T>(r0 + mj) : 0.f;
    v[5] = (unsigned)(mj - 1) < (unsigned)D ? load_q<T>(r0 + mj - 1) : 0.f;
    v[6] = (unsigned)mj < (unsigned)D ? load_q<T>(r1 + mj) : 0.f;
    v[7] = (unsigned)(mj - 1) < (unsigned)D ? load_q<T>(r1 + mj - 1) : 0.f;
    float mid[4], slp[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) orbit_mid_slope(v[2 * r], v[2 * r + 1], (r & 1) ? sc1 : sc0, mid[r], slp[r]);
    uint4 out;
    if constexpr (PACKED) {
        out.x = pack16<T>(mid[0], mid[1]);
        out.y = pack16<T>(slp[0], slp[1]);
        out.z = pack16<T>(mid[2], mid[3]);
        out.w = pack16<T>(slp[2], slp[3]);
    } else {
        out.x = pack16<T>(mid[0], slp[0]);
        out.y = pack16<T>(mid[1], slp[1]);
        out.z = pack16<T>(mid[2], slp[2]);
        out.w = pack16<T>(mid[3], slp[3]);
    }
    return out;
}

// FP32 rows: per segment and row the midpoint (q_j + q_{j+1}) / 2 and the
// slope q_{j+1} - q_j, so that Q(u) = mid + (u' - i) slope; 32 bytes per
// entry as two 16-byte halves, a = (rows th, th + pi/2), b = (mirrored rows).
__device__ __forceinline__ void orbit_entry32(const float *r0, const float *r1, int D, int jj, float4 &a, float4 &b)
{
    const int mj = D - 1 - jj;
    float v[8];
    v[0] = (unsigned)jj < (unsigned)D ? __ldg(r0 + jj) : 0.f;
    v[1] = (unsigned)(jj + 1) < (unsigned)D ? __ldg(r0 + jj + 1) : 0.f;
    v[2] = (unsigned)jj < (unsigned)D ? __ldg(r1 + jj) : 0.f;
    v[3] = (unsigned)(jj + 1) < (unsigned)D ? __ldg(r1 + jj + 1) : 0.f;
    v[4] = (unsigned)mj < (unsigned)D ? __ldg(r0 + mj) : 0.f;
    v[5] = (unsigned)(mj - 1) < (unsigned)D ? __ldg(r0 + mj - 1) : 0.f;
    v[6] = (unsigned)mj < (unsigned)D ? __ldg(r1 + mj) : 0.f;
    v[7] = (unsigned)(mj - 1) < (unsigned)D ? __ldg(r1 + mj - 1) : 0.f;
    float ms[8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        ms[2 * r] = __fmul_rn(0.5f, __fadd_rn(v[2 * r], v[2 * r + 1]));
        ms[2 * r + 1] = __fsub_rn(v[2 * r + 1], v[2 * r]);
    }
    a = make_float4(ms[0], ms[1], ms[2], ms[3]);
    b = make_float4(ms[4], ms[5], ms[6], ms[7]);
}

// One angle pair from FP32 midpoint/slope entries (the FP32 form of
// orbit_pair): per pixel and window the rounded index i and the fraction
// u' - i, two 16-byte loads (rows th, th' at cb, mirrored rows at cb + tab_b),
// four FMAs.
template <int TXT, int TYT, int PX, int PY>
__device__ __forceinline__ void orbit_pair_mid(float (&acc)[4][PY][PX], const float4 pv, const uint32_t cb1,
                                               const uint32_t cb2, const uint32_t tab_b, const float dxt,
                                               const float dyt)
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
                const float fr = __fsub_rn(u, __fsub_rn(t, kRoundMagic));
                const uint32_t e = (win == 0 ? cb1 : cb2) + (__float_as_uint(t) << 4);
                const float4 e0 = lds_f4(e), e1 = lds_f4(e + tab_b);
                // orbit members fed by rows (th, th', th~, th'~), as orbit_pair
                const int m0 = win == 0 ? 0 : 3, m1 = win == 0 ? 1 : 0;
                const int m2 = win == 0 ? 2 : 1, m3 = win == 0 ? 3 : 2;
                acc[m0][iy][ix] += fmaf(fr, e0.y, e0.x);
                acc[m1][iy][ix] += fmaf(fr, e0.w, e0.z);
                acc[m2][iy][ix] += fmaf(fr, e1.y, e1.x);
                acc[m3][iy][ix] += fmaf(fr, e1.w, e1.z);
            }
        }
    }
}

__device__ __forceinline__ bool staged_wait(uint32_t mbar, unsigned parity)
{
    for (long long it = 0; it < kStagedWaitCap; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}


// Shared memory: [0, 128) NS mbarriers, NS "warps done" and NS "times
// issued" counters; [128, 128 + P) the per-stage pair parameters (float4 per
// pair, P rounded to 128 bytes); then NS stage tables of 2 KT windows of Wp
// entries (16 bytes each; Wp a multiple of 8, so every window starts on a
// 128-byte boundary).  The dynamic buffer is rounded up to 128 bytes first.
template <int KT, int NS>
__host__ __device__ constexpr size_t staged_params_bytes()
{
    return ((size_t)NS * KT * 16 + 127) / 128 * 128;
}
// HALVES: 16-byte halves per entry (1 for 16-bit rows, 2 for FP32 rows).
template <int KT, int NS, int HALVES>
__host__ __device__ constexpr size_t staged_smem_bytes(int Wp)
{
    return 128 + 128 + staged_params_bytes<KT, NS>() + (size_t)NS * HALVES * 2 * KT * Wp * 16;
}

}  // namespace fbp
