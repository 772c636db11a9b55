// bp_tile.cuh -- K2: pixel-driven backprojection of one output tile over all
// angles (the O(N_p N_x N_y) step of Sec. V-A(c) stage 2), shared by the
// uniform launch and the persistent ragged-batch launch.
//
// For pixel (r, c) and angle k the detector coordinate is
//   u = alpha (X cos th_k + Y sin th_k) + c_d,  X = c - (N-1)/2, Y = r - (N-1)/2,
// and the pixel gains Q_k(u), the linear interpolation of the filtered row
// (zero outside [0, D)).  At N = 8192 |u| reaches ~5800, where float has
// only ~5e-4 of resolution, so the coordinate is split:
//   * per (tile, angle), in FP64: u_c at the tile centre, j_c = floor(u_c),
//     f_c = u_c - j_c - 1/2 (kept as float);
//   * per pixel, in FP32: u' = f_c + alpha (dx cos + dy sin), with (dx, dy)
//     the pixel's small offset from the tile centre, so |u'| < ~50.
// Then i = rne(u') (one FADD of 1.5*2^23; the index is read from the float's
// bits) picks the segment between bins j_c+i and j_c+i+1, on which
//   Q(u) = a_i + u' d_i,  d_i = q[j_c+i+1] - q[j_c+i],  a_i = q[j_c+i] + (1/2 - i) d_i.
// The block stages (a_i, d_i) for i in [-H, H] and every angle of an angle
// tile in shared memory, so each (pixel, angle) update is
//   FFMA (u') + FADD (index) + integer add (address) + 8-byte LDS + FFMA + FADD.
// Rounding to the nearest index instead of flooring needs no care at ties:
// both neighbouring segments give the same value there (the interpolant is
// continuous).
//
// Thread layout: a warp covers an 8 x 4 block of pixels, so the 32 lanes of
// one LDS touch at most ~10 distinct table entries (broadcast, no bank
// conflicts); each thread owns PX x PY pixels strided by the thread grid.
#pragma once

#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "fbp_internal.cuh"

namespace fbp {

constexpr float kRoundMagic = 12582912.0f;        // 1.5 * 2^23
constexpr unsigned kRoundMagicBits = 0x4B400000u;

template <typename T> __device__ __forceinline__ float load_q(const T *p);
template <> __device__ __forceinline__ float load_q<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_q<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <> __device__ __forceinline__ float load_q<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}

__device__ __forceinline__ float2 lds_f2(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

// One tile of one slice.
struct BpTileJob {
    const void *filt;          // this slice's [K][D] rows (dtype T)
    const float *row_scale;    // this slice's [K] scales, or null
    float *out;                // this slice's [N][N]
    unsigned short *out16;     // or, when set, this slice's [N][N] uint16 CT-number codes
    float hu_a, hu_b;          // code = clamp(rint(RN(RN(hu_a * mu) + hu_b)), 0, 65535)
    const double2 *cs;         // [K] cos, sin (FP64)
    int K, D, N;
    double alpha, det_center;
    float scale;
    int accumulate;
    int H, W;                  // staged window: indices [-H, H], W = 2H + 1
    int x0, y0;                // tile origin (pixels)
    unsigned *status;
};

// Output of one pixel: the attenuation (written or added), or its stage-4
// code (Sec. V-A(c): HU window quantised to uint16), taken in FP32 as two
// single roundings, rounded to nearest even and clamped to [0, 65535].
__device__ __forceinline__ void store_pixel(float *out, unsigned short *out16, float hu_a, float hu_b,
                                            int accumulate, size_t idx, float v)
{
    if (out16) {
        const float t = rintf(__fadd_rn(__fmul_rn(hu_a, v), hu_b));
        out16[idx] = (unsigned short)fminf(fmaxf(t, 0.f), 65535.f);
    } else {
        float *o = out + idx;
        *o = accumulate ? *o + v : v;
    }
}

// Shared memory: [KT] float4 per-angle parameters, [KT] int window starts,
// [KT][W] float2 (a, d) table.
template <int KT>
__host__ __device__ constexpr size_t bp_smem_size(int W)
{
    return (size_t)KT * (sizeof(float4) + sizeof(int)) + (size_t)KT * W * sizeof(float2);
}

template <int TXT, int TYT, int PX, int PY, int KT, typename T, bool CHECKED>
__device__ __forceinline__ void bp_tile(const BpTileJob &j, unsigned char *smem)
{
    constexpr int NT = TXT * TYT;
    constexpr int TW = TXT * PX, TH = TYT * PY;
    constexpr int WX = TXT / 8;                          // warps along x
    static_assert(TXT % 8 == 0 && TYT % 4 == 0, "warp covers 8 x 4 pixels");
    static_assert((TXT / 8) * (TYT / 4) * 32 == NT, "thread grid");

    float4 *prm = reinterpret_cast<float4 *>(smem);
    int *jlo = reinterpret_cast<int *>(smem + KT * sizeof(float4));
    float2 *tab = reinterpret_cast<float2 *>(smem + KT * (sizeof(float4) + sizeof(int)));
    const uint32_t tab_s = (uint32_t)__cvta_generic_to_shared(tab);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tx = (warp % WX) * 8 + (lane & 7);
    const int ty = (warp / WX) * 4 + (lane >> 3);
    const double Xc = (double)j.x0 + 0.5 * (TW - 1) - 0.5 * (j.N - 1);
    const double Yc = (double)j.y0 + 0.5 * (TH - 1) - 0.5 * (j.N - 1);
    const float dxt = (float)tx - 0.5f * (TW - 1);
    const float dyt = (float)ty - 0.5f * (TH - 1);
    const T *q = static_cast<const T *>(j.filt);
    const int H = j.H, W = j.W;

    float acc[PY][PX];
#pragma unroll
    for (int iy = 0; iy < PY; ++iy)
#pragma unroll
        for (int ix = 0; ix < PX; ++ix) acc[iy][ix] = 0.f;

    for (int k0 = 0; k0 < j.K; k0 += KT) {
        const int na = min(KT, j.K - k0);
        __syncthreads();                                  // previous tile's table fully used
        if (tid < KT) {
            // per-angle parameters in FP64
            float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
            int jl = 0;
            if (tid < na) {
                const double2 cs = j.cs[k0 + tid];
                const double c = j.alpha * cs.x, s = j.alpha * cs.y;
                const double uc = fma(c, Xc, fma(s, Yc, j.det_center));
                const double jc = floor(uc);
                pv.x = (float)c;
                pv.y = (float)s;
                pv.z = (float)(uc - jc - 0.5);
                jl = (int)jc - H;
            }
            const uint32_t cb = tab_s + 8u * (uint32_t)(tid * W + H) - 8u * kRoundMagicBits;
            pv.w = __uint_as_float(cb);
            prm[tid] = pv;
            jlo[tid] = jl;
        }
        __syncthreads();
        // stage (a, d) for every angle of the tile, zero outside the detector
        for (int a = warp; a < KT; a += NT / 32) {
            const bool valid = a < na;
            const int jl = jlo[a];
            const T *row = q + (size_t)(k0 + (valid ? a : 0)) * j.D;
            const float sc = (valid && j.row_scale) ? __ldg(j.row_scale + k0 + a) : 1.f;
            for (int i = lane; i < W; i += 32) {
                const int jj = jl + i;
                float q0 = 0.f, q1 = 0.f;
                if (valid && (unsigned)jj < (unsigned)j.D) q0 = load_q<T>(row + jj) * sc;
                if (valid && (unsigned)(jj + 1) < (unsigned)j.D) q1 = load_q<T>(row + jj + 1) * sc;
                const float d = q1 - q0;
                tab[a * W + i] = make_float2(fmaf(0.5f - (float)(i - H), d, q0), d);
            }
        }
        __syncthreads();
        // accumulate
        for (int a = 0; a < na; ++a) {
            const float4 pv = prm[a];
            const uint32_t cb = __float_as_uint(pv.w);
            const float u0 = fmaf(dxt, pv.x, fmaf(dyt, pv.y, pv.z));
            const float stx = (float)TXT * pv.x, sty = (float)TYT * pv.y;
#pragma unroll
            for (int iy = 0; iy < PY; ++iy) {
                const float ur = iy == 0 ? u0 : fmaf((float)iy, sty, u0);
#pragma unroll
                for (int ix = 0; ix < PX; ++ix) {
                    const float u = ix == 0 ? ur : fmaf((float)ix, stx, ur);
                    const float t = __fadd_rn(u, kRoundMagic);
                    uint32_t tb = __float_as_uint(t);
                    if (CHECKED) {
                        const int i = (int)(tb - kRoundMagicBits);
                        if (i < -H || i > H) {
                            atomicCAS(j.status, 0u, (unsigned)FAULT_TABLE_INDEX);
                            tb = kRoundMagicBits;
                        }
                    }
                    const float2 ad = lds_f2(cb + (tb << 3));
                    acc[iy][ix] += fmaf(u, ad.y, ad.x);
                }
            }
        }
    }

    // store (every pixel of the N x N square that this tile covers)
#pragma unroll
    for (int iy = 0; iy < PY; ++iy) {
        const int r = j.y0 + ty + TYT * iy;
#pragma unroll
        for (int ix = 0; ix < PX; ++ix) {
            const int c = j.x0 + tx + TXT * ix;
            if (r < j.N && c < j.N)
                store_pixel(j.out, j.out16, j.hu_a, j.hu_b, j.accumulate, (size_t)r * j.N + c,
                            acc[iy][ix] * j.scale);
        }
    }
}

}  // namespace fbp
