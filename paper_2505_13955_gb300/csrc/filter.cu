// filter.cu -- K1: the ramp-filter step of FBP (Sec. V-A(c) stage 2,
// "filtering", after Kak & Slaney ch. 3), as an FFT convolution in shared
// memory.
//
// Each projection row p (length D) is linearly convolved with the truncated
// kernel h (|n| <= D-1):  q[j] = tau * sum_m h[j-m] p[m], j in [0, D).
// The kernel transforms the row's first differences d[m] = p[m] - p[m-1]
// (m in [0, D], p = 0 outside) with the cumulative kernel
// g[n] = sum_{k<=n} h[k]; by summation by parts this is the same linear
// convolution, but the FP32 transform's rounding error then scales with |d|
// rather than |p| -- line integrals are large and the ramp filter removes
// most of their magnitude, so at N = 8192 this is ~600x more accurate.
// With L >= 2D a circular convolution of length L gives the same values on
// [0, D).  g is real, so two rows a, b are packed as one complex sequence
// z = a + i b; IFFT(FFT(z) G) = (a*g) + i (b*g) returns both filtered rows at
// once, with no real-FFT packing.
//
// The length-L transform is split four-step as L = N1 * 512 with
// n = n1 + N1 * n2 and k = k2 + 512 * k1:
//   step 1  each warp n1 takes the 512 samples x[n1 + N1 n2]; a lane holds
//           16 of them in registers (n2 = 16 l + r).  The 32-point DFT over
//           the lane index l runs as radix-2 butterflies over warp shuffles,
//           the 16-point DFT over r in registers; then the four-step twiddle
//           W_L^{n1 k2}.  One shared-memory transpose follows.
//   step 2  lanes of the group hold the N1 values of one k2; the N1-point
//           DFT runs over shuffles again, the product with G is taken in
//           registers, and the inverse N1-point DFT undoes it in place.
//   step 3  the inverse of step 1 returns the row in natural order.
// Shared memory holds one padded complex row per row pair; both access
// patterns (stride 16*N1 and the transpose) are padded to avoid bank
// conflicts.  Global loads and stores are coalesced and, where alignment
// allows, 16-byte vectors.
//
// The spectrum G already contains tau and 1/L; FP32 throughout, with the
// spectrum and twiddles rounded once from FP64 tables.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "bp_batch.cuh"
#include "fbp_internal.cuh"

namespace fbp {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 shfl_xor2(float2 v, int m)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// W16^m = exp(-2 pi i m / 16), m in [0, 8): (cos, -sin)
__device__ __forceinline__ float2 w16(int m)
{
    const float c1 = 0.92387953251128675613f;   // cos(pi/8)
    const float s1 = 0.38268343236508977173f;   // sin(pi/8)
    const float r2 = 0.70710678118654752440f;   // cos(pi/4)
    switch (m & 7) {
        case 0: return make_float2(1.f, 0.f);
        case 1: return make_float2(c1, -s1);
        case 2: return make_float2(r2, -r2);
        case 3: return make_float2(s1, -c1);
        case 4: return make_float2(0.f, -1.f);
        case 5: return make_float2(-s1, -c1);
        case 6: return make_float2(-r2, -r2);
        default: return make_float2(-c1, -s1);
    }
}

// In-register 16-point DFT, natural order in and out (radix-2 DIT after a
// compile-time bit-reversal).  INV = true: exponent sign +1, unnormalised.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16])
{
    // bit reversal of 4-bit indices
    float2 t;
    t = v[1]; v[1] = v[8]; v[8] = t;
    t = v[2]; v[2] = v[4]; v[4] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[5]; v[5] = v[10]; v[10] = t;
    t = v[7]; v[7] = v[14]; v[14] = t;
    t = v[11]; v[11] = v[13]; v[13] = t;
#pragma unroll
    for (int h = 1; h < 16; h <<= 1) {
#pragma unroll
        for (int blk = 0; blk < 16; blk += 2 * h) {
#pragma unroll
            for (int m = 0; m < h; ++m) {
                float2 w = w16(m * (8 / h));        // W_{2h}^m = W16^{m*16/(2h)}
                if (INV) w.y = -w.y;
                float2 b = cmul(v[blk + m + h], w);
                v[blk + m + h] = csub(v[blk + m], b);
                v[blk + m] = cadd(v[blk + m], b);
            }
        }
    }
}

__device__ __forceinline__ int brev5(int x) { return (int)(__brev((unsigned)x) >> 27); }

// Decimation-in-frequency radix-2 DFT over the low `bits` lane bits (forward,
// natural order in, bit-reversed out), on NV values per lane.
template <int NV>
__device__ __forceinline__ void lane_dif(float2 (&v)[NV], int lane, int bits,
                                         const float2 *__restrict__ tw, int L)
{
    for (int b = bits - 1; b >= 0; --b) {
        const int h = 1 << b;
        const bool hi = (lane & h) != 0;
        const float2 w = __ldg(&tw[(lane & (h - 1)) * (L / (2 * h))]);
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float2 o = shfl_xor2(v[i], h);
            v[i] = hi ? cmul(csub(o, v[i]), w) : cadd(v[i], o);
        }
    }
}

// Inverse of lane_dif: decimation-in-time over the low `bits` lane bits with
// conjugate twiddles (bit-reversed in, natural out), unnormalised.
template <int NV>
__device__ __forceinline__ void lane_dit_inv(float2 (&v)[NV], int lane, int bits,
                                             const float2 *__restrict__ tw, int L)
{
    for (int b = 0; b < bits; ++b) {
        const int h = 1 << b;
        const bool hi = (lane & h) != 0;
        const float2 w = __ldg(&tw[(lane & (h - 1)) * (L / (2 * h))]);
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float2 o = shfl_xor2(v[i], h);
            // low lane: mine + other * conj(w); high lane: other - mine * conj(w)
            v[i] = hi ? csub(o, cmulc(v[i], w)) : cadd(v[i], cmulc(o, w));
        }
    }
}

struct RowPairJob {
    const float *a;       // first row (length D)
    const float *b;       // second row or nullptr
    void *qa, *qb;        // outputs (dtype), qb may be nullptr
    float *sa, *sb;       // row scales (16-bit dtypes) or nullptr
};

template <typename T>
__device__ __forceinline__ T cvt_out(float x);
template <> __device__ __forceinline__ float cvt_out<float>(float x) { return x; }
template <> __device__ __forceinline__ __half cvt_out<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// Store one filtered row (real or imaginary part of the group's buffer);
// 16-bit types store RNE(q / scale).
template <typename T, bool IMAG>
__device__ __forceinline__ void store_row(T *__restrict__ out, const float2 *S, int D, int padsh,
                                          float scale, bool zero, int tid, int nthr)
{
    const uintptr_t align = sizeof(T) == 4 ? 15 : 7;
    const bool vec = ((D & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & align) == 0);
    if (vec) {
        for (int c = tid; c < (D >> 2); c += nthr) {
            const int n = c << 2;
            const float2 *s0 = S + n + (n >> padsh);
            float x[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = zero ? 0.f : (IMAG ? s0[i].y : s0[i].x);
            if constexpr (sizeof(T) == 4) {
                reinterpret_cast<float4 *>(out)[c] = make_float4(x[0], x[1], x[2], x[3]);
            } else {
                T y[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) y[i] = cvt_out<T>(__fdiv_rn(x[i], scale));
                reinterpret_cast<uint2 *>(out)[c] = *reinterpret_cast<uint2 *>(y);
            }
        }
    } else {
        for (int n = tid; n < D; n += nthr) {
            const float2 v = S[n + (n >> padsh)];
            const float x = zero ? 0.f : (IMAG ? v.y : v.x);
            if constexpr (sizeof(T) == 4) out[n] = x;
            else out[n] = cvt_out<T>(__fdiv_rn(x, scale));
        }
    }
}

// The full row-pair transform for one group of N1 warps.  S points at the
// group's shared buffer of (L + 32) float2.  All threads of the block call
// this together (block-wide barriers inside).
template <int NW, typename T>
__device__ void filter_group(const RowPairJob &job, bool active, int D, int L, int N1, int logN1,
                             const float2 *__restrict__ Gs, const float2 *__restrict__ tw,
                             float2 *S, float *red, int gw, int lane)
{
    const int gtid = gw * 32 + lane;          // thread index inside the group
    const int gthr = N1 * 32;
    const int padsh = 4 + logN1;              // one pad slot per 16*N1 samples
    const int P = 512 + (N1 >= 16 ? 1 : 16 / N1);   // transposed row pitch

    // ---- load: z[n] = (a[n], b[n]) for n < D, 0 beyond; layout A.  Whether
    // a and b have any nonzero sample is kept so that an all-zero input row can be
    // written as exact zeros (the paired transform would otherwise leave
    // rounding cross-talk from its partner row in it).
    float in_a = 0.f, in_b = 0.f;
    if (active) {
        const bool vec = ((D & 3) == 0) &&
                         ((reinterpret_cast<uintptr_t>(job.a) & 15) == 0) &&
                         (!job.b || (reinterpret_cast<uintptr_t>(job.b) & 15) == 0);
        for (int c = gtid; c < (L >> 2); c += gthr) {
            const int n = c << 2;
            float av[4], bv[4];      // first differences p[m] - p[m-1], m = n..n+3 (m <= D)
            float ra[4], rb[4];      // raw samples p[m] (0 for m >= D), for the zero-row flags
            if (vec && n + 3 < D) {
                const float4 x = __ldg(reinterpret_cast<const float4 *>(job.a) + c);
                const float xm = n > 0 ? __ldg(job.a + n - 1) : 0.f;
                ra[0] = x.x; ra[1] = x.y; ra[2] = x.z; ra[3] = x.w;
                av[0] = x.x - xm; av[1] = x.y - x.x; av[2] = x.z - x.y; av[3] = x.w - x.z;
                if (job.b) {
                    const float4 y = __ldg(reinterpret_cast<const float4 *>(job.b) + c);
                    const float ym = n > 0 ? __ldg(job.b + n - 1) : 0.f;
                    rb[0] = y.x; rb[1] = y.y; rb[2] = y.z; rb[3] = y.w;
                    bv[0] = y.x - ym; bv[1] = y.y - y.x; bv[2] = y.z - y.y; bv[3] = y.w - y.z;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) rb[i] = bv[i] = 0.f;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int m = n + i;
                    ra[i] = (m < D) ? __ldg(job.a + m) : 0.f;
                    rb[i] = (job.b && m < D) ? __ldg(job.b + m) : 0.f;
                    const float pa = (m >= 1 && m - 1 < D) ? __ldg(job.a + m - 1) : 0.f;
                    const float pb = (job.b && m >= 1 && m - 1 < D) ? __ldg(job.b + m - 1) : 0.f;
                    av[i] = (m <= D) ? ra[i] - pa : 0.f;
                    bv[i] = (m <= D) ? rb[i] - pb : 0.f;
                }
            }
            float2 *d = S + n + (n >> padsh);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                d[i] = make_float2(av[i], bv[i]);
                if (ra[i] != 0.f) in_a = 1.f;   // NaN counts as nonzero
                if (rb[i] != 0.f) in_b = 1.f;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        in_a = fmaxf(in_a, __shfl_xor_sync(0xffffffffu, in_a, o));
        in_b = fmaxf(in_b, __shfl_xor_sync(0xffffffffu, in_b, o));
    }
    if (lane == 0) { red[2 * N1 + 2 * gw] = in_a; red[2 * N1 + 2 * gw + 1] = in_b; }
    __syncthreads();
    bool zero_a = true, zero_b = true;
    for (int w = 0; w < N1; ++w) {
        zero_a = zero_a && !(red[2 * N1 + 2 * w] > 0.f);
        zero_b = zero_b && !(red[2 * N1 + 2 * w + 1] > 0.f);
    }

    float2 v[16];
    const int p = brev5(lane);
    // ---- step 1 (forward): warp n1 = gw
    if (active) {
        const int n1 = gw;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int n = n1 + N1 * (16 * lane + r);
            v[r] = S[n + (n >> padsh)];
        }
        lane_dif<16>(v, lane, 5, tw, L);                      // DFT over l -> p (bit-reversed)
#pragma unroll
        for (int r = 1; r < 16; ++r)                          // W512^{r p}
            v[r] = cmul(v[r], __ldg(&tw[(r * p * N1) & (L - 1)]));
        dft16<false>(v);                                      // DFT over r -> q
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int k2 = p + 32 * q;
            if (n1) v[q] = cmul(v[q], __ldg(&tw[(n1 * k2) & (L - 1)]));   // W_L^{n1 k2}
        }
    }
    __syncthreads();   // every warp has read layout A before it is overwritten
    if (active) {
        const int n1 = gw;
#pragma unroll
        for (int q = 0; q < 16; ++q) S[n1 * P + p + 32 * q] = v[q];
    }
    __syncthreads();

    // ---- step 2: N1-point DFT over lanes, times G, inverse
    if (active) {
        const int n1 = lane & (N1 - 1);
        const int sg = lane >> logN1;
        const int grp = gw * (32 >> logN1) + sg;              // k2 group, 0..31
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = S[n1 * P + 32 * r + grp];
        if (logN1) lane_dif<16>(v, lane, logN1, tw, L);
        const int k1 = logN1 ? (int)(__brev((unsigned)n1) >> (32 - logN1)) : 0;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], __ldg(&Gs[32 * r + grp + 512 * k1]));
        if (logN1) {
            lane_dit_inv<16>(v, lane, logN1, tw, L);
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (n1) v[r] = cmulc(v[r], __ldg(&tw[(n1 * (32 * r + grp)) & (L - 1)]));
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) S[n1 * P + 32 * r + grp] = v[r];
    }
    __syncthreads();

    // ---- step 3 (inverse of step 1)
    if (active) {
        const int n1 = gw;
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = S[n1 * P + p + 32 * q];
        dft16<true>(v);                                       // q -> r
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = cmulc(v[r], __ldg(&tw[(r * p * N1) & (L - 1)]));
        lane_dit_inv<16>(v, lane, 5, tw, L);                  // p -> l
    }
    __syncthreads();
    if (active) {
        const int n1 = gw;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int n = n1 + N1 * (16 * lane + r);
            S[n + (n >> padsh)] = v[r];
        }
    }
    __syncthreads();

    // ---- store (16-bit: per-row amax scale first)
    float scale_a = 1.f, scale_b = 1.f;
    if (sizeof(T) != 4) {
        float ma = 0.f, mb = 0.f;
        if (active)
            for (int n = gtid; n < D; n += gthr) {
                float2 z = S[n + (n >> padsh)];
                ma = fmaxf(ma, fabsf(z.x));
                mb = fmaxf(mb, fabsf(z.y));
            }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
            mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        }
        if (lane == 0) { red[2 * gw] = ma; red[2 * gw + 1] = mb; }
        __syncthreads();
        if (active) {
            ma = 0.f; mb = 0.f;
            for (int w = 0; w < N1; ++w) { ma = fmaxf(ma, red[2 * w]); mb = fmaxf(mb, red[2 * w + 1]); }
            scale_a = (ma > 0.f && !zero_a) ? ma : 1.f;
            scale_b = (mb > 0.f && !zero_b) ? mb : 1.f;
            if (gtid == 0) {
                job.sa[0] = scale_a;
                if (job.sb) job.sb[0] = scale_b;
            }
        }
    }
    if (active) {
        store_row<T, false>(static_cast<T *>(job.qa), S, D, padsh, scale_a, zero_a, gtid, gthr);
        if (job.qb) store_row<T, true>(static_cast<T *>(job.qb), S, D, padsh, scale_b, zero_b, gtid, gthr);
    }
}

struct FilterArgs {
    const float *sino;
    void *filt;
    float *row_scale;
    long long rows;
    int D, L, N1, logN1;
    const float2 *G;
    const float2 *tw;
};

template <int NW, typename T>
__global__ void __launch_bounds__(NW * 32) filter_kernel(FilterArgs a)
{
    extern __shared__ float2 smem_f2[];
    __shared__ float red[4 * NW];   // per-warp maxima: output amax, input amax (both rows)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = NW / a.N1;                       // row pairs per block
    const int g = warp / a.N1, gw = warp % a.N1;
    const long long pair = (long long)blockIdx.x * G + g;
    const bool active = 2 * pair < a.rows;
    RowPairJob job;
    const long long ra = 2 * pair, rb = 2 * pair + 1;
    const size_t esz = sizeof(T);
    job.a = active ? a.sino + ra * a.D : nullptr;
    job.b = (active && rb < a.rows) ? a.sino + rb * a.D : nullptr;
    job.qa = active ? static_cast<char *>(a.filt) + ra * a.D * esz : nullptr;
    job.qb = (active && rb < a.rows) ? static_cast<char *>(a.filt) + rb * a.D * esz : nullptr;
    job.sa = (active && a.row_scale) ? a.row_scale + ra : nullptr;
    job.sb = (active && rb < a.rows && a.row_scale) ? a.row_scale + rb : nullptr;
    float2 *S = smem_f2 + (size_t)g * (a.L + 32);
    filter_group<NW, T>(job, active, a.D, a.L, a.N1, a.logN1, a.G, a.tw, S, red + 4 * g * a.N1,
                        gw, lane);
}

template <int NW, typename T>
fbp_status launch_nw(const FilterArgs &fa, cudaStream_t s)
{
    const int G = NW / fa.N1;
    const long long pairs = (fa.rows + 1) / 2;
    const long long blocks = (pairs + G - 1) / G;
    const size_t smem = (size_t)G * (fa.L + 32) * sizeof(float2);
    auto kern = filter_kernel<NW, T>;
    fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (st != FBP_OK) return st;
    if (blocks > 0x7fffffffLL) return fail(FBP_ERR_UNSUPPORTED, "too many rows");
    kern<<<(unsigned)blocks, NW * 32, smem, s>>>(fa);
    FBP_CUDA_TRY(cudaGetLastError());
    return FBP_OK;
}

template <typename T>
fbp_status launch_t(const FilterArgs &fa, cudaStream_t s)
{
    if (fa.N1 <= 8) return launch_nw<8, T>(fa, s);
    if (fa.N1 == 16) return launch_nw<16, T>(fa, s);
    return launch_nw<32, T>(fa, s);
}

// Ragged batch: one launch over every item's rows.  32 warps per block; an
// item with transform length L = 512 N1 puts 32/N1 row pairs in a block, so
// the shared buffer is the same size for every item.
template <typename T>
__global__ void __launch_bounds__(1024) filter_batched_kernel(FilterBatchArgs a)
{
    extern __shared__ float2 smem_f2[];
    __shared__ float red[4 * 32];
    int lo = 0, hi = a.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.items[mid].group_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const FilterBatchItem &it = a.items[lo];
    const int N1 = it.L / 512;
    int logN1 = 0;
    while ((1 << logN1) < N1) ++logN1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = 32 / N1;
    const int g = warp / N1, gw = warp % N1;
    const long long pair = (long long)(blockIdx.x - it.group_begin) * G + g;
    const long long rows = it.K;
    const bool active = 2 * pair < rows;
    const long long ra = 2 * pair, rb = 2 * pair + 1;
    RowPairJob job;
    job.a = active ? it.sino + ra * it.D : nullptr;
    job.b = (active && rb < rows) ? it.sino + rb * it.D : nullptr;
    job.qa = active ? static_cast<char *>(it.filt) + ra * it.D * sizeof(T) : nullptr;
    job.qb = (active && rb < rows) ? static_cast<char *>(it.filt) + rb * it.D * sizeof(T) : nullptr;
    job.sa = (active && it.row_scale) ? it.row_scale + ra : nullptr;
    job.sb = (active && rb < rows && it.row_scale) ? it.row_scale + rb : nullptr;
    float2 *S = smem_f2 + (size_t)g * (it.L + 32);
    filter_group<32, T>(job, active, it.D, it.L, N1, logN1, it.G, it.tw, S, red + 4 * g * N1, gw, lane);
}

template <typename T>
fbp_status launch_batched_t(const FilterBatchArgs &a, int groups, cudaStream_t s)
{
    // worst case over L: (32/N1) * (512 N1 + 32) float2
    const size_t smem = (size_t)(16384 + 1024) * sizeof(float2);
    auto kern = filter_batched_kernel<T>;
    fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (st != FBP_OK) return st;
    kern<<<groups, 1024, smem, s>>>(a);
    FBP_CUDA_TRY(cudaGetLastError());
    return FBP_OK;
}

}  // namespace

fbp_status launch_filter(const FilterLaunch &a, cudaStream_t s)
{
    if (a.rows <= 0) return FBP_OK;
    FilterArgs fa;
    fa.sino = a.sino;
    fa.filt = a.filt;
    fa.row_scale = a.row_scale;
    fa.rows = a.rows;
    fa.D = a.D;
    fa.L = a.L;
    fa.N1 = a.L / 512;
    fa.logN1 = 0;
    while ((1 << fa.logN1) < fa.N1) ++fa.logN1;
    fa.G = a.G;
    fa.tw = a.tw;
    if (fa.N1 < 1 || fa.N1 > 32 || (1 << fa.logN1) != fa.N1)
        return fail(FBP_ERR_UNSUPPORTED, "filter length %d", a.L);
    switch (a.dtype) {
        case FBP_F32: return launch_t<float>(fa, s);
        case FBP_F16: return launch_t<__half>(fa, s);
        case FBP_BF16: return launch_t<__nv_bfloat16>(fa, s);
    }
    return fail(FBP_ERR_INVALID_ARG, "dtype");
}

fbp_status launch_filter_batched(const FilterBatchArgs &a, int total_groups, fbp_dtype dtype,
                                 cudaStream_t s)
{
    if (total_groups <= 0) return FBP_OK;
    switch (dtype) {
        case FBP_F32: return launch_batched_t<float>(a, total_groups, s);
        case FBP_F16: return launch_batched_t<__half>(a, total_groups, s);
        case FBP_BF16: return launch_batched_t<__nv_bfloat16>(a, total_groups, s);
    }
    return fail(FBP_ERR_INVALID_ARG, "dtype");
}

}  // namespace fbp
