// filter_impl.cuh -- K1: the ramp-filter step of FBP (Sec. V-A(c) stage 2,
// "filtering", after Kak & Slaney ch. 3), as an FFT convolution.
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
// The length-L transform is split as L = R * C, C = 32 * VPL, with
// n = C n1 + n2 and k = k1 + R k2 (R, VPL compile-time per L); a group of C
// threads transforms one row pair, thread t owning n2 = t:
//   step 1  thread t loads z[C n1 + t] for every n1 straight from global
//           memory (coalesced across t), forms the differences, runs the
//           R-point DFT over n1 in registers, multiplies by W_L^{t k1} and
//           writes row k1 of an R x C shared buffer.
//   step 2  each warp takes whole rows k1 (R / VPL of them): the C-point
//           DFT over n2 = l + 32 r is a VPL-point DFT over r in registers
//           (lane l), the twiddle W_C^{l kr}, and R VPL = R 32-point DFTs
//           over l, one per (row, kr).  For those the warp exchanges its
//           rows through the shared buffer (swizzled, so neither side has
//           a bank conflict): lane j = c + R s takes l = s + (32/R) i,
//           runs the R-point DFT over i in registers, and finishes with a
//           (32/R)-point DFT over the lanes j, j ^ R, ... (warp shuffles;
//           none at L = 16384, where R = 32).  The product with
//           G[k1 + R k2] is taken in registers and the inverse undoes the
//           forward steps in place, so the spectrum never leaves the warp.
//   step 3  thread t reads column t, multiplies by W_L^{-t k1}, runs the
//           inverse R-point DFT and stores its outputs n = C n1 + t < D
//           straight to global memory (coalesced across t).
// Steps 1 and 3 and the natural-order side of step 2 access the buffer
// row-contiguously, and the exchange inside step 2 is XOR-swizzled within
// 32-entry runs, so no access has a bank conflict and no padding is needed.
//
// The spectrum G already contains tau and 1/L and is stored in step 2's
// read order; the twiddles come from a plan laid out in the order each step
// reads them (fbp_internal.cuh), so every table load is coalesced.  FP32
// throughout, with the spectrum and twiddles rounded once from FP64 tables.
//
// This header holds the kernels; filter.cu dispatches, and the
// translation units filter_{plain,stream,batched}_{f32,f16,bf16}.cu each
// instantiate one kernel family for one output type, so that the long
// transform instantiations compile in parallel.
#pragma once
#include <algorithm>
#include <cstdlib>

#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "bp_batch.cuh"
#include "fbp_internal.cuh"
#include "filter_launch.cuh"

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
// a / b, correctly rounded, from y = RN(1 / b): q = RN(a y) is within an
// ulp of a / b, the residual a - b q is exact in one FMA, and the
// correction RN(q + (a - b q) y) rounds the quotient correctly (Markstein,
// IBM J. Res. Dev. 34(1), 1990).  Holds while the quotient is normal; the
// 16-bit rows divide values by their row's largest magnitude, so the
// quotient lies in [-1, 1].
__device__ __forceinline__ float div_rn(float a, float b, float y)
{
    const float q = a * y;
    return fmaf(fmaf(-q, b, a), y, q);
}

// The same table pointer, opaque to the compiler: loads through it are
// issued where they are used, instead of being merged with an earlier load
// of the same entry or hoisted out of the row-pair loop, either of which
// keeps whole twiddle sets live in registers across the transform.
__device__ __forceinline__ const float2 *fresh(const float2 *p)
{
    const float2 *q;
    asm volatile("mov.b64 %0, %1;" : "=l"(q) : "l"(p));
    return q;
}


// Step 2's 32-point transforms over l run on lanes j = c + R s (c < R,
// s < SL = 32 / R): lane j holds, for one transform c, the R values
// l = s + SL i (i < R).  After the R-point transform over i (-> m) and the
// twiddle W_32^{s m}, an SL-point transform over s across the lanes
// j, j ^ R, j ^ 2R, ... completes it (none when R = 32).
//
// lane_dif_s: that SL-point transform, radix-2 decimation in frequency
// (natural s in, bit-reversed q out).  Written as v' = sgn v + other, then a
// per-lane twiddle (1 on the low lane), so each stage costs two shuffles,
// two FMAs and one complex product per value (none in the last stage).
template <int NV, int R>
__device__ __forceinline__ void lane_dif_s(float2 (&v)[NV], int s, const float2 *__restrict__ w32t)
{
    constexpr int SL = 32 / R;
#pragma unroll
    for (int h = SL / 2; h >= 1; h >>= 1) {
        const bool hi = (s & h) != 0;
        const float sg = hi ? -1.f : 1.f;
        float2 w = make_float2(1.f, 0.f);
        if (h > 1 && hi) w = __ldg(&w32t[(s & (h - 1)) * (16 / h)]);      // W_{2h}^{s mod h}
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const float2 o = shfl_xor2(v[i], R * h);
            float2 x = make_float2(fmaf(sg, v[i].x, o.x), fmaf(sg, v[i].y, o.y));
            if (h > 1) x = cmul(x, w);
            v[i] = x;
        }
    }
}

// Inverse of lane_dif_s: decimation in time over s with conjugate twiddles
// (bit-reversed in, natural out), unnormalised.  The high lane first takes
// its own value times conj(w), then low: own + other, high: other - own.
template <int NV, int R>
__device__ __forceinline__ void lane_dit_inv_s(float2 (&v)[NV], int s, const float2 *__restrict__ w32t)
{
    constexpr int SL = 32 / R;
#pragma unroll
    for (int h = 1; h < SL; h <<= 1) {
        const bool hi = (s & h) != 0;
        const float sg = hi ? -1.f : 1.f;
        float2 w = make_float2(1.f, 0.f);
        if (h > 1 && hi) {
            w = __ldg(&w32t[(s & (h - 1)) * (16 / h)]);
            w.y = -w.y;
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float2 x = v[i];
            if (h > 1) x = cmul(x, w);
            const float2 o = shfl_xor2(x, R * h);
            v[i] = make_float2(fmaf(sg, x.x, o.x), fmaf(sg, x.y, o.y));
        }
    }
}

// XOR key of transform c in the swizzled layout of step 2: row k1, value
// (kr, l) sits at k1 C + 32 kr + (l ^ key(c)), c = (k1 mod RPW) VPL + kr.
// Both accesses are then free of bank conflicts: the lanes l of one kr
// write a permutation of one 32-entry run, and the 16 lanes of a half-warp
// reading (c, l = s + SL i) in one round of pass B hit 16 different 8-byte
// bank pairs (SL = 32 / min(R, 16) lanes per transform).
template <int R>
__host__ __device__ constexpr int swz_key(int c)
{
    return R >= 16 ? c : c * (16 / R);
}

struct RowPairJob {
    const float *a;       // first row (length D; the physical row in offset mode)
    const float *b;       // second row or nullptr
    const float *a2, *b2; // offset mode with fold: the rows half a turn later
    void *qa, *qb;        // outputs (dtype), qb may be nullptr
    float *sa, *sb;       // row scales (16-bit dtypes) or nullptr
};

template <typename T>
__device__ __forceinline__ T cvt_out(float x);
template <> __device__ __forceinline__ __half cvt_out<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }


// cos(pi j / 16), j in [0, 8]
__device__ __forceinline__ float cos16(int j)
{
    switch (j) {
        case 0: return 1.0f;
        case 1: return 0.98078528040323044913f;
        case 2: return 0.92387953251128675613f;
        case 3: return 0.83146961230254523708f;
        case 4: return 0.70710678118654752440f;
        case 5: return 0.55557023301960222474f;
        case 6: return 0.38268343236508977173f;
        case 7: return 0.19509032201612826785f;
        default: return 0.0f;
    }
}
// cos(2 pi m / 32) for any m (folded to a constant when m is)
__device__ __forceinline__ float cos32(int m)
{
    m &= 31;
    if (m <= 8) return cos16(m);
    if (m <= 16) return -cos16(16 - m);
    if (m <= 24) return -cos16(m - 16);
    return cos16(32 - m);
}
// W_32^m = exp(-2 pi i m / 32) = (cos, -sin)
__device__ __forceinline__ float2 w32(int m) { return make_float2(cos32(m), -cos32(m - 8)); }

template <int M>
__host__ __device__ constexpr int brev_c(int i)
{
    int r = 0;
    for (int b = 1; b < M; b <<= 1) {
        r <<= 1;
        if (i & b) r |= 1;
    }
    return r;
}

// In-register M-point DFT (M a power of two <= 32), natural order in and out
// (radix-2 decimation in time after a compile-time bit reversal).
// INV = true: exponent sign +1, unnormalised.
template <int M, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[M])
{
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const int j = brev_c<M>(i);
        if (j > i) {
            const float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int h = 1; h < M; h <<= 1) {
#pragma unroll
        for (int blk = 0; blk < M; blk += 2 * h) {
#pragma unroll
            for (int m = 0; m < h; ++m) {
                const float2 a = v[blk + m];
                float2 b = v[blk + m + h];
                const int j = m * (16 / h);             // W_{2h}^m = W_32^j
                if (m == 0 || j == 8) {
                    if (j == 8)                         // W_32^8 = -i (conjugate: +i): a swap
                        b = INV ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
                    v[blk + m + h] = csub(a, b);
                    v[blk + m] = cadd(a, b);
                } else {
                    // a +- b w with w = wc + i ws in six FMAs: factor out the
                    // larger of |wc|, |ws| (Linzer & Feig, IBM J. Res. Dev.
                    // 37(5), 1993), b w = wc (b.x - r b.y, b.y + r b.x) with
                    // r = ws / wc, or ws (r b.x - b.y, r b.y + b.x) with r = wc / ws
                    const float2 w = w32(j);
                    const float wc = w.x, ws = INV ? -w.y : w.y;
                    float f, tx, ty;
                    if (fabsf(wc) >= fabsf(ws)) {
                        const float r = ws / wc;
                        f = wc;
                        tx = fmaf(-r, b.y, b.x);
                        ty = fmaf(r, b.x, b.y);
                    } else {
                        const float r = wc / ws;
                        f = ws;
                        tx = fmaf(r, b.x, -b.y);
                        ty = fmaf(r, b.y, b.x);
                    }
                    v[blk + m + h] = make_float2(fmaf(-f, tx, a.x), fmaf(-f, ty, a.y));
                    v[blk + m] = make_float2(fmaf(f, tx, a.x), fmaf(f, ty, a.y));
                }
            }
        }
    }
}

__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

constexpr int kFilterThreads = kFilterBlockThreads;   // 512 / C row pairs per block

__host__ __device__ constexpr int group_threads(int L) { return 32 * fft_VPL(L); }

// Stage-2 pre-processing fused into the load (Sec. V-A(c)): detector counts
// I -> line integrals p = mu_scale * -ln(max(I, floor) / I0) (Beer-Lambert),
// then a Gaussian blur along the detector with taps w_{-r..r} (zero outside
// [0, D)).  The two rows are staged in the group's buffer, which step 1 then
// overwrites.
constexpr int kPrePad = 16;              // zero border of a staged row (>= the blur radius)
constexpr int kMaxBlurRadius = 16;

struct PreArgs {
    int on;                              // 0: rows are line integrals already
    const float *flat;                   // per-bin I0 [D], or null
    float flat_value, floor, mu_scale;
    int r;                               // blur radius, 0 = no blur
    float taps[2 * kMaxBlurRadius + 1];  // w_{-r..r}
    float dtaps[2 * kMaxBlurRadius + 2]; // c_m = w_m - w_{m-1}, m in [-r, r+1]
};

// Blurred line integral at n (the full, untruncated sum); row[kPrePad + m] = p[m],
// zero for m outside [0, D) within the border.
__device__ __forceinline__ float blur_at(const float *row, int n, const PreArgs &pre)
{
    const float *c = row + kPrePad + n;
    float acc = pre.taps[pre.r] * c[0];
    for (int k = 1; k <= pre.r; ++k) acc = fmaf(pre.taps[pre.r + k], c[-k] + c[k], acc);
    return acc;
}

// First difference of the blurred row truncated to [0, D): for 0 < n < D it
// is sum_m c_m p[n - m]; at n = 0 it is the blur at 0, at n = D minus the
// blur at D - 1, beyond D zero.
__device__ __forceinline__ float blur_diff(const float *row, int n, int D, const PreArgs &pre)
{
    if (n > D) return 0.f;
    if (n == 0) return blur_at(row, 0, pre);
    if (n == D) return -blur_at(row, D - 1, pre);
    const float *c = row + kPrePad + n;
    float acc = 0.f;
    for (int m = -pre.r; m <= pre.r + 1; ++m) acc = fmaf(pre.dtaps[m + pre.r], c[-m], acc);
    return acc;
}

// Offset scans (Sec. V-A(b): the sample is shifted laterally and turned a
// full circle, so the detector covers one side of a wider field of view).
// The transform runs on a virtual detector of D bins centred on the axis;
// physical bin m sits at virtual bin m + off.  Each virtual sample is
// weighted by the smooth overlap weight w(t) = (1 + sin(pi t / (2 Delta))) / 2
// on |t| <= Delta (0 below, 1 above), t = sgn (n - cv) the signed distance
// from the axis towards the long side, so w(t) + w(-t) = 1 and each line
// counts once.  With fold, the row half a turn later is added at the
// mirrored bin D - 1 - n with weight 1 - w: the line (th + pi, -s) is the
// line (th, s), so one half-turn row carries both measurements.
struct OffArgs {
    int on;                // 0: the rows are the transform's rows
    int Dp;                // physical bins per row
    int off;               // virtual index of physical bin 0
    int fold;              // 1: add the mirrored row half a turn later
    long long K_in, K_out; // rows per slice read and written (K_out = K_in / 2 with fold)
    float cv, sgn, inv_delta;
};

__device__ __forceinline__ float overlap_weight(int n, const OffArgs &o)
{
    const float x = o.sgn * ((float)n - o.cv) * o.inv_delta;
    if (x >= 1.f) return 1.f;
    if (x <= -1.f) return 0.f;
    return 0.5f + 0.5f * sinpif(0.5f * x);
}

// Weighted (and folded) virtual sample n of one row, zero outside [0, D).
__device__ __forceinline__ float offset_sample(const float *p, const float *p2, int n, int D,
                                              const OffArgs &o)
{
    if (!p || n < 0 || n >= D) return 0.f;
    const float w = overlap_weight(n, o);
    const int m = n - o.off;
    float v = (m >= 0 && m < o.Dp) ? w * __ldg(p + m) : 0.f;
    if (o.fold) {
        const int m2 = D - 1 - n - o.off;
        if (m2 >= 0 && m2 < o.Dp) v = fmaf(1.f - w, __ldg(p2 + m2), v);
    }
    return v;
}

// Streamed rows (filter_stream_kernel): the next row pair is copied into a
// shared staging buffer by the bulk-copy (TMA) engine while the current pair
// is transformed; completion is signalled on an mbarrier.
struct StreamNext {
    bool issue;                  // a next pair exists
    const float *src;            // its first row (16-byte aligned); the second follows at src + D
    unsigned row_bytes;          // 4 D, a multiple of 16
    int nrows;                   // 1 or 2
    uint32_t stage_a, stage_b;   // shared addresses of the two rows' slots (16-byte aligned)
    uint32_t mbar;               // the mbarrier the copies complete on
};

__device__ __forceinline__ void bulk_rows(const StreamNext &nx)
{
    // the staging buffer was last read through the generic proxy: order those
    // reads before the asynchronous copy overwrites it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(nx.mbar),
                 "r"(nx.row_bytes * (unsigned)nx.nrows)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(nx.stage_a), "l"(nx.src), "r"(nx.row_bytes), "r"(nx.mbar)
                 : "memory");
    if (nx.nrows == 2)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(nx.stage_b), "l"(nx.src + nx.row_bytes / 4), "r"(nx.row_bytes), "r"(nx.mbar)
                     : "memory");
}

// Wait for the mbarrier phase with the given parity; false after `cap` polls.
// The non-blocking test form keeps every poll short, so the cap bounds the
// time (4M polls: well under a second).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, unsigned parity, long long cap)
{
    for (long long it = 0; it < cap; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// One row pair by one group of C threads (t = thread index in the group).
// S: the group's R x C complex buffer; red: 4 * C/32 floats of the group;
// bar_id: the group's named barrier.
// STAGED: job.a / job.b point to the rows in shared memory (filled by the
// bulk-copy engine); after step 1 has read them, thread 0 starts the copy
// described by *nx into the same buffer.
template <int L, typename T, bool STAGED = false>
__device__ __forceinline__ void fft_pair(const RowPairJob &job, bool active, int D,
                                         const float2 *__restrict__ Gs,
                                         const float2 *__restrict__ tw, float2 *S, float *red,
                                         int t, int bar_id, const PreArgs &pre, const OffArgs &off,
                                         const StreamNext *nx = nullptr)
{
    constexpr int R = fft_R(L), VPL = fft_VPL(L);
    constexpr int C = 32 * VPL;
    const float2 *__restrict__ w32t = tw + L + C;     // W_32^m
    constexpr int NWG = C / 32;                 // warps in the group
    constexpr int RPW = R / NWG;                // rows k1 per warp in step 2
    static_assert(R * C == L && RPW >= 1 && R % NWG == 0, "shape");
    const int lane = t & 31, gw = t >> 5;

    // ---- step 1: differences of z[C n1 + t], R-point DFT over n1.
    // L is even and >= 2D - 1, so D <= L / 2 = C R / 2: the differences are
    // zero for n1 > R / 2 and step 3 stores only n1 < R / 2; the tests on
    // n1 let the compiler drop that half of the first and last butterflies.
    float2 v[R];
    bool nz_a = false, nz_b = false;     // any nonzero (or NaN) sample in the row
    if (pre.on) {
        // stage p for both rows (row stride RS floats, zero borders), then
        // take differences of the blurred rows at n = C n1 + t; the buffer is
        // rewritten below
        float *st = reinterpret_cast<float *>(S);
        const int RS = D + 2 * kPrePad;
        // positions m = t - kPrePad + C i cover [-kPrePad, D + kPrePad) since
        // D + 2 kPrePad <= L/2 + 32 <= C (R/2 + 1); every load is issued
        // before any of them is used
        constexpr int NST = R / 2 + 1;
#pragma unroll
        for (int row = 0; row < 2; ++row) {
            const float *src = row ? job.b : job.a;
            float *dst = st + row * RS + kPrePad;
            float x[NST], f0[NST];
#pragma unroll
            for (int i = 0; i < NST; ++i) {
                const int m = t - kPrePad + C * i;
                const bool in = active && src && m >= 0 && m < D;
                x[i] = in ? __ldg(src + m) : 0.f;
                f0[i] = (in && pre.flat) ? __ldg(pre.flat + m) : pre.flat_value;
            }
#pragma unroll
            for (int i = 0; i < NST; ++i) {
                const int m = t - kPrePad + C * i;
                if (m < D + kPrePad) {
                    const bool in = active && src && m >= 0 && m < D;
                    dst[m] = in ? pre.mu_scale * -logf(__fdiv_rn(fmaxf(x[i], pre.floor), f0[i])) : 0.f;
                }
            }
        }
        group_sync(bar_id, C);
#pragma unroll
        for (int n1 = 0; n1 < R; ++n1) {
            const int n = C * n1 + t;
            float da = 0.f, db = 0.f;
            if (active && n1 <= R / 2 && C * n1 <= D) {   // uniform over the group
                da = blur_diff(st, n, D, pre);
                if (job.b) db = blur_diff(st + RS, n, D, pre);
                nz_a |= (da != 0.f);
                nz_b |= (db != 0.f);
            }
            v[n1] = make_float2(da, db);
        }
        group_sync(bar_id, C);                    // staged rows read before S is written
    } else if (STAGED) {
        // rows already in shared memory with zero borders (index -1 and
        // [D, D + C) read as 0): each difference reads its two samples with
        // no bounds test; nonzero samples are found from an OR of their bits
        const float *sa = job.a, *sb = job.b;
        unsigned bits_a = 0u, bits_b = 0u;
#pragma unroll
        for (int n1 = 0; n1 < R; ++n1) {
            const int n = C * n1 + t;
            float a = 0.f, b = 0.f, am = 0.f, bm = 0.f;
            if (n1 <= R / 2 && C * n1 <= D) {     // uniform over the group
                a = sa[n];
                am = sa[n - 1];
                if (sb) {
                    b = sb[n];
                    bm = sb[n - 1];
                }
                bits_a |= __float_as_uint(a);
                bits_b |= __float_as_uint(b);
            }
            v[n1] = make_float2(a - am, b - bm);
        }
        nz_a = (bits_a & 0x7fffffffu) != 0u;      // some sample with a nonzero magnitude (or NaN)
        nz_b = (bits_b & 0x7fffffffu) != 0u;
    } else if (off.on) {
        // offset scans: weighted (and folded) virtual samples, then differences
#pragma unroll
        for (int n1 = 0; n1 < R; ++n1) {
            const int n = C * n1 + t;
            float a = 0.f, b = 0.f, am = 0.f, bm = 0.f;
            if (active && n1 <= R / 2 && C * n1 <= D) {   // uniform over the group
                a = offset_sample(job.a, job.a2, n, D, off);
                b = offset_sample(job.b, job.b2, n, D, off);
                am = __shfl_up_sync(0xffffffffu, a, 1);
                bm = __shfl_up_sync(0xffffffffu, b, 1);
                if (lane == 0) {
                    am = offset_sample(job.a, job.a2, n - 1, D, off);
                    bm = offset_sample(job.b, job.b2, n - 1, D, off);
                }
                nz_a |= (a != 0.f);
                nz_b |= (b != 0.f);
            }
            v[n1] = make_float2(a - am, b - bm);
        }
    } else {
#pragma unroll
        for (int n1 = 0; n1 < R; ++n1) {
            const int n = C * n1 + t;
            float a = 0.f, b = 0.f, am = 0.f, bm = 0.f;
            if (active && n1 <= R / 2 && C * n1 <= D) {   // uniform over the group
                a = n < D ? __ldg(job.a + n) : 0.f;
                b = (job.b && n < D) ? __ldg(job.b + n) : 0.f;
                am = __shfl_up_sync(0xffffffffu, a, 1);
                bm = __shfl_up_sync(0xffffffffu, b, 1);
                if (lane == 0) {
                    am = (n >= 1 && n - 1 < D) ? __ldg(job.a + n - 1) : 0.f;
                    bm = (job.b && n >= 1 && n - 1 < D) ? __ldg(job.b + n - 1) : 0.f;
                }
                nz_a |= (a != 0.f);
                nz_b |= (b != 0.f);
            }
            v[n1] = make_float2(a - am, b - bm);
        }
    }
    dft_reg<R, false>(v);
    {
        const float2 *twl = fresh(tw);
#pragma unroll
        for (int k1 = 1; k1 < R; ++k1) v[k1] = cmul(v[k1], __ldg(&twl[k1 * C + t]));  // W_L^{t k1}
    }
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) S[k1 * C + t] = v[k1];
    const unsigned za = __ballot_sync(0xffffffffu, nz_a), zb = __ballot_sync(0xffffffffu, nz_b);
    if (lane == 0) {
        red[2 * gw] = za ? 1.f : 0.f;
        red[2 * gw + 1] = zb ? 1.f : 0.f;
    }
    group_sync(bar_id, C);
    if constexpr (STAGED) {
        if (t == 0 && nx->issue) bulk_rows(*nx);     // step 1 is done with the staged rows
    }
    bool zero_a = true, zero_b = true;
#pragma unroll
    for (int w = 0; w < NWG; ++w) {
        zero_a = zero_a && !(red[2 * w] > 0.f);
        zero_b = zero_b && !(red[2 * w + 1] > 0.f);
    }

    // ---- step 2: per row k1, C-point DFT over n2, times G, inverse.
    // Pass A: lane l, per row, the VPL-point DFT over r and W_C^{l kr}; the
    // values go to the swizzled layout.  Pass B: lane j = c + RB s, per round,
    // the 32-point DFTs over l of transforms c (RB-point in registers,
    // W_32^{s m}, SL-point over lanes), the product with G and the inverse.
    // Pass C undoes pass A.
    if (active) {
        constexpr int RB = R < 16 ? R : 16;       // values per lane in pass B
        constexpr int NRD = R / RB;               // pass B rounds (transforms c of round rd: rd RB + j mod RB)
        constexpr int SL = 32 / RB;               // lanes per 32-point transform
        float2 wc[VPL];                            // W_C^{l kr}, the same for every row of the warp
        {
            const float2 *twc = fresh(tw + L);
#pragma unroll
            for (int kr = 1; kr < VPL; ++kr) wc[kr] = __ldg(&twc[32 * kr + lane]);
        }
#pragma unroll 1
        for (int rr = 0; rr < RPW; ++rr) {
            float2 *row = S + (gw * RPW + rr) * C;
            float2 u[VPL];
#pragma unroll
            for (int r = 0; r < VPL; ++r) u[r] = row[lane + 32 * r];
            dft_reg<VPL, false>(u);                                   // r -> kr
#pragma unroll
            for (int kr = 1; kr < VPL; ++kr) u[kr] = cmul(u[kr], wc[kr]);
            __syncwarp();                                             // the row is read before it is rewritten
#pragma unroll
            for (int kr = 0; kr < VPL; ++kr) row[32 * kr + (lane ^ swz_key<R>(rr * VPL + kr))] = u[kr];
        }
        __syncwarp();
#pragma unroll 1
        for (int rd = 0; rd < NRD; ++rd) {
            const int c = rd * RB + (lane & (RB - 1)), s = lane / RB;
            float2 *run = S + (gw * RPW + c / VPL) * C + 32 * (c % VPL);
            const int key = swz_key<R>(c);
            float2 x[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i) x[i] = run[(s + SL * i) ^ key];
            dft_reg<RB, false>(x);                                    // i -> m
            if constexpr (SL == 2) {                                  // W_32^{s m}: s = 0 or 1, constants
#pragma unroll
                for (int m = 1; m < RB; ++m) if (s) x[m] = cmul(x[m], w32(m));
            } else if constexpr (SL > 2) {
#pragma unroll
                for (int m = 1; m < RB; ++m) x[m] = cmul(x[m], __ldg(&w32t[(s * m) & 31]));   // W_32^{s m}
            }
            lane_dif_s<RB, RB>(x, s, w32t);                           // s -> q, kl = m + RB q
            // G is stored in this order: entry ((gw NRD + rd) RB + m) 32 + j is
            // k = k1 + R (kr + VPL (m + RB brev(s)))
            const float2 *g = fresh(Gs + ((gw * NRD + rd) * RB) * 32);
#pragma unroll
            for (int m = 0; m < RB; ++m) x[m] = cmul(x[m], __ldg(&g[m * 32 + lane]));
            lane_dit_inv_s<RB, RB>(x, s, w32t);                       // q -> s
            if constexpr (SL == 2) {
#pragma unroll
                for (int m = 1; m < RB; ++m) if (s) x[m] = cmulc(x[m], w32(m));
            } else if constexpr (SL > 2) {
#pragma unroll
                for (int m = 1; m < RB; ++m) x[m] = cmulc(x[m], __ldg(&w32t[(s * m) & 31]));
            }
            dft_reg<RB, true>(x);                                     // m -> i
#pragma unroll
            for (int i = 0; i < RB; ++i) run[(s + SL * i) ^ key] = x[i];
        }
        __syncwarp();
        {
            const float2 *twc = fresh(tw + L);
#pragma unroll
            for (int kr = 1; kr < VPL; ++kr) wc[kr] = __ldg(&twc[32 * kr + lane]);
        }
#pragma unroll 1
        for (int rr = 0; rr < RPW; ++rr) {
            float2 *row = S + (gw * RPW + rr) * C;
            float2 u[VPL];
#pragma unroll
            for (int kr = 0; kr < VPL; ++kr) u[kr] = row[32 * kr + (lane ^ swz_key<R>(rr * VPL + kr))];
#pragma unroll
            for (int kr = 1; kr < VPL; ++kr) u[kr] = cmulc(u[kr], wc[kr]);
            dft_reg<VPL, true>(u);                                    // kr -> r
            __syncwarp();
#pragma unroll
            for (int r = 0; r < VPL; ++r) row[lane + 32 * r] = u[r];
        }
    }
    group_sync(bar_id, C);

    // ---- step 3: column t, W_L^{-t k1}, inverse R-point DFT over k1
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) v[k1] = S[k1 * C + t];
    {
        const float2 *twl = fresh(tw);
#pragma unroll
        for (int k1 = 1; k1 < R; ++k1) v[k1] = cmulc(v[k1], __ldg(&twl[k1 * C + t]));
    }
    dft_reg<R, true>(v);                                              // k1 -> n1

    // ---- store (16-bit: per-row amax scale first)
    float scale_a = 1.f, scale_b = 1.f;
    if constexpr (sizeof(T) != 4) {
        float ma = 0.f, mb = 0.f;
#pragma unroll
        for (int n1 = 0; n1 < R; ++n1)
            if (n1 < R / 2 && C * n1 + t < D) {
                ma = fmaxf(ma, fabsf(v[n1].x));
                mb = fmaxf(mb, fabsf(v[n1].y));
            }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
            mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        }
        if (lane == 0) {
            red[2 * NWG + 2 * gw] = ma;
            red[2 * NWG + 2 * gw + 1] = mb;
        }
        group_sync(bar_id, C);
        ma = 0.f;
        mb = 0.f;
#pragma unroll
        for (int w = 0; w < NWG; ++w) {
            ma = fmaxf(ma, red[2 * NWG + 2 * w]);
            mb = fmaxf(mb, red[2 * NWG + 2 * w + 1]);
        }
        scale_a = (ma > 0.f && !zero_a) ? ma : 1.f;
        scale_b = (mb > 0.f && !zero_b) ? mb : 1.f;
        if (active && t == 0) {
            job.sa[0] = scale_a;
            if (job.sb) job.sb[0] = scale_b;
        }
    }
    if (active) {
        T *qa = static_cast<T *>(job.qa), *qb = static_cast<T *>(job.qb);
        const float inv_a = __frcp_rn(scale_a), inv_b = __frcp_rn(scale_b);
#pragma unroll
        for (int n1 = 0; n1 < R; ++n1) {
            const int n = C * n1 + t;
            if (n1 < R / 2 && n < D) {
                const float xa = zero_a ? 0.f : v[n1].x, xb = zero_b ? 0.f : v[n1].y;
                if constexpr (sizeof(T) == 4) {
                    qa[n] = xa;
                    if (qb) qb[n] = xb;
                } else {
                    qa[n] = cvt_out<T>(div_rn(xa, scale_a, inv_a));
                    if (qb) qb[n] = cvt_out<T>(div_rn(xb, scale_b, inv_b));
                }
            }
        }
    }
}

struct FilterArgs {
    const float *sino;          // line integrals, or counts when pre.on
    void *filt;
    float *row_scale;
    long long rows;
    int D;
    const float2 *G;
    const float2 *tw;
    PreArgs pre;
    OffArgs off;
};

__device__ __forceinline__ RowPairJob make_job(const float *sino, void *filt, float *row_scale,
                                               long long rows, int D, long long pair, size_t esz,
                                               bool &active)
{
    RowPairJob job;
    active = 2 * pair < rows;
    const long long ra = 2 * pair, rb = 2 * pair + 1;
    const bool has_b = active && rb < rows;
    job.a = active ? sino + ra * D : nullptr;
    job.b = has_b ? sino + rb * D : nullptr;
    job.a2 = job.b2 = nullptr;
    job.qa = active ? static_cast<char *>(filt) + ra * D * esz : nullptr;
    job.qb = has_b ? static_cast<char *>(filt) + rb * D * esz : nullptr;
    job.sa = (active && row_scale) ? row_scale + ra : nullptr;
    job.sb = (has_b && row_scale) ? row_scale + rb : nullptr;
    return job;
}

// Offset mode: output row r of slice s = r / K_out, angle k = r % K_out reads
// physical row s K_in + k (and, with fold, s K_in + k + K_in / 2).
__device__ __forceinline__ void offset_inputs(RowPairJob &job, const float *sino, long long rows,
                                              long long pair, const OffArgs &o)
{
    const long long r[2] = {2 * pair, 2 * pair + 1};
    const float *in[2] = {nullptr, nullptr}, *in2[2] = {nullptr, nullptr};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        if (r[i] < rows) {
            const long long s = r[i] / o.K_out, k = r[i] - s * o.K_out;
            const long long src = s * o.K_in + k;
            in[i] = sino + src * o.Dp;
            in2[i] = o.fold ? sino + (src + o.K_in / 2) * o.Dp : nullptr;
        }
    }
    job.a = job.a ? in[0] : nullptr;
    job.b = job.b ? in[1] : nullptr;
    job.a2 = job.a ? in2[0] : nullptr;
    job.b2 = job.b ? in2[1] : nullptr;
}

template <int L, typename T>
__global__ void __launch_bounds__(kFilterThreads, L <= 2048 ? 2 : 1) filter_kernel(FilterArgs a)
{
    constexpr int C = group_threads(L);
    constexpr int GP = kFilterThreads / C;        // row pairs per block
    extern __shared__ float2 smem_f2[];
    __shared__ float red[GP][4 * (C / 32)];
    const int g = threadIdx.x / C, t = threadIdx.x % C;
    const long long pair = (long long)blockIdx.x * GP + g;
    bool active;
    RowPairJob job = make_job(a.sino, a.filt, a.row_scale, a.rows, a.D, pair, sizeof(T), active);
    if (a.off.on) offset_inputs(job, a.sino, a.rows, pair, a.off);
    fft_pair<L, T>(job, active, a.D, a.G, a.tw, smem_f2 + (size_t)g * L, red[g], t, 1 + g, a.pre, a.off);
}

template <int L, typename T>
fbp_status launch_l(const FilterArgs &fa, cudaStream_t s)
{
    constexpr int GP = kFilterThreads / group_threads(L);
    const long long pairs = (fa.rows + 1) / 2;
    const long long blocks = (pairs + GP - 1) / GP;
    const size_t smem = (size_t)GP * L * sizeof(float2);
    auto kern = filter_kernel<L, T>;
    fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (st != FBP_OK) return st;
    if (blocks > 0x7fffffffLL) return fail(FBP_ERR_UNSUPPORTED, "too many rows");
    kern<<<(unsigned)blocks, kFilterThreads, smem, s>>>(fa);
    FBP_CUDA_TRY(cudaGetLastError());
    return FBP_OK;
}

// Persistent, streamed form for the lengths with one row pair per block
// (L = 8192, 16384): one block per SM walks the row pairs; the bulk-copy
// engine brings pair i+1's rows into a staging buffer beside the transform
// buffer while pair i is transformed.  Plain line-integral rows only, D a
// multiple of 4 and 16-byte aligned rows.  A wait past its cap records
// FAULT_STREAM_WAIT and ends the block (after waiting, also capped, for its
// copy in flight).
constexpr long long kStreamWaitCap = 1LL << 22;   // a 64 KB copy needs ~1000 polls at most

// skip_copies (failure-detection tests only): no row copy is issued, so
// every wait runs out at its cap, records FAULT_STREAM_WAIT and the block
// returns; nothing is written.
template <int L, typename T>
__global__ void __launch_bounds__(kFilterThreads) filter_stream_kernel(FilterArgs a, unsigned *status,
                                                                      int skip_copies)
{
    static_assert(group_threads(L) == kFilterThreads, "one row pair per block");
    extern __shared__ __align__(128) float2 smem_f2[];
    __shared__ float red[4 * (kFilterThreads / 32)];
    __shared__ __align__(8) unsigned long long mbar_store;
    constexpr int C = kFilterThreads;
    float2 *S = smem_f2;
    // staging: 4 zero floats, row a, then C + 4 zero floats and row b, and
    // C + 4 zero floats: each row reads 0 at index -1 and on [D, D + C)
    float *stage = reinterpret_cast<float *>(smem_f2 + L);
    const int RS = a.D + C + 4;                                     // row stride, a multiple of 4
    float *row_a = stage + 4, *row_b = stage + 4 + RS;
    const int t = threadIdx.x;
    for (int i = t; i < C + 4; i += kFilterThreads) {
        if (i < 4) stage[i] = 0.f;
        row_a[a.D + i] = 0.f;
        row_b[a.D + i] = 0.f;
    }
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&mbar_store);
    const long long pairs = (a.rows + 1) / 2;
    auto next_of = [&](long long p) {
        StreamNext nx;
        nx.issue = p < pairs;
        const long long r0 = 2 * p;
        nx.nrows = (r0 + 1 < a.rows) ? 2 : 1;
        nx.src = a.sino + (nx.issue ? r0 : 0) * a.D;
        nx.row_bytes = (unsigned)(a.D * 4);
        nx.stage_a = (uint32_t)__cvta_generic_to_shared(row_a);
        nx.stage_b = (uint32_t)__cvta_generic_to_shared(row_b);
        nx.mbar = mbar;
        return nx;
    };
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    long long pair = blockIdx.x;
    if (t == 0 && pair < pairs && !skip_copies) bulk_rows(next_of(pair));
    unsigned parity = 0;
    bool pending = pair < pairs && !skip_copies;   // a copy this block issued is in flight
    for (; pair < pairs; pair += gridDim.x) {
        // the decision is block-wide, so no thread reaches the transform's
        // barriers while another has left
        const bool ok = mbar_wait(mbar, parity, kStreamWaitCap);
        if (__syncthreads_or(!ok)) {
            if (t == 0) atomicCAS(status, 0u, (unsigned)FAULT_STREAM_WAIT);
            break;
        }
        parity ^= 1u;
        bool active;
        RowPairJob job = make_job(a.sino, a.filt, a.row_scale, a.rows, a.D, pair, sizeof(T), active);
        job.a = row_a;
        job.b = job.b ? row_b : nullptr;
        const StreamNext nx = next_of(pair + gridDim.x);
        pending = nx.issue;
        fft_pair<L, T, true>(job, true, a.D, a.G, a.tw, S, red, t, 1, a.pre, a.off, &nx);   // pre, off: off
    }
    if (pending) mbar_wait(mbar, parity, kStreamWaitCap);   // only after a failed wait
}

template <int L, typename T>
fbp_status launch_stream_l(const FilterArgs &fa, unsigned *status, int skip_copies, cudaStream_t s)
{
    // transform buffer + staging for two rows of D <= L / 2 with zero borders
    const size_t smem = (size_t)L * sizeof(float2) + (size_t)(L + 2 * kFilterThreads + 12) * sizeof(float);
    auto kern = filter_stream_kernel<L, T>;
    fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (st != FBP_OK) return st;
    int per_sm = 0;
    st = blocks_per_sm(reinterpret_cast<const void *>(kern), kFilterThreads, smem, &per_sm);
    if (st != FBP_OK) return st;
    int dev = 0, sms = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    FBP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long pairs = (fa.rows + 1) / 2;
    const long long grid = std::max(1LL, std::min<long long>(pairs, (long long)sms * std::max(1, per_sm)));
    kern<<<(unsigned)grid, kFilterThreads, smem, s>>>(fa, status, skip_copies);
    FBP_CUDA_TRY(cudaGetLastError());
    return FBP_OK;
}

template <typename T>
fbp_status launch_stream_t(const FilterArgs &fa, int L, unsigned *status, int skip, cudaStream_t s)
{
    if (L == 8192) return launch_stream_l<8192, T>(fa, status, skip, s);
    return launch_stream_l<16384, T>(fa, status, skip, s);
}

template <typename T>
fbp_status launch_t(const FilterArgs &fa, int L, cudaStream_t s)
{
    switch (L) {
        case 512: return launch_l<512, T>(fa, s);
        case 1024: return launch_l<1024, T>(fa, s);
        case 2048: return launch_l<2048, T>(fa, s);
        case 4096: return launch_l<4096, T>(fa, s);
        case 8192: return launch_l<8192, T>(fa, s);
        case 16384: return launch_l<16384, T>(fa, s);
    }
    return fail(FBP_ERR_UNSUPPORTED, "filter length %d", L);
}

// Ragged batch: one launch over every item's rows.  A block holds 512 / C
// row pairs of one item (C = the item's group size), so every block's
// groups run the same transform; the shared buffer is sized for the batch's
// longest transform.
template <typename T>
__global__ void __launch_bounds__(kFilterThreads) filter_batched_kernel(FilterBatchArgs a)
{
    extern __shared__ float2 smem_f2[];
    __shared__ float red[4 * kFilterThreads / 32];     // 4 floats per warp
    int lo = 0, hi = a.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.items[mid].group_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const FilterBatchItem &it = a.items[lo];
    const int C = group_threads(it.L);
    const int GP = kFilterThreads / C;
    const int g = threadIdx.x / C, t = threadIdx.x % C;
    const long long pair = (long long)(blockIdx.x - it.group_begin) * GP + g;
    bool active;
    RowPairJob job = make_job(it.sino, it.filt, it.row_scale, it.K, it.D, pair, sizeof(T), active);
    float2 *S = smem_f2 + (size_t)g * it.L;
    float *rd = red + g * 4 * (C / 32);
    PreArgs pre;
    pre.on = 0;
    pre.r = 0;
    OffArgs off;
    off.on = 0;
    if (it.Dp > 0) {
        off.on = 1;
        off.Dp = it.Dp;
        off.off = it.off;
        off.fold = it.fold;
        off.K_in = it.K_in;
        off.K_out = it.K;
        off.cv = it.cv;
        off.sgn = it.sgn;
        off.inv_delta = it.inv_delta;
        RowPairJob oj = job;
        offset_inputs(oj, it.sino, it.K, pair, off);
        job.a = oj.a;
        job.b = oj.b;
        job.a2 = oj.a2;
        job.b2 = oj.b2;
    }
    switch (it.L) {
        case 512: fft_pair<512, T>(job, active, it.D, it.G, it.tw, S, rd, t, 1 + g, pre, off); break;
        case 1024: fft_pair<1024, T>(job, active, it.D, it.G, it.tw, S, rd, t, 1 + g, pre, off); break;
        case 2048: fft_pair<2048, T>(job, active, it.D, it.G, it.tw, S, rd, t, 1 + g, pre, off); break;
        case 4096: fft_pair<4096, T>(job, active, it.D, it.G, it.tw, S, rd, t, 1 + g, pre, off); break;
        case 8192: fft_pair<8192, T>(job, active, it.D, it.G, it.tw, S, rd, t, 1 + g, pre, off); break;
        default: fft_pair<16384, T>(job, active, it.D, it.G, it.tw, S, rd, t, 1 + g, pre, off); break;
    }
}

template <typename T>
fbp_status launch_batched_t(const FilterBatchArgs &a, int groups, int max_L, cudaStream_t s)
{
    // (512 / C) pairs x L float2 = 4096 R bytes, largest for the longest L
    const size_t smem = (size_t)(kFilterThreads / group_threads(max_L)) * max_L * sizeof(float2);
    auto kern = filter_batched_kernel<T>;
    fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (st != FBP_OK) return st;
    kern<<<groups, kFilterThreads, smem, s>>>(a);
    FBP_CUDA_TRY(cudaGetLastError());
    return FBP_OK;
}


// Kernel arguments of one filter launch (FilterLaunch, fbp_internal.cuh).
inline fbp_status make_filter_args(const FilterLaunch &a, FilterArgs &fa)
{
    fa.sino = a.sino;
    fa.filt = a.filt;
    fa.row_scale = a.row_scale;
    fa.rows = a.rows;
    fa.D = a.D;
    fa.G = a.G;
    fa.tw = a.tw;
    fa.pre.on = 0;
    fa.pre.r = 0;
    fa.off.on = 0;
    if (a.offset) {
        const FilterOffset &o = *a.offset;
        if (a.pre) return fail(FBP_ERR_UNSUPPORTED, "offset rows from counts");
        fa.off.on = 1;
        fa.off.Dp = o.Dp;
        fa.off.off = o.off;
        fa.off.fold = o.fold;
        fa.off.K_in = o.K_in;
        fa.off.K_out = o.fold ? o.K_in / 2 : o.K_in;
        fa.off.cv = o.cv;
        fa.off.sgn = o.sgn;
        fa.off.inv_delta = o.inv_delta;
    }
    if (a.pre) {
        const FilterPre &p = *a.pre;
        if (p.blur_radius < 0 || p.blur_radius > kMaxBlurRadius)
            return fail(FBP_ERR_UNSUPPORTED, "blur radius %d", p.blur_radius);
        fa.pre.on = 1;
        fa.pre.flat = p.flat;
        fa.pre.flat_value = p.flat_value;
        fa.pre.floor = p.floor;
        fa.pre.mu_scale = p.mu_scale;
        fa.pre.r = p.blur_radius;
        for (int k = 0; k <= 2 * p.blur_radius; ++k) fa.pre.taps[k] = p.taps[k];
        for (int m = 0; m <= 2 * p.blur_radius + 1; ++m)     // c_m = w_m - w_{m-1}
            fa.pre.dtaps[m] = (m <= 2 * p.blur_radius ? p.taps[m] : 0.f) - (m >= 1 ? p.taps[m - 1] : 0.f);
    }
    return FBP_OK;
}

template <typename T>
fbp_status launch_plain_rows(const FilterLaunch &a, cudaStream_t s)
{
    FilterArgs fa;
    const fbp_status st = make_filter_args(a, fa);
    if (st != FBP_OK) return st;
    return launch_t<T>(fa, a.L, s);
}

template <typename T>
fbp_status launch_streamed_rows(const FilterLaunch &a, unsigned *status, int skip, cudaStream_t s)
{
    FilterArgs fa;
    const fbp_status st = make_filter_args(a, fa);
    if (st != FBP_OK) return st;
    return launch_stream_t<T>(fa, a.L, status, skip, s);
}

}  // namespace
}  // namespace fbp
