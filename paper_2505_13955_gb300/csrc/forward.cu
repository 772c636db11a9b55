// forward.cu -- K3: the matched forward projector A, the exact transpose of
// the backprojection with linear interpolation (scale 1):
//   (A f)_k[j] = sum_{r,c} f[r][c] * max(0, 1 - |u_k(r,c) - j|).
// (The paper's simulated data come from a forward model, Sec. V-B(a); here
// the projector is written as the adjoint of the library's own backprojector,
// so that least-squares refinement has the exact gradient.)
//
// Two forms share one support solve.  For bin j and a line of the image
// along the axis where |cos| or |sin| is smaller (rows when |cos th| >=
// |sin th|), the pixels whose coordinate lies within one bin of j form a run
// of at most ceil(2/g) candidates along the other axis, g = alpha *
// max(|cos|, |sin|); the run's start moves linearly from line to line and is
// kept in fixed point, so the weights keep full precision without FP64 per
// line:
//   xm(w) = B - slope * w   (first candidate = floor(xm) + 1)
//   weight_i = max(0, 1 - |g (delta + i) - 1|), delta = 1 - frac(xm).
//
// * Gather form (fwd_strip_kernel, fwd_kernel): one thread per output bin
//   (k, j) walks every line; no atomics, deterministic.  A block covers 128
//   consecutive bins of one angle; their candidates on 32 consecutive lines
//   lie in one strip of the image, which the block stages in shared memory
//   with coalesced loads (rows of the strip for the row walk, 32-column
//   segments for the column walk, transposed into shared memory).  Pixels
//   outside the image are staged as zeros.  Geometries whose strip would not
//   fit (pixel_size / det_spacing < 1/4) use the same walk with direct
//   global loads.
// * Tile-owned form (fwd_tile_kernel, below): one block per image tile visits
//   every angle, so the image is read once per call rather than once per
//   angle; partial bins are combined with floating-point atomics.
#include <algorithm>
#include <cmath>

#include "fbp_internal.cuh"

namespace fbp {
namespace {

constexpr int kBins = 128;      // bins (threads) per block
constexpr int kLines = 32;      // lines per staged chunk

struct FwdArgs {
    const float *slice;
    float *sino;
    const double2 *cs;
    int K, D, N;
    double alpha, det_center;
    int bins_blocks;     // ceil(D / 128)
    int slice_base;
    int span_pitch;      // staged strip width (+1 pad), 0 = no staging
};

// Per-bin walk setup (FP64), shared by both kernels.
struct Walk {
    bool walk_rows;
    double g, h, slope, B;
    int nc;
};

__device__ __forceinline__ Walk walk_setup(const FwdArgs &a, int k, double j, int ncmax)
{
    Walk w;
    const double2 cs = a.cs[k];
    w.walk_rows = fabs(cs.x) >= fabs(cs.y);
    const double cp = a.alpha * (w.walk_rows ? cs.x : cs.y);   // along the solved axis
    const double cq = a.alpha * (w.walk_rows ? cs.y : cs.x);   // along the walked axis
    w.g = fabs(cp);
    w.h = 1.0 / w.g;
    w.nc = min(ncmax, (int)ceil(2.0 * w.h));
    const double m = 0.5 * (a.N - 1);
    w.slope = cq / cp;
    w.B = (j - a.det_center + cq * m) / cp + m - w.h;
    return w;
}

// Lines w on which some candidate of this walk can fall inside [0, N);
// clamped in double before conversion (near th = pi/2 the slope is ~1e-17 and
// the unclamped quotients overflow int).
__device__ __forceinline__ void walk_lines(const Walk &w, int N, int &w0, int &w1)
{
    double lo_d = 0.0, hi_d = (double)(N - 1);
    if (w.slope > 0.0) {
        lo_d = fmax(lo_d, floor((w.B - N) / w.slope) - 1.0);
        hi_d = fmin(hi_d, ceil((w.B + w.nc + 1) / w.slope) + 1.0);
    } else if (w.slope < 0.0) {
        lo_d = fmax(lo_d, floor((w.B + w.nc + 1) / w.slope) - 1.0);
        hi_d = fmin(hi_d, ceil((w.B - N) / w.slope) + 1.0);
    } else if (!(w.B > -w.nc - 1.0 && w.B < (double)N)) {
        hi_d = -1.0;
    }
    lo_d = fmin(lo_d, (double)N);     // both now lie in [-1, N]
    hi_d = fmax(hi_d, -1.0);
    w0 = (int)lo_d;
    w1 = (int)hi_d;
}

// Direct-load walk (small pixel/bin ratios, whose strips are too wide).
template <int NCMAX>
__global__ void __launch_bounds__(128) fwd_kernel(FwdArgs a)
{
    const int k = blockIdx.x / a.bins_blocks;
    const int j = (blockIdx.x % a.bins_blocks) * 128 + threadIdx.x;
    const int sl = a.slice_base + blockIdx.y;
    if (j >= a.D) return;
    const int N = a.N;
    const float *f = a.slice + (size_t)sl * N * N;
    const Walk wk = walk_setup(a, k, (double)j, NCMAX);
    int w0, w1;
    walk_lines(wk, N, w0, w1);
    float acc = 0.f;
    if (w0 <= w1) {
        const double two32 = 4294967296.0;
        long long XM = __double2ll_rn((wk.B - wk.slope * (double)w0) * two32);
        const long long SL = __double2ll_rn(wk.slope * two32);
        const float gf = (float)wk.g;
        for (int w = w0; w <= w1; ++w) {
            const int start = (int)(XM >> 32) + 1;
            const unsigned lo = (unsigned)(XM & 0xffffffffLL);
            const float delta = 2.0f - __uint_as_float(0x3f800000u | (lo >> 9));
            const float gd = gf * delta;
#pragma unroll
            for (int i = 0; i < NCMAX; ++i) {
                if (i < wk.nc) {
                    const int col = start + i;
                    const float wgt = fmaxf(0.f, 1.f - fabsf(fmaf(gf, (float)i, gd) - 1.f));
                    if ((unsigned)col < (unsigned)N) {
                        const float v = wk.walk_rows ? __ldg(f + (size_t)w * N + col)
                                                     : __ldg(f + (size_t)col * N + w);
                        acc = fmaf(wgt, v, acc);
                    }
                }
            }
            XM -= SL;
        }
    }
    a.sino[((size_t)sl * a.K + k) * a.D + j] = acc;
}

// Block-uniform walk parameters, formed once per block by thread 0 in FP64.
struct BlockWalk {
    double inv_cp, cq, h, slope;
    long long SL;            // slope in 32.32 fixed point
    long long XMa, XMb;      // first / last bin's position at line blo
    float g;
    int nc, walk_rows, blo, bhi;
};

// Staged walk: the block's strip, kLines lines at a time, in shared memory.
// FP64 is used only for the block setup and each bin's starting position;
// the per-line walk and the per-chunk strip bounds are exact integer
// arithmetic on the 32.32 fixed-point positions.
template <int NCMAX>
__global__ void __launch_bounds__(kBins) fwd_strip_kernel(FwdArgs a)
{
    extern __shared__ float strip[];                     // [kLines][span_pitch]
    __shared__ BlockWalk bw;
    const int k = blockIdx.x / a.bins_blocks;
    const int j0 = (blockIdx.x % a.bins_blocks) * kBins;
    const int tid = threadIdx.x;
    const int j = j0 + tid;
    const int sl = a.slice_base + blockIdx.y;
    const int N = a.N, P = a.span_pitch;
    const float *f = a.slice + (size_t)sl * N * N;
    const int jl = min(j0 + kBins - 1, a.D - 1);
    const double two32 = 4294967296.0;
    const double m = 0.5 * (N - 1);

    if (tid == 0) {
        const Walk wa = walk_setup(a, k, (double)j0, NCMAX);
        const Walk wb = walk_setup(a, k, (double)jl, NCMAX);
        int blo = 0, bhi = N - 1;
        if (wa.slope != 0.0) {       // (a zero slope -- th = 0 or pi/2 exactly -- takes every line)
            int wa0, wa1, wb0, wb1;
            walk_lines(wa, N, wa0, wa1);
            walk_lines(wb, N, wb0, wb1);
            blo = max(0, min(wa0, wb0));
            bhi = min(N - 1, max(wa1, wb1));
        }
        const double2 cs = a.cs[k];
        const double cp = a.alpha * (wa.walk_rows ? cs.x : cs.y);
        bw.inv_cp = 1.0 / cp;
        bw.cq = a.alpha * (wa.walk_rows ? cs.y : cs.x);
        bw.h = wa.h;
        bw.slope = wa.slope;
        bw.SL = __double2ll_rn(wa.slope * two32);
        bw.XMa = __double2ll_rn((wa.B - wa.slope * (double)blo) * two32);
        bw.XMb = __double2ll_rn((wb.B - wb.slope * (double)blo) * two32);
        bw.g = (float)wa.g;
        bw.nc = wa.nc;
        bw.walk_rows = wa.walk_rows;
        bw.blo = blo;
        bw.bhi = bhi;
    }
    __syncthreads();
    const int blo = bw.blo, bhi = bw.bhi, nc = bw.nc;
    const bool walk_rows = bw.walk_rows;
    const long long SL = bw.SL;
    // this bin's position at line blo (padding threads j >= D walk like the last bin)
    const double B = ((double)min(j, a.D - 1) - a.det_center + bw.cq * m) * bw.inv_cp + m - bw.h;
    long long XM = __double2ll_rn((B - bw.slope * (double)blo) * two32);
    const float gf = bw.g;
    const uint32_t strip_s = (uint32_t)__cvta_generic_to_shared(strip);
    float acc = 0.f;

    for (int wc = blo; wc <= bhi; wc += kLines) {
        // strip columns for lines [wc, wc + kLines): candidates start at
        // floor(xm) + 1 and span nc; xm is affine in (bin, line), so the end
        // bins' positions at the chunk's first and last lines bound every
        // bin's; one extra column each side absorbs the per-bin rounding
        const long long d0 = (long long)(wc - blo) * SL, d1 = (long long)(wc + kLines - 1 - blo) * SL;
        const long long c00 = (bw.XMa - d0) >> 32, c01 = (bw.XMa - d1) >> 32;
        const long long c10 = (bw.XMb - d0) >> 32, c11 = (bw.XMb - d1) >> 32;
        const int s_lo = (int)min(min(c00, c01), min(c10, c11));
        const int s_hi = (int)max(max(c00, c01), max(c10, c11)) + NCMAX + 1;
        const int span = s_hi - s_lo + 1;            // <= P - 1 by the pitch bound
        __syncthreads();
        if (walk_rows) {
            // line w = image row, s = column: row segments, coalesced
            for (int l = 0; l < kLines; ++l) {
                const int w = wc + l;
                const bool wok = (unsigned)w < (unsigned)N;
                const float *row = f + (size_t)(wok ? w : 0) * N;
                for (int s = tid; s < span; s += kBins) {
                    const int c = s_lo + s;
                    strip[l * P + s] = (wok && (unsigned)c < (unsigned)N) ? __ldg(row + c) : 0.f;
                }
            }
        } else {
            // line w = image column, s = row: 32 consecutive columns of a row
            // per warp-read, transposed into [line][s] (odd pitch: no conflicts)
            const int l = tid & (kLines - 1);
            const int w = wc + l;
            const bool wok = (unsigned)w < (unsigned)N;
            for (int s = tid / kLines; s < span; s += kBins / kLines) {
                const int r = s_lo + s;
                strip[l * P + s] = (wok && (unsigned)r < (unsigned)N) ? __ldg(f + (size_t)r * N + w) : 0.f;
            }
        }
        __syncthreads();
        const int lend = min(kLines, bhi - wc + 1);
        uint32_t line_base = strip_s - 4u * (uint32_t)s_lo;
        for (int l = 0; l < lend; ++l) {
            const int start = (int)(XM >> 32) + 1;
            const unsigned lo = (unsigned)(XM & 0xffffffffLL);
            const float delta = 2.0f - __uint_as_float(0x3f800000u | (lo >> 9));
            const float gd = gf * delta;
            const uint32_t base = line_base + 4u * (uint32_t)start;
#pragma unroll
            for (int i = 0; i < NCMAX; ++i) {
                if (i < nc) {
                    const float wgt = fmaxf(0.f, 1.f - fabsf(fmaf(gf, (float)i, gd) - 1.f));
                    float v;
                    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(base + 4u * i));
                    acc = fmaf(wgt, v, acc);
                }
            }
            XM -= SL;
            line_base += 4u * (uint32_t)P;
        }
    }
    if (j < a.D) a.sino[((size_t)sl * a.K + k) * a.D + j] = acc;
}


// ---------------------------------------------------------------------------
// Tile-owned form.  One block per 64 x 64 pixel tile (and slice group, and
// share of the angles: fwd_angle_parts) stages the tile once in shared
// memory and visits its angles; per angle it walks only
// the bins the tile's footprint covers, over the tile's own lines, with the
// same support solve as above, and adds each bin's partial sum to the
// sinogram with a global floating-point reduction.  The image is therefore
// read from memory once per call instead of once per angle, at the price of
// a summation order over tiles that is not fixed from run to run.
//
// Positions on a line are kept in 9.23 fixed point (plus an integer bias of
// 4, so that floor(P) + 4 is the first candidate's index in the padded
// tile); each bin's position at its first line is formed exactly from 32.32
// per-(tile, angle) values computed in FP64, and the per-line step is
// rounded to 2^-24, so after the at most 64 / LS steps of one walk the
// position is within 1e-6 pixel.
//
// Candidate weights, with e = g * (x1 - P) in (0, g] for the first candidate
// x1 = floor(P) + 1 and g in [2/3, 1] (pixel / bin ratio alpha in
// [0.9429, 1]): w0 = e, w1 = 1 - |e + g - 1|, w2 = max(0, 2 - 2g - e); a
// fourth candidate would have weight max(0, 2 - 3g - e) = 0.
// ---------------------------------------------------------------------------
constexpr int kTT = 64;                  // tile side
constexpr int kTPad = 3;                 // zero border; clamped candidate reads land in it
constexpr int kTSide = kTT + 2 * kTPad;  // 70
constexpr int kTPitch = 71;              // odd: a column walk's lanes read distinct banks
// Threads per block: the four-slice form runs 384 (12 warps; 79 registers,
// so two blocks -- as many as its 80 KB tile allows -- give 24 warps per SM
// to cover the shared-load latency: 2.12 -> 2.27 Tupdates/s at N = 1024,
// K = 1800); the one- and two-slice forms run 256, four blocks per SM.
// Each thread stages one angle's walk parameters per chunk.
template <int NS> constexpr int tile_threads() { return NS == 4 ? 384 : 256; }
constexpr int kFrac = 23;                // fraction bits of a walk position
constexpr int kBias = 4;

struct alignas(16) TileAngle {
    long long P0;          // first-candidate position of bin jbase at line 0, 32.32, + kBias
    long long BJ;          // step per bin, 32.32
    long long SL;          // step per line (subtracted), 32.32
    float g;               // alpha * max(|cos|, |sin|)
    float p0f, bjf, slf;   // P0 (unbiased), BJ, SL as floats, for the line ranges
    int jbase, W, walk_rows, pad_;
};
static_assert(sizeof(TileAngle) == 64, "TileAngle layout");

struct FwdTileArgs {
    const float *slice;
    float *sino;
    const double2 *cs;
    int K, D, N;
    double alpha, det_center;
    int tiles_x;
    int slice_base;
    int k_parts;         // blocks per tile along z, each a contiguous share of the angles
};

// Walk parameters of tile (r0, c0) for angle k, in FP64.  Bin j's ray meets
// line l of the tile (row r0 + l for a row walk, column c0 + l otherwise) at
// tile-local coordinate t = (j - c_d - cq (l0 + l - m)) / cp - s0 + m, and
// the bins that any tile pixel touches are floor(u_min) .. floor(u_max) + 1.
__device__ __forceinline__ TileAngle tile_angle_setup(const FwdTileArgs &a, int k, int r0, int c0)
{
    const double2 cs = a.cs[k];
    const double m = 0.5 * (a.N - 1);
    const double ax = a.alpha * cs.x, ay = a.alpha * cs.y;
    const double ua = ax * ((double)c0 - m) + ay * ((double)r0 - m) + a.det_center;
    const double dx = ax * (kTT - 1), dy = ay * (kTT - 1);
    const double umin = ua + fmin(0.0, dx) + fmin(0.0, dy);
    const double umax = ua + fmax(0.0, dx) + fmax(0.0, dy);
    TileAngle p;
    p.jbase = (int)floor(umin);
    p.W = (int)floor(umax) + 2 - p.jbase;
    p.walk_rows = fabs(cs.x) >= fabs(cs.y);
    const double cp = p.walk_rows ? ax : ay;          // along the solved axis
    const double cq = p.walk_rows ? ay : ax;          // along the line axis
    const double s0 = p.walk_rows ? c0 : r0, l0 = p.walk_rows ? r0 : c0;
    const double P0 = ((double)p.jbase - a.det_center - cq * (l0 - m)) / cp - s0 + m - 1.0 / fabs(cp);
    const double BJ = 1.0 / cp, SL = cq / cp;
    const double two32 = 4294967296.0;
    p.P0 = __double2ll_rn((P0 + kBias) * two32);
    p.BJ = __double2ll_rn(BJ * two32);
    p.SL = __double2ll_rn(SL * two32);
    p.g = (float)fabs(cp);
    p.p0f = (float)P0;
    p.bjf = (float)BJ;
    p.slf = (float)SL;
    p.pad_ = 0;
    return p;
}

// Vector of NS slices' pixels at one tile position (NS = 1, 2 or 4): the
// multi-slice kernels read the same candidates of NS slices with one 8- or
// 16-byte shared load and share the position and weight arithmetic.
template <int NS> struct PixVec;
template <> struct PixVec<1> { using T = float; };
template <> struct PixVec<2> { using T = float2; };
template <> struct PixVec<4> { using T = float4; };
__device__ __forceinline__ float comp(const float &v, int) { return v; }
__device__ __forceinline__ float comp(const float2 &v, int s) { return s == 0 ? v.x : v.y; }
__device__ __forceinline__ float comp(const float4 &v, int s)
{
    return s == 0 ? v.x : s == 1 ? v.y : s == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_comp(float &v, int, float x) { v = x; }
__device__ __forceinline__ void set_comp(float2 &v, int s, float x) { (s == 0 ? v.x : v.y) = x; }
__device__ __forceinline__ void set_comp(float4 &v, int s, float x)
{
    (s == 0 ? v.x : s == 1 ? v.y : s == 2 ? v.z : v.w) = x;
}

// One lane's walk over lines lo + lsub, lo + lsub + LS, ... <= hi.
template <int LS, bool ROWS, int NS>
__device__ __forceinline__ void tile_walk(const typename PixVec<NS>::T *tile, long long Pb,
                                          long long SL, int lo, int hi, int lsub, float g,
                                          float (&acc)[NS])
{
    using V = typename PixVec<NS>::T;
    constexpr int LW = ROWS ? kTPitch : 1;   // elements between lines
    constexpr int SW = ROWS ? 1 : kTPitch;   // elements between candidates
    int l = lo + lsub;
    if (l > hi) return;
    const float twog = 2.f * g, gm1 = g - 1.f, c2 = 2.f - 2.f * g;
    int P = (int)((Pb - (long long)l * SL) >> (32 - kFrac));
    const int dP = (int)(((long long)LS * SL + (1LL << (31 - kFrac))) >> (32 - kFrac));
    int lb = (l + kTPad) * LW;
#pragma unroll 4
    for (; l <= hi; l += LS) {
        // first candidate's padded index, clamped into the zero border when
        // every candidate lies outside the tile (negative -> huge unsigned)
        const uint32_t c = min((uint32_t)(P >> kFrac), (uint32_t)(kTT + kTPad));
        const V *e = tile + lb + (int)c * SW;
        const float F = __uint_as_float(((uint32_t)P & 0x7fffffu) | 0x3f800000u);   // 1 + frac(P)
        const float w0 = fmaf(-g, F, twog);                                          // g * (2 - F)
        const float w1 = 1.f - fabsf(w0 + gm1);
        const float w2 = fmaxf(0.f, c2 - w0);
        // the third candidate carries weight only when e < 2 - 2g (a quarter
        // of the (bin, line) pairs over a half turn): the multi-slice forms
        // skip its 8- or 16-byte load otherwise; the one-slice form loads it
        // always (a 4-byte read inside the padded tile, weight 0), which
        // costs fewer instructions than the predicate
        const V v0 = e[0], v1 = e[SW];
        V v2;
        if constexpr (NS == 1) {
            v2 = e[2 * SW];
        } else {
#pragma unroll
            for (int t = 0; t < NS; ++t) set_comp(v2, t, 0.f);
            if (w2 > 0.f) v2 = e[2 * SW];
        }
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            acc[t] = fmaf(w0, comp(v0, t), acc[t]);
            acc[t] = fmaf(w1, comp(v1, t), acc[t]);
            acc[t] = fmaf(w2, comp(v2, t), acc[t]);
        }
        P -= dP;
        lb += LS * LW;
    }
}

template <int NS>
constexpr size_t tile_bytes() { return ((size_t)kTSide * kTPitch * 4 * NS + 63) / 64 * 64; }
template <int NS>
constexpr size_t tile_smem() { return tile_bytes<NS>() + (size_t)tile_threads<NS>() * sizeof(TileAngle); }

// NS slices per block (slices slice_base + NS * blockIdx.y + [0, NS)).
template <int BPW, int NS>
__global__ void __launch_bounds__(tile_threads<NS>(), NS == 4 ? 2 : 4) fwd_tile_kernel(FwdTileArgs a)
{
    using V = typename PixVec<NS>::T;
    constexpr int kTThreads = tile_threads<NS>();
    constexpr int kTChunk = kTThreads;       // angles whose walk parameters are staged together
    constexpr int LS = 32 / BPW;             // lines walked side by side in a warp
    extern __shared__ __align__(64) unsigned char fwd_smem[];
    V *tile = reinterpret_cast<V *>(fwd_smem);
    TileAngle *prm = reinterpret_cast<TileAngle *>(fwd_smem + tile_bytes<NS>());
    const int N = a.N;
    const int ty = blockIdx.x / a.tiles_x, tx = blockIdx.x - ty * a.tiles_x;
    const int r0 = ty * kTT, c0 = tx * kTT;
    const int sl0 = a.slice_base + NS * blockIdx.y;
    const float *f = a.slice + (size_t)sl0 * N * N;
    for (int i = threadIdx.x; i < kTSide * kTPitch; i += kTThreads) {
        const int rr = i / kTPitch, cc = i - rr * kTPitch;
        const int r = r0 + rr - kTPad, c = c0 + cc - kTPad;
        const bool in = rr >= kTPad && rr < kTPad + kTT && cc >= kTPad && cc < kTPad + kTT &&
                        r < N && c < N;
        V v;
#pragma unroll
        for (int t = 0; t < NS; ++t)
            set_comp(v, t, in ? __ldg(f + (size_t)t * N * N + (size_t)r * N + c) : 0.f);
        tile[i] = v;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bl = lane % BPW, lsub = lane / BPW;
    // this block's angles (the bins of an angle are the same sums whichever
    // block adds them)
    const int kb = (int)((long long)blockIdx.z * a.K / a.k_parts);
    const int ke = (int)((long long)(blockIdx.z + 1) * a.K / a.k_parts);
    for (int k0 = kb; k0 < ke; k0 += kTChunk) {
        __syncthreads();                     // tile staged / previous chunk consumed
        if (k0 + (int)threadIdx.x < ke)
            prm[threadIdx.x] = tile_angle_setup(a, k0 + threadIdx.x, r0, c0);
        __syncthreads();
        const int kc = min(kTChunk, ke - k0);
        for (int ki = warp; ki < kc; ki += kTThreads / 32) {
            const TileAngle p = prm[ki];
            float *out = a.sino + ((size_t)sl0 * a.K + (k0 + ki)) * a.D;
            const int ng = (p.W + BPW - 1) / BPW;
            for (int q = 0; q < ng; ++q) {
                // lines on which some bin of the group has a candidate inside
                // the tile: max_b P >= -3 and min_b P < T - 1, P = P(b,0) - l SL
                // (float bounds with slack; excluded lines contribute nothing)
                const int bA = q * BPW, bB = min(bA + BPW - 1, p.W - 1);
                const float PA = fmaf((float)bA, p.bjf, p.p0f), PB = fmaf((float)bB, p.bjf, p.p0f);
                const float Pl = fminf(PA, PB) - 0.01f, Ph = fmaxf(PA, PB) + 0.01f;
                float lo_f = 0.f, hi_f = (float)(kTT - 1);
                if (p.slf > 0.f) {
                    hi_f = fminf(hi_f, (Ph + 3.f) / p.slf);
                    lo_f = fmaxf(lo_f, (Pl - (float)(kTT - 1)) / p.slf);
                } else if (p.slf < 0.f) {
                    lo_f = fmaxf(lo_f, (Ph + 3.f) / p.slf);
                    hi_f = fminf(hi_f, (Pl - (float)(kTT - 1)) / p.slf);
                } else if (!(Ph >= -3.f && Pl < (float)(kTT - 1))) {
                    hi_f = -1.f;
                }
                lo_f = fminf(lo_f, (float)kTT);
                hi_f = fmaxf(hi_f, -1.f);
                const int lo = max(0, (int)floorf(lo_f) - 1);
                const int hi = min(kTT - 1, (int)floorf(hi_f) + 1);
                const int b = bA + bl;
                const long long Pb = p.P0 + (long long)b * p.BJ;
                float acc[NS];
#pragma unroll
                for (int t = 0; t < NS; ++t) acc[t] = 0.f;
                if (p.walk_rows) tile_walk<LS, true, NS>(tile, Pb, p.SL, lo, hi, lsub, p.g, acc);
                else tile_walk<LS, false, NS>(tile, Pb, p.SL, lo, hi, lsub, p.g, acc);
#pragma unroll
                for (int t = 0; t < NS; ++t) {
#pragma unroll
                    for (int o = BPW; o < 32; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
                }
                const int j = p.jbase + b;
                if (lsub == 0 && b < p.W && (unsigned)j < (unsigned)a.D) {
#pragma unroll
                    for (int t = 0; t < NS; ++t)
                        if (acc[t] != 0.f) atomicAdd(out + (size_t)t * a.K * a.D + j, acc[t]);
                }
            }
        }
    }
}

}  // namespace

// Staged strip width for a geometry: candidates of 128 bins over 32 lines
// span at most 127/g + 31 |slope| + ncmax + 3 columns (g >= alpha/sqrt 2,
// |slope| <= 1, one margin column each side, floors); 0 when that exceeds
// the shared-memory budget.
int fwd_span_pitch(double alpha, int ncmax)
{
    const double span = 127.0 * 1.4142135623730951 / alpha + 31.0 + ncmax + 5.0;
    const int pitch = ((int)std::ceil(span) | 1);       // odd pitch: conflict-free transposed stores
    return (size_t)kLines * pitch * sizeof(float) <= 160 * 1024 ? pitch : 0;
}

bool fwd_tile_eligible(double alpha)
{
    // g = alpha * max(|cos|, |sin|) must lie in [2/3, 1] for the three-candidate weights
    return alpha >= 0.9429 && alpha <= 1.0;
}

int fwd_variant_count() { return 6; }

// Angle parts per tile: the block count B = tiles x slice groups fills
// ceil(B P / R) waves of R resident blocks in time proportional to
// ceil(B P / R) / P; the P in [1, 8] (at least 64 angles each) with the
// least time, plus 0.5 % per part for restaging the tile, trims the last,
// partly filled wave (N = 1024, 16 slices: 1024 blocks on 304 slots).
int fwd_angle_parts(long long blocks, long long resident, int K)
{
    if (blocks <= 0 || resident <= 0) return 1;
    int best = 1;
    double best_t = 1e300;
    for (int P = 1; P <= 8 && (P == 1 || K / P >= 64); ++P) {
        const long long waves = (blocks * P + resident - 1) / resident;
        const double t = (double)waves / P * (1.0 + 0.005 * P);
        if (t < best_t - 1e-12) {
            best_t = t;
            best = P;
        }
    }
    return best;
}

template <int BPW, int NS>
static fbp_status launch_tile_group(FwdTileArgs a, int first, int count, unsigned tiles, cudaStream_t s)
{
    // count slices from `first`, NS per block
    const void *kern = reinterpret_cast<const void *>(fwd_tile_kernel<BPW, NS>);
    constexpr size_t smem = tile_smem<NS>();
    fbp_status st = ensure_dynamic_smem(kern, smem);
    if (st != FBP_OK) return st;
    int per_sm = 0, sms = 0;
    st = blocks_per_sm(kern, tile_threads<NS>(), smem, &per_sm);
    if (st == FBP_OK) st = device_sm_count(&sms);
    if (st != FBP_OK) return st;
    const int groups = count / NS;
    a.k_parts = fwd_angle_parts((long long)tiles * std::min(65535, groups), (long long)sms * std::max(per_sm, 1),
                                a.K);
    for (int g0 = 0; g0 < groups; g0 += 65535) {
        a.slice_base = first + NS * g0;
        dim3 grid(tiles, (unsigned)std::min(65535, groups - g0), (unsigned)a.k_parts);
        fwd_tile_kernel<BPW, NS><<<grid, tile_threads<NS>(), smem, s>>>(a);
        FBP_CUDA_TRY(cudaGetLastError());
    }
    return FBP_OK;
}

// Variants 1-3: one slice per block, 8 / 16 / 32 bins per warp.  Variant 4:
// four slices per block (8 bins per warp, one 16-byte load per candidate),
// variant 5: two slices per block (16 bins per warp); leftover slices of
// either go through the narrower kernels.
static fbp_status launch_forward_tile(const FwdLaunch &L, int v, cudaStream_t s)
{
    if (!fwd_tile_eligible(L.alpha))
        return fail(FBP_ERR_UNSUPPORTED, "tile forward projector needs pixel_size / det_spacing in [0.9429, 1]");
    FwdTileArgs a;
    a.slice = L.slice;
    a.sino = L.sino;
    a.cs = L.cs;
    a.K = L.K;
    a.D = L.D;
    a.N = L.N;
    a.alpha = L.alpha;
    a.det_center = L.det_center;
    a.tiles_x = (L.N + kTT - 1) / kTT;
    const long long tiles = (long long)a.tiles_x * a.tiles_x;
    if (tiles > 0x7fffffffLL) return fail(FBP_ERR_UNSUPPORTED, "too many image tiles");
    const unsigned nt = (unsigned)tiles;
    FBP_CUDA_TRY(cudaMemsetAsync(L.sino, 0, (size_t)L.S * L.K * L.D * sizeof(float), s));
    fbp_status st = FBP_OK;
    int done = 0;
    if (v == 4) {
        const int n4 = L.S / 4 * 4;
        if (n4) st = launch_tile_group<8, 4>(a, 0, n4, nt, s);
        done = n4;
    }
    if (st == FBP_OK && (v == 4 || v == 5)) {
        const int n2 = (L.S - done) / 2 * 2;
        if (n2) st = launch_tile_group<16, 2>(a, done, n2, nt, s);
        done += n2;
    }
    if (st != FBP_OK || done == L.S) return st;
    switch (v) {
    case 1: return launch_tile_group<8, 1>(a, done, L.S - done, nt, s);
    case 3: return launch_tile_group<32, 1>(a, done, L.S - done, nt, s);
    default: return launch_tile_group<16, 1>(a, done, L.S - done, nt, s);
    }
}

fbp_status launch_forward(const FwdLaunch &L, cudaStream_t s)
{
    if (L.S <= 0) return FBP_OK;
    int v = L.variant;
    if (v < 0) v = fwd_tile_eligible(L.alpha) ? 4 : 0;      // four slices per block measured fastest
    if (v >= fwd_variant_count()) return fail(FBP_ERR_INVALID_ARG, "forward variant %d out of range", v);
    if (v > 0) return launch_forward_tile(L, v, s);
    FwdArgs a;
    a.slice = L.slice;
    a.sino = L.sino;
    a.cs = L.cs;
    a.K = L.K;
    a.D = L.D;
    a.N = L.N;
    a.alpha = L.alpha;
    a.det_center = L.det_center;
    a.bins_blocks = (L.D + kBins - 1) / kBins;
    const long long blocks = (long long)a.bins_blocks * L.K;
    if (blocks > 0x7fffffffLL) return fail(FBP_ERR_UNSUPPORTED, "too many projection bins");
    // worst-case candidates per line: ceil(2 / (alpha / sqrt 2))
    const int ncmax = (int)std::ceil(2.0 * 1.4142135623730951 / L.alpha);
    const int nct = ncmax <= 4 ? 4 : 24;
    a.span_pitch = fwd_span_pitch(L.alpha, nct);
    const size_t smem = (size_t)kLines * a.span_pitch * sizeof(float);
    if (a.span_pitch) {
        const void *kern = nct == 4 ? reinterpret_cast<const void *>(fwd_strip_kernel<4>)
                                    : reinterpret_cast<const void *>(fwd_strip_kernel<24>);
        fbp_status st = ensure_dynamic_smem(kern, smem);
        if (st != FBP_OK) return st;
    }
    for (int base = 0; base < L.S; base += 65535) {
        a.slice_base = base;
        dim3 grid((unsigned)blocks, (unsigned)std::min(65535, L.S - base));
        if (a.span_pitch) {
            if (nct == 4) fwd_strip_kernel<4><<<grid, kBins, smem, s>>>(a);
            else fwd_strip_kernel<24><<<grid, kBins, smem, s>>>(a);
        } else {
            if (nct == 4) fwd_kernel<4><<<grid, 128, 0, s>>>(a);
            else fwd_kernel<24><<<grid, 128, 0, s>>>(a);
        }
        FBP_CUDA_TRY(cudaGetLastError());
    }
    return FBP_OK;
}

}  // namespace fbp
