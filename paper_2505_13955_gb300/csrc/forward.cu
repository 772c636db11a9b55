// forward.cu -- K3: the matched forward projector A, the exact transpose of
// the backprojection with linear interpolation (scale 1):
//   (A f)_k[j] = sum_{r,c} f[r][c] * max(0, 1 - |u_k(r,c) - j|).
// (The paper's simulated data come from a forward model, Sec. V-B(a); here
// the projector is written as the adjoint of the library's own backprojector,
// so that least-squares refinement has the exact gradient.)
//
// Gather form, one thread per output bin (k, j), no atomics, deterministic:
// the thread walks the image along the axis where |cos| or |sin| is smaller
// (rows when |cos th| >= |sin th|) and, on each line of that axis, visits the
// few pixels whose coordinate lies within one bin of j.  Along the solved
// axis the support is 2/g pixels wide, g = alpha * max(|cos|, |sin|), so at
// most ceil(2/g) candidates contribute.  The position of the support on each
// line moves linearly; it is kept in 32.32 fixed point (exact integer adds),
// so the weights keep full precision over 8192 lines without FP64 per line:
//   xm(w) = B - slope * w   (first candidate = floor(xm) + 1)
//   weight_i = max(0, 1 - |g (delta + i) - 1|), delta = 1 - frac(xm).
// B and slope are formed once per thread in FP64 from the FP64 angle table.
//
// A block covers 128 consecutive bins of one angle; their candidates on 32
// consecutive lines lie in one strip of the image, which the block stages in
// shared memory with coalesced loads (rows of the strip for the row walk,
// 32-column segments for the column walk, transposed into shared memory), so
// every candidate is a shared-memory read.  Pixels outside the image are
// staged as zeros.  Geometries whose strip would not fit (pixel_size /
// det_spacing < 1/4) use the same walk with direct global loads.
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

fbp_status launch_forward(const FwdLaunch &L, cudaStream_t s)
{
    if (L.S <= 0) return FBP_OK;
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
