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
#include <cmath>

#include "fbp_internal.cuh"

namespace fbp {
namespace {

struct FwdArgs {
    const float *slice;
    float *sino;
    const double2 *cs;
    int K, D, N;
    double alpha, det_center;
    int bins_blocks;     // ceil(D / 128)
    int slice_base;
};

template <int NCMAX>
__global__ void __launch_bounds__(128) fwd_kernel(FwdArgs a)
{
    const int k = blockIdx.x / a.bins_blocks;
    const int j = (blockIdx.x % a.bins_blocks) * 128 + threadIdx.x;
    const int sl = a.slice_base + blockIdx.y;
    if (j >= a.D) return;
    const int N = a.N;
    const float *f = a.slice + (size_t)sl * N * N;

    const double2 cs = a.cs[k];
    const bool walk_rows = fabs(cs.x) >= fabs(cs.y);
    const double cp = a.alpha * (walk_rows ? cs.x : cs.y);   // along the solved axis
    const double cq = a.alpha * (walk_rows ? cs.y : cs.x);   // along the walked axis
    const double g = fabs(cp);
    const double h = 1.0 / g;
    const int nc = min(NCMAX, (int)ceil(2.0 * h));
    const double m = 0.5 * (N - 1);
    const double slope = cq / cp;
    const double B = ((double)j - a.det_center + cq * m) / cp + m - h;

    // lines w on which some candidate can fall inside [0, N); the bounds are
    // clamped in double before conversion (near th = pi/2 the slope is ~1e-17
    // and the unclamped quotients overflow int)
    double lo_d = 0.0, hi_d = (double)(N - 1);
    if (slope > 0.0) {
        lo_d = fmax(lo_d, floor((B - N) / slope) - 1.0);
        hi_d = fmin(hi_d, ceil((B + nc + 1) / slope) + 1.0);
    } else if (slope < 0.0) {
        lo_d = fmax(lo_d, floor((B + nc + 1) / slope) - 1.0);
        hi_d = fmin(hi_d, ceil((B - N) / slope) + 1.0);
    } else if (!(B > -nc - 1.0 && B < (double)N)) {
        hi_d = -1.0;
    }
    lo_d = fmin(lo_d, (double)N);     // both now lie in [-1, N]
    hi_d = fmax(hi_d, -1.0);
    const int w0 = (int)lo_d, w1 = (int)hi_d;

    float acc = 0.f;
    if (w0 <= w1) {
        const double two32 = 4294967296.0;
        long long XM = __double2ll_rn((B - slope * (double)w0) * two32);
        const long long SL = __double2ll_rn(slope * two32);
        const float gf = (float)g;
        for (int w = w0; w <= w1; ++w) {
            const int start = (int)(XM >> 32) + 1;
            const unsigned lo = (unsigned)(XM & 0xffffffffLL);
            const float delta = 2.0f - __uint_as_float(0x3f800000u | (lo >> 9));
            const float gd = gf * delta;
#pragma unroll
            for (int i = 0; i < NCMAX; ++i) {
                if (i < nc) {
                    const int col = start + i;
                    const float wgt = fmaxf(0.f, 1.f - fabsf(fmaf(gf, (float)i, gd) - 1.f));
                    if ((unsigned)col < (unsigned)N) {
                        const float v = walk_rows ? __ldg(f + (size_t)w * N + col)
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

}  // namespace

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
    a.bins_blocks = (L.D + 127) / 128;
    const long long blocks = (long long)a.bins_blocks * L.K;
    if (blocks > 0x7fffffffLL) return fail(FBP_ERR_UNSUPPORTED, "too many projection bins");
    // worst-case candidates per line: ceil(2 / (alpha / sqrt 2))
    const int ncmax = (int)std::ceil(2.0 * 1.4142135623730951 / L.alpha);
    for (int base = 0; base < L.S; base += 65535) {
        a.slice_base = base;
        dim3 grid((unsigned)blocks, (unsigned)std::min(65535, L.S - base));
        if (ncmax <= 4) fwd_kernel<4><<<grid, 128, 0, s>>>(a);
        else fwd_kernel<24><<<grid, 128, 0, s>>>(a);
        FBP_CUDA_TRY(cudaGetLastError());
    }
    return FBP_OK;
}

}  // namespace fbp
