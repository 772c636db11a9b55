// runtime.cu -- the host-side runtime of libfbp.so: error reporting, the
// device status word, geometry validation, and the per-device cache of
// constant tables (angle table, filter spectrum, FFT twiddles), which are
// computed on the device in double precision.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fbp_internal.cuh"

namespace fbp {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local char tl_msg[512] = "";

fbp_status fail(fbp_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(tl_msg, sizeof(tl_msg), fmt, ap);
    va_end(ap);
    return st;
}

fbp_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(FBP_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e),
                cudaGetErrorName(e));
}

void clear_error() { tl_msg[0] = '\0'; }

// ---------------------------------------------------------------------------
// Device status word
// ---------------------------------------------------------------------------
__device__ unsigned g_fbp_device_status;

fbp_status device_status_word(unsigned **out)
{
    static std::mutex mu;
    static std::map<int, unsigned *> addr;
    int dev = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = addr.find(dev);
    if (it == addr.end()) {
        void *p = nullptr;
        FBP_CUDA_TRY(cudaGetSymbolAddress(&p, g_fbp_device_status));
        it = addr.emplace(dev, static_cast<unsigned *>(p)).first;
    }
    *out = it->second;
    return FBP_OK;
}

bool stream_is_capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st != cudaStreamCaptureStatusNone;
}

fbp_status ensure_dynamic_smem(const void *func, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> done;
    int dev = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = done[std::make_pair(dev, func)];
    if (cur >= bytes) return FBP_OK;
    FBP_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return FBP_OK;
}

fbp_status blocks_per_sm(const void *func, int threads, size_t smem, int *out)
{
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> done;
    int dev = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(dev, func, threads, smem);
    auto it = done.find(key);
    if (it == done.end()) {
        int n = 0;
        FBP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, threads, smem));
        it = done.emplace(key, n).first;
    }
    *out = it->second;
    return FBP_OK;
}

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
fbp_status check_geometry(const fbp_geometry *g, bool for_filter, bool for_projection)
{
    if (!g) return fail(FBP_ERR_INVALID_ARG, "geometry is NULL");
    if (g->n_angles < 1 || g->n_det < 1 || g->n < 1)
        return fail(FBP_ERR_INVALID_ARG, "n_angles, n_det and n must be >= 1 (got %d, %d, %d)",
                    g->n_angles, g->n_det, g->n);
    if (!std::isfinite(g->angle_start) || !std::isfinite(g->angle_step) ||
        !std::isfinite(g->det_center) || !std::isfinite(g->det_spacing) ||
        !std::isfinite(g->pixel_size))
        return fail(FBP_ERR_INVALID_ARG, "geometry has a non-finite field");
    if (!(g->det_spacing > 0.0) || !(g->pixel_size > 0.0))
        return fail(FBP_ERR_INVALID_ARG, "det_spacing and pixel_size must be > 0");
    if (g->n_angles > (1 << 24))
        return fail(FBP_ERR_UNSUPPORTED, "n_angles > 2^24");
    if (for_filter && g->n_det > 8192)
        return fail(FBP_ERR_UNSUPPORTED, "n_det = %d > 8192 (filter transform limit)", g->n_det);
    if (for_projection) {
        double alpha = g->pixel_size / g->det_spacing;
        if (alpha < 0.125 || alpha > 2.5)
            return fail(FBP_ERR_UNSUPPORTED,
                        "pixel_size/det_spacing = %g outside [0.125, 2.5]", alpha);
        if (g->n > 65536 || g->n_det > (1 << 20))
            return fail(FBP_ERR_UNSUPPORTED, "n > 65536 or n_det > 2^20");
        // detector coordinates must stay far inside int range
        double umax = alpha * 0.7072 * (double)g->n + std::fabs(g->det_center) + g->n_det;
        if (umax > (double)(1 << 28))
            return fail(FBP_ERR_UNSUPPORTED, "detector coordinates out of range");
    }
    return FBP_OK;
}

int bp_window_half(double alpha, int tile_w, int tile_h)
{
    double hx = 0.5 * (tile_w - 1), hy = 0.5 * (tile_h - 1);
    double delta = alpha * std::sqrt(hx * hx + hy * hy);
    // |u'| <= 0.5 + delta, i = rne(u') => |i| <= floor(delta) + 1; +1 more for
    // FP32 rounding of the in-tile offsets.
    return (int)std::ceil(delta) + 2;
}

// ---------------------------------------------------------------------------
// Table kernels (double precision)
// ---------------------------------------------------------------------------
__global__ void angle_table_kernel(double2 *cs, int K, double start, double step)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double s, c;
    sincos(start + (double)k * step, &s, &c);
    cs[k] = make_double2(c, s);
}

// The filter's twiddle plan for length L = R C (layout in fbp_internal.cuh),
// each entry exp(-2 pi i x / M) rounded once from double.
__global__ void twiddle_kernel(float2 *tw, int L, int R, int C)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= L + C + 32) return;
    long long x;
    int M;
    if (o < L) {                       // W_L^{t k1}
        x = (long long)(o % C) * (o / C);
        M = L;
    } else if (o < L + C) {            // W_C^{l kr}
        const int i = o - L;
        x = (long long)(i % 32) * (i / 32);
        M = C;
    } else {                           // W_32^m
        x = o - L - C;
        M = 32;
    }
    double s, c;
    sincospi(2.0 * (double)(x % M) / (double)M, &s, &c);
    tw[o] = make_float2((float)c, (float)-s);
}

// Filter taps h_tau(n), n in [0, D) (the kernel is even), double precision.
__global__ void taps_kernel(double *h, int D, int kind, double tau)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= D) return;
    const double pi2 = 9.8696044010893586188344909998762;  // pi^2
    double t2 = tau * tau, v;
    if (kind == FBP_FILTER_RAMLAK) {
        if (n == 0) v = 1.0 / (4.0 * t2);
        else if ((n & 1) == 0) v = 0.0;
        else v = -1.0 / (pi2 * (double)n * (double)n * t2);
    } else {
        v = -2.0 / (pi2 * t2 * (4.0 * (double)n * (double)n - 1.0));
    }
    h[n] = v;
}

__global__ void cos_table_kernel(double *c, int L)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L) return;
    c[m] = cospi(2.0 * (double)m / (double)L);
}

// Hr[k] = h(0) + 2 sum_{n=1}^{D-1} h(n) cos(2 pi k n / L): the (real, even)
// L-point DFT of the truncated kernel laid out circularly, in double.
__global__ void spectrum_kernel(double *Hr, const double *h, const double *ctab, int D, int L,
                                int kind)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > L / 2) return;
    double acc = 0.0;
    const int mask = L - 1;
    const int nstep = (kind == FBP_FILTER_RAMLAK) ? 2 : 1;   // Ram-Lak: only odd n
    for (int n = 1; n < D; n += nstep) {
        int m = (int)(((long long)k * n) & mask);
        acc = fma(h[n], ctab[m], acc);
    }
    const double v = h[0] + 2.0 * acc;
    Hr[k] = v;
    if (k > 0 && k < L / 2) Hr[L - k] = v;
}

// Spectrum of the difference-form kernel.  The filter is applied to the
// first differences d[m] = p[m] - p[m-1] (m in [0, D], p = 0 outside) with
// the cumulative kernel g[n] = sum_{k <= n} h(k), n in [-D, D-1]; summation by
// parts gives the same linear convolution, but the FP32 transform's rounding
// then scales with |d| instead of |p| (line integrals are large and the ramp
// filter removes most of their magnitude).  On the circle of length L >= 2D,
// G (1 - W^k) = H - DC W^{kD} with W = exp(-2 pi i / L), DC = sum h = H(0),
// so G[k] = (H[k] - DC W^{kD}) / (1 - W^k) for k > 0, and G[0] = D * DC
// (h is even).  Stored as (tau / L) G in float2.
__global__ void diff_spectrum_kernel(float2 *G, const double *Hr, int D, int L, double tau)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= L) return;
    // stored in the order step 2 of the transform reads it:
    // o = ((w NRD + rd) RB + m) 32 + j for warp w, round rd, value m of lane
    // j; RB = min(R, 16) values per lane, NRD = R / RB rounds.  Lane j works
    // on transform c = rd RB + j mod RB (row k1 = w (R / VPL) + c / VPL,
    // kr = c mod VPL) and holds kl = m + RB brev(s), s = j / RB
    const int R = fft_R(L), VPL = fft_VPL(L);
    const int RB = R < 16 ? R : 16, NRD = R / RB;
    const int j = o & 31, m = (o >> 5) % RB, rd = (o / (32 * RB)) % NRD, w = o / (32 * R);
    const int c = rd * RB + j % RB, s = j / RB;
    const int k1 = w * (R / VPL) + c / VPL, kr = c % VPL;
    const int sbits = __ffs(32 / RB) - 1;                     // log2 (32 / RB) >= 1
    const int q = (int)(__brev((unsigned)s) >> (32 - sbits));
    const int k = k1 + R * (kr + VPL * (m + RB * q));
    const double dc = Hr[0];
    double gr, gi;
    if (k == 0) {
        gr = (double)D * dc;
        gi = 0.0;
    } else {
        double s1, c1, sD, cD;
        sincospi(2.0 * (double)k / (double)L, &s1, &c1);                            // W^k = c1 - i s1
        sincospi(2.0 * (double)(((long long)k * D) % L) / (double)L, &sD, &cD);     // W^{kD}
        const double nr = Hr[k] - dc * cD, ni = dc * sD;                            // H - DC W^{kD}
        const double dr = 1.0 - c1, di = s1;                                        // 1 - W^k
        const double den = dr * dr + di * di;
        gr = (nr * dr + ni * di) / den;
        gi = (ni * dr - nr * di) / den;
    }
    const double sc = tau / (double)L;
    G[o] = make_float2((float)(gr * sc), (float)(gi * sc));
}

// ---------------------------------------------------------------------------
// Table cache
// ---------------------------------------------------------------------------
namespace {

struct FilterEntry {
    float2 *G = nullptr;      // L complex
    double *scratch = nullptr;
    int L = 0;
};

std::mutex g_mu;
std::map<std::tuple<int, int, uint64_t, uint64_t>, double2 *> g_angles;      // (dev, K, start, step)
std::map<std::tuple<int, int, int, uint64_t>, FilterEntry> g_filters;      // (dev, D, kind, tau)
std::map<std::pair<int, int>, float2 *> g_twiddles;                          // (dev, L)

uint64_t bits(double d)
{
    uint64_t u;
    std::memcpy(&u, &d, sizeof(u));
    return u;
}

}  // namespace

int filter_length(int D)
{
    if (D < 1 || D > 8192) return 0;
    int L = 512;
    while (L < 2 * D - 1) L <<= 1;
    return L;
}

cudaError_t enqueue_angle_table(double2 *cs, int K, double start, double step, cudaStream_t s)
{
    if (K <= 0) return cudaSuccess;
    angle_table_kernel<<<(K + 255) / 256, 256, 0, s>>>(cs, K, start, step);
    return cudaGetLastError();
}

fbp_status angle_table(const fbp_geometry &g, cudaStream_t s, const double2 **out)
{
    int dev = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    auto key = std::make_tuple(dev, g.n_angles, bits(g.angle_start), bits(g.angle_step));
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_angles.find(key);
    if (it != g_angles.end()) {
        *out = it->second;
        return FBP_OK;
    }
    if (stream_is_capturing(s))
        return fail(FBP_ERR_UNSUPPORTED,
                    "angle table for K=%d not built yet; call fbp_prepare (or run once) before stream capture",
                    g.n_angles);
    double2 *p = nullptr;
    FBP_CUDA_TRY(cudaMalloc(&p, sizeof(double2) * (size_t)g.n_angles));
    cudaError_t e = enqueue_angle_table(p, g.n_angles, g.angle_start, g.angle_step, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_fail(e, "angle_table_kernel");
    }
    g_angles.emplace(key, p);
    *out = p;
    return FBP_OK;
}

fbp_status filter_tables(int D, int kind, double tau, cudaStream_t s,
                         const float2 **G, const float2 **tw, int *Lout)
{
    int L = filter_length(D);
    if (!L) return fail(FBP_ERR_UNSUPPORTED, "n_det = %d outside [1, 8192]", D);
    int dev = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_mu);
    auto fkey = std::make_tuple(dev, D, kind, bits(tau));
    auto tkey = std::make_pair(dev, L);
    auto fit = g_filters.find(fkey);
    auto tit = g_twiddles.find(tkey);
    if (fit != g_filters.end() && tit != g_twiddles.end()) {
        *G = fit->second.G;
        *tw = tit->second;
        *Lout = L;
        return FBP_OK;
    }
    if (stream_is_capturing(s))
        return fail(FBP_ERR_UNSUPPORTED,
                    "filter tables for n_det=%d not built yet; call fbp_prepare (or run once) before stream capture",
                    D);
    if (tit == g_twiddles.end()) {
        float2 *t = nullptr;
        const int C = 32 * fft_VPL(L), n = L + C + 32;
        FBP_CUDA_TRY(cudaMalloc(&t, sizeof(float2) * (size_t)n));
        twiddle_kernel<<<(n + 255) / 256, 256, 0, s>>>(t, L, fft_R(L), C);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(t);
            return cuda_fail(e, "twiddle_kernel");
        }
        tit = g_twiddles.emplace(tkey, t).first;
    }
    if (fit == g_filters.end()) {
        FilterEntry fe;
        fe.L = L;
        FBP_CUDA_TRY(cudaMalloc(&fe.G, sizeof(float2) * (size_t)L));
        cudaError_t e = cudaMalloc(&fe.scratch, sizeof(double) * ((size_t)D + 2 * (size_t)L));
        if (e != cudaSuccess) {
            cudaFree(fe.G);
            return cuda_fail(e, "cudaMalloc(filter scratch)");
        }
        double *h = fe.scratch, *ctab = fe.scratch + D, *Hr = fe.scratch + D + L;
        taps_kernel<<<(D + 255) / 256, 256, 0, s>>>(h, D, kind, tau);
        cos_table_kernel<<<(L + 255) / 256, 256, 0, s>>>(ctab, L);
        spectrum_kernel<<<(L / 2 + 1 + 127) / 128, 128, 0, s>>>(Hr, h, ctab, D, L, kind);
        diff_spectrum_kernel<<<(L + 255) / 256, 256, 0, s>>>(fe.G, Hr, D, L, tau);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(fe.scratch);
        fe.scratch = nullptr;
        if (e != cudaSuccess) {
            cudaFree(fe.G);
            return cuda_fail(e, "spectrum_kernel");
        }
        fit = g_filters.emplace(fkey, fe).first;
    }
    *G = fit->second.G;
    *tw = tit->second;
    *Lout = L;
    return FBP_OK;
}

void release_tables()
{
    std::lock_guard<std::mutex> lock(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    auto on = [&](int dev) { cudaSetDevice(dev); cudaDeviceSynchronize(); };
    for (auto &kv : g_angles) { on(std::get<0>(kv.first)); cudaFree(kv.second); }
    for (auto &kv : g_filters) { on(std::get<0>(kv.first)); cudaFree(kv.second.G); }
    for (auto &kv : g_twiddles) { on(kv.first.first); cudaFree(kv.second); }
    g_angles.clear();
    g_filters.clear();
    g_twiddles.clear();
    cudaSetDevice(cur);
    cudaGetLastError();
}

}  // namespace fbp

extern "C" const char *fbp_last_error_message(void) { return fbp::tl_msg; }
