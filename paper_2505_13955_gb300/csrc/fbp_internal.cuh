// fbp_internal.cuh -- declarations shared by the translation units of
// libfbp.so (never by the oracle, which is a separate program).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "fbp.h"

namespace fbp {

// ---------------------------------------------------------------------------
// Error reporting (thread-local message; see fbp_last_error_message()).
// ---------------------------------------------------------------------------
fbp_status fail(fbp_status st, const char *fmt, ...);
fbp_status cuda_fail(cudaError_t e, const char *what);
#define FBP_CUDA_TRY(call)                                              \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::fbp::cuda_fail(e_, #call);      \
    } while (0)

// Device status word: kernels record fault codes here instead of trapping.
enum DeviceFault : unsigned {
    FAULT_NONE = 0,
    FAULT_QUEUE_CAP = 1,      // persistent work loop ran past its iteration cap
    FAULT_TABLE_INDEX = 2,    // checked build: interpolation index outside the staged window
    FAULT_RESERVED_3 = 3,     // unused: transform lengths are checked on the host
    FAULT_UNION_CAP = 4,      // patching: a union-find loop ran past its cap
    FAULT_LEAF = 5,           // patching: a quadtree leaf entry outside the slice
    FAULT_STREAM_WAIT = 6,    // streamed filter: a wait for its row copy ran past its cap
    FAULT_BP_STAGE_WAIT = 7,  // bulk-copy-fed backprojection: a wait for a window copy ran past its cap
    FAULT_BP_WINDOW = 8,      // staged batch: a window outside its item's padded table (copy clamped)
};
fbp_status device_status_word(unsigned **out);   // current device

// ---------------------------------------------------------------------------
// Constant tables, built on the device in FP64 and cached per device.
// ---------------------------------------------------------------------------
struct AngleKey {
    int K;
    double start, step;
};
// cos/sin of theta_k = start + k*step, k in [0, K), in double precision.
fbp_status angle_table(const fbp_geometry &g, cudaStream_t s, const double2 **out);
// The kernel behind angle_table, enqueued on s into caller-owned cs[K]
// (returns the launch's error; allocates nothing).
cudaError_t enqueue_angle_table(double2 *cs, int K, double start, double step, cudaStream_t s);

// Filter transform shape: L = R * C, C = 32 * VPL threads per row pair
// (n = C n1 + n2, k = k1 + R k2, k2 = kr + VPL kl; see filter.cu).
__host__ __device__ constexpr int fft_R(int L)
{
    return L == 512 ? 4 : L <= 2048 ? 8 : L <= 8192 ? 16 : 32;
}
__host__ __device__ constexpr int fft_VPL(int L)
{
    return L <= 1024 ? 4 : L <= 4096 ? 8 : 16;
}

// Filter tables for detector width D:
//   L   = transform length (power of two >= max(512, 2D-1), so L >= 2D; <= 16384)
//   G   = spectrum of the cumulative (difference-form) kernel, times tau / L,
//         complex, in the order the transform's step 2 reads it:
//         G[((w NRD + rd) RB + m) 32 + j] = spectrum at
//         k = k1 + R (kr + VPL (m + RB brev(s))) for warp w, round rd < NRD,
//         lane j, RB = min(R, 16), NRD = R / RB: c = rd RB + j mod RB,
//         s = j / RB, k1 = w (R / VPL) + c / VPL, kr = c mod VPL, and brev
//         the log2(32 / RB)-bit reversal
//   tw  = twiddle plan (float2), L + C + 32 entries: W_L^{t k1} at k1 C + t,
//         then W_C^{l kr} at L + 32 kr + l, then W_32^m at L + C + m,
//         W_M^x = exp(-2 pi i x / M), each rounded once from double
fbp_status filter_tables(int D, int kind, double tau, cudaStream_t s,
                         const float2 **G, const float2 **tw, int *L);
int filter_length(int D);   // 0 if D is outside [1, 8192]

bool stream_is_capturing(cudaStream_t s);

// Per-device, per-kernel caches of launch attributes, so that a call repeated
// inside stream capture only enqueues work.
fbp_status ensure_dynamic_smem(const void *func, size_t bytes);
fbp_status blocks_per_sm(const void *func, int threads, size_t smem, int *out);

// ---------------------------------------------------------------------------
// Geometry validation shared by the entry points.
// ---------------------------------------------------------------------------
fbp_status check_geometry(const fbp_geometry *g, bool for_filter, bool for_projection);

// Half-width H of the detector window one backprojection tile needs:
// every tile pixel's interpolation index lies in [-H, H] around the tile
// centre's bin.  Returns -1 if the window would exceed max_w entries.
int bp_window_half(double alpha, int tile_w, int tile_h);

// ---------------------------------------------------------------------------
// Kernel launchers (defined next to their kernels).
// ---------------------------------------------------------------------------
// Stage-2 pre-processing fused into the filter's load (counts -> blurred
// line integrals); taps w_{-r..r} of the Gaussian, rounded once from double.
struct FilterPre {
    const float *flat;     // per-bin I0 [D] (device) or null
    float flat_value, floor, mu_scale;
    int blur_radius;       // r <= 16
    float taps[33];
};

// Offset scans: rows of Dp physical bins weighted and embedded in the
// transform's virtual detector (physical bin m at virtual bin m + off),
// optionally folded with the row half a turn later (see filter.cu).
struct FilterOffset {
    int Dp, off, fold;
    long long K_in;        // physical rows per slice (even with fold)
    float cv, sgn, inv_delta;
};

struct FilterLaunch {
    const float *sino;     // [rows][D] line integrals, or counts when pre is set
    void *filt;            // [rows][D] of dtype
    float *row_scale;      // [rows] (16-bit dtypes)
    long long rows;        // n_slices * K
    int D, L;
    const float2 *G;
    const float2 *tw;
    fbp_dtype dtype;
    const FilterPre *pre = nullptr;
    const FilterOffset *offset = nullptr;   // rows = output rows; sino is [S][K_in][Dp]
};
fbp_status launch_filter(const FilterLaunch &a, cudaStream_t s);

struct BpLaunch {
    const void *filt;        // [S][K][D]
    const float *row_scale;  // [S][K] or null
    float *slice;            // [S][N][N]
    const double2 *cs;       // [K]
    int K, D, N, S;
    double alpha, det_center;
    double angle_step;       // for the symmetric (orbit) kernels' eligibility
    float scale;
    int accumulate;
    fbp_dtype dtype;
    unsigned short *slice16 = nullptr;   // uint16 CT-number codes instead of `slice`
    float hu_a = 0.f, hu_b = 0.f;        // code = clamp(rint(RN(RN(hu_a * mu) + hu_b)))
    int split = 0;                       // orbit kernels may split small slices' angle pairs (default path)
};
fbp_status launch_backproject(const BpLaunch &a, int variant, cudaStream_t s);
bool bp_orbit_eligible(const BpLaunch &a, int tile);
bool bp_variant_fits(int variant, const BpLaunch &a);   // geometry + shared-memory budget
int orbit_split_parts(long long orbits, int K2, int KT, long long resident);
fbp_status device_sm_count(int *out);                    // current device, cached
int bp_default_variant(const BpLaunch &a);
int bp_variant_count();
bool bp_variant_shape(int v, fbp_bp_shape *out);
size_t bp_smem_bytes(int v, int W);
// The texture-unit variant (bp_texture.cu): eligibility and launch.  The
// launch synchronises `s` before releasing its texture objects.
bool bp_texture_shape_ok(const BpLaunch &a);
fbp_status launch_backproject_texture(const BpLaunch &a, cudaStream_t s);

struct FwdLaunch {
    const float *slice;   // [S][N][N]
    float *sino;          // [S][K][D]
    const double2 *cs;
    int K, D, N, S;
    double alpha, det_center;
    int variant;          // -1 default, 0 gather, 1..3 tile-owned (8 / 16 / 32 bins per warp)
};
fbp_status launch_forward(const FwdLaunch &a, cudaStream_t s);
int fwd_variant_count();
bool fwd_tile_eligible(double alpha);

}  // namespace fbp
