// bp_staged.cu -- K2 with the window staging taken off the threads:
// fbp_backproject_staged (FP32 and 16-bit rows) and its uint16-code form.
//
// The orbit kernel (bp_orbit.cuh) forms, per block, per angle pair and per
// window, the table entries (midpoints and slopes of the rows th, th + pi/2
// and their mirrors; 16-bit rows scaled by s_k / S) from the filtered rows,
// behind two block barriers per stage.  Here a pass over the filtered rows
// writes those entries once per slice, for every detector segment, into the
// caller's workspace:
//     table[s][k][e], k < K/2 the angle pair, e = j + 1 for segment j in
//     [-1, D-1] (the segment between bins j and j+1, zero outside [0, D)),
//     16 bytes per entry for 16-bit rows, 32 for FP32 rows (two 16-byte
//     halves: rows th, th' | mirrored rows),
// and the backprojection moves each window of W entries with one tiled
// bulk-tensor copy per half into shared memory -- out-of-range entries
// (windows that reach past the detector) are filled with zeros by the copy
// engine, which is exactly the staged kernel's zero padding.  Stages cycle
// through NS buffers; each copy completes on the buffer's mbarrier (capped
// waits), and the last warp to finish reading a buffer refills it with the
// stage NS ahead, so the compute loop has no block-wide barrier.  For 16-bit
// rows the entries and the per-pair arithmetic (orbit_mid_slope, orbit_pair)
// are the orbit kernel's own, so the results are bit-identical to
// fbp_backproject_variant with the same shape; FP32 rows use the midpoint
// form (orbit_pair_mid), within FP32 rounding of the orbit kernel.  The
// device code shared with the batched form (bp_staged_batch.cu) is in
// bp_staged.cuh.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "bp_batch.cuh"
#include "bp_staged.cuh"

namespace fbp {
void clear_error();
}

namespace fbp {
namespace {

// S of each slice: the largest row scale (1 if none is positive), as the
// orbit kernel forms it.
__global__ void slice_scale_kernel(const float *row_scale, int K, float *smax)
{
    __shared__ float red[32];
    const float *rs = row_scale + (size_t)blockIdx.x * K;
    float mx = 0.f;
    for (int k = threadIdx.x; k < K; k += blockDim.x) mx = fmaxf(mx, __ldg(rs + k));
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        mx = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
        smax[blockIdx.x] = mx > 0.f ? mx : 1.f;
    }
}

// One entry per thread: table[pair][e] for the chunk's S x K/2 pairs.
template <typename T, bool PACKED>
__global__ void orbit_prestage_kernel(const T *filt, const float *row_scale, const float *smax, uint4 *table,
                                      int K, int D, long long pairs)
{
    const int K2 = K / 2, E = D + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int jj = e - 1;                   // segment between bins jj and jj + 1
    for (long long p = blockIdx.y; p < pairs; p += gridDim.y) {
        const long long s = p / K2;
        const int k = (int)(p - s * K2);
        const T *r0 = filt + ((size_t)s * K + k) * D;
        const T *r1 = r0 + (size_t)K2 * D;
        const float invS = __frcp_rn(__ldg(smax + s));
        const float sc0 = __fmul_rn(__ldg(row_scale + (size_t)s * K + k), invS);
        const float sc1 = __fmul_rn(__ldg(row_scale + (size_t)s * K + k + K2), invS);
        const uint4 out = orbit_entry16<T, PACKED>(r0, r1, D, jj, sc0, sc1);
        table[(size_t)p * E + e] = out;
    }
}

// FP32 rows: 32-byte midpoint/slope entries (orbit_entry32), whose two
// 16-byte halves (rows th, th' | mirrored rows) land in separate shared
// arrays.
__global__ void orbit_prestage_f32_kernel(const float *filt, float4 *table, int K, int D, long long pairs)
{
    const int K2 = K / 2, E = D + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int jj = e - 1;
    for (long long p = blockIdx.y; p < pairs; p += gridDim.y) {
        const long long s = p / K2;
        const int k = (int)(p - s * K2);
        const float *r0 = filt + ((size_t)s * K + k) * D;
        const float *r1 = r0 + (size_t)K2 * D;
        float4 *o = table + ((size_t)p * E + e) * 2;
        orbit_entry32(r0, r1, D, jj, o[0], o[1]);
    }
}

struct StagedArgs {
    const double2 *cs;         // [K] angle table (k < K/2 is read)
    float *out;                // the chunk's first slice [N][N], or null when out16 is set
    unsigned short *out16;     // or the chunk's first slice of uint16 codes (bp_tile.cuh: store_pixel)
    float hu_a, hu_b;
    const float *smax;         // the chunk's S per slice
    int K2, N, H, W, Wp, orbits_x;
    double alpha, det_center;
    float scale;
    int accumulate;
    unsigned *status;
};

// CODES: the epilogue writes uint16 CT-number codes (out16) instead of FP32.
template <int TXT, int TYT, int PX, int PY, int KT, int NS, typename T, bool PACKED, int MINB, bool CODES>
__global__ void __launch_bounds__(TXT *TYT, MINB) bp_staged_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                   StagedArgs a)
{
    constexpr int NT = TXT * TYT, NW = NT / 32, TILE = TXT * PX, WX = TXT / 8;
    constexpr int HALVES = sizeof(T) == 4 ? 2 : 1;   // 16-byte halves per entry
    static_assert(TXT * PX == TYT * PY, "square tile");
    static_assert(KT <= 32 && NS >= 2 && NS <= 4, "stage shape");
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t base_s = (raw_s + 127u) & ~127u;
    unsigned char *base = smem_raw + (base_s - raw_s);
    const uint32_t full_s = base_s;                           // NS x 8 bytes
    int *done = reinterpret_cast<int *>(base + 8 * NS);
    int *issued = reinterpret_cast<int *>(base + 12 * NS);
    float4 *prm = reinterpret_cast<float4 *>(base + 128);
    const uint32_t tab0 = base_s + 128u + (uint32_t)staged_params_bytes<KT, NS>();
    const int H = a.H, W = a.W, Wp = a.Wp, K2 = a.K2;
    const uint32_t half_bytes = (uint32_t)(2 * KT * Wp * 16);   // one half-array of a stage
    const uint32_t stage_bytes = HALVES * half_bytes;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tx = (warp % WX) * 8 + (lane & 7);
    const int ty = (warp / WX) * 4 + (lane >> 3);
    const int sl = blockIdx.y;
    const int x0 = (int)(blockIdx.x % a.orbits_x) * TILE, y0 = (int)(blockIdx.x / a.orbits_x) * TILE;
    const double m = 0.5 * (a.N - 1);
    const double Xc = (double)x0 + 0.5 * (TILE - 1) - m;
    const double Yc = (double)y0 + 0.5 * (TILE - 1) - m;
    const float dxt = (float)tx - 0.5f * (TILE - 1);
    const float dyt = (float)ty - 0.5f * (TILE - 1);
    const int n_stages = (K2 + KT - 1) / KT;
    const long long zbase = (long long)sl * K2;

    // one warp fills buffer b with stage t: the pairs' parameters (FP64 base
    // coordinates, as bp_orbit) and two window copies per pair
    auto issue = [&](int t, int b) {
        const int k0 = t * KT, na = min(KT, K2 - k0);
        int jl1 = 0, jl2 = 0;
        if (lane < KT) {
            float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (lane < na) {
                const double2 cs = a.cs[k0 + lane];
                const double c = a.alpha * cs.x, s = a.alpha * cs.y;
                const double v1 = fma(c, Xc, fma(s, Yc, a.det_center));
                const double v2 = fma(-s, Xc, fma(c, Yc, a.det_center));
                const double jc1 = floor(v1), jc2 = floor(v2);
                pv = make_float4((float)c, (float)s, (float)(v1 - jc1 - 0.5), (float)(v2 - jc2 - 0.5));
                jl1 = (int)jc1 - H;
                jl2 = (int)jc2 - H;
            }
            prm[b * KT + lane] = pv;
        }
        // the block's earlier reads of buffer b (ordered before this warp by
        // the done counter) come before the copy engine's writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        const uint32_t mbar = full_s + 8u * b;
        if (lane == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         ::"r"(mbar), "r"((uint32_t)(na * 2 * W * 16 * HALVES)) : "memory");
            issued[b] += 1;
        }
        __syncwarp();
        if (lane != 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
        if (lane < na) {
            const uint32_t dst = tab0 + (uint32_t)b * stage_bytes + (uint32_t)(2 * lane * Wp * 16);
            const int z = (int)(zbase + k0 + lane);
            const unsigned long long map = reinterpret_cast<unsigned long long>(&tmap);
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                         " [%0], [%1, {%2, %3, %4}], [%5];"
                         ::"r"(dst), "l"(map), "r"(0), "r"(jl1 + 1), "r"(z), "r"(mbar) : "memory");
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                         " [%0], [%1, {%2, %3, %4}], [%5];"
                         ::"r"(dst + (uint32_t)(Wp * 16)), "l"(map), "r"(0), "r"(jl2 + 1), "r"(z), "r"(mbar)
                         : "memory");
            if constexpr (HALVES == 2) {
                // FP32: the entries' second halves (words 4..7) into the mirrored-row array
                asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                             " [%0], [%1, {%2, %3, %4}], [%5];"
                             ::"r"(dst + half_bytes), "l"(map), "r"(4), "r"(jl1 + 1), "r"(z), "r"(mbar)
                             : "memory");
                asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                             " [%0], [%1, {%2, %3, %4}], [%5];"
                             ::"r"(dst + half_bytes + (uint32_t)(Wp * 16)), "l"(map), "r"(4), "r"(jl2 + 1), "r"(z),
                               "r"(mbar)
                             : "memory");
            }
        }
    };

    if (tid == 0) {
        for (int b = 0; b < NS; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" ::"r"(full_s + 8u * b) : "memory");
            done[b] = 0;
            issued[b] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0)
        for (int t = 0; t < min(NS, n_stages); ++t) issue(t, t);

    float acc[4][PY][PX];
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int iy = 0; iy < PY; ++iy)
#pragma unroll
            for (int ix = 0; ix < PX; ++ix) acc[o][iy][ix] = 0.f;

    bool ok = true;
    for (int t = 0; t < n_stages; ++t) {
        const int b = t % NS;
        if (!staged_wait(full_s + 8u * b, (unsigned)((t / NS) & 1))) {
            ok = false;
            break;
        }
        const int na = min(KT, K2 - t * KT);
        const uint32_t tabb = tab0 + (uint32_t)b * stage_bytes;
        for (int p = 0; p < na; ++p) {
            const uint32_t cb1 = tabb + 16u * (uint32_t)(2 * p * Wp + H) - 16u * kRoundMagicBits;
            const uint32_t cb2 = cb1 + 16u * (uint32_t)Wp;
            if constexpr (HALVES == 2)
                orbit_pair_mid<TXT, TYT, PX, PY>(acc, prm[b * KT + p], cb1, cb2, half_bytes, dxt, dyt);
            else
                orbit_pair<TXT, TYT, PX, PY, T, false, PACKED>(acc, prm[b * KT + p], cb1, cb2, 0u, dxt, dyt, H,
                                                               a.status);
        }
        // release buffer b; the last warp to do so refills it with stage t + NS
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&done[b], 1) == NW - 1;
            if (last) {
                done[b] = 0;
                __threadfence_block();
            }
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last && t + NS < n_stages) issue(t + NS, b);
    }
    const bool failed = __syncthreads_or(!ok);
    if (failed) {
        // a wait ran out: record it, let every copy this block started land
        // (capped) and write nothing
        if (tid == 0) {
            atomicCAS(a.status, 0u, (unsigned)FAULT_BP_STAGE_WAIT);
            for (int b = 0; b < NS; ++b)
                if (issued[b] > 0) staged_wait(full_s + 8u * b, (unsigned)((issued[b] - 1) & 1));
        }
        return;
    }
    const size_t so = (size_t)sl * a.N * a.N;
    const float S = HALVES == 2 ? 1.f : __ldg(a.smax + sl);
    if constexpr (CODES)
        orbit_store<TXT, TYT, PX, PY>(acc, nullptr, a.out16 + so, a.hu_a, a.hu_b, 0, a.N, x0 + tx, y0 + ty,
                                      a.scale * S);
    else
        orbit_store<TXT, TYT, PX, PY>(acc, a.out + so, nullptr, 0.f, 0.f, a.accumulate, a.N, x0 + tx, y0 + ty,
                                      a.scale * S);
}

// Compiled shapes.  16-bit rows: the orbit kernel's 64 x 64 (256 threads,
// 4 x 4 pixels) and 32 x 32 (128 threads, 2 x 4) tiles, packed pair
// arithmetic.  FP32 rows: 32-byte entries, so fewer pairs per stage keep
// several blocks per SM.
struct StagedShape {
    int txt, tyt, px, py, kt, ns, minb;
};
constexpr StagedShape kStagedShapes16[] = {
    {16, 16, 4, 4, 8, 3, 2},    // 0: 64 x 64 orbit, 8 pairs per stage, 3 buffers
    {16, 16, 4, 4, 16, 2, 2},   // 1: 64 x 64, 16 pairs, 2 buffers
    {16, 8, 2, 4, 16, 3, 4},    // 2: 32 x 32 orbit, 16 pairs, 3 buffers
    {16, 8, 2, 4, 8, 4, 4},     // 3: 32 x 32, 8 pairs, 4 buffers
    {16, 8, 2, 4, 8, 3, 5},     // 4: 32 x 32, 8 pairs, 3 buffers, five blocks per SM
    {16, 8, 2, 4, 8, 2, 6},     // 5: 32 x 32, 8 pairs, 2 buffers, six blocks per SM
};
constexpr StagedShape kStagedShapes32[] = {
    {16, 8, 2, 4, 4, 2, 6},     // 0: 32 x 32 orbit, 4 pairs per stage, 2 buffers, six blocks per SM
    {16, 8, 2, 4, 4, 3, 5},     // 1: 32 x 32, 4 pairs, 3 buffers, five blocks per SM
    {16, 8, 2, 4, 8, 2, 3},     // 2: 32 x 32, 8 pairs, 2 buffers, three blocks per SM
    {16, 16, 4, 4, 8, 2, 2},    // 3: 64 x 64, 8 pairs, 2 buffers, two blocks per SM
};
constexpr int kNumStagedShapes16 = sizeof(kStagedShapes16) / sizeof(kStagedShapes16[0]);
constexpr int kNumStagedShapes32 = sizeof(kStagedShapes32) / sizeof(kStagedShapes32[0]);

template <typename T> constexpr const StagedShape *staged_shapes()
{
    if constexpr (sizeof(T) == 4) return kStagedShapes32;
    else return kStagedShapes16;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

struct StagedLaunch {
    const void *filt;
    const float *row_scale;
    float *slice;
    unsigned short *slice16;   // uint16 codes instead of slice, or null
    float hu_a, hu_b;
    const double2 *cs;
    int K, D, N, S;
    double alpha, det_center;
    float scale;
    int accumulate;
    fbp_dtype dtype;
    char *ws;
    int chunk;                 // slices per pass through the workspace
};

size_t staged_table_bytes(int K, int D, fbp_dtype dtype)
{
    return (size_t)(K / 2) * (size_t)(D + 1) * (dtype == FBP_F32 ? 32 : 16);
}
size_t staged_scale_bytes(int chunk) { return ((size_t)chunk * 4 + 255) / 256 * 256; }

template <int V, typename T, bool CODES>
fbp_status launch_staged_t(const StagedLaunch &L, cudaStream_t s, unsigned *status)
{
    constexpr StagedShape sd = staged_shapes<T>()[V];
    constexpr int TILE = sd.txt * sd.px;
    constexpr bool kF32 = sizeof(T) == 4;
    constexpr int HALVES = kF32 ? 2 : 1;
    if (L.N % (2 * TILE) != 0) return fail(FBP_ERR_UNSUPPORTED, "n must be a multiple of %d", 2 * TILE);
    auto kern = bp_staged_kernel<sd.txt, sd.tyt, sd.px, sd.py, sd.kt, sd.ns, T, !kF32, sd.minb, CODES>;
    StagedArgs a;
    a.cs = L.cs;
    a.K2 = L.K / 2;
    a.N = L.N;
    a.H = bp_window_half(L.alpha, TILE, TILE);
    a.W = 2 * a.H + 1;
    a.Wp = (a.W + 7) / 8 * 8;
    if (a.H < 0 || a.W > 256) return fail(FBP_ERR_UNSUPPORTED, "backprojection window too wide for a bulk copy");
    a.orbits_x = L.N / TILE / 2;
    a.alpha = L.alpha;
    a.det_center = L.det_center;
    a.scale = L.scale;
    a.accumulate = L.accumulate;
    a.status = status;
    const size_t smem = staged_smem_bytes<sd.kt, sd.ns, HALVES>(a.Wp);
    if (smem > 220 * 1024) return fail(FBP_ERR_UNSUPPORTED, "backprojection window too wide");
    fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (st != FBP_OK) return st;
    auto encode = tensor_map_encoder();
    if (!encode) return fail(FBP_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const long long orbits = (long long)a.orbits_x * a.orbits_x;
    if (orbits > INT_MAX) return fail(FBP_ERR_UNSUPPORTED, "too many tiles");
    const int E = L.D + 1;
    float *smax = reinterpret_cast<float *>(L.ws);
    void *table = L.ws + staged_scale_bytes(L.chunk);
    const size_t kd = (size_t)L.K * L.D;
    for (int s0 = 0; s0 < L.S; s0 += L.chunk) {
        const int n = std::min(L.chunk, L.S - s0);
        const T *filt = static_cast<const T *>(L.filt) + (size_t)s0 * kd;
        const long long pairs = (long long)n * (L.K / 2);
        dim3 pg((unsigned)((E + 255) / 256), (unsigned)std::min<long long>(pairs, 65535));
        if constexpr (kF32) {
            // FP32 rows carry no scale: S = 1
            orbit_prestage_f32_kernel<<<pg, 256, 0, s>>>(reinterpret_cast<const float *>(filt),
                                                         static_cast<float4 *>(table), L.K, L.D, pairs);
            FBP_CUDA_TRY(cudaGetLastError());
        } else {
            const float *rs = L.row_scale + (size_t)s0 * L.K;
            slice_scale_kernel<<<n, 256, 0, s>>>(rs, L.K, smax);
            FBP_CUDA_TRY(cudaGetLastError());
            orbit_prestage_kernel<T, true><<<pg, 256, 0, s>>>(filt, rs, smax, static_cast<uint4 *>(table), L.K,
                                                              L.D, pairs);
            FBP_CUDA_TRY(cudaGetLastError());
        }
        // the chunk's table as a 3-D tensor of 32-bit words: {4 or 8 words, E entries, pairs}
        CUtensorMap map;
        const cuuint64_t words = 4 * HALVES;
        const cuuint64_t dims[3] = {words, (cuuint64_t)E, (cuuint64_t)pairs};
        const cuuint64_t strides[2] = {words * 4, (cuuint64_t)E * words * 4};
        const cuuint32_t box[3] = {4, (cuuint32_t)a.W, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        const CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, table, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return fail(FBP_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
        a.out = L.slice16 ? nullptr : L.slice + (size_t)s0 * L.N * L.N;
        a.out16 = L.slice16 ? L.slice16 + (size_t)s0 * L.N * L.N : nullptr;
        a.hu_a = L.hu_a;
        a.hu_b = L.hu_b;
        a.smax = kF32 ? nullptr : smax;
        dim3 grid((unsigned)orbits, (unsigned)n);
        kern<<<grid, sd.txt * sd.tyt, smem, s>>>(map, a);
        FBP_CUDA_TRY(cudaGetLastError());
    }
    return FBP_OK;
}

template <typename T, bool CODES>
fbp_status launch_staged_shape(const StagedLaunch &L, int v, cudaStream_t s, unsigned *status)
{
    if constexpr (sizeof(T) == 4) {
        switch (v) {
            case 0: return launch_staged_t<0, T, CODES>(L, s, status);
            case 1: return launch_staged_t<1, T, CODES>(L, s, status);
            case 2: return launch_staged_t<2, T, CODES>(L, s, status);
            case 3: return launch_staged_t<3, T, CODES>(L, s, status);
        }
    } else {
        switch (v) {
            case 0: return launch_staged_t<0, T, CODES>(L, s, status);
            case 1: return launch_staged_t<1, T, CODES>(L, s, status);
            case 2: return launch_staged_t<2, T, CODES>(L, s, status);
            case 3: return launch_staged_t<3, T, CODES>(L, s, status);
            case 4: return launch_staged_t<4, T, CODES>(L, s, status);
            case 5: return launch_staged_t<5, T, CODES>(L, s, status);
        }
    }
    return fail(FBP_ERR_INVALID_ARG, "staged shape %d", v);
}

template <typename T>
fbp_status launch_staged_dtype(const StagedLaunch &L, int v, cudaStream_t s, unsigned *status)
{
    return L.slice16 ? launch_staged_shape<T, true>(L, v, s, status) : launch_staged_shape<T, false>(L, v, s, status);
}

}  // namespace
}  // namespace fbp

using namespace fbp;

extern "C" int fbp_backproject_staged_shape_count(fbp_dtype dtype)
{
    return dtype == FBP_F32 ? kNumStagedShapes32 : (dtype == FBP_F16 || dtype == FBP_BF16) ? kNumStagedShapes16 : 0;
}

extern "C" size_t fbp_backproject_staged_workspace_bytes(const fbp_geometry *g, fbp_dtype dtype, int chunk)
{
    clear_error();
    if (!g || chunk < 1 || g->n_angles < 2 || g->n_det < 1) return 0;
    if (dtype != FBP_F32 && dtype != FBP_F16 && dtype != FBP_BF16) return 0;
    return staged_scale_bytes(chunk) + (size_t)chunk * staged_table_bytes(g->n_angles, g->n_det, dtype);
}

namespace {

fbp_status staged_impl(const void *filt, const float *row_scale, fbp_dtype dtype, float *slice,
                       unsigned short *slice16, float hu_a, float hu_b, const fbp_geometry *g, int n_slices,
                       float scale, int accumulate, int shape, void *workspace, size_t ws_bytes,
                       fbp_stream_t stream)
{
    fbp_status st = check_geometry(g, false, true);
    if (st != FBP_OK) return st;
    if (dtype != FBP_F32 && dtype != FBP_F16 && dtype != FBP_BF16)
        return fail(FBP_ERR_INVALID_ARG, "dtype %d", (int)dtype);
    if (shape < -1 || shape >= fbp_backproject_staged_shape_count(dtype))
        return fail(FBP_ERR_INVALID_ARG, "shape %d", shape);
    if (n_slices < 0) return fail(FBP_ERR_INVALID_ARG, "n_slices < 0");
    if (!(scale == scale) || scale > 3.4e38f || scale < -3.4e38f)
        return fail(FBP_ERR_INVALID_ARG, "scale is not finite");
    if (!bp_orbit_geometry(g->n_angles, g->angle_step, g->n_det, g->det_center, g->n, 16))
        return fail(FBP_ERR_UNSUPPORTED, "fbp_backproject_staged needs angle step pi/K with K even and "
                    "det_center = (D-1)/2");
    if (n_slices == 0) return FBP_OK;
    if (!filt || !(slice || slice16)) return fail(FBP_ERR_INVALID_ARG, "filt or slice is NULL");
    if (dtype != FBP_F32 && !row_scale) return fail(FBP_ERR_INVALID_ARG, "row_scale is required for 16-bit input");
    const size_t nin = (size_t)n_slices * g->n_angles * g->n_det * (dtype == FBP_F32 ? 4 : 2);
    const size_t nout = (size_t)n_slices * g->n * g->n * (slice16 ? 2 : 4);
    const char *pi = static_cast<const char *>(filt);
    const char *po = slice16 ? reinterpret_cast<const char *>(slice16) : reinterpret_cast<const char *>(slice);
    if (pi < po + nout && po < pi + nin) return fail(FBP_ERR_INVALID_ARG, "slice overlaps filt");
    if (!workspace) return fail(FBP_ERR_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) & 255)
        return fail(FBP_ERR_WORKSPACE, "workspace is not 256-byte aligned");
    const size_t per = staged_table_bytes(g->n_angles, g->n_det, dtype);
    int chunk = 0;
    for (int c = std::min(n_slices, 1 << 16); c >= 1; c = c > 8 ? c / 2 : c - 1)
        if (staged_scale_bytes(c) + (size_t)c * per <= ws_bytes) {
            chunk = c;
            break;
        }
    if (chunk < 1)
        return fail(FBP_ERR_WORKSPACE, "workspace has %zu bytes, one slice needs %zu", ws_bytes,
                    staged_scale_bytes(1) + per);
    if ((long long)chunk * (g->n_angles / 2) > INT_MAX)
        chunk = (int)std::max(1LL, (long long)INT_MAX / (g->n_angles / 2));
    const double2 *cs = nullptr;
    st = angle_table(*g, stream, &cs);
    if (st != FBP_OK) return st;
    unsigned *status = nullptr;
    st = device_status_word(&status);
    if (st != FBP_OK) return st;
    StagedLaunch L;
    L.filt = filt;
    L.row_scale = row_scale;
    L.slice = slice;
    L.slice16 = slice16;
    L.hu_a = hu_a;
    L.hu_b = hu_b;
    L.cs = cs;
    L.K = g->n_angles;
    L.D = g->n_det;
    L.N = g->n;
    L.S = n_slices;
    L.alpha = g->pixel_size / g->det_spacing;
    L.det_center = g->det_center;
    L.scale = scale;
    L.accumulate = accumulate ? 1 : 0;
    L.dtype = dtype;
    L.ws = static_cast<char *>(workspace);
    L.chunk = chunk;
    // 16-bit default (measured at N = 8192, K = 4096, 16 slices: shape 1 8264,
    // shape 5 8243, shape 0 8001 Gupdates/s): the 64 x 64 orbit where n allows it
    if (shape < 0) shape = dtype == FBP_F32 ? 0 : (g->n % 128 == 0 ? 1 : 5);
    L.row_scale = dtype == FBP_F32 ? nullptr : row_scale;
    switch (dtype) {
        case FBP_F32: return launch_staged_dtype<float>(L, shape, stream, status);
        case FBP_F16: return launch_staged_dtype<__half>(L, shape, stream, status);
        default: return launch_staged_dtype<__nv_bfloat16>(L, shape, stream, status);
    }
}

}  // namespace

extern "C" fbp_status fbp_backproject_staged(const void *filt, const float *row_scale, fbp_dtype dtype,
                                             float *slice, const fbp_geometry *g, int n_slices, float scale,
                                             int accumulate, int shape, void *workspace, size_t ws_bytes,
                                             fbp_stream_t stream)
{
    clear_error();
    if (n_slices > 0 && !slice) return fail(FBP_ERR_INVALID_ARG, "slice is NULL");
    return staged_impl(filt, row_scale, dtype, slice, nullptr, 0.f, 0.f, g, n_slices, scale, accumulate, shape,
                       workspace, ws_bytes, stream);
}

extern "C" fbp_status fbp_backproject_staged_u16(const void *filt, const float *row_scale, fbp_dtype dtype,
                                                 unsigned short *slice, const fbp_geometry *g, int n_slices,
                                                 float scale, const fbp_hu_window *w, int shape, void *workspace,
                                                 size_t ws_bytes, fbp_stream_t stream)
{
    float a = 0.f, b = 0.f;
    fbp_status st = fbp_hu_coefficients(w, &a, &b);     // validates the window (and clears the error)
    if (st != FBP_OK) return st;
    if (n_slices > 0 && !slice) return fail(FBP_ERR_INVALID_ARG, "slice is NULL");
    return staged_impl(filt, row_scale, dtype, nullptr, slice, a, b, g, n_slices, scale, 0, shape, workspace,
                       ws_bytes, stream);
}
