// backproject.cu -- launches of the backprojection tile routine (bp_tile.cuh):
// a uniform grid over (tile, slice) for fbp_backproject, and a persistent
// work-queue kernel for ragged batches.
#include <algorithm>
#include <climits>
#include <cmath>
#include <map>
#include <mutex>

#include "bp_tile.cuh"
#include "bp_orbit.cuh"
#include "bp_batch.cuh"

namespace fbp {

// Blocks per orbit for the default path's split launch: when a slice has
// fewer than half as many orbits as the GPU holds resident blocks, its angle
// pairs are shared among up to 16 blocks (one cluster), each with at least
// one stage.  The count depends on the geometry and the device only, so a
// slice gets the same sums whatever the number of slices in the call.
int orbit_split_parts(long long orbits, int K2, int KT, long long resident)
{
    if (orbits <= 0 || orbits * 2 >= resident) return 1;
    long long P = std::min(16LL, resident / (2 * orbits));
    P = std::min(P, (long long)((K2 + KT - 1) / KT));
    return (int)std::max(P, 1LL);
}

fbp_status device_sm_count(int *out)
{
    static std::mutex mu;
    static std::map<int, int> counts;
    int dev = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = counts.find(dev);
    if (it == counts.end()) {
        int sms = 0;
        FBP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        it = counts.emplace(dev, sms).first;
    }
    *out = it->second;
    return FBP_OK;
}

namespace {

// Compiled tile shapes: threads TXT x TYT, pixels per thread PX x PY,
// angles (generic) or angle pairs (orbit) per staged tile KT.  Orbit shapes
// use the 90-degree symmetry (bp_orbit.cuh) and need the standard geometry.
// minb: resident blocks per SM the orbit kernels are compiled for (the
// register cap is 65536 / (minb x threads)).  Variant 7 runs six 128-thread
// blocks (80 registers, 8 bytes of spill): 24 warps per SM instead of 16 hide
// more shared-load latency, +3 % over four blocks at N = 8192 (seven blocks
// spill 68 bytes, eight fit 64 registers without spill but measure between).
struct ShapeDesc {
    int txt, tyt, px, py, kt, orbit, packed, minb;
};
constexpr ShapeDesc kShapes[] = {
    {16, 16, 4, 4, 32, 0, 0, 0},   // 0: 64 x 64 tile
    {16, 16, 4, 4, 16, 0, 0, 0},   // 1
    {16, 16, 4, 2, 32, 0, 0, 0},   // 2: 64 x 32
    {16, 16, 2, 4, 32, 0, 0, 0},   // 3: 32 x 64
    {16, 16, 4, 4, 64, 0, 0, 0},   // 4
    {32, 8, 2, 8, 32, 0, 0, 0},    // 5: 64 x 64, warps 4 x 2
    {16, 8, 2, 4, 16, 1, 0, 4},    // 6: orbit of 32 x 32 tiles, 16 angle pairs per stage
    {16, 8, 2, 4, 8, 1, 0, 6},     // 7: orbit of 32 x 32 tiles, 8 pairs
    {16, 16, 4, 4, 8, 1, 0, 2},    // 8: orbit of 64 x 64 tiles, 8 pairs
    {16, 8, 2, 4, 32, 1, 0, 4},    // 9: orbit of 32 x 32 tiles, 32 pairs
    {16, 16, 4, 4, 8, 1, 1, 2},    // 10: as 8, packed pair arithmetic (16-bit rows only)
    {16, 8, 2, 4, 16, 1, 1, 4},    // 11: as 6, packed pair arithmetic (16-bit rows only)
    {16, 8, 4, 4, 32, 0, 0, 0},    // 12: 64 x 32, 128 threads (the 128-thread orbits' batch fallback)
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

struct BpArgs {
    const void *filt;
    const float *row_scale;
    float *slice;
    const double2 *cs;
    int K, D, N;
    double alpha, det_center;
    float scale;
    int accumulate;
    unsigned short *slice16;   // uint16 codes instead of `slice`, or null
    float hu_a, hu_b;
    int H, W;
    int tiles_x;
    int slice_base;
    int parts;                 // orbit kernels: blocks (a cluster) per orbit, each a share of the angle pairs
    unsigned *status;
};

template <int TXT, int TYT, int PX, int PY, int KT, typename T, bool CHECKED>
__global__ void __launch_bounds__(TXT *TYT) bp_kernel(BpArgs a)
{
    extern __shared__ __align__(16) unsigned char bp_smem[];
    constexpr int TW = TXT * PX, TH = TYT * PY;
    const int tile = blockIdx.x;
    const int sl = a.slice_base + blockIdx.y;
    BpTileJob j;
    const size_t kd = (size_t)a.K * a.D;
    j.filt = static_cast<const char *>(a.filt) + (size_t)sl * kd * sizeof(T);
    j.row_scale = a.row_scale ? a.row_scale + (size_t)sl * a.K : nullptr;
    j.out = a.slice ? a.slice + (size_t)sl * a.N * a.N : nullptr;
    j.out16 = a.slice16 ? a.slice16 + (size_t)sl * a.N * a.N : nullptr;
    j.hu_a = a.hu_a;
    j.hu_b = a.hu_b;
    j.cs = a.cs;
    j.K = a.K;
    j.D = a.D;
    j.N = a.N;
    j.alpha = a.alpha;
    j.det_center = a.det_center;
    j.scale = a.scale;
    j.accumulate = a.accumulate;
    j.H = a.H;
    j.W = a.W;
    j.x0 = (tile % a.tiles_x) * TW;
    j.y0 = (tile / a.tiles_x) * TH;
    j.status = a.status;
    bp_tile<TXT, TYT, PX, PY, KT, T, CHECKED>(j, bp_smem);
}

// SPLIT: a.parts blocks per orbit, launched as clusters of a.parts blocks
// along x; block part p of the cluster sums angle pairs [p K2 / P, (p+1) K2 / P).
template <int TXT, int TYT, int PX, int PY, int KT, typename T, bool CHECKED, bool PACKED, int MINB,
          bool SPLIT = false>
__global__ void __launch_bounds__(TXT *TYT, MINB) bp_orbit_kernel(BpArgs a)
{
    extern __shared__ __align__(16) unsigned char bp_smem[];
    constexpr int TILE = TXT * PX;
    const int half = a.tiles_x;                 // orbits per row of the top-left quadrant
    const int P = SPLIT ? a.parts : 1;
    const int o = blockIdx.x / P, part = blockIdx.x - o * P;
    const int sl = a.slice_base + blockIdx.y;
    BpOrbitJob j;
    const size_t kd = (size_t)a.K * a.D;
    j.filt = static_cast<const char *>(a.filt) + (size_t)sl * kd * sizeof(T);
    j.row_scale = a.row_scale ? a.row_scale + (size_t)sl * a.K : nullptr;
    j.out = a.slice ? a.slice + (size_t)sl * a.N * a.N : nullptr;
    j.out16 = a.slice16 ? a.slice16 + (size_t)sl * a.N * a.N : nullptr;
    j.hu_a = a.hu_a;
    j.hu_b = a.hu_b;
    j.cs = a.cs;
    j.K = a.K;
    j.D = a.D;
    j.N = a.N;
    j.alpha = a.alpha;
    j.det_center = a.det_center;
    j.scale = a.scale;
    j.accumulate = a.accumulate;
    j.H = a.H;
    j.W = a.W;
    j.x0 = (o % half) * TILE;
    j.y0 = (o / half) * TILE;
    j.kb = (int)((long long)part * (a.K / 2) / P);
    j.ke = (int)((long long)(part + 1) * (a.K / 2) / P);
    j.status = a.status;
    bp_orbit<TILE, TXT, TYT, PX, PY, KT, T, CHECKED, PACKED, SPLIT>(j, bp_smem);
}

// FP32 rows of small slices on the default path: orbits of 16 x 16 tiles
// (64 threads, 2 x 2 pixels each), split over clusters like the variants.
// Four times the orbits of variant 7's 32 x 32 tiles, so more blocks share
// each slice's angle pairs and more warps hide the staging latency.
constexpr ShapeDesc kSmallSplitShape = {8, 8, 2, 2, 16, 1, 0, 12};

// The orbit launch of one shape (V: the variant it serves, for messages).
template <int V, int TXT, int TYT, int PX, int PY, int KT, int PK, int MINB, typename T>
fbp_status launch_orbit_desc(const BpLaunch &L, cudaStream_t s, unsigned *status)
{
    constexpr ShapeDesc sd = {TXT, TYT, PX, PY, KT, 1, PK, MINB};
    constexpr int TILE = sd.txt * sd.px;
#ifdef FBP_CHECKED
    constexpr bool kChecked = true;
#else
    constexpr bool kChecked = false;
#endif
    if (!bp_orbit_eligible(L, TILE))
        return fail(FBP_ERR_UNSUPPORTED, "variant %d needs angle step pi/K with K even, "
                    "det_center = (D-1)/2 and N a multiple of %d", V, 2 * TILE);
    constexpr bool kPacked = sd.packed && sizeof(T) == 2;
    if (sd.packed && sizeof(T) != 2)
        return fail(FBP_ERR_UNSUPPORTED, "variant %d is for 16-bit rows", V);
    static_assert(sd.minb >= 1, "orbit shapes state their blocks per SM");
    auto kern = bp_orbit_kernel<sd.txt, sd.tyt, sd.px, sd.py, sd.kt, T, kChecked, kPacked, sd.minb>;
    BpArgs a;
    a.filt = L.filt;
    a.row_scale = L.row_scale;
    a.slice = L.slice;
    a.cs = L.cs;
    a.K = L.K;
    a.D = L.D;
    a.N = L.N;
    a.alpha = L.alpha;
    a.det_center = L.det_center;
    a.scale = L.scale;
    a.accumulate = L.accumulate;
    a.slice16 = L.slice16;
    a.hu_a = L.hu_a;
    a.hu_b = L.hu_b;
    a.H = bp_window_half(L.alpha, TILE, TILE);
    a.W = 2 * a.H + 1;
    a.status = status;
    const size_t smem = bp_orbit_smem_size<sd.kt, T>(a.W);
    if (smem > 200 * 1024) return fail(FBP_ERR_UNSUPPORTED, "backprojection window too wide");
    fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (st != FBP_OK) return st;
    a.tiles_x = L.N / TILE / 2;
    a.parts = 1;
    const long long orbits = (long long)a.tiles_x * a.tiles_x;
    if (orbits > INT_MAX) return fail(FBP_ERR_UNSUPPORTED, "too many tiles");
    if (L.split) {
        int sms = 0;
        st = device_sm_count(&sms);
        if (st != FBP_OK) return st;
        int parts = orbit_split_parts(orbits, L.K / 2, sd.kt, (long long)sms * sd.minb);
        if (parts > 1) {
            // clusters of `parts` blocks per orbit, partial sums reduced in shared memory
            auto skern = bp_orbit_kernel<sd.txt, sd.tyt, sd.px, sd.py, sd.kt, T, kChecked, kPacked, sd.minb, true>;
            const size_t ssmem = std::max(smem, bp_orbit_split_bytes<sd.txt, sd.tyt, sd.px, sd.py>());
            st = ensure_dynamic_smem(reinterpret_cast<const void *>(skern), ssmem);
            if (st != FBP_OK) return st;
            if (parts > 8) {
                // above the portable 8: allowed per kernel, capped by what the
                // device schedules (asked once per device, kernel and shared
                // memory size, so that a call being captured only launches)
                static std::mutex mu;
                static std::map<std::pair<int, size_t>, int> max_cluster;
                int dev = 0;
                FBP_CUDA_TRY(cudaGetDevice(&dev));
                std::lock_guard<std::mutex> lock(mu);
                auto it = max_cluster.find(std::make_pair(dev, ssmem));
                if (it == max_cluster.end()) {
                    FBP_CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(skern),
                                                      cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
                    cudaLaunchConfig_t q = {};
                    q.gridDim = dim3(16, 1);
                    q.blockDim = dim3(sd.txt * sd.tyt);
                    q.dynamicSmemBytes = ssmem;
                    int maxc = 0;
                    FBP_CUDA_TRY(cudaOccupancyMaxPotentialClusterSize(&maxc, skern, &q));
                    it = max_cluster.emplace(std::make_pair(dev, ssmem), maxc).first;
                }
                if (it->second < parts) parts = std::max(std::min(it->second, 8), 1);
            }
            a.parts = parts;
            for (int base = 0; base < L.S; base += 65535) {
                a.slice_base = base;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)(orbits * parts), (unsigned)std::min(65535, L.S - base));
                cfg.blockDim = dim3(sd.txt * sd.tyt);
                cfg.dynamicSmemBytes = ssmem;
                cfg.stream = s;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = (unsigned)parts;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                FBP_CUDA_TRY(cudaLaunchKernelEx(&cfg, skern, a));
            }
            return FBP_OK;
        }
    }
    for (int base = 0; base < L.S; base += 65535) {
        a.slice_base = base;
        dim3 grid((unsigned)orbits, (unsigned)std::min(65535, L.S - base));
        kern<<<grid, sd.txt * sd.tyt, smem, s>>>(a);
        FBP_CUDA_TRY(cudaGetLastError());
    }
    return FBP_OK;
}

template <int V, typename T>
fbp_status launch_orbit_shape(const BpLaunch &L, cudaStream_t s, unsigned *status)
{
    constexpr ShapeDesc sd = kShapes[V];
    return launch_orbit_desc<V, sd.txt, sd.tyt, sd.px, sd.py, sd.kt, sd.packed, sd.minb, T>(L, s, status);
}

// Whether the default FP32 path takes kSmallSplitShape: the geometry has
// the orbit symmetry at that tile size and its 16 x 16 orbits are few enough
// that each is still shared by at least 8 blocks.  Measured with one slice
// (µs per call, eager): N = 192 16.0 against 18.5 for variant 7's split,
// N = 256 19.6 against 21.4; at N = 512 (3 blocks per orbit) 101 against 81.
// Depends on the geometry and the device only.
bool small_split_applies(const BpLaunch &L)
{
    constexpr ShapeDesc sd = kSmallSplitShape;
    constexpr int TILE = sd.txt * sd.px;
    if (L.dtype != FBP_F32 || !L.split || !bp_orbit_eligible(L, TILE)) return false;
    int sms = 0;
    if (device_sm_count(&sms) != FBP_OK) return false;
    const long long half = L.N / TILE / 2;
    return orbit_split_parts(half * half, L.K / 2, sd.kt, (long long)sms * sd.minb) >= 8;
}

template <int V, typename T>
fbp_status launch_shape(const BpLaunch &L, cudaStream_t s, unsigned *status)
{
    if constexpr (kShapes[V].orbit) return launch_orbit_shape<V, T>(L, s, status);
    constexpr ShapeDesc sd = kShapes[V];
    constexpr int TW = sd.txt * sd.px, TH = sd.tyt * sd.py;
#ifdef FBP_CHECKED
    constexpr bool kChecked = true;
#else
    constexpr bool kChecked = false;
#endif
    auto kern = bp_kernel<sd.txt, sd.tyt, sd.px, sd.py, sd.kt, T, kChecked>;
    BpArgs a;
    a.filt = L.filt;
    a.row_scale = L.row_scale;
    a.slice = L.slice;
    a.cs = L.cs;
    a.K = L.K;
    a.D = L.D;
    a.N = L.N;
    a.alpha = L.alpha;
    a.det_center = L.det_center;
    a.scale = L.scale;
    a.accumulate = L.accumulate;
    a.slice16 = L.slice16;
    a.hu_a = L.hu_a;
    a.hu_b = L.hu_b;
    a.H = bp_window_half(L.alpha, TW, TH);
    a.W = 2 * a.H + 1;
    a.status = status;
    const size_t smem = bp_smem_size<sd.kt>(a.W);
    if (smem > 200 * 1024) return fail(FBP_ERR_UNSUPPORTED, "backprojection window too wide");
    fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (st != FBP_OK) return st;
    a.tiles_x = (L.N + TW - 1) / TW;
    const long long tiles = (long long)a.tiles_x * ((L.N + TH - 1) / TH);
    if (tiles > INT_MAX) return fail(FBP_ERR_UNSUPPORTED, "too many tiles");
    for (int base = 0; base < L.S; base += 65535) {
        a.slice_base = base;
        dim3 grid((unsigned)tiles, (unsigned)std::min(65535, L.S - base));
        kern<<<grid, sd.txt * sd.tyt, smem, s>>>(a);
        FBP_CUDA_TRY(cudaGetLastError());
    }
    return FBP_OK;
}

template <typename T>
fbp_status launch_variant(const BpLaunch &L, int v, cudaStream_t s, unsigned *status)
{
    switch (v) {
        case 0: return launch_shape<0, T>(L, s, status);
        case 1: return launch_shape<1, T>(L, s, status);
        case 2: return launch_shape<2, T>(L, s, status);
        case 3: return launch_shape<3, T>(L, s, status);
        case 4: return launch_shape<4, T>(L, s, status);
        case 5: return launch_shape<5, T>(L, s, status);
        case 6: return launch_shape<6, T>(L, s, status);
        case 7:
            if constexpr (sizeof(T) == 4) {
                if (small_split_applies(L)) {
                    constexpr ShapeDesc sd = kSmallSplitShape;
                    return launch_orbit_desc<7, sd.txt, sd.tyt, sd.px, sd.py, sd.kt, sd.packed, sd.minb, T>(
                        L, s, status);
                }
            }
            return launch_shape<7, T>(L, s, status);
        case 8: return launch_shape<8, T>(L, s, status);
        case 9: return launch_shape<9, T>(L, s, status);
        case 10: return launch_shape<10, T>(L, s, status);
        case 11: return launch_shape<11, T>(L, s, status);
        case 12: return launch_shape<12, T>(L, s, status);
    }
    return fail(FBP_ERR_INVALID_ARG, "backprojection variant %d", v);
}

// ---------------------------------------------------------------------------
// Persistent ragged-batch kernel: blocks pull work units from a global
// counter (or take every P-th unit, cyclic order) until the queue is empty.
// A unit is one 90-degree orbit of four tiles (bp_orbit.cuh) for an item
// whose geometry has the symmetry, else one tile of the generic routine
// (bp_tile.cuh); the two shapes share the block's threads.  Both routines are
// the single-slice kernels' own, so every item equals its single-slice run
// with the same shape bit for bit.  The loop is capped at total+1 iterations
// per block; past the cap it records FAULT_QUEUE_CAP and exits (it cannot
// wait on anything).
// ---------------------------------------------------------------------------
template <int GTX, int GTY, int GPX, int GPY, int GKT, int OTX, int OTY, int OPX, int OPY, int OKT,
          bool ORBIT, bool PACKED, int MINB, typename T>
__global__ void __launch_bounds__(GTX *GTY, MINB) bp_persistent_kernel(BpBatchArgs a)
{
    static_assert(!ORBIT || OTX * OTY == GTX * GTY, "orbit and tile shapes share the block");
    extern __shared__ __align__(16) unsigned char bp_smem[];
    __shared__ int s_unit;
    constexpr int TW = GTX * GPX, TH = GTY * GPY;
    constexpr int OTILE = OTX * OPX;
    for (int iter = 0;; ++iter) {
        int u;
        if (a.cyclic) {
            const long long uc = (long long)blockIdx.x + (long long)iter * gridDim.x;
            u = uc < a.total_units ? (int)uc : a.total_units;
        } else {
            if (threadIdx.x == 0) s_unit = atomicAdd(a.counter, 1);
            __syncthreads();
            u = s_unit;
            __syncthreads();
        }
        if (u >= a.total_units) break;
        if (iter > a.total_units) {
            if (threadIdx.x == 0) atomicCAS(a.status, 0u, (unsigned)FAULT_QUEUE_CAP);
            break;
        }
        // item owning unit u (unit_begin is ascending)
        int lo = 0, hi = a.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.items[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
        }
        const BpBatchItem &it = a.items[lo];
        const int t = u - it.unit_begin;
        if constexpr (ORBIT) {
            if (it.orbit) {
                BpOrbitJob j;
                j.filt = it.filt;
                j.row_scale = it.row_scale;
                j.out = it.slice;
                j.out16 = nullptr;
                j.hu_a = j.hu_b = 0.f;
                j.cs = it.cs;
                j.K = it.K;
                j.D = it.D;
                j.N = it.N;
                j.alpha = it.alpha;
                j.det_center = it.det_center;
                j.scale = it.scale;
                j.accumulate = 0;
                j.H = it.H;
                j.W = 2 * it.H + 1;
                j.x0 = (t % it.tiles_x) * OTILE;
                j.y0 = (t / it.tiles_x) * OTILE;
                j.kb = 0;
                j.ke = it.K / 2;
                j.status = a.status;
                bp_orbit<OTILE, OTX, OTY, OPX, OPY, OKT, T, false, PACKED>(j, bp_smem);
                continue;
            }
        }
        BpTileJob j;
        j.filt = it.filt;
        j.row_scale = it.row_scale;
        j.out = it.slice;
        j.out16 = nullptr;
        j.hu_a = j.hu_b = 0.f;
        j.cs = it.cs;
        j.K = it.K;
        j.D = it.D;
        j.N = it.N;
        j.alpha = it.alpha;
        j.det_center = it.det_center;
        j.scale = it.scale;
        j.accumulate = 0;
        j.H = it.H;
        j.W = 2 * it.H + 1;
        j.x0 = (t % it.tiles_x) * TW;
        j.y0 = (t / it.tiles_x) * TH;
        j.status = a.status;
        bp_tile<GTX, GTY, GPX, GPY, GKT, T, false>(j, bp_smem);
    }
}

// Generic variant an orbit variant falls back to for items without the
// symmetry, with the same threads: 12 (64 x 32 tiles) for 128-thread orbits,
// 0 (64 x 64) for 256-thread ones.
constexpr int fallback_variant(int threads) { return threads == 128 ? 12 : 0; }

template <int V, typename T>
fbp_status launch_persistent_shape(BpBatchArgs &a, int sms, cudaStream_t s)
{
    constexpr ShapeDesc sd = kShapes[V];
    constexpr bool kOrbit = sd.orbit != 0;
    if constexpr (sd.packed && sizeof(T) != 2) {
        return fail(FBP_ERR_UNSUPPORTED, "variant %d is for 16-bit rows", V);
    } else {
        constexpr ShapeDesc gd = kOrbit ? kShapes[fallback_variant(sd.txt * sd.tyt)] : sd;
        constexpr bool kPacked = sd.packed && sizeof(T) == 2;
        auto kern = bp_persistent_kernel<gd.txt, gd.tyt, gd.px, gd.py, gd.kt, sd.txt, sd.tyt, sd.px, sd.py,
                                         sd.kt, kOrbit, kPacked, (kOrbit ? sd.minb : 1), T>;
        size_t smem = 0;
        bool any_tile = false, any_orbit = false;
        for (int i = 0; i < a.count; ++i) (a.items[i].orbit ? any_orbit : any_tile) = true;
        if (any_tile) smem = bp_smem_size<gd.kt>(2 * a.max_H + 1);
        if (any_orbit) smem = std::max(smem, bp_orbit_smem_size<sd.kt, T>(2 * a.max_H_orbit + 1));
        if (smem > 200 * 1024) return fail(FBP_ERR_UNSUPPORTED, "backprojection window too wide");
        fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
        if (st != FBP_OK) return st;
        int per_sm = 0;
        st = blocks_per_sm(reinterpret_cast<const void *>(kern), sd.txt * sd.tyt, smem, &per_sm);
        if (st != FBP_OK) return st;
        if (per_sm < 1) return fail(FBP_ERR_UNSUPPORTED, "persistent kernel does not fit on an SM");
        const int grid = std::max(1, std::min(sms * per_sm, a.total_units));
        kern<<<grid, sd.txt * sd.tyt, smem, s>>>(a);
        FBP_CUDA_TRY(cudaGetLastError());
        return FBP_OK;
    }
}

template <typename T>
fbp_status launch_persistent_t(BpBatchArgs &a, int v, int sms, cudaStream_t s)
{
    switch (v) {
        case 0: return launch_persistent_shape<0, T>(a, sms, s);
        case 1: return launch_persistent_shape<1, T>(a, sms, s);
        case 2: return launch_persistent_shape<2, T>(a, sms, s);
        case 3: return launch_persistent_shape<3, T>(a, sms, s);
        case 4: return launch_persistent_shape<4, T>(a, sms, s);
        case 5: return launch_persistent_shape<5, T>(a, sms, s);
        case 6: return launch_persistent_shape<6, T>(a, sms, s);
        case 7: return launch_persistent_shape<7, T>(a, sms, s);
        case 8: return launch_persistent_shape<8, T>(a, sms, s);
        case 9: return launch_persistent_shape<9, T>(a, sms, s);
        case 10: return launch_persistent_shape<10, T>(a, sms, s);
        case 11: return launch_persistent_shape<11, T>(a, sms, s);
        case 12: return launch_persistent_shape<12, T>(a, sms, s);
    }
    return fail(FBP_ERR_UNSUPPORTED, "variant %d is not available for ragged batches", v);
}

}  // namespace

// One more variant after the table's: the texture-unit kernel (bp_texture.cu).
constexpr int kTextureVariant = kNumShapes;

int bp_variant_count() { return kNumShapes + 1; }

bool bp_variant_shape(int v, fbp_bp_shape *out)
{
    if (!out) return false;
    if (v == kTextureVariant) {
        out->angle_tile = 256;
        out->tile_x = out->tile_y = 64;
        out->px = out->py = 4;
        out->threads = 256;
        out->symmetric = 0;
        out->packed16 = 0;
        out->texture = 1;
        return true;
    }
    if (v < 0 || v >= kNumShapes) return false;
    out->texture = 0;
    const ShapeDesc &d = kShapes[v];
    out->angle_tile = d.kt;
    out->tile_x = d.txt * d.px;
    out->tile_y = d.tyt * d.py;
    out->px = d.px;
    out->py = d.py;
    out->threads = d.txt * d.tyt;
    out->symmetric = d.orbit;
    out->packed16 = d.packed;
    if (d.orbit) out->angle_tile = 2 * d.kt;
    return true;
}

int bp_tile_w(int v) { return v >= 0 && v < kNumShapes ? kShapes[v].txt * kShapes[v].px : 64; }
int bp_tile_h(int v) { return v >= 0 && v < kNumShapes ? kShapes[v].tyt * kShapes[v].py : 64; }

bool bp_persistent_shape(int v, fbp_dtype dtype, BpPersistentShape *out)
{
    if (v < 0 || v >= kNumShapes || !out) return false;
    const ShapeDesc &d = kShapes[v];
    if (d.packed && dtype == FBP_F32) return false;
    if (!d.orbit) {
        *out = {0, d.txt * d.px, d.tyt * d.py};
        return true;
    }
    const ShapeDesc &f = kShapes[fallback_variant(d.txt * d.tyt)];
    *out = {d.txt * d.px, f.txt * f.px, f.tyt * f.py};
    return true;
}

bool bp_orbit_geometry(int K, double angle_step, int D, double det_center, int N, int tile)
{
    const double pi = 3.14159265358979323846;
    if (K % 2 != 0 || N % (2 * tile) != 0) return false;
    if (std::fabs(angle_step * K - pi) > 1e-9 * pi) return false;
    if (std::fabs(det_center - 0.5 * (D - 1)) > 1e-9 * (1.0 + D)) return false;
    return true;
}

bool bp_orbit_eligible(const BpLaunch &L, int tile)
{
    return bp_orbit_geometry(L.K, L.angle_step, L.D, L.det_center, L.N, tile);
}

constexpr size_t kSmemBudget = 200 * 1024;

template <int V>
size_t variant_smem(const BpLaunch &L)
{
    constexpr ShapeDesc sd = kShapes[V];
    const int TW = sd.txt * sd.px, TH = sd.tyt * sd.py;
    const int W = 2 * bp_window_half(L.alpha, TW, TH) + 1;
    if constexpr (sd.orbit)
        return L.dtype == FBP_F32 ? bp_orbit_smem_size<sd.kt, float>(W)
                                  : bp_orbit_smem_size<sd.kt, __half>(W);
    return bp_smem_size<sd.kt>(W);
}

bool bp_variant_fits(int v, const BpLaunch &L)
{
    if (v == kTextureVariant) return bp_texture_shape_ok(L);
    size_t smem = 0;
    switch (v) {
        case 0: smem = variant_smem<0>(L); break;
        case 1: smem = variant_smem<1>(L); break;
        case 2: smem = variant_smem<2>(L); break;
        case 3: smem = variant_smem<3>(L); break;
        case 4: smem = variant_smem<4>(L); break;
        case 5: smem = variant_smem<5>(L); break;
        case 6: smem = variant_smem<6>(L); break;
        case 7: smem = variant_smem<7>(L); break;
        case 8: smem = variant_smem<8>(L); break;
        case 9: smem = variant_smem<9>(L); break;
        case 10: smem = variant_smem<10>(L); break;
        case 11: smem = variant_smem<11>(L); break;
        case 12: smem = variant_smem<12>(L); break;
        default: return false;
    }
    if (smem > kSmemBudget) return false;
    const ShapeDesc &d = kShapes[v];
    if (d.packed && L.dtype == FBP_F32) return false;
    return !d.orbit || bp_orbit_eligible(L, d.txt * d.px);
}

// Measured at N = 8192, K = 4096 on GB300 (Gupdates/s): FP32 rows --
// generic 64 x 64 tile (variant 5) 4290, symmetric 32 x 32 orbit (7) 4330;
// 16-bit rows -- packed 64 x 64 orbit (10) 7170-7210, unpacked (8) 6340-6370.
int bp_default_variant(const BpLaunch &L)
{
    if (L.dtype != FBP_F32) {
        for (int v : {10, 8, 11, 6})
            if (bp_variant_fits(v, L)) return v;
    } else {
        for (int v : {7, 5})
            if (bp_variant_fits(v, L)) return v;
    }
    return 0;
}

fbp_status launch_backproject(const BpLaunch &L, int variant, cudaStream_t s)
{
    if (L.S <= 0) return FBP_OK;
    // the default path may split small slices' angle pairs across clusters
    BpLaunch Ld = L;
    if (variant < 0) {
        variant = bp_default_variant(L);
        Ld.split = 1;
    }
    if (variant == kTextureVariant) return launch_backproject_texture(L, s);
    unsigned *status = nullptr;
    fbp_status st = device_status_word(&status);
    if (st != FBP_OK) return st;
    switch (L.dtype) {
        case FBP_F32: return launch_variant<float>(Ld, variant, s, status);
        case FBP_F16: return launch_variant<__half>(Ld, variant, s, status);
        case FBP_BF16: return launch_variant<__nv_bfloat16>(Ld, variant, s, status);
    }
    return fail(FBP_ERR_INVALID_ARG, "dtype");
}

fbp_status launch_bp_persistent(BpBatchArgs &a, int variant, fbp_dtype dtype, cudaStream_t s)
{
    if (variant < 0) variant = 0;
    int dev = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::map<int, int> sm_count;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = sm_count.find(dev);
        if (it == sm_count.end()) {
            FBP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            it = sm_count.emplace(dev, sms).first;
        }
        sms = it->second;
    }
    switch (dtype) {
        case FBP_F32: return launch_persistent_t<float>(a, variant, sms, s);
        case FBP_F16: return launch_persistent_t<__half>(a, variant, sms, s);
        case FBP_BF16: return launch_persistent_t<__nv_bfloat16>(a, variant, sms, s);
    }
    return fail(FBP_ERR_INVALID_ARG, "dtype");
}

}  // namespace fbp
