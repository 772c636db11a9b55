// bp_staged_batch.cu -- the staged backprojection for ragged batches: the
// default backprojection of fbp_batched / fbp_batched_scans for the items
// whose geometry has the 90-degree orbit symmetry (Sec. V-A(b): specimens of
// different sizes reconstructed together).
//
// fbp_backproject_staged moves each window with a bulk-tensor copy through a
// tensor map of one chunk's table, and the copy engine fills the part of a
// window that lies past the detector with zeros.  A batch holds up to 256
// tables of different shapes, and a tensor map per item would not fit in the
// kernel parameters; each item's table is padded instead, so that every
// window an orbit tile of the item reads lies inside its padded row and is
// one contiguous run of W entries, moved by a plain bulk copy.  Item i's
// table (in the batch workspace), entry e' holding detector segment
// e' - P_lo - 1 (zero outside [-1, D-1], as the tensor copy's fill):
//     16-bit rows: [K/2][Ep] 16-byte entries
//     FP32 rows:   plane a [K/2][Ep], then plane b [K/2][Ep] (the two 16-byte
//                  halves of the 32-byte midpoint/slope entry)
// One persistent launch runs orbit units (four tiles: 32 x 32 for FP32
// rows, 64 x 64 for 16-bit rows) of every such item, taken from an atomic
// counter or in group-cyclic order.  The stage ring, the entries, the
// per-pair arithmetic and the epilogue are fbp_backproject_staged's
// (bp_staged.cuh), so every item's slice is bit-identical to
// fbp_backproject_staged with the same shape (FP32 rows: shape 0, 16-bit
// rows: shape 1).  Stages are numbered per block across its units, so each
// buffer's mbarrier parity follows from that running count.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>

#include "bp_batch.cuh"
#include "bp_staged.cuh"

namespace fbp {
namespace {

constexpr int sb_tile(fbp_dtype dtype) { return dtype == FBP_F32 ? 32 : 64; }
constexpr int sb_max_wp(fbp_dtype dtype) { return dtype == FBP_F32 ? 72 : 104; }

// 16-bit rows: S of each item, the largest row scale (1 if none is positive),
// as fbp_backproject_staged forms it per slice.
__global__ void __launch_bounds__(256) staged_batch_scale_kernel(const __grid_constant__ StagedPrepArgs p)
{
    __shared__ float red[8];
    const StagedPrepItem &it = p.items[blockIdx.x];
    const float *rs = it.row_scale;
    float mx = 0.f;
    for (int k = threadIdx.x; k < it.K; k += blockDim.x) mx = fmaxf(mx, __ldg(rs + k));
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        mx = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
        *it.smax = mx > 0.f ? mx : 1.f;
    }
}

// One block per angle pair of one item: the pair's padded table row.
template <typename T, bool PACKED>
__global__ void __launch_bounds__(256) staged_batch_prep_kernel(const __grid_constant__ StagedPrepArgs p)
{
    const int q = blockIdx.x;
    int lo = 0, hi = p.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.items[mid].pair_begin <= q) lo = mid; else hi = mid - 1;
    }
    const StagedPrepItem &it = p.items[lo];
    const int k = q - it.pair_begin, K2 = it.K / 2, D = it.D, Ep = it.Ep, P_lo = it.P_lo;
    const T *r0 = static_cast<const T *>(it.filt) + (size_t)k * D;
    const T *r1 = r0 + (size_t)K2 * D;
    if constexpr (sizeof(T) == 4) {
        float4 *pa = static_cast<float4 *>(it.table) + (size_t)k * Ep;
        float4 *pb = pa + (size_t)K2 * Ep;
        for (int e = threadIdx.x; e < Ep; e += blockDim.x) {
            float4 va, vb;
            orbit_entry32(reinterpret_cast<const float *>(r0), reinterpret_cast<const float *>(r1), D,
                          e - P_lo - 1, va, vb);
            pa[e] = va;
            pb[e] = vb;
        }
    } else {
        const float invS = __frcp_rn(__ldg(it.smax));
        const float sc0 = __fmul_rn(__ldg(it.row_scale + k), invS);
        const float sc1 = __fmul_rn(__ldg(it.row_scale + k + K2), invS);
        uint4 *row = static_cast<uint4 *>(it.table) + (size_t)k * Ep;
        for (int e = threadIdx.x; e < Ep; e += blockDim.x)
            row[e] = orbit_entry16<T, PACKED>(r0, r1, D, e - P_lo - 1, sc0, sc1);
    }
}

// The persistent kernel: TXT x TYT threads, orbit tiles of PX x PY pixels
// per thread, KT angle pairs per stage, NS stage buffers.  Thread 0 takes
// each unit and publishes its item, tile origin and FP64 tile centre in
// shared memory; the item's fields are read from the kernel parameters where
// they are used (the issuing warp reads most of them once per stage), so that
// the pair loop keeps its registers.
template <int TXT, int TYT, int PX, int PY, int KT, int NS, typename T, bool PACKED, int MINB>
__global__ void __launch_bounds__(TXT *TYT, MINB) bp_staged_batch_kernel(const __grid_constant__ StagedBatchArgs a)
{
    constexpr int NW = TXT * TYT / 32, TILE = TXT * PX, WX = TXT / 8;
    constexpr int HALVES = sizeof(T) == 4 ? 2 : 1;
    static_assert(TXT * PX == TYT * PY, "square tile");
    static_assert(KT <= 32 && (NS == 2 || NS == 4), "stage shape");
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_unit;
    __shared__ double s_xy[2];             // the unit's base tile centre (X, Y)
    const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t base_s = (raw_s + 127u) & ~127u;
    unsigned char *base = smem_raw + (base_s - raw_s);
    const uint32_t full_s = base_s;                           // NS x 8 bytes
    int *done = reinterpret_cast<int *>(base + 8 * NS);
    int *issued = reinterpret_cast<int *>(base + 12 * NS);
    float4 *prm = reinterpret_cast<float4 *>(base + 128);
    const uint32_t tab0 = base_s + 128u + (uint32_t)staged_params_bytes<KT, NS>();
    const int Wp = a.Wp;
    const uint32_t half_bytes = (uint32_t)(2 * KT * Wp * 16);   // one half-array of a stage
    const uint32_t stage_bytes = HALVES * half_bytes;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tx = (warp % WX) * 8 + (lane & 7);
    const int ty = (warp / WX) * 4 + (lane >> 3);
    const float dxt = (float)tx - 0.5f * (TILE - 1);
    const float dyt = (float)ty - 0.5f * (TILE - 1);

    if (tid == 0) {
        for (int b = 0; b < NS; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" ::"r"(full_s + 8u * b) : "memory");
            done[b] = 0;
            issued[b] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // stages this block has consumed, over all its units; NS divides 2^32, so
    // the buffer (g mod NS) and the parity (bit log2 NS of g) survive a wrap
    unsigned gs = 0;
    __shared__ int s_item, s_x0, s_y0;
    for (int iter = 0;; ++iter) {
        // (every thread has read the previous unit's state: the unit ends
        // with a block barrier)
        if (tid == 0) {
            int u;
            if (a.cyclic) {
                const long long uc = (long long)blockIdx.x + (long long)iter * gridDim.x;
                u = uc < a.total_units ? (int)uc : a.total_units;
            } else {
                u = atomicAdd(a.counter, 1);
            }
            if (u < a.total_units && iter > a.total_units) {
                atomicCAS(a.status, 0u, (unsigned)FAULT_QUEUE_CAP);
                u = a.total_units;
            }
            s_unit = u;
            if (u < a.total_units) {
                int lo = 0, hi = a.count - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.items[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
                }
                const StagedBatchItem &it = a.items[lo];
                const int t = u - it.unit_begin;
                const int x0 = (t % it.tiles_x) * TILE, y0 = (t / it.tiles_x) * TILE;
                const double m = 0.5 * (it.N - 1);
                s_item = lo;
                s_x0 = x0;
                s_y0 = y0;
                s_xy[0] = (double)x0 + 0.5 * (TILE - 1) - m;
                s_xy[1] = (double)y0 + 0.5 * (TILE - 1) - m;
            }
        }
        __syncthreads();
        if (s_unit >= a.total_units) break;
        const StagedBatchItem &it = a.items[s_item];
        const int K2 = it.K2, H = it.H, W = it.W, Ep = it.Ep, P_lo = it.P_lo;
        const int n_stages = (K2 + KT - 1) / KT;
        const unsigned char *tab_a = static_cast<const unsigned char *>(it.table);
        const size_t plane = (size_t)K2 * Ep * 16;

        // one warp fills buffer b with the unit's stage tl: the pairs'
        // parameters (FP64 base coordinates) and two window copies per pair
        // (four for FP32 rows), each a run of W entries of the padded table
        auto issue = [&](int tl, int b) {
            const int k0 = tl * KT, na = min(KT, K2 - k0);
            int e1 = 0, e2 = 0;
            if (lane < KT) {
                float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (lane < na) {
                    const double2 cs = it.cs[k0 + lane];
                    const double c = it.alpha * cs.x, s = it.alpha * cs.y;
                    const double v1 = fma(c, s_xy[0], fma(s, s_xy[1], it.det_center));
                    const double v2 = fma(-s, s_xy[0], fma(c, s_xy[1], it.det_center));
                    const double jc1 = floor(v1), jc2 = floor(v2);
                    pv = make_float4((float)c, (float)s, (float)(v1 - jc1 - 0.5), (float)(v2 - jc2 - 0.5));
                    // first entry of each window: segment jc - H, padded
                    e1 = (int)jc1 - H + 1 + P_lo;
                    e2 = (int)jc2 - H + 1 + P_lo;
                    if ((unsigned)e1 > (unsigned)(Ep - W) || (unsigned)e2 > (unsigned)(Ep - W)) {
                        // outside the padding the host sized for this item: clamp
                        // (the copy stays inside the table) and record it
                        atomicCAS(a.status, 0u, (unsigned)FAULT_BP_WINDOW);
                        e1 = min(max(e1, 0), Ep - W);
                        e2 = min(max(e2, 0), Ep - W);
                    }
                }
                prm[b * KT + lane] = pv;
            }
            // the block's earlier reads of buffer b (ordered before this warp
            // by the done counter or the unit barrier) come before the copy
            // engine's writes
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
                const uint32_t bytes = (uint32_t)(W * 16);
                const unsigned char *row = tab_a + (size_t)(k0 + lane) * Ep * 16;
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(dst), "l"(row + (size_t)e1 * 16), "r"(bytes), "r"(mbar) : "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(dst + (uint32_t)(Wp * 16)), "l"(row + (size_t)e2 * 16), "r"(bytes), "r"(mbar)
                             : "memory");
                if constexpr (HALVES == 2) {
                    // FP32: the entries' second halves (plane b) into the mirrored-row array
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(dst + half_bytes), "l"(row + plane + (size_t)e1 * 16), "r"(bytes), "r"(mbar)
                                 : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(dst + half_bytes + (uint32_t)(Wp * 16)), "l"(row + plane + (size_t)e2 * 16),
                                   "r"(bytes), "r"(mbar)
                                 : "memory");
                }
            }
        };

        if (warp == 0)
            for (int tl = 0; tl < min(NS, n_stages); ++tl) issue(tl, (int)((gs + tl) % NS));

        float acc[4][PY][PX];
#pragma unroll
        for (int o = 0; o < 4; ++o)
#pragma unroll
            for (int iy = 0; iy < PY; ++iy)
#pragma unroll
                for (int ix = 0; ix < PX; ++ix) acc[o][iy][ix] = 0.f;

        bool ok = true;
        for (int tl = 0; tl < n_stages; ++tl) {
            const unsigned g = gs + (unsigned)tl;
            const int b = (int)(g % NS);
            if (!staged_wait(full_s + 8u * b, (unsigned)((g / NS) & 1))) {
                ok = false;
                break;
            }
            const int na = min(KT, K2 - tl * KT);
            const uint32_t tabb = tab0 + (uint32_t)b * stage_bytes;
            for (int p = 0; p < na; ++p) {
                const uint32_t cb1 = tabb + 16u * (uint32_t)(2 * p * Wp + H) - 16u * kRoundMagicBits;
                const uint32_t cb2 = cb1 + 16u * (uint32_t)Wp;
                if constexpr (HALVES == 2)
                    orbit_pair_mid<TXT, TYT, PX, PY>(acc, prm[b * KT + p], cb1, cb2, half_bytes, dxt, dyt);
                else
                    orbit_pair<TXT, TYT, PX, PY, T, false, PACKED>(acc, prm[b * KT + p], cb1, cb2, 0u, dxt, dyt,
                                                                   H, a.status);
            }
            // release buffer b; the last warp to do so refills it with stage tl + NS
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
            if (last && tl + NS < n_stages) issue(tl + NS, b);
        }
        gs += (unsigned)n_stages;
        const int x0 = s_x0, y0 = s_y0;
        // every warp is done with the buffers and the unit's shared state
        // (thread 0 rewrites both for the next unit)
        const bool failed = __syncthreads_or(!ok);
        if (failed) {
            // a wait ran out: record it, let every copy this block started land
            // (capped) and stop
            if (tid == 0) {
                atomicCAS(a.status, 0u, (unsigned)FAULT_BP_STAGE_WAIT);
                for (int b = 0; b < NS; ++b)
                    if (issued[b] > 0) staged_wait(full_s + 8u * b, (unsigned)((issued[b] - 1) & 1));
            }
            return;
        }
        const float S = HALVES == 2 ? 1.f : __ldg(it.smax);
        orbit_store<TXT, TYT, PX, PY>(acc, it.slice, nullptr, 0.f, 0.f, 0, it.N, x0 + tx, y0 + ty, it.scale * S);
    }
}

template <int TXT, int TYT, int PX, int PY, int KT, int NS, typename T, bool PACKED, int MINB>
fbp_status launch_staged_batch_t(const StagedPrepArgs &p, StagedBatchArgs &a, fbp_dtype dtype, cudaStream_t s)
{
    constexpr int HALVES = sizeof(T) == 4 ? 2 : 1;
    static_assert(TXT * PX == (HALVES == 2 ? 32 : 64), "tile of the dtype");
    if (a.Wp <= 0 || a.Wp > sb_max_wp(dtype) || a.Wp % 8 != 0)
        return fail(FBP_ERR_UNSUPPORTED, "staged batch window %d", a.Wp);
    if constexpr (sizeof(T) == 2) {
        staged_batch_scale_kernel<<<p.count, 256, 0, s>>>(p);
        FBP_CUDA_TRY(cudaGetLastError());
    }
    staged_batch_prep_kernel<T, PACKED><<<(unsigned)p.total_pairs, 256, 0, s>>>(p);
    FBP_CUDA_TRY(cudaGetLastError());
    auto kern = bp_staged_batch_kernel<TXT, TYT, PX, PY, KT, NS, T, PACKED, MINB>;
    const size_t smem = staged_smem_bytes<KT, NS, HALVES>(a.Wp);
    fbp_status st = ensure_dynamic_smem(reinterpret_cast<const void *>(kern), smem);
    if (st != FBP_OK) return st;
    int per_sm = 0;
    st = blocks_per_sm(reinterpret_cast<const void *>(kern), TXT * TYT, smem, &per_sm);
    if (st != FBP_OK) return st;
    if (per_sm < 1) return fail(FBP_ERR_UNSUPPORTED, "staged batch kernel does not fit on an SM");
    int dev = 0, sms = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    FBP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min(sms * per_sm, a.total_units));
    kern<<<grid, TXT * TYT, smem, s>>>(a);
    FBP_CUDA_TRY(cudaGetLastError());
    return FBP_OK;
}

}  // namespace

bool staged_batch_geometry(int K, double angle_step, int D, double det_center, int N, double alpha,
                           fbp_dtype dtype, StagedItemGeom *out)
{
    const int T = sb_tile(dtype);
    if (!bp_orbit_geometry(K, angle_step, D, det_center, N, T)) return false;
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return false;
    const int H = bp_window_half(alpha, T, T);
    const int W = 2 * H + 1, Wp = (W + 7) / 8 * 8;
    if (H < 0 || Wp > sb_max_wp(dtype)) return false;
    // |v - det_center| <= alpha * |(Xc, Yc)| <= alpha (N - T) / sqrt 2 over
    // the orbit base tiles (|Xc|, |Yc| <= (N - T) / 2); slack for rounding
    const double R = alpha * (N - T) / std::sqrt(2.0) * (1.0 + 1e-12) + 1e-6;
    const double lo = std::floor(det_center - R), hi = std::floor(det_center + R);
    // first entry of a window: floor(v) - H + 1 + P_lo >= 0; its last:
    // floor(v) + H + 1 + P_lo <= Ep - 1; two entries of margin each side
    const long long P_lo = std::max(0LL, (long long)H + 1 - (long long)lo);
    const long long Ep = std::max((long long)D + 1, (long long)hi + H + 4) + P_lo;
    const long long bytes = (long long)(K / 2) * Ep * 16 * (dtype == FBP_F32 ? 2 : 1);
    if (Ep > INT_MAX / 16 || bytes <= 0) return false;
    if (out) {
        out->H = H;
        out->W = W;
        out->Wp = Wp;
        out->P_lo = (int)P_lo;
        out->Ep = (int)Ep;
        out->table_bytes = (size_t)bytes;
    }
    return true;
}

int staged_batch_tile(fbp_dtype dtype) { return sb_tile(dtype); }

// FP32 rows: fbp_backproject_staged's shape 0 (32 x 32 orbits, 128 threads,
// 4 pairs per stage, 2 buffers, six blocks per SM); 16-bit rows: its shape 1
// (64 x 64 orbits, 256 threads, 16 pairs, 2 buffers, two blocks per SM).
fbp_status launch_staged_batch(const StagedPrepArgs &p, StagedBatchArgs &a, fbp_dtype dtype, cudaStream_t s)
{
    if (a.total_units <= 0 || p.count <= 0) return FBP_OK;
    switch (dtype) {
        case FBP_F32: return launch_staged_batch_t<16, 8, 2, 4, 4, 2, float, false, 6>(p, a, dtype, s);
        case FBP_F16: return launch_staged_batch_t<16, 16, 4, 4, 16, 2, __half, true, 2>(p, a, dtype, s);
        case FBP_BF16: return launch_staged_batch_t<16, 16, 4, 4, 16, 2, __nv_bfloat16, true, 2>(p, a, dtype, s);
    }
    return fail(FBP_ERR_INVALID_ARG, "dtype");
}

}  // namespace fbp
