// sap.cu -- symmetric adaptive patching (SAP) of a reconstructed slice and
// the 2-bit masks (Sec. V-B(c), Eq. (1); Sec. V-C(a)); the definitions are in
// include/sap.h.  Everything is exact: integer arithmetic, or a fixed
// sequence of IEEE double operations for the variance key and the patch means.
//
// Edges: one fused kernel per 32 x 32 tile stages the codes with a halo of 4
// and computes smoothing, Sobel, magnitude, non-maximum suppression and the
// two thresholds in shared memory (each staged array holds the value at the
// border-clamped coordinate, which is what replicated borders mean stage by
// stage).  Hysteresis is connected-component labelling of the candidate
// pixels (weak or strong) with a lock-free union-find (links made only from
// roots by compare-and-swap, larger root under smaller); a component is
// kept if it holds a strong pixel.  Connectivity does not depend on the
// order of the unions, so the result is deterministic.
//
// Quadtree: nodes are stored level by level (level l has 4^l nodes of side
// n >> l, indexed by their Morton code, so node m's children are 4m .. 4m+3
// in Z-order).  Sums (edge count, S1, S2) are built bottom-up, the monotone
// variance key top-down, and each splittable node gets a 128-bit key
// (V | variance key | shallower level | smaller Morton code) that orders
// nodes as the greedy split does.  The greedy split set is then the top M =
// (length - 1) / 3 keys: one block radix-selects the M-th key.  Leaf counts
// go bottom-up and Z-order offsets top-down; each leaf writes its entry.
#include <climits>
#include <cstdint>

#include "fbp_internal.cuh"
#include "sap.h"

namespace fbp {
void clear_error();
namespace {

constexpr int kTile = 32, kHalo = 4, kSpan = kTile + 2 * kHalo;   // 40
constexpr int kTan22 = 13573, kTan67 = 79109;                     // tan(22.5), tan(67.5) x 2^15
constexpr int kUnionCap = 1 << 22;
constexpr int kFlag = 1 << 30;            // "component holds a strong pixel", on the root's entry
constexpr int kLabelMask = kFlag - 1;

__device__ __forceinline__ int clampi(int v, int hi) { return v < 0 ? 0 : v > hi ? hi : v; }

// ---------------------------------------------------------------------------
// Canny: classes (0 none, 1 weak, 2 strong), the edge map cleared, and the
// candidates appended to a list with their labels initialised
// ---------------------------------------------------------------------------
template <bool CLAMP>
__device__ __forceinline__ int cl(int v, int nm) { return CLAMP ? clampi(v, nm) : v; }

struct CannyArgs {
    const unsigned short *img;
    int n, lo, hi;
    int vec;                     // img is 8-byte aligned: interior tiles load 4 codes at a time
    unsigned char *cls, *edges;
    int *label, *list, *count;
};

// Every staged array is indexed by (y - (ty0 - 4), x - (tx0 - 4)) and holds
// the stage's value at the clamped coordinate (clamp(y), clamp(x)); in an
// interior tile no coordinate needs clamping.  Border tiles run canny_tile
// (CLAMP true), whose stages walk a region W wide with a linear thread
// index; a warp that wraps into the next row is conflict-free when the row
// stride S satisfies S = W (mod 32), so each array's stride matches the
// width its main reader walks: the input and the horizontal pass are read
// 36 wide (S = 68), the smoothed image 34 wide (S = 66), the magnitude 32
// wide (S = 64).  Interior tiles run canny_interior, whose warps read 32
// consecutive words of one row (conflict-free at any stride).  The
// gradients reuse the first two buffers, which are dead by then.
constexpr int kSin = 68, kShh = 68, kSss = 66, kSmm = 64;
constexpr int kCannySmem = kSpan * (kSin + kShh + kSss + kSmm);   // ints

__device__ __forceinline__ void canny_nms(const CannyArgs &a, const int *GX, const int *GY, const int *MM);

template <bool CLAMP>
__device__ __forceinline__ void canny_tile(const CannyArgs &a, int *IN, int *HH, int *SS, int *MM)
{
    int *GX = IN, *GY = HH;
    const int n = a.n, nm = n - 1;
    const int ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
    const int oy = ty0 - kHalo, ox = tx0 - kHalo;
    const int t = threadIdx.x;
    auto iy = [&](int y) { return cl<CLAMP>(y, nm) - oy; };
    auto ix = [&](int x) { return cl<CLAMP>(x, nm) - ox; };

    if (CLAMP) {
        for (int i = t; i < kSpan * kSpan; i += 256) {
            const int r = i / kSpan, c = i - r * kSpan;
            IN[r * kSin + c] = a.img[(size_t)clampi(oy + r, nm) * n + clampi(ox + c, nm)];
        }
    } else {
        // rows of 40 codes from an 8-byte aligned start (ox = 32 bx - 4): 10 x 8 bytes,
        // stored as one 16-byte vector (the row stride is a multiple of 4 words)
        for (int i = t; i < kSpan * (kSpan / 4); i += 256) {
            const int r = i / (kSpan / 4), c4 = i - r * (kSpan / 4);
            const uint2 v = *reinterpret_cast<const uint2 *>(a.img + (size_t)(oy + r) * n + ox + 4 * c4);
            *reinterpret_cast<int4 *>(IN + r * kSin + 4 * c4) =
                make_int4((int)(v.x & 0xffffu), (int)(v.x >> 16), (int)(v.y & 0xffffu), (int)(v.y >> 16));
        }
    }
    __syncthreads();
    // horizontal binomial, columns needed by the vertical pass: [2, 38)
    for (int i = t; i < kSpan * (kSpan - 4); i += 256) {
        const int r = i / (kSpan - 4), c = 2 + i % (kSpan - 4);
        const int x = cl<CLAMP>(ox + c, nm);
        const int *row = IN + r * kSin;
        HH[r * kShh + c] = row[ix(x - 2)] + 4 * row[ix(x - 1)] + 6 * row[ix(x)] + 4 * row[ix(x + 1)] +
                           row[ix(x + 2)];
    }
    __syncthreads();
    // vertical binomial on [2, 38) x [2, 38)
    for (int i = t; i < (kSpan - 4) * (kSpan - 4); i += 256) {
        const int r = 2 + i / (kSpan - 4), c = 2 + i % (kSpan - 4);
        const int y = cl<CLAMP>(oy + r, nm);
        SS[r * kSss + c] = HH[iy(y - 2) * kShh + c] + 4 * HH[iy(y - 1) * kShh + c] + 6 * HH[iy(y) * kShh + c] +
                           4 * HH[iy(y + 1) * kShh + c] + HH[iy(y + 2) * kShh + c];
    }
    __syncthreads();
    // Sobel and L1 magnitude on [3, 37) x [3, 37)
    for (int i = t; i < (kSpan - 6) * (kSpan - 6); i += 256) {
        const int r = 3 + i / (kSpan - 6), c = 3 + i % (kSpan - 6);
        const int y = cl<CLAMP>(oy + r, nm), x = cl<CLAMP>(ox + c, nm);
        const int *rm = SS + iy(y - 1) * kSss, *r0 = SS + iy(y) * kSss, *rp = SS + iy(y + 1) * kSss;
        const int xm = ix(x - 1), x0 = ix(x), xp = ix(x + 1);
        const int gx = (rm[xp] + 2 * r0[xp] + rp[xp]) - (rm[xm] + 2 * r0[xm] + rp[xm]);
        const int gy = (rp[xm] + 2 * rp[x0] + rp[xp]) - (rm[xm] + 2 * rm[x0] + rm[xp]);
        GX[r * kSin + c] = gx;
        GY[r * kShh + c] = gy;
        MM[r * kSmm + c] = abs(gx) + abs(gy);
    }
    __syncthreads();
    canny_nms(a, GX, GY, MM);
}

// Non-maximum suppression and thresholds on the tile; every thread runs all
// four rounds (1024 pixels / 256 threads) so the warp votes are full.
__device__ __forceinline__ void canny_nms(const CannyArgs &a, const int *GX, const int *GY, const int *MM)
{
    const int n = a.n;
    const int oy = blockIdx.y * kTile - kHalo, ox = blockIdx.x * kTile - kHalo;
    const int t = threadIdx.x, lane = t & 31;
    for (int i = t; i < kTile * kTile; i += 256) {
        const int r = kHalo + i / kTile, c = kHalo + i % kTile;
        const int y = oy + r, x = ox + c;
        const bool inside = y < n && x < n;
        unsigned char k = 0;
        const int m = MM[r * kSmm + c];
        if (inside && m > a.lo) {
            const int gx = GX[r * kSin + c], gy = GY[r * kShh + c];
            const long long ax = abs(gx), ay = abs(gy);
            int dy, dx;
            if (ay * 32768 <= (long long)kTan22 * ax) { dy = 0; dx = 1; }
            else if (ay * 32768 >= (long long)kTan67 * ax) { dy = 1; dx = 0; }
            else if ((gx > 0) == (gy > 0)) { dy = 1; dx = 1; }
            else { dy = 1; dx = -1; }
            const int py = y - dy, px = x - dx, qy = y + dy, qx = x + dx;
            const int prev = (py >= 0 && py < n && px >= 0 && px < n) ? MM[(r - dy) * kSmm + c - dx] : 0;
            const int next = (qy >= 0 && qy < n && qx >= 0 && qx < n) ? MM[(r + dy) * kSmm + c + dx] : 0;
            if (m > prev && m >= next) k = m > a.hi ? 2 : 1;
        }
        const size_t p = (size_t)y * n + x;
        if (inside) {
            a.cls[p] = k;
            a.edges[p] = 0;
        }
        const unsigned vote = __ballot_sync(0xffffffffu, k != 0);
        int base = 0;
        if (lane == 0 && vote) base = atomicAdd(a.count, __popc(vote));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (k) {
            a.list[base + __popc(vote & ((1u << lane) - 1))] = (int)p;
            a.label[p] = (int)p;
        }
    }
}

// Interior tiles (no coordinate needs clamping, 8-byte aligned rows): the
// same integer stages as canny_tile, with fewer loads and index operations
// per output.  The horizontal binomial takes four outputs per work item from
// two 16-byte loads; the vertical binomial and the Sobel pass take a run of
// rows of one column per item and slide a register window down it, so each
// input is loaded once per run.  Work items are numbered so that a warp's
// lanes read consecutive words (or 16-byte slots) of a row.
constexpr int kRuns = 8;   // row runs of the vertical and Sobel passes

__device__ __forceinline__ void canny_interior(const CannyArgs &a, int *IN, int *HH, int *SS, int *MM)
{
    int *GX = IN, *GY = HH;
    const int n = a.n;
    const int oy = blockIdx.y * kTile - kHalo, ox = blockIdx.x * kTile - kHalo;
    const int t = threadIdx.x;
    for (int i = t; i < kSpan * (kSpan / 4); i += 256) {
        const int r = i / (kSpan / 4), c4 = i - r * (kSpan / 4);
        const uint2 v = *reinterpret_cast<const uint2 *>(a.img + (size_t)(oy + r) * n + ox + 4 * c4);
        *reinterpret_cast<int4 *>(IN + r * kSin + 4 * c4) =
            make_int4((int)(v.x & 0xffffu), (int)(v.x >> 16), (int)(v.y & 0xffffu), (int)(v.y >> 16));
    }
    __syncthreads();
    // horizontal binomial, rows [0, 40), columns [2, 38): item (r, g) reads
    // columns 4g .. 4g+7 and writes columns 4g+2 .. 4g+5
    constexpr int G = (kSpan - 4) / 4;                    // 9 groups per row
    for (int it = t; it < kSpan * G; it += 256) {
        const int r = it / G, g = it - r * G;
        const int *row = IN + r * kSin + 4 * g;
        const int4 A = *reinterpret_cast<const int4 *>(row);
        const int4 B = *reinterpret_cast<const int4 *>(row + 4);
        int *h = HH + r * kShh + 4 * g + 2;
        *reinterpret_cast<int2 *>(h) = make_int2(A.x + 4 * A.y + 6 * A.z + 4 * A.w + B.x,
                                                 A.y + 4 * A.z + 6 * A.w + 4 * B.x + B.y);
        *reinterpret_cast<int2 *>(h + 2) = make_int2(A.z + 4 * A.w + 6 * B.x + 4 * B.y + B.z,
                                                     A.w + 4 * B.x + 6 * B.y + 4 * B.z + B.w);
    }
    __syncthreads();
    // vertical binomial on [2, 38)^2: item (run, c), runs of 5, 5, 5, 5, 4, 4, 4, 4 rows
    constexpr int CV = kSpan - 4;                         // 36 columns
    for (int it = t; it < kRuns * CV; it += 256) {
        const int run = it / CV, c = 2 + (it - run * CV);
        const int r0 = run < 4 ? 2 + 5 * run : 22 + 4 * (run - 4);
        const int len = run < 4 ? 5 : 4;
        const int *col = HH + c;
        int w0 = col[(r0 - 2) * kShh], w1 = col[(r0 - 1) * kShh];
        int w2 = col[r0 * kShh], w3 = col[(r0 + 1) * kShh];
        for (int k = 0; k < len; ++k) {
            const int r = r0 + k;
            const int w4 = col[(r + 2) * kShh];
            SS[r * kSss + c] = w0 + 4 * w1 + 6 * w2 + 4 * w3 + w4;
            w0 = w1;
            w1 = w2;
            w2 = w3;
            w3 = w4;
        }
    }
    __syncthreads();
    // Sobel and L1 magnitude on [3, 37)^2: item (run, c), runs of 5, 5, 4 x 6
    // rows; rows r-1, r, r+1 of columns c-1, c, c+1 slide down
    constexpr int CS = kSpan - 6;                         // 34 columns
    for (int it = t; it < kRuns * CS; it += 256) {
        const int run = it / CS, c = 3 + (it - run * CS);
        const int r0 = run < 2 ? 3 + 5 * run : 13 + 4 * (run - 2);
        const int len = run < 2 ? 5 : 4;
        const int *sc = SS + c;
        int um = sc[(r0 - 1) * kSss - 1], u0 = sc[(r0 - 1) * kSss], up = sc[(r0 - 1) * kSss + 1];
        int vm = sc[r0 * kSss - 1], v0 = sc[r0 * kSss], vp = sc[r0 * kSss + 1];
        for (int k = 0; k < len; ++k) {
            const int r = r0 + k;
            const int wm = sc[(r + 1) * kSss - 1], w0 = sc[(r + 1) * kSss], wp = sc[(r + 1) * kSss + 1];
            const int gx = (up + 2 * vp + wp) - (um + 2 * vm + wm);
            const int gy = (wm + 2 * w0 + wp) - (um + 2 * u0 + up);
            GX[r * kSin + c] = gx;
            GY[r * kShh + c] = gy;
            MM[r * kSmm + c] = abs(gx) + abs(gy);
            um = vm;
            u0 = v0;
            up = vp;
            vm = wm;
            v0 = w0;
            vp = wp;
        }
    }
    __syncthreads();
    canny_nms(a, GX, GY, MM);
}

__global__ void __launch_bounds__(256) canny_kernel(CannyArgs a)
{
    __shared__ __align__(16) int smem[kCannySmem];
    int *IN = smem, *HH = IN + kSpan * kSin, *SS = HH + kSpan * kShh, *MM = SS + kSpan * kSss;
    const int oy = (int)blockIdx.y * kTile - kHalo, ox = (int)blockIdx.x * kTile - kHalo;
    if (a.vec && oy >= 0 && ox >= 0 && oy + kSpan <= a.n && ox + kSpan <= a.n)
        canny_interior(a, IN, HH, SS, MM);
    else
        canny_tile<true>(a, IN, HH, SS, MM);
}

// ---------------------------------------------------------------------------
// Hysteresis as connected components of the candidates
// ---------------------------------------------------------------------------
__device__ __forceinline__ int uf_find(int *L, int x, unsigned *status)
{
    // parent pointers only ever point to smaller indices, so the walk ends;
    // loads bypass L1 so that links made by other blocks are seen
    for (int it = 0; it < kUnionCap; ++it) {
        const int p = __ldcg(L + x);
        if (p == x) return x;
        const int gp = __ldcg(L + p);
        if (gp != p) L[x] = gp;            // path halving: every write moves to an ancestor
        x = gp;
    }
    atomicCAS(status, 0u, (unsigned)FAULT_UNION_CAP);
    return x;
}

// The root of x without writing: used once every union is done, where a
// path-halving write could otherwise replace another pixel's final root
// with an intermediate ancestor.
__device__ __forceinline__ int uf_root(const int *L, int x, unsigned *status)
{
    for (int it = 0; it < kUnionCap; ++it) {
        const int p = __ldcg(L + x);
        if (p == x) return x;
        x = p;
    }
    atomicCAS(status, 0u, (unsigned)FAULT_UNION_CAP);
    return x;
}

__device__ __forceinline__ void uf_unite(int *L, int a, int b, unsigned *status)
{
    for (int it = 0; it < kUnionCap; ++it) {
        a = uf_find(L, a, status);
        b = uf_find(L, b, status);
        if (a == b) return;
        if (a < b) { const int tmp = a; a = b; b = tmp; }   // link the larger root under the smaller
        const int old = atomicCAS(&L[a], a, b);
        if (old == a) return;
        a = old;                                             // a was linked meanwhile: retry from there
    }
    atomicCAS(status, 0u, (unsigned)FAULT_UNION_CAP);
}

// The passes below visit the candidates only (the list canny_kernel wrote).
__global__ void ccl_merge_kernel(const int *list, const int *count, const unsigned char *cls, int *label,
                                 int n, unsigned *status)
{
    const int c = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) {
        const int p = list[i];
        const int y = p / n, x = p - y * n;
        // forward neighbours: right, down-left, down, down-right
        if (x + 1 < n && cls[p + 1]) uf_unite(label, p, p + 1, status);
        if (y + 1 < n) {
            const int q = p + n;
            if (x > 0 && cls[q - 1]) uf_unite(label, p, q - 1, status);
            if (cls[q]) uf_unite(label, p, q, status);
            if (x + 1 < n && cls[q + 1]) uf_unite(label, p, q + 1, status);
        }
    }
}

__global__ void ccl_flatten_kernel(const int *list, const int *count, int *label, unsigned *status)
{
    const int c = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) {
        const int p = list[i];
        label[p] = uf_root(label, p, status);      // only this thread writes entry p
    }
}

__global__ void ccl_mark_kernel(const int *list, const int *count, const unsigned char *cls, int *label)
{
    const int c = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) {
        const int p = list[i];
        if (cls[p] == 2) atomicOr(&label[label[p] & kLabelMask], kFlag);
    }
}

__global__ void ccl_output_kernel(const int *list, const int *count, const int *label, unsigned char *edges)
{
    const int c = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) {
        const int p = list[i];
        if (label[label[p] & kLabelMask] & kFlag) edges[p] = 1;
    }
}

// ---------------------------------------------------------------------------
// Quadtree
// ---------------------------------------------------------------------------
__host__ __device__ constexpr long long level_base(int l) { return ((1LL << (2 * l)) - 1) / 3; }

__device__ __forceinline__ unsigned compact1(unsigned long long v)   // even bits -> integer
{
    v &= 0x5555555555555555ULL;
    v = (v | (v >> 1)) & 0x3333333333333333ULL;
    v = (v | (v >> 2)) & 0x0f0f0f0f0f0f0f0fULL;
    v = (v | (v >> 4)) & 0x00ff00ff00ff00ffULL;
    v = (v | (v >> 8)) & 0x0000ffff0000ffffULL;
    v = (v | (v >> 16)) & 0x00000000ffffffffULL;
    return (unsigned)v;
}

struct TreeArgs {
    const unsigned short *img;
    const unsigned char *edges;
    int n, P, L;                 // slice side, patch side, finest level (side P)
    int *V;                      // [T] edge counts
    long long *S1, *S2;          // [T] sums of codes and of squared codes
    double *KE;                  // [Ns] monotone variance keys
    ulonglong2 *K;               // [Ns] 128-bit keys (x = high word)
    unsigned char *split;        // [Ns]
    int *cnt, *off;              // [T] leaf counts, Z-order offsets
    ulonglong2 *thr;             // [1] the M-th largest key
    long long M;                 // splits
    int length;
    int *leaves;                 // [length][3]
    unsigned *status;
};

__global__ void stats_leaf_kernel(TreeArgs a)
{
    const long long count = 1LL << (2 * a.L);
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= count) return;
    const int X = (int)compact1((unsigned long long)m), Y = (int)compact1((unsigned long long)m >> 1);
    const int x0 = X * a.P, y0 = Y * a.P;
    int v = 0;
    long long s1 = 0, s2 = 0;
    for (int r = 0; r < a.P; ++r) {
        const size_t row = (size_t)(y0 + r) * a.n + x0;
        unsigned r1 = 0;
        unsigned long long r2 = 0;
        for (int c = 0; c < a.P; ++c) {
            const unsigned x = a.img[row + c];
            r1 += x;
            r2 += (unsigned long long)x * x;
            v += a.edges[row + c] ? 1 : 0;
        }
        s1 += r1;
        s2 += (long long)r2;
    }
    const long long idx = level_base(a.L) + m;
    a.V[idx] = v;
    a.S1[idx] = s1;
    a.S2[idx] = s2;
}

__global__ void stats_up_kernel(TreeArgs a, int l)
{
    const long long count = 1LL << (2 * l);
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= count) return;
    const long long c0 = level_base(l + 1) + 4 * m, idx = level_base(l) + m;
    a.V[idx] = a.V[c0] + a.V[c0 + 1] + a.V[c0 + 2] + a.V[c0 + 3];
    a.S1[idx] = a.S1[c0] + a.S1[c0 + 1] + a.S1[c0 + 2] + a.S1[c0 + 3];
    a.S2[idx] = a.S2[c0] + a.S2[c0 + 1] + a.S2[c0 + 2] + a.S2[c0 + 3];
}

// order-preserving map of a double to an unsigned integer
__device__ __forceinline__ unsigned long long sortable(double d)
{
    const long long b = __double_as_longlong(d);
    return b < 0 ? ~(unsigned long long)b : (unsigned long long)b | (1ULL << 63);
}

__global__ void keys_kernel(TreeArgs a, int l)
{
    const long long count = 1LL << (2 * l);
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= count) return;
    const long long idx = level_base(l) + m;
    const long long side = (long long)a.n >> l;
    // d(S2) - d(S1) * d(S1) / d(n), each operation rounded once
    const double s1 = __ll2double_rn(a.S1[idx]);
    const double t = __ddiv_rn(__dmul_rn(s1, s1), __ll2double_rn(side * side));
    double ke = __dsub_rn(__ll2double_rn(a.S2[idx]), t);
    if (l > 0) ke = fmin(ke, a.KE[level_base(l - 1) + (m >> 2)]);
    a.KE[idx] = ke;
    const unsigned long long s = sortable(ke);
    const unsigned long long mort = (unsigned long long)m << (2 * (a.L - l));   // corner in units of P
    ulonglong2 k;
    k.x = ((unsigned long long)a.V[idx] << 35) | (s >> 29);
    k.y = ((s & ((1ULL << 29) - 1)) << 35) | ((unsigned long long)(15 - l) << 31) | (0x7fffffffULL - mort);
    a.K[idx] = k;
}

// The M-th largest of the Ns keys, by MSB-first radix selection (8-bit
// digits) in one block: each pass counts the digit of every remaining key
// (per-warp histograms, one atomic per distinct digit in a warp) and picks
// the digit holding the M-th largest.  The remaining keys are those that
// match the digits chosen so far; when a pass drops at least a quarter of
// them they are copied to the other buffer (later passes read fewer keys),
// otherwise they stay in place and later passes check the prefix.
__device__ __forceinline__ unsigned digit_of(ulonglong2 k, int pass)
{
    const int sh = 56 - 8 * (pass & 7);
    return (unsigned)(((pass < 8 ? k.x : k.y) >> sh) & 0xff);
}

constexpr int kSelectBatch = 8;   // rounds of 1024 keys whose loads are issued together

__global__ void __launch_bounds__(1024) select_kernel(TreeArgs a, long long Ns, ulonglong2 *bufB,
                                                      ulonglong2 *bufC)
{
    __shared__ unsigned hist[32][256];
    __shared__ unsigned tot[256];
    __shared__ unsigned s_digit, s_next, s_pos;
    __shared__ long long s_krem;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (a.M <= 0) {
        if (t == 0) *a.thr = make_ulonglong2(~0ULL, ~0ULL);   // above every key (their top bit is 0)
        return;
    }
    if (t == 0) s_krem = a.M;
    const ulonglong2 *src = a.K;
    ulonglong2 *dst = bufB;
    long long cnt = Ns;                               // keys in src (some may not match the prefix)
    long long live = Ns;                              // keys matching the prefix
    unsigned long long tx = 0, ty = 0, mx = 0, my = 0;   // prefix and its mask
    for (int pass = 0; pass < 16; ++pass) {
        for (int i = t; i < 32 * 256; i += 1024) (&hist[0][0])[i] = 0;
        __syncthreads();
        // every warp runs the same number of rounds, so the warp-wide votes see
        // all lanes; the keys of kSelectBatch rounds are loaded before any is
        // counted, so their global-load latencies overlap
        for (long long b0 = 0; b0 < cnt; b0 += 1024 * kSelectBatch) {
            ulonglong2 kk[kSelectBatch];
#pragma unroll
            for (int u = 0; u < kSelectBatch; ++u) {
                const long long i = b0 + (long long)u * 1024 + t;
                kk[u] = i < cnt ? src[i] : make_ulonglong2(0, 0);
            }
#pragma unroll
            for (int u = 0; u < kSelectBatch; ++u) {
                const long long i = b0 + (long long)u * 1024 + t;
                const bool valid = i < cnt && (kk[u].x & mx) == tx && (kk[u].y & my) == ty;
                const unsigned d = valid ? digit_of(kk[u], pass) : 256u;
                const unsigned same = __match_any_sync(0xffffffffu, d);
                if (valid && lane == __ffs(same) - 1) atomicAdd(&hist[warp][d], __popc(same));
            }
        }
        __syncthreads();
        if (t < 256) {
            unsigned v = 0;
            for (int w = 0; w < 32; ++w) v += hist[w][t];
            tot[t] = v;
        }
        __syncthreads();
        if (t == 0) {
            long long cum = 0;
            int d = 255;
            for (; d > 0; --d) {
                if (cum + tot[d] >= s_krem) break;
                cum += tot[d];
            }
            s_krem -= cum;
            s_digit = (unsigned)d;
            s_next = tot[d];
            s_pos = 0;
        }
        __syncthreads();
        const unsigned d = s_digit;
        const int sh = 56 - 8 * (pass & 7);
        if (pass < 8) {
            tx |= (unsigned long long)d << sh;
            mx |= 0xffULL << sh;
        } else {
            ty |= (unsigned long long)d << sh;
            my |= 0xffULL << sh;
        }
        const long long next = s_next;
        if (pass == 15) break;
        if (4 * (live - next) < live) {               // drops under a quarter: keep the keys in place
            live = next;
            continue;
        }
        for (long long b0 = 0; b0 < cnt; b0 += 1024 * kSelectBatch) {
            ulonglong2 kk[kSelectBatch];
#pragma unroll
            for (int u = 0; u < kSelectBatch; ++u) {
                const long long i = b0 + (long long)u * 1024 + t;
                kk[u] = i < cnt ? src[i] : make_ulonglong2(0, 0);
            }
#pragma unroll
            for (int u = 0; u < kSelectBatch; ++u) {
                const long long i = b0 + (long long)u * 1024 + t;
                const bool keep = i < cnt && (kk[u].x & mx) == tx && (kk[u].y & my) == ty;
                const unsigned vote = __ballot_sync(0xffffffffu, keep);
                unsigned base = 0;
                if (lane == 0 && vote) base = atomicAdd(&s_pos, __popc(vote));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (keep) dst[base + __popc(vote & ((1u << lane) - 1))] = kk[u];
            }
        }
        __syncthreads();
        cnt = live = next;
        src = dst;
        dst = dst == bufB ? bufC : bufB;
    }
    if (t == 0) *a.thr = make_ulonglong2(tx, ty);
}

__device__ __forceinline__ bool key_ge(ulonglong2 k, ulonglong2 t)
{
    return k.x > t.x || (k.x == t.x && k.y >= t.y);
}

// bottom-up: split flags (levels < L) and leaf counts
__global__ void counts_kernel(TreeArgs a, int l)
{
    const long long count = 1LL << (2 * l);
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= count) return;
    const long long idx = level_base(l) + m;
    if (l == a.L) {
        a.cnt[idx] = 1;
        return;
    }
    const bool sp = key_ge(a.K[idx], *a.thr);
    a.split[idx] = sp ? 1 : 0;
    const long long c0 = level_base(l + 1) + 4 * m;
    a.cnt[idx] = sp ? a.cnt[c0] + a.cnt[c0 + 1] + a.cnt[c0 + 2] + a.cnt[c0 + 3] : 1;
}

// top-down: Z-order offsets, and the leaves' entries
__global__ void offsets_kernel(TreeArgs a, int l)
{
    const long long count = 1LL << (2 * l);
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= count) return;
    const long long idx = level_base(l) + m;
    bool reached = true;
    int o = 0;
    if (l > 0) {
        const long long pidx = level_base(l - 1) + (m >> 2);
        reached = a.split[pidx] != 0;
        o = a.off[pidx];
        const long long c0 = level_base(l) + (m & ~3LL);
        for (long long j = c0; j < idx; ++j) o += a.cnt[j];
    }
    a.off[idx] = o;
    const bool leaf = reached && (l == a.L || a.split[idx] == 0);
    if (!leaf) return;
    if (o < 0 || o >= a.length) {
        atomicCAS(a.status, 0u, (unsigned)FAULT_LEAF);
        return;
    }
    const int s = a.n >> l;
    a.leaves[3 * o + 0] = (int)compact1((unsigned long long)m) * s;
    a.leaves[3 * o + 1] = (int)compact1((unsigned long long)m >> 1) * s;
    a.leaves[3 * o + 2] = s;
}

__device__ __forceinline__ bool leaf_ok(int x0, int y0, int s, int n, int P)
{
    return s >= P && s <= n && (s & (s - 1)) == 0 && x0 >= 0 && y0 >= 0 && x0 % s == 0 && y0 % s == 0 &&
           x0 <= n - s && y0 <= n - s;
}

__device__ __forceinline__ unsigned long long spread1(unsigned v)      // integer -> even bits
{
    unsigned long long x = v;
    x = (x | (x << 16)) & 0x0000ffff0000ffffULL;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffULL;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0fULL;
    x = (x | (x << 2)) & 0x3333333333333333ULL;
    x = (x | (x << 1)) & 0x5555555555555555ULL;
    return x;
}

// one thread per patch element: the mean of its f x f block.  A block of
// side f >= P is a quadtree node, whose exact sum S1 is already in the
// pyramid; smaller blocks (f < P) are summed from the codes.
__global__ void extract_kernel(TreeArgs a, float *patches)
{
    const int P = a.P;
    const long long total = (long long)a.length * P * P;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int i = (int)(e / (P * P)), rc = (int)(e - (long long)i * P * P);
    const int r = rc / P, c = rc - r * P;
    const int x0 = a.leaves[3 * i], y0 = a.leaves[3 * i + 1], s = a.leaves[3 * i + 2];
    if (!leaf_ok(x0, y0, s, a.n, P)) {
        atomicCAS(a.status, 0u, (unsigned)FAULT_LEAF);
        return;
    }
    const int f = s / P;
    long long sum = 0;
    if (f >= P) {
        const int lf = (__ffs(a.n) - 1) - (__ffs(f) - 1);          // level whose side is f
        const unsigned bx = (unsigned)(x0 / f + c), by = (unsigned)(y0 / f + r);
        sum = a.S1[level_base(lf) + (long long)(spread1(bx) | (spread1(by) << 1))];
    } else {
        for (int yy = 0; yy < f; ++yy) {
            const unsigned short *row = a.img + (size_t)(y0 + r * f + yy) * a.n + x0 + c * f;
            unsigned rs = 0;
            for (int xx = 0; xx < f; ++xx) rs += row[xx];
            sum += rs;
        }
    }
    patches[e] = __double2float_rn(__ddiv_rn(__ll2double_rn(sum), __ll2double_rn((long long)f * f)));
}

// one block per (leaf, row phase): writes the leaf's packed bytes, a 4-byte
// word (16 pixels) at a time where the leaf is at least 16 pixels wide.
// f = s / P is a power of two, so patch coordinates are shifts; where
// f >= 16 one patch value covers the whole word.
constexpr int kRowPhases = 4;
__global__ void __launch_bounds__(128) depatch_pack_kernel(const unsigned char *mask, const int *leaves, int n,
                                                          int P, unsigned char *packed, int words,
                                                          unsigned *status)
{
    const int i = blockIdx.x;
    const int x0 = leaves[3 * i], y0 = leaves[3 * i + 1], s = leaves[3 * i + 2];
    if (!leaf_ok(x0, y0, s, n, P)) {
        if (threadIdx.x == 0 && blockIdx.y == 0) atomicCAS(status, 0u, (unsigned)FAULT_LEAF);
        return;
    }
    const int by = blockIdx.y;
    if (by >= s) return;
    const int lf = (__ffs(s) - 1) - (__ffs(P) - 1);             // log2 f
    const int rows = (s - by + kRowPhases - 1) / kRowPhases;     // rows by, by + 4, ... < s
    const unsigned char *mp = mask + (size_t)i * P * P;
    if (words && s >= 16) {
        const int wpr = s >> 4;
        for (int it = threadIdx.x; it < rows * wpr; it += blockDim.x) {
            const int yy = by + kRowPhases * (it / wpr), w = it % wpr;
            const unsigned char *prow = mp + (size_t)(yy >> lf) * P;
            unsigned v;
            if (lf >= 4) {
                v = (unsigned)(prow[(16 * w) >> lf] & 3) * 0x55555555u;     // one value, 16 copies
            } else {
                v = 0;
#pragma unroll
                for (int q = 0; q < 16; ++q) v |= (unsigned)(prow[(16 * w + q) >> lf] & 3) << (2 * q);
            }
            *reinterpret_cast<unsigned *>(packed + (size_t)(y0 + yy) * (n / 4) + x0 / 4 + 4 * w) = v;
        }
    } else {
        const int bpr = s / 4;
        for (int it = threadIdx.x; it < rows * bpr; it += blockDim.x) {
            const int yy = by + kRowPhases * (it / bpr), k = it % bpr;
            const unsigned char *prow = mp + (size_t)(yy >> lf) * P;
            unsigned b = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) b |= (unsigned)(prow[(4 * k + q) >> lf] & 3) << (2 * q);
            packed[(size_t)(y0 + yy) * (n / 4) + x0 / 4 + k] = (unsigned char)b;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int log2i(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

fbp_status check_params(const sap_params *p)
{
    if (!p) return fail(FBP_ERR_INVALID_ARG, "params is NULL");
    if (p->n < 16 || p->n > 16384 || (p->n & (p->n - 1)))
        return fail(FBP_ERR_INVALID_ARG, "n = %d must be a power of two in [16, 16384]", p->n);
    if (p->patch != 4 && p->patch != 8 && p->patch != 16 && p->patch != 32 && p->patch != 64)
        return fail(FBP_ERR_INVALID_ARG, "patch = %d must be 4, 8, 16, 32 or 64", p->patch);
    if (p->patch > p->n) return fail(FBP_ERR_INVALID_ARG, "patch %d > n %d", p->patch, p->n);
    const long long cells = (long long)(p->n / p->patch) * (p->n / p->patch);
    if (p->length < 1 || p->length > cells || (p->length - 1) % 3)
        return fail(FBP_ERR_INVALID_ARG, "length %d must be 1 mod 3 and in [1, %lld]", p->length, cells);
    if (p->canny_lo < 0 || p->canny_hi < p->canny_lo)
        return fail(FBP_ERR_INVALID_ARG, "need 0 <= canny_lo <= canny_hi");
    return FBP_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t label, cls, list, count, edges_end;                     // sap_edges
    size_t V, S1, S2, KE, K, KB, KC, split, cnt, off, thr, tree_end;   // sap_patches
    long long T, Ns;
    int L;
};

Layout layout(const sap_params &p)
{
    Layout o{};
    const size_t px = (size_t)p.n * p.n;
    o.label = 0;
    o.list = align256(px * 4);
    o.cls = o.list + align256(px * 4);
    o.count = o.cls + align256(px);
    o.edges_end = o.count + 256;
    o.L = log2i(p.n / p.patch);
    o.T = level_base(o.L + 1);
    o.Ns = level_base(o.L);
    size_t q = 0;
    o.V = q;     q += align256((size_t)o.T * 4);
    o.S1 = q;    q += align256((size_t)o.T * 8);
    o.S2 = q;    q += align256((size_t)o.T * 8);
    o.KE = q;    q += align256((size_t)(o.Ns ? o.Ns : 1) * 8);
    o.K = q;     q += align256((size_t)(o.Ns ? o.Ns : 1) * 16);
    o.KB = q;    q += align256((size_t)(o.Ns ? o.Ns : 1) * 16);
    o.KC = q;    q += align256((size_t)(o.Ns ? o.Ns : 1) * 16);
    o.split = q; q += align256((size_t)(o.Ns ? o.Ns : 1));
    o.cnt = q;   q += align256((size_t)o.T * 4);
    o.off = q;   q += align256((size_t)o.T * 4);
    o.thr = q;   q += 256;
    o.tree_end = q;
    return o;
}

fbp_status check_ws(void *ws, size_t bytes, size_t need)
{
    if (!ws) return fail(FBP_ERR_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(FBP_ERR_WORKSPACE, "workspace is not 256-byte aligned");
    if (bytes < need) return fail(FBP_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", bytes, need);
    return FBP_OK;
}

unsigned grid_for(long long items, int threads)
{
    const long long g = (items + threads - 1) / threads;
    return (unsigned)(g < 1 ? 1 : g);
}

template <typename F>
fbp_status guarded(F &&f)
{
    clear_error();
    try {
        return f();
    } catch (...) {
        return fail(FBP_ERR_CUDA, "unexpected host exception");
    }
}

}  // namespace
}  // namespace fbp

using namespace fbp;

extern "C" {

size_t sap_workspace_bytes(const sap_params *p)
{
    if (check_params(p) != FBP_OK) return 0;
    const Layout o = layout(*p);
    return o.edges_end > o.tree_end ? o.edges_end : o.tree_end;
}

fbp_status sap_edges(const unsigned short *slice, unsigned char *edges, const sap_params *p, void *workspace,
                     size_t ws_bytes, fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        fbp_status st = check_params(p);
        if (st != FBP_OK) return st;
        if (!slice || !edges) return fail(FBP_ERR_INVALID_ARG, "slice or edges is NULL");
        st = check_ws(workspace, ws_bytes, sap_workspace_bytes(p));
        if (st != FBP_OK) return st;
        unsigned *status = nullptr;
        st = device_status_word(&status);
        if (st != FBP_OK) return st;
        const Layout o = layout(*p);
        char *ws = static_cast<char *>(workspace);
        CannyArgs ca;
        ca.img = slice;
        ca.n = p->n;
        ca.lo = p->canny_lo;
        ca.hi = p->canny_hi;
        ca.vec = (reinterpret_cast<uintptr_t>(slice) & 7) == 0 ? 1 : 0;
        ca.cls = reinterpret_cast<unsigned char *>(ws + o.cls);
        ca.edges = edges;
        ca.label = reinterpret_cast<int *>(ws + o.label);
        ca.list = reinterpret_cast<int *>(ws + o.list);
        ca.count = reinterpret_cast<int *>(ws + o.count);
        const int n = p->n;
        FBP_CUDA_TRY(cudaMemsetAsync(ca.count, 0, sizeof(int), stream));
        dim3 tiles((n + kTile - 1) / kTile, (n + kTile - 1) / kTile);
        canny_kernel<<<tiles, 256, 0, stream>>>(ca);
        FBP_CUDA_TRY(cudaGetLastError());
        const unsigned g = 152u * 8u;        // grid-stride over the candidate list
        ccl_merge_kernel<<<g, 256, 0, stream>>>(ca.list, ca.count, ca.cls, ca.label, n, status);
        FBP_CUDA_TRY(cudaGetLastError());
        ccl_flatten_kernel<<<g, 256, 0, stream>>>(ca.list, ca.count, ca.label, status);
        FBP_CUDA_TRY(cudaGetLastError());
        ccl_mark_kernel<<<g, 256, 0, stream>>>(ca.list, ca.count, ca.cls, ca.label);
        FBP_CUDA_TRY(cudaGetLastError());
        ccl_output_kernel<<<g, 256, 0, stream>>>(ca.list, ca.count, ca.label, edges);
        FBP_CUDA_TRY(cudaGetLastError());
        return FBP_OK;
    });
}

fbp_status sap_patches(const unsigned short *slice, const unsigned char *edges, float *patches, int *leaves,
                       const sap_params *p, void *workspace, size_t ws_bytes, fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        fbp_status st = check_params(p);
        if (st != FBP_OK) return st;
        if (!slice || !edges || !patches || !leaves)
            return fail(FBP_ERR_INVALID_ARG, "slice, edges, patches or leaves is NULL");
        st = check_ws(workspace, ws_bytes, sap_workspace_bytes(p));
        if (st != FBP_OK) return st;
        unsigned *status = nullptr;
        st = device_status_word(&status);
        if (st != FBP_OK) return st;
        const Layout o = layout(*p);
        char *ws = static_cast<char *>(workspace);
        TreeArgs a;
        a.img = slice;
        a.edges = edges;
        a.n = p->n;
        a.P = p->patch;
        a.L = o.L;
        a.V = reinterpret_cast<int *>(ws + o.V);
        a.S1 = reinterpret_cast<long long *>(ws + o.S1);
        a.S2 = reinterpret_cast<long long *>(ws + o.S2);
        a.KE = reinterpret_cast<double *>(ws + o.KE);
        a.K = reinterpret_cast<ulonglong2 *>(ws + o.K);
        a.split = reinterpret_cast<unsigned char *>(ws + o.split);
        a.cnt = reinterpret_cast<int *>(ws + o.cnt);
        a.off = reinterpret_cast<int *>(ws + o.off);
        a.thr = reinterpret_cast<ulonglong2 *>(ws + o.thr);
        a.M = (p->length - 1) / 3;
        a.length = p->length;
        a.leaves = leaves;
        a.status = status;
        const int L = o.L;
        stats_leaf_kernel<<<grid_for(1LL << (2 * L), 256), 256, 0, stream>>>(a);
        FBP_CUDA_TRY(cudaGetLastError());
        for (int l = L - 1; l >= 0; --l) {
            stats_up_kernel<<<grid_for(1LL << (2 * l), 256), 256, 0, stream>>>(a, l);
            FBP_CUDA_TRY(cudaGetLastError());
        }
        for (int l = 0; l < L; ++l) {
            keys_kernel<<<grid_for(1LL << (2 * l), 256), 256, 0, stream>>>(a, l);
            FBP_CUDA_TRY(cudaGetLastError());
        }
        select_kernel<<<1, 1024, 0, stream>>>(a, o.Ns, reinterpret_cast<ulonglong2 *>(ws + o.KB),
                                              reinterpret_cast<ulonglong2 *>(ws + o.KC));
        FBP_CUDA_TRY(cudaGetLastError());
        for (int l = L; l >= 0; --l) {
            counts_kernel<<<grid_for(1LL << (2 * l), 256), 256, 0, stream>>>(a, l);
            FBP_CUDA_TRY(cudaGetLastError());
        }
        for (int l = 0; l <= L; ++l) {
            offsets_kernel<<<grid_for(1LL << (2 * l), 256), 256, 0, stream>>>(a, l);
            FBP_CUDA_TRY(cudaGetLastError());
        }
        extract_kernel<<<grid_for((long long)p->length * p->patch * p->patch, 256), 256, 0, stream>>>(a, patches);
        FBP_CUDA_TRY(cudaGetLastError());
        return FBP_OK;
    });
}

fbp_status sap_depatch_pack(const unsigned char *mask_patches, const int *leaves, unsigned char *packed,
                            const sap_params *p, fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        fbp_status st = check_params(p);
        if (st != FBP_OK) return st;
        if (!mask_patches || !leaves || !packed)
            return fail(FBP_ERR_INVALID_ARG, "mask_patches, leaves or packed is NULL");
        unsigned *status = nullptr;
        st = device_status_word(&status);
        if (st != FBP_OK) return st;
        dim3 grid((unsigned)p->length, kRowPhases);
        const int words = (reinterpret_cast<uintptr_t>(packed) & 3) == 0 ? 1 : 0;
        depatch_pack_kernel<<<grid, 128, 0, stream>>>(mask_patches, leaves, p->n, p->patch, packed, words, status);
        FBP_CUDA_TRY(cudaGetLastError());
        return FBP_OK;
    });
}

}  // extern "C"
