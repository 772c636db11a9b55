// bp_batch.cuh -- descriptors of a ragged batch, passed by value as kernel
// parameters (so a captured CUDA graph holds them and no host->device copy
// is needed per call).
#pragma once

#include "fbp_internal.cuh"

namespace fbp {

constexpr int kMaxBatch = 256;

struct BpBatchItem {            // one slice of the batch, 80 bytes
    const void *filt;           // [K][D] filtered rows in the workspace
    const float *row_scale;     // [K] or null
    float *slice;               // [N][N] output
    const double2 *cs;          // [K] angle table
    double alpha, det_center;
    int K, D, N;
    float scale;                // angle_step
    int tiles_x, H;             // tiles (orbits) per row, staged half-window
    int unit_begin;             // first work unit (tile, or orbit of four tiles) of this item
    int orbit;                  // 1: units are 90-degree orbits (bp_orbit.cuh), 0: tiles
};

struct BpBatchArgs {
    BpBatchItem items[kMaxBatch];
    int count, total_units;
    int max_H, max_H_orbit;     // widest staged half-windows of the tile and the orbit items
    int cyclic;                 // 1: block b takes units b, b + P, b + 2P (P = grid); 0: atomic queue
    int *counter;               // work-queue counter (workspace), zeroed before launch
    unsigned *status;
};

static_assert(sizeof(BpBatchItem) == 80, "batch item layout");

struct FilterBatchItem {        // 88 bytes
    const float *sino;          // [K][D], or the offset scan's [K_in][Dp] physical rows
    void *filt;                 // [K][D] in the workspace
    float *row_scale;           // [K] or null
    const float2 *G;            // difference-form spectrum for (D, kind, tau), length L
    const float2 *tw;           // twiddles for L
    int K, D, L, group_begin;   // group = one block's filter_pairs_per_block(L) row pairs
    // offset scans (Dp > 0): physical bins, virtual index of bin 0, fold,
    // physical rows, virtual centre, side sign and 1 / overlap (filter.cu)
    int Dp, off, fold, K_in;
    float cv, sgn, inv_delta;
    int pad_;
};

struct FilterBatchArgs {
    FilterBatchItem items[kMaxBatch];
    int count;
};

// Staged ragged batches (bp_staged_batch.cu): orbit units (32 x 32 tiles for
// FP32 rows, 64 x 64 for 16-bit rows) fed by plain bulk copies from per-item
// padded tables.
struct StagedBatchItem {        // 88 bytes
    const void *table;          // padded table (16-bit: [K/2][Ep]; FP32: planes a, b of [K/2][Ep])
    float *slice;               // [N][N] output
    const double2 *cs;          // [K] angle table
    const float *smax;          // 16-bit rows: the item's S (written by the table pass); FP32: null
    double alpha, det_center;
    int K2, N, H, W, Ep, P_lo;  // angle pairs, image side, half-window, window, padded row, padding
    int tiles_x, unit_begin;    // orbits per row (N / (2 tile)), first unit of this item
    float scale;                // angle_step
    int pad_;
};

static_assert(sizeof(StagedBatchItem) == 88, "staged batch item layout");

struct StagedBatchArgs {
    StagedBatchItem items[kMaxBatch];
    int count, total_units;
    int Wp;                     // window pitch in shared memory (entries, multiple of 8, >= every W)
    int cyclic;                 // as BpBatchArgs
    int *counter;
    unsigned *status;
};

struct StagedPrepItem {         // 56 bytes
    const void *filt;           // [K][D] filtered rows
    const float *row_scale;     // [K] (16-bit rows) or null
    void *table;                // the item's padded table
    float *smax;                // 16-bit rows: where S goes; FP32: null
    int K, D, Ep, P_lo;
    int pair_begin, pad_;       // first angle pair of this item in the table pass's grid
};

static_assert(sizeof(StagedPrepItem) == 56, "table pass item layout");

struct StagedPrepArgs {
    StagedPrepItem items[kMaxBatch];
    int count, total_pairs;
};

// The padded table of one item: half-window H, window W and its pitch Wp,
// leading zero entries P_lo, padded row Ep, bytes of the table.
struct StagedItemGeom {
    int H, W, Wp, P_lo, Ep;
    size_t table_bytes;
};
// true if the item can run staged batch units (the orbit symmetry with the
// dtype's tile, a window of at most 72 (FP32) / 104 (16-bit) entries); fills
// *out.  Host only.
bool staged_batch_geometry(int K, double angle_step, int D, double det_center, int N, double alpha,
                           fbp_dtype dtype, StagedItemGeom *out);
int staged_batch_tile(fbp_dtype dtype);
fbp_status launch_staged_batch(const StagedPrepArgs &p, StagedBatchArgs &a, fbp_dtype dtype, cudaStream_t s);

fbp_status launch_bp_persistent(BpBatchArgs &a, int variant, fbp_dtype dtype, cudaStream_t s);
fbp_status launch_filter_batched(const FilterBatchArgs &a, int total_groups, fbp_dtype dtype,
                                 cudaStream_t s);
int filter_pairs_per_block(int L);   // row pairs one filter block transforms for length L
int bp_tile_w(int variant);
int bp_tile_h(int variant);
// The persistent kernel's shapes for `variant`: the orbit tile side (0 if the
// variant has no orbit form) and the generic tile it falls back to for items
// whose geometry has no 90-degree symmetry.
struct BpPersistentShape {
    int orbit_tile;
    int tile_w, tile_h;
};
bool bp_persistent_shape(int variant, fbp_dtype dtype, BpPersistentShape *out);
bool bp_orbit_geometry(int K, double angle_step, int D, double det_center, int N, int tile);

}  // namespace fbp
