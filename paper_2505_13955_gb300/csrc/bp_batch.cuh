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
    int tiles_x, H;             // tiles per row, staged half-window
    int unit_begin;             // first work unit (tile) of this item
    int pad_;
};

struct BpBatchArgs {
    BpBatchItem items[kMaxBatch];
    int count, total_units, max_H;
    int cyclic;                 // 1: block b takes units b, b + P, b + 2P (P = grid); 0: atomic queue
    int *counter;               // work-queue counter (workspace), zeroed before launch
    unsigned *status;
};

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

fbp_status launch_bp_persistent(BpBatchArgs &a, int variant, fbp_dtype dtype, cudaStream_t s);
fbp_status launch_filter_batched(const FilterBatchArgs &a, int total_groups, fbp_dtype dtype,
                                 cudaStream_t s);
int filter_pairs_per_block(int L);   // row pairs one filter block transforms for length L
int bp_tile_w(int variant);
int bp_tile_h(int variant);

}  // namespace fbp
