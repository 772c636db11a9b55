// filter_launch.cuh -- entry points of K1's per-output-type translation
// units (filter_{plain,stream,batched}_{f32,f16,bf16}.cu; kernels in
// filter_impl.cuh), called by the dispatch in filter.cu.
#pragma once

#include "bp_batch.cuh"
#include "fbp_internal.cuh"

namespace fbp {

constexpr int kFilterBlockThreads = 512;   // threads per filter block

// One launch over a.rows rows: a grid of row-pair groups (any length L).
fbp_status filter_plain_f32(const FilterLaunch &a, cudaStream_t s);
fbp_status filter_plain_f16(const FilterLaunch &a, cudaStream_t s);
fbp_status filter_plain_bf16(const FilterLaunch &a, cudaStream_t s);

// The persistent streamed form (L = 8192 or 16384, plain line-integral rows,
// D a multiple of 4, 16-byte aligned rows); status receives FAULT_STREAM_WAIT.
fbp_status filter_stream_f32(const FilterLaunch &a, unsigned *status, int skip_copies, cudaStream_t s);
fbp_status filter_stream_f16(const FilterLaunch &a, unsigned *status, int skip_copies, cudaStream_t s);
fbp_status filter_stream_bf16(const FilterLaunch &a, unsigned *status, int skip_copies, cudaStream_t s);

// A ragged batch in one launch of `groups` blocks; max_L = the batch's longest transform.
fbp_status filter_batched_f32(const FilterBatchArgs &a, int groups, int max_L, cudaStream_t s);
fbp_status filter_batched_f16(const FilterBatchArgs &a, int groups, int max_L, cudaStream_t s);
fbp_status filter_batched_bf16(const FilterBatchArgs &a, int groups, int max_L, cudaStream_t s);

}  // namespace fbp
