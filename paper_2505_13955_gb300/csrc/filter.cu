// filter.cu -- K1: the ramp-filter step of FBP (Sec. V-A(c) stage 2,
// "filtering", after Kak & Slaney ch. 3), as an FFT convolution of each
// projection row with the truncated band-limited ramp kernel.  The kernels
// and the transform's design are in filter_impl.cuh; this file chooses the
// kernel family and output type of each launch.
#include <cstdint>
#include <cstdlib>

#include "filter_launch.cuh"

namespace fbp {

int filter_pairs_per_block(int L) { return kFilterBlockThreads / (32 * fft_VPL(L)); }

fbp_status launch_filter(const FilterLaunch &a, cudaStream_t s)
{
    if (a.rows <= 0) return FBP_OK;
    // the persistent streamed form covers the one-pair-per-block lengths for
    // plain line-integral rows that the bulk-copy engine can move
    const bool streamed = !a.pre && !a.offset && (a.L == 8192 || a.L == 16384) && a.D % 4 == 0 &&
                          (reinterpret_cast<uintptr_t>(a.sino) & 15) == 0;
    if (streamed) {
        unsigned *status = nullptr;
        fbp_status st = device_status_word(&status);
        if (st != FBP_OK) return st;
        // failure-detection tests set FBP_TEST_STREAM_NO_COPY=1 so that the
        // kernel's waits run out (see filter_stream_kernel)
        const char *env = std::getenv("FBP_TEST_STREAM_NO_COPY");
        const int skip = (env && env[0] == '1') ? 1 : 0;
        switch (a.dtype) {
            case FBP_F32: return filter_stream_f32(a, status, skip, s);
            case FBP_F16: return filter_stream_f16(a, status, skip, s);
            case FBP_BF16: return filter_stream_bf16(a, status, skip, s);
        }
        return fail(FBP_ERR_INVALID_ARG, "dtype");
    }
    switch (a.dtype) {
        case FBP_F32: return filter_plain_f32(a, s);
        case FBP_F16: return filter_plain_f16(a, s);
        case FBP_BF16: return filter_plain_bf16(a, s);
    }
    return fail(FBP_ERR_INVALID_ARG, "dtype");
}

fbp_status launch_filter_batched(const FilterBatchArgs &a, int total_groups, fbp_dtype dtype,
                                 cudaStream_t s)
{
    if (total_groups <= 0) return FBP_OK;
    int max_L = 512;
    for (int i = 0; i < a.count; ++i) max_L = a.items[i].L > max_L ? a.items[i].L : max_L;
    switch (dtype) {
        case FBP_F32: return filter_batched_f32(a, total_groups, max_L, s);
        case FBP_F16: return filter_batched_f16(a, total_groups, max_L, s);
        case FBP_BF16: return filter_batched_bf16(a, total_groups, max_L, s);
    }
    return fail(FBP_ERR_INVALID_ARG, "dtype");
}

}  // namespace fbp
