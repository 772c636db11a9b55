// filter_stream_bf16.cu -- K1's persistent streamed kernels with BF16 output
// (filter_impl.cuh), in a translation unit of their own.
#include "filter_impl.cuh"
#include "filter_launch.cuh"

namespace fbp {

fbp_status filter_stream_bf16(const FilterLaunch &a, unsigned *status, int skip_copies, cudaStream_t s)
{
    return launch_streamed_rows<__nv_bfloat16>(a, status, skip_copies, s);
}

}  // namespace fbp
