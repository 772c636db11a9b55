// filter_stream_f32.cu -- K1's persistent streamed kernels with FP32 output
// (filter_impl.cuh), in a translation unit of their own.
#include "filter_impl.cuh"
#include "filter_launch.cuh"

namespace fbp {

fbp_status filter_stream_f32(const FilterLaunch &a, unsigned *status, int skip_copies, cudaStream_t s)
{
    return launch_streamed_rows<float>(a, status, skip_copies, s);
}

}  // namespace fbp
