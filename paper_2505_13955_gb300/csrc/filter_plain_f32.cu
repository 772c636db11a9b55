// filter_plain_f32.cu -- K1's plain row-pair kernels with FP32 output
// (filter_impl.cuh), in a translation unit of their own.
#include "filter_impl.cuh"
#include "filter_launch.cuh"

namespace fbp {

fbp_status filter_plain_f32(const FilterLaunch &a, cudaStream_t s)
{
    return launch_plain_rows<float>(a, s);
}

}  // namespace fbp
