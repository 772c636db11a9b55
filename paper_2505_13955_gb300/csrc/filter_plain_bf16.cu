// filter_plain_bf16.cu -- K1's plain row-pair kernels with BF16 output
// (filter_impl.cuh), in a translation unit of their own.
#include "filter_impl.cuh"
#include "filter_launch.cuh"

namespace fbp {

fbp_status filter_plain_bf16(const FilterLaunch &a, cudaStream_t s)
{
    return launch_plain_rows<__nv_bfloat16>(a, s);
}

}  // namespace fbp
