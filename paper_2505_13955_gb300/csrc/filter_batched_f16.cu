// filter_batched_f16.cu -- K1's ragged-batch kernel with FP16 output
// (filter_impl.cuh), in a translation unit of their own.
#include "filter_impl.cuh"
#include "filter_launch.cuh"

namespace fbp {

fbp_status filter_batched_f16(const FilterBatchArgs &a, int groups, int max_L, cudaStream_t s)
{
    return launch_batched_t<__half>(a, groups, max_L, s);
}

}  // namespace fbp
