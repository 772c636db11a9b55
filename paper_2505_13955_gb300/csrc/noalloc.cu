// noalloc.cu -- fbp_backproject_noalloc: the backprojection of
// fbp_backproject for callers that cannot allocate device memory.
//
// fbp_backproject reads its FP64 angle table from a per-geometry cache that
// the library fills with cudaMalloc on the first call for each geometry.  Some
// callers cannot allow that: code running under a framework that owns every
// byte of device memory through its own pool (any cudaMalloc outside it can
// fail or fragment the pool), and code whose device memory is fixed up front
// (embedded and real-time pipelines, where a failed allocation mid-run is not
// an option).  This entry point keeps
// the angle table in a file-scope static device array of fixed size instead,
// recomputes it on the caller's stream at every call, and calls no allocating
// routine.  The caller still provides the input rows and the output slices.
//
// The array lives for as long as the library is loaded, on every device that
// runs this entry point, and is shared by all calls: a call overwrites it
// completely before the backprojection reads it, but two calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// it and can read each other's angles.  Order such calls on one stream.
#include <map>
#include <mutex>

#include "fbp_internal.cuh"

namespace fbp {
namespace {

constexpr int kNoAllocMaxAngles = 16384;   // 16384 x 16 B = 256 KB per device

static __device__ __align__(256) double2 g_noalloc_angles[kNoAllocMaxAngles];

// Device address of the static array on the current device.  In host code
// the name g_noalloc_angles is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
fbp_status noalloc_table(double2 **out)
{
    static std::mutex mu;
    static std::map<int, double2 *> addr;
    int dev = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = addr.find(dev);
    if (it == addr.end()) {
        double2 *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_angles);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_angles)");
        it = addr.emplace(dev, p).first;
    }
    *out = it->second;
    return FBP_OK;
}

}  // namespace
}  // namespace fbp

using namespace fbp;

namespace fbp {
void clear_error();
}

extern "C" fbp_status fbp_backproject_noalloc(const void *filt, const float *row_scale,
                                              fbp_dtype dtype, float *slice,
                                              const fbp_geometry *g, int n_slices, float scale,
                                              int accumulate, fbp_stream_t stream)
{
    clear_error();
    fbp_status st = check_geometry(g, false, true);
    if (st != FBP_OK) return st;
    if (g->n_angles > kNoAllocMaxAngles)
        return fail(FBP_ERR_UNSUPPORTED,
                    "fbp_backproject_noalloc: n_angles = %d exceeds its fixed table of %d angles",
                    g->n_angles, kNoAllocMaxAngles);
    if (dtype != FBP_F32 && dtype != FBP_F16 && dtype != FBP_BF16)
        return fail(FBP_ERR_INVALID_ARG, "dtype %d", (int)dtype);
    if (n_slices < 0) return fail(FBP_ERR_INVALID_ARG, "n_slices < 0");
    if (!(scale == scale) || scale > 3.4e38f || scale < -3.4e38f)
        return fail(FBP_ERR_INVALID_ARG, "scale is not finite");
    if (n_slices == 0) return FBP_OK;
    if (!filt || !slice) return fail(FBP_ERR_INVALID_ARG, "filt or slice is NULL");
    if (dtype != FBP_F32 && !row_scale)
        return fail(FBP_ERR_INVALID_ARG, "row_scale is required for 16-bit input");
    // the same aliasing rule as fbp_backproject: the rows and the slices may not overlap
    const size_t nin = (size_t)n_slices * g->n_angles * g->n_det * (dtype == FBP_F32 ? 4 : 2);
    const size_t nout = (size_t)n_slices * g->n * g->n * 4;
    const char *pi = static_cast<const char *>(filt), *po = reinterpret_cast<const char *>(slice);
    if (pi < po + nout && po < pi + nin) return fail(FBP_ERR_INVALID_ARG, "slice overlaps filt");

    double2 *cs = nullptr;
    st = noalloc_table(&cs);
    if (st != FBP_OK) return st;
    const int K = g->n_angles;
    // the kernel that fills fbp_backproject's cached tables, so both read the same angles
    FBP_CUDA_TRY(enqueue_angle_table(cs, K, g->angle_start, g->angle_step, stream));

    BpLaunch a;
    a.filt = filt;
    a.row_scale = dtype == FBP_F32 ? nullptr : row_scale;
    a.slice = slice;
    a.cs = cs;
    a.K = K;
    a.D = g->n_det;
    a.N = g->n;
    a.S = n_slices;
    a.alpha = g->pixel_size / g->det_spacing;
    a.det_center = g->det_center;
    a.angle_step = g->angle_step;
    a.scale = scale;
    a.accumulate = accumulate ? 1 : 0;
    a.dtype = dtype;
    return launch_backproject(a, -1, stream);
}
