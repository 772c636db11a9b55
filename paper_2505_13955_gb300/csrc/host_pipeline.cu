// host_pipeline.cu -- fbp_host: filtered backprojection of a stack held in
// host memory, with the copies of one chunk of slices overlapping the kernels
// of another.
//
// The paper's reconstruction stage moves projections in, reconstructs and
// stores slices as an overlapped pipeline (Sec. V-A(c): load, FBP
// computation, reduction, store), so that data movement hides behind
// computation.  On one GPU the load and the store are the host<->device
// copies: the stack is cut into chunks of `chunk` slices and chunk i runs on
// stream i mod n_streams -- copy in, filter, backproject, copy out -- each
// stream with its own buffers in the caller's workspace, so one stream's
// copies run while another's kernels do.  Every step is a call of the
// library's own device entry points on the chunk (fbp_backproject_staged or,
// for uint16 codes, fbp_backproject_staged_u16, with the chunk's tables in the
// stream's buffers, where the geometry has the orbit symmetry).  The internal
// streams and the start event come from a per-device pool, so a call on a
// small stack does not pay for creating and destroying them.
#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "bp_batch.cuh"
#include "fbp_internal.cuh"

using namespace fbp;

namespace fbp {
void clear_error();
}

namespace {

constexpr int kMaxHostStreams = 16;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct HostLayout {
    size_t in, filt, scale, out, table, per_stream;
};

// Slices whose geometry has the orbit symmetry (n a multiple of 64, at least
// 1024: smaller slices are launch-bound, and the table pass costs more than
// it saves) backproject through fbp_backproject_staged (FP32 out) or
// fbp_backproject_staged_u16 (codes out): each stream's buffers then include
// one chunk's tables.
bool host_staged(const fbp_geometry &g, bool)
{
    return g.n % 64 == 0 && g.n >= 1024 &&
           bp_orbit_geometry(g.n_angles, g.angle_step, g.n_det, g.det_center, g.n, 32);
}

// Internal streams and start events, kept per device and handed to one call
// at a time (a call takes what it needs from the free list and returns it).
struct HostResources {
    std::vector<cudaStream_t> streams;
    cudaEvent_t ready = nullptr;
};
std::mutex g_pool_mu;
std::map<int, std::vector<HostResources>> g_pool;

cudaError_t take_resources(int used, HostResources *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        std::vector<HostResources> &free = g_pool[dev];
        for (size_t i = 0; i < free.size(); ++i) {
            if ((int)free[i].streams.size() >= used) {
                *out = free[i];
                free.erase(free.begin() + (long)i);
                return cudaSuccess;
            }
        }
    }
    HostResources r;
    e = cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming);
    for (int i = 0; i < used && e == cudaSuccess; ++i) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) r.streams.push_back(s);
    }
    if (e != cudaSuccess) {
        for (cudaStream_t s : r.streams) cudaStreamDestroy(s);
        if (r.ready) cudaEventDestroy(r.ready);
        return e;
    }
    *out = r;
    return cudaSuccess;
}

void give_back(const HostResources &r)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lock(g_pool_mu);
    g_pool[dev].push_back(r);
}

HostLayout host_layout(const fbp_geometry &g, fbp_dtype dtype, int chunk, bool codes)
{
    HostLayout l;
    const size_t rows = (size_t)chunk * g.n_angles;
    l.in = align256(rows * g.n_det * sizeof(float));
    l.filt = align256(rows * g.n_det * (dtype == FBP_F32 ? 4 : 2));
    l.scale = dtype == FBP_F32 ? 0 : align256(rows * sizeof(float));
    l.out = align256((size_t)chunk * g.n * g.n * (codes ? 2 : 4));
    l.table = host_staged(g, codes) ? align256(fbp_backproject_staged_workspace_bytes(&g, dtype, chunk)) : 0;
    l.per_stream = l.in + l.filt + l.scale + l.out + l.table;
    return l;
}

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice;
}

}  // namespace

extern "C" size_t fbp_host_workspace_bytes(const fbp_geometry *g, fbp_dtype dtype, int chunk,
                                           int n_streams, int codes)
{
    clear_error();
    if (!g || chunk < 1 || n_streams < 1 || n_streams > kMaxHostStreams) return 0;
    if (dtype != FBP_F32 && dtype != FBP_F16 && dtype != FBP_BF16) return 0;
    if (check_geometry(g, true, true) != FBP_OK) return 0;
    return (size_t)n_streams * host_layout(*g, dtype, chunk, codes != 0).per_stream;
}

extern "C" fbp_status fbp_host(const float *sino_host, void *slice_host, const fbp_geometry *g,
                               int n_slices, fbp_filter_kind kind, fbp_dtype dtype, int bp_variant,
                               const fbp_preprocess *pre, const fbp_hu_window *window, int chunk,
                               int n_streams, void *workspace, size_t ws_bytes, fbp_stream_t stream)
{
    clear_error();
    fbp_status st = check_geometry(g, true, true);
    if (st != FBP_OK) return st;
    if (dtype != FBP_F32 && dtype != FBP_F16 && dtype != FBP_BF16)
        return fail(FBP_ERR_INVALID_ARG, "dtype %d", (int)dtype);
    if (kind != FBP_FILTER_RAMLAK && kind != FBP_FILTER_SHEPP_LOGAN)
        return fail(FBP_ERR_INVALID_ARG, "filter kind %d", (int)kind);
    if (n_slices < 0) return fail(FBP_ERR_INVALID_ARG, "n_slices < 0");
    if (chunk < 1) return fail(FBP_ERR_INVALID_ARG, "chunk < 1");
    if (n_streams < 1 || n_streams > kMaxHostStreams)
        return fail(FBP_ERR_INVALID_ARG, "n_streams %d outside [1, %d]", n_streams, kMaxHostStreams);
    if (bp_variant < -1 || bp_variant >= bp_variant_count())
        return fail(FBP_ERR_INVALID_ARG, "variant %d", bp_variant);
    if (n_slices == 0) return FBP_OK;
    if (!sino_host || !slice_host) return fail(FBP_ERR_INVALID_ARG, "sino_host or slice_host is NULL");
    if (is_device_pointer(sino_host) || is_device_pointer(slice_host))
        return fail(FBP_ERR_INVALID_ARG, "sino_host and slice_host must be host memory");
    // the pre-processing and the window are checked here, before anything is
    // enqueued (a zero-slice call validates and enqueues nothing)
    if (pre && (st = fbp_filter_counts(nullptr, nullptr, nullptr, dtype, kind, g, 0, pre, stream)) != FBP_OK)
        return st;
    float hu_a = 0.f, hu_b = 0.f;
    if (window && (st = fbp_hu_coefficients(window, &hu_a, &hu_b)) != FBP_OK) return st;
    const bool codes = window != nullptr;
    const HostLayout l = host_layout(*g, dtype, chunk, codes);
    if (!workspace) return fail(FBP_ERR_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) & 255)
        return fail(FBP_ERR_WORKSPACE, "workspace is not 256-byte aligned");
    const int used = (int)std::min<long long>(n_streams, ((long long)n_slices + chunk - 1) / chunk);
    if (ws_bytes < (size_t)n_streams * l.per_stream)
        return fail(FBP_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", ws_bytes,
                    (size_t)n_streams * l.per_stream);

    const size_t K = (size_t)g->n_angles, D = (size_t)g->n_det, N = (size_t)g->n;
    const size_t in_slice = K * D * sizeof(float);
    const size_t out_slice = N * N * (codes ? 2 : 4);
    HostResources res;
    cudaError_t e = take_resources(used, &res);
    if (e != cudaSuccess) return cuda_fail(e, "fbp_host: streams");
    const std::vector<cudaStream_t> streams(res.streams.begin(), res.streams.begin() + used);
    // the pipeline starts after the work already enqueued on the caller's stream
    e = cudaEventRecord(res.ready, stream);
    for (int i = 0; i < used && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(streams[i], res.ready, 0);
    if (e != cudaSuccess) {
        give_back(res);
        return cuda_fail(e, "fbp_host: streams");
    }

    char *ws = static_cast<char *>(workspace);
    const char *src = reinterpret_cast<const char *>(sino_host);
    char *dst = static_cast<char *>(slice_host);
    st = FBP_OK;
    for (int c = 0, i0 = 0; i0 < n_slices && st == FBP_OK; ++c, i0 += chunk) {
        const int n = std::min(chunk, n_slices - i0);
        const int si = c % used;
        cudaStream_t s = streams[si];
        char *base = ws + (size_t)si * l.per_stream;
        float *d_in = reinterpret_cast<float *>(base);
        void *d_filt = base + l.in;
        float *d_scale = dtype == FBP_F32 ? nullptr : reinterpret_cast<float *>(base + l.in + l.filt);
        void *d_out = base + l.in + l.filt + l.scale;
        e = cudaMemcpyAsync(d_in, src + (size_t)i0 * in_slice, (size_t)n * in_slice, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "fbp_host: copy in");
            break;
        }
        st = pre ? fbp_filter_counts(d_in, d_filt, d_scale, dtype, kind, g, n, pre, s)
                 : fbp_filter(d_in, d_filt, d_scale, dtype, kind, g, n, s);
        if (st != FBP_OK) break;
        const float scale = (float)g->angle_step;
        if (codes && l.table && bp_variant < 0)
            st = fbp_backproject_staged_u16(d_filt, d_scale, dtype, static_cast<unsigned short *>(d_out), g, n,
                                            scale, window, -1, base + l.in + l.filt + l.scale + l.out, l.table, s);
        else if (codes)
            st = fbp_backproject_u16(d_filt, d_scale, dtype, static_cast<unsigned short *>(d_out), g, n, scale,
                                     window, bp_variant, s);
        else if (l.table && bp_variant < 0)
            st = fbp_backproject_staged(d_filt, d_scale, dtype, static_cast<float *>(d_out), g, n, scale, 0, -1,
                                        base + l.in + l.filt + l.scale + l.out, l.table, s);
        else
            st = fbp_backproject_variant(d_filt, d_scale, dtype, static_cast<float *>(d_out), g, n, scale, 0,
                                         bp_variant, s);
        if (st != FBP_OK) break;
        e = cudaMemcpyAsync(dst + (size_t)i0 * out_slice, d_out, (size_t)n * out_slice, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = cuda_fail(e, "fbp_host: copy out");
    }
    // wait for every stream (also after an error: nothing may still write the buffers)
    for (cudaStream_t s : streams) {
        const cudaError_t se = cudaStreamSynchronize(s);
        if (se != cudaSuccess && st == FBP_OK) st = cuda_fail(se, "fbp_host: synchronise");
    }
    give_back(res);
    return st;
}
