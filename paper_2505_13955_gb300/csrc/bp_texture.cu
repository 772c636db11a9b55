// bp_texture.cu -- K2 through the texture unit: the measured alternative to
// the shared-memory tables.  Each slice's filtered rows [K][D] are bound as
// a pitched 2-D texture with linear filtering along the detector and zero
// outside it (border addressing); a fetch at (u + 1/2, k + 1/2) lands on
// angle k's texel centre, so the angle direction does not interpolate, and
// the hardware returns the linear interpolation of row k at u -- with the
// fraction quantised to the texture unit's fixed-point weights (8 fraction
// bits), which is this variant's accuracy cost.
//
// Layout: a block owns a 64 x 64 tile of one slice (256 threads, 4 x 4
// pixels each); per chunk of 256 angles, each thread forms one angle's
// tile-centre coordinate in FP64 (u_c + 1/2, split into an integer and a
// float fraction, as the table kernels do) and stores it in shared memory;
// each pixel then adds its small FP32 offset and fetches.  One texture
// covers a group of G consecutive slices (rows s K + k), so only the group's
// first row has to meet the texture unit's address alignment.
#include <algorithm>
#include <climits>
#include <vector>

#include "bp_tile.cuh"

namespace fbp {
namespace {

constexpr int kTexTile = 64, kTexThreads = 256, kTexChunk = 256;

struct TexArgs {
    cudaTextureObject_t tex;    // rows of the group's slices, [G K][D]
    float *out;                 // the group's first slice's [N][N], or null
    unsigned short *out16;      // or its uint16 codes
    float hu_a, hu_b;
    const double2 *cs;
    int K, N, tiles_x;
    double alpha, det_center;
    float scale;
    int accumulate;
};

__global__ void __launch_bounds__(kTexThreads) bp_texture_kernel(TexArgs a)
{
    __shared__ float4 prm[kTexChunk];             // (j_c, f_c, alpha cos, alpha sin)
    const int tile = blockIdx.x, sl = blockIdx.y;                 // slice within the group
    const int x0 = (tile % a.tiles_x) * kTexTile, y0 = (tile / a.tiles_x) * kTexTile;
    const float yrow = (float)sl * (float)a.K + 0.5f;             // texel centre of row (sl, 0)
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const double m = 0.5 * (a.N - 1);
    const double Xc = x0 + 0.5 * (kTexTile - 1) - m, Yc = y0 + 0.5 * (kTexTile - 1) - m;
    float acc[4][4];
#pragma unroll
    for (int iy = 0; iy < 4; ++iy)
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) acc[iy][ix] = 0.f;
    for (int k0 = 0; k0 < a.K; k0 += kTexChunk) {
        const int na = min(kTexChunk, a.K - k0);
        __syncthreads();
        if ((int)threadIdx.x < na) {
            const double2 cs = a.cs[k0 + threadIdx.x];
            const double c = a.alpha * cs.x, s = a.alpha * cs.y;
            const double uc = fma(c, Xc, fma(s, Yc, a.det_center)) + 0.5;   // texel-centre convention
            const double jc = floor(uc);
            prm[threadIdx.x] = make_float4((float)jc, (float)(uc - jc), (float)c, (float)s);
        }
        __syncthreads();
        for (int i = 0; i < na; ++i) {
            const float4 p = prm[i];
            const float yk = yrow + (float)(k0 + i);
#pragma unroll
            for (int iy = 0; iy < 4; ++iy) {
                const float dy = (float)(ty + 16 * iy) - 0.5f * (kTexTile - 1);
#pragma unroll
                for (int ix = 0; ix < 4; ++ix) {
                    const float dx = (float)(tx + 16 * ix) - 0.5f * (kTexTile - 1);
                    const float up = fmaf(dx, p.z, fmaf(dy, p.w, p.y));
                    acc[iy][ix] += tex2D<float>(a.tex, p.x + up, yk);
                }
            }
        }
    }
#pragma unroll
    for (int iy = 0; iy < 4; ++iy) {
        const int r = y0 + ty + 16 * iy;
        if (r >= a.N) continue;
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) {
            const int c = x0 + tx + 16 * ix;
            if (c >= a.N) continue;
            store_pixel(a.out, a.out16, a.hu_a, a.hu_b, a.accumulate,
                        ((size_t)sl * a.N + r) * a.N + c, acc[iy][ix] * a.scale);
        }
    }
}

struct TexAttrs {
    int align = 0, pitch_align = 0, max_w = 0, max_h = 0, max_pitch = 0;
};

fbp_status tex_attrs(TexAttrs *t)
{
    int dev = 0;
    FBP_CUDA_TRY(cudaGetDevice(&dev));
    FBP_CUDA_TRY(cudaDeviceGetAttribute(&t->align, cudaDevAttrTextureAlignment, dev));
    FBP_CUDA_TRY(cudaDeviceGetAttribute(&t->pitch_align, cudaDevAttrTexturePitchAlignment, dev));
    FBP_CUDA_TRY(cudaDeviceGetAttribute(&t->max_w, cudaDevAttrMaxTexture2DLinearWidth, dev));
    FBP_CUDA_TRY(cudaDeviceGetAttribute(&t->max_h, cudaDevAttrMaxTexture2DLinearHeight, dev));
    FBP_CUDA_TRY(cudaDeviceGetAttribute(&t->max_pitch, cudaDevAttrMaxTexture2DLinearPitch, dev));
    return FBP_OK;
}

}  // namespace

bool bp_texture_shape_ok(const BpLaunch &L)
{
    // FP32 rows whose row pitch (4 D bytes) is a multiple of 32 bytes and at
    // most 65,000 angles; the device limits are checked again at launch
    return L.dtype == FBP_F32 && L.D % 8 == 0 && L.K <= 65000 && L.D <= 131072;
}

fbp_status launch_backproject_texture(const BpLaunch &L, cudaStream_t s)
{
    if (!bp_texture_shape_ok(L))
        return fail(FBP_ERR_UNSUPPORTED, "texture variant needs FP32 rows, D a multiple of 8, K <= 65000");
    if (stream_is_capturing(s))
        return fail(FBP_ERR_UNSUPPORTED, "texture variant synchronises: not inside stream capture");
    TexAttrs ta;
    fbp_status st = tex_attrs(&ta);
    if (st != FBP_OK) return st;
    const size_t pitch = (size_t)L.D * sizeof(float);
    if (pitch % (size_t)ta.pitch_align || L.D > ta.max_w || L.K > ta.max_h || pitch > (size_t)ta.max_pitch)
        return fail(FBP_ERR_UNSUPPORTED, "rows exceed the texture unit's pitched 2-D limits");
    if (reinterpret_cast<uintptr_t>(L.filt) % (size_t)ta.align)
        return fail(FBP_ERR_UNSUPPORTED, "rows are not %d-byte aligned for a texture", ta.align);
    // slices per texture: at most max_h / K rows, and a multiple of the
    // smallest count m whose rows end on an aligned address
    const size_t slice_bytes = (size_t)L.K * pitch;
    size_t m = 1;
    while ((m * slice_bytes) % (size_t)ta.align) ++m;        // m <= align / 4
    const long long gmax = ta.max_h / L.K;
    long long G = (gmax / (long long)m) * (long long)m;
    if (G < 1) {
        if (L.S > gmax) return fail(FBP_ERR_UNSUPPORTED, "slices cannot be grouped into aligned textures");
        G = L.S;
    }
    G = std::min<long long>(G, std::min<long long>(L.S, 65535));
    const int tiles_x = (L.N + kTexTile - 1) / kTexTile;
    const long long tiles = (long long)tiles_x * tiles_x;
    if (tiles > INT_MAX) return fail(FBP_ERR_UNSUPPORTED, "too many tiles");

    std::vector<cudaTextureObject_t> texs;
    fbp_status result = FBP_OK;
    for (long long s0 = 0; s0 < L.S && result == FBP_OK; s0 += G) {
        const long long ns = std::min<long long>(G, L.S - s0);
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypePitch2D;
        rd.res.pitch2D.devPtr = const_cast<char *>(static_cast<const char *>(L.filt)) + (size_t)s0 * slice_bytes;
        rd.res.pitch2D.desc = cudaCreateChannelDesc<float>();
        rd.res.pitch2D.width = (size_t)L.D;
        rd.res.pitch2D.height = (size_t)(ns * L.K);
        rd.res.pitch2D.pitchInBytes = pitch;
        cudaTextureDesc td = {};
        td.addressMode[0] = cudaAddressModeBorder;     // zero outside the detector
        td.addressMode[1] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModeLinear;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        cudaTextureObject_t tex = 0;
        cudaError_t e = cudaCreateTextureObject(&tex, &rd, &td, nullptr);
        if (e != cudaSuccess) {
            result = cuda_fail(e, "cudaCreateTextureObject");
            break;
        }
        texs.push_back(tex);
        TexArgs a;
        a.tex = tex;
        a.out = L.slice ? L.slice + (size_t)s0 * L.N * L.N : nullptr;
        a.out16 = L.slice16 ? L.slice16 + (size_t)s0 * L.N * L.N : nullptr;
        a.hu_a = L.hu_a;
        a.hu_b = L.hu_b;
        a.cs = L.cs;
        a.K = L.K;
        a.N = L.N;
        a.tiles_x = tiles_x;
        a.alpha = L.alpha;
        a.det_center = L.det_center;
        a.scale = L.scale;
        a.accumulate = L.accumulate;
        bp_texture_kernel<<<dim3((unsigned)tiles, (unsigned)ns), kTexThreads, 0, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) result = cuda_fail(e, "bp_texture_kernel launch");
    }
    // the objects may only go once the launches that read them are done
    const cudaError_t es = cudaStreamSynchronize(s);
    for (cudaTextureObject_t t : texs) cudaDestroyTextureObject(t);
    if (result == FBP_OK && es != cudaSuccess) result = cuda_fail(es, "cudaStreamSynchronize");
    return result;
}

}  // namespace fbp
