// fbp_api.cu -- the exported C ABI of libfbp.so (declared in include/fbp.h).
// Validation happens here, synchronously, before anything is enqueued.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <new>
#include <numeric>
#include <vector>

#include "bp_batch.cuh"
#include "fbp_internal.cuh"

namespace fbp {
void clear_error();
void release_tables();
}  // namespace fbp

using namespace fbp;

namespace {

size_t dtype_size(fbp_dtype d) { return d == FBP_F32 ? 4 : 2; }
bool dtype_ok(int d) { return d == FBP_F32 || d == FBP_F16 || d == FBP_BF16; }
bool kind_ok(int k) { return k == FBP_FILTER_RAMLAK || k == FBP_FILTER_SHEPP_LOGAN; }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
    return pa < pb + nb && pb < pa + na;
}

template <typename F>
fbp_status guarded(F &&f)
{
    clear_error();
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return fail(FBP_ERR_CUDA, "host allocation failed");
    } catch (...) {
        return fail(FBP_ERR_CUDA, "unexpected host exception");
    }
}

}  // namespace

extern "C" {

int fbp_version(void) { return 100; }

fbp_geometry fbp_geometry_default(int n_angles, int n_det, int n)
{
    fbp_geometry g;
    g.n_angles = n_angles;
    g.n_det = n_det;
    g.n = n;
    g.angle_start = 0.0;
    g.angle_step = n_angles > 0 ? 3.14159265358979323846 / (double)n_angles : 0.0;
    g.det_center = 0.5 * (double)(n_det - 1);
    g.det_spacing = 1.0;
    g.pixel_size = 1.0;
    return g;
}

const char *fbp_status_string(fbp_status s)
{
    switch (s) {
        case FBP_OK: return "FBP_OK";
        case FBP_ERR_INVALID_ARG: return "FBP_ERR_INVALID_ARG";
        case FBP_ERR_UNSUPPORTED: return "FBP_ERR_UNSUPPORTED";
        case FBP_ERR_WORKSPACE: return "FBP_ERR_WORKSPACE";
        case FBP_ERR_CUDA: return "FBP_ERR_CUDA";
        case FBP_ERR_DEVICE_STATUS: return "FBP_ERR_DEVICE_STATUS";
    }
    return "FBP_UNKNOWN_STATUS";
}

const char *fbp_last_error_message(void);

static fbp_status filter_impl(const float *sino, void *filt, float *row_scale, fbp_dtype dtype,
                              fbp_filter_kind kind, const fbp_geometry *g, int n_slices,
                              const FilterPre *pre, fbp_stream_t stream)
{
    fbp_status st = check_geometry(g, true, false);
    if (st != FBP_OK) return st;
    if (!dtype_ok(dtype)) return fail(FBP_ERR_INVALID_ARG, "dtype %d", (int)dtype);
    if (!kind_ok(kind)) return fail(FBP_ERR_INVALID_ARG, "filter kind %d", (int)kind);
    if (n_slices < 0) return fail(FBP_ERR_INVALID_ARG, "n_slices < 0");
    if (n_slices == 0) return FBP_OK;
    if (!sino || !filt) return fail(FBP_ERR_INVALID_ARG, "sino or filt is NULL");
    if (dtype != FBP_F32 && !row_scale)
        return fail(FBP_ERR_INVALID_ARG, "row_scale is required for 16-bit output");
    const long long rows = (long long)n_slices * g->n_angles;
    const size_t nin = (size_t)rows * g->n_det * 4, nout = (size_t)rows * g->n_det * dtype_size(dtype);
    if (overlap(sino, nin, filt, nout)) return fail(FBP_ERR_INVALID_ARG, "filt overlaps sino");
    const float2 *G = nullptr;
    const float2 *tw = nullptr;
    int L = 0;
    st = filter_tables(g->n_det, kind, g->det_spacing, stream, &G, &tw, &L);
    if (st != FBP_OK) return st;
    FilterLaunch a;
    a.sino = sino;
    a.filt = filt;
    a.row_scale = dtype == FBP_F32 ? nullptr : row_scale;
    a.rows = rows;
    a.D = g->n_det;
    a.L = L;
    a.G = G;
    a.tw = tw;
    a.dtype = dtype;
    a.pre = pre;
    return launch_filter(a, stream);
}

fbp_status fbp_filter(const float *sino, void *filt, float *row_scale, fbp_dtype dtype,
                      fbp_filter_kind kind, const fbp_geometry *g, int n_slices,
                      fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        return filter_impl(sino, filt, row_scale, dtype, kind, g, n_slices, nullptr, stream);
    });
}

fbp_status fbp_filter_counts(const float *counts, void *filt, float *row_scale, fbp_dtype dtype,
                             fbp_filter_kind kind, const fbp_geometry *g, int n_slices,
                             const fbp_preprocess *pre, fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        if (!pre) return fail(FBP_ERR_INVALID_ARG, "pre is NULL");
        if (!pre->flat && !(pre->flat_value > 0.f && std::isfinite(pre->flat_value)))
            return fail(FBP_ERR_INVALID_ARG, "flat_value must be positive when flat is NULL");
        if (!(pre->count_floor > 0.f && std::isfinite(pre->count_floor)))
            return fail(FBP_ERR_INVALID_ARG, "count_floor must be positive");
        if (!(pre->mu_scale > 0.f && std::isfinite(pre->mu_scale)))
            return fail(FBP_ERR_INVALID_ARG, "mu_scale must be positive");
        if (!(pre->blur_sigma >= 0.f && pre->blur_sigma <= 3.875f))
            return fail(FBP_ERR_INVALID_ARG, "blur_sigma must lie in [0, 3.875]");
        FilterPre fp;
        fp.flat = pre->flat;
        fp.flat_value = pre->flat_value;
        fp.floor = pre->count_floor;
        fp.mu_scale = pre->mu_scale;
        // taps exp(-k^2 / (2 sigma^2)), |k| <= floor(4 sigma + 1/2), normalised in double
        const double sg = pre->blur_sigma;
        fp.blur_radius = sg > 0.0 ? (int)(4.0 * sg + 0.5) : 0;
        double w[33], sum = 0.0;
        for (int k = -fp.blur_radius; k <= fp.blur_radius; ++k) {
            w[k + fp.blur_radius] = sg > 0.0 ? std::exp(-(double)k * k / (2.0 * sg * sg)) : 1.0;
            sum += w[k + fp.blur_radius];
        }
        for (int i = 0; i <= 2 * fp.blur_radius; ++i) fp.taps[i] = (float)(w[i] / sum);
        if (g && pre->flat && overlap(pre->flat, (size_t)g->n_det * 4, filt,
                                      (size_t)n_slices * g->n_angles * g->n_det * dtype_size(dtype)))
            return fail(FBP_ERR_INVALID_ARG, "flat overlaps filt");
        return filter_impl(counts, filt, row_scale, dtype, kind, g, n_slices, &fp, stream);
    });
}

// Virtual detector of an offset scan (fbp.h, fbp_offset_geometry).
static fbp_status offset_virtual(const fbp_geometry *g, const fbp_offset_scan *o, fbp_geometry *gv,
                                 FilterOffset *fo)
{
    if (!g || !o || !gv) return fail(FBP_ERR_INVALID_ARG, "g, o or gv is NULL");
    fbp_status st = check_geometry(g, false, false);
    if (st != FBP_OK) return st;
    const double pi = 3.14159265358979323846;
    const int D = g->n_det, K = g->n_angles;
    const double c = g->det_center;
    if (!(c >= 0.0 && c <= D - 1.0) || std::fabs(2.0 * c - std::rint(2.0 * c)) > 1e-9)
        return fail(FBP_ERR_INVALID_ARG, "offset scan needs det_center in [0, D-1], a multiple of 1/2");
    if (std::fabs((double)K * g->angle_step - 2.0 * pi) > 1e-9 * 2.0 * pi)
        return fail(FBP_ERR_INVALID_ARG, "offset scan needs a full turn: n_angles * angle_step = 2 pi");
    if (o->fold != 0 && o->fold != 1) return fail(FBP_ERR_INVALID_ARG, "fold must be 0 or 1");
    if (o->fold && K % 2) return fail(FBP_ERR_INVALID_ARG, "fold needs an even number of angles");
    const bool long_pos = (D - 1 - c) >= c;
    const double long_side = long_pos ? D - 1 - c : c, short_side = long_pos ? c : D - 1 - c;
    if (!(o->overlap > 0.0 && o->overlap <= short_side + 1e-12))
        return fail(FBP_ERR_INVALID_ARG, "overlap %g outside (0, %g]", o->overlap, short_side);
    const long long nv = (long long)std::llround(2.0 * long_side) + 1;
    if (nv > 8192) return fail(FBP_ERR_UNSUPPORTED, "virtual detector of %lld bins > 8192", nv);
    const double cv = 0.5 * (double)(nv - 1);
    const int off = long_pos ? (int)std::llround(cv - c) : 0;
    *gv = *g;
    gv->n_angles = o->fold ? K / 2 : K;
    gv->n_det = (int)nv;
    gv->det_center = cv;
    if (fo) {
        fo->Dp = D;
        fo->off = off;
        fo->fold = o->fold;
        fo->K_in = K;
        fo->cv = (float)cv;
        fo->sgn = long_pos ? 1.f : -1.f;
        fo->inv_delta = (float)(1.0 / o->overlap);
    }
    return FBP_OK;
}

fbp_status fbp_offset_geometry(const fbp_geometry *g, const fbp_offset_scan *o, fbp_geometry *gv,
                               int *offset)
{
    return guarded([&]() -> fbp_status {
        FilterOffset fo;
        fbp_status st = offset_virtual(g, o, gv, &fo);
        if (st == FBP_OK && offset) *offset = fo.off;
        return st;
    });
}

fbp_status fbp_filter_offset(const float *sino, void *filt, float *row_scale, fbp_dtype dtype,
                             fbp_filter_kind kind, const fbp_geometry *g, int n_slices,
                             const fbp_offset_scan *o, fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        fbp_geometry gv;
        FilterOffset fo;
        fbp_status st = offset_virtual(g, o, &gv, &fo);
        if (st != FBP_OK) return st;
        st = check_geometry(&gv, true, false);
        if (st != FBP_OK) return st;
        if (!dtype_ok(dtype)) return fail(FBP_ERR_INVALID_ARG, "dtype %d", (int)dtype);
        if (!kind_ok(kind)) return fail(FBP_ERR_INVALID_ARG, "filter kind %d", (int)kind);
        if (n_slices < 0) return fail(FBP_ERR_INVALID_ARG, "n_slices < 0");
        if (n_slices == 0) return FBP_OK;
        if (!sino || !filt) return fail(FBP_ERR_INVALID_ARG, "sino or filt is NULL");
        if (dtype != FBP_F32 && !row_scale)
            return fail(FBP_ERR_INVALID_ARG, "row_scale is required for 16-bit output");
        const long long rows = (long long)n_slices * gv.n_angles;
        const size_t nin = (size_t)n_slices * g->n_angles * g->n_det * 4;
        const size_t nout = (size_t)rows * gv.n_det * dtype_size(dtype);
        if (overlap(sino, nin, filt, nout)) return fail(FBP_ERR_INVALID_ARG, "filt overlaps sino");
        const float2 *G = nullptr;
        const float2 *tw = nullptr;
        int L = 0;
        st = filter_tables(gv.n_det, kind, gv.det_spacing, stream, &G, &tw, &L);
        if (st != FBP_OK) return st;
        FilterLaunch a;
        a.sino = sino;
        a.filt = filt;
        a.row_scale = dtype == FBP_F32 ? nullptr : row_scale;
        a.rows = rows;
        a.D = gv.n_det;
        a.L = L;
        a.G = G;
        a.tw = tw;
        a.dtype = dtype;
        a.offset = &fo;
        return launch_filter(a, stream);
    });
}

static fbp_status backproject_impl(const void *filt, const float *row_scale, fbp_dtype dtype,
                                   float *slice, unsigned short *slice16, float hu_a, float hu_b,
                                   const fbp_geometry *g, int n_slices, float scale,
                                   int accumulate, int variant, fbp_stream_t stream)
{
    fbp_status st = check_geometry(g, false, true);
    if (st != FBP_OK) return st;
    if (!dtype_ok(dtype)) return fail(FBP_ERR_INVALID_ARG, "dtype %d", (int)dtype);
    if (n_slices < 0) return fail(FBP_ERR_INVALID_ARG, "n_slices < 0");
    if (variant < -1 || variant >= bp_variant_count())
        return fail(FBP_ERR_INVALID_ARG, "variant %d", variant);
    if (!std::isfinite(scale)) return fail(FBP_ERR_INVALID_ARG, "scale is not finite");
    if (n_slices == 0) return FBP_OK;
    if (!filt || !(slice || slice16)) return fail(FBP_ERR_INVALID_ARG, "filt or slice is NULL");
    if (dtype != FBP_F32 && !row_scale)
        return fail(FBP_ERR_INVALID_ARG, "row_scale is required for 16-bit input");
    const size_t nin = (size_t)n_slices * g->n_angles * g->n_det * dtype_size(dtype);
    const size_t nout = (size_t)n_slices * g->n * g->n * (slice16 ? 2 : 4);
    if (overlap(filt, nin, slice16 ? (const void *)slice16 : (const void *)slice, nout))
        return fail(FBP_ERR_INVALID_ARG, "slice overlaps filt");
    const double2 *cs = nullptr;
    st = angle_table(*g, stream, &cs);
    if (st != FBP_OK) return st;
    BpLaunch a;
    a.filt = filt;
    a.row_scale = dtype == FBP_F32 ? nullptr : row_scale;
    a.slice = slice;
    a.cs = cs;
    a.K = g->n_angles;
    a.D = g->n_det;
    a.N = g->n;
    a.S = n_slices;
    a.alpha = g->pixel_size / g->det_spacing;
    a.det_center = g->det_center;
    a.angle_step = g->angle_step;
    a.scale = scale;
    a.accumulate = accumulate ? 1 : 0;
    a.dtype = dtype;
    a.slice16 = slice16;
    a.hu_a = hu_a;
    a.hu_b = hu_b;
    return launch_backproject(a, variant, stream);
}

fbp_status fbp_backproject_variant(const void *filt, const float *row_scale, fbp_dtype dtype,
                                   float *slice, const fbp_geometry *g, int n_slices, float scale,
                                   int accumulate, int variant, fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        return backproject_impl(filt, row_scale, dtype, slice, nullptr, 0.f, 0.f, g, n_slices, scale,
                                accumulate, variant, stream);
    });
}

static fbp_status hu_coeffs(const fbp_hu_window *w, float *a, float *b)
{
    if (!w) return fail(FBP_ERR_INVALID_ARG, "window is NULL");
    const double dw = w->mu_water - w->mu_air, dh = w->hu_max - w->hu_min;
    if (!std::isfinite(w->mu_water) || !std::isfinite(w->mu_air) || !std::isfinite(w->hu_min) ||
        !std::isfinite(w->hu_max) || !(dw != 0.0) || !(dh > 0.0))
        return fail(FBP_ERR_INVALID_ARG, "HU window needs finite values, mu_water != mu_air, hu_max > hu_min");
    // code = (HU - hu_min) / (hu_max - hu_min) * 65535, HU = 1000 (mu - mu_water) / (mu_water - mu_air)
    const double s = 65535.0 / dh;
    *a = (float)(1000.0 / dw * s);
    *b = (float)(-(1000.0 * w->mu_water / dw + w->hu_min) * s);
    return FBP_OK;
}

fbp_status fbp_hu_coefficients(const fbp_hu_window *w, float *a, float *b)
{
    return guarded([&]() -> fbp_status {
        if (!a || !b) return fail(FBP_ERR_INVALID_ARG, "a or b is NULL");
        return hu_coeffs(w, a, b);
    });
}

fbp_status fbp_backproject_u16(const void *filt, const float *row_scale, fbp_dtype dtype,
                               unsigned short *slice, const fbp_geometry *g, int n_slices,
                               float scale, const fbp_hu_window *w, int variant,
                               fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        float a = 0.f, b = 0.f;
        fbp_status st = hu_coeffs(w, &a, &b);
        if (st != FBP_OK) return st;
        if (n_slices > 0 && !slice) return fail(FBP_ERR_INVALID_ARG, "slice is NULL");
        return backproject_impl(filt, row_scale, dtype, nullptr, slice, a, b, g, n_slices, scale, 0,
                                variant, stream);
    });
}

fbp_status fbp_backproject(const void *filt, const float *row_scale, fbp_dtype dtype, float *slice,
                           const fbp_geometry *g, int n_slices, float scale, int accumulate,
                           fbp_stream_t stream)
{
    return fbp_backproject_variant(filt, row_scale, dtype, slice, g, n_slices, scale, accumulate,
                                   -1, stream);
}

fbp_status radon_forward(const float *slice, float *sino, const fbp_geometry *g, int n_slices,
                         fbp_stream_t stream)
{
    return radon_forward_variant(slice, sino, g, n_slices, -1, stream);
}

fbp_status radon_forward_variant(const float *slice, float *sino, const fbp_geometry *g,
                                 int n_slices, int variant, fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        fbp_status st = check_geometry(g, false, true);
        if (st != FBP_OK) return st;
        if (n_slices < 0) return fail(FBP_ERR_INVALID_ARG, "n_slices < 0");
        if (variant < -1 || variant >= fwd_variant_count())
            return fail(FBP_ERR_INVALID_ARG, "forward variant %d out of range", variant);
        const double alpha = g->pixel_size / g->det_spacing;
        if (variant > 0 && !fwd_tile_eligible(alpha))
            return fail(FBP_ERR_UNSUPPORTED,
                        "tile forward projector needs pixel_size / det_spacing in [0.9429, 1]");
        if (n_slices == 0) return FBP_OK;
        if (!slice || !sino) return fail(FBP_ERR_INVALID_ARG, "slice or sino is NULL");
        const size_t nin = (size_t)n_slices * g->n * g->n * 4;
        const size_t nout = (size_t)n_slices * g->n_angles * g->n_det * 4;
        if (overlap(slice, nin, sino, nout)) return fail(FBP_ERR_INVALID_ARG, "sino overlaps slice");
        const double2 *cs = nullptr;
        st = angle_table(*g, stream, &cs);
        if (st != FBP_OK) return st;
        FwdLaunch a;
        a.slice = slice;
        a.sino = sino;
        a.cs = cs;
        a.K = g->n_angles;
        a.D = g->n_det;
        a.N = g->n;
        a.S = n_slices;
        a.alpha = alpha;
        a.det_center = g->det_center;
        a.variant = variant;
        return launch_forward(a, stream);
    });
}

int radon_forward_variant_count(void) { return fwd_variant_count(); }

int fbp_bp_variant_count(void) { return bp_variant_count(); }

int fbp_bp_variant_supports(int variant, fbp_dtype dtype, const fbp_geometry *g)
{
    clear_error();
    fbp_bp_shape sh;
    if (!bp_variant_shape(variant, &sh) || check_geometry(g, false, true) != FBP_OK) return 0;
    if (!dtype_ok(dtype)) return 0;
    BpLaunch a{};
    a.K = g->n_angles;
    a.D = g->n_det;
    a.N = g->n;
    a.alpha = g->pixel_size / g->det_spacing;
    a.det_center = g->det_center;
    a.angle_step = g->angle_step;
    a.dtype = dtype;
    return bp_variant_fits(variant, a) ? 1 : 0;
}

fbp_status fbp_bp_variant_info(int variant, fbp_bp_shape *out)
{
    return guarded([&]() -> fbp_status {
        if (!out) return fail(FBP_ERR_INVALID_ARG, "out is NULL");
        if (!bp_variant_shape(variant, out)) return fail(FBP_ERR_INVALID_ARG, "variant %d", variant);
        return FBP_OK;
    });
}

// ---------------------------------------------------------------------------
// Ragged batches (normal and offset scans)
// ---------------------------------------------------------------------------
struct ScanPlan {
    const float *sino;
    float *slice;
    fbp_geometry g;        // the scan's geometry
    fbp_geometry gb;       // geometry of the filtered rows (virtual detector for offset scans)
    bool offset;
    FilterOffset fo;
};

static fbp_status plan_items(const fbp_scan_item *items, int count, std::vector<ScanPlan> *plan)
{
    if (!items) return fail(FBP_ERR_INVALID_ARG, "items is NULL");
    if (count < 1 || count > kMaxBatch)
        return fail(FBP_ERR_INVALID_ARG, "count %d outside [1, %d]", count, kMaxBatch);
    plan->resize(count);
    for (int i = 0; i < count; ++i) {
        ScanPlan &p = (*plan)[i];
        p.sino = items[i].sino;
        p.slice = items[i].slice;
        p.g = items[i].g;
        p.offset = items[i].overlap != 0.0;
        p.fo = FilterOffset{};
        fbp_status st = FBP_OK;
        if (p.offset) {
            fbp_offset_scan o;
            o.overlap = items[i].overlap;
            o.fold = items[i].fold;
            st = offset_virtual(&items[i].g, &o, &p.gb, &p.fo);
            if (st == FBP_OK) st = check_geometry(&p.gb, true, true);
        } else {
            p.gb = items[i].g;
            st = check_geometry(&items[i].g, true, true);
        }
        if (st != FBP_OK) {
            const std::string why = fbp_last_error_message();
            return fail(st, "item %d: %s", i, why.c_str());
        }
        if (!p.sino || !p.slice) return fail(FBP_ERR_INVALID_ARG, "item %d: sino or slice is NULL", i);
    }
    return FBP_OK;
}

// Padded table of an item that runs staged batch units (bp_staged_batch.cu):
// the 90-degree orbit symmetry with the dtype's tile and a window that fits.
static bool staged_item(const ScanPlan &p, fbp_dtype dtype, StagedItemGeom *out)
{
    const fbp_geometry &g = p.gb;
    return staged_batch_geometry(g.n_angles, g.angle_step, g.n_det, g.det_center, g.n,
                                 g.pixel_size / g.det_spacing, dtype, out);
}

// Workspace: [256 B: two work-queue counters] then, per item, its filtered
// rows, (16-bit dtypes) its row scales and (items that can run staged batch
// units) its padded table, each 256-byte aligned; then (16-bit dtypes) one
// float S per item.
struct BatchLayout {
    std::vector<size_t> filt, scale, table;   // table 0: the item has none
    size_t smax = 0, total = 0;
};

static BatchLayout workspace_layout(const std::vector<ScanPlan> &plan, fbp_dtype dtype)
{
    BatchLayout L;
    size_t off = 256;
    for (const ScanPlan &p : plan) {
        const size_t rows = (size_t)p.gb.n_angles;
        L.filt.push_back(off);
        off += align256(rows * p.gb.n_det * dtype_size(dtype));
        L.scale.push_back(dtype == FBP_F32 ? 0 : off);
        if (dtype != FBP_F32) off += align256(rows * 4);
        StagedItemGeom sg;
        if (staged_item(p, dtype, &sg)) {
            L.table.push_back(off);
            off += align256(sg.table_bytes);
        } else {
            L.table.push_back(0);
        }
    }
    if (dtype != FBP_F32) {
        L.smax = off;
        off += align256(plan.size() * 4);
    }
    L.total = off;
    return L;
}

static fbp_status batched_impl(const std::vector<ScanPlan> &plan, fbp_filter_kind kind,
                               fbp_dtype dtype, int bp_variant, int order, void *workspace,
                               size_t ws_bytes, fbp_stream_t stream)
{
    const int count = (int)plan.size();
    if (!dtype_ok(dtype)) return fail(FBP_ERR_INVALID_ARG, "dtype %d", (int)dtype);
    if (!kind_ok(kind)) return fail(FBP_ERR_INVALID_ARG, "filter kind %d", (int)kind);
    if (bp_variant < -1 || bp_variant >= bp_variant_count())
        return fail(FBP_ERR_INVALID_ARG, "variant %d", bp_variant);
    if (order != FBP_ORDER_QUEUE && order != FBP_ORDER_GROUP_CYCLIC)
        return fail(FBP_ERR_INVALID_ARG, "order %d", order);
    // the persistent tile kernel's shape (items that do not run staged batch
    // units by default, every item when a variant is given): the 64 x 64
    // orbit (FP32 rows: variant 8, 16-bit rows: the packed variant 10),
    // generic tiles for items without the symmetry.  For batches of many
    // smaller slices the 64 x 64 orbit beats the 32 x 32 one that single
    // N = 8192 slices prefer (ragged workload: 512 vs 569 ms).
    const int variant = bp_variant >= 0 ? bp_variant : (dtype == FBP_F32 ? 8 : 10);
    BpPersistentShape shape;
    if (!bp_persistent_shape(variant, dtype, &shape))
        return fail(FBP_ERR_UNSUPPORTED, "variant %d is not available for ragged batches of this dtype", variant);
    const BatchLayout lay = workspace_layout(plan, dtype);
    const std::vector<size_t> &foff = lay.filt, &soff = lay.scale;
    const size_t need = lay.total;
    if (!workspace) return fail(FBP_ERR_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) & 255)
        return fail(FBP_ERR_WORKSPACE, "workspace is not 256-byte aligned");
    if (ws_bytes < need)
        return fail(FBP_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", ws_bytes, need);
    char *ws = static_cast<char *>(workspace);
    unsigned *status = nullptr;
    fbp_status st = device_status_word(&status);
    if (st != FBP_OK) return st;

    // tables (all before any launch, so a failure enqueues nothing)
    std::vector<const double2 *> cs(count);
    std::vector<const float2 *> Gs(count);
    std::vector<const float2 *> tws(count);
    std::vector<int> Ls(count);
    for (int i = 0; i < count; ++i) {
        st = angle_table(plan[i].gb, stream, &cs[i]);
        if (st != FBP_OK) return st;
        st = filter_tables(plan[i].gb.n_det, kind, plan[i].gb.det_spacing, stream, &Gs[i], &tws[i], &Ls[i]);
        if (st != FBP_OK) return st;
    }

    // filter descriptors, in item order
    auto *fa = new FilterBatchArgs();
    std::unique_ptr<FilterBatchArgs> fa_owner(fa);
    int groups = 0;
    for (int i = 0; i < count; ++i) {
        const ScanPlan &p = plan[i];
        FilterBatchItem &f = fa->items[i];
        f.sino = p.sino;
        f.filt = ws + foff[i];
        f.row_scale = dtype == FBP_F32 ? nullptr : reinterpret_cast<float *>(ws + soff[i]);
        f.G = Gs[i];
        f.tw = tws[i];
        f.K = p.gb.n_angles;
        f.D = p.gb.n_det;
        f.L = Ls[i];
        f.group_begin = groups;
        f.Dp = p.offset ? p.fo.Dp : 0;
        f.off = p.offset ? p.fo.off : 0;
        f.fold = p.offset ? p.fo.fold : 0;
        f.K_in = p.offset ? (int)p.fo.K_in : f.K;
        f.cv = p.fo.cv;
        f.sgn = p.fo.sgn;
        f.inv_delta = p.fo.inv_delta;
        f.pad_ = 0;
        const int G = filter_pairs_per_block(Ls[i]);
        const long long pairs = ((long long)f.K + 1) / 2;
        const long long gi = (pairs + G - 1) / G;
        if ((long long)groups + gi > 0x7fffffffLL) return fail(FBP_ERR_UNSUPPORTED, "batch too large");
        groups += (int)gi;
    }
    fa->count = count;

    // backprojection.  By default (bp_variant -1) the items with a padded
    // table run staged batch units (bp_staged_batch.cu: 90-degree orbits of
    // 32 x 32 (FP32) or 64 x 64 (16-bit) tiles, windows moved by bulk
    // copies); the others -- and every
    // item when a variant is given -- run the persistent tile kernel, where
    // an item whose geometry has the 90-degree symmetry runs orbit units
    // (four tiles each) and any other generic tiles.  Queue: items by total
    // cost K n^2, largest first.  Group-cyclic: by cost per unit, largest
    // first, so every run of P consecutive units holds units of similar cost.
    std::vector<char> staged(count, 0);
    std::vector<StagedItemGeom> sg(count);
    if (bp_variant < 0)
        for (int i = 0; i < count; ++i) staged[i] = lay.table[i] != 0 && staged_item(plan[i], dtype, &sg[i]);
    std::vector<int> orbit(count), tiles_x(count), H(count);
    std::vector<long long> n_units(count), unit_cost(count);
    for (int i = 0; i < count; ++i) {
        const fbp_geometry &g = plan[i].gb;
        const double alpha = g.pixel_size / g.det_spacing;
        if (staged[i]) {
            const int T = staged_batch_tile(dtype);
            orbit[i] = 1;
            tiles_x[i] = g.n / T / 2;
            H[i] = sg[i].H;
            n_units[i] = (long long)tiles_x[i] * tiles_x[i];
            unit_cost[i] = 4LL * T * T * g.n_angles;
            continue;
        }
        orbit[i] = shape.orbit_tile > 0 &&
                   bp_orbit_geometry(g.n_angles, g.angle_step, g.n_det, g.det_center, g.n, shape.orbit_tile);
        if (orbit[i]) {
            const int T = shape.orbit_tile;
            tiles_x[i] = g.n / T / 2;
            H[i] = bp_window_half(alpha, T, T);
            n_units[i] = (long long)tiles_x[i] * tiles_x[i];
            unit_cost[i] = 4LL * T * T * g.n_angles;
        } else {
            const int TW = shape.tile_w, TH = shape.tile_h;
            tiles_x[i] = (g.n + TW - 1) / TW;
            H[i] = bp_window_half(alpha, TW, TH);
            n_units[i] = (long long)tiles_x[i] * ((g.n + TH - 1) / TH);
            unit_cost[i] = (long long)TW * TH * g.n_angles;
        }
    }
    std::vector<int> idx(count);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        const fbp_geometry &a = plan[x].gb, &b = plan[y].gb;
        if (order == FBP_ORDER_GROUP_CYCLIC) return unit_cost[x] > unit_cost[y];
        return (long long)a.n_angles * a.n * a.n > (long long)b.n_angles * b.n * b.n;
    });
    auto *ba = new BpBatchArgs();
    std::unique_ptr<BpBatchArgs> ba_owner(ba);
    auto *sa = new StagedBatchArgs();
    std::unique_ptr<StagedBatchArgs> sa_owner(sa);
    auto *sp = new StagedPrepArgs();
    std::unique_ptr<StagedPrepArgs> sp_owner(sp);
    long long units = 0, s_units = 0, s_pairs = 0;
    int nb = 0, ns = 0, max_H = 0, max_H_orbit = 0, Wp = 8;
    for (int r = 0; r < count; ++r) {
        const int i = idx[r];
        const fbp_geometry &g = plan[i].gb;
        if (staged[i]) {
            StagedBatchItem &b = sa->items[ns];
            StagedPrepItem &q = sp->items[ns];
            ++ns;
            float *smax = dtype == FBP_F32 ? nullptr : reinterpret_cast<float *>(ws + lay.smax) + i;
            q.filt = ws + foff[i];
            q.row_scale = dtype == FBP_F32 ? nullptr : reinterpret_cast<const float *>(ws + soff[i]);
            q.table = ws + lay.table[i];
            q.smax = smax;
            q.K = g.n_angles;
            q.D = g.n_det;
            q.Ep = sg[i].Ep;
            q.P_lo = sg[i].P_lo;
            q.pair_begin = (int)s_pairs;
            q.pad_ = 0;
            b.table = q.table;
            b.slice = plan[i].slice;
            b.cs = cs[i];
            b.smax = smax;
            b.alpha = g.pixel_size / g.det_spacing;
            b.det_center = g.det_center;
            b.K2 = g.n_angles / 2;
            b.N = g.n;
            b.H = sg[i].H;
            b.W = sg[i].W;
            b.Ep = sg[i].Ep;
            b.P_lo = sg[i].P_lo;
            b.tiles_x = tiles_x[i];
            b.unit_begin = (int)s_units;
            b.scale = (float)g.angle_step;
            b.pad_ = 0;
            Wp = std::max(Wp, sg[i].Wp);
            s_units += n_units[i];
            s_pairs += g.n_angles / 2;
            if (s_units > 0x7fffffffLL || s_pairs > 0x7fffffffLL)
                return fail(FBP_ERR_UNSUPPORTED, "batch too large");
            continue;
        }
        BpBatchItem &b = ba->items[nb++];
        b.filt = ws + foff[i];
        b.row_scale = dtype == FBP_F32 ? nullptr : reinterpret_cast<const float *>(ws + soff[i]);
        b.slice = plan[i].slice;
        b.cs = cs[i];
        b.alpha = g.pixel_size / g.det_spacing;
        b.det_center = g.det_center;
        b.K = g.n_angles;
        b.D = g.n_det;
        b.N = g.n;
        b.scale = (float)g.angle_step;
        b.tiles_x = tiles_x[i];
        b.H = H[i];
        b.unit_begin = (int)units;
        b.orbit = orbit[i];
        if (orbit[i])
            max_H_orbit = std::max(max_H_orbit, H[i]);
        else
            max_H = std::max(max_H, H[i]);
        units += n_units[i];
        if (units > 0x7fffffffLL) return fail(FBP_ERR_UNSUPPORTED, "batch too large");
    }
    const int cyclic = order == FBP_ORDER_GROUP_CYCLIC ? 1 : 0;
    ba->count = nb;
    ba->total_units = (int)units;
    ba->max_H = max_H;
    ba->max_H_orbit = max_H_orbit;
    ba->cyclic = cyclic;
    ba->counter = reinterpret_cast<int *>(ws);
    ba->status = status;
    sa->count = ns;
    sa->total_units = (int)s_units;
    sa->Wp = Wp;
    sa->cyclic = cyclic;
    sa->counter = reinterpret_cast<int *>(ws) + 1;
    sa->status = status;
    sp->count = ns;
    sp->total_pairs = (int)s_pairs;

    if (!cyclic) FBP_CUDA_TRY(cudaMemsetAsync(ws, 0, 2 * sizeof(int), stream));
    st = launch_filter_batched(*fa, groups, dtype, stream);
    if (st != FBP_OK) return st;
    if (ns > 0) {
        st = launch_staged_batch(*sp, *sa, dtype, stream);
        if (st != FBP_OK) return st;
    }
    if (nb > 0) return launch_bp_persistent(*ba, variant, dtype, stream);
    return FBP_OK;
}

static fbp_status plan_plain(const fbp_batch_item *items, int count, std::vector<ScanPlan> *plan)
{
    if (!items) return fail(FBP_ERR_INVALID_ARG, "items is NULL");
    if (count < 1 || count > kMaxBatch)
        return fail(FBP_ERR_INVALID_ARG, "count %d outside [1, %d]", count, kMaxBatch);
    std::vector<fbp_scan_item> scans(count);
    for (int i = 0; i < count; ++i) {
        scans[i].sino = items[i].sino;
        scans[i].slice = items[i].slice;
        scans[i].g = items[i].g;
        scans[i].overlap = 0.0;
        scans[i].fold = 0;
    }
    return plan_items(scans.data(), count, plan);
}

size_t fbp_batched_workspace_bytes(const fbp_batch_item *items, int count, fbp_dtype dtype)
{
    clear_error();
    std::vector<ScanPlan> plan;
    if (!dtype_ok(dtype) || plan_plain(items, count, &plan) != FBP_OK) return 0;
    return workspace_layout(plan, dtype).total;
}

int fbp_batched_item_staged(const fbp_geometry *g, fbp_dtype dtype)
{
    clear_error();
    if (!g || !dtype_ok(dtype) || check_geometry(g, false, true) != FBP_OK) return 0;
    return staged_batch_geometry(g->n_angles, g->angle_step, g->n_det, g->det_center, g->n,
                                 g->pixel_size / g->det_spacing, dtype, nullptr) ? 1 : 0;
}

fbp_status fbp_batched(const fbp_batch_item *items, int count, fbp_filter_kind kind,
                       fbp_dtype dtype, int bp_variant, void *workspace, size_t ws_bytes,
                       fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        std::vector<ScanPlan> plan;
        fbp_status st = plan_plain(items, count, &plan);
        if (st != FBP_OK) return st;
        return batched_impl(plan, kind, dtype, bp_variant, FBP_ORDER_QUEUE, workspace, ws_bytes, stream);
    });
}

size_t fbp_batched_scans_workspace_bytes(const fbp_scan_item *items, int count, fbp_dtype dtype)
{
    clear_error();
    std::vector<ScanPlan> plan;
    if (!dtype_ok(dtype) || plan_items(items, count, &plan) != FBP_OK) return 0;
    return workspace_layout(plan, dtype).total;
}

fbp_status fbp_batched_scans(const fbp_scan_item *items, int count, fbp_filter_kind kind,
                             fbp_dtype dtype, int bp_variant, fbp_batch_order order,
                             void *workspace, size_t ws_bytes, fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        std::vector<ScanPlan> plan;
        fbp_status st = plan_items(items, count, &plan);
        if (st != FBP_OK) return st;
        return batched_impl(plan, kind, dtype, bp_variant, (int)order, workspace, ws_bytes, stream);
    });
}

fbp_status fbp_last_device_status(fbp_stream_t stream, int *code)
{
    return guarded([&]() -> fbp_status {
        unsigned *p = nullptr;
        fbp_status st = device_status_word(&p);
        if (st != FBP_OK) return st;
        FBP_CUDA_TRY(cudaStreamSynchronize(stream));
        unsigned v = 0;
        FBP_CUDA_TRY(cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost));
        if (v) {
            const unsigned zero = 0;
            FBP_CUDA_TRY(cudaMemcpy(p, &zero, sizeof(zero), cudaMemcpyHostToDevice));
        }
        if (code) *code = (int)v;
        if (v) return fail(FBP_ERR_DEVICE_STATUS, "device status word = %u", v);
        return FBP_OK;
    });
}

fbp_status fbp_prepare(const fbp_geometry *g, int kind, fbp_stream_t stream)
{
    return guarded([&]() -> fbp_status {
        fbp_status st = check_geometry(g, kind >= 0, false);
        if (st != FBP_OK) return st;
        const double2 *cs = nullptr;
        st = angle_table(*g, stream, &cs);
        if (st != FBP_OK) return st;
        if (kind >= 0) {
            if (!kind_ok(kind)) return fail(FBP_ERR_INVALID_ARG, "filter kind %d", kind);
            const float2 *G;
            const float2 *tw;
            int L;
            st = filter_tables(g->n_det, kind, g->det_spacing, stream, &G, &tw, &L);
            if (st != FBP_OK) return st;
        }
        unsigned *p = nullptr;
        return device_status_word(&p);
    });
}

void fbp_release_tables(void) { release_tables(); }

}  // extern "C"
