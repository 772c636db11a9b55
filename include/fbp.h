/*
 * fbp.h -- C ABI of libfbp.so: parallel-beam filtered backprojection (FBP)
 * on one NVIDIA GB300 GPU (sm_103a), with its matched forward projector.
 *
 * The operation.  FBP reconstructs each slice of a parallel-beam scan in two
 * steps (paper Sec. IV-B; Sec. V-A(c), stage 2 "FBP Computation"): every
 * projection row is filtered, then the filtered rows are backprojected onto
 * the image and summed over all angles, at cost O(N_p * N_x * N_y) per slice.
 * Each detector row maps to one independent slice (Sec. V-A(a), "Scan-rows
 * Partition"), so a call takes a stack of per-row sinograms
 * [n_angles, n_det] and returns one N x N slice per row.  The paper cites
 * Kak & Slaney ch. 3 for the filter; the discrete sums implemented here are:
 *
 *   filter      q_k[j] = tau * sum_{m=0}^{D-1} h[j-m] p_k[m]    (linear, zero-padded)
 *               h = band-limited Ram-Lak or Shepp-Logan kernel, tau = det_spacing
 *   backproject f[r][c] = scale * sum_k Q_k(u_k(r,c))           (scale = dtheta for FBP)
 *               u_k = (pixel_size/det_spacing) (X cos th_k + Y sin th_k) + det_center
 *               X = c - (N-1)/2, Y = r - (N-1)/2, th_k = angle_start + k*angle_step
 *               Q_k = linear interpolation of q_k, zero outside [0, D)
 *   forward     (A f)_k[j] = sum_{r,c} f[r][c] max(0, 1 - |u_k(r,c) - j|)
 *               (exactly the transpose of backproject with scale 1)
 *
 * Conventions for every call.
 *   * Pointers to arrays are DEVICE pointers owned by the caller, unless a
 *     parameter says "host".  The library never frees caller memory.
 *   * Arrays are dense and row-major: sino/filt [n_slices][n_angles][n_det],
 *     row_scale [n_slices][n_angles], slice [n_slices][n][n].
 *   * Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream).  Argument validation is synchronous: a call that
 *     returns an error other than FBP_ERR_CUDA has enqueued nothing.
 *   * No C++ exception crosses this boundary.  fbp_last_error_message()
 *     gives a human-readable reason for the calling thread's last error.
 *   * Constant tables (the FP64 angle table, the filter spectrum and the FFT
 *     twiddles) are built on the device in double precision the first time a
 *     geometry is seen on a device, and cached by the library until
 *     fbp_release_tables() or process exit.  That first call allocates device
 *     memory and must not happen inside CUDA stream capture (it returns
 *     FBP_ERR_UNSUPPORTED there); later calls with the same geometry allocate
 *     nothing and may be captured.
 *   * Limits: 1 <= n_det <= 8192 for filtering; n_angles >= 1; n >= 1;
 *     pixel_size/det_spacing in [1/8, 2.5] for backprojection and projection.
 */
#ifndef FBP_H
#define FBP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
/* Same type as cudaStream_t. */
typedef struct CUstream_st *fbp_stream_t;

typedef enum {
    FBP_OK = 0,
    FBP_ERR_INVALID_ARG = -1,   /* NULL pointer, bad size, bad enum, bad geometry */
    FBP_ERR_UNSUPPORTED = -2,   /* valid but outside the limits above, or table
                                   creation requested during stream capture */
    FBP_ERR_WORKSPACE = -3,     /* workspace NULL, too small or misaligned */
    FBP_ERR_CUDA = -4,          /* a CUDA runtime call or launch failed */
    FBP_ERR_DEVICE_STATUS = -5  /* a kernel reported a fault through the
                                   device status word (see below) */
} fbp_status;

typedef enum {
    FBP_FILTER_RAMLAK = 0,      /* h(0)=1/(4 tau^2), h(odd n)=-1/(pi^2 n^2 tau^2), 0 else */
    FBP_FILTER_SHEPP_LOGAN = 1  /* h(n) = -2 / (pi^2 tau^2 (4 n^2 - 1))                    */
} fbp_filter_kind;

typedef enum {
    FBP_F32 = 0,                /* filtered rows stored as float                      */
    FBP_F16 = 1,                /* as IEEE half, q / s_k rounded to nearest even       */
    FBP_BF16 = 2                /* as bfloat16, q / s_k rounded to nearest even        */
} fbp_dtype;

/* Geometry of one slice (paper Table I: N_p = n_angles, N_c = n_det,
 * N_x = N_y = n).  Angles and det_center are doubles: at n = 8192 the
 * detector coordinate needs more than float precision. */
typedef struct {
    int n_angles;        /* K >= 1                                          */
    int n_det;           /* D >= 1                                          */
    int n;               /* output slice is n x n, n >= 1                   */
    double angle_start;  /* theta_0, radians                                */
    double angle_step;   /* dtheta, radians (pi/K for a half turn)          */
    double det_center;   /* bin coordinate of the rotation axis ((D-1)/2)   */
    double det_spacing;  /* tau: bin width, > 0 (1)                          */
    double pixel_size;   /* pixel width, same unit as det_spacing, > 0 (1)  */
} fbp_geometry;

/* One slice of a ragged batch: its own sinogram [n_angles][n_det] (device,
 * float), its own output [n][n] (device, float) and its own geometry. */
typedef struct {
    const float *sino;
    float *slice;
    fbp_geometry g;
} fbp_batch_item;

/* Tile shape of one compiled backprojection variant. */
typedef struct {
    int angle_tile;      /* angles staged in shared memory per pass         */
    int tile_x, tile_y;  /* output pixels per thread block                  */
    int px, py;          /* output pixels per thread (x, y)                 */
    int threads;         /* threads per block                               */
    int symmetric;       /* 1: uses the 90-degree symmetry of the standard
                            geometry (angle step pi/K with K even, centred
                            detector, n a multiple of 2*tile_x); the block
                            owns a tile and its three rotations            */
    int packed16;        /* 1: 16-bit rows only; interpolates two rows with
                            one packed 16-bit FMA (the interpolated value is
                            rounded to the 16-bit type, then summed in FP32) */
    int texture;         /* 1: interpolates with the texture unit's linear
                            filtering instead of staged tables (FP32 rows, D a
                            multiple of 8, K <= 65000, `filt` aligned for a
                            texture: 512 bytes on current GPUs; slices are bound
                            in groups of up to 65000 rows); its fraction is
                            quantised to 8 bits,
                            and the call synchronises `stream` before it returns
                            (so it cannot be captured in a CUDA graph).  Never
                            the default; kept as the measured alternative   */
} fbp_bp_shape;

/* Library version (major*10000 + minor*100 + patch). */
int fbp_version(void);

/* Geometry with the defaults: angles k*pi/K on [0, pi), det_center (D-1)/2,
 * det_spacing 1, pixel_size 1. */
fbp_geometry fbp_geometry_default(int n_angles, int n_det, int n);

/* Short name of a status code (static string, never NULL). */
const char *fbp_status_string(fbp_status s);

/* Reason for the calling thread's most recent non-OK status ("" if none). */
const char *fbp_last_error_message(void);

/*
 * fbp_filter -- the filtering step (Sec. V-A(c) stage 2, "filtering").
 *   sino       device, float [n_slices][K][D]: line integrals p_k[m].
 *   filt       device, [n_slices][K][D] of `dtype`: receives q_k[j]
 *              (F32), or RNE(q_k[j] / s_k) (F16/BF16).  May not alias sino.
 *   row_scale  device, float [n_slices][K]: receives s_k = max_j |q_k[j]|
 *              (1 where the row is all zero).  Required for F16/BF16,
 *              ignored (may be NULL) for F32.
 *   kind       filter kernel; g->det_spacing is tau.
 *   n_slices   >= 0 slices sharing geometry g (0 enqueues nothing).
 * The convolution is computed in FP32 as a length-L FFT, L the smallest
 * power of two >= max(512, 2D-1), with the spectrum of the truncated FP64
 * kernel; it equals the linear convolution over the D detector samples.
 */
fbp_status fbp_filter(const float *sino, void *filt, float *row_scale,
                      fbp_dtype dtype, fbp_filter_kind kind,
                      const fbp_geometry *g, int n_slices, fbp_stream_t stream);

/*
 * fbp_backproject -- the backprojection step (Sec. V-A(c) stage 2,
 * "back-projection computation O(N_p N_x N_y N_z)").
 *   filt       device, [n_slices][K][D] of `dtype` (as written by fbp_filter).
 *   row_scale  device, float [n_slices][K] for F16/BF16 (NULL for F32):
 *              each row is multiplied by s_k before interpolation.
 *   slice      device, float [n_slices][n][n]: receives scale * sum_k Q_k,
 *              or has it added when `accumulate` is nonzero.
 *   scale      angle_step for FBP; 1 for the transpose of radon_forward.
 * Every pixel of the n x n square is computed.  Accumulation is FP32; the
 * per-(tile, angle) base coordinate is formed in FP64.  The kernel and its
 * tile are chosen from the geometry, dtype and device; a slice with too few
 * tiles to fill the GPU has its angle pairs shared among the blocks of a
 * thread-block cluster (partial sums added in a fixed order), so a slice's
 * result is the same run to run and whatever n_slices is.
 */
fbp_status fbp_backproject(const void *filt, const float *row_scale,
                           fbp_dtype dtype, float *slice, const fbp_geometry *g,
                           int n_slices, float scale, int accumulate,
                           fbp_stream_t stream);

/* fbp_backproject with an explicit compiled tile variant
 * (0 <= variant < fbp_bp_variant_count(); -1 = the library's default). */
fbp_status fbp_backproject_variant(const void *filt, const float *row_scale,
                                   fbp_dtype dtype, float *slice,
                                   const fbp_geometry *g, int n_slices,
                                   float scale, int accumulate, int variant,
                                   fbp_stream_t stream);

/*
 * Stage-2 pre-processing fused into the filter (Sec. V-A(c) stage 2: the
 * Beer-Lambert conversion and a Gaussian blur precede the filtering).  The
 * paper fixes neither the blur width nor the flat field; they are inputs.
 */
typedef struct {
    const float *flat;   /* device, float [n_det]: incident intensity I0 per detector
                            bin, or NULL to use flat_value for every bin */
    float flat_value;    /* I0 when flat is NULL (> 0) */
    float count_floor;   /* counts are raised to at least this before the log (> 0) */
    float mu_scale;      /* line integral unit: p = mu_scale * -ln(I / I0) (> 0);
                            n for line integrals in pixel units of an n-pixel field
                            of view whose attenuation is given per field width */
    float blur_sigma;    /* Gaussian blur along the detector, in bins, in [0, 3.875];
                            0 = none.  Taps exp(-k^2 / (2 sigma^2)), |k| <= floor(4 sigma
                            + 1/2), normalised to sum 1 in double, zero outside [0, D) */
} fbp_preprocess;

/*
 * fbp_filter_counts -- fbp_filter on detector counts: each sample I becomes
 * p = mu_scale * -ln(max(I, count_floor) / I0), each row is blurred with
 * the Gaussian, and the result is filtered exactly as fbp_filter filters
 * line integrals, in one pass (the line integrals are never written to
 * memory).  counts: device, float [n_slices][K][D]; the other arguments and
 * errors are fbp_filter's.  FBP_ERR_INVALID_ARG for a NULL pre, a
 * non-positive floor, scale or flat_value (flat NULL), or sigma outside
 * [0, 3.875].
 */
fbp_status fbp_filter_counts(const float *counts, void *filt, float *row_scale,
                             fbp_dtype dtype, fbp_filter_kind kind, const fbp_geometry *g,
                             int n_slices, const fbp_preprocess *pre, fbp_stream_t stream);

/*
 * Stage-4 output mapping (Sec. V-A(c) stage 4: slices normalised by CT
 * number (HU) range and quantised to uint16).  HU = 1000 (mu - mu_water) /
 * (mu_water - mu_air); the window [hu_min, hu_max] maps linearly onto
 * [0, 65535].
 */
typedef struct {
    double mu_water, mu_air;   /* attenuation of water and air in the slice's units */
    double hu_min, hu_max;     /* the window, hu_max > hu_min */
} fbp_hu_window;

/* FP32 coefficients the kernels use: code = clamp(rint(RN(RN(a * mu) + b)),
 * 0, 65535), rounded to nearest even; a and b are formed in double as
 * a = 1000 s / (mu_water - mu_air), b = -(1000 mu_water / (mu_water - mu_air)
 * + hu_min) s, s = 65535 / (hu_max - hu_min), then rounded to float.
 * FBP_ERR_INVALID_ARG for a NULL argument, a non-finite value,
 * mu_water == mu_air or hu_max <= hu_min.  Host-only. */
fbp_status fbp_hu_coefficients(const fbp_hu_window *w, float *a, float *b);

/*
 * fbp_backproject_u16 -- fbp_backproject_variant with the stage-4 mapping in
 * the epilogue: each pixel's value scale * sum_k Q_k is mapped to its uint16
 * code (see fbp_hu_coefficients) instead of being stored as FP32.
 *   slice  device, uint16 [n_slices][n][n]: receives the codes.
 * No accumulate mode.  Other arguments and errors as fbp_backproject_variant,
 * plus fbp_hu_coefficients' errors for the window.
 */
fbp_status fbp_backproject_u16(const void *filt, const float *row_scale, fbp_dtype dtype,
                               unsigned short *slice, const fbp_geometry *g, int n_slices,
                               float scale, const fbp_hu_window *w, int variant,
                               fbp_stream_t stream);

/*
 * Offset scans (Sec. V-A(b), "Addressing Load Imbalance in XCT Offset
 * Scans": the sample is shifted laterally so that a full-turn scan images a
 * field of view wider than the detector).  The rotation axis sits at
 * det_center, off the detector's centre, and the angles cover a full turn
 * (n_angles * angle_step = 2 pi).  A line (th + pi, -s) is the line (th, s),
 * so lines within `overlap` bins of the axis are measured twice and lines
 * farther out on the long side once.  The paper gives no weighting; this
 * library weights each sample before filtering with the smooth overlap
 * weight w(t) = (1 + sin(pi t / (2 overlap))) / 2 for |t| <= overlap, 0 for
 * t < -overlap and 1 for t > overlap, t the signed distance (bins) of the
 * sample's line from the axis, positive towards the long side; w(t) + w(-t)
 * = 1, so every line counts once.  The ramp filter spreads a weighted row
 * past the detector's short edge, so rows are filtered on a virtual detector
 * centred on the axis that spans the long side on both sides:
 *   n_v = 2 * (long side length) + 1 bins (long side = max(c, D-1-c) for
 *   c = det_center), centre (n_v - 1) / 2, physical bin m at virtual bin
 *   m + offset (offset = n_v - D when the long side is above c, else 0).
 */
typedef struct {
    double overlap;   /* half-width of the overlap weight, bins, 0 < overlap <=
                         the short side min(c, D-1-c)                        */
    int fold;         /* 1: fold the row at th + pi into the row at th (its
                         mirror, weight 1 - w), giving K/2 half-turn rows; K must
                         be even.  0: K weighted full-turn rows               */
} fbp_offset_scan;

/*
 * fbp_offset_geometry -- the geometry of the rows fbp_filter_offset writes,
 * for fbp_backproject: n_angles = K/2 (fold) or K, n_det = n_v,
 * det_center = (n_v - 1)/2; angle_start, angle_step, det_spacing,
 * pixel_size and n as in g.  Backproject with scale = angle_step: the
 * weights make each line count once over the full turn.  *offset (may be
 * NULL) receives the virtual index of physical bin 0.  Host-only, no CUDA
 * call.  FBP_ERR_INVALID_ARG for a NULL g/o/gv, an invalid geometry, a
 * det_center outside [0, D-1] or not a multiple of 1/2, overlap outside
 * (0, short side], angles not covering a full turn (|K angle_step - 2 pi| >
 * 1e-9 2 pi), or fold with K odd; FBP_ERR_UNSUPPORTED if n_v > 8192.
 */
fbp_status fbp_offset_geometry(const fbp_geometry *g, const fbp_offset_scan *o,
                               fbp_geometry *gv, int *offset);

/*
 * fbp_filter_offset -- fbp_filter for an offset scan: each physical row is
 * weighted, embedded in the virtual detector (zero elsewhere), folded when
 * o->fold is set, and filtered on the virtual detector, in one pass.
 *   sino   device, float [n_slices][K][D]: line integrals of the physical
 *          detector (g is the scan's geometry, full turn).
 *   filt   device, [n_slices][K'][n_v] of `dtype`, K' = K/2 (fold) or K:
 *          the filtered virtual rows, for fbp_backproject with the geometry
 *          from fbp_offset_geometry.  May not alias sino.
 *   row_scale  device, float [n_slices][K'] for F16/BF16 (as fbp_filter).
 * Errors: fbp_offset_geometry's, then fbp_filter's.
 */
fbp_status fbp_filter_offset(const float *sino, void *filt, float *row_scale, fbp_dtype dtype,
                             fbp_filter_kind kind, const fbp_geometry *g, int n_slices,
                             const fbp_offset_scan *o, fbp_stream_t stream);

/*
 * fbp_backproject_noalloc -- fbp_backproject for callers that cannot
 * allocate device memory.  The paper has no counterpart: this is a library
 * service, not a step of the method.
 *
 * fbp_backproject caches its FP64 angle table in device memory it allocates
 * with cudaMalloc the first time it sees a geometry.  Callers whose device
 * memory is owned by a framework's pool or fixed up front cannot allow that
 * allocation.  This variant
 * computes the angle table on `stream` into a static device array of at most
 * 16384 angles (256 KB, held on every device that runs it until the library
 * is unloaded) and calls no allocating routine; inputs and outputs are as for
 * fbp_backproject, and the result equals fbp_backproject's.
 *   * n_angles > 16384 returns FBP_ERR_UNSUPPORTED; filt and slice may not
 *     overlap (FBP_ERR_INVALID_ARG), as for fbp_backproject.
 *   * The first call on a device looks up the array's device address; make
 *     that first call before any stream capture.
 *   * All calls share the array and overwrite it completely.  Calls whose
 *     work overlaps on the GPU (unordered streams) race on it: order them.
 */
fbp_status fbp_backproject_noalloc(const void *filt, const float *row_scale,
                                   fbp_dtype dtype, float *slice,
                                   const fbp_geometry *g, int n_slices,
                                   float scale, int accumulate,
                                   fbp_stream_t stream);

/*
 * fbp_backproject_staged -- fbp_backproject with the backprojection tables
 * formed once per slice instead of once per thread block (the same step,
 * Sec. V-A(c) stage 2, for the symmetric orbit geometry).  A pass over the
 * filtered rows writes, for every angle pair (th_k, th_k + pi/2) and
 * detector segment, one table entry -- the segment midpoints and slopes of
 * the two rows and of their mirrors -- into the workspace; the
 * backprojection then moves each tile's window of entries into shared memory
 * with one bulk-tensor copy (zero-filled past the detector) and interpolates
 * with no block-wide barrier per stage.
 *   16-bit rows (FBP_F16, FBP_BF16): 16-byte entries of the orbit kernel
 *              (scaled by s_k / S, S = max_k s_k of the slice); the result is
 *              bit-identical to fbp_backproject_variant with the packed orbit
 *              variant of the same tile (10 for shapes 0-1, 11 for 2-5).
 *   FP32 rows: 32-byte entries, Q = midpoint + (u' - i) slope on the segment
 *              of the rounded index i (the orbit kernel's FP32 tables use
 *              block-relative intercepts instead, so results agree with it to
 *              FP32 rounding, not bit for bit).
 *   filt, row_scale, dtype, slice, g, n_slices, scale, accumulate  as
 *              fbp_backproject (row_scale only for 16-bit rows).
 *   shape      -1 default, or one of fbp_backproject_staged_shape_count(dtype):
 *              16-bit -- 0: 64 x 64 orbit tiles, 8 angle pairs per stage, 3
 *              buffers; 1: 64 x 64, 16 pairs, 2 buffers (default when n is a
 *              multiple of 128); 2: 32 x 32, 16 pairs, 3 buffers; 3: 32 x 32,
 *              8 pairs, 4 buffers; 4: 32 x 32, 8 pairs, 3 buffers, five blocks
 *              per SM; 5: 32 x 32, 8 pairs, 2 buffers, six blocks per SM (the
 *              default otherwise).  FP32 -- 0: 32 x 32, 4 pairs, 2 buffers, six
 *              blocks per SM (default); 1: 32 x 32, 4 pairs, 3 buffers, five
 *              blocks; 2: 32 x 32, 8 pairs, 2 buffers, three blocks; 3: 64 x 64,
 *              8 pairs, 2 buffers, two blocks.
 *   workspace  device, 256-byte aligned, owned by the caller, at least
 *              fbp_backproject_staged_workspace_bytes(g, dtype, 1) bytes; the
 *              call works through the stack in as many slices at a time as the
 *              workspace holds (c slices: (K/2) (D+1) 16 bytes per slice for
 *              16-bit rows, 32 for FP32, plus 256).
 * Geometry: angle step pi/K with K even, det_center = (D-1)/2, n a multiple
 * of twice the tile (FBP_ERR_UNSUPPORTED otherwise).  The table write and the
 * backprojection run on `stream`; the call may be captured once g's angle
 * table exists.
 */
size_t fbp_backproject_staged_workspace_bytes(const fbp_geometry *g, fbp_dtype dtype, int chunk);
int fbp_backproject_staged_shape_count(fbp_dtype dtype);
fbp_status fbp_backproject_staged(const void *filt, const float *row_scale, fbp_dtype dtype,
                                  float *slice, const fbp_geometry *g, int n_slices, float scale,
                                  int accumulate, int shape, void *workspace, size_t ws_bytes,
                                  fbp_stream_t stream);

/* fbp_backproject_staged with the stage-4 mapping in the epilogue (as
 * fbp_backproject_u16): each pixel's value scale * sum_k Q_k becomes its
 * uint16 code (fbp_hu_coefficients) in slice [n_slices][n][n] (device).
 * Arguments and errors as fbp_backproject_staged, plus the window's. */
fbp_status fbp_backproject_staged_u16(const void *filt, const float *row_scale, fbp_dtype dtype,
                                      unsigned short *slice, const fbp_geometry *g, int n_slices,
                                      float scale, const fbp_hu_window *w, int shape, void *workspace,
                                      size_t ws_bytes, fbp_stream_t stream);

/*
 * radon_forward -- the matched forward projector A (the adjoint of
 * fbp_backproject with scale 1; the paper's data generation uses a forward
 * model, Sec. V-B(a)):  (A f)_k[j] = sum_{r,c} f[r][c] max(0, 1 - |u_k(r,c) - j|).
 *   slice  device, float [n_slices][n][n].
 *   sino   device, float [n_slices][K][D]: receives A f (overwritten).
 * Uses the library's default variant (see radon_forward_variant).
 */
fbp_status radon_forward(const float *slice, float *sino, const fbp_geometry *g,
                         int n_slices, fbp_stream_t stream);

/*
 * radon_forward with an explicit kernel:
 *   0   gather form: one thread per output bin walks the image; deterministic,
 *       any pixel_size / det_spacing in [1/8, 2.5].
 *   1-5 tile-owned form: one block per 64 x 64 pixel tile visits every angle
 *       and adds per-tile partial bins with floating-point atomics; 1-3 take
 *       one slice per block (8, 16 or 32 bins per warp), 4 takes four slices
 *       per block and 5 two (one shared-memory load serves every slice;
 *       leftover slices run through the narrower forms).  The sum over
 *       tiles is not in a fixed order, so results may differ between runs
 *       in the last bits.  Needs
 *       pixel_size / det_spacing in [0.9429, 1] (FBP_ERR_UNSUPPORTED
 *       otherwise).  The sinogram is cleared on `stream` first.
 *  -1   the default: the fastest tile-owned variant where it applies, else 0.
 * Other values return FBP_ERR_INVALID_ARG.
 */
fbp_status radon_forward_variant(const float *slice, float *sino, const fbp_geometry *g,
                                 int n_slices, int variant, fbp_stream_t stream);

/* Number of forward-projector variants (valid variant values are 0 .. count-1). */
int radon_forward_variant_count(void);

/* Number of compiled backprojection tile variants, and the shape of one. */
int fbp_bp_variant_count(void);
fbp_status fbp_bp_variant_info(int variant, fbp_bp_shape *out);

/* 1 if fbp_backproject_variant accepts `variant` for rows of `dtype` and
 * geometry g (symmetric variants need the standard geometry; every variant
 * needs its staged window to fit in shared memory), 0 otherwise.  Host-only,
 * no CUDA call. */
int fbp_bp_variant_supports(int variant, fbp_dtype dtype, const fbp_geometry *g);

/*
 * Ragged batches (Sec. V-A(b): specimens with various N_p and N_c
 * reconstructed together).  One persistent filter launch and persistent
 * backprojection launches cover every item; items may differ in K, D, n and
 * geometry.
 *   items      HOST array of `count` items (1 <= count <= 256); each item's
 *              sino/slice are device pointers as above.  n_det <= 8192.
 *   workspace  device, >= fbp_batched_workspace_bytes(items, count, dtype)
 *              bytes, 256-byte aligned, owned by the caller.  It holds the
 *              work-queue counters, the filtered rows of every item and, for
 *              each item that fbp_batched_item_staged accepts, its padded
 *              angle-pair table (about 4-6x its FP32 rows, 2-3x its 16-bit
 *              rows; the size does not depend on bp_variant).
 *   bp_variant -1 = default: the items that fbp_batched_item_staged accepts
 *              run in one persistent launch of staged units (90-degree orbits
 *              of four tiles, 32 x 32 for FP32 rows and 64 x 64 for 16-bit
 *              rows, whose windows are moved by bulk copies from their padded
 *              tables; each such slice is bit-identical to
 *              fbp_backproject_staged with shape 0 for FP32 rows, shape 1 for
 *              16-bit rows), the others in the persistent tile kernel with
 *              variant 8 (FP32 rows) or 10 (16-bit rows).  A tile variant
 *              (fbp_bp_variant_info) runs every item in the persistent tile
 *              kernel: with a symmetric variant, items whose geometry has the
 *              90-degree symmetry (angle step pi/K with K even, det_center =
 *              (D-1)/2, n a multiple of twice the variant's tile) run its
 *              orbit units and every other item runs generic tiles of the
 *              same thread count (64 x 32 for 128-thread variants, 64 x 64 for
 *              256); with a generic variant every item runs that variant's
 *              tiles.  Each item's slice is then bit-identical to
 *              fbp_backproject_variant on the same rows with the shape the
 *              item ran.  Packed variants (10, 11) with FP32 rows return
 *              FBP_ERR_UNSUPPORTED.
 * The call captures into a CUDA graph once each item's geometry has been
 * seen by the library (tables exist).
 */
size_t fbp_batched_workspace_bytes(const fbp_batch_item *items, int count,
                                   fbp_dtype dtype);
fbp_status fbp_batched(const fbp_batch_item *items, int count,
                       fbp_filter_kind kind, fbp_dtype dtype, int bp_variant,
                       void *workspace, size_t ws_bytes, fbp_stream_t stream);

/* 1 if a batch item whose filtered rows have geometry g and dtype runs
 * staged units under fbp_batched's default, 0 otherwise: the 90-degree
 * symmetry with n a multiple of twice the dtype's tile (FP32 rows: 64,
 * 16-bit rows: 128) and a backprojection window of at most 72 (FP32) / 104
 * (16-bit) detector segments, i.e. pixel_size / det_spacing up to about 1.5
 * (FP32) / 1.1 (16-bit).  For an offset item of fbp_batched_scans pass its
 * virtual geometry (fbp_offset_geometry).  Host-only, no CUDA call. */
int fbp_batched_item_staged(const fbp_geometry *g, fbp_dtype dtype);

/*
 * Mixed batches of normal and offset scans (Sec. V-A(b): specimens with
 * various N_p, N_r, N_c, "both normal scan CT and offset scan CT",
 * reconstructed simultaneously).  An item with overlap > 0 is a full-turn
 * offset scan (g as for fbp_filter_offset, weighted and optionally folded on
 * its virtual detector); overlap == 0 is a normal scan (g as for fbp_filter).
 */
typedef struct {
    const float *sino;   /* device, float [n_angles][n_det]: the scan's rows     */
    float *slice;        /* device, float [n][n]: the reconstruction             */
    fbp_geometry g;      /* the scan's geometry                                  */
    double overlap;      /* 0: normal scan; > 0: offset scan (fbp_offset_scan)   */
    int fold;            /* offset scans: 1 = fold the half turns (K even)       */
} fbp_scan_item;

/* Work order of the batch's persistent backprojection launch.  A work unit
 * is one output tile of one item. */
typedef enum {
    FBP_ORDER_QUEUE = 0,        /* items by total cost K n^2, largest first; blocks
                                   take the next unit from an atomic counter      */
    FBP_ORDER_GROUP_CYCLIC = 1  /* the paper's group-and-cyclic mapping (Sec.
                                   V-A(b)): units sorted by cost per unit, so each
                                   run of P consecutive units (P = resident blocks)
                                   is a group of similar cost, and block b takes
                                   units b, b + P, b + 2P, ...: one unit of every
                                   group, no atomics                              */
} fbp_batch_order;

/*
 * fbp_batched_scans -- fbp_batched for mixed items, with a chosen work
 * order.  Arguments and errors as fbp_batched, plus fbp_offset_geometry's
 * errors for offset items and FBP_ERR_INVALID_ARG for an unknown order.
 * Each item's virtual detector must have n_v <= 8192 bins.  The workspace
 * holds each item's filtered rows ([K'][n_v] for offset items, K' = K/2
 * when folded).
 */
size_t fbp_batched_scans_workspace_bytes(const fbp_scan_item *items, int count,
                                         fbp_dtype dtype);
fbp_status fbp_batched_scans(const fbp_scan_item *items, int count,
                             fbp_filter_kind kind, fbp_dtype dtype, int bp_variant,
                             fbp_batch_order order, void *workspace, size_t ws_bytes,
                             fbp_stream_t stream);

/*
 * fbp_host -- filtered backprojection of a stack held in HOST memory, with
 * host<->device copies overlapped with the kernels (the paper's overlapped
 * load / FBP computation / store pipeline, Sec. V-A(c), on one GPU).  The
 * stack is cut into chunks of `chunk` slices; chunk i runs on internal stream
 * i mod n_streams: copy in, fbp_filter (fbp_filter_counts when pre != NULL),
 * the backprojection with scale = angle_step -- where bp_variant is -1 and
 * the geometry has the orbit symmetry with n a multiple of 64 and at least
 * 1024, fbp_backproject_staged (FP32 out) or fbp_backproject_staged_u16
 * (window != NULL), else fbp_backproject_variant or fbp_backproject_u16 --
 * copy out, so the copies of one chunk run while another chunk's kernels
 * do.  The results equal those calls on device buffers.  The internal
 * streams are kept per device between calls (created on first need).
 *   sino_host   HOST, float [n_slices][K][D]: line integrals, or detector
 *               counts when pre != NULL.  Pinned memory (cudaHostAlloc or
 *               cudaHostRegister) lets the copies overlap; pageable memory
 *               works but serialises them.
 *   slice_host  HOST, [n_slices][n][n]: float slices, or uint16 codes when
 *               window != NULL.
 *   kind, dtype as fbp_filter; bp_variant as fbp_backproject_variant.
 *   pre         NULL, or the stage-2 pre-processing (fbp_filter_counts; its
 *               flat is a device pointer).
 *   window      NULL, or the stage-4 HU window (fbp_backproject_u16).
 *   chunk       slices per chunk, >= 1; n_streams in [1, 16].
 *   workspace   device, >= fbp_host_workspace_bytes(g, dtype, chunk,
 *               n_streams, window != NULL) bytes, 256-byte aligned, owned
 *               by the caller: per stream one chunk's input, filtered rows,
 *               row scales, output and (staged path) tables.
 *   stream      the pipeline starts after the work already enqueued on it.
 * Blocking: returns when every slice is in slice_host (or after an error,
 * once nothing is in flight).  Creates and destroys its streams; allocates
 * no device memory beyond the first call's constant tables for g (not for
 * stream capture).  Errors: those of the calls above, FBP_ERR_WORKSPACE,
 * FBP_ERR_INVALID_ARG for a device pointer as sino_host or slice_host.
 * fbp_host_workspace_bytes returns 0 for invalid arguments.
 */
size_t fbp_host_workspace_bytes(const fbp_geometry *g, fbp_dtype dtype, int chunk, int n_streams,
                                int codes);
fbp_status fbp_host(const float *sino_host, void *slice_host, const fbp_geometry *g, int n_slices,
                    fbp_filter_kind kind, fbp_dtype dtype, int bp_variant,
                    const fbp_preprocess *pre, const fbp_hu_window *window, int chunk,
                    int n_streams, void *workspace, size_t ws_bytes, fbp_stream_t stream);

/*
 * Device status word.  Kernels never trap: a kernel that detects a fault
 * records a nonzero code in a device word and returns.  Codes: 1 a
 * work-queue loop past its iteration cap; 2 (checked build) an
 * interpolation index outside the staged table; 3 reserved; 4 a
 * union-find loop of the patching kernels (sap.h) past its cap; 5 a
 * quadtree leaf entry outside the slice (sap.h); 6 a wait of the streamed
 * filter for its row copy past its cap (the block then stops; after two
 * expired waits a copy into its shared memory may still be in flight, so
 * treat code 6 as voiding that launch's output and any kernel enqueued after
 * it on the stream: synchronise and discard those results); 7 a wait of
 * fbp_backproject_staged or a staged batch unit for a window copy past its
 * cap (the block writes nothing, after a capped wait for its copies); 8 a
 * staged batch window outside its item's padded table (the copy is
 * clamped into the table; that item's slice is wrong).  The
 * first fault recorded stays until read.  This call synchronises `stream`,
 * reads and clears the word, and returns FBP_OK or FBP_ERR_DEVICE_STATUS
 * (code in *code if non-NULL).
 */
fbp_status fbp_last_device_status(fbp_stream_t stream, int *code);

/* Build the constant tables for geometry g on the current device (the same
 * work the first fbp_* call for g does), so that later calls can be captured
 * in a CUDA graph.  kind < 0 skips the filter tables. */
fbp_status fbp_prepare(const fbp_geometry *g, int kind, fbp_stream_t stream);

/* Free every cached table on every device (synchronises those devices). */
void fbp_release_tables(void);

/*
 * Measured on-chip ceilings of the current device, for the roofline of the
 * backprojection and the forward projector (the paper has no counterpart:
 * this is a measurement service).  Both kernels are bound by the path that
 * carries shared-memory loads into registers and by the FP32 lanes, so
 * their ceilings are per-SM rates rather than HBM bandwidth.  Two probe
 * kernels run on every SM (eight 256-thread blocks each): conflict-free
 * 16-byte shared loads, and eight independent FP32 FMA chains per thread;
 * each SM's cycles come from its own clock64 counter, so the rates are per
 * clock and per SM, whatever clock the GPU ran at (median over SMs).
 *   lds_bytes_per_clk_per_sm  bytes delivered by ld.shared.v4 per SM cycle
 *   fma_per_clk_per_sm        FP32 FMA lane operations per SM cycle
 *   sm_clock_mhz              cycles / event time of the shared-load probe
 *   sm_count                  multiprocessors of the device
 * Synchronous (runs on the legacy default stream and waits, ~10 ms); not for
 * stream capture.  Returns FBP_ERR_INVALID_ARG for a NULL out.
 */
typedef struct {
    double lds_bytes_per_clk_per_sm;
    double fma_per_clk_per_sm;
    double sm_clock_mhz;
    int sm_count;
} fbp_onchip_peaks;
fbp_status fbp_measure_onchip_peaks(fbp_onchip_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* FBP_H */
