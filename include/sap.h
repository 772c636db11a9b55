/*
 * sap.h -- C ABI (in libfbp.so) of symmetric adaptive patching (SAP) of
 * reconstructed slices and of the 2-bit masks, on one GB300 GPU.
 *
 * The paper's AI stage (Sec. V-B(c), "Symmetric Adaptive Patching") turns
 * each reconstructed slice into a fixed-length sequence of patches for the
 * segmentation model: (1) Canny edge detection, (2) a quadtree grown by
 * splitting the leaf whose edge image has the largest sum (Eq. (1), argmax_i
 * V(L_n[i]), s = 4 children in 2-D), then by pixel-intensity variance so that
 * every slice gives the same sequence length, ordered along a Z-order curve,
 * (3) depatching of the mask patches through the stored quadtree.  The fused
 * reconstruction + AI pipeline stores four-class masks as 2 bits per pixel
 * (Sec. V-C(a)).  The paper fixes none of the numbers or tie rules; this
 * library's are:
 *
 *   edges     integer Canny on the uint16 codes: 5-tap binomial (1 4 6 4 1)
 *             smoothing along each axis, 3x3 Sobel, M = |gx| + |gy| (borders
 *             replicated); non-maximum suppression along the gradient
 *             quantised to 0/45/90/135 degrees (|gy| 2^15 against 13573 |gx|
 *             and 79109 |gx|); a pixel survives if M exceeds the previous
 *             neighbour's and is not below the next one's (0 outside the
 *             slice); strong if M > canny_hi, weak if canny_lo < M <= hi;
 *             edges = strong pixels and weak pixels 8-connected to them
 *             through weak pixels.
 *   quadtree  V(node) = edge pixels in the node; variance key = the node's
 *             sum of squared deviations d(S2) - d(S1) d(S1) / d(n) in IEEE
 *             double (S1, S2 exact integer sums of codes and squared codes),
 *             replaced by its parent's key where larger; a node of side > P
 *             is split while the leaf count is below `length`, taking the
 *             largest (V, variance key), then the shallower node, then the
 *             smaller Morton code; i.e. the split set is the top
 *             (length - 1) / 3 nodes in that order.
 *   sequence  leaves in Z-order (Morton code of the top-left corner in units
 *             of P, x in the even bits); leaf i of side s = P 2^j is patch i:
 *             P x P means of 2^j x 2^j blocks, float(d(block sum) / d(4^j)).
 *   masks     depatching writes patch value [r][c] of leaf i to its pixels
 *             [y0 + r 2^j + a][x0 + c 2^j + b]; the 2-bit mask holds pixel
 *             4k + t of a row in bits 2t..2t+1 of byte k.
 *
 * Conventions as in fbp.h: device pointers owned by the caller, row-major
 * arrays, work enqueued on `stream`, synchronous validation (an error other
 * than FBP_ERR_CUDA enqueues nothing).  Results are exact: every decision
 * is taken in integer arithmetic or in a fixed sequence of IEEE operations.
 */
#ifndef SAP_H
#define SAP_H

#include <stddef.h>

#include "fbp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n;          /* slice side: a power of two, 16 <= n <= 16384          */
    int patch;      /* P: patch side, 4, 8, 16, 32 or 64, P <= n             */
    int length;     /* patches per slice: 1 <= length <= (n / P)^2 and
                       length = 1 (mod 3) (each split adds three leaves)     */
    int canny_lo;   /* weak threshold on M, >= 0                             */
    int canny_hi;   /* strong threshold on M, >= canny_lo                    */
} sap_params;

/* Device workspace bytes sap_edges and sap_patches need (one buffer serves
 * both, used in turn); 0 if the parameters are invalid.  Host-only. */
size_t sap_workspace_bytes(const sap_params *p);

/*
 * sap_edges -- step (1): the Canny edge map of one slice.
 *   slice   device, uint16 [n][n]: the slice's codes (e.g. the output of
 *           fbp_backproject_u16).
 *   edges   device, uint8 [n][n]: receives 1 on edges, 0 elsewhere.
 *   workspace  device, >= sap_workspace_bytes(p), 256-byte aligned.
 * FBP_ERR_INVALID_ARG for bad parameters or NULL pointers,
 * FBP_ERR_WORKSPACE for a missing, small or misaligned workspace.  The
 * union-find loops are capped; a cap reached records a fault in the device
 * status word (fbp_last_device_status).
 */
fbp_status sap_edges(const unsigned short *slice, unsigned char *edges, const sap_params *p,
                     void *workspace, size_t ws_bytes, fbp_stream_t stream);

/*
 * sap_patches -- step (2): the adaptive quadtree of one slice and its patch
 * sequence.
 *   slice    device, uint16 [n][n]; edges device, uint8 [n][n] (sap_edges).
 *   patches  device, float [length][P][P]: receives the patches in Z-order.
 *   leaves   device, int [length][3]: receives (x0, y0, side) of each patch's
 *            quadtree leaf, in the same order (the structure depatching uses).
 * Errors as sap_edges.
 */
fbp_status sap_patches(const unsigned short *slice, const unsigned char *edges, float *patches,
                       int *leaves, const sap_params *p, void *workspace, size_t ws_bytes,
                       fbp_stream_t stream);

/*
 * sap_depatch_pack -- step (3) and the 2-bit mask: four-class mask patches
 * scaled back onto the slice through the quadtree and packed 4 pixels per
 * byte.
 *   mask_patches  device, uint8 [length][P][P], classes 0..3 (higher bits
 *                 are ignored).
 *   leaves        device, int [length][3] as written by sap_patches.
 *   packed        device, uint8 [n][n / 4]: receives the 2-bit mask.
 * The leaves must tile the slice (as sap_patches writes them); nothing else
 * is written.  A leaf that lies outside the slice, or whose side is not
 * P 2^j or whose corner is not a multiple of its side, is skipped and
 * recorded in the device status word (code 5, fbp_last_device_status); the
 * other leaves are still written.  No workspace.
 */
fbp_status sap_depatch_pack(const unsigned char *mask_patches, const int *leaves,
                            unsigned char *packed, const sap_params *p, fbp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SAP_H */
