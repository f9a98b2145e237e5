/*
 * gsff.h -- C ABI of the GB300 feature-field Gaussian rasterizer.
 *
 * The library renders a set of 3D Gaussians (paper Sec. 3.1: mean mu,
 * quaternion q, scale s, opacity alpha, colour c, feature embedding f in R^N)
 * at a camera pose T_CW into RGB, depth, accumulated opacity and an N-channel
 * feature map by front-to-back alpha compositing (Eq. 2-3), and back-propagates
 * a loss through it, including the Lie-algebra pose gradient (Eq. 4) and a
 * feature gradient that reaches only f (Sec. 3.1, "decoupled").
 *
 * Conventions shared by every call:
 *  - Every array pointer is DEVICE memory owned by the caller; the library
 *    never allocates. Scratch space comes from the caller through the
 *    *_workspace_bytes queries (256-byte aligned base required).
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL is the legacy default stream). Host pointers (the camera, bg) are
 *    read before the call returns.
 *  - Invalid arguments are reported synchronously by the return value and
 *    nothing is launched. Errors found on the device are OR-ed as bit flags
 *    (1 << gs_status) into *status (a device int32 the caller zeroes); kernels
 *    never trap and never spin without a bound.
 *  - Gradient outputs are ACCUMULATED (+=): the caller zeroes them.
 *  - Array shapes below are row-major; [P,3] means 3 consecutive floats per
 *    Gaussian.
 */
#ifndef GSFF_H
#define GSFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1,  /* synchronous: a null/misaligned pointer or a size out of range */
  GS_ERR_CAPACITY = 2,     /* device: more tile instances than the caller's capacity */
  GS_ERR_TIMEOUT = 3,      /* device: a bounded wait gave up */
  GS_ERR_CUDA = 4,         /* a CUDA launch or runtime call failed */
  GS_ERR_UNSUPPORTED = 5,  /* a valid but unimplemented combination of options */
  GS_ERR_BOUNDS = 6        /* device, bounds-checked build only: an index read from the inputs (a Gaussian id
                              of the sorted lists, a saved last index) was out of range; it was not followed */
} gs_status;

/* Pinhole camera and world->camera transform T_CW: mu_c = R mu + t.
 * OpenCV axes (x right, y down, z forward); pixel (i, j) has its centre at
 * (i + 0.5, j + 0.5). R is row-major. Gaussians with z_c <= near_z are culled. */
typedef struct gs_camera {
  int32_t width, height;
  float fx, fy, cx, cy;
  float R[9];
  float t[3];
  float near_z;
  /* Optional device copy of the pose: 12 floats (R row-major, then t). When
   * not NULL the kernels read the world -> camera transform from it instead
   * of R and t, so a pose updated on the device (gs_pose_update) is used by
   * the next frame's calls without a host round trip. */
  const float* pose_dev;
} gs_camera;

/* flags of gs_render_fwd / gs_render_bwd */
enum {
  GS_FEAT_OFF = 0,          /* Eq. 3 "otherwise": no feature work at all */
  GS_FEAT_ON = 1,           /* render (and back-propagate) the N feature channels */
  GS_FEAT_TENSOR_CORE = 2   /* with GS_FEAT_ON and BF16 features: tcgen05 contraction */
};
enum { GS_FEAT_GRAD_DECOUPLED = 0, GS_FEAT_GRAD_COUPLED = 1 };
enum { GS_F32 = 0, GS_BF16 = 1 };
enum { GS_LAYOUT_CHW = 0, GS_LAYOUT_HWC = 1 };

enum { GS_TILE = 16 };      /* tiles are 16 x 16 pixels, numbered row-major */

/* ---------------------------------------------------------------------------
 * gs_project -- per-Gaussian EWA projection (Eq. 1 and the 3DGS projection
 * the paper builds on, Sec. 3.1).
 *
 * In:  means [P,3], scales [P,3] (linear, > 0), quats [P,4] (w,x,y,z, not
 *      necessarily unit), opacity [P] (already in (0,1)).
 * Out: uv [P,2] pixel coordinates of the projected mean; conic_opacity [P,4]
 *      = (A, B, C, opacity) with [[A,B],[B,C]] the inverse of the 2D
 *      covariance J W Sigma W^T J^T + 0.3 I; depth [P] = z_c; rect [P,4] =
 *      tile rectangle (x0, y0, x1, y1), ends exclusive; tiles_touched [P] =
 *      (x1-x0)(y1-y0), 0 for a culled Gaussian.
 *      n_instances (optional, device int64): set to sum(tiles_touched).
 * Every output is computed in binary32 in one fixed order of operations (no
 * fused multiply-add), so tile rectangles and depth keys are reproducible
 * bit for bit by an independent binary32 evaluation.
 * Culling: non-finite input, z_c <= near_z, zero quaternion, non-positive or
 * non-finite determinant, or a 3-sigma box outside the image.
 */
gs_status gs_project(const gs_camera* cam, int32_t P, const float* means, const float* scales,
                     const float* quats, const float* opacity, float* uv, float* conic_opacity,
                     float* depth, int32_t* rect, int32_t* tiles_touched, int64_t* n_instances,
                     void* stream);

/* ---------------------------------------------------------------------------
 * gs_bin_sort -- the per-tile depth-sorted instance lists (Sec. 3.1: the
 * projected Gaussians are sorted front to back per 16x16 tile).
 *
 * For every Gaussian g and every tile k of its rectangle there is one
 * instance; the instances are ordered by the key (k << 32) | bits(depth_g)
 * with equal keys in ascending g (bits(depth) orders like depth, as depth > 0).
 * Computed per tile: the instances are counted and placed into their tiles'
 * ranges, then each tile's (depth bits, g) pairs are sorted on their own.
 * In:  depth [P], rect [P,4], tiles_touched [P] from gs_project.
 * Out: gids [capacity] (u32), first I entries valid; keys [capacity] (u64,
 *      may be NULL) = the sorted keys; tile_ranges [num_tiles,2] = [start,
 *      end) into gids, (0,0) if empty; n_instances (device int64) = I.
 * If I > capacity, GS_ERR_CAPACITY is flagged in *status and the lists are
 * truncated: tiles that start past the capacity get (0, 0) and the tile
 * across it a shortened range over some of its instances (which ones is
 * unspecified); every range covers written ids < P only. workspace must hold
 * gs_bin_sort_workspace_bytes(P, capacity, num_tiles) bytes (0 is returned
 * for sizes out of range); the caller need not clear it. The sort has no
 * wait on other blocks.
 */
size_t gs_bin_sort_workspace_bytes(int32_t P, int64_t capacity, int32_t num_tiles);
gs_status gs_bin_sort(const gs_camera* cam, int32_t P, const float* depth, const int32_t* rect,
                      const int32_t* tiles_touched, int64_t capacity, void* workspace,
                      size_t workspace_bytes, uint64_t* keys, uint32_t* gids, int32_t* tile_ranges,
                      int64_t* n_instances, int32_t* status, void* stream);

/* gs_count_nonfinite -- adds to *count (device uint64, the caller zeroes it)
 * the number of NaN or infinite values among the n floats at x (device,
 * 4-byte aligned): the scan of an output or gradient buffer for non-finite
 * values. The paper has no counterpart. */
gs_status gs_count_nonfinite(int64_t n, const float* x, uint64_t* count, void* stream);

/* ---------------------------------------------------------------------------
 * gs_bin_sort_static -- gs_bin_sort for callers that cannot allocate device
 * memory. The paper has no counterpart; this is a deployment addition.
 *
 * Some callers cannot call cudaMalloc: a camera-tracking thread that must
 * meet a per-frame deadline (cudaMalloc and cudaFree can synchronise the
 * whole device and stall it), or a host application that owns every device
 * allocation and only lends the library its input and output buffers. This
 * entry point takes the same inputs and outputs as gs_bin_sort and runs the
 * same kernels, but keeps its scratch space in a fixed device array of
 * GS_BIN_SORT_STATIC_SCRATCH_BYTES (32 MiB) inside the library instead of a
 * caller workspace. It calls no allocator. Every device that loads the
 * library holds that array until the process exits.
 * Limit: gs_bin_sort_workspace_bytes(P, capacity, num_tiles) must not exceed
 * GS_BIN_SORT_STATIC_SCRATCH_BYTES (about 2.08 million instances of capacity
 * with up to 65,536 tiles: 16 bytes per instance plus 4 per tile, whatever P);
 * larger sizes return GS_ERR_INVALID_ARG and launch nothing.
 * keys may be NULL, as for gs_bin_sort.
 * The first call on a device looks up the array's device address with that
 * device current (a CUDA runtime query); make that first call before any
 * stream capture. The address is kept per device and context: a call that
 * finds a different context current on the device (for instance after
 * cudaDeviceReset) looks it up again. All calls share the one array and it keeps the previous
 * call's contents (the caller zeroes nothing: the sort clears the counters
 * it needs with a kernel on its stream): calls whose work
 * overlaps on the GPU (several streams or host threads) race on the array and
 * must be serialised by the caller.
 */
#define GS_BIN_SORT_STATIC_SCRATCH_BYTES (32u << 20)
gs_status gs_bin_sort_static(const gs_camera* cam, int32_t P, const float* depth, const int32_t* rect,
                             const int32_t* tiles_touched, int64_t capacity, uint64_t* keys, uint32_t* gids,
                             int32_t* tile_ranges, int64_t* n_instances, int32_t* status, void* stream);

/* ---------------------------------------------------------------------------
 * gs_zero -- clears `bytes` bytes of device memory at `ptr` (4-byte aligned,
 * bytes a multiple of 4) with one kernel that, like the library's other
 * kernels, is launched as a programmatic dependent of the previous one on the
 * stream, so a caller's clear between two library calls does not end their
 * overlap (e.g. the gradient outputs before gs_render_bwd, which accumulates).
 */
gs_status gs_zero(void* ptr, size_t bytes, void* stream);

/* ---------------------------------------------------------------------------
 * gs_tile_order -- a launch order for the compositing kernels: the tiles by
 * descending length of their lists, so that the longest tiles start first
 * and the shortest fill the end of the grid. The paper has no counterpart
 * (a scheduling aid; no result depends on it).
 * In:  tile_ranges [num_tiles,2] from gs_bin_sort.
 * Out: tile_order [num_tiles] (int32), a permutation of 0..num_tiles-1 in
 *      which the lengths fall in non-increasing buckets of 8 instances
 *      (lengths of 8184 and more share the first bucket); the order within
 *      a bucket is unspecified.
 * The render calls take it as tile_order (NULL = tiles in index order).
 */
gs_status gs_tile_order(int32_t num_tiles, const int32_t* tile_ranges, int32_t* tile_order, void* stream);

/* ---------------------------------------------------------------------------
 * gs_render_fwd -- front-to-back alpha compositing per pixel (Eq. 2-3).
 *
 * For pixel p in tile k, walking k's list in order with T = 1:
 *   power = -(A dx^2 + C dy^2)/2 - B dx dy, (dx, dy) = (u, v) - p;
 *   skip if power > 0; alpha = min(0.99, o exp(power)); skip if alpha < 1/255;
 *   stop (without blending) if T (1 - alpha) < 1e-4; else w = alpha T,
 *   C += w c, D += w d, F += w f, T *= 1 - alpha.
 * Out: out_rgb [3,H,W] = C + T bg; out_depth [H,W] = D; out_alpha [H,W] = 1 - T;
 *      out_feat [N,H,W] (layout CHW) or [H,W,N] (HWC), only with GS_FEAT_ON;
 *      T_final [H,W]; last_idx [H,W] = list position (from the tile's start)
 *      of the last blended Gaussian + 1; n_contrib [H,W] = blended count.
 * visible [P] (u8, may be NULL): set to 1 for every Gaussian blended at some
 *      pixel with T > 0.5 in front of it (the visibility V_id of the keyframe
 *      selection, Sec. 3.2, Eq. 5); other entries are left unchanged, so the
 *      caller zeroes the array (or keeps OR-ing frames into it).
 * feats [P,N] is float32 (GS_F32) or bfloat16 (GS_BF16); may be NULL with
 * GS_FEAT_OFF. bg: 3 host floats, NULL = black.
 * GS_FEAT_TENSOR_CORE (N % 64 == 0, N <= 512, GS_BF16, layout HWC): the
 * feature channels are computed per half tile as the product of a 128 x 32
 * weight matrix per step of 32 Gaussians (w = alpha T, rounded to bf16) and
 * the 32 x N bf16 feature rows on tcgen05 tensor cores, fp32 accumulation.
 * tile_order: NULL, or a permutation of the tiles (gs_tile_order) giving the
 * order in which tile blocks are launched; the outputs do not depend on it
 * (in the adjoints, only the summation order of the per-tile float atomics).
 * inst_masks: NULL, or [capacity] bytes indexed like gids: for every instance
 * it loads, the forward writes which of the tile's four 8x8 pixel blocks the
 * instance's Gaussian can reach (bit b: block b, 2 across by 2 down; the
 * conservative alpha >= 1/255 test). gs_render_bwd of the same frame (same
 * projection, lists and forward) reads them instead of testing again; its
 * masks must come from that forward (NULL there: computed in the adjoint).
 * They change no result, only which pixel blocks skip a Gaussian.
 */
gs_status gs_render_fwd(const gs_camera* cam, int32_t P, const int32_t* tile_ranges,
                        const int32_t* tile_order, const uint32_t* gids, uint8_t* inst_masks,
                        const float* uv, const float* conic_opacity,
                        const float* depth, const float* colors, const void* feats, int32_t N,
                        int32_t feat_dtype, int32_t layout, int32_t flags, const float* bg,
                        float* out_rgb, float* out_depth, float* out_alpha, float* out_feat,
                        float* T_final, int32_t* last_idx, int32_t* n_contrib, uint8_t* visible,
                        int32_t* status, void* stream);

/* ---------------------------------------------------------------------------
 * gs_visibility_iou -- co-visibility of two frames for keyframe selection
 * (Sec. 3.2): counts[0] = |{g : a_g and b_g}|, counts[1] = |{g : a_g or b_g}|
 * over two visibility vectors of gs_render_fwd (u8 [P], nonzero = visible).
 * counts: 2 device int64, overwritten (cleared by a memset on the stream);
 * IoU = counts[0] / counts[1]; a frame becomes a keyframe when its IoU with
 * the last keyframe is below the caller's threshold.
 */
gs_status gs_visibility_iou(int32_t P, const uint8_t* vis_a, const uint8_t* vis_b, int64_t* counts,
                            void* stream);

/* ---------------------------------------------------------------------------
 * gs_render_bwd -- adjoint of gs_render_fwd and gs_project, plus the pose
 * gradient of Eq. 4.
 *
 * Walks each pixel's list backwards from last_idx, recovering the
 * transmittance in front of each blended Gaussian as T_i = T_{i+1}/(1-alpha_i)
 * from the saved T_final (no per-pair storage). Cotangents dL_drgb [3,H,W],
 * dL_ddepth [H,W], dL_dalpha [H,W], dL_dfeat (layout as out_feat) may be NULL
 * (zero). feat_grad_mode GS_FEAT_GRAD_DECOUPLED is the paper's rule (Sec. 3.1):
 * dL_dfeat reaches d_feats only; GS_FEAT_GRAD_COUPLED also sends it through
 * alpha into the geometry (the full derivative).
 * Out (accumulated): d_means [P,3], d_scales [P,3], d_quats [P,4],
 *      d_opacity [P], d_colors [P,3], d_feats [P,N] (fp32 even for bf16
 *      features), d_pose [6] = (rho, theta) of the left perturbation
 *      T_CW <- Exp(tau) T_CW at tau = 0. d_pose is required; d_means,
 *      d_scales, d_quats, d_opacity and d_colors may each be NULL (not
 *      written), as in tracking, where the Gaussians are frozen (Sec. 3.2).
 * GS_FEAT_TENSOR_CORE (decoupled mode, bf16 features, layout HWC, N % 128
 * == 0, N <= 512): the feature gradient is computed per half tile as the
 * tcgen05 product dL/dF^T [N x 128 px] (rounded to bf16) times the weights
 * W [128 px x 32 Gaussians] (bf16), fp32 accumulation; the geometry
 * gradients stay on the fp32 SIMT kernel. Coupled mode is GS_ERR_UNSUPPORTED
 * there; dL_dfeat and d_feats must be 16-byte aligned (GS_ERR_INVALID_ARG
 * otherwise), since d_feats rows are accumulated with vector atomics.
 * workspace must hold gs_render_bwd_workspace_bytes(P) bytes.
 * tile_order and inst_masks as for gs_render_fwd: any permutation or NULL,
 * and the masks of the forward this call differentiates or NULL.
 */
size_t gs_render_bwd_workspace_bytes(int32_t P);
gs_status gs_render_bwd(const gs_camera* cam, int32_t P, const float* means, const float* scales,
                        const float* quats, const float* colors, const void* feats, int32_t N,
                        int32_t feat_dtype, int32_t layout, int32_t flags, const float* bg,
                        const int32_t* tile_ranges, const int32_t* tile_order, const uint32_t* gids,
                        const uint8_t* inst_masks, const float* uv, const float* conic_opacity, const float* depth,
                        const float* T_final, const int32_t* last_idx, const float* dL_drgb, const float* dL_ddepth,
                        const float* dL_dalpha, const float* dL_dfeat, int32_t feat_grad_mode,
                        void* workspace, size_t workspace_bytes, float* d_means, float* d_scales,
                        float* d_quats, float* d_opacity, float* d_colors, float* d_feats,
                        float* d_pose, int32_t* status, void* stream);

/* ---------------------------------------------------------------------------
 * Per-pair saved state (the alternative to the saved T_final and last index
 * that gs_render_bwd recovers the transmittance from, Sec. 3.1): the
 * transmittance in front of every blended (pixel, Gaussian) pair, so that an
 * adjoint reads T_i instead of dividing, T_i = T_{i+1} / (1 - alpha_i), which
 * loses accuracy where alpha nears the 0.99 clamp. The paper has no
 * counterpart; the calls exist to measure the two against each other
 * (memory: 8 bytes per pixel against 4 bytes per blended pair).
 *
 * gs_render_fwd_pairs -- after gs_render_fwd (its last_idx and n_contrib):
 * pair_off [H*W + 1] (int64) = the exclusive scan of n_contrib (pixels row
 * major; pair_off[H*W] = the number of blended pairs), and pair_T[k] for k in
 * [pair_off[q], pair_off[q + 1]) = T in front of pixel q's blended Gaussians
 * in list order, bit for bit the forward's values. More pairs than capacity
 * flags GS_ERR_CAPACITY (pair_T holds the first capacity). workspace: at least
 * gs_pair_state_workspace_bytes(width, height) bytes, 256-byte aligned.
 * gs_render_bwd_pairs -- gs_render_bwd (same arguments without inst_masks,
 * no GS_FEAT_TENSOR_CORE) on the SIMT adjoint in 32-channel chunks, the
 * transmittance read from pair_T (pair_off/pair_T of gs_render_fwd_pairs for
 * the same frame) or, with pair_T NULL, recovered by division as in
 * gs_render_bwd.
 */
size_t gs_pair_state_workspace_bytes(int32_t width, int32_t height);
gs_status gs_render_fwd_pairs(const gs_camera* cam, int32_t P, const int32_t* tile_ranges, const int32_t* tile_order,
                              const uint32_t* gids, const float* uv, const float* conic_opacity,
                              const int32_t* last_idx, const int32_t* n_contrib, void* workspace,
                              size_t workspace_bytes, int64_t capacity, int64_t* pair_off, float* pair_T,
                              int32_t* status, void* stream);
gs_status gs_render_bwd_pairs(const gs_camera* cam, int32_t P, const float* means, const float* scales,
                              const float* quats, const float* colors, const void* feats, int32_t N,
                              int32_t feat_dtype, int32_t layout, int32_t flags, const float* bg,
                              const int32_t* tile_ranges, const int32_t* tile_order, const uint32_t* gids,
                              const float* uv, const float* conic_opacity, const float* depth, const float* T_final,
                              const int32_t* last_idx, const float* dL_drgb, const float* dL_ddepth,
                              const float* dL_dalpha, const float* dL_dfeat, int32_t feat_grad_mode,
                              const int64_t* pair_off, const float* pair_T, void* workspace,
                              size_t workspace_bytes, float* d_means, float* d_scales, float* d_quats,
                              float* d_opacity, float* d_colors, float* d_feats, float* d_pose, int32_t* status,
                              void* stream);

/* ---------------------------------------------------------------------------
 * L1 image loss fused into compositing: the colour and depth L1 terms of the
 * mapping loss (Sec. 3.2) and the feature L1 term (Eq. 11 on the rendered
 * field),
 *   L = w_rgb sum |rgb - rgb*| + w_depth sum |D - D*| + w_feat sum |F - F*|
 * (sums over pixels and channels), with dL/dpred = w sign(pred - target),
 * sign(0) = 0 -- the values gs_l1_loss_grad writes, never stored as floats.
 *
 * gs_render_fwd_l1 -- gs_render_fwd (same arguments and outputs) that also
 * adds L to *loss (device float, atomic; the caller zeroes it; may be NULL)
 * and writes l1_signs [H*W][2] (uint32): for each pixel, word 0 has bit c set
 * where the cotangent of channel c is nonzero and word 1 where it is
 * negative; bits 0..15 are features 0..15, bits 16, 17, 18 red, green, blue
 * and bit 19 depth. A NULL target drops its term (its bits stay 0).
 * gs_render_bwd_l1 -- gs_render_bwd (same arguments and outputs, no
 * cotangent images, no alpha cotangent) whose cotangents are w sign(...)
 * rebuilt from the l1_signs of the forward it differentiates and the weights
 * of l1 (its targets and loss are not used).
 * Both: features with N <= 16 on the fp32 path and decoupled feature
 * gradients; other configurations return GS_ERR_UNSUPPORTED (use
 * gs_l1_loss_grad with gs_render_fwd / gs_render_bwd there).
 */
typedef struct {
  const float* target_rgb;    /* [3,H,W] */
  const float* target_depth;  /* [H,W] */
  const float* target_feat;   /* layout of out_feat */
  float w_rgb, w_depth, w_feat;
  float* loss;
} gs_l1_terms;

gs_status gs_render_fwd_l1(const gs_camera* cam, int32_t P, const int32_t* tile_ranges,
                           const int32_t* tile_order, const uint32_t* gids, uint8_t* inst_masks,
                           const float* uv, const float* conic_opacity,
                           const float* depth, const float* colors, const void* feats, int32_t N,
                           int32_t feat_dtype, int32_t layout, int32_t flags, const float* bg,
                           float* out_rgb, float* out_depth, float* out_alpha, float* out_feat,
                           float* T_final, int32_t* last_idx, int32_t* n_contrib, uint8_t* visible,
                           const gs_l1_terms* l1, uint32_t* l1_signs, int32_t* status, void* stream);

gs_status gs_render_bwd_l1(const gs_camera* cam, int32_t P, const float* means, const float* scales,
                           const float* quats, const float* colors, const void* feats, int32_t N,
                           int32_t feat_dtype, int32_t layout, int32_t flags, const float* bg,
                           const int32_t* tile_ranges, const int32_t* tile_order, const uint32_t* gids,
                           const uint8_t* inst_masks, const float* uv, const float* conic_opacity,
                           const float* depth,
                           const float* T_final, const int32_t* last_idx, const gs_l1_terms* l1, const uint32_t* l1_signs,
                           void* workspace, size_t workspace_bytes, float* d_means, float* d_scales,
                           float* d_quats, float* d_opacity, float* d_colors, float* d_feats,
                           float* d_pose, int32_t* status, void* stream);

/* ---------------------------------------------------------------------------
 * gs_l1_signs -- the L1 terms of gs_render_fwd_l1 as a separate pass over
 * images that gs_render_fwd rendered: adds L to *l1->loss (the caller zeroes
 * it; may be NULL) and writes l1_signs [H*W][2] exactly as gs_render_fwd_l1
 * writes them for the same images (each image holds the value the fused
 * epilogue compares), for gs_render_bwd_l1. The paper has no counterpart:
 * with targets still being copied from the host, the forward can run
 * before they arrive and only this pass waits for them.
 * rgb [3,H,W], depth [H,W], feat [N,H,W] (CHW) or [H,W,N] (HWC), N <= 16
 * (GS_ERR_UNSUPPORTED above; 0 = no feature term); an image may be NULL when
 * its target is NULL.
 */
gs_status gs_l1_signs(int32_t width, int32_t height, int32_t N, int32_t layout, const float* rgb,
                      const float* depth, const float* feat, const gs_l1_terms* l1, uint32_t* l1_signs,
                      void* stream);

/* ---------------------------------------------------------------------------
 * gs_l1_loss_grad -- the L1 photometric term of the tracking and mapping
 * losses (Eq. 6, Eq. 8): grad[i] = scale * sign(pred[i] - target[i]) (sign(0)
 * = 0) and *loss_sum += scale * sum |pred - target| (device float, atomic).
 */
gs_status gs_l1_loss_grad(int64_t n, const float* pred, const float* target, float scale,
                          float* grad, float* loss_sum, void* stream);

/* ---------------------------------------------------------------------------
 * Camera tracking (Sec. 3.2, Eq. 6): with the Gaussians frozen, the pose is
 * refined on its tangent until the update converges.
 *
 * gs_edge_mask -- m_e, the pixels of the observed image with a significant
 * gradient: L = (r + g + b)/3 per pixel (rgb [3,H,W]); Sobel gx, gy of L with
 * replicated borders, divided by 8 (a unit step gives 0.5); m_e [H,W] (u8) =
 * gx^2 + gy^2 > tau^2. Every step is one binary32 operation in a fixed
 * order: (r + g) + b, then * (1/3); a = (L(x+1,y-1) + 2 L(x+1,y)) +
 * L(x+1,y+1), b likewise at x-1, gx = (a - b) * 0.125; gy alike with rows
 * y+1 and y-1 (summed from x-1 to x+1); (gx gx) + (gy gy) > tau tau.
 */
gs_status gs_edge_mask(int32_t width, int32_t height, const float* rgb, float tau, uint8_t* m_e,
                       void* stream);

/* gs_tracking_loss_grad -- cotangents of Eq. 6 for one render:
 *   m_v = alpha_ref > alpha_min (alpha_ref: the opacity of the frame's first
 *   render, the 2D visibility map); colour term on m_v m_e, depth term on
 *   m_v and gt_depth > 0;
 *   g_rgb [3,H,W] = lambda_t / (3 H W) sign(rgb - gt_rgb) on the colour mask,
 *   g_depth [H,W] = (1 - lambda_t) / (H W) sign(depth - gt_depth) on the depth
 *   mask, 0 elsewhere (sign(0) = 0); *loss_sum (device float, may be NULL)
 *   += the loss, accumulated atomically. Feed g_rgb and g_depth to
 *   gs_render_bwd for the pose gradient.
 */
gs_status gs_tracking_loss_grad(int32_t width, int32_t height, const float* rgb, const float* depth,
                                const float* gt_rgb, const float* gt_depth, const float* alpha_ref,
                                float alpha_min, const uint8_t* m_e, float lambda_t, float* g_rgb,
                                float* g_depth, float* loss_sum, void* stream);

/* gs_tracking_loss_signs -- the same loss and cotangents as
 * gs_tracking_loss_grad, kept as the sign words of gs_render_fwd_l1
 * (l1_signs [H*W][2]: bits 16, 17, 18 colour, 19 depth; a bit of word 0 is
 * set where the cotangent is nonzero, of word 1 where it is negative) with
 * their weights written to weights[0] = lambda_t / (3 H W) (colour) and
 * weights[1] = (1 - lambda_t) / (H W) (depth) (host floats). gs_render_bwd_l1
 * with those weights (features off) then gives the pose gradient of
 * gs_render_bwd on gs_tracking_loss_grad's images. *loss_sum as there.
 */
gs_status gs_tracking_loss_signs(int32_t width, int32_t height, const float* rgb, const float* depth,
                                 const float* gt_rgb, const float* gt_depth, const float* alpha_ref, float alpha_min,
                                 const uint8_t* m_e, float lambda_t, uint32_t* l1_signs, float* weights,
                                 float* loss_sum, void* stream);


/* gs_pose_update -- one optimiser step of the pose (device arrays):
 *   Adam on d_pose [6] (tangent (rho, theta) of the left perturbation, from
 *   gs_render_bwd) with moments adam_m [6], adam_v [6] (zero at the frame's
 *   first step), bias-corrected at `step` (1-based), step sizes lr_trans for
 *   rho and lr_rot for theta: delta = -lr m_hat / (sqrt(v_hat) + eps);
 *   pose_dev [12] (R row-major, t) <- Exp(delta) pose, with
 *   Exp(rho, theta) = [R(theta), V(theta) rho], R(theta) = I + A K + B K^2,
 *   V(theta) = I + B K + C K^2, K = [theta]x, phi = |theta|,
 *   A = sin(phi)/phi, B = (1 - cos phi)/phi^2, C = (phi - sin phi)/phi^3
 *   (series below phi = 1e-4);
 *   *converged (device int32, may be NULL) = |V rho| < tol_trans and
 *   phi < tol_rot.
 * Use pose_dev as gs_camera.pose_dev so the next render reads it.
 */
gs_status gs_pose_update(float* pose_dev, const float* d_pose, float* adam_m, float* adam_v, int32_t step,
                         float lr_trans, float lr_rot, float beta1, float beta2, float eps,
                         float tol_trans, float tol_rot, int32_t* converged, void* stream);

/* ---------------------------------------------------------------------------
 * View-dependent colour from spherical harmonics (Sec. 3.1: third-order SH
 * coefficients per Gaussian).
 *
 * gs_sh_colors -- colors [P,3] = max(0, sum_k sh[g][k][c] Y_k(d) + 0.5) per
 * Gaussian and channel, with d the unit direction from the camera centre
 * C = -R^T t (the pose of cam, or cam->pose_dev) to means[g]; sh [P, K, 3]
 * (coefficient-major, K = (degree + 1)^2, degree 0..3); k = l^2 + l + m;
 * Y_k the real SH basis with the Condon-Shortley phase. The result is the
 * colors input of gs_render_fwd / gs_render_bwd.
 */
gs_status gs_sh_colors(const gs_camera* cam, int32_t P, int32_t degree, const float* means, const float* sh,
                       float* colors, void* stream);

/* gs_sh_colors_bwd -- adjoint of gs_sh_colors for d_colors [P,3] (the d_colors
 * of gs_render_bwd); ACCUMULATES d_sh [P, K, 3], d_means [P,3] (through the
 * view direction) and d_pose [6] (the camera centre moves with rho only at
 * first order: d rho += R sum_g dL/dmu_g|_view); each output may be NULL.
 * Clamped channels pass no gradient.
 */
gs_status gs_sh_colors_bwd(const gs_camera* cam, int32_t P, int32_t degree, const float* means,
                           const float* sh, const float* d_colors, float* d_sh, float* d_means,
                           float* d_pose, void* stream);

/* ---------------------------------------------------------------------------
 * Semantic supervision and read-out of the feature field (Sec. 3.3).
 *
 * gs_semantic_ce_grad -- the ground-truth loss of Eq. 9 on the rendered map
 * feat (N channels, layout CHW [N,H,W] or HWC [H,W,N]) read as per-pixel
 * logits normalised by a softmax over the channels:
 *   loss_sum += (1/HW) sum_p [logsumexp_c F_p(c) - F_p(l_p)],
 *   grad (same layout, may be NULL) = (softmax(F_p) - onehot(l_p)) / HW,
 * labels [H,W] int32; a label outside [0, N) marks an ignored pixel (no loss,
 * zero gradient). grad is the feature cotangent for gs_render_bwd.
 */
gs_status gs_semantic_ce_grad(int32_t width, int32_t height, int32_t N, int32_t layout, const float* feat,
                              const int32_t* labels, float* grad, float* loss_sum, void* stream);

/* gs_argmax_labels -- predicted labels argmax_c F_p(c) (Eq. 10; ties take the
 * lowest channel) of feat (layout as above) into labels [H,W] int32.
 */
gs_status gs_argmax_labels(int32_t width, int32_t height, int32_t N, int32_t layout, const float* feat,
                           int32_t* labels, void* stream);

/* gs_label_probs -- label probabilities of Eq. 12 for npix pixel features
 * feat [npix, M] (fp32 rows, 16-byte aligned; M % 4 == 0) against L query
 * vectors queries [L, M] (1 <= L <= 64, L M <= 51200):
 *   probs [npix, L] (may be NULL) = softmax_l(f . q(l)),
 *   labels [npix] int32 (may be NULL) = argmax_l f . q(l) (ties: lowest l).
 * At least one output must be given.
 */
gs_status gs_label_probs(int64_t npix, int32_t M, int32_t L, const float* feat, const float* queries,
                         float* probs, int32_t* labels, void* stream);

/* ---------------------------------------------------------------------------
 * Per-pixel feature decoder o(.) of Eq. 11, read as a 1x1 lift of a rendered
 * latent map (a din-channel render of per-Gaussian latents):
 *     y = W2^T gelu(W1^T z + b1) + b2,   gelu(x) = x (1 + erf(x / sqrt 2)) / 2.
 * W1 [din, dh] and W2 [dh, dout] are row-major fp32 arrays whose values are
 * bf16-representable (the bf16 weights; gs_adam_step can write that
 * rounding), b1 [dh], b2 [dout] fp32; accumulation is fp32.
 * Limits: din <= 64, dh <= 1024, dout <= 4096; fewer than 2^31 pixels.
 */
typedef struct gs_decoder {
  int32_t din, dh, dout;
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
} gs_decoder;

/* Workspace for gs_decoder_fwd over n pixels (training = 0) or for
 * gs_decoder_train with n samples (training = 1). */
size_t gs_decoder_workspace_bytes(const gs_decoder* dec, int64_t n, int32_t training);

/* z [npix, din] -> y [npix, dout]. */
gs_status gs_decoder_fwd(const gs_decoder* dec, int64_t npix, const float* z, float* y, void* workspace,
                         size_t workspace_bytes, void* stream);

/* One training evaluation on nsample pixels drawn with replacement from the
 * npix pixels of z_map [npix, din] / target [npix, dout]: sample s is pixel
 * splitmix64(seed + (s + 1) * 0x9E3779B97F4A7C15) mod npix. Loss
 * L = loss_scale * sum_s sum_c (y - target)^2 is added to *loss_sum (device,
 * may be NULL); its gradients are ACCUMULATED into dW1, db1, dW2, db2 and,
 * at the sampled pixels, into dz_map [npix, din] (may be NULL). */
gs_status gs_decoder_train(const gs_decoder* dec, int64_t nsample, int64_t npix, uint64_t seed,
                           const float* z_map, const float* target, float loss_scale, void* workspace,
                           size_t workspace_bytes, float* dW1, float* db1, float* dW2, float* db2,
                           float* dz_map, float* loss_sum, void* stream);

/* The same training evaluation on tcgen05 tensor cores, for din = 16,
 * dh = 128, dout = 512 (GS_ERR_UNSUPPORTED otherwise), in two fused kernels:
 * the first takes each 128-sample tile through W1, the GELU, W2, the loss
 * and its cotangent dY, then back through W2 and the GELU to dPRE, dz and
 * dW1 / db1 (db1 and db2 from the fp32 values); the second forms dW2 from the
 * tiles' H and dY, which the first leaves in the workspace. z, H, dY and
 * dPRE enter the products rounded to bf16 (unit roundoff u = 2^-8), every
 * sum is fp32: to first order each gradient's error is bounded by u times
 * the sum of |terms| of every rounded operand it passes through (the
 * tensor-core training test states the bound per gradient). The GELU and
 * its derivative take erf from Abramowitz & Stegun 7.1.26 (absolute error
 * at most 1.5e-7, far below u). Same sampling
 * rule, loss and accumulation as gs_decoder_train; z_map, dz_map, dW1, db1
 * and dW2 16-byte aligned (vector atomics), workspace 256-byte aligned with
 * gs_decoder_train_tc_workspace_bytes(nsample) bytes (1.25 KB per sample).
 * Device errors (a bounded wait that gave up) are OR-ed into *status (may be
 * NULL). */
size_t gs_decoder_train_tc_workspace_bytes(int64_t nsample);
gs_status gs_decoder_train_tc(const gs_decoder* dec, int64_t nsample, int64_t npix, uint64_t seed,
                              const float* z_map, const float* target, float loss_scale, void* workspace,
                              size_t workspace_bytes, float* dW1, float* db1, float* dW2, float* db2,
                              float* dz_map, float* loss_sum, int32_t* status, void* stream);

/* The decoder forward on tcgen05 tensor cores for din = 16, dh = 128,
 * dout = 512: z and W rounded to bf16, fp32 accumulation, the hidden layer
 * rounded to bf16 after the exact GELU; y = D + b2 in fp32. No workspace.
 * Device errors (a bounded wait that gave up) are OR-ed into *status
 * (may be NULL). */
gs_status gs_decoder_fwd_tc(const gs_decoder* dec, int64_t npix, const float* z, float* y, int32_t* status,
                            void* stream);

/* Label read-out of the decoded field without forming it (Eq. 11 composed
 * with Eq. 12): since y = W2^T h + b2, the logit of query l is
 * y . q(l) = h . G(:, l) + c(l) with G = W2 q^T and c = b2 . q^T, so per
 * pixel the 16-d latent z [npix, 16] goes through W1, the GELU (rounded to
 * bf16) and one tcgen05 product with G (folded in fp32, rounded to bf16);
 * probs [npix, L] (may be NULL) = softmax_l, labels [npix] (may be NULL) =
 * argmax_l (ties: lowest l). queries [L, 512], 1 <= L <= 64; din = 16,
 * dh = 128, dout = 512. Device errors are OR-ed into *status (may be NULL).
 */
gs_status gs_decoder_labels_tc(const gs_decoder* dec, int64_t npix, const float* z, int32_t L,
                               const float* queries, float* probs, int32_t* labels, int32_t* status,
                               void* stream);

/* Adam (Kingma and Ba 2015) with bias correction on n parameters at step
 * `step` (>= 1); param_bf16 (may be NULL) receives the updated parameters
 * rounded to bf16 (stored as fp32), the copy the decoder multiplies with. */
gs_status gs_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr,
                       float beta1, float beta2, float eps, int32_t step, float* param_bf16, void* stream);

/* ---------------------------------------------------------------------------
 * Tracing: when enabled, every kernel the library launches is bracketed by
 * CUDA events on its stream (up to `capacity` launches, then recording stops).
 * gs_trace_get synchronizes on the i-th end event and returns the kernel's
 * name (static storage) and its duration in milliseconds.
 */
gs_status gs_trace_enable(int32_t capacity); /* 0 disables and frees the events */
void gs_trace_reset(void);
int32_t gs_trace_count(void);
gs_status gs_trace_get(int32_t i, const char** name, float* ms);

/* ---------------------------------------------------------------------------
 * gs_peak_probe -- throughput probes for the arithmetic rooflines (the paper
 * has no counterpart): one launch of `blocks` x `threads` threads (threads a
 * multiple of 32, <= 1024), each running 8 independent dependency chains of
 * `iters` operations of one kind:
 *   0: fp32 fused multiply-add (2 flop each);
 *   1: packed two-lane fp32 fused multiply-add (4 flop each);
 *   2: ex2.approx.ftz.f32 (1 op each);
 *   3: mma.sync m16n8k16 bf16 x bf16 -> fp32 per warp (4096 flop each).
 * *ops (host double) receives the operations the launch performs; sink
 * (device, >= blocks floats) is written only to keep the work alive. The
 * caller times the launch on its stream.
 */
gs_status gs_peak_probe(int32_t kind, int32_t blocks, int32_t threads, int32_t iters, float* sink, double* ops,
                        void* stream);

/* ---------------------------------------------------------------------------
 * gs_test_hold_tc_producer -- test hook of the bounded waits (failure
 * detection; the paper has no counterpart). While `on` is nonzero, the
 * tensor-core feature kernels (gs_render_fwd and gs_render_bwd with
 * GS_FEAT_TENSOR_CORE) run with their producer warps idle: no stage of
 * records is ever filled, so the other roles' mbarrier waits run out after
 * their bound (1 s of %globaltimer). The launch then ORs 1 << GS_ERR_TIMEOUT
 * into the status word, waits for the copies it issued, frees its tensor
 * memory and returns; the feature map (forward) or the feature gradient
 * (adjoint) is unspecified, everything else the call writes is as usual. No
 * product is issued before the waits give up, so the context stays usable.
 * Process-wide, read at each launch; not for use while other threads render.
 * Returns GS_OK.
 */
gs_status gs_test_hold_tc_producer(int32_t on);

const char* gs_status_string(gs_status s);
int32_t gs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GSFF_H */
