/*
 * gs_topk.h -- C ABI of the Top-K feature renderer (B300, sm_103a).
 *
 * The library renders colour, depth and a D-dimensional language feature per pixel
 * from 3D Gaussians, and back-propagates a loss to the Gaussians:
 *   colour / depth  C(p) = sum_i c_i w_i,  D(p) = sum_i z_i w_i           (Sec. 3.1, Eq. 1)
 *   weights         w_i = alpha_i prod_{j<i} (1 - alpha_j), front to back  (Eq. 1; Sec. 3.3 text of Eq. 8)
 *   Top-K set       the K contributors of largest w                        (Sec. 3.2, Eq. 2)
 *   renormalised    w'_k = w_k / sum_{j in K} w_j                          (Eq. 3)
 *   feature         F(p) = sum_{k in K} w'_k f_k                           (Eq. 4)
 * Colour and depth keep the full alpha blend; only the feature uses Top-K (Sec. 3.2).
 * The projection and the per-pixel constants follow 3D Gaussian Splatting, which
 * Sec. 3.1 defers to: EWA covariance with a 0.3 px^2 dilation, alpha = min(0.99,
 * o exp(-q/2)); a Gaussian takes part at a pixel iff q <= 9, alpha >= 1/255 and the
 * transmittance would stay >= 1e-4.  Pixel (i, j) is sampled at (i + 0.5, j + 0.5).
 *
 * Conventions for every call
 *   - All array pointers are DEVICE memory owned by the caller (camera and config
 *     structs are host memory, read during the call).  The library never allocates
 *     device memory: scratch lives in the caller's workspace `ws` of at least
 *     gs_workspace_size() bytes, 256-byte aligned.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream); none synchronises except gs_sync_status().
 *   - Return value: GS_OK or an error code below.  Argument errors are detected on
 *     the host before anything is launched.  Data-dependent failures (instance
 *     overflow) are recorded in a device error word inside `ws`; kernels of later
 *     calls on the same workspace skip their work once it is set, and
 *     gs_sync_status() reads it back.
 *   - Layouts: row-major; Gaussians are indexed 0..N-1; the pixels of camera c occupy
 *     the flat range [pix_off(c), pix_off(c) + W_c H_c) of every per-pixel array,
 *     pix_off(c) being the sum of W H over cameras 0..c-1; within a camera pixel
 *     (x, y) is x + W y.  Feature rows (N x D) start 16-byte aligned, D is a multiple
 *     of 8.
 *   - One render = gs_preprocess, gs_bin_sort, gs_topk_select, gs_feature_blend in
 *     this order on one workspace, which must stay untouched until gs_backward of
 *     that render has run.
 */
#ifndef GS_TOPK_H
#define GS_TOPK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_MAX_CAMERAS 16
#define GS_MAX_K 32
#define GS_PROJ_FLOATS 16      /* floats per (camera, Gaussian) projected record */

enum gs_status_code {
    GS_OK = 0,
    GS_ERR_ARG = 1,            /* bad argument (null pointer, size, unsupported shape) */
    GS_ERR_WORKSPACE = 2,      /* workspace smaller than gs_workspace_size() or misaligned */
    GS_ERR_CUDA = 3,           /* a CUDA launch or runtime call failed */
    GS_ERR_TIMEOUT = 4,        /* a bounded device-side wait ran out */
    GS_ERR_OVERFLOW = 5,       /* more (Gaussian, tile) instances than the configured capacity */
    GS_ERR_UNSUPPORTED = 6     /* configuration not compiled into this library */
};

enum gs_dtype { GS_F32 = 0, GS_BF16 = 1 };

/* Pinhole camera.  viewmat: row-major 4x4 world->camera transform (camera looks
 * along +z, x right, y down).  u = fx x/z + cx, v = fy y/z + cy. */
typedef struct {
    float viewmat[16];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_z;              /* Gaussians with camera depth <= near_z are culled */
} gs_camera;

/* Render configuration. */
typedef struct {
    int32_t K;                 /* Top-K size, 1..GS_MAX_K */
    int32_t D;                 /* feature width, multiple of 8, 8..1024 */
    int32_t tile_w, tile_h;    /* screen tile: 16x16, 32x8, 16x8 or 8x8 */
    int32_t feat_dtype;        /* GS_F32 or GS_BF16: feature rows, F and dL/dF */
    int32_t max_instances;     /* capacity of (Gaussian, tile) instances; 0: 32 per (camera, Gaussian) */
    int32_t max_feature_rows;  /* capacity of gs_backward's partial feature-gradient rows, one per (pixel
                                  block, selected Gaussian); 0: 32 per block, or max_instances per
                                  (camera, Gaussian) when that is larger */
    int32_t topk_layout;       /* how gs_topk_select keeps each pixel's K-buffer while it walks: 0 in
                                  registers, 1 in shared memory (K <= 16; fewer registers per thread),
                                  2 in shared memory with warp-level insertion (K <= 16: the warp
                                  inserts each new member, one lane per slot).  The outputs are
                                  identical; a performance choice for an autotuner */
    int32_t depth_cut;         /* 1: the per-tile depth cut (see gs_bin_sort) carried from one render to
                                  the next on the same workspace; 0: every instance sorted.  Every
                                  output of a render is bit-identical either way */
} gs_config;

/* Per-Gaussian gradient outputs of gs_backward (device, caller-allocated, fully
 * overwritten).  feat is N x D float32 whatever the feature dtype.  mean2d and conic
 * are per camera: n_cams x N x 2 and n_cams x N x 3, conic as (a, b, c) with
 * q = a dx^2 + 2 b dx dy + c dy^2 and d = pixel - mean2d; they may be NULL. */
typedef struct {
    float *feat;               /* N x D  */
    float *opacity;            /* N      */
    float *rgb;                /* N x 3  */
    float *mean3d;             /* N x 3  */
    float *cov3d;              /* N x 6 (xx, xy, xz, yy, yz, zz); an off-diagonal entry stands for both symmetric entries */
    float *mean2d;             /* n_cams x N x 2, or NULL */
    float *conic;              /* n_cams x N x 3, or NULL */
    float *viewmat;            /* n_cams x 12, or NULL: the gradient with respect to each camera's world-to-camera
                                  [R | t] (row-major 3 x 4; through p = R mu + t and the EWA Jacobian term J R),
                                  summed over the Gaussians in a fixed order -- for rendering-loss pose refinement */
} gs_grads;

/* Human-readable name of a status code (static string). */
const char *gs_status_string(int status);

/* Library version and the compute capability it was built for (e.g. 103). */
int gs_version(int *major, int *minor, int *built_sm);

/* Workspace bytes needed by one render (forward and backward) of n_gauss Gaussians
 * seen by n_cams cameras under cfg.  Returns 0 on a bad argument. */
size_t gs_workspace_size(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss);

/* Total pixel count of the cameras (the P of every per-pixel array); -1 on a bad argument. */
int64_t gs_pixel_count(const gs_camera *cams, int32_t n_cams);

/* a1. EWA projection (Sec. 3.1, after 3DGS).  Inputs: mean3d N x 3, cov3d N x 6
 * (xx, xy, xz, yy, yz, zz), opacity N, rgb N x 3, all float32.  Output proj:
 * n_cams x N records of GS_PROJ_FLOATS floats (16-byte aligned); a culled Gaussian
 * (depth <= near_z, or opacity too low to ever reach alpha >= 1/255) gets a record
 * with zero extent.  Also clears the workspace error word. */
int gs_preprocess(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                  const float *mean3d, const float *cov3d, const float *opacity, const float *rgb,
                  float *proj, void *ws, size_t ws_bytes, void *stream);

/* a2. Tile binning: every (camera, Gaussian) is duplicated into each screen tile its
 * ellipse reaches (alpha >= 1/255 at some pixel centre of the tile is possible), and the
 * instances are ordered by (tile, depth) with the library's own device radix sort;
 * per-tile instance ranges stay in ws.  Instance overflow sets GS_ERR_OVERFLOW in the
 * error word.
 * Depth cut (cfg->depth_cut = 1): a tile's walk stops where its last pixel saturates,
 * usually far in front of the tile's deepest instance.  Each render records, per tile,
 * the depth where that happened (with a 6% margin, or none if the tile did not
 * saturate), and the next render on the same workspace sorts only the instances in
 * front of their tile's recorded depth.  gs_topk_select then completes, within the
 * same render, every tile that this shorter list leaves unsaturated: it sorts that
 * tile's remaining instances and walks the tile again over the whole list.  So every
 * walk sees exactly the full list up to where it stops, and the outputs are identical
 * to depth_cut = 0; only the amount of sorting changes.  A render uses the cuts an
 * earlier render on the workspace recorded for the same tile grid (a signature in the
 * header says which); a workspace whose first 256 bytes are zero, or one whose tile grid
 * changed, starts without cuts.  The lists are complete for every later call once
 * gs_topk_select has run. */
int gs_bin_sort(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                const float *proj, void *ws, size_t ws_bytes, void *stream);

/* a3. Front-to-back walk of each pixel's tile list (Eq. 1) keeping the pixel's
 * Top-K contributors (Eq. 2).  Outputs (P = gs_pixel_count): rgb_out P x 3, depth_out
 * P, T_final P (transmittance after the walk), n_contrib P (contributor count),
 * topk_idx P x K (Gaussian ids by descending w, -1 padded), topk_w P x K (the raw
 * weights w, 0 padded). */
int gs_topk_select(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                   const float *proj, void *ws, size_t ws_bytes,
                   float *rgb_out, float *depth_out, float *T_final, int32_t *n_contrib,
                   int32_t *topk_idx, float *topk_w, void *stream);

/* a4. Gather-blend (Eqs. 3-4): F[p] = sum_k (w_k / S_p) feats[idx_k], S_p = sum_k w_k,
 * F[p] = 0 where S_p = 0.  feats: N x D rows of cfg->feat_dtype; F_out: n_pix x D of
 * cfg->feat_dtype (accumulation is float32 either way).  Needs no workspace. */
int gs_feature_blend(const gs_config *cfg, int64_t n_pix, int32_t n_gauss, const int32_t *topk_idx,
                     const float *topk_w, const void *feats, void *F_out, void *stream);

/* a5. Adjoint of a1-a4.  Takes the forward inputs and outputs and the upstream
 * gradients dL_dF (P x D, cfg->feat_dtype), dL_dC (P x 3), dL_dD (P), and writes
 * every gradient in `grads`.  dL_dF == NULL is the geometry-only adjoint of the hybrid
 * schedule (Sec. 3.4): no feature loss, so no feature gradient (feats and grads->feat
 * are not used and may be NULL) and no feature term in dL/dw.  The walk is recomputed, not stored; feature gradients
 * are reduced per Gaussian after a sort of the Top-K (pixel, slot) pairs by
 * Gaussian, and geometry gradients per (Gaussian, tile) instance, without atomics,
 * so the results are deterministic.  Streams: the feature-gradient reduction runs on
 * a library-owned auxiliary stream of the current device (created by the first call
 * made outside a stream capture, kept until exit), forked after the work queued on
 * `stream` and joined back to `stream` before the call returns, so all outputs are
 * ordered on `stream` as if everything ran there; a call made while `stream` is being
 * captured uses the auxiliary stream only if it already exists (the fork and join are
 * then captured), otherwise everything runs on `stream`. */
int gs_backward(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                const float *mean3d, const float *cov3d, const float *opacity, const float *rgb,
                const void *feats, const float *proj,
                const float *rgb_out, const float *depth_out, const int32_t *topk_idx, const float *topk_w,
                const void *dL_dF, const float *dL_dC, const float *dL_dD,
                const gs_grads *grads, void *ws, size_t ws_bytes, void *stream);

/* gs_backward with options.  flags: 0, or GS_BWD_H_FROM_LOSS -- dL_dF is the gradient
 * that the last gs_feature_blend_loss call on this workspace wrote, unmodified since:
 * that call also left the per-slot terms h = dL/dF . f_idx of the re-walk in ws
 * (computed from rows it had just read), and they are reused instead of being
 * recomputed from dL_dF.  Passing the flag for any other dL_dF gives wrong gradients.
 * Unknown flag bits: GS_ERR_ARG. */
#define GS_BWD_H_FROM_LOSS 1u
int gs_backward_ex(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                   const float *mean3d, const float *cov3d, const float *opacity, const float *rgb,
                   const void *feats, const float *proj,
                   const float *rgb_out, const float *depth_out, const int32_t *topk_idx, const float *topk_w,
                   const void *dL_dF, const float *dL_dC, const float *dL_dD,
                   const gs_grads *grads, uint32_t flags, void *ws, size_t ws_bytes, void *stream);

/* Training loss of the benchmark workloads (Eqs. 5-7 leave the weights and the
 * feature distance open; this one takes 1 - cosine for the feature, as the workload
 * specifies): L = w_feat mean_p(1 - cos(F_p, Fgt_p)) + w_rgb mean_p |C_p - Cgt_p|_1 / 3
 * + w_depth mean_p |D_p - Dgt_p|; a pixel with |F_p| = 0 or |Fgt_p| = 0 contributes
 * w_feat to the cosine term and no gradient.  Writes dL_dF (P x D, cfg->feat_dtype),
 * dL_dC, dL_dD and the scalar loss (device float, summed in a fixed order).
 * `scratch` is caller device memory of gs_loss_scratch_size(n_pix) bytes. */
size_t gs_loss_scratch_size(int64_t n_pix);
int gs_loss_cos_l1(const gs_config *cfg, int64_t n_pix, const void *F, const void *F_gt,
                   const float *rgb, const float *rgb_gt, const float *depth, const float *depth_gt,
                   float w_feat, float w_rgb, float w_depth,
                   void *dL_dF, float *dL_dC, float *dL_dD, float *loss,
                   void *scratch, size_t scratch_bytes, void *stream);

/* Training form of a4 + loss in one pass (same results as gs_feature_blend followed
 * by gs_loss_cos_l1 on the same inputs, without reading F back): pixels are processed
 * in screen-tile order, so needs the cameras and the workspace of the render (it reads
 * the error word).  Outputs F_out (P x D) and the loss gradients as gs_loss_cos_l1;
 * scratch of gs_loss_scratch_size(P) bytes.  It also writes into ws the re-walk's
 * per-slot terms h = dL/dF . f for the dL_dF it outputs, which gs_backward_ex with
 * GS_BWD_H_FROM_LOSS reuses. */
int gs_feature_blend_loss(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                          const int32_t *topk_idx, const float *topk_w, const void *feats, const void *F_gt,
                          const float *rgb, const float *rgb_gt, const float *depth, const float *depth_gt,
                          float w_feat, float w_rgb, float w_depth, void *F_out, void *dL_dF, float *dL_dC,
                          float *dL_dD, float *loss, void *ws, size_t ws_bytes, void *scratch, size_t scratch_bytes,
                          void *stream);

/* Same loss as gs_loss_cos_l1, for callers that cannot allocate device memory (code in
 * a real-time loop where cudaMalloc may stall the device, a plug-in inside a host
 * framework that owns all device memory, a component handed only its buffers).  The
 * paper has no counterpart; this is a property of the library.  No scratch argument:
 * the per-pixel partial sums live in a fixed array the library holds on every GPU that
 * loads it (GS_LOSS_NOALLOC_MAX_PIX + 360 floats, about 16.8 MB, kept until exit).
 * n_pix > GS_LOSS_NOALLOC_MAX_PIX returns GS_ERR_WORKSPACE without launching; other
 * arguments follow gs_loss_cos_l1's rules.  The first call on a device looks up the
 * array's device address for that device; make it before any stream capture.  Later
 * calls outside a capture look the address up again (it belongs to the device's current
 * context, e.g. it changes after cudaDeviceReset); a call on a capturing stream reuses
 * the last one found.  All calls share the array: calls whose kernels overlap on the
 * GPU race.  Allocates nothing. */
#define GS_LOSS_NOALLOC_MAX_PIX (1 << 22)
int gs_loss_cos_l1_noalloc(const gs_config *cfg, int64_t n_pix, const void *F, const void *F_gt,
                           const float *rgb, const float *rgb_gt, const float *depth, const float *depth_gt,
                           float w_feat, float w_rgb, float w_depth,
                           void *dL_dF, float *dL_dC, float *dL_dD, float *loss, void *stream);

/* Geometric reconstruction loss of the hybrid schedule's geometry-only iterations
 * (Sec. 3.4, Eq. 6 read as in gs_loss_cos_l1 without the feature term): mean over pixels
 * of w_rgb |C - C_gt|_1 / 3 + w_depth |D - D_gt|, with its gradients dL_dC (P x 3) and
 * dL_dD (P); loss (1 float, device) summed in a fixed order.  Scratch as gs_loss_cos_l1. */
int gs_loss_geo_l1(int64_t n_pix, const float *rgb, const float *rgb_gt, const float *depth, const float *depth_gt,
                   float w_rgb, float w_depth, float *dL_dC, float *dL_dD, float *loss, void *scratch,
                   size_t scratch_bytes, void *stream);

/* One Adam step over up to GS_ADAM_MAX_TENSORS float32 parameter tensors in a single
 * launch (the optimiser of the mapping iterations; the paper leaves it to 3DGS):
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps),
 * element-wise; param, exp_avg (m) and exp_avg_sq (v) are updated in place, step >= 1.
 * param_bf16 (optional, may be NULL): n bf16 values that receive the updated param
 * rounded to nearest -- the BF16 copy a renderer with GS_BF16 feature rows reads, kept
 * beside float32 master weights; 8-byte aligned. */
#define GS_ADAM_MAX_TENSORS 16
typedef struct {
    float *param;
    const float *grad;
    float *exp_avg;
    float *exp_avg_sq;
    int64_t n;
    float lr;
    void *param_bf16;
} gs_adam_tensor;
int gs_adam_step(const gs_adam_tensor *tensors, int32_t n_tensors, int32_t step, float beta1, float beta2, float eps,
                 void *stream);

/* The full alpha-blending feature baseline (Sec. 3.2, Tab. 4 "vanilla"; Feature3DGS's
 * way of rendering features): F_out[p] = sum over every contributor i of w_i f_i -- Eq. 1
 * applied to the feature rows, with the walk's own contributor rule, no Top-K and no
 * renormalisation.  F_out: P x D of cfg->feat_dtype (float32 accumulation).  Call after
 * gs_topk_select on the same workspace (it walks the binned tile lists, which that call
 * completes; with cfg->depth_cut = 0, gs_bin_sort is enough). */
int gs_feature_blend_vanilla(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                             const float *proj, const void *feats, void *F_out, void *ws, size_t ws_bytes,
                             void *stream);

/* Consistency-pruning statistics of one rendered view (Sec. 3.3), accumulated into
 * caller-owned per-Gaussian arrays that the caller zeroes at the start of a pruning
 * window and passes for every view of it:
 *   topk_count[g] += the number of pixels whose Top-K set (Eq. 2) holds g (int32, N);
 *   S[g] = max(S[g], w) over every pixel where g contributes, w the alpha-blending
 *          weight of Eq. 1 -- the geometric importance of Eq. 8 (float32, N, >= 0).
 * Call after gs_topk_select on the same workspace (it re-walks the binned tile lists)
 * with that call's topk_idx.  Exact: integer counts, and the maximum of float32
 * weights taken with the walk's own contributor rule. */
int gs_prune_stats(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss, const float *proj,
                   const int32_t *topk_idx, void *ws, size_t ws_bytes, int32_t *topk_count, float *S, void *stream);

/* Survival selection of Sec. 3.3 (Eq. 9).  Candidates G_prune: Gaussians with
 * topk_count < tau.  m = floor(ratio |G_prune| + 1/2) candidates survive, drawn by
 * weighted sampling without replacement with probability S_i / sum S over the remaining
 * candidates, realised as an exponential race: candidate i finishes at expo[i] / S[i]
 * (float32 division), expo[i] ~ Exp(1) supplied by the caller (the random numbers of
 * the method are inputs); S = 0 never finishes; equal times go to the smaller id.
 * keep[g] (uint8, N) = 1 for survivors and every non-candidate, 0 for the pruned.
 * Device workspace of gs_prune_select_workspace_size(n_gauss) bytes, 256-aligned. */
size_t gs_prune_select_workspace_size(int32_t n_gauss);
int gs_prune_select(int32_t n_gauss, const int32_t *topk_count, const float *S, int32_t tau, double ratio,
                    const float *expo, uint8_t *keep, void *ws, size_t ws_bytes, void *stream);

/* Bound, in SM clock cycles, of the device-side waits of the current render on this
 * workspace (the mbarrier waits of the feature-gradient pipeline in gs_backward): each
 * wait gives up once more than `cycles` cycles have passed, records GS_ERR_TIMEOUT in the
 * error word, and its kernel finishes early (after waiting, with the default bound, for
 * the copies it has in flight), so later kernels on the workspace skip their work and
 * gs_sync_status reports the timeout.  cycles <= 0 selects the default, 2e9 cycles
 * (about 1 s); gs_preprocess resets it to the default at the start of every render.
 * Queued on `stream` like the other calls.  For failure-detection tests: a limit of a
 * few cycles makes the first wait run out. */
int gs_set_wait_limit(void *ws, size_t ws_bytes, int64_t cycles, void *stream);

/* Synchronises `stream` and reads two counts of the last render on the workspace: the
 * (Gaussian, tile) instances that gs_bin_sort produced and the partial feature-gradient
 * rows that gs_backward needed -- whether or not they fitted the capacities, so a caller
 * can size max_instances and max_feature_rows after a GS_ERR_OVERFLOW.  Either pointer
 * may be NULL. */
int gs_workspace_counts(const void *ws, size_t ws_bytes, void *stream, int64_t *n_instances,
                        int64_t *n_feature_rows);

/* Synchronises `stream` and returns the workspace error word as a status (GS_OK if
 * clear).  If n_instances is not NULL it receives the instance count of the last
 * gs_bin_sort. */
int gs_sync_status(const void *ws, size_t ws_bytes, void *stream, int64_t *n_instances);

/* Binning statistics of the last render on ws (synchronises `stream`, reads the
 * workspace header): out[0] the instance slots -- every (Gaussian, tile) instance without
 * cuts; with cuts, those of the Gaussians in front of some cut of their rows plus those
 * the completion emitted -- out[1] the instances sorted by gs_bin_sort (in front of the
 * depth cut), out[2] those sorted by gs_topk_select to complete unsaturated tiles, out[3]
 * the tiles it completed. */
int gs_binning_stats(const void *ws, size_t ws_bytes, void *stream, int64_t out[4]);

/* Kernel timers, for measurement.  While enabled (gs_timer_enable(1)), each launch of a
 * timed stage below that is not being captured into a graph is bracketed by a CUDA event
 * pair recorded on the stream it runs on (the feature-gradient blocks run on the
 * library's auxiliary stream).  gs_timer_read(id, &ms) waits for the end event of the
 * stage's last recorded launch and returns its elapsed milliseconds in *ms; GS_ERR_ARG
 * for an unknown id or when none was recorded since gs_timer_enable(1).  Process-wide
 * state, for one device.  Recording adds two event records per timed stage; disabled (the
 * default) it adds one flag test. */
#define GS_TIMER_BINNING 0     /* gs_bin_sort: tile counts, their scan, instance emission */
#define GS_TIMER_TILE_SORT 1   /* gs_bin_sort: radix sort of the instances by tile */
#define GS_TIMER_WALK_FWD 2    /* gs_topk_select: the (first) forward walk */
#define GS_TIMER_BLOCK_GRAD 3  /* gs_backward: per-block partial feature-gradient rows */
#define GS_TIMER_WALK_BWD 4    /* gs_backward: the re-walk adjoint */
#define GS_TIMER_COMPLETE 5    /* gs_topk_select: completing the tiles the depth cut left unsaturated */
#define GS_TIMER_COUNT 6
int gs_timer_enable(int on);
int gs_timer_read(int id, float *ms);

#ifdef __cplusplus
}
#endif
#endif /* GS_TOPK_H */
