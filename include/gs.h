/*
 * gs.h -- C ABI of the GB300 (sm_103a) differentiable Gaussian splatting
 * library for the mapping and pose-refinement hot path of TAMBRIDGE
 * (arXiv 2405.19614).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are DEVICE pointers unless marked "host".  The caller
 *    owns every buffer, including workspaces; the library never allocates,
 *    never frees and never synchronises the stream inside a call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is only enqueued; results are ready when the stream is.
 *  - Synchronous argument errors return a gs_status_t and enqueue nothing.
 *    Asynchronous errors (pair capacity exceeded, bounded wait expired) are
 *    OR-ed into a device status word (bit 1 << GS_ERR_CAPACITY,
 *    1 << GS_ERR_TIMEOUT) that the caller reads after the stream; outputs are
 *    then incomplete but every access stays in bounds.
 *  - Views: up to GS_MAX_VIEWS cameras per call, possibly of different sizes.
 *    Per-view arrays are concatenated: projected records and radii at
 *    [v * n + i]; pixels at pix_base[v] + y * width + x with pix_base the
 *    running sum of width*height; tiles at tile_base[v] + ty * tiles_x + tx with
 *    tile_base the running sum of tiles_x * tiles_y, tiles_x = ceil(width /
 *    tile_w) and tiles_y = ceil(height / tile_h) for the view's tile shape.
 *  - Pixel (x, y) is sampled at (x + 0.5, y + 0.5); u = fx * X/Z + cx.
 *  - Poses are world -> camera row-major 3x4 [R | t] (device, FP32) so that an
 *    on-device pose update needs no host round trip; the twist is
 *    xi = (rho, phi) with pose(xi) = Exp(xi) * E and gradients at xi = 0.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_MAX_VIEWS 64
#define GS_TILE 16 /* default tile width and height in pixels */

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,
    GS_ERR_CUDA = 2,
    GS_ERR_CAPACITY = 3,
    GS_ERR_TIMEOUT = 4,
    GS_ERR_UNSUPPORTED = 5
} gs_status_t;

/* Host-side camera intrinsics and image size (Sec. 3.4 "Projection": K). */
/* A view: pinhole intrinsics, image size and the tile shape that bins and
 * composites it (Sec. 3.4 "Differentiable Rasterization" sorts Gaussians per
 * screen tile; the shape is this library's choice, picked by its autotuner).
 * tile_w, tile_h: 8, 16, 32 or 64 pixels with tile_w * tile_h <= 2048, or 0
 * for GS_TILE.  Every call that takes the views of one configuration must
 * get the same tile shapes (they define the tile ids and ranges). */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
    int32_t tile_w, tile_h;
} gs_view_t;

/* Gaussian parameters, structure of arrays (Sec. 3.4 "Gaussian
 * Representation", generalised to anisotropic scales and SH colour):
 * means [n,3], log_scales [n,3], quats [n,4] as (w, x, y, z), not necessarily
 * normalised, opacity_logit [n] (opacity = sigmoid), sh [n, (deg+1)^2, 3]. */
typedef struct {
    const float *means, *log_scales, *quats, *opacity_logit, *sh;
    int64_t n;
    int32_t sh_degree; /* 0..3 */
} gs_params_t;

/* Gradients with the same layouts as gs_params_t; accumulated (+=), or
 * written (=) where gs_options_t.overwrite_grads is set. */
typedef struct {
    float *means, *log_scales, *quats, *opacity_logit, *sh;
} gs_param_grads_t;

typedef struct {
    float near_z; /* cull if camera z <= near_z (0.2) */
    float blur;   /* low-pass variance added to the 2D covariance (0.3 px^2) */
    int32_t overwrite_grads; /* gs_project_bwd: 0 adds to grads (+=); 1 writes every
                              * Gaussian's gradients (=), so grads need no zeroing */
} gs_options_t;

/* Output of gs_project, one entry per (view, Gaussian) at [v * n + i]:
 *   rec [., 12] floats: (u, v, z, log2 o), (A', B', C', du),
 *                       (red, green, blue, dv); u, v, z are the FP32 values of
 *                       the binning contract and du, dv the remainders
 *                       u* - u, v* - v of the 2D mean computed in double-FP32
 *                       arithmetic, so the compositing sees the mean to
 *                       ~1e-7 px; log2 o is the opacity's base-2 logarithm
 *                       and (A', B', C') = -log2(e) (A/2, B, C/2) the conic
 *                       (A, B, C) = (c, -b, a) / det of the 2D covariance
 *                       (a, b, c) in base 2, so that log2(o exp(power)) =
 *                       log2 o + A' dx^2 + B' dx dy + C' dy^2.  u, v, du, dv,
 *                       log2 o and A', B', C' follow one fixed sequence of
 *                       correctly rounded FP32 operations (the compositing's
 *                       alpha decisions are taken on them); 16-byte aligned;
 *   rect [., 2] uint32: x0 | y0 << 16 and x1 | y1 << 16, the inclusive tile
 *                       rectangle;
 *   radii [.]   int32 support radius in pixels, 0 = not drawn in that view;
 *   tile_mask [.] uint64, written for drawn records whose rectangle has
 *                       w x h <= 64 tiles: bit (j * w + i) set when the splat
 *                       can reach alpha >= 1/255 in tile (x0 + i, y0 + j) (a
 *                       conservative FP32 test of the record's quadratic form
 *                       over the tile's pixel centres, per tile row: a
 *                       cleared tile is one where every pixel would skip the
 *                       splat); 8-byte aligned;
 *   tiles_touched [.] uint32 number of tiles kept (the set bits of tile_mask,
 *                       or every tile of a larger rectangle); 0 = no pair. */
typedef struct {
    float *rec;
    uint32_t *rect;
    int32_t *radii;
    uint32_t *tiles_touched;
    uint64_t *tile_mask;
} gs_projected_t;

/* Output of gs_bin_sort:
 *   keys [capacity] uint64: (global tile id << 32) | bits(z), ascending;
 *   vals [capacity] uint32: Gaussian index within its view;
 *   ranges [n_tiles_total, 2] uint32: [start, end) of each tile's list;
 *   n_pairs: device uint32, number of (Gaussian, tile) pairs (may exceed the
 *            capacity, in which case status has the capacity bit set);
 *   status: device uint32 error word (see above); never cleared by the library. */
typedef struct {
    uint64_t *keys;
    uint32_t *vals;
    uint32_t *ranges;
    uint32_t *n_pairs;
    uint32_t *status;
    int64_t capacity;
} gs_bins_t;

/* Forward image outputs, per pixel (see pixel layout above):
 * rgb [P,3], depth [P], alpha [P] (= border mask M_b), final_T [P],
 * n_contrib [P] (list entries consumed up to the last blended one). */
typedef struct {
    float *rgb, *depth, *alpha, *final_T;
    uint32_t *n_contrib;
} gs_image_t;

/* Library version string. */
const char *gs_version(void);

/* Text for a status code. */
const char *gs_status_string(gs_status_t s);

/* Host read of an asynchronous error word (the status of gs_bins_t, or of
 * any call that takes one): copies *status_dev (device uint32) to
 * *status_host after the work already enqueued on stream, and waits for it.
 * This is the one call of the library that synchronises.  Bit
 * 1 << GS_ERR_CAPACITY: a pair capacity was exceeded; 1 << GS_ERR_TIMEOUT: a
 * bounded wait expired.  GS_ERR_INVALID_ARG for null pointers, GS_ERR_CUDA if
 * the copy fails. */
gs_status_t gs_get_device_status(const uint32_t *status_dev, uint32_t *status_host, void *stream);

/* Workspace bytes of one operation in one place (each also has its own size
 * call): GS_OP_BIN_SORT (n_views * n records, pair_capacity),
 * GS_OP_GRAD2D (the 2D gradient buffer of n Gaussians in n_views views),
 * GS_OP_SSIM (n_pixels), GS_OP_SELECT (n items: densification and pruning),
 * GS_OP_SPATIAL_ORDER (n Gaussians), GS_OP_CHECK_LOOKBACK.  0 for an unknown
 * op or negative sizes. */
enum {
    GS_OP_BIN_SORT = 0,
    GS_OP_GRAD2D = 1,
    GS_OP_SSIM = 2,
    GS_OP_SELECT = 3,
    GS_OP_SPATIAL_ORDER = 4,
    GS_OP_CHECK_LOOKBACK = 5
};
size_t gs_workspace_size(int32_t op, int64_t n, int32_t n_views, int64_t pair_capacity, int64_t n_pixels);

/* Check of the asynchronous timeout path of the radix passes (the paper has
 * no counterpart; the bounded waits of the onesweep look-back are this
 * library's design).  Enqueues one onesweep counting pass over 8,192
 * pseudo-random uint32 keys (key i = i * 2654435761 mod 2^32, value i) in
 * two 4,096-key tiles, sorted stably by their low byte.  With
 * withhold_first_tile = 0 the pass runs normally: the sorted keys and values
 * are left at byte offsets 0 and 32,768 of the workspace and *status is not
 * touched.  With withhold_first_tile != 0 the pass starts its tile counter at
 * 1, so tile 0 is never published: tile 1's look-back gives up after
 * spin_limit waits of about 32 ns, ORs 1 << GS_ERR_TIMEOUT into *status
 * (device uint32) and the kernel returns; its outputs are then meaningless
 * but every write stays inside the workspace.  spin_limit 0 takes the
 * library's default (2^22).  workspace: device, 256-byte aligned,
 * >= gs_check_lookback_timeout_workspace_size() bytes.  GS_ERR_INVALID_ARG
 * for a null or short workspace or a null status. */
size_t gs_check_lookback_timeout_workspace_size(void);
gs_status_t gs_check_lookback_timeout(uint32_t spin_limit, int32_t withhold_first_tile, uint32_t *status,
                                      void *workspace, size_t workspace_bytes, void *stream);

/* Total tiles and pixels over the views (host helper). */
gs_status_t gs_layout(const gs_view_t *views /* host */, int32_t n_views, int64_t *n_tiles_total,
                      int64_t *n_pixels_total);

/* a1. Projection (Sec. 3.4 "Projection": mu2D = K E_t mu / d, r2D = f r / d;
 * EWA footprint of the rasteriser of Sec. 4.1).  For every view and Gaussian:
 * camera transform, 2D covariance J W S W^T J^T + blur, support radius
 * ceil(3 sqrt(lambda_max)), tile rectangle, conic, opacity = sigmoid(logit),
 * colour = max(0, SH(dir) + 0.5).  Radius, rectangle and depth follow a fixed
 * FP32 operation order so that binning is reproducible bit for bit.
 * params: device SoA; views: host [n_views]; viewmats: device [n_views, 12].
 * out: caller-allocated arrays of n_views * params->n entries.
 * Errors: GS_ERR_INVALID_ARG for null pointers, n < 0, n_views outside
 * [1, GS_MAX_VIEWS], sh_degree outside [0, 3] or non-positive image sizes. */
gs_status_t gs_project(const gs_params_t *params, const gs_view_t *views, const float *viewmats,
                       int32_t n_views, const gs_options_t *opt, gs_projected_t *out, void *stream);

/* Bytes of workspace gs_bin_sort needs for n_records = n_views * n and the
 * given pair capacity (about 8 bytes per pair of capacity and 16 per record;
 * n_tiles_total does not enter); 0 for invalid sizes. */
size_t gs_bin_sort_workspace_size(int64_t n_records, int64_t pair_capacity, int64_t n_tiles_total);

/* a2-a4. Binning in front-to-back order (Sec. 3.4 "Differentiable
 * Rasterization": Gaussians arranged front to back before alpha blending).
 * Produces exactly the pairs a stable sort of the keys (global tile << 32) |
 * bits(depth), values = Gaussian index, would: per tile, entries by depth,
 * equal depths in index order, and each tile's [start, end) ([0, 0) when
 * empty).  Built by sorting the drawn records by depth, emitting their pairs
 * in that order and sorting the pairs stably by tile id (onesweep radix
 * passes over 32-bit keys).  n_views * n must be below 2^32.  When the pair
 * total exceeds bins->capacity, n_pairs still reports the total, the
 * capacity bit is set in the status word and only the pairs of the nearest
 * records that fit are binned.
 * workspace: device, >= gs_bin_sort_workspace_size bytes, 256-byte aligned. */
gs_status_t gs_bin_sort(const gs_projected_t *proj, int64_t n, const gs_view_t *views, int32_t n_views,
                        gs_bins_t *bins, void *workspace, size_t workspace_bytes, void *stream);

/* Allocation-free gs_bin_sort (the paper has no counterpart: this serves
 * callers that cannot allocate device memory, such as code in the middle of a
 * CUDA graph capture, fixed-rate tracking loops that cannot take the device
 * synchronisation an allocation may cause, or host frameworks that own all
 * device memory and pass a plugin only its inputs and outputs).  Same inputs,
 * outputs and results as gs_bin_sort, but the scratch workspace is a
 * static device array inside the library (about 65 MiB: exactly gs_bin_sort's
 * workspace at both limits), held on every GPU that loads it until the
 * process exits.  Limits: n_views * n <= 2,097,152 records and
 * bins->capacity <= 2,097,152 pairs; every call within them fits, larger
 * calls return GS_ERR_CAPACITY and enqueue nothing.  The first call on a device looks up
 * the array's address (cudaGetSymbolAddress) and should come before any
 * stream capture.  All
 * calls share the array and it keeps the last call's contents (what must
 * start at zero is cleared inside each call); calls that may overlap on the
 * GPU race on it and must not be issued. */
gs_status_t gs_bin_sort_noalloc(const gs_projected_t *proj, int64_t n, const gs_view_t *views, int32_t n_views,
                                gs_bins_t *bins, void *stream);

/* a5. Forward compositing (Sec. 3.4: C(p) = sum c_i f_i prod_{j<i} (1 - f_j),
 * D(p) likewise with the depths d_i; Sec. 3.3: M_b(p) = sum f_i prod (1 - f_j)).
 * alpha_i = min(0.99, o_i exp(-1/2 d^T conic d)); entries with alpha < 1/255
 * are skipped; compositing stops before an entry that would bring T below
 * 1e-4.  One persistent launch over all (view, tile) work items.
 * work_counter: device uint32 scratch, reset inside the call. */
gs_status_t gs_render_fwd(const gs_projected_t *proj, int64_t n, const gs_bins_t *bins,
                          const gs_view_t *views, int32_t n_views, gs_image_t *img,
                          uint32_t *work_counter, void *stream);

/* a5 + a6 fused: gs_render_fwd that also evaluates gs_loss_l1 on each pixel as
 * it finishes (same arguments and results as gs_loss_l1 over all pixels of the
 * views: adds L to *loss, WRITES d_rgb [P,3] and d_depth [P]), so the image is
 * not read back by a separate loss launch.  d_rgb and d_depth equal
 * gs_loss_l1's bit for bit; *loss differs only in summation order.
 * Errors as gs_render_fwd, and GS_ERR_INVALID_ARG for null loss arguments. */
gs_status_t gs_render_fwd_l1(const gs_projected_t *proj, int64_t n, const gs_bins_t *bins, const gs_view_t *views,
                             int32_t n_views, gs_image_t *img, uint32_t *work_counter, const float *target_rgb,
                             const float *target_depth, float w_c, float w_d, int32_t use_gate, float gamma,
                             float *loss, float *d_rgb, float *d_depth, void *stream);

/* Work counts of a5 for measurement: per pixel, the list entries evaluated
 * (n_eval [P]) and blended (n_blend [P]) by the forward compositing under the
 * same skip and stop rules.  Writes no image. */
gs_status_t gs_render_stats(const gs_projected_t *proj, int64_t n, const gs_bins_t *bins,
                            const gs_view_t *views, int32_t n_views, uint32_t *n_eval, uint32_t *n_blend,
                            uint32_t *work_counter, void *stream);

/* Kernel variants of the compositing (a5, a7), 0..23 for both the forward and
 * the backward: index % 6 is the band shape (pixels per thread, band width
 * BW), a warp's band of a tile being BW x (pixels per thread * 32 / BW)
 * pixels, in (1,8) (2,8) (2,16) (4,8) (4,16) (8,16); index / 6 the staging of
 * the list entries in shared memory: 32 loaded by the lanes into registers,
 * 32 copied by the lanes' asynchronous copies into a second buffer, or 32 or
 * 64 gathered by the tensor memory accelerator (a band that does not divide
 * a view's tile falls back to the (2, 8) band of the same staging; defaults:
 * forward 7, backward 9, the asynchronous-copy (2, 8) and (4, 8)).  All
 * variants compute the same result; the autotuner times them on the workload
 * and sets the fastest.  The setting is process-wide and read when a kernel
 * is launched.  GS_ERR_INVALID_ARG for an index out of range. */
gs_status_t gs_set_render_variants(int32_t fwd, int32_t bwd);

/* Current variants and the number of each (any pointer may be NULL). */
gs_status_t gs_get_render_variants(int32_t *fwd, int32_t *bwd, int32_t *n_fwd, int32_t *n_bwd);

/* a6. L1 rendering losses with the optional filter gate (Sec. 3.3
 * G(p) = [D_c > 0][D_g > 0][M_b > gamma]; Sec. 3.3 joint loss w2 L_c + w3 L_d;
 * Sec. 3.4 L_m L1 terms):  L = w_c/(3P) sum G |C - C^| + w_d/P sum G |D - D^|
 * over all P pixels of the batch.  Adds L to *loss (device float) and WRITES
 * d_rgb [P,3] and d_depth [P] (sign(0) = 0; zero where the gate is closed). */
gs_status_t gs_loss_l1(const float *rgb, const float *depth, const float *alpha, const float *target_rgb,
                       const float *target_depth, int64_t n_pixels, float w_c, float w_d,
                       int32_t use_gate, float gamma, float *loss, float *d_rgb, float *d_depth,
                       void *stream);

/* Keyframe decoding (Sec. 4: RGB-D frames of TUM RGB-D, 8-bit colour and
 * 16-bit depth): rgb8 [P,3] bytes and depth16 [P] (device, as uploaded from
 * the sensor) to the FP32 loss targets rgb [P,3] = c / 255 and depth [P] =
 * d * depth_scale (metres per depth unit, e.g. 1/5000 for TUM RGB-D; 0 stays
 * 0), each one correctly rounded FP32 operation.  Alignment: rgb8 4 bytes,
 * depth16 8 bytes, rgb and depth 16 bytes, else GS_ERR_INVALID_ARG. */
gs_status_t gs_decode_keyframes(const uint8_t *rgb8, const uint16_t *depth16, int64_t n_pixels, float depth_scale,
                                float *rgb, float *depth, void *stream);

/* Bytes of workspace gs_loss_ssim needs for n_pixels (9 floats per pixel). */
size_t gs_ssim_workspace_size(int64_t n_pixels);

/* SSIM term of the mapping loss (Sec. 3.4: L_m = (1 - zeta)(w4 L1(D) +
 * w5 L1(C)) + zeta L_SSIM, zeta = 0.3).  The paper does not define its SSIM;
 * this is the usual one: per colour channel, moments under an 11x11 Gaussian
 * window (sigma 1.5, normalised, zero padding), C1 = 0.01^2, C2 = 0.03^2.
 * Adds weight * (1 - mean SSIM) over all pixels and channels of the views to
 * *loss and its gradient to d_rgb [P,3] (+=, so it sums with gs_loss_l1's).
 * rgb, target_rgb [P,3] device; views host; workspace device, >=
 * gs_ssim_workspace_size(P) bytes, 16-byte aligned for the staged gradient
 * pass (else a slower pass runs).  status: device error word, may be NULL; an
 * asynchronous copy that never completes sets bit GS_ERR_TIMEOUT there (the
 * bounded wait gives up, the affected tiles' gradients are missing). */
gs_status_t gs_loss_ssim(const float *rgb, const float *target_rgb, const gs_view_t *views, int32_t n_views,
                         float weight, float *loss, float *d_rgb, void *workspace, size_t workspace_bytes,
                         uint32_t *status, void *stream);

/* Check of the asynchronous timeout path of the SSIM gradient pass (the
 * paper has no counterpart; the staged copies and their bounded waits are this
 * library's design).  Runs gs_loss_ssim with weight 1 on the same arguments,
 * but the gradient pass's barrier expects 16 bytes more than its staged copy
 * delivers, so every block's bounded wait gives up: each block sets bit
 * GS_ERR_TIMEOUT in *status and returns without touching d_rgb (the loss is
 * still added).  The copies themselves complete, so nothing is left in
 * flight.  GS_ERR_UNSUPPORTED when the staged pass cannot run for these views
 * (a width or first pixel not a multiple of 4, or a workspace not 16-byte
 * aligned); GS_ERR_INVALID_ARG for a null status. */
gs_status_t gs_check_ssim_timeout(const float *rgb, const float *target_rgb, const gs_view_t *views,
                                  int32_t n_views, float *loss, float *d_rgb, void *workspace, size_t workspace_bytes,
                                  uint32_t *status, void *stream);

/* Bytes of the per-(view, Gaussian) 2D gradient buffer: n_views * n * 12 floats. */
size_t gs_grad2d_size(int64_t n, int32_t n_views);

/* a7. Backward of the compositing for upstream gradients d_rgb [P,3],
 * d_depth [P], d_alpha [P] (each may be NULL = zero).  Recomputes each
 * pixel's blend state from final_T and n_contrib, reduces per-Gaussian
 * gradients over each warp (three list entries at a time, through a table in
 * shared memory) and adds them with atomics into grad2d [n_views * n, 12]
 * laid out as
 * (du, dv, dconicA, dconicB), (dconicC, dopacity, dred, dgreen),
 * (dblue, dz, 0, 0).  grad2d is accumulated (+=). */
gs_status_t gs_render_bwd_splats(const gs_projected_t *proj, int64_t n, const gs_bins_t *bins,
                                 const gs_view_t *views, int32_t n_views, const gs_image_t *img,
                                 const float *d_rgb, const float *d_depth, const float *d_alpha,
                                 float *grad2d, uint32_t *work_counter, void *stream);

/* a8. Backward of the projection: chains grad2d to the parameter gradients
 * (summed over views, accumulated into grads) and to each view's twist
 * gradient d_twist [n_views, 6] (+=; NULL to skip); with opt->overwrite_grads
 * set, grads are written (=) instead of accumulated.  grads = NULL selects the
 * pose-only mode of tracking (Sec. 3.3: the pose is refined, the map is not):
 * only d_twist is written.  Entries of grad2d it reads are set back to zero,
 * so a buffer that starts zeroed is zero again when the call completes.
 * grad2d and params->quats must be 16-byte aligned (GS_ERR_INVALID_ARG
 * otherwise); params->sh and grads->sh need only 4-byte alignment (when both
 * are 16-byte aligned the SH rows are copied 16 bytes at a time; the results
 * are the same bit for bit). */
gs_status_t gs_project_bwd(const gs_params_t *params, const gs_view_t *views, const float *viewmats,
                           int32_t n_views, const gs_options_t *opt, const gs_projected_t *proj,
                           float *grad2d, gs_param_grads_t *grads, float *d_twist, void *stream);

/* a7 + a8. The whole backward of the render (reverse of Sec. 3.4 projection and
 * compositing): gs_render_bwd_splats followed by gs_project_bwd.  grad2d must
 * be zero on entry (it is zero again on completion); parameter gradients and
 * d_twist are accumulated; grads may be NULL (pose only).  Used for mapping (pose fixed, Sec. 3.4) with
 * d_twist = NULL and for pose refinement (Sec. 3.3) with d_twist set. */
gs_status_t gs_render_bwd(const gs_params_t *params, const gs_view_t *views, const float *viewmats,
                          int32_t n_views, const gs_options_t *opt, const gs_projected_t *proj,
                          const gs_bins_t *bins, const gs_image_t *img, const float *d_rgb,
                          const float *d_depth, const float *d_alpha, float *grad2d,
                          gs_param_grads_t *grads, float *d_twist, uint32_t *work_counter, void *stream);

/* a9. Keypoint re-projection loss (Sec. 3.2 Eq. lba; Sec. 3.3 tracking-centred
 * encoder):  L = (weight/n) sum_i || obs_i - pi(K_v, E_v, P_i) ||_2 over
 * points P_i [n,3] (world) observed at obs [n,2] pixels in view view_ids[i]
 * ([n] int32, NULL = view 0).  Points with camera z <= near_z are left out.
 * Adds L to *loss and dL/dxi (at xi = 0) to d_twist [n_views, 6]. */
gs_status_t gs_reproj_loss_grad(const float *points, const float *obs, const int32_t *view_ids, int64_t n,
                                const gs_view_t *views, const float *viewmats, int32_t n_views,
                                float weight, float near_z, float *loss, float *d_twist, void *stream);

/* One Adam learning-rate group: elements [offset, offset + count). */
typedef struct {
    int64_t offset, count;
    float lr;
} gs_adam_group_t;

#define GS_MAX_ADAM_GROUPS 8

/* a10. Adam step (Sec. 3.4: "iteratively refined using gradient-based
 * optimization"; the optimiser is not named): for each group, m = b1 m +
 * (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 -
 * b2^t)) + eps) with t = step[0] + 1.  step: device int32[2] = {steps done,
 * scratch that must start at 0}; the call sets step[0] = t on completion, so
 * a captured graph replays successive steps.  groups: host array. */
gs_status_t gs_adam_step(float *param, const float *grad, float *m, float *v, const gs_adam_group_t *groups,
                         int32_t n_groups, float beta1, float beta2, float eps, int32_t *step, void *stream);

/* Pose update of the tracking loop: E_v <- Exp(xi_v) E_v, then xi_v <- 0, for
 * viewmats [n_views, 12] and twist [n_views, 6] (device). */
gs_status_t gs_pose_update(float *viewmats, float *twist, int32_t n_views, void *stream);

/* ------------------------------------------------------------------------ */
/* Map maintenance and keyframe choice                                      */
/* ------------------------------------------------------------------------ */

/* Bytes of workspace of gs_densify / gs_prune_select for n_items pixels or
 * Gaussians. */
size_t gs_select_workspace_size(int64_t n_items);

/* Densification (Sec. 3.4 "Densification", Eq. d: d = r f).  Every pixel of
 * the views whose border mask alpha [P] is below threshold and whose sensor
 * depth target_depth [P] is positive gets one new Gaussian, appended in pixel
 * order at indices n_old, n_old + 1, ... of the parameter arrays (capacity
 * rows each): mean = back-projection of the pixel centre at that depth through
 * the view's pose viewmats [n_views,12]; log-scales = log(d / fx) on all axes
 * (radius of one pixel on the image plane); quaternion (1,0,0,0); SH degree-0
 * band = (rgb - 0.5) / C0 from target_rgb [P,3], higher bands 0; opacity logit
 * as given.  *n_added (device) receives the number written; pixels beyond the
 * capacity are dropped and flagged in *status (device, may be NULL).  The
 * gs_param_grads_t struct is used here for its five writable pointers. */
gs_status_t gs_densify(const float *alpha, const float *target_rgb, const float *target_depth,
                       const gs_view_t *views, const float *viewmats, int32_t n_views, float threshold,
                       float opacity_logit, gs_param_grads_t *params, int32_t sh_degree, int64_t n_old,
                       int64_t capacity, uint32_t *n_added, uint32_t *status, void *workspace,
                       size_t workspace_bytes, void *stream);

/* Pruning (Sec. 3.4 "Gaussian Pruning", tau = 0.005 in Table hyper): a
 * Gaussian is kept when its opacity sigmoid(logit) >= tau, decided on the
 * logit against log(tau / (1 - tau)) rounded once to FP32.  Writes
 * new_index [n] (its row after compaction, order kept, or -1) and *n_kept
 * (device).  tau in (0, 1). */
gs_status_t gs_prune_select(const float *opacity_logit, int64_t n, float tau, int32_t *new_index,
                            uint32_t *n_kept, void *workspace, size_t workspace_bytes, void *stream);

#define GS_MAX_COMPACT_ARRAYS 16

/* One array of rows to compact: row i of src (row_floats floats) goes to row
 * new_index[i] of dst when new_index[i] >= 0.  src and dst must not alias. */
typedef struct {
    const float *src;
    float *dst;
    int32_t row_floats;
} gs_rows_t;

/* Compacts up to GS_MAX_COMPACT_ARRAYS arrays (parameters and optimiser state)
 * with the indices of gs_prune_select, in one launch.  arrays: host. */
gs_status_t gs_compact_rows(const int32_t *new_index, int64_t n, const gs_rows_t *arrays, int32_t n_arrays,
                            void *stream);

/* Bytes of workspace of gs_spatial_order for n Gaussians (0 for n < 1). */
size_t gs_spatial_order_workspace_size(int64_t n);

/* Spatial order of the map (a layout service; the paper has no counterpart):
 * new_index [n] (device) receives each Gaussian's rank in the Morton (Z-order)
 * sequence of its mean, quantised to 1024 cells per axis of the means'
 * bounding box in correctly rounded FP32 (q = min(1023, floor((m - lo) *
 * (1024 / (hi - lo)))), 0 on a flat axis; x in the lowest bit); equal codes
 * keep index order.  Applied with gs_compact_rows to every per-Gaussian array
 * it stores Gaussians that are close in space next to each other, as a map
 * grown by densification is, so that the 32 Gaussians of a warp are drawn in
 * the same views.  means [n,3] device; workspace >= the size above, 256-byte
 * aligned; status (device, may be NULL) receives GS_ERR_TIMEOUT if a bounded
 * wait of the sort expires.  n < 2^31. */
gs_status_t gs_spatial_order(const float *means, int64_t n, int32_t *new_index, void *workspace,
                             size_t workspace_bytes, uint32_t *status, void *stream);

/* View point selection (Sec. 3.3): keyframe i (i >= 1) is selected when
 * beta <= matches[i] < alpha * totals[i], with matches[i] = M_{i-1,i} the
 * feature matches between keyframes i-1 and i and totals[i] = T_{i-1,i} the
 * total matches of keyframe i-1 (alpha = 0.75, beta = 20 in Table hyper); the
 * first keyframe is always selected.  Host arrays; writes selected [n] as 0/1. */
gs_status_t gs_select_views(const int32_t *matches, const int32_t *totals, int32_t n, float alpha, int32_t beta,
                            int32_t *selected);

#ifdef __cplusplus
}
#endif
#endif /* GS_H_ */
