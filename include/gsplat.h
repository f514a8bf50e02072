/*
 * gsplat.h - C ABI of the GB300 pose-differentiable Gaussian-splatting
 * renderer ("Look Gauss, No Pose", arXiv 2410.08743).
 *
 * The library renders a set of 3D Gaussians (Sec. 3.1, Eq. 1-4) into one or
 * more views and back-propagates an image loss to every Gaussian parameter
 * and, per view, to the 6-DoF world-to-camera pose as a tangent-space
 * gradient of a left perturbation T <- Exp(tau) T, tau = (rho, phi)
 * (Sec. 3.2, Eq. 5-13).  All arithmetic runs in the library's own sm_103a
 * CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Return codes: GS_OK (0), GS_PENDING (> 0, polling only), or a negative
 *     GS_E* code; gs_last_error() returns a thread-local message for the
 *     calling thread's last failure.  No C++ exception crosses this ABI.
 *   - Pointers are DEVICE pointers unless the argument says host.  Device
 *     inputs are borrowed for the duration of the call's stream work; the
 *     caller must keep them alive and unmodified until that work completes.
 *   - Every call is asynchronous on the caller's CUDA stream (`stream`, a
 *     cudaStream_t passed as void*; NULL = legacy default stream) unless it
 *     says otherwise.  Workspaces live in the gs_ctx / gs_frames objects and
 *     grow on demand; a growth may synchronise the stream.
 *   - Layouts:
 *       Gaussians (structure of arrays, float32): means [N][3], scales [N][3]
 *       (activated, > 0), quats [N][4] (w, x, y, z; any non-zero length, 16-byte
 *       aligned; the
 *       renderer normalises), opacities [N] (activated, in [0, 1]), sh
 *       [N][16][3] (real SH, degree <= 3, l = 0..3, m = -l..l; the stride is
 *       16 coefficients whatever sh_degree is).
 *       Poses: float64 [V][12] = world->camera rotation R (row-major 3x3)
 *       then translation t, so a world point x maps to R x + t.
 *       Images: packed float32 planar, view v occupies [3][H_v][W_v] starting
 *       at sum_{u<v} 3 H_u W_u; the pixel (px, py) samples the image-plane
 *       point (px, py) (integer pixel centres).
 *       Per-view pose gradients: float64 [V][6] = (rho[3], phi[3]).
 */
#ifndef GSPLAT_H
#define GSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GS_OK = 0,
    GS_PENDING = 1,       /* solve not finished yet (gs_solve_poll) */
    GS_EINVAL = -1,       /* bad argument */
    GS_ENOMEM = -2,       /* device or host allocation failed */
    GS_ETIMEOUT = -3,     /* a bounded device or host wait gave up */
    GS_EBUSY = -4,        /* object in use / queue full */
    GS_ECUDA = -5,        /* a CUDA runtime call failed */
    GS_EOVERFLOW = -6     /* a fixed-capacity buffer was too small (no-sync mode) */
};

/* Render option flags. */
enum {
    GS_F_NO_SYNC = 1u << 0,   /* never synchronise inside the call: use the
                                 capacities reserved so far and report
                                 GS_EOVERFLOW through gs_status() instead of
                                 growing (required inside CUDA-graph capture) */
    GS_F_HOST_IO = 1u << 1,   /* gs_step only: every array argument is host memory */
    GS_F_RECOMPUTE = 1u << 3, /* gs_render_backward only: rebuild the forward state
                                 (projection, tile lists, sorted prefixes, per-pixel
                                 state) of THESE views instead of requiring that `fr`
                                 still holds it, so one frames object can serve many
                                 view batches in turn and memory stays bounded by
                                 one batch's tile lists (the forward is deterministic,
                                 so the result is the same) */
    GS_F_FULL_SORT = 1u << 2, /* sort every tile's whole list before blending.  By
                                 default a tile is sorted only as far as the forward
                                 blend consumes it (identical image and gradients);
                                 GS_Q_SORTED_IDX then holds each tile's sorted prefix
                                 of GS_Q_SORTED_COUNT entries. */
    GS_F_COUNT = 1u << 4      /* the blends accumulate the work counters that
                                 gs_frames_counters reads (off by default: counting
                                 costs a few percent of the blends' instructions;
                                 results are the same either way) */
};

typedef struct gs_ctx gs_ctx;
typedef struct gs_scene gs_scene;
typedef struct gs_frames gs_frames;

/* Gaussians, structure of arrays (layout above). */
typedef struct {
    int64_t n;
    int32_t sh_degree;        /* 0..3 */
    const float* means;
    const float* scales;
    const float* quats;
    const float* opacities;
    const float* sh;
} gs_scene_desc;

/* Pinhole intrinsics and image size of one view (host memory). */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
} gs_view;

/* Rendering options (Sec. 3.1; values the paper leaves open are the prior
 * art's: see gs_default_opts). */
typedef struct {
    float bg[3];              /* background colour composited with T_final */
    float z_near;             /* cull Gaussians with camera-space z <= z_near */
    float eps2d;              /* low-pass dilation added to Sigma_hat's diagonal */
    float clamp_factor;       /* frustum clamp of x/z, y/z in J; 0 disables */
    float alpha_min;          /* skip a splat whose alpha < alpha_min */
    float alpha_max;          /* clamp alpha to alpha_max */
    float t_min;              /* stop before a splat that would bring T below t_min */
    uint32_t flags;           /* GS_F_* */
} gs_render_opts;

/* Fills the defaults: black background, z_near 0.2, eps2d 0.3,
 * clamp_factor 1.3, alpha_min 1/255, alpha_max 0.99, t_min 1e-4, flags 0. */
void gs_default_opts(gs_render_opts* opts);

/* Loss applied inside gs_render_backward. */
enum {
    GS_LOSS_DLDC = 0,         /* dl_dimage holds dL/dC directly */
    GS_LOSS_L1 = 1,           /* w_l1 * mean_{3HW} |C - target| per view (Eq. 16, L1 term) */
    GS_LOSS_L1_DSSIM = 2,     /* w_l1 * L1 + w_dssim * (1 - SSIM), 11x11 Gaussian window
                                 (Eq. 16 with beta = w_dssim) */
    GS_LOSS_L1_MASKED = 3     /* confidence-masked L1 of pose estimation (Sec. 3.4, Eq. 20-21):
                                 w_l1 * mean_{3HW} M |C - target| with the per-pixel mask
                                 M = [accumulated alpha 1 - T_final > mask_alpha]; the mask is
                                 piecewise constant, so it carries no gradient */
};

typedef struct {
    int32_t kind;             /* GS_LOSS_* */
    float w_l1, w_dssim;
    const float* target;      /* device, packed like the image (L1 / D-SSIM) */
    const float* dl_dimage;   /* device, packed like the image (GS_LOSS_DLDC) */
    double* loss;             /* device [V], nullable: per-view loss values (written) */
    float mask_alpha;         /* GS_LOSS_L1_MASKED threshold; 0 means the paper's 0.99 */
} gs_loss;

/* Per-Gaussian gradient outputs (device, same layouts as the parameters).
 * gs_render_backward ADDS into them, so a per-view loop accumulates; zero
 * them first for a fresh gradient.  Any member may be NULL to skip it. */
typedef struct {
    float* means;
    float* scales;
    float* quats;
    float* opacities;
    float* sh;
} gs_grads;

/* ---------------------------------------------------------------- objects */

/* Creates a context on CUDA device `device` (made current for the call).
 * The context owns per-call scratch and a device status word. */
int gs_ctx_create(int device, gs_ctx** out);
void gs_ctx_destroy(gs_ctx* ctx);

/* Copies a scene (host or device source, `src_on_device` 0/1) into
 * library-owned device memory.  Synchronous. */
int gs_scene_load(gs_ctx* ctx, const gs_scene_desc* desc, int src_on_device, gs_scene** out);
/* Wraps caller-owned DEVICE arrays without copying (the caller keeps them
 * alive for every call that uses the handle). */
int gs_scene_borrow(const gs_scene_desc* desc, gs_scene** out);
void gs_scene_free(gs_scene* scene);

/* Forward state kept for the backward pass: per-(view, Gaussian) splats,
 * tile lists, per-pixel final transmittance and list lengths.  One frames
 * object serves one forward/backward pair at a time. */
int gs_frames_create(gs_ctx* ctx, gs_frames** out);
void gs_frames_destroy(gs_frames* fr);
/* Reserves capacity (in keys, in (view, Gaussian) pairs, in pixels and in
 * tiles) so that GS_F_NO_SYNC calls up to that size cannot overflow. */
int gs_frames_reserve(gs_frames* fr, int64_t keys, int64_t pairs, int64_t pixels, int64_t tiles);

/* ---------------------------------------------------------------- render */

/* Sec. 3.1: projects every Gaussian into every view (Eq. 1-2, SH colour),
 * builds the depth-sorted per-tile lists (deterministic: ties in depth go
 * to the lower Gaussian index) and alpha-composites front to back (Eq. 3-4).
 *   views  host [n_views]; poses device [n_views][12];
 *   image  device output, packed planar float32.
 *   target device, nullable: with a target the per-view L1 loss (mean over
 *          3HW of |C - target|) is written to loss_out [n_views] (device,
 *          float64, nullable).
 * Keeps its state in `fr` for gs_render_backward.  Errors: GS_EINVAL for
 * bad sizes/pointers, GS_ENOMEM, GS_ECUDA. */
int gs_render_forward(gs_ctx* ctx, const gs_scene* scene, int n_views, const gs_view* views,
                      const double* poses, const gs_render_opts* opts, gs_frames* fr, float* image,
                      const float* target, double* loss_out, void* stream);

/* Sec. 3.2: back-propagates the loss through compositing, projection and SH
 * to the Gaussians (accumulated into `grads`, NULL = pose only) and to each
 * view's pose (pose_grad device [n_views][6], float64, written, nullable).
 * The pose gradient is the tangent-space gradient of L(Exp(tau) T) at tau = 0
 * (Eq. 7 with Eq. 8-13).  `image` is the forward's output; the other
 * arguments must equal the forward's. */
int gs_render_backward(gs_ctx* ctx, const gs_scene* scene, int n_views, const gs_view* views,
                       const double* poses, const gs_render_opts* opts, gs_frames* fr,
                       const float* image, const gs_loss* loss, gs_grads* grads, double* pose_grad,
                       void* stream);

/* One fused forward + loss + backward step (Sec. 3.3): renders the views,
 * evaluates `loss` and writes fresh gradients (overwritten, not accumulated)
 * into `grads` (NULL = pose only) and pose_grad [n_views][6], and the per-view
 * loss into loss_out [n_views] (nullable).  image_out (nullable) receives the
 * rendered image.  Without GS_F_HOST_IO in opts->flags every array is a device
 * pointer.  With GS_F_HOST_IO every array (the scene's parameters, poses,
 * loss->target / loss->dl_dimage, image_out, grads, pose_grad, loss_out) is
 * HOST memory, preferably pinned: the call copies the inputs to library-owned
 * device staging, runs the step and copies the outputs back, ordered after
 * the work already queued on `stream`; the outputs are valid after `stream`
 * synchronises.  The copies overlap the computation on an internal stream:
 * the parameters go up in slices of Gaussians (four from 2^18 Gaussians on),
 * each slice's forward preprocess starting once its slice has landed; the
 * loss input goes up and the image comes down while the other kernels run;
 * each slice's gradients come down as soon as the backward has finished
 * them.  The results equal those of the device-buffer call. */
int gs_step(gs_ctx* ctx, gs_frames* fr, const gs_scene_desc* scene, int n_views, const gs_view* views,
            const double* poses, const gs_render_opts* opts, const gs_loss* loss, float* image_out,
            gs_grads* grads, double* pose_grad, double* loss_out, void* stream);

/* One optimisation step of the view poses (Sec. 3.2-3.3): Adam on the
 * tangent vector (moments m, v device [n_views][6] float64, kept in the
 * tangent space), then the left update T <- Exp(-lr m_hat/(sqrt(v_hat)+eps)) T
 * on poses (device [n_views][12], float64, in place).  step is 1-based. */
int gs_pose_step(gs_ctx* ctx, int n_views, double* poses, double* adam_m, double* adam_v,
                 const double* pose_grad, double lr, double beta1, double beta2, double eps,
                 int step, void* stream);

/* Pose parametrisations of the Adam step. */
enum {
    GS_POSE_SE3 = 0,          /* tau = (rho, phi) in se(3), left update T <- Exp(delta) T */
    GS_POSE_TXSO3 = 1         /* camera centre and rotation stepped separately (Sec. 4.2) */
};

/* The same step in T x SO(3) (Sec. 4.2 contrasts it with SE(3), whose
 * exponential couples camera position and orientation): the camera centre
 * o = -R^T t and the rotation are updated separately, o <- o + d_o and
 * R <- Exp(d_phi) R (a rotation about the centre), then t = -R o.  pose_grad is
 * the left-SE(3) gradient gs_render_backward writes; its T x SO(3) form is
 * (g_o, g_phi) = (-R^T g_rho, g_phi), and the moments m, v [n_views][6] hold
 * that form (do not mix them with gs_pose_step's). */
int gs_pose_step_txso3(gs_ctx* ctx, int n_views, double* poses, double* adam_m, double* adam_v,
                       const double* pose_grad, double lr, double beta1, double beta2, double eps,
                       int step, void* stream);

/* ------------------------------------------------------------ regularisers and pruning
 * Joint refinement's extra terms (Sec. 3.3).  gs_regularize ADDS to
 * grad_scales [n][3] / grad_opacities [n] (device, each nullable) the
 * gradients of
 *   lambda_aniso * (1/n) sum_i [max(s_i) / min(s_i) - aniso_r]_+   (Eq. 17)
 *   + lambda_opacity * (1/n) sum_i o_i      (the opacity L1 the paper adds
 *                                            during the first 10k steps)
 * on the ACTIVATED scales s and opacities o, and writes that value to *loss
 * (device double, nullable; summed in a fixed order).  The ratio's
 * subgradient goes to the first largest and the first smallest axis; a ratio
 * exactly at aniso_r, or all axes equal, gives none.  aniso_r >= 1.  Errors:
 * GS_EINVAL, GS_ENOMEM (scratch), GS_ECUDA.  Asynchronous on `stream`. */
int gs_regularize(gs_ctx* ctx, int64_t n, const float* scales, const float* opacities, float aniso_r,
                  float lambda_aniso, float lambda_opacity, float* grad_scales, float* grad_opacities,
                  double* loss, void* stream);

/* Adaptive opacity threshold (Sec. 3.3: the threshold is adapted so that at
 * most n_target Gaussians remain): the smallest value t >= min_opacity such
 * that at most n_target opacities (device [n]) exceed t, namely
 * max(min_opacity, the (n - n_target)-th smallest opacity) when n > n_target,
 * else min_opacity.  Writes t and the number of Gaussians with o > t (host
 * outputs; synchronises `stream`).  Opacities must be positive. */
int gs_prune_threshold(gs_ctx* ctx, int64_t n, const float* opacities, int64_t n_target, float min_opacity,
                       float* threshold, int64_t* n_keep, void* stream);

/* Stable out-of-place compaction of n_arrays (<= 24) row-major float arrays
 * (src[a] device [n][widths[a]]) into dst[a] (device, [n_keep][widths[a]],
 * allocated by the caller, not aliasing src): row i is kept iff
 * opacities[i] > threshold, in index order.  Use it to prune every parameter
 * array and Adam moment of a scene at once.  Writes *n_keep (host;
 * synchronises `stream`). */
int gs_compact(gs_ctx* ctx, int64_t n, const float* opacities, float threshold, int n_arrays,
               const float* const* src, float* const* dst, const int32_t* widths, int64_t* n_keep, void* stream);

/* ------------------------------------------------------------ spatial order
 * (No counterpart in the paper: a data-layout step.)  The renderer's passes
 * over (view, Gaussian) pairs run in Gaussian index order, so Gaussians that
 * are close in space but far apart in memory scatter every block's keys over
 * many tiles and its gathers over many cache lines.  gs_spatial_order writes
 * to perm (device uint32 [n]) the order of the Gaussians by the Morton
 * (Z-order) code of their means (device [n][3]) on a 1024^3 grid over the
 * means' bounding box, ties by index; gs_gather_rows then writes
 * dst[a][j] = src[a][perm[j]] (rows of widths[a] floats, out of place, up to
 * 24 arrays), e.g. every parameter array of a scene before it is loaded.
 * Rendering a reordered scene gives the same image (up to the order of
 * Gaussians at exactly equal depth) and the gradients in the new order.
 * Errors: GS_EINVAL, GS_ENOMEM (scratch of 16 bytes per Gaussian), GS_ECUDA.
 * Asynchronous. */
int gs_spatial_order(gs_ctx* ctx, int64_t n, const float* means, uint32_t* perm, void* stream);
int gs_gather_rows(gs_ctx* ctx, int64_t n, const uint32_t* perm, int n_arrays, const float* const* src,
                   float* const* dst, const int32_t* widths, void* stream);

/* ------------------------------------------------------------ tuning
 * Launch parameters that change performance but never results: the number of
 * Gaussians per CTA of the tile counting / key scatter (1024..8192), the run
 * length of the forward blend's lazy tile sort (1024 or 2048 keys), the
 * block size of the forward preprocess (128 or 256 threads) and the pixels
 * each thread of the backward and of the forward blend handles (1 or 2). */
typedef struct {
    int32_t scatter_chunk;
    int32_t sort_chunk;
    int32_t preprocess_threads;
    int32_t bwd_pixels_per_thread;  /* backward blend: 1 (256-thread tiles) or 2 (128) */
    int32_t fwd_pixels_per_thread;  /* forward blend: 1 or 2, likewise */
} gs_tuning;

/* A GS_F_NO_SYNC call after a tuning change needs workspaces grown by one
 * synchronising call with the new tuning (a smaller scatter_chunk needs more
 * per-CTA tile-list entries); otherwise it fails with GS_EOVERFLOW. */
int gs_ctx_set_tuning(gs_ctx* ctx, const gs_tuning* t);
int gs_ctx_get_tuning(gs_ctx* ctx, gs_tuning* t);

/* Autotuner: times one forward + backward of the given workload (the loss and
 * gradient targets as for gs_render_backward; grads may be NULL) for every
 * candidate tuning, `repeats` times each after one warm-up, keeps the fastest
 * in the context and returns it in *best (and its time in *best_ms).
 * Synchronous. */
int gs_autotune(gs_ctx* ctx, gs_frames* fr, const gs_scene* scene, int n_views, const gs_view* views,
                const double* poses, const gs_render_opts* opts, float* image, const gs_loss* loss,
                gs_grads* grads, double* pose_grad, int repeats, gs_tuning* best, double* best_ms, void* stream);

/* Raw (unactivated) Gaussian parameters optimised in joint refinement
 * (device; layouts as the scene's, log-scales and logit-opacities in place of
 * the activated values). */
typedef struct {
    float* means;
    float* log_scales;
    float* quats;
    float* logit_opacities;
    float* sh;
} gs_raw_params;

/* Per-group Adam learning rates (sh_dc for the degree-0 coefficients,
 * sh_rest for the others). */
typedef struct {
    float means, scales, quats, opacities, sh_dc, sh_rest;
} gs_gaussian_lrs;

/* One Adam step on the raw Gaussian parameters (joint reconstruction and pose
 * refinement, Sec. 3.3).  `grads` are the renderer's gradients w.r.t. the
 * ACTIVATED scales and opacities; the step chains them through s = exp(log s)
 * and o = sigmoid(logit o), updates `raw` in place and writes the activated
 * scales_out [n][3] and opacities_out [n] that the next render reads.
 * adam_m, adam_v: device float [59 n] each, groups at offsets means 0,
 * log-scales 3n, quats 6n, opacities 10n, sh 11n.  step is 1-based.  SH
 * coefficients above sh_degree are left untouched. */
int gs_gaussian_adam(gs_ctx* ctx, int64_t n, int sh_degree, gs_raw_params* raw, float* scales_out,
                     float* opacities_out, const gs_grads* grads, float* adam_m, float* adam_v,
                     const gs_gaussian_lrs* lrs, float beta1, float beta2, float eps, int step, void* stream);

/* ------------------------------------------------------------ Gaussians from a depth map
 * The initialisation of relative pose estimation (Sec. 3.4): a subset of a
 * frame's pixels is unprojected with the intrinsics and a depth map into a
 * point cloud, and every point becomes an isotropic Gaussian with the pixel's
 * colour and a scale equal to the mean 3D distance to its three nearest
 * neighbours.
 *
 * gs_unproject: the pixels (u, v) = (i * stride, j * stride) with z-depth
 * d = depth[v][u] > 0 (device [H][W]; <= 0 or NaN = no depth) become camera
 * points ((u - cx) / fx * d, (v - cy) / fy * d, d), in pixel order, with the
 * colours image[c][v][u] (device planar [3][H][W], nullable -> colours not
 * written).  points / colours: device [capacity][3] with capacity >=
 * ceil(W / stride) * ceil(H / stride).  Writes the point count to *n_out (host;
 * synchronises `stream`). */
int gs_unproject(gs_ctx* ctx, const gs_view* view, const float* depth, const float* image, int stride,
                 float* points, float* colours, int64_t capacity, int64_t* n_out, void* stream);

/* Mean Euclidean distance of each of n points (device [n][3]) to its k
 * (1..8) nearest other points (exhaustive search; coincident points count at
 * distance 0), into mean_dist (device [n]).  Asynchronous. */
int gs_knn_mean_dist(gs_ctx* ctx, int64_t n, const float* points, int k, float* mean_dist, void* stream);

/* Raw parameters (gs_raw_params, device arrays of n rows) of isotropic
 * Gaussians at the points: log-scale = log(max(mean_dist, min_scale)) on all
 * three axes, identity quaternion, logit(opacity), SH DC = (colour - 0.5) / C0
 * (the renderer's colour is C0 f0 + 0.5), every other SH coefficient 0.  The
 * paper gives no initial opacity (the prior art uses 0.1; a per-frame fit for
 * the confidence-masked pose loss needs accumulated alpha above 0.99, reached
 * in ~100 steps from 0.5).  Asynchronous. */
int gs_init_from_points(gs_ctx* ctx, int64_t n, const float* points, const float* colours, const float* mean_dist,
                        float min_scale, float opacity, gs_raw_params* raw, void* stream);


/* ------------------------------------------------------------ pose serving
 * A request loop of 6-DoF pose-estimation solves against a device-resident
 * scene (Sec. 3.4 / Sec. 4.2: estimate the camera pose of a query image from a
 * trained model by gradient descent on the photometric L1 loss).  Continuous
 * batching: a worker thread admits queued requests into free slots as slots
 * and memory allow, and each iteration runs ONE batched forward + L1 +
 * pose-only backward + Adam step over every active solve, so solves that
 * arrive while others run share the device.  Each solve's result depends only
 * on its own view (equal alone and in the mix up to FP32 summation order). */
typedef struct gs_server gs_server;

typedef struct {
    int32_t max_slots;        /* solves batched per iteration (1 = one solve at a time) */
    int32_t max_width;        /* largest accepted query image */
    int32_t max_height;
    int64_t mem_budget;       /* admission by memory: 0 (default) admits while the modelled working
                                 set of the batch fits the device memory that is free (queried before
                                 each admission) plus what the server's workspaces hold, less a
                                 reserve of max(256 MiB, 2% of the device); > 0 also caps it at this
                                 many bytes; < 0 admits without a memory check */
    int32_t queue_capacity;   /* pending requests beyond which submit returns GS_EBUSY */
    float mask_alpha;         /* 0: plain L1; > 0: confidence-masked L1 (GS_LOSS_L1_MASKED)
                                 with this accumulated-alpha threshold (the paper uses 0.99) */
    int32_t pose_param;       /* GS_POSE_SE3 or GS_POSE_TXSO3 */
    gs_tuning tuning;         /* launch parameters of the server's renderer (all zero: defaults) */
} gs_server_config;

typedef struct {
    gs_view view;             /* intrinsics and size of the query image */
    const float* image;       /* host, planar float32 [3][H][W]; copied by gs_solve_submit */
    double init_pose[12];     /* world->camera initial estimate */
    int32_t steps;            /* Adam steps (> 0) */
    double lr_start, lr_end;  /* pose learning rate, cosine decay from start to end */
} gs_solve_request;

typedef struct {
    double pose[12];          /* final world->camera estimate */
    double loss;              /* L1 loss of the last step's render */
    double latency_ms;        /* submission to completion (host clock) */
    double queue_ms;          /* submission to admission */
    int32_t steps_done;
    int32_t status;           /* GS_OK, or the error that ended the solve */
} gs_solve_result;

typedef struct {
    int64_t submitted, completed, failed, iterations, active, queued;
    double busy_ms;           /* wall time spent in iterations */
    double views_per_iteration; /* mean batch size */
    int64_t max_active;       /* largest batch so far */
    int64_t budget_bytes;     /* working-set limit at the last admission decision (-1: none) */
    int64_t requeued;         /* admitted requests put back in the queue after GS_ENOMEM */
} gs_server_stats;

/* Starts a server on `scene` (which must outlive it).  The server owns its own
 * context, stream, forward state and slot storage. */
int gs_server_create(int device, const gs_scene* scene, const gs_render_opts* opts, const gs_server_config* cfg,
                     gs_server** out);
/* Queues a solve; the image is copied.  GS_EBUSY when the queue is full,
 * GS_EINVAL for an image larger than the configured maximum. */
int gs_solve_submit(gs_server* srv, const gs_solve_request* req, uint64_t* ticket);
/* GS_PENDING while the solve runs; GS_OK once it has finished (the result is
 * returned and the ticket is released); GS_EINVAL for an unknown ticket. */
int gs_solve_poll(gs_server* srv, uint64_t ticket, gs_solve_result* out);
/* Like poll, but waits up to timeout_ms; GS_ETIMEOUT if still running. */
int gs_solve_wait(gs_server* srv, uint64_t ticket, int timeout_ms, gs_solve_result* out);
/* Cancels a queued or running solve (its result reports GS_EBUSY). */
int gs_solve_cancel(gs_server* srv, uint64_t ticket);
int gs_server_stats_get(gs_server* srv, gs_server_stats* out);
/* Stops the worker (running solves end with GS_EBUSY) and frees the server. */
void gs_server_destroy(gs_server* srv);
/* Test hook for the out-of-memory path, made on the host: the next
 * `iterations` iterations report GS_ENOMEM before any device work, as a failed
 * workspace growth would, so their new solves go back to the queue. */
int gs_server_inject_enomem(gs_server* srv, int iterations);

/* Synchronises `stream`, returns and clears the context's device status word
 * (GS_OK, GS_EOVERFLOW from a GS_F_NO_SYNC call, ...). */
int gs_status(gs_ctx* ctx, void* stream);

/* Copies an internal forward array of `fr` to host memory (synchronous):
 * what = GS_Q_*; bytes must be at least the array size; the size in bytes
 * is returned through *size_out (may be called with dst = NULL to query). */
enum {
    GS_Q_NUM_KEYS = 0,        /* int64: total (tile, Gaussian) keys */
    GS_Q_DEPTH = 1,           /* float [V*N]: key-path depth (0 where culled) */
    GS_Q_RECT = 2,            /* int32 [V*N][4]: tile rectangle x0,y0,x1,y1 (0 where culled) */
    GS_Q_RADIUS = 3,          /* int32 [V*N]: screen radius (0 where culled) */
    GS_Q_TILE_RANGES = 4,     /* uint32 [tiles][2]: [start, end) in the sorted list */
    GS_Q_SORTED_IDX = 5,      /* uint32 [keys]: Gaussian index per sorted key */
    GS_Q_T_FINAL = 6,         /* float [pixels]: final transmittance */
    GS_Q_N_CONTRIB = 7,       /* uint32 [pixels]: 1 + last blended list position in the tile */
    GS_Q_MEAN2D = 8,          /* float [V*N][2]: FP32 key-path projected mean that decides the
                                 tile rectangle (0 where culled) */
    GS_Q_SPLAT = 9,           /* float [V*N][9]: mu_hat(2) as blended (exact to ~1e-9 px, then
                                 rounded to float), conic(3), opacity, colour(3) */
    GS_Q_SORTED_COUNT = 10,   /* uint32 [tiles]: length of each tile's sorted prefix */
    GS_Q_DSSIM_GRAD = 11      /* float [sum 3HW]: the D-SSIM term's dL/dC (w_dssim included) of the
                                 last GS_LOSS_L1_DSSIM backward of these frames (GS_EINVAL if none) */
};
int gs_frames_query(gs_frames* fr, int what, void* dst, size_t bytes, size_t* size_out);

/* Per-kernel timing with CUDA events recorded on the launching stream
 * around every kernel the library launches (off by default).  While enabled,
 * calls must not be captured into a CUDA graph. */
int gs_ctx_set_profiling(gs_ctx* ctx, int enable);
/* Synchronises the device and returns, per kernel kind, the name, the summed
 * event time in milliseconds and the launch count since the last read; then
 * resets them.  names is [max_kinds][32]; *n_kinds receives the count. */
int gs_ctx_profile(gs_ctx* ctx, int max_kinds, char (*names)[32], double* total_ms, int64_t* launches,
                   int* n_kinds);

/* Measured arithmetic rates of a device, the peaks of the "alu" roofline of
 * the blending kernels (which are bound by FP32 and MUFU issue; the paper has
 * no counterpart, it reports no kernel rates), and of the atomic adds the
 * backward blend ends with.  Runs four probe kernels of one wave of resident
 * blocks each and two atomic probes on `device` (synchronous, some tens of ms,
 * uses the legacy default stream and allocates about 20 MB that it frees):
 *   sm_count               multiprocessors of the device;
 *   probe_sm_mhz           SM clock seen by the probes (clock64 cycles over
 *                          CUDA-event time); the GPU's clocks are not touched;
 *   fp32_fma_per_sm_clk    FP32 FMA lane operations per SM per cycle (FFMA);
 *   fp32x2_fma_per_sm_clk  the same with paired fma.rn.f32x2 (both halves);
 *   ex2_per_sm_clk         MUFU ex2 lane operations per SM per cycle;
 *   fp64_fma_per_sm_clk    FP64 FMA lane operations per SM per cycle (DFMA);
 *   *_per_s                the same rates per second at the probe's clock;
 *   red_f32_per_s          global atomic float adds without a return value,
 *                          every thread its own address (16 MB of addresses
 *                          that stay in L2), per second;
 *   red_f32x4_per_s        the same with 16-byte vector adds (float4).
 * Returns GS_EINVAL for a NULL out, GS_ECUDA / GS_ENOMEM on a CUDA error. */
typedef struct gs_alu_peaks {
    int sm_count;
    double probe_sm_mhz;
    double fp32_fma_per_sm_clk, fp32x2_fma_per_sm_clk, ex2_per_sm_clk;
    double fp32_fma_per_s, fp32x2_fma_per_s, ex2_per_s;
    double fp64_fma_per_sm_clk, fp64_fma_per_s;
    double red_f32_per_s, red_f32x4_per_s;
} gs_alu_peaks;
int gs_measure_alu_peaks(int device, gs_alu_peaks* out);

/* Number of CUDA kernels this context has launched so far (host counter). */
int64_t gs_ctx_launch_count(gs_ctx* ctx);

/* Work counters of the last forward/backward of `fr` (synchronous), counted
 * only by passes run with GS_F_COUNT (zero otherwise):
 * out[0] (pixel, splat) pairs whose alpha the forward blend evaluated (pairs
 * inside the splat's alpha box), out[1] pairs blended, out[2] pairs whose
 * alpha the backward blend evaluated, out[3] pairs that
 * contributed gradients in the backward, out[4] sorted-list entries read by
 * the forward blend, out[5] sorted-list entries read by the backward blend,
 * out[6] list entries the forward sorted (all keys with GS_F_FULL_SORT),
 * out[7] (warp, splat) entries the forward blend walked (after the per-warp
 * compaction), out[8] / out[9] (warp, splat) entries of the backward blend with
 * a pixel in the splat's alpha box / with a contributing pixel, out[10]
 * visible (view, Gaussian) pairs N_vis (non-empty tile rectangle). */
#define GS_N_COUNTERS 11
int gs_frames_counters(gs_frames* fr, int64_t out[GS_N_COUNTERS]);

/* D-SSIM loss term and its image gradient for ONE view, allocating nothing.
 * (The paper has no counterpart: this is a deployment variant of the D-SSIM
 * part of GS_LOSS_L1_DSSIM.)  It is for callers that cannot call cudaMalloc
 * at the point where they need the loss: serving loops that fix their device
 * footprint at start-up (a later cudaMalloc can fail once other tenants have
 * taken the memory, and it synchronises the device, stalling every stream),
 * real-time loops that forbid allocator calls after initialisation, and hosts
 * that own all device memory and give the library only the buffers it
 * passes.  Its scratch is a file-scope device array that every GPU loading
 * the library holds until the process exits: 11 planes of
 * GS_DSSIM_STATIC_MAX_PIXELS floats (11.5 MiB), a safe upper bound on what
 * one call uses (9 planes for the SSIM partials plus 3 floats per 32x32 tile
 * for the per-tile SSIM sums).
 *   image, target  device, planar float32 [3][height][width];
 *   dl_dimage      device output [3][height][width]: w_dssim * d(1 - SSIM)/dC;
 *   loss           device float64 [1], nullable: w_dssim * (1 - mean SSIM).
 * width * height above GS_DSSIM_STATIC_MAX_PIXELS is rejected with GS_EINVAL
 * before any device work.  The first call on a device resolves the scratch's
 * device address and uploads the filter window (once per device, with that
 * device current); make that first call before any stream capture.  All
 * calls share the one scratch array, which keeps the last call's contents:
 * calls whose GPU work overlaps (other streams, other host threads) race and
 * must be serialised by the caller.  No scratch needs clearing: each call
 * writes every scratch value it reads. */
#define GS_DSSIM_STATIC_MAX_PIXELS (512 * 512)
int gs_loss_dssim_static(const float* image, const float* target, int width, int height, float w_dssim,
                         float* dl_dimage, double* loss, void* stream);

/* Thread-local message describing the calling thread's last error. */
const char* gs_last_error(void);

/* Library version string. */
const char* gs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSPLAT_H */
