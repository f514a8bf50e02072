// gs_internal.cuh - device-side data layout and helpers shared by the
// renderer's kernels (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "gsplat.h"

#define GS_TILE 16
#define GS_TILE_PIX (GS_TILE * GS_TILE)

// Per-view constants the kernels read (built on device from the float64 pose
// so that CUDA-graph replays see pose updates made by gs_pose_step).
struct ViewDev {
    float fx, fy, cx, cy;
    int W, H, gw, gh;
    int tile_base;          // global id of the view's first tile
    int pad0;
    long long img_off;      // float offset of the planar [3][H][W] image
    long long pix_off;      // offset of the view's [H][W] per-pixel planes
    float Rf[9], tf[3];     // pose rounded to FP32 (key path and value path)
    float oc[3];            // camera centre -R^T t (FP32)
    float limx, limy;       // frustum-clamp limits on x/z and y/z
    float inv_npix3;        // 1 / (3 H W)
    float Rlo[9], tlo[3];   // pose - (Rf, tf): with them the pose is exact to ~2^-48
};

// Per-(view, Gaussian) splat record written by the forward preprocess.
//   A  = (mu_hat.x, mu_hat.y, conic.a, conic.b)
//   B  = (conic.c, opacity, colour.r, colour.g)
//   Cb = colour.b
//   rect = (x0 | y0 << 16, x1 | y1 << 16); x1 <= x0 marks a culled splat
//   depth = key-path camera-space z
//   Mlo = mu_hat - A.xy: the projected mean to ~1e-9 px is A.xy + Mlo, which
//         the blends apply in tile-relative coordinates (A.xy itself is the
//         FP32 key-path value that decides the tile rectangle)
struct SplatArrays {
    float4* A;
    float2* Mlo;
    float4* B;
    float* Cb;
    uint2* rect;
    float* depth;
    int* radius;
};

// Per-(view, Gaussian) 2D gradients accumulated by the backward blend.
//   gA = (dmu.x, dmu.y, dconic.a, dconic.b), gB = (dconic.c, dopacity, dcol.r, dcol.g), gC = dcol.b
struct Grad2DArrays {
    float4* gA;
    float4* gB;
    float* gC;
};

struct SceneDev {
    int n;
    int sh_degree;
    const float* means;
    const float* scales;
    const float* quats;
    const float* opac;
    const float* sh;
};

struct RenderParams {
    float bg[3];
    float z_near, eps2d, clamp_factor, alpha_min, alpha_max, t_min;
};

// ------------------------------------------------------------ status codes
// Device status word bits (OR-ed); the host maps them to GS_E* codes.
#define GS_DEV_OVERFLOW 1
#define GS_DEV_BADRANGE 2

__device__ __forceinline__ void gs_set_status(int* status, int bit) {
    if (status) atomicOr(status, bit);
}

// ------------------------------------------------------------ small helpers
__device__ __forceinline__ uint32_t pack16(int lo, int hi) {
    return (uint32_t)(lo & 0xffff) | ((uint32_t)(hi & 0xffff) << 16);
}

__device__ __forceinline__ int view_of_tile(const int* tile_base, int n_views, int t) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {  // last v with tile_base[v] <= t
        int mid = (lo + hi + 1) >> 1;
        if (tile_base[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// 2^x with the SFU's approximate exponential (flush-to-zero).
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

#define GS_LOG2E 1.4426950408889634f

// Approximate reciprocal (MUFU); for arguments in normal range.
__device__ __forceinline__ float fast_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------ kernel entry
// Host-side launchers (defined in the .cu files).
namespace gs {

// Runs set() the first time it is reached on the current device (kernel
// attributes such as the dynamic shared-memory limit are per device); safe to
// reach from several threads, where set() may run more than once (it only
// sets the same values).
template <class F>
inline void once_per_device(std::atomic<unsigned long long>& done, F set) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    set(dev);
    done.fetch_or(bit, std::memory_order_acq_rel);
}

void launch_setup_views(const gs_view* dummy, int n_views, const double* poses, ViewDev* views_dev,
                        const RenderParams& rp, cudaStream_t s);

// [i_begin, i_end): the Gaussians this launch covers (i_end < 0: to the end)
void launch_preprocess_fwd(const SceneDev& sc, int threads, int n_views, const ViewDev* views, const RenderParams& rp,
                           SplatArrays sp, uint32_t* tile_counts, cudaStream_t s, int i_begin = 0, int i_end = -1);

void launch_scan_u32(const uint32_t* in, uint32_t* out, int n, void* tmp, size_t tmp_bytes, cudaStream_t s);
size_t scan_tmp_bytes(int n);

// Per-CTA (tile, offset) lists of the count pass, read back by the scatter
// pass of the same chunking: entries needed for n Gaussians in chunks of
// `chunk` over views with total_tiles tiles; plus one length per (view, chunk).
size_t cta_list_entries(int n, int chunk, int total_tiles);

void launch_scatter_keys(int n, int chunk, int n_views, const ViewDev* views, SplatArrays sp, const uint32_t* starts,
                         uint32_t* cursor, const uint2* cta_lists, const uint32_t* cta_list_len,
                         unsigned long long* keys, uint32_t cap, int* status, cudaStream_t s);

void launch_count_tiles(int n, int chunk, int n_views, const ViewDev* views, const uint2* rect,
                        uint32_t* tile_counts, uint2* cta_lists, uint32_t* cta_list_len, cudaStream_t s);

// lists: [3][n_tiles] work lists; counters: 6 words (list lengths, work cursors)
void launch_segment_sort(int n_tiles, const uint32_t* starts, unsigned long long* keys,
                         unsigned long long* tmp_keys, uint32_t* sorted_idx, uint32_t cap, uint32_t* lists,
                         uint32_t* counters, cudaStream_t s);

void launch_blend_fwd(int n_tiles, int n_views, const int* tile_base, const ViewDev* views,
                      const RenderParams& rp, SplatArrays sp, int n, const uint32_t* starts,
                      const uint32_t* sorted_idx, uint32_t cap, float* image, float* T_final,
                      uint32_t* n_contrib, const float* target, float* tile_loss, unsigned long long* counters,
                      cudaStream_t s);

void launch_blend_fwd_lazy(int n_tiles, int sort_chunk, int px_per_thread, int n_views, const int* tile_base,
                           const ViewDev* views, const RenderParams& rp, SplatArrays sp, int n, const uint32_t* starts,
                           unsigned long long* keys, unsigned long long* tmp, uint32_t* sorted_idx,
                           uint32_t* sorted_count, uint32_t cap, float* image, float* T_final, uint32_t* n_contrib,
                           const float* target, float* tile_loss, unsigned long long* counters, cudaStream_t s);

void launch_loss_finalize(int n_views, const ViewDev* views, const float* tile_loss, double w, const double* addend,
                          double* loss_out, cudaStream_t s);

void launch_blend_bwd(int n_tiles, int n_views, const int* tile_base, const ViewDev* views,
                      const RenderParams& rp, SplatArrays sp, int n, const uint32_t* starts,
                      const uint32_t* sorted_idx, uint32_t cap, const float* image, const float* T_final,
                      const uint32_t* n_contrib, int loss_kind, float w_l1, float l1_mask_t, const float* target,
                      const float* dldc, Grad2DArrays g2d, float* tile_loss, unsigned long long* counters,
                      int px_per_thread, cudaStream_t s);

// [i_begin, i_end): the Gaussians this launch covers (i_begin a multiple of the
// block, 128; i_end < 0: to the end); n_blocks bounds the launch's blocks
void launch_preprocess_bwd(const SceneDev& sc, int n_views, const ViewDev* views, const RenderParams& rp,
                           SplatArrays sp, Grad2DArrays g2d, gs_grads grads, double* pose_partials,
                           int n_blocks, cudaStream_t s, int i_begin = 0, int i_end = -1);
int preprocess_bwd_blocks(int n);

// scratch: pose_reduce_groups(n_blocks) * n_views * 6 doubles
int pose_reduce_groups(int n_blocks);
void launch_pose_reduce(int n_views, int n_blocks, const double* partials, double* scratch, double* pose_grad,
                        cudaStream_t s);

void launch_pose_adam(int n_views, double* poses, double* m, double* v, const double* grad, double lr,
                      double b1, double b2, double eps, int step, int param, cudaStream_t s);


void launch_gather_poses(int n, const int* slot_of, const double* slot_poses, double* packed, cudaStream_t s);
void launch_pose_adam_slots(int n, const int* slot_of, double* poses, double* m, double* v, const double* grad,
                            const int* steps, const double* lrs, double b1, double b2, double eps, int param,
                            cudaStream_t s);

// Row arrays moved together by the opacity compaction (gs_reg.cu).
#define GS_COMPACT_MAX 24
struct CompactArrays {
    int count;
    const float* src[GS_COMPACT_MAX];
    float* dst[GS_COMPACT_MAX];
    int width[GS_COMPACT_MAX];
};
int regularize_blocks(int n);
void launch_regularize(int n, const float* scales, const float* opac, float r, float w_an, float w_op,
                       float* g_scales, float* g_opac, double* partial, double* loss, cudaStream_t s);
void launch_select_kth(int n, const float* x, uint32_t k, uint32_t* state, uint32_t* hist, cudaStream_t s);
void launch_compact(int n, const float* opac, float thr, const CompactArrays& ca, uint32_t* counts,
                    uint32_t* total, cudaStream_t s);

// Gaussians from a depth map (gs_init.cu).
void launch_unproject(int W, int H, int stride, float fx, float fy, float cx, float cy, const float* depth,
                      const float* image, float* pts, float* cols, float* key, cudaStream_t s);
void launch_knn_mean(int n, const float* pts, int k, float* out, cudaStream_t s);
void launch_init_raw(int n, const float* pts, const float* cols, const float* dist, float min_scale, float logit_o,
                     float* means, float* log_scales, float* quats, float* logit_opac, float* sh, cudaStream_t s);

int spatial_order_blocks(int n);
void launch_spatial_keys(int n, const float* means, float* part, unsigned long long* keys, uint32_t* starts,
                         cudaStream_t s);
void launch_gather_rows(int n, const uint32_t* perm, const CompactArrays& ca, cudaStream_t s);

// One parameter group of the Gaussian Adam update (gs_pose.cu).
struct AdamGroup {
    float* p;          // raw parameter
    const float* g;    // gradient w.r.t. the activated parameter
    float* m;
    float* v;
    float* act;        // activated output (scales / opacities) or nullptr
    int width;         // floats per Gaussian
    int used;          // leading floats per Gaussian that are optimised
    int act_kind;      // 0 none, 1 exp, 2 sigmoid
    float lr;
    float lr_tail;     // learning rate of elements >= tail_from (SH beyond DC)
    int tail_from;
};
void launch_gaussian_adam(int64_t n, const AdamGroup* groups, int n_groups, float b1, float b2, float eps, int step,
                          cudaStream_t s);

// Adds the number of (view, Gaussian) pairs with a non-empty tile rectangle to *count.
void launch_count_visible(size_t vn, const uint2* rect, unsigned long long* count, cudaStream_t s);
// Returns the error of the per-device window upload (nothing is launched then).
cudaError_t launch_dssim(int n_views, const gs_view* views_host, const long long* img_off_host, const float* image,
                         const float* target, float w_dssim, float* dldc_out, double* loss_out, float* tmp,
                         cudaStream_t s);
// Uploads the D-SSIM filter window to the current device once (thread-safe).
cudaError_t ensure_dssim_window();

// Records a message for gs_last_error() and returns `code` (defined in gs_api.cu).
int set_error(int code, const char* msg);

// Accessors of the opaque ABI objects (gs_api.cu).
int scene_count(const gs_scene* scene);
uint32_t frames_num_keys(const gs_frames* fr);
// Device bytes the frames' workspaces hold (they grow on demand and are kept).
size_t frames_device_bytes(const gs_frames* fr);

// Slices of the Gaussians for a step whose parameters arrive from and whose
// gradients return to host memory: the forward preprocess of slice c waits
// for ready[c] (its parameters are on the device), and the backward records
// done[c] on the stream once slice c's gradients are final, so that copies of
// one slice overlap the preprocess of the others.  bounds[c] are multiples of
// 256 (a multiple of the backward preprocess's block), bounds[n_slices] = N.
// Odd slices run on `aux` (forked from and joined back into the caller's
// stream around each sliced pass), so that one slice's last wave overlaps the
// next slice's first.
#define GS_MAX_SLICES 8
struct SlicePipe {
    int n_slices = 0;
    int bounds[GS_MAX_SLICES + 1] = {};
    cudaEvent_t ready[GS_MAX_SLICES] = {};
    cudaEvent_t done[GS_MAX_SLICES] = {};
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

// Forward / backward with optional per-view float offsets of the planar
// images (img_offs == nullptr: packed layout).  Used by the serving loop,
// whose views keep their images in fixed per-slot storage.
int render_forward_impl(gs_ctx* ctx, const gs_scene* scene, int n_views, const gs_view* views,
                        const long long* img_offs, const double* poses, const gs_render_opts* opts, gs_frames* fr,
                        float* image, const float* target, double* loss_out, cudaStream_t s,
                        const SlicePipe* pipe = nullptr);
int render_backward_impl(gs_ctx* ctx, const gs_scene* scene, int n_views, const gs_view* views,
                         const long long* img_offs, const double* poses, const gs_render_opts* opts, gs_frames* fr,
                         const float* image, const gs_loss* loss, gs_grads* grads, double* pose_grad, cudaStream_t s,
                         const SlicePipe* pipe = nullptr);

}  // namespace gs
