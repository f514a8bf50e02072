// gs_api.cu - the C ABI: contexts, scenes, forward state, and the
// orchestration of the kernels of one forward / backward pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gs_internal.cuh"

// ------------------------------------------------------------ errors
static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

namespace gs {
int set_error(int code, const char* msg);
}

namespace gs {
int set_error(int code, const char* msg) {
    g_err = msg ? msg : "";
    return code;
}
}  // namespace gs

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? GS_ENOMEM : GS_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                           \
    } while (0)

#define CK_LAUNCH()                                                                            \
    do {                                                                                       \
        cudaError_t e_ = cudaGetLastError();                                                   \
        if (e_ != cudaSuccess)                                                                 \
            return fail(GS_ECUDA, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// ------------------------------------------------------------ objects
// Kernel kinds reported by the profiler.
enum ProfKind {
    PK_SETUP = 0, PK_PRE_FWD, PK_SCAN, PK_SCATTER, PK_SORT, PK_BLEND_FWD, PK_LOSS, PK_DSSIM, PK_BLEND_BWD,
    PK_PRE_BWD, PK_POSE_REDUCE, PK_POSE_ADAM, PK_MEMSET, PK_COUNT_TILES, PK_GAUSS_ADAM, PK_REG, PK_PRUNE, PK_INIT,
    PK_COUNT
};
static const char* kProfNames[PK_COUNT] = {"setup_views", "preprocess_fwd", "scan_tiles", "scatter_keys",
                                           "segment_sort", "blend_fwd", "loss_finalize", "dssim", "blend_bwd",
                                           "preprocess_bwd", "pose_reduce", "pose_adam", "memset", "count_tiles",
                                           "gaussian_adam", "regularize", "prune", "init_gaussians"};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};

struct gs_ctx {
    int device = 0;
    int* status = nullptr;          // device status word
    long long* pinned = nullptr;    // small pinned host scratch
    bool prof = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    double prof_ms[PK_COUNT] = {};
    long long prof_n[PK_COUNT] = {};
    long long launches = 0;         // kernels launched by this context
    gs_tuning tune{4096, 2048, 256, 1, 1};  // result-neutral launch parameters
    // scratch of the regularisers and the pruning select/compaction
    void* reg_scratch = nullptr;
    size_t reg_cap = 0;
};

static cudaEvent_t pool_event(gs_ctx* c) {
    if (!c->pool.empty()) { cudaEvent_t e = c->pool.back(); c->pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records an event pair around one kernel launch on the launching stream.
struct ProfScope {
    gs_ctx* c;
    cudaStream_t s;
    int idx = -1;
    ProfScope(gs_ctx* c_, int kind, cudaStream_t s_, int n_kernels) : c(c_), s(s_) {
        if (c) c->launches += n_kernels;
        if (!c || !c->prof) return;
        ProfRec r{kind, pool_event(c), pool_event(c)};
        cudaEventRecord(r.a, s);
        c->recs.push_back(r);
        idx = (int)c->recs.size() - 1;
    }
    ~ProfScope() {
        if (idx >= 0) cudaEventRecord(c->recs[idx].b, s);
    }
};
#define PROF(kind, nk) ProfScope prof_scope_##kind(ctx, kind, s, nk)

struct gs_scene {
    SceneDev d{};
    bool owned = false;
};

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;  // elements
    int ensure(size_t n, bool allow_grow, const char* what) {
        if (n <= cap && p) return GS_OK;
        if (!allow_grow) return fail(GS_EOVERFLOW, "%s: capacity %zu < %zu in no-sync mode", what, cap, n);
        size_t nc = std::max<size_t>(n + n / 4, 256);
        T* q = nullptr;
        cudaError_t e = cudaMalloc(&q, nc * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            nc = n;
            e = cudaMalloc(&q, nc * sizeof(T));
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(GS_ENOMEM, "%s: cudaMalloc of %zu bytes failed", what, nc * sizeof(T));
            }
        }
        if (p) cudaFree(p);
        p = q;
        cap = nc;
        return GS_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// Device tables of one view configuration (intrinsics and sizes); the
// pose-dependent fields are refreshed on the device by every forward.  Each
// table keeps its own pinned staging so that switching configurations never
// waits for an earlier upload.
struct ViewTable {
    std::vector<gs_view> views;
    std::vector<long long> offs;      // custom image offsets (empty: packed)
    std::vector<ViewDev> vdev_host;
    std::vector<int> tile_base_host;
    ViewDev* vdev_pinned = nullptr;
    int* tb_pinned = nullptr;
    DevBuf<ViewDev> vdev;
    DevBuf<int> tile_base;
    size_t pinned_cap = 0;
    int total_tiles = 0;
    long long total_pixels = 0;
    long long total_image = 0;
    void release() {
        vdev.release();
        tile_base.release();
        if (vdev_pinned) cudaFreeHost(vdev_pinned);
        if (tb_pinned) cudaFreeHost(tb_pinned);
        vdev_pinned = nullptr;
        tb_pinned = nullptr;
        pinned_cap = 0;
    }
};

static const size_t kMaxViewTables = 64;

struct gs_frames {
    gs_ctx* ctx = nullptr;
    // gs_step with host buffers: the stream that uploads the parameters and the
    // loss input while the forward runs (fork: after the caller's queued work;
    // join: before the backward) and the stream that downloads the image and
    // the gradients while the backward runs
    cudaStream_t side = nullptr, down = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // ... the events of its Gaussian slices (parameters uploaded, gradients
    // final), of the rendered image, and of the end of the downloads
    gs::SlicePipe pipe;
    cudaEvent_t ev_down = nullptr, ev_img = nullptr;
    // launch configuration of the last forward
    int n_views = 0;
    int n = 0;
    int total_tiles = 0;
    long long total_pixels = 0;
    long long total_image = 0;
    uint32_t n_keys = 0;
    bool have_forward = false;
    std::vector<ViewTable*> tables;   // cache of view configurations
    size_t evict_next = 0;            // next entry to recycle when the cache is full
    ViewTable* cur = nullptr;         // configuration of the last forward
    std::vector<gs_view> views_host;
    std::vector<ViewDev> vdev_host;
    DevBuf<ViewDev> vdev;             // aliases cur->vdev (not owned)
    DevBuf<int> tile_base;            // aliases cur->tile_base (not owned)
    // per (view, Gaussian)
    DevBuf<float4> A, B, gA, gB;
    DevBuf<float> Cb, depth, gC;
    // leading (view, Gaussian) records of gA/gB/gC known to be zero: the
    // backward preprocess clears every record it consumes, so after a complete
    // backward the next one needs no clearing pass over the records it uses
    size_t g2d_zero = 0;
    DevBuf<uint2> rect;
    DevBuf<float2> Mlo;
    DevBuf<int> radius;
    // per tile
    DevBuf<uint32_t> counts, starts, cursor, scan_tmp, sort_lists, sort_counters, sorted_count;
    DevBuf<uint2> cta_lists;          // per (view, chunk) CTA: (tile, offset) of its keys in the tile
    DevBuf<uint32_t> cta_list_len;
    bool full_sort = false;           // the last forward sorted whole lists
    DevBuf<float> tile_loss;
    // per key
    DevBuf<unsigned long long> keys, tmp_keys;
    DevBuf<uint32_t> sorted_idx;
    // per pixel
    DevBuf<float> T_final;
    DevBuf<uint32_t> n_contrib;
    // backward
    DevBuf<double> pose_partials;
    DevBuf<float> dldc_ssim, ssim_tmp;
    bool have_dssim_grad = false;     // dldc_ssim holds the last backward's D-SSIM dL/dC
    DevBuf<long long> img_off_dev;
    DevBuf<double> loss_tmp;
    DevBuf<unsigned long long> counters;  // [8] pair / entry counters
    // gs_step staging (host I/O and fresh gradients)
    DevBuf<float> st_params, st_target, st_image, st_grads;
    DevBuf<double> st_poses, st_pose_grad, st_loss;

    SplatArrays splats() {
        SplatArrays s;
        s.A = A.p; s.Mlo = Mlo.p; s.B = B.p; s.Cb = Cb.p; s.rect = rect.p; s.depth = depth.p; s.radius = radius.p;
        return s;
    }
    Grad2DArrays g2d() {
        Grad2DArrays g;
        g.gA = gA.p; g.gB = gB.p; g.gC = gC.p;
        return g;
    }
    void release() {
        DevBuf<float4>* f4[] = {&A, &B, &gA, &gB};
        for (auto* b : f4) b->release();
        DevBuf<float>* f1[] = {&Cb, &depth, &gC, &tile_loss, &T_final, &dldc_ssim, &ssim_tmp};
        for (auto* b : f1) b->release();
        rect.release(); Mlo.release(); radius.release(); counts.release(); starts.release(); cursor.release(); scan_tmp.release();
        cta_lists.release(); cta_list_len.release();
        sort_lists.release(); sort_counters.release(); sorted_count.release();
        keys.release(); tmp_keys.release(); sorted_idx.release(); n_contrib.release(); pose_partials.release();
        loss_tmp.release(); counters.release();
        st_params.release(); st_target.release(); st_image.release(); st_grads.release();
        st_poses.release(); st_pose_grad.release(); st_loss.release();
        img_off_dev.release();
        for (ViewTable* t : tables) { t->release(); delete t; }
        tables.clear();
        cur = nullptr;
        vdev.p = nullptr; tile_base.p = nullptr;
    }
};

static const int kViewChunk = 64;  // views per preprocess launch (bounds shared memory)
static const size_t kHostSlices = 8;  // Gaussian slices of a gs_step with host buffers (at most GS_MAX_SLICES)

// ------------------------------------------------------------ helpers
static int check_scene(const gs_scene* sc) {
    if (!sc) return fail(GS_EINVAL, "scene is NULL");
    if (sc->d.n < 0) return fail(GS_EINVAL, "negative Gaussian count");
    if (sc->d.sh_degree < 0 || sc->d.sh_degree > 3) return fail(GS_EINVAL, "sh_degree %d not in 0..3", sc->d.sh_degree);
    if (sc->d.n > 0 && (!sc->d.means || !sc->d.scales || !sc->d.quats || !sc->d.opac || !sc->d.sh))
        return fail(GS_EINVAL, "scene has a NULL parameter array");
    if (reinterpret_cast<uintptr_t>(sc->d.quats) % 16 != 0)
        return fail(GS_EINVAL, "quats must be 16-byte aligned (read as float4)");
    return GS_OK;
}

static int check_views(int n_views, const gs_view* views) {
    if (n_views < 0) return fail(GS_EINVAL, "negative view count");
    if (n_views > 0 && !views) return fail(GS_EINVAL, "views is NULL");
    for (int v = 0; v < n_views; v++) {
        const gs_view& w = views[v];
        if (w.width <= 0 || w.height <= 0 || w.width > 16 * 4095 || w.height > 16 * 4095)
            return fail(GS_EINVAL, "view %d: bad size %dx%d", v, w.width, w.height);
        if (!(w.fx > 0.0f) || !(w.fy > 0.0f)) return fail(GS_EINVAL, "view %d: focal lengths must be > 0", v);
    }
    return GS_OK;
}

static RenderParams make_params(const gs_render_opts* o) {
    RenderParams rp;
    for (int k = 0; k < 3; k++) rp.bg[k] = o->bg[k];
    rp.z_near = o->z_near; rp.eps2d = o->eps2d; rp.clamp_factor = o->clamp_factor;
    rp.alpha_min = o->alpha_min; rp.alpha_max = o->alpha_max; rp.t_min = o->t_min;
    return rp;
}

static bool same_views(const std::vector<gs_view>& a, int n, const gs_view* b) {
    if ((int)a.size() != n) return false;
    for (int v = 0; v < n; v++)
        if (memcmp(&a[v], &b[v], sizeof(gs_view)) != 0) return false;
    return true;
}

static bool same_offs(const std::vector<long long>& a, int n, const long long* b) {
    if (!b) return a.empty();
    if ((int)a.size() != n) return false;
    for (int v = 0; v < n; v++)
        if (a[v] != b[v]) return false;
    return true;
}

// Selects (or builds and uploads) the device tables of a view configuration.
static int upload_views(gs_frames* fr, int n_views, const gs_view* views, const long long* offs, bool allow_grow,
                        cudaStream_t s) {
    ViewTable* hit = nullptr;
    if (fr->cur && same_views(fr->cur->views, n_views, views) && same_offs(fr->cur->offs, n_views, offs)) hit = fr->cur;
    for (size_t k = 0; !hit && k < fr->tables.size(); k++)
        if (same_views(fr->tables[k]->views, n_views, views) && same_offs(fr->tables[k]->offs, n_views, offs))
            hit = fr->tables[k];
    if (!hit) {
        if (!allow_grow) return fail(GS_EOVERFLOW, "new view configuration in no-sync mode (run it once without GS_F_NO_SYNC)");
        ViewTable* t = nullptr;
        if (fr->tables.size() >= kMaxViewTables) {
            // recycle an entry other than the current one; its pinned staging
            // may still feed a pending upload, so drain the stream first
            CK(cudaStreamSynchronize(s));
            for (size_t k = 0; k < fr->tables.size(); k++) {
                ViewTable* c = fr->tables[(fr->evict_next + k) % fr->tables.size()];
                if (c != fr->cur) { t = c; fr->evict_next = (fr->evict_next + k + 1) % fr->tables.size(); break; }
            }
        }
        if (!t) {
            t = new (std::nothrow) ViewTable();
            if (!t) return fail(GS_ENOMEM, "host allocation failed");
            fr->tables.push_back(t);
        }
        t->views.assign(views, views + n_views);
        t->offs.clear();
        if (offs) t->offs.assign(offs, offs + n_views);
        t->vdev_host.assign(n_views, ViewDev{});
        t->tile_base_host.assign(n_views + 1, 0);
        long long img = 0, pix = 0;
        int tb = 0;
        for (int v = 0; v < n_views; v++) {
            ViewDev& d = t->vdev_host[v];
            const gs_view& w = views[v];
            d.fx = w.fx; d.fy = w.fy; d.cx = w.cx; d.cy = w.cy;
            d.W = w.width; d.H = w.height;
            d.gw = (w.width + GS_TILE - 1) / GS_TILE;
            d.gh = (w.height + GS_TILE - 1) / GS_TILE;
            d.tile_base = tb;
            d.img_off = offs ? offs[v] : img;
            d.pix_off = pix;
            t->tile_base_host[v] = tb;
            tb += d.gw * d.gh;
            img = offs ? std::max(img, offs[v] + 3LL * w.width * w.height) : img + 3LL * w.width * w.height;
            pix += (long long)w.width * w.height;
        }
        t->tile_base_host[n_views] = tb;
        t->total_tiles = tb;
        t->total_pixels = pix;
        t->total_image = img;
        int rc;
        if ((rc = t->vdev.ensure(std::max(n_views, 1), true, "views")) ||
            (rc = t->tile_base.ensure(n_views + 1, true, "tile_base")))
            return rc;
        if (t->pinned_cap < (size_t)n_views + 1) {
            if (t->vdev_pinned) cudaFreeHost(t->vdev_pinned);
            if (t->tb_pinned) cudaFreeHost(t->tb_pinned);
            t->vdev_pinned = nullptr;
            t->tb_pinned = nullptr;
            const size_t c = (size_t)n_views + 16;
            cudaError_t e = cudaMallocHost(&t->vdev_pinned, sizeof(ViewDev) * c);
            if (e == cudaSuccess) e = cudaMallocHost(&t->tb_pinned, sizeof(int) * (c + 1));
            if (e != cudaSuccess) { t->pinned_cap = 0; return fail(GS_ENOMEM, "pinned allocation failed"); }
            t->pinned_cap = c;
        }
        memcpy(t->vdev_pinned, t->vdev_host.data(), sizeof(ViewDev) * n_views);
        memcpy(t->tb_pinned, t->tile_base_host.data(), sizeof(int) * (n_views + 1));
        if (n_views > 0)
            CK(cudaMemcpyAsync(t->vdev.p, t->vdev_pinned, sizeof(ViewDev) * n_views, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(t->tile_base.p, t->tb_pinned, sizeof(int) * (n_views + 1), cudaMemcpyHostToDevice, s));
        hit = t;
    }
    fr->cur = hit;
    fr->views_host = hit->views;
    fr->vdev_host = hit->vdev_host;
    fr->vdev.p = hit->vdev.p; fr->vdev.cap = hit->vdev.cap;
    fr->tile_base.p = hit->tile_base.p; fr->tile_base.cap = hit->tile_base.cap;
    fr->total_tiles = hit->total_tiles;
    fr->total_pixels = hit->total_pixels;
    fr->total_image = hit->total_image;
    return GS_OK;
}

static int ensure_pair_buffers(gs_frames* fr, size_t vn, bool grow) {
    int rc;
    if ((rc = fr->A.ensure(vn, grow, "splat A")) || (rc = fr->Mlo.ensure(vn, grow, "splat Mlo")) ||
        (rc = fr->B.ensure(vn, grow, "splat B")) ||
        (rc = fr->Cb.ensure(vn, grow, "splat Cb")) || (rc = fr->rect.ensure(vn, grow, "splat rect")) ||
        (rc = fr->depth.ensure(vn, grow, "splat depth")) || (rc = fr->radius.ensure(vn, grow, "splat radius")))
        return rc;
    return GS_OK;
}

static int ensure_tile_buffers(gs_frames* fr, size_t tiles, bool grow) {
    int rc;
    if ((rc = fr->counts.ensure(tiles + 1, grow, "tile counts")) || (rc = fr->starts.ensure(tiles + 1, grow, "tile starts")) ||
        (rc = fr->cursor.ensure(tiles + 1, grow, "tile cursor")) || (rc = fr->tile_loss.ensure(tiles + 1, grow, "tile loss")) ||
        (rc = fr->scan_tmp.ensure(gs::scan_tmp_bytes((int)tiles + 1) / 4 + 1, grow, "scan tmp")) ||
        (rc = fr->sort_lists.ensure(3 * (tiles + 1), grow, "sort lists")) ||
        (rc = fr->sort_counters.ensure(8, grow, "sort counters")) ||
        (rc = fr->sorted_count.ensure(tiles + 1, grow, "sorted count")))
        return rc;
    return GS_OK;
}

static int ensure_key_buffers(gs_frames* fr, size_t keys, bool grow) {
    int rc;
    if ((rc = fr->keys.ensure(keys, grow, "keys")) || (rc = fr->tmp_keys.ensure(keys, grow, "tmp keys")) ||
        (rc = fr->sorted_idx.ensure(keys, grow, "sorted idx")))
        return rc;
    return GS_OK;
}

// ------------------------------------------------------------ ABI
extern "C" {

const char* gs_last_error(void) { return g_err.c_str(); }

const char* gs_version(void) { return "gsplat-gb300 0.1 (sm_103a)"; }

void gs_default_opts(gs_render_opts* o) {
    if (!o) return;
    o->bg[0] = o->bg[1] = o->bg[2] = 0.0f;
    o->z_near = 0.2f;
    o->eps2d = 0.3f;
    o->clamp_factor = 1.3f;
    o->alpha_min = 1.0f / 255.0f;
    o->alpha_max = 0.99f;
    o->t_min = 1e-4f;
    o->flags = 0u;
}

int gs_ctx_create(int device, gs_ctx** out) {
    if (!out) return fail(GS_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(GS_EINVAL, "device %d out of range (%d devices)", device, ndev);
    CK(cudaSetDevice(device));
    gs_ctx* c = new (std::nothrow) gs_ctx();
    if (!c) return fail(GS_ENOMEM, "host allocation failed");
    c->device = device;
    cudaError_t e = cudaMalloc(&c->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->pinned, 64 * sizeof(long long));
    if (e != cudaSuccess) {
        if (c->status) cudaFree(c->status);
        delete c;
        return fail(GS_ECUDA, "context setup: %s", cudaGetErrorString(e));
    }
    *out = c;
    return GS_OK;
}

void gs_ctx_destroy(gs_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (const ProfRec& r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    if (c->status) cudaFree(c->status);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->reg_scratch) cudaFree(c->reg_scratch);
    delete c;
}

int gs_scene_borrow(const gs_scene_desc* d, gs_scene** out) {
    if (!d || !out) return fail(GS_EINVAL, "NULL argument");
    if (d->n < 0 || d->n > 0x7fffffff) return fail(GS_EINVAL, "Gaussian count %lld out of range", (long long)d->n);
    gs_scene* s = new (std::nothrow) gs_scene();
    if (!s) return fail(GS_ENOMEM, "host allocation failed");
    s->d.n = (int)d->n;
    s->d.sh_degree = d->sh_degree;
    s->d.means = d->means; s->d.scales = d->scales; s->d.quats = d->quats;
    s->d.opac = d->opacities; s->d.sh = d->sh;
    s->owned = false;
    int rc = check_scene(s);
    if (rc != GS_OK) { delete s; return rc; }
    *out = s;
    return GS_OK;
}

int gs_scene_load(gs_ctx* ctx, const gs_scene_desc* d, int src_on_device, gs_scene** out) {
    if (!ctx || !d || !out) return fail(GS_EINVAL, "NULL argument");
    if (d->n < 0 || d->n > 0x7fffffff) return fail(GS_EINVAL, "Gaussian count out of range");
    if (d->sh_degree < 0 || d->sh_degree > 3) return fail(GS_EINVAL, "sh_degree %d not in 0..3", d->sh_degree);
    if (d->n > 0 && (!d->means || !d->scales || !d->quats || !d->opacities || !d->sh))
        return fail(GS_EINVAL, "scene has a NULL parameter array");
    CK(cudaSetDevice(ctx->device));
    const size_t n = (size_t)d->n;
    const size_t bytes = n * sizeof(float) * (3 + 3 + 4 + 1 + 48);
    char* base = nullptr;
    if (n > 0) CK(cudaMalloc(&base, bytes));
    gs_scene* s = new (std::nothrow) gs_scene();
    if (!s) { if (base) cudaFree(base); return fail(GS_ENOMEM, "host allocation failed"); }
    float* p = reinterpret_cast<float*>(base);
    float* quats = p; float* means = quats + 4 * n; float* scales = means + 3 * n;
    float* opac = scales + 3 * n; float* sh = opac + n;
    const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (n > 0) {
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = cudaMemcpy(means, d->means, 3 * n * sizeof(float), kind);
        if (e == cudaSuccess) e = cudaMemcpy(scales, d->scales, 3 * n * sizeof(float), kind);
        if (e == cudaSuccess) e = cudaMemcpy(quats, d->quats, 4 * n * sizeof(float), kind);
        if (e == cudaSuccess) e = cudaMemcpy(opac, d->opacities, n * sizeof(float), kind);
        if (e == cudaSuccess) e = cudaMemcpy(sh, d->sh, 48 * n * sizeof(float), kind);
        if (e != cudaSuccess) {
            cudaFree(base);
            delete s;
            return fail(GS_ECUDA, "scene copy: %s", cudaGetErrorString(e));
        }
    }
    s->d.n = (int)n; s->d.sh_degree = d->sh_degree;
    s->d.means = means; s->d.scales = scales; s->d.quats = quats; s->d.opac = opac; s->d.sh = sh;
    s->owned = true;
    *out = s;
    return GS_OK;
}

void gs_scene_free(gs_scene* s) {
    if (!s) return;
    if (s->owned && s->d.quats) cudaFree(const_cast<float*>(s->d.quats));
    delete s;
}

int gs_frames_create(gs_ctx* ctx, gs_frames** out) {
    if (!ctx || !out) return fail(GS_EINVAL, "NULL argument");
    gs_frames* f = new (std::nothrow) gs_frames();
    if (!f) return fail(GS_ENOMEM, "host allocation failed");
    f->ctx = ctx;
    *out = f;
    return GS_OK;
}

void gs_frames_destroy(gs_frames* f) {
    if (!f) return;
    cudaSetDevice(f->ctx->device);
    cudaDeviceSynchronize();
    f->release();
    if (f->ev_fork) cudaEventDestroy(f->ev_fork);
    if (f->ev_join) cudaEventDestroy(f->ev_join);
    if (f->ev_down) cudaEventDestroy(f->ev_down);
    if (f->ev_img) cudaEventDestroy(f->ev_img);
    for (int c = 0; c < GS_MAX_SLICES; c++) {
        if (f->pipe.ready[c]) cudaEventDestroy(f->pipe.ready[c]);
        if (f->pipe.done[c]) cudaEventDestroy(f->pipe.done[c]);
    }
    if (f->pipe.fork) cudaEventDestroy(f->pipe.fork);
    if (f->pipe.join) cudaEventDestroy(f->pipe.join);
    if (f->pipe.aux) cudaStreamDestroy(f->pipe.aux);
    if (f->side) cudaStreamDestroy(f->side);
    if (f->down) cudaStreamDestroy(f->down);
    delete f;
}

int gs_frames_reserve(gs_frames* fr, int64_t keys, int64_t pairs, int64_t pixels, int64_t tiles) {
    if (!fr || keys < 0 || pairs < 0 || pixels < 0 || tiles < 0) return fail(GS_EINVAL, "bad reserve arguments");
    if (keys > 0xfffffff0LL) return fail(GS_EINVAL, "key capacity above 2^32");
    CK(cudaSetDevice(fr->ctx->device));
    int rc;
    if ((rc = ensure_pair_buffers(fr, (size_t)pairs, true))) return rc;
    if ((rc = fr->gA.ensure(pairs, true, "g2d A")) || (rc = fr->gB.ensure(pairs, true, "g2d B")) ||
        (rc = fr->gC.ensure(pairs, true, "g2d C")))
        return rc;
    if ((rc = ensure_tile_buffers(fr, (size_t)tiles, true))) return rc;
    if ((rc = ensure_key_buffers(fr, (size_t)keys, true))) return rc;
    if ((rc = fr->T_final.ensure(pixels, true, "T_final")) || (rc = fr->n_contrib.ensure(pixels, true, "n_contrib")))
        return rc;
    return GS_OK;
}

int gs_render_forward(gs_ctx* ctx, const gs_scene* scene, int n_views, const gs_view* views, const double* poses,
                      const gs_render_opts* opts, gs_frames* fr, float* image, const float* target, double* loss_out,
                      void* stream) {
    return gs::render_forward_impl(ctx, scene, n_views, views, nullptr, poses, opts, fr, image, target, loss_out,
                                   static_cast<cudaStream_t>(stream));
}

int gs_render_backward(gs_ctx* ctx, const gs_scene* scene, int n_views, const gs_view* views, const double* poses,
                       const gs_render_opts* opts, gs_frames* fr, const float* image, const gs_loss* loss,
                       gs_grads* grads, double* pose_grad, void* stream) {
    return gs::render_backward_impl(ctx, scene, n_views, views, nullptr, poses, opts, fr, image, loss, grads, pose_grad,
                                    static_cast<cudaStream_t>(stream));
}

}  // extern "C"

int gs::render_forward_impl(gs_ctx* ctx, const gs_scene* scene, int n_views, const gs_view* views,
                            const long long* img_offs, const double* poses, const gs_render_opts* opts, gs_frames* fr,
                            float* image, const float* target, double* loss_out, cudaStream_t s,
                            const SlicePipe* pipe) {
    if (!ctx || !fr || !opts) return fail(GS_EINVAL, "NULL ctx/frames/opts");
    if (fr->ctx != ctx) return fail(GS_EINVAL, "frames belong to another context");
    int rc;
    if ((rc = check_scene(scene)) || (rc = check_views(n_views, views))) return rc;
    if (n_views > 0 && (!poses || !image)) return fail(GS_EINVAL, "poses/image is NULL");
    const bool grow = !(opts->flags & GS_F_NO_SYNC);
    CK(cudaSetDevice(ctx->device));
    fr->have_forward = false;
    fr->have_dssim_grad = false;     // a D-SSIM gradient belongs to the forward it followed
    if ((rc = upload_views(fr, n_views, views, img_offs, grow, s))) return rc;
    const int n = scene->d.n;
    const size_t vn = (size_t)n * n_views;
    const int T = fr->total_tiles;
    if ((rc = ensure_pair_buffers(fr, std::max<size_t>(vn, 1), grow))) return rc;
    if ((rc = ensure_tile_buffers(fr, (size_t)T, grow))) return rc;
    if ((rc = fr->T_final.ensure(std::max<long long>(fr->total_pixels, 1), grow, "T_final")) ||
        (rc = fr->n_contrib.ensure(std::max<long long>(fr->total_pixels, 1), grow, "n_contrib")))
        return rc;
    if ((rc = ensure_key_buffers(fr, std::max<size_t>(fr->keys.cap, 1024), grow))) return rc;
    fr->n_views = n_views;
    fr->n = n;
    if (n_views == 0) { fr->have_forward = true; return GS_OK; }
    const RenderParams rp = make_params(opts);
    SplatArrays sp = fr->splats();
    if ((rc = fr->counters.ensure(12, grow, "counters"))) return rc;
    {
        const int chunk = ctx->tune.scatter_chunk;
        if ((rc = fr->cta_lists.ensure(std::max<size_t>(gs::cta_list_entries(n, chunk, T), 1), grow, "CTA tile lists")) ||
            (rc = fr->cta_list_len.ensure((size_t)((n + chunk - 1) / chunk) * n_views + 1, grow, "CTA list lengths")))
            return rc;
    }
    {
        PROF(PK_SETUP, 1);
        gs::launch_setup_views(views, n_views, poses, fr->vdev.p, rp, s);
    }
    CK_LAUNCH();
    {
        PROF(PK_MEMSET, 0);
        CK(cudaMemsetAsync(fr->counts.p, 0, sizeof(uint32_t) * (T + 1), s));
        CK(cudaMemsetAsync(fr->cursor.p, 0, sizeof(uint32_t) * (T + 1), s));
        CK(cudaMemsetAsync(fr->counters.p, 0, sizeof(unsigned long long) * 12, s));
    }
    for (int v0 = 0; v0 < n_views; v0 += kViewChunk) {
        const int nv = std::min(kViewChunk, n_views - v0);
        SplatArrays spc = sp;
        const size_t off = (size_t)v0 * n;
        spc.A += off; spc.B += off; spc.Cb += off; spc.rect += off; spc.depth += off; spc.radius += off;
        if (pipe && pipe->n_slices > 0) {
            // slice by slice, each as soon as its parameters are on the device
            PROF(PK_PRE_FWD, pipe->n_slices);
            CK(cudaEventRecord(pipe->fork, s));
            CK(cudaStreamWaitEvent(pipe->aux, pipe->fork, 0));
            for (int c = 0; c < pipe->n_slices; c++) {
                cudaStream_t cs = (c & 1) ? pipe->aux : s;
                if (v0 == 0) CK(cudaStreamWaitEvent(cs, pipe->ready[c], 0));
                gs::launch_preprocess_fwd(scene->d, ctx->tune.preprocess_threads, nv, fr->vdev.p + v0, rp, spc,
                                          nullptr, cs, pipe->bounds[c], pipe->bounds[c + 1]);
            }
            CK(cudaEventRecord(pipe->join, pipe->aux));
            CK(cudaStreamWaitEvent(s, pipe->join, 0));
        } else {
            PROF(PK_PRE_FWD, 1);
            gs::launch_preprocess_fwd(scene->d, ctx->tune.preprocess_threads, nv, fr->vdev.p + v0, rp, spc, nullptr, s);
        }
        CK_LAUNCH();
    }
    {
        PROF(PK_COUNT_TILES, 1);
        gs::launch_count_tiles(n, ctx->tune.scatter_chunk, n_views, fr->vdev.p, sp.rect, fr->counts.p,
                               fr->cta_lists.p, fr->cta_list_len.p, s);
    }
    CK_LAUNCH();
    if (opts->flags & GS_F_COUNT) {
        gs::launch_count_visible(vn, sp.rect, fr->counters.p + 11, s);
        CK_LAUNCH();
    }
    {
        PROF(PK_SCAN, (T + 1 > 4096) ? 3 : 1);
        gs::launch_scan_u32(fr->counts.p, fr->starts.p, T + 1, fr->scan_tmp.p, fr->scan_tmp.cap * 4, s);
    }
    CK_LAUNCH();
    if (grow) {
        CK(cudaMemcpyAsync(ctx->pinned, fr->starts.p + T, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const uint32_t K = *reinterpret_cast<uint32_t*>(ctx->pinned);
        fr->n_keys = K;
        if ((rc = ensure_key_buffers(fr, std::max<uint32_t>(K, 1), true))) return rc;
    }
    const uint32_t cap = (uint32_t)std::min<size_t>(fr->keys.cap, 0xffffffffu);
    {
        PROF(PK_SCATTER, 1);
        gs::launch_scatter_keys(n, ctx->tune.scatter_chunk, n_views, fr->vdev.p, sp, fr->starts.p, fr->cursor.p,
                                fr->cta_lists.p, fr->cta_list_len.p, fr->keys.p, cap,
                                ctx->status, s);
    }
    CK_LAUNCH();
    fr->full_sort = (opts->flags & GS_F_FULL_SORT) != 0;
    unsigned long long* counters = (opts->flags & GS_F_COUNT) ? fr->counters.p : nullptr;
    if (fr->full_sort) {
        {
            PROF(PK_SORT, 4);
            gs::launch_segment_sort(T, fr->starts.p, fr->keys.p, fr->tmp_keys.p, fr->sorted_idx.p, cap,
                                    fr->sort_lists.p, fr->sort_counters.p, s);
        }
        CK_LAUNCH();
        {
            PROF(PK_BLEND_FWD, 1);
            gs::launch_blend_fwd(T, n_views, fr->tile_base.p, fr->vdev.p, rp, sp, n, fr->starts.p, fr->sorted_idx.p,
                                 cap, image, fr->T_final.p, fr->n_contrib.p, target,
                                 target ? fr->tile_loss.p : nullptr, counters, s);
        }
        CK_LAUNCH();
    } else {
        PROF(PK_BLEND_FWD, 1);
        gs::launch_blend_fwd_lazy(T, ctx->tune.sort_chunk, ctx->tune.fwd_pixels_per_thread, n_views, fr->tile_base.p, fr->vdev.p, rp, sp, n, fr->starts.p, fr->keys.p,
                                  fr->tmp_keys.p, fr->sorted_idx.p, fr->sorted_count.p, cap, image, fr->T_final.p,
                                  fr->n_contrib.p, target, target ? fr->tile_loss.p : nullptr, counters, s);
        CK_LAUNCH();
    }
    if (target && loss_out) {
        PROF(PK_LOSS, 1);
        gs::launch_loss_finalize(n_views, fr->vdev.p, fr->tile_loss.p, 1.0, nullptr, loss_out, s);
        CK_LAUNCH();
    }
    fr->have_forward = true;
    return GS_OK;
}

int gs::render_backward_impl(gs_ctx* ctx, const gs_scene* scene, int n_views, const gs_view* views,
                             const long long* img_offs, const double* poses, const gs_render_opts* opts, gs_frames* fr,
                             const float* image, const gs_loss* loss, gs_grads* grads, double* pose_grad,
                             cudaStream_t s, const SlicePipe* pipe) {
    if (!ctx || !fr || !opts || !loss) return fail(GS_EINVAL, "NULL ctx/frames/opts/loss");
    int rc;
    if ((rc = check_scene(scene)) || (rc = check_views(n_views, views))) return rc;
    if (opts->flags & GS_F_RECOMPUTE) {
        // rebuild the forward state of these views in fr (into scratch image storage)
        long long n_img = 0;
        for (int v = 0; v < n_views; v++) {
            const long long end = (img_offs ? img_offs[v] : n_img) + 3LL * views[v].width * views[v].height;
            n_img = img_offs ? std::max(n_img, end) : end;
        }
        if ((rc = fr->st_image.ensure(std::max<long long>(n_img, 1), !(opts->flags & GS_F_NO_SYNC), "recompute image")))
            return rc;
        gs_render_opts o2 = *opts;
        o2.flags &= ~(uint32_t)GS_F_RECOMPUTE;
        if ((rc = gs::render_forward_impl(ctx, scene, n_views, views, img_offs, poses, &o2, fr, fr->st_image.p, nullptr,
                                          nullptr, s)))
            return rc;
    }
    if (!fr->have_forward || fr->n_views != n_views || fr->n != scene->d.n || !fr->cur ||
        !same_views(fr->views_host, n_views, views) || !same_offs(fr->cur->offs, n_views, img_offs))
        return fail(GS_EINVAL, "backward does not match the frames' last forward");
    if (n_views == 0) return GS_OK;
    if (!image) return fail(GS_EINVAL, "image is NULL");
    if (loss->kind == GS_LOSS_DLDC && !loss->dl_dimage) return fail(GS_EINVAL, "GS_LOSS_DLDC without dl_dimage");
    if (loss->kind < 0 || loss->kind > 3) return fail(GS_EINVAL, "unknown loss kind %d", loss->kind);
    const bool l1_kind = loss->kind == GS_LOSS_L1 || loss->kind == GS_LOSS_L1_DSSIM || loss->kind == GS_LOSS_L1_MASKED;
    if (l1_kind && !loss->target) return fail(GS_EINVAL, "loss needs a target");
    if (loss->kind == GS_LOSS_L1_MASKED && !(loss->mask_alpha >= 0.0f && loss->mask_alpha < 1.0f))
        return fail(GS_EINVAL, "mask_alpha must lie in [0, 1)");
    const bool grow = !(opts->flags & GS_F_NO_SYNC);
    CK(cudaSetDevice(ctx->device));
    const int n = scene->d.n;
    const size_t vn = (size_t)n * n_views;
    {
        const void* before[3] = {fr->gA.p, fr->gB.p, fr->gC.p};
        if ((rc = fr->gA.ensure(std::max<size_t>(vn, 1), grow, "g2d A")) ||
            (rc = fr->gB.ensure(std::max<size_t>(vn, 1), grow, "g2d B")) ||
            (rc = fr->gC.ensure(std::max<size_t>(vn, 1), grow, "g2d C"))) {
            fr->g2d_zero = 0;
            return rc;
        }
        if (before[0] != fr->gA.p || before[1] != fr->gB.p || before[2] != fr->gC.p) fr->g2d_zero = 0;  // new storage
    }
    const int nblk = gs::preprocess_bwd_blocks(n);
    const int nchunks = (n_views + kViewChunk - 1) / kViewChunk;
    // the block partials of a view chunk, then the reduction's group sums
    const size_t part_n = (size_t)std::max(nblk, 1) * std::min(n_views, kViewChunk) * 6 + 6;
    const size_t red_n = (size_t)gs::pose_reduce_groups(nblk) * std::min(n_views, kViewChunk) * 6;
    if ((rc = fr->pose_partials.ensure(part_n + red_n, grow, "pose partials"))) return rc;
    const RenderParams rp = make_params(opts);
    const float* dldc = loss->dl_dimage;
    const bool l1_loss = loss->loss && l1_kind;
    // the L1 term counts pixels whose final transmittance is below this bound
    // (1 - mask_alpha for the masked loss; everything otherwise)
    const float l1_mask_t = loss->kind == GS_LOSS_L1_MASKED
                                ? 1.0f - (loss->mask_alpha > 0.0f ? loss->mask_alpha : 0.99f)
                                : 2.0f;
    if (loss->kind == GS_LOSS_L1_DSSIM) {
        if ((rc = fr->dldc_ssim.ensure(fr->total_image, grow, "dssim grad")) ||
            (rc = fr->ssim_tmp.ensure(fr->total_image * 4, grow, "dssim tmp")))
            return rc;
        std::vector<long long> offs(n_views);
        for (int v = 0; v < n_views; v++) offs[v] = fr->vdev_host[v].img_off;
        if (loss->loss && (rc = fr->loss_tmp.ensure(n_views, grow, "loss tmp"))) return rc;
        {
            PROF(PK_DSSIM, n_views * (12 + (loss->loss ? 1 : 0)));
            CK(gs::launch_dssim(n_views, views, offs.data(), image, loss->target, loss->w_dssim, fr->dldc_ssim.p,
                                loss->loss ? fr->loss_tmp.p : nullptr, fr->ssim_tmp.p, s));
        }
        CK_LAUNCH();
        fr->have_dssim_grad = true;
        dldc = fr->dldc_ssim.p;
    }
    // the backward blend accumulates into records [0, vn), which must start at zero
    const size_t g2d_zero_after = std::max(fr->g2d_zero, vn);
    if (fr->g2d_zero < vn) {
        PROF(PK_MEMSET, 0);
        CK(cudaMemsetAsync(fr->gA.p, 0, sizeof(float4) * vn, s));
        CK(cudaMemsetAsync(fr->gB.p, 0, sizeof(float4) * vn, s));
        CK(cudaMemsetAsync(fr->gC.p, 0, sizeof(float) * vn, s));
    }
    fr->g2d_zero = 0;   // until the backward preprocess has cleared them again
    const uint32_t cap = (uint32_t)std::min<size_t>(fr->keys.cap, 0xffffffffu);
    {
        PROF(PK_BLEND_BWD, 1);
        gs::launch_blend_bwd(fr->total_tiles, n_views, fr->tile_base.p, fr->vdev.p, rp, fr->splats(), n, fr->starts.p,
                             fr->sorted_idx.p, cap, image, fr->T_final.p, fr->n_contrib.p, loss->kind, loss->w_l1,
                             l1_mask_t, loss->target, dldc, fr->g2d(), l1_loss ? fr->tile_loss.p : nullptr,
                             (opts->flags & GS_F_COUNT) ? fr->counters.p + 2 : nullptr,
                             ctx->tune.bwd_pixels_per_thread, s);
    }
    CK_LAUNCH();
    if (l1_loss) {
        PROF(PK_LOSS, 1);
        gs::launch_loss_finalize(n_views, fr->vdev.p, fr->tile_loss.p, (double)loss->w_l1,
                                 loss->kind == GS_LOSS_L1_DSSIM ? fr->loss_tmp.p : nullptr, loss->loss, s);
        CK_LAUNCH();
    }
    gs_grads gg{};
    if (grads) gg = *grads;
    if (gg.quats && reinterpret_cast<uintptr_t>(gg.quats) % 16 != 0)
        return fail(GS_EINVAL, "grads->quats must be 16-byte aligned");
    SplatArrays sp = fr->splats();
    Grad2DArrays g2 = fr->g2d();
    for (int c = 0; c < nchunks; c++) {
        const int v0 = c * kViewChunk;
        const int nv = std::min(kViewChunk, n_views - v0);
        SplatArrays spc = sp;
        Grad2DArrays g2c = g2;
        const size_t off = (size_t)v0 * n;
        spc.A += off; spc.B += off; spc.Cb += off; spc.rect += off; spc.depth += off; spc.radius += off;
        g2c.gA += off; g2c.gB += off; g2c.gC += off;
        double* part = fr->pose_partials.p;
        if (pipe && pipe->n_slices > 0) {
            // slice by slice; after the last view chunk a slice's gradients are final
            PROF(PK_PRE_BWD, pipe->n_slices);
            CK(cudaEventRecord(pipe->fork, s));
            CK(cudaStreamWaitEvent(pipe->aux, pipe->fork, 0));
            for (int k = 0; k < pipe->n_slices; k++) {
                cudaStream_t cs = (k & 1) ? pipe->aux : s;
                gs::launch_preprocess_bwd(scene->d, nv, fr->vdev.p + v0, rp, spc, g2c, gg, part, nblk, cs,
                                          pipe->bounds[k], pipe->bounds[k + 1]);
                if (c == nchunks - 1) CK(cudaEventRecord(pipe->done[k], cs));
            }
            CK(cudaEventRecord(pipe->join, pipe->aux));
            CK(cudaStreamWaitEvent(s, pipe->join, 0));
        } else {
            PROF(PK_PRE_BWD, 1);
            gs::launch_preprocess_bwd(scene->d, nv, fr->vdev.p + v0, rp, spc, g2c, gg, part, nblk, s);
        }
        CK_LAUNCH();
        if (pose_grad) {
            PROF(PK_POSE_REDUCE, 2);
            gs::launch_pose_reduce(nv, nblk, part, part + part_n, pose_grad + 6 * v0, s);
            CK_LAUNCH();
        }
    }
    fr->g2d_zero = g2d_zero_after;   // every record of [0, vn) was consumed and cleared
    return GS_OK;
}

extern "C" {

int gs_step(gs_ctx* ctx, gs_frames* fr, const gs_scene_desc* sd, int n_views, const gs_view* views,
            const double* poses, const gs_render_opts* opts, const gs_loss* loss, float* image_out, gs_grads* grads,
            double* pose_grad, double* loss_out, void* stream) {
    if (!ctx || !fr || !sd || !opts || !loss) return fail(GS_EINVAL, "NULL argument");
    int rc;
    if ((rc = check_views(n_views, views))) return rc;
    if (sd->n < 0 || sd->n > 0x7fffffff) return fail(GS_EINVAL, "Gaussian count out of range");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool host = (opts->flags & GS_F_HOST_IO) != 0;
    const bool grow = !(opts->flags & GS_F_NO_SYNC);
    const size_t n = (size_t)sd->n;
    long long n_img = 0;
    for (int v = 0; v < n_views; v++) n_img += 3LL * views[v].width * views[v].height;
    const bool need_target =
        loss->kind == GS_LOSS_L1 || loss->kind == GS_LOSS_L1_DSSIM || loss->kind == GS_LOSS_L1_MASKED;
    const float* in_img = need_target ? loss->target : loss->dl_dimage;
    if (n_views > 0 && (!poses || !in_img)) return fail(GS_EINVAL, "poses or loss input is NULL");
    gs_scene_desc dd = *sd;
    const double* dposes = poses;
    gs_loss dl = *loss;
    float* dimage = image_out;
    gs_grads dg{};
    if (grads) dg = *grads;
    double* dpose_grad = pose_grad;
    double* dloss = loss_out;
    // parameter layout inside the staging block: quats (16-byte aligned), means, scales, opac, sh
    const size_t off_q = 0, off_m = 4 * n, off_s = 7 * n, off_o = 10 * n, off_sh = 11 * n, nparam = 59 * n;
    if (host) {
        if ((rc = fr->st_params.ensure(std::max<size_t>(nparam, 1), grow, "staging params")) ||
            (rc = fr->st_target.ensure(std::max<long long>(n_img, 1), grow, "staging target")) ||
            (rc = fr->st_image.ensure(std::max<long long>(n_img, 1), grow, "staging image")) ||
            (rc = fr->st_grads.ensure(std::max<size_t>(nparam, 1), grow, "staging grads")) ||
            (rc = fr->st_poses.ensure(std::max(12 * n_views, 1), grow, "staging poses")) ||
            (rc = fr->st_pose_grad.ensure(std::max(6 * n_views, 1), grow, "staging pose grad")) ||
            (rc = fr->st_loss.ensure(std::max(n_views, 1), grow, "staging loss")))
            return rc;
        float* P = fr->st_params.p;
        if (n_views > 0 && !fr->side) {
            CK(cudaStreamCreateWithFlags(&fr->side, cudaStreamNonBlocking));
            CK(cudaStreamCreateWithFlags(&fr->down, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&fr->ev_fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&fr->ev_join, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&fr->ev_down, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&fr->ev_img, cudaEventDisableTiming));
            for (int c = 0; c < GS_MAX_SLICES; c++) {
                CK(cudaEventCreateWithFlags(&fr->pipe.ready[c], cudaEventDisableTiming));
                CK(cudaEventCreateWithFlags(&fr->pipe.done[c], cudaEventDisableTiming));
            }
            CK(cudaStreamCreateWithFlags(&fr->pipe.aux, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&fr->pipe.fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&fr->pipe.join, cudaEventDisableTiming));
        }
        // The parameters go up in slices of Gaussians on the side stream (after
        // everything already queued on s, which may still read the staging
        // block), and the forward preprocess of a slice starts once its copy
        // has landed; the loss input, first read by the backward, follows.
        fr->pipe.n_slices = 0;
        if (n_views > 0) {
            CK(cudaEventRecord(fr->ev_fork, s));
            CK(cudaStreamWaitEvent(fr->side, fr->ev_fork, 0));
            if (n > 0) {
                const size_t k = n >= ((size_t)1 << 18) ? kHostSlices : 1;
                const size_t step = ((n + k - 1) / k + 255) / 256 * 256;
                int c = 0;
                for (size_t b = 0; b < n && c < GS_MAX_SLICES; b += step, c++) fr->pipe.bounds[c] = (int)b;
                fr->pipe.n_slices = c;
                fr->pipe.bounds[c] = (int)n;
            }
        }
        const int n_up = n_views > 0 ? fr->pipe.n_slices : (n > 0 ? 1 : 0);
        for (int c = 0; c < n_up; c++) {
            const size_t b0 = n_views > 0 ? (size_t)fr->pipe.bounds[c] : 0;
            const size_t m = (n_views > 0 ? (size_t)fr->pipe.bounds[c + 1] : n) - b0;
            cudaStream_t cs = n_views > 0 ? fr->side : s;
            CK(cudaMemcpyAsync(P + off_m + 3 * b0, sd->means + 3 * b0, 3 * m * 4, cudaMemcpyHostToDevice, cs));
            CK(cudaMemcpyAsync(P + off_s + 3 * b0, sd->scales + 3 * b0, 3 * m * 4, cudaMemcpyHostToDevice, cs));
            CK(cudaMemcpyAsync(P + off_q + 4 * b0, sd->quats + 4 * b0, 4 * m * 4, cudaMemcpyHostToDevice, cs));
            CK(cudaMemcpyAsync(P + off_o + b0, sd->opacities + b0, m * 4, cudaMemcpyHostToDevice, cs));
            CK(cudaMemcpyAsync(P + off_sh + 48 * b0, sd->sh + 48 * b0, 48 * m * 4, cudaMemcpyHostToDevice, cs));
            if (n_views > 0) CK(cudaEventRecord(fr->pipe.ready[c], cs));
        }
        dd.means = P + off_m; dd.scales = P + off_s; dd.quats = P + off_q; dd.opacities = P + off_o; dd.sh = P + off_sh;
        if (n_views > 0) {
            CK(cudaMemcpyAsync(fr->st_poses.p, poses, 12 * sizeof(double) * n_views, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(fr->st_target.p, in_img, n_img * sizeof(float), cudaMemcpyHostToDevice, fr->side));
            CK(cudaEventRecord(fr->ev_join, fr->side));
        }
        dposes = fr->st_poses.p;
        if (need_target) dl.target = fr->st_target.p; else dl.dl_dimage = fr->st_target.p;
        dimage = fr->st_image.p;
        float* G = fr->st_grads.p;
        if (grads) {
            dg.means = grads->means ? G + off_m : nullptr; dg.scales = grads->scales ? G + off_s : nullptr;
            dg.quats = grads->quats ? G + off_q : nullptr; dg.opacities = grads->opacities ? G + off_o : nullptr;
            dg.sh = grads->sh ? G + off_sh : nullptr;
            if (nparam) CK(cudaMemsetAsync(G, 0, nparam * sizeof(float), s));
        }
        dpose_grad = pose_grad ? fr->st_pose_grad.p : nullptr;
        dloss = loss_out ? fr->st_loss.p : nullptr;
    } else {
        if (!dimage) {
            if ((rc = fr->st_image.ensure(std::max<long long>(n_img, 1), grow, "image"))) return rc;
            dimage = fr->st_image.p;
        }
        if (grads && n > 0) {
            if (dg.means) CK(cudaMemsetAsync(dg.means, 0, 3 * n * 4, s));
            if (dg.scales) CK(cudaMemsetAsync(dg.scales, 0, 3 * n * 4, s));
            if (dg.quats) CK(cudaMemsetAsync(dg.quats, 0, 4 * n * 4, s));
            if (dg.opacities) CK(cudaMemsetAsync(dg.opacities, 0, n * 4, s));
            if (dg.sh) CK(cudaMemsetAsync(dg.sh, 0, 48 * n * 4, s));
        }
    }
    gs_scene* sc = nullptr;
    if ((rc = gs_scene_borrow(&dd, &sc))) return rc;
    gs_render_opts o2 = *opts;
    o2.flags &= ~(uint32_t)GS_F_HOST_IO;
    dl.loss = dloss;
    const gs::SlicePipe* pipe = (host && fr->pipe.n_slices > 0) ? &fr->pipe : nullptr;
    rc = gs::render_forward_impl(ctx, sc, n_views, views, nullptr, dposes, &o2, fr, dimage, nullptr, nullptr, s, pipe);
    if (rc == GS_OK && host && n_views > 0) {
        if (image_out && n_img) {
            // the rendered image goes down on the download stream while the backward runs
            cudaError_t e = cudaEventRecord(fr->ev_img, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(fr->down, fr->ev_img, 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(image_out, dimage, n_img * sizeof(float), cudaMemcpyDeviceToHost, fr->down);
            if (e != cudaSuccess) rc = fail(GS_ECUDA, "image download: %s", cudaGetErrorString(e));
        }
        const cudaError_t e = cudaStreamWaitEvent(s, fr->ev_join, 0);
        if (rc == GS_OK && e != cudaSuccess) rc = fail(GS_ECUDA, "join of the loss-input upload: %s", cudaGetErrorString(e));
    }
    if (rc == GS_OK)
        rc = gs::render_backward_impl(ctx, sc, n_views, views, nullptr, dposes, &o2, fr, dimage, &dl,
                                      grads ? &dg : nullptr, dpose_grad, s, grads ? pipe : nullptr);
    gs_scene_free(sc);
    if (rc != GS_OK) {
        // a failed step still leaves nothing of it pending on the download stream
        if (host && n_views > 0 && cudaEventRecord(fr->ev_down, fr->down) == cudaSuccess)
            cudaStreamWaitEvent(s, fr->ev_down, 0);
        return rc;
    }
    if (host) {
        if (image_out && n_img && n_views == 0)
            CK(cudaMemcpyAsync(image_out, dimage, n_img * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (grads && n > 0) {
            // slice by slice on the download stream as each slice's gradients
            // become final (one slice on s without the pipeline); s then waits
            const float* G = fr->st_grads.p;
            const int ns = pipe ? pipe->n_slices : 1;
            cudaStream_t ds = pipe ? fr->down : s;
            for (int c = 0; c < ns; c++) {
                const size_t b0 = pipe ? (size_t)pipe->bounds[c] : 0;
                const size_t m = (pipe ? (size_t)pipe->bounds[c + 1] : n) - b0;
                if (pipe) CK(cudaStreamWaitEvent(ds, pipe->done[c], 0));
                if (grads->means)
                    CK(cudaMemcpyAsync(grads->means + 3 * b0, G + off_m + 3 * b0, 3 * m * 4, cudaMemcpyDeviceToHost, ds));
                if (grads->scales)
                    CK(cudaMemcpyAsync(grads->scales + 3 * b0, G + off_s + 3 * b0, 3 * m * 4, cudaMemcpyDeviceToHost, ds));
                if (grads->quats)
                    CK(cudaMemcpyAsync(grads->quats + 4 * b0, G + off_q + 4 * b0, 4 * m * 4, cudaMemcpyDeviceToHost, ds));
                if (grads->opacities)
                    CK(cudaMemcpyAsync(grads->opacities + b0, G + off_o + b0, m * 4, cudaMemcpyDeviceToHost, ds));
                if (grads->sh)
                    CK(cudaMemcpyAsync(grads->sh + 48 * b0, G + off_sh + 48 * b0, 48 * m * 4, cudaMemcpyDeviceToHost, ds));
            }
        }
        if (n_views > 0) {
            // the downloads (image and gradients) are done when s passes this
            // point; the uploads were joined before the backward
            CK(cudaEventRecord(fr->ev_down, fr->down));
            CK(cudaStreamWaitEvent(s, fr->ev_down, 0));
        }
        if (pose_grad && n_views)
            CK(cudaMemcpyAsync(pose_grad, dpose_grad, 6 * sizeof(double) * n_views, cudaMemcpyDeviceToHost, s));
        if (loss_out && n_views) CK(cudaMemcpyAsync(loss_out, dloss, sizeof(double) * n_views, cudaMemcpyDeviceToHost, s));
    }
    return GS_OK;
}

int gs_gaussian_adam(gs_ctx* ctx, int64_t n, int sh_degree, gs_raw_params* raw, float* scales_out,
                     float* opacities_out, const gs_grads* grads, float* m, float* v, const gs_gaussian_lrs* lrs,
                     float b1, float b2, float eps, int step, void* stream) {
    if (!ctx || !raw || !grads || !lrs) return fail(GS_EINVAL, "NULL argument");
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || step < 1) return fail(GS_EINVAL, "bad n, sh_degree or step");
    if (n > 0 && (!raw->means || !raw->log_scales || !raw->quats || !raw->logit_opacities || !raw->sh || !m || !v ||
                  !scales_out || !opacities_out))
        return fail(GS_EINVAL, "NULL parameter, moment or output array");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = n;
    gs::AdamGroup G[5];
    G[0] = {raw->means, grads->means, m, v, nullptr, 3, 3, 0, lrs->means, lrs->means, 3};
    G[1] = {raw->log_scales, grads->scales, m + 3 * N, v + 3 * N, scales_out, 3, 3, 1, lrs->scales, lrs->scales, 3};
    G[2] = {raw->quats, grads->quats, m + 6 * N, v + 6 * N, nullptr, 4, 4, 0, lrs->quats, lrs->quats, 4};
    G[3] = {raw->logit_opacities, grads->opacities, m + 10 * N, v + 10 * N, opacities_out, 1, 1, 2, lrs->opacities,
            lrs->opacities, 1};
    G[4] = {raw->sh, grads->sh, m + 11 * N, v + 11 * N, nullptr, 48, 3 * (sh_degree + 1) * (sh_degree + 1), 0,
            lrs->sh_dc, lrs->sh_rest, 3};
    {
        PROF(PK_GAUSS_ADAM, 1);
        gs::launch_gaussian_adam(N, G, 5, b1, b2, eps, step, s);
    }
    CK_LAUNCH();
    return GS_OK;
}

static int pose_step_param(gs_ctx* ctx, int n_views, double* poses, double* m, double* v, const double* g, double lr,
                           double b1, double b2, double eps, int step, int param, void* stream) {
    if (!ctx) return fail(GS_EINVAL, "ctx is NULL");
    if (n_views < 0 || step < 1) return fail(GS_EINVAL, "bad n_views or step");
    if (n_views > 0 && (!poses || !m || !v || !g)) return fail(GS_EINVAL, "NULL pose/moment/gradient array");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        PROF(PK_POSE_ADAM, 1);
        gs::launch_pose_adam(n_views, poses, m, v, g, lr, b1, b2, eps, step, param, s);
    }
    CK_LAUNCH();
    return GS_OK;
}

int gs_pose_step(gs_ctx* ctx, int n_views, double* poses, double* m, double* v, const double* g, double lr, double b1,
                 double b2, double eps, int step, void* stream) {
    return pose_step_param(ctx, n_views, poses, m, v, g, lr, b1, b2, eps, step, GS_POSE_SE3, stream);
}

int gs_pose_step_txso3(gs_ctx* ctx, int n_views, double* poses, double* m, double* v, const double* g, double lr,
                       double b1, double b2, double eps, int step, void* stream) {
    return pose_step_param(ctx, n_views, poses, m, v, g, lr, b1, b2, eps, step, GS_POSE_TXSO3, stream);
}

// Grows the context's regulariser scratch to `bytes` (not during capture).
static int reg_scratch(gs_ctx* ctx, size_t bytes) {
    if (ctx->reg_cap >= bytes) return GS_OK;
    if (ctx->reg_scratch) cudaFree(ctx->reg_scratch);
    ctx->reg_scratch = nullptr;
    ctx->reg_cap = 0;
    size_t cap = std::max<size_t>(bytes, 4096);
    if (cudaMalloc(&ctx->reg_scratch, cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(GS_ENOMEM, "regulariser scratch (%zu bytes)", cap);
    }
    ctx->reg_cap = cap;
    return GS_OK;
}

int gs_regularize(gs_ctx* ctx, int64_t n, const float* scales, const float* opacities, float aniso_r,
                  float lambda_aniso, float lambda_opacity, float* grad_scales, float* grad_opacities, double* loss,
                  void* stream) {
    if (!ctx) return fail(GS_EINVAL, "ctx is NULL");
    if (n < 0 || n > INT32_MAX) return fail(GS_EINVAL, "bad n");
    if (n > 0 && ((lambda_aniso != 0.0f && !scales) || (lambda_opacity != 0.0f && !opacities)))
        return fail(GS_EINVAL, "NULL scales or opacities");
    if (!(aniso_r >= 1.0f)) return fail(GS_EINVAL, "aniso_r must be >= 1");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    const int nb = gs::regularize_blocks((int)n);
    if (loss && (rc = reg_scratch(ctx, sizeof(double) * (size_t)std::max(nb, 1)))) return rc;
    const float inv_n = n > 0 ? 1.0f / (float)n : 0.0f;
    {
        PROF(PK_REG, loss ? 2 : 1);
        gs::launch_regularize((int)n, scales, opacities, aniso_r, lambda_aniso * inv_n, lambda_opacity * inv_n,
                              grad_scales, grad_opacities, static_cast<double*>(ctx->reg_scratch), loss, s);
    }
    CK_LAUNCH();
    return GS_OK;
}

int gs_prune_threshold(gs_ctx* ctx, int64_t n, const float* opacities, int64_t n_target, float min_opacity,
                       float* threshold, int64_t* n_keep, void* stream) {
    if (!ctx || !threshold || !n_keep) return fail(GS_EINVAL, "NULL argument");
    if (n < 0 || n > INT32_MAX || n_target < 0) return fail(GS_EINVAL, "bad n or n_target");
    if (n > 0 && !opacities) return fail(GS_EINVAL, "opacities is NULL");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    const int nb = gs::regularize_blocks((int)n);
    const size_t bytes = sizeof(uint32_t) * (2 + 256 + (size_t)std::max(nb, 1) + 1);
    if ((rc = reg_scratch(ctx, bytes))) return rc;
    uint32_t* state = static_cast<uint32_t*>(ctx->reg_scratch);
    uint32_t* hist = state + 2;
    uint32_t* counts = hist + 256;
    uint32_t* total = counts + std::max(nb, 1);
    float thr = min_opacity;
    if (n > n_target) {
        PROF(PK_PRUNE, 9);
        gs::launch_select_kth((int)n, opacities, (uint32_t)(n - n_target - 1), state, hist, s);
        uint32_t st[2];
        CK(cudaMemcpyAsync(st, state, sizeof(st), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        float kth;
        memcpy(&kth, &st[0], sizeof(float));
        thr = std::max(thr, kth);
    }
    gs::CompactArrays none{};
    {
        PROF(PK_PRUNE, 2);
        // counting only: a compaction with no arrays
        gs::launch_compact((int)n, opacities, thr, none, counts, total, s);
    }
    CK_LAUNCH();
    uint32_t kept = 0;
    CK(cudaMemcpyAsync(&kept, total, sizeof(kept), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *threshold = thr;
    *n_keep = (int64_t)kept;
    return GS_OK;
}

int gs_unproject(gs_ctx* ctx, const gs_view* view, const float* depth, const float* image, int stride, float* points,
                 float* colours, int64_t capacity, int64_t* n_out, void* stream) {
    if (!ctx || !view || !depth || !points || !n_out) return fail(GS_EINVAL, "NULL argument");
    if (view->width < 1 || view->height < 1 || stride < 1) return fail(GS_EINVAL, "bad view size or stride");
    if (!(view->fx > 0.0f) || !(view->fy > 0.0f)) return fail(GS_EINVAL, "bad focal length");
    const int gw = (view->width + stride - 1) / stride, gh = (view->height + stride - 1) / stride;
    const int64_t ng = (int64_t)gw * gh;
    if (capacity < ng) return fail(GS_EINVAL, "capacity %lld < %lld grid pixels", (long long)capacity, (long long)ng);
    if (ng > INT32_MAX / 8) return fail(GS_EINVAL, "too many grid pixels");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    const int nb = gs::regularize_blocks((int)ng);
    const size_t fl = (size_t)ng * 7;
    if ((rc = reg_scratch(ctx, sizeof(float) * fl + sizeof(uint32_t) * ((size_t)nb + 2)))) return rc;
    float* pts = static_cast<float*>(ctx->reg_scratch);
    float* cols = pts + 3 * ng;
    float* key = cols + 3 * ng;
    uint32_t* counts = reinterpret_cast<uint32_t*>(key + ng);
    uint32_t* total = counts + nb + 1;
    gs::CompactArrays ca{};
    ca.count = colours ? 2 : 1;
    ca.src[0] = pts; ca.dst[0] = points; ca.width[0] = 3;
    if (colours) { ca.src[1] = cols; ca.dst[1] = colours; ca.width[1] = 3; }
    {
        PROF(PK_INIT, 4);
        gs::launch_unproject(view->width, view->height, stride, view->fx, view->fy, view->cx, view->cy, depth, image,
                             pts, cols, key, s);
        gs::launch_compact((int)ng, key, 0.0f, ca, counts, total, s);
    }
    CK_LAUNCH();
    uint32_t kept = 0;
    CK(cudaMemcpyAsync(&kept, total, sizeof(kept), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n_out = (int64_t)kept;
    return GS_OK;
}

int gs_knn_mean_dist(gs_ctx* ctx, int64_t n, const float* points, int k, float* mean_dist, void* stream) {
    if (!ctx) return fail(GS_EINVAL, "ctx is NULL");
    if (n < 0 || n > INT32_MAX || k < 1 || k > 8) return fail(GS_EINVAL, "bad n or k (1..8)");
    if (n > 0 && (!points || !mean_dist)) return fail(GS_EINVAL, "NULL points or output");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        PROF(PK_INIT, 1);
        gs::launch_knn_mean((int)n, points, k, mean_dist, s);
    }
    CK_LAUNCH();
    return GS_OK;
}

int gs_init_from_points(gs_ctx* ctx, int64_t n, const float* points, const float* colours, const float* mean_dist,
                        float min_scale, float opacity, gs_raw_params* raw, void* stream) {
    if (!ctx || !raw) return fail(GS_EINVAL, "NULL argument");
    if (n < 0 || n > INT32_MAX) return fail(GS_EINVAL, "bad n");
    if (!(opacity > 0.0f && opacity < 1.0f) || !(min_scale > 0.0f)) return fail(GS_EINVAL, "bad opacity or min_scale");
    if (n > 0 && (!points || !colours || !mean_dist || !raw->means || !raw->log_scales || !raw->quats ||
                  !raw->logit_opacities || !raw->sh))
        return fail(GS_EINVAL, "NULL array");
    CK(cudaSetDevice(ctx->device));
    const float logit_o = logf(opacity / (1.0f - opacity));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        PROF(PK_INIT, 1);
        gs::launch_init_raw((int)n, points, colours, mean_dist, min_scale, logit_o, raw->means, raw->log_scales,
                            raw->quats, raw->logit_opacities, raw->sh, s);
    }
    CK_LAUNCH();
    return GS_OK;
}

int gs_spatial_order(gs_ctx* ctx, int64_t n, const float* means, uint32_t* perm, void* stream) {
    if (!ctx) return fail(GS_EINVAL, "ctx is NULL");
    if (n < 0 || n > INT32_MAX / 4) return fail(GS_EINVAL, "bad n");
    if (n == 0) return GS_OK;
    if (!means || !perm) return fail(GS_EINVAL, "NULL means or perm");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    const int nb = gs::spatial_order_blocks((int)n);
    const size_t key_bytes = sizeof(unsigned long long) * (size_t)n;
    const size_t bytes = 2 * key_bytes + sizeof(float) * 6 * (size_t)nb + sizeof(uint32_t) * 16;
    if ((rc = reg_scratch(ctx, bytes))) return rc;
    unsigned long long* keys = static_cast<unsigned long long*>(ctx->reg_scratch);
    unsigned long long* tmp = keys + n;
    float* part = reinterpret_cast<float*>(tmp + n);
    uint32_t* small = reinterpret_cast<uint32_t*>(part + 6 * nb);
    uint32_t* starts = small;          // [2]
    uint32_t* lists = small + 2;       // [3]
    uint32_t* counters = small + 5;    // [8]
    {
        PROF(PK_INIT, 7);
        gs::launch_spatial_keys((int)n, means, part, keys, starts, s);
        gs::launch_segment_sort(1, starts, keys, tmp, perm, (uint32_t)n, lists, counters, s);
    }
    CK_LAUNCH();
    return GS_OK;
}

int gs_gather_rows(gs_ctx* ctx, int64_t n, const uint32_t* perm, int n_arrays, const float* const* src,
                   float* const* dst, const int32_t* widths, void* stream) {
    if (!ctx) return fail(GS_EINVAL, "ctx is NULL");
    if (n < 0 || n > INT32_MAX) return fail(GS_EINVAL, "bad n");
    if (n_arrays < 0 || n_arrays > GS_COMPACT_MAX) return fail(GS_EINVAL, "at most %d arrays", GS_COMPACT_MAX);
    if (n > 0 && (!perm || (n_arrays > 0 && (!src || !dst || !widths)))) return fail(GS_EINVAL, "NULL argument");
    gs::CompactArrays ca{};
    ca.count = n_arrays;
    for (int a = 0; a < n_arrays; a++) {
        if (!src[a] || !dst[a] || widths[a] < 1) return fail(GS_EINVAL, "bad array %d", a);
        if (src[a] == dst[a]) return fail(GS_EINVAL, "array %d: the gather is out of place", a);
        ca.src[a] = src[a]; ca.dst[a] = dst[a]; ca.width[a] = widths[a];
    }
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        PROF(PK_INIT, 1);
        gs::launch_gather_rows((int)n, perm, ca, s);
    }
    CK_LAUNCH();
    return GS_OK;
}

int gs_compact(gs_ctx* ctx, int64_t n, const float* opacities, float threshold, int n_arrays, const float* const* src,
               float* const* dst, const int32_t* widths, int64_t* n_keep, void* stream) {
    if (!ctx || !n_keep) return fail(GS_EINVAL, "NULL argument");
    if (n < 0 || n > INT32_MAX) return fail(GS_EINVAL, "bad n");
    if (n_arrays < 0 || n_arrays > GS_COMPACT_MAX) return fail(GS_EINVAL, "at most %d arrays", GS_COMPACT_MAX);
    if (n > 0 && !opacities) return fail(GS_EINVAL, "opacities is NULL");
    if (n_arrays > 0 && (!src || !dst || !widths)) return fail(GS_EINVAL, "NULL array lists");
    gs::CompactArrays ca{};
    ca.count = n_arrays;
    for (int a = 0; a < n_arrays; a++) {
        if (!src[a] || !dst[a] || widths[a] < 1) return fail(GS_EINVAL, "bad array %d", a);
        if (src[a] == dst[a]) return fail(GS_EINVAL, "array %d: compaction is out of place", a);
        ca.src[a] = src[a]; ca.dst[a] = dst[a]; ca.width[a] = widths[a];
    }
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    const int nb = gs::regularize_blocks((int)n);
    if ((rc = reg_scratch(ctx, sizeof(uint32_t) * ((size_t)std::max(nb, 1) + 1)))) return rc;
    uint32_t* counts = static_cast<uint32_t*>(ctx->reg_scratch);
    uint32_t* total = counts + std::max(nb, 1);
    {
        PROF(PK_PRUNE, 3);
        gs::launch_compact((int)n, opacities, threshold, ca, counts, total, s);
    }
    CK_LAUNCH();
    uint32_t kept = 0;
    CK(cudaMemcpyAsync(&kept, total, sizeof(kept), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n_keep = (int64_t)kept;
    return GS_OK;
}

int gs_status(gs_ctx* ctx, void* stream) {
    if (!ctx) return fail(GS_EINVAL, "ctx is NULL");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(ctx->pinned, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    const int st = *reinterpret_cast<int*>(ctx->pinned);
    if (st & GS_DEV_OVERFLOW) return fail(GS_EOVERFLOW, "a key buffer overflowed in no-sync mode");
    if (st) return fail(GS_ECUDA, "device status 0x%x", st);
    return GS_OK;
}

int gs_ctx_set_tuning(gs_ctx* ctx, const gs_tuning* t) {
    if (!ctx || !t) return fail(GS_EINVAL, "NULL argument");
    if (t->scatter_chunk < 256 || t->scatter_chunk > 65536 || (t->scatter_chunk & (t->scatter_chunk - 1)))
        return fail(GS_EINVAL, "scatter_chunk must be a power of two in [256, 65536]");
    if (t->sort_chunk != 1024 && t->sort_chunk != 2048) return fail(GS_EINVAL, "sort_chunk must be 1024 or 2048");
    if (t->preprocess_threads != 128 && t->preprocess_threads != 256)
        return fail(GS_EINVAL, "preprocess_threads must be 128 or 256");
    if (t->bwd_pixels_per_thread != 1 && t->bwd_pixels_per_thread != 2)
        return fail(GS_EINVAL, "bwd_pixels_per_thread must be 1 or 2");
    if (t->fwd_pixels_per_thread != 1 && t->fwd_pixels_per_thread != 2)
        return fail(GS_EINVAL, "fwd_pixels_per_thread must be 1 or 2");
    ctx->tune = *t;
    return GS_OK;
}

int gs_ctx_get_tuning(gs_ctx* ctx, gs_tuning* t) {
    if (!ctx || !t) return fail(GS_EINVAL, "NULL argument");
    *t = ctx->tune;
    return GS_OK;
}

int gs_autotune(gs_ctx* ctx, gs_frames* fr, const gs_scene* scene, int n_views, const gs_view* views,
                const double* poses, const gs_render_opts* opts, float* image, const gs_loss* loss, gs_grads* grads,
                double* pose_grad, int repeats, gs_tuning* best, double* best_ms, void* stream) {
    if (!ctx || !fr || !opts || !loss || !best) return fail(GS_EINVAL, "NULL argument");
    if (repeats < 1) return fail(GS_EINVAL, "repeats must be >= 1");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const gs_tuning saved = ctx->tune;
    const bool prof = ctx->prof;
    ctx->prof = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int chunks[] = {1024, 2048, 4096, 8192};
    const int sorts[] = {1024, 2048};
    const int threads[] = {128, 256};
    const int bwd_px[] = {1, 2};
    double bms = 1e300;
    gs_tuning bt = saved;
    int rc = GS_OK;
    for (int a : chunks)
        for (int b : sorts)
            for (int c : threads)
              for (int d : bwd_px)
                for (int f : bwd_px) {
                ctx->tune = gs_tuning{a, b, c, d, f};
                for (int r = 0; r <= repeats && rc == GS_OK; r++) {
                    if (r == 1) cudaEventRecord(e0, s);
                    rc = gs_render_forward(ctx, scene, n_views, views, poses, opts, fr, image, nullptr, nullptr, stream);
                    if (rc == GS_OK)
                        rc = gs_render_backward(ctx, scene, n_views, views, poses, opts, fr, image, loss, grads,
                                                pose_grad, stream);
                }
                if (rc != GS_OK) break;
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms / repeats < bms) { bms = ms / repeats; bt = ctx->tune; }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->prof = prof;
    if (rc != GS_OK) { ctx->tune = saved; return rc; }
    ctx->tune = bt;
    *best = bt;
    if (best_ms) *best_ms = bms;
    return GS_OK;
}

int gs_ctx_set_profiling(gs_ctx* ctx, int enable) {
    if (!ctx) return fail(GS_EINVAL, "ctx is NULL");
    ctx->prof = enable != 0;
    return GS_OK;
}

int gs_ctx_profile(gs_ctx* ctx, int max_kinds, char (*names)[32], double* total_ms, int64_t* launches,
                   int* n_kinds) {
    if (!ctx) return fail(GS_EINVAL, "ctx is NULL");
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    for (const ProfRec& r : ctx->recs) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            ctx->prof_ms[r.kind] += ms;
            ctx->prof_n[r.kind] += 1;
        } else {
            cudaGetLastError();
        }
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
    int k = 0;
    for (int i = 0; i < PK_COUNT && k < max_kinds; i++) {
        if (ctx->prof_n[i] == 0) continue;
        if (names) { strncpy(names[k], kProfNames[i], 31); names[k][31] = 0; }
        if (total_ms) total_ms[k] = ctx->prof_ms[i];
        if (launches) launches[k] = ctx->prof_n[i];
        k++;
    }
    if (n_kinds) *n_kinds = k;
    for (int i = 0; i < PK_COUNT; i++) { ctx->prof_ms[i] = 0.0; ctx->prof_n[i] = 0; }
    return GS_OK;
}

int64_t gs_ctx_launch_count(gs_ctx* ctx) { return ctx ? ctx->launches : -1; }

int gs_frames_counters(gs_frames* fr, int64_t out[GS_N_COUNTERS]) {
    if (!fr || !out) return fail(GS_EINVAL, "NULL argument");
    for (int k = 0; k < GS_N_COUNTERS; k++) out[k] = 0;
    if (!fr->counters.p) return GS_OK;
    CK(cudaSetDevice(fr->ctx->device));
    unsigned long long c[12];
    CK(cudaMemcpy(c, fr->counters.p, sizeof(c), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 4; k++) out[k] = (int64_t)c[k];
    out[4] = (int64_t)c[4];
    out[5] = (int64_t)c[6];
    out[6] = fr->full_sort ? (int64_t)fr->n_keys : (int64_t)c[5];
    out[7] = (int64_t)c[8];
    out[8] = (int64_t)c[9];
    out[9] = (int64_t)c[10];
    out[10] = (int64_t)c[11];
    return GS_OK;
}

int gs_frames_query(gs_frames* fr, int what, void* dst, size_t bytes, size_t* size_out) {
    if (!fr) return fail(GS_EINVAL, "frames is NULL");
    if (!fr->have_forward) return fail(GS_EINVAL, "no forward pass recorded");
    CK(cudaSetDevice(fr->ctx->device));
    CK(cudaDeviceSynchronize());
    const size_t vn = (size_t)fr->n * fr->n_views;
    size_t need = 0;
    switch (what) {
        case GS_Q_NUM_KEYS: need = sizeof(int64_t); break;
        case GS_Q_DEPTH: need = vn * sizeof(float); break;
        case GS_Q_RECT: need = vn * 4 * sizeof(int32_t); break;
        case GS_Q_RADIUS: need = vn * sizeof(int32_t); break;
        case GS_Q_TILE_RANGES: need = (size_t)fr->total_tiles * 2 * sizeof(uint32_t); break;
        case GS_Q_SORTED_IDX: need = (size_t)fr->n_keys * sizeof(uint32_t); break;
        case GS_Q_T_FINAL: need = (size_t)fr->total_pixels * sizeof(float); break;
        case GS_Q_N_CONTRIB: need = (size_t)fr->total_pixels * sizeof(uint32_t); break;
        case GS_Q_MEAN2D: need = vn * 2 * sizeof(float); break;
        case GS_Q_SPLAT: need = vn * 9 * sizeof(float); break;
        case GS_Q_SORTED_COUNT: need = (size_t)fr->total_tiles * sizeof(uint32_t); break;
        case GS_Q_DSSIM_GRAD:
            if (!fr->have_dssim_grad) return fail(GS_EINVAL, "no D-SSIM backward recorded for these frames");
            need = (size_t)fr->total_image * sizeof(float);
            break;
        default: return fail(GS_EINVAL, "unknown query %d", what);
    }
    if (size_out) *size_out = need;
    if (!dst) return GS_OK;
    if (bytes < need) return fail(GS_EINVAL, "destination too small (%zu < %zu)", bytes, need);
    if (what == GS_Q_NUM_KEYS) {
        uint32_t K = 0;
        CK(cudaMemcpy(&K, fr->starts.p + fr->total_tiles, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        int64_t k64 = K;
        memcpy(dst, &k64, sizeof(k64));
        return GS_OK;
    }
    if (what == GS_Q_DSSIM_GRAD) { CK(cudaMemcpy(dst, fr->dldc_ssim.p, need, cudaMemcpyDeviceToHost)); return GS_OK; }
    if (what == GS_Q_DEPTH) { CK(cudaMemcpy(dst, fr->depth.p, need, cudaMemcpyDeviceToHost)); return GS_OK; }
    if (what == GS_Q_RADIUS) { CK(cudaMemcpy(dst, fr->radius.p, need, cudaMemcpyDeviceToHost)); return GS_OK; }
    if (what == GS_Q_T_FINAL) { CK(cudaMemcpy(dst, fr->T_final.p, need, cudaMemcpyDeviceToHost)); return GS_OK; }
    if (what == GS_Q_N_CONTRIB) { CK(cudaMemcpy(dst, fr->n_contrib.p, need, cudaMemcpyDeviceToHost)); return GS_OK; }
    if (what == GS_Q_SORTED_IDX) {
        uint32_t K = 0;
        CK(cudaMemcpy(&K, fr->starts.p + fr->total_tiles, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        const size_t nb = std::min<size_t>((size_t)K * 4, need);
        if (nb) CK(cudaMemcpy(dst, fr->sorted_idx.p, nb, cudaMemcpyDeviceToHost));
        return GS_OK;
    }
    if (what == GS_Q_SORTED_COUNT) {
        std::vector<uint32_t> st(fr->total_tiles + 1);
        CK(cudaMemcpy(st.data(), fr->starts.p, st.size() * 4, cudaMemcpyDeviceToHost));
        uint32_t* o = static_cast<uint32_t*>(dst);
        if (fr->full_sort) {
            for (int t = 0; t < fr->total_tiles; t++) o[t] = st[t + 1] - st[t];
        } else if (fr->total_tiles) {
            CK(cudaMemcpy(o, fr->sorted_count.p, need, cudaMemcpyDeviceToHost));
        }
        return GS_OK;
    }
    if (what == GS_Q_TILE_RANGES) {
        std::vector<uint32_t> st(fr->total_tiles + 1);
        CK(cudaMemcpy(st.data(), fr->starts.p, st.size() * 4, cudaMemcpyDeviceToHost));
        uint32_t* o = static_cast<uint32_t*>(dst);
        for (int t = 0; t < fr->total_tiles; t++) { o[2 * t] = st[t]; o[2 * t + 1] = st[t + 1]; }
        return GS_OK;
    }
    std::vector<uint2> rc(vn);
    if (vn) CK(cudaMemcpy(rc.data(), fr->rect.p, vn * sizeof(uint2), cudaMemcpyDeviceToHost));
    if (what == GS_Q_RECT) {
        int32_t* o = static_cast<int32_t*>(dst);
        for (size_t k = 0; k < vn; k++) {
            const int x0 = rc[k].x & 0xffff, y0 = rc[k].x >> 16, x1 = rc[k].y & 0xffff, y1 = rc[k].y >> 16;
            const bool ok = x1 > x0;
            o[4 * k] = ok ? x0 : 0; o[4 * k + 1] = ok ? y0 : 0; o[4 * k + 2] = ok ? x1 : 0; o[4 * k + 3] = ok ? y1 : 0;
        }
        return GS_OK;
    }
    std::vector<float4> a(vn), b(vn);
    std::vector<float2> lo(vn);
    std::vector<float> c(vn);
    if (vn) {
        CK(cudaMemcpy(a.data(), fr->A.p, vn * sizeof(float4), cudaMemcpyDeviceToHost));
        if (what == GS_Q_SPLAT) CK(cudaMemcpy(lo.data(), fr->Mlo.p, vn * sizeof(float2), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(b.data(), fr->B.p, vn * sizeof(float4), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(c.data(), fr->Cb.p, vn * sizeof(float), cudaMemcpyDeviceToHost));
    }
    float* o = static_cast<float*>(dst);
    for (size_t k = 0; k < vn; k++) {
        const bool ok = (rc[k].y & 0xffff) > (rc[k].x & 0xffff);
        if (what == GS_Q_MEAN2D) {
            o[2 * k] = ok ? a[k].x : 0.f; o[2 * k + 1] = ok ? a[k].y : 0.f;
        } else {
            float r[9] = {a[k].x + lo[k].x, a[k].y + lo[k].y, a[k].z, a[k].w, b[k].x, b[k].y, b[k].z, b[k].w, c[k]};
            for (int j = 0; j < 9; j++) o[9 * k + j] = ok ? r[j] : 0.f;
        }
    }
    return GS_OK;
}

}  // extern "C"

int gs::scene_count(const gs_scene* scene) { return scene ? scene->d.n : 0; }

uint32_t gs::frames_num_keys(const gs_frames* fr) { return fr ? fr->n_keys : 0u; }

size_t gs::frames_device_bytes(const gs_frames* fr) {
    if (!fr) return 0;
    size_t b = 0;
    auto add = [&](const auto& buf) { b += buf.cap * sizeof(*buf.p); };
    add(fr->A); add(fr->B); add(fr->gA); add(fr->gB); add(fr->Cb); add(fr->depth); add(fr->gC); add(fr->rect);
    add(fr->Mlo); add(fr->radius); add(fr->counts); add(fr->starts); add(fr->cursor); add(fr->scan_tmp);
    add(fr->sort_lists); add(fr->sort_counters); add(fr->sorted_count); add(fr->tile_loss); add(fr->keys);
    add(fr->cta_lists); add(fr->cta_list_len);
    add(fr->tmp_keys); add(fr->sorted_idx); add(fr->T_final); add(fr->n_contrib); add(fr->pose_partials);
    add(fr->dldc_ssim); add(fr->ssim_tmp); add(fr->img_off_dev); add(fr->loss_tmp); add(fr->counters);
    add(fr->st_params); add(fr->st_target); add(fr->st_image); add(fr->st_grads); add(fr->st_poses);
    add(fr->st_pose_grad); add(fr->st_loss);
    return b;
}

