// gs_server.cu - continuous-batching server of 6-DoF pose-estimation solves
// against a device-resident scene (the pose estimation of Sec. 3.4 / 4.2:
// gradient descent on the photometric L1 loss w.r.t. the camera pose).
//
// A worker thread owns a private context, stream and forward state.  Each
// iteration it (1) admits queued requests into free slots while the modelled
// device working set of the batch fits the memory the server may use (by
// default the device memory that is free, plus what its workspaces already
// hold, less a reserve; queried before each admission), (2) runs ONE batched
// forward + L1 + pose-only backward + per-slot Adam step over every active
// solve, and (3) completes the solves whose step count is reached.  If the
// workspaces cannot grow (GS_ENOMEM), the requests admitted for that
// iteration go back to the head of the queue and the iteration runs without
// them; a running solve that no longer fits goes back too and restarts later.
// Query images, poses and Adam moments stay on the device in fixed per-slot
// storage; only the batch bookkeeping (which slot is view k, its step and
// learning rate) is uploaded per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gs_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Req {
    uint64_t ticket = 0;
    gs_view view{};
    std::vector<float> image;
    double pose[12] = {};
    int steps = 0;
    double lr0 = 0.0, lr1 = 0.0;
    int slot = -1;
    int done_steps = 0;
    int enomem = 0;          // consecutive iterations that failed to grow the workspaces with it alone
    bool finished = false;
    bool cancelled = false;
    int status = GS_OK;
    double loss = 0.0;
    Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct gs_server {
    int device = 0;
    gs_ctx* ctx = nullptr;
    gs_frames* fr = nullptr;
    const gs_scene* scene = nullptr;
    gs_render_opts opts{};
    gs_server_config cfg{};
    cudaStream_t stream = nullptr;
    size_t slot_floats = 0;
    // device slot storage
    float* d_targets = nullptr;
    float* d_images = nullptr;
    double* d_pose_slot = nullptr;
    double* d_m = nullptr;
    double* d_v = nullptr;
    // device per-batch arrays (packed in batch order)
    double* d_pose_packed = nullptr;
    double* d_grad = nullptr;
    double* d_loss = nullptr;
    int* d_slot_of = nullptr;
    int* d_steps = nullptr;
    double* d_lrs = nullptr;
    // pinned staging
    int* h_slot_of = nullptr;
    int* h_steps = nullptr;
    double* h_lrs = nullptr;
    double* h_loss = nullptr;
    double* h_pose = nullptr;   // [slots][12] poses read back at completion
    // queue and slots
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker
    std::condition_variable cv_done;  // wakes waiters
    std::deque<Req*> queue;
    std::vector<Req*> slots;
    std::unordered_map<uint64_t, Req*> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    // statistics
    gs_server_stats st{};
    double views_sum = 0.0;
    double keys_per_pixel = 30.0;  // running estimate for the memory model
    double model_scale = 1.0;      // raised after a failed growth, decays back
    int inject_enomem = 0;         // test hook: iterations that report GS_ENOMEM before any device work
};

static int srv_fail(int code, const char* msg) { return gs::set_error(code, msg); }

// Modelled device bytes of a batch: per view the per-(view, Gaussian) splat
// and 2D-gradient records (96 B), per pixel the keys (20 B each in three
// arrays, at the running keys-per-pixel estimate) and the per-pixel state
// (8 B), per (chunk of 1024 Gaussians, tile) the key pass's 8 B CTA list
// entry; workspaces grow by a quarter beyond the request.
static double model_bytes(const gs_server* s, const std::vector<const gs_view*>& views) {
    double b = 0.0;
    const double n = (double)gs::scene_count(s->scene);
    for (const gs_view* v : views) {
        const double px = (double)v->width * v->height;
        const double tiles = (double)((v->width + 15) / 16) * (double)((v->height + 15) / 16);
        b += n * 96.0 + s->keys_per_pixel * px * 20.0 + px * 8.0 + std::ceil(n / 1024.0) * tiles * 8.0;
    }
    return 1.25 * s->model_scale * b;
}

// Bytes the batch's working set may occupy: the configured budget, and unless
// the budget is negative (no limit) at most what the workspaces hold plus the
// device memory that is free now, less a reserve of max(256 MiB, 2% of the
// device) for everything else on it.
static double admission_limit(gs_server* s) {
    if (s->cfg.mem_budget < 0) return 1e300;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return s->cfg.mem_budget > 0 ? (double)s->cfg.mem_budget : 1e300;
    }
    const double reserve = std::max(256.0 * (1 << 20), 0.02 * (double)total_b);
    const double avail = std::max(0.0, (double)gs::frames_device_bytes(s->fr) + (double)free_b - reserve);
    return s->cfg.mem_budget > 0 ? std::min((double)s->cfg.mem_budget, avail) : avail;
}

// Puts an admitted request back at the head of the queue (its slot freed);
// it restarts from its initial pose when admitted again.
static void requeue_locked(gs_server* s, Req* r) {
    if (r->slot >= 0 && r->slot < (int)s->slots.size() && s->slots[r->slot] == r) s->slots[r->slot] = nullptr;
    r->slot = -1;
    r->done_steps = 0;
    r->t_admit = Clock::time_point{};
    s->queue.push_front(r);
    s->st.requeued++;
}

static void finish_locked(gs_server* s, Req* r, int status) {
    r->finished = true;
    r->status = status;
    r->t_done = Clock::now();
    if (r->slot >= 0 && r->slot < (int)s->slots.size() && s->slots[r->slot] == r) s->slots[r->slot] = nullptr;
    r->slot = -1;
    if (status == GS_OK) s->st.completed++; else s->st.failed++;
}

static void worker_main(gs_server* s) {
    cudaSetDevice(s->device);
    const int S = s->cfg.max_slots;
    std::vector<gs_view> views;
    std::vector<long long> offs;
    std::vector<Req*> batch;
    std::vector<Req*> fresh;
    for (;;) {
        fresh.clear();
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            for (int k = 0; k < S; k++)
                if (s->slots[k] && s->slots[k]->cancelled) finish_locked(s, s->slots[k], GS_EBUSY);
            std::vector<const gs_view*> act;
            for (int k = 0; k < S; k++)
                if (s->slots[k]) act.push_back(&s->slots[k]->view);
            double limit = 0.0;
            bool have_limit = false;
            while (!s->queue.empty()) {
                Req* r = s->queue.front();
                if (r->cancelled) {
                    s->queue.pop_front();
                    finish_locked(s, r, GS_EBUSY);
                    continue;
                }
                int free_slot = -1;
                for (int k = 0; k < S; k++)
                    if (!s->slots[k]) { free_slot = k; break; }
                if (free_slot < 0) break;
                if (!have_limit) {
                    limit = admission_limit(s);
                    have_limit = true;
                    s->st.budget_bytes = limit >= 1e299 ? -1 : (int64_t)limit;
                }
                act.push_back(&r->view);
                // the first solve is always admitted (its growth may still fail
                // and send it back); later ones wait until the batch fits
                if (act.size() > 1 && model_bytes(s, act) > limit) {
                    act.pop_back();
                    break;
                }
                s->queue.pop_front();
                s->slots[free_slot] = r;
                r->slot = free_slot;
                r->t_admit = Clock::now();
                fresh.push_back(r);
            }
            s->st.queued = (int64_t)s->queue.size();
            bool any = false;
            for (int k = 0; k < S; k++) any |= s->slots[k] != nullptr;
            if (!any) {
                s->st.active = 0;
                s->cv.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
            batch.clear();
            for (int k = 0; k < S; k++)
                if (s->slots[k]) batch.push_back(s->slots[k]);
            s->st.active = (int64_t)batch.size();
            s->st.max_active = std::max(s->st.max_active, s->st.active);
        }
        const Clock::time_point t0 = Clock::now();
        int rc = GS_OK;
        cudaError_t e = cudaSuccess;
        // new solves: query image, initial pose, zero moments into their slot
        for (Req* r : fresh) {
            const size_t nb = sizeof(float) * 3 * (size_t)r->view.width * r->view.height;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->d_targets + (size_t)r->slot * s->slot_floats, r->image.data(), nb,
                                    cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->d_pose_slot + 12 * (size_t)r->slot, r->pose, sizeof(r->pose),
                                    cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(s->d_m + 6 * (size_t)r->slot, 0, 6 * sizeof(double), s->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(s->d_v + 6 * (size_t)r->slot, 0, 6 * sizeof(double), s->stream);
        }
        const int A = (int)batch.size();
        views.resize(A);
        offs.resize(A);
        for (int k = 0; k < A; k++) {
            Req* r = batch[k];
            views[k] = r->view;
            offs[k] = (long long)r->slot * (long long)s->slot_floats;
            s->h_slot_of[k] = r->slot;
            s->h_steps[k] = r->done_steps + 1;
            const double ph = 3.14159265358979323846 * (double)r->done_steps / (double)r->steps;
            s->h_lrs[k] = r->lr1 + 0.5 * (r->lr0 - r->lr1) * (1.0 + cos(ph));
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_slot_of, s->h_slot_of, sizeof(int) * A, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_steps, s->h_steps, sizeof(int) * A, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_lrs, s->h_lrs, sizeof(double) * A, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) rc = GS_ECUDA;
        if (rc == GS_OK && s->inject_enomem > 0) {
            s->inject_enomem--;
            rc = gs::set_error(GS_ENOMEM, "server: injected workspace growth failure");
        }
        if (rc == GS_OK) {
            gs::launch_gather_poses(A, s->d_slot_of, s->d_pose_slot, s->d_pose_packed, s->stream);
            rc = gs::render_forward_impl(s->ctx, s->scene, A, views.data(), offs.data(), s->d_pose_packed, &s->opts,
                                         s->fr, s->d_images, s->d_targets, nullptr, s->stream);
        }
        if (rc == GS_OK) {
            gs_loss L{};
            L.kind = s->cfg.mask_alpha > 0.0f ? GS_LOSS_L1_MASKED : GS_LOSS_L1;
            L.mask_alpha = s->cfg.mask_alpha;
            L.w_l1 = 1.0f;
            L.target = s->d_targets;
            L.loss = s->d_loss;
            rc = gs::render_backward_impl(s->ctx, s->scene, A, views.data(), offs.data(), s->d_pose_packed, &s->opts,
                                          s->fr, s->d_images, &L, nullptr, s->d_grad, s->stream);
        }
        if (rc == GS_OK) {
            gs::launch_pose_adam_slots(A, s->d_slot_of, s->d_pose_slot, s->d_m, s->d_v, s->d_grad, s->d_steps,
                                       s->d_lrs, 0.9, 0.999, 1e-8, s->cfg.pose_param, s->stream);
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->h_loss, s->d_loss, sizeof(double) * A, cudaMemcpyDeviceToHost, s->stream);
            for (int k = 0; k < A && e == cudaSuccess; k++)
                if (batch[k]->done_steps + 1 >= batch[k]->steps)
                    e = cudaMemcpyAsync(s->h_pose + 12 * (size_t)batch[k]->slot,
                                        s->d_pose_slot + 12 * (size_t)batch[k]->slot, 12 * sizeof(double),
                                        cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            if (e != cudaSuccess) rc = GS_ECUDA;
        } else {
            cudaStreamSynchronize(s->stream);
        }
        if (rc == GS_ENOMEM) {
            // the workspaces could not grow: this iteration's new solves go back
            // to the queue; without new ones, the most recently admitted running
            // solve does; a solve that fails alone three times in a row fails
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->model_scale = std::min(8.0, s->model_scale * 1.25);
                if (A == 1) {
                    if (++batch[0]->enomem >= 3) finish_locked(s, batch[0], GS_ENOMEM);
                    else requeue_locked(s, batch[0]);
                } else if (!fresh.empty()) {
                    for (auto it = fresh.rbegin(); it != fresh.rend(); ++it) requeue_locked(s, *it);
                } else {
                    Req* last = batch[0];
                    for (Req* r : batch)
                        if (r->t_admit > last->t_admit) last = r;
                    requeue_locked(s, last);
                }
                s->st.queued = (int64_t)s->queue.size();
                s->st.busy_ms += ms_between(t0, Clock::now());
            }
            s->cv_done.notify_all();
            std::this_thread::sleep_for(std::chrono::milliseconds(5));   // let memory come free
            continue;
        }
        s->model_scale = std::max(1.0, s->model_scale * 0.98);
        uint32_t nk = gs::frames_num_keys(s->fr);
        double px = 0.0;
        for (const gs_view& v : views) px += (double)v.width * v.height;
        if (px > 0 && nk > 0) s->keys_per_pixel = 0.7 * s->keys_per_pixel + 0.3 * ((double)nk / px);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->st.iterations++;
            s->views_sum += A;
            s->st.busy_ms += ms_between(t0, Clock::now());
            for (int k = 0; k < A; k++) {
                Req* r = batch[k];
                if (rc != GS_OK) {
                    finish_locked(s, r, rc);
                    continue;
                }
                r->done_steps++;
                r->enomem = 0;
                r->loss = s->h_loss[k];
                if (r->done_steps >= r->steps) {
                    memcpy(r->pose, s->h_pose + 12 * (size_t)r->slot, sizeof(r->pose));
                    finish_locked(s, r, GS_OK);
                }
            }
        }
        s->cv_done.notify_all();
    }
}

extern "C" {

int gs_server_create(int device, const gs_scene* scene, const gs_render_opts* opts, const gs_server_config* cfg,
                     gs_server** out) {
    if (!scene || !opts || !cfg || !out) return srv_fail(GS_EINVAL, "gs_server_create: NULL argument");
    if (cfg->max_slots < 1 || cfg->max_slots > 4096 || cfg->max_width < 1 || cfg->max_height < 1 ||
        cfg->queue_capacity < 1 || !(cfg->mask_alpha >= 0.0f && cfg->mask_alpha < 1.0f) ||
        (cfg->pose_param != GS_POSE_SE3 && cfg->pose_param != GS_POSE_TXSO3))
        return srv_fail(GS_EINVAL, "gs_server_create: bad configuration");
    *out = nullptr;
    gs_server* s = new (std::nothrow) gs_server();
    if (!s) return srv_fail(GS_ENOMEM, "gs_server_create: host allocation failed");
    s->device = device;
    s->scene = scene;
    s->opts = *opts;
    s->opts.flags = 0;
    s->cfg = *cfg;
    int rc = gs_ctx_create(device, &s->ctx);
    if (rc == GS_OK && cfg->tuning.scatter_chunk != 0) rc = gs_ctx_set_tuning(s->ctx, &cfg->tuning);
    if (rc == GS_OK) rc = gs_frames_create(s->ctx, &s->fr);
    if (rc != GS_OK) { gs_server_destroy(s); return rc; }
    const int S = cfg->max_slots;
    s->slot_floats = ((size_t)3 * cfg->max_width * cfg->max_height + 63) & ~(size_t)63;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    auto dm = [&](void** p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
    auto hm = [&](void** p, size_t b) { if (e == cudaSuccess) e = cudaMallocHost(p, b); };
    dm((void**)&s->d_targets, sizeof(float) * s->slot_floats * S);
    dm((void**)&s->d_images, sizeof(float) * s->slot_floats * S);
    dm((void**)&s->d_pose_slot, sizeof(double) * 12 * S);
    dm((void**)&s->d_m, sizeof(double) * 6 * S);
    dm((void**)&s->d_v, sizeof(double) * 6 * S);
    dm((void**)&s->d_pose_packed, sizeof(double) * 12 * S);
    dm((void**)&s->d_grad, sizeof(double) * 6 * S);
    dm((void**)&s->d_loss, sizeof(double) * S);
    dm((void**)&s->d_slot_of, sizeof(int) * S);
    dm((void**)&s->d_steps, sizeof(int) * S);
    dm((void**)&s->d_lrs, sizeof(double) * S);
    hm((void**)&s->h_slot_of, sizeof(int) * S);
    hm((void**)&s->h_steps, sizeof(int) * S);
    hm((void**)&s->h_lrs, sizeof(double) * S);
    hm((void**)&s->h_loss, sizeof(double) * S);
    hm((void**)&s->h_pose, sizeof(double) * 12 * S);
    if (e != cudaSuccess) {
        cudaGetLastError();
        gs_server_destroy(s);
        return srv_fail(GS_ENOMEM, "gs_server_create: device or pinned allocation failed");
    }
    s->slots.assign(S, nullptr);
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        gs_server_destroy(s);
        return srv_fail(GS_ENOMEM, "gs_server_create: cannot start the worker thread");
    }
    *out = s;
    return GS_OK;
}

int gs_solve_submit(gs_server* s, const gs_solve_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket) return srv_fail(GS_EINVAL, "gs_solve_submit: NULL argument");
    const gs_view& v = req->view;
    if (v.width < 1 || v.height < 1 || v.width > s->cfg.max_width || v.height > s->cfg.max_height ||
        (size_t)3 * v.width * v.height > s->slot_floats)
        return srv_fail(GS_EINVAL, "gs_solve_submit: image size outside the server's limits");
    if (!(v.fx > 0.0f) || !(v.fy > 0.0f) || !req->image || req->steps < 1)
        return srv_fail(GS_EINVAL, "gs_solve_submit: bad intrinsics, image or step count");
    for (int k = 0; k < 12; k++)
        if (!std::isfinite(req->init_pose[k])) return srv_fail(GS_EINVAL, "gs_solve_submit: non-finite pose");
    Req* r = new (std::nothrow) Req();
    if (!r) return srv_fail(GS_ENOMEM, "gs_solve_submit: host allocation failed");
    r->view = v;
    try {
        r->image.assign(req->image, req->image + (size_t)3 * v.width * v.height);
    } catch (...) {
        delete r;
        return srv_fail(GS_ENOMEM, "gs_solve_submit: host allocation failed");
    }
    memcpy(r->pose, req->init_pose, sizeof(r->pose));
    r->steps = req->steps;
    r->lr0 = req->lr_start;
    r->lr1 = req->lr_end;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if ((int)s->queue.size() >= s->cfg.queue_capacity) {
            delete r;
            return srv_fail(GS_EBUSY, "gs_solve_submit: queue full");
        }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
        s->st.submitted++;
        s->st.queued = (int64_t)s->queue.size();
        *ticket = r->ticket;
    }
    s->cv.notify_one();
    return GS_OK;
}

static void fill_result(const Req* r, gs_solve_result* out) {
    memcpy(out->pose, r->pose, sizeof(out->pose));
    out->loss = r->loss;
    out->latency_ms = ms_between(r->t_submit, r->t_done);
    out->queue_ms = r->t_admit != Clock::time_point{} ? ms_between(r->t_submit, r->t_admit) : 0.0;
    out->steps_done = r->done_steps;
    out->status = r->status;
}

int gs_solve_wait(gs_server* s, uint64_t ticket, int timeout_ms, gs_solve_result* out) {
    if (!s || !out) return srv_fail(GS_EINVAL, "gs_solve_wait: NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return srv_fail(GS_EINVAL, "gs_solve_wait: unknown ticket");
    Req* r = it->second;
    if (!r->finished && timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->finished; });
    if (!r->finished) return timeout_ms > 0 ? srv_fail(GS_ETIMEOUT, "gs_solve_wait: timed out") : GS_PENDING;
    fill_result(r, out);
    s->reqs.erase(it);
    delete r;
    return GS_OK;
}

int gs_solve_poll(gs_server* s, uint64_t ticket, gs_solve_result* out) { return gs_solve_wait(s, ticket, 0, out); }

int gs_solve_cancel(gs_server* s, uint64_t ticket) {
    if (!s) return srv_fail(GS_EINVAL, "gs_solve_cancel: NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return srv_fail(GS_EINVAL, "gs_solve_cancel: unknown ticket");
        it->second->cancelled = true;
    }
    s->cv.notify_one();
    return GS_OK;
}

int gs_server_inject_enomem(gs_server* s, int iterations) {
    if (!s || iterations < 0) return srv_fail(GS_EINVAL, "gs_server_inject_enomem: bad argument");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->inject_enomem = iterations;
    }
    s->cv.notify_one();
    return GS_OK;
}

int gs_server_stats_get(gs_server* s, gs_server_stats* out) {
    if (!s || !out) return srv_fail(GS_EINVAL, "gs_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->views_per_iteration = s->st.iterations ? s->views_sum / (double)s->st.iterations : 0.0;
    return GS_OK;
}

void gs_server_destroy(gs_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (auto& kv : s->reqs) delete kv.second;
    s->reqs.clear();
    void* dptr[] = {s->d_targets, s->d_images, s->d_pose_slot, s->d_m, s->d_v, s->d_pose_packed, s->d_grad,
                    s->d_loss, s->d_slot_of, s->d_steps, s->d_lrs};
    for (void* p : dptr)
        if (p) cudaFree(p);
    void* hptr[] = {s->h_slot_of, s->h_steps, s->h_lrs, s->h_loss, s->h_pose};
    for (void* p : hptr)
        if (p) cudaFreeHost(p);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->fr) gs_frames_destroy(s->fr);
    if (s->ctx) gs_ctx_destroy(s->ctx);
    delete s;
}

}  // extern "C"
