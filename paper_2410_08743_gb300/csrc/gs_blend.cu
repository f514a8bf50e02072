// gs_blend.cu - per-tile alpha compositing (Sec. 3.1, Eq. 3-4) and its
// reverse-replay backward (the prior art's gradients w.r.t. the 2D splat
// parameters, the inputs of the pose chain rule of Sec. 3.2).
//
// One CTA per 16x16 tile.  The forward consumes the tile's depth-sorted list
// in batches of 128 splats staged in shared memory; each warp compacts a batch
// to the entries that can reach its pixel block and walks them in lock step,
// a pixel stopping before the splat that would bring its transmittance below
// t_min, and the CTA leaves once every pixel has stopped.  The backward walks
// the same lists back to front from each pixel's last blended entry,
// rebuilding T by division; with two pixels per thread each warp stages its
// own 32-entry chunks (no block barrier), and every splat's nine 2D gradients
// are reduced over the warp before one set of vector atomics per warp.
#include <cuda_runtime.h>

#include "gs_block_sort.cuh"
#include "gs_internal.cuh"

namespace gs {

#define BATCH 128

// ------------------------------------------------------------ paired FP32
// add/sub/mul/fma.rn.f32x2 (sm_100 and later) compute two IEEE
// round-to-nearest results in one instruction, bit for bit those of the
// scalar operations, so the two pixels of a lane share their issue slots and
// every decision stays the one the scalar sequence takes.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float f2_lo(f2_t x) {
    float lo;
    asm("{.reg .f32 hi;\n\tmov.b64 {%0, hi}, %1;}" : "=f"(lo) : "l"(x));
    return lo;
}
__device__ __forceinline__ float f2_hi(f2_t x) {
    float hi;
    asm("{.reg .f32 lo;\n\tmov.b64 {lo, %0}, %1;}" : "=f"(hi) : "l"(x));
    return hi;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Shared-memory splat batch.  The fields of the per-pixel arithmetic are
// stored twice, as (x, x) pairs, so that the paired operations of the
// two-pixel blends take a splat operand straight from one (broadcast) load:
//   P0 = (mu.x, mu.x, a', a'), P1 = (mu.y, mu.y, b', b'), P2 = (c', c', o, o),
//   P3 = (r, r, g, g), P4 = (blue, blue), with (a', b', c') the scaled conic.
struct SplatBatch {
    ulonglong2 P0[BATCH];
    ulonglong2 P1[BATCH];
    ulonglong2 P2[BATCH];
    ulonglong2 P3[BATCH];
    f2_t P4[BATCH];
    float2 H[BATCH];   // half-extents of the box holding every pixel with alpha >= alpha_min
    float Qt[BATCH];   // widened bound on the conic's quadratic form at such pixels (INFINITY: no bound)
};

// Per-warp chunk of WCH staged entries (the records as in SplatBatch) and the
// warp's accumulator slots, nine per entry, of the backward.
#define WCH 32
struct WarpChunk {
    ulonglong2 P0[WCH];
    ulonglong2 P1[WCH];
    ulonglong2 P2[WCH];
    ulonglong2 P3[WCH];
    f2_t P4[WCH];
    float acc[WCH * 9];
};

// Entry j as the scalar records A = (mu.x, mu.y, a', b'), B = (c', o, r, g)
// and blue.
__device__ __forceinline__ float4 sb_A(const SplatBatch& sb, int j) {
    const ulonglong2 p0 = sb.P0[j], p1 = sb.P1[j];
    return make_float4(f2_lo(p0.x), f2_lo(p1.x), f2_lo(p0.y), f2_lo(p1.y));
}
__device__ __forceinline__ float4 sb_B(const SplatBatch& sb, int j) {
    const ulonglong2 p2 = sb.P2[j], p3 = sb.P3[j];
    return make_float4(f2_lo(p2.x), f2_lo(p2.y), f2_lo(p3.x), f2_lo(p3.y));
}
__device__ __forceinline__ float sb_Cb(const SplatBatch& sb, int j) { return f2_lo(sb.P4[j]); }

// Conservative half-extents of {d : o exp(-1/2 d^T Q d) >= alpha_min}, the
// ellipse d^T Q d <= R^2 with R^2 = 2 ln(o / alpha_min): |dx| <= R sqrt(Q^-1_xx),
// |dy| <= R sqrt(Q^-1_yy), widened by 1% + 0.01 px (far above the FP32 error
// of the alpha test), so a pixel outside the box is certainly skipped by
// pair_alpha and the box changes no decision.  Conics with det < 1e-4 a c get
// no box: there FP32 cancellation in det (relative error ~1e-7 a c / det)
// could approach the 1% margin.  The hardware approximations used here (log,
// quotient, reciprocal square root) are off by a few units in the last place,
// relatively far inside the 1% margin; R^2 gets 2e-6 more, above the
// logarithm's absolute error near o = alpha_min.
__device__ __forceinline__ float2 alpha_box(const float4 a, const float4 b, float amin) {
    if (!(b.y >= amin)) return make_float2(-1.0f, -1.0f);
    const float R2 = fmaf(2.0f, __logf(__fdividef(b.y, amin)), 2e-6f);
    const float dq = a.z * b.x - a.w * a.w;
    if (!(dq > 1e-4f * a.z * b.x)) return make_float2(INFINITY, INFINITY);
    const float s = __fdividef(R2, dq);
    const float hx2 = s * b.x, hy2 = s * a.z;
    const float hx = hx2 * rsqrtf(hx2), hy = hy2 * rsqrtf(hy2);
    return make_float2(fmaf(hx, 1.01f, 0.01f), fmaf(hy, 1.01f, 0.01f));
}

// Bound for the per-warp ellipse test: a pixel with alpha >= alpha_min has
// q = d^T Q d <= R^2 = 2 ln(o / alpha_min).  The returned threshold is
// R^2 widened by 2% + 1e-3, which keeps the alpha of every pixel whose FP32 q
// exceeds it below alpha_min (1 - 5e-4) whatever the exp error.  The bound is
// only given for well-conditioned positive-definite conics (det >= 1e-2 a c),
// where the FP32 error of a q evaluation is below 1e-3 q; others get INFINITY.
__device__ __forceinline__ float ellipse_bound(const float4 a, const float4 b, float amin) {
    if (!(b.y >= amin)) return INFINITY;
    const float dq = a.z * b.x - a.w * a.w;
    if (!(a.z > 0.0f && b.x > 0.0f && dq >= 1e-2f * a.z * b.x)) return INFINITY;
    return fmaf(2.0f * __logf(__fdividef(b.y, amin)), 1.02f, 1e-3f);   // 1e-3 >> the approximations' error
}

// The staged conic is scaled so that the exponent of Eq. 3 comes out in base
// 2, ready for ex2: with L = log2(e),
//   a' = -L a / 2, b' = -L b, c' = -L c / 2, and
//   power2 = a' dx^2 + b' dx dy + c' dy^2 = L power, alpha = o 2^power2.
// The ellipse bound is staged in the same units (q <= Qt iff power2 >= Qt').
#define GS_KA (-0.72134752044448170f)   // -L / 2
#define GS_KB (-1.44269504088896340f)   // -L
#define GS_IKA (-1.38629436111989061f)  // 1 / GS_KA = -2 ln 2
#define GS_IKB (-0.69314718055994531f)  // 1 / GS_KB = -ln 2

// Culling bounds of a splat record a = (mu.x, mu.y, a, b), b = (c, o, r, g)
// from its conic, which is then scaled in place (a.z, a.w, b.x).
__device__ __forceinline__ void stage_prepare(float4& a, float4& b, float amin, float2& h, float& qt) {
    h = alpha_box(a, b, amin);
    qt = GS_KA * ellipse_bound(a, b, amin);   // -INFINITY: no bound
    a.z *= GS_KA;
    a.w *= GS_KB;
    b.x *= GS_KA;
}

// Stores the prepared record (scaled conic) as entry j of a batch in pairs;
// cb = blue.
template <class Batch>
__device__ __forceinline__ void stage_store(Batch& sb, int j, const float4 a, const float4 b, float cb) {
    sb.P0[j] = make_ulonglong2(f2_pack(a.x, a.x), f2_pack(a.z, a.z));
    sb.P1[j] = make_ulonglong2(f2_pack(a.y, a.y), f2_pack(a.w, a.w));
    sb.P2[j] = make_ulonglong2(f2_pack(b.x, b.x), f2_pack(b.y, b.y));
    sb.P3[j] = make_ulonglong2(f2_pack(b.z, b.z), f2_pack(b.w, b.w));
    sb.P4[j] = f2_pack(cb, cb);
}

// Stages batch entry j: culling bounds from the unscaled conic, then the
// scaled record.
__device__ __forceinline__ void stage_entry(SplatBatch& sb, int j, float4 a, float4 b, float cb, float amin) {
    float2 h;
    float qt;
    stage_prepare(a, b, amin, h, qt);
    sb.H[j] = h;
    sb.Qt[j] = qt;
    stage_store(sb, j, a, b, cb);
}

// Splat record A of entry k with its projected mean moved to the tile origin
// (ox, oy) and corrected by the residual Mlo.  A.x - ox is exact whenever the
// FP32 mean lies within a factor of two of the origin (or ox = 0); otherwise it
// is off by at most half an ulp of an offset far larger than the tile, where the
// splat's alpha varies slowly.  So the staged mean keeps ~1e-9 px where it
// matters, and pixel offsets in the tile are small exact integers.
__device__ __forceinline__ float4 stage_mean(const SplatArrays& sp, size_t k, float ox, float oy) {
    float4 a = sp.A[k];
    const float2 lo = sp.Mlo[k];
    a.x = __fadd_rn(__fsub_rn(a.x, ox), lo.x);
    a.y = __fadd_rn(__fsub_rn(a.y, oy), lo.y);
    return a;
}

// Pixel of thread tid within its 16x16 tile.  Each warp covers an 8x4 block
// (the 8 warps tile the 16x16 pixels as 2 columns x 4 rows), which a small
// splat's alpha box overlaps in fewer warps than a 16x2 strip would.
#define WARP_W 8
#define WARP_H 4
__device__ __forceinline__ int tile_px(int tid) { return ((tid >> 5) & 1) * WARP_W + (tid & (WARP_W - 1)); }
__device__ __forceinline__ int tile_py(int tid) { return (tid >> 6) * WARP_H + ((tid & 31) >> 3); }
__device__ __forceinline__ float warp_x0(int tid) { return (float)(((tid >> 5) & 1) * WARP_W); }
__device__ __forceinline__ float warp_y0(int tid) { return (float)((tid >> 6) * WARP_H); }

// Per-warp compaction of a staged batch: the entries (in order) whose alpha
// box can touch a pixel of this warp's 8 x fh footprint (x in [fx0, fx0+7],
// y in [fy0, fy0+fh-1]) and whose ellipse q <= Qt meets the footprint's
// rectangle.  Both tests are conservative (0.01 px slack over the per-pixel
// box test; the widened Qt of ellipse_bound), so skipping the other entries
// changes no decision.  The ellipse test drops the entries whose box corner
// alone reaches the footprint: about a fifth of the box hits for the
// rotated, elongated splats of real scenes.
// Returns the number of entries written to wl.
// Footprint test of one staged entry: a = (mu.x, mu.y, a', b') and c' the
// scaled conic, h its alpha box, qt its scaled ellipse bound (-INFINITY: none).
__device__ __forceinline__ bool footprint_hit(const float4 a, float cc, const float2 h, float qt, float fx0, float fy0,
                                              int fh) {
    const float fx1 = fx0 + (float)(WARP_W - 1), fy1 = fy0 + (float)(fh - 1);
    bool hit = (a.x + h.x + 0.01f >= fx0) && (a.x - h.x - 0.01f <= fx1) && (a.y + h.y + 0.01f >= fy0) &&
               (a.y - h.y - 0.01f <= fy1);
    if (hit && qt > -INFINITY) {
        // Maximum of the scaled exponent p(d) = a' dx^2 + b' dx dy + c' dy^2
        // (d = p - mu; -L/2 times the quadratic form q) over the
        // footprint.  With the centre outside, a concave p is largest on
        // an edge whose outside holds the centre: on such an edge the
        // other offset is the 1D maximiser clamped to the edge.
        const float dxl = fx0 - a.x, dxr = fx1 - a.x, dyl = fy0 - a.y, dyr = fy1 - a.y;
        float best = 0.0f;
        const bool ox = dxl > 0.0f || dxr < 0.0f, oy = dyl > 0.0f || dyr < 0.0f;
        if (ox || oy) best = -INFINITY;
        // (the 1D maximiser needs no exact quotient: an error e in it
        // lowers p by only |c'| e^2, far inside the bound's 2% margin,
        // and the p evaluated is that of a point of the edge either way)
        if (ox) {
            const float dx = dxl > 0.0f ? dxl : dxr;
            const float dy = fminf(fmaxf(__fdividef(-0.5f * a.w * dx, cc), dyl), dyr);
            best = fmaxf(best, fmaf(a.z * dx, dx, fmaf(a.w * dx, dy, cc * dy * dy)));
        }
        if (oy) {
            const float dy = dyl > 0.0f ? dyl : dyr;
            const float dx = fminf(fmaxf(__fdividef(-0.5f * a.w * dy, a.z), dxl), dxr);
            best = fmaxf(best, fmaf(a.z * dx, dx, fmaf(a.w * dx, dy, cc * dy * dy)));
        }
        hit = best >= qt;
    }
    return hit;
}

__device__ __forceinline__ int warp_compact(const SplatBatch& sb, int cnt, float fx0, float fy0,
                                            unsigned char* wl, int fh = WARP_H) {
    const int lane = threadIdx.x & 31;
    int n = 0;
    for (int r = 0; r < cnt; r += 32) {
        const int e = r + lane;
        const bool hit = e < cnt && footprint_hit(sb_A(sb, e), f2_lo(sb.P2[e].x), sb.H[e], sb.Qt[e], fx0, fy0, fh);
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) wl[n + __popc(m & ((1u << lane) - 1u))] = (unsigned char)e;
        n += __popc(m);
    }
    __syncwarp();
    return n;
}

// alpha of one (pixel, splat) pair from the staged (scaled) conic with a fixed
// operation sequence, which every blend uses, so that the forward and the
// backward take the same skip decisions:
//   power2 = (a' dx^2 + c' dy^2) + b' dx dy = log2(e) power, d = p - mu_hat,
//   power = -1/2 (a dx^2 + c dy^2) - b dx dy (Eq. 3), alpha = o 2^power2;
//   returns false when the pair is skipped (power > 0 or alpha < alpha_min).
__device__ __forceinline__ float pair_power2(const float4 a, const float4 b, float dxx_a, float dx, float dy) {
    return __fmaf_rn(a.w, __fmul_rn(dx, dy), __fmaf_rn(b.x, __fmul_rn(dy, dy), dxx_a));
}
__device__ __forceinline__ bool pair_alpha(const float4 a, const float4 b, float dx, float dy, float amin, float amax,
                                           float& G, float& alpha, bool& clamped) {
    const float pw = pair_power2(a, b, __fmul_rn(a.z, __fmul_rn(dx, dx)), dx, dy);
    if (pw > 0.0f) return false;
    G = fast_exp2(pw);
    const float ar = __fmul_rn(b.y, G);
    clamped = ar > amax;
    alpha = clamped ? amax : ar;
    return alpha >= amin;
}

__global__ void __launch_bounds__(GS_TILE_PIX) k_blend_fwd(int n_views, const int* __restrict__ tile_base,
                                                           const ViewDev* __restrict__ views, RenderParams rp,
                                                           SplatArrays sp, int n, const uint32_t* __restrict__ starts,
                                                           const uint32_t* __restrict__ sorted_idx, uint32_t cap,
                                                           float* __restrict__ image, float* __restrict__ T_final,
                                                           uint32_t* __restrict__ n_contrib,
                                                           const float* __restrict__ target,
                                                           float* __restrict__ tile_loss,
                                                           unsigned long long* __restrict__ counters) {
    __shared__ SplatBatch sb;
    __shared__ float s_red[GS_TILE_PIX / 32];
    const int t = blockIdx.x;
    const int v = view_of_tile(tile_base, n_views, t);
    const ViewDev& vd = views[v];
    const int W = vd.W, H = vd.H, gw = vd.gw;
    const int lt = t - vd.tile_base;
    const int px = (lt % gw) * GS_TILE + tile_px(threadIdx.x);
    const int py = (lt / gw) * GS_TILE + tile_py(threadIdx.x);
    const bool inside = px < W && py < H;
    // tile-relative pixel coordinates (the staged means are moved to the same origin)
    const float ox = (float)((lt % gw) * GS_TILE), oy = (float)((lt / gw) * GS_TILE);
    const float fpx = (float)tile_px(threadIdx.x), fpy = (float)tile_py(threadIdx.x);
    uint32_t s = starts[t], e = starts[t + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    const size_t vbase = (size_t)v * n;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last = 0, n_eval = 0, n_blend = 0;
    bool done = !inside;
    for (uint32_t base = s; base < e; base += BATCH) {
        if (__syncthreads_count(done) == GS_TILE_PIX) break;
        const uint32_t j = base + threadIdx.x;
        if (counters && threadIdx.x == 0) atomicAdd(counters + 4, (unsigned long long)min((uint32_t)BATCH, e - base));
        if (threadIdx.x < BATCH && j < e) {
            const size_t k = vbase + sorted_idx[j];
            stage_entry(sb, threadIdx.x, stage_mean(sp, k, ox, oy), sp.B[k], sp.Cb[k], rp.alpha_min);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)BATCH, e - base);
        if (!done) {
            for (int jj = 0; jj < cnt; jj++) {
                const float4 a = sb_A(sb, jj);
                const float2 h = sb.H[jj];
                n_eval++;
                const float dx = __fsub_rn(fpx, a.x), dy = __fsub_rn(fpy, a.y);
                if (fabsf(dx) > h.x || fabsf(dy) > h.y) continue;
                const float4 b = sb_B(sb, jj);
                float G, alpha;
                bool cl;
                if (!pair_alpha(a, b, dx, dy, rp.alpha_min, rp.alpha_max, G, alpha, cl)) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < rp.t_min) { done = true; break; }
                n_blend++;
                const float w = alpha * T;
                C0 = fmaf(b.z, w, C0);
                C1 = fmaf(b.w, w, C1);
                C2 = fmaf(sb_Cb(sb, jj), w, C2);
                T = Tn;
                last = base - s + jj + 1;
            }
        }
    }
    float l1 = 0.0f;
    if (inside) {
        const size_t p = (size_t)py * W + px;
        const size_t np = (size_t)W * H;
        float* img = image + vd.img_off;
        C0 = fmaf(T, rp.bg[0], C0);
        C1 = fmaf(T, rp.bg[1], C1);
        C2 = fmaf(T, rp.bg[2], C2);
        img[p] = C0;
        img[np + p] = C1;
        img[2 * np + p] = C2;
        T_final[vd.pix_off + p] = T;
        n_contrib[vd.pix_off + p] = last;
        if (target) {
            const float* tg = target + vd.img_off;
            l1 = fabsf(C0 - tg[p]) + fabsf(C1 - tg[np + p]) + fabsf(C2 - tg[2 * np + p]);
        }
    }
    if (target) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = l1;
        __syncthreads();
        if (threadIdx.x == 0) {
            float acc = 0.0f;
            for (int w = 0; w < GS_TILE_PIX / 32; w++) acc += s_red[w];
            tile_loss[t] = acc;
        }
    }
    if (counters) {
        unsigned long long ce = n_eval, cbl = n_blend;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ce += __shfl_xor_sync(0xffffffffu, ce, o);
            cbl += __shfl_xor_sync(0xffffffffu, cbl, o);
        }
        if ((threadIdx.x & 31) == 0) { atomicAdd(counters, ce); atomicAdd(counters + 1, cbl); }
    }
}

// ------------------------------------------------------------ forward with lazy tile sort
// The forward blend usually stops long before the end of a tile's list (every
// pixel saturates), so the tile's keys are sorted only as far as they are
// consumed.  A list of at most LZ_CAP keys is sorted whole in shared memory.
// A longer list is bucketed by depth (LZ_NB buckets spanning the tile's depth
// range; bucket order is depth order and equal depths share a bucket), then
// runs of consecutive buckets of at most LZ_CAP keys are sorted and blended one
// after another until every pixel has stopped.  The concatenation of the
// sorted runs is exactly the (depth, index) order, so the image equals the one
// of a fully sorted list.  A run is gathered grouped by bucket and each bucket
// is sorted on its own (buckets hold a few keys each), with a radix sort of
// the whole run where a bucket is large.  The sorted prefix and its length go
// to sorted_idx / sorted_count for the backward pass, which never reads past
// it.
#define LZ_NB_BITS 9
#define LZ_NB (1 << LZ_NB_BITS)
// the first run of buckets is cut at LZ_FIRST keys: most tiles stop within
// a few hundred entries, so a short first run sorts little that is not used
#define LZ_FIRST 512
// buckets of at most LZ_SMALL keys are insertion-sorted by one thread
#define LZ_SMALL 32
#define LZ_T GS_TILE_PIX

template <int LZ_CAP, int NT>
struct LazySmem {
    union {
        struct {
            unsigned long long b0[LZ_CAP];
            unsigned long long b1[LZ_CAP];
        } srt;
        SplatBatch sb;  // blending reuses the sort buffers
    } u;
    uint32_t hist[(NT / 32) * 256];  // radix histograms, then bucket cursors
    uint32_t bstart[LZ_NB + 1];
    unsigned char wl[NT / 32][BATCH];  // per-warp compacted batch entries
};

// PX pixels per thread (1 or 2): each warp covers an 8 x (4 PX) pixel block.
// Two pixels per thread share every shared-memory read of a splat and give
// each thread two independent compositing chains.
// CNT: accumulate the work counters (pairs evaluated and blended, entries read
// and sorted, warp entries); the timed variant carries none of that bookkeeping.
template <int LZ_CAP, int PX, bool CNT>
__global__ void __launch_bounds__(GS_TILE_PIX / PX, PX == 1 ? 4 : 8) k_blend_fwd_lazy(
    int n_views, const int* __restrict__ tile_base, const ViewDev* __restrict__ views, RenderParams rp, SplatArrays sp,
    int n, const uint32_t* __restrict__ starts, unsigned long long* __restrict__ keys,
    unsigned long long* __restrict__ tmp, uint32_t* __restrict__ sorted_idx, uint32_t* __restrict__ sorted_count,
    uint32_t cap, float* __restrict__ image, float* __restrict__ T_final, uint32_t* __restrict__ n_contrib,
    const float* __restrict__ target, float* __restrict__ tile_loss, unsigned long long* __restrict__ counters) {
    constexpr int NT = GS_TILE_PIX / PX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LazySmem<LZ_CAP, NT>& sm = *reinterpret_cast<LazySmem<LZ_CAP, NT>*>(smem_raw);
    __shared__ float s_red[NT / 32];
    __shared__ uint32_t s_warp[NT / 32];
    __shared__ uint32_t s_mm[2];
    const int t = blockIdx.x;
    const int v = view_of_tile(tile_base, n_views, t);
    const ViewDev& vd = views[v];
    const int W = vd.W, H = vd.H, gw = vd.gw;
    const int lt = t - vd.tile_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int wx0 = (wid & 1) * WARP_W, wy0 = (wid >> 1) * (WARP_H * PX);
    const int lx = wx0 + (lane & (WARP_W - 1)), ly = wy0 + (lane >> 3);
    const int tx0 = (lt % gw) * GS_TILE, ty0 = (lt / gw) * GS_TILE;
    // tile-relative pixel coordinates (the staged means are moved to the same origin)
    const float ox = (float)tx0, oy = (float)ty0;
    const float fpx = (float)lx;
    uint32_t s = starts[t], e = starts[t + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    const uint32_t n_list = e - s;
    const size_t vbase = (size_t)v * n;
    float pT[PX], C0[PX], C1[PX], C2[PX];
    uint32_t last[PX];
    bool done[PX];
#pragma unroll
    for (int q = 0; q < PX; q++) {
        pT[q] = 1.0f; C0[q] = C1[q] = C2[q] = 0.0f; last[q] = 0;
        done[q] = !(tx0 + lx < W && ty0 + ly + WARP_H * q < H);
    }
    auto all_done = [&]() -> bool {
        bool d = true;
#pragma unroll
        for (int q = 0; q < PX; q++) d = d && done[q];
        return d;
    };
    uint32_t n_eval = 0, n_blend = 0, n_read = 0, n_went = 0;
    uint32_t n_sorted = 0;
    // two-pixel state in pairs: (transmittance, colour) of the lane's pixels
    const float amin = rp.alpha_min, amax = rp.alpha_max, tmin = rp.t_min;
    const f2_t fpx2 = f2_pack(fpx, fpx), fpy2 = f2_pack((float)ly, (float)(ly + WARP_H));
    const f2_t one2 = f2_pack(1.0f, 1.0f);
    f2_t pT2 = one2, Cr2 = f2_pack(0.0f, 0.0f), Cg2 = Cr2, Cb2 = Cr2;

    // Blends list positions [p0, p1) read from sorted_idx; returns true when
    // every pixel of the tile has stopped.
    auto blend_range = [&](uint32_t p0, uint32_t p1) -> bool {
        static_assert(NT >= BATCH, "one staged entry per thread");
        for (uint32_t base = p0; base < p1; base += BATCH) {
            const int cnt = (int)min((uint32_t)BATCH, p1 - base);
            // the entry's records are loaded before the barrier (their latency
            // overlaps the wait) and staged after it
            const bool have = (int)threadIdx.x < cnt;
            float4 ra = make_float4(0.0f, 0.0f, 0.0f, 0.0f), rb = ra;
            float rc = 0.0f;
            if (have) {
                const size_t k = vbase + sorted_idx[s + base + threadIdx.x];
                ra = stage_mean(sp, k, ox, oy);
                rb = sp.B[k];
                rc = sp.Cb[k];
            }
            if (__syncthreads_count(all_done()) == NT) return true;
            n_read += (threadIdx.x == 0) ? (uint32_t)cnt : 0u;
            if (have) stage_entry(sm.u.sb, threadIdx.x, ra, rb, rc, rp.alpha_min);
            __syncthreads();
            unsigned char* wl = sm.wl[wid];
            // a warp whose pixels have all stopped skips the batch
            const int nw = __all_sync(0xffffffffu, all_done())
                               ? 0
                               : warp_compact(sm.u.sb, cnt, (float)wx0, (float)wy0, wl, WARP_H * PX);
            // the warp walks its entries in lock step; a pixel that has stopped
            // or whose alpha is below alpha_min blends nothing (weight 0)
            if (CNT) n_went += (uint32_t)nw;
            if constexpr (PX == 2) {
                for (int qq = 0; qq < nw; qq++) {
                    const int jj = wl[qq];
                    const uint32_t pos1 = base + (uint32_t)jj + 1u;
                    const ulonglong2 p0 = sm.u.sb.P0[jj], p1 = sm.u.sb.P1[jj], p2 = sm.u.sb.P2[jj];
                    // alpha of both pixels (Eq. 3) with pair_alpha's operation
                    // sequence, paired: the lanes of each pair share dx
                    const f2_t dx2 = f2_sub(fpx2, p0.x), dy2 = f2_sub(fpy2, p1.x);
                    const f2_t pw2 =
                        f2_fma(p1.y, f2_mul(dx2, dy2), f2_fma(p2.x, f2_mul(dy2, dy2), f2_mul(p0.y, f2_mul(dx2, dx2))));
                    const float pw0 = f2_lo(pw2), pw1 = f2_hi(pw2);
                    const f2_t ar2 = f2_mul(p2.y, f2_pack(fast_exp2(pw0), fast_exp2(pw1)));
                    const float ar0 = f2_lo(ar2), ar1 = f2_hi(ar2);
                    // the decisions of pair_alpha (alpha >= alpha_min iff the
                    // unclamped ar is, as alpha_max >= alpha_min; a NaN skips)
                    const bool ok0 = !done[0] && !(pw0 > 0.0f) && ar0 >= amin;
                    const bool ok1 = !done[1] && !(pw1 > 0.0f) && ar1 >= amin;
                    const float al0 = fminf(ar0, amax), al1 = fminf(ar1, amax);
                    if (CNT) {
                        const float2 h = sm.u.sb.H[jj];
                        const bool inx = fabsf(f2_lo(dx2)) <= h.x;
                        n_eval += (!done[0] && inx && fabsf(f2_lo(dy2)) <= h.y) +
                                  (!done[1] && inx && fabsf(f2_hi(dy2)) <= h.y);
                    }
                    if (!__any_sync(0xffffffffu, ok0 || ok1)) {
                        // no pixel blends: the warp leaves once all have stopped
                        if (__all_sync(0xffffffffu, done[0] && done[1])) break;
                        continue;
                    }
                    // Eq. 4 front to back; stop before the splat that would take
                    // the transmittance below t_min
                    const f2_t Tn2 = f2_mul(pT2, f2_sub(one2, f2_pack(al0, al1)));
                    const float Tn0 = f2_lo(Tn2), Tn1 = f2_hi(Tn2);
                    const bool st0 = ok0 && Tn0 < tmin, st1 = ok1 && Tn1 < tmin;
                    const bool bl0 = ok0 && !st0, bl1 = ok1 && !st1;
                    done[0] = done[0] || st0;
                    done[1] = done[1] || st1;
                    const f2_t w2 = f2_mul(f2_pack(bl0 ? al0 : 0.0f, bl1 ? al1 : 0.0f), pT2);
                    const ulonglong2 p3 = sm.u.sb.P3[jj];
                    Cr2 = f2_fma(p3.x, w2, Cr2);
                    Cg2 = f2_fma(p3.y, w2, Cg2);
                    Cb2 = f2_fma(sm.u.sb.P4[jj], w2, Cb2);
                    pT2 = f2_pack(bl0 ? Tn0 : f2_lo(pT2), bl1 ? Tn1 : f2_hi(pT2));
                    last[0] = bl0 ? pos1 : last[0];
                    last[1] = bl1 ? pos1 : last[1];
                    if (CNT) n_blend += bl0 + bl1;
                }
            } else {
                for (int qq = 0; qq < nw; qq++) {
                    if (__all_sync(0xffffffffu, done[0])) break;
                    const int jj = wl[qq];
                    const uint32_t pos1 = base + (uint32_t)jj + 1u;
                    const float4 a = sb_A(sm.u.sb, jj);
                    const float2 h = sm.u.sb.H[jj];
                    const float dx = __fsub_rn(fpx, a.x), dy = __fsub_rn((float)ly, a.y);
                    const bool u = !done[0] && fabsf(dx) <= h.x && fabsf(dy) <= h.y;
                    if (CNT) n_eval += u;
                    if (!__any_sync(0xffffffffu, u)) continue;
                    const float4 b = sb_B(sm.u.sb, jj);
                    const float pw = pair_power2(a, b, __fmul_rn(a.z, __fmul_rn(dx, dx)), dx, dy);
                    const float ar = __fmul_rn(b.y, fast_exp2(pw));
                    const float alpha = ar > amax ? amax : ar;
                    const bool ok = u && !(pw > 0.0f) && alpha >= amin;
                    const float Tn = pT[0] * (1.0f - alpha);
                    const bool stop = ok && Tn < tmin;
                    const bool blend = ok && !stop;
                    done[0] = done[0] || stop;
                    const float w = blend ? alpha * pT[0] : 0.0f;
                    C0[0] = fmaf(b.z, w, C0[0]);
                    C1[0] = fmaf(b.w, w, C1[0]);
                    C2[0] = fmaf(sb_Cb(sm.u.sb, jj), w, C2[0]);
                    pT[0] = blend ? Tn : pT[0];
                    last[0] = blend ? pos1 : last[0];
                    if (CNT) n_blend += blend;
                }
            }
        }
        return __syncthreads_count(all_done()) == NT;
    };
    // Sorts list positions [c0, c0 + m) found in src (shared b0 or global) and
    // writes their indices to sorted_idx.
    auto sort_write = [&](unsigned long long* src, unsigned long long* scratch, uint32_t c0, int m) {
        unsigned long long* r = sort_tile_keys<NT>(src, scratch, m, sm.hist);
        for (int j = threadIdx.x; j < m; j += NT) sorted_idx[s + c0 + j] = (uint32_t)(r[j] & 0xffffffffull);
        __syncthreads();
    };
    // Sorts the run [c0, c0 + m) of buckets [cb, cb1) held in b0 grouped by
    // bucket (bucket b at [bstart[b] - c0, bstart[b + 1] - c0)): the buckets
    // are depth intervals in order, so sorting each bucket on its own sorts the
    // run; a thread insertion-sorts a bucket of at most LZ_SMALL keys.  A run
    // with a larger bucket is radix-sorted whole instead.  Either way b0 ends
    // in the exact (depth, index) order.
    auto sort_buckets_write = [&](int cb, int cb1, uint32_t c0, int m) {
        bool big = false;
        unsigned long long* k0 = sm.u.srt.b0;
        for (int b = cb + (int)threadIdx.x; b < cb1; b += NT) {
            const uint32_t bl = sm.bstart[b] - c0, bh = sm.bstart[b + 1] - c0;
            if (bh - bl > LZ_SMALL) {
                big = true;
                continue;
            }
            for (uint32_t i = bl + 1; i < bh; i++) {
                const unsigned long long x = k0[i];
                uint32_t j = i;
                while (j > bl && k0[j - 1] > x) {
                    k0[j] = k0[j - 1];
                    j--;
                }
                k0[j] = x;
            }
        }
        if (__syncthreads_or(big)) {
            sort_write(k0, sm.u.srt.b1, c0, m);
            return;
        }
        for (int j = threadIdx.x; j < m; j += NT) sorted_idx[s + c0 + j] = (uint32_t)(k0[j] & 0xffffffffull);
        __syncthreads();
    };

    if (n_list <= LZ_CAP) {
        for (uint32_t j = threadIdx.x; j < n_list; j += NT) sm.u.srt.b0[j] = keys[s + j];
        __syncthreads();
        if (n_list > 0) sort_write(sm.u.srt.b0, sm.u.srt.b1, 0, (int)n_list);
        n_sorted = n_list;
        blend_range(0, n_list);
    } else {
        // depth range of the tile
        uint32_t lo = 0xffffffffu, hi = 0u;
        for (uint32_t j = threadIdx.x; j < n_list; j += NT) {
            const uint32_t d = (uint32_t)(keys[s + j] >> 32);
            lo = min(lo, d);
            hi = max(hi, d);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (threadIdx.x == 0) { s_mm[0] = 0xffffffffu; s_mm[1] = 0u; }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) { atomicMin(&s_mm[0], lo); atomicMax(&s_mm[1], hi); }
        __syncthreads();
        lo = s_mm[0];
        hi = s_mm[1];
        if (lo == hi) {
            // one depth for the whole list: index order, sorted in global memory
            sort_write(keys + s, tmp + s, 0, (int)n_list);
            n_sorted = n_list;
            blend_range(0, n_list);
        } else {
            const int bits = 32 - __clz(hi - lo);
            const int shift = bits > LZ_NB_BITS ? bits - LZ_NB_BITS : 0;  // bucket index < LZ_NB
            for (int b = threadIdx.x; b <= LZ_NB; b += NT) sm.bstart[b] = 0u;
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < n_list; j += NT)
                atomicAdd(&sm.bstart[((uint32_t)(keys[s + j] >> 32) - lo) >> shift], 1u);
            __syncthreads();
            {
                uint32_t c[LZ_NB / NT], sum = 0;
#pragma unroll
                for (int k = 0; k < LZ_NB / NT; k++) { c[k] = sm.bstart[threadIdx.x * (LZ_NB / NT) + k]; sum += c[k]; }
                uint32_t off = block_scan_excl<NT>(sum, s_warp);
#pragma unroll
                for (int k = 0; k < LZ_NB / NT; k++) {
                    const int b = threadIdx.x * (LZ_NB / NT) + k;
                    sm.bstart[b] = off;
                    off += c[k];
                }
                if (threadIdx.x == 0) sm.bstart[LZ_NB] = n_list;
            }
            __syncthreads();
            // The first runs of buckets are gathered straight into shared memory
            // by a filtering pass over the tile's keys (most tiles stop within
            // them, and the rest of the list is never moved).  From the third run
            // on, or for a bucket larger than the shared buffer, every key is
            // scattered once into bucket order in global memory instead.
            bool scattered = false;
            int cb = 0, run = 0;
            while (cb < LZ_NB) {
                const uint32_t c0 = sm.bstart[cb];
                if (c0 >= n_list) break;
                int cb1 = cb + 1;
                while (cb1 < LZ_NB && sm.bstart[cb1 + 1] - c0 <= (run == 0 ? (uint32_t)LZ_FIRST : (uint32_t)LZ_CAP)) cb1++;
                const int m = (int)(sm.bstart[cb1] - c0);
                if (!scattered && (m > LZ_CAP || run >= 2)) {
                    for (int b = threadIdx.x; b < LZ_NB; b += NT) sm.hist[b] = sm.bstart[b];
                    __syncthreads();
                    for (uint32_t j = threadIdx.x; j < n_list; j += NT) {
                        const unsigned long long x = keys[s + j];
                        const uint32_t pos = atomicAdd(&sm.hist[((uint32_t)(x >> 32) - lo) >> shift], 1u);
                        tmp[s + pos] = x;
                    }
                    __syncthreads();
                    scattered = true;
                }
                if (m > LZ_CAP) {
                    sort_write(tmp + s + c0, keys + s + c0, c0, m);  // one oversized bucket
                } else if (scattered) {
                    // the scattered copy is grouped by bucket already
                    for (int j = threadIdx.x; j < m; j += NT) sm.u.srt.b0[j] = tmp[s + c0 + j];
                    __syncthreads();
                    sort_buckets_write(cb, cb1, c0, m);
                } else {
                    // gathered into b0 grouped by bucket (a cursor per bucket)
                    for (int b = cb + (int)threadIdx.x; b < cb1; b += NT) sm.hist[b] = sm.bstart[b] - c0;
                    __syncthreads();
                    for (uint32_t j = threadIdx.x; j < n_list; j += NT) {
                        const unsigned long long x = keys[s + j];
                        const int b = (int)(((uint32_t)(x >> 32) - lo) >> shift);
                        if (b >= cb && b < cb1) sm.u.srt.b0[atomicAdd(&sm.hist[b], 1u)] = x;
                    }
                    __syncthreads();
                    sort_buckets_write(cb, cb1, c0, m);
                }
                n_sorted = c0 + (uint32_t)m;
                run++;
                if (blend_range(c0, c0 + (uint32_t)m)) break;
                cb = cb1;
            }
        }
    }
    if (threadIdx.x == 0) sorted_count[t] = n_sorted;
    if constexpr (PX == 2) {
        pT[0] = f2_lo(pT2); pT[1] = f2_hi(pT2);
        C0[0] = f2_lo(Cr2); C0[1] = f2_hi(Cr2);
        C1[0] = f2_lo(Cg2); C1[1] = f2_hi(Cg2);
        C2[0] = f2_lo(Cb2); C2[1] = f2_hi(Cb2);
    }
    float l1 = 0.0f;
#pragma unroll
    for (int q = 0; q < PX; q++) {
        const int px = tx0 + lx, py = ty0 + ly + WARP_H * q;
        if (px < W && py < H) {
            const size_t p = (size_t)py * W + px;
            const size_t np = (size_t)W * H;
            float* img = image + vd.img_off;
            const float c0 = fmaf(pT[q], rp.bg[0], C0[q]);
            const float c1 = fmaf(pT[q], rp.bg[1], C1[q]);
            const float c2 = fmaf(pT[q], rp.bg[2], C2[q]);
            img[p] = c0;
            img[np + p] = c1;
            img[2 * np + p] = c2;
            T_final[vd.pix_off + p] = pT[q];
            n_contrib[vd.pix_off + p] = last[q];
            if (target) {
                const float* tg = target + vd.img_off;
                l1 += fabsf(c0 - tg[p]) + fabsf(c1 - tg[np + p]) + fabsf(c2 - tg[2 * np + p]);
            }
        }
    }
    if (target) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        if (lane == 0) s_red[wid] = l1;
        __syncthreads();
        if (threadIdx.x == 0) {
            float acc = 0.0f;
            for (int w = 0; w < NT / 32; w++) acc += s_red[w];
            tile_loss[t] = acc;
        }
    }
    if (CNT) {
        unsigned long long ce = n_eval, cbl = n_blend;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ce += __shfl_xor_sync(0xffffffffu, ce, o);
            cbl += __shfl_xor_sync(0xffffffffu, cbl, o);
        }
        if (lane == 0) {
            atomicAdd(counters, ce);
            atomicAdd(counters + 1, cbl);
            atomicAdd(counters + 8, (unsigned long long)n_went);   // warp-entries walked
        }
        if (threadIdx.x == 0) {
            atomicAdd(counters + 4, (unsigned long long)n_read);
            atomicAdd(counters + 5, (unsigned long long)n_sorted);
        }
    }
}

template <int CAP, int PX, bool CNT>
static void launch_lazy_cnt(int n_tiles, int n_views, const int* tile_base, const ViewDev* views,
                            const RenderParams& rp, SplatArrays sp, int n, const uint32_t* starts,
                            unsigned long long* keys, unsigned long long* tmp, uint32_t* sorted_idx,
                            uint32_t* sorted_count, uint32_t cap, float* image, float* T_final, uint32_t* n_contrib,
                            const float* target, float* tile_loss, unsigned long long* counters, cudaStream_t s) {
    constexpr int NT = GS_TILE_PIX / PX;
    static std::atomic<unsigned long long> attr{0};
    once_per_device(attr, [](int) {
        cudaFuncSetAttribute(k_blend_fwd_lazy<CAP, PX, CNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(LazySmem<CAP, NT>));
    });
    k_blend_fwd_lazy<CAP, PX, CNT><<<n_tiles, NT, sizeof(LazySmem<CAP, NT>), s>>>(
        n_views, tile_base, views, rp, sp, n, starts, keys, tmp, sorted_idx, sorted_count, cap, image, T_final,
        n_contrib, target, tile_loss, counters);
}

template <int CAP, int PX>
static void launch_lazy(int n_tiles, int n_views, const int* tile_base, const ViewDev* views, const RenderParams& rp,
                        SplatArrays sp, int n, const uint32_t* starts, unsigned long long* keys,
                        unsigned long long* tmp, uint32_t* sorted_idx, uint32_t* sorted_count, uint32_t cap,
                        float* image, float* T_final, uint32_t* n_contrib, const float* target, float* tile_loss,
                        unsigned long long* counters, cudaStream_t s) {
    if (counters)
        launch_lazy_cnt<CAP, PX, true>(n_tiles, n_views, tile_base, views, rp, sp, n, starts, keys, tmp, sorted_idx,
                                       sorted_count, cap, image, T_final, n_contrib, target, tile_loss, counters, s);
    else
        launch_lazy_cnt<CAP, PX, false>(n_tiles, n_views, tile_base, views, rp, sp, n, starts, keys, tmp, sorted_idx,
                                        sorted_count, cap, image, T_final, n_contrib, target, tile_loss, counters, s);
}

void launch_blend_fwd_lazy(int n_tiles, int sort_chunk, int px_per_thread, int n_views, const int* tile_base,
                           const ViewDev* views, const RenderParams& rp, SplatArrays sp, int n, const uint32_t* starts,
                           unsigned long long* keys, unsigned long long* tmp, uint32_t* sorted_idx,
                           uint32_t* sorted_count, uint32_t cap, float* image, float* T_final, uint32_t* n_contrib,
                           const float* target, float* tile_loss, unsigned long long* counters, cudaStream_t s) {
    if (n_tiles <= 0) return;
#define GS_LAZY_ARGS n_tiles, n_views, tile_base, views, rp, sp, n, starts, keys, tmp, sorted_idx, sorted_count, cap, \
                     image, T_final, n_contrib, target, tile_loss, counters, s
    if (sort_chunk <= 1024) {
        if (px_per_thread == 2) launch_lazy<1024, 2>(GS_LAZY_ARGS);
        else launch_lazy<1024, 1>(GS_LAZY_ARGS);
    } else {
        if (px_per_thread == 2) launch_lazy<2048, 2>(GS_LAZY_ARGS);
        else launch_lazy<2048, 1>(GS_LAZY_ARGS);
    }
#undef GS_LAZY_ARGS
}

void launch_blend_fwd(int n_tiles, int n_views, const int* tile_base, const ViewDev* views, const RenderParams& rp,
                      SplatArrays sp, int n, const uint32_t* starts, const uint32_t* sorted_idx, uint32_t cap,
                      float* image, float* T_final, uint32_t* n_contrib, const float* target, float* tile_loss,
                      unsigned long long* counters, cudaStream_t s) {
    if (n_tiles <= 0) return;
    k_blend_fwd<<<n_tiles, GS_TILE_PIX, 0, s>>>(n_views, tile_base, views, rp, sp, n, starts, sorted_idx, cap, image,
                                                 T_final, n_contrib, target, tile_loss, counters);
}

// Per-view loss w * mean_{3HW} |C - target| (+ addend[v]) from the per-tile
// partial sums, summed in tile order (deterministic).
__global__ void k_loss_finalize(int n_views, const ViewDev* __restrict__ views, const float* __restrict__ tile_loss,
                                double w, const double* __restrict__ addend, double* __restrict__ out) {
    __shared__ double sm[256];
    const int v = blockIdx.x;
    const ViewDev& vd = views[v];
    const int nt = vd.gw * vd.gh;
    double acc = 0.0;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) acc += (double)tile_loss[vd.tile_base + t];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = w * sm[0] / (3.0 * (double)vd.W * (double)vd.H) + (addend ? addend[v] : 0.0);
}

void launch_loss_finalize(int n_views, const ViewDev* views, const float* tile_loss, double w, const double* addend,
                          double* loss_out, cudaStream_t s) {
    if (n_views <= 0) return;
    k_loss_finalize<<<n_views, 256, 0, s>>>(n_views, views, tile_loss, w, addend, loss_out);
}

// ------------------------------------------------------------ backward
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Per-pixel state of the backward blend.
struct BwdPixel {
    float T, g0, g1, g2, sg;
    uint32_t last;
    bool inside;
};

// Per-pixel setup of the backward blend: T_final, n_contrib and dL/dC at
// pixel (px, py) of view vd (a given dL/dC, the L1 term of Eq. 16 or its
// confidence-masked form of Eq. 20-21), with the pixel's L1 sum added to l1.
__device__ __forceinline__ BwdPixel bwd_pixel(const ViewDev& vd, int px, int py, const RenderParams& rp,
                                              const float* __restrict__ image, const float* __restrict__ T_final,
                                              const uint32_t* __restrict__ n_contrib, int loss_kind, float w_l1,
                                              float l1_mask_t, const float* __restrict__ target,
                                              const float* __restrict__ dldc, float& l1) {
    BwdPixel P;
    const int W = vd.W, H = vd.H;
    P.inside = px < W && py < H;
    P.T = 1.0f; P.g0 = P.g1 = P.g2 = 0.0f; P.last = 0;
    if (P.inside) {
        const size_t p = (size_t)py * W + px;
        const size_t np = (size_t)W * H;
        P.T = T_final[vd.pix_off + p];
        P.last = n_contrib[vd.pix_off + p];
        const float* img = image + vd.img_off;
        if (loss_kind == GS_LOSS_DLDC || loss_kind == GS_LOSS_L1_DSSIM) {
            const float* d = dldc + vd.img_off;
            P.g0 = d[p]; P.g1 = d[np + p]; P.g2 = d[2 * np + p];
        }
        // L1 term (Eq. 16), or its confidence-masked form (Eq. 20-21): pixels
        // whose accumulated alpha 1 - T is not above the mask threshold
        // contribute nothing
        if ((loss_kind == GS_LOSS_L1 || loss_kind == GS_LOSS_L1_DSSIM || loss_kind == GS_LOSS_L1_MASKED) &&
            P.T < l1_mask_t) {
            const float* tg = target + vd.img_off;
            const float sc = w_l1 * vd.inv_npix3;
            const float d0 = img[p] - tg[p], d1 = img[np + p] - tg[np + p], d2 = img[2 * np + p] - tg[2 * np + p];
            P.g0 += d0 > 0.f ? sc : (d0 < 0.f ? -sc : 0.f);
            P.g1 += d1 > 0.f ? sc : (d1 < 0.f ? -sc : 0.f);
            P.g2 += d2 > 0.f ? sc : (d2 < 0.f ? -sc : 0.f);
            l1 += fabsf(d0) + fabsf(d1) + fabsf(d2);
        }
    }
    // dL/dC . (colour accumulated behind the current splat), starting with
    // the background: sg = sum_{behind} w_j (c_j . g) + T_final (bg . g)
    P.sg = P.T * (rp.bg[0] * P.g0 + rp.bg[1] * P.g1 + rp.bg[2] * P.g2);
    if (!(P.inside && ((P.g0 != 0.f) | (P.g1 != 0.f) | (P.g2 != 0.f)))) P.last = 0;  // takes no part
    return P;
}

// One pixel per thread in block-wide batches: 8 warps per tile, each an 8 x 4
// pixel block (the two-pixel form is k_blend_bwd_warp).
template <bool CNT>
__global__ void __launch_bounds__(GS_TILE_PIX, 6) k_blend_bwd(
    int n_views, const int* __restrict__ tile_base, const ViewDev* __restrict__ views, RenderParams rp, SplatArrays sp,
    int n, const uint32_t* __restrict__ starts, const uint32_t* __restrict__ sorted_idx, uint32_t cap,
    const float* __restrict__ image, const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
    int loss_kind, float w_l1, float l1_mask_t, const float* __restrict__ target, const float* __restrict__ dldc,
    Grad2DArrays g2d, float* __restrict__ tile_loss, unsigned long long* __restrict__ counters) {
    constexpr int PX = 1;
    constexpr int NT = GS_TILE_PIX;   // threads
    constexpr int NW = NT / 32;       // warps
    __shared__ SplatBatch sb;
    __shared__ uint32_t s_idx[BATCH];
    __shared__ uint32_t s_max[NW];
    __shared__ float s_acc[BATCH * 9];
    __shared__ unsigned char s_wl[NW][BATCH];
    const int t = blockIdx.x;
    const int v = view_of_tile(tile_base, n_views, t);
    const ViewDev& vd = views[v];
    const int gw = vd.gw;
    const int lt = t - vd.tile_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // warp footprint origin and this lane's first pixel (tile-relative)
    const int wx0 = (wid & 1) * WARP_W, wy0 = (wid >> 1) * (WARP_H * PX);
    const int lx = wx0 + (lane & (WARP_W - 1)), ly = wy0 + (lane >> 3);
    const int tx0 = (lt % gw) * GS_TILE, ty0 = (lt / gw) * GS_TILE;
    // tile-relative pixel coordinates (the staged means are moved to the same origin)
    const float ox = (float)tx0, oy = (float)ty0;
    const float fpx = (float)lx;
    uint32_t s = starts[t], e = starts[t + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    const size_t vbase = (size_t)v * n;
    BwdPixel pix[PX];
    float l1 = 0.0f;
#pragma unroll
    for (int q = 0; q < PX; q++)
        pix[q] = bwd_pixel(vd, tx0 + lx, ty0 + ly + WARP_H * q, rp, image, T_final, n_contrib, loss_kind, w_l1,
                           l1_mask_t, target, dldc, l1);
    if (tile_loss) {
        float r = l1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (lane == 0) s_max[wid] = __float_as_uint(r);
        __syncthreads();
        if (threadIdx.x == 0) {
            float acc = 0.0f;
            for (int w = 0; w < NW; w++) acc += __uint_as_float(s_max[w]);
            tile_loss[t] = acc;
        }
        __syncthreads();
    }
    // longest list prefix used by any pixel of the tile (n_contrib of the
    // pixels that take part)
    uint32_t mx = 0;
#pragma unroll
    for (int q = 0; q < PX; q++) mx = max(mx, pix[q].last);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_max[wid] = mx;
    __syncthreads();
    uint32_t tile_last = 0;
    for (int w = 0; w < NW; w++) tile_last = max(tile_last, s_max[w]);
    if (tile_last > e - s) tile_last = e - s;
    if (CNT && threadIdx.x == 0) atomicAdd(counters + 4, (unsigned long long)tile_last);
    uint32_t n_eval = 0, n_used = 0, n_w1 = 0, n_w2 = 0;
    // component held by this lane after the transposed reduction
    const int comp = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    // per-pixel state in registers, walked in lock step: a pixel that takes no
    // part in an entry gets alpha 0, so its state is unchanged and its share of
    // every sum is 0; the warp leaves an entry early only when no pixel of the
    // warp is in the splat's box, or none gets an alpha above alpha_min
    float pT[PX], psg[PX], pg0[PX], pg1[PX], pg2[PX], fpy[PX];
    uint32_t plast[PX];
#pragma unroll
    for (int q = 0; q < PX; q++) {
        pT[q] = pix[q].T; psg[q] = pix[q].sg; plast[q] = pix[q].last;
        pg0[q] = pix[q].g0; pg1[q] = pix[q].g1; pg2[q] = pix[q].g2;
        fpy[q] = (float)(ly + WARP_H * q);
    }
    const float amin = rp.alpha_min, amax = rp.alpha_max;
    for (int bend = (int)tile_last; bend > 0; bend -= BATCH) {
        const int bstart = max(0, bend - BATCH);
        const int cnt = bend - bstart;
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += NT) {
            const uint32_t id = sorted_idx[s + bstart + j];
            const size_t k = vbase + id;
            s_idx[j] = id;
            stage_entry(sb, j, stage_mean(sp, k, ox, oy), sp.B[k], sp.Cb[k], rp.alpha_min);
        }
        for (int q = threadIdx.x; q < BATCH * 9; q += NT) s_acc[q] = 0.0f;
        __syncthreads();
        unsigned char* wl = s_wl[wid];
        const int nw = warp_compact(sb, cnt, (float)wx0, (float)wy0, wl, WARP_H * PX);
        for (int qq = nw - 1; qq >= 0; qq--) {
            const int jj = wl[qq];
            const uint32_t pos = (uint32_t)(bstart + jj);
            // Per pixel, back to front: T_i = T_{i+1} / (1 - alpha_i), weight
            // w = alpha T_i, dL/dalpha = T_i (c . g) - S / (1 - alpha) with S the
            // colour behind (incl. background) dotted with g.  dL/dpower =
            // alpha dL/dalpha where alpha is not clamped.  Per entry the lane
            // sums dp = dL/dpower into the moments D = sum dp, My = sum dp dy,
            // Myy = sum dp dy^2 (its pixels share dx); the conic and mean
            // gradients are linear in the moments and formed once per splat.
            float r[9];
            {
                const float4 a = sb_A(sb, jj);
                const float2 h = sb.H[jj];
                const float dx = __fsub_rn(fpx, a.x), dy = __fsub_rn(fpy[0], a.y);
                bool u = fabsf(dx) <= h.x && fabsf(dy) <= h.y && pos < plast[0];
                if (CNT) n_eval += u;
                if (!__any_sync(0xffffffffu, u)) continue;
                if (CNT) n_w1++;
                const float4 b = sb_B(sb, jj);
                const float dxx = __fmul_rn(dx, dx), yy = __fmul_rn(dy, dy);
                const float pw = __fmaf_rn(a.w, __fmul_rn(dx, dy), __fmaf_rn(b.x, yy, __fmul_rn(a.z, dxx)));
                const float G = fast_exp2(pw);
                const float ar = __fmul_rn(b.y, G);
                const bool cl = ar > amax;
                const float al = cl ? amax : ar;
                u = u && !(pw > 0.0f) && al >= amin;
                if (!__any_sync(0xffffffffu, u)) continue;
                if (CNT) { n_w2++; n_used += u; }
                const float alq = u ? al : 0.0f;
                const float Gq = (u && !cl) ? G : 0.0f;
                const float inv = fast_rcp(1.0f - alq);    // 1 - alpha lies in [0.01, 1]
                const float Ti = pT[0] * inv;
                const float w = alq * Ti;
                const float cg = fmaf(sb_Cb(sb, jj), pg2[0], fmaf(b.w, pg1[0], b.z * pg0[0]));
                const float dL = fmaf(Ti, cg, -(psg[0] * inv));
                psg[0] = fmaf(w, cg, psg[0]);
                pT[0] = u ? Ti : pT[0];
                const float t = Gq * dL;                   // dL/do contribution
                const float dp = b.y * t;                  // dL/dpower
                r[0] = dx * dp;
                r[1] = dp * dy;
                r[2] = dxx * dp;
                r[3] = dx * r[1];
                r[4] = dp * yy;
                r[5] = t;
                r[6] = w * pg0[0];
                r[7] = w * pg1[0];
                r[8] = w * pg2[0];
            }
            // transposed reduce-scatter of r[0..7]: afterwards lane L (L % 4 == 0)
            // holds the warp sum of component comp(L)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const bool hi = lane & 16;
                const float send = hi ? r[k] : r[k + 4];
                const float keep = hi ? r[k + 4] : r[k];
                r[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const bool hi = lane & 8;
                const float send = hi ? r[k] : r[k + 2];
                const float keep = hi ? r[k + 2] : r[k];
                r[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
            {
                const bool hi = lane & 4;
                const float send = hi ? r[0] : r[1];
                const float keep = hi ? r[1] : r[0];
                r[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            r[0] += __shfl_xor_sync(0xffffffffu, r[0], 2);
            r[0] += __shfl_xor_sync(0xffffffffu, r[0], 1);
            const float r8 = warp_sum(r[8]);
            if ((lane & 3) == 0) atomicAdd(&s_acc[jj * 9 + comp], r[0]);
            if (lane == 1) atomicAdd(&s_acc[jj * 9 + 8], r8);
        }
        __syncthreads();
        // one set of vector atomics per (tile, splat) of the batch: the conic
        // and mean gradients from the moments (power = -1/2 (a dx^2 + c dy^2)
        // - b dx dy, d = p - mu: dpower/dmu = (a dx + b dy, b dx + c dy),
        // dpower/d(a, b, c) = (-dx^2 / 2, -dx dy, -dy^2 / 2))
        for (int j = threadIdx.x; j < cnt; j += NT) {
            const float* acc = s_acc + j * 9;
            const float ca = f2_lo(sb.P0[j].y) * GS_IKA, cb_ = f2_lo(sb.P1[j].y) * GS_IKB,
                        cc = f2_lo(sb.P2[j].x) * GS_IKA;
            const float Mx = acc[0], My = acc[1];
            const float4 ga = make_float4(fmaf(ca, Mx, cb_ * My), fmaf(cb_, Mx, cc * My), -0.5f * acc[2], -acc[3]);
            const float4 gb = make_float4(-0.5f * acc[4], acc[5], acc[6], acc[7]);
            const bool nz = (ga.x != 0.f) | (ga.y != 0.f) | (ga.z != 0.f) | (ga.w != 0.f) | (gb.x != 0.f) |
                            (gb.y != 0.f) | (gb.z != 0.f) | (gb.w != 0.f) | (acc[8] != 0.f);
            if (nz) {
                const size_t k = vbase + s_idx[j];
                atomicAdd(g2d.gA + k, ga);
                atomicAdd(g2d.gB + k, gb);
                atomicAdd(g2d.gC + k, acc[8]);
            }
        }
    }
    if (CNT) {
        unsigned long long ce = n_eval, cu = n_used;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ce += __shfl_xor_sync(0xffffffffu, ce, o);
            cu += __shfl_xor_sync(0xffffffffu, cu, o);
        }
        if (lane == 0) {
            atomicAdd(counters, ce);
            atomicAdd(counters + 1, cu);
            atomicAdd(counters + 7, (unsigned long long)n_w1);   // warp-entries with a pixel in the box
            atomicAdd(counters + 8, (unsigned long long)n_w2);   // warp-entries with a contributing pixel
        }
    }
}

// Backward blend in per-warp chunks (two pixels per thread, 4 warps per
// tile, each warp an 8 x 8 pixel block).  Every warp walks the tile's list
// back to front from the longest prefix its own pixels use, in chunks of 32
// entries that it stages itself: lane l stages entry l of the chunk and tests
// it against the warp's footprint from the values it staged, so no entry list
// and no block barrier is needed and the warps of a tile never wait for one
// another.  A warp's nine reduced sums of an entry go to its own accumulator
// slots; the lanes then flush the chunk's entries in parallel, one set of
// vector atomics per (warp, splat).
template <bool CNT>
__global__ void __launch_bounds__(GS_TILE_PIX / 2, 8) k_blend_bwd_warp(
    int n_views, const int* __restrict__ tile_base, const ViewDev* __restrict__ views, RenderParams rp, SplatArrays sp,
    int n, const uint32_t* __restrict__ starts, const uint32_t* __restrict__ sorted_idx, uint32_t cap,
    const float* __restrict__ image, const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
    int loss_kind, float w_l1, float l1_mask_t, const float* __restrict__ target, const float* __restrict__ dldc,
    Grad2DArrays g2d, float* __restrict__ tile_loss, unsigned long long* __restrict__ counters) {
    constexpr int NT = GS_TILE_PIX / 2;   // threads
    constexpr int NW = NT / 32;           // warps
    __shared__ WarpChunk s_wc[NW];
    __shared__ uint32_t s_red[NW];
    const int t = blockIdx.x;
    const int v = view_of_tile(tile_base, n_views, t);
    const ViewDev& vd = views[v];
    const int gw = vd.gw;
    const int lt = t - vd.tile_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // warp footprint origin and this lane's first pixel (tile-relative)
    const int wx0 = (wid & 1) * WARP_W, wy0 = (wid >> 1) * (WARP_H * 2);
    const int lx = wx0 + (lane & (WARP_W - 1)), ly = wy0 + (lane >> 3);
    const int tx0 = (lt % gw) * GS_TILE, ty0 = (lt / gw) * GS_TILE;
    // tile-relative pixel coordinates (the staged means are moved to the same origin)
    const float ox = (float)tx0, oy = (float)ty0;
    uint32_t s = starts[t], e = starts[t + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    const size_t vbase = (size_t)v * n;
    float l1 = 0.0f;
    const BwdPixel P0 = bwd_pixel(vd, tx0 + lx, ty0 + ly, rp, image, T_final, n_contrib, loss_kind, w_l1, l1_mask_t,
                                  target, dldc, l1);
    const BwdPixel P1 = bwd_pixel(vd, tx0 + lx, ty0 + ly + WARP_H, rp, image, T_final, n_contrib, loss_kind, w_l1,
                                  l1_mask_t, target, dldc, l1);
    if (tile_loss) {
        const float r = warp_sum(l1);
        if (lane == 0) s_red[wid] = __float_as_uint(r);
        __syncthreads();
        if (threadIdx.x == 0) {
            float acc = 0.0f;
            for (int w = 0; w < NW; w++) acc += __uint_as_float(s_red[w]);
            tile_loss[t] = acc;
        }
        __syncthreads();
    }
    // longest list prefix used by a pixel of this warp
    uint32_t wlast = max(P0.last, P1.last);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, o));
    if (wlast > e - s) wlast = e - s;
    if (CNT) {
        // list entries the tile reads: the longest of its warps' prefixes
        if (lane == 0) s_red[wid] = wlast;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t m = 0;
            for (int w = 0; w < NW; w++) m = max(m, s_red[w]);
            atomicAdd(counters + 4, (unsigned long long)m);
        }
    }
    uint32_t n_eval = 0, n_used = 0, n_w1 = 0, n_w2 = 0;
    // component held by this lane after the transposed reduction
    const int comp = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    const float amin = rp.alpha_min, amax = rp.alpha_max;
    const float fx0 = (float)wx0, fy0 = (float)wy0;
    // per-pixel state in pairs, walked in lock step: a pixel that takes no
    // part in an entry gets alpha 0, so its state is unchanged and its share of
    // every sum is 0
    const f2_t fpx2 = f2_pack((float)lx, (float)lx), fpy2 = f2_pack((float)ly, (float)(ly + WARP_H));
    const f2_t one2 = f2_pack(1.0f, 1.0f);
    const f2_t g0_2 = f2_pack(P0.g0, P1.g0), g1_2 = f2_pack(P0.g1, P1.g1), g2_2 = f2_pack(P0.g2, P1.g2);
    f2_t pT2 = f2_pack(P0.T, P1.T), S2 = f2_pack(P0.sg, P1.sg);
    const uint32_t plast0 = P0.last, plast1 = P1.last;
    WarpChunk& wc = s_wc[wid];
    for (int cend = (int)wlast; cend > 0; cend -= WCH) {
        const int cstart = max(0, cend - WCH);
        __syncwarp();   // the previous chunk's flush has read the slots
        // lane l stages entry cstart + l and tests it against the footprint
        bool hit = false;
        uint32_t id = 0;
        if (cstart + lane < cend) {
            id = sorted_idx[s + cstart + lane];
            const size_t k = vbase + id;
            float4 a = stage_mean(sp, k, ox, oy);
            float4 b = sp.B[k];
            float2 h;
            float qt;
            stage_prepare(a, b, amin, h, qt);
            stage_store(wc, lane, a, b, sp.Cb[k]);
            hit = footprint_hit(a, b.x, h, qt, fx0, fy0, WARP_H * 2);
        }
        unsigned mm = __ballot_sync(0xffffffffu, hit);
        __syncwarp();
        unsigned pm = 0;   // entries with a contributing pixel
        while (mm) {
            const int jj = 31 - __clz(mm);
            mm &= ~(1u << jj);
            const uint32_t pos = (uint32_t)(cstart + jj);
            // (the warp walks only positions below its longest prefix, so some
            // lane's pixel always takes part here)
            const bool u0 = pos < plast0, u1 = pos < plast1;
            // alpha of both pixels (Eq. 3) with pair_alpha's operation
            // sequence, paired: the lanes of each pair share dx
            const ulonglong2 p0 = wc.P0[jj], p1 = wc.P1[jj], p2 = wc.P2[jj];
            const f2_t dx2 = f2_sub(fpx2, p0.x), dy2 = f2_sub(fpy2, p1.x);
            const f2_t dxx2 = f2_mul(dx2, dx2), yy2 = f2_mul(dy2, dy2);
            const f2_t pw2 = f2_fma(p1.y, f2_mul(dx2, dy2), f2_fma(p2.x, yy2, f2_mul(p0.y, dxx2)));
            const float pw0 = f2_lo(pw2), pw1 = f2_hi(pw2);
            const float G0 = fast_exp2(pw0), G1 = fast_exp2(pw1);
            const f2_t ar2 = f2_mul(p2.y, f2_pack(G0, G1));
            const float ar0 = f2_lo(ar2), ar1 = f2_hi(ar2);
            // the decisions of pair_alpha (alpha >= alpha_min iff the unclamped ar
            // is, as alpha_max >= alpha_min; a NaN skips)
            const bool cl0 = ar0 > amax, cl1 = ar1 > amax;
            const float al0 = fminf(ar0, amax), al1 = fminf(ar1, amax);
            const bool v0 = u0 && !(pw0 > 0.0f) && ar0 >= amin;
            const bool v1 = u1 && !(pw1 > 0.0f) && ar1 >= amin;
            if (CNT) {
                // pixels inside the splat's alpha box (recomputed from the record)
                const float4 a = make_float4(f2_lo(p0.x), f2_lo(p1.x), f2_lo(p0.y) * GS_IKA, f2_lo(p1.y) * GS_IKB);
                const float4 b = make_float4(f2_lo(p2.x) * GS_IKA, f2_lo(p2.y), 0.0f, 0.0f);
                const float2 h = alpha_box(a, b, amin);
                const bool inx = fabsf(f2_lo(dx2)) <= h.x;
                const bool b0 = u0 && inx && fabsf(f2_lo(dy2)) <= h.y;
                const bool b1 = u1 && inx && fabsf(f2_hi(dy2)) <= h.y;
                n_eval += b0 + b1;
                n_w1 += __any_sync(0xffffffffu, b0 || b1) ? 1u : 0u;
            }
            if (!__any_sync(0xffffffffu, v0 || v1)) continue;
            if (CNT) { n_w2++; n_used += v0 + v1; }
            pm |= 1u << jj;
            const f2_t alq2 = f2_pack(v0 ? al0 : 0.0f, v1 ? al1 : 0.0f);
            const f2_t Gq2 = f2_pack((v0 && !cl0) ? G0 : 0.0f, (v1 && !cl1) ? G1 : 0.0f);
            const f2_t om2 = f2_sub(one2, alq2);   // 1 - alpha lies in [0.01, 1]
            const f2_t inv2 = f2_pack(fast_rcp(f2_lo(om2)), fast_rcp(f2_hi(om2)));
            const f2_t Ti2 = f2_mul(pT2, inv2);
            const f2_t w2 = f2_mul(alq2, Ti2);
            const ulonglong2 p3 = wc.P3[jj];
            const f2_t cg2 = f2_fma(wc.P4[jj], g2_2, f2_fma(p3.y, g1_2, f2_mul(p3.x, g0_2)));
            const f2_t dL2 = f2_sub(f2_mul(Ti2, cg2), f2_mul(S2, inv2));
            S2 = f2_fma(w2, cg2, S2);
            pT2 = f2_pack(v0 ? f2_lo(Ti2) : f2_lo(pT2), v1 ? f2_hi(Ti2) : f2_hi(pT2));
            const f2_t t2 = f2_mul(Gq2, dL2);      // dL/do contributions
            const f2_t dp2 = f2_mul(p2.y, t2);     // dL/dpower
            const f2_t My2 = f2_mul(dp2, dy2), Myy2 = f2_mul(dp2, yy2);
            const f2_t c0 = f2_mul(w2, g0_2), c1 = f2_mul(w2, g1_2), c2 = f2_mul(w2, g2_2);
            const float dx = f2_lo(dx2), D = f2_lo(dp2) + f2_hi(dp2), My = f2_lo(My2) + f2_hi(My2);
            float r[9];
            r[0] = dx * D;                          // sum dp dx
            r[1] = My;                              // sum dp dy
            r[2] = f2_lo(dxx2) * D;                 // sum dp dx^2
            r[3] = dx * My;                         // sum dp dx dy
            r[4] = f2_lo(Myy2) + f2_hi(Myy2);       // sum dp dy^2
            r[5] = f2_lo(t2) + f2_hi(t2);
            r[6] = f2_lo(c0) + f2_hi(c0);
            r[7] = f2_lo(c1) + f2_hi(c1);
            r[8] = f2_lo(c2) + f2_hi(c2);
            // transposed reduce-scatter of r[0..7]: afterwards lane L (L % 4 == 0)
            // holds the warp sum of component comp(L)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const bool hi = lane & 16;
                const float send = hi ? r[k] : r[k + 4];
                const float keep = hi ? r[k + 4] : r[k];
                r[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const bool hi = lane & 8;
                const float send = hi ? r[k] : r[k + 2];
                const float keep = hi ? r[k + 2] : r[k];
                r[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
            {
                const bool hi = lane & 4;
                const float send = hi ? r[0] : r[1];
                const float keep = hi ? r[1] : r[0];
                r[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            r[0] += __shfl_xor_sync(0xffffffffu, r[0], 2);
            r[0] += __shfl_xor_sync(0xffffffffu, r[0], 1);
            const float r8 = warp_sum(r[8]);
            if ((lane & 3) == 0) wc.acc[jj * 9 + comp] = r[0];
            if (lane == 1) wc.acc[jj * 9 + 8] = r8;
        }
        __syncwarp();
        // lane l flushes entry l: the conic and mean gradients from the moments
        // (power = -1/2 (a dx^2 + c dy^2) - b dx dy, d = p - mu:
        // dpower/dmu = (a dx + b dy, b dx + c dy), dpower/d(a, b, c) =
        // (-dx^2 / 2, -dx dy, -dy^2 / 2))
        if ((pm >> lane) & 1u) {
            const float* acc = wc.acc + lane * 9;
            const float ca = f2_lo(wc.P0[lane].y) * GS_IKA, cb_ = f2_lo(wc.P1[lane].y) * GS_IKB,
                        cc = f2_lo(wc.P2[lane].x) * GS_IKA;
            const float Mx = acc[0], My = acc[1];
            const float4 ga = make_float4(fmaf(ca, Mx, cb_ * My), fmaf(cb_, Mx, cc * My), -0.5f * acc[2], -acc[3]);
            const float4 gb = make_float4(-0.5f * acc[4], acc[5], acc[6], acc[7]);
            const size_t k = vbase + id;
            atomicAdd(g2d.gA + k, ga);
            atomicAdd(g2d.gB + k, gb);
            atomicAdd(g2d.gC + k, acc[8]);
        }
    }
    if (CNT) {
        unsigned long long ce = n_eval, cu = n_used;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ce += __shfl_xor_sync(0xffffffffu, ce, o);
            cu += __shfl_xor_sync(0xffffffffu, cu, o);
        }
        if (lane == 0) {
            atomicAdd(counters, ce);
            atomicAdd(counters + 1, cu);
            atomicAdd(counters + 7, (unsigned long long)n_w1);   // warp-entries with a pixel in the box
            atomicAdd(counters + 8, (unsigned long long)n_w2);   // warp-entries with a contributing pixel
        }
    }
}

void launch_blend_bwd(int n_tiles, int n_views, const int* tile_base, const ViewDev* views, const RenderParams& rp,
                      SplatArrays sp, int n, const uint32_t* starts, const uint32_t* sorted_idx, uint32_t cap,
                      const float* image, const float* T_final, const uint32_t* n_contrib, int loss_kind, float w_l1,
                      float l1_mask_t, const float* target, const float* dldc, Grad2DArrays g2d, float* tile_loss,
                      unsigned long long* counters, int px_per_thread, cudaStream_t s) {
    if (n_tiles <= 0) return;
#define GS_BWD_LAUNCH(KERNEL, NT)                                                                                   \
    KERNEL<<<n_tiles, NT, 0, s>>>(n_views, tile_base, views, rp, sp, n, starts, sorted_idx, cap, image, T_final,     \
                                  n_contrib, loss_kind, w_l1, l1_mask_t, target, dldc, g2d, tile_loss, counters)
    if (px_per_thread == 2) {
        if (counters) GS_BWD_LAUNCH(k_blend_bwd_warp<true>, GS_TILE_PIX / 2);
        else GS_BWD_LAUNCH(k_blend_bwd_warp<false>, GS_TILE_PIX / 2);
    } else {
        if (counters) GS_BWD_LAUNCH(k_blend_bwd<true>, GS_TILE_PIX);
        else GS_BWD_LAUNCH(k_blend_bwd<false>, GS_TILE_PIX);
    }
#undef GS_BWD_LAUNCH
}

}  // namespace gs
