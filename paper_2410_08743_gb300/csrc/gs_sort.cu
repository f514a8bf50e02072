// gs_sort.cu - depth-sorted per-tile lists (Sec. 3.1: "sorted by depth and
// composited front to back"; tile-based rasterisation).
//
// Layout: every (view, Gaussian) splat with tile rectangle R emits one key per
// tile of R.  Tiles of all views of a launch share one global numbering, so a
// single pass serves a whole batch of views.
//   1. the preprocess counts keys per tile (atomics on tile_counts);
//   2. an exclusive scan of the counts gives each tile's [start, end);
//   3. scatter: each splat writes (depth bits << 32 | Gaussian index) into
//      its tiles' ranges (arbitrary order within a tile);
//   4. per-tile LSD radix sort of those 64-bit keys in shared memory.  Keys
//      within a tile are unique (one Gaussian appears once per tile), so the
//      result is the unique (depth, index) order: ties in depth go to the
//      lower index, independent of the scatter's order.
#include <cuda_runtime.h>

#include "gs_internal.cuh"

namespace gs {

// ------------------------------------------------------------ exclusive scan
#define SCAN_T 1024
#define SCAN_IPT 4
#define SCAN_ITEMS (SCAN_T * SCAN_IPT)

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_sums, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? warp_sums[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) warp_sums[lane] = wi - w;
        if (lane == nw - 1 && total) *total = wi;
    }
    __syncthreads();
    uint32_t r = inc - x + warp_sums[warp];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                        int n, uint32_t* __restrict__ block_sums) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t tot;
    const size_t base = (size_t)blockIdx.x * SCAN_ITEMS + (size_t)threadIdx.x * SCAN_IPT;
    uint32_t v[SCAN_IPT], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; k++) { v[k] = (base + k < (size_t)n) ? in[base + k] : 0u; s += v[k]; }
    uint32_t off = block_exclusive_scan(s, ws, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_IPT; k++) {
        if (base + k < (size_t)n) out[base + k] = off;
        off += v[k];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_sums(uint32_t* __restrict__ sums, int nb) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += SCAN_T) {
        const int i = base + threadIdx.x;
        uint32_t x = i < nb ? sums[i] : 0u;
        __shared__ uint32_t tot;
        uint32_t off = block_exclusive_scan(x, ws, &tot);
        if (i < nb) sums[i] = off + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int n, const uint32_t* __restrict__ sums) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (size_t)n) out[i] += sums[i / SCAN_ITEMS];
}

size_t scan_tmp_bytes(int n) { return sizeof(uint32_t) * (size_t)((n + SCAN_ITEMS - 1) / SCAN_ITEMS + 1); }

void launch_scan_u32(const uint32_t* in, uint32_t* out, int n, void* tmp, size_t, cudaStream_t s) {
    if (n <= 0) return;
    const int nb = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
    uint32_t* sums = static_cast<uint32_t*>(tmp);
    k_scan_blocks<<<nb, SCAN_T, 0, s>>>(in, out, n, sums);
    if (nb > 1) {
        k_scan_sums<<<1, SCAN_T, 0, s>>>(sums, nb);
        k_scan_add<<<(n + 255) / 256, 256, 0, s>>>(out, n, sums);
    }
}

// ------------------------------------------------------------ scatter
__global__ void __launch_bounds__(256) k_scatter_keys(int n, int n_views, const ViewDev* __restrict__ views,
                                                      const uint2* __restrict__ rect, const float* __restrict__ depth,
                                                      const uint32_t* __restrict__ starts, uint32_t* __restrict__ cursor,
                                                      unsigned long long* __restrict__ keys, uint32_t cap,
                                                      int* __restrict__ status) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * n_views) return;
    const uint2 r = rect[k];
    const int x0 = r.x & 0xffff, y0 = r.x >> 16, x1 = r.y & 0xffff, y1 = r.y >> 16;
    if (x1 <= x0) return;
    const int v = (int)(k / (size_t)n);
    const uint32_t i = (uint32_t)(k - (size_t)v * n);
    const int gw = views[v].gw, tb = views[v].tile_base;
    const unsigned long long key = ((unsigned long long)__float_as_uint(depth[k]) << 32) | i;
    for (int ty = y0; ty < y1; ty++)
        for (int tx = x0; tx < x1; tx++) {
            const int t = tb + ty * gw + tx;
            const uint32_t pos = starts[t] + atomicAdd(cursor + t, 1u);
            if (pos < cap) keys[pos] = key;
            else gs_set_status(status, GS_DEV_OVERFLOW);
        }
}

void launch_scatter_keys(int n, int n_views, const ViewDev* views, SplatArrays sp, const uint32_t* starts,
                         uint32_t* cursor, unsigned long long* keys, uint32_t cap, int* status, cudaStream_t s) {
    const size_t total = (size_t)n * n_views;
    if (total == 0) return;
    k_scatter_keys<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n, n_views, views, sp.rect, sp.depth, starts, cursor,
                                                                   keys, cap, status);
}

// ------------------------------------------------------------ segment sort
// Stable LSD radix sort (8-bit digits) of one tile's 64-bit keys held in
// `src`/`dst` (shared or global memory).  Digits on which every key agrees
// are skipped.  Each warp owns a contiguous chunk; ranks inside a 32-key step
// come from match_any, so equal digits keep their order and the sort is
// stable.  Returns the buffer holding the result.
template <int THREADS>
__device__ unsigned long long* block_radix_sort(unsigned long long* src, unsigned long long* dst, int n,
                                                uint32_t* hist /* [THREADS/32][256] */) {
    constexpr int W = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    // bits that vary across the segment
    __shared__ unsigned long long s_or[W], s_and[W];
    unsigned long long vo = 0ull, va = ~0ull;
    for (int j = threadIdx.x; j < n; j += THREADS) { unsigned long long x = src[j]; vo |= x; va &= x; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) { vo |= __shfl_xor_sync(0xffffffffu, vo, o); va &= __shfl_xor_sync(0xffffffffu, va, o); }
    if (lane == 0) { s_or[warp] = vo; s_and[warp] = va; }
    __syncthreads();
    unsigned long long vary = 0ull;
    {
        unsigned long long o2 = 0ull, a2 = ~0ull;
        for (int w = 0; w < W; w++) { o2 |= s_or[w]; a2 &= s_and[w]; }
        vary = o2 ^ a2;
    }
    const int chunk = ((n + W - 1) / W + 31) & ~31;
    const int cb = warp * chunk;
    const int ce = min(n, cb + chunk);
    for (int shift = 0; shift < 64; shift += 8) {
        if (((vary >> shift) & 0xffull) == 0ull) continue;
        for (int d = threadIdx.x; d < W * 256; d += THREADS) hist[d] = 0u;
        __syncthreads();
        // A: per-warp digit histograms
        for (int b = cb; b < ce; b += 32) {
            const int j = b + lane;
            const bool ok = j < ce;
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const unsigned d = (unsigned)(src[j] >> shift) & 0xffu;
                const unsigned peers = __match_any_sync(act, d);
                if ((peers & lt_mask) == 0u) hist[warp * 256 + d] += __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        // B: offsets in (digit, warp) order.  Threads 0..255 own one digit
        // each: warp prefix within the digit, then a scan of digit totals.
        if (threadIdx.x < 256) {
            __shared__ uint32_t s_ws[8];
            const int d = threadIdx.x;
            uint32_t run = 0;
            for (int w = 0; w < W; w++) { const uint32_t c = hist[w * 256 + d]; hist[w * 256 + d] = run; run += c; }
            uint32_t inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_ws[warp] = inc;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            uint32_t wpre = 0;
            for (int w = 0; w < warp; w++) wpre += s_ws[w];
            const uint32_t dbase = inc - run + wpre;
            for (int w = 0; w < W; w++) hist[w * 256 + d] += dbase;
        }
        __syncthreads();
        // C: stable scatter
        for (int b = cb; b < ce; b += 32) {
            const int j = b + lane;
            const bool ok = j < ce;
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const unsigned long long x = src[j];
                const unsigned d = (unsigned)(x >> shift) & 0xffu;
                const unsigned peers = __match_any_sync(act, d);
                const uint32_t pos = hist[warp * 256 + d] + __popc(peers & lt_mask);
                dst[pos] = x;
                __syncwarp(act);
                if ((peers & lt_mask) == 0u) hist[warp * 256 + d] += __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        unsigned long long* t = src; src = dst; dst = t;
    }
    return src;
}

// Shared-memory variant for segments of at most CAP keys; segments outside
// (lo, hi] are left to another launch.
template <int THREADS, int CAP>
__global__ void __launch_bounds__(THREADS) k_segsort_smem(int n_tiles, const uint32_t* __restrict__ starts,
                                                          const unsigned long long* __restrict__ keys,
                                                          uint32_t* __restrict__ sorted_idx, uint32_t cap, int lo,
                                                          int hi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* b0 = reinterpret_cast<unsigned long long*>(smem_raw);
    unsigned long long* b1 = b0 + CAP;
    uint32_t* hist = reinterpret_cast<uint32_t*>(b1 + CAP);
    const int t = blockIdx.x;
    if (t >= n_tiles) return;
    uint32_t s = starts[t], e = starts[t + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    const int n = (int)(e - s);
    if (n <= lo || n > hi) return;
    for (int j = threadIdx.x; j < n; j += THREADS) b0[j] = keys[s + j];
    __syncthreads();
    unsigned long long* r = block_radix_sort<THREADS>(b0, b1, n, hist);
    for (int j = threadIdx.x; j < n; j += THREADS) sorted_idx[s + j] = (uint32_t)(r[j] & 0xffffffffull);
}

// Global-memory variant for long segments (one block per segment).
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_segsort_global(int n_tiles, const uint32_t* __restrict__ starts,
                                                            unsigned long long* __restrict__ keys,
                                                            unsigned long long* __restrict__ tmp,
                                                            uint32_t* __restrict__ sorted_idx, uint32_t cap, int lo) {
    __shared__ uint32_t hist[(THREADS / 32) * 256];
    const int t = blockIdx.x;
    if (t >= n_tiles) return;
    uint32_t s = starts[t], e = starts[t + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    const int n = (int)(e - s);
    if (n <= lo) return;
    unsigned long long* r = block_radix_sort<THREADS>(keys + s, tmp + s, n, hist);
    for (int j = threadIdx.x; j < n; j += THREADS) sorted_idx[s + j] = (uint32_t)(r[j] & 0xffffffffull);
}

#define SEG_SMALL_T 256
#define SEG_SMALL_CAP 2048
#define SEG_MED_T 512
#define SEG_MED_CAP 12288

void launch_segment_sort(int n_tiles, const uint32_t* starts, unsigned long long* keys, unsigned long long* tmp_keys,
                         uint32_t* sorted_idx, uint32_t cap, int, cudaStream_t s) {
    if (n_tiles <= 0) return;
    static bool attr_done = false;
    const size_t sm_small = 2 * sizeof(unsigned long long) * SEG_SMALL_CAP + sizeof(uint32_t) * (SEG_SMALL_T / 32) * 256;
    const size_t sm_med = 2 * sizeof(unsigned long long) * SEG_MED_CAP + sizeof(uint32_t) * (SEG_MED_T / 32) * 256;
    if (!attr_done) {
        cudaFuncSetAttribute(k_segsort_smem<SEG_SMALL_T, SEG_SMALL_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm_small);
        cudaFuncSetAttribute(k_segsort_smem<SEG_MED_T, SEG_MED_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm_med);
        attr_done = true;
    }
    k_segsort_smem<SEG_SMALL_T, SEG_SMALL_CAP><<<n_tiles, SEG_SMALL_T, sm_small, s>>>(n_tiles, starts, keys, sorted_idx,
                                                                                      cap, 0, SEG_SMALL_CAP);
    k_segsort_smem<SEG_MED_T, SEG_MED_CAP><<<n_tiles, SEG_MED_T, sm_med, s>>>(n_tiles, starts, keys, sorted_idx, cap,
                                                                              SEG_SMALL_CAP, SEG_MED_CAP);
    k_segsort_global<1024><<<n_tiles, 1024, 0, s>>>(n_tiles, starts, keys, tmp_keys, sorted_idx, cap, SEG_MED_CAP);
}

}  // namespace gs
