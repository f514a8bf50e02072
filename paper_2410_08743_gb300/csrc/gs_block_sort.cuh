// gs_block_sort.cuh - block-wide sort of one tile's (depth, index) keys in
// shared or global memory, shared by the standalone tile sort and the
// forward blend's lazy per-tile sort.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gs {

// Keys are (depth bits << 32 | Gaussian index), unique within a tile.  A tile
// is sorted by a stable LSD radix sort (8-bit digits) over the depth digits
// that vary within it; equal depths then sit in runs that are put in index
// order by a short insertion sort.  If some run is longer than RUN_MAX the
// whole list is re-sorted on every varying digit (index digits first).
#define RUN_MAX 32

// Block-wide exclusive scan of `v` (one value per thread); returns the
// thread's offset.  s_warp holds THREADS/32 words.
template <int THREADS>
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t v, uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < THREADS / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < THREADS / 32) s_warp[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t r = inc - v + s_warp[warp];
    __syncthreads();
    return r;
}

// Stable LSD radix passes (8-bit digits) over the digits set in `vary`.  Each
// warp owns a contiguous chunk; ranks inside a 32-key step come from
// match_any, so equal digits keep their order.  hist is [THREADS/32][256].
// Returns the buffer holding the result.
template <int THREADS>
__device__ unsigned long long* block_radix_sort_bits(unsigned long long* src, unsigned long long* dst, int n,
                                                     unsigned long long vary, uint32_t* hist) {
    constexpr int W = THREADS / 32;
    constexpr int E = 256 * W / THREADS;  // = 8 digit-major counters per thread
    __shared__ uint32_t s_warp[W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
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
        // B: exclusive scan in (digit, warp) order; thread t owns entries
        // [E t, E t + E) of that order.
        {
            uint32_t c[E], sum = 0;
#pragma unroll
            for (int k = 0; k < E; k++) {
                const int q = E * threadIdx.x + k;        // q = d * W + w
                c[k] = hist[(q % W) * 256 + q / W];
                sum += c[k];
            }
            uint32_t off = block_scan_excl<THREADS>(sum, s_warp);
#pragma unroll
            for (int k = 0; k < E; k++) {
                const int q = E * threadIdx.x + k;
                hist[(q % W) * 256 + q / W] = off;
                off += c[k];
            }
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

// OR and AND of n keys over the block -> bits that vary.
template <int THREADS>
__device__ unsigned long long block_vary_bits(const unsigned long long* src, int n) {
    constexpr int W = THREADS / 32;
    __shared__ unsigned long long s_or[W], s_and[W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long vo = 0ull, va = ~0ull;
    for (int j = threadIdx.x; j < n; j += THREADS) { const unsigned long long x = src[j]; vo |= x; va &= x; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) { vo |= __shfl_xor_sync(0xffffffffu, vo, o); va &= __shfl_xor_sync(0xffffffffu, va, o); }
    if (lane == 0) { s_or[warp] = vo; s_and[warp] = va; }
    __syncthreads();
    unsigned long long o2 = 0ull, a2 = ~0ull;
    for (int w = 0; w < W; w++) { o2 |= s_or[w]; a2 &= s_and[w]; }
    __syncthreads();
    return o2 ^ a2;
}

// Longest run of equal depth bits in a depth-sorted list (block-wide max).
template <int THREADS>
__device__ int block_max_depth_run(const unsigned long long* a, int n) {
    __shared__ int s_max;
    if (threadIdx.x == 0) s_max = 1;
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += THREADS) {
        const uint32_t dj = (uint32_t)(a[j] >> 32);
        if (j > 0 && (uint32_t)(a[j - 1] >> 32) == dj) continue;  // not a run start
        int m = 1;
        while (j + m < n && (uint32_t)(a[j + m] >> 32) == dj && m <= RUN_MAX) m++;
        if (m > 1) atomicMax(&s_max, m);
    }
    __syncthreads();
    const int r = s_max;
    __syncthreads();
    return r;
}

// Puts every run of equal depth in index order (runs of at most RUN_MAX).
template <int THREADS>
__device__ void block_fix_ties(unsigned long long* a, int n) {
    for (int j = threadIdx.x; j < n; j += THREADS) {
        const uint32_t dj = (uint32_t)(a[j] >> 32);
        if (j > 0 && (uint32_t)(a[j - 1] >> 32) == dj) continue;
        int m = 1;
        while (j + m < n && (uint32_t)(a[j + m] >> 32) == dj) m++;
        for (int p = j + 1; p < j + m; p++) {  // insertion sort of the run
            const unsigned long long x = a[p];
            int q = p - 1;
            while (q >= j && a[q] > x) { a[q + 1] = a[q]; q--; }
            a[q + 1] = x;
        }
    }
    __syncthreads();
}

// Sorts n unique keys held in b0 (b1 is scratch of the same size) into
// (depth, index) order; returns the buffer holding the result.
template <int THREADS>
__device__ unsigned long long* sort_tile_keys(unsigned long long* b0, unsigned long long* b1, int n, uint32_t* hist) {
    const unsigned long long vary = block_vary_bits<THREADS>(b0, n);
    unsigned long long* r = block_radix_sort_bits<THREADS>(b0, b1, n, vary & 0xffffffff00000000ull, hist);
    if (block_max_depth_run<THREADS>(r, n) > RUN_MAX) {
        unsigned long long* o = (r == b0) ? b1 : b0;
        r = block_radix_sort_bits<THREADS>(r, o, n, vary, hist);
    } else {
        block_fix_ties<THREADS>(r, n);
    }
    return r;
}

}  // namespace gs
