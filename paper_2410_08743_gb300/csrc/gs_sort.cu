// gs_sort.cu - depth-sorted per-tile lists (Sec. 3.1: "sorted by depth and
// composited front to back"; tile-based rasterisation).
//
// Layout: every (view, Gaussian) splat with tile rectangle R emits one key per
// tile of R.  Tiles of all views of a launch share one global numbering, so a
// single pass serves a whole batch of views.
//   1. count: a CTA takes a chunk of Gaussians of one view, counts their keys
//      per tile in shared memory and reserves its range in each touched tile
//      with one global atomic, recording (tile, offset) for step 3;
//   2. an exclusive scan of the counts gives each tile's [start, end);
//   3. scatter: each splat writes (depth bits << 32 | Gaussian index) into
//      its tiles' ranges at the CTA's reserved slots (arbitrary order within
//      a tile);
//   4. sort: normally lazily inside the forward blend (gs_blend.cu), which
//      sorts only the list prefixes it consumes; with GS_F_FULL_SORT the
//      segmented sorts below sort every tile's whole list.  Keys within a tile
//      are unique (one Gaussian appears once per tile), so either gives the
//      unique (depth, index) order: ties in depth go to the lower index,
//      independent of the scatter's order.
#include <cuda_runtime.h>

#include <algorithm>

#include "gs_block_sort.cuh"
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

// ------------------------------------------------------------ visible pairs
// Number of (view, Gaussian) pairs that passed the preprocess (non-empty tile
// rectangle), added to *count.  Only the counting passes run it.
__global__ void k_count_visible(size_t vn, const uint2* __restrict__ rect, unsigned long long* __restrict__ count) {
    unsigned long long c = 0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < vn; k += (size_t)gridDim.x * blockDim.x) {
        const uint2 r = rect[k];
        c += ((r.y & 0xffffu) > (r.x & 0xffffu)) ? 1ull : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

void launch_count_visible(size_t vn, const uint2* rect, unsigned long long* count, cudaStream_t s) {
    if (vn == 0) return;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t want = (vn + 255) / 256;
    const int grid = (int)std::min<size_t>(want, (size_t)std::max(1, sms) * 8);
    k_count_visible<<<grid, 256, 0, s>>>(vn, rect, count);
}

// ------------------------------------------------------------ count + scatter
// One CTA per (view, chunk of `chunk` Gaussians; a tuning knob).  The count
// CTA builds a shared-memory histogram of its keys over the view's tiles and
// reserves its range in every touched tile with one global atomic per (CTA,
// tile): tile_counts[t] += hist[t] returns the CTA's offset inside tile t,
// which it records as (t, offset) in its own list.  After the scan of the
// counts, the scatter CTA of the same chunk loads that list as its per-tile
// cursors (starts[t] + offset) and places each key with a shared-memory
// atomic: it neither rebuilds the histogram nor touches a global counter.
// Views with more than SMEM_TILES tiles use one global atomic per key in both
// passes instead (a per-tile cursor).
#define SMEM_TILES 8192
#define CS_THREADS 256

__device__ __forceinline__ void rect_of(const uint2 r, int& x0, int& y0, int& x1, int& y1) {
    x0 = r.x & 0xffff; y0 = r.x >> 16; x1 = r.y & 0xffff; y1 = r.y >> 16;
}

// Rectangles of four chunk entries per thread are loaded before any of them
// is used, so that the loads overlap.
#define CS_PREFETCH 4

// Warp-cooperative key scatter.  The 32 lanes of a warp hold consecutive
// Gaussians (Morton-ordered, so their rectangles cluster).  When the union of
// the warp's rectangles spans at most GS_BIN_BOX tiles, the warp walks that
// box: per tile, a ballot of the lanes whose rectangle covers it, and one
// slot atomic by the first of them for all (instead of one returning atomic
// per key, which the atomic unit serialises when lanes share a tile).  A wider
// union falls back to each lane walking its own rectangle, whose per-tile
// ballots would cost more than the atomics they save.  (The count pass keeps
// one atomic per key: without a return value they are cheap.)
#define GS_BIN_BOX 16

// Union box of the valid rectangles of the warp; returns false when none.
__device__ __forceinline__ bool warp_box(bool valid, int x0, int y0, int x1, int y1, int& bx0, int& by0, int& bx1,
                                         int& by1) {
    if (!__any_sync(0xffffffffu, valid)) return false;
    bx0 = (int)__reduce_min_sync(0xffffffffu, valid ? (unsigned)x0 : 0xffffffffu);
    by0 = (int)__reduce_min_sync(0xffffffffu, valid ? (unsigned)y0 : 0xffffffffu);
    bx1 = (int)__reduce_max_sync(0xffffffffu, valid ? (unsigned)x1 : 0u);
    by1 = (int)__reduce_max_sync(0xffffffffu, valid ? (unsigned)y1 : 0u);
    return true;
}

// Scatters the lane's key to every tile of its rectangle at the slots that
// hist (tile -> next global position) hands out; every lane of the warp
// calls it.  over is set when a position reaches cap.
__device__ __forceinline__ void warp_scatter(int x0, int y0, int x1, int y1, int gw, uint32_t* hist,
                                             unsigned long long key, unsigned long long* __restrict__ keys,
                                             uint32_t cap, bool& over) {
    const bool valid = x1 > x0 && y1 > y0;
    int bx0, by0, bx1, by1;
    if (!warp_box(valid, x0, y0, x1, y1, bx0, by0, bx1, by1)) return;
    if ((bx1 - bx0) * (by1 - by0) <= GS_BIN_BOX) {
        const int lane = threadIdx.x & 31;
        const unsigned lt = (1u << lane) - 1u;
        for (int ty = by0; ty < by1; ty++) {
            const bool iny = valid && y0 <= ty && ty < y1;
            for (int tx = bx0; tx < bx1; tx++) {
                const bool cov = iny && x0 <= tx && tx < x1;
                const unsigned m = __ballot_sync(0xffffffffu, cov);
                if (!m) continue;
                const int leader = __ffs(m) - 1;
                uint32_t base = 0u;
                if (lane == leader) base = atomicAdd(hist + ty * gw + tx, (uint32_t)__popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (cov) {
                    const uint32_t pos = base + (uint32_t)__popc(m & lt);
                    if (pos < cap) keys[pos] = key; else over = true;
                }
            }
        }
    } else {
        for (int ty = y0; ty < y1; ty++)
            for (int tx = x0; tx < x1; tx++) {
                const uint32_t pos = atomicAdd(hist + ty * gw + tx, 1u);
                if (pos < cap) keys[pos] = key; else over = true;
            }
    }
}

// Adds every key of this thread's entries of [i0, i1) to the shared histogram.
__device__ __forceinline__ void chunk_histogram(const uint2* __restrict__ rect, size_t vb, int i0, int i1, int gw,
                                                uint32_t* hist) {
    for (int i = i0 + threadIdx.x; i < i1; i += CS_THREADS * CS_PREFETCH) {
        uint2 r[CS_PREFETCH];
#pragma unroll
        for (int u = 0; u < CS_PREFETCH; u++) {
            const int iu = i + u * CS_THREADS;
            r[u] = iu < i1 ? rect[vb + iu] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < CS_PREFETCH; u++) {
            int x0, y0, x1, y1;
            rect_of(r[u], x0, y0, x1, y1);
            for (int ty = y0; ty < y1; ty++)
                for (int tx = x0; tx < x1; tx++) atomicAdd(hist + ty * gw + tx, 1u);
        }
    }
}

// First entry of the (tile, offset) list of the CTA of chunk c of view v: the
// lists of view v hold n_chunks * ntile(v) entries from n_chunks * tile_base(v).
__device__ __forceinline__ size_t cta_list_base(int n_chunks, int tile_base, int chunk_idx, int ntile) {
    return (size_t)n_chunks * (size_t)tile_base + (size_t)chunk_idx * (size_t)ntile;
}

__global__ void __launch_bounds__(CS_THREADS) k_count_tiles(int n, int chunk, const ViewDev* __restrict__ views,
                                                           const uint2* __restrict__ rect,
                                                           uint32_t* __restrict__ tile_counts,
                                                           uint2* __restrict__ cta_lists,
                                                           uint32_t* __restrict__ cta_list_len) {
    __shared__ uint32_t hist[SMEM_TILES];
    __shared__ uint32_t s_len;
    const int v = blockIdx.y;
    const int gw = views[v].gw, ntile = gw * views[v].gh, tb = views[v].tile_base;
    const int i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    const size_t vb = (size_t)v * n;
    if (ntile > SMEM_TILES) {
        for (int i = i0 + threadIdx.x; i < i1; i += CS_THREADS) {
            int x0, y0, x1, y1;
            rect_of(rect[vb + i], x0, y0, x1, y1);
            for (int ty = y0; ty < y1; ty++)
                for (int tx = x0; tx < x1; tx++) atomicAdd(tile_counts + tb + ty * gw + tx, 1u);
        }
        return;
    }
    for (int t = threadIdx.x; t < ntile; t += CS_THREADS) hist[t] = 0u;
    if (threadIdx.x == 0) s_len = 0u;
    __syncthreads();
    chunk_histogram(rect, vb, i0, i1, gw, hist);
    __syncthreads();
    // reserve the CTA's range in each touched tile; record (tile, offset)
    uint2* list = cta_lists + cta_list_base(gridDim.x, tb, blockIdx.x, ntile);
    const int lane = threadIdx.x & 31;
    for (int t0 = 0; t0 < ntile; t0 += CS_THREADS) {
        const int t = t0 + threadIdx.x;
        const uint32_t c = t < ntile ? hist[t] : 0u;
        const unsigned m = __ballot_sync(0xffffffffu, c != 0u);
        uint32_t w = 0u;
        if (lane == 0 && m) w = atomicAdd(&s_len, (uint32_t)__popc(m));
        w = __shfl_sync(0xffffffffu, w, 0);
        if (c) {
            const uint32_t off = atomicAdd(tile_counts + tb + t, c);
            list[w + __popc(m & ((1u << lane) - 1u))] = make_uint2((uint32_t)t, off);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) cta_list_len[(size_t)v * gridDim.x + blockIdx.x] = s_len;
}

__global__ void __launch_bounds__(CS_THREADS) k_scatter_tiles(int n, int chunk, const ViewDev* __restrict__ views,
                                                             const uint2* __restrict__ rect,
                                                             const float* __restrict__ depth,
                                                             const uint32_t* __restrict__ starts,
                                                             uint32_t* __restrict__ cursor,
                                                             const uint2* __restrict__ cta_lists,
                                                             const uint32_t* __restrict__ cta_list_len,
                                                             unsigned long long* __restrict__ keys, uint32_t cap,
                                                             int* __restrict__ status) {
    __shared__ uint32_t hist[SMEM_TILES];
    __shared__ int s_over;
    const int v = blockIdx.y;
    const int gw = views[v].gw, ntile = gw * views[v].gh, tb = views[v].tile_base;
    const int i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    const size_t vb = (size_t)v * n;
    if (threadIdx.x == 0) s_over = 0;
    if (ntile > SMEM_TILES) {
        __syncthreads();
        for (int i = i0 + threadIdx.x; i < i1; i += CS_THREADS) {
            int x0, y0, x1, y1;
            rect_of(rect[vb + i], x0, y0, x1, y1);
            if (x1 <= x0) continue;
            const unsigned long long key = ((unsigned long long)__float_as_uint(depth[vb + i]) << 32) | (uint32_t)i;
            for (int ty = y0; ty < y1; ty++)
                for (int tx = x0; tx < x1; tx++) {
                    const int t = tb + ty * gw + tx;
                    const uint32_t pos = starts[t] + atomicAdd(cursor + t, 1u);
                    if (pos < cap) keys[pos] = key; else s_over = 1;
                }
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_over) gs_set_status(status, GS_DEV_OVERFLOW);
        return;
    }
    // this CTA's cursor in every tile it touches (the tiles its keys go to)
    {
        const uint2* list = cta_lists + cta_list_base(gridDim.x, tb, blockIdx.x, ntile);
        const uint32_t len = cta_list_len[(size_t)v * gridDim.x + blockIdx.x];
        for (uint32_t k = threadIdx.x; k < len; k += CS_THREADS) {
            const uint2 e = list[k];
            hist[e.x] = starts[tb + e.x] + e.y;
        }
    }
    __syncthreads();
    bool over = false;
    const int lane = threadIdx.x & 31;
    // warp-uniform bases (lane i = base + lane), so that every lane takes part
    // in the warp's ballots; entries past the chunk get an empty rectangle
    for (int ib = i0 + (int)(threadIdx.x & ~31u); ib < i1; ib += CS_THREADS * CS_PREFETCH) {
        const int i = ib + lane;
        uint2 r[CS_PREFETCH];
        float dz[CS_PREFETCH];
#pragma unroll
        for (int u = 0; u < CS_PREFETCH; u++) {
            const int iu = i + u * CS_THREADS;
            r[u] = iu < i1 ? rect[vb + iu] : make_uint2(0u, 0u);
            dz[u] = iu < i1 ? depth[vb + iu] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < CS_PREFETCH; u++) {
            int x0, y0, x1, y1;
            rect_of(r[u], x0, y0, x1, y1);
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(dz[u]) << 32) | (uint32_t)(i + u * CS_THREADS);
            warp_scatter(x0, y0, x1, y1, gw, hist, key, keys, cap, over);
        }
    }
    if (over) s_over = 1;
    __syncthreads();
    if (threadIdx.x == 0 && s_over) gs_set_status(status, GS_DEV_OVERFLOW);
}

size_t cta_list_entries(int n, int chunk, int total_tiles) {
    return (size_t)((n + chunk - 1) / chunk) * (size_t)total_tiles;
}

void launch_count_tiles(int n, int chunk, int n_views, const ViewDev* views, const uint2* rect, uint32_t* tile_counts,
                        uint2* cta_lists, uint32_t* cta_list_len, cudaStream_t s) {
    if (n <= 0 || n_views <= 0) return;
    dim3 grid((n + chunk - 1) / chunk, n_views);
    k_count_tiles<<<grid, CS_THREADS, 0, s>>>(n, chunk, views, rect, tile_counts, cta_lists, cta_list_len);
}

void launch_scatter_keys(int n, int chunk, int n_views, const ViewDev* views, SplatArrays sp, const uint32_t* starts,
                         uint32_t* cursor, const uint2* cta_lists, const uint32_t* cta_list_len,
                         unsigned long long* keys, uint32_t cap, int* status, cudaStream_t s) {
    if (n <= 0 || n_views <= 0) return;
    dim3 grid((n + chunk - 1) / chunk, n_views);
    k_scatter_tiles<<<grid, CS_THREADS, 0, s>>>(n, chunk, views, sp.rect, sp.depth, starts, cursor, cta_lists,
                                                cta_list_len, keys, cap, status);
}

// ------------------------------------------------------------ segment sort
// The block-wide sort helpers live in gs_block_sort.cuh.

// Classifies tiles by list length into work lists: [0] <= SMALL_CAP keys,
// [1] <= MED_CAP, [2] longer.  Single-key tiles are written directly.
#define SMALL_T 256
#define SMALL_CAP 2048
#define MED_T 512
#define MED_CAP 5632
#define LARGE_T 512

__global__ void k_classify_tiles(int n_tiles, const uint32_t* __restrict__ starts, uint32_t cap,
                                 const unsigned long long* __restrict__ keys, uint32_t* __restrict__ sorted_idx,
                                 uint32_t* __restrict__ lists, uint32_t* __restrict__ counts) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    uint32_t s = starts[t], e = starts[t + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    const uint32_t n = e - s;
    if (n == 0) return;
    if (n == 1) { sorted_idx[s] = (uint32_t)(keys[s] & 0xffffffffull); return; }
    const int c = n <= SMALL_CAP ? 0 : (n <= MED_CAP ? 1 : 2);
    const uint32_t pos = atomicAdd(counts + c, 1u);
    lists[(size_t)c * n_tiles + pos] = (uint32_t)t;
}

// Persistent shared-memory sort over a work list (small or medium tiles).
template <int THREADS, int CAP>
__global__ void __launch_bounds__(THREADS) k_segsort_list(int n_tiles, const uint32_t* __restrict__ starts, uint32_t cap,
                                                          const unsigned long long* __restrict__ keys,
                                                          uint32_t* __restrict__ sorted_idx,
                                                          const uint32_t* __restrict__ list,
                                                          const uint32_t* __restrict__ list_count,
                                                          uint32_t* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* b0 = reinterpret_cast<unsigned long long*>(smem_raw);
    unsigned long long* b1 = b0 + CAP;
    uint32_t* hist = reinterpret_cast<uint32_t*>(b1 + CAP);
    __shared__ uint32_t s_item;
    const uint32_t total = *list_count;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= total) break;
        const uint32_t t = list[item];
        uint32_t s = starts[t], e = starts[t + 1];
        if (s > cap) s = cap;
        if (e > cap) e = cap;
        const int n = (int)(e - s);
        for (int j = threadIdx.x; j < n; j += THREADS) b0[j] = keys[s + j];
        __syncthreads();
        unsigned long long* r = sort_tile_keys<THREADS>(b0, b1, n, hist);
        for (int j = threadIdx.x; j < n; j += THREADS) sorted_idx[s + j] = (uint32_t)(r[j] & 0xffffffffull);
        __syncthreads();
    }
}

// Long lists: one MSD pass in global memory on the highest varying digit
// splits the list into 256 buckets (written to tmp), then runs of whole
// buckets of at most MED_CAP keys are sorted in shared memory.  A bucket
// longer than MED_CAP is sorted in global memory.
__global__ void __launch_bounds__(LARGE_T) k_segsort_large(int n_tiles, const uint32_t* __restrict__ starts,
                                                           uint32_t cap, unsigned long long* __restrict__ keys,
                                                           unsigned long long* __restrict__ tmp,
                                                           uint32_t* __restrict__ sorted_idx,
                                                           const uint32_t* __restrict__ list,
                                                           const uint32_t* __restrict__ list_count,
                                                           uint32_t* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* b0 = reinterpret_cast<unsigned long long*>(smem_raw);
    unsigned long long* b1 = b0 + MED_CAP;
    uint32_t* hist = reinterpret_cast<uint32_t*>(b1 + MED_CAP);
    __shared__ uint32_t s_item;
    __shared__ uint32_t s_bucket[257];
    __shared__ uint32_t s_start[257];
    const uint32_t total = *list_count;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= total) break;
        const uint32_t t = list[item];
        uint32_t s = starts[t], e = starts[t + 1];
        if (s > cap) s = cap;
        if (e > cap) e = cap;
        const int n = (int)(e - s);
        unsigned long long* src = keys + s;
        unsigned long long* dst = tmp + s;
        const unsigned long long vary = block_vary_bits<LARGE_T>(src, n);
        int top = 56;
        while (top > 0 && ((vary >> top) & 0xffull) == 0ull) top -= 8;
        for (int d = threadIdx.x; d < 257; d += LARGE_T) s_bucket[d] = 0u;
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += LARGE_T) atomicAdd(&s_bucket[(src[j] >> top) & 0xffull], 1u);
        __syncthreads();
        {
            const uint32_t c = threadIdx.x < 256 ? s_bucket[threadIdx.x] : 0u;
            __shared__ uint32_t s_w[LARGE_T / 32];
            const uint32_t off = block_scan_excl<LARGE_T>(c, s_w);
            if (threadIdx.x < 256) { s_bucket[threadIdx.x] = off; s_start[threadIdx.x] = off; }
            if (threadIdx.x == 0) s_start[256] = (uint32_t)n;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += LARGE_T) {
            const unsigned long long x = src[j];
            const uint32_t pos = atomicAdd(&s_bucket[(x >> top) & 0xffull], 1u);
            dst[pos] = x;
        }
        __syncthreads();
        int d0 = 0;
        while (d0 < 256) {
            const uint32_t c0 = s_start[d0];
            int d1 = d0 + 1;
            while (d1 < 256 && s_start[d1 + 1] - c0 <= (uint32_t)MED_CAP) d1++;
            const int m = (int)(s_start[d1] - c0);
            if (m > MED_CAP) {
                // one oversized bucket: sort in global memory (tmp <-> keys)
                unsigned long long* r = sort_tile_keys<LARGE_T>(dst + c0, src + c0, m, hist);
                for (int j = threadIdx.x; j < m; j += LARGE_T) sorted_idx[s + c0 + j] = (uint32_t)(r[j] & 0xffffffffull);
            } else if (m > 0) {
                for (int j = threadIdx.x; j < m; j += LARGE_T) b0[j] = dst[c0 + j];
                __syncthreads();
                unsigned long long* r = sort_tile_keys<LARGE_T>(b0, b1, m, hist);
                for (int j = threadIdx.x; j < m; j += LARGE_T) sorted_idx[s + c0 + j] = (uint32_t)(r[j] & 0xffffffffull);
            }
            __syncthreads();
            d0 = d1;
        }
        __syncthreads();
    }
}


void launch_segment_sort(int n_tiles, const uint32_t* starts, unsigned long long* keys, unsigned long long* tmp_keys,
                         uint32_t* sorted_idx, uint32_t cap, uint32_t* lists, uint32_t* counters, cudaStream_t s) {
    if (n_tiles <= 0) return;
    static std::atomic<unsigned long long> attr_done{0};
    static std::atomic<int> num_sms[64];   // SM count per device
    const size_t sm_small = 2 * sizeof(unsigned long long) * SMALL_CAP + sizeof(uint32_t) * (SMALL_T / 32) * 256;
    const size_t sm_med = 2 * sizeof(unsigned long long) * MED_CAP + sizeof(uint32_t) * (MED_T / 32) * 256;
    const size_t sm_large = 2 * sizeof(unsigned long long) * MED_CAP + sizeof(uint32_t) * (LARGE_T / 32) * 256;
    once_per_device(attr_done, [&](int dev) {
        cudaFuncSetAttribute(k_segsort_list<SMALL_T, SMALL_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm_small);
        cudaFuncSetAttribute(k_segsort_list<MED_T, MED_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_med);
        cudaFuncSetAttribute(k_segsort_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_large);
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        num_sms[dev & 63].store(sms);
    });
    int dev = 0;
    cudaGetDevice(&dev);
    // counters: [0..2] list lengths, [3..5] work cursors
    cudaMemsetAsync(counters, 0, 6 * sizeof(uint32_t), s);
    k_classify_tiles<<<(n_tiles + 255) / 256, 256, 0, s>>>(n_tiles, starts, cap, keys, sorted_idx, lists, counters);
    const int sms_seen = num_sms[dev & 63].load();
    const int sms = sms_seen > 0 ? sms_seen : 152;
    k_segsort_large<<<sms * 2, LARGE_T, sm_large, s>>>(n_tiles, starts, cap, keys, tmp_keys, sorted_idx,
                                                       lists + 2 * (size_t)n_tiles, counters + 2, counters + 5);
    k_segsort_list<MED_T, MED_CAP><<<sms * 2, MED_T, sm_med, s>>>(n_tiles, starts, cap, keys, sorted_idx,
                                                                  lists + (size_t)n_tiles, counters + 1, counters + 4);
    k_segsort_list<SMALL_T, SMALL_CAP><<<sms * 5, SMALL_T, sm_small, s>>>(n_tiles, starts, cap, keys, sorted_idx,
                                                                          lists, counters, counters + 3);
}

}  // namespace gs
