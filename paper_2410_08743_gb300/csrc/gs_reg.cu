// gs_reg.cu - regularisers and opacity pruning of joint refinement (Sec. 3.3).
//
// Eq. 17: L_An = (1/N) sum_i [max(s_i) / min(s_i) - r]_+ on the activated
// scales, which keeps Gaussians from degenerating into thin spikes; the
// opacity L1 term L_o = (1/N) sum_i o_i (opacities are positive) that the
// paper adds during the first 10k steps; and the adaptive pruning threshold:
// the opacity below which Gaussians are removed so that at most N_tgt remain.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_internal.cuh"

namespace gs {

#define REG_T 256

// Per Gaussian: the hinge of the axis ratio and the opacity term, their
// gradients added into g_scales / g_opac, and a per-block FP64 partial sum of
// w_an * [ratio - r]_+ + w_op * o (the caller's 1/N is folded into the weights).
// The ratio's subgradient picks the first largest and the first smallest axis;
// all-equal axes (ratio 1) and a ratio exactly at r give no gradient.
__global__ void __launch_bounds__(REG_T) k_regularize(int n, const float* __restrict__ scales,
                                                      const float* __restrict__ opac, float r, float w_an,
                                                      float w_op, float* __restrict__ g_scales,
                                                      float* __restrict__ g_opac, double* __restrict__ partial) {
    __shared__ double red[REG_T / 32];
    const int i = blockIdx.x * REG_T + threadIdx.x;
    double term = 0.0;
    if (i < n) {
        const float s0 = scales[3 * i], s1 = scales[3 * i + 1], s2 = scales[3 * i + 2];
        if (w_an != 0.0f) {
            int imax = 0, imin = 0;
            float smax = s0, smin = s0;
            if (s1 > smax) { smax = s1; imax = 1; }
            if (s2 > smax) { smax = s2; imax = 2; }
            if (s1 < smin) { smin = s1; imin = 1; }
            if (s2 < smin) { smin = s2; imin = 2; }
            const float ratio = smax / smin;
            if (ratio > r && imax != imin) {
                term += (double)w_an * (double)(ratio - r);
                if (g_scales) {
                    g_scales[3 * i + imax] += w_an / smin;
                    g_scales[3 * i + imin] -= w_an * ratio / smin;
                }
            }
        }
        if (w_op != 0.0f) {
            term += (double)w_op * (double)opac[i];
            if (g_opac) g_opac[i] += w_op;
        }
    }
    if (partial) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
        __syncthreads();
        if (threadIdx.x == 0) {
            double acc = 0.0;
            for (int w = 0; w < REG_T / 32; w++) acc += red[w];
            partial[blockIdx.x] = acc;
        }
    }
}

// Sums the per-block partials in block order (deterministic) into *loss.
__global__ void k_sum_partials(int nb, const double* __restrict__ partial, double* __restrict__ loss) {
    __shared__ double red[REG_T];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += REG_T) acc += partial[b];
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < REG_T; k++) t += red[k];
        *loss = t;
    }
}

int regularize_blocks(int n) { return (n + REG_T - 1) / REG_T; }

void launch_regularize(int n, const float* scales, const float* opac, float r, float w_an, float w_op,
                       float* g_scales, float* g_opac, double* partial, double* loss, cudaStream_t s) {
    const int nb = regularize_blocks(n);
    if (n > 0) k_regularize<<<nb, REG_T, 0, s>>>(n, scales, opac, r, w_an, w_op, g_scales, g_opac, loss ? partial : nullptr);
    if (loss) k_sum_partials<<<1, REG_T, 0, s>>>(n > 0 ? nb : 0, partial, loss);
}

// ------------------------------------------------------------ radix select
// k-th smallest (0-based) of n positive floats: four passes over the 8-bit
// digits of the IEEE bit pattern (monotone for positive values), each a
// histogram of the values that share the digits found so far, then a pick.
// state[0] = bit prefix found so far, state[1] = remaining rank.
__global__ void __launch_bounds__(REG_T) k_select_hist(int n, const float* __restrict__ x,
                                                       const uint32_t* __restrict__ state, int shift,
                                                       uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t prefix = state[0];
    const uint32_t hi_mask = shift >= 24 ? 0u : (0xffffffffu << (shift + 8));
    for (int i = blockIdx.x * REG_T + threadIdx.x; i < n; i += gridDim.x * REG_T) {
        const uint32_t b = __float_as_uint(x[i]);
        if ((b & hi_mask) == (prefix & hi_mask)) atomicAdd(&h[(b >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_select_pick(uint32_t* __restrict__ state, int shift, uint32_t* __restrict__ hist) {
    if (threadIdx.x != 0) return;
    uint32_t k = state[1], acc = 0;
    int d = 0;
    for (; d < 256; d++) {
        if (acc + hist[d] > k) break;
        acc += hist[d];
    }
    if (d > 255) d = 255;  // unreachable for k < n
    state[0] |= (uint32_t)d << shift;
    state[1] = k - acc;
    for (int j = 0; j < 256; j++) hist[j] = 0;
}

__global__ void k_select_init(uint32_t* __restrict__ state, uint32_t k, uint32_t* __restrict__ hist) {
    if (threadIdx.x == 0) { state[0] = 0u; state[1] = k; }
    for (int j = threadIdx.x; j < 256; j += blockDim.x) hist[j] = 0u;
}

void launch_select_kth(int n, const float* x, uint32_t k, uint32_t* state, uint32_t* hist, cudaStream_t s) {
    k_select_init<<<1, 256, 0, s>>>(state, k, hist);
    const int nb = min(regularize_blocks(n), 4 * 152);
    for (int shift = 24; shift >= 0; shift -= 8) {
        k_select_hist<<<nb, REG_T, 0, s>>>(n, x, state, shift, hist);
        k_select_pick<<<1, 32, 0, s>>>(state, shift, hist);
    }
}

// ------------------------------------------------------------ compaction
// Stable compaction of the rows with opacity > thr: per-block counts, an
// exclusive scan of the counts (one block), then each block writes its kept
// rows in order.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* ws, uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = lane < REG_T / 32 ? ws[lane] : 0u;
        uint32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        if (lane < REG_T / 32) ws[lane] = xi - x;
        if (lane == REG_T / 32 - 1) *total = xi;
    }
    __syncthreads();
    const uint32_t r = ws[w] + inc - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(REG_T) k_keep_count(int n, const float* __restrict__ opac, float thr,
                                                      uint32_t* __restrict__ counts) {
    __shared__ uint32_t ws[REG_T / 32], tot;
    const int i = blockIdx.x * REG_T + threadIdx.x;
    const uint32_t keep = (i < n && opac[i] > thr) ? 1u : 0u;
    block_excl_scan(keep, ws, &tot);
    if (threadIdx.x == 0) counts[blockIdx.x] = tot;
}

// exclusive scan of nb block counts in place (one block, sequential chunks)
__global__ void __launch_bounds__(REG_T) k_scan_counts(int nb, uint32_t* __restrict__ counts,
                                                       uint32_t* __restrict__ total) {
    __shared__ uint32_t ws[REG_T / 32], tot;
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += REG_T) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? counts[i] : 0u;
        const uint32_t ex = block_excl_scan(v, ws, &tot);
        if (i < nb) counts[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(REG_T) k_compact_rows(int n, const float* __restrict__ opac, float thr,
                                                        const uint32_t* __restrict__ offsets, CompactArrays ca) {
    __shared__ uint32_t ws[REG_T / 32], tot;
    const int i = blockIdx.x * REG_T + threadIdx.x;
    const bool keep = i < n && opac[i] > thr;
    const uint32_t pos = offsets[blockIdx.x] + block_excl_scan(keep ? 1u : 0u, ws, &tot);
    if (!keep) return;
    for (int a = 0; a < ca.count; a++) {
        const int w = ca.width[a];
        const float* src = ca.src[a] + (size_t)i * w;
        float* dst = ca.dst[a] + (size_t)pos * w;
        for (int c = 0; c < w; c++) dst[c] = src[c];
    }
}

void launch_compact(int n, const float* opac, float thr, const CompactArrays& ca, uint32_t* counts,
                    uint32_t* total, cudaStream_t s) {
    const int nb = regularize_blocks(n);
    if (n <= 0) {
        k_scan_counts<<<1, REG_T, 0, s>>>(0, counts, total);
        return;
    }
    k_keep_count<<<nb, REG_T, 0, s>>>(n, opac, thr, counts);
    k_scan_counts<<<1, REG_T, 0, s>>>(nb, counts, total);
    k_compact_rows<<<nb, REG_T, 0, s>>>(n, opac, thr, counts, ca);
}

}  // namespace gs
