// gs_init.cu - preparing Gaussians.
//  * From one frame and a depth map, the first stage of relative pose
//    estimation (Sec. 3.4): a subset of the pixels is unprojected with the
//    intrinsics into a point cloud, every point becomes an isotropic Gaussian
//    with the pixel's colour, and its scale is the mean 3D distance to its
//    three nearest neighbours.
//  * A spatial (Morton) order of a scene's Gaussians and the row gather that
//    applies it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gs_internal.cuh"

namespace gs {

#define INIT_T 256

// Pixel (u, v) = (gx * stride, gy * stride) with z-depth d becomes the camera
// point ((u - cx) / fx * d, (v - cy) / fy * d, d) (the pixel samples the point
// (u, v), as in the renderer).  Dense output over the stride grid; key[g] is
// the depth (<= 0 or NaN marks an invalid pixel, dropped by the compaction).
__global__ void k_unproject(int W, int H, int stride, int gw, int gh, float fx, float fy, float cx, float cy,
                            const float* __restrict__ depth, const float* __restrict__ image,
                            float* __restrict__ pts, float* __restrict__ cols, float* __restrict__ key) {
    const int g = blockIdx.x * INIT_T + threadIdx.x;
    if (g >= gw * gh) return;
    const int u = (g % gw) * stride, v = (g / gw) * stride;
    const size_t p = (size_t)v * W + u;
    const float d = depth[p];
    key[g] = d;
    pts[3 * g + 0] = (((float)u - cx) / fx) * d;
    pts[3 * g + 1] = (((float)v - cy) / fy) * d;
    pts[3 * g + 2] = d;
    const size_t np = (size_t)W * H;
    cols[3 * g + 0] = image ? image[p] : 0.0f;
    cols[3 * g + 1] = image ? image[np + p] : 0.0f;
    cols[3 * g + 2] = image ? image[2 * np + p] : 0.0f;
}

void launch_unproject(int W, int H, int stride, float fx, float fy, float cx, float cy, const float* depth,
                      const float* image, float* pts, float* cols, float* key, cudaStream_t s) {
    const int gw = (W + stride - 1) / stride, gh = (H + stride - 1) / stride;
    const int n = gw * gh;
    if (n <= 0) return;
    k_unproject<<<(n + INIT_T - 1) / INIT_T, INIT_T, 0, s>>>(W, H, stride, gw, gh, fx, fy, cx, cy, depth, image, pts,
                                                              cols, key);
}

// Mean Euclidean distance of every point to its K nearest other points, by
// brute force: the block stages tiles of points in shared memory and every
// thread keeps the K smallest squared distances of its own point (a point's
// own index is skipped; coincident points count at distance 0).
#define KNN_TILE 1024
template <int K>
__global__ void __launch_bounds__(INIT_T) k_knn_mean(int n, const float* __restrict__ pts, float* __restrict__ out) {
    __shared__ float4 tile[KNN_TILE];
    const int i = blockIdx.x * INIT_T + threadIdx.x;
    float qx = 0.f, qy = 0.f, qz = 0.f;
    if (i < n) { qx = pts[3 * i]; qy = pts[3 * i + 1]; qz = pts[3 * i + 2]; }
    float best[K];
#pragma unroll
    for (int k = 0; k < K; k++) best[k] = INFINITY;
    for (int base = 0; base < n; base += KNN_TILE) {
        __syncthreads();
        for (int j = threadIdx.x; j < KNN_TILE; j += INIT_T) {
            const int q = base + j;
            tile[j] = q < n ? make_float4(pts[3 * q], pts[3 * q + 1], pts[3 * q + 2], 0.f)
                            : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        }
        __syncthreads();
        if (i >= n) continue;
        const int cnt = min(KNN_TILE, n - base);
        for (int j = 0; j < cnt; j++) {
            const float4 t = tile[j];
            const float dx = t.x - qx, dy = t.y - qy, dz = t.z - qz;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (d2 < best[K - 1] && base + j != i) {
                // insert into the sorted list
                float v = d2;
#pragma unroll
                for (int k = 0; k < K; k++) {
                    const float lo = fminf(best[k], v), hi = fmaxf(best[k], v);
                    best[k] = lo;
                    v = hi;
                }
            }
        }
    }
    if (i < n) {
        float acc = 0.f;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < K; k++)
            if (best[k] < INFINITY) { acc += sqrtf(best[k]); cnt++; }
        out[i] = cnt ? acc / (float)cnt : 0.f;
    }
}

void launch_knn_mean(int n, const float* pts, int k, float* out, cudaStream_t s) {
    if (n <= 0) return;
    const int nb = (n + INIT_T - 1) / INIT_T;
    switch (k) {
        case 1: k_knn_mean<1><<<nb, INIT_T, 0, s>>>(n, pts, out); break;
        case 2: k_knn_mean<2><<<nb, INIT_T, 0, s>>>(n, pts, out); break;
        case 3: k_knn_mean<3><<<nb, INIT_T, 0, s>>>(n, pts, out); break;
        case 4: k_knn_mean<4><<<nb, INIT_T, 0, s>>>(n, pts, out); break;
        case 5: k_knn_mean<5><<<nb, INIT_T, 0, s>>>(n, pts, out); break;
        case 6: k_knn_mean<6><<<nb, INIT_T, 0, s>>>(n, pts, out); break;
        case 7: k_knn_mean<7><<<nb, INIT_T, 0, s>>>(n, pts, out); break;
        default: k_knn_mean<8><<<nb, INIT_T, 0, s>>>(n, pts, out); break;
    }
}

// Raw parameters of isotropic Gaussians at the points: log-scale = log of the
// neighbour distance (floored at min_scale), identity quaternion, logit of
// the initial opacity, SH DC from the colour (c = f0 * C0 + 0.5, so
// f0 = (c - 0.5) / C0), higher SH coefficients zero.
__global__ void k_init_raw(int n, const float* __restrict__ pts, const float* __restrict__ cols,
                           const float* __restrict__ dist, float min_scale, float logit_o, float* __restrict__ means,
                           float* __restrict__ log_scales, float* __restrict__ quats, float* __restrict__ logit_opac,
                           float* __restrict__ sh) {
    const int i = blockIdx.x * INIT_T + threadIdx.x;
    if (i >= n) return;
    const float ls = logf(fmaxf(dist[i], min_scale));
    for (int a = 0; a < 3; a++) {
        means[3 * i + a] = pts[3 * i + a];
        log_scales[3 * i + a] = ls;
    }
    quats[4 * i] = 1.0f; quats[4 * i + 1] = 0.0f; quats[4 * i + 2] = 0.0f; quats[4 * i + 3] = 0.0f;
    logit_opac[i] = logit_o;
    const float inv_c0 = 3.5449077018110318f;   // 1 / C0 = 2 sqrt(pi)
    float* f = sh + (size_t)48 * i;
    for (int k = 0; k < 48; k++) f[k] = 0.0f;
    for (int a = 0; a < 3; a++) f[a] = (cols[3 * i + a] - 0.5f) * inv_c0;
}

void launch_init_raw(int n, const float* pts, const float* cols, const float* dist, float min_scale, float logit_o,
                     float* means, float* log_scales, float* quats, float* logit_opac, float* sh, cudaStream_t s) {
    if (n <= 0) return;
    k_init_raw<<<(n + INIT_T - 1) / INIT_T, INIT_T, 0, s>>>(n, pts, cols, dist, min_scale, logit_o, means,
                                                             log_scales, quats, logit_opac, sh);
}

// ------------------------------------------------------------ spatial order
// Morton (Z-order) code of every Gaussian mean on a 1024^3 grid over the
// means' bounding box; sorting by it places Gaussians that are close in space
// close in memory, so the per-(view, Gaussian) passes of the renderer touch
// few tiles per block of Gaussians and read their records coherently.
__global__ void __launch_bounds__(INIT_T) k_bbox_partial(int n, const float* __restrict__ means,
                                                         float* __restrict__ part) {
    __shared__ float red[6][INIT_T / 32];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * INIT_T + threadIdx.x; i < n; i += gridDim.x * INIT_T)
        for (int a = 0; a < 3; a++) {
            const float x = means[3 * i + a];
            mn[a] = fminf(mn[a], x);
            mx[a] = fmaxf(mx[a], x);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        for (int a = 0; a < 3; a++) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; a++) { red[a][threadIdx.x >> 5] = mn[a]; red[3 + a][threadIdx.x >> 5] = mx[a]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = red[threadIdx.x][0];
        for (int w = 1; w < INIT_T / 32; w++)
            v = threadIdx.x < 3 ? fminf(v, red[threadIdx.x][w]) : fmaxf(v, red[threadIdx.x][w]);
        part[6 * blockIdx.x + threadIdx.x] = v;
    }
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    // bits b0..b9 of v to positions 0, 3, 6, ..., 27
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// key = morton << 32 | index; the box comes from nb partial boxes.  The grid
// coordinate is floor((x - lo) * (1024 / (hi - lo))) in FP32 with every
// operation rounded (no contraction), clamped to [0, 1023].
__global__ void k_morton_keys(int n, int nb, const float* __restrict__ means, const float* __restrict__ part,
                              unsigned long long* __restrict__ keys) {
    __shared__ float lo[3], sc[3];
    if (threadIdx.x < 3) {
        float a = INFINITY, b = -INFINITY;
        for (int k = 0; k < nb; k++) {
            a = fminf(a, part[6 * k + threadIdx.x]);
            b = fmaxf(b, part[6 * k + 3 + threadIdx.x]);
        }
        const float ext = __fsub_rn(b, a);
        lo[threadIdx.x] = a;
        sc[threadIdx.x] = ext > 0.0f ? __fdiv_rn(1024.0f, ext) : 0.0f;
    }
    __syncthreads();
    const int i = blockIdx.x * INIT_T + threadIdx.x;
    if (i >= n) return;
    uint32_t code = 0;
    for (int a = 0; a < 3; a++) {
        float q = floorf(__fmul_rn(__fsub_rn(means[3 * i + a], lo[a]), sc[a]));
        q = fminf(fmaxf(q, 0.0f), 1023.0f);
        code |= spread3((uint32_t)q) << a;
    }
    keys[i] = ((unsigned long long)code << 32) | (uint32_t)i;
}

__global__ void k_one_segment(uint32_t n, uint32_t* __restrict__ starts) {
    if (threadIdx.x == 0) { starts[0] = 0u; starts[1] = n; }
}

int spatial_order_blocks(int n) { return max(1, min((n + INIT_T - 1) / INIT_T, 4 * 152)); }

void launch_spatial_keys(int n, const float* means, float* part, unsigned long long* keys, uint32_t* starts,
                         cudaStream_t s) {
    const int nb = spatial_order_blocks(n);
    k_bbox_partial<<<nb, INIT_T, 0, s>>>(n, means, part);
    k_morton_keys<<<(n + INIT_T - 1) / INIT_T, INIT_T, 0, s>>>(n, nb, means, part, keys);
    k_one_segment<<<1, 32, 0, s>>>((uint32_t)n, starts);
}

// dst[j] = src[perm[j]] for row arrays (gather by a permutation).
__global__ void k_gather_rows(int n, const uint32_t* __restrict__ perm, CompactArrays ca) {
    const int j = blockIdx.x * INIT_T + threadIdx.x;
    if (j >= n) return;
    const size_t i = perm[j];
    for (int a = 0; a < ca.count; a++) {
        const int w = ca.width[a];
        const float* src = ca.src[a] + i * w;
        float* dst = ca.dst[a] + (size_t)j * w;
        for (int c = 0; c < w; c++) dst[c] = src[c];
    }
}

void launch_gather_rows(int n, const uint32_t* perm, const CompactArrays& ca, cudaStream_t s) {
    if (n <= 0) return;
    k_gather_rows<<<(n + INIT_T - 1) / INIT_T, INIT_T, 0, s>>>(n, perm, ca);
}

}  // namespace gs
