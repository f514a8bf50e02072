// gs_init.cu - Gaussians initialised from one frame and a depth map, the
// first stage of relative pose estimation (Sec. 3.4): a subset of the pixels
// is unprojected with the intrinsics into a point cloud, every point becomes
// an isotropic Gaussian with the pixel's colour, and its scale is the mean
// 3D distance to its three nearest neighbours.
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

}  // namespace gs
