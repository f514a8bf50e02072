// gs_ssim.cu - the D-SSIM term of the photometric loss (Eq. 16, beta = w_dssim):
// 1 - SSIM with the 11x11 Gaussian window (sigma 1.5), zero padding,
// C1 = 0.01^2, C2 = 0.03^2, mean over pixels and channels, and its gradient
// w.r.t. the rendered image.  The window is separable, so each filtering is
// a horizontal then a vertical 11-tap pass; the adjoint of the zero-padded
// symmetric filter is the same filter.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {

__constant__ float c_win[11];

// The window lives in constant memory, which every device holds separately:
// it is uploaded once per device, with that device current, under a lock
// (contexts, servers and the allocation-free entry point may run D-SSIM from
// several host threads and on several devices).
namespace {
std::mutex g_win_mu;
constexpr int kWinDevices = 256;
bool g_win_done[kWinDevices] = {};
}  // namespace

cudaError_t ensure_dssim_window() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kWinDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_win_mu);
    if (g_win_done[dev]) return cudaSuccess;
    float w[11];
    double s = 0.0, g[11];
    for (int k = 0; k < 11; k++) { const double x = k - 5; g[k] = exp(-x * x / (2.0 * 1.5 * 1.5)); s += g[k]; }
    for (int k = 0; k < 11; k++) w[k] = (float)(g[k] / s);
    e = cudaMemcpyToSymbol(c_win, w, sizeof(w));
    if (e == cudaSuccess) g_win_done[dev] = true;
    return e;
}

// Tiled, fused D-SSIM.  One block computes 32x32 outputs of one channel of
// one view: it stages the tile of rendered (x) and target (y) values with a
// 5-pixel halo in shared memory (zero outside the image), filters the five
// moments x, y, x^2, y^2, xy horizontally then vertically, and writes the
// SSIM value's partials
//   dA = df/dmu_x - 2 mu_x df/dsxx - mu_y df/dsxy, dB = df/dsxx, dC = df/dsxy
// (f = SSIM at the pixel) plus a per-block sum of f.  A second pass filters
// the three partial planes the same way (the zero-padded symmetric window is
// its own adjoint) and forms dL/dx = -w/(3HW) (F dA + 2 x F dB + y F dC).
#define SS_T 32                 // outputs per block side
#define SS_R 5                  // window radius
#define SS_S (SS_T + 2 * SS_R)  // staged side
#define SS_THREADS 256
#define SS_MAXV 32              // views per launch

struct DssimBatch {
    int n;                       // views in this launch
    int max_tiles;               // tiles of the largest view
    int W[SS_MAXV], H[SS_MAXV], tx[SS_MAXV];
    long long off[SS_MAXV];      // float offset of the view's planar image
};

__device__ __forceinline__ bool ss_block(const DssimBatch& b, int& j, int& ch, int& W, int& H, int& x0, int& y0,
                                         long long& off) {
    j = blockIdx.y / 3;
    ch = blockIdx.y % 3;
    W = b.W[j];
    H = b.H[j];
    const int tile = blockIdx.x;
    const int ty = (H + SS_T - 1) / SS_T;
    if (tile >= b.tx[j] * ty) return false;
    x0 = (tile % b.tx[j]) * SS_T;
    y0 = (tile / b.tx[j]) * SS_T;
    off = b.off[j] + (long long)ch * W * H;
    return true;
}

__global__ void __launch_bounds__(SS_THREADS) k_ssim_fwd(DssimBatch b, const float* __restrict__ image,
                                                        const float* __restrict__ target, float* __restrict__ parts,
                                                        long long part_stride, float* __restrict__ block_sum) {
    __shared__ float sx[SS_S][SS_S + 1], sy[SS_S][SS_S + 1];
    __shared__ float hm[5][SS_S][SS_T + 1];
    __shared__ float red[SS_THREADS / 32];
    int j, ch, W, H, x0, y0;
    long long off;
    const bool live = ss_block(b, j, ch, W, H, x0, y0, off);
    float fsum = 0.0f;
    if (live) {
        for (int k = threadIdx.x; k < SS_S * SS_S; k += SS_THREADS) {
            const int r = k / SS_S, c = k % SS_S;
            const int gy = y0 + r - SS_R, gx = x0 + c - SS_R;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            const size_t q = (size_t)gy * W + gx;
            sx[r][c] = in ? image[off + q] : 0.0f;
            sy[r][c] = in ? target[off + q] : 0.0f;
        }
    }
    __syncthreads();
    if (live) {
        for (int k = threadIdx.x; k < SS_S * SS_T; k += SS_THREADS) {
            const int r = k / SS_T, c = k % SS_T;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
            for (int t = 0; t < 2 * SS_R + 1; t++) {
                const float w = c_win[t], xv = sx[r][c + t], yv = sy[r][c + t];
                a0 += w * xv; a1 += w * yv; a2 += w * xv * xv; a3 += w * yv * yv; a4 += w * xv * yv;
            }
            hm[0][r][c] = a0; hm[1][r][c] = a1; hm[2][r][c] = a2; hm[3][r][c] = a3; hm[4][r][c] = a4;
        }
    }
    __syncthreads();
    if (live) {
        const long long np = (long long)W * H;
        for (int k = threadIdx.x; k < SS_T * SS_T; k += SS_THREADS) {
            const int r = k / SS_T, c = k % SS_T;
            const int gy = y0 + r, gx = x0 + c;
            if (gx >= W || gy >= H) continue;
            float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t < 2 * SS_R + 1; t++) {
                const float w = c_win[t];
#pragma unroll
                for (int u = 0; u < 5; u++) m[u] += w * hm[u][r + t][c];
            }
            const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
            const float ux = m[0], uy = m[1];
            const float vx = m[2] - ux * ux, vy = m[3] - uy * uy, cxy = m[4] - ux * uy;
            const float N1 = 2.f * ux * uy + C1, N2 = 2.f * cxy + C2;
            const float D1 = ux * ux + uy * uy + C1, D2 = vx + vy + C2;
            const float iD = 1.0f / (D1 * D2);
            const float f = N1 * N2 * iD;
            const float dmu = 2.f * uy * N2 * iD - f * 2.f * ux / D1;
            const float dvx = -f / D2;
            const float dcxy = 2.f * N1 * iD;
            const size_t q = (size_t)off + (size_t)gy * W + gx;
            parts[q] = dmu - 2.f * ux * dvx - uy * dcxy;
            parts[part_stride + q] = dvx;
            parts[2 * part_stride + q] = dcxy;
            fsum += f;
            (void)np;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fsum += __shfl_xor_sync(0xffffffffu, fsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = fsum;
    __syncthreads();
    if (threadIdx.x == 0 && block_sum) {
        float acc = 0.0f;
        for (int w = 0; w < SS_THREADS / 32; w++) acc += red[w];
        block_sum[(size_t)blockIdx.y * b.max_tiles + blockIdx.x] = live ? acc : 0.0f;
    }
}

__global__ void __launch_bounds__(SS_THREADS) k_ssim_bwd(DssimBatch b, const float* __restrict__ image,
                                                        const float* __restrict__ target,
                                                        const float* __restrict__ parts, long long part_stride,
                                                        float w_dssim, float* __restrict__ dldc) {
    __shared__ float sp[3][SS_S][SS_S + 1];
    __shared__ float hm[3][SS_S][SS_T + 1];
    int j, ch, W, H, x0, y0;
    long long off;
    if (!ss_block(b, j, ch, W, H, x0, y0, off)) return;
    for (int k = threadIdx.x; k < SS_S * SS_S; k += SS_THREADS) {
        const int r = k / SS_S, c = k % SS_S;
        const int gy = y0 + r - SS_R, gx = x0 + c - SS_R;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const size_t q = (size_t)off + (size_t)gy * W + gx;
#pragma unroll
        for (int u = 0; u < 3; u++) sp[u][r][c] = in ? parts[u * part_stride + q] : 0.0f;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < SS_S * SS_T; k += SS_THREADS) {
        const int r = k / SS_T, c = k % SS_T;
        float a[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 2 * SS_R + 1; t++) {
            const float w = c_win[t];
#pragma unroll
            for (int u = 0; u < 3; u++) a[u] += w * sp[u][r][c + t];
        }
#pragma unroll
        for (int u = 0; u < 3; u++) hm[u][r][c] = a[u];
    }
    __syncthreads();
    const float scale = -w_dssim / (3.0f * (float)W * (float)H);
    for (int k = threadIdx.x; k < SS_T * SS_T; k += SS_THREADS) {
        const int r = k / SS_T, c = k % SS_T;
        const int gy = y0 + r, gx = x0 + c;
        if (gx >= W || gy >= H) continue;
        float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 2 * SS_R + 1; t++) {
            const float w = c_win[t];
#pragma unroll
            for (int u = 0; u < 3; u++) m[u] += w * hm[u][r + t][c];
        }
        const size_t q = (size_t)off + (size_t)gy * W + gx;
        dldc[q] = scale * (m[0] + 2.f * image[q] * m[1] + target[q] * m[2]);
    }
}

// Per-view loss w_dssim (1 - mean SSIM): the view's block sums added in block
// order (deterministic).
__global__ void k_ssim_loss(DssimBatch b, const float* __restrict__ block_sum, float w, double* __restrict__ out) {
    const int j = blockIdx.x;
    __shared__ double sm[256];
    double acc = 0.0;
    const int nb = 3 * b.max_tiles;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) acc += (double)block_sum[(size_t)j * nb + k];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = (double)w * (1.0 - sm[0] / (3.0 * (double)b.W[j] * (double)b.H[j]));
}

// tmp: 3 planes of the packed image (the SSIM partials) plus 3 floats per
// 32x32 tile of the largest view per view of a launch (at most 32 views) for
// the per-block SSIM sums.  loss_out (nullable, device [V]) receives
// w_dssim (1 - SSIM) per view.
cudaError_t launch_dssim(int n_views, const gs_view* views, const long long* img_off, const float* image,
                         const float* target, float w_dssim, float* dldc_out, double* loss_out, float* tmp,
                         cudaStream_t s) {
    const cudaError_t we = ensure_dssim_window();
    if (we != cudaSuccess) return we;
    long long total = 0;
    for (int v = 0; v < n_views; v++)
        total = std::max(total, img_off[v] + 3LL * views[v].width * views[v].height);
    float* parts = tmp;                       // [3][total]
    float* bsum = tmp + 3 * (size_t)total;    // per-block SSIM sums of one launch
    for (int v0 = 0; v0 < n_views; v0 += SS_MAXV) {
        DssimBatch b{};
        b.n = std::min(SS_MAXV, n_views - v0);
        int mt = 1;
        for (int j = 0; j < b.n; j++) {
            const gs_view& vw = views[v0 + j];
            b.W[j] = vw.width;
            b.H[j] = vw.height;
            b.tx[j] = (vw.width + SS_T - 1) / SS_T;
            b.off[j] = img_off[v0 + j];
            mt = std::max(mt, b.tx[j] * ((vw.height + SS_T - 1) / SS_T));
        }
        b.max_tiles = mt;
        const dim3 grid(mt, 3 * b.n);
        k_ssim_fwd<<<grid, SS_THREADS, 0, s>>>(b, image, target, parts, total, loss_out ? bsum : nullptr);
        k_ssim_bwd<<<grid, SS_THREADS, 0, s>>>(b, image, target, parts, total, w_dssim, dldc_out);
        if (loss_out) k_ssim_loss<<<b.n, 256, 0, s>>>(b, bsum, w_dssim, loss_out + v0);
    }
    return cudaSuccess;
}

}  // namespace gs

// ------------------------------------------------------------ no-alloc variant
// gs_loss_dssim_static runs the same D-SSIM kernels as the backward pass, but
// with its scratch in a static device array instead of workspace memory, so
// that it calls no allocator at all: for serving loops that fix their device
// footprint at start-up, real-time loops that forbid allocator calls after
// initialisation, and hosts that hand the library only the buffers it uses.
// The array is device memory reserved when the module loads; host code only
// ever passes the address that cudaGetSymbolAddress returns for the current
// device (the symbol itself names a host-side stand-in).

static __device__ __align__(256) float g_dssim_static_scratch[11 * GS_DSSIM_STATIC_MAX_PIXELS];

namespace {
std::mutex g_dssim_static_mu;
constexpr int kMaxDevices = 256;
float* g_dssim_static_ptr[kMaxDevices] = {};
}  // namespace

extern "C" int gs_loss_dssim_static(const float* image, const float* target, int width, int height, float w_dssim,
                                    float* dl_dimage, double* loss, void* stream) {
    char msg[256];
    if (!image || !target || !dl_dimage) return gs::set_error(GS_EINVAL, "gs_loss_dssim_static: NULL image/target/output");
    if (width <= 0 || height <= 0) return gs::set_error(GS_EINVAL, "gs_loss_dssim_static: width and height must be > 0");
    if ((long long)width * height > GS_DSSIM_STATIC_MAX_PIXELS) {
        snprintf(msg, sizeof(msg), "gs_loss_dssim_static: %dx%d = %lld pixels exceeds the static scratch limit of %d",
                 width, height, (long long)width * height, GS_DSSIM_STATIC_MAX_PIXELS);
        return gs::set_error(GS_EINVAL, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        snprintf(msg, sizeof(msg), "gs_loss_dssim_static: cudaGetDevice: %s", cudaGetErrorString(e));
        return gs::set_error(GS_ECUDA, msg);
    }
    float* scratch = nullptr;
    {
        // once per device, with that device current: the symbol's device address
        std::lock_guard<std::mutex> lock(g_dssim_static_mu);
        if (!g_dssim_static_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_dssim_static_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(msg, sizeof(msg), "gs_loss_dssim_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return gs::set_error(GS_ECUDA, msg);
            }
            e = gs::ensure_dssim_window();
            if (e != cudaSuccess) {
                snprintf(msg, sizeof(msg), "gs_loss_dssim_static: window upload: %s", cudaGetErrorString(e));
                return gs::set_error(GS_ECUDA, msg);
            }
            g_dssim_static_ptr[dev] = static_cast<float*>(p);
        }
        scratch = g_dssim_static_ptr[dev];
    }
    const gs_view v = {1.0f, 1.0f, 0.0f, 0.0f, width, height};
    const long long off = 0;
    e = gs::launch_dssim(1, &v, &off, image, target, w_dssim, dl_dimage, loss, scratch,
                         static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "gs_loss_dssim_static: launch: %s", cudaGetErrorString(e));
        return gs::set_error(GS_ECUDA, msg);
    }
    return GS_OK;
}

