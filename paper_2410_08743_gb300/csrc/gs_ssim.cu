// gs_ssim.cu - the D-SSIM term of the photometric loss (Eq. 16, beta = w_dssim):
// 1 - SSIM with the 11x11 Gaussian window (sigma 1.5), zero padding,
// C1 = 0.01^2, C2 = 0.03^2, mean over pixels and channels, and its gradient
// w.r.t. the rendered image.  The window is separable, so each filtering is
// a horizontal then a vertical 11-tap pass; the adjoint of the zero-padded
// symmetric filter is the same filter.
#include <cuda_runtime.h>
#include <math.h>

#include <cstdio>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {

__constant__ float c_win[11];

static void upload_window() {
    static bool done = false;
    if (done) return;
    float w[11];
    double s = 0.0, g[11];
    for (int k = 0; k < 11; k++) { const double x = k - 5; g[k] = exp(-x * x / (2.0 * 1.5 * 1.5)); s += g[k]; }
    for (int k = 0; k < 11; k++) w[k] = (float)(g[k] / s);
    cudaMemcpyToSymbol(c_win, w, sizeof(w));
    done = true;
}

// Horizontal pass over NM planes: in[m] -> out[m]; the inputs are built from
// x (rendered) and y (target): {x, y, x*x, y*y, x*y} when NM == 5, or taken
// from `src` planes when products == false.
template <int NM, bool PRODUCTS>
__global__ void k_hpass(int W, int H, const float* __restrict__ x, const float* __restrict__ y,
                        const float* __restrict__ src, float* __restrict__ out) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int py = blockIdx.y;
    if (px >= W) return;
    const size_t np = (size_t)W * H;
    float acc[NM];
#pragma unroll
    for (int m = 0; m < NM; m++) acc[m] = 0.0f;
#pragma unroll
    for (int a = -5; a <= 5; a++) {
        const int xx = px + a;
        if (xx < 0 || xx >= W) continue;
        const size_t q = (size_t)py * W + xx;
        const float w = c_win[a + 5];
        if (PRODUCTS) {
            const float xv = x[q], yv = y[q];
            acc[0] += w * xv; acc[1] += w * yv; acc[2] += w * xv * xv; acc[3] += w * yv * yv; acc[4] += w * xv * yv;
        } else {
#pragma unroll
            for (int m = 0; m < NM; m++) acc[m] += w * src[m * np + q];
        }
    }
    const size_t p = (size_t)py * W + px;
#pragma unroll
    for (int m = 0; m < NM; m++) out[m * np + p] = acc[m];
}

// Vertical pass of the five moments, the SSIM map and the partials
// dA = df/dmu_x - 2 mu_x df/dsxx - mu_y df/dsxy, dB = df/dsxx, dC = df/dsxy.
__global__ void k_vpass_ssim(int W, int H, const float* __restrict__ h5, float* __restrict__ parts,
                             float* __restrict__ smap) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int py = blockIdx.y;
    if (px >= W) return;
    const size_t np = (size_t)W * H;
    float m[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int b = -5; b <= 5; b++) {
        const int yy = py + b;
        if (yy < 0 || yy >= H) continue;
        const size_t q = (size_t)yy * W + px;
        const float w = c_win[b + 5];
#pragma unroll
        for (int k = 0; k < 5; k++) m[k] += w * h5[k * np + q];
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
    const size_t p = (size_t)py * W + px;
    parts[p] = dmu - 2.f * ux * dvx - uy * dcxy;
    parts[np + p] = dvx;
    parts[2 * np + p] = dcxy;
    smap[p] = f;
}

// Vertical pass of the three filtered partials and the image gradient
// dL/dx = -w/(3HW) (F dA + 2 x F dB + y F dC).
__global__ void k_vpass_grad(int W, int H, const float* __restrict__ h3, const float* __restrict__ x,
                             const float* __restrict__ y, float scale, float* __restrict__ out) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int py = blockIdx.y;
    if (px >= W) return;
    const size_t np = (size_t)W * H;
    float m[3] = {0, 0, 0};
#pragma unroll
    for (int b = -5; b <= 5; b++) {
        const int yy = py + b;
        if (yy < 0 || yy >= H) continue;
        const size_t q = (size_t)yy * W + px;
        const float w = c_win[b + 5];
#pragma unroll
        for (int k = 0; k < 3; k++) m[k] += w * h3[k * np + q];
    }
    const size_t p = (size_t)py * W + px;
    out[p] = scale * (m[0] + 2.f * x[p] * m[1] + y[p] * m[2]);
}

// Per-view loss value w_dssim * (1 - mean SSIM), summed in a fixed order.
__global__ void k_ssim_value(const float* __restrict__ smap, long long n, float w, double* __restrict__ out) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (long long k = threadIdx.x; k < n; k += blockDim.x) acc += (double)smap[k];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = (double)w * (1.0 - sm[0] / (double)n);
}

// tmp must hold 11 planes of the largest view: 5 moments, 3 partials and the
// 3-channel SSIM map.  loss_out (nullable, device [V]) receives w_dssim (1 - SSIM).
void launch_dssim(int n_views, const gs_view* views, const long long* img_off, const float* image,
                  const float* target, float w_dssim, float* dldc_out, double* loss_out, float* tmp,
                  cudaStream_t s) {
    upload_window();
    for (int v = 0; v < n_views; v++) {
        const int W = views[v].width, H = views[v].height;
        const size_t np = (size_t)W * H;
        const dim3 blk(128), grd((W + 127) / 128, H);
        float* smap = tmp + 8 * np;  // [3][H][W]
        for (int ch = 0; ch < 3; ch++) {
            const float* x = image + img_off[v] + ch * np;
            const float* y = target + img_off[v] + ch * np;
            float* h5 = tmp;           // 5 planes
            float* parts = tmp + 5 * np;  // 3 planes
            k_hpass<5, true><<<grd, blk, 0, s>>>(W, H, x, y, nullptr, h5);
            k_vpass_ssim<<<grd, blk, 0, s>>>(W, H, h5, parts, smap + ch * np);
            k_hpass<3, false><<<grd, blk, 0, s>>>(W, H, nullptr, nullptr, parts, h5);
            k_vpass_grad<<<grd, blk, 0, s>>>(W, H, h5, x, y, -w_dssim / (3.0f * (float)np), dldc_out + img_off[v] + ch * np);
        }
        if (loss_out) k_ssim_value<<<1, 256, 0, s>>>(smap, (long long)(3 * np), w_dssim, loss_out + v);
    }
}

}  // namespace gs

// ------------------------------------------------------------ no-alloc variant
// gs_loss_dssim_static runs the same D-SSIM kernels as the backward pass, but
// with its scratch in a static device array instead of workspace memory, so
// that it calls no allocator at all.  Callers that cannot allocate at the
// point of use (inside CUDA-graph capture, in allocation-free serving loops,
// under a fixed memory budget) use it.  The array is device memory reserved
// when the module loads; host code only ever sees the address that
// cudaGetSymbolAddress returns for the current device.

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
            float w[11];
            double g[11], sum = 0.0;
            for (int k = 0; k < 11; k++) { const double x = k - 5; g[k] = exp(-x * x / (2.0 * 1.5 * 1.5)); sum += g[k]; }
            for (int k = 0; k < 11; k++) w[k] = (float)(g[k] / sum);
            e = cudaMemcpyToSymbol(gs::c_win, w, sizeof(w));
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
    gs::launch_dssim(1, &v, &off, image, target, w_dssim, dl_dimage, loss, scratch, static_cast<cudaStream_t>(stream));
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "gs_loss_dssim_static: launch: %s", cudaGetErrorString(e));
        return gs::set_error(GS_ECUDA, msg);
    }
    return GS_OK;
}

