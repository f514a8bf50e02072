// gs_preprocess.cu - per-(view, Gaussian) projection (Sec. 3.1, Eq. 1-2 and
// the SH colour) and its backward with the fused camera-pose gradient
// (Sec. 3.2, Eq. 7-13).
//
// Batched form: one thread per Gaussian reads its parameters once and loops
// over every view of the launch, so a batch of V views costs one read of the
// scene instead of V.
//
// Key path.  Culling, the screen radius, the tile rectangle and the depth key
// are computed as FP32 operations in a fixed order with explicit round-to-
// nearest intrinsics (no contraction), so that the tile lists are a defined
// function of the inputs and reproducible bit for bit.
#include <cuda_runtime.h>

#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

// ------------------------------------------------------------ view setup
__global__ void k_setup_views(int n_views, const double* __restrict__ poses, ViewDev* __restrict__ views,
                              float clamp_factor) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_views) return;
    ViewDev vd = views[v];
    const double* P = poses + 12 * v;
    for (int k = 0; k < 9; k++) {
        vd.Rf[k] = __double2float_rn(P[k]);
        vd.Rlo[k] = __double2float_rn(P[k] - (double)vd.Rf[k]);
    }
    for (int k = 0; k < 3; k++) {
        vd.tf[k] = __double2float_rn(P[9 + k]);
        vd.tlo[k] = __double2float_rn(P[9 + k] - (double)vd.tf[k]);
    }
    for (int a = 0; a < 3; a++)
        vd.oc[a] = __double2float_rn(-(P[0 * 3 + a] * P[9] + P[1 * 3 + a] * P[10] + P[2 * 3 + a] * P[11]));
    if (clamp_factor > 0.0f) {
        float tanx = __fdiv_rn((float)vd.W, __fmul_rn(2.0f, vd.fx));
        float tany = __fdiv_rn((float)vd.H, __fmul_rn(2.0f, vd.fy));
        vd.limx = __fmul_rn(clamp_factor, tanx);
        vd.limy = __fmul_rn(clamp_factor, tany);
    } else {
        vd.limx = vd.limy = 0.0f;
    }
    vd.inv_npix3 = 1.0f / (3.0f * (float)vd.W * (float)vd.H);
    views[v] = vd;
}

void launch_setup_views(const gs_view*, int n_views, const double* poses, ViewDev* views_dev, const RenderParams& rp,
                        cudaStream_t s) {
    if (n_views <= 0) return;
    k_setup_views<<<(n_views + 63) / 64, 64, 0, s>>>(n_views, poses, views_dev, rp.clamp_factor);
}

// ------------------------------------------------------------ FP32 key path
#define FM(a, b) __fmul_rn((a), (b))
#define FA(a, b) __fadd_rn((a), (b))
#define FS(a, b) __fsub_rn((a), (b))
#define FD(a, b) __fdiv_rn((a), (b))

// View-independent part: normalised quaternion -> R -> M = R diag(s) ->
// Sigma = M M^T (six unique entries S00 S01 S02 S11 S12 S22).
__device__ __forceinline__ void key_sigma(const float q[4], const float sc[3], float S[6]) {
    float n2 = FM(q[0], q[0]);
    n2 = FA(n2, FM(q[1], q[1]));
    n2 = FA(n2, FM(q[2], q[2]));
    n2 = FA(n2, FM(q[3], q[3]));
    float inv = FD(1.0f, __fsqrt_rn(n2));
    float w = FM(q[0], inv), x = FM(q[1], inv), y = FM(q[2], inv), z = FM(q[3], inv);
    float R[9];
    R[0] = FS(1.0f, FM(2.0f, FA(FM(y, y), FM(z, z))));
    R[1] = FM(2.0f, FS(FM(x, y), FM(w, z)));
    R[2] = FM(2.0f, FA(FM(x, z), FM(w, y)));
    R[3] = FM(2.0f, FA(FM(x, y), FM(w, z)));
    R[4] = FS(1.0f, FM(2.0f, FA(FM(x, x), FM(z, z))));
    R[5] = FM(2.0f, FS(FM(y, z), FM(w, x)));
    R[6] = FM(2.0f, FS(FM(x, z), FM(w, y)));
    R[7] = FM(2.0f, FA(FM(y, z), FM(w, x)));
    R[8] = FS(1.0f, FM(2.0f, FA(FM(x, x), FM(y, y))));
    float M[9];
#pragma unroll
    for (int j = 0; j < 3; j++)
#pragma unroll
        for (int k = 0; k < 3; k++) M[j * 3 + k] = FM(R[j * 3 + k], sc[k]);
    int t = 0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++) {
            float s0 = FM(M[a * 3 + 0], M[b * 3 + 0]);
            float s1 = FM(M[a * 3 + 1], M[b * 3 + 1]);
            float s2 = FM(M[a * 3 + 2], M[b * 3 + 2]);
            S[t++] = FA(FA(s0, s1), s2);
        }
}

__device__ __forceinline__ float sym3(const float S[6], int a, int b) {
    // index into the upper triangle (00 01 02 11 12 22)
    if (a > b) { int t = a; a = b; b = t; }
    return a == 0 ? S[b] : (a == 1 ? S[2 + b] : S[5]);
}

struct KeyOut {
    float depth, mx, my, A, B, C, det;
    int radius;
    int x0, y0, x1, y1;
};

// View-dependent part; returns false if culled.
__device__ __forceinline__ bool key_view(const float mu[3], const float S[6], const ViewDev& vd,
                                         const RenderParams& rp, KeyOut& o) {
    const float* Rc = vd.Rf;
    float mc[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float t0 = FM(Rc[a * 3 + 0], mu[0]);
        float t1 = FM(Rc[a * 3 + 1], mu[1]);
        float t2 = FM(Rc[a * 3 + 2], mu[2]);
        mc[a] = FA(FA(FA(t0, t1), t2), vd.tf[a]);
    }
    float zc = mc[2];
    if (!(zc > rp.z_near)) return false;
    float Tm[9];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            float t0 = FM(Rc[a * 3 + 0], sym3(S, 0, b));
            float t1 = FM(Rc[a * 3 + 1], sym3(S, 1, b));
            float t2 = FM(Rc[a * 3 + 2], sym3(S, 2, b));
            Tm[a * 3 + b] = FA(FA(t0, t1), t2);
        }
    float Sc[6];
    int t = 0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++) {
            float t0 = FM(Tm[a * 3 + 0], Rc[b * 3 + 0]);
            float t1 = FM(Tm[a * 3 + 1], Rc[b * 3 + 1]);
            float t2 = FM(Tm[a * 3 + 2], Rc[b * 3 + 2]);
            Sc[t++] = FA(FA(t0, t1), t2);
        }
    // Sc: 0=00 1=01 2=02 3=11 4=12 5=22
    float txv = mc[0], tyv = mc[1];
    if (rp.clamp_factor > 0.0f) {
        float ux = FD(mc[0], zc), uy = FD(mc[1], zc);
        float nlx = -vd.limx, nly = -vd.limy;
        ux = ux < nlx ? nlx : ux; ux = ux > vd.limx ? vd.limx : ux;
        uy = uy < nly ? nly : uy; uy = uy > vd.limy ? vd.limy : uy;
        txv = FM(ux, zc); tyv = FM(uy, zc);
    }
    float zz = FM(zc, zc);
    float j00 = FD(vd.fx, zc), j11 = FD(vd.fy, zc);
    float j02 = -FD(FM(vd.fx, txv), zz);
    float j12 = -FD(FM(vd.fy, tyv), zz);
    float U00 = FA(FM(j00, Sc[0]), FM(j02, Sc[2]));
    float U01 = FA(FM(j00, Sc[1]), FM(j02, Sc[4]));
    float U02 = FA(FM(j00, Sc[2]), FM(j02, Sc[5]));
    float U11 = FA(FM(j11, Sc[3]), FM(j12, Sc[4]));
    float U12 = FA(FM(j11, Sc[4]), FM(j12, Sc[5]));
    float A = FA(FM(U00, j00), FM(U02, j02));
    float B = FA(FM(U01, j11), FM(U02, j12));
    float C = FA(FM(U11, j11), FM(U12, j12));
    A = FA(A, rp.eps2d);
    C = FA(C, rp.eps2d);
    float det = FS(FM(A, C), FM(B, B));
    if (!(det > 0.0f)) return false;
    float mid = FM(0.5f, FA(A, C));
    float disc = FS(FM(mid, mid), det);
    if (!(disc > 0.1f)) disc = 0.1f;
    float lam = FA(mid, __fsqrt_rn(disc));
    float rf = ceilf(FM(3.0f, __fsqrt_rn(lam)));
    float mx = FA(FD(FM(vd.fx, mc[0]), zc), vd.cx);
    float my = FA(FD(FM(vd.fy, mc[1]), zc), vd.cy);
    const float invt = 1.0f / (float)GS_TILE;
    float rb = FA(rf, (float)(GS_TILE - 1));
    float fx0 = floorf(FM(FS(mx, rf), invt));
    float fy0 = floorf(FM(FS(my, rf), invt));
    float fx1 = floorf(FM(FA(mx, rb), invt));
    float fy1 = floorf(FM(FA(my, rb), invt));
    float gwf = (float)vd.gw, ghf = (float)vd.gh;
    if (!(fx0 >= 0.0f)) fx0 = 0.0f; if (fx0 > gwf) fx0 = gwf;
    if (!(fy0 >= 0.0f)) fy0 = 0.0f; if (fy0 > ghf) fy0 = ghf;
    if (!(fx1 >= 0.0f)) fx1 = 0.0f; if (fx1 > gwf) fx1 = gwf;
    if (!(fy1 >= 0.0f)) fy1 = 0.0f; if (fy1 > ghf) fy1 = ghf;
    o.x0 = (int)fx0; o.y0 = (int)fy0; o.x1 = (int)fx1; o.y1 = (int)fy1;
    if (o.x1 <= o.x0 || o.y1 <= o.y0) return false;
    o.depth = zc; o.mx = mx; o.my = my; o.A = A; o.B = B; o.C = C; o.det = det;
    o.radius = (int)rf;
    return true;
}

#undef FM
#undef FA
#undef FS
#undef FD

// ------------------------------------------------------------ SH basis
// Real SH constants sqrt(k/pi) with the Condon-Shortley phase, l <= 3.
#define SH_C0 0.28209479177387814f
#define SH_C1 0.48860251190291992f
#define SH_C2a 1.0925484305920792f
#define SH_C2b 0.31539156525252005f
#define SH_C2c 0.54627421529603959f
#define SH_C3a 0.59004358992664352f
#define SH_C3b 2.8906114426405538f
#define SH_C3c 0.45704579946446572f
#define SH_C3d 0.37317633259011546f
#define SH_C3e 1.4453057213202769f

template <int D>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    Y[0] = SH_C0;
    if (D >= 1) { Y[1] = -SH_C1 * y; Y[2] = SH_C1 * z; Y[3] = -SH_C1 * x; }
    if (D >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = SH_C2a * x * y;
        Y[5] = -SH_C2a * y * z;
        Y[6] = SH_C2b * (2.0f * zz - xx - yy);
        Y[7] = -SH_C2a * x * z;
        Y[8] = SH_C2c * (xx - yy);
        if (D >= 3) {
            Y[9] = -SH_C3a * y * (3.0f * xx - yy);
            Y[10] = SH_C3b * x * y * z;
            Y[11] = -SH_C3c * y * (4.0f * zz - xx - yy);
            Y[12] = SH_C3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -SH_C3c * x * (4.0f * zz - xx - yy);
            Y[14] = SH_C3e * z * (xx - yy);
            Y[15] = -SH_C3a * x * (xx - 3.0f * yy);
        }
    }
}

// Gradient of sum_k c_k Y_k(x, y, z) w.r.t. (x, y, z) for coefficient
// weights c[k] (treating the components as independent).
template <int D>
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float c[16], float g[3]) {
    g[0] = g[1] = g[2] = 0.0f;
    if (D >= 1) { g[1] += -SH_C1 * c[1]; g[2] += SH_C1 * c[2]; g[0] += -SH_C1 * c[3]; }
    if (D >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        g[0] += SH_C2a * y * c[4]; g[1] += SH_C2a * x * c[4];
        g[1] += -SH_C2a * z * c[5]; g[2] += -SH_C2a * y * c[5];
        g[0] += -2.0f * SH_C2b * x * c[6]; g[1] += -2.0f * SH_C2b * y * c[6]; g[2] += 4.0f * SH_C2b * z * c[6];
        g[0] += -SH_C2a * z * c[7]; g[2] += -SH_C2a * x * c[7];
        g[0] += 2.0f * SH_C2c * x * c[8]; g[1] += -2.0f * SH_C2c * y * c[8];
        if (D >= 3) {
            g[0] += -SH_C3a * 6.0f * x * y * c[9]; g[1] += -SH_C3a * (3.0f * xx - 3.0f * yy) * c[9];
            g[0] += SH_C3b * y * z * c[10]; g[1] += SH_C3b * x * z * c[10]; g[2] += SH_C3b * x * y * c[10];
            g[0] += SH_C3c * 2.0f * x * y * c[11]; g[1] += -SH_C3c * (4.0f * zz - xx - 3.0f * yy) * c[11];
            g[2] += -SH_C3c * 8.0f * y * z * c[11];
            g[0] += -SH_C3d * 6.0f * x * z * c[12]; g[1] += -SH_C3d * 6.0f * y * z * c[12];
            g[2] += SH_C3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * c[12];
            g[0] += -SH_C3c * (4.0f * zz - 3.0f * xx - yy) * c[13]; g[1] += SH_C3c * 2.0f * x * y * c[13];
            g[2] += -SH_C3c * 8.0f * x * z * c[13];
            g[0] += SH_C3e * 2.0f * x * z * c[14]; g[1] += -SH_C3e * 2.0f * y * z * c[14];
            g[2] += SH_C3e * (xx - yy) * c[14];
            g[0] += -SH_C3a * (3.0f * xx - 3.0f * yy) * c[15]; g[1] += SH_C3a * 6.0f * x * y * c[15];
        }
    }
}

// ------------------------------------------------------------ precise mean
// The projected mean mu_hat = f (x_c / z_c) + c evaluated with FP32 pairs
// (value = hi + lo) built from the classical error-free transformations:
// Knuth's TwoSum and the FMA-based TwoProduct (Dekker, Ogita-Rump-Oishi).
// Relative error about 2^-44, against about 2^-22 for plain FP32: at 1280 px
// a plain FP32 mu_hat is off by ~1e-4 px, which moves alpha near its 1/255
// threshold by ~3e-4 relative and flips skip decisions.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// camera coordinate a of mu (exact FP32 inputs) under the split pose
__device__ __forceinline__ void cam_coord_ff(const ViewDev& vd, int a, const float mu[3], float& hi, float& lo) {
    float s = vd.tf[a], e = vd.tlo[a];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        float p, pe, se;
        two_prod(vd.Rf[a * 3 + j], mu[j], p, pe);
        two_sum(s, p, s, se);
        e = __fadd_rn(e, __fadd_rn(__fadd_rn(pe, se), __fmul_rn(vd.Rlo[a * 3 + j], mu[j])));
    }
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}
// f * (x / z) + c as a pair
__device__ __forceinline__ void project_ff(float xh, float xl, float zh, float zl, float f, float c, float& hi,
                                           float& lo) {
    // q need not be the rounded quotient: the residual below is exact for any q
    // within a few units in the last place of x / z, and the correction ql
    // carries it (the pair keeps its ~2^-44 relative error)
    const float q = __fdividef(xh, zh);
    float p, pe;
    two_prod(q, zh, p, pe);
    const float r = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(xh, p), pe), xl), __fmul_rn(q, zl));
    const float ql = __fdividef(r, zh);
    float m, me, s, se;
    two_prod(f, q, m, me);
    me = __fmaf_rn(f, ql, me);
    two_sum(m, c, s, se);
    const float e = __fadd_rn(se, me);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// ------------------------------------------------------------ forward
// 16-byte shared-memory read that the compiler keeps where it is written
// (inside the view loop, not hoisted into 48 live registers).
__device__ __forceinline__ float4 lds_f4(const float4* p) {
    float4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// Gaussians [i_begin, i_end) of the scene (a launch may cover a slice, so that
// the slices can start while later ones are still being uploaded), one per
// thread, looping over the views (in shared memory); the thread's SH
// coefficients are staged in shared memory once and read per view, which keeps
// the kernel near 60 registers instead of 124.
template <int D>
__global__ void __launch_bounds__(256) k_preprocess_fwd(SceneDev sc, int i_begin, int i_end, int n_views,
                                                        const ViewDev* __restrict__ views, RenderParams rp,
                                                        SplatArrays sp, uint32_t* __restrict__ tile_counts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ViewDev* sv = reinterpret_cast<ViewDev*>(smem_raw);
    constexpr int NC = (D + 1) * (D + 1);
    // the block's SH coefficients in groups of four, [group][thread]: the
    // 16-byte reads of consecutive lanes are consecutive
    constexpr int NG = (NC * 3 + 3) / 4;
    float4* ssh = reinterpret_cast<float4*>(smem_raw + sizeof(ViewDev) * n_views);
    {
        const int words = n_views * (int)(sizeof(ViewDev) / 4);
        const int* src = reinterpret_cast<const int*>(views);
        int* dst = reinterpret_cast<int*>(sv);
        for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
        const int g0 = i_begin + blockIdx.x * blockDim.x;
        const int ng = min((int)blockDim.x, i_end - g0);
        const float4* shb = reinterpret_cast<const float4*>(sc.sh + (size_t)g0 * 48);
        for (int w = threadIdx.x; w < ng * 12; w += blockDim.x) {
            const int g = w / 12, k4 = w - g * 12;
            if (k4 < NG) ssh[k4 * blockDim.x + g] = shb[w];
        }
    }
    __syncthreads();
    const int i = i_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= i_end) return;
    const float4* frow = ssh + threadIdx.x;
    float mu[3], s[3], q[4];
#pragma unroll
    for (int k = 0; k < 3; k++) { mu[k] = sc.means[3 * i + k]; s[k] = sc.scales[3 * i + k]; }
    {
        float4 qq = reinterpret_cast<const float4*>(sc.quats)[i];
        q[0] = qq.x; q[1] = qq.y; q[2] = qq.z; q[3] = qq.w;
    }
    const float op = sc.opac[i];
    float S[6];
    key_sigma(q, s, S);
    for (int v = 0; v < n_views; v++) {
        const ViewDev& vd = sv[v];
        const size_t k = (size_t)v * sc.n + i;
        KeyOut ko;
        if (!key_view(mu, S, vd, rp, ko)) {
            sp.rect[k] = make_uint2(0u, 0u);
            sp.depth[k] = 0.0f;
            sp.radius[k] = 0;
            continue;
        }
        // value path: conic and view-dependent colour
        float inv_det = fast_rcp(ko.det);   // value path: a unit in the last place is far inside its tolerance
        float ca = ko.C * inv_det, cb = -ko.B * inv_det, cc = ko.A * inv_det;
        float dx = mu[0] - vd.oc[0], dy = mu[1] - vd.oc[1], dz = mu[2] - vd.oc[2];
        float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= il; dy *= il; dz *= il;
        float Y[16];
        sh_basis<D>(dx, dy, dz, Y);
        // colour = sum_b f[b][ch] Y[b] + 1/2 per channel, in b order, the
        // coefficients read from the shared row for each view (not kept live
        // across the view loop)
        float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int k4 = 0; k4 < NG; k4++) {
            const float4 v4 = lds_f4(frow + k4 * blockDim.x);
            const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int idx = 4 * k4 + e;
                if (idx < NC * 3) col[idx % 3] = fmaf(vv[e], Y[idx / 3], col[idx % 3]);
            }
        }
#pragma unroll
        for (int ch = 0; ch < 3; ch++) col[ch] = fmaxf(col[ch], 0.0f);
        {
            float xh, xl, yh, yl, zh, zl, mxh, mxl, myh, myl;
            cam_coord_ff(vd, 0, mu, xh, xl);
            cam_coord_ff(vd, 1, mu, yh, yl);
            cam_coord_ff(vd, 2, mu, zh, zl);
            project_ff(xh, xl, zh, zl, vd.fx, vd.cx, mxh, mxl);
            project_ff(yh, yl, zh, zl, vd.fy, vd.cy, myh, myl);
            sp.Mlo[k] = make_float2(__fadd_rn(__fsub_rn(mxh, ko.mx), mxl), __fadd_rn(__fsub_rn(myh, ko.my), myl));
        }
        sp.A[k] = make_float4(ko.mx, ko.my, ca, cb);
        sp.B[k] = make_float4(cc, op, col[0], col[1]);
        sp.Cb[k] = col[2];
        sp.rect[k] = make_uint2(pack16(ko.x0, ko.y0), pack16(ko.x1, ko.y1));
        sp.depth[k] = ko.depth;
        sp.radius[k] = ko.radius;
        if (tile_counts) {  // direct per-key counting (the sort stage normally counts per chunk)
            uint32_t* tc = tile_counts + vd.tile_base;
            for (int ty = ko.y0; ty < ko.y1; ty++)
                for (int tx = ko.x0; tx < ko.x1; tx++) atomicAdd(tc + ty * vd.gw + tx, 1u);
        }
    }
}

void launch_preprocess_fwd(const SceneDev& sc, int threads, int n_views, const ViewDev* views, const RenderParams& rp,
                           SplatArrays sp, uint32_t* tile_counts, cudaStream_t s, int i_begin, int i_end) {
    if (i_end < 0 || i_end > sc.n) i_end = sc.n;
    if (i_begin < 0) i_begin = 0;
    if (i_end <= i_begin || n_views <= 0) return;
    const int T = threads == 128 ? 128 : 256;
    const int grid = (i_end - i_begin + T - 1) / T;
    const int deg = sc.sh_degree < 3 ? sc.sh_degree : 3;
    const size_t sm = sizeof(ViewDev) * (size_t)n_views + sizeof(float4) * ((3 * (deg + 1) * (deg + 1) + 3) / 4) * T;
    static std::atomic<unsigned long long> attr{0};
    once_per_device(attr, [](int) {
        const int mx = 200 * 1024;
        cudaFuncSetAttribute(k_preprocess_fwd<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_fwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_fwd<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    });
#define GS_PRE_FWD(D) k_preprocess_fwd<D><<<grid, T, sm, s>>>(sc, i_begin, i_end, n_views, views, rp, sp, tile_counts)
    switch (sc.sh_degree) {
        case 0: GS_PRE_FWD(0); break;
        case 1: GS_PRE_FWD(1); break;
        case 2: GS_PRE_FWD(2); break;
        default: GS_PRE_FWD(3); break;
    }
#undef GS_PRE_FWD
}

// ------------------------------------------------------------ backward
// Chain rule per (view, Gaussian), in the oracle's order:
//   conic -> Sigma_hat -> (J, Sigma_c) -> mu_c, Sigma -> M -> (s, R -> q)
//   colour -> SH coefficients and viewing direction -> mu
//   pose: rho += g_mu_c + R_c g_mu(SH);  phi += mu_c x g_mu_c + 2 w(Sigma_c G_Sigma_c)
// Asynchronous global -> shared copies (cp.async): a thread copies its own
// 2D gradients of the next views into shared memory and reads them back after
// waiting for their group, so several views' loads are in flight without
// holding registers.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// views of 2D gradients staged ahead of their use
#define PB_STAGES 5
#define PB_T 128

// Gaussians [i_begin, i_end) of the scene; i_begin is a multiple of the block
// size, and block b of the launch writes pose partial row i_begin / PB_T + b, so
// a sliced pass gives the same partials as one launch over all Gaussians.
template <int D, bool POSE_ONLY>
__global__ void __launch_bounds__(PB_T, 3) k_preprocess_bwd(SceneDev sc, int i_begin, int i_end, int n_views,
                                                        const ViewDev* __restrict__ views, RenderParams rp,
                                                        SplatArrays sp, Grad2DArrays g2d, gs_grads grads,
                                                        double* __restrict__ pose_partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ViewDev* sv = reinterpret_cast<ViewDev*>(smem_raw);
    const int nwarps = blockDim.x >> 5;
    double* spose = reinterpret_cast<double*>(smem_raw + ((sizeof(ViewDev) * n_views + 15) & ~(size_t)15));
    // SH-coefficient gradient accumulators of every thread, [coefficient][thread]
    // with rows padded to PB_T + 1 floats, so that both a thread's walk over its
    // coefficients and the block's row-major copies to and from global memory
    // are free of bank conflicts.  Before the view loop it holds the block's SH
    // coefficients on their way into registers.
    constexpr int SGS = PB_T + 1;
    float* sgf = reinterpret_cast<float*>(spose + (size_t)nwarps * n_views * 6);
    // staged 2D gradients, [stage][thread]
    constexpr int NC3 = 3 * (D + 1) * (D + 1);
    float4* stA = reinterpret_cast<float4*>(
        (reinterpret_cast<uintptr_t>(sgf + (size_t)NC3 * SGS) + 15) & ~(uintptr_t)15);
    float4* stB = stA + PB_STAGES * PB_T;
    float* stC = reinterpret_cast<float*>(stB + PB_STAGES * PB_T);
    {
        const int words = n_views * (int)(sizeof(ViewDev) / 4);
        const int* src = reinterpret_cast<const int*>(views);
        int* dst = reinterpret_cast<int*>(sv);
        for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
        for (int k = threadIdx.x; k < nwarps * n_views * 6; k += blockDim.x) spose[k] = 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i0 = i_begin + blockIdx.x * PB_T;            // the block's first Gaussian
    const int m_blk = min(PB_T, i_end - i0);               // its Gaussians
    const int i = i0 + threadIdx.x;
    const bool live = i < i_end;
    constexpr int NC = (D + 1) * (D + 1);
    float mu[3] = {0, 0, 0}, s[3] = {1, 1, 1}, qn[4] = {1, 0, 0, 0}, qlen = 1.0f;
    // SH coefficients: the block's rows (48 floats per Gaussian) read row-major
    // (coalesced) into shared memory, then each thread takes its own
    {
        // eight loads per thread in flight before their stores
        const int tot = m_blk * 48;
        const float* src = sc.sh + (size_t)i0 * 48;
        for (int e0 = threadIdx.x; e0 < tot; e0 += PB_T * 8) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int e = e0 + u * PB_T;
                x[u] = e < tot ? src[e] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int e = e0 + u * PB_T;
                const int r = e / 48, c = e - r * 48;
                if (e < tot && c < NC3) sgf[c * SGS + r] = x[u];
            }
        }
    }
    __syncthreads();
    float f[NC * 3];
#pragma unroll
    for (int k = 0; k < NC * 3; k++) f[k] = live ? sgf[k * SGS + threadIdx.x] : 0.0f;
    __syncthreads();
    if (live) {
#pragma unroll
        for (int k = 0; k < 3; k++) { mu[k] = sc.means[3 * i + k]; s[k] = sc.scales[3 * i + k]; }
        float4 qq = reinterpret_cast<const float4*>(sc.quats)[i];
        qlen = sqrtf(qq.x * qq.x + qq.y * qq.y + qq.z * qq.z + qq.w * qq.w);
        float il = 1.0f / qlen;
        qn[0] = qq.x * il; qn[1] = qq.y * il; qn[2] = qq.z * il; qn[3] = qq.w * il;
    }
    // rotation, M = R diag(s), Sigma = M M^T (value path)
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    float R[9];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
    float M[9], Sig[9];
#pragma unroll
    for (int j = 0; j < 3; j++)
#pragma unroll
        for (int k = 0; k < 3; k++) M[j * 3 + k] = R[j * 3 + k] * s[k];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) Sig[a * 3 + b] = M[a * 3 + 0] * M[b * 3 + 0] + M[a * 3 + 1] * M[b * 3 + 1] + M[a * 3 + 2] * M[b * 3 + 2];

    float gmu[3] = {0, 0, 0}, gSig[9];
#pragma unroll
    for (int k = 0; k < 9; k++) gSig[k] = 0.0f;
    float gop = 0.0f;
#pragma unroll
    for (int k = 0; k < NC * 3; k++) sgf[k * SGS + threadIdx.x] = 0.0f;

    // The 2D gradients are zero for every culled (view, Gaussian) pair (the
    // records are zero before the backward blend), so they are read without
    // consulting the tile rectangle, PB_STAGES - 1 views ahead of their use;
    // each record is cleared once read, which restores that state.
    const int tid = threadIdx.x;
    auto stage_view = [&](int vv) {
        if (live && vv < n_views) {
            const size_t k = (size_t)vv * sc.n + i;
            const int st = (vv % PB_STAGES) * PB_T + tid;
            cp_async16(stA + st, g2d.gA + k);
            cp_async16(stB + st, g2d.gB + k);
            cp_async4(stC + st, g2d.gC + k);
        }
        cp_async_commit();   // one group per view, empty past the last view
    };
#pragma unroll
    for (int vv = 0; vv < PB_STAGES - 1; vv++) stage_view(vv);
    for (int v = 0; v < n_views; v++) {
        const ViewDev& vd = sv[v];
        float pr[6] = {0, 0, 0, 0, 0, 0};
        cp_async_wait<PB_STAGES - 2>();   // view v's group has landed
        float4 a4 = make_float4(0, 0, 0, 0), b4 = make_float4(0, 0, 0, 0);
        float c1 = 0.0f;
        if (live) {
            const int st = (v % PB_STAGES) * PB_T + tid;
            a4 = stA[st]; b4 = stB[st]; c1 = stC[st];
        }
        // refill the stage consumed in the previous view
        stage_view(v + PB_STAGES - 1);
        const bool act = (a4.x != 0.f) | (a4.y != 0.f) | (a4.z != 0.f) | (a4.w != 0.f) | (b4.x != 0.f) |
                         (b4.y != 0.f) | (b4.z != 0.f) | (b4.w != 0.f) | (c1 != 0.f);
        if (act) {
            // consumed: cleared for the next backward blend, which accumulates into it
            const size_t k = (size_t)v * sc.n + i;
            g2d.gA[k] = make_float4(0, 0, 0, 0);
            g2d.gB[k] = make_float4(0, 0, 0, 0);
            g2d.gC[k] = 0.0f;
            const float* Rc = vd.Rf;
            const float fx = vd.fx, fy = vd.fy;
            float mc[3];
#pragma unroll
            for (int a = 0; a < 3; a++) mc[a] = Rc[a * 3 + 0] * mu[0] + Rc[a * 3 + 1] * mu[1] + Rc[a * 3 + 2] * mu[2] + vd.tf[a];
            float T1[9], Sc[9];
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) T1[a * 3 + b] = Rc[a * 3 + 0] * Sig[0 * 3 + b] + Rc[a * 3 + 1] * Sig[1 * 3 + b] + Rc[a * 3 + 2] * Sig[2 * 3 + b];
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) Sc[a * 3 + b] = T1[a * 3 + 0] * Rc[b * 3 + 0] + T1[a * 3 + 1] * Rc[b * 3 + 1] + T1[a * 3 + 2] * Rc[b * 3 + 2];
            const float zc = mc[2], iz = 1.0f / zc, iz2 = iz * iz;
            float ux = mc[0] * iz, uy = mc[1] * iz;
            bool clx = false, cly = false;
            if (rp.clamp_factor > 0.0f) {
                if (ux < -vd.limx) { ux = -vd.limx; clx = true; } else if (ux > vd.limx) { ux = vd.limx; clx = true; }
                if (uy < -vd.limy) { uy = -vd.limy; cly = true; } else if (uy > vd.limy) { uy = vd.limy; cly = true; }
            }
            const float J00 = fx * iz, J02 = -fx * ux * iz, J11 = fy * iz, J12 = -fy * uy * iz;
            // Sigma_hat and its inverse (the conic)
            float JS0[3], JS1[3];
#pragma unroll
            for (int b = 0; b < 3; b++) { JS0[b] = J00 * Sc[0 * 3 + b] + J02 * Sc[2 * 3 + b]; JS1[b] = J11 * Sc[1 * 3 + b] + J12 * Sc[2 * 3 + b]; }
            const float A = JS0[0] * J00 + JS0[2] * J02 + rp.eps2d;
            const float B = JS0[1] * J11 + JS0[2] * J12;
            const float C = JS1[1] * J11 + JS1[2] * J12 + rp.eps2d;
            const float idet = 1.0f / (A * C - B * B);
            const float qa = C * idet, qb = -B * idet, qc = A * idet;
            // dL/dSigma_hat = -Q G_Q Q
            const float ga = a4.z, gb = 0.5f * a4.w, gc = b4.x;
            const float m00 = qa * ga + qb * gb, m01 = qa * gb + qb * gc, m10 = qb * ga + qc * gb, m11 = qb * gb + qc * gc;
            const float G00 = -(m00 * qa + m01 * qb), G01 = -(m00 * qb + m01 * qc), G11 = -(m10 * qb + m11 * qc);
            // dL/dSigma_c = J^T G J (3x3) ; dL/dJ = 2 G J Sigma_c
            const float Jm[6] = {J00, 0.0f, J02, 0.0f, J11, J12};
            float GSc[9];
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++)
                    GSc[a * 3 + b] = Jm[a] * (G00 * Jm[b] + G01 * Jm[3 + b]) + Jm[3 + a] * (G01 * Jm[b] + G11 * Jm[3 + b]);
            // rows of G J
            float GJ0[3], GJ1[3];
#pragma unroll
            for (int b = 0; b < 3; b++) { GJ0[b] = G00 * Jm[b] + G01 * Jm[3 + b]; GJ1[b] = G01 * Jm[b] + G11 * Jm[3 + b]; }
            float dJ00 = 0, dJ02 = 0, dJ11 = 0, dJ12 = 0;
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                dJ00 += GJ0[kk] * Sc[kk * 3 + 0];
                dJ02 += GJ0[kk] * Sc[kk * 3 + 2];
                dJ11 += GJ1[kk] * Sc[kk * 3 + 1];
                dJ12 += GJ1[kk] * Sc[kk * 3 + 2];
            }
            dJ00 *= 2.f; dJ02 *= 2.f; dJ11 *= 2.f; dJ12 *= 2.f;
            float gmc[3];
            gmc[0] = a4.x * fx * iz;
            gmc[1] = a4.y * fy * iz;
            gmc[2] = -(a4.x * fx * mc[0] + a4.y * fy * mc[1]) * iz2;
            gmc[2] += -(dJ00 * fx + dJ11 * fy) * iz2;
            if (!clx) { gmc[0] += -dJ02 * fx * iz2; gmc[2] += dJ02 * 2.0f * fx * mc[0] * iz2 * iz; }
            else { gmc[2] += dJ02 * fx * ux * iz2; }
            if (!cly) { gmc[1] += -dJ12 * fy * iz2; gmc[2] += dJ12 * 2.0f * fy * mc[1] * iz2 * iz; }
            else { gmc[2] += dJ12 * fy * uy * iz2; }
            // dL/dSigma (world) += R_c^T GSc R_c
            float T2[9];
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) T2[a * 3 + b] = Rc[0 * 3 + a] * GSc[0 * 3 + b] + Rc[1 * 3 + a] * GSc[1 * 3 + b] + Rc[2 * 3 + a] * GSc[2 * 3 + b];
            if constexpr (!POSE_ONLY) {
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++) gSig[a * 3 + b] += T2[a * 3 + 0] * Rc[0 * 3 + b] + T2[a * 3 + 1] * Rc[1 * 3 + b] + T2[a * 3 + 2] * Rc[2 * 3 + b];
                gop += b4.y;  // opacity
            }
            // SH colour
            float dx = mu[0] - vd.oc[0], dy = mu[1] - vd.oc[1], dz = mu[2] - vd.oc[2];
            const float vl = sqrtf(dx * dx + dy * dy + dz * dz), ivl = 1.0f / vl;
            dx *= ivl; dy *= ivl; dz *= ivl;
            float Y[16];
            sh_basis<D>(dx, dy, dz, Y);
            const float gcol[3] = {b4.z, b4.w, c1};
            float wsum[16];
#pragma unroll
            for (int b = 0; b < 16; b++) wsum[b] = 0.0f;
#pragma unroll
            for (int ch = 0; ch < 3; ch++) {
                float raw = 0.5f;
#pragma unroll
                for (int b = 0; b < NC; b++) raw = fmaf(f[b * 3 + ch], Y[b], raw);
                const float gch = raw < 0.0f ? 0.0f : gcol[ch];
#pragma unroll
                for (int b = 0; b < NC; b++) {
                    if constexpr (!POSE_ONLY) sgf[(b * 3 + ch) * SGS + threadIdx.x] += Y[b] * gch;
                    wsum[b] += f[b * 3 + ch] * gch;
                }
            }
            float gd[3];
            sh_grad<D>(dx, dy, dz, wsum, gd);
            const float dd = gd[0] * dx + gd[1] * dy + gd[2] * dz;
            const float gsh0 = (gd[0] - dx * dd) * ivl, gsh1 = (gd[1] - dy * dd) * ivl, gsh2 = (gd[2] - dz * dd) * ivl;
#pragma unroll
            for (int a = 0; a < 3; a++)
                gmu[a] += Rc[0 * 3 + a] * gmc[0] + Rc[1 * 3 + a] * gmc[1] + Rc[2 * 3 + a] * gmc[2];
            gmu[0] += gsh0; gmu[1] += gsh1; gmu[2] += gsh2;
            // pose (left perturbation)
            float Am[9];
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) Am[a * 3 + b] = Sc[a * 3 + 0] * GSc[0 * 3 + b] + Sc[a * 3 + 1] * GSc[1 * 3 + b] + Sc[a * 3 + 2] * GSc[2 * 3 + b];
            pr[0] = gmc[0] + Rc[0] * gsh0 + Rc[1] * gsh1 + Rc[2] * gsh2;
            pr[1] = gmc[1] + Rc[3] * gsh0 + Rc[4] * gsh1 + Rc[5] * gsh2;
            pr[2] = gmc[2] + Rc[6] * gsh0 + Rc[7] * gsh1 + Rc[8] * gsh2;
            pr[3] = mc[1] * gmc[2] - mc[2] * gmc[1] + 2.0f * (Am[5] - Am[7]);
            pr[4] = mc[2] * gmc[0] - mc[0] * gmc[2] + 2.0f * (Am[6] - Am[2]);
            pr[5] = mc[0] * gmc[1] - mc[1] * gmc[0] + 2.0f * (Am[1] - Am[3]);
        }
        // warp reduction of the pose contribution (skipped when no lane is active)
        if (__any_sync(0xffffffffu, act)) {
#pragma unroll
            for (int c = 0; c < 6; c++) {
                float t = pr[c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                pr[c] = t;
            }
            if (lane == 0) {
                double* dst = spose + ((size_t)warp * n_views + v) * 6;
#pragma unroll
                for (int c = 0; c < 6; c++) dst[c] += (double)pr[c];
            }
        }
    }
    cp_async_wait_all();
    if (live && !POSE_ONLY) {
        // Sigma = M M^T -> dL/dM = 2 gSig M  (gSig symmetric)
        float GM[9];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) GM[a * 3 + b] = 2.0f * (gSig[a * 3 + 0] * M[0 * 3 + b] + gSig[a * 3 + 1] * M[1 * 3 + b] + gSig[a * 3 + 2] * M[2 * 3 + b]);
        float gsc[3], GR[9];
#pragma unroll
        for (int kk = 0; kk < 3; kk++) {
            gsc[kk] = GM[0 * 3 + kk] * R[0 * 3 + kk] + GM[1 * 3 + kk] * R[1 * 3 + kk] + GM[2 * 3 + kk] * R[2 * 3 + kk];
#pragma unroll
            for (int j = 0; j < 3; j++) GR[j * 3 + kk] = GM[j * 3 + kk] * s[kk];
        }
        float gq[4];
        gq[0] = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
        gq[1] = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] - 2.f * x * GR[8]);
        gq[2] = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] - 2.f * y * GR[8]);
        gq[3] = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] + x * GR[6] + y * GR[7]);
        const float dq = gq[0] * qn[0] + gq[1] * qn[1] + gq[2] * qn[2] + gq[3] * qn[3];
        const float iq = 1.0f / qlen;
        // every old value is loaded before the first store, so the loads are in
        // flight together (the arrays may alias as far as the compiler knows)
        float om[3] = {0, 0, 0}, os[3] = {0, 0, 0}, oo = 0.0f;
        float4 o4 = make_float4(0, 0, 0, 0);
        float4* gqp = grads.quats ? reinterpret_cast<float4*>(grads.quats) + i : nullptr;
        if (grads.means) { om[0] = grads.means[3 * i]; om[1] = grads.means[3 * i + 1]; om[2] = grads.means[3 * i + 2]; }
        if (grads.scales) { os[0] = grads.scales[3 * i]; os[1] = grads.scales[3 * i + 1]; os[2] = grads.scales[3 * i + 2]; }
        if (gqp) o4 = *gqp;
        if (grads.opacities) oo = grads.opacities[i];
        if (grads.means) {
#pragma unroll
            for (int a = 0; a < 3; a++) grads.means[3 * i + a] = om[a] + gmu[a];
        }
        if (grads.scales) {
#pragma unroll
            for (int a = 0; a < 3; a++) grads.scales[3 * i + a] = os[a] + gsc[a];
        }
        if (gqp) {
            o4.x += (gq[0] - qn[0] * dq) * iq; o4.y += (gq[1] - qn[1] * dq) * iq;
            o4.z += (gq[2] - qn[2] * dq) * iq; o4.w += (gq[3] - qn[3] * dq) * iq;
            *gqp = o4;
        }
        if (grads.opacities) grads.opacities[i] = oo + gop;
    }
    __syncthreads();
    if (!POSE_ONLY && grads.sh) {
        // SH gradients added row-major (coalesced) from the accumulators
        const int tot = m_blk * 48;
        float* dst = grads.sh + (size_t)i0 * 48;
        for (int e0 = threadIdx.x; e0 < tot; e0 += PB_T * 8) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int e = e0 + u * PB_T;
                const int c = e % 48;
                x[u] = (e < tot && c < NC3) ? dst[e] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int e = e0 + u * PB_T;
                const int r = e / 48, c = e - r * 48;
                if (e < tot && c < NC3) dst[e] = x[u] + sgf[c * SGS + r];
            }
        }
    }
    // block partial of every view's pose gradient, warps summed in order
    for (int t = threadIdx.x; t < n_views * 6; t += blockDim.x) {
        double acc = 0.0;
        for (int wi = 0; wi < nwarps; wi++) acc += spose[(size_t)wi * n_views * 6 + t];
        pose_partials[((size_t)(i_begin / blockDim.x) + blockIdx.x) * n_views * 6 + t] = acc;
    }
}

int preprocess_bwd_blocks(int n) { return (n + PB_T - 1) / PB_T; }

void launch_preprocess_bwd(const SceneDev& sc, int n_views, const ViewDev* views, const RenderParams& rp,
                           SplatArrays sp, Grad2DArrays g2d, gs_grads grads, double* pose_partials, int n_blocks,
                           cudaStream_t s, int i_begin, int i_end) {
    const int T = PB_T;
    if (i_end < 0 || i_end > sc.n) i_end = sc.n;
    if (i_begin < 0) i_begin = 0;
    i_begin -= i_begin % T;  // block-aligned
    if (i_end <= i_begin || n_views <= 0) return;
    n_blocks = std::min(n_blocks, (i_end - i_begin + T - 1) / T);
    const int nc3 = 3 * (sc.sh_degree + 1) * (sc.sh_degree + 1);
    const size_t sm = ((sizeof(ViewDev) * n_views + 15) & ~(size_t)15) + sizeof(double) * (T / 32) * n_views * 6 +
                      sizeof(float) * nc3 * (T + 1) + 16 + (size_t)PB_STAGES * T * (16 + 16 + 4);
    static std::atomic<unsigned long long> attr{0};
    once_per_device(attr, [](int) {
        const int mx = 200 * 1024;
        cudaFuncSetAttribute(k_preprocess_bwd<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_bwd<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_bwd<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_bwd<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_bwd<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_bwd<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_bwd<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_preprocess_bwd<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    });
    const bool po = !grads.means && !grads.scales && !grads.quats && !grads.opacities && !grads.sh;
#define GS_PRE_BWD(D)                                                                                          \
    if (po)                                                                                                    \
        k_preprocess_bwd<D, true><<<n_blocks, T, sm, s>>>(sc, i_begin, i_end, n_views, views, rp, sp, g2d, grads, \
                                                          pose_partials);                                      \
    else                                                                                                       \
        k_preprocess_bwd<D, false><<<n_blocks, T, sm, s>>>(sc, i_begin, i_end, n_views, views, rp, sp, g2d, grads, \
                                                           pose_partials)
    switch (sc.sh_degree) {
        case 0: GS_PRE_BWD(0); break;
        case 1: GS_PRE_BWD(1); break;
        case 2: GS_PRE_BWD(2); break;
        default: GS_PRE_BWD(3); break;
    }
#undef GS_PRE_BWD
}

// Deterministic sum of the block partials in two passes (FP64 runs at a small
// fraction of the FP32 rate on this GPU, so the sum is spread over many SMs
// instead of one block per view): pass 1, block (g, v) sums the partials of
// blocks [g PRD_CHUNK, (g + 1) PRD_CHUNK) of view v (thread-strided, then a
// butterfly over the warp, then the warps in order) into scratch[v][g]; pass
// 2, one warp per view sums scratch[v][0 .. G) the same way.  The split and
// every order are fixed, so the result is bit-reproducible.
#define PRD_T 128
#define PRD_CHUNK 256

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);   // a + b = b + a: all lanes agree
    return x;
}

__global__ void __launch_bounds__(PRD_T) k_pose_reduce_part(int n_views, int n_blocks,
                                                            const double* __restrict__ partials,
                                                            double* __restrict__ scratch) {
    __shared__ double sm[PRD_T / 32][6];
    const int g = blockIdx.x, v = blockIdx.y;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int b0 = g * PRD_CHUNK, b1 = min(n_blocks, b0 + PRD_CHUNK);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = b0 + threadIdx.x; b < b1; b += PRD_T) {
        const double* p = partials + ((size_t)b * n_views + v) * 6;
#pragma unroll
        for (int c = 0; c < 6; c++) acc[c] += p[c];
    }
#pragma unroll
    for (int c = 0; c < 6; c++) acc[c] = warp_sum_d(acc[c]);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 6; c++) sm[wid][c] = acc[c];
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = 0.0;
        for (int w = 0; w < PRD_T / 32; w++) t += sm[w][threadIdx.x];
        scratch[((size_t)v * gridDim.x + g) * 6 + threadIdx.x] = t;
    }
}

__global__ void k_pose_reduce_final(int n_groups, const double* __restrict__ scratch, double* __restrict__ out) {
    const int v = blockIdx.x, lane = threadIdx.x;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int g = lane; g < n_groups; g += 32) {
        const double* p = scratch + ((size_t)v * n_groups + g) * 6;
#pragma unroll
        for (int c = 0; c < 6; c++) acc[c] += p[c];
    }
    double r = 0.0;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const double t = warp_sum_d(acc[c]);
        if (lane == c) r = t;
    }
    if (lane < 6) out[v * 6 + lane] = r;
}

int pose_reduce_groups(int n_blocks) { return (std::max(n_blocks, 1) + PRD_CHUNK - 1) / PRD_CHUNK; }

void launch_pose_reduce(int n_views, int n_blocks, const double* partials, double* scratch, double* pose_grad,
                        cudaStream_t s) {
    if (n_views <= 0) return;
    const int G = pose_reduce_groups(n_blocks);
    k_pose_reduce_part<<<dim3(G, n_views), PRD_T, 0, s>>>(n_views, n_blocks, partials, scratch);
    k_pose_reduce_final<<<n_views, 32, 0, s>>>(G, scratch, pose_grad);
}

}  // namespace gs
