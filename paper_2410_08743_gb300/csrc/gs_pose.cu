// gs_pose.cu - pose optimisation step (Sec. 3.2: T = Exp(tau), gradients on
// the tangent space; Sec. 4.1: the camera learning rate schedule is the
// caller's).  Adam keeps its moments in the tangent space of each view's
// current pose; the SE(3) step is applied on the left, T <- Exp(delta) T,
// matching the left-perturbation pose gradient; the T x SO(3) step moves the
// camera centre and the rotation separately (Sec. 4.2).  FP64 throughout (a
// group of eight lanes per view).
#include <cuda_runtime.h>
#include <math.h>

#include "gs_internal.cuh"

namespace gs {

// SE(3) exponential of tau = (rho, phi): R = I + A K + B K^2 and t = V rho,
// V = I + B K + C K^2 with K = [phi]x, A = sin(th)/th, B = (1-cos(th))/th^2,
// C = (th - sin(th))/th^3, by their Taylor series for small th.
__device__ void se3_exp(const double tau[6], double E[9], double te[3]) {
    const double p0 = tau[3], p1 = tau[4], p2 = tau[5];
    const double th2 = p0 * p0 + p1 * p1 + p2 * p2;
    const double th = sqrt(th2);
    double A, B, Cc;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        Cc = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        double sn, cs;
        sincos(th, &sn, &cs);
        A = sn / th;
        B = (1.0 - cs) / th2;
        Cc = (th - sn) / (th2 * th);
    }
    const double K[9] = {0.0, -p2, p1, p2, 0.0, -p0, -p1, p0, 0.0};
    double K2[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) K2[i * 3 + j] = K[i * 3 + 0] * K[0 * 3 + j] + K[i * 3 + 1] * K[1 * 3 + j] + K[i * 3 + 2] * K[2 * 3 + j];
    double Vm[9];
    for (int k = 0; k < 9; k++) {
        const double I = (k % 4 == 0) ? 1.0 : 0.0;
        E[k] = I + A * K[k] + B * K2[k];
        Vm[k] = I + B * K[k] + Cc * K2[k];
    }
    for (int a = 0; a < 3; a++) te[a] = Vm[a * 3 + 0] * tau[0] + Vm[a * 3 + 1] * tau[1] + Vm[a * 3 + 2] * tau[2];
}

// One Adam step on one pose.  g is the left-SE(3) tangent gradient the
// backward produces.  param GS_POSE_SE3: moments on tau = (rho, phi), update
// T <- Exp(delta) T.  param GS_POSE_TXSO3 (Sec. 4.2 names T x SO(3) as the
// parametrisation without the SE(3) coupling of position and orientation):
// the camera centre o = -R^T t and the rotation are stepped separately,
// o <- o + d_o and R <- Exp(d_phi) R (a rotation about the centre), t = -R o.
// A step (d_o, d_phi) equals the left step (rho, phi) = (-R d_o, d_phi) to
// first order, so its gradient is (g_o, g_phi) = (-R^T g_rho, g_phi); the
// moments live in those coordinates.
//
// The step is taken by a group of POSE_LANES consecutive lanes per pose (GB300
// runs FP64 at a small fraction of the FP32 rate, so the length of the
// dependent FP64 chain sets the time): lane k < 6 of the group updates the
// moments of tangent component k and its step, lanes 6 and 7 the two bias
// corrections where they are per pose, and the group's first lane applies the
// step to the pose.  The operations per component are those of a one-thread
// step.  Every lane of the warp calls it (ok false: a lane group with no pose).
#define POSE_LANES 8

// Applies the tangent step d to pose P (first lane of the group).
__device__ void pose_apply(double* P, const double d[6], int param) {
    double E[9], te[3], R[9], t[3];
    if (param == GS_POSE_TXSO3) {
        double o[3];
        for (int a = 0; a < 3; a++)
            o[a] = -(P[0 * 3 + a] * P[9] + P[1 * 3 + a] * P[10] + P[2 * 3 + a] * P[11]) + d[a];
        const double rot[6] = {0.0, 0.0, 0.0, d[3], d[4], d[5]};
        se3_exp(rot, E, te);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) R[a * 3 + b] = E[a * 3 + 0] * P[0 * 3 + b] + E[a * 3 + 1] * P[1 * 3 + b] + E[a * 3 + 2] * P[2 * 3 + b];
        for (int a = 0; a < 3; a++) t[a] = -(R[a * 3 + 0] * o[0] + R[a * 3 + 1] * o[1] + R[a * 3 + 2] * o[2]);
    } else {
        se3_exp(d, E, te);
        for (int a = 0; a < 3; a++) {
            for (int b = 0; b < 3; b++) R[a * 3 + b] = E[a * 3 + 0] * P[0 * 3 + b] + E[a * 3 + 1] * P[1 * 3 + b] + E[a * 3 + 2] * P[2 * 3 + b];
            t[a] = E[a * 3 + 0] * P[9] + E[a * 3 + 1] * P[10] + E[a * 3 + 2] * P[11] + te[a];
        }
    }
    for (int k = 0; k < 9; k++) P[k] = R[k];
    for (int k = 0; k < 3; k++) P[9 + k] = t[k];
}

// step > 0: bias corrections 1 - b^step computed in the group (lanes 6, 7);
// step <= 0: c1, c2 as given.
__device__ void pose_adam_group(bool ok, double* P, double* m, double* v, const double* g_in, double lr, double b1,
                                double b2, double eps, double c1, double c2, int step, int param) {
    const int k = threadIdx.x & (POSE_LANES - 1);
    if (step > 0) {
        double c = 0.0;
        if (k == 6) c = 1.0 - pow(b1, (double)step);
        if (k == 7) c = 1.0 - pow(b2, (double)step);
        c1 = __shfl_sync(0xffffffffu, c, 6, POSE_LANES);
        c2 = __shfl_sync(0xffffffffu, c, 7, POSE_LANES);
    }
    double dk = 0.0;
    if (ok && k < 6) {
        double gk = g_in[k];
        if (param == GS_POSE_TXSO3 && k < 3)
            gk = -(P[0 * 3 + k] * g_in[0] + P[1 * 3 + k] * g_in[1] + P[2 * 3 + k] * g_in[2]);
        const double mk = b1 * m[k] + (1.0 - b1) * gk;
        const double vk = b2 * v[k] + (1.0 - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        dk = -lr * (mk / c1) / (sqrt(vk / c2) + eps);
    }
    double d[6];
#pragma unroll
    for (int j = 0; j < 6; j++) d[j] = __shfl_sync(0xffffffffu, dk, j, POSE_LANES);
    if (ok && k == 0) pose_apply(P, d, param);
}

// POSE_LANES lanes per view (pose_adam_group)
__global__ void k_pose_adam(int n_views, double* __restrict__ poses, double* __restrict__ m, double* __restrict__ v,
                            const double* __restrict__ g, double lr, double b1, double b2, double eps, double c1,
                            double c2, int param) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) / POSE_LANES;
    const bool ok = i < n_views;
    const int j = ok ? i : 0;
    pose_adam_group(ok, poses + 12 * j, m + 6 * j, v + 6 * j, g + 6 * j, lr, b1, b2, eps, c1, c2, 0, param);
}

void launch_pose_adam(int n_views, double* poses, double* m, double* v, const double* grad, double lr, double b1,
                      double b2, double eps, int step, int param, cudaStream_t s) {
    if (n_views <= 0) return;
    const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    k_pose_adam<<<(n_views + 7) / 8, 8 * POSE_LANES, 0, s>>>(n_views, poses, m, v, grad, lr, b1, b2, eps, c1, c2,
                                                            param);
}

// Slot-indexed variants for a batch of independent solves whose state lives
// in fixed slots: view k of the batch is slot slot_of[k], with its own step
// count (1-based; <= 0 leaves the slot alone) and learning rate, as the solves
// started at different times.
__global__ void k_gather_poses(int n, const int* __restrict__ slot_of, const double* __restrict__ slot_poses,
                               double* __restrict__ packed) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * 12) return;
    packed[k] = slot_poses[(size_t)slot_of[k / 12] * 12 + k % 12];
}

__global__ void k_pose_adam_slots(int n, const int* __restrict__ slot_of, double* __restrict__ poses,
                                  double* __restrict__ m, double* __restrict__ v, const double* __restrict__ g,
                                  const int* __restrict__ steps, const double* __restrict__ lrs, double b1, double b2,
                                  double eps, int param) {
    const int kv = (blockIdx.x * blockDim.x + threadIdx.x) / POSE_LANES;
    const int k = kv < n ? kv : 0;
    const int i = slot_of[k];
    const int step = kv < n ? steps[k] : 0;
    pose_adam_group(step > 0, poses + 12 * (size_t)i, m + 6 * (size_t)i, v + 6 * (size_t)i, g + 6 * k, lrs[k], b1, b2,
                    eps, 1.0, 1.0, step > 0 ? step : 1, param);
}

void launch_gather_poses(int n, const int* slot_of, const double* slot_poses, double* packed, cudaStream_t s) {
    if (n <= 0) return;
    k_gather_poses<<<(n * 12 + 255) / 256, 256, 0, s>>>(n, slot_of, slot_poses, packed);
}

void launch_pose_adam_slots(int n, const int* slot_of, double* poses, double* m, double* v, const double* grad,
                            const int* steps, const double* lrs, double b1, double b2, double eps, int param,
                            cudaStream_t s) {
    if (n <= 0) return;
    k_pose_adam_slots<<<(n + 7) / 8, 8 * POSE_LANES, 0, s>>>(n, slot_of, poses, m, v, grad, steps, lrs, b1, b2, eps,
                                                            param);
}

// ------------------------------------------------------------ Gaussian Adam
// Adam on the raw Gaussian parameters of joint refinement (Sec. 3.3): means,
// log-scales, quaternions, logit-opacities and SH coefficients.  The renderer
// differentiates the activated scales s = exp(log s) and opacities
// o = sigmoid(logit o), so the update first chains ds/dlog s = s and
// do/dlogit = o (1 - o); it then writes the activated values the next render
// reads.  Element k of Gaussian i in a group of width w lives at i * w + k in
// both the parameter and moment arrays.  Blocks are assigned to groups in
// order (each group's elements padded to whole blocks), and a thread updates
// ADAM_UNR elements of its group a block-width apart, so its loads of all of
// them are in flight together.
#define ADAM_T 256
#define ADAM_UNR 4
struct AdamGroups {
    AdamGroup g[5];
    long long count_of[5];   // elements of each group (n * width)
    int blk_end[5];          // exclusive end of each group's block range (cumulative)
    int count;
};

__global__ void __launch_bounds__(ADAM_T) k_gaussian_adam(AdamGroups A, float b1, float b2, float eps, float ic1,
                                                          float ic2) {
    int gi = 0;
    while (gi + 1 < A.count && (int)blockIdx.x >= A.blk_end[gi]) gi++;
    const AdamGroup& G = A.g[gi];
    const long long cnt = A.count_of[gi];
    const long long base = (long long)(blockIdx.x - (gi ? A.blk_end[gi - 1] : 0)) * (ADAM_T * ADAM_UNR) + threadIdx.x;
    // the element's place in its Gaussian matters only for groups with unused
    // or separately scheduled trailing elements (the SH coefficients)
    const bool need_k = G.used < G.width || G.tail_from < G.width;
    float p[ADAM_UNR], g[ADAM_UNR], m[ADAM_UNR], v[ADAM_UNR];
#pragma unroll
    for (int u = 0; u < ADAM_UNR; u++) {
        const long long idx = base + u * ADAM_T;
        p[u] = g[u] = m[u] = v[u] = 0.0f;
        if (idx < cnt) {
            p[u] = G.p[idx];
            g[u] = G.g ? G.g[idx] : 0.0f;
            m[u] = G.m[idx];
            v[u] = G.v[idx];
        }
    }
    // k of the first element, then stepped by ADAM_T mod width
    int k = 0, dk = 0;
    if (need_k) {
        k = base < 0x7fffffffLL ? (int)((unsigned)base % (unsigned)G.width) : (int)(base % G.width);
        dk = ADAM_T % G.width;
    }
#pragma unroll
    for (int u = 0; u < ADAM_UNR; u++, k = (k + dk >= G.width) ? k + dk - G.width : k + dk) {
        const long long idx = base + u * ADAM_T;
        if (idx >= cnt) continue;
        if (k >= G.used) continue;
        float pu = p[u], gu = g[u];
        if (G.act_kind == 1) gu *= expf(pu);
        else if (G.act_kind == 2) { const float o = 1.0f / (1.0f + expf(-pu)); gu *= o * (1.0f - o); }
        const float mk = b1 * m[u] + (1.0f - b1) * gu;
        const float vk = b2 * v[u] + (1.0f - b2) * gu * gu;
        G.m[idx] = mk;
        G.v[idx] = vk;
        const float lr = k >= G.tail_from ? G.lr_tail : G.lr;
        pu -= lr * (mk * ic1) / (sqrtf(vk * ic2) + eps);
        G.p[idx] = pu;
        if (G.act) G.act[idx] = G.act_kind == 1 ? expf(pu) : 1.0f / (1.0f + expf(-pu));
    }
}

// All groups in one launch.
void launch_gaussian_adam(int64_t n, const AdamGroup* groups, int n_groups, float b1, float b2, float eps, int step,
                          cudaStream_t s) {
    if (n <= 0 || n_groups <= 0) return;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    AdamGroups A{};
    A.count = n_groups > 5 ? 5 : n_groups;
    long long blocks = 0;
    for (int k = 0; k < A.count; k++) {
        A.g[k] = groups[k];
        A.count_of[k] = n * groups[k].width;
        blocks += (A.count_of[k] + ADAM_T * ADAM_UNR - 1) / (ADAM_T * ADAM_UNR);
        A.blk_end[k] = (int)blocks;
    }
    if (blocks <= 0) return;
    k_gaussian_adam<<<(unsigned)blocks, ADAM_T, 0, s>>>(A, b1, b2, eps, 1.0f / c1, 1.0f / c2);
}

}  // namespace gs

