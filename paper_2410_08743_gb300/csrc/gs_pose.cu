// gs_pose.cu - pose optimisation step (Sec. 3.2: T = Exp(tau), gradients on
// the tangent space; Sec. 4.1: the camera learning rate schedule is the
// caller's).  Adam keeps its moments in the tangent space of each view's
// current pose; the step is applied on the left, T <- Exp(delta) T, matching
// the left-perturbation pose gradient.  FP64 throughout (one thread per view).
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

__global__ void k_pose_adam(int n_views, double* __restrict__ poses, double* __restrict__ m, double* __restrict__ v,
                            const double* __restrict__ g, double lr, double b1, double b2, double eps, double c1,
                            double c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_views) return;
    double d[6];
    for (int k = 0; k < 6; k++) {
        const double gk = g[6 * i + k];
        const double mk = b1 * m[6 * i + k] + (1.0 - b1) * gk;
        const double vk = b2 * v[6 * i + k] + (1.0 - b2) * gk * gk;
        m[6 * i + k] = mk;
        v[6 * i + k] = vk;
        d[k] = -lr * (mk / c1) / (sqrt(vk / c2) + eps);
    }
    double E[9], te[3];
    se3_exp(d, E, te);
    double* P = poses + 12 * i;
    double R[9], t[3];
    for (int a = 0; a < 3; a++) {
        for (int b = 0; b < 3; b++) R[a * 3 + b] = E[a * 3 + 0] * P[0 * 3 + b] + E[a * 3 + 1] * P[1 * 3 + b] + E[a * 3 + 2] * P[2 * 3 + b];
        t[a] = E[a * 3 + 0] * P[9] + E[a * 3 + 1] * P[10] + E[a * 3 + 2] * P[11] + te[a];
    }
    for (int k = 0; k < 9; k++) P[k] = R[k];
    for (int k = 0; k < 3; k++) P[9 + k] = t[k];
}

void launch_pose_adam(int n_views, double* poses, double* m, double* v, const double* grad, double lr, double b1,
                      double b2, double eps, int step, cudaStream_t s) {
    if (n_views <= 0) return;
    const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    k_pose_adam<<<(n_views + 63) / 64, 64, 0, s>>>(n_views, poses, m, v, grad, lr, b1, b2, eps, c1, c2);
}

}  // namespace gs
