/*
 * gs_oracle.c - plain, slow FP64 CPU oracle of the pose-differentiable
 * Gaussian-splatting renderer ("Look Gauss, No Pose", Sec. 3.1-3.2).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the package's smoke check and the
 * benchmark's CPU-baseline leg call it; the CUDA product path never does, and
 * this file shares no code, header or constant table with it.
 *
 * What it computes, in the paper's order:
 *   Sec. 3.1 Eq. 1   Sigma = R(q) diag(s) diag(s)^T R(q)^T
 *   Sec. 3.1         mu_hat = pi(K T mu), pi(p) = (px/pz, py/pz)
 *   Sec. 3.1 Eq. 2   Sigma_hat = [J R_c Sigma R_c^T J^T]_2x2
 *   Sec. 3.1 Eq. 3   alpha = o exp(-1/2 d^T Sigma_hat^-1 d), d = p - mu_hat
 *   Sec. 3.1         c = SH(f, d_view), d_view = (mu - o_c)/|mu - o_c|, o_c = -R_c^T t_c
 *   Sec. 3.1 Eq. 4   C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j), depth order
 *   Sec. 3.2 Eq. 7   dL/dT = sum_i [mean term + covariance term (via J and via R_c)
 *                    + SH term], the tangent-space gradient of a left perturbation
 *                    Exp(tau) T (Eq. 5-6), with
 *                    Eq. 8/10  d mu_c / dT = (I | -[mu_c]x)
 *                    Eq. 12-13 d R_c / dT = ([e1]x R_c | [e2]x R_c | [e3]x R_c)
 *                    and the camera-centre term for the SH colour.
 *
 * Readings of points the paper leaves open:
 *   - Eq. 3 is printed without the inverse: read as d^T Sigma_hat^{-1} d.
 *   - Eq. 4's "transmittance" is read as T_i = prod_{j<i}(1 - alpha_j).
 *   - J of the perspective map with the prior-art frustum clamp of x/z, y/z to
 *     +-clamp_factor * W/(2 fx) (resp. H/(2 fy)); the clamped coordinate has zero
 *     derivative.  A low-pass dilation eps2d is added to Sigma_hat's diagonal.
 *   - Cull z <= z_near.  Screen support: radius r = ceil(3 sqrt(lambda_max)),
 *     tile rectangle of 16x16-pixel tiles; a pixel sees a Gaussian iff its tile
 *     lies in that rectangle.
 *   - Blending: alpha = min(alpha_max, o exp(power)); skip if power > 0 or
 *     alpha < alpha_min; with T_next = T (1 - alpha), stop before blending when
 *     T_next < t_min.  The clamped alpha has zero derivative.
 *   - Tile membership, culling and the depth key are FP32 functions with a
 *     fixed operation order (every op rounded to FP32, no contraction): this
 *     file must be compiled with -ffp-contract=off.  Ties in depth go to the
 *     lower Gaussian index.  The colour/geometry values used in blending and in
 *     the backward pass are FP64.
 *   - SH: real basis, degree <= 3, Condon-Shortley signs, colour =
 *     max(0, sum f Y + 0.5); the clamped channel has zero derivative.
 *   - Pose: left perturbation T <- Exp(tau) T, tau = (rho, phi), translation
 *     first; SE(3) Exp via Rodrigues and the V matrix.
 *
 * Fragility: wherever a discrete decision (alpha thresholds, the stop rule, the
 * sign of power) lies within a small margin of its threshold, FP32 and FP64
 * evaluations may legitimately differ; such pixels are flagged so that parity
 * tests compare only what is unique.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_TILE 16

/* ------------------------------------------------------------------ types */

typedef struct {
    int n;            /* number of Gaussians */
    int sh_degree;    /* 0..3 */
    const float* means;   /* [n][3] */
    const float* scales;  /* [n][3] activated */
    const float* quats;   /* [n][4] (w,x,y,z), normalised here */
    const float* opac;    /* [n] activated */
    const float* sh;      /* [n][16][3] */
} or_scene;

typedef struct {
    float fx, fy, cx, cy;
    int width, height;
    double pose[12];      /* world->camera: R row-major (9) then t (3) */
} or_cam;

typedef struct {
    double bg[3];
    float z_near;
    float eps2d;
    float clamp_factor;   /* 0 disables the frustum clamp in J */
    float alpha_min;
    float alpha_max;
    float t_min;
} or_opts;

/* Per-(view, Gaussian) results of the projection. */
typedef struct {
    int valid;            /* passes the FP32 key path (not culled) */
    float depth;          /* FP32 camera-space z: the depth key */
    float mu2f[2];        /* FP32 projected mean (key path) */
    int radius;
    int rect[4];          /* tiles [x0,x1) x [y0,y1) */
    /* FP64 value path */
    double qn[4], qlen;
    double R[9], M[9], Sig[9];
    double mc[3], Rc[9], Sc[9];
    double J[6];          /* row-major 2x3 */
    int clampx, clampy;
    double uxc, uyc;      /* clamped x/z, y/z */
    double Sh[3];         /* Sigma_hat entries A, B, C incl. eps2d */
    double conic[3];      /* inverse entries a, b, c */
    double mu2[2];
    double vdir[3], vlen, dir[3];
    double raw[3], col[3];
    int colclamp[3];
    double opac;          /* activated opacity */
    int fragile;          /* a Gaussian-level decision is near its threshold */
} or_splat;

/* ------------------------------------------------------------ utilities */

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void mat3_mul(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[i * 3 + k] * B[k * 3 + j];
            C[i * 3 + j] = s;
        }
}

static void mat3_mul_bt(const double* A, const double* B, double* C) { /* A B^T */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[i * 3 + k] * B[j * 3 + k];
            C[i * 3 + j] = s;
        }
}

static void mat3_mul_at(const double* A, const double* B, double* C) { /* A^T B */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[k * 3 + i] * B[k * 3 + j];
            C[i * 3 + j] = s;
        }
}

static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static int tiles_x(const or_cam* c) { return (c->width + OR_TILE - 1) / OR_TILE; }
static int tiles_y(const or_cam* c) { return (c->height + OR_TILE - 1) / OR_TILE; }

/* ------------------------------------------------- real spherical harmonics
 * Orthonormal real SH on the unit sphere, degree <= 3, ordered l = 0..3,
 * m = -l..l, with the Condon-Shortley phase.  The normalisation constants are
 * computed from their definitions sqrt(k / pi).                              */

static double SHK[16];
static int sh_ready = 0;

static void sh_init(void) {
    if (sh_ready) return;
    const double pi = 3.14159265358979323846;
    SHK[0] = sqrt(1.0 / (4.0 * pi));
    SHK[1] = -sqrt(3.0 / (4.0 * pi));   /* y */
    SHK[2] = sqrt(3.0 / (4.0 * pi));    /* z */
    SHK[3] = -sqrt(3.0 / (4.0 * pi));   /* x */
    SHK[4] = sqrt(15.0 / (4.0 * pi));   /* xy */
    SHK[5] = -sqrt(15.0 / (4.0 * pi));  /* yz */
    SHK[6] = sqrt(5.0 / (16.0 * pi));   /* 2zz - xx - yy */
    SHK[7] = -sqrt(15.0 / (4.0 * pi));  /* xz */
    SHK[8] = sqrt(15.0 / (16.0 * pi));  /* xx - yy */
    SHK[9] = -sqrt(35.0 / (32.0 * pi)); /* y (3xx - yy) */
    SHK[10] = sqrt(105.0 / (4.0 * pi)); /* xyz */
    SHK[11] = -sqrt(21.0 / (32.0 * pi));/* y (4zz - xx - yy) */
    SHK[12] = sqrt(7.0 / (16.0 * pi));  /* z (2zz - 3xx - 3yy) */
    SHK[13] = -sqrt(21.0 / (32.0 * pi));/* x (4zz - xx - yy) */
    SHK[14] = sqrt(105.0 / (16.0 * pi));/* z (xx - yy) */
    SHK[15] = -sqrt(35.0 / (32.0 * pi));/* x (xx - 3yy) */
    sh_ready = 1;
}

/* Basis values Y[k] and their gradients dY[k][3] w.r.t. the (x, y, z)
 * components, treated as independent variables. */
static void sh_basis(const double* d, int deg, double* Y, double (*dY)[3]) {
    const double x = d[0], y = d[1], z = d[2];
    const double xx = x * x, yy = y * y, zz = z * z;
    int nb = (deg + 1) * (deg + 1);
    for (int k = 0; k < 16; k++) { Y[k] = 0.0; if (dY) dY[k][0] = dY[k][1] = dY[k][2] = 0.0; }
    Y[0] = SHK[0];
    if (nb > 1) {
        Y[1] = SHK[1] * y; Y[2] = SHK[2] * z; Y[3] = SHK[3] * x;
        if (dY) { dY[1][1] = SHK[1]; dY[2][2] = SHK[2]; dY[3][0] = SHK[3]; }
    }
    if (nb > 4) {
        Y[4] = SHK[4] * x * y;
        Y[5] = SHK[5] * y * z;
        Y[6] = SHK[6] * (2.0 * zz - xx - yy);
        Y[7] = SHK[7] * x * z;
        Y[8] = SHK[8] * (xx - yy);
        if (dY) {
            dY[4][0] = SHK[4] * y; dY[4][1] = SHK[4] * x;
            dY[5][1] = SHK[5] * z; dY[5][2] = SHK[5] * y;
            dY[6][0] = -2.0 * SHK[6] * x; dY[6][1] = -2.0 * SHK[6] * y; dY[6][2] = 4.0 * SHK[6] * z;
            dY[7][0] = SHK[7] * z; dY[7][2] = SHK[7] * x;
            dY[8][0] = 2.0 * SHK[8] * x; dY[8][1] = -2.0 * SHK[8] * y;
        }
    }
    if (nb > 9) {
        Y[9] = SHK[9] * y * (3.0 * xx - yy);
        Y[10] = SHK[10] * x * y * z;
        Y[11] = SHK[11] * y * (4.0 * zz - xx - yy);
        Y[12] = SHK[12] * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
        Y[13] = SHK[13] * x * (4.0 * zz - xx - yy);
        Y[14] = SHK[14] * z * (xx - yy);
        Y[15] = SHK[15] * x * (xx - 3.0 * yy);
        if (dY) {
            dY[9][0] = SHK[9] * 6.0 * x * y; dY[9][1] = SHK[9] * (3.0 * xx - 3.0 * yy);
            dY[10][0] = SHK[10] * y * z; dY[10][1] = SHK[10] * x * z; dY[10][2] = SHK[10] * x * y;
            dY[11][0] = SHK[11] * (-2.0 * x * y); dY[11][1] = SHK[11] * (4.0 * zz - xx - 3.0 * yy);
            dY[11][2] = SHK[11] * 8.0 * y * z;
            dY[12][0] = SHK[12] * (-6.0 * x * z); dY[12][1] = SHK[12] * (-6.0 * y * z);
            dY[12][2] = SHK[12] * (6.0 * zz - 3.0 * xx - 3.0 * yy);
            dY[13][0] = SHK[13] * (4.0 * zz - 3.0 * xx - yy); dY[13][1] = SHK[13] * (-2.0 * x * y);
            dY[13][2] = SHK[13] * 8.0 * x * z;
            dY[14][0] = SHK[14] * 2.0 * x * z; dY[14][1] = SHK[14] * (-2.0 * y * z);
            dY[14][2] = SHK[14] * (xx - yy);
            dY[15][0] = SHK[15] * (3.0 * xx - 3.0 * yy); dY[15][1] = SHK[15] * (-6.0 * x * y);
        }
    }
}

/* Exposed for the orthonormality pin. */
void or_sh_eval(const double* dirs, int n, int deg, double* out /*[n][16]*/) {
    sh_init();
    for (int i = 0; i < n; i++) sh_basis(dirs + 3 * i, deg, out + 16 * i, NULL);
}

/* ------------------------------------------------------- FP32 key path
 * Culling, the screen radius, the tile rectangle and the depth key as FP32
 * functions with a fixed operation order.  Each statement is one rounded FP32
 * operation; -ffp-contract=off keeps the compiler from fusing them.          */

static int keypath_f32(const float* mu, const float* sc, const float* q,
                       const double* pose, float fx, float fy, float cx, float cy,
                       int W, int H, const or_opts* o,
                       float* depth, float* mx_out, float* my_out, int* radius, int* rect) {
    /* quaternion normalisation */
    float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    float n2 = qw * qw; n2 = n2 + qx * qx; n2 = n2 + qy * qy; n2 = n2 + qz * qz;
    float inv = 1.0f / sqrtf(n2);
    float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
    /* rotation matrix of the unit quaternion */
    float R[9];
    { float a = y * y, b = z * z; float s = a + b; R[0] = 1.0f - 2.0f * s; }
    { float a = x * y, b = w * z; R[1] = 2.0f * (a - b); }
    { float a = x * z, b = w * y; R[2] = 2.0f * (a + b); }
    { float a = x * y, b = w * z; R[3] = 2.0f * (a + b); }
    { float a = x * x, b = z * z; float s = a + b; R[4] = 1.0f - 2.0f * s; }
    { float a = y * z, b = w * x; R[5] = 2.0f * (a - b); }
    { float a = x * z, b = w * y; R[6] = 2.0f * (a - b); }
    { float a = y * z, b = w * x; R[7] = 2.0f * (a + b); }
    { float a = x * x, b = y * y; float s = a + b; R[8] = 1.0f - 2.0f * s; }
    /* M = R diag(s); Sigma = M M^T (upper triangle) */
    float M[9];
    for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++) M[j * 3 + k] = R[j * 3 + k] * sc[k];
    float S[9];
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++) {
            float t0 = M[a * 3 + 0] * M[b * 3 + 0];
            float t1 = M[a * 3 + 1] * M[b * 3 + 1];
            float t2 = M[a * 3 + 2] * M[b * 3 + 2];
            float s = t0 + t1; s = s + t2;
            S[a * 3 + b] = s; S[b * 3 + a] = s;
        }
    /* camera (pose rounded to FP32) */
    float Rc[9], tc[3];
    for (int k = 0; k < 9; k++) Rc[k] = (float)pose[k];
    for (int k = 0; k < 3; k++) tc[k] = (float)pose[9 + k];
    float mc[3];
    for (int a = 0; a < 3; a++) {
        float t0 = Rc[a * 3 + 0] * mu[0];
        float t1 = Rc[a * 3 + 1] * mu[1];
        float t2 = Rc[a * 3 + 2] * mu[2];
        float s = t0 + t1; s = s + t2; s = s + tc[a];
        mc[a] = s;
    }
    float zc = mc[2];
    if (!(zc > o->z_near)) return 0;
    /* Sigma_c = Rc Sigma Rc^T: Tm = Rc Sigma, then Tm Rc^T (upper triangle) */
    float Tm[9];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            float t0 = Rc[a * 3 + 0] * S[0 * 3 + b];
            float t1 = Rc[a * 3 + 1] * S[1 * 3 + b];
            float t2 = Rc[a * 3 + 2] * S[2 * 3 + b];
            float s = t0 + t1; s = s + t2;
            Tm[a * 3 + b] = s;
        }
    float Sc[9];
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++) {
            float t0 = Tm[a * 3 + 0] * Rc[b * 3 + 0];
            float t1 = Tm[a * 3 + 1] * Rc[b * 3 + 1];
            float t2 = Tm[a * 3 + 2] * Rc[b * 3 + 2];
            float s = t0 + t1; s = s + t2;
            Sc[a * 3 + b] = s; Sc[b * 3 + a] = s;
        }
    /* Jacobian of the perspective map, with the frustum clamp */
    float txv = mc[0], tyv = mc[1];
    if (o->clamp_factor > 0.0f) {
        float twofx = 2.0f * fx, twofy = 2.0f * fy;
        float tanx = (float)W / twofx, tany = (float)H / twofy;
        float limx = o->clamp_factor * tanx, limy = o->clamp_factor * tany;
        float ux = mc[0] / zc, uy = mc[1] / zc;
        float nlx = -limx, nly = -limy;
        ux = ux < nlx ? nlx : ux; ux = ux > limx ? limx : ux;
        uy = uy < nly ? nly : uy; uy = uy > limy ? limy : uy;
        txv = ux * zc; tyv = uy * zc;
    }
    float zz = zc * zc;
    float j00 = fx / zc, j11 = fy / zc;
    float j02, j12;
    { float a = fx * txv; float b = a / zz; j02 = -b; }
    { float a = fy * tyv; float b = a / zz; j12 = -b; }
    /* U = J Sigma_c, then Sigma_hat = U J^T */
    float U00, U01, U02, U11, U12;
    { float a = j00 * Sc[0]; float b = j02 * Sc[6]; U00 = a + b; }
    { float a = j00 * Sc[1]; float b = j02 * Sc[7]; U01 = a + b; }
    { float a = j00 * Sc[2]; float b = j02 * Sc[8]; U02 = a + b; }
    { float a = j11 * Sc[4]; float b = j12 * Sc[7]; U11 = a + b; }
    { float a = j11 * Sc[5]; float b = j12 * Sc[8]; U12 = a + b; }
    float A, B, C;
    { float a = U00 * j00; float b = U02 * j02; A = a + b; }
    { float a = U01 * j11; float b = U02 * j12; B = a + b; }
    { float a = U11 * j11; float b = U12 * j12; C = a + b; }
    A = A + o->eps2d; C = C + o->eps2d;
    float det;
    { float a = A * C; float b = B * B; det = a - b; }
    if (!(det > 0.0f)) return 0;
    /* largest eigenvalue and the 3-sigma radius */
    float mid; { float a = A + C; mid = 0.5f * a; }
    float disc; { float a = mid * mid; disc = a - det; }
    if (!(disc > 0.1f)) disc = 0.1f;
    float lam; { float a = sqrtf(disc); lam = mid + a; }
    float rf; { float a = sqrtf(lam); float b = 3.0f * a; rf = ceilf(b); }
    /* projected mean */
    float mx, my;
    { float a = fx * mc[0]; float b = a / zc; mx = b + cx; }
    { float a = fy * mc[1]; float b = a / zc; my = b + cy; }
    /* tile rectangle */
    int gw = (W + OR_TILE - 1) / OR_TILE, gh = (H + OR_TILE - 1) / OR_TILE;
    const float invt = 1.0f / (float)OR_TILE;
    float rb = rf + (float)(OR_TILE - 1);
    float fx0, fy0, fx1, fy1;
    { float a = mx - rf; fx0 = floorf(a * invt); }
    { float a = my - rf; fy0 = floorf(a * invt); }
    { float a = mx + rb; fx1 = floorf(a * invt); }
    { float a = my + rb; fy1 = floorf(a * invt); }
    float gwf = (float)gw, ghf = (float)gh;
    if (!(fx0 >= 0.0f)) fx0 = 0.0f; if (fx0 > gwf) fx0 = gwf;
    if (!(fy0 >= 0.0f)) fy0 = 0.0f; if (fy0 > ghf) fy0 = ghf;
    if (!(fx1 >= 0.0f)) fx1 = 0.0f; if (fx1 > gwf) fx1 = gwf;
    if (!(fy1 >= 0.0f)) fy1 = 0.0f; if (fy1 > ghf) fy1 = ghf;
    rect[0] = (int)fx0; rect[1] = (int)fy0; rect[2] = (int)fx1; rect[3] = (int)fy1;
    if (rect[2] <= rect[0] || rect[3] <= rect[1]) return 0;
    *depth = zc; *mx_out = mx; *my_out = my;
    *radius = (int)rf;
    return 1;
}

/* --------------------------------------------------------- FP64 value path */

static void camera_center(const double* pose, double* oc) {
    /* o_c = -R_c^T t_c (Sec. 3.1) */
    for (int a = 0; a < 3; a++)
        oc[a] = -(pose[0 * 3 + a] * pose[9] + pose[1 * 3 + a] * pose[10] + pose[2 * 3 + a] * pose[11]);
}

static void value_path(const or_scene* s, int i, const or_cam* cam, const double* oc,
                       const or_opts* o, or_splat* g) {
    const float* q = s->quats + 4 * i;
    double qq[4] = {q[0], q[1], q[2], q[3]};
    double len = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
    g->qlen = len;
    g->opac = (double)s->opac[i];
    for (int k = 0; k < 4; k++) g->qn[k] = qq[k] / len;
    double w = g->qn[0], x = g->qn[1], y = g->qn[2], z = g->qn[3];
    double* R = g->R;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
    const float* sc = s->scales + 3 * i;
    for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++) g->M[j * 3 + k] = R[j * 3 + k] * (double)sc[k];
    mat3_mul_bt(g->M, g->M, g->Sig);                       /* Eq. 1 */
    for (int k = 0; k < 9; k++) g->Rc[k] = cam->pose[k];
    const float* mu = s->means + 3 * i;
    for (int a = 0; a < 3; a++)
        g->mc[a] = g->Rc[a * 3 + 0] * mu[0] + g->Rc[a * 3 + 1] * mu[1] + g->Rc[a * 3 + 2] * mu[2]
                   + cam->pose[9 + a];
    double T1[9];
    mat3_mul(g->Rc, g->Sig, T1);
    mat3_mul_bt(T1, g->Rc, g->Sc);                         /* R_c Sigma R_c^T */
    const double fx = cam->fx, fy = cam->fy;
    const double zc = g->mc[2];
    double ux = g->mc[0] / zc, uy = g->mc[1] / zc;
    g->clampx = g->clampy = 0;
    if (o->clamp_factor > 0.0f) {
        double limx = (double)o->clamp_factor * (double)cam->width / (2.0 * fx);
        double limy = (double)o->clamp_factor * (double)cam->height / (2.0 * fy);
        if (fabs(fabs(ux) - limx) < 1e-6 * limx) g->fragile = 1;
        if (fabs(fabs(uy) - limy) < 1e-6 * limy) g->fragile = 1;
        if (ux < -limx) { ux = -limx; g->clampx = 1; } else if (ux > limx) { ux = limx; g->clampx = 1; }
        if (uy < -limy) { uy = -limy; g->clampy = 1; } else if (uy > limy) { uy = limy; g->clampy = 1; }
    }
    g->uxc = ux; g->uyc = uy;
    /* J = d pi / d mu_c at mu_c, with the clamped lateral coordinates */
    g->J[0] = fx / zc; g->J[1] = 0.0; g->J[2] = -fx * ux / zc;
    g->J[3] = 0.0; g->J[4] = fy / zc; g->J[5] = -fy * uy / zc;
    /* Sigma_hat = [J Sigma_c J^T]_2x2 + eps2d I (Eq. 2) */
    double JS[6];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 3; b++) {
            double t = 0.0;
            for (int k = 0; k < 3; k++) t += g->J[a * 3 + k] * g->Sc[k * 3 + b];
            JS[a * 3 + b] = t;
        }
    double S00 = 0, S01 = 0, S11 = 0;
    for (int k = 0; k < 3; k++) {
        S00 += JS[0 * 3 + k] * g->J[0 * 3 + k];
        S01 += JS[0 * 3 + k] * g->J[1 * 3 + k];
        S11 += JS[1 * 3 + k] * g->J[1 * 3 + k];
    }
    g->Sh[0] = S00 + (double)o->eps2d; g->Sh[1] = S01; g->Sh[2] = S11 + (double)o->eps2d;
    double det = g->Sh[0] * g->Sh[2] - g->Sh[1] * g->Sh[1];
    g->conic[0] = g->Sh[2] / det; g->conic[1] = -g->Sh[1] / det; g->conic[2] = g->Sh[0] / det;
    /* mu_hat = pi(K T mu) */
    g->mu2[0] = fx * g->mc[0] / zc + (double)cam->cx;
    g->mu2[1] = fy * g->mc[1] / zc + (double)cam->cy;
    /* view-dependent colour */
    double v[3] = {mu[0] - oc[0], mu[1] - oc[1], mu[2] - oc[2]};
    double vl = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int a = 0; a < 3; a++) { g->vdir[a] = v[a]; g->dir[a] = v[a] / vl; }
    g->vlen = vl;
    double Y[16];
    sh_basis(g->dir, s->sh_degree, Y, NULL);
    int nb = (s->sh_degree + 1) * (s->sh_degree + 1);
    const float* f = s->sh + 48 * (size_t)i;
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.0, mag = 0.5;
        for (int k = 0; k < nb; k++) { acc += (double)f[k * 3 + ch] * Y[k]; mag += fabs((double)f[k * 3 + ch] * Y[k]); }
        double r = acc + 0.5;
        g->raw[ch] = r;
        if (fabs(r) < 1e-6 * mag) g->fragile = 1;
        g->colclamp[ch] = r < 0.0;
        g->col[ch] = r < 0.0 ? 0.0 : r;
    }
}

static void project_all(const or_scene* s, int V, const or_cam* cams, const or_opts* o, or_splat* out) {
    sh_init();
    for (int v = 0; v < V; v++) {
        double oc[3];
        camera_center(cams[v].pose, oc);
        #pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int i = 0; i < s->n; i++) {
            or_splat* g = out + (size_t)v * s->n + i;
            memset(g, 0, sizeof(*g));
            const or_cam* c = cams + v;
            g->valid = keypath_f32(s->means + 3 * i, s->scales + 3 * i, s->quats + 4 * i, c->pose,
                                   c->fx, c->fy, c->cx, c->cy, c->width, c->height, o,
                                   &g->depth, &g->mu2f[0], &g->mu2f[1], &g->radius, g->rect);
            if (g->valid) value_path(s, i, c, oc, o, g);
        }
    }
}

/* ----------------------------------------------------------- tile lists */

typedef struct { uint64_t key; uint32_t idx; } or_kv;

static int kv_cmp(const void* a, const void* b) {
    const or_kv* x = (const or_kv*)a; const or_kv* y = (const or_kv*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

static uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

typedef struct {
    int64_t n_keys;
    int total_tiles;
    int* tile_base;       /* [V+1] global tile id of each view's first tile */
    uint32_t* ranges;     /* [total_tiles][2] */
    uint32_t* idx;        /* [n_keys] Gaussian index in sorted order */
} or_lists;

/* Keys (global tile << 32 | depth bits) with value = Gaussian index, sorted
 * by key then index: a library sort as one step. */
static void build_lists(const or_scene* s, int V, const or_cam* cams, const or_splat* sp, or_lists* L) {
    L->tile_base = (int*)malloc(sizeof(int) * (V + 1));
    L->tile_base[0] = 0;
    for (int v = 0; v < V; v++) L->tile_base[v + 1] = L->tile_base[v] + tiles_x(cams + v) * tiles_y(cams + v);
    L->total_tiles = L->tile_base[V];
    int64_t K = 0;
    for (int v = 0; v < V; v++)
        for (int i = 0; i < s->n; i++) {
            const or_splat* g = sp + (size_t)v * s->n + i;
            if (g->valid) K += (int64_t)(g->rect[2] - g->rect[0]) * (g->rect[3] - g->rect[1]);
        }
    or_kv* kv = (or_kv*)malloc(sizeof(or_kv) * (K > 0 ? K : 1));
    int64_t p = 0;
    for (int v = 0; v < V; v++) {
        int gw = tiles_x(cams + v);
        for (int i = 0; i < s->n; i++) {
            const or_splat* g = sp + (size_t)v * s->n + i;
            if (!g->valid) continue;
            for (int ty = g->rect[1]; ty < g->rect[3]; ty++)
                for (int tx = g->rect[0]; tx < g->rect[2]; tx++) {
                    uint64_t tile = (uint64_t)(L->tile_base[v] + ty * gw + tx);
                    kv[p].key = (tile << 32) | fbits(g->depth);
                    kv[p].idx = (uint32_t)i;
                    p++;
                }
        }
    }
    qsort(kv, (size_t)K, sizeof(or_kv), kv_cmp);
    L->n_keys = K;
    L->ranges = (uint32_t*)calloc((size_t)L->total_tiles * 2 + 2, sizeof(uint32_t));
    L->idx = (uint32_t*)malloc(sizeof(uint32_t) * (K > 0 ? K : 1));
    for (int64_t k = 0; k < K; k++) {
        L->idx[k] = kv[k].idx;
        uint32_t t = (uint32_t)(kv[k].key >> 32);
        if (k == 0 || (uint32_t)(kv[k - 1].key >> 32) != t) L->ranges[2 * t] = (uint32_t)k;
        if (k == K - 1 || (uint32_t)(kv[k + 1].key >> 32) != t) L->ranges[2 * t + 1] = (uint32_t)k + 1;
    }
    free(kv);
}

static void free_lists(or_lists* L) { free(L->tile_base); free(L->ranges); free(L->idx); }

/* ------------------------------------------------------------- blending */

typedef struct {
    int j;               /* Gaussian index */
    double alpha, G, T;  /* alpha, exp(power), transmittance before blending */
    double d[2];         /* p - mu_hat */
    int clamped;         /* o exp(power) exceeded alpha_max */
} or_rec;

/* Front-to-back compositing of one pixel over a depth-ordered candidate list
 * (Eq. 3-4).  When use_rect_filter is set the candidate list is the whole view
 * and a Gaussian is used only if the pixel's tile lies in its rectangle (the
 * brute-force mode).  Records the blended entries when recs != NULL.  Returns
 * 1 + the list position of the last blended entry (0 if none), sets *nb to the
 * number of blended entries and *fragile when a decision is near a threshold. */
static int blend_pixel(const or_splat* sp, const uint32_t* list, int n, int px, int py,
                       int tx, int ty, int use_rect_filter, const or_opts* o,
                       double* C, double* Tout, or_rec* recs, int* nb, int* fragile) {
    double T = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    int last = 0, cnt = 0;
    const double amin = (double)o->alpha_min, amax = (double)o->alpha_max, tmin = (double)o->t_min;
    for (int k = 0; k < n; k++) {
        const or_splat* g = sp + list[k];
        if (use_rect_filter &&
            !(tx >= g->rect[0] && tx < g->rect[2] && ty >= g->rect[1] && ty < g->rect[3]))
            continue;
        /* Eq. 3: power = -1/2 d^T Sigma_hat^{-1} d, d = p - mu_hat */
        double dx = (double)px - g->mu2[0], dy = (double)py - g->mu2[1];
        double pa = g->conic[0] * dx * dx, pc = g->conic[2] * dy * dy, pb = g->conic[1] * dx * dy;
        double power = -0.5 * (pa + pc) - pb;
        double scale = 0.5 * (fabs(pa) + fabs(pc)) + fabs(pb);
        if (fabs(power) <= 1e-5 * scale + 1e-9) *fragile = 1;
        if (power > 0.0) continue;
        double G = exp(power);
        double ar = g->opac * G;
        double margin = 2e-5 + 5e-6 * scale;
        if (fabs(ar - amin) <= margin * amin) *fragile = 1;
        if (fabs(ar - amax) <= margin * amax) *fragile = 1;
        int clamped = ar > amax;
        double alpha = clamped ? amax : ar;
        if (alpha < amin) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - tmin) <= 5e-5 * tmin) *fragile = 1;
        if (Tn < tmin) break;
        if (recs) {
            recs[cnt].j = (int)list[k]; recs[cnt].alpha = alpha; recs[cnt].G = G; recs[cnt].T = T;
            recs[cnt].d[0] = dx; recs[cnt].d[1] = dy; recs[cnt].clamped = clamped;
        }
        /* Eq. 4 */
        for (int ch = 0; ch < 3; ch++) C[ch] += g->col[ch] * alpha * T;
        T = Tn;
        cnt++;
        last = k + 1;
    }
    for (int ch = 0; ch < 3; ch++) C[ch] += T * o->bg[ch];
    *Tout = T;
    *nb = cnt;
    return last;
}

/* Global depth order of one view (brute-force mode): all valid splats sorted
 * by (depth bits, index). */
static uint32_t* view_depth_order(const or_scene* s, const or_splat* spv, int* n_out) {
    or_kv* kv = (or_kv*)malloc(sizeof(or_kv) * (s->n > 0 ? s->n : 1));
    int m = 0;
    for (int i = 0; i < s->n; i++)
        if (spv[i].valid) { kv[m].key = fbits(spv[i].depth); kv[m].idx = (uint32_t)i; m++; }
    qsort(kv, (size_t)m, sizeof(or_kv), kv_cmp);
    uint32_t* ord = (uint32_t*)malloc(sizeof(uint32_t) * (m > 0 ? m : 1));
    for (int k = 0; k < m; k++) ord[k] = kv[k].idx;
    free(kv);
    *n_out = m;
    return ord;
}

static uint64_t fnv(uint64_t h, uint64_t x) {
    for (int b = 0; b < 8; b++) { h ^= (x >> (8 * b)) & 0xff; h *= 1099511628211ULL; }
    return h;
}

/* ------------------------------------------------------------- forward */

/* Render V views.  image: packed planar [3][H][W] per view (float64);
 * T_final, n_contrib, fragile_px: packed [H][W] per view (each nullable).
 * brute != 0 uses the brute-force order (no tiles).  hash_out (nullable)
 * receives a hash of every discrete decision: culling, rectangles, list order,
 * the blended set of every pixel, alpha and colour clamps. */
int or_render(const or_scene* s, int V, const or_cam* cams, const or_opts* o, int brute,
              double* image, double* T_final, int32_t* n_contrib, uint8_t* fragile_px,
              uint64_t* hash_out) {
    or_splat* sp = (or_splat*)malloc(sizeof(or_splat) * (size_t)V * (s->n > 0 ? s->n : 1));
    if (!sp) return -1;
    project_all(s, V, cams, o, sp);
    or_lists L;
    build_lists(s, V, cams, sp, &L);
    uint64_t h = 1469598103934665603ULL;
    size_t img_off = 0, pix_off = 0;
    for (int v = 0; v < V; v++) {
        const or_cam* c = cams + v;
        const or_splat* spv = sp + (size_t)v * s->n;
        int W = c->width, H = c->height, gw = tiles_x(c), gh = tiles_y(c);
        int nord = 0;
        uint32_t* ord = brute ? view_depth_order(s, spv, &nord) : NULL;
        uint64_t* th = (uint64_t*)calloc((size_t)gw * gh, sizeof(uint64_t));
        #pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
        for (int t = 0; t < gw * gh; t++) {
            int tx = t % gw, ty = t / gw;
            const uint32_t* list; int n;
            if (brute) { list = ord; n = nord; }
            else {
                uint32_t gt = (uint32_t)(L.tile_base[v] + t);
                list = L.idx + L.ranges[2 * gt]; n = (int)(L.ranges[2 * gt + 1] - L.ranges[2 * gt]);
            }
            or_rec* recs = (or_rec*)malloc(sizeof(or_rec) * (n > 0 ? n : 1));
            uint64_t hh = 1469598103934665603ULL;
            for (int py = ty * OR_TILE; py < (ty + 1) * OR_TILE && py < H; py++)
                for (int px = tx * OR_TILE; px < (tx + 1) * OR_TILE && px < W; px++) {
                    double C[3], T; int nb = 0, fr = 0;
                    int last = blend_pixel(spv, list, n, px, py, tx, ty, brute, o, C, &T, recs, &nb, &fr);
                    size_t p = (size_t)py * W + px;
                    for (int ch = 0; ch < 3; ch++) image[img_off + (size_t)ch * W * H + p] = C[ch];
                    if (T_final) T_final[pix_off + p] = T;
                    if (n_contrib) n_contrib[pix_off + p] = brute ? nb : last;
                    if (fragile_px) fragile_px[pix_off + p] = (uint8_t)fr;
                    hh = fnv(hh, (uint64_t)nb);
                    for (int r = 0; r < nb; r++) hh = fnv(hh, ((uint64_t)recs[r].j << 1) | (uint64_t)recs[r].clamped);
                }
            th[t] = hh;
            free(recs);
        }
        for (int t = 0; t < gw * gh; t++) h = fnv(h, th[t]);
        free(th);
        if (ord) free(ord);
        img_off += (size_t)3 * W * H;
        pix_off += (size_t)W * H;
    }
    for (size_t k = 0; k < (size_t)V * s->n; k++) {
        h = fnv(h, (uint64_t)sp[k].valid);
        if (sp[k].valid) {
            h = fnv(h, ((uint64_t)sp[k].rect[0] << 48) ^ ((uint64_t)sp[k].rect[1] << 32) ^
                           ((uint64_t)sp[k].rect[2] << 16) ^ (uint64_t)sp[k].rect[3]);
            h = fnv(h, (uint64_t)(sp[k].colclamp[0] | (sp[k].colclamp[1] << 1) | (sp[k].colclamp[2] << 2) |
                                  (sp[k].clampx << 3) | (sp[k].clampy << 4)));
        }
    }
    for (int64_t k = 0; k < L.n_keys; k++) h = fnv(h, L.idx[k]);
    if (hash_out) *hash_out = h;
    free_lists(&L);
    free(sp);
    return 0;
}

/* Key-path outputs of every (view, Gaussian) and the sorted tile lists, for
 * bit-exact comparison.  Per (v,i): valid, depth, FP32 mu_hat, radius, rect.
 * ranges [total_tiles][2] and idx [n_keys] are written when idx_cap suffices.
 * Returns the number of keys (or -1 on allocation failure). */
int64_t or_keys(const or_scene* s, int V, const or_cam* cams, const or_opts* o,
                uint8_t* valid, float* depth, float* mu2f, int32_t* radius, int32_t* rect,
                uint32_t* ranges, uint32_t* idx, int64_t idx_cap) {
    or_splat* sp = (or_splat*)malloc(sizeof(or_splat) * (size_t)V * (s->n > 0 ? s->n : 1));
    if (!sp) return -1;
    project_all(s, V, cams, o, sp);
    for (size_t k = 0; k < (size_t)V * s->n; k++) {
        if (valid) valid[k] = (uint8_t)sp[k].valid;
        if (depth) depth[k] = sp[k].valid ? sp[k].depth : 0.0f;
        if (mu2f) { mu2f[2 * k] = sp[k].valid ? sp[k].mu2f[0] : 0.0f; mu2f[2 * k + 1] = sp[k].valid ? sp[k].mu2f[1] : 0.0f; }
        if (radius) radius[k] = sp[k].valid ? sp[k].radius : 0;
        if (rect) for (int a = 0; a < 4; a++) rect[4 * k + a] = sp[k].valid ? sp[k].rect[a] : 0;
    }
    or_lists L;
    build_lists(s, V, cams, sp, &L);
    int64_t K = L.n_keys;
    if (ranges) memcpy(ranges, L.ranges, sizeof(uint32_t) * 2 * (size_t)L.total_tiles);
    if (idx && idx_cap >= K) memcpy(idx, L.idx, sizeof(uint32_t) * (size_t)K);
    free_lists(&L);
    free(sp);
    return K;
}

/* FP64 per-(v,i) values consumed by blending: mu_hat (2), conic (3),
 * opacity (1), colour (3) -> [V*n][9]; zero where culled. */
int or_project_values(const or_scene* s, int V, const or_cam* cams, const or_opts* o, double* out9) {
    or_splat* sp = (or_splat*)malloc(sizeof(or_splat) * (size_t)V * (s->n > 0 ? s->n : 1));
    if (!sp) return -1;
    project_all(s, V, cams, o, sp);
    for (size_t k = 0; k < (size_t)V * s->n; k++) {
        double* r = out9 + 9 * k;
        memset(r, 0, 9 * sizeof(double));
        if (!sp[k].valid) continue;
        r[0] = sp[k].mu2[0]; r[1] = sp[k].mu2[1];
        r[2] = sp[k].conic[0]; r[3] = sp[k].conic[1]; r[4] = sp[k].conic[2];
        r[5] = sp[k].opac;
        r[6] = sp[k].col[0]; r[7] = sp[k].col[1]; r[8] = sp[k].col[2];
    }
    free(sp);
    return 0;
}

/* ------------------------------------------------------------- backward */

/* Chain rule of one (view, Gaussian) from its 2D gradients
 * g9 = (dL/dmu_hat[2], dL/dconic[a,b,c], dL/do, dL/dc[3]) to the world
 * parameters and to the camera pose (Eq. 7-13).  Accumulates into the
 * per-Gaussian gradients and into pose6 = (rho[3], phi[3]). */
static void chain_one(const or_scene* s, int i, const or_cam* cam, const or_splat* g,
                      const double* g9, double* gm, double* gs, double* gq, double* go,
                      double* gsh, double* pose6) {
    const double fx = cam->fx, fy = cam->fy;
    const double x = g->mc[0], y = g->mc[1], z = g->mc[2];
    /* conic = Sigma_hat^{-1}: dL/dSigma_hat = -Q G_Q Q, Q and G_Q symmetric,
     * G_Q's off-diagonal entries carrying half of dL/db each. */
    double Q[4] = {g->conic[0], g->conic[1], g->conic[1], g->conic[2]};
    double GQ[4] = {g9[2], 0.5 * g9[3], 0.5 * g9[3], g9[4]};
    double QG[4], GS[4];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) QG[a * 2 + b] = Q[a * 2 + 0] * GQ[0 * 2 + b] + Q[a * 2 + 1] * GQ[1 * 2 + b];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) GS[a * 2 + b] = -(QG[a * 2 + 0] * Q[0 * 2 + b] + QG[a * 2 + 1] * Q[1 * 2 + b]);
    /* Sigma_hat = J Sigma_c J^T (+ eps2d I): dL/dSigma_c = J^T GS J,
     * dL/dJ = 2 GS J Sigma_c */
    const double* J = g->J;
    double GSc[9];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double t = 0.0;
            for (int p = 0; p < 2; p++)
                for (int q = 0; q < 2; q++) t += J[p * 3 + a] * GS[p * 2 + q] * J[q * 3 + b];
            GSc[a * 3 + b] = t;
        }
    double GJ[6];
    for (int p = 0; p < 2; p++)
        for (int b = 0; b < 3; b++) {
            double t = 0.0;
            for (int q = 0; q < 2; q++)
                for (int k = 0; k < 3; k++) t += GS[p * 2 + q] * J[q * 3 + k] * g->Sc[k * 3 + b];
            GJ[p * 3 + b] = 2.0 * t;
        }
    /* dL/dmu_c: through mu_hat (pi) and through J */
    double gmc[3];
    gmc[0] = g9[0] * fx / z;
    gmc[1] = g9[1] * fy / z;
    gmc[2] = -(g9[0] * fx * x + g9[1] * fy * y) / (z * z);
    /* J00 = fx/z, J11 = fy/z, J02 = -fx u/z, J12 = -fy v/z with u = clamp(x/z) */
    gmc[2] += GJ[0] * (-fx / (z * z)) + GJ[4] * (-fy / (z * z));
    if (!g->clampx) {
        gmc[0] += GJ[2] * (-fx / (z * z));
        gmc[2] += GJ[2] * (2.0 * fx * x / (z * z * z));
    } else {
        gmc[2] += GJ[2] * (fx * g->uxc / (z * z));
    }
    if (!g->clampy) {
        gmc[1] += GJ[5] * (-fy / (z * z));
        gmc[2] += GJ[5] * (2.0 * fy * y / (z * z * z));
    } else {
        gmc[2] += GJ[5] * (fy * g->uyc / (z * z));
    }
    /* Sigma_c = R_c Sigma R_c^T -> dL/dSigma = R_c^T GSc R_c */
    double T1[9], GSig[9];
    mat3_mul_at(g->Rc, GSc, T1);
    mat3_mul(T1, g->Rc, GSig);
    /* Sigma = M M^T -> dL/dM = 2 GSig M (GSig symmetric) */
    double GM[9];
    mat3_mul(GSig, g->M, GM);
    for (int k = 0; k < 9; k++) GM[k] *= 2.0;
    /* M = R diag(s) */
    const float* sc = s->scales + 3 * i;
    double GR[9];
    for (int k = 0; k < 3; k++) {
        double t = 0.0;
        for (int j = 0; j < 3; j++) { t += GM[j * 3 + k] * g->R[j * 3 + k]; GR[j * 3 + k] = GM[j * 3 + k] * (double)sc[k]; }
        gs[3 * i + k] += t;
    }
    /* R(q_hat) -> q_hat */
    const double w = g->qn[0], qx = g->qn[1], qy = g->qn[2], qz = g->qn[3];
    double gqh[4];
    gqh[0] = 2.0 * (-qz * GR[1] + qy * GR[2] + qz * GR[3] - qx * GR[5] - qy * GR[6] + qx * GR[7]);
    gqh[1] = 2.0 * (qy * GR[1] + qz * GR[2] + qy * GR[3] - 2.0 * qx * GR[4] - w * GR[5] + qz * GR[6] + w * GR[7]
                    - 2.0 * qx * GR[8]);
    gqh[2] = 2.0 * (-2.0 * qy * GR[0] + qx * GR[1] + w * GR[2] + qx * GR[3] + qz * GR[5] - w * GR[6] + qz * GR[7]
                    - 2.0 * qy * GR[8]);
    gqh[3] = 2.0 * (-2.0 * qz * GR[0] - w * GR[1] + qx * GR[2] + w * GR[3] - 2.0 * qz * GR[4] + qy * GR[5]
                    + qx * GR[6] + qy * GR[7]);
    /* q_hat = q / |q| */
    double dq = gqh[0] * g->qn[0] + gqh[1] * g->qn[1] + gqh[2] * g->qn[2] + gqh[3] * g->qn[3];
    for (int k = 0; k < 4; k++) gq[4 * i + k] += (gqh[k] - g->qn[k] * dq) / g->qlen;
    /* opacity */
    go[i] += g9[5];
    /* SH colour: c = max(0, sum f Y(d) + 0.5) */
    double Y[16], dY[16][3];
    sh_basis(g->dir, s->sh_degree, Y, dY);
    int nb = (s->sh_degree + 1) * (s->sh_degree + 1);
    double gdir[3] = {0, 0, 0};
    const float* f = s->sh + 48 * (size_t)i;
    for (int ch = 0; ch < 3; ch++) {
        if (g->colclamp[ch]) continue;
        double gc = g9[6 + ch];
        for (int k = 0; k < nb; k++) {
            gsh[48 * (size_t)i + k * 3 + ch] += Y[k] * gc;
            for (int a = 0; a < 3; a++) gdir[a] += (double)f[k * 3 + ch] * dY[k][a] * gc;
        }
    }
    /* d = v/|v|, v = mu - o_c */
    double dd = gdir[0] * g->dir[0] + gdir[1] * g->dir[1] + gdir[2] * g->dir[2];
    double gmu_sh[3];
    for (int a = 0; a < 3; a++) gmu_sh[a] = (gdir[a] - g->dir[a] * dd) / g->vlen;
    /* mu_c = R_c mu + t_c */
    for (int a = 0; a < 3; a++)
        gm[3 * i + a] += g->Rc[0 * 3 + a] * gmc[0] + g->Rc[1 * 3 + a] * gmc[1] + g->Rc[2 * 3 + a] * gmc[2]
                         + gmu_sh[a];
    /* Pose, left perturbation Exp(tau) T with tau = (rho, phi):
     *   mu_c -> mu_c + rho + phi x mu_c             (Eq. 8/10)
     *   R_c  -> (I + [phi]x) R_c, hence Sigma_c -> Sigma_c + [phi]x Sigma_c - Sigma_c [phi]x  (Eq. 12-13)
     *   o_c  -> o_c - R_c^T rho                      (camera centre; SH term) */
    double cr[3];
    cross3(g->mc, gmc, cr);
    double A[9];
    mat3_mul(g->Sc, GSc, A);
    double Rg[3];
    for (int a = 0; a < 3; a++)
        Rg[a] = g->Rc[a * 3 + 0] * gmu_sh[0] + g->Rc[a * 3 + 1] * gmu_sh[1] + g->Rc[a * 3 + 2] * gmu_sh[2];
    pose6[0] += gmc[0] + Rg[0];
    pose6[1] += gmc[1] + Rg[1];
    pose6[2] += gmc[2] + Rg[2];
    pose6[3] += cr[0] + 2.0 * (A[1 * 3 + 2] - A[2 * 3 + 1]);
    pose6[4] += cr[1] + 2.0 * (A[2 * 3 + 0] - A[0 * 3 + 2]);
    pose6[5] += cr[2] + 2.0 * (A[0 * 3 + 1] - A[1 * 3 + 0]);
}

/* Backward of the rendering given dL/dC (packed planar per view, FP64).
 * Outputs (accumulated with +=, caller zeroes): g_means [n][3], g_scales
 * [n][3], g_quats [n][4], g_opac [n], g_sh [n][16][3], pose_grad [V][6]
 * (rho, phi).  g2d [V*n][9] (nullable) receives the per-(view, Gaussian) 2D
 * gradients.  fragile_g [V*n] (nullable) marks Gaussians with a near-threshold
 * Gaussian-level decision. */
int or_backward(const or_scene* s, int V, const or_cam* cams, const or_opts* o, const double* dldc,
                double* g_means, double* g_scales, double* g_quats, double* g_opac, double* g_sh,
                double* pose_grad, double* g2d_out, uint8_t* fragile_g) {
    size_t VN = (size_t)V * s->n;
    or_splat* sp = (or_splat*)malloc(sizeof(or_splat) * (VN > 0 ? VN : 1));
    if (!sp) return -1;
    project_all(s, V, cams, o, sp);
    or_lists L;
    build_lists(s, V, cams, sp, &L);
    int nthr = g_threads;
    double* g2d = (double*)calloc((VN > 0 ? VN : 1) * 9 * (size_t)nthr, sizeof(double));
    if (!g2d) { free_lists(&L); free(sp); return -1; }
    size_t img_off = 0;
    for (int v = 0; v < V; v++) {
        const or_cam* c = cams + v;
        const or_splat* spv = sp + (size_t)v * s->n;
        int W = c->width, H = c->height, gw = tiles_x(c), gh = tiles_y(c);
        const double* dv = dldc + img_off;
        #pragma omp parallel for schedule(static, 1) num_threads(nthr)
        for (int t = 0; t < gw * gh; t++) {
#ifdef _OPENMP
            int tid = omp_get_thread_num();
#else
            int tid = 0;
#endif
            double* acc = g2d + (size_t)tid * VN * 9 + (size_t)v * s->n * 9;
            int tx = t % gw, ty = t / gw;
            uint32_t gt = (uint32_t)(L.tile_base[v] + t);
            const uint32_t* list = L.idx + L.ranges[2 * gt];
            int n = (int)(L.ranges[2 * gt + 1] - L.ranges[2 * gt]);
            or_rec* recs = (or_rec*)malloc(sizeof(or_rec) * (n > 0 ? n : 1));
            for (int py = ty * OR_TILE; py < (ty + 1) * OR_TILE && py < H; py++)
                for (int px = tx * OR_TILE; px < (tx + 1) * OR_TILE && px < W; px++) {
                    double C[3], Tf; int nb = 0, fr = 0;
                    blend_pixel(spv, list, n, px, py, tx, ty, 0, o, C, &Tf, recs, &nb, &fr);
                    size_t p = (size_t)py * W + px;
                    double gC[3] = {dv[p], dv[(size_t)W * H + p], dv[(size_t)2 * W * H + p]};
                    if (gC[0] == 0.0 && gC[1] == 0.0 && gC[2] == 0.0) continue;
                    /* C = sum_i c_i a_i T_i + T_final bg.
                     * dC/dc_i = a_i T_i;
                     * dC/da_i = c_i T_i - (sum_{k>i} c_k a_k T_k + T_final bg) / (1 - a_i). */
                    double Sb[3] = {Tf * o->bg[0], Tf * o->bg[1], Tf * o->bg[2]};
                    for (int r = nb - 1; r >= 0; r--) {
                        const or_rec* e = recs + r;
                        const or_splat* g = spv + e->j;
                        double* a9 = acc + (size_t)e->j * 9;
                        double dLda = 0.0;
                        for (int ch = 0; ch < 3; ch++) {
                            double dCda = g->col[ch] * e->T - Sb[ch] / (1.0 - e->alpha);
                            dLda += gC[ch] * dCda;
                            a9[6 + ch] += gC[ch] * e->alpha * e->T;
                        }
                        for (int ch = 0; ch < 3; ch++) Sb[ch] += g->col[ch] * e->alpha * e->T;
                        if (e->clamped) continue;
                        /* alpha = o G, G = exp(power) */
                        a9[5] += e->G * dLda;
                        double dLdp = e->alpha * dLda;
                        double dx = e->d[0], dy = e->d[1];
                        /* d power / d mu_hat = Q d; d power / d(a, b, c) = (-dx^2/2, -dx dy, -dy^2/2) */
                        a9[0] += dLdp * (g->conic[0] * dx + g->conic[1] * dy);
                        a9[1] += dLdp * (g->conic[1] * dx + g->conic[2] * dy);
                        a9[2] += dLdp * (-0.5 * dx * dx);
                        a9[3] += dLdp * (-dx * dy);
                        a9[4] += dLdp * (-0.5 * dy * dy);
                    }
                }
            free(recs);
        }
        img_off += (size_t)3 * W * H;
    }
    /* reduce the per-thread 2D gradients in thread order */
    for (int tid = 1; tid < nthr; tid++)
        for (size_t k = 0; k < VN * 9; k++) g2d[k] += g2d[(size_t)tid * VN * 9 + k];
    if (g2d_out) memcpy(g2d_out, g2d, sizeof(double) * VN * 9);
    /* per-Gaussian chain: each Gaussian sums its views in view order */
    double* pacc = (double*)calloc((size_t)nthr * V * 6, sizeof(double));
    #pragma omp parallel for schedule(static) num_threads(nthr)
    for (int i = 0; i < s->n; i++) {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        for (int v = 0; v < V; v++) {
            const or_splat* g = sp + (size_t)v * s->n + i;
            if (!g->valid) continue;
            const double* g9 = g2d + ((size_t)v * s->n + i) * 9;
            int any = 0;
            for (int k = 0; k < 9; k++) any |= g9[k] != 0.0;
            if (!any) continue;
            chain_one(s, i, cams + v, g, g9, g_means, g_scales, g_quats, g_opac, g_sh,
                      pacc + ((size_t)tid * V + v) * 6);
        }
    }
    for (int tid = 0; tid < nthr; tid++)
        for (int k = 0; k < V * 6; k++) pose_grad[k] += pacc[(size_t)tid * V * 6 + k];
    if (fragile_g)
        for (size_t k = 0; k < VN; k++) fragile_g[k] = (uint8_t)sp[k].fragile;
    free(pacc);
    free(g2d);
    free_lists(&L);
    free(sp);
    return 0;
}

/* ---------------------------------------------------------------- losses */

/* L1 (Eq. 16's first term): L = w * sum_v mean_{3HW} |C - I|.
 * dldc (nullable) receives w * sign(C - I) / (3HW), sign(0) = 0; fragile_px
 * (nullable, packed [H][W]) is set where 0 < |C - I| < 1e-5 in some channel. */
double or_loss_l1(int V, const int* wh, const double* img, const float* target, double w,
                  double* dldc, uint8_t* fragile_px) {
    double total = 0.0;
    size_t off = 0, poff = 0;
    for (int v = 0; v < V; v++) {
        size_t np = (size_t)wh[2 * v] * wh[2 * v + 1];
        double m = 3.0 * (double)np, acc = 0.0;
        for (int ch = 0; ch < 3; ch++)
            for (size_t p = 0; p < np; p++) {
                size_t k = off + ch * np + p;
                double d = img[k] - (double)target[k];
                acc += fabs(d);
                if (dldc) dldc[k] = d > 0 ? w / m : (d < 0 ? -w / m : 0.0);
                if (fragile_px && d != 0.0 && fabs(d) < 1e-5) fragile_px[poff + p] = 1;
            }
        total += w * acc / m;
        off += 3 * np;
        poff += np;
    }
    return total;
}

/* Sec. 3.4, Eq. 20-21: confidence-masked L1 for pose estimation.  The mask
 * keeps a pixel when its accumulated alpha 1 - T_final (the sum of the blend
 * weights, which the paper calls transmittances) exceeds mask_alpha.  Eq. 21
 * prints a sum; read as the mean over 3HW with masked-out pixels counting 0,
 * so that it has the scale of the unmasked L1.  The mask is piecewise
 * constant in the parameters, so dL/dC = w M sign(C - I) / (3HW).
 * fragile_px flags pixels whose mask decision lies within 1e-5 of the
 * threshold, and kept pixels whose sign is in doubt. */
double or_loss_l1_masked(int V, const int* wh, const double* img, const float* target, const double* T_final,
                         double mask_alpha, double w, double* dldc, uint8_t* fragile_px) {
    double total = 0.0;
    size_t off = 0, poff = 0;
    for (int v = 0; v < V; v++) {
        size_t np = (size_t)wh[2 * v] * wh[2 * v + 1];
        double m = 3.0 * (double)np, acc = 0.0;
        for (int ch = 0; ch < 3; ch++)
            for (size_t p = 0; p < np; p++) {
                const double a = 1.0 - T_final[poff + p];
                const int keep = a > mask_alpha;
                if (fragile_px && fabs(a - mask_alpha) <= 1e-5) fragile_px[poff + p] = 1;
                size_t k = off + ch * np + p;
                double d = img[k] - (double)target[k];
                if (!keep) {
                    if (dldc) dldc[k] = 0.0;
                    continue;
                }
                acc += fabs(d);
                if (dldc) dldc[k] = d > 0 ? w / m : (d < 0 ? -w / m : 0.0);
                if (fragile_px && d != 0.0 && fabs(d) < 1e-5) fragile_px[poff + p] = 1;
            }
        total += w * acc / m;
        off += 3 * np;
        poff += np;
    }
    return total;
}

/* Normalised 11-tap Gaussian window, sigma = 1.5 (the prior art's SSIM window). */
static void ssim_window(double* g11) {
    double s = 0.0;
    for (int k = 0; k < 11; k++) { double x = k - 5; g11[k] = exp(-x * x / (2.0 * 1.5 * 1.5)); s += g11[k]; }
    for (int k = 0; k < 11; k++) g11[k] /= s;
}

/* Zero-padded "same" 2D filtering with the 11x11 window w(a) w(b), written as
 * the plain double sum over the window. */
static void filt2(const double* x, int W, int H, const double* g, double* out) {
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            double s = 0.0;
            for (int b = -5; b <= 5; b++) {
                int yy = py + b;
                if (yy < 0 || yy >= H) continue;
                for (int a = -5; a <= 5; a++) {
                    int xx = px + a;
                    if (xx < 0 || xx >= W) continue;
                    s += g[a + 5] * g[b + 5] * x[(size_t)yy * W + xx];
                }
            }
            out[(size_t)py * W + px] = s;
        }
}

/* D-SSIM term: L = w * sum_v (1 - mean_{3HW} SSIM), SSIM with the 11x11
 * Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2.
 * dldc (nullable) receives the gradient; ssim_map (nullable) the SSIM map. */
double or_loss_dssim(int V, const int* wh, const double* img, const float* target, double w,
                     double* dldc, double* ssim_map) {
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double g[11];
    ssim_window(g);
    double total = 0.0;
    size_t off = 0;
    for (int v = 0; v < V; v++) {
        int W = wh[2 * v], H = wh[2 * v + 1];
        size_t np = (size_t)W * H;
        double m = 3.0 * (double)np;
        double* buf = (double*)malloc(sizeof(double) * np * 14);
        double *X = buf, *Y = buf + np, *XX = buf + 2 * np, *YY = buf + 3 * np, *XY = buf + 4 * np;
        double *mx = buf + 5 * np, *my = buf + 6 * np, *sxx = buf + 7 * np, *syy = buf + 8 * np, *sxy = buf + 9 * np;
        double *dA = buf + 10 * np, *dB = buf + 11 * np, *dCc = buf + 12 * np, *tmp = buf + 13 * np;
        double acc = 0.0;
        for (int ch = 0; ch < 3; ch++) {
            for (size_t p = 0; p < np; p++) {
                X[p] = img[off + ch * np + p]; Y[p] = (double)target[off + ch * np + p];
                XX[p] = X[p] * X[p]; YY[p] = Y[p] * Y[p]; XY[p] = X[p] * Y[p];
            }
            filt2(X, W, H, g, mx); filt2(Y, W, H, g, my);
            filt2(XX, W, H, g, sxx); filt2(YY, W, H, g, syy); filt2(XY, W, H, g, sxy);
            for (size_t p = 0; p < np; p++) {
                double ux = mx[p], uy = my[p];
                double vx = sxx[p] - ux * ux, vy = syy[p] - uy * uy, cxy = sxy[p] - ux * uy;
                double N1 = 2.0 * ux * uy + C1, N2 = 2.0 * cxy + C2;
                double D1 = ux * ux + uy * uy + C1, D2 = vx + vy + C2;
                double f = (N1 * N2) / (D1 * D2);
                acc += f;
                if (ssim_map) ssim_map[off + ch * np + p] = f;
                /* partial derivatives of f w.r.t. mu_x, sigma_x^2, sigma_xy */
                double dmu = 2.0 * uy * N2 / (D1 * D2) - f * 2.0 * ux / D1;
                double dvx = -f / D2;
                double dcxy = 2.0 * N1 / (D1 * D2);
                /* sigma_x^2 = F(x^2) - mu_x^2, sigma_xy = F(xy) - mu_x mu_y */
                dA[p] = dmu - 2.0 * ux * dvx - uy * dcxy;
                dB[p] = dvx;
                dCc[p] = dcxy;
            }
            if (dldc) {
                /* adjoint of the zero-padded symmetric filter is the same filter */
                double* out = dldc + off + ch * np;
                filt2(dA, W, H, g, tmp);
                for (size_t p = 0; p < np; p++) out[p] = tmp[p];
                filt2(dB, W, H, g, tmp);
                for (size_t p = 0; p < np; p++) out[p] += 2.0 * X[p] * tmp[p];
                filt2(dCc, W, H, g, tmp);
                for (size_t p = 0; p < np; p++) out[p] += Y[p] * tmp[p];
                for (size_t p = 0; p < np; p++) out[p] *= -w / m;
            }
        }
        total += w * (1.0 - acc / m);
        free(buf);
        off += 3 * np;
    }
    return total;
}

/* Conditioning of the D-SSIM gradient (a diagnostic for tolerances, not part
 * of the loss): per element, w/(3HW) times the sum of the magnitudes of the
 * terms whose signed sum or_loss_dssim returns as dL/dC,
 *   F(|dmu| + 2|mu_x dvx| + |mu_y dcxy|) + 2|x| F(|dvx|) + |y| F(|dcxy|),
 * with the partials of f = SSIM at each window centre as in or_loss_dssim.
 * A computation of dL/dC in a precision with unit roundoff u that rounds
 * each of those terms a bounded number k of times is off by at most about
 * k u cond (the classical bound for sums of n terms, (n - 1) u sum |t_i|). */
void or_loss_dssim_cond(int V, const int* wh, const double* img, const float* target, double w, double* cond) {
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double g[11];
    ssim_window(g);
    size_t off = 0;
    for (int v = 0; v < V; v++) {
        int W = wh[2 * v], H = wh[2 * v + 1];
        size_t np = (size_t)W * H;
        double m = 3.0 * (double)np;
        double* buf = (double*)malloc(sizeof(double) * np * 14);
        double *X = buf, *Y = buf + np, *XX = buf + 2 * np, *YY = buf + 3 * np, *XY = buf + 4 * np;
        double *mx = buf + 5 * np, *my = buf + 6 * np, *sxx = buf + 7 * np, *syy = buf + 8 * np, *sxy = buf + 9 * np;
        double *aA = buf + 10 * np, *aB = buf + 11 * np, *aC = buf + 12 * np, *tmp = buf + 13 * np;
        for (int ch = 0; ch < 3; ch++) {
            for (size_t p = 0; p < np; p++) {
                X[p] = img[off + ch * np + p]; Y[p] = (double)target[off + ch * np + p];
                XX[p] = X[p] * X[p]; YY[p] = Y[p] * Y[p]; XY[p] = X[p] * Y[p];
            }
            filt2(X, W, H, g, mx); filt2(Y, W, H, g, my);
            filt2(XX, W, H, g, sxx); filt2(YY, W, H, g, syy); filt2(XY, W, H, g, sxy);
            for (size_t p = 0; p < np; p++) {
                double ux = mx[p], uy = my[p];
                double vx = sxx[p] - ux * ux, vy = syy[p] - uy * uy, cxy = sxy[p] - ux * uy;
                double N1 = 2.0 * ux * uy + C1, N2 = 2.0 * cxy + C2;
                double D1 = ux * ux + uy * uy + C1, D2 = vx + vy + C2;
                double f = (N1 * N2) / (D1 * D2);
                double dmu = 2.0 * uy * N2 / (D1 * D2) - f * 2.0 * ux / D1;
                double dvx = -f / D2;
                double dcxy = 2.0 * N1 / (D1 * D2);
                aA[p] = fabs(dmu) + 2.0 * fabs(ux * dvx) + fabs(uy * dcxy);
                aB[p] = fabs(dvx);
                aC[p] = fabs(dcxy);
            }
            double* out = cond + off + ch * np;
            filt2(aA, W, H, g, tmp);
            for (size_t p = 0; p < np; p++) out[p] = tmp[p];
            filt2(aB, W, H, g, tmp);
            for (size_t p = 0; p < np; p++) out[p] += 2.0 * fabs(X[p]) * tmp[p];
            filt2(aC, W, H, g, tmp);
            for (size_t p = 0; p < np; p++) out[p] += fabs(Y[p]) * tmp[p];
            for (size_t p = 0; p < np; p++) out[p] *= fabs(w) / m;
        }
        free(buf);
        off += 3 * np;
    }
}

/* Exposed for the window pin: zero-padded Gaussian filtering of one plane. */
void or_ssim_filter(const double* x, int W, int H, double* out) {
    double g[11];
    ssim_window(g);
    filt2(x, W, H, g, out);
}

/* ------------------------------------------------------------- SE(3) */

static void hat3(const double* p, double* K) {
    K[0] = 0; K[1] = -p[2]; K[2] = p[1];
    K[3] = p[2]; K[4] = 0; K[5] = -p[0];
    K[6] = -p[1]; K[7] = p[0]; K[8] = 0;
}

/* Exp: R6 -> SE(3), tau = (rho, phi): R = I + A K + B K^2, t = V rho with
 * V = I + B K + C K^2, K = [phi]x, A = sin t/t, B = (1 - cos t)/t^2,
 * C = (t - sin t)/t^3 (series below 1e-4).  T is [12]: R row-major, t. */
void or_se3_exp(const double* tau, double* T) {
    const double* rho = tau; const double* phi = tau + 3;
    double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    double th = sqrt(th2);
    double A, B, Cc;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        Cc = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        A = sin(th) / th; B = (1.0 - cos(th)) / th2; Cc = (th - sin(th)) / (th2 * th);
    }
    double K[9], K2[9];
    hat3(phi, K);
    mat3_mul(K, K, K2);
    double Vm[9];
    for (int k = 0; k < 9; k++) {
        double I = (k % 4 == 0) ? 1.0 : 0.0;
        T[k] = I + A * K[k] + B * K2[k];
        Vm[k] = I + B * K[k] + Cc * K2[k];
    }
    for (int a = 0; a < 3; a++) T[9 + a] = Vm[a * 3 + 0] * rho[0] + Vm[a * 3 + 1] * rho[1] + Vm[a * 3 + 2] * rho[2];
}

/* Log: SE(3) -> R6, the inverse of or_se3_exp for rotation angles below pi. */
void or_se3_log(const double* T, double* tau) {
    double tr = T[0] + T[4] + T[8];
    double c = 0.5 * (tr - 1.0);
    if (c > 1.0) c = 1.0; if (c < -1.0) c = -1.0;
    double th = acos(c);
    double w[3] = {T[7] - T[5], T[2] - T[6], T[3] - T[1]};
    double f = th < 1e-6 ? 0.5 + th * th / 12.0 : th / (2.0 * sin(th));
    double phi[3] = {f * w[0], f * w[1], f * w[2]};
    double K[9], K2[9];
    hat3(phi, K);
    mat3_mul(K, K, K2);
    double th2 = th * th;
    double D;
    if (th < 1e-4) D = 1.0 / 12.0 + th2 / 720.0;
    else {
        double A = sin(th) / th, B = (1.0 - cos(th)) / th2;
        D = (1.0 - A / (2.0 * B)) / th2;
    }
    double Vi[9];
    for (int k = 0; k < 9; k++) Vi[k] = ((k % 4 == 0) ? 1.0 : 0.0) - 0.5 * K[k] + D * K2[k];
    for (int a = 0; a < 3; a++) tau[a] = Vi[a * 3 + 0] * T[9] + Vi[a * 3 + 1] * T[10] + Vi[a * 3 + 2] * T[11];
    for (int a = 0; a < 3; a++) tau[3 + a] = phi[a];
}

/* T <- Exp(tau) T (left update), T [12]. */
void or_se3_left_update(const double* tau, double* T) {
    double E[12], R[9], t[3];
    or_se3_exp(tau, E);
    mat3_mul(E, T, R);
    for (int a = 0; a < 3; a++) t[a] = E[a * 3 + 0] * T[9] + E[a * 3 + 1] * T[10] + E[a * 3 + 2] * T[11] + E[9 + a];
    memcpy(T, R, sizeof(R));
    memcpy(T + 9, t, sizeof(t));
}

/* Adam on the pose tangent (moments kept in the tangent space), then the
 * left update T <- Exp(-lr m_hat / (sqrt(v_hat) + eps)) T.  step is 1-based.
 * poses [V][12], m, v [V][6], grad [V][6]. */
void or_pose_adam(int V, double* poses, double* m, double* v, const double* grad, double lr,
                  double b1, double b2, double eps, int step) {
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (int i = 0; i < V; i++) {
        double d[6];
        for (int k = 0; k < 6; k++) {
            double g = grad[6 * i + k];
            m[6 * i + k] = b1 * m[6 * i + k] + (1.0 - b1) * g;
            v[6 * i + k] = b2 * v[6 * i + k] + (1.0 - b2) * g * g;
            double mh = m[6 * i + k] / c1, vh = v[6 * i + k] / c2;
            d[k] = -lr * mh / (sqrt(vh) + eps);
        }
        or_se3_left_update(d, poses + 12 * i);
    }
}

/* T x SO(3) variant (Sec. 4.2 names it as the parametrisation free of the
 * SE(3) coupling of camera position and orientation): the camera centre
 * o = -R^T t and the rotation are stepped separately, o <- o + d_o and
 * R <- Exp_SO3(d_phi) R (a rotation about the centre), then t = -R o.  The
 * input gradient is the left-SE(3) one (g_rho, g_phi).  Moving the centre by
 * d_o is the left step rho = -R d_o, so the gradient in these coordinates is
 * g_o = -R^T g_rho; a left step with rho = 0 rotates about the centre, so
 * g_phi carries over.  Adam moments are kept in (g_o, g_phi). */
void or_pose_adam_txso3(int V, double* poses, double* m, double* v, const double* grad, double lr,
                        double b1, double b2, double eps, int step) {
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (int i = 0; i < V; i++) {
        double* P = poses + 12 * i;
        const double* g_se3 = grad + 6 * i;
        double g[6];
        for (int a = 0; a < 3; a++)
            g[a] = -(P[0 * 3 + a] * g_se3[0] + P[1 * 3 + a] * g_se3[1] + P[2 * 3 + a] * g_se3[2]);
        for (int a = 3; a < 6; a++) g[a] = g_se3[a];
        double d[6];
        for (int k = 0; k < 6; k++) {
            m[6 * i + k] = b1 * m[6 * i + k] + (1.0 - b1) * g[k];
            v[6 * i + k] = b2 * v[6 * i + k] + (1.0 - b2) * g[k] * g[k];
            double mh = m[6 * i + k] / c1, vh = v[6 * i + k] / c2;
            d[k] = -lr * mh / (sqrt(vh) + eps);
        }
        double o[3];
        for (int a = 0; a < 3; a++) o[a] = -(P[0 * 3 + a] * P[9] + P[1 * 3 + a] * P[10] + P[2 * 3 + a] * P[11]) + d[a];
        double rot[6] = {0.0, 0.0, 0.0, d[3], d[4], d[5]}, E[12], R[9];
        or_se3_exp(rot, E);
        mat3_mul(E, P, R);
        memcpy(P, R, sizeof(R));
        for (int a = 0; a < 3; a++) P[9 + a] = -(R[a * 3 + 0] * o[0] + R[a * 3 + 1] * o[1] + R[a * 3 + 2] * o[2]);
    }
}

/* Joint refinement's regularisers (Sec. 3.3) on activated scales [n][3] and
 * opacities [n]: lam_an * (1/n) sum_i [max(s_i)/min(s_i) - r]_+ (Eq. 17) plus
 * lam_op * (1/n) sum_i o_i.  Adds the gradients into g_scales / g_opac
 * (nullable) and returns the value.  The ratio's subgradient goes to the
 * first largest and the first smallest axis; no gradient when the ratio is
 * exactly r or all axes are equal. */
double or_regularize(int n, const float* scales, const float* opac, double r, double lam_an, double lam_op,
                     double* g_scales, double* g_opac) {
    double total = 0.0;
    if (n <= 0) return 0.0;
    const double w_an = lam_an / n, w_op = lam_op / n;
    for (int i = 0; i < n; i++) {
        const double s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
        int imax = 0, imin = 0;
        for (int k = 1; k < 3; k++) {
            if (s[k] > s[imax]) imax = k;
            if (s[k] < s[imin]) imin = k;
        }
        const double ratio = s[imax] / s[imin];
        if (lam_an != 0.0 && ratio > r && imax != imin) {
            total += w_an * (ratio - r);
            if (g_scales) {
                g_scales[3 * i + imax] += w_an / s[imin];
                g_scales[3 * i + imin] -= w_an * ratio / s[imin];
            }
        }
        if (lam_op != 0.0) {
            total += w_op * opac[i];
            if (g_opac) g_opac[i] += w_op;
        }
    }
    return total;
}

static int cmp_float(const void* a, const void* b) {
    const float x = *(const float*)a, y = *(const float*)b;
    return (x > y) - (x < y);
}

/* The adaptive pruning threshold (Sec. 3.3: at most n_target Gaussians stay):
 * max(min_opacity, the (n - n_target)-th smallest opacity) when n > n_target,
 * else min_opacity; *n_keep = #{o > threshold}. */
float or_prune_threshold(int n, const float* opac, long long n_target, float min_opacity, long long* n_keep) {
    float thr = min_opacity;
    if ((long long)n > n_target) {
        float* sorted = (float*)malloc(sizeof(float) * (size_t)n);
        memcpy(sorted, opac, sizeof(float) * (size_t)n);
        qsort(sorted, (size_t)n, sizeof(float), cmp_float);
        const float kth = sorted[(size_t)(n - n_target - 1)];
        free(sorted);
        if (kth > thr) thr = kth;
    }
    long long kept = 0;
    for (int i = 0; i < n; i++) kept += opac[i] > thr;
    *n_keep = kept;
    return thr;
}

/* Sec. 3.4, relative pose initialisation: the pixels (u, v) = (i s, j s) of
 * the stride grid with z-depth d > 0 become camera points
 * ((u - cx) / fx d, (v - cy) / fy d, d) in pixel order (the pixel samples the
 * point (u, v)), with their colours (planar image, nullable).  Returns the
 * count; points / colours hold ceil(W/s) ceil(H/s) rows. */
int or_unproject(int W, int H, double fx, double fy, double cx, double cy, const float* depth, const float* image,
                 int stride, double* points, double* colours) {
    int n = 0;
    const size_t np = (size_t)W * H;
    for (int v = 0; v < H; v += stride)
        for (int u = 0; u < W; u += stride) {
            const double d = depth[(size_t)v * W + u];
            if (!(d > 0.0)) continue;
            points[3 * n + 0] = (u - cx) / fx * d;
            points[3 * n + 1] = (v - cy) / fy * d;
            points[3 * n + 2] = d;
            if (colours && image)
                for (int c = 0; c < 3; c++) colours[3 * n + c] = image[c * np + (size_t)v * W + u];
            n++;
        }
    return n;
}

/* Mean distance of every point to its k nearest other points (exhaustive,
 * FP64; coincident points count at distance 0), for the Gaussian scales of
 * Sec. 3.4. */
void or_knn_mean_dist(int n, const double* pts, int k, double* out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; i++) {
        double best[16];
        for (int j = 0; j < k; j++) best[j] = INFINITY;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            const double dx = pts[3 * j] - pts[3 * i], dy = pts[3 * j + 1] - pts[3 * i + 1],
                         dz = pts[3 * j + 2] - pts[3 * i + 2];
            double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 >= best[k - 1]) continue;
            int p = k - 1;
            while (p > 0 && best[p - 1] > d2) { best[p] = best[p - 1]; p--; }
            best[p] = d2;
        }
        double acc = 0.0;
        int cnt = 0;
        for (int j = 0; j < k; j++)
            if (best[j] < INFINITY) { acc += sqrt(best[j]); cnt++; }
        out[i] = cnt ? acc / cnt : 0.0;
    }
}

/* Adam on the raw Gaussian parameters of joint refinement (Sec. 3.3).  The
 * renderer's gradients are w.r.t. the activated scales s = exp(log s) and
 * opacities o = 1/(1 + exp(-logit)); the chain rule gives the raw gradients
 * g_log_s = g_s s and g_logit = g_o o (1 - o).  Group order and widths:
 * means 3, log-scales 3, quats 4, logit-opacities 1, SH 48 (only the first
 * 3 (deg+1)^2 coefficients are updated; SH DC at lr[4], the rest at lr[5]).
 * raw/grad/m/v are [n * width] per group, passed as 5 pointers each. */
void or_gaussian_adam(int n, int sh_degree, double** raw, double** grad, double** m, double** v,
                      const double* lr, double b1, double b2, double eps, int step,
                      double* scales_out, double* opac_out) {
    static const int width[5] = {3, 3, 4, 1, 48};
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    int used_sh = 3 * (sh_degree + 1) * (sh_degree + 1);
    for (int gi = 0; gi < 5; gi++) {
        int w = width[gi];
        int used = gi == 4 ? used_sh : w;
        for (int i = 0; i < n; i++)
            for (int k = 0; k < used; k++) {
                size_t id = (size_t)i * w + k;
                double p = raw[gi][id];
                double g = grad[gi][id];
                if (gi == 1) g *= exp(p);
                if (gi == 3) { double o = 1.0 / (1.0 + exp(-p)); g *= o * (1.0 - o); }
                m[gi][id] = b1 * m[gi][id] + (1.0 - b1) * g;
                v[gi][id] = b2 * v[gi][id] + (1.0 - b2) * g * g;
                double l = gi < 4 ? lr[gi] : (k < 3 ? lr[4] : lr[5]);
                p -= l * (m[gi][id] / c1) / (sqrt(v[gi][id] / c2) + eps);
                raw[gi][id] = p;
            }
    }
    for (size_t id = 0; id < (size_t)n * 3; id++) scales_out[id] = exp(raw[1][id]);
    for (int i = 0; i < n; i++) opac_out[i] = 1.0 / (1.0 + exp(-raw[3][i]));
}
