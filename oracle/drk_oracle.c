/*
 * drk_oracle.c -- plain FP64 CPU oracle for Deformable Radial Kernel (DRK)
 * splatting.  TEST INFRASTRUCTURE ONLY: it exists to check the CUDA path and
 * is called from the test-suite, the smoke check and the benchmark's CPU
 * baseline leg, never from the product path.  It shares no code, header or
 * constant table with the CUDA library.
 *
 * What it computes (per pixel, brute force over every primitive, no culling,
 * no tiles, no cache):
 *   1. ray of the pixel centre, ray-plane intersection and local (u, v)
 *      coordinates                                           -- Eq. 4, Eq. 5
 *   2. polar angle, sector k, relative angle, radial L2 term -- Eq. 6
 *   3. L1 norm through the inverse endpoint matrix           -- Eq. 7
 *   4. L1/L2 blend and exponential                           -- Eq. 8
 *   5. sharpening Psi                                        -- Eq. 9
 *   6. view-dependent low-pass filter (max)                  -- Eq. 10
 *   7. contributors sorted by ray depth r_t                  -- Eq. 13
 *   8. front-to-back alpha compositing                       -- Eq. 1
 * and the exact reverse-mode derivative of that image, evaluated
 * back-to-front over each pixel's sorted contributor list.
 *
 * Readings where the paper is silent or garbled (each one is stated where it
 * is used below):
 *   R1  the polar angle is atan2(v, u) on the full circle (Sec. 4.1 writes
 *       arccos, which only covers half of it); K angles theta_0..theta_{K-1}
 *       ascending with span < 2 pi, the last sector wraps to theta_0 + 2 pi
 *       with scale s_0; a point on theta_{k+1} belongs to sector k.
 *   R2  R_x, R_y, R_z are the columns of R(q) (Eq. 5 speaks of rows of R,
 *       i.e. the rows of R^T); q = (w, x, y, z) is normalised first.
 *   R3  camera: pinhole, x right / y down / z forward, pixel centres at +0.5;
 *       the ray direction has unit camera-space z, so r_t of Eq. 13 is the
 *       view-space depth of the intersection.  Skip a pair when the
 *       normalised ray is within 1e-7 of parallel to the plane or r_t <= near.
 *   R4  low-pass filter: r_d in Eq. 10 is normalised; Delta p is measured
 *       from the pinhole projection of mu (only when mu lies beyond the near
 *       plane); s_l is an option (0 = filter off); the max is taken after Psi.
 *   R5  alpha_tilde = min(max(alpha, filter), alpha_max); a pair contributes
 *       iff alpha_tilde >= alpha_min; compositing stops before the first
 *       contributor whose T (1 - alpha_tilde) would fall below T_min.
 *   R6  contributors are ordered by (r_t, primitive index).
 *   R7  colour: plain RGB, or real spherical harmonics of degree <= 3 in the
 *       view direction camera centre -> mu, plus 0.5, clamped below at 0.
 *   R8  background colour bg is added with the final transmittance.
 *   R10 cull_paper 1 applies the paper's tile culling as printed (Sec. 4.4,
 *       Eq. 11 - Eq. 12): a primitive reaches the pixels of a 16 x 16 tile only
 *       if the polygon of its basis endpoints at s_k sqrt(-log
 *       Psi^-1(alpha_min / o)) meets the tile, tested in the primitive's
 *       plane against the quad of the tile's corner pixel centres; tiles whose
 *       corner rays do not all meet the plane in front of the camera are kept.
 *   R9  order_mode 1 composites in the order of the paper's cache-sorting
 *       (Sec. 4.4 "Cache Sorting", supplementary Algorithm 1) instead of the
 *       exact order: pre-sort by centre depth, a cache of cache_len entries
 *       sorted by r_t whose smallest is composited when it overflows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORD_PI 3.14159265358979323846
#define ORD_TWO_PI (2.0 * ORD_PI)
#define ORD_MAXK 64

typedef struct {
    int64_t n;
    int K;
    int sh_degree;          /* -1: plain RGB */
    const double *mu;       /* n x 3 */
    const double *quat;     /* n x 4 (w, x, y, z) */
    const double *scale;    /* n x K */
    const double *theta;    /* n x K ascending */
    const double *eta;      /* n */
    const double *tau;      /* n */
    const double *opacity;  /* n */
    const double *color;    /* n x 3 or n x (deg+1)^2 x 3 */
} ord_params;

typedef struct {
    double *mu, *quat, *scale, *theta, *eta, *tau, *opacity, *color;
} ord_grads;

typedef struct {
    int width, height;
    double fx, fy, cx, cy;
    double w2c[12];         /* row-major 3 x 4 [R | t] */
} ord_camera;

typedef struct {
    double alpha_min, T_min, alpha_max, lowpass_sl, near_plane;
    double bg[3];
    int order_mode;         /* 0: exact (r_t, index) order; 1: the paper's cache-sorting */
    int cache_len;          /* cache length of order_mode 1 (the paper uses 8) */
    int cull_paper;         /* 1: the paper's endpoint-polygon tile culling (lossy), reading R10 */
} ord_options;

/* parity flags written per pixel by ord_render */
#define ORD_FLAG_ALPHA_MIN 1   /* some alpha_tilde within 1e-4 (rel) of alpha_min (informational) */
#define ORD_FLAG_T_MIN     2   /* a stop decision within FP32 margin and with visible effect */
#define ORD_FLAG_DEPTH_TIE 4   /* two contributors with near-equal depth and visible order effect */
#define ORD_FLAG_STEEP     8   /* float32 error of the alphas could exceed half the tolerance
                                  (near-hard edges: Psi's middle slope (1+tau)/(1-tau)) */
#define ORD_FLAG_KINK      32  /* a composited contributor within float32 rounding of a point where
                                  the derivative of its alpha_tilde changes branch (see branch_kink):
                                  images are continuous there, gradients take a side */
#define ORD_FLAG_CULL      16  /* a contributor whose paper-culling decision for the pixel's
                                  tile is within float32 margin */

/* ------------------------------------------------------------------------ */
/* Sharpening, Eq. 9, and its inverse (used by tests and by the culling
 * radius of Eq. 11).                                                        */

double ord_psi(double g, double tau)
{
    if (g < (1.0 + tau) / 4.0) return (1.0 - tau) / (1.0 + tau) * g;
    if (g < (3.0 - tau) / 4.0) return (1.0 + tau) / (1.0 - tau) * g - tau / (1.0 - tau);
    return (1.0 - tau) / (1.0 + tau) * g + 2.0 * tau / (1.0 + tau);
}

/* derivative of Psi with respect to g and to tau on the piece containing g */
static void psi_grad(double g, double tau, double *dg, double *dtau)
{
    double p = 1.0 + tau, m = 1.0 - tau;
    if (g < p / 4.0) {
        *dg = m / p;
        *dtau = -2.0 * g / (p * p);
    } else if (g < (3.0 - tau) / 4.0) {
        *dg = p / m;
        *dtau = 2.0 * g / (m * m) - 1.0 / (m * m);
    } else {
        *dg = m / p;
        *dtau = -2.0 * g / (p * p) + 2.0 / (p * p);
    }
}

/* inverse of Psi on [0, 1] (Psi is continuous and strictly increasing) */
double ord_psi_inv(double y, double tau)
{
    if (y < (1.0 - tau) / 4.0) return y * (1.0 + tau) / (1.0 - tau);
    if (y < (3.0 + tau) / 4.0) return (y * (1.0 - tau) + tau) / (1.0 + tau);
    return ((1.0 + tau) * y - 2.0 * tau) / (1.0 - tau);
}

/* ------------------------------------------------------------------------ */
/* Rotation from a quaternion (w, x, y, z), normalised first.  R is
 * row-major; its columns are R_x, R_y, R_z (reading R2).                   */

void ord_rotation(const double *q, double *R)
{
    double nrm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / nrm, x = q[1] / nrm, y = q[2] / nrm, z = q[3] / nrm;
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* gradient of a loss with respect to the (unnormalised) quaternion, given
 * its gradient with respect to the row-major R */
static void rotation_backward(const double *q, const double *dR, double *dq)
{
    double nrm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / nrm, x = q[1] / nrm, y = q[2] / nrm, z = q[3] / nrm;
    double gw = 0, gx = 0, gy = 0, gz = 0;
    /* R00 */ gy += -4 * y * dR[0]; gz += -4 * z * dR[0];
    /* R01 */ gw += -2 * z * dR[1]; gx += 2 * y * dR[1]; gy += 2 * x * dR[1]; gz += -2 * w * dR[1];
    /* R02 */ gw += 2 * y * dR[2]; gx += 2 * z * dR[2]; gy += 2 * w * dR[2]; gz += 2 * x * dR[2];
    /* R10 */ gw += 2 * z * dR[3]; gx += 2 * y * dR[3]; gy += 2 * x * dR[3]; gz += 2 * w * dR[3];
    /* R11 */ gx += -4 * x * dR[4]; gz += -4 * z * dR[4];
    /* R12 */ gw += -2 * x * dR[5]; gx += -2 * w * dR[5]; gy += 2 * z * dR[5]; gz += 2 * y * dR[5];
    /* R20 */ gw += -2 * y * dR[6]; gx += 2 * z * dR[6]; gy += -2 * w * dR[6]; gz += 2 * x * dR[6];
    /* R21 */ gw += 2 * x * dR[7]; gx += 2 * w * dR[7]; gy += 2 * z * dR[7]; gz += 2 * y * dR[7];
    /* R22 */ gx += -4 * x * dR[8]; gy += -4 * y * dR[8];
    double dotp = w * gw + x * gx + y * gy + z * gz;
    dq[0] = (gw - w * dotp) / nrm;
    dq[1] = (gx - x * dotp) / nrm;
    dq[2] = (gy - y * dotp) / nrm;
    dq[3] = (gz - z * dotp) / nrm;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3 (reading R7), written as
 * polynomials in the unit direction (x, y, z).  Index l*l + l + m,
 * m = -l..l.  Convention: y_lm = sqrt(2) Im Y_l^|m| (m < 0), Y_l^0 (m = 0),
 * sqrt(2) Re Y_l^m (m > 0), with Y_l^m carrying the Condon-Shortley phase.
 * Normalisation constants are written in closed form.                      */

void ord_sh_basis(int degree, const double *d, double *Y)
{
    double x = d[0], y = d[1], z = d[2];
    Y[0] = 0.5 * sqrt(1.0 / ORD_PI);
    if (degree < 1) return;
    double c1 = sqrt(3.0 / (4.0 * ORD_PI));
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    if (degree < 2) return;
    double a = 0.5 * sqrt(15.0 / ORD_PI), b = 0.25 * sqrt(5.0 / ORD_PI), c = 0.25 * sqrt(15.0 / ORD_PI);
    Y[4] = a * x * y;
    Y[5] = -a * y * z;
    Y[6] = b * (2.0 * z * z - x * x - y * y);
    Y[7] = -a * x * z;
    Y[8] = c * (x * x - y * y);
    if (degree < 3) return;
    double e = 0.25 * sqrt(35.0 / (2.0 * ORD_PI)), f = 0.5 * sqrt(105.0 / ORD_PI);
    double h = 0.25 * sqrt(21.0 / (2.0 * ORD_PI)), k = 0.25 * sqrt(7.0 / ORD_PI), l = 0.25 * sqrt(105.0 / ORD_PI);
    Y[9] = -e * y * (3.0 * x * x - y * y);
    Y[10] = f * x * y * z;
    Y[11] = -h * y * (4.0 * z * z - x * x - y * y);
    Y[12] = k * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -h * x * (4.0 * z * z - x * x - y * y);
    Y[14] = l * z * (x * x - y * y);
    Y[15] = -e * x * (x * x - 3.0 * y * y);
}

/* gradient of each basis polynomial with respect to (x, y, z): G[3*j + c] */
static void sh_basis_grad(int degree, const double *d, double *G)
{
    double x = d[0], y = d[1], z = d[2];
    memset(G, 0, sizeof(double) * 48);
    if (degree < 1) return;
    double c1 = sqrt(3.0 / (4.0 * ORD_PI));
    G[3 * 1 + 1] = -c1;
    G[3 * 2 + 2] = c1;
    G[3 * 3 + 0] = -c1;
    if (degree < 2) return;
    double a = 0.5 * sqrt(15.0 / ORD_PI), b = 0.25 * sqrt(5.0 / ORD_PI), c = 0.25 * sqrt(15.0 / ORD_PI);
    G[3 * 4 + 0] = a * y;  G[3 * 4 + 1] = a * x;
    G[3 * 5 + 1] = -a * z; G[3 * 5 + 2] = -a * y;
    G[3 * 6 + 0] = -2.0 * b * x; G[3 * 6 + 1] = -2.0 * b * y; G[3 * 6 + 2] = 4.0 * b * z;
    G[3 * 7 + 0] = -a * z; G[3 * 7 + 2] = -a * x;
    G[3 * 8 + 0] = 2.0 * c * x; G[3 * 8 + 1] = -2.0 * c * y;
    if (degree < 3) return;
    double e = 0.25 * sqrt(35.0 / (2.0 * ORD_PI)), f = 0.5 * sqrt(105.0 / ORD_PI);
    double h = 0.25 * sqrt(21.0 / (2.0 * ORD_PI)), k = 0.25 * sqrt(7.0 / ORD_PI), l = 0.25 * sqrt(105.0 / ORD_PI);
    /* Y9 = -e (3 x^2 y - y^3) */
    G[3 * 9 + 0] = -e * 6.0 * x * y; G[3 * 9 + 1] = -e * (3.0 * x * x - 3.0 * y * y);
    /* Y10 = f x y z */
    G[3 * 10 + 0] = f * y * z; G[3 * 10 + 1] = f * x * z; G[3 * 10 + 2] = f * x * y;
    /* Y11 = -h (4 y z^2 - x^2 y - y^3) */
    G[3 * 11 + 0] = -h * (-2.0 * x * y);
    G[3 * 11 + 1] = -h * (4.0 * z * z - x * x - 3.0 * y * y);
    G[3 * 11 + 2] = -h * (8.0 * y * z);
    /* Y12 = k (2 z^3 - 3 x^2 z - 3 y^2 z) */
    G[3 * 12 + 0] = k * (-6.0 * x * z); G[3 * 12 + 1] = k * (-6.0 * y * z);
    G[3 * 12 + 2] = k * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    /* Y13 = -h (4 x z^2 - x^3 - x y^2) */
    G[3 * 13 + 0] = -h * (4.0 * z * z - 3.0 * x * x - y * y);
    G[3 * 13 + 1] = -h * (-2.0 * x * y);
    G[3 * 13 + 2] = -h * (8.0 * x * z);
    /* Y14 = l (x^2 z - y^2 z) */
    G[3 * 14 + 0] = l * 2.0 * x * z; G[3 * 14 + 1] = -l * 2.0 * y * z; G[3 * 14 + 2] = l * (x * x - y * y);
    /* Y15 = -e (x^3 - 3 x y^2) */
    G[3 * 15 + 0] = -e * (3.0 * x * x - 3.0 * y * y); G[3 * 15 + 1] = -e * (-6.0 * x * y);
}

/* ------------------------------------------------------------------------ */
/* Camera helpers (reading R3). */

static void cam_center(const ord_camera *c, double *o)
{
    const double *M = c->w2c;
    /* o = -R^T t */
    for (int i = 0; i < 3; i++)
        o[i] = -(M[0 * 4 + i] * M[3] + M[1 * 4 + i] * M[7] + M[2 * 4 + i] * M[11]);
}

/* world-space ray direction of pixel (px, py); camera-space z component 1 */
static void cam_ray(const ord_camera *c, int px, int py, double *d)
{
    const double *M = c->w2c;
    double dc[3] = {(px + 0.5 - c->cx) / c->fx, (py + 0.5 - c->cy) / c->fy, 1.0};
    for (int i = 0; i < 3; i++)
        d[i] = M[0 * 4 + i] * dc[0] + M[1 * 4 + i] * dc[1] + M[2 * 4 + i] * dc[2];
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------------ */
/* Kernel function in local (u, v) coordinates: Eq. 6 - Eq. 9.  Everything
 * the derivative needs is kept in this record.                             */

typedef struct {
    int k, k1;                  /* sector (k, k+1 mod K) */
    double r2sq, phi, th_k, th_k1, gap, dtheta, c, Q;
    double a, b, r1, E, g, psi, alpha;
    double Minv[4];             /* inverse of [e_k e_{k+1}], row-major */
} kernel_eval;

static void kernel_uv(int K, const double *s, const double *th, double eta, double tau, double o,
                      double u, double v, kernel_eval *ke)
{
    ke->r2sq = u * u + v * v;
    /* reading R1: full-circle polar angle reduced into [theta_0, theta_0 + 2 pi) */
    double phi = atan2(v, u);
    double rel = fmod(phi - th[0], ORD_TWO_PI);
    if (rel < 0.0) rel += ORD_TWO_PI;
    phi = th[0] + rel;
    int k = 0;
    for (int j = 1; j < K; j++)
        if (th[j] < phi) k = j;
    int k1 = (k + 1) % K;
    double th_k = th[k];
    double th_k1 = (k + 1 < K) ? th[k + 1] : th[0] + ORD_TWO_PI;
    ke->k = k; ke->k1 = k1; ke->phi = phi; ke->th_k = th_k; ke->th_k1 = th_k1;
    ke->gap = th_k1 - th_k;
    /* Eq. 6: relative angle and cosine-weighted inverse squared radius */
    ke->dtheta = (phi - th_k) * ORD_PI / ke->gap;
    ke->c = cos(ke->dtheta);
    ke->Q = (1.0 + ke->c) / (2.0 * s[k] * s[k]) + (1.0 - ke->c) / (2.0 * s[k1] * s[k1]);
    /* Eq. 7: L1 norm of the coordinates in the basis of the two endpoints */
    double e0x = s[k] * cos(th_k), e0y = s[k] * sin(th_k);
    double e1x = s[k1] * cos(th_k1), e1y = s[k1] * sin(th_k1);
    double det = e0x * e1y - e1x * e0y;
    ke->Minv[0] = e1y / det;  ke->Minv[1] = -e1x / det;
    ke->Minv[2] = -e0y / det; ke->Minv[3] = e0x / det;
    ke->a = ke->Minv[0] * u + ke->Minv[1] * v;
    ke->b = ke->Minv[2] * u + ke->Minv[3] * v;
    ke->r1 = fabs(ke->a) + fabs(ke->b);
    /* Eq. 8: blend and exponential */
    ke->E = eta * ke->r1 * ke->r1 + (1.0 - eta) * ke->r2sq * ke->Q;
    ke->g = exp(-0.5 * ke->E);
    /* Eq. 9 */
    ke->psi = ord_psi(ke->g, tau);
    ke->alpha = o * ke->psi;
}

double ord_kernel_uv(int K, const double *s, const double *th, double eta, double tau, double o,
                     double u, double v)
{
    kernel_eval ke;
    kernel_uv(K, s, th, eta, tau, o, u, v, &ke);
    return ke.alpha;
}

double ord_l1_norm(int K, const double *s, const double *th, double u, double v)
{
    kernel_eval ke;
    kernel_uv(K, s, th, 0.0, 0.0, 1.0, u, v, &ke);
    return ke.r1;
}

/* ------------------------------------------------------------------------ */
/* One (pixel, primitive) pair: geometry (Eq. 4, 5), kernel (Eq. 6-9),
 * filter (Eq. 10), clamp and threshold (reading R5).                       */

typedef struct {
    int valid;                  /* ray meets the plane in front of the near plane */
    double t, u, v;
    double R[9], m[3], d[3], dn, p[3];
    kernel_eval ke;
    int filt_on;                /* filter evaluated */
    double filt, dpx, dpy, cosv, dp2, muc[3];
    int use_filter;             /* alpha_tilde taken from the filter */
    int clamped;                /* alpha_tilde clamped to alpha_max */
    double alpha_tilde;
} pair_eval;

static void eval_pair(const ord_params *P, int64_t i, const ord_camera *cam, const ord_options *opt,
                      const double *ocam, int px, int py, pair_eval *pe)
{
    memset(pe, 0, sizeof(*pe));
    int K = P->K;
    ord_rotation(P->quat + 4 * i, pe->R);
    const double *mu = P->mu + 3 * i;
    double Rx[3] = {pe->R[0], pe->R[3], pe->R[6]};
    double Ry[3] = {pe->R[1], pe->R[4], pe->R[7]};
    double Rz[3] = {pe->R[2], pe->R[5], pe->R[8]};
    cam_ray(cam, px, py, pe->d);
    for (int c = 0; c < 3; c++) pe->m[c] = mu[c] - ocam[c];
    pe->dn = dot3(pe->d, Rz);
    double dnorm = sqrt(dot3(pe->d, pe->d));
    if (fabs(pe->dn) < 1e-7 * dnorm) return;                 /* reading R3 */
    /* Eq. 4 (ray depth r_t of Eq. 13) */
    pe->t = dot3(pe->m, Rz) / pe->dn;
    if (!(pe->t > opt->near_plane)) return;
    pe->valid = 1;
    /* Eq. 5: p = i - mu with i = o + t d */
    for (int c = 0; c < 3; c++) pe->p[c] = pe->t * pe->d[c] - pe->m[c];
    pe->u = dot3(Rx, pe->p);
    pe->v = dot3(Ry, pe->p);
    double o = P->opacity[i];
    kernel_uv(K, P->scale + (int64_t)K * i, P->theta + (int64_t)K * i, P->eta[i], P->tau[i], o,
              pe->u, pe->v, &pe->ke);
    double at = pe->ke.alpha;
    /* Eq. 10 (reading R4) */
    const double *M = cam->w2c;
    for (int r = 0; r < 3; r++)
        pe->muc[r] = M[r * 4 + 0] * mu[0] + M[r * 4 + 1] * mu[1] + M[r * 4 + 2] * mu[2] + M[r * 4 + 3];
    if (opt->lowpass_sl > 0.0 && pe->muc[2] > opt->near_plane) {
        pe->filt_on = 1;
        double prx = cam->fx * pe->muc[0] / pe->muc[2] + cam->cx;
        double pry = cam->fy * pe->muc[1] / pe->muc[2] + cam->cy;
        pe->dpx = px + 0.5 - prx;
        pe->dpy = py + 0.5 - pry;
        pe->dp2 = pe->dpx * pe->dpx + pe->dpy * pe->dpy;
        pe->cosv = fabs(pe->dn) / dnorm;
        double sl = opt->lowpass_sl;
        pe->filt = o * exp(-pe->dp2 / (2.0 * pe->cosv * pe->cosv * sl * sl));
        if (pe->filt > at) { at = pe->filt; pe->use_filter = 1; }
    }
    if (at > opt->alpha_max) { at = opt->alpha_max; pe->clamped = 1; }
    pe->alpha_tilde = at;
}

int ord_pair(const ord_params *P, int64_t i, const ord_camera *cam, const ord_options *opt,
             int px, int py, double *alpha_tilde, double *t)
{
    double ocam[3];
    cam_center(cam, ocam);
    pair_eval pe;
    eval_pair(P, i, cam, opt, ocam, px, py, &pe);
    *alpha_tilde = pe.valid ? pe.alpha_tilde : 0.0;
    *t = pe.t;
    return pe.valid;
}

/* colour of primitive i seen from the camera centre (reading R7) */
static int ncoef_of(int deg) { return deg < 0 ? 1 : (deg + 1) * (deg + 1); }

static void prim_color(const ord_params *P, int64_t i, const double *ocam, double *rgb, int *clamped)
{
    if (P->sh_degree < 0) {
        for (int c = 0; c < 3; c++) { rgb[c] = P->color[3 * i + c]; clamped[c] = 0; }
        return;
    }
    int nc = ncoef_of(P->sh_degree);
    const double *sh = P->color + (int64_t)3 * nc * i;
    double dir[3];
    for (int c = 0; c < 3; c++) dir[c] = P->mu[3 * i + c] - ocam[c];
    double nr = sqrt(dot3(dir, dir));
    for (int c = 0; c < 3; c++) dir[c] /= nr;
    double Y[16];
    ord_sh_basis(P->sh_degree, dir, Y);
    for (int c = 0; c < 3; c++) {
        double acc = 0.5;
        for (int j = 0; j < nc; j++) acc += sh[3 * j + c] * Y[j];
        clamped[c] = acc < 0.0;
        rgb[c] = acc < 0.0 ? 0.0 : acc;
    }
}

void ord_color(const ord_params *P, int64_t i, const ord_camera *cam, double *rgb)
{
    double ocam[3];
    int cl[3];
    cam_center(cam, ocam);
    prim_color(P, i, ocam, rgb, cl);
}

/* ------------------------------------------------------------------------ */
/* Per-pixel contributor list, sorted by (r_t, index) -- Eq. 13, reading R6 */

typedef struct {
    double t;
    int64_t idx;
    double alpha, dalpha;   /* alpha_tilde and its float32 error model */
    int cull_und;           /* the paper's culling decision is within float32 margin */
    int kink;               /* alpha_tilde within float32 rounding of a branch point (branch_kink) */
} contrib;

/* Rounding-error model of a float32 evaluation of alpha_tilde.  It decides
 * nothing in the rendered image; it only bounds how far a float32
 * evaluation of the pair may land from this one, to set the parity budget
 * of a pixel.  First-order error propagation, where the sensitivities are
 * taken from the kernel itself by re-evaluating it (FP64) at perturbed
 * inputs:
 *   - the plane coordinates (u, v) of Eq. 5 carry a relative error d_r of
 *     about 2e-6 (a float32 product and sum of quantities of the size of
 *     the camera distance that cancel down to r_2), plus, near grazing
 *     incidence, t |d| 1.2e-7 / (cos r_2): one float32 rounding of the ray
 *     direction moves the ray-plane intersection of Eq. 4 by t |d| 1.2e-7 /
 *     cos, cos being the cosine between the ray and the plane normal;
 *     (u, v) is moved by d_r radially and turned by d_r + 5e-7 rad (the
 *     polar angle adds the rounding of atan2 and of theta_k - theta_0, a
 *     few half-ulps of 2 pi);
 *   - the sector endpoints theta_k, theta_k+1 carry 5e-7 rad and the
 *     scales s_k, s_k+1 a relative 3e-7 (their float32 trigonometry and
 *     products); narrow sectors amplify both through pi / gap (Eq. 6) and
 *     the inverse endpoint matrix (Eq. 7), which is why they are measured
 *     on the kernel and not estimated;
 *   - the exponent E of Eq. 8 itself carries 4e-6 (1 + E) from its own
 *     rounding, the cosine and the exponential: o Psi'(g) g dE / 2;
 *   - the affine pieces of Eq. 9 and the product with o round a few times
 *     more: 3e-7 alpha (this dominates on the flat pieces of Psi).
 * The perturbed kernels are re-evaluated in the sector each point falls
 * in; Eq. 6 - Eq. 7 are continuous across sectors.  For the filter of
 * Eq. 10 the exponent carries 4e-6 (1 + 2 X_f) / 2 plus the grazing term.
 * A clamped alpha has no error.                                            */
/* float32 error of the filter branch of Eq. 10 (see above) */
static double filter_alpha_err(const pair_eval *pe, double o)
{
    double Xf = -log(pe->filt / o);
    return pe->filt * (0.5 * 4e-6 * (1.0 + 2.0 * Xf) + Xf * 2.4e-7 / pe->cosv);
}

/* float32 error of the kernel branch (Eq. 6 - Eq. 9, see above); *dg gets
 * the matching bound on g of Eq. 8 (the same perturbations, measured on g) */
static double kernel_alpha_err(const ord_params *P, int64_t i, const pair_eval *pe, double *dg)
{
    const double tau = P->tau[i], o = P->opacity[i];
    double dnorm = sqrt(dot3(pe->d, pe->d));
    double cosv = fabs(pe->dn) / dnorm;
    const int K = P->K;
    const double *s0 = P->scale + (int64_t)K * i, *th0 = P->theta + (int64_t)K * i;
    const double eta = P->eta[i];
    const double a0 = pe->ke.alpha, g0 = pe->ke.g;
    double dpsi, dtau;
    psi_grad(pe->ke.g, tau, &dpsi, &dtau);
    double err = o * dpsi * pe->ke.g * 0.5 * 4e-6 * (1.0 + pe->ke.E) + 3e-7 * a0;
    double errg = pe->ke.g * 0.5 * 4e-6 * (1.0 + pe->ke.E);
    double r2 = sqrt(pe->ke.r2sq);
    if (r2 <= 0.0) {
        *dg = errg;
        return err;
    }
    const double d_r = 2e-6 + (pe->t * dnorm / r2) * 1.2e-7 / cosv;
    const double d_phi = d_r + 5e-7;
    double s[ORD_MAXK], th[ORD_MAXK];
    memcpy(s, s0, sizeof(double) * (size_t)K);
    memcpy(th, th0, sizeof(double) * (size_t)K);
    kernel_eval ke;
    double worst, worstg;
    /* radial */
    worst = worstg = 0.0;
    for (int sg = -1; sg <= 1; sg += 2) {
        const double f = 1.0 + sg * d_r;
        kernel_uv(K, s, th, eta, tau, o, pe->u * f, pe->v * f, &ke);
        worst = fmax(worst, fabs(ke.alpha - a0));
        worstg = fmax(worstg, fabs(ke.g - g0));
    }
    err += worst;
    errg += worstg;
    /* angular */
    worst = worstg = 0.0;
    for (int sg = -1; sg <= 1; sg += 2) {
        const double c = cos(sg * d_phi), sn = sin(sg * d_phi);
        kernel_uv(K, s, th, eta, tau, o, c * pe->u - sn * pe->v, sn * pe->u + c * pe->v, &ke);
        worst = fmax(worst, fabs(ke.alpha - a0));
        worstg = fmax(worstg, fabs(ke.g - g0));
    }
    err += worst;
    errg += worstg;
    /* sector endpoints and scales of the pair's sector (each one alone;
     * angles stay ascending because every gap is far above 5e-7) */
    const int ks[2] = {pe->ke.k, pe->ke.k1};
    for (int e = 0; e < 2; e++) {
        const int k = ks[e];
        worst = worstg = 0.0;
        for (int sg = -1; sg <= 1; sg += 2) {
            th[k] = th0[k] + sg * 5e-7;
            kernel_uv(K, s, th, eta, tau, o, pe->u, pe->v, &ke);
            worst = fmax(worst, fabs(ke.alpha - a0));
            worstg = fmax(worstg, fabs(ke.g - g0));
        }
        th[k] = th0[k];
        err += worst;
        errg += worstg;
        worst = worstg = 0.0;
        for (int sg = -1; sg <= 1; sg += 2) {
            s[k] = s0[k] * (1.0 + sg * 3e-7);
            kernel_uv(K, s, th, eta, tau, o, pe->u, pe->v, &ke);
            worst = fmax(worst, fabs(ke.alpha - a0));
            worstg = fmax(worstg, fabs(ke.g - g0));
        }
        s[k] = s0[k];
        err += worst;
        errg += worstg;
    }
    *dg = errg;
    return err;
}

static double alpha_fp32_error(const ord_params *P, int64_t i, const pair_eval *pe)
{
    if (pe->clamped) return 0.0;
    if (pe->use_filter) return filter_alpha_err(pe, P->opacity[i]);
    double dg;
    return kernel_alpha_err(P, i, pe, &dg);
}

/* Does alpha_tilde of this contributing pair sit, within float32 rounding,
 * at a point where its derivative changes branch?  Four such points:
 *   - g of Eq. 8 at a breakpoint of Psi (Eq. 9), g = (1 + tau)/4 or
 *     (3 - tau)/4, while the kernel sets alpha_tilde: Psi is continuous
 *     there but its slope jumps from (1 - tau)/(1 + tau) to its inverse
 *     (a factor 40000 at tau = 0.99), and so do its tau derivatives;
 *   - the kernel and the filter equal in the max of Eq. 10;
 *   - max(kernel, filter) at the clamp alpha_max;
 *   - the polar angle at a sector boundary theta_k (Eq. 6 - Eq. 7).
 * The image is continuous at all four, so it needs no flag; the gradient
 * is not, and a float32 evaluation on the other side of the point is
 * equally right.  The margins are the float32 error models of g and of the
 * two alpha branches, plus the rounding of the breakpoints and of alpha_max
 * to float32.                                                              */
static int branch_kink(const ord_params *P, int64_t i, const pair_eval *pe, const ord_options *opt)
{
    const double tau = P->tau[i], o = P->opacity[i];
    double dg;
    const double dk = kernel_alpha_err(P, i, pe, &dg);
    const double ak = pe->ke.alpha;
    const double df = pe->filt_on && pe->filt > 0.0 ? filter_alpha_err(pe, o) : 0.0;
    const double af = pe->filt_on ? pe->filt : 0.0;
    const double raw = fmax(ak, af);
    const double draw = ak >= af ? dk : df;
    /* the clamp */
    if (fabs(raw - opt->alpha_max) <= draw + 1e-7 * opt->alpha_max) return 1;
    if (pe->clamped) return 0;
    /* the max of Eq. 10 */
    if (pe->filt_on && fabs(ak - af) <= dk + df + 1e-12) return 1;
    if (pe->use_filter) return 0;
    /* the breakpoints of Psi (no slope jump when tau = 0) */
    if (fabs(tau) > 1e-6) {
        const double g = pe->ke.g;
        const double b1 = 0.25 * (1.0 + tau), b2 = 0.25 * (3.0 - tau);
        if (fabs(g - b1) <= dg + 1e-7 * b1 || fabs(g - b2) <= dg + 1e-7 * b2) return 1;
    }
    /* a sector boundary: the polar angle within its float32 error (the
     * error model's angle term plus the endpoint's own 5e-7) of theta_k or
     * theta_k+1.  Eq. 6 - Eq. 7 are continuous there, but the L1 term
     * |a| + |b| changes basis and has a kink, and the angle derivatives
     * change sector.  Near the centre every angle is uncertain, but the
     * jump of the derivative shrinks with the radius: below 1e-3 of the
     * sector's smaller scale it is negligible and not flagged */
    const double r2 = sqrt(pe->ke.r2sq);
    const double *sc = P->scale + (int64_t)P->K * i;
    if (r2 > 1e-3 * fmin(sc[pe->ke.k], sc[pe->ke.k1])) {
        const double dnorm = sqrt(dot3(pe->d, pe->d));
        const double cosv = fabs(pe->dn) / dnorm;
        const double d_phi = 2e-6 + (pe->t * dnorm / r2) * 1.2e-7 / cosv + 5e-7 + 5e-7;
        if (pe->ke.phi - pe->ke.th_k <= d_phi || pe->ke.th_k1 - pe->ke.phi <= d_phi) return 1;
    }
    return 0;
}

/* A batch of (pixel, primitive) pairs: alpha_tilde (0 where the ray misses
 * the plane in front of the near plane), r_t, and the float32 error model
 * of alpha_tilde (alpha_fp32_error) -- so that tests can hold the model
 * against float32 evaluations.  pix: m x 2 (x, y).                          */
void ord_pairs(const ord_params *P, const ord_camera *cam, const ord_options *opt, int64_t m, const int64_t *idx,
               const int32_t *pix, double *alpha_tilde, double *t, double *dalpha, int32_t *valid)
{
    double ocam[3];
    cam_center(cam, ocam);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < m; q++) {
        pair_eval pe;
        const int64_t i = idx[q];
        eval_pair(P, i, cam, opt, ocam, pix[2 * q], pix[2 * q + 1], &pe);
        valid[q] = pe.valid;
        alpha_tilde[q] = pe.valid ? pe.alpha_tilde : 0.0;
        t[q] = pe.t;
        dalpha[q] = pe.valid ? alpha_fp32_error(P, i, &pe) : 0.0;
    }
}

static int contrib_cmp(const void *pa, const void *pb)
{
    const contrib *a = (const contrib *)pa, *b = (const contrib *)pb;
    if (a->t < b->t) return -1;
    if (a->t > b->t) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* view-space depth of the primitive centre (the pre-sort key of the paper's
 * cache-sorting study, "vanilla" 3D-GS ordering)                           */
static double centre_depth(const ord_params *P, const ord_camera *cam, int64_t i)
{
    const double *m = P->mu + 3 * i, *M = cam->w2c;
    return M[8] * m[0] + M[9] * m[1] + M[10] * m[2] + M[11];
}

typedef struct { double zc; int64_t idx; int64_t pos; } presort_key;

static int presort_cmp(const void *pa, const void *pb)
{
    const presort_key *a = (const presort_key *)pa, *b = (const presort_key *)pb;
    if (a->zc < b->zc) return -1;
    if (a->zc > b->zc) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* The paper's cache-sorting (Sec. 4.4 "Cache Sorting", supplementary
 * Algorithm 1) applied to the contributors of one pixel, which buf holds
 * sorted by (r_t, index): the pixel meets them in the order of the pre-sort
 * (keys: centre depth, index); each is inserted into a cache kept sorted by
 * (r_t, index); when the cache holds more than cache_len entries, its
 * smallest is composited (reading: Sec. 4.4 pops "the kernel with the
 * smallest r_t" once the array is full); at the end of the list the cache
 * is composited in order.  rank[j] is the (r_t, index) rank of buf[j]
 * (NULL: j itself).  Writes the compositing order to out.                  */
static void cache_sort_order(const contrib *buf, int64_t cnt, int cache_len, const presort_key *keys,
                             const int64_t *rank, int64_t *cache, contrib *out)
{
    int64_t nc = 0, no = 0;
    for (int64_t j = 0; j < cnt; j++) {
        int64_t q = keys[j].pos, w = nc++;
        int64_t rq = rank ? rank[q] : q;
        while (w > 0 && (rank ? rank[cache[w - 1]] : cache[w - 1]) > rq) { cache[w] = cache[w - 1]; w--; }
        cache[w] = q;
        if (nc > cache_len) {
            out[no++] = buf[cache[0]];
            for (int64_t l = 1; l < nc; l++) cache[l - 1] = cache[l];
            nc--;
        }
    }
    for (int64_t l = 0; l < nc; l++) out[no++] = buf[cache[l]];
}

/* colour of a compositing order (Eq. 1 with the T_min stop of reading R5) */
static void order_colour(const ord_params *P, const double *ocam, const ord_options *opt, const contrib *buf,
                         int64_t cnt, double *rgb)
{
    double T = 1.0;
    rgb[0] = rgb[1] = rgb[2] = 0.0;
    for (int64_t j = 0; j < cnt; j++) {
        double Tn = T * (1.0 - buf[j].alpha);
        if (Tn < opt->T_min) break;
        double cj[3];
        int cl[3];
        prim_color(P, buf[j].idx, ocam, cj, cl);
        for (int c = 0; c < 3; c++) rgb[c] += T * buf[j].alpha * cj[c];
        T = Tn;
    }
    for (int c = 0; c < 3; c++) rgb[c] += T * opt->bg[c];
}

static double max_abs_diff3(const double *a, const double *b);

/* Rewrites buf (sorted by (r_t, index)) in the cache-sorting order.
 * Returns 1 where float32 may take another order with a visible effect:
 * two neighbours in the pre-sort with centre depths within 1e-6
 * (relative), or two r_t within 2e-6 (relative), whose exchange moves the
 * colour by more than 5e-5.  Each tie is tested by re-running the cache
 * with the pair exchanged: an exchange changes which entries the cache
 * pops later, so its effect is not bounded by the two contributors alone.
 * Returns -1 on allocation failure.                                        */
static int cache_sort_pixel(const ord_params *P, const ord_camera *cam, const ord_options *opt,
                            const double *ocam, contrib *buf, int64_t cnt, double *tie_move)
{
    const int cache_len = opt->cache_len > 0 ? opt->cache_len : 8;
    presort_key *keys = (presort_key *)malloc(sizeof(presort_key) * (size_t)cnt);
    contrib *out = (contrib *)malloc(sizeof(contrib) * (size_t)cnt);
    int64_t *rank = (int64_t *)malloc(sizeof(int64_t) * (size_t)cnt);
    int64_t *cache = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cache_len + 1));
    int tie = 0;
    if (!keys || !out || !rank || !cache) {
        tie = -1;
        goto done;
    }
    for (int64_t j = 0; j < cnt; j++) {
        keys[j].zc = centre_depth(P, cam, buf[j].idx);
        keys[j].idx = buf[j].idx;
        keys[j].pos = j;
        rank[j] = j;
    }
    qsort(keys, (size_t)cnt, sizeof(presort_key), presort_cmp);
    double base[3], alt[3];
    cache_sort_order(buf, cnt, cache_len, keys, NULL, cache, out);
    order_colour(P, ocam, opt, out, cnt, base);
    for (int64_t j = 1; j < cnt; j++) {
        if (keys[j].zc - keys[j - 1].zc > 1e-6 * fabs(keys[j].zc)) continue;
        presort_key k = keys[j];
        keys[j] = keys[j - 1];
        keys[j - 1] = k;
        cache_sort_order(buf, cnt, cache_len, keys, NULL, cache, out);
        order_colour(P, ocam, opt, out, cnt, alt);
        if (max_abs_diff3(base, alt) > 5e-5) tie = 1;
        *tie_move = fmax(*tie_move, max_abs_diff3(base, alt));
        keys[j - 1] = keys[j];
        keys[j] = k;
    }
    for (int64_t j = 0; j < cnt; j++)
        for (int64_t l = j + 1; l < cnt && buf[l].t - buf[j].t <= 2e-6 * buf[l].t; l++) {
            rank[j] = l;
            rank[l] = j;
            cache_sort_order(buf, cnt, cache_len, keys, rank, cache, out);
            order_colour(P, ocam, opt, out, cnt, alt);
            if (max_abs_diff3(base, alt) > 5e-5) tie = 1;
            *tie_move = fmax(*tie_move, max_abs_diff3(base, alt));
            rank[j] = j;
            rank[l] = l;
        }
    cache_sort_order(buf, cnt, cache_len, keys, NULL, cache, out);
    memcpy(buf, out, sizeof(contrib) * (size_t)cnt);
done:
    free(keys);
    free(out);
    free(rank);
    free(cache);
    return tie;
}

/* Does the convex quad (qu, qv) meet the polygon (px, py) of K vertices,
 * star-shaped about the origin?  Either holds a vertex of the other (the
 * origin stands for the polygon), or two edges cross.                       */
static int quad_meets_polygon(const double *qu, const double *qv, const double *px, const double *py, int K)
{
    double pts[17][2];
    pts[0][0] = 0.0;
    pts[0][1] = 0.0;
    for (int k = 0; k < K; k++) {
        pts[k + 1][0] = px[k];
        pts[k + 1][1] = py[k];
    }
    for (int j = 0; j <= K; j++) {
        int pos = 0, neg = 0;
        for (int c = 0; c < 4; c++) {
            int n = (c + 1) & 3;
            double cr = (qu[n] - qu[c]) * (pts[j][1] - qv[c]) - (qv[n] - qv[c]) * (pts[j][0] - qu[c]);
            pos += cr > 0.0;
            neg += cr < 0.0;
        }
        if (pos == 0 || neg == 0) return 1;
    }
    for (int c = 0; c < 4; c++) {           /* even-odd rule, ray towards +u */
        int in = 0;
        for (int k = 0; k < K; k++) {
            int k1 = (k + 1) % K;
            if ((py[k] > qv[c]) != (py[k1] > qv[c])) {
                double xc = px[k] + (qv[c] - py[k]) * (px[k1] - px[k]) / (py[k1] - py[k]);
                if (qu[c] < xc) in = !in;
            }
        }
        if (in) return 1;
    }
    for (int k = 0; k < K; k++) {
        int k1 = (k + 1) % K;
        for (int c = 0; c < 4; c++) {
            int n = (c + 1) & 3;
            double d1 = (px[k1] - px[k]) * (qv[c] - py[k]) - (py[k1] - py[k]) * (qu[c] - px[k]);
            double d2 = (px[k1] - px[k]) * (qv[n] - py[k]) - (py[k1] - py[k]) * (qu[n] - px[k]);
            double d3 = (qu[n] - qu[c]) * (py[k] - qv[c]) - (qv[n] - qv[c]) * (px[k] - qu[c]);
            double d4 = (qu[n] - qu[c]) * (py[k1] - qv[c]) - (qv[n] - qv[c]) * (px[k1] - qu[c]);
            if (((d1 > 0.0) != (d2 > 0.0)) && ((d3 > 0.0) != (d4 > 0.0))) return 1;
        }
    }
    return 0;
}

/* The paper's tile culling (reading R10) for primitive i and the tile of
 * pixel (px, py).  Returns 1 to keep; *undecided is set when the decision
 * changes with the polygon scaled by 1 -+ delta (delta covers the float32
 * error of the corner mapping) or a corner ray is nearly parallel to the
 * plane.                                                                    */
static int paper_tile_keep(const ord_params *P, int64_t i, const ord_camera *cam, const ord_options *opt,
                           const double *ocam, int px, int py, int *undecided)
{
    *undecided = 0;
    const int K = P->K;
    const double o = P->opacity[i];
    if (o < opt->alpha_min) return 0;
    double R[9];
    ord_rotation(P->quat + 4 * i, R);
    const double Rx[3] = {R[0], R[3], R[6]}, Ry[3] = {R[1], R[4], R[7]}, Rz[3] = {R[2], R[5], R[8]};
    const double *mu = P->mu + 3 * i;
    double m[3];
    for (int c = 0; c < 3; c++) m[c] = mu[c] - ocam[c];
    const double mz = dot3(m, Rz);
    const int tx = px / 16, ty = py / 16;
    const int xs[2] = {tx * 16, (tx * 16 + 15 < cam->width - 1) ? tx * 16 + 15 : cam->width - 1};
    const int ys[2] = {ty * 16, (ty * 16 + 15 < cam->height - 1) ? ty * 16 + 15 : cam->height - 1};
    const int cx[4] = {xs[0], xs[1], xs[1], xs[0]}, cy[4] = {ys[0], ys[0], ys[1], ys[1]};
    double w[4], wmin = 1e300, wmax = -1e300, qu[4], qv[4], wabs = 0.0;
    for (int c = 0; c < 4; c++) {
        double d[3];
        cam_ray(cam, cx[c], cy[c], d);
        w[c] = dot3(d, Rz) / mz;                  /* 1 / r_t at the corner */
        wmin = fmin(wmin, w[c]);
        wmax = fmax(wmax, w[c]);
        wabs = fmax(wabs, fabs(w[c]));
        if (w[c] > 0.0) {
            double p[3];
            for (int r = 0; r < 3; r++) p[r] = d[r] / w[c] - m[r];
            qu[c] = dot3(p, Rx);
            qv[c] = dot3(p, Ry);
        }
    }
    if (wmax <= 0.0) return 0;
    if (fabs(wmin) <= 1e-5 * wabs) *undecided = 1;
    if (wmin <= 0.0) return 1;
    const double cl = sqrt(fmax(-log(ord_psi_inv(opt->alpha_min / o, P->tau[i])), 0.0));
    double pxs[16], pys[16], ext_p = 0.0, ext_q = 0.0;
    for (int k = 0; k < K; k++) {
        pxs[k] = cl * P->scale[K * i + k] * cos(P->theta[K * i + k]);
        pys[k] = cl * P->scale[K * i + k] * sin(P->theta[K * i + k]);
        ext_p = fmax(ext_p, hypot(pxs[k], pys[k]));
    }
    for (int c = 0; c < 4; c++) ext_q = fmax(ext_q, hypot(qu[c], qv[c]));
    const int keep = quad_meets_polygon(qu, qv, pxs, pys, K);
    const double delta = 1e-4 * fmax(1.0, ext_q / fmax(ext_p, 1e-300));
    double sx[16], sy[16];
    for (int sgn = -1; sgn <= 1; sgn += 2) {
        for (int k = 0; k < K; k++) {
            sx[k] = pxs[k] * (1.0 + sgn * delta);
            sy[k] = pys[k] * (1.0 + sgn * delta);
        }
        if (quad_meets_polygon(qu, qv, sx, sy, K) != keep) *undecided = 1;
    }
    return keep;
}

/* Contributors of pixel (px, py), sorted by (r_t, index) (or in the
 * cache-sorting order).  With the paper's culling, a contributor whose
 * culling decision is within float32 margin is marked (cull_und) when it
 * is kept, and copied to und (if not NULL) when it is culled.  In the
 * cache-sorting order *tie_move (if not NULL) gets the largest colour move
 * of a float32-undecidable exchange.                                      */
static int64_t gather_contributors(const ord_params *P, const ord_camera *cam, const ord_options *opt,
                                   const double *ocam, int px, int py, contrib *buf, int *near_amin,
                                   contrib *und, int64_t *n_und, double *tie_move)
{
    int64_t cnt = 0;
    *near_amin = 0;
    if (n_und) *n_und = 0;
    if (tie_move) *tie_move = 0.0;
    for (int64_t i = 0; i < P->n; i++) {
        pair_eval pe;
        eval_pair(P, i, cam, opt, ocam, px, py, &pe);
        if (!pe.valid) continue;
        int undecided = 0;
        if (opt->cull_paper) {
            const int keep = paper_tile_keep(P, i, cam, opt, ocam, px, py, &undecided);
            undecided = undecided && pe.alpha_tilde >= opt->alpha_min;
            if (undecided) *near_amin |= 4;
            if (!keep) {
                if (undecided && und) {
                    und[*n_und].t = pe.t;
                    und[*n_und].idx = i;
                    und[*n_und].alpha = pe.alpha_tilde;
                    und[*n_und].dalpha = 0.0;
                    und[*n_und].cull_und = 1;
                    und[*n_und].kink = 0;
                    (*n_und)++;
                }
                continue;
            }
        }
        if (fabs(pe.alpha_tilde / opt->alpha_min - 1.0) < 1e-4) *near_amin |= 1;
        if (pe.alpha_tilde >= opt->alpha_min) {
            buf[cnt].t = pe.t;
            buf[cnt].idx = i;
            buf[cnt].alpha = pe.alpha_tilde;
            buf[cnt].dalpha = alpha_fp32_error(P, i, &pe);
            buf[cnt].cull_und = undecided;
            buf[cnt].kink = branch_kink(P, i, &pe, opt);
            cnt++;
        }
    }
    qsort(buf, (size_t)cnt, sizeof(contrib), contrib_cmp);
    if (opt->order_mode == 1 && cnt > 0) {
        double move = 0.0;
        int r = cache_sort_pixel(P, cam, opt, ocam, buf, cnt, &move);
        if (r < 0) return -1;
        if (r) *near_amin |= 2;
        if (tie_move) *tie_move = move;
    }
    return cnt;
}

/* number of contributors composited before the T_min stop (reading R5) */
static int64_t composite_count(const contrib *buf, int64_t cnt, double T_min)
{
    double T = 1.0;
    for (int64_t j = 0; j < cnt; j++) {
        double Tn = T * (1.0 - buf[j].alpha);
        if (Tn < T_min) return j;
        T = Tn;
    }
    return cnt;
}

static double max_abs_diff3(const double *a, const double *b)
{
    double m = 0.0;
    for (int c = 0; c < 3; c++) {
        double d = fabs(a[c] - b[c]);
        if (d > m) m = d;
    }
    return m;
}

/* Render the listed pixels.  pix: npix x 2 (x, y).  Outputs per pixel:
 * rgb (npix x 3, includes T_final * bg), T_final, number of composited
 * contributors, parity flags, and tol (may be NULL): how far a float32
 * evaluation of the same pixel may legitimately land from this result
 * (colour units, any channel), the sum of
 *   - the alpha error model of every composited contributor and of the
 *     first one not composited, carried through Eq. 1: T_j dalpha_j 2 c_max;
 *   - for every stop decision within its float32 margin, the exact colour
 *     change if that decision went the other way (stop before j: the
 *     contributions of j .. last are replaced by the background; go on past
 *     the stop: one more contributor is composited);
 *   - for every pair of contributors with depths within 2e-6 (relative),
 *     the exact change of exchanging them when adjacent, T a_j a_l |c_j - c_l|;
 *   - in the cache-sorting order, the largest colour move of an exchange of
 *     a float32-undecidable pair (re-running the cache);
 *   - with the paper's culling, for a contributor whose culling decision
 *     is within float32 margin, T a 2 c_max (T at its depth).
 * Returns 0, or -1 on allocation failure.                                  */
int ord_render(const ord_params *P, const ord_camera *cam, const ord_options *opt, int64_t npix,
               const int32_t *pix, double *rgb, double *T_final, int32_t *n_contrib, int32_t *flags, double *tol)
{
    double ocam[3];
    cam_center(cam, ocam);
    int fail = 0;
    const size_t nb = (size_t)(P->n > 0 ? P->n : 1);
#pragma omp parallel
    {
        contrib *buf = (contrib *)malloc(sizeof(contrib) * nb);
        contrib *und = opt->cull_paper ? (contrib *)malloc(sizeof(contrib) * nb) : NULL;
        double *w = (double *)malloc(sizeof(double) * 4 * (nb + 1));   /* T_j a_j (c_j - bg), then T_j */
        if (!buf || !w || (opt->cull_paper && !und)) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < npix; q++) {
            if (!buf || !w || (opt->cull_paper && !und)) continue;
            int px = pix[2 * q], py = pix[2 * q + 1];
            int near_amin;
            int64_t n_und = 0;
            double tie_move = 0.0;
            int64_t cnt = gather_contributors(P, cam, opt, ocam, px, py, buf, &near_amin, und, &n_und, &tie_move);
            if (cnt < 0) {
#pragma omp atomic write
                fail = 1;
                continue;
            }
            int64_t nc = composite_count(buf, cnt, opt->T_min);
            double C[3] = {0, 0, 0}, T = 1.0;
            int flag = (near_amin & 1) ? ORD_FLAG_ALPHA_MIN : 0;
            if (near_amin & 2) flag |= ORD_FLAG_DEPTH_TIE;
            if (near_amin & 4) flag |= ORD_FLAG_CULL;
            double cmax = 1.0;
            for (int c = 0; c < 3; c++) cmax = fmax(cmax, fabs(opt->bg[c]));
            double dT_rel = 0.0;     /* float32 error estimate of T (relative) */
            double budget = 0.0;     /* float32 error estimate of the colour */
            double extra = tie_move; /* undecided stops, ties and culling decisions */
            for (int64_t j = 0; j <= nc && j < cnt; j++) {
                double cj[3];
                int cl[3];
                prim_color(P, buf[j].idx, ocam, cj, cl);
                double a = buf[j].alpha, da = buf[j].dalpha;
                double cm = fmax(cmax, fmax(fabs(cj[0]), fmax(fabs(cj[1]), fabs(cj[2]))));
                for (int c = 0; c < 3; c++) w[4 * j + c] = T * a * (cj[c] - opt->bg[c]);
                w[4 * j + 3] = 0.0;      /* marks an undecided stop before j */
                /* a stop decision within the float32 error of T (1 - alpha)
                 * whose flip would move the colour by more than 5e-5 */
                double rel = fabs(T * (1.0 - a) / opt->T_min - 1.0);
                double margin = 3.0 * (dT_rel + da / (1.0 - a)) + 1e-6;
                if (opt->T_min > 0.0 && rel < margin) {
                    if (T * a * max_abs_diff3(cj, opt->bg) > 5e-5) flag |= ORD_FLAG_T_MIN;
                    w[4 * j + 3] = 1.0;
                }
                budget += T * da * 2.0 * cm;
                if (j == nc) break;
                if (buf[j].kink) flag |= ORD_FLAG_KINK;
                if (buf[j].cull_und) extra += T * a * 2.0 * cm;
                /* near-equal depths whose swap is visible */
                for (int64_t l = j + 1; opt->order_mode == 0 && l < cnt && buf[l].t - buf[j].t <= 2e-6 * buf[l].t; l++) {
                    double cl_rgb[3];
                    int cl2[3];
                    prim_color(P, buf[l].idx, ocam, cl_rgb, cl2);
                    const double sw = T * a * buf[l].alpha * max_abs_diff3(cj, cl_rgb);
                    if (sw > 5e-5) flag |= ORD_FLAG_DEPTH_TIE;
                    extra += sw;
                }
                dT_rel += da / (1.0 - a) + 1e-7;
                for (int c = 0; c < 3; c++) C[c] += T * a * cj[c];
                T *= 1.0 - a;
            }
            /* undecided stops: stopping before j < nc drops j .. nc-1 (their
             * colour replaced by the background); going on past nc adds nc */
            double suffix[3] = {0.0, 0.0, 0.0};
            for (int64_t j = (nc < cnt ? nc : cnt - 1); j >= 0; j--) {
                if (j < nc)
                    for (int c = 0; c < 3; c++) suffix[c] += w[4 * j + c];
                if (w[4 * j + 3] != 0.0) {
                    const double zero[3] = {0.0, 0.0, 0.0};
                    extra += j < nc ? max_abs_diff3(suffix, zero)
                                    : fmax(fabs(w[4 * j]), fmax(fabs(w[4 * j + 1]), fabs(w[4 * j + 2])));
                }
            }
            /* culled contributors whose culling decision is undecided */
            for (int64_t u = 0; u < n_und; u++) {
                double Tu = 1.0;
                for (int64_t j = 0; j < nc && contrib_cmp(&buf[j], &und[u]) < 0; j++) Tu *= 1.0 - buf[j].alpha;
                double cu[3];
                int cl[3];
                prim_color(P, und[u].idx, ocam, cu, cl);
                const double cm = fmax(cmax, fmax(fabs(cu[0]), fmax(fabs(cu[1]), fabs(cu[2]))));
                extra += Tu * und[u].alpha * 2.0 * cm;
            }
            if (budget > 1e-4) flag |= ORD_FLAG_STEEP;
            for (int c = 0; c < 3; c++) rgb[3 * q + c] = C[c] + T * opt->bg[c];
            if (T_final) T_final[q] = T;
            if (n_contrib) n_contrib[q] = (int32_t)nc;
            if (flags) flags[q] = flag;
            if (tol) tol[q] = budget + extra;
        }
        free(buf);
        free(und);
        free(w);
    }
    return fail ? -1 : 0;
}

/* Depth and normal images of the listed pixels (supplementary "Converting
 * Mesh to DRK": rendered depth and normal images), composited with the
 * weights of the colour (Eq. 1): depth = sum_i T_i alpha_i r_t,i (r_t of
 * Eq. 13, the view depth) and normal = sum_i T_i alpha_i n_i, n_i the unit
 * normal R_z of primitive i's plane in camera coordinates, oriented towards
 * the camera (the side of the plane the camera is on).  Reading: the paper
 * shows these images without defining them; unnormalised sums (divide by
 * 1 - T_final for the mean over the covered part).  depth: npix, normal:
 * npix x 3.  Returns 0, or -1 on allocation failure.                        */
int ord_render_aux(const ord_params *P, const ord_camera *cam, const ord_options *opt, int64_t npix,
                   const int32_t *pix, double *depth, double *normal)
{
    double ocam[3];
    cam_center(cam, ocam);
    const double *M = cam->w2c;
    int fail = 0;
#pragma omp parallel
    {
        contrib *buf = (contrib *)malloc(sizeof(contrib) * (size_t)(P->n > 0 ? P->n : 1));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < npix; q++) {
            if (!buf) continue;
            int near_amin;
            int64_t cnt = gather_contributors(P, cam, opt, ocam, pix[2 * q], pix[2 * q + 1], buf, &near_amin, NULL, NULL, NULL);
            if (cnt < 0) {
#pragma omp atomic write
                fail = 1;
                continue;
            }
            int64_t nc = composite_count(buf, cnt, opt->T_min);
            double D = 0.0, N[3] = {0.0, 0.0, 0.0}, T = 1.0;
            for (int64_t j = 0; j < nc; j++) {
                const int64_t i = buf[j].idx;
                double R[9];
                ord_rotation(P->quat + 4 * i, R);
                double nw[3] = {R[2], R[5], R[8]}, nc3[3];
                for (int r = 0; r < 3; r++) nc3[r] = M[4 * r] * nw[0] + M[4 * r + 1] * nw[1] + M[4 * r + 2] * nw[2];
                /* the camera is on the side of the plane that n points to */
                double side = 0.0;
                for (int c = 0; c < 3; c++) side += nw[c] * (ocam[c] - P->mu[3 * i + c]);
                const double sg = side >= 0.0 ? 1.0 : -1.0;
                const double w = T * buf[j].alpha;
                D += w * buf[j].t;
                for (int c = 0; c < 3; c++) N[c] += w * sg * nc3[c];
                T *= 1.0 - buf[j].alpha;
            }
            depth[q] = D;
            for (int c = 0; c < 3; c++) normal[3 * q + c] = N[c];
        }
        free(buf);
    }
    return fail ? -1 : 0;
}

/* Sorted contributor list of one pixel (for inspection by tests).
 * Writes up to cap entries; returns the total count; *n_composited gets the
 * number composited before the stop.                                        */
int64_t ord_contributors(const ord_params *P, const ord_camera *cam, const ord_options *opt, int px, int py,
                         int64_t cap, int64_t *idx, double *t, double *alpha, int64_t *n_composited)
{
    double ocam[3];
    cam_center(cam, ocam);
    contrib *buf = (contrib *)malloc(sizeof(contrib) * (size_t)(P->n > 0 ? P->n : 1));
    if (!buf) return -1;
    int near_amin;
    int64_t cnt = gather_contributors(P, cam, opt, ocam, px, py, buf, &near_amin, NULL, NULL, NULL);
    if (cnt < 0) {
        free(buf);
        return -1;
    }
    for (int64_t j = 0; j < cnt && j < cap; j++) {
        idx[j] = buf[j].idx;
        t[j] = buf[j].t;
        alpha[j] = buf[j].alpha;
    }
    *n_composited = composite_count(buf, cnt, opt->T_min);
    free(buf);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode.  For one pair, given dL/d(alpha_tilde), accumulate the
 * gradient with respect to every DRK parameter of primitive i.  The chain
 * follows the forward steps above in reverse order.                        */

static void acc(double *dst, double v)
{
#pragma omp atomic update
    *dst += v;
}

static void pair_backward(const ord_params *P, int64_t i, const ord_camera *cam, const ord_options *opt,
                          const double *ocam, int px, int py, double g_at, ord_grads *G)
{
    pair_eval pe;
    eval_pair(P, i, cam, opt, ocam, px, py, &pe);
    if (!pe.valid || pe.clamped) return;
    int K = P->K;
    const double *s = P->scale + (int64_t)K * i;
    double o = P->opacity[i];
    double tau = P->tau[i], eta = P->eta[i];
    double dmu[3] = {0, 0, 0}, dR[9] = {0};
    const double *M = cam->w2c;

    if (pe.use_filter) {
        /* f = o exp(-dp2 / (2 cosv^2 sl^2)) */
        double sl = opt->lowpass_sl, f = pe.filt;
        acc(&G->opacity[i], g_at * f / o);
        double dQf = -g_at * f;                                  /* dL/dQf */
        double d_dp2 = dQf / (2.0 * pe.cosv * pe.cosv * sl * sl);
        double d_cos = dQf * (-pe.dp2 / (pe.cosv * pe.cosv * pe.cosv * sl * sl));
        /* projection of mu */
        double z = pe.muc[2];
        double dprx = -2.0 * pe.dpx * d_dp2, dpry = -2.0 * pe.dpy * d_dp2;
        double dmuc[3] = {dprx * cam->fx / z, dpry * cam->fy / z,
                          -dprx * cam->fx * pe.muc[0] / (z * z) - dpry * cam->fy * pe.muc[1] / (z * z)};
        for (int c = 0; c < 3; c++)
            dmu[c] += M[0 * 4 + c] * dmuc[0] + M[1 * 4 + c] * dmuc[1] + M[2 * 4 + c] * dmuc[2];
        /* cosv = |d . Rz| / |d| */
        double dnorm = sqrt(dot3(pe.d, pe.d));
        double sg = pe.dn >= 0.0 ? 1.0 : -1.0;
        for (int c = 0; c < 3; c++) dR[3 * c + 2] += d_cos * sg * pe.d[c] / dnorm;
    } else {
        kernel_eval *ke = &pe.ke;
        double dpsi_dg, dpsi_dtau;
        psi_grad(ke->g, tau, &dpsi_dg, &dpsi_dtau);
        acc(&G->opacity[i], g_at * ke->psi);
        acc(&G->tau[i], g_at * o * dpsi_dtau);
        double dE = -0.5 * ke->g * g_at * o * dpsi_dg;
        acc(&G->eta[i], dE * (ke->r1 * ke->r1 - ke->r2sq * ke->Q));
        double d_r1 = dE * 2.0 * eta * ke->r1;
        double d_r2sq = dE * (1.0 - eta) * ke->Q;
        double d_Q = dE * (1.0 - eta) * ke->r2sq;
        int k = ke->k, k1 = ke->k1;
        double *ds = G->scale + (int64_t)K * i, *dth = G->theta + (int64_t)K * i;
        /* Q = (1 + c)/(2 s_k^2) + (1 - c)/(2 s_k1^2) */
        double d_c = d_Q * (1.0 / (2.0 * s[k] * s[k]) - 1.0 / (2.0 * s[k1] * s[k1]));
        acc(&ds[k], d_Q * (1.0 + ke->c) * (-1.0 / (s[k] * s[k] * s[k])));
        acc(&ds[k1], d_Q * (1.0 - ke->c) * (-1.0 / (s[k1] * s[k1] * s[k1])));
        /* c = cos(dtheta), dtheta = (phi - th_k) pi / gap */
        double d_dth = -sin(ke->dtheta) * d_c;
        double gap = ke->gap;
        double d_phi = d_dth * ORD_PI / gap;
        acc(&dth[k], d_dth * ORD_PI * (ke->phi - ke->th_k1) / (gap * gap));
        acc(&dth[k1], d_dth * (-(ke->phi - ke->th_k) * ORD_PI / (gap * gap)));
        double du = 0.0, dv = 0.0;
        if (ke->r2sq > 0.0) {
            du += d_phi * (-pe.v / ke->r2sq);
            dv += d_phi * (pe.u / ke->r2sq);
        }
        du += d_r2sq * 2.0 * pe.u;
        dv += d_r2sq * 2.0 * pe.v;
        /* r1 = |a| + |b|, (a, b) = Minv (u, v) */
        double sa = ke->a > 0.0 ? 1.0 : (ke->a < 0.0 ? -1.0 : 0.0);
        double sb = ke->b > 0.0 ? 1.0 : (ke->b < 0.0 ? -1.0 : 0.0);
        double wx = ke->Minv[0] * sa + ke->Minv[2] * sb;   /* Minv^T (sa, sb) */
        double wy = ke->Minv[1] * sa + ke->Minv[3] * sb;
        du += d_r1 * wx;
        dv += d_r1 * wy;
        double ck = cos(ke->th_k), sk = sin(ke->th_k), ck1 = cos(ke->th_k1), sk1 = sin(ke->th_k1);
        acc(&ds[k], d_r1 * (-ke->a) * (wx * ck + wy * sk));
        acc(&dth[k], d_r1 * (-ke->a) * s[k] * (-wx * sk + wy * ck));
        acc(&ds[k1], d_r1 * (-ke->b) * (wx * ck1 + wy * sk1));
        acc(&dth[k1], d_r1 * (-ke->b) * s[k1] * (-wx * sk1 + wy * ck1));
        /* geometry: u = Rx . p, v = Ry . p, p = t d - m, t = (m . Rz)/(d . Rz) */
        double dp[3];
        for (int c = 0; c < 3; c++) {
            dR[3 * c + 0] += du * pe.p[c];
            dR[3 * c + 1] += dv * pe.p[c];
            dp[c] = du * pe.R[3 * c + 0] + dv * pe.R[3 * c + 1];
        }
        double dt = dot3(dp, pe.d);
        for (int c = 0; c < 3; c++) {
            double dm = -dp[c] + dt * pe.R[3 * c + 2] / pe.dn;
            dmu[c] += dm;
            dR[3 * c + 2] += -dt * pe.p[c] / pe.dn;
        }
    }
    for (int c = 0; c < 3; c++) acc(&G->mu[3 * i + c], dmu[c]);
    double dq[4];
    rotation_backward(P->quat + 4 * i, dR, dq);
    for (int c = 0; c < 4; c++) acc(&G->quat[4 * i + c], dq[c]);
}

static void color_backward(const ord_params *P, int64_t i, const double *ocam, const double *gc, ord_grads *G)
{
    if (P->sh_degree < 0) {
        for (int c = 0; c < 3; c++) acc(&G->color[3 * i + c], gc[c]);
        return;
    }
    int nc = ncoef_of(P->sh_degree);
    const double *sh = P->color + (int64_t)3 * nc * i;
    double dir[3];
    for (int c = 0; c < 3; c++) dir[c] = P->mu[3 * i + c] - ocam[c];
    double nr = sqrt(dot3(dir, dir));
    for (int c = 0; c < 3; c++) dir[c] /= nr;
    double Y[16], Gy[48];
    ord_sh_basis(P->sh_degree, dir, Y);
    sh_basis_grad(P->sh_degree, dir, Gy);
    double rgb_pre[3];
    for (int c = 0; c < 3; c++) {
        rgb_pre[c] = 0.5;
        for (int j = 0; j < nc; j++) rgb_pre[c] += sh[3 * j + c] * Y[j];
    }
    double ddir[3] = {0, 0, 0};
    for (int c = 0; c < 3; c++) {
        if (rgb_pre[c] < 0.0) continue;       /* clamped channel */
        for (int j = 0; j < nc; j++) {
            acc(&G->color[(int64_t)3 * nc * i + 3 * j + c], gc[c] * Y[j]);
            for (int a = 0; a < 3; a++) ddir[a] += gc[c] * sh[3 * j + c] * Gy[3 * j + a];
        }
    }
    double proj = dot3(ddir, dir);
    for (int a = 0; a < 3; a++) acc(&G->mu[3 * i + a], (ddir[a] - dir[a] * proj) / nr);
}

/* Gradient of L = sum_q dL_drgb[q] . rgb[q] over the listed pixels with
 * respect to every parameter (accumulated into G, which the caller zeroes).
 * Back-to-front over each pixel's composited contributors:
 *   dC/dc_j = T_j alpha_j,   dC/dalpha_j = T_j (c_j - B_j),
 * where B_j is the colour composited behind contributor j (bg behind the
 * last).  Returns 0, or -1 on allocation failure.                           */
int ord_render_backward(const ord_params *P, const ord_camera *cam, const ord_options *opt, int64_t npix,
                        const int32_t *pix, const double *dL_drgb, ord_grads *G)
{
    double ocam[3];
    cam_center(cam, ocam);
    int fail = 0;
#pragma omp parallel
    {
        contrib *buf = (contrib *)malloc(sizeof(contrib) * (size_t)(P->n > 0 ? P->n : 1));
        double *Tj = (double *)malloc(sizeof(double) * (size_t)(P->n > 0 ? P->n : 1));
        double *cj = (double *)malloc(sizeof(double) * 3 * (size_t)(P->n > 0 ? P->n : 1));
        if (!buf || !Tj || !cj) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < npix; q++) {
            if (!buf || !Tj || !cj) continue;
            int px = pix[2 * q], py = pix[2 * q + 1];
            const double *gC = dL_drgb + 3 * q;
            int near_amin;
            int64_t cnt = gather_contributors(P, cam, opt, ocam, px, py, buf, &near_amin, NULL, NULL, NULL);
            if (cnt < 0) {
#pragma omp atomic write
                fail = 1;
                continue;
            }
            int64_t nc = composite_count(buf, cnt, opt->T_min);
            double T = 1.0;
            for (int64_t j = 0; j < nc; j++) {
                int cl[3];
                Tj[j] = T;
                prim_color(P, buf[j].idx, ocam, cj + 3 * j, cl);
                T *= 1.0 - buf[j].alpha;
            }
            double B[3] = {opt->bg[0], opt->bg[1], opt->bg[2]};
            for (int64_t j = nc - 1; j >= 0; j--) {
                double a = buf[j].alpha;
                double gc[3], ga = 0.0;
                for (int c = 0; c < 3; c++) {
                    gc[c] = gC[c] * Tj[j] * a;
                    ga += gC[c] * Tj[j] * (cj[3 * j + c] - B[c]);
                }
                color_backward(P, buf[j].idx, ocam, gc, G);
                pair_backward(P, buf[j].idx, cam, opt, ocam, px, py, ga, G);
                for (int c = 0; c < 3; c++) B[c] = a * cj[3 * j + c] + (1.0 - a) * B[c];
            }
        }
        free(buf);
        free(Tj);
        free(cj);
    }
    return fail ? -1 : 0;
}

int ord_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ord_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
