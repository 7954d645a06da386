// preprocess.cu -- per-primitive preprocess, conservative tile culling and
// pair emission, and the per-primitive part of the backward pass.
//
// Sec. 4.4 ("Kernel Culling"): the paper bounds a DRK by its radial-basis
// endpoints at a calibrated length (Eq. 11, Eq. 12) and culls the tiles that
// the projected endpoint polygon misses.  That bound is not conservative
// (Eq. 11 omits the factor 2 of the Gaussian exponent, and the L2 contour
// bulges beyond the chord between endpoints), so this file uses a bound
// derived from the kernel itself:
//   - alpha = o Psi(g) >= alpha_min  <=>  g >= g* = Psi^-1(alpha_min / o)
//     <=> E <= E* = -2 ln g*  (Eq. 8, Eq. 9; Psi is increasing);
//   - in sector k, r1 >= r2 / max(s_k, s_k1) (triangle inequality on
//     a e_k + b e_k1) and 1/sbar^2 >= 1 / max(s_k, s_k1)^2, so E >= r2^2 /
//     max(s_k, s_k1)^2 and the support lies within radius
//     rho_k = sqrt(E*) max(s_k, s_k1) inside the sector;
//   - each sector is covered by a five-vertex tangent polygon, the
//     polygons are projected (their convex hull contains the support), and
//     the low-pass filter adds a disc of radius s_l sqrt(2 ln(o/alpha_min))
//     pixels around the projected centre (|cos| <= 1 in Eq. 10).
// The per-tile test maps the tile's pixel-centre rectangle into the plane
// with the primitive's homography and keeps the tile if the quad comes
// within rho_k of the centre inside the angular range of any sector it
// spans, or if the tile touches the filter disc.
#include "drk_internal.h"

namespace drk {

// ---------------------------------------------------------------------------
// real spherical harmonics, degree <= 3, closed-form constants.  Index
// l*l + l + m; y_lm = sqrt(2) Im Y_l^|m| (m < 0), Y_l^0, sqrt(2) Re Y_l^m
// (m > 0), with the Condon-Shortley phase.
namespace sh {
constexpr float C0 = (float)(0.5 * csqrt(1.0 / kPiD));
constexpr float C1 = (float)csqrt(3.0 / (4.0 * kPiD));
constexpr float C2a = (float)(0.5 * csqrt(15.0 / kPiD));
constexpr float C2b = (float)(0.25 * csqrt(5.0 / kPiD));
constexpr float C2c = (float)(0.25 * csqrt(15.0 / kPiD));
constexpr float C3a = (float)(0.25 * csqrt(35.0 / (2.0 * kPiD)));
constexpr float C3b = (float)(0.5 * csqrt(105.0 / kPiD));
constexpr float C3c = (float)(0.25 * csqrt(21.0 / (2.0 * kPiD)));
constexpr float C3d = (float)(0.25 * csqrt(7.0 / kPiD));
constexpr float C3e = (float)(0.25 * csqrt(105.0 / kPiD));
}  // namespace sh

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
    using namespace sh;
    Y[0] = C0;
    if (deg < 1) return;
    Y[1] = -C1 * y;
    Y[2] = C1 * z;
    Y[3] = -C1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = C2a * x * y;
    Y[5] = -C2a * y * z;
    Y[6] = C2b * (2.0f * zz - xx - yy);
    Y[7] = -C2a * x * z;
    Y[8] = C2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -C3a * y * (3.0f * xx - yy);
    Y[10] = C3b * x * y * z;
    Y[11] = -C3c * y * (4.0f * zz - xx - yy);
    Y[12] = C3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -C3c * x * (4.0f * zz - xx - yy);
    Y[14] = C3e * z * (xx - yy);
    Y[15] = -C3a * x * (xx - 3.0f * yy);
}

// d/d(x, y, z) of each basis polynomial, accumulated against weights w_j:
// out = sum_j w_j grad Y_j
__device__ __forceinline__ void sh_basis_vjp(int deg, float x, float y, float z, const float* w, float* out) {
    using namespace sh;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (deg >= 1) {
        gy += -C1 * w[1];
        gz += C1 * w[2];
        gx += -C1 * w[3];
    }
    if (deg >= 2) {
        gx += C2a * y * w[4];            gy += C2a * x * w[4];
        gy += -C2a * z * w[5];           gz += -C2a * y * w[5];
        gx += -2.f * C2b * x * w[6];     gy += -2.f * C2b * y * w[6];     gz += 4.f * C2b * z * w[6];
        gx += -C2a * z * w[7];           gz += -C2a * x * w[7];
        gx += 2.f * C2c * x * w[8];      gy += -2.f * C2c * y * w[8];
    }
    if (deg >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        gx += -C3a * 6.f * x * y * w[9];                 gy += -C3a * (3.f * xx - 3.f * yy) * w[9];
        gx += C3b * y * z * w[10];  gy += C3b * x * z * w[10];  gz += C3b * x * y * w[10];
        gx += C3c * 2.f * x * y * w[11];
        gy += -C3c * (4.f * zz - xx - 3.f * yy) * w[11];
        gz += -C3c * 8.f * y * z * w[11];
        gx += -C3d * 6.f * x * z * w[12];  gy += -C3d * 6.f * y * z * w[12];
        gz += C3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
        gx += -C3c * (4.f * zz - 3.f * xx - yy) * w[13];
        gy += C3c * 2.f * x * y * w[13];
        gz += -C3c * 8.f * x * z * w[13];
        gx += C3e * 2.f * x * z * w[14];  gy += -C3e * 2.f * y * z * w[14];  gz += C3e * (xx - yy) * w[14];
        gx += -C3a * (3.f * xx - 3.f * yy) * w[15];  gy += C3a * 6.f * x * y * w[15];
    }
    out[0] = gx; out[1] = gy; out[2] = gz;
}

// rotation matrix (row-major, columns R_x, R_y, R_z) of a normalised quaternion
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float* R) {
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ float dot3(const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Psi^-1 of Eq. 9 on [0, 1]
__device__ __forceinline__ float psi_inv(float y, float tau) {
    if (y < (1.f - tau) * 0.25f) return y * (1.f + tau) / (1.f - tau);
    if (y < (3.f + tau) * 0.25f) return (y * (1.f - tau) + tau) / (1.f + tau);
    return ((1.f + tau) * y - 2.f * tau) / (1.f - tau);
}

// Geometry shared by the forward preprocess and its backward.
struct PrimGeom {
    float qn[4], qnorm;
    float R[9];          // world rotation, columns Rx, Ry, Rz
    float muc[3];        // camera-space centre
    float Rxc[3], Ryc[3], nc[3];
    float c0, s0;        // cos / sin theta_0
    float Rxp[3], Ryp[3];// rotated-frame axes (camera space)
    float N, U0, V0;     // mu_c . n_c, Rx'. mu_c, Ry'. mu_c
};

__device__ __forceinline__ void prim_geom(const PreArgs& A, int64_t i, PrimGeom& G) {
    const float q0 = A.p.quat[4 * i], q1 = A.p.quat[4 * i + 1], q2 = A.p.quat[4 * i + 2], q3 = A.p.quat[4 * i + 3];
    G.qnorm = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float inv = 1.f / G.qnorm;
    G.qn[0] = q0 * inv; G.qn[1] = q1 * inv; G.qn[2] = q2 * inv; G.qn[3] = q3 * inv;
    quat_to_rot(G.qn[0], G.qn[1], G.qn[2], G.qn[3], G.R);
    const float* M = A.cam.w2c;
    const float mu[3] = {A.p.mu[3 * i], A.p.mu[3 * i + 1], A.p.mu[3 * i + 2]};
    for (int r = 0; r < 3; r++) {
        G.muc[r] = M[4 * r] * mu[0] + M[4 * r + 1] * mu[1] + M[4 * r + 2] * mu[2] + M[4 * r + 3];
        G.Rxc[r] = M[4 * r] * G.R[0] + M[4 * r + 1] * G.R[3] + M[4 * r + 2] * G.R[6];
        G.Ryc[r] = M[4 * r] * G.R[1] + M[4 * r + 1] * G.R[4] + M[4 * r + 2] * G.R[7];
        G.nc[r] = M[4 * r] * G.R[2] + M[4 * r + 1] * G.R[5] + M[4 * r + 2] * G.R[8];
    }
    const float th0 = A.p.theta[(int64_t)A.p.K * i];
    sincosf(th0, &G.s0, &G.c0);
    for (int r = 0; r < 3; r++) {
        G.Rxp[r] = G.c0 * G.Rxc[r] + G.s0 * G.Ryc[r];
        G.Ryp[r] = -G.s0 * G.Rxc[r] + G.c0 * G.Ryc[r];
    }
    G.N = dot3(G.muc, G.nc);
    G.U0 = dot3(G.Rxp, G.muc);
    G.V0 = dot3(G.Ryp, G.muc);
}

__device__ __forceinline__ void row_of(const PreArgs& A, const float* v, float* out) {
    out[0] = v[0] * A.fc.ifx;
    out[1] = v[1] * A.fc.ify;
    out[2] = v[0] * A.fc.ox + v[1] * A.fc.oy + v[2];
}

// ---------------------------------------------------------------------------
// K1: per-primitive preprocess.
template <int KMAX>
__global__ void __launch_bounds__(128) preprocess_kernel(PreArgs A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.p.n) return;
    const int K = A.p.K;
    float* rec = A.rec + (int64_t)Rec<KMAX>::STRIDE * i;
    float* bnd = A.bnd + (int64_t)Bnd<KMAX>::STRIDE * i;
    PrimGeom G;
    prim_geom(A, i, G);
    const float o = A.p.opacity[i];
    const float tau = A.p.tau[i];
    const float eta = A.p.eta[i];
    const float* th = A.p.theta + (int64_t)K * i;
    const float* s = A.p.scale + (int64_t)K * i;

    // homography rows in the rotated frame (Eq. 4, Eq. 5 per pixel)
    const bool plane_ok = fabsf(G.N) > 1e-20f;
    float Hrows[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (plane_ok) {
        const float al = G.U0 / G.N, be = G.V0 / G.N, invN = 1.f / G.N;
        float av[3], bv[3], mv[3];
        for (int r = 0; r < 3; r++) {
            av[r] = G.Rxp[r] - al * G.nc[r];
            bv[r] = G.Ryp[r] - be * G.nc[r];
            mv[r] = G.nc[r] * invN;
        }
        row_of(A, av, Hrows);
        row_of(A, bv, Hrows + 3);
        row_of(A, mv, Hrows + 6);
    }
    for (int j = 0; j < 9; j++) rec[j] = Hrows[j];
    rec[R_ETA2] = eta * (0.5f * kLog2e);
    rec[R_ETA2C] = (1.f - eta) * (0.5f * kLog2e);
    rec[R_OPA] = o;
    rec[R_B1] = (1.f + tau) * 0.25f;
    rec[R_B2] = (3.f - tau) * 0.25f;
    rec[R_SLO] = o * (1.f - tau) / (1.f + tau);
    rec[R_SMID] = o * (1.f + tau) / (1.f - tau);
    rec[R_OMID] = -o * tau / (1.f - tau);
    rec[R_OHI] = 2.f * o * tau / (1.f + tau);
    rec[R_TAU] = tau;

    // Eq. 10 low-pass filter
    const bool filt_on = A.sl > 0.f && G.muc[2] > A.fc.near_plane && plane_ok && o > 0.5f * A.fc.alpha_min;
    float fpx = 0.f, fpy = 0.f;
    if (filt_on) {
        fpx = A.cam.fx * G.muc[0] / G.muc[2] + A.cam.cx - 0.5f;
        fpy = A.cam.fy * G.muc[1] / G.muc[2] + A.cam.cy - 0.5f;
        rec[R_FPX] = fpx;
        rec[R_FPY] = fpy;
        rec[R_FCOEF] = kLog2e / (2.f * A.sl * A.sl * G.N * G.N);
        rec[R_FCUT] = log2f(2.f * o / A.fc.alpha_min);
    } else {
        rec[R_FPX] = 0.f; rec[R_FPY] = 0.f; rec[R_FCOEF] = 0.f; rec[R_FCUT] = -1.f;
    }

    // angles relative to theta_0 (sector thresholds, the K-th is 2 pi) and
    // the basis table e_j, A_j the evaluation forms sector constants from
    // (Eq. 6, Eq. 7)
    using RK = Rec<KMAX>;
    for (int j = 1; j <= KMAX; j++) rec[RK::TH + j - 1] = (j < K) ? th[j] - th[0] : (j == K ? kTwoPi : 1e30f);
    for (int j = 0; j < KMAX; j++) {
        if (j >= K) {
            rec[RK::EX + j] = 0.f; rec[RK::EY + j] = 0.f; rec[RK::AA + j] = 0.f;
            continue;
        }
        const float tj = (j == 0) ? 0.f : th[j] - th[0];
        float sn, cs;
        sincosf(tj, &sn, &cs);
        rec[RK::EX + j] = s[j] * cs;
        rec[RK::EY + j] = s[j] * sn;
        rec[RK::AA + j] = 1.f / (2.f * s[j] * s[j]);
    }

    // colour (Eq. 1's SH term), clamped below at 0
    float rgb[3];
    if (A.p.sh_degree < 0) {
        for (int c = 0; c < 3; c++) rgb[c] = A.p.color[3 * i + c];
    } else {
        const int nc = (A.p.sh_degree + 1) * (A.p.sh_degree + 1);
        float d[3];
        for (int c = 0; c < 3; c++) d[c] = A.p.mu[3 * i + c] - A.cam_center[c];
        const float inv = rsqrtf(dot3(d, d));
        float Y[16];
        sh_basis(A.p.sh_degree, d[0] * inv, d[1] * inv, d[2] * inv, Y);
        const float* shc = A.p.color + (int64_t)3 * nc * i;
        for (int c = 0; c < 3; c++) {
            float acc = 0.5f;
            for (int j = 0; j < nc; j++) acc += shc[3 * j + c] * Y[j];
            rgb[c] = fmaxf(acc, 0.f);
        }
    }
    A.rgb[i] = make_float4(rgb[0], rgb[1], rgb[2], 0.f);

    // ---- conservative screen bound
    int flags = 0;
    float rho[KMAX];
    float rho_max = 0.f, c_paper = 0.f, l1_bound = 0.f;
    const bool kernel_on = plane_ok && A.fc.alpha_min <= o;
    if (kernel_on) {
        const float gstar = psi_inv(A.fc.alpha_min / o, tau);
        // Eq. 11 as printed (no factor 2): endpoints at s_k sqrt(-log g*)
        c_paper = sqrtf(fmaxf(-logf(fmaxf(gstar, 1e-38f)), 0.f));
        const float Estar = -2.f * logf(fmaxf(gstar, 1e-38f)) * 1.004f + 1e-4f;
        const float sq = sqrtf(Estar) * 1.002f;
        // Eq. 8's exponent is at least eta r1^2, so alpha >= alpha_min needs
        // r1 <= sqrt(E* / eta): inside the polygon of the endpoints e_k scaled
        // by that factor (Eq. 7's r1 is 1 on the chord between e_k and e_k1)
        if (eta > 1e-3f) l1_bound = sqrtf(Estar / eta) * 1.002f;
        for (int k = 0; k < KMAX; k++) {
            if (k < K) {
                const int k1 = (k + 1 == K) ? 0 : k + 1;
                rho[k] = sq * fmaxf(s[k], s[k1]);
                rho_max = fmaxf(rho_max, rho[k]);
            } else {
                rho[k] = 0.f;
            }
        }
        flags |= 1;
    } else {
        for (int k = 0; k < KMAX; k++) rho[k] = 0.f;
    }
    rec[R_RHO2] = kernel_on ? rho_max * rho_max : -1.f;
    float minx = 1e30f, miny = 1e30f, maxx = -1e30f, maxy = -1e30f;
    float zlb = 1e30f, zub = -1e30f;
    bool crosses_near = false;
    if (kernel_on) {
        auto add_pt = [&](float x, float y) {   // point in the rotated plane frame
            float pc[3];
            for (int r = 0; r < 3; r++) pc[r] = G.muc[r] + x * G.Rxp[r] + y * G.Ryp[r];
            zlb = fminf(zlb, pc[2]);
            zub = fmaxf(zub, pc[2]);
            if (pc[2] <= A.fc.near_plane) { crosses_near = true; return; }
            const float iz = 1.f / pc[2];
            const float sx = A.cam.fx * pc[0] * iz + A.cam.cx - 0.5f;
            const float sy = A.cam.fy * pc[1] * iz + A.cam.cy - 0.5f;
            minx = fminf(minx, sx); maxx = fmaxf(maxx, sx);
            miny = fminf(miny, sy); maxy = fmaxf(maxy, sy);
        };
        add_pt(0.f, 0.f);
        for (int k = 0; k < K; k++) {
            const float tk = (k == 0) ? 0.f : th[k] - th[0];
            const float tk1 = (k + 1 == K) ? kTwoPi : th[k + 1] - th[0];
            const float gap = tk1 - tk;
            const float r0 = rho[k], r1 = rho[k] / cosf(0.25f * gap);
            for (int m = 0; m <= 4; m++) {
                const float ang = tk + 0.25f * gap * m;
                const float rr = (m & 1) ? r1 : r0;
                float sa, ca;
                sincosf(ang, &sa, &ca);
                add_pt(rr * ca, rr * sa);
            }
        }
        if (crosses_near) flags |= 2;
    }
    // filter disc
    float fr2 = -1.f;
    if (filt_on) {
        const float Rf = A.sl * sqrtf(2.f * fmaxf(logf(o / A.fc.alpha_min), 0.f)) + 1.0f;
        if (o >= A.fc.alpha_min) {
            fr2 = Rf * Rf;
            minx = fminf(minx, fpx - Rf); maxx = fmaxf(maxx, fpx + Rf);
            miny = fminf(miny, fpy - Rf); maxy = fmaxf(maxy, fpy + Rf);
        }
    }
    int x0, y0, x1, y1;
    const int TX = A.fc.tiles_x, TY = A.fc.tiles_y;
    if (A.cull_level == 0 || (kernel_on && crosses_near)) {
        x0 = 0; y0 = 0; x1 = TX - 1; y1 = TY - 1;
    } else if (minx > maxx) {
        x0 = 1; y0 = 1; x1 = 0; y1 = 0;   // empty
    } else {
        // pixel indices p in [minx - 1, maxx + 1] may be covered
        const float lx = fmaxf(minx - 1.f, -1.f), hx = fminf(maxx + 1.f, (float)A.fc.width);
        const float ly = fmaxf(miny - 1.f, -1.f), hy = fminf(maxy + 1.f, (float)A.fc.height);
        x0 = max(0, (int)floorf(lx / kTile));
        y0 = max(0, (int)floorf(ly / kTile));
        x1 = min(TX - 1, (int)floorf(hx / kTile));
        y1 = min(TY - 1, (int)floorf(hy / kTile));
        if (hx < 0.f || hy < 0.f || lx > (float)A.fc.width - 1.f || ly > (float)A.fc.height - 1.f) {
            x0 = 1; y0 = 1; x1 = 0; y1 = 0;
        }
    }
    int* bi = reinterpret_cast<int*>(bnd);
    bi[B_X0] = x0; bi[B_Y0] = y0; bi[B_X1] = x1; bi[B_Y1] = y1;
    bnd[B_ZLB] = (kernel_on && !crosses_near) ? zlb * (1.f - 1e-5f) : A.fc.near_plane;
    bnd[B_FCX] = fpx;
    bnd[B_FCY] = fpy;
    bnd[B_FR2] = fr2;
    bi[B_FLAGS] = flags;
    bnd[B_RHOMAX] = rho_max;
    for (int k = 0; k < KMAX; k++) bnd[B_RHO + k] = rho[k];
    for (int j = B_RHO + KMAX; j < Bnd<KMAX>::STRIDE; j++) bnd[j] = 0.f;
    bnd[Bnd<KMAX>::CPAPER] = c_paper;
    bnd[Bnd<KMAX>::CL1] = l1_bound;
    bnd[Bnd<KMAX>::ZC] = G.muc[2];
    const bool nonempty = x1 >= x0 && y1 >= y0;
    A.count[i] = nonempty ? (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1)) : 0u;
    if (nonempty && kernel_on && !crosses_near) atomicMax(A.zmax_bits, __float_as_int(fmaxf(zub, A.fc.near_plane)));
}

// ---------------------------------------------------------------------------
// Per-(primitive, tile) test.  Returns whether the pair may contribute and
// a lower bound of r_t over the tile's contributing pixels.
// Does the quad q (the corner pixels of a tile mapped into the plane frame,
// convex) meet the polygon of the K endpoints cl (EX_k, EY_k) (star-shaped
// about the origin, counter-clockwise)?  Either contains a vertex of the
// other, or two edges cross.
template <int KMAX>
__device__ bool quad_meets_polygon(const float (&qu)[4], const float (&qv)[4], const float* __restrict__ ex,
                                   const float* __restrict__ ey, int K, float cl) {
    float px[KMAX], py[KMAX];
    for (int k = 0; k < KMAX; k++) {
        px[k] = k < K ? cl * ex[k] : 0.f;
        py[k] = k < K ? cl * ey[k] : 0.f;
    }
    // a polygon vertex (or the origin, inside the polygon) inside the quad
    auto in_quad = [&](float x, float y) {
        int pos = 0, neg = 0;
        for (int c = 0; c < 4; c++) {
            const int n = (c + 1) & 3;
            const float cr = (qu[n] - qu[c]) * (y - qv[c]) - (qv[n] - qv[c]) * (x - qu[c]);
            pos += cr > 0.f;
            neg += cr < 0.f;
        }
        return pos == 0 || neg == 0;
    };
    if (in_quad(0.f, 0.f)) return true;
    for (int k = 0; k < K; k++)
        if (in_quad(px[k], py[k])) return true;
    // a quad corner inside the polygon (crossings of a ray towards +u)
    for (int c = 0; c < 4; c++) {
        bool in = false;
        for (int k = 0; k < K; k++) {
            const int k1 = (k + 1 == K) ? 0 : k + 1;
            const float ya = py[k], yb = py[k1];
            if ((ya > qv[c]) != (yb > qv[c])) {
                const float xc = px[k] + (qv[c] - ya) * (px[k1] - px[k]) / (yb - ya);
                if (qu[c] < xc) in = !in;
            }
        }
        if (in) return true;
    }
    // proper edge crossings
    for (int k = 0; k < K; k++) {
        const int k1 = (k + 1 == K) ? 0 : k + 1;
        const float ax = px[k], ay = py[k], bx = px[k1], by = py[k1];
        for (int c = 0; c < 4; c++) {
            const int n = (c + 1) & 3;
            const float d1 = (bx - ax) * (qv[c] - ay) - (by - ay) * (qu[c] - ax);
            const float d2 = (bx - ax) * (qv[n] - ay) - (by - ay) * (qu[n] - ax);
            const float d3 = (qu[n] - qu[c]) * (ay - qv[c]) - (qv[n] - qv[c]) * (ax - qu[c]);
            const float d4 = (qu[n] - qu[c]) * (by - qv[c]) - (qv[n] - qv[c]) * (bx - qu[c]);
            if (((d1 > 0.f) != (d2 > 0.f)) && ((d3 > 0.f) != (d4 > 0.f))) return true;
        }
    }
    return false;
}

template <int KMAX>
__device__ __forceinline__ bool tile_test(const float* __restrict__ rec, const float* __restrict__ bnd, int K,
                                          const FrameConst& fc, int tx, int ty, int cull, float& lb) {
    const bool do_cull = cull >= DRK_CULL_TILE, paper = cull == DRK_CULL_PAPER;
    const float x0 = (float)(tx * kTile), y0 = (float)(ty * kTile);
    const float x1 = (float)min(tx * kTile + kTile - 1, fc.width - 1);
    const float y1 = (float)min(ty * kTile + kTile - 1, fc.height - 1);
    const float cx[4] = {x0, x1, x1, x0}, cy[4] = {y0, y0, y1, y1};
    float w[4], wmax = -1e30f, wmin = 1e30f;
    for (int c = 0; c < 4; c++) {
        w[c] = fmaf(rec[R_HW0], cx[c], fmaf(rec[R_HW1], cy[c], rec[R_HW2]));
        wmax = fmaxf(wmax, w[c]);
        wmin = fminf(wmin, w[c]);
    }
    // t = 1/w over the rectangle is at least 1/wmax where w > 0
    const float tile_lb = wmax > 0.f ? fmaxf(1.f / wmax, fc.near_plane) * (1.f - 2e-6f) : fc.near_plane;
    const int flags = reinterpret_cast<const int*>(bnd)[B_FLAGS];
    const bool kernel_on = flags & 1, crosses = flags & 2;
    // filter disc
    bool keep_f = false;
    if (bnd[B_FR2] >= 0.f) {
        const float dx = fmaxf(fmaxf(x0 - bnd[B_FCX], bnd[B_FCX] - x1), 0.f);
        const float dy = fmaxf(fmaxf(y0 - bnd[B_FCY], bnd[B_FCY] - y1), 0.f);
        keep_f = dx * dx + dy * dy <= bnd[B_FR2];
    }
    lb = keep_f ? tile_lb : fmaxf(tile_lb, bnd[B_ZLB]);
    if (!do_cull) return true;
    if (wmax <= 0.f) return false;                                 // plane behind every pixel
    if (wmin * fc.near_plane >= 1.f + 1e-5f) return false;         // every r_t below the near plane
    if (keep_f && !paper) return true;
    if (!kernel_on) return false;
    // no quad: keep (the paper's polygon test needs only w > 0 at the corners:
    // then the tile maps to a convex quad of the plane, whatever the bound)
    if ((crosses && !paper) || wmin <= 0.f) return true;
    // tile corners in the rotated plane frame
    float qu[4], qv[4];
    for (int c = 0; c < 4; c++) {
        const float it = 1.f / w[c];
        qu[c] = fmaf(rec[R_HU0], cx[c], fmaf(rec[R_HU1], cy[c], rec[R_HU2])) * it;
        qv[c] = fmaf(rec[R_HV0], cx[c], fmaf(rec[R_HV1], cy[c], rec[R_HV2])) * it;
    }
    if (paper) {
        // the paper's culling (Sec. 4.4, Eq. 11 - Eq. 12): the polygon of the
        // basis endpoints at the calibrated lengths; lossy (see DRK_CULL_PAPER)
        using RK = Rec<KMAX>;
        const float cl = bnd[Bnd<KMAX>::CPAPER];
        return cl > 0.f && quad_meets_polygon<KMAX>(qu, qv, rec + RK::EX, rec + RK::EY, K, cl);
    }
    // distance from the centre to the quad, and whether it contains it
    float dmin2 = 1e30f;
    int pos = 0, neg = 0;
    for (int c = 0; c < 4; c++) {
        const int n = (c + 1) & 3;
        const float ex = qu[n] - qu[c], ey = qv[n] - qv[c];
        const float cr = qu[c] * qv[n] - qu[n] * qv[c];
        pos += cr > 0.f;
        neg += cr < 0.f;
        const float l2 = ex * ex + ey * ey;
        float tpar = l2 > 0.f ? -(qu[c] * ex + qv[c] * ey) / l2 : 0.f;
        tpar = fminf(fmaxf(tpar, 0.f), 1.f);
        const float px = qu[c] + tpar * ex, py = qv[c] + tpar * ey;
        dmin2 = fminf(dmin2, px * px + py * py);
    }
    if (pos == 0 || neg == 0) return true;                          // centre inside the quad
    const float rmax = bnd[B_RHOMAX];
    if (dmin2 > rmax * rmax * 1.002f) return false;                 // quad beyond every sector radius
    // angular range of the quad seen from the centre (< pi since the quad is
    // convex and excludes the centre)
    float ang[4];
    for (int c = 0; c < 4; c++) {
        float a = atan2f(qv[c], qu[c]);
        ang[c] = a < 0.f ? a + kTwoPi : a;
    }
    // sort four angles
#define DRK_CSWAP(i, j) { const float lo = fminf(ang[i], ang[j]), hi = fmaxf(ang[i], ang[j]); ang[i] = lo; ang[j] = hi; }
    DRK_CSWAP(0, 1) DRK_CSWAP(2, 3) DRK_CSWAP(0, 2) DRK_CSWAP(1, 3) DRK_CSWAP(1, 2)
#undef DRK_CSWAP
    float best = ang[0] + kTwoPi - ang[3];
    float A0 = ang[0];
    for (int c = 0; c < 3; c++) {
        const float gap = ang[c + 1] - ang[c];
        if (gap > best) { best = gap; A0 = ang[c + 1]; }
    }
    const float eps = 2e-3f;
    const float lo = A0 - eps, hi = A0 + (kTwoPi - best) + eps;
    // In each sector the quad overlaps: the wedge radius, and the chord of
    // the L1 bound (a sector's part of the polygon {r1 <= L} is the triangle
    // (0, L e_k, L e_k1); a convex quad meets the origin's side of the chord
    // only if one of its corners does)
    using RK = Rec<KMAX>;
    const float L = bnd[Bnd<KMAX>::CL1];
    float rho_arc = 0.f;
    bool chord_ok = !(L > 0.f);
    for (int k = 0; k < K; k++) {
        const float tk = (k == 0) ? 0.f : rec[R_TH + k - 1];
        const float tk1 = (k + 1 == K) ? kTwoPi : rec[R_TH + k];
        const bool ov = (tk <= hi && lo <= tk1) || (tk + kTwoPi <= hi && lo <= tk1 + kTwoPi) ||
                        (tk - kTwoPi <= hi && lo <= tk1 - kTwoPi);
        if (ov) {
            rho_arc = fmaxf(rho_arc, bnd[B_RHO + k]);
            if (!chord_ok) {
                const int k1 = (k + 1 == K) ? 0 : k + 1;
                const float ex = rec[RK::EX + k], ey = rec[RK::EY + k];
                const float nx = rec[RK::EY + k1] - ey, ny = ex - rec[RK::EX + k1];   // outward normal
                const float lim = L * (nx * ex + ny * ey);
                for (int c = 0; c < 4; c++)
                    if (nx * qu[c] + ny * qv[c] <= lim) chord_ok = true;
            }
        }
    }
    return chord_ok && dmin2 <= rho_arc * rho_arc * 1.002f;
}

// ---------------------------------------------------------------------------
// Row-interval culling (DRK_CULL_TILE).  The kernel's support lies in the
// union over sectors k of the sector of radius rho_k -- covered by a
// polygon of kArcSeg tangent segments, which lies inside the polygon the
// screen rectangle is built from -- cut by the chord of its L1 bound, the
// triangle (0, L e_k, L e_k1) with L = sqrt(E* / eta) (E >= eta r1^2,
// Eq. 7 - Eq. 8).  Each piece is convex and lies in front of the near plane
// (else the primitive takes the per-tile test), so it projects to a convex
// polygon.  In every row of tiles, the tiles kept are those whose columns
// hold a pixel centre (integer pixel index) within the x-range of the
// pieces (and of the filter disc) over the row's band of pixel rows, both
// widened by 0.1 pixel, far above the float32 error of the projection.
// The count pass stores each row's span of tiles, and the emission writes
// exactly those tiles.
constexpr int kArcSeg = 4;    // tangent segments per sector arc (the cover exceeds the arc by 1/cos(gap/8))
constexpr int kPieceV = 2 * kArcSeg + 3;   // centre, 2 kArcSeg + 1 arc points, one cut point

template <int KMAX>
struct Pieces {
    float2 v[KMAX][kPieceV];
    float ylo[KMAX], yhi[KMAX];   // the piece's extent in pixel rows
    int n[KMAX];
};

// Lane k < K builds piece k of primitive i in pixel-index coordinates.
template <int KMAX>
__device__ void build_pieces(const PreArgs& A, int64_t i, const float* __restrict__ rec,
                             const float* __restrict__ bnd, Pieces<KMAX>& P) {
    using RK = Rec<KMAX>;
    const int lane = threadIdx.x & 31;
    const int K = A.p.K;
    if (lane >= K) return;
    PrimGeom G;
    prim_geom(A, i, G);
    const int k = lane, k1 = (k + 1 == K) ? 0 : k + 1;
    const float tk = k == 0 ? 0.f : rec[RK::TH + k - 1];
    const float tk1 = rec[RK::TH + k];
    const float gap = tk1 - tk;
    const float rho = bnd[B_RHO + k];
    // the arc of radius rho over [tk, tk1], covered by kArcSeg tangent
    // segments: points on the arc alternate with the tangents' crossings
    // (directions by rotation from theta'_k in steps of gap / (2 kArcSeg); the
    // last one exact, so neighbouring pieces share their boundary ray; the
    // rotation's float32 drift, ~1e-6 rad, is far inside rho's 0.2 % margin)
    const float half = gap / (2 * kArcSeg);
    float sh, ch, sa, ca;
    sincosf(half, &sh, &ch);
    sincosf(tk, &sa, &ca);
    const float rt = rho / ch;
    float px[kPieceV], py[kPieceV];
    int n = 0;
    px[n] = 0.f; py[n] = 0.f; n++;
    for (int m = 0; m <= 2 * kArcSeg; m++) {
        if (m == 2 * kArcSeg) sincosf(tk1, &sa, &ca);
        const float rr = (m & 1) ? rt : rho;
        px[n] = rr * ca; py[n] = rr * sa; n++;
        const float cn = ca * ch - sa * sh;
        sa = sa * ch + ca * sh;
        ca = cn;
    }
    const float L = bnd[Bnd<KMAX>::CL1];
    float qx[kPieceV], qy[kPieceV];
    int m = 0;
    if (L > 0.f) {
        // keep the side of the chord the centre is on: n . p <= L n . e_k
        const float ex = rec[RK::EX + k], ey = rec[RK::EY + k];
        const float nx = rec[RK::EY + k1] - ey, ny = ex - rec[RK::EX + k1];
        const float lim = L * (nx * ex + ny * ey);
        for (int a = 0; a < n; a++) {
            const int b = (a + 1 == n) ? 0 : a + 1;
            const float da = nx * px[a] + ny * py[a] - lim, db = nx * px[b] + ny * py[b] - lim;
            if (da <= 0.f) { qx[m] = px[a]; qy[m] = py[a]; m++; }
            if ((da < 0.f && db > 0.f) || (da > 0.f && db < 0.f)) {
                const float t = da / (da - db);
                qx[m] = px[a] + t * (px[b] - px[a]);
                qy[m] = py[a] + t * (py[b] - py[a]);
                m++;
            }
        }
    } else {
        for (int a = 0; a < n; a++) { qx[a] = px[a]; qy[a] = py[a]; }
        m = n;
    }
    float ylo = 1e30f, yhi = -1e30f;
    for (int a = 0; a < m; a++) {
        float pc[3];
        for (int r = 0; r < 3; r++) pc[r] = G.muc[r] + qx[a] * G.Rxp[r] + qy[a] * G.Ryp[r];
        const float iz = 1.f / pc[2];
        const float2 q = make_float2(A.cam.fx * pc[0] * iz + A.cam.cx - 0.5f, A.cam.fy * pc[1] * iz + A.cam.cy - 0.5f);
        P.v[k][a] = q;
        ylo = fminf(ylo, q.y);
        yhi = fmaxf(yhi, q.y);
    }
    P.ylo[k] = ylo;
    P.yhi[k] = yhi;
    P.n[k] = m;
}

// Tiles [a, b] of row ty (clamped to the rectangle's columns x0 .. x1) whose
// columns meet the pieces or the filter disc within the row's pixel band.
template <int KMAX>
__device__ void row_span(const Pieces<KMAX>& P, int K, const float* __restrict__ bnd, const FrameConst& fc, int ty,
                         int x0, int x1, int& a, int& b) {
    // pixel centres sit at integer pixel indices; 0.1 px covers the float32
    // error of the projection many times over
    const float yl = (float)(ty * kTile) - 0.1f;
    const float yh = (float)min(ty * kTile + kTile - 1, fc.height - 1) + 0.1f;
    float xmin = 1e30f, xmax = -1e30f;
    for (int k = 0; k < K; k++) {
        const int n = P.n[k];
        if (n == 0 || P.yhi[k] < yl || P.ylo[k] > yh) continue;   // the piece misses the band
        for (int e = 0; e < n; e++) {
            float2 p = P.v[k][e], q = P.v[k][(e + 1 == n) ? 0 : e + 1];
            if (p.y > q.y) { const float2 t = p; p = q; q = t; }
            if (q.y < yl || p.y > yh) continue;
            const float dy = q.y - p.y;
            const float xa = (p.y >= yl || dy <= 0.f) ? p.x : p.x + (q.x - p.x) * ((yl - p.y) / dy);
            const float xb = (q.y <= yh || dy <= 0.f) ? q.x : p.x + (q.x - p.x) * ((yh - p.y) / dy);
            xmin = fminf(xmin, fminf(xa, xb));
            xmax = fmaxf(xmax, fmaxf(xa, xb));
        }
    }
    const float fr2 = bnd[B_FR2];
    if (fr2 >= 0.f) {
        const float fy = bnd[B_FCY];
        const float d = fmaxf(fmaxf(yl - fy, fy - yh), 0.f);
        if (d * d <= fr2) {
            const float dx = sqrtf(fr2 - d * d);
            xmin = fminf(xmin, bnd[B_FCX] - dx);
            xmax = fmaxf(xmax, bnd[B_FCX] + dx);
        }
    }
    // integer pixel columns within [xmin - 0.1, xmax + 0.1]
    const float lx = ceilf(fmaxf(xmin - 0.1f, -1.f)), hx = floorf(fminf(xmax + 0.1f, (float)fc.width));
    if (!(lx <= hx)) { a = 1; b = 0; return; }
    a = max(x0, (int)floorf(lx / kTile));
    b = min(x1, (int)floorf(hx / kTile));
}

// Lower bound of r_t over the pixels of tile (tx, ty) the primitive can
// reach (the depth field of its pair key; as in tile_test).
__device__ __forceinline__ float tile_depth_bound(const float* __restrict__ rec, const float* __restrict__ bnd,
                                                  const FrameConst& fc, int tx, int ty) {
    const float x0 = (float)(tx * kTile), y0 = (float)(ty * kTile);
    const float x1 = (float)min(tx * kTile + kTile - 1, fc.width - 1);
    const float y1 = (float)min(ty * kTile + kTile - 1, fc.height - 1);
    const float cx[4] = {x0, x1, x1, x0}, cy[4] = {y0, y0, y1, y1};
    float wmax = -1e30f;
    for (int c = 0; c < 4; c++) wmax = fmaxf(wmax, fmaf(rec[R_HW0], cx[c], fmaf(rec[R_HW1], cy[c], rec[R_HW2])));
    const float tile_lb = wmax > 0.f ? fmaxf(1.f / wmax, fc.near_plane) * (1.f - 2e-6f) : fc.near_plane;
    bool keep_f = false;
    if (bnd[B_FR2] >= 0.f) {
        const float dx = fmaxf(fmaxf(x0 - bnd[B_FCX], bnd[B_FCX] - x1), 0.f);
        const float dy = fmaxf(fmaxf(y0 - bnd[B_FCY], bnd[B_FCY] - y1), 0.f);
        keep_f = dx * dx + dy * dy <= bnd[B_FR2];
    }
    return keep_f ? tile_lb : fmaxf(tile_lb, bnd[B_ZLB]);
}

// Does primitive i take the row-interval test?  Only when its rectangle
// holds more tiles than one warp tests at once: below that the per-tile
// test costs less than building the pieces.  (Either test is conservative;
// the count and the emission take the same choice.)
__device__ __forceinline__ bool row_culled(const PreArgs& A, const float* __restrict__ bnd) {
    const int* bi = reinterpret_cast<const int*>(bnd);
    const int area = (bi[B_X1] - bi[B_X0] + 1) * (bi[B_Y1] - bi[B_Y0] + 1);
    return A.cull_level == DRK_CULL_TILE && !(bi[B_FLAGS] & 2) && area > 32;
}

constexpr int kCullThreads = 256;

// K2a: count the pairs of each primitive (one warp per primitive).
template <int KMAX>
__global__ void __launch_bounds__(kCullThreads) count_kernel(PreArgs A) {
    __shared__ Pieces<KMAX> pieces[kCullThreads / 32];
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= A.p.n) return;
    const float* rec = A.rec + (int64_t)Rec<KMAX>::STRIDE * i;
    const float* bnd = A.bnd + (int64_t)Bnd<KMAX>::STRIDE * i;
    const int* bi = reinterpret_cast<const int*>(bnd);
    const int x0 = bi[B_X0], y0 = bi[B_Y0], x1 = bi[B_X1], y1 = bi[B_Y1];
    if (x1 < x0 || y1 < y0) {
        if (lane == 0) A.count[i] = 0;
        return;
    }
    if (row_culled(A, bnd)) {
        Pieces<KMAX>& P = pieces[threadIdx.x >> 5];
        if (lane < KMAX) P.n[lane] = 0;
        if (bi[B_FLAGS] & 1) build_pieces<KMAX>(A, i, rec, bnd, P);
        __syncwarp();
        uint32_t cnt = 0;
        uint32_t* sp = A.spans + (size_t)A.fc.tiles_y * i;
        // the same trip count on every lane: a shuffle after a loop whose
        // trip count differed between lanes returned stale values to the
        // lanes that ran longer (observed with nvcc 13.0 on sm_103a)
        for (int r0 = y0; r0 <= y1; r0 += 32) {
            const int ty = r0 + lane;
            if (ty <= y1) {
                int a, b;
                row_span<KMAX>(P, A.p.K, bnd, A.fc, ty, x0, x1, a, b);
                cnt += b >= a ? (uint32_t)(b - a + 1) : 0u;
                sp[ty] = b >= a ? ((uint32_t)a | ((uint32_t)b << 16)) : 1u;   // 1: a = 1 > b = 0, empty
            }
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) A.count[i] = cnt;
        return;
    }
    const int wdt = x1 - x0 + 1;
    const int area = wdt * (y1 - y0 + 1);
    uint32_t cnt = 0;
    for (int base = 0; base < area; base += 32) {
        const int j = base + lane;
        bool keep = false;
        if (j < area) {
            float lb;
            keep = tile_test<KMAX>(rec, bnd, A.p.K, A.fc, x0 + j % wdt, y0 + j / wdt, A.cull_level, lb);
        }
        cnt += __popc(__ballot_sync(0xffffffffu, keep));
    }
    if (lane == 0) A.count[i] = cnt;
}

// K2b: emit (key, value) pairs: key = tile << depth_bits | quantised lower
// bound of r_t, value = primitive index.  Pairs of primitive i start at
// offsets[i]; within a primitive they are in tile order.
template <int KMAX>
__global__ void __launch_bounds__(kCullThreads) emit_kernel(PreArgs A) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= A.p.n) return;
    const float* rec = A.rec + (int64_t)Rec<KMAX>::STRIDE * i;
    const float* bnd = A.bnd + (int64_t)Bnd<KMAX>::STRIDE * i;
    const int* bi = reinterpret_cast<const int*>(bnd);
    const int x0 = bi[B_X0], y0 = bi[B_Y0], x1 = bi[B_X1], y1 = bi[B_Y1];
    if (x1 < x0 || y1 < y0) return;
    if (lane == 0 && A.count[i] > 0 && A.counters) atomicAdd(A.counters + 3, 1ull);
    const DepthQuant dq = *A.dq;
    const uint32_t qmax = (1u << dq.depth_bits) - 1u;
    const int wdt = x1 - x0 + 1;
    int area = wdt * (y1 - y0 + 1);
    uint64_t out = A.offsets[i];
    const uint64_t end = A.offsets[i + 1];
    const int cull = A.cull_level >= DRK_CULL_TILE ? A.cull_level : DRK_CULL_NONE;
    // depth field of a pair key: the quantised lower bound of r_t (or, in the
    // cache-sorting mode, the primitive's centre-depth rank)
    auto depth_field = [&](float lb) -> uint32_t {
        if (A.rank) return A.rank[i];
        const float qf = floorf((lb - dq.zmin) * dq.scale);
        return qf <= 0.f ? 0u : (qf >= (float)qmax ? qmax : (uint32_t)qf);
    };
    if (row_culled(A, bnd)) {
        // the row spans the count pass found; each lane writes the tiles of
        // its rows, after those of lower lanes
        const uint32_t* sp = A.spans + (size_t)A.fc.tiles_y * i;
        for (int r0 = y0; r0 <= y1; r0 += 32) {
            const int ty = r0 + lane;
            int a = 1, b = 0;
            if (ty <= y1) {
                const uint32_t ab = sp[ty];
                a = (int)(ab & 0xffffu);
                b = (int)(ab >> 16);
            }
            const uint32_t c = b >= a ? (uint32_t)(b - a + 1) : 0u;
            uint32_t incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            uint64_t pos = out + (incl - c);
            for (int tx = a; tx <= b; tx++, pos++) {
                if (pos < end) {   // never write past the slots the count pass allotted
                    A.keys[pos] = ((uint32_t)(ty * A.fc.tiles_x + tx) << dq.depth_bits) |
                                  depth_field(tile_depth_bound(rec, bnd, A.fc, tx, ty));
                    A.vals[pos] = (uint32_t)i;
                }
            }
            out += __shfl_sync(0xffffffffu, incl, 31);
        }
        area = 0;   // the per-tile loop below has nothing left to do
    }
    for (int base = 0; base < area; base += 32) {
        const int j = base + lane;
        bool keep = false;
        uint32_t key = 0;
        if (j < area) {
            const int tx = x0 + j % wdt, ty = y0 + j / wdt;
            float lb;
            keep = tile_test<KMAX>(rec, bnd, A.p.K, A.fc, tx, ty, cull, lb);
            key = ((uint32_t)(ty * A.fc.tiles_x + tx) << dq.depth_bits) | depth_field(lb);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const uint64_t pos = out + __popc(m & ((1u << lane) - 1u));
            if (pos < end) {   // never write past the slots the count pass allotted
                A.keys[pos] = key;
                A.vals[pos] = (uint32_t)i;
            }
        }
        out += __popc(m);
    }
    // the count pass and this pass take the same decisions; should they ever
    // differ, the allotted slots stay in bounds: surplus pairs are dropped
    // and flagged, missing ones become sentinel keys past the last tile
    if (out != end && lane == 0 && A.status) atomicOr(A.status, 1 << DRK_ERR_CAPACITY);
    const uint32_t sentinel = ((uint32_t)(A.fc.tiles_x * A.fc.tiles_y) << dq.depth_bits) | qmax;
    for (uint64_t pos = out + lane; pos < end; pos += 32) {
        A.keys[pos] = sentinel;
        A.vals[pos] = (uint32_t)i;
    }
}

// Pre-sort of the cache-sorting mode: the rank of every primitive in the
// order (view-space depth of mu, index).  keys: order-preserving bits of the
// depth; a stable sort by them leaves equal depths in index order.
__global__ void centre_key_kernel(const float* __restrict__ bnd, int stride, int zc, int64_t n,
                                  uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t b = __float_as_uint(bnd[(int64_t)stride * i + zc]);
    keys[i] = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    vals[i] = (uint32_t)i;
}
__global__ void rank_scatter_kernel(const uint32_t* __restrict__ vals, int64_t n, uint32_t* __restrict__ rank) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    rank[vals[k]] = (uint32_t)k;
}

template <int KMAX>
void launch_centre_rank(const PreArgs& A, uint32_t* keys, uint32_t* vals, uint32_t* kalt, uint32_t* valt,
                        void* scratch, uint32_t* rank, cudaStream_t st) {
    const int64_t n = A.p.n;
    if (n <= 0) return;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    centre_key_kernel<<<blocks, 256, 0, st>>>(A.bnd, Bnd<KMAX>::STRIDE, Bnd<KMAX>::ZC, n, keys, vals); note_launch();
    radix_sort_pairs(keys, vals, kalt, valt, n, 32, scratch, st);
    rank_scatter_kernel<<<blocks, 256, 0, st>>>(vals, n, rank); note_launch();
}
template void launch_centre_rank<8>(const PreArgs&, uint32_t*, uint32_t*, uint32_t*, uint32_t*, void*, uint32_t*,
                                    cudaStream_t);
template void launch_centre_rank<16>(const PreArgs&, uint32_t*, uint32_t*, uint32_t*, uint32_t*, void*, uint32_t*,
                                     cudaStream_t);

// depth quantisation from the device-side maximum depth
__global__ void depth_quant_kernel(PreArgs A) {
    DepthQuant dq;
    dq.zmin = A.fc.near_plane;
    float zmax = __int_as_float(*A.zmax_bits);
    if (!(zmax > dq.zmin)) zmax = dq.zmin + 1.f;
    dq.depth_bits = A.depth_bits;
    const float levels = (float)((1u << A.depth_bits) - 1u);
    dq.scale = levels / (zmax - dq.zmin);
    dq.inv_scale = (zmax - dq.zmin) / levels;
    *A.dq = dq;
}

// ---------------------------------------------------------------------------
// K7: per-primitive backward.  Consumes the record-space gradients of the
// raster backward (homography rows, filter centre and coefficient, colour)
// and writes the gradients of mu, quat and colour; completes theta_0.
template <int KMAX>
__global__ void __launch_bounds__(128) preprocess_backward_kernel(PreArgs A, const float* __restrict__ gtmp,
                                                                  drk_params_grad_t grads) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.p.n) return;
    const int K = A.p.K;
    const float* gr = gtmp + (int64_t)G_STRIDE * i;
    PrimGeom G;
    prim_geom(A, i, G);
    float dmuc[3] = {0.f, 0.f, 0.f}, dRxc[3] = {0.f, 0.f, 0.f}, dRyc[3] = {0.f, 0.f, 0.f}, dnc[3] = {0.f, 0.f, 0.f};
    float dth0 = 0.f;
    const bool plane_ok = fabsf(G.N) > 1e-20f;
    if (plane_ok) {
        // rows: U' = row(a), V' = row(b), W = row(m)
        auto drow = [&](const float* dr, float* dv) {
            dv[0] = dr[0] * A.fc.ifx + dr[2] * A.fc.ox;
            dv[1] = dr[1] * A.fc.ify + dr[2] * A.fc.oy;
            dv[2] = dr[2];
        };
        float da[3], db[3], dm[3];
        drow(gr + G_HU0, da);
        drow(gr + G_HV0, db);
        drow(gr + G_HW0, dm);
        const float N = G.N, invN = 1.f / N;
        const float al = G.U0 * invN, be = G.V0 * invN;
        float dRxp[3], dRyp[3], dN = 0.f;
        for (int r = 0; r < 3; r++) {
            dRxp[r] = da[r];
            dRyp[r] = db[r];
            dnc[r] += -al * da[r] - be * db[r] + dm[r] * invN;
        }
        const float dal = -dot3(da, G.nc), dbe = -dot3(db, G.nc);
        dN += -dot3(dm, G.nc) * invN * invN;
        const float dU0 = dal * invN, dV0 = dbe * invN;
        dN += -dal * G.U0 * invN * invN - dbe * G.V0 * invN * invN;
        // filter: coefficient log2(e)/(2 sl^2 N^2), projected centre
        if (A.sl > 0.f && G.muc[2] > A.fc.near_plane) {
            const float fcoef = kLog2e / (2.f * A.sl * A.sl * N * N);
            dN += gr[G_FCOEF] * (-2.f * fcoef * invN);
            const float iz = 1.f / G.muc[2];
            dmuc[0] += gr[G_FPX] * A.cam.fx * iz;
            dmuc[1] += gr[G_FPY] * A.cam.fy * iz;
            dmuc[2] += -(gr[G_FPX] * A.cam.fx * G.muc[0] + gr[G_FPY] * A.cam.fy * G.muc[1]) * iz * iz;
        }
        for (int r = 0; r < 3; r++) {
            dRxp[r] += dU0 * G.muc[r];
            dRyp[r] += dV0 * G.muc[r];
            dmuc[r] += dU0 * G.Rxp[r] + dV0 * G.Ryp[r] + dN * G.nc[r];
            dnc[r] += dN * G.muc[r];
        }
        for (int r = 0; r < 3; r++) {
            dRxc[r] = G.c0 * dRxp[r] - G.s0 * dRyp[r];
            dRyc[r] = G.s0 * dRxp[r] + G.c0 * dRyp[r];
        }
        dth0 += dot3(dRxp, G.Ryp) - dot3(dRyp, G.Rxp);
    }
    // back to world space: mu_c = Rc mu + t, Rxc = Rc Rx, ...
    const float* M = A.cam.w2c;
    float dmu[3], dR[9];
    for (int c = 0; c < 3; c++) {
        dmu[c] = M[c] * dmuc[0] + M[4 + c] * dmuc[1] + M[8 + c] * dmuc[2];
        dR[3 * c + 0] = M[c] * dRxc[0] + M[4 + c] * dRxc[1] + M[8 + c] * dRxc[2];
        dR[3 * c + 1] = M[c] * dRyc[0] + M[4 + c] * dRyc[1] + M[8 + c] * dRyc[2];
        dR[3 * c + 2] = M[c] * dnc[0] + M[4 + c] * dnc[1] + M[8 + c] * dnc[2];
    }
    // colour
    const float drgb[3] = {gr[G_R], gr[G_G], gr[G_B]};
    if (A.p.sh_degree < 0) {
        for (int c = 0; c < 3; c++) grads.color[3 * i + c] = drgb[c];
    } else {
        const int deg = A.p.sh_degree;
        const int nc = (deg + 1) * (deg + 1);
        float d[3];
        for (int c = 0; c < 3; c++) d[c] = A.p.mu[3 * i + c] - A.cam_center[c];
        const float nrm = sqrtf(dot3(d, d));
        const float x = d[0] / nrm, y = d[1] / nrm, z = d[2] / nrm;
        float Y[16];
        sh_basis(deg, x, y, z, Y);
        const float* shc = A.p.color + (int64_t)3 * nc * i;
        float wgt[16];
        float gc[3];
        for (int c = 0; c < 3; c++) {
            float acc = 0.5f;
            for (int j = 0; j < nc; j++) acc += shc[3 * j + c] * Y[j];
            gc[c] = acc < 0.f ? 0.f : drgb[c];
        }
        for (int j = 0; j < nc; j++) {
            wgt[j] = gc[0] * shc[3 * j] + gc[1] * shc[3 * j + 1] + gc[2] * shc[3 * j + 2];
            for (int c = 0; c < 3; c++) grads.color[(int64_t)3 * nc * i + 3 * j + c] = gc[c] * Y[j];
        }
        float gdir[3];
        sh_basis_vjp(deg, x, y, z, wgt, gdir);
        const float pr = gdir[0] * x + gdir[1] * y + gdir[2] * z;
        dmu[0] += (gdir[0] - x * pr) / nrm;
        dmu[1] += (gdir[1] - y * pr) / nrm;
        dmu[2] += (gdir[2] - z * pr) / nrm;
    }
    for (int c = 0; c < 3; c++) grads.mu[3 * i + c] = dmu[c];
    // quaternion: R(qn), qn = q / |q|
    {
        const float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
        float gw = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        gy += -4.f * y * dR[0]; gz += -4.f * z * dR[0];
        gw += -2.f * z * dR[1]; gx += 2.f * y * dR[1]; gy += 2.f * x * dR[1]; gz += -2.f * w * dR[1];
        gw += 2.f * y * dR[2];  gx += 2.f * z * dR[2]; gy += 2.f * w * dR[2]; gz += 2.f * x * dR[2];
        gw += 2.f * z * dR[3];  gx += 2.f * y * dR[3]; gy += 2.f * x * dR[3]; gz += 2.f * w * dR[3];
        gx += -4.f * x * dR[4]; gz += -4.f * z * dR[4];
        gw += -2.f * x * dR[5]; gx += -2.f * w * dR[5]; gy += 2.f * z * dR[5]; gz += 2.f * y * dR[5];
        gw += -2.f * y * dR[6]; gx += 2.f * z * dR[6]; gy += -2.f * w * dR[6]; gz += 2.f * x * dR[6];
        gw += 2.f * x * dR[7];  gx += 2.f * w * dR[7]; gy += 2.f * z * dR[7]; gz += 2.f * y * dR[7];
        gx += -4.f * x * dR[8]; gy += -4.f * y * dR[8];
        const float pr = w * gw + x * gx + y * gy + z * gz;
        const float inv = 1.f / G.qnorm;
        grads.quat[4 * i + 0] = (gw - w * pr) * inv;
        grads.quat[4 * i + 1] = (gx - x * pr) * inv;
        grads.quat[4 * i + 2] = (gy - y * pr) * inv;
        grads.quat[4 * i + 3] = (gz - z * pr) * inv;
    }
    // theta_0: the relative angles theta'_j = theta_j - theta_0 and the frame
    float* dth = grads.theta + (int64_t)K * i;
    float sum = 0.f;
    for (int j = 1; j < K; j++) sum += dth[j];
    dth[0] = dth0 - sum;
}

// ---------------------------------------------------------------------------
template <int KMAX>
void launch_preprocess(const PreArgs& A, cudaStream_t st) {
    const int64_t n = A.p.n;
    if (n == 0) return;
    preprocess_kernel<KMAX><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(A); note_launch();
}
template <int KMAX>
void launch_count(const PreArgs& A, cudaStream_t st) {
    const int64_t n = A.p.n;
    if (n == 0) return;
    count_kernel<KMAX><<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(A); note_launch();
}
template <int KMAX>
void launch_emit(const PreArgs& A, cudaStream_t st) {
    const int64_t n = A.p.n;
    if (n == 0) return;
    emit_kernel<KMAX><<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(A); note_launch();
}
template <int KMAX>
void launch_preprocess_backward(const PreArgs& A, const float* gtmp, const drk_params_grad_t& g, cudaStream_t st) {
    const int64_t n = A.p.n;
    if (n == 0) return;
    preprocess_backward_kernel<KMAX><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(A, gtmp, g); note_launch();
}

void launch_depth_quant(const PreArgs& A, cudaStream_t st) { depth_quant_kernel<<<1, 1, 0, st>>>(A); }

template void launch_preprocess<8>(const PreArgs&, cudaStream_t);
template void launch_preprocess<16>(const PreArgs&, cudaStream_t);
template void launch_count<8>(const PreArgs&, cudaStream_t);
template void launch_count<16>(const PreArgs&, cudaStream_t);
template void launch_emit<8>(const PreArgs&, cudaStream_t);
template void launch_emit<16>(const PreArgs&, cudaStream_t);
template void launch_preprocess_backward<8>(const PreArgs&, const float*, const drk_params_grad_t&, cudaStream_t);
template void launch_preprocess_backward<16>(const PreArgs&, const float*, const drk_params_grad_t&, cudaStream_t);

}  // namespace drk
