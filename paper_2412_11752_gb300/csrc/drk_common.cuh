// drk_common.cuh -- device-side data layout and per-pair math of the DRK
// rasterizer (sm_103a).  Shared by the preprocess, raster and backward
// translation units of libdrk.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace drk {

constexpr double kPiD = 3.14159265358979323846;
constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kLog2e = 1.44269504088896340736f;
constexpr float kLn2 = 0.69314718055994530942f;
constexpr int kTile = 16;                 // 16 x 16 pixel tiles (Sec. 4.4)
constexpr int kTilePix = kTile * kTile;   // one thread per pixel

// compile-time square root (Newton) for closed-form constants
constexpr double csqrt_iter(double x, double g, int n) {
    return n == 0 ? g : csqrt_iter(x, 0.5 * (g + x / g), n - 1);
}
constexpr double csqrt(double x) { return csqrt_iter(x, x > 1.0 ? x : 1.0, 60); }

// ---------------------------------------------------------------------------
// Raster record: everything the per-pixel evaluation needs, per primitive,
// float32, 16-byte aligned so that a CTA stages it into shared memory with
// 16-byte vector copies.
//
// The plane coordinates are taken in a frame rotated by -theta_0 about the
// normal, so that the polar angle of the evaluation is measured from the
// first radial basis directly (theta'_j = theta_j - theta_0).
//
// header (floats):
//   0..8   homography rows U', V', W over integer pixel indices (x, y):
//          w = W.(x, y, 1), t = 1/w is the ray depth r_t (Eq. 13),
//          (u', v') = (U'.(x, y, 1), V'.(x, y, 1)) * t  (Eq. 4, Eq. 5)
//   9      squared radius of the kernel support in the plane (max over
//          sectors of rho_k, see the preprocess); < 0 when the kernel
//          term cannot reach alpha_min
//   10     filter cut: evaluate the filter only while its base-2 exponent
//          is below this (beyond it the filter is < alpha_min / 2); < 0 = off
//   11,12  projected centre minus 0.5 (pixel-index coordinates)   (Eq. 10)
//   13     log2(e) / (2 s_l^2 N^2)    filter exponent per (px^2 |d|^2 t^2)
//   14     o
//   15     eta * log2(e) / 2         (Eq. 8, base-2 exponent)
//          (floats 0-15, the first 64 bytes, are all the geometry stage
//          of the evaluation reads)
//   16     (1 - eta) * log2(e) / 2
//   17,18  Psi breakpoints (1 + tau)/4, (3 - tau)/4          (Eq. 9)
//   19     o (1 - tau)/(1 + tau)      outer slope (x o)
//   20     o (1 + tau)/(1 - tau)      middle slope (x o)
//   21     -o tau/(1 - tau)           middle offset (x o)
//   22     2 o tau/(1 + tau)          upper offset (x o)
//   23     tau
//   24 .. 24+KMAX-1           theta'_1 .. theta'_{K-1}, then theta'_K = 2 pi,
//                             padded with +1e30 (sector thresholds)
//   EX = 24+KMAX .. +KMAX-1   e_j.x = s_j cos theta'_j   (Eq. 7 basis)
//   EY = EX+KMAX ..           e_j.y = s_j sin theta'_j
//   AA = EY+KMAX ..           A_j = 1 / (2 s_j^2)         (Eq. 6)
// The sector constants (pi / gap, A_k +- A_k1, the inverse of
// [e_k e_k1]) are formed from these during the evaluation, so the whole
// evaluation reads the record header only.
// ---------------------------------------------------------------------------
enum : int {
    R_HU0 = 0, R_HU1, R_HU2, R_HV0, R_HV1, R_HV2, R_HW0, R_HW1, R_HW2,
    R_RHO2, R_FCUT, R_FPX, R_FPY, R_FCOEF, R_OPA, R_ETA2,
    R_ETA2C, R_B1, R_B2, R_SLO, R_SMID, R_OMID, R_OHI, R_TAU,
    R_TH = 24
};
constexpr int R_GEO4 = 4;   // float4 count of the geometry part
constexpr int R_FIX4 = 6;   // float4 count of the fixed part (floats 0-23)

template <int KMAX>
struct Rec {
    static constexpr int TH = R_TH;
    static constexpr int EX = TH + KMAX;
    static constexpr int EY = EX + KMAX;
    static constexpr int AA = EY + KMAX;
    static constexpr int HDR = AA + KMAX;                     // floats
    static constexpr int STRIDE = HDR;
    static constexpr int STRIDE4 = STRIDE / 4;                // float4
    static_assert(STRIDE % 4 == 0, "record must be float4 aligned");
};

// Bound record used by tile culling and pair emission (floats; ints in
// the first four slots).
//   0..3  tile rect x0, y0, x1, y1 (inclusive; x1 < x0 means empty)
//   4     lower bound of r_t over the kernel support (polygon vertices)
//   5,6   projected centre minus 0.5 (filter disc centre, pixel indices)
//   7     squared filter disc radius in pixels (< 0: filter off)
//   8     flags: bit0 kernel support non-empty, bit1 support crosses the
//         near plane (no polygon bound)
//   9     max_k rho_k
//   10..  rho_k (KMAX), the per-sector radius of the support (Eq. 11
//         corrected, see preprocess)
enum : int { B_X0 = 0, B_Y0, B_X1, B_Y1, B_ZLB, B_FCX, B_FCY, B_FR2, B_FLAGS, B_RHOMAX, B_RHO = 10 };
template <int KMAX>
struct Bnd {
    static constexpr int ZC = B_RHO + KMAX;                    // view-space depth of mu
    static constexpr int CPAPER = ZC + 1;                      // sqrt(-log g*) of Eq. 11 as printed
    static constexpr int CL1 = CPAPER + 1;                     // L1 bound sqrt(E* / eta) (0: none)
    static constexpr int STRIDE = ((CL1 + 1) + 3) / 4 * 4;
};

// Per-primitive record-space gradient accumulator used between the raster
// backward and the preprocess backward (floats).
enum : int { G_HU0 = 0, G_HU1, G_HU2, G_HV0, G_HV1, G_HV2, G_HW0, G_HW1, G_HW2,
             G_FPX, G_FPY, G_FCOEF, G_R, G_G, G_B, G_STRIDE };

// ---------------------------------------------------------------------------
// Small PTX helpers (documented PTX instructions).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Polar angle of (u, v) in [0, 2 pi): the octant is reduced to r = min/max
// in [0, 1], atan(r) = r P(r^2) with a degree-7 polynomial P fitted here
// (weighted least squares on [0, 1], absolute error below 4e-8 in exact
// arithmetic, 1.2e-7 evaluated in float32), then the octant is restored.
// With the reciprocal (1 ulp) and the restoring subtractions the angle is
// within about 4e-7 rad, as close as atan2f; (0, 0) gives 0.
__device__ __forceinline__ float polar_angle(float u, float v) {
    const float ax = fabsf(u), ay = fabsf(v);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float r = mx > 1e-30f ? __fmul_rn(mn, rcp_approx(mx)) : 0.0f;
    const float s = __fmul_rn(r, r);
    float p = -0.0040557123720645905f;
    p = fmaf(p, s, 0.02186696231365204f);
    p = fmaf(p, s, -0.0559178851544857f);
    p = fmaf(p, s, 0.09642587602138519f);
    p = fmaf(p, s, -0.1390877515077591f);
    p = fmaf(p, s, 0.19946593046188354f);
    p = fmaf(p, s, -0.33329862356185913f);
    p = fmaf(p, s, 0.9999993443489075f);
    float a = __fmul_rn(r, p);
    if (ay > ax) a = __fadd_rn(1.57079632679489662f, -a);
    if (u < 0.0f) a = __fadd_rn(kPi, -a);
    if (v < 0.0f) a = __fadd_rn(kTwoPi, -a);
    return a;
}

// ---------------------------------------------------------------------------
// Per-pixel constants of the camera ray (integer pixel indices).
struct PixelRay {
    float x, y;    // pixel indices as float
    float d2;      // |d|^2 of the unnormalised camera-space ray (z = 1)
};

// Intermediate values of one evaluation, kept when the derivative is needed.
struct EvalInfo {
    float t, u, v, phi, r2sq, dth, c, Q, a, b, r1, X, g, al_k, Xf, f;
    float pg, dif;                  // pi / gap_k, A_k - A_k1
    float ekx, eky, e1x, e1y, idet; // e_k, e_k1 and 1 / det [e_k e_k1]
    int k;
    bool filt_eval, use_filter, clamped;
};

// Record header loads (16-byte, read-only path): the fixed part (floats
// 0-23) into registers; the geometry stage needs the first R_GEO4 float4.
__device__ __forceinline__ void load_head_geo(const float4* __restrict__ r4, float* h) {
#pragma unroll
    for (int q = 0; q < R_GEO4; q++) {
        const float4 v = __ldg(r4 + q);
        h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
    }
}
__device__ __forceinline__ void load_head_fix(const float4* __restrict__ r4, float* h) {
    load_head_geo(r4, h);
#pragma unroll
    for (int q = R_GEO4; q < R_FIX4; q++) {
        const float4 v = __ldg(r4 + q);
        h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
    }
}

// Geometry of one (pixel, primitive) pair: ray-plane intersection and local
// coordinates (Eq. 4, Eq. 5, ray depth of Eq. 13).
struct Geo {
    float t, u, v, r2sq;
};

// Stage 1.  Returns false when the pair cannot contribute: the ray misses
// the plane in front of the near plane, or the point lies beyond the
// conservative support radius of the kernel and the low-pass filter is out
// of reach too (then alpha_tilde < alpha_min; skipping never changes a
// result).  Every rounding step is explicit (fmaf / __fmul_rn / __fadd_rn)
// so that the forward pass and the backward reproduce identical values.
__device__ __forceinline__ bool eval_geometry(const float* h, const PixelRay& pr, float near_plane, Geo& g) {
    const float w = fmaf(h[R_HW0], pr.x, fmaf(h[R_HW1], pr.y, h[R_HW2]));
    if (!(w > 0.0f)) return false;
    const float t = rcp_approx(w);
    if (!(t > near_plane)) return false;
    const float U = fmaf(h[R_HU0], pr.x, fmaf(h[R_HU1], pr.y, h[R_HU2]));
    const float V = fmaf(h[R_HV0], pr.x, fmaf(h[R_HV1], pr.y, h[R_HV2]));
    const float u = __fmul_rn(U, t);
    const float v = __fmul_rn(V, t);
    const float r2sq = fmaf(u, u, __fmul_rn(v, v));
    g.t = t; g.u = u; g.v = v; g.r2sq = r2sq;
    if (r2sq > h[R_RHO2]) {
        if (!(h[R_FCUT] > 0.0f)) return false;
        const float dx = __fadd_rn(pr.x, -h[R_FPX]);
        const float dy = __fadd_rn(pr.y, -h[R_FPY]);
        const float dp2 = fmaf(dx, dx, __fmul_rn(dy, dy));
        const float Xf = __fmul_rn(__fmul_rn(dp2, pr.d2), __fmul_rn(__fmul_rn(t, t), h[R_FCOEF]));
        if (!(Xf < h[R_FCUT])) return false;
    }
    return true;
}

// Stage 2: the deformable radial kernel (Eq. 6 - Eq. 9), the low-pass
// filter (Eq. 10) and the clamp.  h holds header floats 0-23; hb points to
// the whole header (staged shared memory or the record in global memory)
// for the thresholds and the basis table; K is the basis count.  Returns
// true iff alpha_tilde >= alpha_min.
template <int KMAX, bool INFO>
__device__ __forceinline__ bool eval_kernel(const float* h, const float* hb, int K, const PixelRay& pr,
                                            const Geo& gm, float alpha_min, float alpha_max, float& a_out,
                                            EvalInfo* info = nullptr) {
    using RK = Rec<KMAX>;
    const float t = gm.t, u = gm.u, v = gm.v, r2sq = gm.r2sq;
    // polar angle from the first basis (Eq. 6 with reading: full circle)
    const float phi = polar_angle(u, v);
    // sector k: theta'_k <= phi < theta'_k1 (thresholds 1 .. K-1; the K-th is 2 pi)
    int k = 0;
#pragma unroll
    for (int q = 0; q < KMAX / 4; q++) {
        const float4 th4 = *reinterpret_cast<const float4*>(hb + RK::TH + 4 * q);
        if (4 * q + 1 < KMAX) k += (th4.x < phi) ? 1 : 0;
        if (4 * q + 2 < KMAX) k += (th4.y < phi) ? 1 : 0;
        if (4 * q + 3 < KMAX) k += (th4.z < phi) ? 1 : 0;
        if (4 * q + 4 < KMAX) k += (th4.w < phi) ? 1 : 0;
    }
    const int k1 = (k + 1 == K) ? 0 : k + 1;
    const float thk = k == 0 ? 0.0f : hb[RK::TH + k - 1];
    const float thk1 = hb[RK::TH + k];
    const float Ak = hb[RK::AA + k], Ak1 = hb[RK::AA + k1];
    const float ekx = hb[RK::EX + k], eky = hb[RK::EY + k];
    const float e1x = hb[RK::EX + k1], e1y = hb[RK::EY + k1];
    // Eq. 6: relative angle, cosine weight, inverse squared radius
    const float pg = __fmul_rn(kPi, rcp_approx(__fadd_rn(thk1, -thk)));
    const float dth = __fmul_rn(__fadd_rn(phi, -thk), pg);
    const float c = __cosf(dth);
    const float dif = __fadd_rn(Ak, -Ak1);
    const float Q = fmaf(c, dif, __fadd_rn(Ak, Ak1));
    // Eq. 7: L1 norm in the endpoint basis, (a, b) = [e_k e_k1]^-1 (u, v)
    const float idet = rcp_approx(fmaf(ekx, e1y, -__fmul_rn(eky, e1x)));
    const float a = __fmul_rn(fmaf(e1y, u, -__fmul_rn(e1x, v)), idet);
    const float b = __fmul_rn(fmaf(ekx, v, -__fmul_rn(eky, u)), idet);
    const float r1 = __fadd_rn(fabsf(a), fabsf(b));
    // Eq. 8 in base 2: g = 2^-X, X = log2(e)/2 (eta r1^2 + (1 - eta) r2^2 Q)
    const float X = fmaf(h[R_ETA2], __fmul_rn(r1, r1), __fmul_rn(h[R_ETA2C], __fmul_rn(r2sq, Q)));
    const float g = ex2_approx(-X);
    // Eq. 9 with o folded into the pieces
    float al;
    if (g < h[R_B1]) al = __fmul_rn(h[R_SLO], g);
    else if (g < h[R_B2]) al = fmaf(h[R_SMID], g, h[R_OMID]);
    else al = fmaf(h[R_SLO], g, h[R_OHI]);
    const float al_k = al;
    // Eq. 10: view-dependent low-pass filter, max with the kernel
    bool filt_eval = false, use_filter = false;
    float Xf = 0.0f, f = 0.0f;
    if (h[R_FCUT] > 0.0f) {
        const float dx = __fadd_rn(pr.x, -h[R_FPX]);
        const float dy = __fadd_rn(pr.y, -h[R_FPY]);
        const float dp2 = fmaf(dx, dx, __fmul_rn(dy, dy));
        Xf = __fmul_rn(__fmul_rn(dp2, pr.d2), __fmul_rn(__fmul_rn(t, t), h[R_FCOEF]));
        if (Xf < h[R_FCUT]) {
            filt_eval = true;
            f = __fmul_rn(h[R_OPA], ex2_approx(-Xf));
            if (f > al) { al = f; use_filter = true; }
        }
    }
    bool clamped = false;
    if (al > alpha_max) { al = alpha_max; clamped = true; }
    a_out = al;
    if (INFO) {
        info->t = t; info->u = u; info->v = v; info->phi = phi; info->r2sq = r2sq; info->dth = dth;
        info->c = c; info->Q = Q; info->a = a; info->b = b; info->r1 = r1; info->X = X; info->g = g;
        info->al_k = al_k; info->Xf = Xf; info->f = f; info->k = k;
        info->pg = pg; info->dif = dif;
        info->ekx = ekx; info->eky = eky; info->e1x = e1x; info->e1y = e1y; info->idet = idet;
        info->filt_eval = filt_eval; info->use_filter = use_filter; info->clamped = clamped;
    }
    return al >= alpha_min;
}

// Both stages for a record in global memory.
template <int KMAX, bool INFO>
__device__ __forceinline__ bool eval_pair(const float* __restrict__ rec, int K, const PixelRay& pr, float near_plane,
                                          float alpha_min, float alpha_max, float& t_out, float& a_out,
                                          EvalInfo* info = nullptr) {
    float h[R_FIX4 * 4];
    load_head_fix(reinterpret_cast<const float4*>(rec), h);
    Geo gm;
    if (!eval_geometry(h, pr, near_plane, gm)) return false;
    t_out = gm.t;
    return eval_kernel<KMAX, INFO>(h, rec, K, pr, gm, alpha_min, alpha_max, a_out, info);
}

// Launch-wide constants of one render.
struct FrameConst {
    int width, height, tiles_x, tiles_y;
    float ifx, ify, ox, oy;          // ray: d = (x ifx + ox, y ify + oy, 1)
    float near_plane, alpha_min, alpha_max, T_min;
    float bg[3];
    int order_mode;                  // DRK_ORDER_EXACT or DRK_ORDER_CACHE_SORT
};

__device__ __forceinline__ PixelRay make_ray(const FrameConst& fc, int x, int y) {
    PixelRay pr;
    pr.x = (float)x;
    pr.y = (float)y;
    const float dx = fmaf((float)x, fc.ifx, fc.ox);
    const float dy = fmaf((float)y, fc.ify, fc.oy);
    pr.d2 = __fadd_rn(fmaf(dx, dx, __fmul_rn(dy, dy)), 1.0f);
    return pr;
}

// Depth quantisation of sort keys (written by the preprocess on the device).
struct DepthQuant {
    float zmin, scale, inv_scale;
    int depth_bits;
};

}  // namespace drk
