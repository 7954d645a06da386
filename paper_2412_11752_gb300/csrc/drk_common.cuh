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
//   9      eta * log2(e) / 2         (Eq. 8, base-2 exponent)
//   10     (1 - eta) * log2(e) / 2
//   11     o
//   12,13  Psi breakpoints (1 + tau)/4, (3 - tau)/4          (Eq. 9)
//   14     o (1 - tau)/(1 + tau)      outer slope (x o)
//   15     o (1 + tau)/(1 - tau)      middle slope (x o)
//   16     -o tau/(1 - tau)           middle offset (x o)
//   17     2 o tau/(1 + tau)          upper offset (x o)
//   18,19  projected centre minus 0.5 (pixel-index coordinates)   (Eq. 10)
//   20     log2(e) / (2 s_l^2 N^2)    filter exponent per (px^2 |d|^2 t^2)
//   21     filter cut: evaluate the filter only while its base-2 exponent
//          is below this (beyond it the filter is < alpha_min / 2); < 0 = off
//   22     tau
//   23     unused
//   24..   theta'_1 .. theta'_{KMAX-1}, padded with +1e30
// then KMAX sectors of 8 floats:
//   theta'_k, pi / gap_k, A_k + A_k1, A_k - A_k1, Minv (row-major, 4)
//   with A_j = 1 / (2 s_j^2) (Eq. 6) and Minv = [e_k e_k1]^-1 (Eq. 7),
//   e_j = s_j (cos theta'_j, sin theta'_j).
// ---------------------------------------------------------------------------
enum : int {
    R_HU0 = 0, R_HU1, R_HU2, R_HV0, R_HV1, R_HV2, R_HW0, R_HW1, R_HW2,
    R_ETA2, R_ETA2C, R_OPA, R_B1, R_B2, R_SLO, R_SMID, R_OMID, R_OHI,
    R_FPX, R_FPY, R_FCOEF, R_FCUT, R_TAU, R_UNUSED,
    R_TH = 24
};
enum : int { S_TH = 0, S_PG, S_SUM, S_DIF, S_M00, S_M01, S_M10, S_M11, S_STRIDE };

template <int KMAX>
struct Rec {
    static constexpr int HDR = ((R_TH + KMAX - 1) + 3) / 4 * 4;
    static constexpr int STRIDE = HDR + S_STRIDE * KMAX;      // floats
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
    static constexpr int STRIDE = ((B_RHO + KMAX) + 3) / 4 * 4;
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

// ---------------------------------------------------------------------------
// Per-pixel constants of the camera ray (integer pixel indices).
struct PixelRay {
    float x, y;    // pixel indices as float
    float d2;      // |d|^2 of the unnormalised camera-space ray (z = 1)
};

// Intermediate values of one evaluation, kept when the derivative is needed.
struct EvalInfo {
    float t, u, v, phi, r2sq, dth, c, Q, a, b, r1, X, g, al_k, Xf, f;
    int k;
    bool filt_eval, use_filter, clamped;
};

// One (pixel, primitive) evaluation: Eq. 4 - Eq. 10 and the clamp.  Every
// rounding step is explicit (fmaf / __fmul_rn / __fadd_rn) so that the
// forward pass and the backward replay produce bit-identical values.
// Returns true iff the pair contributes (alpha_tilde >= alpha_min).
template <int KMAX, bool INFO>
__device__ __forceinline__ bool eval_pair(const float* __restrict__ r, const PixelRay& pr, float near_plane,
                                          float alpha_min, float alpha_max, float& t_out, float& a_out,
                                          EvalInfo* info = nullptr) {
    constexpr int HDR = Rec<KMAX>::HDR;
    const float w = fmaf(r[R_HW0], pr.x, fmaf(r[R_HW1], pr.y, r[R_HW2]));
    if (!(w > 0.0f)) return false;
    const float t = rcp_approx(w);
    if (!(t > near_plane)) return false;
    const float U = fmaf(r[R_HU0], pr.x, fmaf(r[R_HU1], pr.y, r[R_HU2]));
    const float V = fmaf(r[R_HV0], pr.x, fmaf(r[R_HV1], pr.y, r[R_HV2]));
    const float u = __fmul_rn(U, t);
    const float v = __fmul_rn(V, t);
    const float r2sq = fmaf(u, u, __fmul_rn(v, v));
    // polar angle from the first basis (Eq. 6 with reading: full circle)
    float phi = atan2f(v, u);
    phi = phi < 0.0f ? __fadd_rn(phi, kTwoPi) : phi;
    int k = 0;
#pragma unroll
    for (int j = 1; j < KMAX; j++) k += (r[R_TH + j - 1] < phi) ? 1 : 0;
    const float4 s0 = *reinterpret_cast<const float4*>(r + HDR + S_STRIDE * k);
    const float4 s1 = *reinterpret_cast<const float4*>(r + HDR + S_STRIDE * k + 4);
    // Eq. 6: relative angle, cosine weight, inverse squared radius
    const float dth = __fmul_rn(__fadd_rn(phi, -s0.x), s0.y);
    const float c = __cosf(dth);
    const float Q = fmaf(c, s0.w, s0.z);
    // Eq. 7: L1 norm in the endpoint basis
    const float a = fmaf(s1.x, u, __fmul_rn(s1.y, v));
    const float b = fmaf(s1.z, u, __fmul_rn(s1.w, v));
    const float r1 = __fadd_rn(fabsf(a), fabsf(b));
    // Eq. 8 in base 2: g = 2^-X, X = log2(e)/2 (eta r1^2 + (1 - eta) r2^2 Q)
    const float X = fmaf(r[R_ETA2], __fmul_rn(r1, r1), __fmul_rn(r[R_ETA2C], __fmul_rn(r2sq, Q)));
    const float g = ex2_approx(-X);
    // Eq. 9 with o folded into the pieces
    float al;
    if (g < r[R_B1]) al = __fmul_rn(r[R_SLO], g);
    else if (g < r[R_B2]) al = fmaf(r[R_SMID], g, r[R_OMID]);
    else al = fmaf(r[R_SLO], g, r[R_OHI]);
    const float al_k = al;
    // Eq. 10: view-dependent low-pass filter, max with the kernel
    bool filt_eval = false, use_filter = false;
    float Xf = 0.0f, f = 0.0f;
    if (r[R_FCUT] > 0.0f) {
        const float dx = __fadd_rn(pr.x, -r[R_FPX]);
        const float dy = __fadd_rn(pr.y, -r[R_FPY]);
        const float dp2 = fmaf(dx, dx, __fmul_rn(dy, dy));
        Xf = __fmul_rn(__fmul_rn(dp2, pr.d2), __fmul_rn(__fmul_rn(t, t), r[R_FCOEF]));
        if (Xf < r[R_FCUT]) {
            filt_eval = true;
            f = __fmul_rn(r[R_OPA], ex2_approx(-Xf));
            if (f > al) { al = f; use_filter = true; }
        }
    }
    bool clamped = false;
    if (al > alpha_max) { al = alpha_max; clamped = true; }
    t_out = t;
    a_out = al;
    if (INFO) {
        info->t = t; info->u = u; info->v = v; info->phi = phi; info->r2sq = r2sq; info->dth = dth;
        info->c = c; info->Q = Q; info->a = a; info->b = b; info->r1 = r1; info->X = X; info->g = g;
        info->al_k = al_k; info->Xf = Xf; info->f = f; info->k = k;
        info->filt_eval = filt_eval; info->use_filter = use_filter; info->clamped = clamped;
    }
    return al >= alpha_min;
}

// ---------------------------------------------------------------------------
// Per-pixel depth-order buffer (the exact variant of the paper's
// cache-sorting, Sec. 4.4 and the supplementary algorithm).
//
// Entries are (key, alpha) with key = (float bits of r_t) << 32 | index, so
// an unsigned compare orders by (r_t, primitive index).  The buffer is kept
// sorted ascending in registers; empty slots hold key = ~0.  Because the
// tile list is visited in ascending order of a per-(primitive, tile) lower
// bound of r_t, every buffered entry whose r_t is below the bound of the
// next list item can be composited: no later item can precede it.  When the
// buffer is full, the largest key is evicted and becomes the pass horizon;
// keys at or beyond the horizon are left for another pass over the list,
// which starts at that horizon.  The composited order is therefore exactly
// the (r_t, index) order for any capacity.
// ---------------------------------------------------------------------------
template <int CAP>
struct KBuf {
    uint64_t key[CAP];
    float alpha[CAP];

    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int i = 0; i < CAP; i++) { key[i] = ~0ull; alpha[i] = 0.0f; }
    }
    __device__ __forceinline__ bool empty() const { return key[0] == ~0ull; }
    __device__ __forceinline__ float front_t() const { return __uint_as_float((uint32_t)(key[0] >> 32)); }
    // insert; returns the key that fell off the end (~0 if none)
    __device__ __forceinline__ uint64_t insert(uint64_t k, float a) {
#pragma unroll
        for (int i = 0; i < CAP; i++) {
            const bool sw = k < key[i];
            const uint64_t tk = sw ? k : key[i];
            const float ta = sw ? a : alpha[i];
            k = sw ? key[i] : k;
            a = sw ? alpha[i] : a;
            key[i] = tk;
            alpha[i] = ta;
        }
        return k;
    }
    __device__ __forceinline__ void pop_front() {
#pragma unroll
        for (int i = 0; i < CAP - 1; i++) { key[i] = key[i + 1]; alpha[i] = alpha[i + 1]; }
        key[CAP - 1] = ~0ull;
        alpha[CAP - 1] = 0.0f;
    }
};

// Launch-wide constants of one render.
struct FrameConst {
    int width, height, tiles_x, tiles_y;
    float ifx, ify, ox, oy;          // ray: d = (x ifx + ox, y ify + oy, 1)
    float near_plane, alpha_min, alpha_max, T_min;
    float bg[3];
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
