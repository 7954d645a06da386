// train.cu -- activations of the learnable DRK parameters (supplementary
// "Parametrization") and the fused Adam update that fits them (supplementary
// "Model Training").
//
// One thread per primitive handles the arrays whose activation couples a
// primitive's values (quat, scale, theta, eta, tau, opacity): it reads the
// raw values once, forms the raw gradient by the chain rule, applies Adam,
// and writes the new raw values, the moments and the activated values the
// renderer reads next.  mu and color are not activated; their Adam update
// runs element by element in the same launch (blocks past the per-primitive
// ones), coalesced over the flat arrays.  The update is HBM-bound: every
// float of the raw parameters is read with its gradient and two moments and
// written back with the moments (28 bytes), and the activated arrays are
// written once more (32 bytes per activated float).
#include <algorithm>
#include <cmath>

#include "host.h"

namespace drk {
namespace {

constexpr float kSigCap = 1.f - 1e-3f;      // keeps every angular gap below pi
constexpr float kTauLo = -0.1f, kTauSpan = 1.09f;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr int kTrainThreads = 128;

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }
// sigmoid'(x) = sigmoid(x) sigmoid(-x): unlike s (1 - s) it keeps its relative
// accuracy where the sigmoid saturates (Adam's update does not shrink with
// the gradient, so a derivative rounded to 0 would change the step)
__device__ __forceinline__ float dsigm(float x) { return sigm(x) * sigm(-x); }

struct AdamK {
    float step_size[DRK_ARR_COUNT];   // lr / (1 - beta1^t)
    float inv_bc2;                    // 1 / sqrt(1 - beta2^t)
    float b1, b2, eps;
};

__device__ __forceinline__ void adam1(float& x, float g, float* __restrict__ m, float* __restrict__ v,
                                      const AdamK& h, int arr) {
    const float mm = h.b1 * *m + (1.f - h.b1) * g;
    const float vv = h.b2 * *v + (1.f - h.b2) * g * g;
    *m = mm;
    *v = vv;
    x -= h.step_size[arr] * mm / (sqrtf(vv) * h.inv_bc2 + h.eps);
}

// theta_k = 2 pi (w_0 + ... + w_{k-1}) / S,  w_j = min(sigmoid(x_j), cap) + 1/(K-2)
template <int KMAX>
__device__ __forceinline__ void theta_act(const float (&x)[KMAX], int K, float (&th)[KMAX]) {
    const float res = 1.f / (float)(K - 2);
    float w[KMAX], S = 0.f;
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
        w[k] = k < K ? fminf(sigm(x[k]), kSigCap) + res : 0.f;
        S += w[k];
    }
    const float sc = kTwoPiF / S;
    float c = 0.f;
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
        th[k] = c * sc;
        c += w[k];
    }
}

// raw-angle gradient: d theta_k / d w_j = 2 pi ([j < k] / S - C_k / S^2)
template <int KMAX>
__device__ __forceinline__ void theta_grad(const float (&x)[KMAX], const float (&g)[KMAX], int K,
                                           float (&gx)[KMAX]) {
    const float res = 1.f / (float)(K - 2);
    float sg[KMAX], w[KMAX], S = 0.f;
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
        sg[k] = k < K ? sigm(x[k]) : 0.f;
        w[k] = k < K ? fminf(sg[k], kSigCap) + res : 0.f;
        S += w[k];
    }
    float c = 0.f, D = 0.f;
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
        D += g[k] * c;           // sum_k g_k C_k
        c += w[k];
    }
    const float a = kTwoPiF / S, b = kTwoPiF * D / (S * S);
    float after = 0.f;           // sum over k > j of g_k
#pragma unroll
    for (int j = KMAX - 1; j >= 0; j--) {
        const float gw = a * after - b;
        gx[j] = (j < K && sg[j] < kSigCap) ? gw * dsigm(x[j]) : 0.f;
        after += g[j];
    }
}

__device__ __forceinline__ void quat_act(const float (&x)[4], float (&q)[4]) {
    const float nr2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2] + x[3] * x[3];
    if (nr2 > 0.f) {
        const float inv = 1.f / sqrtf(nr2);
#pragma unroll
        for (int c = 0; c < 4; c++) q[c] = x[c] * inv;
    } else {
        q[0] = 1.f;
        q[1] = q[2] = q[3] = 0.f;
    }
}

__device__ __forceinline__ void quat_grad(const float (&x)[4], const float (&g)[4], float (&gx)[4]) {
    const float nr2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2] + x[3] * x[3];
    if (!(nr2 > 0.f)) {
        gx[0] = gx[1] = gx[2] = gx[3] = 0.f;
        return;
    }
    const float inv = 1.f / sqrtf(nr2);
    float q[4], qg = 0.f;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        q[c] = x[c] * inv;
        qg += q[c] * g[c];
    }
#pragma unroll
    for (int c = 0; c < 4; c++) gx[c] = (g[c] - q[c] * qg) * inv;
}

// ---- per-primitive kernels ------------------------------------------------

enum Mode { ACTIVATE = 0, BACKWARD = 1, ADAM = 2 };

struct PrimArgs {
    drk_raw_params_t raw;
    drk_params_grad_t g, m, v, out;    // out: activated (ACTIVATE, ADAM) or raw gradient (BACKWARD)
    AdamK h;
    int64_t n_elem_mu, n_elem_col;     // flat sizes of mu and color
    int64_t prim_blocks;
};

template <int KMAX, int MODE>
__global__ void __launch_bounds__(kTrainThreads) train_kernel(PrimArgs A) {
    const int K = A.raw.K;
    if ((int64_t)blockIdx.x >= A.prim_blocks) {
        // element-wise part: mu then color (identity activations)
        if (MODE == ACTIVATE) return;
        const int64_t stride = (int64_t)(gridDim.x - A.prim_blocks) * blockDim.x;
        const int64_t total = A.n_elem_mu + A.n_elem_col;
        for (int64_t e = ((int64_t)blockIdx.x - A.prim_blocks) * blockDim.x + threadIdx.x; e < total; e += stride) {
            const bool is_mu = e < A.n_elem_mu;
            const int64_t j = is_mu ? e : e - A.n_elem_mu;
            float* x = is_mu ? A.raw.mu : A.raw.color;
            const float g = is_mu ? A.g.mu[j] : A.g.color[j];
            if (MODE == BACKWARD) {
                (is_mu ? A.out.mu : A.out.color)[j] = g;
            } else {
                float xv = x[j];
                adam1(xv, g, (is_mu ? A.m.mu : A.m.color) + j, (is_mu ? A.v.mu : A.v.color) + j, A.h,
                      is_mu ? DRK_ARR_MU : DRK_ARR_COLOR);
                x[j] = xv;
            }
        }
        return;
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.raw.n) return;

    // quaternion
    {
        float x[4], q[4];
#pragma unroll
        for (int c = 0; c < 4; c++) x[c] = A.raw.quat[4 * i + c];
        if (MODE != ACTIVATE) {
            float g[4], gx[4];
#pragma unroll
            for (int c = 0; c < 4; c++) g[c] = A.g.quat[4 * i + c];
            quat_grad(x, g, gx);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                if (MODE == BACKWARD) {
                    A.out.quat[4 * i + c] = gx[c];
                } else {
                    adam1(x[c], gx[c], A.m.quat + 4 * i + c, A.v.quat + 4 * i + c, A.h, DRK_ARR_QUAT);
                    A.raw.quat[4 * i + c] = x[c];
                }
            }
        }
        if (MODE != BACKWARD) {
            quat_act(x, q);
#pragma unroll
            for (int c = 0; c < 4; c++) A.out.quat[4 * i + c] = q[c];
        }
    }
    // radial lengths s_k = exp(x_k)
    const int64_t base = (int64_t)K * i;
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
        if (k >= K) break;
        float x = A.raw.scale[base + k];
        if (MODE != ACTIVATE) {
            const float gx = A.g.scale[base + k] * expf(x);
            if (MODE == BACKWARD) {
                A.out.scale[base + k] = gx;
            } else {
                adam1(x, gx, A.m.scale + base + k, A.v.scale + base + k, A.h, DRK_ARR_SCALE);
                A.raw.scale[base + k] = x;
            }
        }
        if (MODE != BACKWARD) A.out.scale[base + k] = expf(x);
    }
    // polar angles
    {
        float x[KMAX], th[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; k++) x[k] = k < K ? A.raw.theta[base + k] : 0.f;
        if (MODE != ACTIVATE) {
            float g[KMAX], gx[KMAX];
#pragma unroll
            for (int k = 0; k < KMAX; k++) g[k] = k < K ? A.g.theta[base + k] : 0.f;
            theta_grad<KMAX>(x, g, K, gx);
#pragma unroll
            for (int k = 0; k < KMAX; k++) {
                if (k >= K) break;
                if (MODE == BACKWARD) {
                    A.out.theta[base + k] = gx[k];
                } else {
                    adam1(x[k], gx[k], A.m.theta + base + k, A.v.theta + base + k, A.h, DRK_ARR_THETA);
                    A.raw.theta[base + k] = x[k];
                }
            }
        }
        if (MODE != BACKWARD) {
            theta_act<KMAX>(x, K, th);
#pragma unroll
            for (int k = 0; k < KMAX; k++)
                if (k < K) A.out.theta[base + k] = th[k];
        }
    }
    // eta, tau, opacity: sigmoid with a linear remap
    {
        float* const rs[3] = {A.raw.eta, A.raw.tau, A.raw.opacity};
        const float* const gs[3] = {A.g.eta, A.g.tau, A.g.opacity};
        float* const ms[3] = {A.m.eta, A.m.tau, A.m.opacity};
        float* const vs[3] = {A.v.eta, A.v.tau, A.v.opacity};
        float* const os[3] = {A.out.eta, A.out.tau, A.out.opacity};
        const float lo[3] = {0.f, kTauLo, 0.f}, span[3] = {1.f, kTauSpan, 1.f};
        const int arr[3] = {DRK_ARR_ETA, DRK_ARR_TAU, DRK_ARR_OPACITY};
#pragma unroll
        for (int p = 0; p < 3; p++) {
            float x = rs[p][i];
            if (MODE != ACTIVATE) {
                const float gx = gs[p][i] * span[p] * dsigm(x);
                if (MODE == BACKWARD) {
                    os[p][i] = gx;
                } else {
                    adam1(x, gx, ms[p] + i, vs[p] + i, A.h, arr[p]);
                    rs[p][i] = x;
                }
            }
            if (MODE != BACKWARD) os[p][i] = lo[p] + span[p] * sigm(x);
        }
    }
}

int64_t color_count(const drk_raw_params_t* r) {
    const int64_t per = r->sh_degree < 0 ? 3 : 3 * (int64_t)(r->sh_degree + 1) * (r->sh_degree + 1);
    return per * r->n;
}

drk_status_t check_raw(const drk_raw_params_t* r) {
    if (!r) return fail(DRK_ERR_INVALID_ARG, "raw parameters are NULL");
    if (r->n < 0 || r->n >= (int64_t(1) << 31)) return fail(DRK_ERR_INVALID_ARG, "n = %lld out of range", (long long)r->n);
    if (r->K < 3 || r->K > 16) return fail(DRK_ERR_INVALID_ARG, "K = %d not in [3, 16]", r->K);
    if (r->sh_degree < -1 || r->sh_degree > 3)
        return fail(DRK_ERR_INVALID_ARG, "sh_degree = %d not in [-1, 3]", r->sh_degree);
    if (r->n > 0 && (!r->mu || !r->quat || !r->scale || !r->theta || !r->eta || !r->tau || !r->opacity || !r->color))
        return fail(DRK_ERR_INVALID_ARG, "a raw parameter array is NULL");
    return DRK_OK;
}

drk_status_t check_arrays(const drk_params_grad_t* a, int64_t n, bool need_mu_color, const char* what) {
    if (!a) return fail(DRK_ERR_INVALID_ARG, "%s is NULL", what);
    if (n > 0 && (!a->quat || !a->scale || !a->theta || !a->eta || !a->tau || !a->opacity))
        return fail(DRK_ERR_INVALID_ARG, "an array of %s is NULL", what);
    if (n > 0 && need_mu_color && (!a->mu || !a->color))
        return fail(DRK_ERR_INVALID_ARG, "mu or color of %s is NULL", what);
    return DRK_OK;
}

template <int MODE>
drk_status_t launch(PrimArgs& A, cudaStream_t st) {
    const drk_raw_params_t& r = A.raw;
    A.n_elem_mu = 3 * r.n;
    A.n_elem_col = color_count(&r);
    A.prim_blocks = (r.n + kTrainThreads - 1) / kTrainThreads;
    int64_t elem_blocks = 0;
    if (MODE != ACTIVATE) {
        // grid-stride over the flat arrays; eight blocks per SM at most
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        elem_blocks = std::min<int64_t>((A.n_elem_mu + A.n_elem_col + kTrainThreads - 1) / kTrainThreads,
                                        (int64_t)std::max(sms, 1) * 8);
    }
    const int64_t blocks = A.prim_blocks + elem_blocks;
    if (blocks == 0) return DRK_OK;
    if (r.K <= 8)
        train_kernel<8, MODE><<<(unsigned)blocks, kTrainThreads, 0, st>>>(A);
    else
        train_kernel<16, MODE><<<(unsigned)blocks, kTrainThreads, 0, st>>>(A);
    note_launch();
    return check_launch();
}

}  // namespace
}  // namespace drk

using namespace drk;

extern "C" {

drk_status_t drk_activate(const drk_raw_params_t* raw, const drk_params_grad_t* out, void* stream) {
    drk_status_t s;
    if ((s = check_raw(raw)) != DRK_OK) return s;
    if ((s = check_arrays(out, raw->n, false, "out")) != DRK_OK) return s;
    PrimArgs A{};
    A.raw = *raw;
    A.out = *out;
    return launch<ACTIVATE>(A, reinterpret_cast<cudaStream_t>(stream));
}

drk_status_t drk_activate_backward(const drk_raw_params_t* raw, const drk_params_grad_t* g_act,
                                   const drk_params_grad_t* g_raw, void* stream) {
    drk_status_t s;
    if ((s = check_raw(raw)) != DRK_OK) return s;
    if ((s = check_arrays(g_act, raw->n, true, "g_act")) != DRK_OK) return s;
    if ((s = check_arrays(g_raw, raw->n, true, "g_raw")) != DRK_OK) return s;
    PrimArgs A{};
    A.raw = *raw;
    A.g = *g_act;
    A.out = *g_raw;
    return launch<BACKWARD>(A, reinterpret_cast<cudaStream_t>(stream));
}

drk_status_t drk_adam_step(const drk_raw_params_t* raw, const drk_params_grad_t* g_act, const drk_params_grad_t* m,
                           const drk_params_grad_t* v, const drk_adam_t* hp, const drk_params_grad_t* act,
                           void* stream) {
    drk_status_t s;
    if ((s = check_raw(raw)) != DRK_OK) return s;
    if ((s = check_arrays(g_act, raw->n, true, "g_act")) != DRK_OK) return s;
    if ((s = check_arrays(m, raw->n, true, "m")) != DRK_OK) return s;
    if ((s = check_arrays(v, raw->n, true, "v")) != DRK_OK) return s;
    if ((s = check_arrays(act, raw->n, false, "act")) != DRK_OK) return s;
    if (!hp) return fail(DRK_ERR_INVALID_ARG, "hyper-parameters are NULL");
    if (hp->step < 1) return fail(DRK_ERR_INVALID_ARG, "step = %lld < 1", (long long)hp->step);
    if (!(hp->beta1 >= 0.f && hp->beta1 < 1.f) || !(hp->beta2 >= 0.f && hp->beta2 < 1.f))
        return fail(DRK_ERR_INVALID_ARG, "beta1 = %g, beta2 = %g not in [0, 1)", hp->beta1, hp->beta2);
    if (!(hp->eps >= 0.f) || !std::isfinite(hp->eps)) return fail(DRK_ERR_INVALID_ARG, "eps = %g", hp->eps);
    for (int k = 0; k < DRK_ARR_COUNT; k++)
        if (!std::isfinite(hp->lr[k]) || hp->lr[k] < 0.f)
            return fail(DRK_ERR_INVALID_ARG, "lr[%d] = %g", k, hp->lr[k]);
    PrimArgs A{};
    A.raw = *raw;
    A.g = *g_act;
    A.m = *m;
    A.v = *v;
    A.out = *act;
    const double t = (double)hp->step;
    const double bc1 = 1.0 - std::pow((double)hp->beta1, t);
    const double bc2 = 1.0 - std::pow((double)hp->beta2, t);
    for (int k = 0; k < DRK_ARR_COUNT; k++) A.h.step_size[k] = (float)((double)hp->lr[k] / bc1);
    A.h.inv_bc2 = (float)(1.0 / std::sqrt(bc2));
    A.h.b1 = hp->beta1;
    A.h.b2 = hp->beta2;
    A.h.eps = hp->eps;
    return launch<ADAM>(A, reinterpret_cast<cudaStream_t>(stream));
}

double drk_lr_exponential(int64_t step, double lr_init, double lr_final, int64_t max_steps) {
    double r = max_steps > 0 ? (double)step / (double)max_steps : 1.0;
    r = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
    return std::exp((1.0 - r) * std::log(lr_init) + r * std::log(lr_final));
}

}  // extern "C"
