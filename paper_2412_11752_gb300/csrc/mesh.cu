// mesh.cu -- conversion of polygon meshes to DRKs (Sec. 5.4 "Converting
// Mesh to DRK" and the supplementary section of the same name).
//
// One thread per face: gather the face's vertices, build the plane frame
// (Newell normal, R_x towards the first vertex), project the vertices into
// the plane, spread the extra endpoints over the edges, and write one DRK
// whose L1 contours (eta = 1, Eq. 7-8) are scaled copies of the polygon,
// the polygon itself being the contour g = edge_density.  Nothing here is
// iterative; the conversion is a single pass over the faces.
#include <cmath>

#include "host.h"

namespace drk {
namespace {

constexpr int kMeshThreads = 128;
constexpr int kMaxFace = 16;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kPiF = 3.14159265358979323846f;
constexpr float kGapMargin = 1e-3f;

struct MeshArgs {
    const float* verts;
    int64_t n_verts;
    const int32_t* faces;
    int64_t n_faces;
    int face_size;
    const float* face_color;
    int K;
    float inv_edge;          // 1 / sqrt(-2 ln edge_density)
    float tau, opacity, ambient, diffuse;
    float lx, ly, lz;        // unit light direction
    drk_params_grad_t out;
    int32_t* status;
};

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// unit quaternion (w, x, y, z), w >= 0, of the rotation whose columns are
// the axes X, Y, Z (divide by the largest of 4w^2, 4x^2, 4y^2, 4z^2)
__device__ void quat_of_frame(const float X[3], const float Y[3], const float Z[3], float q[4]) {
    // R[r][c]: column c is the c-th axis
    const float r00 = X[0], r10 = X[1], r20 = X[2];
    const float r01 = Y[0], r11 = Y[1], r21 = Y[2];
    const float r02 = Z[0], r12 = Z[1], r22 = Z[2];
    const float tr = r00 + r11 + r22;
    if (tr >= r00 && tr >= r11 && tr >= r22) {
        const float w = 0.5f * sqrtf(1.f + tr), i4 = 0.25f / w;
        q[0] = w; q[1] = (r21 - r12) * i4; q[2] = (r02 - r20) * i4; q[3] = (r10 - r01) * i4;
    } else if (r00 >= r11 && r00 >= r22) {
        const float x = 0.5f * sqrtf(1.f + r00 - r11 - r22), i4 = 0.25f / x;
        q[0] = (r21 - r12) * i4; q[1] = x; q[2] = (r01 + r10) * i4; q[3] = (r02 + r20) * i4;
    } else if (r11 >= r22) {
        const float y = 0.5f * sqrtf(1.f - r00 + r11 - r22), i4 = 0.25f / y;
        q[0] = (r02 - r20) * i4; q[1] = (r01 + r10) * i4; q[2] = y; q[3] = (r12 + r21) * i4;
    } else {
        const float z = 0.5f * sqrtf(1.f - r00 - r11 + r22), i4 = 0.25f / z;
        q[0] = (r10 - r01) * i4; q[1] = (r02 + r20) * i4; q[2] = (r12 + r21) * i4; q[3] = z;
    }
    const float inv = 1.f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float sg = q[0] < 0.f ? -inv : inv;
    for (int c = 0; c < 4; c++) q[c] *= sg;
}

__global__ void __launch_bounds__(kMeshThreads) mesh_kernel(MeshArgs A) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= A.n_faces) return;
    const int K = A.K;
    const int32_t* row = A.faces + (int64_t)A.face_size * f;
    int m = 0;
    while (m < A.face_size && row[m] >= 0) m++;
    int st = (m < 3 || m > K) ? 1 : 0;
    for (int j = m; j < A.face_size; j++)
        if (row[j] >= 0) st = 1;
    for (int j = 0; j < m; j++)
        if ((int64_t)row[j] >= A.n_verts) st = 1;

    float mu[3] = {0.f, 0.f, 0.f}, q[4] = {1.f, 0.f, 0.f, 0.f}, col[3] = {0.f, 0.f, 0.f};
    float ex[kMaxFace], ey[kMaxFace];
    if (st == 0) {
        float P[kMaxFace][3];
        for (int j = 0; j < m; j++) {
            const float* v = A.verts + 3 * (int64_t)row[j];
            for (int c = 0; c < 3; c++) P[j][c] = v[c];
        }
        for (int c = 0; c < 3; c++) {
            float s = 0.f;
            for (int j = 0; j < m; j++) s += P[j][c];
            mu[c] = s / (float)m;
        }
        float size2 = 0.f, n[3] = {0.f, 0.f, 0.f};
        for (int j = 0; j < m; j++) {
            float a[3], b[3], c3[3];
            for (int c = 0; c < 3; c++) {
                a[c] = P[j][c] - mu[c];
                b[c] = P[(j + 1) % m][c] - mu[c];
            }
            size2 = fmaxf(size2, dot3(a, a));
            cross3(a, b, c3);
            for (int c = 0; c < 3; c++) n[c] += c3[c];
        }
        const float nn = sqrtf(dot3(n, n));
        if (!(nn > 1e-12f * size2)) st = 1;
        float Z[3], X[3], Y[3];
        if (st == 0) {
            for (int c = 0; c < 3; c++) Z[c] = n[c] / nn;
            float d0[3];
            for (int c = 0; c < 3; c++) d0[c] = P[0][c] - mu[c];
            const float dz = dot3(d0, Z);
            for (int c = 0; c < 3; c++) d0[c] -= Z[c] * dz;
            const float l0 = sqrtf(dot3(d0, d0));
            if (!(l0 > 1e-12f * sqrtf(size2))) st = 1;
            else {
                for (int c = 0; c < 3; c++) X[c] = d0[c] / l0;
                cross3(Z, X, Y);
            }
        }
        if (st == 0) {
            // vertices in the plane, then the K endpoints (extra ones on edges)
            float lx[kMaxFace], ly[kMaxFace];
            for (int j = 0; j < m; j++) {
                float d[3];
                for (int c = 0; c < 3; c++) d[c] = P[j][c] - mu[c];
                lx[j] = dot3(d, X);
                ly[j] = dot3(d, Y);
            }
            const int extra = K - m;
            int e = 0;
            for (int j = 0; j < m; j++) {
                const int jn = (j + 1) % m;
                const int cnt = extra / m + (j < extra % m ? 1 : 0);
                ex[e] = lx[j];
                ey[e] = ly[j];
                e++;
                for (int i = 1; i <= cnt; i++) {
                    const float t = (float)i / (float)(cnt + 1);
                    ex[e] = lx[j] + (lx[jn] - lx[j]) * t;
                    ey[e] = ly[j] + (ly[jn] - ly[j]) * t;
                    e++;
                }
            }
            // angles: strictly increasing, every cyclic gap below pi - margin
            float prev = 0.f;
            for (int k = 1; k <= K; k++) {
                float th = kTwoPiF;
                if (k < K) {
                    th = atan2f(ey[k], ex[k]);
                    if (th < 0.f) th += kTwoPiF;
                }
                const float gap = th - prev;
                if (!(gap > 0.f) || !(gap < kPiF - kGapMargin)) st = 2;
                prev = th;
            }
            quat_of_frame(X, Y, Z, q);
            const float shade = A.ambient + A.diffuse * fabsf(Z[0] * A.lx + Z[1] * A.ly + Z[2] * A.lz);
            for (int c = 0; c < 3; c++) col[c] = (A.face_color ? A.face_color[3 * f + c] : 1.f) * shade;
        }
    }

    const int64_t kb = (int64_t)K * f;
    if (st == 0) {
        for (int c = 0; c < 3; c++) A.out.mu[3 * f + c] = mu[c];
        for (int c = 0; c < 4; c++) A.out.quat[4 * f + c] = q[c];
        for (int k = 0; k < K; k++) {
            float th = 0.f;
            if (k > 0) {
                th = atan2f(ey[k], ex[k]);
                if (th < 0.f) th += kTwoPiF;
            }
            A.out.theta[kb + k] = th;
            A.out.scale[kb + k] = sqrtf(ex[k] * ex[k] + ey[k] * ey[k]) * A.inv_edge;
        }
        A.out.eta[f] = 1.f;
        A.out.tau[f] = A.tau;
        A.out.opacity[f] = A.opacity;
        for (int c = 0; c < 3; c++) A.out.color[3 * f + c] = col[c];
    } else {
        for (int c = 0; c < 3; c++) A.out.mu[3 * f + c] = 0.f;
        A.out.quat[4 * f] = 1.f;
        for (int c = 1; c < 4; c++) A.out.quat[4 * f + c] = 0.f;
        for (int k = 0; k < K; k++) {
            A.out.theta[kb + k] = kTwoPiF * (float)k / (float)K;
            A.out.scale[kb + k] = 1e-3f;
        }
        A.out.eta[f] = 1.f;
        A.out.tau[f] = A.tau;
        A.out.opacity[f] = 0.f;
        for (int c = 0; c < 3; c++) A.out.color[3 * f + c] = 0.f;
    }
    if (A.status) A.status[f] = st;
}

}  // namespace
}  // namespace drk

using namespace drk;

extern "C" {

void drk_mesh_options_default(drk_mesh_options_t* opt) {
    if (!opt) return;
    opt->K = 4;
    opt->edge_density = 0.5f;
    opt->tau = 0.95f;
    opt->opacity = 1.f;
    opt->light[0] = 0.3f;
    opt->light[1] = -0.5f;
    opt->light[2] = -0.8f;
    opt->ambient = 0.35f;
    opt->diffuse = 0.65f;
}

drk_status_t drk_mesh_to_drk(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                             int32_t face_size, const float* face_color, const drk_mesh_options_t* opt,
                             const drk_params_grad_t* out, int32_t* face_status, void* stream) {
    if (!opt || !out) return fail(DRK_ERR_INVALID_ARG, "options or outputs are NULL");
    if (n_verts < 0 || n_faces < 0 || n_faces >= (int64_t(1) << 31))
        return fail(DRK_ERR_INVALID_ARG, "n_verts = %lld, n_faces = %lld", (long long)n_verts, (long long)n_faces);
    if (face_size < 3 || face_size > kMaxFace)
        return fail(DRK_ERR_INVALID_ARG, "face_size = %d not in [3, %d]", face_size, kMaxFace);
    if (opt->K < 3 || opt->K > 16) return fail(DRK_ERR_INVALID_ARG, "K = %d not in [3, 16]", opt->K);
    if (!(opt->edge_density > 0.f && opt->edge_density < 1.f))
        return fail(DRK_ERR_INVALID_ARG, "edge_density = %g not in (0, 1)", opt->edge_density);
    if (!(opt->tau > -1.f && opt->tau < 1.f)) return fail(DRK_ERR_INVALID_ARG, "tau = %g not in (-1, 1)", opt->tau);
    if (!(opt->opacity > 0.f && opt->opacity <= 1.f))
        return fail(DRK_ERR_INVALID_ARG, "opacity = %g not in (0, 1]", opt->opacity);
    const double l2 = (double)opt->light[0] * opt->light[0] + (double)opt->light[1] * opt->light[1] +
                      (double)opt->light[2] * opt->light[2];
    if (!(l2 > 0.0) || !std::isfinite(l2) || !std::isfinite(opt->ambient) || !std::isfinite(opt->diffuse))
        return fail(DRK_ERR_INVALID_ARG, "light direction or shading coefficients invalid");
    if (n_faces == 0) return DRK_OK;
    if (!faces || (n_verts > 0 && !verts))
        return fail(DRK_ERR_INVALID_ARG, "faces or verts are NULL");
    if (!out->mu || !out->quat || !out->scale || !out->theta || !out->eta || !out->tau || !out->opacity ||
        !out->color)
        return fail(DRK_ERR_INVALID_ARG, "an output array is NULL");
    MeshArgs A{};
    A.verts = verts;
    A.n_verts = n_verts;
    A.faces = faces;
    A.n_faces = n_faces;
    A.face_size = face_size;
    A.face_color = face_color;
    A.K = opt->K;
    A.inv_edge = (float)(1.0 / std::sqrt(-2.0 * std::log((double)opt->edge_density)));
    A.tau = opt->tau;
    A.opacity = opt->opacity;
    A.ambient = opt->ambient;
    A.diffuse = opt->diffuse;
    const double il = 1.0 / std::sqrt(l2);
    A.lx = (float)(opt->light[0] * il);
    A.ly = (float)(opt->light[1] * il);
    A.lz = (float)(opt->light[2] * il);
    A.out = *out;
    A.status = face_status;
    const unsigned blocks = (unsigned)((n_faces + kMeshThreads - 1) / kMeshThreads);
    mesh_kernel<<<blocks, kMeshThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(A);
    note_launch();
    return check_launch();
}

}  // extern "C"
