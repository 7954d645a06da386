// raster.cu -- per-tile rasterizer (Sec. 4.4) and its reverse mode.
//
// Forward.  One CTA per 16 x 16 tile, one thread per pixel (the paper's 2D
// thread grid), each warp an 8 x 4 block that walks the tile's pair list
// (sorted by a per-(primitive, tile) lower bound of the ray depth) on its
// own.  Each pixel evaluates every primitive of the list (Eq. 4 - Eq. 10),
// keeps contributors in a shared-memory depth-order buffer (the exact form
// of the paper's cache-sorting), and composites front to back (Eq. 1) in
// exact (r_t, index) order, stopping when the transmittance would fall
// below T_min.  A warp leaves the list as soon as its 32 pixels are
// finished.  When a backward will follow, each pixel also records the list
// positions it composited, in order.
//
// Reverse.  For a composited contributor i of a pixel,
//   dC/dc_i = T_i alpha_i,  dC/dalpha_i = T_i c_i - S_i / (1 - alpha_i),
// with S_i = C_final - P_i the colour composited behind i (P_i the prefix
// including i).  The forward writes one record per composited contributor
// (primitive, pixel, T_i, P_i) in the order it composites, which is the
// front-to-back order the supplementary "Cache-Sorting" paragraph asks the
// backward to follow; each record then carries its own T_i and P_i, so the
// backward treats records independently: grouped by primitive, each warp
// recomputes a range of them 32 at a time, keeps per-lane partial sums of
// the current primitive and adds them over the warp into one global
// atomic per component only when the primitive changes.
// Tiles whose records did not fit the pool use the replay kernel instead,
// which re-runs the forward traversal exactly and accumulates with global
// atomics.
#include <algorithm>

#include "drk_internal.h"

namespace drk {

// Staging of record headers by the bulk-copy (TMA) engine: one
// cp.async.bulk per header row, completed on an mbarrier of the warp.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
// one arrival that also announces the bytes the copies will deliver
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// global -> shared bulk copy of `bytes` (16-byte aligned ends and size)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}
// bound of a stage wait (try_wait polls, each with the hardware's own
// time limit): far beyond any copy's latency; past it the raster records
// DRK_ERR_TIMEOUT, and the warp issues no further copies and waits no
// more until its last task is done (its images are then wrong, but the
// kernel ends)
constexpr int kStageSpin = 1 << 20;

// The warp's two stage buffers: their mbarriers, the parity of each one's
// current phase and which ones have copies in flight.
struct StageSync {
    uint64_t* mbar;        // 2 mbarriers in shared memory
    unsigned phase;        // bit b: parity of buffer b's current phase
    unsigned pending;      // bit b: buffer b has copies not yet waited for
    bool failed;           // a wait ran out: no more copies or waits
};

// After a wait ran out: waits once more, with the same bound, for the
// copies still in flight into the warp's buffers, so that none of them
// lands in shared memory after the CTA has ended (called by all lanes).
__device__ __forceinline__ void stage_settle(const StageSync& ss) {
    for (int b = 0; b < 2; b++) {
        if (!((ss.pending >> b) & 1u)) continue;
        const unsigned par = (ss.phase >> b) & 1u;
        for (int spins = 0; spins < kStageSpin; spins++)
            if (__all_sync(0xffffffffu, mbar_try_wait(ss.mbar + b, par))) break;
    }
    __syncwarp();
}

constexpr int kMaxPasses = 1 << 20;
constexpr int kRasterThreads = 128;   // persistent raster CTAs: 4 independent warps
constexpr int kChunk = 16;            // list items staged and composited per step

// per-item gradient accumulator layout (floats)
enum : int { A_H = 0, A_FPX = 9, A_FPY = 10, A_FCOEF = 11, A_RGB = 12, A_OPA = 15, A_TAU = 16, A_ETA = 17, A_NFIX = 18 };
static_assert((int)A_H == (int)G_HU0 && (int)A_FPX == (int)G_FPX && (int)A_FPY == (int)G_FPY &&
                  (int)A_FCOEF == (int)G_FCOEF && (int)A_RGB == (int)G_R,
              "the first 15 accumulator entries mirror the record-gradient layout");

struct PixelState {
    float T;
    float C[3];     // forward: composited colour; backward: prefix P
    int n_emit;
    bool done;
};

__device__ __forceinline__ uint64_t key_of(float t, uint32_t idx) {
    return ((uint64_t)__float_as_uint(t) << 32) | idx;
}

// Entries of a pixel's overflow column in global memory.
constexpr int kOvfCap = 2048;
// Children per node of the depth-order heap.
constexpr int kHeapArity = 8;
// Shared heap slots for a capacity option of cap (8, 16, 32): at least one
// more, and 1 modulo the arity, so that no group of siblings straddles
// shared and global memory.
template <int CAP>
struct HeapSlots {
    static constexpr int value = (CAP + kHeapArity - 1) / kHeapArity * kHeapArity + 1;
    static_assert(value % kHeapArity == 1 % kHeapArity, "sibling groups must not straddle the shared slots");
};

// Per-pixel depth-order buffer (the exact form of the paper's cache-sorting,
// Sec. 4.4 and the supplementary algorithm): a D-ary min-heap of pending
// contributors keyed by (r_t, primitive index) as one 64-bit word (r_t > 0,
// so its float bits order like the value; the index breaks ties), with
// alpha beside it.  Its first SLOTS slots live in shared memory (slot s of
// this pixel at [s * STRIDE] from its column base, so a warp touching the
// same slot index hits distinct banks); deeper slots continue in the
// pixel's overflow column in global memory (keys and alphas in two arrays,
// lane-contiguous, L1/L2-resident for the usual depths).  The D children
// of node i are slots D i + 1 .. D i + D; with SLOTS = 1 (mod D) a group of
// siblings lies wholly in shared or wholly in global memory, where its keys
// fill one aligned 8 D-byte block and its alphas one 4 D-byte block, read
// together.  A removal walks log_D(n) levels (a binary heap of the same
// size walks twice as many, most of them in global memory).  Items arrive
// nearly in depth order, so an insertion usually stops at the first parent.
// In the cache-sorting mode the heap holds at most `lim` entries (the
// paper's cache length) and has no global part.
template <int D, int SLOTS, int STRIDE>
struct HeapBuf {
    static_assert(SLOTS % D == 1 % D, "sibling groups must not straddle the shared slots");
    static_assert(D % 4 == 0, "column groups are read in 16-byte pieces");
    static constexpr int OFF = 0;   // slot SLOTS + j is column entry OFF + j (groups start on multiples of D)
    uint64_t* sk;           // shared keys
    float* sa;              // shared alphas
    uint64_t* ck;           // column keys (null: no global part)
    float* ca;              // column alphas
    int lim;                // capacity (entries)
    int n;
    uint64_t fk;            // key of the root (~0 when empty), kept in a register
    __device__ __forceinline__ void init(uint64_t* k, float* a, uint4* col, int ncol_req, int cache_len) {
        sk = k; sa = a;
        if (col) {
            ck = reinterpret_cast<uint64_t*>(col);
            ca = reinterpret_cast<float*>(ck + kOvfCap);
            lim = SLOTS + min(ncol_req, kOvfCap - D);
        } else {
            ck = nullptr; ca = nullptr;
            lim = cache_len > 0 ? min(cache_len, SLOTS) : SLOTS;
        }
        n = 0;
        fk = ~0ull;
    }
    __device__ __forceinline__ int capacity() const { return lim; }
    __device__ __forceinline__ bool empty() const { return n == 0; }
    __device__ __forceinline__ bool full() const { return n >= lim; }
    __device__ __forceinline__ float front_t() const { return __uint_as_float((uint32_t)(fk >> 32)); }
    __device__ __forceinline__ uint32_t front_i() const { return (uint32_t)fk; }
    __device__ __forceinline__ float front_a() const { return sa[0]; }
    __device__ __forceinline__ void clear() { n = 0; fk = ~0ull; }
    __device__ __forceinline__ uint64_t getk(int i) const {
        return i < SLOTS ? sk[i * STRIDE] : ck[OFF + i - SLOTS];
    }
    __device__ __forceinline__ float geta(int i) const {
        return i < SLOTS ? sa[i * STRIDE] : ca[OFF + i - SLOTS];
    }
    __device__ __forceinline__ void put(int i, uint64_t k, float a) {
        if (i < SLOTS) {
            sk[i * STRIDE] = k; sa[i * STRIDE] = a;
        } else {
            ck[OFF + i - SLOTS] = k; ca[OFF + i - SLOTS] = a;
        }
    }
    // (t1, i1) < (t2, i2)?
    __device__ __forceinline__ bool less(float t1, uint32_t i1, float t2, uint32_t i2) const {
        return t1 < t2 || (t1 == t2 && i1 < i2);
    }
    // the root's key is at or after (t, idx)?
    __device__ __forceinline__ bool front_at_or_after(float t, uint32_t idx) const { return fk >= key_of(t, idx); }
    __device__ __forceinline__ void sift_up(int i, uint64_t k, float a) {
        while (i > 0) {
            const int up = (i - 1) / D;
            const uint64_t uk = getk(up);
            if (!(k < uk)) break;
            put(i, uk, geta(up));
            i = up;
        }
        put(i, k, a);
        if (i == 0) fk = k;
    }
    // requires !full()
    __device__ __forceinline__ void push(float t, uint32_t p, float a) { sift_up(n++, key_of(t, p), a); }
    // Full heap: keeps the smallest keys among the old entries and the new
    // one, so every pass composites at least one entry.  The largest key is
    // on a leaf (slots ceil((n - 1) / D) .. n - 1); it leaves unless the new
    // entry is larger.  Returns the key of the entry that does not stay.
    __device__ __forceinline__ uint64_t push_full(float t, uint32_t p, float a) {
        const uint64_t k = key_of(t, p);
        int m = (n + D - 2) / D;
        uint64_t mk = getk(m);
        for (int i = m + 1; i < n; i++) {
            const uint64_t ik = getk(i);
            if (ik > mk) { m = i; mk = ik; }
        }
        if (!(k < mk)) return k;
        sift_up(m, k, a);
        return mk;
    }
    // removes the root; requires !empty()
    __device__ __forceinline__ void pop() {
        n--;
        if (n == 0) {
            fk = ~0ull;
            return;
        }
        const uint64_t lk = getk(n);
        const float la = geta(n);
        int i = 0;
        while (true) {
            const int c = D * i + 1;
            if (c >= n) break;
            // the smallest key of the sibling group c .. c + D - 1 (slots at
            // or past n read as +inf); alpha is selected along with it
            uint64_t gk[D];
            uint64_t mk;
            float ma;
            int m = 0;
            if (c < SLOTS) {
#pragma unroll
                for (int j = 0; j < D; j++) gk[j] = sk[(c + j) * STRIDE];
                if (c + D > n) {
#pragma unroll
                    for (int j = 1; j < D; j++)
                        if (c + j >= n) gk[j] = ~0ull;
                }
                mk = gk[0];
#pragma unroll
                for (int j = 1; j < D; j++)
                    if (gk[j] < mk) { mk = gk[j]; m = j; }
                if (!(mk < lk)) break;
                ma = sa[(c + m) * STRIDE];   // one shared load for the chosen child
            } else {
                // global: keys and alphas of the group in aligned 16-byte
                // pieces, loaded together (a dependent load costs more here)
                const int e = OFF + c - SLOTS;
                float ga[D];
                const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(ck + e);
#pragma unroll
                for (int j = 0; j < D / 2; j++) {
                    const ulonglong2 v = k2[j];
                    gk[2 * j] = v.x; gk[2 * j + 1] = v.y;
                }
                const float4* a4 = reinterpret_cast<const float4*>(ca + e);
#pragma unroll
                for (int j = 0; j < D / 4; j++) {
                    const float4 v = a4[j];
                    ga[4 * j] = v.x; ga[4 * j + 1] = v.y; ga[4 * j + 2] = v.z; ga[4 * j + 3] = v.w;
                }
                if (c + D > n) {
#pragma unroll
                    for (int j = 1; j < D; j++)
                        if (c + j >= n) gk[j] = ~0ull;
                }
                mk = gk[0];
                ma = ga[0];
#pragma unroll
                for (int j = 1; j < D; j++)
                    if (gk[j] < mk) { mk = gk[j]; ma = ga[j]; m = j; }
                if (!(mk < lk)) break;
            }
            put(i, mk, ma);
            i = c + m;
        }
        put(i, lk, la);
        fk = sk[0];
    }
};

// Gradient of G * alpha_tilde for one pair with respect to the record
// quantities (homography rows, filter centre and coefficient) and the
// activated parameters o, tau, eta, s_k, s_k1, theta'_k, theta'_k1.
struct PairGrad {
    float v[A_NFIX];          // A_RGB entries are filled by the caller
    int k, k1;
    float ds_k, ds_k1, dth_k, dth_k1;
    bool has_k, has_k1;       // theta'_k (k >= 1) and theta'_k1 (k + 1 < K) are free
};

template <int KMAX>
__device__ __forceinline__ void grad_from_info(const RasterArgs& A, const float* __restrict__ r, uint32_t idx,
                                               const PixelRay& pr, const EvalInfo& e, float G, PairGrad& out) {
#pragma unroll
    for (int j = 0; j < A_NFIX; j++) out.v[j] = 0.f;
    out.k = 0; out.k1 = 0;
    out.ds_k = out.ds_k1 = out.dth_k = out.dth_k1 = 0.f;
    out.has_k = out.has_k1 = false;
    if (e.clamped) return;
    const float t = e.t;
    const float o = r[R_OPA];
    float dL_dt = 0.f, dL_du = 0.f, dL_dv = 0.f;
    if (e.use_filter) {
        // f = o 2^-Xf, Xf = dp2 d2 t^2 fcoef
        out.v[A_OPA] = G * __fdividef(e.f, o);
        const float dXf = -G * e.f * kLn2;
        const float dx = pr.x - r[R_FPX], dy = pr.y - r[R_FPY];
        const float k2 = pr.d2 * t * t * r[R_FCOEF];
        out.v[A_FPX] = dXf * (-2.f * dx * k2);
        out.v[A_FPY] = dXf * (-2.f * dy * k2);
        out.v[A_FCOEF] = dXf * (dx * dx + dy * dy) * pr.d2 * t * t;
        dL_dt = __fdividef(dXf * 2.f * e.Xf, t);
    } else {
        const float tau = r[R_TAU];
        const float g = e.g;
        float slope, dpsi_dtau;
        const float p1 = 1.f + tau, m1 = 1.f - tau;
        if (g < r[R_B1]) {
            slope = __fdividef(m1, p1);
            dpsi_dtau = __fdividef(-2.f * g, p1 * p1);
        } else if (g < r[R_B2]) {
            slope = __fdividef(p1, m1);
            dpsi_dtau = __fdividef(2.f * g - 1.f, m1 * m1);
        } else {
            slope = __fdividef(m1, p1);
            dpsi_dtau = __fdividef(2.f - 2.f * g, p1 * p1);
        }
        out.v[A_OPA] = G * __fdividef(e.al_k, o);
        out.v[A_TAU] = G * o * dpsi_dtau;
        const float dX = -G * o * slope * kLn2 * g;
        out.v[A_ETA] = dX * (0.5f * kLog2e) * (e.r1 * e.r1 - e.r2sq * e.Q);
        const float d_r1 = dX * 2.f * r[R_ETA2] * e.r1;
        const float d_r2sq = dX * r[R_ETA2C] * e.Q;
        const float d_Q = dX * r[R_ETA2C] * e.r2sq;
        const int K = A.K;
        const int k = e.k, k1 = (k + 1 == K) ? 0 : k + 1;
        const float* sc = A.p.scale + (size_t)K * idx;
        const float sk = __ldg(sc + k), sk1 = __ldg(sc + k1);
        // Q = (A_k + A_k1) + c (A_k - A_k1), A = 1/(2 s^2)
        float ds_k = -d_Q * (1.f + e.c) * rcp_approx(sk * sk * sk);
        float ds_k1 = -d_Q * (1.f - e.c) * rcp_approx(sk1 * sk1 * sk1);
        const float d_c = d_Q * e.dif;
        // c = cos(dth), dth = (phi - th_k) pi / gap
        const float d_dth = -d_c * __sinf(e.dth);
        const float pg = e.pg;
        const float d_phi = d_dth * pg;
        float dth_k = d_dth * pg * (e.dth * (1.f / kPi) - 1.f);
        float dth_k1 = -d_dth * pg * e.dth * (1.f / kPi);
        if (e.r2sq > 1e-30f) {
            const float ir2 = rcp_approx(e.r2sq);
            dL_du -= d_phi * e.v * ir2;
            dL_dv += d_phi * e.u * ir2;
        }
        dL_du += d_r2sq * 2.f * e.u;
        dL_dv += d_r2sq * 2.f * e.v;
        // r1 = |a| + |b|, (a, b) = Minv (u, v), Minv = [e_k e_k1]^-1
        const float sa = e.a > 0.f ? 1.f : (e.a < 0.f ? -1.f : 0.f);
        const float sb = e.b > 0.f ? 1.f : (e.b < 0.f ? -1.f : 0.f);
        // Minv = [e_k e_k1]^-1 = [[e1y, -e1x], [-eky, ekx]] / det
        const float ekx = e.ekx, eky = e.eky, e1x = e.e1x, e1y = e.e1y;
        const float wx = (e1y * sa - eky * sb) * e.idet;
        const float wy = (-e1x * sa + ekx * sb) * e.idet;
        dL_du += d_r1 * wx;
        dL_dv += d_r1 * wy;
        ds_k -= __fdividef(d_r1 * e.a * (wx * ekx + wy * eky), sk);
        dth_k += d_r1 * (-e.a) * (wy * ekx - wx * eky);
        ds_k1 -= __fdividef(d_r1 * e.b * (wx * e1x + wy * e1y), sk1);
        dth_k1 += d_r1 * (-e.b) * (wy * e1x - wx * e1y);
        out.k = k;
        out.k1 = k1;
        out.ds_k = ds_k;
        out.ds_k1 = ds_k1;
        // theta'_0 = 0 and theta'_K = 2 pi are constants of the frame
        out.dth_k = dth_k;
        out.dth_k1 = dth_k1;
        out.has_k = k >= 1;
        out.has_k1 = k + 1 < K;
        // u = U t, v = V t
        const float dU = dL_du * t, dV = dL_dv * t;
        out.v[A_H + 0] = dU * pr.x;
        out.v[A_H + 1] = dU * pr.y;
        out.v[A_H + 2] = dU;
        out.v[A_H + 3] = dV * pr.x;
        out.v[A_H + 4] = dV * pr.y;
        out.v[A_H + 5] = dV;
        dL_dt = __fdividef(dL_du * e.u + dL_dv * e.v, t);
    }
    // t = 1 / w
    const float dw = -dL_dt * t * t;
    out.v[A_H + 6] = dw * pr.x;
    out.v[A_H + 7] = dw * pr.y;
    out.v[A_H + 8] = dw;
}

template <int KMAX>
__device__ __forceinline__ void pair_grad(const RasterArgs& A, const float* __restrict__ r, uint32_t idx,
                                          const PixelRay& pr, float G, PairGrad& out) {
    float t, al;
    EvalInfo e;
    eval_pair<KMAX, true>(r, A.K, pr, A.fc.near_plane, A.fc.alpha_min, A.fc.alpha_max, t, al, &e);
    grad_from_info<KMAX>(A, r, idx, pr, e, G, out);
}

__device__ __forceinline__ void add_global(const RasterArgs& A, uint32_t idx, const PairGrad& g) {
    float* gt = A.gtmp + (size_t)G_STRIDE * idx;
#pragma unroll
    for (int j = 0; j < A_OPA; j++)
        if (g.v[j] != 0.f) atomicAdd(gt + j, g.v[j]);
    if (g.v[A_OPA] != 0.f) atomicAdd(A.grads.opacity + idx, g.v[A_OPA]);
    if (g.v[A_TAU] != 0.f) atomicAdd(A.grads.tau + idx, g.v[A_TAU]);
    if (g.v[A_ETA] != 0.f) atomicAdd(A.grads.eta + idx, g.v[A_ETA]);
    const size_t base = (size_t)A.K * idx;
    if (g.ds_k != 0.f) atomicAdd(A.grads.scale + base + g.k, g.ds_k);
    if (g.ds_k1 != 0.f) atomicAdd(A.grads.scale + base + g.k1, g.ds_k1);
    if (g.has_k && g.dth_k != 0.f) atomicAdd(A.grads.theta + base + g.k, g.dth_k);
    if (g.has_k1 && g.dth_k1 != 0.f) atomicAdd(A.grads.theta + base + g.k + 1, g.dth_k1);
}

// The warp's current chunk of contributor-record slots [base, end).
struct RecChunk {
    uint32_t base, end;
};

// Called by all 32 lanes: takes the next chunk of kRecChunk record slots
// from the pool (one atomic per chunk).  The slots left in the previous
// chunk are marked unused first (the pool is not cleared).  When the pool
// is exhausted the chunk stays empty and the tile is marked for the exact
// replay.
__device__ __forceinline__ void take_record_chunk(const RasterArgs& A, RecChunk& rc, int tile) {
    // the same trip count on every lane: a shuffle after a loop whose trip
    // count differed between lanes returned stale values to the lanes that
    // ran longer (observed with nvcc 13.0 on sm_103a)
    for (uint32_t q0 = rc.base; q0 < rc.end; q0 += 32) {
        const uint32_t q = q0 + (threadIdx.x & 31);
        if (q < rc.end) A.rec_key[q] = kNoSlot;
    }
    uint32_t c = 0;
    if ((threadIdx.x & 31) == 0) c = atomicAdd(A.rec_ctr, 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if ((uint64_t)(c + 1) * kRecChunk <= (uint64_t)A.rec_cap) {
        rc.base = c * kRecChunk;
        rc.end = rc.base + kRecChunk;
    } else {
        rc.base = rc.end = 0;
        if ((threadIdx.x & 31) == 0) A.tile_overflow[tile] = 1;
    }
}

// ---------------------------------------------------------------------------
// Counters a warp accumulates over its tasks.
// Per lane in 32 bits (a lane would need 2^32 evaluations in one launch to
// wrap; the counters are statistics), summed over the warp in 32 bits and
// added to the 64-bit device counters.
// Only `passes` bounds the traversal; the others are statistics, kept
// when the kernel is instantiated with STATS (their registers cost the
// frame forward at 1080p about 1.5 % of its time).
struct WarpCounters {
    uint32_t evals = 0, emit = 0, passes = 0, contrib = 0, geo = 0, spills = 0;
};

// One task of the forward (or replay) traversal: the 8 x 4 block `blk` of
// `tile` in the frame (fc, rec, rgb, vals, keys, ranges, dq, out).
template <int KMAX, int CAP, bool BWD, bool AUX, bool STATS>
__device__ __forceinline__ void run_task(const RasterArgs& A, const FrameConst& fc, const float* __restrict__ recp,
                                         const float4* __restrict__ rgbp, const uint32_t* __restrict__ valsp,
                                         const uint32_t* __restrict__ keysp, const uint2* __restrict__ rangesp,
                                         const DepthQuant* __restrict__ dqp, float* __restrict__ outp, bool batched,
                                         int K, int tile, uint32_t task, float4* stage, StageSync& ss, float* ring,
                                         uint4* ovf,
                                         HeapBuf<kHeapArity, HeapSlots<CAP>::value, kRasterThreads>& kb, WarpCounters& wc, RecChunk& rc) {
    constexpr int HDR4 = Rec<KMAX>::HDR / 4;
    constexpr int STRIDE4 = Rec<KMAX>::STRIDE4;
    const int lane = threadIdx.x & 31;
    const DepthQuant dq = *dqp;
    const uint32_t qmask = (1u << dq.depth_bits) - 1u;
    const float4* rec4 = reinterpret_cast<const float4*>(recp);
    const size_t npix = (size_t)fc.width * fc.height;
    const int blk = (int)(task & 7u);
    if (BWD && A.tile_overflow && A.tile_overflow[tile] == 0) return;   // handled by the list kernel
    const int tx = tile % fc.tiles_x, ty = tile / fc.tiles_x;
    const int x = tx * kTile + (blk & 1) * 8 + (lane & 7);
    const int y = ty * kTile + (blk >> 1) * 4 + (lane >> 3);
    const bool inside = x < fc.width && y < fc.height;
    // pixel-index corners of this 8 x 4 block (for the depth bounds of the items)
    const float bx0 = (float)(tx * kTile + (blk & 1) * 8), by0 = (float)(ty * kTile + (blk >> 1) * 4);
    const float2 bxs = make_float2(bx0, bx0 + 7.0f), bys = make_float2(by0, by0 + 3.0f);
    const uint2 rg = rangesp[tile];
    const uint32_t L = rg.y - rg.x;
    const uint32_t* list = valsp + rg.x;
    const uint32_t* lkeys = keysp + rg.x;
    const PixelRay pr = make_ray(fc, x, y);
    const size_t pix = (size_t)y * fc.width + x;

    PixelState ps;
    ps.T = 1.f;
    ps.C[0] = ps.C[1] = ps.C[2] = 0.f;
    ps.n_emit = 0;
    ps.done = !inside;
    float dL[3] = {0.f, 0.f, 0.f}, Cf[3] = {0.f, 0.f, 0.f};
    if (BWD && inside) {
        for (int c = 0; c < 3; c++) {
            dL[c] = A.dL[c * npix + pix];
            Cf[c] = A.Cfin[c * npix + pix];
        }
    }
    // contributor records for the backward
    const bool rec_on = !BWD && A.rec_key != nullptr;
    const bool literal = fc.order_mode == DRK_ORDER_CACHE_SORT;
    // shared heap: keys [slots][threads] (u64), then alphas [slots][threads]
    constexpr int kSlots = HeapSlots<CAP>::value;
    kb.init(reinterpret_cast<uint64_t*>(ring) + threadIdx.x, ring + 2 * kSlots * kRasterThreads + threadIdx.x,
            literal ? nullptr : ovf, A.ovf_cap, literal ? CAP : 0);
    // Exact order with a bounded heap.  When a contributor finds the heap
    // full, the largest key among the heap and the new entry is dropped;
    // `lost` is the smallest dropped key (every key in the heap stays below
    // it).  Keys at or after it are not composited in this pass: the list
    // is walked again from the start for keys at or above it (an extra
    // pass), which keeps the order exact for any capacity.
    uint64_t lo = 0ull;        // keys below lo were composited in earlier passes
    uint64_t lost = ~0ull;     // smallest dropped key
    bool finished = ps.done;

    // depth and normal images (AUX): the plane normal in camera coordinates
    // follows from the homography row of 1/r_t: with the ray d = (x ifx + ox,
    // y ify + oy, 1), 1/r_t = n . d / c, so n / c = (HW0 / ifx, HW1 / ify,
    // HW2 - ox HW0 / ifx - oy HW1 / ify); n / c . d = 1/r_t > 0, so -n / c
    // points towards the camera
    float aux_d = 0.f, aux_n[3] = {0.f, 0.f, 0.f};
    const float fxp = AUX ? 1.f / fc.ifx : 0.f, fyp = AUX ? 1.f / fc.ify : 0.f;

    // composites contributor (r_t t, alpha a, primitive idx, colour c4);
    // `slot` is its record slot (kNoSlot: not recorded).  Returns the
    // primitive index recorded (kNoSlot: none)
    auto composite = [&](float t, float a, uint32_t idx, const float4 c4, uint32_t slot) -> uint32_t {
        const float Tn = __fmul_rn(ps.T, __fsub_rn(1.f, a));
        if (Tn < fc.T_min) {
            // the pixel stops here: its slot of this round stays unused
            if (!BWD && slot != kNoSlot) A.rec_key[slot] = kNoSlot;
            ps.done = true;
            return kNoSlot;
        }
        const float col[3] = {c4.x, c4.y, c4.z};
        uint32_t recorded = kNoSlot;
        const float wgt = __fmul_rn(a, ps.T);
        if (AUX) {
            const float* h = recp + (size_t)Rec<KMAX>::STRIDE * idx;
            const float nx = __ldg(h + R_HW0) * fxp, ny = __ldg(h + R_HW1) * fyp;
            const float nz = __ldg(h + R_HW2) - fc.ox * nx - fc.oy * ny;
            const float s = -wgt * rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
            aux_n[0] = fmaf(s, nx, aux_n[0]);
            aux_n[1] = fmaf(s, ny, aux_n[1]);
            aux_n[2] = fmaf(s, nz, aux_n[2]);
            aux_d = fmaf(wgt, t, aux_d);
        }
        if (!BWD) {
            const float T_i = ps.T;
            for (int c = 0; c < 3; c++) ps.C[c] = fmaf(wgt, col[c], ps.C[c]);
            if (slot != kNoSlot) {
                // read only by the backward: streaming stores keep them from
                // evicting the primitive records this kernel re-reads from L2
                recorded = idx;
                __stcs(A.rec_key + slot, recorded);
                __stcs(A.rec_rd + 2 * (size_t)slot, make_uint4(recorded, (uint32_t)pix, __float_as_uint(T_i),
                                                               __float_as_uint(ps.C[0])));
                __stcs(A.rec_rd + 2 * (size_t)slot + 1,
                       make_uint4(__float_as_uint(ps.C[1]), __float_as_uint(ps.C[2]), 0u, 0u));
            }
        } else {
            float G = 0.f;
            const float inv1ma = 1.f / (1.f - a);
            for (int c = 0; c < 3; c++) {
                ps.C[c] = fmaf(wgt, col[c], ps.C[c]);
                const float S = Cf[c] - ps.C[c];
                G += dL[c] * (ps.T * col[c] - S * inv1ma);
            }
            PairGrad g;
            pair_grad<KMAX>(A, A.rec + (size_t)Rec<KMAX>::STRIDE * idx, idx, pr, G, g);
            for (int c = 0; c < 3; c++) g.v[A_RGB + c] = dL[c] * wgt;
            add_global(A, idx, g);
        }
        ps.T = Tn;
        ps.n_emit++;
        return recorded;
    };
    // composites the root of this lane's heap
    // composites the root of this lane's heap and removes it: the colour
    // load is issued first so that the removal's memory accesses overlap it
    // (a pixel that stops here leaves its heap unused)
    auto emit_front = [&](uint32_t slot) {
        const float t = kb.front_t(), a = kb.front_a();
        const uint32_t i = kb.front_i();
        const float4 c4 = __ldg(rgbp + i);
        kb.pop();
        return composite(t, a, i, c4, slot);
    };

    // a contributor of primitive j with key kk = (t, j)
    auto offer = [&](float t, uint32_t j, float a, uint64_t kk) {
        if (literal) {
            // the paper's cache-sorting: a full cache composites the smaller
            // of its smallest entry and the new one (Sec. 4.4)
            if (!kb.full()) {
                kb.push(t, j, a);
            } else if (kb.less(t, j, kb.front_t(), kb.front_i())) {
                composite(t, a, j, __ldg(rgbp + j), kNoSlot);
            } else {
                const float ra = kb.front_a(), rt = kb.front_t();
                const uint32_t rp = kb.front_i();
                composite(rt, ra, rp, __ldg(rgbp + rp), kNoSlot);
                if (!ps.done) {
                    kb.pop();
                    kb.push(t, j, a);
                }
            }
            return;
        }
        if (kk < lo || kk >= lost) return;
        if (!kb.full()) {
            if (STATS && kb.n >= HeapSlots<CAP>::value) wc.spills++;
            kb.push(t, j, a);
        } else {
            const uint64_t d = kb.push_full(t, j, a);
            if (d < lost) lost = d;
        }
    };


    // Called by all 32 lanes.  For each lane with `go`, composites every
    // pending entry that no item at or after a list position with depth
    // bound thr can precede, in rounds in which every lane that still has
    // one composites one entry; the round's records take consecutive slots
    // of the warp's record chunk.  Returns false for a lane whose next entry
    // is at or after its smallest dropped key (its pass ends).
    auto drain = [&](bool go, float thr) -> bool {
        const float lt = __uint_as_float((uint32_t)(lost >> 32));
        bool ok = true;
        while (true) {
            bool want = go && ok && !ps.done && !kb.empty() && kb.front_t() < thr;
            if (want && lost != ~0ull && kb.front_at_or_after(lt, (uint32_t)lost)) {
                ok = false;
                want = false;
            }
            const unsigned m = __ballot_sync(0xffffffffu, want);
            if (m == 0) break;
            uint32_t slot = kNoSlot;
            if (rec_on) {
                const uint32_t cnt = (uint32_t)__popc(m);
                if (rc.end - rc.base < cnt) take_record_chunk(A, rc, tile);
                if (rc.end - rc.base >= cnt) {
                    slot = rc.base + (uint32_t)__popc(m & ((1u << lane) - 1u));
                    rc.base += cnt;
                }
            }
            uint32_t rk = kNoSlot;
            if (want) rk = emit_front(slot);
            // records per primitive: one atomic per recorded lane (cheaper
            // here than grouping equal primitives of the round with a
            // match-any first)
            if (rec_on && rk != kNoSlot) atomicAdd(A.rec_count + rk, 1u);
        }
        // nothing left below the smallest dropped key can come before thr
        if (go && ok) ok = !(lost != ~0ull && lt < thr);
        return ok;
    };

    // copies the headers of the chunk starting at list position base, whose
    // indices lanes 0 .. kChunk-1 hold in idxv, into stage buffer b: lane 0
    // arms the buffer's mbarrier with the chunk's bytes, then lane l < kChunk
    // issues one bulk copy of item l's header row (called by all lanes)
    constexpr unsigned kHdrBytes = (unsigned)(HDR4 * sizeof(float4));
    auto stage_chunk = [&](uint32_t base, uint32_t idxv, int b) {
        const uint32_t avail = base < L ? min((uint32_t)kChunk, L - base) : 0u;
        if (avail == 0u || ss.failed) return;
        float4* bufp = stage + b * kChunk * HDR4;
        // the warp's earlier reads of this buffer come before the copies
        // into it (generic then async proxy)
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (lane == 0) mbar_arrive_expect_tx(ss.mbar + b, avail * kHdrBytes);
        __syncwarp();
        if ((uint32_t)lane < avail) bulk_g2s(bufp + lane * HDR4, rec4 + (size_t)idxv * STRIDE4, kHdrBytes, ss.mbar + b);
        ss.pending |= 1u << b;
    };
    // waits for buffer b's copies (called by all lanes)
    auto stage_wait = [&](int b) {
        if (!((ss.pending >> b) & 1u) || ss.failed) return;
        const unsigned par = (ss.phase >> b) & 1u;
        // every lane polls; the loop ends for the whole warp at once (the
        // same trip count on every lane, see take_record_chunk)
        for (int spins = 0;; spins++) {
            if (__all_sync(0xffffffffu, mbar_try_wait(ss.mbar + b, par))) break;
            if (spins >= kStageSpin) {
                // buffer b stays pending: the kernel settles it at its end
                ss.failed = true;
                if (lane == 0 && A.status) atomicOr(A.status, 1 << DRK_ERR_TIMEOUT);
                return;
            }
        }
        ss.phase ^= 1u << b;
        ss.pending &= ~(1u << b);
        __syncwarp();
    };

    while (true) {   // passes over the list
        bool pass_done = finished;
        // chunk c covers list positions [kChunk c, kChunk (c + 1)); lane l < kChunk holds item kChunk c + l
        const bool lo_lane = lane < kChunk;
        uint32_t idx_a = lo_lane && (uint32_t)lane < L ? __ldg(list + lane) : 0u;
        uint32_t key_a = lo_lane && (uint32_t)lane < L ? __ldg(lkeys + lane) : 0u;
        uint32_t idx_b = lo_lane && kChunk + (uint32_t)lane < L ? __ldg(list + kChunk + lane) : 0u;
        uint32_t key_b = lo_lane && kChunk + (uint32_t)lane < L ? __ldg(lkeys + kChunk + lane) : 0u;
        stage_chunk(0u, idx_a, 0);
        for (uint32_t c0 = 0; c0 < L; c0 += kChunk) {
            const int buf = (int)((c0 / kChunk) & 1u);
            // stage the next chunk's headers, fetch the one after's entries
            stage_chunk(c0 + kChunk, idx_b, buf ^ 1);
            const uint32_t n2 = c0 + 2 * kChunk + lane;
            const uint32_t idx_c = lo_lane && n2 < L ? __ldg(list + n2) : 0u;
            const uint32_t key_c = lo_lane && n2 < L ? __ldg(lkeys + n2) : 0u;
            stage_wait(buf);
            const uint32_t cn = min((uint32_t)kChunk, L - c0);
            // Composite, once per chunk and with every lane together, each
            // pending entry that no item of this chunk or later can precede
            // (the chunk's first bound is the smallest).  Compositing later
            // than possible never changes the order; a pixel that finishes
            // inside the chunk only evaluates a few items more.
            // The threshold is a lower bound of r_t over this block's pixels
            // for every item still to come: for this chunk's items the
            // larger of the item's key bound and 1 / max w over the block's
            // corners (w is affine in the pixel indices), deflated for FP32;
            // for the items after the chunk the next chunk's first key bound.
            if (!literal) {
                float bb = __int_as_float(0x7f800000);
                if (lo_lane && c0 + (uint32_t)lane < L) {
                    const float* hs = reinterpret_cast<const float*>(stage + (buf * kChunk + lane) * HDR4);
                    const float W0 = hs[R_HW0], W1 = hs[R_HW1], W2 = hs[R_HW2];
                    const float wy0 = fmaf(W1, bys.x, W2), wy1 = fmaf(W1, bys.y, W2);
                    const float mw = fmaxf(fmaxf(fmaf(W0, bxs.x, wy0), fmaf(W0, bxs.y, wy0)),
                                           fmaxf(fmaf(W0, bxs.x, wy1), fmaf(W0, bxs.y, wy1)));
                    const float kb = fmaf((float)(key_a & qmask), dq.inv_scale, dq.zmin);
                    bb = mw > 0.0f ? fmaxf(kb, __fmul_rn(rcp_approx(mw), 1.0f - 2e-5f)) : __int_as_float(0x7f800000);
                }
                for (int o = 8; o > 0; o >>= 1) bb = fminf(bb, __shfl_xor_sync(0xffffffffu, bb, o));
                bb = __shfl_sync(0xffffffffu, bb, 0);
                const uint32_t keyn = __shfl_sync(0xffffffffu, key_b, 0);
                const float thr_next = c0 + kChunk < L ? fmaf((float)(keyn & qmask), dq.inv_scale, dq.zmin)
                                                      : __int_as_float(0x7f800000);
                const float thr0 = fminf(bb, thr_next);
                const bool ok = drain(!pass_done, thr0);
                if (!pass_done && (!ok || ps.done)) pass_done = true;
            }
            if (!literal) {
                // exact order: two items per step, both evaluated before
                // either is offered (in list order), so that their two
                // dependency chains interleave
                for (uint32_t jj = 0; jj < cn; jj += 2) {
                    const bool two = jj + 1 < cn;
                    const uint32_t idxA = __shfl_sync(0xffffffffu, idx_a, jj);
                    const uint32_t idxB = __shfl_sync(0xffffffffu, idx_a, two ? jj + 1 : jj);
                    const float4* sgA = stage + (buf * kChunk + jj) * HDR4;
                    const float4* sgB = sgA + HDR4;
                    float hA[R_FIX4 * 4], hB[R_FIX4 * 4];
                    Geo gA{0.f, 0.f, 0.f, 0.f}, gB{0.f, 0.f, 0.f, 0.f};
                    bool geoA = false, geoB = false;
                    if (!pass_done) {
                        if (STATS) wc.evals += two ? 2 : 1;
#pragma unroll
                        for (int q = 0; q < R_GEO4; q++) {
                            const float4 v = sgA[q];
                            hA[4 * q] = v.x; hA[4 * q + 1] = v.y; hA[4 * q + 2] = v.z; hA[4 * q + 3] = v.w;
                            const float4 w = sgB[q];
                            hB[4 * q] = w.x; hB[4 * q + 1] = w.y; hB[4 * q + 2] = w.z; hB[4 * q + 3] = w.w;
                        }
                        geoA = eval_geometry(hA, pr, fc.near_plane, gA);
                        geoB = two && eval_geometry(hB, pr, fc.near_plane, gB);
                    }
                    if (__any_sync(0xffffffffu, geoA || geoB)) {
                        if (STATS) wc.geo += (geoA ? 1 : 0) + (geoB ? 1 : 0);
#pragma unroll
                        for (int q = R_GEO4; q < R_FIX4; q++) {
                            const float4 v = sgA[q];
                            hA[4 * q] = v.x; hA[4 * q + 1] = v.y; hA[4 * q + 2] = v.z; hA[4 * q + 3] = v.w;
                            const float4 w = sgB[q];
                            hB[4 * q] = w.x; hB[4 * q + 1] = w.y; hB[4 * q + 2] = w.z; hB[4 * q + 3] = w.w;
                        }
                        float aA = 0.f, aB = 0.f;
                        const bool okA = eval_kernel<KMAX, false>(hA, reinterpret_cast<const float*>(sgA), K, pr, gA,
                                                                  fc.alpha_min, fc.alpha_max, aA) && geoA;
                        const bool okB = eval_kernel<KMAX, false>(hB, reinterpret_cast<const float*>(sgB), K, pr, gB,
                                                                  fc.alpha_min, fc.alpha_max, aB) && geoB;
                        if (okA) {
                            if (STATS) wc.contrib++;
                            offer(gA.t, idxA, aA, key_of(gA.t, idxA));
                        }
                        if (okB) {
                            if (STATS) wc.contrib++;
                            offer(gB.t, idxB, aB, key_of(gB.t, idxB));
                        }
                    }
                }
            } else {
                for (uint32_t jj = 0; jj < cn; jj++) {
                    const uint32_t idx = __shfl_sync(0xffffffffu, idx_a, jj);
                    float h[R_FIX4 * 4];
                    Geo gm;
                    bool geo = false;
                    const float4* sg = stage + (buf * kChunk + jj) * HDR4;
                    if (!pass_done) {
                        if (STATS) wc.evals++;
    #pragma unroll
                        for (int q = 0; q < R_GEO4; q++) {
                            const float4 v = sg[q];
                            h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
                        }
                        geo = eval_geometry(h, pr, fc.near_plane, gm);
                    }
                    if (__any_sync(0xffffffffu, geo)) {
                        if (geo) {
                            if (STATS) wc.geo++;
    #pragma unroll
                            for (int q = R_GEO4; q < R_FIX4; q++) {
                                const float4 v = sg[q];
                                h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
                            }
                            float a;
                            if (eval_kernel<KMAX, false>(h, reinterpret_cast<const float*>(sg), K, pr, gm, fc.alpha_min,
                                                         fc.alpha_max, a)) {
                                if (STATS) wc.contrib++;
                                offer(gm.t, idx, a, key_of(gm.t, idx));
                                if (ps.done) pass_done = true;
                            }
                        }
                    }
                }
            }
            __syncwarp();
            idx_a = idx_b; key_a = key_b;
            idx_b = idx_c; key_b = key_c;
            if (__all_sync(0xffffffffu, pass_done)) break;
        }
        // a pass that ended early leaves the next chunk's copies in flight
        stage_wait(0);
        stage_wait(1);
        // end of the list for this pass: composite what is left in order
        drain(!ps.done, __int_as_float(0x7f800000));
        bool need = !ps.done && lost != ~0ull;
        if (need && wc.passes >= (unsigned long long)kMaxPasses) {
            // every pass composites at least CAP entries, so this bound is
            // never reached by a correct traversal; it only guards the loop
            need = false;
            if (A.status) atomicOr(A.status, 1 << DRK_ERR_CAPACITY);
        }
        if (need) {
            lo = lost;
            lost = ~0ull;
            kb.clear();
            wc.passes++;
        }
        finished = !need;
        if (!__any_sync(0xffffffffu, need)) break;
    }

    if (!BWD && inside) {
        for (int c = 0; c < 3; c++) outp[c * npix + pix] = fmaf(ps.T, fc.bg[c], ps.C[c]);
        if (!batched && A.out_T) A.out_T[pix] = ps.T;
        if (!batched && A.out_n) A.out_n[pix] = ps.n_emit;
        if (AUX && !batched) {
            if (A.out_depth) A.out_depth[pix] = aux_d;
            if (A.out_normal)
                for (int c = 0; c < 3; c++) A.out_normal[c * npix + pix] = aux_n[c];
        }
    }
    if (STATS) wc.emit += (uint32_t)ps.n_emit;
}

// Forward traversal; with BWD it is the exact replay used by the backward of
// tiles whose composited lists were not recorded in full; with BATCH it
// renders every tile of a batch of frames in one launch (serving).
//
// Persistent warps.  The work unit is an 8 x 4 block of a tile (a task;
// 8 per tile); each warp takes tasks from a global counter until none are
// left and walks the tile's list on its own, so there is no block-wide
// barrier anywhere.  List entries (primitive index, depth key) are fetched
// 16 at a time with one coalesced load and broadcast by shuffle; the
// headers of the next 16 records are copied into the warp's shared-memory
// stage by bulk copies (one per header row) one chunk ahead of use,
// completed on the warp's mbarrier of that stage buffer; two items are
// evaluated per step, and the kernel stage runs only when some lane of the
// warp passes the geometry stage.  Tasks are taken heaviest tile first
// (longest list), which keeps the tail short.
// The register budget is that of the CTAs per SM the shared memory allows:
// four with 16 or more heap slots (and for the batch variant, which keeps a
// frame slot per task), five with 8.
template <int KMAX, int CAP, bool BWD, bool BATCH, bool AUX = false, bool STATS = true>
__global__ void __launch_bounds__(kRasterThreads, (BATCH || CAP >= 16) ? 4 : 5) raster_kernel(RasterArgs A) {
    constexpr int kWarps = kRasterThreads / 32;
    constexpr int HDR4 = Rec<KMAX>::HDR / 4;
    extern __shared__ float4 smem4[];
    // [kWarps][2 chunks][kChunk items][HDR4] float4 staging of record
    // headers, then the shared part of the depth-order heaps
    float4* stage_all = smem4;
    float* ring = reinterpret_cast<float*>(smem4 + kWarps * 2 * kChunk * HDR4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* stage = stage_all + warp * (2 * kChunk * HDR4);
    __shared__ FrameConst fc_sh[BATCH ? kWarps : 1];   // batch: the current task's frame constants
    __shared__ __align__(8) uint64_t stage_mbar[kWarps][2];
    StageSync ss{stage_mbar[warp], 0u, 0u, false};
    if (lane == 0) {
        mbar_init(ss.mbar, 1u);
        mbar_init(ss.mbar + 1, 1u);
    }
    // the initialised barriers are visible to the bulk-copy engine
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    const int slot = blockIdx.x * kWarps + warp;
    // lane-contiguous columns: a lane's deep heap levels are adjacent, and
    // the footprint is what the pixels actually hold
    uint4* ovf = (A.ovf && A.ovf_cap > 0 && slot < A.ovf_slots)
                     ? A.ovf + ((size_t)slot * 32 + lane) * kOvfCap
                     : nullptr;
    const uint32_t n_tasks = BATCH ? (uint32_t)A.n_batch_tiles * 8u : (uint32_t)(A.fc.tiles_x * A.fc.tiles_y) * 8u;
    WarpCounters wc;

    HeapBuf<kHeapArity, HeapSlots<CAP>::value, kRasterThreads> kb;
    RecChunk rc{0u, 0u};

    while (true) {
        uint32_t task = 0;
        if (lane == 0) task = atomicAdd(A.task_counter, 1u);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= n_tasks) break;
        const int tile = A.tile_order ? (int)A.tile_order[task >> 3] : (int)(task >> 3);
        if (BATCH) {
            const FrameSlot& sl = A.slots[(uint32_t)tile >> 20];
            // the frame's constants, read in every evaluation, into this
            // warp's shared slot (the single-frame kernel has them in its
            // parameter space; read through the global slot they cost an
            // L1 access per use)
            constexpr int kFcWords = (int)(sizeof(FrameConst) / sizeof(int));
            static_assert(sizeof(FrameConst) % sizeof(int) == 0 && kFcWords <= 32, "frame constants fit one warp copy");
            __syncwarp();
            if (lane < kFcWords) reinterpret_cast<int*>(&fc_sh[warp])[lane] = reinterpret_cast<const int*>(&sl.fc)[lane];
            __syncwarp();
            run_task<KMAX, CAP, BWD, false, STATS>(A, fc_sh[warp], sl.rec, sl.rgb, sl.vals, sl.keys, sl.ranges, sl.dq,
                                            sl.out_rgb, true, sl.K, tile & ((1 << 20) - 1), task, stage, ss, ring, ovf,
                                            kb, wc, rc);
            // the warp that finishes a frame's last task publishes it: its
            // image is complete in device memory once the flag is visible
            __syncwarp();
            if (lane == 0 && sl.task_left) {
                __threadfence();
                if (atomicSub(sl.task_left, 1u) == 1u) {
                    __threadfence_system();
                    *reinterpret_cast<volatile unsigned int*>(sl.done_flag) = 1u;
                }
            }
        } else {
            run_task<KMAX, CAP, BWD, AUX, STATS>(A, A.fc, A.rec, A.rgb, A.vals, A.keys, A.ranges, A.dq, A.out_rgb, false, A.K, tile,
                                     task, stage, ss, ring, ovf, kb, wc, rc);
        }
    }
    // copies abandoned by a wait that ran out are waited for once more
    if (ss.failed) stage_settle(ss);
    // the unused tail of the warp's last record chunk holds no record
    if (!BWD && !BATCH && A.rec_key)
        for (uint32_t q0 = rc.base; q0 < rc.end; q0 += 32)
            if (q0 + lane < rc.end) A.rec_key[q0 + lane] = kNoSlot;
    // counters: one atomic per warp
    if (A.counters) {
        for (int o = 16; o > 0; o >>= 1) {
            wc.evals += __shfl_down_sync(0xffffffffu, wc.evals, o);
            wc.emit += __shfl_down_sync(0xffffffffu, wc.emit, o);
            wc.passes += __shfl_down_sync(0xffffffffu, wc.passes, o);
            wc.contrib += __shfl_down_sync(0xffffffffu, wc.contrib, o);
            wc.geo += __shfl_down_sync(0xffffffffu, wc.geo, o);
            wc.spills += __shfl_down_sync(0xffffffffu, wc.spills, o);
        }
        if (lane == 0) {
            atomicAdd(A.counters + 0, (unsigned long long)wc.evals);
            atomicAdd(A.counters + 1, (unsigned long long)wc.emit);
            atomicAdd(A.counters + 2, (unsigned long long)wc.passes);
            atomicAdd(A.counters + 5, (unsigned long long)wc.contrib);
            atomicAdd(A.counters + 6, (unsigned long long)wc.geo);
            atomicAdd(A.counters + 8, (unsigned long long)wc.spills);
        }
    }

}

// ---------------------------------------------------------------------------
// Backward over the contributor records, grouped by primitive.
// Each record (pixel, T before, colour prefix after) is independent: a lane
// recomputes its pair with all intermediates, forms
// dC/dalpha = T c - S / (1 - alpha) with S = C_final - P, and chains
// through Eq. 10 - Eq. 4 to the record quantities.  Records of one
// primitive (all its pixels, over all tiles) are contiguous, a few thousand
// on average, so a warp walks a range of kRecWin windows of 32 records and
// keeps per-lane partial sums of the current primitive: the fixed terms in
// registers, the per-basis terms (scale and angle of the pixel's sector
// and of the next one) in a per-lane shared-memory column.  Only when the
// primitive changes are the partial sums added over the warp and sent to
// global memory, one atomic per parameter.  Records of tiles marked for
// the replay are skipped.
constexpr int kRecWin = 32;          // 32-record windows per warp
constexpr int kRecThreads = 128;     // 4 warps per block

template <int KMAX>
struct RecAcc {
    static constexpr int ROWS = A_NFIX + 2 * KMAX;   // fixed terms, then scale[KMAX], theta[KMAX]
    float* sh;                                       // this warp's [ROWS][32] columns
    float v[A_NFIX];
};

// Adds the warp's partial sums of primitive g to its gradients and clears
// them (every lane calls it).
template <int KMAX>
__device__ __forceinline__ void rec_flush(const RasterArgs& A, RecAcc<KMAX>& acc, uint32_t g) {
    const int lane = threadIdx.x & 31;
    float* sh = acc.sh;
#pragma unroll
    for (int j = 0; j < A_NFIX; j++) {
        sh[j * 32 + lane] = acc.v[j];
        acc.v[j] = 0.f;
    }
    __syncwarp();
    const int K = A.K;
    // every lane runs the same passes (see take_record_chunk)
#pragma unroll
    for (int pass = 0; pass < (RecAcc<KMAX>::ROWS + 31) / 32; pass++) {
        const int r = pass * 32 + lane;
        // rotated reads: the lanes of one step hit 32 distinct banks
        float s = 0.f;
        if (r < RecAcc<KMAX>::ROWS) {
#pragma unroll 8
            for (int m = 0; m < 32; m++) s += sh[r * 32 + ((m + lane) & 31)];
        }
        if (r >= RecAcc<KMAX>::ROWS || s == 0.f) continue;
        if (r < A_OPA) {
            atomicAdd(A.gtmp + (size_t)G_STRIDE * g + r, s);
        } else if (r == A_OPA) {
            atomicAdd(A.grads.opacity + g, s);
        } else if (r == A_TAU) {
            atomicAdd(A.grads.tau + g, s);
        } else if (r == A_ETA) {
            atomicAdd(A.grads.eta + g, s);
        } else if (r < A_NFIX + KMAX) {
            const int q = r - A_NFIX;
            if (q < K) atomicAdd(A.grads.scale + (size_t)K * g + q, s);
        } else {
            // theta'_0 = 0 and theta'_K = 2 pi are constants of the frame
            const int q = r - A_NFIX - KMAX;
            if (q >= 1 && q < K) atomicAdd(A.grads.theta + (size_t)K * g + q, s);
        }
    }
    __syncwarp();
#pragma unroll
    for (int r = A_NFIX; r < RecAcc<KMAX>::ROWS; r++) sh[r * 32 + lane] = 0.f;
    __syncwarp();
}

template <int KMAX>
__global__ void __launch_bounds__(kRecThreads) raster_backward_records_kernel(RasterArgs A,
                                                                              const uint32_t* __restrict__ sslot,
                                                                              uint32_t n) {
    constexpr int kWarps = kRecThreads / 32;
    constexpr int ROWS = RecAcc<KMAX>::ROWS;
    __shared__ float sh_all[kWarps * ROWS * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base = ((uint64_t)blockIdx.x * kWarps + warp) * (32u * kRecWin);
    if (base >= n) return;
    const FrameConst& fc = A.fc;
    const int K = A.K;
    RecAcc<KMAX> acc;
    acc.sh = sh_all + warp * ROWS * 32;
#pragma unroll
    for (int j = 0; j < A_NFIX; j++) acc.v[j] = 0.f;
#pragma unroll
    for (int r = A_NFIX; r < ROWS; r++) acc.sh[r * 32 + lane] = 0.f;
    __syncwarp();
    float* S = acc.sh + A_NFIX * 32 + lane;            // scale column
    float* H = acc.sh + (A_NFIX + KMAX) * 32 + lane;   // theta column

    // software pipeline: the records of window w + 1 and the slots of
    // window w + 2 are loaded while window w is computed.  Records and
    // slots are read once: streaming loads (evict first) keep them from
    // evicting the per-pixel inputs and the primitive headers from L2
    auto load_rec = [&](uint32_t slot, uint4& r0, uint4& r1) {
        r0 = make_uint4(kNoSlot, 0u, 0u, 0u);
        r1 = make_uint4(0u, 0u, 0u, 0u);
        if (slot < A.rec_cap) {
            r0 = __ldcs(A.rec_rd + 2 * (size_t)slot);
            r1 = __ldcs(A.rec_rd + 2 * (size_t)slot + 1);
        }
    };
    uint64_t i = base + lane;
    uint4 r0, r1;
    load_rec(i < n ? __ldcs(sslot + i) : kNoSlot, r0, r1);
    uint32_t slot_n = i + 32 < n ? __ldcs(sslot + i + 32) : kNoSlot;
    uint32_t gcur = kNoSlot;   // primitive of the partial sums (warp-uniform)
    for (int w = 0; w < kRecWin; w++) {
        if (base + 32u * w >= n) break;
        uint4 n0, n1;
        load_rec(w + 1 < kRecWin ? slot_n : kNoSlot, n0, n1);
        const uint64_t i2 = i + 64;
        const uint32_t slot_nn = (w + 2 < kRecWin && i2 < n) ? __ldcs(sslot + i2) : kNoSlot;

        uint32_t g = r0.x;   // primitive index
        PairGrad pg;
#pragma unroll
        for (int j = 0; j < A_NFIX; j++) pg.v[j] = 0.f;
        pg.k = 0; pg.k1 = 0;
        pg.ds_k = pg.ds_k1 = pg.dth_k = pg.dth_k1 = 0.f;
        if (g != kNoSlot) {
            const uint32_t pix = r0.y;
            const int y = (int)(pix / (uint32_t)fc.width), x = (int)(pix - (uint32_t)y * fc.width);
            const int tile = (y / kTile) * fc.tiles_x + x / kTile;
            if (A.any_overflow && A.tile_overflow[tile] != 0) {
                g = kNoSlot;                      // replayed exactly instead
            } else {
                // the pixel's dL and final colour: one 32-byte sector
                const float4 q0 = A.pixg[2 * (size_t)pix], q1 = A.pixg[2 * (size_t)pix + 1];
                const float* r = A.rec + (size_t)Rec<KMAX>::STRIDE * g;
                const PixelRay pr = make_ray(fc, x, y);
                float t, a;
                EvalInfo e;
                eval_pair<KMAX, true>(r, K, pr, fc.near_plane, fc.alpha_min, fc.alpha_max, t, a, &e);
                const float4 c4 = __ldg(A.rgb + g);
                const float col[3] = {c4.x, c4.y, c4.z};
                const float T = __uint_as_float(r0.z);
                const float P[3] = {__uint_as_float(r0.w), __uint_as_float(r1.x), __uint_as_float(r1.y)};
                const float wgt = __fmul_rn(a, T);
                const float inv1ma = rcp_approx(1.f - a);
                const float dL[3] = {q0.x, q0.y, q0.z}, Cf[3] = {q0.w, q1.x, q1.y};
                float G = 0.f;
                for (int c = 0; c < 3; c++) G += dL[c] * (T * col[c] - (Cf[c] - P[c]) * inv1ma);
                grad_from_info<KMAX>(A, r, g, pr, e, G, pg);
                for (int c = 0; c < 3; c++) pg.v[A_RGB + c] = dL[c] * wgt;
            }
        }
        // runs of equal primitive: lanes of the current one add to the
        // partial sums; a new primitive flushes them first
        while (true) {
            if (g != kNoSlot && g == gcur) {
#pragma unroll
                for (int j = 0; j < A_NFIX; j++) acc.v[j] += pg.v[j];
                S[pg.k * 32] += pg.ds_k;
                S[pg.k1 * 32] += pg.ds_k1;
                H[pg.k * 32] += pg.dth_k;
                if (pg.k + 1 < KMAX) H[(pg.k + 1) * 32] += pg.dth_k1;
                g = kNoSlot;
            }
            const unsigned rest = __ballot_sync(0xffffffffu, g != kNoSlot);
            if (rest == 0u) break;
            __syncwarp();
            if (gcur != kNoSlot) rec_flush<KMAX>(A, acc, gcur);
            gcur = __shfl_sync(0xffffffffu, g, __ffs(rest) - 1);
        }
        r0 = n0; r1 = n1;
        slot_n = slot_nn;
        i += 32;
    }
    __syncwarp();
    if (gcur != kNoSlot) rec_flush<KMAX>(A, acc, gcur);
}

template <int KMAX, int CAP>
constexpr size_t raster_smem() {
    return (size_t)(kRasterThreads / 32) * 2 * kChunk * (Rec<KMAX>::HDR / 4) * sizeof(float4) +
           (size_t)3 * HeapSlots<CAP>::value * kRasterThreads * sizeof(float);
}

// resident CTAs x SMs of one instantiation (computed once)
template <int KMAX, int CAP, bool BWD, bool BATCH, bool AUX = false, bool STATS = true>
static int raster_grid() {
    static int grid = 0;
    if (grid == 0) {
        constexpr size_t smem = raster_smem<KMAX, CAP>();
        cudaFuncSetAttribute(raster_kernel<KMAX, CAP, BWD, BATCH, AUX, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raster_kernel<KMAX, CAP, BWD, BATCH, AUX, STATS>,
                                                      kRasterThreads, smem);
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    return grid;
}

template <int KMAX, int CAP, bool BWD, bool BATCH, bool AUX = false, bool STATS = true>
static int raster_blocks(int n_tiles) {
    constexpr int kWarps = kRasterThreads / 32;
    const int n_tasks = n_tiles * 8;
    return std::min(raster_grid<KMAX, CAP, BWD, BATCH, AUX, STATS>(), (n_tasks + kWarps - 1) / kWarps);
}

template <int KMAX, int CAP, bool BWD, bool BATCH, bool AUX = false, bool STATS = true>
static void launch_raster_t(const RasterArgs& A, int n_tiles, cudaStream_t st) {
    // the depth/normal and the statistics-free instantiations run at most
    // as many resident warps as the plain one (the same bounds and shared
    // memory), so the overflow columns sized by raster_slots cover them;
    // warps past the columns would run without
    const int blocks = raster_blocks<KMAX, CAP, BWD, BATCH, AUX, STATS>(n_tiles);
    if (blocks <= 0) return;
    cudaMemsetAsync(A.task_counter, 0, sizeof(unsigned int), st);
    raster_kernel<KMAX, CAP, BWD, BATCH, AUX, STATS><<<blocks, kRasterThreads, raster_smem<KMAX, CAP>(), st>>>(A);
    note_launch();
}

int raster_slots(int kmax, int cap, bool bwd, bool batch, int n_tiles) {
    if (n_tiles <= 0) return 0;
    constexpr int kWarps = kRasterThreads / 32;
#define DRK_SLOTS_CASE(KM, CP)                                                                   \
    if (kmax == KM && cap == CP) {                                                               \
        if (batch) return kWarps * raster_blocks<KM, CP, false, true>(n_tiles);                  \
        if (bwd) return kWarps * raster_blocks<KM, CP, true, false>(n_tiles);                    \
        return kWarps * raster_blocks<KM, CP, false, false>(n_tiles);                            \
    }
    DRK_SLOTS_CASE(8, 8)
    DRK_SLOTS_CASE(8, 16)
    DRK_SLOTS_CASE(8, 32)
    DRK_SLOTS_CASE(16, 8)
    DRK_SLOTS_CASE(16, 16)
    DRK_SLOTS_CASE(16, 32)
#undef DRK_SLOTS_CASE
    return 0;
}

size_t raster_ovf_bytes(int slots) { return (size_t)slots * kOvfCap * 32 * sizeof(uint4); }

void launch_raster(const RasterArgs& A, int kmax, int cap, bool bwd, bool stats, cudaStream_t st) {
    const int n_tiles = A.fc.tiles_x * A.fc.tiles_y;
    if (n_tiles == 0) return;
    const bool aux = !bwd && (A.out_depth || A.out_normal);
#define DRK_RASTER_CASE(KM, CP)                                                          \
    if (kmax == KM && cap == CP) {                                                       \
        if (bwd) launch_raster_t<KM, CP, true, false>(A, n_tiles, st);                   \
        else if (aux) launch_raster_t<KM, CP, false, false, true>(A, n_tiles, st);       \
        else if (stats) launch_raster_t<KM, CP, false, false>(A, n_tiles, st);           \
        else launch_raster_t<KM, CP, false, false, false, false>(A, n_tiles, st);        \
        return;                                                                          \
    }
    DRK_RASTER_CASE(8, 8)
    DRK_RASTER_CASE(8, 16)
    DRK_RASTER_CASE(8, 32)
    DRK_RASTER_CASE(16, 8)
    DRK_RASTER_CASE(16, 16)
    DRK_RASTER_CASE(16, 32)
#undef DRK_RASTER_CASE
}

void launch_raster_batch(const RasterArgs& A, int kmax, int cap, cudaStream_t st) {
    if (A.n_batch_tiles <= 0) return;
#define DRK_RASTER_CASE(KM, CP)                                                        \
    if (kmax == KM && cap == CP) {                                                     \
        launch_raster_t<KM, CP, false, true>(A, A.n_batch_tiles, st);                  \
        return;                                                                        \
    }
    DRK_RASTER_CASE(8, 8)
    DRK_RASTER_CASE(8, 16)
    DRK_RASTER_CASE(8, 32)
    DRK_RASTER_CASE(16, 8)
    DRK_RASTER_CASE(16, 16)
    DRK_RASTER_CASE(16, 32)
#undef DRK_RASTER_CASE
}

__global__ void pack_pixel_grad_kernel(const float* __restrict__ dL, const float* __restrict__ Cfin, size_t npix,
                                       float4* __restrict__ out) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    out[2 * p] = make_float4(dL[p], dL[npix + p], dL[2 * npix + p], Cfin[p]);
    out[2 * p + 1] = make_float4(Cfin[npix + p], Cfin[2 * npix + p], 0.f, 0.f);
}

void launch_pack_pixel_grad(const float* dL, const float* Cfin, size_t npix, float4* out, cudaStream_t st) {
    if (npix == 0) return;
    pack_pixel_grad_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(dL, Cfin, npix, out);
    note_launch();
}

void launch_raster_backward_records(const RasterArgs& A, const uint32_t* sslot, uint32_t n, int kmax,
                                    cudaStream_t st) {
    if (n == 0) return;
    constexpr uint32_t per_block = kRecThreads * kRecWin;
    const unsigned blocks = (unsigned)((n + per_block - 1u) / per_block);
    if (kmax == 8) raster_backward_records_kernel<8><<<blocks, kRecThreads, 0, st>>>(A, sslot, n);
    else raster_backward_records_kernel<16><<<blocks, kRecThreads, 0, st>>>(A, sslot, n);
    note_launch();
}

}  // namespace drk
