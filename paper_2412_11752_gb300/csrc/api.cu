// api.cu -- C ABI of libdrk: contexts, forward render, backward, counters.
//
// Pipeline of drk_render (Sec. 4.4):
//   K1 preprocess (per primitive)  -> raster records, colours, bounds
//   K2 count (per-tile culling)    -> pairs per primitive; exclusive scan
//      host reads the pair total back once (sizes the sort)
//   K2 emit                        -> (tile | depth) keys, primitive values
//   K3 radix sort                  -> pairs grouped by tile, by depth bound
//   K4 tile ranges
//   K5 raster                      -> image, final transmittance, counts
// drk_render_backward replays K5 (K6) and then runs the per-primitive
// backward (K7).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "host.h"

using namespace drk;

namespace {
std::atomic<long long> g_launches{0};
}
namespace drk {
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace drk

namespace drk {
cudaEvent_t StageTimer::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
cudaEvent_t StageTimer::begin(cudaStream_t st) {
    if (!on) return nullptr;
    cudaEvent_t a = get();
    cudaEventRecord(a, st);
    return a;
}
void StageTimer::end(int stage, cudaEvent_t a, cudaStream_t st) {
    if (!on || !a) return;
    cudaEvent_t b = get();
    cudaEventRecord(b, st);
    pending.push_back({stage, a, b});
}
void StageTimer::collect() {
    for (auto& p : pending) {
        float t = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&t, p.a, p.b);
        ms[p.stage] += t;
        cnt[p.stage] += 1;
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    pending.clear();
}
void StageTimer::destroy() {
    collect();
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
}
}  // namespace drk

struct drk_ctx {
    StageTimer timer;
    int device = 0;
    cudaMemPool_t pool = nullptr;
    cudaStream_t last_stream = nullptr;
    unsigned long long* counters = nullptr;   // evals, emitted, extra passes, visible
    int* zmax_bits = nullptr;                 // counters[4] holds the device status bits
    DepthQuant* dq = nullptr;
    uint64_t* h_total = nullptr;              // pinned: pair total, record chunks of the last forward, backward record chunks
    unsigned int* rec_ctr = nullptr;          // record chunks the last recording forward took
    uint4* ovf = nullptr;                     // overflow columns of the raster's depth-order buffers
    size_t ovf_bytes = 0;
    bool stats = true;                        // the forward raster collects its statistics
    drk_stats_t last{};
};

struct drk_state {
    drk_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    int64_t n = 0, pairs = 0;
    int K = 0, kmax = 0, cap = 0, sh_degree = 0, width = 0, height = 0;
    FrameConst fc{};
    float* rec = nullptr;
    float4* rgb = nullptr;
    uint32_t* keys = nullptr;
    uint32_t* vals = nullptr;
    uint2* ranges = nullptr;
    uint32_t* tile_order = nullptr;
    DepthQuant* dq = nullptr;
    float* Cfin = nullptr;
    uint32_t* rec_key = nullptr;
    uint32_t* rec_count = nullptr;
    uint4* rec_rd = nullptr;
    uint32_t rec_cap = 0;
    unsigned int* rec_chunks = nullptr;       // device: chunks this forward took
    int32_t* tile_overflow = nullptr;
    std::vector<void*> allocs;
};

namespace {
// Gives the raster launch for n_tiles tiles the context's overflow columns,
// grown (stream-ordered) to one slot per warp of the launch.  If the pool
// cannot provide them the raster runs without (extra list passes instead).
void attach_ovf(drk_ctx* c, const drk_options_t* opt, int kmax, int cap, bool bwd, int n_tiles, cudaStream_t st,
                RasterArgs& R) {
    R.ovf = nullptr;
    R.ovf_slots = 0;
    R.ovf_cap = opt->ovf_capacity == 0 ? 2048 : std::max(0, (int)opt->ovf_capacity);
    if (R.ovf_cap == 0) return;
    const int slots = raster_slots(kmax, cap, bwd, false, n_tiles);
    const size_t need = raster_ovf_bytes(slots);
    if (need > c->ovf_bytes) {
        if (c->ovf) cudaFreeAsync(c->ovf, st);
        c->ovf = nullptr;
        c->ovf_bytes = 0;
        void* p = nullptr;
        if (cudaMallocFromPoolAsync(&p, need, c->pool, st) == cudaSuccess) {
            c->ovf = reinterpret_cast<uint4*>(p);
            c->ovf_bytes = need;
        } else {
            cudaGetLastError();
        }
    }
    R.ovf = c->ovf;
    R.ovf_slots = c->ovf ? (int)(c->ovf_bytes / raster_ovf_bytes(1)) : 0;
}
}  // namespace

// device counters of a context: 0 evaluations, 1 composited, 2 extra
// passes, 3 visible primitives, 4 status bits, 5 contributing evaluations,
// 6 geometry passes, 7 raster task counter, 8 spills to overflow columns;
// 16.. the same for the exact replay of the last backward
constexpr int kCtxCounters = 32;
constexpr int kBwdCounters = 16;


namespace drk {

namespace {
thread_local char g_err[512] = "";
}

const char* last_error_message() { return g_err; }

drk_status_t fail(drk_status_t s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

bool finite_pos(float v) { return std::isfinite(v) && v > 0.f; }

drk_status_t validate(const drk_params_t* p, const drk_camera_t* cam, const drk_options_t* opt) {
    if (!p || !cam || !opt) return fail(DRK_ERR_INVALID_ARG, "null params, camera or options");
    if (p->n < 0 || p->n >= (int64_t(1) << 31)) return fail(DRK_ERR_INVALID_ARG, "n = %lld out of range", (long long)p->n);
    if (p->K < 3 || p->K > 16) return fail(DRK_ERR_INVALID_ARG, "K = %d not in [3, 16]", p->K);
    if (p->sh_degree < -1 || p->sh_degree > 3)
        return fail(DRK_ERR_INVALID_ARG, "sh_degree = %d not in [-1, 3]", p->sh_degree);
    if (p->n > 0 && (!p->mu || !p->quat || !p->scale || !p->theta || !p->eta || !p->tau || !p->opacity || !p->color))
        return fail(DRK_ERR_INVALID_ARG, "null parameter array");
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
        return fail(DRK_ERR_INVALID_ARG, "image size %d x %d out of range", cam->width, cam->height);
    if (!finite_pos(cam->fx) || !finite_pos(cam->fy) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
        return fail(DRK_ERR_INVALID_ARG, "bad intrinsics");
    for (int i = 0; i < 12; i++)
        if (!std::isfinite(cam->world_to_cam[i])) return fail(DRK_ERR_INVALID_ARG, "non-finite world_to_cam");
    if (!(opt->alpha_min > 0.f && opt->alpha_min < 1.f)) return fail(DRK_ERR_INVALID_ARG, "alpha_min not in (0, 1)");
    if (!(opt->alpha_max >= opt->alpha_min && opt->alpha_max < 1.f))
        return fail(DRK_ERR_INVALID_ARG, "alpha_max not in [alpha_min, 1)");
    if (!(opt->T_min >= 0.f && opt->T_min < 1.f)) return fail(DRK_ERR_INVALID_ARG, "T_min not in [0, 1)");
    if (!(opt->lowpass_sl >= 0.f) || !std::isfinite(opt->lowpass_sl)) return fail(DRK_ERR_INVALID_ARG, "bad lowpass_sl");
    if (!finite_pos(opt->near_plane)) return fail(DRK_ERR_INVALID_ARG, "near_plane must be > 0");
    if (opt->cull_level < 0 || opt->cull_level > 3) return fail(DRK_ERR_INVALID_ARG, "cull_level not in 0..3");
    if (opt->kbuf_capacity != 8 && opt->kbuf_capacity != 16 && opt->kbuf_capacity != 32)
        return fail(DRK_ERR_INVALID_ARG, "kbuf_capacity must be 8, 16 or 32");
    if (opt->ovf_capacity < -1 || opt->ovf_capacity > 2048)
        return fail(DRK_ERR_INVALID_ARG, "ovf_capacity not in -1..2048");
    if (opt->order_mode != DRK_ORDER_EXACT && opt->order_mode != DRK_ORDER_CACHE_SORT)
        return fail(DRK_ERR_INVALID_ARG, "order_mode not in 0..1");
    if (opt->record_chunks < 0) return fail(DRK_ERR_INVALID_ARG, "record_chunks must be >= 0");
    for (int i = 0; i < 3; i++)
        if (opt->reserved[i] != 0) return fail(DRK_ERR_INVALID_ARG, "reserved option fields must be zero");
    for (int i = 0; i < 3; i++)
        if (!std::isfinite(opt->bg[i])) return fail(DRK_ERR_INVALID_ARG, "non-finite bg");
    return DRK_OK;
}

Frame make_frame(const drk_params_t* p, const drk_camera_t* cam, const drk_options_t* opt) {
    Frame F{};
    FrameConst& fc = F.fc;
    fc.width = cam->width;
    fc.height = cam->height;
    fc.tiles_x = (cam->width + kTile - 1) / kTile;
    fc.tiles_y = (cam->height + kTile - 1) / kTile;
    fc.ifx = (float)(1.0 / cam->fx);
    fc.ify = (float)(1.0 / cam->fy);
    fc.ox = (float)((0.5 - (double)cam->cx) / cam->fx);
    fc.oy = (float)((0.5 - (double)cam->cy) / cam->fy);
    fc.near_plane = opt->near_plane;
    fc.alpha_min = opt->alpha_min;
    fc.alpha_max = opt->alpha_max;
    fc.T_min = opt->T_min;
    for (int c = 0; c < 3; c++) fc.bg[c] = opt->bg[c];
    fc.order_mode = opt->order_mode;
    F.cam.fx = cam->fx; F.cam.fy = cam->fy; F.cam.cx = cam->cx; F.cam.cy = cam->cy;
    for (int i = 0; i < 12; i++) F.cam.w2c[i] = cam->world_to_cam[i];
    const float* M = cam->world_to_cam;
    for (int i = 0; i < 3; i++)
        F.center[i] = (float)(-((double)M[i] * M[3] + (double)M[4 + i] * M[7] + (double)M[8 + i] * M[11]));
    F.n_tiles = fc.tiles_x * fc.tiles_y;
    int tb = 1;
    while ((1 << tb) < F.n_tiles + 1) tb++;   // one spare id for sentinel keys
    F.tile_bits = tb;
    F.depth_bits = 32 - tb;
    F.kmax = p->K <= 8 ? 8 : 16;
    return F;
}

size_t rec_floats(int kmax) { return kmax == 8 ? Rec<8>::STRIDE : Rec<16>::STRIDE; }
size_t bnd_floats(int kmax) { return kmax == 8 ? Bnd<8>::STRIDE : Bnd<16>::STRIDE; }

drk_status_t check_launch() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DRK_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return DRK_OK;
}

drk_status_t frame_phase_a(FrameWork& w, const drk_params_t* params, const drk_camera_t* cam,
                           const drk_options_t* opt, Allocs& al, unsigned long long* counters, int* status,
                           uint64_t* total_host, cudaStream_t st, StageTimer* tm) {
    w.F = make_frame(params, cam, opt);
    const Frame& F = w.F;
    const int64_t n = params->n;
    PreArgs& A = w.A;
    std::memset(&A, 0, sizeof(A));
    A.p = *params;
    A.cam = F.cam;
    for (int c = 0; c < 3; c++) A.cam_center[c] = F.center[c];
    A.fc = F.fc;
    A.sl = opt->lowpass_sl;
    A.cull_level = opt->cull_level;
    A.depth_bits = F.depth_bits;
    A.counters = counters;
    A.status = status;
    drk_status_t s;
    if ((s = al.get(&A.rec, (size_t)n * rec_floats(F.kmax))) != DRK_OK) return s;
    if ((s = al.get(&A.bnd, (size_t)n * bnd_floats(F.kmax))) != DRK_OK) return s;
    if ((s = al.get(&A.rgb, (size_t)n)) != DRK_OK) return s;
    if (opt->cull_level == DRK_CULL_TILE && (s = al.get(&A.spans, (size_t)n * F.fc.tiles_y)) != DRK_OK) return s;
    if ((s = al.get(&A.count, (size_t)n + 1)) != DRK_OK) return s;
    if ((s = al.get(&A.offsets, (size_t)n + 1)) != DRK_OK) return s;
    if ((s = al.get(&A.zmax_bits, 1)) != DRK_OK) return s;
    if ((s = al.get(&A.dq, 1)) != DRK_OK) return s;
    uint8_t* scan_scr = nullptr;
    if ((s = al.get(&scan_scr, scan_scratch_bytes(n + 1))) != DRK_OK) return s;
    // 0.0f: every bound is beyond the near plane, so any maximum wins
    DRK_CUDA(cudaMemsetAsync(A.zmax_bits, 0, sizeof(int), st));
    cudaEvent_t ev = tm ? tm->begin(st) : nullptr;
    if (F.kmax == 8) launch_preprocess<8>(A, st); else launch_preprocess<16>(A, st);
    if (opt->order_mode == DRK_ORDER_CACHE_SORT && n > 0) {
        // pre-sort of the paper's cache-sorting: pair keys carry the rank of
        // the primitive's centre depth instead of the depth bound
        if ((uint64_t)n >= (uint64_t(1) << F.depth_bits) - 1)
            return fail(DRK_ERR_INVALID_ARG, "cache-sorting order: %lld primitives exceed the %d-bit rank field",
                        (long long)n, F.depth_bits);
        uint32_t *rk = nullptr, *rv = nullptr, *ra = nullptr, *rb = nullptr, *rank = nullptr;
        uint8_t* rscr = nullptr;
        if ((s = al.get(&rk, (size_t)n)) != DRK_OK) return s;
        if ((s = al.get(&rv, (size_t)n)) != DRK_OK) return s;
        if ((s = al.get(&ra, (size_t)n)) != DRK_OK) return s;
        if ((s = al.get(&rb, (size_t)n)) != DRK_OK) return s;
        if ((s = al.get(&rank, (size_t)n)) != DRK_OK) return s;
        if ((s = al.get(&rscr, radix_sort_scratch_bytes(n))) != DRK_OK) return s;
        if (F.kmax == 8) launch_centre_rank<8>(A, rk, rv, ra, rb, rscr, rank, st);
        else launch_centre_rank<16>(A, rk, rv, ra, rb, rscr, rank, st);
        A.rank = rank;
    }
    if (opt->cull_level >= 2) {
        if (F.kmax == 8) launch_count<8>(A, st); else launch_count<16>(A, st);
    }
    if ((s = check_launch()) != DRK_OK) return s;
    exclusive_scan_u32_u64(A.count, A.offsets, n, scan_scr, st);
    launch_depth_quant(A, st);
    if (tm) tm->end(ST_PREPROCESS, ev, st);
    DRK_CUDA(cudaMemcpyAsync(total_host, A.offsets + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    return check_launch();
}

drk_status_t frame_phase_b(FrameWork& w, Allocs& al, cudaStream_t st, StageTimer* tm) {
    const Frame& F = w.F;
    PreArgs& A = w.A;
    const int64_t P = w.P;
    if (P >= (int64_t(1) << 32) - 1)
        return fail(DRK_ERR_CAPACITY, "%lld pairs exceed the 2^32 - 1 limit of one render", (long long)P);
    drk_status_t s;
    uint8_t* sort_scr = nullptr;
    uint8_t* order_work = nullptr;
    if ((s = al.get(&A.keys, (size_t)P)) != DRK_OK) return s;
    if ((s = al.get(&A.vals, (size_t)P)) != DRK_OK) return s;
    if ((s = al.get(&w.kalt, (size_t)P)) != DRK_OK) return s;
    if ((s = al.get(&w.valt, (size_t)P)) != DRK_OK) return s;
    if ((s = al.get(&w.ranges, (size_t)F.n_tiles)) != DRK_OK) return s;
    if ((s = al.get(&sort_scr, radix_sort_scratch_bytes(P))) != DRK_OK) return s;
    if ((s = al.get(&w.tile_order, (size_t)F.n_tiles)) != DRK_OK) return s;
    if ((s = al.get(&order_work, tile_order_work_bytes(F.n_tiles))) != DRK_OK) return s;
    cudaEvent_t ev = tm ? tm->begin(st) : nullptr;
    if (F.kmax == 8) launch_emit<8>(A, st); else launch_emit<16>(A, st);
    if (tm) tm->end(ST_EMIT, ev, st);
    ev = tm ? tm->begin(st) : nullptr;
    radix_sort_pairs(A.keys, A.vals, w.kalt, w.valt, P, 32, sort_scr, st);
    launch_tile_ranges(A.keys, P, F.depth_bits, w.ranges, F.n_tiles, st);
    launch_tile_order(w.ranges, F.n_tiles, w.tile_order, order_work, st);
    if (tm) tm->end(ST_SORT, ev, st);
    return check_launch();
}

}  // namespace drk

extern "C" {

void drk_options_default(drk_options_t* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->alpha_min = expf(-9.0f);
    opt->T_min = 1e-4f;
    opt->alpha_max = 0.99f;
    opt->lowpass_sl = 0.70710678f;
    opt->near_plane = 0.2f;
    opt->cull_level = DRK_CULL_TILE;
    opt->kbuf_capacity = 16;
}

const char* drk_last_error(void) { return last_error_message(); }

const char* drk_version(void) { return "libdrk 0.1 (sm_103a)"; }

drk_status_t drk_ctx_create(int device, drk_ctx_t** out) {
    if (!out) return fail(DRK_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    int ndev = 0;
    DRK_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(DRK_ERR_INVALID_ARG, "device %d of %d", device, ndev);
    DRK_CUDA(cudaSetDevice(device));
    drk_ctx* c = new (std::nothrow) drk_ctx();
    if (!c) return fail(DRK_ERR_OOM, "host allocation failed");
    c->device = device;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaError_t e = cudaMemPoolCreate(&c->pool, &props);
    if (e != cudaSuccess) {
        delete c;
        return fail(DRK_ERR_CUDA, "cudaMemPoolCreate: %s", cudaGetErrorString(e));
    }
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (cudaMalloc(&c->counters, kCtxCounters * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->zmax_bits, sizeof(int)) != cudaSuccess || cudaMalloc(&c->dq, sizeof(DepthQuant)) != cudaSuccess ||
        cudaMalloc(&c->rec_ctr, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(c->rec_ctr, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaMallocHost(&c->h_total, 4 * sizeof(uint64_t)) != cudaSuccess) {
        cudaGetLastError();
        drk_ctx_destroy(c);
        return fail(DRK_ERR_OOM, "context buffers");
    }
    *out = c;
    return DRK_OK;
}

void drk_ctx_destroy(drk_ctx_t* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->last_stream) cudaStreamSynchronize(c->last_stream);
    if (c->ovf) cudaFree(c->ovf);
    cudaFree(c->counters);
    cudaFree(c->zmax_bits);
    cudaFree(c->dq);
    if (c->h_total) cudaFreeHost(c->h_total);
    cudaFree(c->rec_ctr);
    c->timer.destroy();
    if (c->pool) cudaMemPoolDestroy(c->pool);
    delete c;
}

drk_status_t drk_render(drk_ctx_t* ctx, const drk_params_t* params, const drk_camera_t* cam, const drk_options_t* opt,
                        const drk_image_t* out, drk_state_t** state, void* stream) {
    if (!ctx) return fail(DRK_ERR_INVALID_ARG, "null context");
    if (state) *state = nullptr;
    drk_status_t s = validate(params, cam, opt);
    if (s != DRK_OK) return s;
    if (!out || !out->rgb) return fail(DRK_ERR_INVALID_ARG, "null output image");
    if (state && opt->order_mode != DRK_ORDER_EXACT)
        return fail(DRK_ERR_INVALID_ARG, "the cache-sorting order has no backward (render without a state)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DRK_CUDA(cudaSetDevice(ctx->device));
    ctx->last_stream = st;
    const int64_t n = params->n;
    Allocs al(ctx->pool, st);
    StageTimer& tm = ctx->timer;
    DRK_CUDA(cudaMemsetAsync(ctx->counters, 0, kBwdCounters * sizeof(unsigned long long), st));

    FrameWork w;
    if ((s = frame_phase_a(w, params, cam, opt, al, ctx->counters, reinterpret_cast<int*>(ctx->counters + 4),
                           ctx->h_total, st, &tm)) != DRK_OK)
        return s;
    if (state) {
        ctx->h_total[1] = 0;
        DRK_CUDA(cudaMemcpyAsync(ctx->h_total + 1, ctx->rec_ctr, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    }
    DRK_CUDA(cudaStreamSynchronize(st));   // the pair total sizes the sort
    w.P = (int64_t)ctx->h_total[0];
    if ((s = frame_phase_b(w, al, st, &tm)) != DRK_OK) return s;
    const Frame& F = w.F;
    const PreArgs& A = w.A;

    RasterArgs R;
    std::memset(&R, 0, sizeof(R));
    R.fc = F.fc;
    R.K = params->K;
    R.rec = A.rec;
    R.rgb = A.rgb;
    R.keys = A.keys;
    R.vals = A.vals;
    R.ranges = w.ranges;
    R.tile_order = w.tile_order;
    R.dq = A.dq;
    R.counters = ctx->counters;
    R.status = reinterpret_cast<int*>(ctx->counters + 4);
    R.task_counter = reinterpret_cast<unsigned int*>(ctx->counters + 7);
    R.out_rgb = out->rgb;
    R.out_T = out->T_final;
    R.out_n = out->n_emitted;
    R.out_depth = out->depth;
    R.out_normal = out->normal;
    R.p = *params;
    if (state) {
        // one record per composited contributor for the backward; the pool
        // is sized from the chunks the previous recording forward on this
        // context took (a quarter of headroom, plus one chunk per warp of the
        // launch), else 128 records per pixel; a record that does not fit
        // sends its tile to the exact replay
        const uint64_t warps = (uint64_t)raster_slots(F.kmax, opt->kbuf_capacity, false, false, F.n_tiles);
        const uint64_t prev = ctx->h_total[1] & 0xffffffffu;
        const uint64_t npix = (uint64_t)cam->width * cam->height;
        uint64_t chunks = prev > 0 ? prev + prev / 4 + warps : (npix * 128 + kRecChunk - 1) / kRecChunk + warps;
        chunks = std::min<uint64_t>(chunks, (0xffffffffull / kRecChunk) - 1);
        if (opt->record_chunks > 0) chunks = std::min<uint64_t>(chunks, (uint64_t)opt->record_chunks);
        R.rec_cap = (uint32_t)(chunks * kRecChunk);
        R.rec_ctr = ctx->rec_ctr;
        if ((s = al.get(&R.rec_key, (size_t)R.rec_cap)) != DRK_OK) return s;
        if ((s = al.get(&R.rec_count, (size_t)n + 1)) != DRK_OK) return s;
        if ((s = al.get(&R.rec_rd, 2 * (size_t)R.rec_cap)) != DRK_OK) return s;
        DRK_CUDA(cudaMemsetAsync(R.rec_count, 0, sizeof(uint32_t) * ((size_t)n + 1), st));
        DRK_CUDA(cudaMemsetAsync(ctx->rec_ctr, 0, sizeof(unsigned int), st));
        if ((s = al.get(&R.tile_overflow, (size_t)F.n_tiles)) != DRK_OK) return s;
        DRK_CUDA(cudaMemsetAsync(R.tile_overflow, 0, sizeof(int32_t) * (size_t)F.n_tiles, st));
    }
    attach_ovf(ctx, opt, F.kmax, opt->kbuf_capacity, false, F.n_tiles, st, R);
    cudaEvent_t ev = tm.begin(st);
    launch_raster(R, F.kmax, opt->kbuf_capacity, false, ctx->stats, st);
    tm.end(ST_RASTER, ev, st);
    if ((s = check_launch()) != DRK_OK) return s;

    ctx->last = drk_stats_t{};
    ctx->last.n_pairs = w.P;
    ctx->last.n_tiles = F.n_tiles;
    ctx->last.key_bits_depth = F.depth_bits;

    if (state) {
        drk_state* S = new (std::nothrow) drk_state();
        if (!S) return fail(DRK_ERR_OOM, "host allocation failed");
        S->ctx = ctx;
        S->stream = st;
        S->n = n;
        S->pairs = w.P;
        S->K = params->K;
        S->kmax = F.kmax;
        S->cap = opt->kbuf_capacity;
        S->sh_degree = params->sh_degree;
        S->width = cam->width;
        S->height = cam->height;
        S->fc = F.fc;
        S->rec = A.rec;
        S->rgb = A.rgb;
        S->keys = A.keys;
        S->vals = A.vals;
        S->ranges = w.ranges;
        S->tile_order = w.tile_order;
        S->dq = A.dq;
        S->rec_key = R.rec_key;
        S->rec_count = R.rec_count;
        S->rec_rd = R.rec_rd;
        S->rec_cap = R.rec_cap;
        S->tile_overflow = R.tile_overflow;
        const size_t npix = (size_t)cam->width * cam->height;
        float* cf = nullptr;
        if ((s = al.get(&cf, 3 * npix)) != DRK_OK) {
            delete S;
            return s;
        }
        DRK_CUDA(cudaMemcpyAsync(cf, out->rgb, 3 * npix * sizeof(float), cudaMemcpyDeviceToDevice, st));
        S->Cfin = cf;
        unsigned int* rch = nullptr;
        if ((s = al.get(&rch, 1)) != DRK_OK) {
            delete S;
            return s;
        }
        DRK_CUDA(cudaMemcpyAsync(rch, ctx->rec_ctr, sizeof(unsigned int), cudaMemcpyDeviceToDevice, st));
        S->rec_chunks = rch;
        S->allocs = al.ptrs;
        al.keep = true;
        *state = S;
    }
    return DRK_OK;
}

drk_status_t drk_render_backward(drk_ctx_t* ctx, const drk_params_t* params, const drk_camera_t* cam,
                                 const drk_options_t* opt, const drk_state_t* state, const float* dL_drgb,
                                 const drk_params_grad_t* grads, void* stream) {
    if (!ctx || !state || !dL_drgb || !grads) return fail(DRK_ERR_INVALID_ARG, "null argument");
    drk_status_t s = validate(params, cam, opt);
    if (s != DRK_OK) return s;
    if (params->n != state->n || params->K != state->K || cam->width != state->width || cam->height != state->height ||
        params->sh_degree != state->sh_degree || opt->kbuf_capacity != state->cap)
        return fail(DRK_ERR_INVALID_ARG, "backward arguments do not match the forward state");
    if (opt->order_mode != DRK_ORDER_EXACT) return fail(DRK_ERR_INVALID_ARG, "the cache-sorting order has no backward");
    const int64_t n = params->n;
    if (n > 0 && (!grads->mu || !grads->quat || !grads->scale || !grads->theta || !grads->eta || !grads->tau ||
                  !grads->opacity || !grads->color))
        return fail(DRK_ERR_INVALID_ARG, "null gradient array");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DRK_CUDA(cudaSetDevice(ctx->device));
    ctx->last_stream = st;
    const Frame F = make_frame(params, cam, opt);
    const int K = params->K;
    const int ncoef = params->sh_degree < 0 ? 1 : (params->sh_degree + 1) * (params->sh_degree + 1);
    if (n == 0) return DRK_OK;
    DRK_CUDA(cudaMemsetAsync(grads->mu, 0, (size_t)n * 3 * sizeof(float), st));
    DRK_CUDA(cudaMemsetAsync(grads->quat, 0, (size_t)n * 4 * sizeof(float), st));
    DRK_CUDA(cudaMemsetAsync(grads->scale, 0, (size_t)n * K * sizeof(float), st));
    DRK_CUDA(cudaMemsetAsync(grads->theta, 0, (size_t)n * K * sizeof(float), st));
    DRK_CUDA(cudaMemsetAsync(grads->eta, 0, (size_t)n * sizeof(float), st));
    DRK_CUDA(cudaMemsetAsync(grads->tau, 0, (size_t)n * sizeof(float), st));
    DRK_CUDA(cudaMemsetAsync(grads->opacity, 0, (size_t)n * sizeof(float), st));
    DRK_CUDA(cudaMemsetAsync(grads->color, 0, (size_t)n * 3 * ncoef * sizeof(float), st));
    Allocs al(ctx->pool, st);
    float* gtmp = nullptr;
    if ((s = al.get(&gtmp, (size_t)n * G_STRIDE)) != DRK_OK) return s;
    DRK_CUDA(cudaMemsetAsync(gtmp, 0, (size_t)n * G_STRIDE * sizeof(float), st));

    RasterArgs R;
    std::memset(&R, 0, sizeof(R));
    R.fc = F.fc;
    R.K = K;
    R.rec = state->rec;
    R.rgb = state->rgb;
    R.keys = state->keys;
    R.vals = state->vals;
    R.ranges = state->ranges;
    R.tile_order = state->tile_order;
    R.dq = state->dq;
    R.counters = ctx->counters + kBwdCounters;
    DRK_CUDA(cudaMemsetAsync(R.counters, 0, 8 * sizeof(unsigned long long), st));
    R.status = reinterpret_cast<int*>(ctx->counters + 4);
    R.task_counter = reinterpret_cast<unsigned int*>(ctx->counters + 7);
    R.p = *params;
    R.dL = dL_drgb;
    R.Cfin = state->Cfin;
    R.gtmp = gtmp;
    R.grads = *grads;
    R.rec_key = state->rec_key;
    R.rec_count = state->rec_count;
    R.rec_rd = state->rec_rd;
    R.rec_cap = state->rec_cap;
    R.tile_overflow = state->tile_overflow;
    attach_ovf(ctx, opt, F.kmax, state->cap, true, F.n_tiles, st, R);

    // records taken by the forward (one readback; the grouping is sized by it)
    DRK_CUDA(cudaMemcpyAsync(ctx->h_total + 2, state->rec_chunks, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    DRK_CUDA(cudaStreamSynchronize(st));
    const uint64_t taken = (uint64_t)(uint32_t)ctx->h_total[2] * kRecChunk;
    const uint64_t nrec = std::min<uint64_t>(taken, state->rec_cap);
    // a chunk request beyond the pool sent tiles to the replay
    R.any_overflow = taken > state->rec_cap ? 1 : 0;
    // records grouped by primitive, from the per-primitive counts of the forward
    uint32_t* sslot = nullptr;
    uint8_t* sort_scr = nullptr;
    const uint32_t n_keys = (uint32_t)state->n;
    if ((s = al.get(&sslot, (size_t)nrec)) != DRK_OK) return s;
    if ((s = al.get(&sort_scr, record_sort_scratch_bytes(n_keys))) != DRK_OK) return s;
    StageTimer& tm = ctx->timer;
    cudaEvent_t ev = tm.begin(st);
    group_records(state->rec_key, (uint32_t)nrec, n_keys, state->rec_count, sslot, sort_scr, st);
    tm.end(ST_REC_SORT, ev, st);
    ev = tm.begin(st);
    float4* pixg = nullptr;
    const size_t npix = (size_t)cam->width * cam->height;
    if ((s = al.get(&pixg, 2 * npix)) != DRK_OK) return s;
    launch_pack_pixel_grad(R.dL, R.Cfin, npix, pixg, st);
    R.pixg = pixg;
    launch_raster_backward_records(R, sslot, (uint32_t)nrec, F.kmax, st);
    tm.end(ST_RASTER_BWD, ev, st);
    ev = tm.begin(st);
    launch_raster(R, F.kmax, state->cap, true, true, st);   // exact replay of the others
    tm.end(ST_REPLAY, ev, st);

    PreArgs A;
    std::memset(&A, 0, sizeof(A));
    A.p = *params;
    A.cam = F.cam;
    for (int c = 0; c < 3; c++) A.cam_center[c] = F.center[c];
    A.fc = F.fc;
    A.sl = opt->lowpass_sl;
    ev = tm.begin(st);
    if (F.kmax == 8) launch_preprocess_backward<8>(A, gtmp, *grads, st);
    else launch_preprocess_backward<16>(A, gtmp, *grads, st);
    tm.end(ST_PREPROCESS_BWD, ev, st);
    return check_launch();
}

drk_status_t drk_timing_enable(drk_ctx_t* ctx, int enable) {
    if (!ctx) return fail(DRK_ERR_INVALID_ARG, "null context");
    DRK_CUDA(cudaSetDevice(ctx->device));
    ctx->timer.collect();
    for (int i = 0; i < ST_COUNT; i++) {
        ctx->timer.ms[i] = 0.0;
        ctx->timer.cnt[i] = 0;
    }
    ctx->timer.on = enable != 0;
    return DRK_OK;
}

drk_status_t drk_stats_enable(drk_ctx_t* ctx, int enable) {
    if (!ctx) return fail(DRK_ERR_INVALID_ARG, "null context");
    ctx->stats = enable != 0;
    return DRK_OK;
}

drk_status_t drk_timing_read(drk_ctx_t* ctx, double* ms, int64_t* launches) {
    if (!ctx || !ms || !launches) return fail(DRK_ERR_INVALID_ARG, "null argument");
    DRK_CUDA(cudaSetDevice(ctx->device));
    ctx->timer.collect();
    for (int i = 0; i < ST_COUNT; i++) {
        ms[i] = ctx->timer.ms[i];
        launches[i] = ctx->timer.cnt[i];
    }
    return DRK_OK;
}

int64_t drk_launch_count(void) { return g_launches.load(); }

void drk_state_free(drk_state_t* S) {
    if (!S) return;
    cudaSetDevice(S->ctx->device);
    for (void* q : S->allocs) cudaFreeAsync(q, S->stream);
    delete S;
}

drk_status_t drk_sort_pairs(drk_ctx_t* ctx, uint32_t* keys, uint32_t* vals, int64_t n, int key_bits, void* stream) {
    if (!ctx) return fail(DRK_ERR_INVALID_ARG, "null context");
    if (n < 0 || n >= (int64_t(1) << 32)) return fail(DRK_ERR_INVALID_ARG, "n = %lld out of range", (long long)n);
    if (key_bits < 1 || key_bits > 32) return fail(DRK_ERR_INVALID_ARG, "key_bits = %d not in [1, 32]", key_bits);
    if (n > 0 && (!keys || !vals)) return fail(DRK_ERR_INVALID_ARG, "null keys or values");
    if (n <= 1) return DRK_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DRK_CUDA(cudaSetDevice(ctx->device));
    Allocs al(ctx->pool, st);
    drk_status_t s;
    uint32_t *kalt = nullptr, *valt = nullptr;
    uint8_t* scr = nullptr;
    if ((s = al.get(&kalt, (size_t)n)) != DRK_OK) return s;
    if ((s = al.get(&valt, (size_t)n)) != DRK_OK) return s;
    if ((s = al.get(&scr, radix_sort_scratch_bytes(n))) != DRK_OK) return s;
    radix_sort_pairs(keys, vals, kalt, valt, n, key_bits, scr, st);
    return check_launch();
}

drk_status_t drk_get_stats(drk_ctx_t* ctx, drk_stats_t* out) {
    if (!ctx || !out) return fail(DRK_ERR_INVALID_ARG, "null argument");
    DRK_CUDA(cudaSetDevice(ctx->device));
    unsigned long long c[kCtxCounters];
    DRK_CUDA(cudaMemcpyAsync(c, ctx->counters, sizeof(c), cudaMemcpyDeviceToHost, ctx->last_stream));
    DRK_CUDA(cudaStreamSynchronize(ctx->last_stream));
    *out = ctx->last;
    out->n_evals = (int64_t)c[0];
    out->n_emitted = (int64_t)c[1];
    out->n_extra_passes = (int64_t)c[2];
    out->n_visible = (int64_t)c[3];
    out->n_contrib_evals = (int64_t)c[5];
    out->n_geo_evals = (int64_t)c[6];
    out->n_spills = (int64_t)c[8];
    out->n_replay_evals = (int64_t)c[kBwdCounters + 0];
    const int bits = (int)(c[4] & 0xffffffffu);
    out->status = DRK_OK;
    for (int b = 1; b < 8; b++)
        if (bits & (1 << b)) { out->status = b; break; }
    return DRK_OK;
}

}  // extern "C"
