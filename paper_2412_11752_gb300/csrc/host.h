// host.h -- host-side pieces of libdrk shared by the render entry points
// (api.cu) and the server (serve.cu).  Not part of the public ABI.
#pragma once

#include <cstdarg>
#include <vector>

#include "drk_internal.h"

namespace drk {

// records the message of the last failure on this thread; returns s
drk_status_t fail(drk_status_t s, const char* fmt, ...);
const char* last_error_message();

#define DRK_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::drk::fail(DRK_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// stream-ordered allocations from a pool, freed together unless kept
struct Allocs {
    cudaMemPool_t pool;
    cudaStream_t st;
    std::vector<void*> ptrs;
    bool keep = false;
    int* fail_countdown = nullptr;   // fault injection: fail when it reaches 0
    Allocs(cudaMemPool_t p, cudaStream_t s) : pool(p), st(s) {}
    ~Allocs() {
        if (!keep)
            for (void* q : ptrs) cudaFreeAsync(q, st);
    }
    template <typename T>
    drk_status_t get(T** out, size_t count) {
        void* q = nullptr;
        const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
        if (fail_countdown && (*fail_countdown)-- == 0)
            return fail(DRK_ERR_OOM, "device allocation of %zu bytes failed (injected)", bytes);
        const cudaError_t e = cudaMallocFromPoolAsync(&q, bytes, pool, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(DRK_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        }
        ptrs.push_back(q);
        *out = reinterpret_cast<T*>(q);
        return DRK_OK;
    }
};

// CUDA-event timing of the pipeline stages (off unless enabled)
enum { ST_PREPROCESS = 0, ST_EMIT, ST_SORT, ST_RASTER, ST_RASTER_BWD, ST_PREPROCESS_BWD, ST_REPLAY, ST_REC_SORT,
       ST_COUNT = 8 };
struct StageTimer {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    double ms[ST_COUNT] = {0};
    long long cnt[ST_COUNT] = {0};
    cudaEvent_t get();
    cudaEvent_t begin(cudaStream_t st);
    void end(int stage, cudaEvent_t a, cudaStream_t st);
    void collect();
    void destroy();
};

drk_status_t validate(const drk_params_t* p, const drk_camera_t* cam, const drk_options_t* opt);

struct Frame {
    FrameConst fc;
    CamDev cam;
    float center[3];
    int n_tiles, tile_bits, depth_bits, kmax;
};
Frame make_frame(const drk_params_t* p, const drk_camera_t* cam, const drk_options_t* opt);
// floats per raster record / per culling bound of a primitive
size_t rec_floats(int kmax);
size_t bnd_floats(int kmax);
drk_status_t check_launch();

// Work of one frame between the two host phases.
struct FrameWork {
    Frame F;
    PreArgs A;
    int64_t P = 0;
    uint32_t* kalt = nullptr;
    uint32_t* valt = nullptr;
    uint2* ranges = nullptr;
    uint32_t* tile_order = nullptr;
};

// Phase A: preprocess, culling count, scan, depth quantisation; the pair
// total is copied to *total_host (pinned) on the stream.
drk_status_t frame_phase_a(FrameWork& w, const drk_params_t* p, const drk_camera_t* cam, const drk_options_t* opt,
                           Allocs& al, unsigned long long* counters, int* status, uint64_t* total_host,
                           cudaStream_t st, StageTimer* tm);
// Phase B (after w.P is known): pair emission, radix sort, tile ranges and
// the heaviest-first tile order.
drk_status_t frame_phase_b(FrameWork& w, Allocs& al, cudaStream_t st, StageTimer* tm);

}  // namespace drk
