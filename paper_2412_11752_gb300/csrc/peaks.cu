// peaks.cu -- drk_measure_pipes: the arithmetic throughput of this GPU's
// FP32 FMA pipe and of its transcendental (MUFU) unit, measured with the
// library's own kernels.  The rasterizer is bound by these two units (no
// dense contraction, records resident in L2), so its roofline takes them
// as the peaks.  A measurement utility of the library; the paper has no
// counterpart.
//
// Each thread runs kChains independent dependent chains (enough to cover
// the pipe latency with the resident warps) for `iters` steps; the grid
// fills every SM.  Times are CUDA events around each launch, after a
// warm-up launch; ops = threads x chains x iters (an FMA counted as one
// operation).
#include "host.h"

namespace {

constexpr int kChains = 8;
constexpr int kPipeThreads = 256;

__global__ void __launch_bounds__(kPipeThreads) fma_kernel(float seed, int iters, float* out) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = seed + (float)(threadIdx.x + c);
    const float b = 0.999999f, d = 1e-7f;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) a[c] = fmaf(a[c], b, d);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += a[c];
    if (s == 12345.f) out[blockIdx.x] = s;   // never true: keeps the chains live
}

// op: 0 ex2.approx, 1 rcp.approx, 2 cos.approx.  Each step also passes
// through the FMA pipe (a multiply or an add; that pipe is eight times
// faster), so that no two transcendental operations meet directly (a
// reciprocal of a reciprocal could otherwise be simplified away) and the
// values stay finite.
template <int OP>
__global__ void __launch_bounds__(kPipeThreads) mufu_kernel(float seed, int iters, float* out) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = seed + 1e-3f * (float)(threadIdx.x + c);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            float y;
            if (OP == 0) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[c]));
            else if (OP == 1) asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[c]));
            else asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[c]));
            a[c] = OP == 0 ? y * 1e-3f : y + 0.25f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += a[c];
    if (s == 12345.f) out[blockIdx.x] = s;
}

// ops per second of one kernel launch (best of `reps` timed launches)
template <typename F>
drk_status_t time_ops(F launch, double ops, int reps, cudaStream_t st, double* rate) {
    cudaEvent_t a = nullptr, b = nullptr;
    DRK_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return drk::fail(DRK_ERR_CUDA, "cudaEventCreate failed");
    }
    launch();   // warm-up
    float best = 1e30f;
    drk_status_t s = DRK_OK;
    for (int r = 0; r < reps && s == DRK_OK; r++) {
        cudaEventRecord(a, st);
        launch();
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            s = drk::fail(DRK_ERR_CUDA, "pipe measurement failed: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        best = ms < best ? ms : best;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s == DRK_OK) *rate = ops / (best * 1e-3);
    return s;
}

}  // namespace

extern "C" drk_status_t drk_measure_pipes(int device, drk_pipe_peaks_t* out) {
    if (!out) return drk::fail(DRK_ERR_INVALID_ARG, "null out");
    int ndev = 0;
    DRK_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return drk::fail(DRK_ERR_INVALID_ARG, "device %d of %d", device, ndev);
    DRK_CUDA(cudaSetDevice(device));
    int sms = 0, per_sm = 0;
    DRK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    DRK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_kernel, kPipeThreads, 0));
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    float* sink = nullptr;
    DRK_CUDA(cudaMalloc(&sink, sizeof(float) * (size_t)blocks));
    cudaStream_t st = nullptr;
    const int it_fma = 1 << 14, it_mufu = 1 << 12;
    const double thr = (double)blocks * kPipeThreads * kChains;
    drk_status_t s = time_ops([&] { fma_kernel<<<blocks, kPipeThreads, 0, st>>>(1.0f, it_fma, sink); },
                              thr * it_fma, 5, st, &out->fma_ops);
    if (s == DRK_OK)
        s = time_ops([&] { mufu_kernel<0><<<blocks, kPipeThreads, 0, st>>>(0.5f, it_mufu, sink); }, thr * it_mufu, 5,
                     st, &out->ex2_ops);
    if (s == DRK_OK)
        s = time_ops([&] { mufu_kernel<1><<<blocks, kPipeThreads, 0, st>>>(1.5f, it_mufu, sink); }, thr * it_mufu, 5,
                     st, &out->rcp_ops);
    if (s == DRK_OK)
        s = time_ops([&] { mufu_kernel<2><<<blocks, kPipeThreads, 0, st>>>(0.5f, it_mufu, sink); }, thr * it_mufu, 5,
                     st, &out->cos_ops);
    cudaFree(sink);
    out->sms = sms;
    return s == DRK_OK ? drk::check_launch() : s;
}
