// noalloc.cu -- drk_sort_pairs_static: the pair sort without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// sort: embedders whose device memory is handed out once at start-up and
// never grows, real-time loops that must not meet the implicit
// synchronisation or the latency of an allocation, or code running inside
// a custom allocator's own bookkeeping, which must not re-enter it.  For
// them this entry point keeps its working memory in a fixed array that
// lives in the library's device image: every GPU that loads the library
// reserves it (9 MiB) until the process exits, and no call allocates or
// frees anything.
#include <mutex>

#include "host.h"

namespace {

// Largest number of (key, value) pairs one call may sort.
constexpr int64_t kStaticMaxPairs = int64_t(1) << 20;
// Histogram, scan and carry space of the radix sort (upper bound for
// kStaticMaxPairs pairs; checked at run time).
constexpr size_t kStaticSortScratch = size_t(1) << 20;
constexpr size_t kStaticBytes = 2 * sizeof(uint32_t) * (size_t)kStaticMaxPairs + kStaticSortScratch;

// The scratch itself.  In host code the name below is only a stand-in for
// the symbol; the device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_sort_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_sort_scratch on the current device, looked up once
// per device with that device current (set-up of the first call on each
// device).  A device reset unloads the library's module, so the cached
// address is valid only until then.
drk_status_t scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return drk::fail(DRK_ERR_INVALID_ARG, "device %d above %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || !p)
            return drk::fail(DRK_ERR_CUDA, "cudaGetSymbolAddress of the sort scratch: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DRK_OK;
}

// A device array of the current device?  Host, managed-on-host and other
// devices' pointers are refused before anything is launched.
drk_status_t on_device(const void* p, int dev, const char* what) {
    cudaPointerAttributes at{};
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();   // an unknown pointer leaves no error behind
        return drk::fail(DRK_ERR_INVALID_ARG, "%s: not a CUDA pointer (%s)", what, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice || at.device != dev)
        return drk::fail(DRK_ERR_INVALID_ARG, "%s is not device memory of the current device %d (type %d, device %d)",
                         what, dev, (int)at.type, at.device);
    return DRK_OK;
}

}  // namespace

extern "C" drk_status_t drk_sort_pairs_static(uint32_t* keys, uint32_t* vals, int64_t n, int key_bits, void* stream) {
    if (n < 0 || n > kStaticMaxPairs)
        return drk::fail(DRK_ERR_CAPACITY, "n = %lld outside 0 .. 2^20", (long long)n);
    if (key_bits < 1 || key_bits > 32) return drk::fail(DRK_ERR_INVALID_ARG, "key_bits = %d not in [1, 32]", key_bits);
    if (n > 0 && (!keys || !vals)) return drk::fail(DRK_ERR_INVALID_ARG, "null keys or values");
    if (n <= 1) return DRK_OK;
    if (drk::radix_sort_scratch_bytes(n) > kStaticSortScratch)
        return drk::fail(DRK_ERR_CAPACITY, "sort scratch for n = %lld above the fixed array", (long long)n);
    int dev = 0;
    DRK_CUDA(cudaGetDevice(&dev));
    drk_status_t s;
    if ((s = on_device(keys, dev, "keys")) != DRK_OK) return s;
    if ((s = on_device(vals, dev, "vals")) != DRK_OK) return s;
    void* base = nullptr;
    if ((s = scratch_address(dev, &base)) != DRK_OK) return s;
    unsigned char* b = static_cast<unsigned char*>(base);
    uint32_t* keys_alt = reinterpret_cast<uint32_t*>(b);
    uint32_t* vals_alt = reinterpret_cast<uint32_t*>(b + sizeof(uint32_t) * (size_t)kStaticMaxPairs);
    void* scratch = b + 2 * sizeof(uint32_t) * (size_t)kStaticMaxPairs;
    // every scratch word the sort reads it writes first in the same call
    // (histograms, scans, carries), so nothing needs clearing
    drk::radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, key_bits, scratch,
                          reinterpret_cast<cudaStream_t>(stream));
    return drk::check_launch();
}
