// noalloc.cu -- drk_sort_pairs_static: the pair sort without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// sort: code running while a CUDA stream is being captured into a graph
// that must not contain allocation nodes, code inside a host callback or a
// custom allocator's own bookkeeping, or embedders whose memory is handed
// out once at start-up and never grows.  For them this entry point keeps
// its working memory in a fixed array that lives in the library's device
// image: every GPU that loads the library reserves it (9 MiB) until the
// process exits, and no call allocates or frees anything.
#include <mutex>

#include "drk_internal.h"

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

// Device address of g_sort_scratch on the current device (looked up once
// per device, with that device current).
drk_status_t scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DRK_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || !p) return DRK_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DRK_OK;
}

}  // namespace

extern "C" drk_status_t drk_sort_pairs_static(uint32_t* keys, uint32_t* vals, int64_t n, int key_bits, void* stream) {
    if (n < 0 || n > kStaticMaxPairs) return DRK_ERR_CAPACITY;
    if (key_bits < 1 || key_bits > 32) return DRK_ERR_INVALID_ARG;
    if (n > 0 && (!keys || !vals)) return DRK_ERR_INVALID_ARG;
    if (n <= 1) return DRK_OK;
    if (drk::radix_sort_scratch_bytes(n) > kStaticSortScratch) return DRK_ERR_CAPACITY;
    void* base = nullptr;
    const drk_status_t s = scratch_address(&base);
    if (s != DRK_OK) return s;
    unsigned char* b = static_cast<unsigned char*>(base);
    uint32_t* keys_alt = reinterpret_cast<uint32_t*>(b);
    uint32_t* vals_alt = reinterpret_cast<uint32_t*>(b + sizeof(uint32_t) * (size_t)kStaticMaxPairs);
    void* scratch = b + 2 * sizeof(uint32_t) * (size_t)kStaticMaxPairs;
    // every scratch word the sort reads it writes first in the same call
    // (histograms, scans, carries), so nothing needs clearing
    drk::radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, key_bits, scratch,
                          reinterpret_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? DRK_OK : DRK_ERR_CUDA;
}
