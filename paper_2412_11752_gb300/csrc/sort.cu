// sort.cu -- device scans, the stable LSD radix sort of (tile | depth) keys
// and the per-tile range extraction (Sec. 4.4: tile-kernel pairs sorted by
// tile and depth before rasterisation).
//
// Radix sort: 8-bit digits.  Per digit pass:
//   1. upsweep   -- each CTA histograms its 4096 keys (per-warp shared
//                   counters) and writes hist[digit][cta];
//   2. scan      -- exclusive scan over hist in digit-major order gives the
//                   global start of every (digit, cta) run;
//   3. downsweep -- each CTA ranks its keys stably (warp match-any groups,
//                   per-warp running counts, prefix over warps), reorders
//                   them in shared memory by digit and writes each digit
//                   run contiguously.
// Stability makes the final order (tile, quantised depth, input position);
// pairs are emitted in primitive order, so ties keep the primitive index
// order.
#include "drk_internal.h"

namespace drk {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// block-wide exclusive scan of one value per thread (256 threads)
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* sh_warp, T& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T s = lane < (int)(blockDim.x >> 5) ? sh_warp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < (int)(blockDim.x >> 5)) sh_warp[lane] = s;
    }
    __syncthreads();
    const T wbase = wid > 0 ? sh_warp[wid - 1] : T(0);
    total = sh_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return wbase + x - v;
}

// per-block exclusive scan; block totals to partial[]
template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) scan_block_kernel(const TI* __restrict__ in, TO* __restrict__ out,
                                                                   TO* __restrict__ partial, int64_t n) {
    __shared__ TO sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    TO v[kScanItems];
    TO sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        v[j] = (base + j < n) ? (TO)in[base + j] : TO(0);
        sum += v[j];
    }
    TO total;
    TO run = block_exclusive_scan<TO>(sum, sh, total);
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

template <typename TO>
__global__ void __launch_bounds__(kScanThreads) scan_add_kernel(TO* __restrict__ out, const TO* __restrict__ partial,
                                                                 int64_t n) {
    const TO add = partial[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int j = threadIdx.x; j < kScanTile; j += kScanThreads)
        if (base + j < n) out[base + j] += add;
}

template <typename TO>
__global__ void set_total_kernel(TO* out, const TO* partial_scanned, const TO* partial_raw, int64_t nb, int64_t n) {
    out[n] = partial_scanned[nb - 1] + partial_raw[nb - 1];
}

// bytes of scratch needed by exclusive_scan for n items
size_t scan_scratch_bytes(int64_t n) {
    size_t b = 0;
    while (n > 1) {
        const int64_t nb = (n + kScanTile - 1) / kScanTile;
        b += 2 * (size_t)(nb + 1) * sizeof(uint64_t);
        n = nb;
    }
    return b + 64;
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total
template <typename TI, typename TO>
static void exclusive_scan_impl(const TI* in, TO* out, int64_t n, TO* scratch, cudaStream_t st) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(TO), st);
        return;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    TO* raw = scratch;
    TO* scanned = scratch + (nb + 1);
    scan_block_kernel<TI, TO><<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, raw, n); note_launch();
    if (nb > 1) {
        exclusive_scan_impl<TO, TO>(raw, scanned, nb, scratch + 2 * (nb + 1), st);
        scan_add_kernel<TO><<<(unsigned)nb, kScanThreads, 0, st>>>(out, scanned, n); note_launch();
    } else {
        cudaMemsetAsync(scanned, 0, sizeof(TO), st);
    }
    set_total_kernel<TO><<<1, 1, 0, st>>>(out, scanned, raw, nb, n); note_launch();
}

void exclusive_scan_u32_u64(const uint32_t* in, uint64_t* out, int64_t n, void* scratch, cudaStream_t st) {
    exclusive_scan_impl<uint32_t, uint64_t>(in, out, n, reinterpret_cast<uint64_t*>(scratch), st);
}

// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096
constexpr int kWarps = kSortThreads / 32;
constexpr int kWarpItems = kSortTile / kWarps;          // 512 per warp
constexpr int kBins = 256;

int64_t sort_num_blocks(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

__global__ void __launch_bounds__(kSortThreads) radix_upsweep_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                                                      int shift, uint32_t* __restrict__ hist,
                                                                      int64_t nblocks) {
    __shared__ uint32_t cnt[kWarps][kBins];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kBins; i += kSortThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)wid * kWarpItems;
    // all of the warp's loads first, then the counting: the loads overlap
    uint32_t dg[kWarpItems / 32];
#pragma unroll
    for (int r = 0; r < kWarpItems / 32; r++) {
        const int64_t i = base + r * 32 + lane;
        dg[r] = i < n ? (__ldg(keys + i) >> shift) & 0xffu : kBins;
    }
#pragma unroll
    for (int r = 0; r < kWarpItems / 32; r++)
        if (dg[r] < kBins) atomicAdd(&cnt[wid][dg[r]], 1u);
    __syncthreads();
    const int d = threadIdx.x;   // one bin per thread
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) s += cnt[w][d];
    hist[(int64_t)d * nblocks + blockIdx.x] = s;
}

__global__ void __launch_bounds__(kSortThreads, 3) radix_downsweep_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, int64_t n, int shift, const uint64_t* __restrict__ hist_scan, int64_t nblocks) {
    __shared__ uint32_t skey[kSortTile];
    __shared__ uint32_t sval[kSortTile];
    __shared__ uint32_t wcnt[kWarps][kBins];
    __shared__ uint32_t dstart[kBins];
    __shared__ uint32_t scan_tmp[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kBins; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t bbase = (int64_t)blockIdx.x * kSortTile;
    const int64_t wbase = bbase + (int64_t)wid * kWarpItems;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t k[kWarpItems / 32], v[kWarpItems / 32], rk[kWarpItems / 32];
    // all of the warp's loads first (the ranking below is a chain of warp
    // barriers, which loads are not moved across), then the ranking
#pragma unroll
    for (int r = 0; r < kWarpItems / 32; r++) {
        const int64_t i = wbase + r * 32 + lane;
        const bool valid = i < n;
        k[r] = valid ? __ldg(keys_in + i) : 0u;
        v[r] = valid ? __ldg(vals_in + i) : 0u;
    }
#pragma unroll
    for (int r = 0; r < kWarpItems / 32; r++) {
        const int64_t i = wbase + r * 32 + lane;
        const bool valid = i < n;
        const int d = valid ? (int)((k[r] >> shift) & 0xffu) : -1;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = valid ? wcnt[wid][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt_mask) == 0u) wcnt[wid][d] = before + __popc(peers);
        __syncwarp();
        rk[r] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, then over digits
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<uint32_t>(run, scan_tmp, tot);
        dstart[d] = ex;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kWarpItems / 32; r++) {
        const int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            const int d = (int)((k[r] >> shift) & 0xffu);
            const uint32_t pos = dstart[d] + wcnt[wid][d] + rk[r];
            skey[pos] = k[r];
            sval[pos] = v[r];
        }
    }
    __syncthreads();
    const int nvalid = (int)min((int64_t)kSortTile, n - bbase);
    for (int p = threadIdx.x; p < nvalid; p += kSortThreads) {
        const uint32_t kk = skey[p];
        const int d = (int)((kk >> shift) & 0xffu);
        const uint64_t g = hist_scan[(int64_t)d * nblocks + blockIdx.x] + (uint64_t)(p - dstart[d]);
        keys_out[g] = kk;
        vals_out[g] = sval[p];
    }
}

size_t radix_sort_scratch_bytes(int64_t n) {
    const int64_t nb = sort_num_blocks(n);
    const int64_t nh = nb * kBins;
    return (size_t)nh * sizeof(uint32_t) + (size_t)(nh + 1) * sizeof(uint64_t) + scan_scratch_bytes(nh) + 256;
}

// Sorts (keys, vals) of length n by the low `bits` bits of the keys.  The
// result lands in keys/vals (the alt buffers are clobbered).
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n, int bits,
                      void* scratch, cudaStream_t st) {
    if (n <= 1) return;
    const int64_t nb = sort_num_blocks(n);
    const int64_t nh = nb * kBins;
    uint32_t* hist = reinterpret_cast<uint32_t*>(scratch);
    uint64_t* hscan = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(hist + nh) + 15) & ~uintptr_t(15));
    void* sscr = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(hscan + nh + 1) + 15) & ~uintptr_t(15));
    uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        radix_upsweep_kernel<<<(unsigned)nb, kSortThreads, 0, st>>>(ki, n, shift, hist, nb); note_launch();
        exclusive_scan_impl<uint32_t, uint64_t>(hist, hscan, nh, reinterpret_cast<uint64_t*>(sscr), st);
        radix_downsweep_kernel<<<(unsigned)nb, kSortThreads, 0, st>>>(ki, vi, ko, vo, n, shift, hscan, nb); note_launch();
        uint32_t* t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    if (ki != keys) {
        cudaMemcpyAsync(keys, ki, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals, vi, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    }
}

// ---------------------------------------------------------------------------
// K4: [start, end) of every tile in the sorted key array.
__global__ void tile_ranges_kernel(const uint32_t* __restrict__ keys, int64_t n, int depth_bits,
                                   uint2* __restrict__ ranges, int n_tiles) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = keys[i] >> depth_bits;
    if (t >= (uint32_t)n_tiles) return;   // sentinel keys sort past the last tile
    if (i == 0 || (keys[i - 1] >> depth_bits) != t) ranges[t].x = (uint32_t)i;
    if (i == n - 1 || (keys[i + 1] >> depth_bits) != t) ranges[t].y = (uint32_t)(i + 1);
}

// key = 2^24 - 1 - min(list length, 2^24 - 1): ascending keys = longest first
__global__ void tile_order_keys_kernel(const uint2* __restrict__ ranges, int n_tiles, uint32_t* __restrict__ keys,
                                       uint32_t* __restrict__ vals) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const uint2 r = ranges[t];
    const uint32_t len = min(r.y - r.x, 0xffffffu);
    keys[t] = 0xffffffu - len;
    vals[t] = (uint32_t)t;
}

// keys/vals of one frame of a batch: key as above, value = slot << 20 | tile
__global__ void batch_order_keys_kernel(const uint2* __restrict__ ranges, int n_tiles, uint32_t slot,
                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const uint2 r = ranges[t];
    // frame-major, heaviest tile first within a frame: a frame's tail runs
    // beside the next frame's heaviest tiles while at most two frames'
    // records compete for L2
    keys[t] = (slot << 20) | (0xfffffu - min(r.y - r.x, 0xfffffu));
    vals[t] = (slot << 20) | (uint32_t)t;
}

void launch_batch_order_keys(const uint2* ranges, int n_tiles, int slot, uint32_t* keys, uint32_t* vals,
                             cudaStream_t st) {
    if (n_tiles <= 0) return;
    batch_order_keys_kernel<<<(n_tiles + 255) / 256, 256, 0, st>>>(ranges, n_tiles, (uint32_t)slot, keys, vals);
    note_launch();
}

// ---------------------------------------------------------------------------
// Grouping of the contributor records by primitive: the forward counted the
// records of every primitive, so an exclusive scan gives each primitive's
// start and one scatter pass places every record's slot in its
// primitive's range.  The scatter aggregates over the warp: lanes holding
// the same primitive (neighbouring slots often do) take a single atomic
// for the group.  (A block-wide aggregation through a shared hash table,
// with the slots of each primitive written as one run, measured slower.)
__global__ void record_scatter_kernel(const uint32_t* __restrict__ key, uint32_t n, uint32_t n_keys,
                                      unsigned long long* __restrict__ cursor, uint32_t* __restrict__ out_idx) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t k = i < n ? key[i] : 0xffffffffu;
    const bool valid = k < n_keys;
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    unsigned long long base = 0ull;
    if (valid && lane == leader) base = atomicAdd(cursor + k, (unsigned long long)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!valid) return;
    // the counts cover every record, so pos < n; the check keeps a
    // miscounted primitive from writing past the array
    const unsigned long long pos = base + (unsigned long long)__popc(peers & ((1u << lane) - 1u));
    if (pos < n) out_idx[pos] = i;
}

// out_idx[offs[n_keys] .. n) = no record
__global__ void record_tail_kernel(const unsigned long long* __restrict__ total, uint32_t n,
                                   uint32_t* __restrict__ out_idx) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = *total + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out_idx[i] = kNoSlot;
}

size_t record_sort_scratch_bytes(uint32_t n_keys) {
    return ((size_t)n_keys + 1) * sizeof(uint64_t) + scan_scratch_bytes((int64_t)n_keys + 1) + 64;
}

void group_records(const uint32_t* key, uint32_t n, uint32_t n_keys, const uint32_t* count, uint32_t* out_idx,
                   void* scratch, cudaStream_t st) {
    if (n == 0) return;
    if (n_keys == 0) {
        cudaMemsetAsync(out_idx, 0xff, sizeof(uint32_t) * (size_t)n, st);
        return;
    }
    uint64_t* offs = reinterpret_cast<uint64_t*>(scratch);
    void* sscr = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(offs + (size_t)n_keys + 1) + 15) & ~uintptr_t(15));
    exclusive_scan_u32_u64(count, offs, (int64_t)n_keys, sscr, st);
    // only the unused tail needs the no-record mark (the scatter writes the
    // rest): out_idx[total .. n), total = offs[n_keys]
    record_tail_kernel<<<1024, 256, 0, st>>>(reinterpret_cast<const unsigned long long*>(offs + n_keys), n, out_idx);
    note_launch();
    record_scatter_kernel<<<(n + 255u) / 256u, 256, 0, st>>>(key, n, n_keys, reinterpret_cast<unsigned long long*>(offs),
                                                           out_idx);
    note_launch();
}

__global__ void iota_kernel(uint32_t* __restrict__ v, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

void launch_iota(uint32_t* v, uint32_t n, cudaStream_t st) {
    if (n == 0) return;
    iota_kernel<<<(n + 255u) / 256u, 256, 0, st>>>(v, n);
    note_launch();
}

size_t tile_order_work_bytes(int n_tiles) {
    return 4 * sizeof(uint32_t) * (size_t)n_tiles + radix_sort_scratch_bytes(n_tiles) + 64;
}

void launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* order, void* work, cudaStream_t st) {
    if (n_tiles <= 0) return;
    uint32_t* keys = reinterpret_cast<uint32_t*>(work);
    uint32_t* kalt = keys + n_tiles;
    uint32_t* valt = kalt + n_tiles;
    void* scr = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(valt + n_tiles) + 15) & ~uintptr_t(15));
    tile_order_keys_kernel<<<(n_tiles + 255) / 256, 256, 0, st>>>(ranges, n_tiles, keys, order); note_launch();
    radix_sort_pairs(keys, order, kalt, valt, n_tiles, 24, scr, st);
}

void launch_tile_ranges(const uint32_t* keys, int64_t n, int depth_bits, uint2* ranges, int n_tiles,
                        cudaStream_t st) {
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, st);
    if (n <= 0) return;
    tile_ranges_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, n, depth_bits, ranges, n_tiles); note_launch();
}

}  // namespace drk
