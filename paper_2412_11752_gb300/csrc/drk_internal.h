// drk_internal.h -- host/device interfaces between the translation units of
// libdrk.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/drk.h"
#include "drk_common.cuh"

namespace drk {

struct CamDev {
    float fx, fy, cx, cy;
    float w2c[12];
};

// arguments of the per-primitive kernels (preprocess, culling, emission,
// preprocess backward)
struct PreArgs {
    drk_params_t p;
    CamDev cam;
    float cam_center[3];
    FrameConst fc;
    float sl;               // low-pass filter radius s_l (pixels), 0 = off
    int cull_level;
    int depth_bits;
    float* rec;             // n x Rec<KMAX>::STRIDE
    float* bnd;             // n x Bnd<KMAX>::STRIDE
    float4* rgb;            // n view-dependent colours (r, g, b, 0)
    uint32_t* spans;        // n x tiles_y: tile span [a, b] (a | b << 16) of each row of a
                            // primitive taking row-interval culling (written by the count pass)
    uint32_t* count;        // n pairs per primitive
    uint64_t* offsets;      // n + 1 exclusive scan of count
    int* zmax_bits;         // max ray depth of any bound (float bits)
    DepthQuant* dq;         // device
    uint32_t* keys;         // pair keys
    uint32_t* vals;         // pair values (primitive index)
    unsigned long long* counters;  // [3]: primitives with at least one pair
    int* status;                   // device status bits (1 << drk_status_t)
    const uint32_t* rank;          // cache-sorting mode: rank of each primitive by centre depth (else null)
};

// One frame of a batched forward raster (serving): everything the raster
// reads per request.  order values of a batch encode (slot << 20) | tile.
struct FrameSlot {
    FrameConst fc;
    const float* rec;
    const float4* rgb;
    const uint32_t* keys;
    const uint32_t* vals;
    const uint2* ranges;
    const DepthQuant* dq;
    float* out_rgb;
    int K;
    unsigned int* task_left;         // device: tasks of this frame not yet finished
    unsigned int* done_flag;         // host-mapped: set to 1 when the last task finished
};

// arguments of the raster kernels
struct RasterArgs {
    FrameConst fc;
    int K;
    const float* rec;
    const float4* rgb;
    const uint32_t* keys;
    const uint32_t* vals;
    const uint2* ranges;
    const DepthQuant* dq;
    unsigned long long* counters;   // evals, emitted, extra passes (may be null)
    int* status;                     // device status bits (may be null)
    unsigned int* task_counter;      // work counter of the persistent raster (zeroed per launch)
    const uint32_t* tile_order;      // tiles by descending list length (may be null)
    // overflow columns of the depth-order buffers: ovf_slots warps x 2048
    // entries x 32 lanes (raster_ovf_bytes); without them (null) a pixel
    // whose buffer fills takes extra passes over the list instead
    uint4* ovf;
    int ovf_slots;
    int ovf_cap;                     // entries used per column (<= 2048)
    // batched forward (serving): when slots != null the kernel renders
    // n_batch_tiles tiles taken from tile_order, each encoding (slot, tile),
    // and reads the frame of each task from slots[slot]
    const FrameSlot* slots;
    int n_batch_tiles;
    // forward outputs
    float* out_rgb;
    float* out_T;
    int32_t* out_n;
    float* out_depth;      // H x W sum of T alpha r_t (null: not computed)
    float* out_normal;     // 3 x H x W sum of T alpha n (camera frame, towards the camera)
    // contributor records written by the forward for the backward (may be
    // null): one per composited contributor, in rec_cap slots handed out in
    // chunks of kRecChunk; rec_key = primitive index, kNoSlot for a slot
    // left unused (the raster marks the unused tail of each warp's last
    // chunk); rec_rd = the record itself, one 32-byte sector per slot:
    // (index, pixel y * width + x, T before the contributor, composited
    // colour after it, two unused words), so that reading one record costs
    // one sector whatever its neighbours; rec_count[i] counts the records
    // of primitive i (zeroed before the forward).  tile_overflow[tile] != 0 if a record did not fit (the
    // backward replays that tile exactly)
    uint32_t* rec_key;
    uint4* rec_rd;                   // 2 per slot
    uint32_t* rec_count;
    uint32_t rec_cap;
    unsigned int* rec_ctr;           // chunks taken (zeroed before the forward)
    int32_t* tile_overflow;
    int any_overflow;                // backward: some record did not fit
    // backward
    drk_params_t p;
    const float* dL;
    const float* Cfin;
    const float4* pixg;    // per pixel {dL0, dL1, dL2, Cf0}, {Cf1, Cf2, -, -} (backward records)
    float* gtmp;                     // n x G_STRIDE
    drk_params_grad_t grads;
};

// contributor records (see RasterArgs)
constexpr uint32_t kRecChunk = 1024;
constexpr uint32_t kNoSlot = 0xffffffffu;

// host-side count of kernel launches made by the library (all threads)
void note_launch();

template <int KMAX> void launch_preprocess(const PreArgs& A, cudaStream_t st);
template <int KMAX> void launch_count(const PreArgs& A, cudaStream_t st);
template <int KMAX> void launch_emit(const PreArgs& A, cudaStream_t st);
template <int KMAX>
void launch_preprocess_backward(const PreArgs& A, const float* gtmp, const drk_params_grad_t& g, cudaStream_t st);
void launch_depth_quant(const PreArgs& A, cudaStream_t st);
// rank of every primitive in (centre depth, index) order (cache-sorting mode)
template <int KMAX>
void launch_centre_rank(const PreArgs& A, uint32_t* keys, uint32_t* vals, uint32_t* kalt, uint32_t* valt,
                        void* scratch, uint32_t* rank, cudaStream_t st);

size_t scan_scratch_bytes(int64_t n);
void exclusive_scan_u32_u64(const uint32_t* in, uint64_t* out, int64_t n, void* scratch, cudaStream_t st);
size_t radix_sort_scratch_bytes(int64_t n);
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n, int bits,
                      void* scratch, cudaStream_t st);
void launch_tile_ranges(const uint32_t* keys, int64_t n, int depth_bits, uint2* ranges, int n_tiles,
                        cudaStream_t st);
// order[] = tile ids by descending list length; work holds 4 x n_tiles words
// followed by radix_sort_scratch_bytes(n_tiles) bytes
size_t tile_order_work_bytes(int n_tiles);
void launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* order, void* work, cudaStream_t st);
// batch tile order: writes n_tiles (key, slot << 20 | tile) entries; sorting
// them by 26-bit key gives frame order, heaviest tile first within a frame
void launch_batch_order_keys(const uint2* ranges, int n_tiles, int slot, uint32_t* keys, uint32_t* vals,
                             cudaStream_t st);
// stats: the forward keeps its per-render statistics (the replay always does)
void launch_raster(const RasterArgs& A, int kmax, int cap, bool bwd, bool stats, cudaStream_t st);
// warps the raster launch for n_tiles tiles runs (one overflow slot each),
// and the bytes of the overflow columns of `slots` warps
int raster_slots(int kmax, int cap, bool bwd, bool batch, int n_tiles);
size_t raster_ovf_bytes(int slots);
// backward over n record slots grouped by pair (sslot; kNoSlot entries skipped)
void launch_pack_pixel_grad(const float* dL, const float* Cfin, size_t npix, float4* out, cudaStream_t st);
void launch_raster_backward_records(const RasterArgs& A, const uint32_t* sslot, uint32_t n, int kmax,
                                    cudaStream_t st);
// v[i] = i for i < n
void launch_iota(uint32_t* v, uint32_t n, cudaStream_t st);
// records grouped by key (rec_key): out_idx[0 .. total) holds the slots of
// the n records whose key is below n_keys (others, kNoSlot, dropped),
// grouped by key (order within a key unspecified), from the per-key counts
// the forward took; then kNoSlot up to n
size_t record_sort_scratch_bytes(uint32_t n_keys);
void group_records(const uint32_t* key, uint32_t n, uint32_t n_keys, const uint32_t* count, uint32_t* out_idx,
                   void* scratch, cudaStream_t st);
// batched forward over A.n_batch_tiles tiles of the frames in A.slots
void launch_raster_batch(const RasterArgs& A, int kmax, int cap, cudaStream_t st);

}  // namespace drk
