// serve.cu -- continuous-batching request loop over resident scenes
// (drk_serve_*).
//
// One worker thread owns two CUDA streams.  Whenever a stream is free and
// requests are queued, it forms a batch (same basis-count class, at most
// max_batch requests, within the memory budget beside the batch in flight)
// and runs it on that stream:
//   phase A per request   preprocess, culling count, scan (pair totals -> host)
//   wait for the totals   (the worker keeps retiring the other stream's batch)
//   phase B per request   emission, radix sort, tile ranges
//   batch tile order      frame by frame (heaviest frame first), heaviest
//                         tile first within a frame
//   one raster launch     persistent warps over every tile of every frame
// and records a completion event.  The next batch's phases A/B run on the
// other stream while this raster runs; its raster waits for this one to
// end (one raster on the SMs at a time).  Each pixel's arithmetic and
// compositing order are those of drk_render, so the images are identical.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host.h"

using namespace drk;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kStreams = 2;
constexpr int kMaxBatch = 64;

struct SceneDev {
    drk_params_t p{};
    void* mem = nullptr;
    size_t bytes = 0;
    int kmax = 8;
    double pairs_per_pixel = -1.0;   // running estimate from served frames
};

struct Request {
    int scene = 0;
    drk_camera_t cam{};
    float* out = nullptr;
    drk_serve_timing_t t{};
    size_t est_bytes = 0;
    bool done = false;
};

struct Batch {
    int stream = 0;
    std::vector<uint64_t> tickets;
    std::vector<int> ok;             // request still live after phase A/B
    std::vector<int> slot;           // its frame slot in the raster (-1: none)
    std::vector<int> early;          // completed before the batch (frame flag)
    std::unique_ptr<Allocs> al;
    cudaEvent_t ev = nullptr;
    size_t bytes = 0;
};

// device bytes of one request with P pairs (phase A + phase B + its share
// of the batch order arrays)
size_t request_bytes(int64_t n, int kmax, int64_t P, int n_tiles, int tiles_y) {
    const size_t per_prim = (rec_floats(kmax) + bnd_floats(kmax) + 4 + 1 + tiles_y) * sizeof(float) + 2 * sizeof(uint64_t);
    const size_t per_pair = 4 * sizeof(uint32_t);
    return (size_t)n * per_prim + scan_scratch_bytes(n + 1) + (size_t)P * per_pair + radix_sort_scratch_bytes(P) +
           (size_t)n_tiles * (sizeof(uint2) + 6 * sizeof(uint32_t)) + tile_order_work_bytes(n_tiles) + 4096;
}

}  // namespace

struct drk_serve {
    int device = 0;
    drk_options_t opt{};
    size_t budget = 0;
    int max_batch = 1;
    cudaMemPool_t pool = nullptr;
    cudaStream_t streams[kStreams] = {nullptr, nullptr};
    Batch* running[kStreams] = {nullptr, nullptr};
    uint64_t* h_totals[kStreams] = {nullptr, nullptr};        // pinned, max_batch each
    FrameSlot* h_slots[kStreams] = {nullptr, nullptr};        // pinned
    FrameSlot* d_slots[kStreams] = {nullptr, nullptr};
    unsigned long long* d_counters[kStreams] = {nullptr, nullptr};   // max_batch x 8 each
    unsigned long long* h_counters[kStreams] = {nullptr, nullptr};   // pinned copy at batch end
    unsigned int* d_task[kStreams] = {nullptr, nullptr};
    unsigned int* d_left[kStreams] = {nullptr, nullptr};      // tasks left per frame slot
    unsigned int* h_left[kStreams] = {nullptr, nullptr};      // pinned staging of d_left
    unsigned int* h_done[kStreams] = {nullptr, nullptr};      // host-mapped frame-done flags
    unsigned int* d_done[kStreams] = {nullptr, nullptr};      // their device address
    uint4* ovf[kStreams] = {nullptr, nullptr};           // raster overflow columns per stream
    size_t ovf_bytes[kStreams] = {0, 0};
    cudaEvent_t ev_phase_a[kStreams] = {nullptr, nullptr};
    cudaEvent_t ev_done[kStreams] = {nullptr, nullptr};
    // device timeline of the running batch per stream: phase A begin / end,
    // phase B end (raster begin), raster end; times against ev_ref
    cudaEvent_t ev_tl[kStreams][4] = {{nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr}};
    cudaEvent_t ev_ref = nullptr;
    std::vector<std::unique_ptr<SceneDev>> scenes;
    std::mutex mu;
    std::condition_variable cv_work;   // worker: new request or stop
    std::condition_variable cv_done;   // waiters: a ticket completed
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    size_t inflight_bytes = 0;
    bool stop = false;
    int fail_countdown = -1;
    int inject_gen = 0;
    std::thread worker;
    Clock::time_point t0;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

// one request of a batch, copied out of the queue
struct Item {
    uint64_t ticket;
    int scene;
    drk_params_t p;
    drk_camera_t cam;
    float* out;
    size_t est;
};

// the running batch of stream s, with what retirement needs
struct BatchInfo {
    std::vector<int64_t> pairs;
    std::vector<int> scene;
    std::vector<double> npix;
};

constexpr int kCountersPer = 8;   // per request: visible, ..., [4] status bits

void sleep_us(int us) { std::this_thread::sleep_for(std::chrono::microseconds(us)); }

// Retires every batch whose completion event has fired: per-request status
// from the device status words, timing, memory accounting, scene estimates;
// frees the batch's allocations on its stream.  Worker thread only.
void retire(drk_serve* S, std::unique_ptr<BatchInfo>* info) {
    for (int s = 0; s < kStreams; s++) {
        Batch* b = S->running[s];
        if (!b) continue;
        const cudaError_t e = cudaEventQuery(b->ev);
        if (e == cudaErrorNotReady) {
            // frames of the running batch whose last task finished
            bool any = false;
            const double t = S->now_ms();
            for (size_t i = 0; i < b->tickets.size(); i++) {
                if (b->early[i] || b->slot[i] < 0) continue;
                if (reinterpret_cast<volatile unsigned int*>(S->h_done[s])[b->slot[i]] == 0u) continue;
                b->early[i] = 1;
                std::lock_guard<std::mutex> lk(S->mu);
                auto it = S->reqs.find(b->tickets[i]);
                if (it == S->reqs.end()) continue;
                it->second.t.status = DRK_OK;
                it->second.t.end_ms = t;
                it->second.done = true;
                any = true;
            }
            if (any) S->cv_done.notify_all();
            continue;
        }
        if (e != cudaSuccess) cudaGetLastError();
        const double t = S->now_ms();
        const int m = (int)b->tickets.size();
        double tl[4] = {0.0, 0.0, 0.0, 0.0};
        if (e == cudaSuccess)
            for (int q = 0; q < 4; q++) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, S->ev_ref, S->ev_tl[s][q]) == cudaSuccess) tl[q] = ms;
                else cudaGetLastError();
            }
        const unsigned long long* hc = S->h_counters[s];
        const unsigned long long batch_bits = hc[(size_t)kMaxBatch * kCountersPer + 4];
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (int i = 0; i < m; i++) {
                auto it = S->reqs.find(b->tickets[i]);
                if (it == S->reqs.end()) continue;
                Request& r = it->second;
                if (b->ok[i]) {
                    const unsigned long long bits = hc[(size_t)i * kCountersPer + 4] | batch_bits;
                    // a failed launch, else the lowest device status bit set
                    // (a capacity overflow, a stage wait that ran out)
                    r.t.status = DRK_OK;
                    if (e != cudaSuccess) r.t.status = DRK_ERR_CUDA;
                    else
                        for (int sb = 1; sb < 8; sb++)
                            if (bits & (1ull << sb)) {
                                r.t.status = sb;
                                break;
                            }
                    // pairs per pixel of this scene, kept as the largest recent value
                    const BatchInfo& bi = *info[s];
                    SceneDev& sc = *S->scenes[bi.scene[i]];
                    const double ppp = bi.npix[i] > 0 ? (double)bi.pairs[i] / bi.npix[i] : 0.0;
                    sc.pairs_per_pixel = sc.pairs_per_pixel < 0 ? ppp : std::max(ppp, 0.9 * sc.pairs_per_pixel);
                }
                if (!b->early[i]) r.t.end_ms = t;
                r.t.dev_a0_ms = tl[0];
                r.t.dev_a1_ms = tl[1];
                r.t.dev_b1_ms = tl[2];
                r.t.dev_r1_ms = tl[3];
                r.t.stream = s;
                r.done = true;
            }
            S->inflight_bytes -= std::min(S->inflight_bytes, b->bytes);
        }
        S->cv_done.notify_all();
        b->al.reset();   // stream-ordered frees behind the completed work
        delete b;
        S->running[s] = nullptr;
        info[s].reset();
    }
}

bool any_running(const drk_serve* S) {
    for (int s = 0; s < kStreams; s++)
        if (S->running[s]) return true;
    return false;
}

// Pops the next batch from the queue (caller holds the lock): requests of
// the head's basis-count class in arrival order, at most max_batch, while
// their estimates fit in the budget beside the batches in flight.  A head
// request whose own estimate exceeds the budget completes with
// DRK_ERR_OOM.  start_ms and batch_size are set here.
std::vector<Item> form_batch_locked(drk_serve* S) {
    std::vector<Item> items;
    size_t bytes = 0;
    int kmax = -1;
    const double t = S->now_ms();
    bool failed_any = false;
    for (auto it = S->pending.begin(); it != S->pending.end() && (int)items.size() < S->max_batch;) {
        Request& r = S->reqs[*it];
        const SceneDev& sc = *S->scenes[r.scene];
        if (kmax < 0 && r.est_bytes > S->budget) {
            r.t.status = DRK_ERR_OOM;
            r.t.start_ms = r.t.end_ms = t;
            r.t.batch_size = 0;
            r.done = true;
            failed_any = true;
            it = S->pending.erase(it);
            continue;
        }
        if (kmax >= 0 && sc.kmax != kmax) {
            ++it;
            continue;
        }
        if (S->inflight_bytes + bytes + r.est_bytes > S->budget) break;
        kmax = sc.kmax;
        items.push_back(Item{*it, r.scene, sc.p, r.cam, r.out, r.est_bytes});
        bytes += r.est_bytes;
        it = S->pending.erase(it);
    }
    for (const Item& x : items) {
        Request& r = S->reqs[x.ticket];
        r.t.start_ms = t;
        r.t.batch_size = (int)items.size();
    }
    S->inflight_bytes += bytes;
    if (failed_any) S->cv_done.notify_all();
    return items;
}

}  // namespace

namespace {

// Waits for an event while retiring the other stream's batches; returns
// the event's final status.
cudaError_t wait_event_retiring(drk_serve* S, cudaEvent_t ev, std::unique_ptr<BatchInfo>* info) {
    cudaError_t e;
    while ((e = cudaEventQuery(ev)) == cudaErrorNotReady) {
        retire(S, info);
        sleep_us(20);
    }
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

// Runs one batch on stream s (worker thread, lock not held).
void run_batch(drk_serve* S, int s, std::vector<Item>& items, int* countdown, std::unique_ptr<BatchInfo>* info) {
    cudaStream_t st = S->streams[s];
    const int m = (int)items.size();
    Batch* b = new Batch();
    b->stream = s;
    b->tickets.resize(m);
    b->ok.assign(m, 1);
    b->slot.assign(m, -1);
    b->early.assign(m, 0);
    std::vector<int> status(m, DRK_OK);
    b->al.reset(new Allocs(S->pool, st));
    if (*countdown >= 0) b->al->fail_countdown = countdown;
    std::unique_ptr<BatchInfo> bi(new BatchInfo());
    bi->pairs.assign(m, 0);
    bi->scene.resize(m);
    bi->npix.resize(m);
    size_t est_total = 0;
    for (int i = 0; i < m; i++) {
        b->tickets[i] = items[i].ticket;
        bi->scene[i] = items[i].scene;
        bi->npix[i] = (double)items[i].cam.width * items[i].cam.height;
        est_total += items[i].est;
    }
    const int kmax = items[0].p.K <= 8 ? 8 : 16;
    std::vector<FrameWork> W(m);

    // phase A of every request; the pair totals come back in one wait
    cudaError_t ce = cudaMemsetAsync(S->d_counters[s], 0, sizeof(unsigned long long) * (kMaxBatch + 1) * kCountersPer, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        for (int i = 0; i < m; i++) { b->ok[i] = 0; status[i] = DRK_ERR_CUDA; }
    }
    cudaEventRecord(S->ev_tl[s][0], st);
    for (int i = 0; i < m; i++) {
        if (!b->ok[i]) continue;
        unsigned long long* ctr = S->d_counters[s] + (size_t)i * kCountersPer;
        const drk_status_t e = frame_phase_a(W[i], &items[i].p, &items[i].cam, &S->opt, *b->al, ctr,
                                             reinterpret_cast<int*>(ctr + 4), S->h_totals[s] + i, st, nullptr);
        if (e != DRK_OK) { b->ok[i] = 0; status[i] = e; }
    }
    cudaEventRecord(S->ev_tl[s][1], st);
    cudaEventRecord(S->ev_phase_a[s], st);
    if (wait_event_retiring(S, S->ev_phase_a[s], info) != cudaSuccess)
        for (int i = 0; i < m; i++)
            if (b->ok[i]) { b->ok[i] = 0; status[i] = fail(DRK_ERR_CUDA, "phase A of a batch failed"); }

    // device bytes counted with the actual pair totals; a request that can
    // never fit the budget fails, and the batch waits for the other stream
    // while the two together would not fit
    size_t actual = 0;
    for (int i = 0; i < m; i++) {
        if (!b->ok[i]) continue;
        W[i].P = (int64_t)S->h_totals[s][i];
        bi->pairs[i] = W[i].P;
        const size_t rb = request_bytes(items[i].p.n, kmax, W[i].P, W[i].F.n_tiles, W[i].F.fc.tiles_y);
        if (rb > S->budget) {
            b->ok[i] = 0;
            status[i] = fail(DRK_ERR_OOM, "request needs %zu device bytes, budget %zu", rb, S->budget);
            continue;
        }
        actual += rb;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->inflight_bytes = S->inflight_bytes - std::min(S->inflight_bytes, est_total) + actual;
    }
    b->bytes = actual;
    while (true) {
        size_t other;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            other = S->inflight_bytes - std::min(S->inflight_bytes, actual);
        }
        if (other + actual <= S->budget || !any_running(S)) break;
        retire(S, info);
        sleep_us(20);
    }

    // phase B of every live request
    for (int i = 0; i < m; i++) {
        if (!b->ok[i]) continue;
        const drk_status_t e = frame_phase_b(W[i], *b->al, st, nullptr);
        if (e != DRK_OK) { b->ok[i] = 0; status[i] = e; }
    }

    // frame-major, heaviest-first order over every tile of every live frame, and the slot
    // table the raster reads each task's frame from
    int live = 0;
    int64_t T = 0;
    for (int i = 0; i < m; i++)
        if (b->ok[i]) { live++; T += W[i].F.n_tiles; }
    drk_status_t bs = DRK_OK;
    uint32_t *okeys = nullptr, *ovals = nullptr, *okalt = nullptr, *ovalt = nullptr;
    uint8_t* oscr = nullptr;
    if (live > 0) {
        if (T >= (int64_t(1) << 31)) bs = fail(DRK_ERR_CAPACITY, "batch of %lld tiles", (long long)T);
        if (bs == DRK_OK) bs = b->al->get(&okeys, (size_t)T);
        if (bs == DRK_OK) bs = b->al->get(&ovals, (size_t)T);
        if (bs == DRK_OK) bs = b->al->get(&okalt, (size_t)T);
        if (bs == DRK_OK) bs = b->al->get(&ovalt, (size_t)T);
        if (bs == DRK_OK) bs = b->al->get(&oscr, radix_sort_scratch_bytes(T));
    }
    if (live > 0 && bs == DRK_OK) {
        // frames in decreasing pair count: the raster finishes the heaviest
        // frames of the batch first (they set the tail latency; the light
        // ones have slack)
        std::vector<int> order;
        for (int i = 0; i < m; i++)
            if (b->ok[i]) order.push_back(i);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return W[x].P > W[y].P; });
        int slot = 0;
        int64_t off = 0;
        for (int i : order) {
            const FrameWork& w = W[i];
            launch_batch_order_keys(w.ranges, w.F.n_tiles, slot, okeys + off, ovals + off, st);
            FrameSlot& fs = S->h_slots[s][slot];
            fs.fc = w.F.fc;
            fs.rec = w.A.rec;
            fs.rgb = w.A.rgb;
            fs.keys = w.A.keys;
            fs.vals = w.A.vals;
            fs.ranges = w.ranges;
            fs.dq = w.A.dq;
            fs.out_rgb = items[i].out;
            fs.K = items[i].p.K;
            fs.task_left = S->d_left[s] + slot;
            fs.done_flag = S->d_done[s] + slot;
            S->h_left[s][slot] = (unsigned int)w.F.n_tiles * 8u;
            S->h_done[s][slot] = 0u;
            b->slot[i] = slot;
            off += w.F.n_tiles;
            slot++;
        }
        cudaMemcpyAsync(S->d_slots[s], S->h_slots[s], sizeof(FrameSlot) * (size_t)live, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(S->d_left[s], S->h_left[s], sizeof(unsigned int) * (size_t)live, cudaMemcpyHostToDevice, st);
        radix_sort_pairs(okeys, ovals, okalt, ovalt, T, 26, oscr, st);
        // one raster at a time: this batch's raster starts when the other
        // stream's has ended (the event holds its latest batch's raster
        // end; an idle stream's has long completed).  Phases A/B and the
        // tile order above ran beside that raster; the older batch's
        // frames keep every SM to themselves, so a heavy frame is not
        // slowed by the requests that arrive while it rasterises.
        cudaStreamWaitEvent(st, S->ev_tl[1 - s][3], 0);
        cudaEventRecord(S->ev_tl[s][2], st);
        RasterArgs R;
        std::memset(&R, 0, sizeof(R));
        R.fc = S->h_slots[s][0].fc;
        R.K = S->h_slots[s][0].K;
        R.status = reinterpret_cast<int*>(S->d_counters[s] + (size_t)kMaxBatch * kCountersPer + 4);
        R.task_counter = S->d_task[s];
        R.tile_order = ovals;
        R.slots = S->d_slots[s];
        R.n_batch_tiles = (int)T;
        // overflow columns of the depth-order buffers, kept per stream
        R.ovf_cap = S->opt.ovf_capacity == 0 ? 2048 : std::max(0, (int)S->opt.ovf_capacity);
        const size_t need =
            R.ovf_cap == 0 ? 0 : raster_ovf_bytes(raster_slots(kmax, S->opt.kbuf_capacity, false, true, (int)T));
        if (need > S->ovf_bytes[s]) {
            if (S->ovf[s]) cudaFreeAsync(S->ovf[s], st);
            S->ovf[s] = nullptr;
            S->ovf_bytes[s] = 0;
            void* q = nullptr;
            if (cudaMallocFromPoolAsync(&q, need, S->pool, st) == cudaSuccess) {
                S->ovf[s] = reinterpret_cast<uint4*>(q);
                S->ovf_bytes[s] = need;
            } else {
                cudaGetLastError();   // the raster takes extra list passes instead
            }
        }
        R.ovf = R.ovf_cap > 0 ? S->ovf[s] : nullptr;
        R.ovf_slots = R.ovf ? (int)(S->ovf_bytes[s] / raster_ovf_bytes(1)) : 0;
        launch_raster_batch(R, kmax, S->opt.kbuf_capacity, st);
        bs = check_launch();
    } else {
        cudaEventRecord(S->ev_tl[s][2], st);
    }
    cudaEventRecord(S->ev_tl[s][3], st);
    if (bs != DRK_OK)
        for (int i = 0; i < m; i++)
            if (b->ok[i]) { b->ok[i] = 0; status[i] = bs; }
    cudaMemcpyAsync(S->h_counters[s], S->d_counters[s], sizeof(unsigned long long) * (kMaxBatch + 1) * kCountersPer,
                    cudaMemcpyDeviceToHost, st);
    if (cudaEventRecord(b->ev = S->ev_done[s], st) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(st);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (int i = 0; i < m; i++)
            if (!b->ok[i]) {
                auto it = S->reqs.find(items[i].ticket);
                if (it != S->reqs.end()) it->second.t.status = status[i];
            }
    }
    S->running[s] = b;
    info[s] = std::move(bi);
}

void worker_main(drk_serve* S) {
    cudaSetDevice(S->device);
    std::unique_ptr<BatchInfo> info[kStreams];
    while (true) {
        retire(S, info);
        int free_s = -1;
        for (int s = 0; s < kStreams && free_s < 0; s++)
            if (!S->running[s]) free_s = s;
        std::vector<Item> items;
        int countdown = -1;
        int gen = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop && S->pending.empty() && !any_running(S)) break;
            if (free_s >= 0 && !S->pending.empty()) items = form_batch_locked(S);
            if (items.empty()) {
                if (any_running(S)) S->cv_work.wait_for(lk, std::chrono::microseconds(50));
                else if (S->pending.empty() && !S->stop) S->cv_work.wait(lk);
                continue;
            }
            countdown = S->fail_countdown;
            gen = S->inject_gen;
        }
        run_batch(S, free_s, items, &countdown, info);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->inject_gen == gen) S->fail_countdown = countdown < 0 ? -1 : countdown;
        }
    }
}

}  // namespace

namespace {

void free_server(drk_serve* S) {
    cudaSetDevice(S->device);
    for (int s = 0; s < kStreams; s++) {
        if (S->streams[s]) cudaStreamSynchronize(S->streams[s]);
        if (S->h_totals[s]) cudaFreeHost(S->h_totals[s]);
        if (S->h_slots[s]) cudaFreeHost(S->h_slots[s]);
        if (S->h_counters[s]) cudaFreeHost(S->h_counters[s]);
        cudaFree(S->d_slots[s]);
        cudaFree(S->d_counters[s]);
        cudaFree(S->d_task[s]);
        if (S->ovf[s]) cudaFree(S->ovf[s]);
        cudaFree(S->d_left[s]);
        if (S->h_left[s]) cudaFreeHost(S->h_left[s]);
        if (S->h_done[s]) cudaFreeHost(S->h_done[s]);
        if (S->ev_phase_a[s]) cudaEventDestroy(S->ev_phase_a[s]);
        if (S->ev_done[s]) cudaEventDestroy(S->ev_done[s]);
        for (int q = 0; q < 4; q++)
            if (S->ev_tl[s][q]) cudaEventDestroy(S->ev_tl[s][q]);
        if (S->streams[s]) cudaStreamDestroy(S->streams[s]);
    }
    if (S->ev_ref) cudaEventDestroy(S->ev_ref);
    for (auto& sc : S->scenes) cudaFree(sc->mem);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    delete S;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" {

drk_status_t drk_serve_create(int device, size_t mem_budget, int max_batch, const drk_options_t* opt,
                              drk_serve_t** out) {
    if (!out || !opt) return fail(DRK_ERR_INVALID_ARG, "null out or options");
    *out = nullptr;
    if (max_batch < 1 || max_batch > kMaxBatch) return fail(DRK_ERR_INVALID_ARG, "max_batch %d not in 1..64", max_batch);
    if (mem_budget == 0) return fail(DRK_ERR_INVALID_ARG, "zero memory budget");
    {
        // options are checked with a minimal valid scene and camera
        drk_params_t p{};
        p.K = 8;
        p.sh_degree = -1;
        drk_camera_t c{};
        c.width = c.height = 1;
        c.fx = c.fy = 1.f;
        const drk_status_t s = validate(&p, &c, opt);
        if (s != DRK_OK) return s;
    }
    int ndev = 0;
    DRK_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(DRK_ERR_INVALID_ARG, "device %d of %d", device, ndev);
    DRK_CUDA(cudaSetDevice(device));
    drk_serve* S = new (std::nothrow) drk_serve();
    if (!S) return fail(DRK_ERR_OOM, "host allocation failed");
    S->device = device;
    S->opt = *opt;
    S->budget = mem_budget;
    S->max_batch = max_batch;
    S->t0 = Clock::now();
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    bool ok = cudaMemPoolCreate(&S->pool, &props) == cudaSuccess;
    if (ok) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    const size_t nctr = (size_t)(kMaxBatch + 1) * kCountersPer;
    for (int s = 0; s < kStreams && ok; s++) {
        ok = cudaStreamCreateWithFlags(&S->streams[s], cudaStreamNonBlocking) == cudaSuccess &&
             cudaMallocHost(&S->h_totals[s], sizeof(uint64_t) * kMaxBatch) == cudaSuccess &&
             cudaMallocHost(&S->h_slots[s], sizeof(FrameSlot) * kMaxBatch) == cudaSuccess &&
             cudaMallocHost(&S->h_counters[s], sizeof(unsigned long long) * nctr) == cudaSuccess &&
             cudaMalloc(&S->d_slots[s], sizeof(FrameSlot) * kMaxBatch) == cudaSuccess &&
             cudaMalloc(&S->d_counters[s], sizeof(unsigned long long) * nctr) == cudaSuccess &&
             cudaMalloc(&S->d_task[s], sizeof(unsigned int)) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->ev_phase_a[s], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->ev_done[s], cudaEventDisableTiming) == cudaSuccess &&
             cudaMalloc(&S->d_left[s], sizeof(unsigned int) * kMaxBatch) == cudaSuccess &&
             cudaMallocHost(&S->h_left[s], sizeof(unsigned int) * kMaxBatch) == cudaSuccess &&
             cudaHostAlloc(&S->h_done[s], sizeof(unsigned int) * kMaxBatch, cudaHostAllocMapped) == cudaSuccess &&
             cudaHostGetDevicePointer(reinterpret_cast<void**>(&S->d_done[s]), S->h_done[s], 0) == cudaSuccess;
    }
    for (int s = 0; s < kStreams && ok; s++)
        for (int q = 0; q < 4 && ok; q++) ok = cudaEventCreate(&S->ev_tl[s][q]) == cudaSuccess;
    // the device-time origin of the batch timelines
    ok = ok && cudaEventCreate(&S->ev_ref) == cudaSuccess && cudaEventRecord(S->ev_ref, S->streams[0]) == cudaSuccess &&
         cudaEventSynchronize(S->ev_ref) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_server(S);
        return fail(DRK_ERR_OOM, "server buffers");
    }
    try {
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        free_server(S);
        return fail(DRK_ERR_OOM, "worker thread");
    }
    *out = S;
    return DRK_OK;
}

drk_status_t drk_serve_add_scene(drk_serve_t* S, const drk_params_t* params, int* scene_id) {
    if (!S || !params || !scene_id) return fail(DRK_ERR_INVALID_ARG, "null argument");
    drk_camera_t c{};
    c.width = c.height = 1;
    c.fx = c.fy = 1.f;
    drk_status_t s = validate(params, &c, &S->opt);
    if (s != DRK_OK) return s;
    DRK_CUDA(cudaSetDevice(S->device));
    const int64_t n = params->n;
    const int K = params->K;
    const size_t ncol = params->sh_degree < 0 ? 3 : (size_t)(params->sh_degree + 1) * (params->sh_degree + 1) * 3;
    const float* src[8] = {params->mu, params->quat, params->scale, params->theta,
                           params->eta, params->tau, params->opacity, params->color};
    const size_t cnt[8] = {3 * (size_t)n, 4 * (size_t)n, (size_t)K * n, (size_t)K * n,
                           (size_t)n, (size_t)n, (size_t)n, ncol * n};
    size_t total = 0;
    for (int j = 0; j < 8; j++) total += align256(cnt[j] * sizeof(float));
    std::unique_ptr<SceneDev> sc(new SceneDev());
    if (cudaMalloc(&sc->mem, total > 0 ? total : 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(DRK_ERR_OOM, "scene copy of %zu bytes", total);
    }
    sc->bytes = total;
    float* dst[8];
    size_t off = 0;
    for (int j = 0; j < 8; j++) {
        dst[j] = reinterpret_cast<float*>(static_cast<char*>(sc->mem) + off);
        if (cnt[j] > 0) {
            const cudaError_t e = cudaMemcpyAsync(dst[j], src[j], cnt[j] * sizeof(float), cudaMemcpyDeviceToDevice, 0);
            if (e != cudaSuccess) {
                cudaFree(sc->mem);
                return fail(DRK_ERR_CUDA, "scene copy: %s", cudaGetErrorString(e));
            }
        }
        off += align256(cnt[j] * sizeof(float));
    }
    // the worker's streams do not synchronise with the legacy stream
    const cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        cudaFree(sc->mem);
        return fail(DRK_ERR_CUDA, "scene copy: %s", cudaGetErrorString(e));
    }
    sc->p = *params;
    sc->p.mu = dst[0]; sc->p.quat = dst[1]; sc->p.scale = dst[2]; sc->p.theta = dst[3];
    sc->p.eta = dst[4]; sc->p.tau = dst[5]; sc->p.opacity = dst[6]; sc->p.color = dst[7];
    sc->kmax = K <= 8 ? 8 : 16;
    std::lock_guard<std::mutex> lk(S->mu);
    *scene_id = (int)S->scenes.size();
    S->scenes.push_back(std::move(sc));
    return DRK_OK;
}

drk_status_t drk_serve_submit(drk_serve_t* S, int scene_id, const drk_camera_t* cam, float* out_rgb,
                              uint64_t* ticket) {
    if (!S || !cam || !ticket) return fail(DRK_ERR_INVALID_ARG, "null argument");
    if (!out_rgb) return fail(DRK_ERR_INVALID_ARG, "null output image");
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(DRK_ERR_INVALID_ARG, "server is shutting down");
    if (scene_id < 0 || scene_id >= (int)S->scenes.size()) return fail(DRK_ERR_NOT_FOUND, "scene %d", scene_id);
    const SceneDev& sc = *S->scenes[scene_id];
    const drk_status_t s = validate(&sc.p, cam, &S->opt);
    if (s != DRK_OK) return s;
    // pairs: the scene's recent pairs per pixel with headroom, else a guess
    // of 12 per pixel (about the clustered 1080p workload) or 16 per primitive
    const double npix = (double)cam->width * cam->height;
    const double pairs = sc.pairs_per_pixel >= 0 ? 1.25 * sc.pairs_per_pixel * npix + 1024
                                                 : std::max(12.0 * npix, 16.0 * (double)sc.p.n);
    const int n_tiles = ((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
    Request r;
    r.scene = scene_id;
    r.cam = *cam;
    r.out = out_rgb;
    r.est_bytes = request_bytes(sc.p.n, sc.kmax, (int64_t)pairs, n_tiles, (cam->height + kTile - 1) / kTile);
    r.t.arrival_ms = S->now_ms();
    r.t.status = DRK_OK;
    const uint64_t tk = S->next_ticket++;
    S->reqs.emplace(tk, r);
    S->pending.push_back(tk);
    *ticket = tk;
    S->cv_work.notify_one();
    return DRK_OK;
}

drk_status_t drk_serve_poll(drk_serve_t* S, uint64_t ticket, int* done, drk_serve_timing_t* t) {
    if (!S || !done) return fail(DRK_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(DRK_ERR_NOT_FOUND, "ticket %llu", (unsigned long long)ticket);
    *done = it->second.done ? 1 : 0;
    if (t) *t = it->second.t;
    return DRK_OK;
}

drk_status_t drk_serve_wait(drk_serve_t* S, uint64_t ticket, double timeout_ms, drk_serve_timing_t* t) {
    if (!S) return fail(DRK_ERR_INVALID_ARG, "null server");
    if (!(timeout_ms >= 0.0)) return fail(DRK_ERR_INVALID_ARG, "negative timeout");
    const auto deadline = Clock::now() + std::chrono::microseconds((long long)(std::min(timeout_ms, 1e9) * 1000.0));
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(DRK_ERR_NOT_FOUND, "ticket %llu", (unsigned long long)ticket);
        if (it->second.done) {
            if (t) *t = it->second.t;
            return DRK_OK;
        }
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto jt = S->reqs.find(ticket);
            if (jt != S->reqs.end() && jt->second.done) {
                if (t) *t = jt->second.t;
                return DRK_OK;
            }
            return fail(DRK_ERR_TIMEOUT, "ticket %llu not done after %.3f ms", (unsigned long long)ticket, timeout_ms);
        }
    }
}

drk_status_t drk_serve_release(drk_serve_t* S, uint64_t ticket) {
    if (!S) return fail(DRK_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(DRK_ERR_NOT_FOUND, "ticket %llu", (unsigned long long)ticket);
    if (!it->second.done) return fail(DRK_ERR_BUSY, "ticket %llu is not done", (unsigned long long)ticket);
    S->reqs.erase(it);
    return DRK_OK;
}

drk_status_t drk_serve_inject_alloc_failure(drk_serve_t* S, int n) {
    if (!S) return fail(DRK_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    S->fail_countdown = n < 0 ? -1 : n;
    S->inject_gen++;
    return DRK_OK;
}

drk_status_t drk_serve_destroy(drk_serve_t* S) {
    if (!S) return DRK_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    free_server(S);
    return DRK_OK;
}

}  // extern "C"
