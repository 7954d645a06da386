/*
 * drk.h -- C ABI of libdrk, the GB300 (sm_103a) hot path of Deformable
 * Radial Kernel (DRK) splatting.
 *
 * The library renders planar DRK primitives (Sec. 4: centre mu, rotation q,
 * K radial bases (s_k, theta_k), L1/L2 blend eta, sharpness tau, opacity o,
 * colour) through a tile-based rasterizer (Sec. 4.4, "Kernel Culling" and
 * "Cache Sorting"): per-primitive preprocess with a conservative K-basis
 * screen bound, per-(primitive, tile) pair emission with tile culling, a
 * device radix sort on tile|depth keys, and a per-tile rasterizer that
 * intersects each pixel ray with the primitive plane (Eq. 4, Eq. 5),
 * evaluates the kernel (Eq. 6 - Eq. 10), and composites front to back in
 * exact per-pixel ray-depth order (Eq. 1, Eq. 13).  The derivative of the
 * rendered image with respect to every primitive parameter is available
 * through drk_render_backward (the paper trains through its renderer,
 * Sec. 1 and the supplementary "Tensor Graph"; the backward visits each
 * pixel's contributors front to back as the supplementary "Cache-Sorting"
 * paragraph requires).
 *
 * Conventions (the paper leaves these open):
 *   - Pinhole camera, OpenCV axes (x right, y down, z forward); pixel (x, y)
 *     has its centre at (x + 0.5, y + 0.5); world_to_cam is the row-major
 *     3 x 4 [R | t] with x_cam = R x_world + t, R orthonormal.
 *   - R_x, R_y, R_z of Eq. 4 / Eq. 5 are the columns of R(q), q = (w, x, y, z)
 *     normalised by the library.
 *   - The polar angle is atan2(v, u) over the full circle; angles
 *     theta_0 < ... < theta_{K-1} with theta_{K-1} - theta_0 < 2 pi and every
 *     cyclic gap below pi; the last sector wraps to theta_0 + 2 pi with s_0.
 *   - r_t (Eq. 13) is the view-space depth of the ray-plane intersection;
 *     pairs with r_t <= near_plane are skipped.
 *   - alpha_tilde = min(max(o Psi(g), filter), alpha_max) (Eq. 9, Eq. 10);
 *     a pair contributes iff alpha_tilde >= alpha_min; compositing stops
 *     before the first contributor with T (1 - alpha_tilde) < T_min;
 *     contributors are composited in (r_t, primitive index) order.
 *   - Colour: plain RGB (sh_degree = -1) or real spherical harmonics of
 *     degree 0..3 evaluated in the direction camera centre -> mu, plus 0.5,
 *     clamped below at 0.  bg is added with the final transmittance.
 *
 * Memory: every pointer argument that refers to per-primitive or per-pixel
 * data is a DEVICE pointer owned by the caller, unless a field says
 * otherwise.  Structures themselves are passed by host pointer and read
 * during the call only.  All calls with a `stream` argument are
 * asynchronous on that stream (a cudaStream_t passed as void*, NULL = the
 * legacy default stream) unless stated; they never call
 * cudaDeviceSynchronize.  Errors detected on the host are returned before
 * anything is launched; errors detected on the device (capacity) are
 * recorded in the context and returned by the next synchronising call.
 * drk_last_error() gives a message for the last failure on the calling
 * thread.  No call traps or asserts on the device.
 */
#ifndef DRK_H
#define DRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DRK_OK = 0,
    DRK_ERR_INVALID_ARG = 1,  /* rejected on the host before any launch */
    DRK_ERR_OOM = 2,          /* device allocation failed or over budget */
    DRK_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    DRK_ERR_CAPACITY = 4,     /* a fixed-capacity buffer was too small */
    DRK_ERR_TIMEOUT = 5,      /* a bounded wait expired */
    DRK_ERR_BUSY = 6,         /* no free slot; retry later */
    DRK_ERR_NOT_FOUND = 7     /* unknown ticket or scene */
} drk_status_t;

/* Activated DRK parameters (Sec. 4), structure of arrays, float32, device.
 *   mu       n x 3           centre
 *   quat     n x 4           rotation (w, x, y, z), any non-zero norm
 *   scale    n x K           radial lengths s_k > 0
 *   theta    n x K           polar angles, ascending (see conventions)
 *   eta      n               L1/L2 blend in [0, 1] (Eq. 8)
 *   tau      n               sharpness in (-1, 1) (Eq. 9)
 *   opacity  n               o in (0, 1]
 *   color    n x 3           plain RGB when sh_degree = -1, else
 *            n x (d+1)^2 x 3 SH coefficients, coefficient-major, RGB inner
 * 3 <= K <= 16, -1 <= sh_degree <= 3, 0 <= n < 2^31. */
typedef struct {
    int64_t n;
    int32_t K;
    int32_t sh_degree;
    const float *mu, *quat, *scale, *theta, *eta, *tau, *opacity, *color;
} drk_params_t;

/* Gradients, same shapes as drk_params_t; written (not accumulated) by
 * drk_render_backward. */
typedef struct {
    float *mu, *quat, *scale, *theta, *eta, *tau, *opacity, *color;
} drk_params_grad_t;

typedef struct {
    int32_t width, height;      /* 1 .. 16384 */
    float fx, fy, cx, cy;       /* pixels */
    float world_to_cam[12];     /* host values, row-major 3 x 4 */
} drk_camera_t;

/* Compositing orders.  DRK_ORDER_EXACT composites each pixel's contributors
 * in exact (r_t, primitive index) order.  DRK_ORDER_CACHE_SORT is the
 * paper's cache-sorting (Sec. 4.4 "Cache Sorting", supplementary
 * Algorithm 1), an approximation kept for comparison: pairs are pre-sorted
 * by the view-space depth of the primitive centre, and each pixel keeps a
 * cache of kbuf_capacity contributors sorted by r_t whose smallest entry is
 * composited when it overflows.  Forward only (no backward state). */
enum {
    DRK_ORDER_EXACT = 0,
    DRK_ORDER_CACHE_SORT = 1
};

/* Tile culling levels (Sec. 4.4, "Kernel Culling").  The first three give
 * the same image bit for bit: culling only removes pairs that cannot reach
 * alpha_min.  DRK_CULL_PAPER is the paper's culling as printed, kept for
 * comparison: a tile is kept iff it meets the polygon of the basis
 * endpoints v_k = mu + s_k sqrt(-log Psi^-1(alpha_min / o)) (cos theta_k
 * R_x + sin theta_k R_y) (Eq. 11 - Eq. 12), tested in the primitive's plane
 * with the tile's corner pixels.  It is lossy: Eq. 11 omits the factor 2
 * of the exponent (the printed radius is 1/sqrt 2 of the alpha_min contour
 * at o = 1, tau = 0), the chords between endpoints cut off the L2 contour,
 * and the low-pass filter's disc is not considered.  Tiles whose corner
 * rays do not all meet the plane in front of the camera are kept. */
enum {
    DRK_CULL_NONE = 0,   /* every primitive is paired with every tile */
    DRK_CULL_RECT = 1,   /* tiles of the screen rectangle of the K-basis bound */
    DRK_CULL_TILE = 2,   /* plus a per-tile test against the per-sector radii */
    DRK_CULL_PAPER = 3   /* the paper's endpoint polygon (lossy) */
};

typedef struct {
    float alpha_min;      /* contribution threshold; default exp(-9) (Eq. 11) */
    float T_min;          /* early-termination transmittance; default 1e-4 */
    float alpha_max;      /* alpha clamp; default 0.99 */
    float lowpass_sl;     /* low-pass filter radius s_l of Eq. 10 in pixels; 0 = off */
    float near_plane;     /* default 0.2 */
    float bg[3];          /* background colour */
    int32_t cull_level;   /* DRK_CULL_*; default DRK_CULL_TILE */
    int32_t kbuf_capacity;/* per-pixel depth-order heap slots in shared
                             memory: 8, 16 (default) or 32 (any value gives
                             the same image; deeper heaps continue in the
                             overflow column); in DRK_ORDER_CACHE_SORT the
                             cache length (the paper uses 8) */
    int32_t ovf_capacity; /* depth-order heap slots per pixel in global memory
                             beyond the kbuf_capacity slots in shared memory
                             (any value gives the same image): 0 = 2048
                             (default), 1..2048, or -1 = none (a full heap
                             then takes extra passes over the list) */
    int32_t order_mode;   /* DRK_ORDER_*; default DRK_ORDER_EXACT */
    int32_t record_chunks;/* upper bound on the contributor records a forward
                             with a backward state keeps, in chunks of 1024
                             records (24 B each); 0 = automatic (sized from
                             the previous recording forward).  Tiles whose
                             records do not fit are replayed exactly by the
                             backward instead (same gradients, slower) */
    int32_t reserved[3];  /* must be zero */
} drk_options_t;

/* Fills *opt with the defaults listed above. */
void drk_options_default(drk_options_t *opt);

/* Output image, device, float32 planar. */
typedef struct {
    float *rgb;           /* 3 x H x W, includes T_final * bg */
    float *T_final;       /* H x W final transmittance, may be NULL */
    int32_t *n_emitted;   /* H x W number of composited contributors, may be NULL */
    /* Depth and normal images (supplementary "Converting Mesh to DRK"),
     * composited with the colour's weights T_i alpha_i: depth = sum of
     * T_i alpha_i r_t,i (view depth, Eq. 13), normal = sum of T_i alpha_i
     * n_i with n_i the unit normal of primitive i's plane in camera
     * coordinates, oriented towards the camera.  Unnormalised: divide by
     * 1 - T_final for the mean over the covered part.  Either may be NULL
     * (not computed); when one is given the forward raster runs a variant
     * that also accumulates them.  Not differentiated by
     * drk_render_backward. */
    float *depth;         /* H x W, may be NULL */
    float *normal;        /* 3 x H x W, may be NULL */
} drk_image_t;

/* Counters of the last render on a context (device-side counts). */
typedef struct {
    int64_t n_visible;    /* primitives with a non-empty bound */
    int64_t n_pairs;      /* (primitive, tile) pairs after culling */
    int64_t n_evals;      /* kernel evaluations (pixel, primitive) */
    int64_t n_emitted;    /* composited contributions */
    int64_t n_extra_passes;/* extra list passes taken by pixels whose depth
                             buffer filled (exactness is kept) */
    int64_t n_tiles;
    int64_t n_contrib_evals;/* evaluations with alpha_tilde >= alpha_min */
    int64_t n_spills;     /* contributors pushed while the shared-memory
                             part of their pixel's depth-order heap was full
                             (they went to the overflow column) */
    int64_t n_replay_evals;/* evaluations made by the exact replay of the
                             last drk_render_backward (tiles whose recorded
                             lists did not fit) */
    int64_t n_geo_evals;  /* evaluations that passed the geometry stage (ray
                             in front, point within the support radius or
                             the filter's reach) */
    int32_t key_bits_depth;
    int32_t status;       /* device-side drk_status_t of the last render */
} drk_stats_t;

typedef struct drk_ctx drk_ctx_t;
typedef struct drk_state drk_state_t;

/* A context owns device scratch memory (grown on demand from a
 * stream-ordered pool) and the counters of its last render.  One context
 * may be used from one host thread at a time.  `device` is the CUDA
 * ordinal. */
drk_status_t drk_ctx_create(int device, drk_ctx_t **out);
void drk_ctx_destroy(drk_ctx_t *ctx);

/* Forward render (Sec. 4.4 pipeline).  params, cam, opt: host structs whose
 * array fields are device pointers.  out: device image buffers of the
 * camera's size.  If state != NULL, *state receives a library-owned object
 * holding what drk_render_backward needs (free it with drk_state_free).
 * The call reads the pair count back to the host once (a stream sync) to
 * size the sort; everything else is asynchronous.  Returns
 * DRK_ERR_INVALID_ARG for bad sizes or options, DRK_ERR_OOM if scratch
 * cannot grow, DRK_ERR_CUDA on a launch failure.  Conditions found on the
 * device (a bounded wait that ran out, a capacity bound) do not change the
 * return value: they surface as drk_stats_t.status of drk_get_stats. */
drk_status_t drk_render(drk_ctx_t *ctx, const drk_params_t *params, const drk_camera_t *cam,
                        const drk_options_t *opt, const drk_image_t *out, drk_state_t **state,
                        void *stream);

/* Reverse mode of drk_render (Eq. 1 and Eq. 4 - Eq. 10, taken front to
 * back as the supplementary "Cache-Sorting" paragraph describes) for the
 * same params, cam and opt and the state it produced:
 * grads <- d(sum dL_drgb * rgb)/d(params), with respect to the activated
 * parameters.  dL_drgb is a device 3 x H x W array; grads holds device
 * arrays of the parameters' shapes, overwritten.  The state stays owned by
 * the caller and may be used again.  The call reads the forward's record
 * count back once (a stream sync) to size the grouping of the records;
 * everything else is asynchronous.  Returns DRK_ERR_INVALID_ARG when
 * params, cam or opt do not match the state, for the cache-sorting order
 * (it has no backward) or for a null gradient array; DRK_ERR_OOM or
 * DRK_ERR_CUDA as drk_render does. */
drk_status_t drk_render_backward(drk_ctx_t *ctx, const drk_params_t *params, const drk_camera_t *cam,
                                 const drk_options_t *opt, const drk_state_t *state,
                                 const float *dL_drgb, const drk_params_grad_t *grads, void *stream);

/* Frees a state of drk_render (stream-ordered on the stream of its
 * render); NULL is a no-op. */
void drk_state_free(drk_state_t *state);

/* Stable ascending sort of n (key, value) pairs by the low key_bits bits of
 * the keys (1..32), in place, on device arrays -- the LSD radix sort the
 * render uses for its (tile | depth) keys (Sec. 4.4).  Scratch comes from
 * the context's pool.  Asynchronous.  n < 2^32. */
drk_status_t drk_sort_pairs(drk_ctx_t *ctx, uint32_t *keys, uint32_t *vals, int64_t n, int key_bits, void *stream);

/* drk_sort_pairs without any device allocation, for callers that cannot
 * allocate when they sort: an embedder whose device memory is handed out
 * once at start-up and never grows, a real-time loop that must not meet the
 * implicit synchronisation or latency of an allocation, or code inside a
 * custom allocator's own bookkeeping, which must not re-enter it.  The
 * paper has no counterpart; this is a service of the library.
 *   keys, vals  device arrays of n uint32 on the CURRENT device (sorted in
 *               place, stable, by the low key_bits bits of the keys, 1..32);
 *               host pointers or arrays of another device are refused with
 *               DRK_ERR_INVALID_ARG before anything is launched
 *   n           0 .. 1048576 (2^20); larger n returns DRK_ERR_CAPACITY
 *               before anything is launched; n <= 1 returns at once
 * Working memory is one fixed device array inside the library (9 MiB per
 * GPU that loads it, held until the process exits); the call allocates and
 * frees nothing.  The first call on a device looks the array's address up
 * with that device current and keeps it; a device reset (which unloads the
 * library's device image) invalidates it, so do not call this entry point
 * after resetting a device it was used on.  All calls share the array and
 * it keeps the contents of the last call: calls whose work could overlap on
 * the GPU (different streams, or different host threads) race on it and
 * must be ordered by the caller.  Asynchronous on `stream`; DRK_ERR_CUDA if
 * a launch fails (message in drk_last_error). */
drk_status_t drk_sort_pairs_static(uint32_t *keys, uint32_t *vals, int64_t n, int key_bits, void *stream);

/* Synchronises the stream of the last render and copies its counters into
 * *out (host).  out->status is the lowest device status bit the last
 * render or backward set (DRK_OK if none).  DRK_ERR_INVALID_ARG for a null
 * argument, DRK_ERR_CUDA if the copy fails. */
drk_status_t drk_get_stats(drk_ctx_t *ctx, drk_stats_t *out);

/* Stage timing with CUDA events recorded on the caller's stream around each
 * stage of drk_render / drk_render_backward.  Stages: 0 preprocess (bounds,
 * culling count, scan), 1 pair emission, 2 radix sort, tile ranges and tile
 * order, 3 raster forward, 4 raster backward over the contributor records,
 * 5 preprocess backward, 6 exact replay of tiles whose records overflowed,
 * 7 grouping of the contributor records.  drk_timing_enable resets the
 * accumulators and switches timing on (enable != 0) or off.
 * drk_timing_read waits for the recorded events and returns, per stage, the
 * summed milliseconds and the number of timed launches (host arrays of 8). */
drk_status_t drk_timing_enable(drk_ctx_t *ctx, int enable);
drk_status_t drk_timing_read(drk_ctx_t *ctx, double *ms, int64_t *launches);

/* Statistics of the forward raster (n_evals, n_geo_evals, n_contrib_evals,
 * n_emitted and n_spills of drk_stats_t) are collected by default.  With
 * enable = 0 the forward of later drk_render calls on this context runs a
 * kernel without them (its per-lane counters cost the 1080p forward about
 * 1.5 % of its time) and those five fields read 0; images, records and
 * gradients are the same bit for bit.  n_visible, n_pairs, n_extra_passes,
 * n_replay_evals and the status word are always kept.  Takes effect at the
 * next render; no device work.  DRK_ERR_INVALID_ARG for a null context. */
drk_status_t drk_stats_enable(drk_ctx_t *ctx, int enable);

/* Measured arithmetic throughput of one GPU (operations per second): the
 * FP32 FMA pipe (an FMA counted as one operation) and the transcendental
 * unit for ex2.approx, rcp.approx and cos.approx, each from the library's
 * own kernels with independent dependent chains filling every SM (best of
 * five timed launches after a warm-up).  A measurement utility: the paper
 * has no counterpart; the rasterizer's roofline takes these as its peaks
 * (it is bound by these two units).  Synchronous, about 20 ms; allocates a
 * few bytes of device memory. */
typedef struct {
    double fma_ops, ex2_ops, rcp_ops, cos_ops;
    int32_t sms;
    int32_t reserved;
} drk_pipe_peaks_t;
drk_status_t drk_measure_pipes(int device, drk_pipe_peaks_t *out);

/* Number of kernel launches the library has issued so far, process-wide
 * (host counter). */
int64_t drk_launch_count(void);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over resident scenes.
 *
 * A server owns a worker thread, two CUDA streams and copies of its scenes
 * in device memory.  drk_serve_submit queues a camera request; the worker
 * forms a batch from the queued requests whenever one of its two streams is
 * free (at most max_batch requests, while their estimated device memory
 * fits in mem_budget beside the batch already running), renders every
 * request of the batch with one preprocess/sort phase per request and ONE
 * rasterizer launch over all tiles of all of them.  A ticket is marked
 * done as soon as its frame is complete: the rasterizer runs the batch
 * frame by frame (heaviest tiles first within a frame), and the warp that
 * finishes a frame's last tile sets a flag in host-mapped memory that the
 * worker polls; at the latest when the batch's completion event fires.
 * Requests that arrive while a batch runs join the next batch, whose
 * preprocess and sort overlap the running batch's rasterizer.  Each image is bit-identical to a
 * drk_render of the same scene and camera (the batch does not change any
 * pixel's arithmetic or order).  All requests of a batch share one basis
 * count class (K <= 8 or K <= 16).  The rendering options are the server's.
 */
typedef struct drk_serve drk_serve_t;

typedef struct {
    double arrival_ms;    /* submit time, ms since the server was created */
    double start_ms;      /* its batch was launched */
    double end_ms;        /* its frame was complete (worker saw the flag or
                             the batch's event) */
    int32_t batch_size;   /* requests in its batch */
    int32_t status;       /* drk_status_t of the request */
    /* device timeline of its batch (CUDA events on the batch's stream, ms
     * since an event recorded when the server was created; 0 until the
     * whole batch has finished): phase A (preprocess, culling count, scan)
     * began, phase A ended, phase B (emission, sort, tile ranges, batch
     * tile order) ended = the batch raster began, the raster ended */
    double dev_a0_ms, dev_a1_ms, dev_b1_ms, dev_r1_ms;
    int32_t stream;       /* the server stream (0 or 1) the batch ran on */
    int32_t reserved;
} drk_serve_timing_t;

/* device: CUDA ordinal; mem_budget: device bytes the in-flight batches may
 * use (estimated before, counted after preprocess); max_batch: 1..64 (1
 * renders one request at a time); opt: rendering options (copied). */
drk_status_t drk_serve_create(int device, size_t mem_budget, int max_batch, const drk_options_t *opt,
                              drk_serve_t **out);
/* Copies the scene's parameter arrays (device pointers) into server-owned
 * device memory; *scene_id receives its index. Synchronous. */
drk_status_t drk_serve_add_scene(drk_serve_t *srv, const drk_params_t *params, int *scene_id);
/* Queues a request; out_rgb is a caller-owned device buffer of
 * 3 x H x W floats that must stay valid until the ticket is done.  Returns
 * DRK_ERR_NOT_FOUND for an unknown scene, DRK_ERR_INVALID_ARG for a bad
 * camera.  A request whose own estimate exceeds mem_budget completes with
 * status DRK_ERR_OOM. */
drk_status_t drk_serve_submit(drk_serve_t *srv, int scene_id, const drk_camera_t *cam, float *out_rgb,
                              uint64_t *ticket);
/* *done = 1 once the ticket's image is complete (or failed; see t->status).
 * t may be NULL.  DRK_ERR_NOT_FOUND for an unknown or released ticket. */
drk_status_t drk_serve_poll(drk_serve_t *srv, uint64_t ticket, int *done, drk_serve_timing_t *t);
/* Waits up to timeout_ms for the ticket (DRK_ERR_TIMEOUT when it is not
 * done by then).  Done tickets are kept until drk_serve_release. */
drk_status_t drk_serve_wait(drk_serve_t *srv, uint64_t ticket, double timeout_ms, drk_serve_timing_t *t);
drk_status_t drk_serve_release(drk_serve_t *srv, uint64_t ticket);
/* Fault injection for tests: the n-th device allocation the worker makes
 * from now on (0 = the next one) fails as if the device were out of
 * memory; the affected request completes with DRK_ERR_OOM and the server
 * continues.  n < 0 switches it off. */
drk_status_t drk_serve_inject_alloc_failure(drk_serve_t *srv, int n);
/* Drains the queue, joins the worker and frees everything. */
drk_status_t drk_serve_destroy(drk_serve_t *srv);

/* ------------------------------------------------------------------------
 * Training: the activations of the learnable parameters (supplementary
 * "Parametrization") and the optimiser step that fits them ("Model
 * Training": Adam as in 3D-GS, learning rates decayed exponentially).
 *
 * Raw parameters are unconstrained float32 device arrays with the shapes
 * of drk_params_t.  The activated parameters the renderer reads are
 *   opacity = sigmoid(x),  eta = sigmoid(x),  scale_k = exp(x_k),
 *   tau     = -0.1 + 1.09 sigmoid(x)          (the range (-0.1, 0.99)),
 *   quat    = x / |x|                          ((1, 0, 0, 0) when x = 0),
 *   theta_0 = 0, theta_k = 2 pi (w_0 + ... + w_{k-1}) / (w_0 + ... + w_{K-1})
 *             with w_j = min(sigmoid(x_j), 1 - 1e-3) + 1 / (K - 2),
 * so every cyclic gap between angles stays below pi (the cap keeps it
 * below pi even where float32 sigmoids saturate).  mu and color are used
 * as they are: the renderer reads the raw arrays. */
typedef struct {
    int64_t n;
    int32_t K;            /* 3 .. 16 */
    int32_t sh_degree;    /* -1 .. 3, as in drk_params_t */
    float *mu, *quat, *scale, *theta, *eta, *tau, *opacity, *color;
} drk_raw_params_t;

/* Writes the activated quat, scale, theta, eta, tau and opacity of raw
 * into out (device arrays of drk_params_t shapes; out->mu and out->color
 * are not touched).  Returns DRK_ERR_INVALID_ARG for n < 0, K outside
 * 3..16 or a NULL array when n > 0. */
drk_status_t drk_activate(const drk_raw_params_t *raw, const drk_params_grad_t *out, void *stream);

/* Chain rule through the activations: from gradients of the activated
 * parameters (g_act, as drk_render_backward writes them) to gradients of
 * the raw ones (g_raw, written; mu and color are copied). */
drk_status_t drk_activate_backward(const drk_raw_params_t *raw, const drk_params_grad_t *g_act,
                                   const drk_params_grad_t *g_raw, void *stream);

/* Adam hyper-parameters of one step.  lr[] has one rate per array in the
 * order mu, quat, scale, theta, eta, tau, opacity, color (index with the
 * DRK_ARR_* constants); step is the 1-based step t of the bias corrections
 * 1 - beta1^t and 1 - beta2^t. */
enum { DRK_ARR_MU = 0, DRK_ARR_QUAT, DRK_ARR_SCALE, DRK_ARR_THETA, DRK_ARR_ETA, DRK_ARR_TAU,
       DRK_ARR_OPACITY, DRK_ARR_COLOR, DRK_ARR_COUNT };
typedef struct {
    float lr[DRK_ARR_COUNT];
    float beta1, beta2, eps;  /* 0.9, 0.999, 1e-15 in 3D-GS */
    int64_t step;
} drk_adam_t;

/* One fused training update in a single launch: raw gradients from g_act
 * (chain rule through the activations), the Adam update of every raw array
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   x -= lr / (1 - b1^t) * m / (sqrt(v) / sqrt(1 - b2^t) + eps),
 * and the activation of the updated raw parameters into act (as
 * drk_activate).  m and v are the moment arrays (shapes of raw, zero
 * before step 1), updated in place; raw is updated in place.  Returns
 * DRK_ERR_INVALID_ARG for bad shapes, NULL arrays, step < 1 or a beta
 * outside [0, 1). */
drk_status_t drk_adam_step(const drk_raw_params_t *raw, const drk_params_grad_t *g_act, const drk_params_grad_t *m,
                           const drk_params_grad_t *v, const drk_adam_t *hp, const drk_params_grad_t *act,
                           void *stream);

/* Learning rate at `step` decayed log-linearly from lr_init to lr_final
 * over max_steps (constant lr_final afterwards): the supplement decays the
 * DRK-specific rate 5e-3 to 1e-2 of it at 35K steps.  Host function. */
double drk_lr_exponential(int64_t step, double lr_init, double lr_final, int64_t max_steps);

/* ------------------------------------------------------------------------
 * Mesh to DRK (Sec. 5.4 "Converting Mesh to DRK", supplementary section of
 * the same name): every convex polygon face becomes one DRK, without any
 * optimisation.
 *
 *   mu      mean of the face's vertices;
 *   frame   R_z = unit normal by Newell's method (sum over the edges of
 *           (v_j - mu) x (v_{j+1} - mu)), so the vertices run
 *           counter-clockwise about R_z; R_x from mu towards the first vertex
 *           projected into the plane; R_y = R_z x R_x; quat of [R_x R_y R_z]
 *           with w >= 0;
 *   bases   endpoints at the vertices projected into the plane, in face
 *           order; a face of m < K vertices gets K - m extra endpoints on its
 *           edges, edge j (vertex j to j+1) receiving (K-m)/m + (j < (K-m) %
 *           m) of them, equally spaced; theta_0 = 0, theta_k the polar angle
 *           of endpoint k in [0, 2 pi); s_k = |endpoint k| / sqrt(-2 ln g_e);
 *   shape   eta = 1 (L1 norm alone, Eq. 7-8): the contours of the kernel
 *           are scaled copies of the polygon and the polygon is the contour
 *           g = g_e (edge_density); g_e = 1/2 puts the edges where Psi = 1/2
 *           for any tau (Eq. 9), g_e = exp(-1/2) puts the endpoints exactly on
 *           the vertices;
 *   colour  face colour x (ambient + diffuse |R_z . light|), plain RGB.
 * A face is rejected (status 1: index out of range, padding inside the row,
 * fewer than 3 or more than K vertices, zero area; status 2: the endpoint
 * angles do not increase strictly with every cyclic gap below pi - 1e-3)
 * and its DRK gets opacity 0 (it renders nothing). */
typedef struct {
    int32_t K;            /* bases per DRK, 3 .. 16, at least the largest face */
    float edge_density;   /* g_e in (0, 1); default 0.5 */
    float tau;            /* sharpness in (-1, 1); default 0.95 */
    float opacity;        /* in (0, 1]; default 1 */
    float light[3];       /* direction of the light (world), any length > 0 */
    float ambient, diffuse;
} drk_mesh_options_t;

/* Fills *opt with K = 4, edge_density 0.5, tau 0.95, opacity 1, light
 * (0.3, -0.5, -0.8), ambient 0.35, diffuse 0.65. */
void drk_mesh_options_default(drk_mesh_options_t *opt);

/* verts: n_verts x 3; faces: n_faces x face_size vertex indices (int32),
 * -1 padding at the end of a row; face_color: n_faces x 3 (may be NULL:
 * white); out: the DRK arrays of n_faces primitives (mu n x 3, quat n x 4,
 * scale n x K, theta n x K, eta, tau, opacity n, color n x 3 with
 * sh_degree -1); face_status: n_faces int32 (may be NULL).  All device
 * pointers.  Returns DRK_ERR_INVALID_ARG for bad sizes or options. */
drk_status_t drk_mesh_to_drk(const float *verts, int64_t n_verts, const int32_t *faces, int64_t n_faces,
                             int32_t face_size, const float *face_color, const drk_mesh_options_t *opt,
                             const drk_params_grad_t *out, int32_t *face_status, void *stream);

/* Message for the last failure on the calling thread ("" if none). */
const char *drk_last_error(void);

/* Library version string. */
const char *drk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DRK_H */
