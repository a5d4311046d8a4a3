/*
 * of.h -- C ABI of libof.so: dense pyramidal Lucas-Kanade optical flow on one GPU.
 *
 * The method is the one of Gautier & Aider, "Real-time planar flow velocity
 * measurements using an optical flow algorithm implemented on GPU"
 * (arXiv:1306.2461), Sect. 2.4: two camera images of a region of interest, a
 * pyramid whose images shrink by 4 in area per level, an iterative Gauss-Newton
 * minimisation of a windowed sum of squared differences (window radius r) on each
 * level starting from zero displacement at the top, each level's result
 * propagated as the starting estimate of the next finer level; one displacement
 * vector per pixel.
 *
 * Conventions shared by every call:
 *  - Images are row-major, pitch = W elements, 8-bit (uint8) or up to 16-bit
 *    (uint16) camera counts. Displacements are FP32 pixels, returned as two planes
 *    u (columns, positive to the right) and v (rows, positive downwards), pitch W,
 *    such that I1(x) ~ I2(x + u(x)).
 *  - Pointers named "device" must be device (or managed) memory of the current
 *    CUDA device; the library never copies them. The caller owns them and keeps
 *    them valid until the work queued on `stream` has completed.
 *  - Calls are asynchronous with respect to the host unless stated otherwise.
 *    Arguments are validated on the host before anything is queued; a call that
 *    returns an error has queued nothing.
 *  - Every call returns an of_status code (0 = OF_OK) and never throws.
 *  - A handle is not thread-safe: one handle per camera stream, used by one host
 *    thread at a time. Different handles may be used concurrently.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).
 */
#ifndef OF_H_
#define OF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *of_stream_t; /* identical to cudaStream_t */

typedef enum of_status {
    OF_OK = 0,
    OF_EINVAL = -1,   /* an argument or the plan is out of range */
    OF_ENOMEM = -2,   /* device allocation failed, or the HBM budget is exceeded */
    OF_ECUDA = -3,    /* a CUDA runtime call failed (launch, copy, graph) */
    OF_EDEVICE = -4,  /* a kernel reported a failed internal check */
    OF_ETIMEOUT = -5, /* a bounded device-side wait ran out */
    OF_ESTATE = -6,   /* the call needs state the handle does not have */
    OF_EBUSY = -7     /* a server queue or slot pool is full */
} of_status;

typedef enum of_in_format { OF_U8 = 0, OF_U16 = 1 } of_in_format;

/* Precision in which the pyramids are stored in HBM. Window sums and the 2x2
 * solve always accumulate in FP32 (FP64 for ill-conditioned pixels). */
typedef enum of_storage { OF_F32 = 0, OF_F16 = 1, OF_BF16 = 2 } of_storage;

/* plan.flags */
#define OF_FLAG_NO_GRAPH 0x1u /* launch kernels one by one instead of replaying a CUDA graph */
#define OF_FLAG_ZNSSD 0x4u    /* normalise both images before the pyramid (Sect. 2.4, Eq. 2): local
                                 mean and standard deviation over a radius of 5 pixels, clipped
                                 to the image; level 0 is then stored at the storage precision */
#define OF_FLAG_GATHER 0x2u   /* gather each iteration tile's taps and estimates from global memory
                                 instead of staging the tile's I2 window and estimate in shared
                                 memory with TMA tensor copies (the default); same results */
#define OF_FLAG_I1GRAD 0x8u   /* the FOLKI-lineage variant (Sect. 2.4): linearise with the gradient
                                 of the FIRST image at integer pixels (central difference, clamped)
                                 instead of the second image's gradient at the displaced position.
                                 The window matrix then depends on I1 only and is summed once per
                                 level; each iteration sums two channels. Batched calls and the
                                 serving loop run it as phase launches (the tuning's phased,
                                 stage_i2 and blocks_per_sm are ignored for it). The workspace
                                 grows by one float4 per level-0 pixel. */

/*
 * Problem statement (Sect. 2.4): image size of the region of interest, number of
 * pyramid levels n_lev and iterations per level n_iter (the two parameters that
 * set the speed, Eq. 1 and Table 1), window radius r.
 */
typedef struct of_plan {
    int32_t H, W;       /* image size in pixels, 1..32768 each, H*W <= 2^28 */
    int32_t levels;     /* pyramid levels including full resolution, 1..16 */
    int32_t radius;     /* window radius r: box of (2r+1)^2 pixels, 1..16 */
    int32_t iterations; /* Gauss-Newton iterations per level, 1..1000 */
    int32_t in_format;  /* OF_U8 or OF_U16 */
    int32_t in_bits;    /* significant bits of the input, 1..8 (U8) or 1..16 (U16) */
    int32_t storage;    /* OF_F32, OF_F16 or OF_BF16 */
    float fp64_cond;    /* a pixel whose window matrix has tr^2/det above this value is
                           solved in FP64; 0 = never (FP32 only). Default 1e3. */
    uint32_t flags;     /* OF_FLAG_* */
} of_plan;

typedef struct of_ctx *of_handle;

/* Fill *p with defaults for an H x W problem: levels 3, radius 4, iterations 5,
 * OF_U8 with 8 bits, OF_F32 storage, fp64_cond 1e3, no flags. Host only. */
void of_plan_init(of_plan *p, int32_t H, int32_t W);

/* Check every field of *p against the ranges above. Host only.
 * Returns OF_OK or OF_EINVAL (p == NULL included). */
int of_plan_validate(const of_plan *p);

/* Eq. 1 (Sect. 2.4): the pyramid should satisfy max_disp / 2^(levels-1) < 3 px.
 * Sets *ok to 1 if it does for the given maximum displacement (pixels, at full
 * resolution), 0 if not. Advisory only: of_create accepts either. Host only. */
int of_plan_check(const of_plan *p, float max_disp_px, int *ok);

/* Size of pyramid level `level` (0 = full resolution): each level has
 * ceil(n/2) pixels along an axis of n pixels at the level below (Sect. 2.4, area
 * reduced by 4 per level). Host only. OF_EINVAL if level is outside [0, levels). */
int of_level_size(const of_plan *p, int32_t level, int32_t *Hl, int32_t *Wl);

/* Bytes of device memory of_create allocates for this plan (both pyramids, two
 * flow buffers, a status word), for admission against an HBM budget. Host only. */
int of_workspace_bytes(const of_plan *p, size_t *bytes);

/* Validate the plan and allocate the workspace on the current CUDA device.
 * On success *out receives the handle; on failure *out is set to NULL and nothing
 * is left allocated. OF_EINVAL (bad plan or out == NULL), OF_ENOMEM, OF_ECUDA. */
int of_create(const of_plan *p, of_handle *out);

/*
 * Compute the displacement field from I1 to I2 (Sect. 2.4).
 *  I1, I2: device, H*W elements of the plan's input format (uint8 or uint16).
 *          I1 == NULL reuses the pyramid of the previous call's I2 on this handle
 *          as the first image: with a time-resolved camera, each field then needs
 *          only one new image to be processed (computing scheme 1 of Sect. 2.4).
 *          OF_ESTATE if the handle has no previous I2.
 *  u, v:   device, H*W floats each, written by the last kernel of the call.
 *  stream: the work is queued on it; buffers must outlive the stream's progress.
 * Returns OF_EINVAL (NULL handle, I2, u or v), OF_ESTATE, OF_ECUDA. Device-side
 * failures are reported by of_sync_status.
 */
int of_compute(of_handle h, const void *I1, const void *I2, float *u, float *v, of_stream_t stream);

/*
 * Compute n independent fields together (fields are independent, Sect. 3.3, so they
 * can share the GPU): one CUDA graph replay per call of either one launch per phase
 * (pyramid pass, one iteration of one level) over the tiles of up to 64 pairs, in one
 * or several concurrent sequences over parts of the batch, or one persistent
 * cooperative launch with bounded grid barriers between phases, as the tuning table
 * says (of_autotune_batch below). hs[i] are handles whose plans have
 * equal levels, radius, iterations, in_format, in_bits, storage and method flags
 * (sizes may differ); a handle may appear at most once. I1s[i] may be NULL (reuse, as
 * in of_compute). All pointers as in of_compute. n == 0 is a no-op. OF_EINVAL on
 * mismatched plans, repeated handles or NULL pointers; OF_ESTATE as in of_compute.
 * The results are those of n separate of_compute calls (bit for bit with the grouped
 * window sums and the default tile height, in any number of sequences).
 */
int of_compute_batch(int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s,
                     float *const *us, float *const *vs, of_stream_t stream);

/*
 * of_compute_batch from and to HOST buffers, with the copies overlapped with the
 * computation. The pairs are taken in chunks of `chunk` pairs (0: about 8 Mpx of level 0
 * per chunk, i.e. eight 1024^2 pairs, at most 24 such chunks, with the first and the last
 * a quarter and the second and the second-to-last half of that when such a chunk holds at
 * least 4 pairs and the batch at least 2.5 chunks' worth, so that the pipeline fills and
 * drains faster): chunk
 * k's frames are uploaded (hI1s/hI2s -> dI1s/dI2s) on an internal stream, its
 * batched launch runs after that upload (even chunks on `stream`, odd chunks on a
 * compute stream the library keeps for the calling thread and device until the thread
 * exits, so that neighbouring chunks' launches overlap), and its fields are downloaded
 * (dus/dvs -> hus/hvs) on a second internal stream after the launch, so the uploads
 * and downloads of neighbouring chunks overlap the launches. The copy streams are kept
 * per thread and device as well. Calls from different threads are independent. hI1s[i] == NULL reuses
 * the previous pyramid (dI1s[i] is then ignored). Host buffers should be pinned (page-
 * locked) for the copies to be asynchronous; device buffers are caller-owned, sized
 * as in of_compute. The call is complete (fields in hus/hvs) when `stream` reaches it.
 * Errors as of_compute_batch; an error after the first chunk was queued leaves the
 * earlier chunks queued, and `stream` waits for all of them (uploads, launches and
 * downloads) before the call returns, so synchronising `stream` after an error makes
 * every buffer of the call free for reuse.
 */
int of_compute_batch_host(int32_t n, const of_handle *hs, const void *const *hI1s, const void *const *hI2s,
                          float *const *hus, float *const *hvs, void *const *dI1s, void *const *dI2s,
                          float *const *dus, float *const *dvs, of_stream_t stream, int32_t chunk);

/*
 * Autotuning of the batched launch (of_compute_batch and the serving loop). Every
 * batch shape has the same results to within the stated tolerances whichever tuning
 * runs it; with grouped sums (generic_sums == 0) they are the results of of_compute bit
 * for bit (with the default tile height and fusion 1, whatever the strip). Without a table
 * entry a batch runs {generic_sums 0, stage_i2 1, blocks_per_sm 0, phased 1, prefetch 0,
 * tile_h 24, branches 1, fusion 1, strip 4}.
 * A tuning:
 *   generic_sums   1: per-output window sums of the run-time-radius kernel;
 *                  0: grouped sums of the kernel specialised for the radius
 *   stage_i2       1: stage each tile's I2 window and estimate in shared memory with TMA tensor
 *                  copies (specialised kernel, phase launches; ignored under OF_FLAG_GATHER);
 *                  0: gather them from global memory
 *   blocks_per_sm  resident blocks per SM of the persistent launch; 0 = as many as fit
 *   phased         1: one ordinary launch per phase (pyramid pass, iteration) over all
 *                  pairs' tiles, the pairs' arguments passed as kernel parameters, in
 *                  place of the one persistent launch with grid barriers (then
 *                  blocks_per_sm must be 0)
 *   prefetch       phase launches: each iteration block warms L2 with the rows the block
 *                  prefetch x (number of SMs) tiles later will read first (0: off, <= 16)
 *   tile_h         phase launches with grouped sums: height of the 64-wide iteration tile,
 *                  24 (the default; 0 means the default) or 32. Tiles other than the
 *                  default move each tile's reference flow, so their fields differ from
 *                  of_compute's by rounding (within the stated tolerances)
 *   branches       phase launches: the pairs split into this many groups of about equal
 *                  pixel counts whose launch sequences run concurrently (forked from and
 *                  joined back into the caller's stream, inside the captured graph), so
 *                  that one group's launches fill the last waves of another's; 1 to 4
 *                  (0 means 1). Each pair's arithmetic is unchanged.
 *   fusion         phase launches with grouped sums at the default tile height: 2 runs two
 *                  consecutive iterations of a level (after its first) in one launch, each
 *                  tile computing the first of them on its whole window region in shared
 *                  memory (iteration fusion depth 2; fields equal to within the FP32
 *                  tolerance, the reference flows of the region's pixels being the tile's);
 *                  0 or 1: one iteration per launch
 *   strip          phase launches with grouped sums: tiles per block along a column of
 *                  tiles, 1, 2 or 4 (0 means 4), halved for a launch while it would have
 *                  fewer than 8 blocks per SM. The tiles of a group of 4 tile rows share one
 *                  reference flow, so a block's tiles after the first take over the window
 *                  sums of the rows they share with the tile above; the fields are the
 *                  same bit for bit for every strip (of_compute runs strip 1)
 *   ms             measured milliseconds per batch (of_autotune_batch output only)
 * The process-wide table is keyed by the method (in_format, storage, radius, levels,
 * iterations, OF_FLAG_ZNSSD, OF_FLAG_I1GRAD) and a size class, round(log2(mean level-0 pixels
 * per pair)).
 */
typedef struct of_tuning {
    int32_t generic_sums;
    int32_t stage_i2;
    int32_t blocks_per_sm;
    int32_t phased;
    int32_t prefetch;
    int32_t tile_h;
    int32_t branches;
    int32_t fusion;
    int32_t strip;
    float ms;
} of_tuning;

/* Time every candidate tuning on this batch (one untimed launch, then `reps` timed
 * launches each, CUDA events on `stream`, synchronised) and record the fastest in the
 * table for the batch's method and size class. Arguments as of_compute_batch, except
 * that every I1s[i] must be non-NULL (repeated launches must not move the reused
 * pyramid) and n >= 1. The outputs hold the last candidate's fields. results (up to
 * max_results entries, may be NULL when max_results == 0) receives each candidate's
 * time; *n_results (may be NULL) their number; *best (may be NULL) the choice.
 * Blocks the calling thread. OF_EINVAL, OF_ECUDA, OF_ETIMEOUT (a device wait ran out;
 * nothing is recorded), or the errors of of_compute_batch. */
int of_autotune_batch(int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s,
                      float *const *us, float *const *vs, of_stream_t stream, int32_t reps, of_tuning *best,
                      of_tuning *results, int32_t max_results, int32_t *n_results);
/* Size class of a batch (its table key). OF_EINVAL for n < 1 or NULL handles. */
int of_batch_size_class(int32_t n, const of_handle *hs, int32_t *size_class);
/* Read or write one table entry (the method is a plan whose H and W are ignored).
 * of_tuning_get: OF_ESTATE when there is no entry. of_tuning_set: OF_EINVAL for an
 * invalid tuning (generic_sums and stage_i2 together, values out of range). Host only. */
int of_tuning_get(const of_plan *method, int32_t size_class, of_tuning *t);
int of_tuning_set(const of_plan *method, int32_t size_class, const of_tuning *t);
int of_tuning_clear(void);

/*
 * of_compute without any device allocation. The paper has no counterpart: this is for
 * callers that cannot call cudaMalloc once running, such as a real-time acquisition
 * loop (cudaMalloc/cudaFree can synchronise the device and stall the camera pipeline)
 * or a host application that owns all device memory through its own allocator.
 * The workspace of of_create lives here in one static device array of
 * OF_NOALLOC_MAX_BYTES (32 MiB: enough for one 1024 x 1024 pair at any storage without
 * OF_FLAG_I1GRAD, whose window matrices add 16 bytes per pixel), reserved on every GPU
 * where the library's code is loaded and held until exit.
 *  p:      the plan, as for of_create; plans whose of_workspace_bytes exceed
 *          OF_NOALLOC_MAX_BYTES are rejected with OF_ENOMEM before anything is queued.
 *  I1, I2, u, v, stream: as for of_compute, except that I1 must not be NULL (there is
 *          no handle, so no previous pyramid to reuse): OF_EINVAL.
 * Nothing is allocated, on the device or by a library routine: kernels are launched
 * directly on `stream` (no graph), and the status word is cleared with a memset. The
 * iteration tiles always run gathered (as with OF_FLAG_GATHER, same fields as
 * of_compute): that form has no bounded device-side wait, so no device-side error can
 * arise that this call, having no handle to report it on, would drop.
 * The first call on a device, with that device current, looks up the array's device
 * address and sets kernel attributes; make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents: calls whose
 * work overlaps on the GPU (different streams, or other host threads) race and give
 * wrong results; serialise them on one stream.
 * Returns OF_OK, OF_EINVAL, OF_ENOMEM or OF_ECUDA.
 */
#define OF_NOALLOC_MAX_BYTES (32u * 1024u * 1024u)
int of_compute_noalloc(const of_plan *p, const void *I1, const void *I2, float *u, float *v, of_stream_t stream);

/*
 * Recirculation-bubble surface, Eq. 3 (Sect. 3.2): S_bubble = (number of vectors whose
 * streamwise component u is <= T_v) / (number of vectors). The paper's fraction is
 * garbled (it divides the count by a sum of velocities); this is the reading of its
 * text, "percentage of velocities below a given threshold".
 *  u:      device, H*W floats (a field from of_compute, or any streamwise component).
 *  count:  device, one unsigned 64-bit integer, overwritten with the count (exact);
 *          S_bubble = count / (H*W).
 * The comparison is in FP32 and inclusive. OF_EINVAL for NULL pointers, empty sizes or
 * a NaN threshold.
 */
int of_sbubble_count(const float *u, int32_t H, int32_t W, float Tv, unsigned long long *count, of_stream_t stream);

/* Minimum and maximum of a device field of H*W floats into minmax[0], minmax[1]
 * (device, 2 floats), ignoring NaNs (NaN results if every value is NaN). With the
 * time-mean streamwise field this gives Eq. 3's threshold T_v = (min + max) / 2. */
int of_field_minmax(const float *field, int32_t H, int32_t W, float *minmax, of_stream_t stream);

/* Wait for the handle's last queued work, then read and clear its device status
 * word. Returns OF_OK, OF_EDEVICE or OF_ETIMEOUT from the device, or OF_ECUDA. */
int of_sync_status(of_handle h);

/* Release the workspace. Waits for the handle's queued work first. NULL is a no-op. */
int of_destroy(of_handle h);

/* Copy pyramid level `level` of image `which` (0 = the first image of the last
 * compute, 1 = the second) into dst (device, Hl*Wl floats, pitch Wl), converted to
 * FP32. Used to check the pyramid step. OF_ESTATE before the first compute. */
int of_get_level(of_handle h, int32_t which, int32_t level, float *dst, of_stream_t stream);

/* The window-sum step alone (Sect. 2.4, window of radius r): out[c] = sum of ch[c]
 * over the (2r+1)^2 box around each pixel, zero outside the image, for the 5
 * planes c = 0..4. ch, out: device, 5*H*W floats (plane c at offset c*H*W).
 * Same device code and summation order as inside the fused iteration. */
int of_window_sums(const float *ch, int32_t H, int32_t W, int32_t r, float *out, of_stream_t stream);

/* Test hook for bounded device waits: launches one kernel that waits for a device
 * flag which nothing sets, giving up after about timeout_us microseconds. Blocks
 * until it returns and reports OF_ETIMEOUT (the expected outcome) or OF_ECUDA. */
int of_debug_wait_timeout(int32_t timeout_us);

/* ------------------------------------------------------------------------------
 * Serving: camera streams of mixed resolutions on one GPU, continuous batching.
 *
 * Each stream delivers frames in order; every frame after the first yields the field
 * from the previous frame to it. The previous frame's pyramid stays resident on the
 * device and is reused as the first image of the next pair (computing scheme 1 of
 * Sect. 2.4), so each field processes one new image. Streams are admitted against an
 * HBM budget. A worker thread packs the next pending frame of every stream into one
 * batched launch ("tick", tuned as of_compute_batch); frames arriving while ticks run join the next
 * tick as soon as fewer than max_inflight ticks are on the device, their host-to-
 * device copies overlapping the running tick. All calls are thread-safe.
 */
typedef struct of_server *of_server_t;

typedef struct of_server_config {
    int32_t levels, radius, iterations; /* the method, as in of_plan, shared by all streams */
    int32_t in_format, in_bits, storage;
    float fp64_cond;
    uint32_t flags;                     /* OF_FLAG_GATHER (OF_FLAG_NO_GRAPH is ignored) */
    uint64_t hbm_budget_bytes;          /* device memory all open streams may hold together */
    int32_t max_batch;                  /* pairs per tick, 1..4096 */
    int32_t max_inflight;               /* ticks queued on the device at once, 1..8 */
} of_server_config;

/* One finished frame. Times are of_server_now_ns() values (host steady clock). */
typedef struct of_result {
    int32_t stream;      /* stream id */
    int32_t status;      /* OF_OK or the error that affected this frame */
    uint64_t tag;        /* the caller's tag from of_server_submit */
    int64_t arrival_ns;  /* when the frame arrived (given to, or taken by, of_server_submit) */
    int64_t launch_ns;   /* when its tick was queued on the device */
    int64_t done_ns;     /* when the worker saw its tick complete */
    int32_t batch;       /* pairs in that tick */
    int32_t has_field;   /* 0 for a stream's first frame (staged only), 1 when u, v were written */
} of_result;

/* Defaults: 3 levels, r = 4, 5 iterations, 12-bit uint16 input, FP16 storage,
 * fp64_cond 1e3, 8 GiB budget, max_batch 64, max_inflight 2. Host only. */
void of_server_config_init(of_server_config *c);

/* Create a server on the current device (streams, launch slots, worker thread).
 * OF_EINVAL, OF_ENOMEM, OF_ECUDA. */
int of_server_create(const of_server_config *c, of_server_t *out);

/* Admit a stream of H x W frames: allocates its workspace (of_workspace_bytes of its
 * plan) and two frame staging buffers. OF_ENOMEM if that would exceed the budget;
 * *id receives the stream id (>= 0, reused after a close). */
int of_server_open_stream(of_server_t s, int32_t H, int32_t W, int32_t *id);

/* Close a stream whose submitted frames have all been taken into ticks: waits for
 * those ticks, then frees its memory. OF_EBUSY if frames are still queued. */
int of_server_close_stream(of_server_t s, int32_t id);

/*
 * Queue one frame of stream `id`.
 *  frame: host memory (pinned for full copy speed), H*W elements of the input format;
 *         it must stay valid and unchanged until this frame's result is reported.
 *  u, v:  device, H*W floats each, receive the field from the stream's previous
 *         frame to this one; may be NULL for the stream's first frame.
 *  tag:   returned in the result. arrival_ns: the frame's arrival time (0 = now);
 *         latency is measured from it, so late submissions are charged in full.
 * OF_EINVAL, OF_EBUSY (256 frames already queued on this stream), or a sticky error.
 */
int of_server_submit(of_server_t s, int32_t id, const void *frame, float *u, float *v, uint64_t tag,
                     int64_t arrival_ns);

/* Move up to `max` finished results into out[0..*n), waiting up to timeout_us for the
 * first one. Returns OF_OK or the server's sticky error. */
int of_server_poll(of_server_t s, of_result *out, int32_t max, int32_t *n, int32_t timeout_us);

/* Wait until every submitted frame is finished (OF_ETIMEOUT after timeout_ms). */
int of_server_drain(of_server_t s, int32_t timeout_ms);

/* Ticks launched, pairs computed, device bytes held by open streams. */
int of_server_stats(of_server_t s, int64_t *ticks, int64_t *pairs, uint64_t *hbm_used);

/* The clock of of_result times (nanoseconds, monotonic). */
int64_t of_server_now_ns(void);

/* Stop the worker, wait for the device, free everything. NULL is a no-op. */
int of_server_destroy(of_server_t s);

/* Test hook for failure handling: the library's next n device allocations (of_create,
 * of_server_open_stream, of_server_create) fail as if the device were out of memory.
 * n = 0 clears it. Returns the previous count. Host only. */
int of_debug_fail_allocs(int32_t n);

/* Static text for a status code. */
const char *of_status_string(int status);

/* Library version as 10000*major + 100*minor + patch. */
int of_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OF_H_ */
