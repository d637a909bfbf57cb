/*
 * veckm: GB300 (sm_103a) local event encoder and normal-flow head.
 *
 * The operation is the pooled local-event encoding of "A Real-Time
 * Event-Based Normal Flow Estimator" (arXiv 2504.19417), Algorithm 1 and
 * Eq. 13-17 of Section 2.2.2, followed by the two-layer perceptron of
 * Eq. 6.  For every requested event k of a slice {(t_j, x_j, y_j)}:
 *
 *   emb_k[d] = (1/n_k) sum_{j : |x_j-x_k|<=dx, |y_j-y_k|<=dy}
 *              exp(i[(t_j-t_k)/dt T_d + (x_j-x_k)/dx X_d + (y_j-y_k)/dy Y_d])
 *
 * (Eq. emb of Section 2.2.1; n_k is the number of slice events in the
 * window, k included; there is no temporal window inside the slice, Eq. 1),
 * and   flow_k = W2 ReLU(W1 [Re emb_k ; Im emb_k] + b1) + b2.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers; pointers named h_* are host
 *     pointers.  The caller owns every buffer it passes; the context owns its
 *     tables, weights and per-pixel accumulators and frees them in
 *     veckm_destroy.
 *   - Work is enqueued on the caller's CUDA stream (a cudaStream_t passed as
 *     void*; NULL means the legacy default stream) and the call returns after
 *     enqueueing, except where a function says it synchronises.
 *   - Host-detectable errors return immediately with a negative status and a
 *     message retrievable through veckm_last_error.  Errors that only the GPU
 *     can see (an event outside the sensor or outside [t_ref, t_ref+t_span],
 *     an index in K outside [0, n)) set a device error word; the affected
 *     event is skipped (its outputs are written as zeros) and the error is
 *     reported as VECKM_ERANGE by veckm_sync_status or by the next
 *     synchronising call.  No kernel traps.
 *   - A context is not thread safe: use one per host thread, or lock.
 *     Calls on one context must be ordered on one stream, since they share the
 *     context's accumulators.
 */
#ifndef VECKM_H
#define VECKM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VECKM_API_VERSION 1

typedef struct veckm_ctx veckm_ctx;

/* Largest n (events of a slice) and nK (requested flows) of one call; larger
 * sizes return VECKM_EINVAL.  Events are indexed with 32-bit integers on the
 * device. */
#define VECKM_MAX_EVENTS ((int64_t)1 << 30)

typedef enum {
    VECKM_OK = 0,
    VECKM_EINVAL = -1,      /* bad argument or configuration */
    VECKM_ENOMEM = -2,      /* a device or host allocation failed */
    VECKM_ECUDA = -3,       /* a CUDA runtime call failed */
    VECKM_ERANGE = -4,      /* an event or index was out of range (device-detected) */
    VECKM_ETIMEOUT = -5,    /* a bounded device wait ran out */
    VECKM_EBUSY = -6,       /* no free slot or memory for the request */
    VECKM_EUNSUPPORTED = -7 /* configuration not supported by this build */
} veckm_status;

/* flags of veckm_config */
#define VECKM_MLP_FP32 0u        /* perceptron in FP32 on the CUDA cores (the plain form) */
#define VECKM_MLP_BF16 (1u << 0) /* first layer on tcgen05 tensor cores, BF16 x BF16 -> FP32 */
#define VECKM_MLP_FP16 (1u << 1) /* first layer on tcgen05 tensor cores, FP16 x FP16 -> FP32 */
/* Store the pooled grid that veckm_predict gathers from as FP16, divided by
 * the window count (half the bytes; the conjugate-phase product is formed in
 * packed half2 arithmetic).  Needs VECKM_MLP_BF16 or VECKM_MLP_FP16;
 * veckm_encode keeps FP32 throughout. */
#define VECKM_ACC_FP16 (1u << 2)

typedef struct {
    int32_t width, height; /* sensor W x H in pixels (Algorithm 1 inputs), 1..32767 */
    int32_t D;             /* encoding dimension (complex), 64, 128, 192 or 256 */
    int32_t dx, dy;        /* pixel radii of the window (Eq. 1), 0..64 */
    int32_t hidden;        /* perceptron hidden width; 128 */
    int64_t dt_us;         /* time radius delta t in microseconds (Eq. 1 slice of 2 dt) */
    int64_t t_span_us;     /* largest accepted t - t_ref; 0 means 2*dt_us */
    double sigma2;         /* variance of the frequencies (Algorithm 1: 25); 0 means 25 */
    uint64_t freq_seed;    /* T, X, Y drawn with seeds s, s+1, s+2 when h_T etc. are NULL */
    const double *h_T, *h_X, *h_Y; /* optional: D frequencies each (copied in create) */
    const float *h_W1;     /* [hidden][2D] row-major, input packed as [Re | Im] */
    const float *h_b1;     /* [hidden] */
    const float *h_W2;     /* [2][hidden] row-major */
    const float *h_b2;     /* [2] */
    uint32_t flags;        /* VECKM_MLP_* | VECKM_ACC_FP16 */
} veckm_config;

/* Create a context: validates cfg, draws or copies the frequencies T, X, Y
 * (Algorithm 1; drawn as SplitMix64 + Box-Muller normals scaled by
 * sqrt(sigma2)), builds the per-axis phase tables in FP64 and stores them in
 * FP32, uploads the weights and allocates the per-pixel accumulators
 * (2 x W x H x D complex FP32 plus counts) on the current device.
 * On success *out owns all of it.  Synchronous. */
veckm_status veckm_create(veckm_ctx **out, const veckm_config *cfg);

/* Free everything the context owns.  NULL-safe.  Synchronises the device. */
void veckm_destroy(veckm_ctx *ctx);

/* Encode: the pooled local event encoding of Algorithm 1 (Eq. 16-17) for the
 * events selected by d_K.
 *   d_x, d_y  int16 pixel coordinates of the n slice events (device)
 *   d_t       uint32 timestamps in microseconds (device); t_ref_us is the slice
 *             start, every t must lie in [t_ref_us, t_ref_us + t_span_us]
 *   d_K       int64 indices into [0, n) of the events to encode, or NULL for all
 *             (then nK must equal n)
 *   d_emb     float [nK][2D] output (device): row i holds Re(emb) for d = 0..D-1
 *             then Im(emb) for d = 0..D-1 of event K[i].
 * nK == 0 is valid (with or without d_K) and does nothing. */
veckm_status veckm_encode(veckm_ctx *ctx, const int16_t *d_x, const int16_t *d_y,
                          const uint32_t *d_t, int64_t n, uint32_t t_ref_us,
                          const int64_t *d_K, int64_t nK, float *d_emb, void *stream);

/* Encode without allocating: the same result as veckm_encode, for callers
 * that may not allocate device memory during a call.  A loop with a real-time
 * budget cannot wait for an allocation and the synchronisation before it; a
 * process that reserves all of a device's memory up front for its own
 * allocator finds cudaMalloc failing.  veckm_encode may grow its per-event
 * buffers with cudaMalloc; this call takes them from a fixed array in device
 * memory that the library declares statically and never calls cudaMalloc,
 * cudaFree or any allocating routine.  The paper has no counterpart; it is a
 * deployment variant.
 *   - At most 1048576 events per call (n); larger n returns VECKM_EINVAL.
 *   - The array (12 MiB) exists on every GPU that loads the library until the
 *     process exits.  The first call on a device looks up its address there
 *     (cudaGetSymbolAddress) and keeps it for that device's CUDA context; make
 *     that first call before any stream capture.  After a device reset the
 *     next call looks the address up again.
 *   - All calls on a device share the array and the context's accumulators:
 *     calls that may overlap on the GPU race and must be serialised.
 *   - It always uses the histogram-and-placement sort and clears the
 *     per-pixel sums in full, so it runs slower than veckm_encode.
 * Arguments, layout and errors are those of veckm_encode. */
veckm_status veckm_encode_noalloc(veckm_ctx *ctx, const int16_t *d_x, const int16_t *d_y,
                                  const uint32_t *d_t, int64_t n, uint32_t t_ref_us,
                                  const int64_t *d_K, int64_t nK, float *d_emb, void *stream);

/* Predict: the encoding above fused with the two-layer perceptron (Eq. 6),
 * in the precision chosen by cfg.flags.  d_flow is float [nK][2] (device):
 * the generalised normal flow (n_x, n_y) of event K[i] in row i. */
veckm_status veckm_predict(veckm_ctx *ctx, const int16_t *d_x, const int16_t *d_y,
                           const uint32_t *d_t, int64_t n, uint32_t t_ref_us,
                           const int64_t *d_K, int64_t nK, float *d_flow, void *stream);

/* Predict from host buffers: copies the events (and K) host-to-device into
 * context-owned staging buffers, runs veckm_predict, copies the flows back to
 * h_flow and synchronises the stream.  Pinned host memory makes the copies
 * asynchronous DMA; pageable memory works but is slower.  Returns
 * VECKM_ERANGE if the device flagged an out-of-range event or index. */
veckm_status veckm_predict_host(veckm_ctx *ctx, const int16_t *h_x, const int16_t *h_y,
                                const uint32_t *h_t, int64_t n, uint32_t t_ref_us,
                                const int64_t *h_K, int64_t nK, float *h_flow, void *stream);

/* Pipelined form of veckm_predict_host (Eq. 6 on host buffers).  Enqueues
 * the call and returns at once with *ticket set; the call's result is ready
 * after veckm_host_wait(ctx, *ticket).  Each context keeps two staging slots
 * and internal upload, compute and download streams: the uploads of one call
 * run while the previous call computes, and its flows come back while the
 * next call computes, so at most two calls are in flight (a third call first
 * waits for the call two back).  Calls run on the device in the order they were made.  h_x, h_y,
 * h_t, h_K must stay unchanged and h_flow untouched until the wait; they
 * should be pinned (cudaHostAlloc), since pageable buffers make the copies
 * block the host.  Until the last ticket is waited for, the context must not
 * be used on another stream.  The device error word is read and cleared
 * after each call, so a ticket's status covers exactly its own call.
 * Argument errors are returned at once (no ticket is issued). */
veckm_status veckm_predict_host_async(veckm_ctx *ctx, const int16_t *h_x, const int16_t *h_y,
                                      const uint32_t *h_t, int64_t n, uint32_t t_ref_us,
                                      const int64_t *h_K, int64_t nK, float *h_flow,
                                      int64_t *ticket);

/* Block until the call with this ticket has finished and its flows are in
 * h_flow; returns its status (VECKM_ERANGE for an out-of-range event or
 * index, VECKM_ETIMEOUT, a CUDA failure).  A ticket may be waited for more
 * than once; the statuses of the last 64 tickets are kept (older ones:
 * VECKM_EINVAL). */
veckm_status veckm_host_wait(veckm_ctx *ctx, int64_t ticket);

/* Switch the perceptron precision and pooled-grid storage of an existing
 * context (VECKM_MLP_* | VECKM_ACC_FP16); tables and accumulators are kept.
 * Synchronous. */
veckm_status veckm_set_mlp_mode(veckm_ctx *ctx, uint32_t flags);

/* Synchronise the stream, then read and clear the device error word:
 * VECKM_ERANGE if any event or index since the last check was out of range. */
veckm_status veckm_sync_status(veckm_ctx *ctx, void *stream);

/* Thread-local message describing the last failure on this thread ("" if none). */
const char *veckm_last_error(void);

/* Copy the context's frequencies T, X, Y (D doubles each) to host arrays. */
veckm_status veckm_get_frequencies(const veckm_ctx *ctx, double *h_T, double *h_X, double *h_Y);

/* Per-stage timing, measured with CUDA events recorded on the launching
 * stream around each stage.  Stages: 0 sort of the events by pixel (and, where
 * the pixel sums need a cleared grid, the wait for its clear on a side stream),
 * 1 per-pixel accumulation (the first loop of Algorithm 1), 2 pooling row pass,
 * 3 window counts (Eq. 17; they run on a side stream, so this is the residual
 * wait for them), 4 pooling column pass (the window sums of Eq. 16), 5 gather
 * + normalise, fused with the perceptron in veckm_predict.
 * veckm_stage_times synchronises, writes the elapsed milliseconds summed over
 * every timed call since the last read into ms[0..nstage-1] and the number of
 * timed calls into calls[0..nstage-1] (may be NULL), then resets. */
veckm_status veckm_set_timing(veckm_ctx *ctx, int enable);
veckm_status veckm_stage_times(veckm_ctx *ctx, double *ms, int64_t *calls, int nstage);

/* Number of kernel launches the last encode/predict call made. */
int veckm_last_launch_count(const veckm_ctx *ctx);

/* Dense pooling or the direct window form.  Algorithm 1 computes each
 * requested flow by looping over its window (its second loop, cost C
 * per flow in Eq. runtime of Section 2.2.2).  The dense form pools every
 * pixel once with separable box sums (cost per pixel, then little per flow);
 * the direct form keeps the window loop, visiting only occupied window pixels
 * (one warp per requested event), and skips the pooling passes.
 * VECKM_PATH_AUTO (default) picks per call the smaller of
 *   dense:  k_pixel * W*H + k_flow_dense * nK
 *   direct: k_flow_window * (2dx+1)(2dy+1) * nK,
 * with coefficients measured on GB300 (settable).  The direct form's
 * perceptron is the FP32 one whatever the flags; with D > 128 predictions
 * stay dense.  Results agree to FP32 rounding. */
#define VECKM_PATH_AUTO 0
#define VECKM_PATH_DENSE 1
#define VECKM_PATH_DIRECT 2
veckm_status veckm_set_path(veckm_ctx *ctx, int32_t path);
/* The path the last encode/predict call took (VECKM_PATH_DENSE or _DIRECT). */
int veckm_last_path(const veckm_ctx *ctx);
/* The model's coefficients in nanoseconds (all positive; flow_dense may be 0). */
veckm_status veckm_set_path_model(veckm_ctx *ctx, double pixel_ns, double flow_dense_ns,
                                  double flow_window_ns);

/* Kernel density read back from encodings (Lemma 1 of Section 2.2.1), the
 * "general-purpose encoder" use of an encoding.  For query i, with e the row
 * d_row[i] of d_emb (float [nrows][2D], as veckm_encode writes it) and the
 * integer offset q = (d_qt[i] microseconds, d_qx[i], d_qy[i] pixels) from
 * that row's event:
 *   d_out[i] = (1/D) sum_d [Re e_d cos a_d + Im e_d sin a_d],
 *   a_d = qt T_d / dt + qx X_d / dx + qy Y_d / dy,
 * i.e. Re((1/D) sum_d e_d conj(exp(i a_d))), which approaches the Gaussian
 * kernel density of the event's window at q as D grows.  Every term of a_d is
 * reduced modulo one turn exactly (64-bit fixed point), whatever the offset.
 * A row outside [0, nrows) gives 0 and sets the device error word
 * (VECKM_ERANGE at the next status check).  Device buffers; nq may be 0. */
veckm_status veckm_kde_query(veckm_ctx *ctx, const float *d_emb, int64_t nrows,
                             const int64_t *d_row, const int32_t *d_qt, const int32_t *d_qx,
                             const int32_t *d_qy, int64_t nq, float *d_out, void *stream);

/* ------------------------------------------------------------------ batches
 * Several slices, possibly from sensors of different sizes, encoded in one
 * pass.  The library lays the sensors out on a canvas, one large virtual
 * sensor of at most the context's width x height, each sensor at an offset
 * (ox, oy) and at least dx empty columns and dy empty rows away from any
 * other.  The encoding of Eq. emb depends on pixel coordinates only through
 * differences inside a (2dx+1) x (2dy+1) window, so a shifted sensor encodes
 * exactly as on its own, and no window reaches another sensor.  Times enter
 * only as differences inside a window too, so each slice keeps its own start
 * t_ref_us.  The canvas then goes through the encoder once: one launch per
 * stage for the whole batch.  Not in the paper (which encodes one slice at a
 * time); results equal those of per-slice calls up to FP32 summation order. */
typedef struct {
    const int16_t *d_x, *d_y; /* device, n events each */
    const uint32_t *d_t;      /* device, microseconds; every t in [t_ref_us, t_ref_us + t_span] */
    int64_t n;                /* events of this slice (0 allowed) */
    uint32_t t_ref_us;        /* slice start */
    int32_t width, height;    /* this slice's sensor; each at most the context's */
} veckm_slice;

/* Host-only shelf packing used by the batch calls: sensors sorted by height
 * (ties by index), placed left to right in shelves no wider than max_width,
 * with gap_x columns between neighbours and gap_y rows between shelves.
 * Writes each sensor's offset to ox[i], oy[i] and the canvas extent (the
 * bounding box of all sensors) to *canvas_w, *canvas_h.  VECKM_EINVAL if a
 * sensor is wider than max_width or a size is not positive. */
veckm_status veckm_canvas_layout(int32_t nslices, const int32_t *widths, const int32_t *heights,
                                 int32_t gap_x, int32_t gap_y, int32_t max_width, int32_t *ox,
                                 int32_t *oy, int32_t *canvas_w, int32_t *canvas_h);

/* Flows of every event of every slice: d_flow (device) is float
 * [sum n][2], slices in order, events in input order within a slice.
 * VECKM_EBUSY if the canvas does not fit the context (width x height) or the
 * records cannot grow while a plan exists.  Out-of-range events are reported
 * as in veckm_predict (their rows are zeroed).  May grow context buffers with
 * cudaMalloc (synchronising the stream) the first time a larger batch comes. */
veckm_status veckm_predict_batch(veckm_ctx *ctx, const veckm_slice *slices, int32_t nslices,
                                 float *d_flow, void *stream);
/* Encodings of every event of every slice: d_emb is float [sum n][2D]. */
veckm_status veckm_encode_batch(veckm_ctx *ctx, const veckm_slice *slices, int32_t nslices,
                                float *d_emb, void *stream);

/* A batch captured once into a CUDA graph and replayed: the slices' buffers,
 * sizes and starts and the output buffer are fixed at creation (new event
 * values in the same buffers are picked up by each launch).  Creation
 * allocates what the batch needs, autotunes the pooling launch shapes for its
 * canvas if veckm_autotune has not, and captures every copy and kernel of the
 * batch call on an internal stream.  predict != 0 captures
 * veckm_predict_batch, else veckm_encode_batch.  While a plan exists its
 * context keeps its buffers (calls needing larger ones return VECKM_EBUSY) and
 * its precision (veckm_set_mlp_mode returns VECKM_EBUSY).  A plan must be
 * destroyed before its context. */
typedef struct veckm_plan veckm_plan;
veckm_status veckm_plan_create(veckm_ctx *ctx, const veckm_slice *slices, int32_t nslices,
                               float *d_out, int32_t predict, veckm_plan **out);
/* Launch the captured graph on stream (ordered after earlier work there). */
veckm_status veckm_plan_launch(veckm_plan *plan, void *stream);
/* Number of kernel launches in one replay of the plan. */
int veckm_plan_kernel_count(const veckm_plan *plan);
void veckm_plan_destroy(veckm_plan *plan);

/* Autotune the launch shapes of the pooling passes (segment length per warp
 * and warps per block of the row and column passes) for a width x height
 * geometry (at most the context's): every candidate is timed with CUDA
 * events on stream over the context's accumulator buffers, and the fastest
 * is kept for calls on that geometry and pooled-grid storage.  Overwrites the
 * context's intermediate buffers (not the caller's).  Synchronous.  The
 * choice never changes results.  Writes the chosen shapes to tuned[0..3]
 * (rows segment, rows warps, columns segment, columns warps) if non-NULL. */
veckm_status veckm_autotune(veckm_ctx *ctx, int32_t width, int32_t height, void *stream,
                            int32_t *tuned);

/* ------------------------------------------------------------------ streams
 * Sliding-window encoding of one sensor's event stream (not in the paper's
 * implementation; it follows from the linearity of the accumulation of
 * Algorithm 1).  A stream keeps its window's per-pixel phase sums and counts
 * resident on the device and updates them per pushed packet: the packet's
 * events are added and the events that left the window subtracted.  The sums
 * are held in 64-bit fixed point (units of 2^-32; each event adds and later
 * subtracts the same integers), so the resident sums stay bit-identical to
 * sums built from the window's events alone, however many packets pass (no
 * drift, no rebuild).
 * The context supplies the sensor, D, the window radii, dt, the weights and
 * its scratch buffers; calls on a stream and on its context are ordered on
 * one CUDA stream. */
typedef struct veckm_stream veckm_stream;

/* window_us: the window length (events with t >= t_hi - window_us stay);
 * capacity: the most events the window may hold (the device ring).  Allocates
 * 32 D bytes per pixel plus 16 bytes per ring slot. */
veckm_status veckm_stream_create(veckm_ctx *ctx, int64_t window_us, int64_t capacity,
                                 veckm_stream **out);
/* Push a packet of n events (device x, y int16; t uint32 microseconds, the
 * stream's absolute times, sorted, all >= the previous packet's) that ends
 * at t_hi_us, which may not be earlier than the previous push's (else
 * VECKM_EINVAL, nothing enqueued).  The window becomes [t_hi_us - window_us,
 * t_hi_us]; the packet's events are encoded against it (predict == 0: d_out
 * float [n][2D] encodings; else d_out float [n][2] flows).  An event outside
 * the sensor or the window is not added, nor one earlier than an event
 * accepted before it (in an earlier packet, or earlier in this one inside
 * the sensor and the window), so the window's events stay in time order;
 * such an event's output row is zeroed (VECKM_ERANGE at the next status
 * check); events beyond the ring's capacity likewise (VECKM_EBUSY).  Never
 * synchronises.  n may be 0 (the window still slides to t_hi_us). */
veckm_status veckm_stream_push(veckm_stream *st, const int16_t *d_x, const int16_t *d_y,
                               const uint32_t *d_t, int64_t n, uint32_t t_hi_us, float *d_out,
                               int32_t predict, void *stream);
/* Events currently in the window (synchronises the stream). */
veckm_status veckm_stream_window(veckm_stream *st, int64_t *h_events, void *stream);
/* Copy the resident sums (int64 [H][W][D/2][4]: re(2u), im(2u), re(2u+1),
 * im(2u+1) in units of 2^-32) and counts (int32 [H][W]) to host memory
 * (synchronises the stream). */
veckm_status veckm_stream_accumulator(veckm_stream *st, int64_t *h_acc, int32_t *h_cnt,
                                      void *stream);
void veckm_stream_destroy(veckm_stream *st);

/* ------------------------------------------------------------------ serving
 * A request loop for event packets from many sensors.  veckm_server_submit
 * admits a packet if its events (8 bytes each, in three 256-byte aligned
 * arrays; with resident windows also its flows, 8 bytes each) fit in the
 * server's device arena, a ring sized from free HBM at creation, and refuses
 * it with VECKM_EBUSY otherwise; an admitted packet's events are copied
 * host-to-device at once on an upload stream.  A native worker thread takes
 * admitted packets in arrival order.  Two modes:
 *   - packets as slices (window_us == 0): each packet is one slice (its
 *     events, its sensor size and its start).  The worker takes as many
 *     waiting packets as fit one canvas batch and runs them as one
 *     veckm_predict_batch on its compute stream (at most two batches in
 *     flight).
 *   - resident windows (window_us > 0): every sensor stream keeps its
 *     window's per-pixel sums resident on the device (a veckm_stream of its
 *     own, on a context of its own sensor size, created with the stream's
 *     first packet; a stream whose state cannot be allocated has its packet
 *     refused with VECKM_EBUSY).  A packet of a stream slides that stream's
 *     window to end at its last event (events must come sorted by time, not
 *     earlier than the stream's previous ones; t_ref_us is unused) and its
 *     flows are those of its events against the window (veckm_stream_push).
 *     Each stream's packets run in order on the stream's own CUDA stream;
 *     packets of different streams run concurrently on the device, up to 64
 *     at once, and complete in any order.
 * Each packet's flows are copied to its host buffer and the packet is
 * reported complete, with its latency from submission to completion.  The
 * paper has no serving layer. */
typedef struct veckm_server veckm_server;

typedef struct {
    veckm_config model;        /* as for veckm_create; width x height is the canvas */
    int64_t arena_bytes;       /* device bytes for packets in flight; 0: a quarter of the
                                  free HBM left after the context is created */
    int32_t max_batch_packets; /* packets per batch; 0: 256 */
    int64_t max_batch_events;  /* events per batch; 0: 2^24 */
    int32_t batch_window_us;   /* a batch that is not full waits for more packets until
                                  its oldest packet is this old; 0: launch at once */
    int32_t window_us;         /* > 0: resident windows of this length per stream; 0:
                                  packets as slices */
    int64_t window_capacity;   /* events one stream's window may hold; 0: 2^22 */
} veckm_server_config;

typedef struct {
    int32_t stream_id;          /* the sensor stream, 0 .. 65535 */
    uint64_t tag;               /* returned with the completion */
    const int16_t *h_x, *h_y;   /* host; pinned memory makes the upload asynchronous */
    const uint32_t *h_t;
    int64_t n;                  /* 1 .. VECKM_MAX_EVENTS */
    uint32_t t_ref_us;
    int32_t width, height;      /* the packet's sensor, at most the canvas */
    float *h_flow;              /* host [n][2]; written before the completion is reported */
} veckm_packet;

typedef struct {
    uint64_t tag;
    int32_t stream_id;
    veckm_status status;        /* VECKM_ERANGE if an event of the batch was out of range */
    int64_t n;
    double latency_ms;          /* submission to completion, host steady clock */
    int32_t batch_packets;      /* packets in the batch that carried this one */
} veckm_completion;

typedef struct {
    int64_t submitted, admitted, refused, completed, batches, events_completed, streams;
    double p50_ms, p99_ms, max_ms;  /* latency over completed packets */
    double wall_s;                  /* first submission to last completion */
    double gpu_busy_s;              /* sum of batch device times (CUDA events); with resident
                                       windows, of per-packet device times, which overlap */
} veckm_server_stats;

/* Create the server, its context (cfg->model) and its worker thread.  The
 * host buffers of a packet must stay valid until its completion is polled. */
veckm_status veckm_server_create(const veckm_server_config *cfg, veckm_server **out);
/* Admit (VECKM_OK) or refuse (VECKM_EBUSY: no room in the arena) one packet.
 * VECKM_EINVAL for a malformed packet.  Thread safe. */
veckm_status veckm_server_submit(veckm_server *srv, const veckm_packet *pkt);
/* Up to max completions, oldest first; waits up to wait_ms for the first.
 * Returns how many were written (or a negative status). */
int32_t veckm_server_poll(veckm_server *srv, veckm_completion *out, int32_t max, int32_t wait_ms);
/* Wait until every admitted packet has completed (completions stay pollable). */
veckm_status veckm_server_drain(veckm_server *srv);
veckm_status veckm_server_get_stats(veckm_server *srv, veckm_server_stats *st);
/* Stops the worker after the packets in flight and frees everything. */
void veckm_server_destroy(veckm_server *srv);

/* ------------------------------------------------------------ error paths
 * Failure detection and its tests (not in the paper).  Every wait of a
 * kernel on another part of itself (the tensor-core head's mbarrier
 * hand-offs) is bounded: when it runs out the kernel releases what it holds
 * and leaves, the rows it did not finish keep whatever they held, and the
 * device error word reports VECKM_ETIMEOUT at the next status check; the
 * context stays usable. */

/* Limit of each bounded wait of the tensor-core head in SM clock cycles;
 * 0 restores the default (4e9 cycles, about 2 s at 2 GHz). */
veckm_status veckm_set_wait_limit(veckm_ctx *ctx, int64_t cycles);

/* Fault injection for tests of the error paths, off by default.
 * VECKM_INJECT_HEAD_STALL: the tensor-core head's producer warps never signal
 * a filled tile, so its waits run out (VECKM_ETIMEOUT); nothing faults and
 * nothing waits without a limit.  VECKM_INJECT_NONE turns it off. */
#define VECKM_INJECT_NONE 0
#define VECKM_INJECT_HEAD_STALL 1
veckm_status veckm_set_injection(veckm_ctx *ctx, int32_t what);

/* Test hook for the out-of-memory paths (host side): counts the library's
 * device (cudaMalloc) and pinned host (cudaMallocHost) allocations from 0
 * again, and makes allocation number fail_at (if >= 0; -1 turns it off) fail
 * as if memory were exhausted, which the calling entry point reports as
 * VECKM_ENOMEM after freeing what it had allocated.  Returns the number of
 * allocations counted since the previous call.  Process wide. */
int64_t veckm_debug_fail_alloc(int64_t fail_at);

/* Bounds-checked build (no counterpart in the paper; a stand-in for a device
 * memory checker).  The library built with -DVECKM_CHECKED
 * (paper_2504_19417_gb300/build.py, build(checked=True):
 * libveckm_checked.so) tests every index its kernels derive from data before
 * the access it guards (the pixel of a sorted record, a slot from an atomic
 * counter, a bucket from an event, a ring position) and, where one would
 * leave its buffer, counts it and skips the access.  veckm_debug_checks waits
 * for the device (cudaDeviceSynchronize), stores the number counted since the
 * previous call in *violations and where the first one was in *first_line
 * (file number * 100000 + source line; files: 1 kernels.cu, 2 mlp_tc.cu,
 * 3 stream.cu; 0 if none), and clears both.  Process wide.  In the normal
 * build it returns VECKM_EUNSUPPORTED and the checks compile away. */
veckm_status veckm_debug_checks(int64_t *violations, int32_t *first_line);

/* SplitMix64 + Box-Muller standard normals (the generator behind freq_seed):
 * writes count normals of stream `seed` to h_out.  Host only. */
void veckm_normals(uint64_t seed, int64_t count, double *h_out);

#ifdef __cplusplus
}
#endif
#endif /* VECKM_H */
