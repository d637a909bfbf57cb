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
 * that may not allocate device memory during a call (graph recording,
 * real-time loops, devices whose memory is reserved up front).  veckm_encode
 * may grow its per-event buffers with cudaMalloc; this call takes them from a
 * fixed array in device memory that the library declares statically and
 * never calls cudaMalloc, cudaFree or any allocating routine.  The paper has
 * no counterpart; it is a deployment variant.
 *   - At most 1048576 events per call (n); larger n returns VECKM_EINVAL.
 *   - The array (12 MiB) exists on every GPU that loads the library until the
 *     process exits.  The first call on a device looks up its address there
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls on a device share the array and the context's accumulators:
 *     calls that may overlap on the GPU race and must be serialised.
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
 * stream around each stage.  Stages: 0 clear (memset of the accumulators),
 * 1 per-pixel accumulation (the first loop of Algorithm 1), 2 pooling row pass,
 * 3 window counts (Eq. 17), 4 pooling column pass (the window sums of
 * Eq. 16), 5 gather + normalise, fused with the perceptron in veckm_predict.
 * veckm_stage_times synchronises, writes the elapsed milliseconds summed over
 * every timed call since the last read into ms[0..nstage-1] and the number of
 * timed calls into calls[0..nstage-1] (may be NULL), then resets. */
veckm_status veckm_set_timing(veckm_ctx *ctx, int enable);
veckm_status veckm_stage_times(veckm_ctx *ctx, double *ms, int64_t *calls, int nstage);

/* Number of kernel launches the last encode/predict call made. */
int veckm_last_launch_count(const veckm_ctx *ctx);

/* SplitMix64 + Box-Muller standard normals (the generator behind freq_seed):
 * writes count normals of stream `seed` to h_out.  Host only. */
void veckm_normals(uint64_t seed, int64_t count, double *h_out);

#ifdef __cplusplus
}
#endif
#endif /* VECKM_H */
