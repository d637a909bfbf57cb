// Internal declarations shared by the library's own translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/veckm.h"

namespace veckm {

// Bits of the device error word.
enum : int { ERR_EVENT_RANGE = 1, ERR_INDEX_RANGE = 2, ERR_TIMEOUT = 4, ERR_CAPACITY = 8 };

// Device view of one slice's events.
struct Events {
  const int16_t *x, *y;
  const uint32_t *t;
  int64_t n;
  uint32_t t_ref;
  uint32_t t_span;  // largest accepted t - t_ref
};

// Device-side constant state of a context.  Complex values are stored as
// interleaved (re, im) FP32 with the channel index fastest; one float4 holds
// channels 2u and 2u+1 ("unit" u), so a pixel has U = D/2 units.
// One slice of a batch as it sits on the canvas (batch.cu): its events, its
// place among the canvas events and the mapping kernel's blocks, and its
// sensor's size and offset on the canvas.
struct CanvasSlice {
  const int16_t *x, *y;
  const uint32_t *t;
  long long n;    // events
  long long off;  // first canvas event (sum of the previous slices' n)
  long long blk;  // first block of the mapping kernel
  uint32_t t_ref;
  int W, H, ox, oy;
};

struct Geometry {
  int W, H, D, U, dx, dy;
  // a batch's canvas (device table of its slices, or null): the pooling
  // passes skip line segments that no slice's outputs depend on
  const CanvasSlice *canvas = nullptr;
  int ncanvas = 0;
};

struct Tables {
  const float4 *tx;     // [dx + W][U] exp(i x X/dx), x in [-dx, W), row x + dx
  const float4 *ty;     // [H][U]      exp(i y Y/dy), y in [0, H)
  const float4 *sx;     // [U]         exp(i X/dx), one step along x
  const float4 *sy;     // [U]         exp(i Y/dy), one step along y
  const uint2 *wt;      // [D]         T_d/(2 pi dt) in turns per microsecond, reduced to
                        //             [-1/2, 1/2], as 64-bit fixed point (lo, hi words)
  const float4 *rx;     // [2dx + 1][U] exp(i o X/dx), offset o in [-dx, dx], row o + dx
  const float4 *ry;     // [2dy + 1][U] exp(i o Y/dy), offset o in [-dy, dy], row o + dy
};

struct MLP {
  const float *W1;       // [hidden][2D] FP32
  const float *W1t;      // [2D][hidden] FP32 (transposed copy for the CUDA-core path)
  const float *b1;       // [hidden]
  const float *W2;       // [2][hidden]
  const float *b2;       // [2]
  const uint16_t *W1h;   // [hidden][2D] BF16 or FP16 bits, core-matrix order for tcgen05
  int hidden;
  int half_kind;         // 0: BF16, 1: FP16 (for W1h)
  int pooled_half;       // tensor-core head: 1, the pooled grid is FP16 and divided by the
                         // counts; 0, FP32 window sums in the launch_pool_cols_pair order
  // host copies of b1, W2, b2 (kernel parameters of the tensor-core head)
  const float *hb1 = nullptr, *hW2 = nullptr, *hb2 = nullptr;
  // [16][hidden] FP16 bits: W2 padded to 16 rows, core-matrix order for
  // the tensor-core head's second layer
  const uint16_t *W2h = nullptr;
  // tensor-core head: limit of each bounded wait in SM cycles, and the test
  // injection that stops its producers from signalling filled tiles
  long long wait_cycles = 4000000000LL;
  int inject_stall = 0;
  // host copy of the fixed-point temporal frequencies (Tables::wt), passed
  // to the D = 64 tensor-core head as a kernel parameter
  const uint2 *hwt = nullptr;
};

// Launch shapes picked by the autotuner (batch.cu); 0 keeps the built-in
// default.  The results do not depend on them.
struct Tune {
  int rows_seg = 0, rows_wpb = 0;  // row pass: segment length in windows, warps per block
  int cols_seg = 0, cols_wpb = 0;  // column pass: the same
};

// Launchers (kernels.cu, mlp_tc.cu).  Each returns the number of kernels it
// launched, or a negative value on a launch failure.
// zero_flow (nullable): flow rows of invalid events are zeroed (sorted prediction).
int launch_hist(const Events &ev, const Geometry &g, int *cnt, int *err, float *zero_flow,
                cudaStream_t s);
int scan_blocks(int64_t P);
int launch_scan(const Geometry &g, const int *cnt, int *bsum, int *off, int *cur, int *total,
                cudaStream_t s, bool chain = false);
int launch_place(const Events &ev, const Geometry &g, int *cur, int2 *rec, int *pix,
                 cudaStream_t s, bool chain = false);
// The same outputs as launch_hist + launch_scan + launch_place (counts per
// pixel, the record total in *total, pixel-grouped records) by a two-level
// bucket sort without global atomics.  bucket_sort_shift: log2 of the pixels
// per bucket for P pixels, or -1 when P is beyond the form's limits
// (launch_bucket_sort returns -1 outside bucket_sort_fits).  A geometry of P pixels has at most
// min(P, bucket_sort_max_buckets()) buckets.  brec: n records; bhist: twice
// that many buckets times bucket_sort_max_tiles() ints (per-tile counts,
// then their prefixes); btot: one per bucket.  zgrid (optional): a grid of
// g.U float4 per pixel whose rows at the per-pixel sums' range edges are
// zeroed, so that launch_pixsum(..., clear = false) may write into it
// uncleared (pixels without records then hold stale values: read it only
// through launch_pool_rows with occ = the counts).
int bucket_sort_shift(int64_t P);
int bucket_sort_max_buckets();
int bucket_sort_max_tiles();
// Whether P pixels and n events are within the bucket form's limits.
bool bucket_sort_fits(int64_t P, int64_t n);
int launch_bucket_sort(const Events &ev, const Geometry &g, int *cnt, int *total, int2 *rec,
                       int *rpix, int4 *brec, int *bhist, int *btot, int *err, float *zero_flow,
                       cudaStream_t s, float4 *zgrid = nullptr);
// Clears acc (unless the caller knows it is zero, or the sort zeroed the
// range-edge rows: clear = false), then sums the *nsorted pixel-sorted
// records (n bounds it).  Pixels without records are not written.
// chain (here and below): the launch may overlap the end of the kernel
// before it in s (programmatic dependent launch, chain.cuh); only for a
// launch whose predecessor in s is a kernel of the same step.
int launch_pixsum(const Geometry &g, const Tables &tb, const int *nsorted, const int2 *rec,
                  const int *rpix, int64_t n, float4 *acc, cudaStream_t s, bool clear = true,
                  bool chain = false);
// Readers of the bounds-checked build's violation words, one per translation
// unit with checks: the count since the previous read (the first source line
// in *line), then cleared; -1 if the device could not be read; 0 in the
// normal build.
int check_read_kernels(int *line);
int check_read_head(int *line);
int check_read_stream(int *line);
// Blocks of `threads` threads with `smem` dynamic bytes that fit on one SM.
int blocks_per_sm(const void *func, int threads, size_t smem);
// Pooling: row pass acc -> hbuf, column pass hbuf -> acc, window counts.
// occ (row pass; window length 2dx+1 <= 32, else -1): per-pixel event counts,
// pixels with none read as zero whatever acc holds there.
int launch_pool_rows(const Geometry &g, const Tables &tb, const float4 *acc, float4 *hbuf,
                     cudaStream_t s, const Tune &tn = Tune{}, const int *occ = nullptr,
                     bool chain = false);
int launch_pool_cols(const Geometry &g, const Tables &tb, const float4 *hbuf, float4 *acc,
                     cudaStream_t s, const Tune &tn = Tune{});
int launch_counts(const Geometry &g, const int *cnt, int *cnt_tmp, int *ncnt, cudaStream_t s);
// Column pass writing the pooled grid divided by the window counts as FP16:
// per pixel D/2 units of 8 bytes (Re 2u, Re 2u+1, Im 2u, Im 2u+1).
int launch_pool_cols_half(const Geometry &g, const Tables &tb, const float4 *hbuf,
                          const int *ncnt, void *pooled16, cudaStream_t s, const Tune &tn = Tune{});
// Column pass writing the pooled grid (the window sums) as FP32 with unit u
// of a pixel = (Re 2u, Re 2u+1, Im 2u, Im 2u+1): the grid the tensor-core head
// reads when the pooled grid is kept in FP32.
int launch_pool_cols_pair(const Geometry &g, const Tables &tb, const float4 *hbuf,
                          float4 *pooled, cudaStream_t s, const Tune &tn = Tune{});
int launch_gather_emb(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                      const Tables &tb, const float4 *pooled, const int *ncnt, float *emb,
                      int *err, cudaStream_t s);
// Perceptron launchers: rec/rpix non-null selects the pixel-sorted order
// (all valid events, *nsorted of them on the device; row i is written to
// flow[rec[i].y]); otherwise K (or the identity).
int launch_predict_fp32(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                        const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                        const float4 *pooled, const int *ncnt, const MLP &mlp, float *flow,
                        int *err, cudaStream_t s);
// pooled: float4 FP32 grid, or (mlp.pooled_half) the FP16 grid divided by the counts
int launch_predict_tc(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                      const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                      const void *pooled, const int *ncnt, const MLP &mlp, float *flow,
                      int *err, cudaStream_t s, const Tune &tn = Tune{},
                      float4 *zero_buf = nullptr, int64_t zero_units = 0,
                      bool *zeroed = nullptr, bool chain = false);
// Forget which grid of the context is known to be zero (for paths that write
// the grids outside the dense pipeline).
void grids_dirty(veckm_ctx *c);

// Direct window form: per-pixel sums written once per occupied pixel (no
// clear), then one warp per requested event summing its window (mlp == NULL:
// the encoding to out [nK][2D]; else the flows to out [nK][2], D <= 128).
int launch_pixsum_owned(const Geometry &g, const Tables &tb, const int *nsorted, const int2 *rec,
                        const int *rpix, int64_t n, float4 *acc, cudaStream_t s,
                        bool chain = false);
int launch_direct(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                  const Tables &tb, const float4 *acc, const int *cnt, const MLP *mlp, float *out,
                  int *err, cudaStream_t s, bool chain = false);

int num_sms();

// Device buffers and geometry of a context (veckm.cu), for entry points that
// live in other translation units.
struct CtxView {
  Geometry g;
  Tables tb;
  float4 *acc, *hbuf;
  int *cnt, *cnt_tmp, *ncnt, *off, *cur, *bsum, *total, *err;
  int64_t t_span;
  Tune tn;  // the pooling launch shapes tuned for g (defaults if none)
};
bool ctx_view(const veckm_ctx *c, CtxView *v);
// Records msg as this thread's last error and returns st.
veckm_status report(veckm_status st, const char *msg);

// Every device (dev_malloc) and pinned-host (host_malloc) allocation of the
// library goes through these: they count allocations and can fail one of them
// on purpose (veckm_debug_fail_alloc) to test the out-of-memory paths.
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t host_malloc(void **p, size_t bytes);

}  // namespace veckm
