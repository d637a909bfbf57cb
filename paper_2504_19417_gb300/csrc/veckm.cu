// Host side of the C ABI declared in include/veckm.h: context creation,
// FP64 phase-table construction, stream-ordered launches, error reporting and
// per-stage timing.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "ctx.h"

namespace veckm {
namespace {
// the allocation counter behind veckm_debug_fail_alloc
std::atomic<long long> g_alloc_count{0};     // allocations since the last reset
std::atomic<long long> g_alloc_fail_at{-1};  // the one to fail (-1: none)

bool alloc_should_fail() {
  const long long k = g_alloc_count.fetch_add(1);
  return k == g_alloc_fail_at.load();
}
}  // namespace
}  // namespace veckm

using namespace veckm;

namespace {

thread_local char g_err[512] = "";

veckm_status fail(veckm_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

veckm_status cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? VECKM_ENOMEM : VECKM_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

// SplitMix64 (Steele, Lea, Flood 2014): output i is mix(seed + (i+1) * gamma).
uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

enum class Out { Emb, Flow };

}  // namespace

namespace {

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
  return dev_malloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

// exp(i (first + n) * step * w_d * scale) for n in [0, rows) as interleaved
// FP32 (re, im), channel fastest.  The angle is formed in FP64 (it stays below
// ~1e6 rad, where FP64 keeps ~1e-10 rad), then rounded once to FP32.
std::vector<float> phase_rows(const std::vector<double> &w, double scale, int64_t first,
                              int64_t rows, int64_t step) {
  const size_t D = w.size();
  std::vector<float> out((size_t)rows * D * 2);
  for (int64_t n = 0; n < rows; ++n)
    for (size_t d = 0; d < D; ++d) {
      const double a = (double)((first + n) * step) * (w[d] * scale);
      out[((size_t)n * D + d) * 2] = (float)std::cos(a);
      out[((size_t)n * D + d) * 2 + 1] = (float)std::sin(a);
    }
  return out;
}

uint16_t half_bits(float v, bool fp16) {
  if (fp16) {
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t *>(&h);
  }
  __nv_bfloat16 b = __float2bfloat16_rn(v);
  return *reinterpret_cast<uint16_t *>(&b);
}

// W1 [hidden][IN] -> the K-major 128-byte-swizzled order the tcgen05 kernel
// reads: K-blocks of 64 columns, each hidden x 128 B; row n of a block at
// (n/8)*1024 + (n%8)*128, its 16-byte chunk c at position c ^ (n%8).
// W1 as the tensor-core B operand: K-major, 128-byte swizzled, with the K
// axis permuted to the order in which the gather writes the A operand: K
// position 4u + {0, 1, 2, 3} holds input Re(2u), Re(2u+1), Im(2u), Im(2u+1),
// i.e. columns 2u, 2u+1, D+2u, D+2u+1 of W1 (whose input is packed [Re | Im]).
// The contraction runs over all of K, so the same permutation of A's columns
// and B's rows leaves W1 x unchanged.
std::vector<uint16_t> w1_core_matrix(const std::vector<float> &W1, int hidden, int IN, bool fp16) {
  std::vector<uint16_t> out((size_t)hidden * IN);
  const int D = IN / 2;
  for (int n = 0; n < hidden; ++n)
    for (int k = 0; k < IN; ++k) {
      const int src = ((k & 2) ? D : 0) + 2 * (k >> 2) + (k & 1);
      const size_t byte = (size_t)(k / 64) * hidden * 128 + (size_t)(n / 8) * 1024 + (n % 8) * 128 +
                          (size_t)((((k / 8) % 8) ^ (n % 8)) * 16) + (k % 8) * 2;
      out[byte / 2] = half_bits(W1[(size_t)n * IN + src], fp16);
    }
  return out;
}

// W2 [2][hidden] as the B operand of the tensor-core head's second layer:
// FP16, padded to 16 rows (rows 2..15 zero), K-major and 128-byte swizzled
// like W1 (K-blocks of 64 columns, each 16 x 128 B), with the K axis in the
// natural order of the hidden units.
std::vector<uint16_t> w2_core_matrix(const std::vector<float> &W2, int hidden) {
  constexpr int N2 = 16;
  std::vector<uint16_t> out((size_t)N2 * hidden, 0);
  for (int n = 0; n < 2; ++n)
    for (int k = 0; k < hidden; ++k) {
      const size_t byte = (size_t)(k / 64) * N2 * 128 + (size_t)(n / 8) * 1024 + (n % 8) * 128 +
                          (size_t)((((k / 8) % 8) ^ (n % 8)) * 16) + (k % 8) * 2;
      out[byte / 2] = half_bits(W2[(size_t)n * hidden + k], true);
    }
  return out;
}

// The tensor-core head rounds ReLU(h) to FP16 for its second layer.  An
// encoding has |Re e_d|, |Im e_d| <= 1 (a mean of unit phasors), so
// |h_j| <= sum_c |W1_jc| + |b1_j|; that must stay well inside FP16's range.
bool tc_head_range_ok(const veckm_ctx *c) {
  const int IN = 2 * c->g.D;
  for (int j = 0; j < c->hidden; ++j) {
    double s = std::fabs((double)c->hb1[j]);
    for (int k = 0; k < IN; ++k) s += std::fabs((double)c->hW1[(size_t)j * IN + k]);
    if (!(s < 32768.0)) return false;
  }
  for (float w : c->hW2)
    if (!(std::fabs(w) < 32768.0f)) return false;
  return true;
}

void free_all(veckm_ctx *c) {
  veckm::destroy_pipe(c->pipe);
  c->pipe = nullptr;
  void *ptrs[] = {c->tx, c->ty, c->sx, c->sy, c->wt, c->W1, c->W1t, c->b1, c->W2, c->b2,
                  c->W1h, c->W2h, c->acc, c->hbuf, c->cnt, c->cnt_tmp, c->ncnt, c->err, c->st_buf,
                  c->off, c->cur, c->bsum, c->total, c->rec, c->rpix, c->brec, c->bhist, c->btot,
                  c->cx, c->cy, c->ct,
                  c->slice_tab, c->wxy, c->rx, c->ry};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->h_slice_tab) cudaFreeHost(c->h_slice_tab);
  if (c->tab_copied) cudaEventDestroy(c->tab_copied);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_fork0) cudaEventDestroy(c->ev_fork0);
  if (c->ev_zero) cudaEventDestroy(c->ev_zero);
  if (c->side) cudaStreamDestroy(c->side);
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  for (auto &v : c->pending)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
}

cudaEvent_t take_event(veckm_ctx *c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

namespace veckm {
veckm_status check_events_args(veckm_ctx *c, const void *x, const void *y, const void *t,
                               int64_t n, const void *K, int64_t nK, const void *out) {
  if (!c) return fail(VECKM_EINVAL, "null context");
  if (n < 0 || nK < 0) return fail(VECKM_EINVAL, "negative size (n=%lld, nK=%lld)", (long long)n, (long long)nK);
  if (n > VECKM_MAX_EVENTS || nK > VECKM_MAX_EVENTS)
    return fail(VECKM_EINVAL, "more than %lld events or requests in one call (n=%lld, nK=%lld)",
                (long long)VECKM_MAX_EVENTS, (long long)n, (long long)nK);
  if (n > 0 && (!x || !y || !t)) return fail(VECKM_EINVAL, "null event buffer with n=%lld", (long long)n);
  if (!K && nK != n && nK != 0)
    return fail(VECKM_EINVAL, "K is NULL but nK (%lld) != n (%lld)", (long long)nK, (long long)n);
  if (nK > 0 && !out) return fail(VECKM_EINVAL, "null output buffer");
  if (nK > 0 && n == 0) return fail(VECKM_EINVAL, "nK > 0 with an empty slice");
  return VECKM_OK;
}
}  // namespace veckm

namespace {

}  // namespace

namespace veckm {

veckm_status ensure_records(veckm_ctx *c, int64_t n, cudaStream_t s) {
  if (n <= c->rec_cap) return VECKM_OK;
  if (c->live_plans > 0)
    return fail(VECKM_EBUSY, "%lld events need larger record buffers, which cannot be "
                "reallocated while a captured plan uses them", (long long)n);
  cudaError_t e = cudaStreamSynchronize(s);
  if (c->rec) cudaFree(c->rec);
  if (c->rpix) cudaFree(c->rpix);
  if (c->brec) cudaFree(c->brec);
  c->rec = nullptr;
  c->rpix = nullptr;
  c->brec = nullptr;
  c->rec_cap = 0;
  if (e == cudaSuccess) e = dalloc(&c->rec, (size_t)n);
  if (e == cudaSuccess) e = dalloc(&c->rpix, (size_t)n);
  if (e == cudaSuccess) e = dalloc(&c->brec, (size_t)n);
  if (e != cudaSuccess) {  // keep none of a partial set
    if (c->rec) cudaFree(c->rec);
    if (c->rpix) cudaFree(c->rpix);
    if (c->brec) cudaFree(c->brec);
    c->rec = nullptr;
    c->rpix = nullptr;
    c->brec = nullptr;
    return cuda_fail(e, "event record buffers");
  }
  c->rec_cap = n;
  return VECKM_OK;
}

veckm_status run_pipeline(veckm_ctx *c, const Geometry &g, const Events &ev, const int64_t *K,
                          int64_t nK, float *out, bool flow, cudaStream_t s, const Tune &tn) {
  const Out what = flow ? Out::Flow : Out::Emb;
  const int64_t n = ev.n;
  c->last_launches = 0;
  if (nK == 0) return VECKM_OK;  // nothing requested: no work
  if ((int64_t)g.W * g.H > (int64_t)c->g.W * c->g.H || g.W > c->g.W || g.H > c->g.H)
    return fail(VECKM_EINVAL, "geometry %dx%d exceeds the context's %dx%d", g.W, g.H, c->g.W,
                c->g.H);
  const Tables tb = c->tables();
  std::vector<cudaEvent_t> evs;
  auto mark = [&]() {
    if (c->timing) {
      cudaEvent_t e = take_event(c);
      cudaEventRecord(e, s);
      evs.push_back(e);
    }
  };
  const size_t P = (size_t)g.W * g.H;
  // pixel-sorted prediction for "all events"; explicit K keeps input order
  const bool sorted = (what == Out::Flow) && K == nullptr;
  if (veckm_status st = ensure_records(c, n, s)) return st;
  int launches = 0, r;
  // Dense pooling or the direct window form, by the runtime model of Eq.
  // runtime (Section 2.2.2): the dense passes cost per pixel, the direct form
  // per requested flow and window pixel.  The direct perceptron is the FP32
  // one (D <= 128).
  const double area = (2.0 * g.dx + 1) * (2.0 * g.dy + 1);
  const double t_dense = c->k_pixel * (double)P + c->k_flow_dense * (double)nK;
  const double t_direct = c->k_flow_window * area * (double)nK;
  const bool direct_ok = what == Out::Emb || g.D <= 128;
  const bool direct = direct_ok && (c->path == VECKM_PATH_DIRECT ||
                                    (c->path == VECKM_PATH_AUTO && t_direct < t_dense));
  c->last_path = direct ? VECKM_PATH_DIRECT : VECKM_PATH_DENSE;
  mark();
  // Side-stream work is forked with an event record and joined back before
  // its consumer, on every return once forked.
  struct Join {
    cudaStream_t s;
    cudaEvent_t ev;
    bool armed = false;
    void wait() {
      if (armed) cudaStreamWaitEvent(s, ev, 0);
      armed = false;
    }
    ~Join() { wait(); }
  };
  auto fork = [&](cudaEvent_t at) {
    cudaError_t fe = cudaEventRecord(at, s);
    if (fe == cudaSuccess) fe = cudaStreamWaitEvent(c->side, at, 0);
    return fe;
  };
  // Dense path: with the bucket sort (and a window of at most 32 columns) the
  // pixel sums need no cleared grid: the sort zeroes the rows of the pixels
  // at the edges of the sums' record ranges, the only ones the sums add
  // into, the sums store the other pixels that have records, and the row
  // pass reads only pixels that have records (occupancy from the counts).
  // Otherwise the sums go to a grid known to be zero when there is one (the
  // previous call's tensor-core head cleared it), else acc is cleared, on the
  // side stream under the sort.  The row pass writes the other grid, the
  // column pass writes back into the first, which the gather reads.  A graph
  // capture cannot know what runs before a replay: it clears, unless the plan
  // capturing it picks the grid (capture_grid) and chooses between its two
  // graphs at each launch.
  const bool bucketed = bucket_sort_fits((int64_t)P, n);
  const bool sparse_rows = bucketed && 2 * g.dx + 1 <= 32;
  const int64_t units = (int64_t)P * g.U;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return cuda_fail(cudaGetLastError(), "capture query");
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  const int zgrid = capturing ? c->capture_grid
                              : (c->zero_grid >= 0 && c->zero_units >= units ? c->zero_grid : -1);
  const bool known_zero = zgrid >= 0;
  const bool may_zero = !capturing || c->capture_grid >= 0;
  float4 *gsum = c->acc, *grow = c->hbuf;
  if (zgrid == 1) std::swap(gsum, grow);
  Join zjoin{s, c->ev_zero};
  if (!direct) {
    c->zero_grid = -1;
    c->capture_zeroed = false;
    if (!known_zero && !sparse_rows) {
      cudaError_t fe = fork(c->ev_fork0);
      if (fe == cudaSuccess) fe = cudaMemsetAsync(gsum, 0, (size_t)units * sizeof(float4), c->side);
      if (fe == cudaSuccess) fe = cudaEventRecord(c->ev_zero, c->side);
      zjoin.armed = true;
      if (fe != cudaSuccess) return cuda_fail(fe, "clearing the pixel sums");
    }
  }
  // Sort by pixel: the bucket form (no global atomics) where the geometry
  // fits its limits, else histogram, scan and placement with global cursors.
  // Both give the per-pixel counts, the record total (off[P]) and the
  // pixel-grouped records.
  float *zero_flow = (sorted && !direct) ? out : nullptr;
  // A launch that follows a kernel of this step in s (after_kernel) is
  // chained to it (programmatic dependent launch, chain.cuh); the step's
  // first kernel and the first after a memset or a join with the side stream
  // keep full ordering.  Event records in between (the forks) change nothing.
  // The stage timing's marks (event records) sit between stages: with timing
  // on, the launches after a mark are plain (chain_marked), so that each
  // stage's events bracket its own kernels in full order.
  bool after_kernel = false;
  const bool chain_marked = !c->timing;
  if (bucketed) {
    if ((r = launch_bucket_sort(ev, g, c->cnt, c->off + P, c->rec, c->rpix, c->brec, c->bhist,
                                c->btot, c->err, zero_flow, s,
                                sparse_rows && !direct ? gsum : nullptr)) < 0)
      return cuda_fail(cudaGetLastError(), "bucket sort launch");
    launches += r;
    after_kernel = r > 0;
  } else {
    cudaError_t e = cudaMemsetAsync(c->cnt, 0, P * sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the counts");
    if ((r = launch_hist(ev, g, c->cnt, c->err, zero_flow, s)) < 0)
      return cuda_fail(cudaGetLastError(), "histogram launch");
    launches += r;
    if ((r = launch_scan(g, c->cnt, c->bsum, c->off, c->cur, c->total, s, r > 0)) < 0)
      return cuda_fail(cudaGetLastError(), "scan launch");
    launches += r;
    after_kernel = true;
  }
  // The window counts need only the per-pixel counts: on the dense path they
  // run on the side stream, under the pixel sums and row pass, and join
  // before the column pass.
  Join join{s, c->ev_join};
  if (!direct) {
    cudaError_t fe = fork(c->ev_fork);
    if (fe != cudaSuccess) return cuda_fail(fe, "forking the window counts");
    r = launch_counts(g, c->cnt, c->cnt_tmp, c->ncnt, c->side);
    fe = cudaEventRecord(c->ev_join, c->side);
    join.armed = true;
    if (r < 0 || fe != cudaSuccess) return cuda_fail(cudaGetLastError(), "window count launch");
    launches += r;
  }
  if (!bucketed) {
    if ((r = launch_place(ev, g, c->cur, c->rec, c->rpix, s, true)) < 0)
      return cuda_fail(cudaGetLastError(), "placement launch");
    launches += r;
  }
  mark();
  if (direct) {
    if (c->zero_grid == 0) c->zero_grid = -1;  // the owned sums write acc
    if ((r = launch_pixsum_owned(g, tb, c->off + P, c->rec, c->rpix, n, c->acc, s,
                                 after_kernel && chain_marked)) < 0)
      return cuda_fail(cudaGetLastError(), "pixel sum launch");
    launches += r;
    after_kernel = after_kernel || r > 0;
    mark();
    mark();  // no row pass, window counts or column pass
    mark();
    mark();
    MLP m = c->mlp();
    if ((r = launch_direct(ev, K, nK, g, tb, c->acc, c->cnt, what == Out::Flow ? &m : nullptr,
                           out, c->err, s, after_kernel && chain_marked)) < 0)
      return cuda_fail(cudaGetLastError(), "direct window launch");
    launches += r;
    mark();
    if (c->timing) c->pending.push_back(evs);
    c->last_launches = launches;
    return VECKM_OK;
  }
  // The pixel sums are chained to the sort unless they wait for the clear,
  // the row pass to the pixel sums, the head to the column pass; the column
  // pass follows the join with the side stream.
  const bool chain_sums = after_kernel && !zjoin.armed && chain_marked;
  zjoin.wait();  // the clear of gsum (side stream)
  if ((r = launch_pixsum(g, tb, c->off + P, c->rec, c->rpix, n, gsum, s, false, chain_sums)) < 0)
    return cuda_fail(cudaGetLastError(), "pixel sum launch");
  launches += r;
  const bool chain_rows = r > 0 && chain_marked;
  mark();
  if ((r = launch_pool_rows(g, tb, gsum, grow, s, tn, sparse_rows ? c->cnt : nullptr,
                            chain_rows)) < 0)
    return cuda_fail(cudaGetLastError(), "pooling (rows) launch");
  launches += r;
  mark();
  join.wait();  // the window counts (side stream)
  mark();
  // The tensor-core head reads the pooled grid as FP16 divided by the window
  // counts (VECKM_ACC_FP16), else as FP32 window sums with each unit's real
  // and imaginary parts paired; the other consumers read the plain sums.
  const bool tc_head = what == Out::Flow && (c->flags & (VECKM_MLP_BF16 | VECKM_MLP_FP16));
  const bool half_grid = tc_head && (c->flags & VECKM_ACC_FP16);
  if (half_grid)
    r = launch_pool_cols_half(g, tb, grow, c->ncnt, gsum, s, tn);
  else if (tc_head)
    r = launch_pool_cols_pair(g, tb, grow, gsum, s, tn);
  else
    r = launch_pool_cols(g, tb, grow, gsum, s, tn);
  if (r < 0) return cuda_fail(cudaGetLastError(), "pooling (columns) launch");
  launches += r;
  mark();
  if (what == Out::Emb) {
    r = launch_gather_emb(ev, K, nK, g, tb, gsum, c->ncnt, out, c->err, s);
  } else if (c->flags & (VECKM_MLP_BF16 | VECKM_MLP_FP16)) {
    MLP m = c->mlp();
    m.pooled_half = half_grid ? 1 : 0;
    bool zeroed = false;
    // a cleared grid serves only a next call whose sums cannot do without one
    r = launch_predict_tc(ev, K, nK, sorted ? c->rec : nullptr, sorted ? c->rpix : nullptr,
                          c->off + P, g, tb, gsum, c->ncnt, m, out, c->err, s, tn,
                          may_zero && !sparse_rows ? grow : nullptr, units, &zeroed,
                          chain_marked);
    if (r >= 0 && zeroed && !capturing) {
      c->zero_grid = grow == c->acc ? 0 : 1;
      c->zero_units = units;
    }
    if (r >= 0 && zeroed && capturing) {
      c->capture_zeroed = true;
      c->capture_units = units;
    }
  } else {
    r = launch_predict_fp32(ev, K, nK, sorted ? c->rec : nullptr, sorted ? c->rpix : nullptr,
                            c->off + P, g, tb, gsum, c->ncnt, c->mlp(), out, c->err, s);
    if (r == -2) return fail(VECKM_EUNSUPPORTED, "FP32 perceptron needs 2D*128 floats of shared memory; D=%d is too large", g.D);
  }
  if (r < 0) return cuda_fail(cudaGetLastError(), "gather launch");
  launches += r;
  mark();
  if (c->timing) c->pending.push_back(evs);
  c->last_launches = launches;
  return VECKM_OK;
}

}  // namespace veckm

namespace {

veckm_status run(veckm_ctx *c, const int16_t *x, const int16_t *y, const uint32_t *t, int64_t n,
                 uint32_t t_ref, const int64_t *K, int64_t nK, float *out, cudaStream_t s, Out what) {
  veckm_status st = check_events_args(c, x, y, t, n, K, nK, out);
  if (st) return st;
  const Events ev{x, y, t, n, t_ref, (uint32_t)c->t_span};
  return run_pipeline(c, c->g, ev, K, nK, out, what == Out::Flow, s, c->tune_for(c->g));
}

bool valid_D(int D) { return D == 64 || D == 128 || D == 192 || D == 256; }

}  // namespace

extern "C" {

const char *veckm_last_error(void) { return g_err; }

void veckm_normals(uint64_t seed, int64_t count, double *h_out) {
  if (!h_out || count <= 0) return;
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t j = 0; 2 * j < count; ++j) {
    const double u1 = (double)(splitmix64_at(seed, 2 * j) >> 11) * 0x1.0p-53;
    const double u2 = (double)(splitmix64_at(seed, 2 * j + 1) >> 11) * 0x1.0p-53;
    const double r = std::sqrt(-2.0 * std::log1p(-u1));
    h_out[2 * j] = r * std::cos(two_pi * u2);
    if (2 * j + 1 < count) h_out[2 * j + 1] = r * std::sin(two_pi * u2);
  }
}

veckm_status veckm_create(veckm_ctx **out, const veckm_config *cfg) {
  g_err[0] = 0;
  if (!out || !cfg) return fail(VECKM_EINVAL, "null argument");
  *out = nullptr;
  if (cfg->width < 1 || cfg->width > 32767 || cfg->height < 1 || cfg->height > 32767)
    return fail(VECKM_EINVAL, "sensor size %dx%d outside 1..32767", cfg->width, cfg->height);
  if (!valid_D(cfg->D)) return fail(VECKM_EINVAL, "D=%d not in {64,128,192,256}", cfg->D);
  if (cfg->dx < 0 || cfg->dx > 64 || cfg->dy < 0 || cfg->dy > 64)
    return fail(VECKM_EINVAL, "window radii (%d,%d) outside 0..64", cfg->dx, cfg->dy);
  if (cfg->hidden != 128) return fail(VECKM_EINVAL, "hidden=%d; this build supports 128", cfg->hidden);
  // the pooling walker streams three windows of D/2 float4 units per warp through shared memory
  if ((size_t)3 * (2 * std::max(cfg->dx, cfg->dy) + 2) * (cfg->D / 2) * 16 > 220 * 1024)
    return fail(VECKM_EUNSUPPORTED, "window %dx%d too large for D=%d", 2 * cfg->dx + 1,
                2 * cfg->dy + 1, cfg->D);
  if (cfg->dt_us <= 0) return fail(VECKM_EINVAL, "dt_us must be positive");
  const int64_t span = cfg->t_span_us > 0 ? cfg->t_span_us : 2 * cfg->dt_us;
  if (span >= ((int64_t)1 << 32)) return fail(VECKM_EINVAL, "t_span_us too large");
  if (!cfg->h_W1 || !cfg->h_b1 || !cfg->h_W2 || !cfg->h_b2)
    return fail(VECKM_EINVAL, "perceptron weights are required");
  const uint32_t known = VECKM_MLP_BF16 | VECKM_MLP_FP16;
  if ((cfg->flags & ~(known | VECKM_ACC_FP16)) ||
      ((cfg->flags & VECKM_MLP_BF16) && (cfg->flags & VECKM_MLP_FP16)) ||
      ((cfg->flags & VECKM_ACC_FP16) && !(cfg->flags & known)))
    return fail(VECKM_EINVAL, "bad flags 0x%x", cfg->flags);
  if ((cfg->flags & known) && cfg->D > 128)
    return fail(VECKM_EUNSUPPORTED, "tensor-core perceptron supports D <= 128");

  veckm_ctx *c = new (std::nothrow) veckm_ctx();
  if (!c) return fail(VECKM_ENOMEM, "host allocation");
  cudaGetDevice(&c->device);
  Geometry &g = c->g;
  g.W = cfg->width; g.H = cfg->height; g.D = cfg->D; g.U = cfg->D / 2;
  g.dx = cfg->dx; g.dy = cfg->dy;
  c->hidden = cfg->hidden;
  c->flags = cfg->flags;
  c->dt_us = cfg->dt_us;
  c->t_span = span;
  c->sigma2 = cfg->sigma2 > 0 ? cfg->sigma2 : 25.0;
  const int D = g.D;
  c->T.resize(D); c->X.resize(D); c->Y.resize(D);
  if (cfg->h_T && cfg->h_X && cfg->h_Y) {
    std::copy(cfg->h_T, cfg->h_T + D, c->T.begin());
    std::copy(cfg->h_X, cfg->h_X + D, c->X.begin());
    std::copy(cfg->h_Y, cfg->h_Y + D, c->Y.begin());
  } else if (cfg->h_T || cfg->h_X || cfg->h_Y) {
    delete c;
    return fail(VECKM_EINVAL, "give all of h_T, h_X, h_Y or none");
  } else {
    const double sd = std::sqrt(c->sigma2);
    veckm_normals(cfg->freq_seed, D, c->T.data());
    veckm_normals(cfg->freq_seed + 1, D, c->X.data());
    veckm_normals(cfg->freq_seed + 2, D, c->Y.data());
    for (int d = 0; d < D; ++d) { c->T[d] *= sd; c->X[d] *= sd; c->Y[d] *= sd; }
  }
  // tables
  const double wx = cfg->dx > 0 ? 1.0 / cfg->dx : 0.0, wy = cfg->dy > 0 ? 1.0 / cfg->dy : 0.0;
  const double wt = 1.0 / (double)cfg->dt_us;
  std::vector<float> htx = phase_rows(c->X, wx, -cfg->dx, (int64_t)g.W + cfg->dx, 1);
  std::vector<float> hty = phase_rows(c->Y, wy, 0, g.H, 1);
  std::vector<float> hsx = phase_rows(c->X, wx, 1, 1, 1);
  std::vector<float> hsy = phase_rows(c->Y, wy, 1, 1, 1);
  std::vector<float> hrx = phase_rows(c->X, wx, -cfg->dx, 2 * (int64_t)cfg->dx + 1, 1);
  std::vector<float> hry = phase_rows(c->Y, wy, -cfg->dy, 2 * (int64_t)cfg->dy + 1, 1);
  // frequencies in turns per unit (microsecond, pixel), reduced to
  // [-1/2, 1/2], as 64-bit fixed point (the device reduces q * w mod 1
  // exactly for an integer q)
  auto fixed_turns = [](double freq_per_unit) {
    const double w = freq_per_unit / (2.0 * 3.14159265358979323846);
    const double r = w - std::nearbyint(w);
    const double q = std::ldexp(r, 64);
    const int64_t qi = q >= 9.2233720368547758e18 ? INT64_MAX : (int64_t)std::llround(q);
    const uint64_t u = (uint64_t)qi;
    return make_uint2((uint32_t)(u & 0xffffffffu), (uint32_t)(u >> 32));
  };
  std::vector<uint2> hwt(D), hwxy(2 * (size_t)D);
  for (int d = 0; d < D; ++d) {
    hwt[d] = fixed_turns(c->T[d] * wt);
    hwxy[d] = fixed_turns(c->X[d] * wx);
    hwxy[D + d] = fixed_turns(c->Y[d] * wy);
  }
  c->hwt = hwt;
  const int IN = 2 * D;
  c->hW1.assign(cfg->h_W1, cfg->h_W1 + (size_t)c->hidden * IN);
  c->hb1.assign(cfg->h_b1, cfg->h_b1 + c->hidden);
  c->hW2.assign(cfg->h_W2, cfg->h_W2 + 2 * (size_t)c->hidden);
  c->hb2.assign(cfg->h_b2, cfg->h_b2 + 2);
  std::vector<float> hW1t((size_t)IN * c->hidden);
  for (int h = 0; h < c->hidden; ++h)
    for (int k = 0; k < IN; ++k) hW1t[(size_t)k * c->hidden + h] = c->hW1[(size_t)h * IN + k];
  std::vector<uint16_t> hW1h = w1_core_matrix(c->hW1, c->hidden, IN, (c->flags & VECKM_MLP_FP16) != 0);
  std::vector<uint16_t> hW2h = w2_core_matrix(c->hW2, c->hidden);
  if ((c->flags & (VECKM_MLP_BF16 | VECKM_MLP_FP16)) && !tc_head_range_ok(c)) {
    delete c;
    return fail(VECKM_EUNSUPPORTED, "tensor-core perceptron: sum_c |W1_jc| + |b1_j| or |W2| "
                "reaches 32768, beyond the FP16 range its second layer needs");
  }

  const size_t P = (size_t)g.W * g.H;
  cudaError_t e = cudaSuccess;
#define VK_TRY(expr)                    \
  do {                                  \
    if (e == cudaSuccess) e = (expr);   \
  } while (0)
  VK_TRY(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  VK_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  VK_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  VK_TRY(cudaEventCreateWithFlags(&c->ev_fork0, cudaEventDisableTiming));
  VK_TRY(cudaEventCreateWithFlags(&c->ev_zero, cudaEventDisableTiming));
  VK_TRY(dalloc(&c->tx, ((size_t)g.W + cfg->dx) * g.U));
  VK_TRY(dalloc(&c->sx, (size_t)g.U));
  VK_TRY(dalloc(&c->sy, (size_t)g.U));
  VK_TRY(dalloc(&c->ty, (size_t)g.H * g.U));
  VK_TRY(dalloc(&c->rx, (2 * (size_t)cfg->dx + 1) * g.U));
  VK_TRY(dalloc(&c->ry, (2 * (size_t)cfg->dy + 1) * g.U));
  VK_TRY(dalloc(&c->wt, (size_t)D));
  VK_TRY(dalloc(&c->wxy, 2 * (size_t)D));
  VK_TRY(dalloc(&c->W1, (size_t)c->hidden * IN));
  VK_TRY(dalloc(&c->W1t, (size_t)c->hidden * IN));
  VK_TRY(dalloc(&c->W1h, (size_t)c->hidden * IN));
  VK_TRY(dalloc(&c->W2h, hW2h.size()));
  VK_TRY(dalloc(&c->b1, (size_t)c->hidden));
  VK_TRY(dalloc(&c->W2, (size_t)2 * c->hidden));
  VK_TRY(dalloc(&c->b2, 2));
  VK_TRY(dalloc(&c->acc, P * g.U));
  VK_TRY(dalloc(&c->hbuf, P * g.U));
  VK_TRY(dalloc(&c->cnt, P));
  VK_TRY(dalloc(&c->cnt_tmp, P));
  VK_TRY(dalloc(&c->ncnt, P));
  VK_TRY(dalloc(&c->off, P + 1));
  VK_TRY(dalloc(&c->cur, P));
  VK_TRY(dalloc(&c->bsum, (size_t)scan_blocks((int64_t)P)));
  VK_TRY(dalloc(&c->total, 1));
  {  // a call's geometry is at most the context's, so at most min(P, max) buckets
    const size_t nbmax = std::min<size_t>(P, (size_t)bucket_sort_max_buckets());
    VK_TRY(dalloc(&c->bhist, 2 * nbmax * bucket_sort_max_tiles()));  // counts, then prefixes
    VK_TRY(dalloc(&c->btot, nbmax));
  }
  VK_TRY(dalloc(&c->err, 1));
  VK_TRY(host_malloc(reinterpret_cast<void **>(&c->h_err), sizeof(int)));
  VK_TRY(cudaMemcpy(c->tx, htx.data(), htx.size() * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->ty, hty.data(), hty.size() * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->sx, hsx.data(), hsx.size() * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->sy, hsy.data(), hsy.size() * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->rx, hrx.data(), hrx.size() * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->ry, hry.data(), hry.size() * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->wt, hwt.data(), hwt.size() * sizeof(uint2), cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->wxy, hwxy.data(), hwxy.size() * sizeof(uint2), cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->W1, c->hW1.data(), c->hW1.size() * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->W1t, hW1t.data(), hW1t.size() * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->W1h, hW1h.data(), hW1h.size() * 2, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->W2h, hW2h.data(), hW2h.size() * 2, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->b1, cfg->h_b1, (size_t)c->hidden * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->W2, cfg->h_W2, (size_t)2 * c->hidden * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemcpy(c->b2, cfg->h_b2, 2 * 4, cudaMemcpyHostToDevice));
  VK_TRY(cudaMemset(c->err, 0, sizeof(int)));
#undef VK_TRY
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    return cuda_fail(e, "veckm_create");
  }
  *out = c;
  return VECKM_OK;
}

void veckm_destroy(veckm_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  free_all(c);
  delete c;
}

int64_t veckm_debug_fail_alloc(int64_t fail_at) {
  const long long n = veckm::g_alloc_count.exchange(0);
  veckm::g_alloc_fail_at.store(fail_at >= 0 ? fail_at : -1);
  return n;
}

veckm_status veckm_debug_checks(int64_t *violations, int32_t *first_line) {
#ifndef VECKM_CHECKED
  (void)violations;
  (void)first_line;
  return fail(VECKM_EUNSUPPORTED, "not the bounds-checked build (build(checked=True))");
#else
  if (!violations || !first_line) return fail(VECKM_EINVAL, "null output");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "waiting for the device");
  int (*readers[])(int *) = {veckm::check_read_kernels, veckm::check_read_head,
                             veckm::check_read_stream};
  int64_t total = 0;
  int32_t first = 0;
  for (int f = 0; f < 3; ++f) {
    int line = 0;
    const int n = readers[f](&line);
    if (n < 0) return cuda_fail(cudaGetLastError(), "reading the check words");
    if (n > 0 && first == 0) first = (f + 1) * 100000 + line;
    total += n;
  }
  *violations = total;
  *first_line = first;
  return VECKM_OK;
#endif
}

veckm_status veckm_set_wait_limit(veckm_ctx *c, int64_t cycles) {
  if (!c) return fail(VECKM_EINVAL, "null context");
  if (cycles < 0) return fail(VECKM_EINVAL, "negative wait limit");
  c->wait_cycles = cycles > 0 ? cycles : kDefaultWaitCycles;
  return VECKM_OK;
}

veckm_status veckm_set_injection(veckm_ctx *c, int32_t what) {
  if (!c) return fail(VECKM_EINVAL, "null context");
  if (what != VECKM_INJECT_NONE && what != VECKM_INJECT_HEAD_STALL)
    return fail(VECKM_EINVAL, "unknown injection %d", what);
  c->inject = what;
  return VECKM_OK;
}

veckm_status veckm_set_mlp_mode(veckm_ctx *c, uint32_t flags) {
  if (!c) return fail(VECKM_EINVAL, "null context");
  if (c->live_plans > 0) return fail(VECKM_EBUSY, "captured plans use this context's mode");
  const uint32_t known = VECKM_MLP_BF16 | VECKM_MLP_FP16;
  if ((flags & ~(known | VECKM_ACC_FP16)) || ((flags & VECKM_MLP_BF16) && (flags & VECKM_MLP_FP16)) ||
      ((flags & VECKM_ACC_FP16) && !(flags & known)))
    return fail(VECKM_EINVAL, "bad flags 0x%x", flags);
  if ((flags & known) && c->g.D > 128)
    return fail(VECKM_EUNSUPPORTED, "tensor-core perceptron supports D <= 128");
  if ((flags & known) && !tc_head_range_ok(c))
    return fail(VECKM_EUNSUPPORTED, "tensor-core perceptron: sum_c |W1_jc| + |b1_j| or |W2| "
                "reaches 32768, beyond the FP16 range its second layer needs");
  if (flags & known) {
    std::vector<uint16_t> h = w1_core_matrix(c->hW1, c->hidden, 2 * c->g.D, (flags & VECKM_MLP_FP16) != 0);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c->W1h, h.data(), h.size() * 2, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "veckm_set_mlp_mode");
  }
  c->flags = flags;
  return VECKM_OK;
}

veckm_status veckm_encode(veckm_ctx *c, const int16_t *x, const int16_t *y, const uint32_t *t,
                          int64_t n, uint32_t t_ref, const int64_t *K, int64_t nK, float *emb,
                          void *stream) {
  return run(c, x, y, t, n, t_ref, K, nK, emb, (cudaStream_t)stream, Out::Emb);
}

veckm_status veckm_predict(veckm_ctx *c, const int16_t *x, const int16_t *y, const uint32_t *t,
                           int64_t n, uint32_t t_ref, const int64_t *K, int64_t nK, float *flow,
                           void *stream) {
  return run(c, x, y, t, n, t_ref, K, nK, flow, (cudaStream_t)stream, Out::Flow);
}

veckm_status veckm_sync_status(veckm_ctx *c, void *stream) {
  if (!c) return fail(VECKM_EINVAL, "null context");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(c->h_err, c->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "veckm_sync_status");
  const int w = *c->h_err;
  if (w & ERR_TIMEOUT) return fail(VECKM_ETIMEOUT, "a bounded device wait ran out");
  if (w & ERR_CAPACITY) return fail(VECKM_EBUSY, "a stream's window held more events than its ring");
  if (w & (ERR_EVENT_RANGE | ERR_INDEX_RANGE))
    return fail(VECKM_ERANGE, "%s%s", (w & ERR_EVENT_RANGE) ? "event outside the sensor or time span; " : "",
                (w & ERR_INDEX_RANGE) ? "index in K outside [0, n)" : "");
  return VECKM_OK;
}

veckm_status veckm_predict_host(veckm_ctx *c, const int16_t *hx, const int16_t *hy,
                                const uint32_t *ht, int64_t n, uint32_t t_ref,
                                const int64_t *hK, int64_t nK, float *hflow, void *stream) {
  veckm_status st = check_events_args(c, hx, hy, ht, n, hK, nK, hflow);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bx = al(n * 2), by = al(n * 2), bt = al(n * 4), bk = hK ? al(nK * 8) : 0,
               bf = al(nK * 8);
  const size_t need = bx + by + bt + bk + bf;
  if (need > c->st_cap) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (c->st_buf) cudaFree(c->st_buf);
    c->st_buf = nullptr;
    c->st_cap = 0;
    if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&c->st_buf), need);
    if (e != cudaSuccess) return cuda_fail(e, "staging buffers");
    c->st_cap = need;
  }
  char *b = (char *)c->st_buf;
  int16_t *dx = (int16_t *)b;
  int16_t *dy = (int16_t *)(b + bx);
  uint32_t *dt = (uint32_t *)(b + bx + by);
  int64_t *dK = hK ? (int64_t *)(b + bx + by + bt) : nullptr;
  float *df = (float *)(b + bx + by + bt + bk);
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    e = cudaMemcpyAsync(dx, hx, n * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, hy, n * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt, ht, n * 4, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess && hK && nK > 0) e = cudaMemcpyAsync(dK, hK, nK * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
  st = veckm_predict(c, dx, dy, dt, n, t_ref, dK, nK, df, stream);
  if (st) return st;
  if (nK > 0) {
    e = cudaMemcpyAsync(hflow, df, nK * 8, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
  }
  return veckm_sync_status(c, stream);
}

veckm_status veckm_get_frequencies(const veckm_ctx *c, double *T, double *X, double *Y) {
  if (!c || !T || !X || !Y) return fail(VECKM_EINVAL, "null argument");
  std::copy(c->T.begin(), c->T.end(), T);
  std::copy(c->X.begin(), c->X.end(), X);
  std::copy(c->Y.begin(), c->Y.end(), Y);
  return VECKM_OK;
}

veckm_status veckm_set_timing(veckm_ctx *c, int enable) {
  if (!c) return fail(VECKM_EINVAL, "null context");
  c->timing = enable != 0;
  return VECKM_OK;
}

veckm_status veckm_stage_times(veckm_ctx *c, double *ms, int64_t *launches, int nstage) {
  if (!c || !ms || nstage < 1) return fail(VECKM_EINVAL, "bad argument");
  for (auto &evs : c->pending) {
    if (evs.size() == kStages + 1) {
      cudaError_t e = cudaEventSynchronize(evs.back());
      if (e != cudaSuccess) return cuda_fail(e, "timing events");
      for (int i = 0; i < kStages; ++i) {
        float t = 0.f;
        cudaEventElapsedTime(&t, evs[i], evs[i + 1]);
        c->stage_ms[i] += t;
        c->stage_launch[i] += 1;
      }
    }
    for (cudaEvent_t e : evs) c->ev_free.push_back(e);
  }
  c->pending.clear();
  for (int i = 0; i < nstage && i < kStages; ++i) {
    ms[i] = c->stage_ms[i];
    if (launches) launches[i] = c->stage_launch[i];
    c->stage_ms[i] = 0;
    c->stage_launch[i] = 0;
  }
  return VECKM_OK;
}

int veckm_last_launch_count(const veckm_ctx *c) { return c ? c->last_launches : 0; }

veckm_status veckm_set_path(veckm_ctx *c, int32_t path) {
  if (!c) return fail(VECKM_EINVAL, "null context");
  if (path != VECKM_PATH_AUTO && path != VECKM_PATH_DENSE && path != VECKM_PATH_DIRECT)
    return fail(VECKM_EINVAL, "unknown path %d", path);
  c->path = path;
  return VECKM_OK;
}

int veckm_last_path(const veckm_ctx *c) { return c ? c->last_path : 0; }

veckm_status veckm_set_path_model(veckm_ctx *c, double pixel_ns, double flow_dense_ns,
                                  double flow_window_ns) {
  if (!c) return fail(VECKM_EINVAL, "null context");
  if (!(pixel_ns > 0) || !(flow_dense_ns >= 0) || !(flow_window_ns > 0))
    return fail(VECKM_EINVAL, "model coefficients must be positive");
  c->k_pixel = pixel_ns * 1e-9;
  c->k_flow_dense = flow_dense_ns * 1e-9;
  c->k_flow_window = flow_window_ns * 1e-9;
  return VECKM_OK;
}

}  // extern "C"

// Read-only view of a context for other translation units of the library.
namespace veckm {

bool ctx_view(const veckm_ctx *c, CtxView *v) {
  if (!c || !v) return false;
  v->g = c->g;
  v->tb = c->tables();
  v->acc = c->acc;
  v->hbuf = c->hbuf;
  v->cnt = c->cnt;
  v->cnt_tmp = c->cnt_tmp;
  v->ncnt = c->ncnt;
  v->off = c->off;
  v->cur = c->cur;
  v->bsum = c->bsum;
  v->total = c->total;
  v->err = c->err;
  v->t_span = c->t_span;
  v->tn = c->tune_for(c->g);
  return true;
}

veckm_status report(veckm_status st, const char *msg) { return fail(st, "%s", msg); }

cudaError_t dev_malloc(void **p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t host_malloc(void **p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

void grids_dirty(veckm_ctx *c) {
  if (c) c->zero_grid = -1;
}

veckm_status fail_msg(veckm_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

veckm_status fail_cuda(cudaError_t e, const char *what) { return cuda_fail(e, what); }

}  // namespace veckm
