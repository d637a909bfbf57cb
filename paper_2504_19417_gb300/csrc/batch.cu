// Batches of slices on one canvas, CUDA-graph plans and the pooling autotuner.
//
// A batch of slices (each on its own sensor, of any size up to the context's)
// is laid out on a canvas: one large virtual sensor holding every slice's
// sensor at an offset (ox, oy), at least dx columns and dy rows away from any
// other.  The encoding (Eq. emb, computed through Eq. 16-17) depends on pixel
// coordinates only through x_j - x_k and y_j - y_k inside a window of radii
// (dx, dy), so a sensor shifted by (ox, oy) encodes exactly as on its own and
// no window reaches across a gap.  Times enter only as t_j - t_k inside a
// window as well, so each event's time is stored relative to its own slice's
// start.  One mapping kernel writes every event's canvas coordinates; the
// canvas then runs through the single-slice pipeline, one launch per stage for
// the whole batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "ctx.h"

namespace veckm {
namespace {

using SliceDev = CanvasSlice;  // one slice as the mapping kernel sees it

constexpr int kMapThreads = 256;
constexpr int kMapPer = 4;  // events per thread
constexpr int kMapBlock = kMapThreads * kMapPer;

// Canvas event j of slice s: (x + ox, y + oy, t - t_ref), or x = -1 for an
// event outside its sensor or time span (the pipeline then reports it and
// writes its outputs as zeros).
__global__ void __launch_bounds__(kMapThreads)
    k_canvas_map(const SliceDev *__restrict__ tab, int ns, int16_t *__restrict__ cx,
                 int16_t *__restrict__ cy, uint32_t *__restrict__ ct, uint32_t t_span) {
  __shared__ int s_slice;
  if (threadIdx.x == 0) {  // the last slice whose first block is at or before this one
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tab[mid].blk <= (long long)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_slice = lo;
  }
  __syncthreads();
  const SliceDev d = tab[s_slice];
  const long long j0 = ((long long)blockIdx.x - d.blk) * kMapBlock + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kMapPer; ++k) {
    const long long j = j0 + (long long)k * kMapThreads;
    if (j >= d.n) break;
    const int x = d.x[j], y = d.y[j];
    const uint32_t t = d.t[j];
    const uint32_t tr = t - d.t_ref;
    const bool ok = x >= 0 && x < d.W && y >= 0 && y < d.H && t >= d.t_ref && tr <= t_span;
    const long long o = d.off + j;
    cx[o] = ok ? (int16_t)(x + d.ox) : (int16_t)-1;
    cy[o] = ok ? (int16_t)(y + d.oy) : (int16_t)0;
    ct[o] = tr;
  }
}

struct Prepared {
  Geometry g{};
  int64_t N = 0;
  long long blocks = 0;
  std::vector<SliceDev> tab;
};

veckm_status layout(int32_t ns, const int32_t *w, const int32_t *h, int32_t gx, int32_t gy,
                    int32_t max_width, int32_t *ox, int32_t *oy, int64_t *cw, int64_t *ch) {
  if (ns < 0 || gx < 0 || gy < 0 || max_width < 1)
    return fail_msg(VECKM_EINVAL, "bad layout arguments");
  if (ns > 0 && (!w || !h || !ox || !oy)) return fail_msg(VECKM_EINVAL, "null layout array");
  for (int32_t i = 0; i < ns; ++i) {
    if (w[i] < 1 || h[i] < 1) return fail_msg(VECKM_EINVAL, "slice %d has size %dx%d", i, w[i], h[i]);
    if (w[i] > max_width)
      return fail_msg(VECKM_EINVAL, "slice %d is %d wide; the canvas is %d", i, w[i], max_width);
  }
  std::vector<int32_t> order(ns);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return h[a] > h[b]; });
  int64_t x = 0, y = 0, shelf = 0, wmax = 0;
  for (int32_t i : order) {
    if (x > 0 && x + w[i] > max_width) {  // next shelf
      y += shelf + gy;
      x = 0;
      shelf = 0;
    }
    ox[i] = (int32_t)x;
    oy[i] = (int32_t)std::min<int64_t>(y, INT32_MAX);
    wmax = std::max<int64_t>(wmax, x + w[i]);
    shelf = std::max<int64_t>(shelf, h[i]);
    x += w[i] + gx;
  }
  *cw = wmax;
  *ch = ns > 0 ? y + shelf : 0;
  return VECKM_OK;
}

veckm_status prepare(veckm_ctx *c, const veckm_slice *sl, int32_t ns, Prepared *p) {
  if (!c) return fail_msg(VECKM_EINVAL, "null context");
  if (ns < 0 || (ns > 0 && !sl)) return fail_msg(VECKM_EINVAL, "bad slice array");
  std::vector<int32_t> w(ns), h(ns), ox(ns), oy(ns);
  int64_t N = 0;
  for (int32_t i = 0; i < ns; ++i) {
    const veckm_slice &s = sl[i];
    if (s.n < 0) return fail_msg(VECKM_EINVAL, "slice %d: negative n", i);
    if (s.n > 0 && (!s.d_x || !s.d_y || !s.d_t))
      return fail_msg(VECKM_EINVAL, "slice %d: null event buffer", i);
    if (s.width < 1 || s.height < 1 || s.width > c->g.W || s.height > c->g.H)
      return fail_msg(VECKM_EINVAL, "slice %d: sensor %dx%d outside 1..%dx%d", i, s.width,
                      s.height, c->g.W, c->g.H);
    N += s.n;
    if (N > VECKM_MAX_EVENTS)
      return fail_msg(VECKM_EINVAL, "more than %lld events in one batch", (long long)VECKM_MAX_EVENTS);
    w[i] = s.width;
    h[i] = s.height;
  }
  int64_t cw = 0, ch = 0;
  if (veckm_status st = layout(ns, w.data(), h.data(), c->g.dx, c->g.dy, c->g.W, ox.data(),
                               oy.data(), &cw, &ch))
    return st;
  if (ch > c->g.H)
    return fail_msg(VECKM_EBUSY, "the batch needs a %lldx%lld canvas; the context is %dx%d",
                    (long long)cw, (long long)ch, c->g.W, c->g.H);
  p->g = c->g;
  p->g.W = (int)std::max<int64_t>(cw, 1);
  p->g.H = (int)std::max<int64_t>(ch, 1);
  p->N = N;
  p->tab.resize(ns);
  long long off = 0, blk = 0;
  for (int32_t i = 0; i < ns; ++i) {
    const veckm_slice &s = sl[i];
    p->tab[i] = SliceDev{s.d_x, s.d_y, s.d_t, (long long)s.n, off, blk, s.t_ref_us,
                         s.width, s.height, ox[i], oy[i]};
    off += s.n;
    blk += (s.n + kMapBlock - 1) / kMapBlock;
  }
  p->blocks = blk;
  return VECKM_OK;
}

template <typename T>
cudaError_t grow(T **p, int64_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  return dev_malloc(reinterpret_cast<void **>(p), (size_t)std::max<int64_t>(count, 1) * sizeof(T));
}

// Canvas event buffers, the device slice table and the records for p.
veckm_status reserve(veckm_ctx *c, const Prepared &p, cudaStream_t s) {
  const size_t tab_bytes = p.tab.size() * sizeof(SliceDev);
  const bool more_events = p.N > c->canvas_cap, more_tab = tab_bytes > c->slice_tab_cap;
  if ((more_events || more_tab) && c->live_plans > 0)
    return fail_msg(VECKM_EBUSY, "batch buffers cannot grow while a captured plan uses them");
  if (more_events || more_tab) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && more_events) {
      e = grow(&c->cx, p.N);
      if (e == cudaSuccess) e = grow(&c->cy, p.N);
      if (e == cudaSuccess) e = grow(&c->ct, p.N);
      c->canvas_cap = e == cudaSuccess ? p.N : 0;
    }
    if (e == cudaSuccess && more_tab) {
      char *q = static_cast<char *>(c->slice_tab);
      e = grow(&q, (int64_t)tab_bytes);
      c->slice_tab = q;
      c->slice_tab_cap = e == cudaSuccess ? tab_bytes : 0;
    }
    if (e != cudaSuccess) return fail_cuda(e, "batch buffers");
  }
  return ensure_records(c, p.N, s);
}

veckm_status launch_map(veckm_ctx *c, const Prepared &p, cudaStream_t s) {
  if (p.blocks == 0) return VECKM_OK;
  k_canvas_map<<<(unsigned)p.blocks, kMapThreads, 0, s>>>(
      static_cast<const SliceDev *>(c->slice_tab), (int)p.tab.size(), c->cx, c->cy, c->ct,
      (uint32_t)c->t_span);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VECKM_OK : fail_cuda(e, "canvas mapping launch");
}

// A batch of one slice: the layout puts it at the canvas origin and sizes the
// canvas to it, so the canvas is that slice and its events need no mapping
// (the pipeline applies the mapping kernel's test of sensor and time span).
bool single_slice(const Prepared &p) {
  return p.tab.size() == 1 && p.tab[0].ox == 0 && p.tab[0].oy == 0 && p.tab[0].W == p.g.W &&
         p.tab[0].H == p.g.H;
}

veckm_status run_canvas(veckm_ctx *c, const Prepared &p, float *out, bool flow, cudaStream_t s) {
  if (single_slice(p)) {
    const SliceDev &d = p.tab[0];
    const Events ev{d.x, d.y, d.t, d.n, d.t_ref, (uint32_t)c->t_span};
    return run_pipeline(c, p.g, ev, nullptr, p.N, out, flow, s, c->tune_for(p.g));
  }
  if (veckm_status st = launch_map(c, p, s)) return st;
  const Events ev{c->cx, c->cy, c->ct, p.N, 0u, (uint32_t)c->t_span};
  // the pooling passes skip what lies away from every slice (canvas gaps)
  Geometry g = p.g;
  g.canvas = static_cast<const SliceDev *>(c->slice_tab);
  g.ncanvas = (int)p.tab.size();
  veckm_status st = run_pipeline(c, g, ev, nullptr, p.N, out, flow, s, c->tune_for(p.g));
  if (st == VECKM_OK && p.blocks > 0) c->last_launches += 1;
  return st;
}

veckm_status batch_call(veckm_ctx *c, const veckm_slice *sl, int32_t ns, float *out, bool flow,
                        cudaStream_t s) {
  Prepared p;
  if (veckm_status st = prepare(c, sl, ns, &p)) return st;
  c->last_launches = 0;
  if (p.N == 0) return VECKM_OK;
  if (!out) return fail_msg(VECKM_EINVAL, "null output buffer");
  if (veckm_status st = reserve(c, p, s)) return st;
  if (single_slice(p)) return run_canvas(c, p, out, flow, s);  // no slice table to upload
  const size_t bytes = p.tab.size() * sizeof(SliceDev);
  cudaError_t e = cudaSuccess;
  if (c->tab_copied) e = cudaEventSynchronize(c->tab_copied);  // the pinned copy is free again
  if (e == cudaSuccess && bytes > c->h_slice_tab_cap) {
    if (c->h_slice_tab) cudaFreeHost(c->h_slice_tab);
    c->h_slice_tab = nullptr;
    c->h_slice_tab_cap = 0;
    e = host_malloc(reinterpret_cast<void **>(&c->h_slice_tab), bytes);
    if (e == cudaSuccess) c->h_slice_tab_cap = bytes;
  }
  if (e == cudaSuccess && !c->tab_copied)
    e = cudaEventCreateWithFlags(&c->tab_copied, cudaEventDisableTiming);
  if (e != cudaSuccess) return fail_cuda(e, "slice table staging");
  std::memcpy(c->h_slice_tab, p.tab.data(), bytes);
  e = cudaMemcpyAsync(c->slice_tab, c->h_slice_tab, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(c->tab_copied, s);
  if (e != cudaSuccess) return fail_cuda(e, "slice table upload");
  return run_canvas(c, p, out, flow, s);
}

// Times one pooling launch shape: the least of a few runs (after one warm-up).
float time_shape(cudaStream_t s, cudaEvent_t a, cudaEvent_t b, int (*go)(void *, cudaStream_t),
                 void *arg) {
  if (go(arg, s) < 0) {
    cudaGetLastError();
    return -1.f;
  }
  float best = -1.f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(a, s);
    if (go(arg, s) < 0) {
      cudaGetLastError();
      return -1.f;
    }
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (best < 0.f || ms < best) best = ms;
  }
  return best;
}

struct TuneArg {
  veckm_ctx *c;
  Geometry g;
  Tune tn;
  bool cols;
};

int tune_go(void *p, cudaStream_t s) {
  const TuneArg &a = *static_cast<TuneArg *>(p);
  const Tables tb = a.c->tables();
  if (!a.cols) return launch_pool_rows(a.g, tb, a.c->acc, a.c->hbuf, s, a.tn);
  if (a.c->flags & VECKM_ACC_FP16)
    return launch_pool_cols_half(a.g, tb, a.c->hbuf, a.c->ncnt, a.c->acc, s, a.tn);
  return launch_pool_cols(a.g, tb, a.c->hbuf, a.c->acc, s, a.tn);
}

veckm_status autotune(veckm_ctx *c, const Geometry &g, cudaStream_t s, int32_t *tuned) {
  grids_dirty(c);  // the timing runs write both grids
  const int segs[] = {2, 3, 4, 6, 8, 12};
  const int wpbs[] = {1, 2, 3, 4};
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return fail_cuda(e, "autotune events");
  }
  Tune best{};
  for (int pass = 0; pass < 2; ++pass) {
    float best_ms = -1.f;
    int best_seg = 0, best_wpb = 0;
    for (int sg : segs)
      for (int wp : wpbs) {
        TuneArg arg{c, g, Tune{}, pass == 1};
        if (pass == 0) { arg.tn.rows_seg = sg; arg.tn.rows_wpb = wp; }
        else { arg.tn.cols_seg = sg; arg.tn.cols_wpb = wp; }
        const float ms = time_shape(s, a, b, tune_go, &arg);
        if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
          best_ms = ms;
          best_seg = sg;
          best_wpb = wp;
        }
      }
    if (pass == 0) { best.rows_seg = best_seg; best.rows_wpb = best_wpb; }
    else { best.cols_seg = best_seg; best.cols_wpb = best_wpb; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e, "autotune");
  const uint32_t acc16 = c->flags & VECKM_ACC_FP16;
  bool found = false;
  for (auto &t : c->tunes)
    if (t.W == g.W && t.H == g.H && t.acc16 == acc16) {
      t.tn = best;
      found = true;
    }
  if (!found) c->tunes.push_back({g.W, g.H, acc16, best});
  if (tuned) {
    tuned[0] = best.rows_seg;
    tuned[1] = best.rows_wpb;
    tuned[2] = best.cols_seg;
    tuned[3] = best.cols_wpb;
  }
  return VECKM_OK;
}

bool tuned_for(const veckm_ctx *c, const Geometry &g) {
  for (const auto &t : c->tunes)
    if (t.W == g.W && t.H == g.H && t.acc16 == (c->flags & VECKM_ACC_FP16)) return true;
  return false;
}

}  // namespace
}  // namespace veckm

using namespace veckm;

// A plan holds one graph that clears the grid its sums go to, or, when the
// captured tensor-core head zeroes the other grid, two graphs with the grids'
// roles swapped: a launch replays the one whose sums go to the grid the
// context knows to be zero (clearing acc first when neither is).
struct veckm_plan {
  veckm_ctx *c = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  bool pingpong = false;
  int64_t units = 0;      // float4 of each grid the canvas uses
  void *h_tab = nullptr;  // pinned slice table read by the graphs' copy nodes
  int kernels = 0;
};

extern "C" {

veckm_status veckm_canvas_layout(int32_t ns, const int32_t *w, const int32_t *h, int32_t gx,
                                 int32_t gy, int32_t max_width, int32_t *ox, int32_t *oy,
                                 int32_t *cw, int32_t *ch) {
  if (!cw || !ch) return fail_msg(VECKM_EINVAL, "null canvas size output");
  int64_t w64 = 0, h64 = 0;
  if (veckm_status st = layout(ns, w, h, gx, gy, max_width, ox, oy, &w64, &h64)) return st;
  if (h64 > INT32_MAX) return fail_msg(VECKM_EINVAL, "canvas taller than 2^31 rows");
  *cw = (int32_t)w64;
  *ch = (int32_t)h64;
  return VECKM_OK;
}

veckm_status veckm_predict_batch(veckm_ctx *c, const veckm_slice *sl, int32_t ns, float *d_flow,
                                 void *stream) {
  return batch_call(c, sl, ns, d_flow, true, (cudaStream_t)stream);
}

veckm_status veckm_encode_batch(veckm_ctx *c, const veckm_slice *sl, int32_t ns, float *d_emb,
                                void *stream) {
  return batch_call(c, sl, ns, d_emb, false, (cudaStream_t)stream);
}

veckm_status veckm_autotune(veckm_ctx *c, int32_t width, int32_t height, void *stream,
                            int32_t *tuned) {
  if (!c) return fail_msg(VECKM_EINVAL, "null context");
  if (width < 1 || height < 1 || width > c->g.W || height > c->g.H)
    return fail_msg(VECKM_EINVAL, "geometry %dx%d outside 1..%dx%d", width, height, c->g.W, c->g.H);
  Geometry g = c->g;
  g.W = width;
  g.H = height;
  return autotune(c, g, (cudaStream_t)stream, tuned);
}

veckm_status veckm_plan_create(veckm_ctx *c, const veckm_slice *sl, int32_t ns, float *d_out,
                               int32_t predict, veckm_plan **out) {
  if (!out) return fail_msg(VECKM_EINVAL, "null plan output");
  *out = nullptr;
  Prepared p;
  if (veckm_status st = prepare(c, sl, ns, &p)) return st;
  if (p.N > 0 && !d_out) return fail_msg(VECKM_EINVAL, "null output buffer");
  veckm_plan *pl = new (std::nothrow) veckm_plan();
  if (!pl) return fail_msg(VECKM_ENOMEM, "host allocation");
  pl->c = c;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  veckm_status st = e == cudaSuccess ? VECKM_OK : fail_cuda(e, "plan stream");
  if (st == VECKM_OK && p.N > 0) st = reserve(c, p, cs);
  if (st == VECKM_OK && p.N > 0 && !tuned_for(c, p.g)) st = autotune(c, p.g, cs, nullptr);
  const size_t bytes = p.tab.size() * sizeof(SliceDev);
  if (st == VECKM_OK && p.N > 0) {
    e = host_malloc(reinterpret_cast<void **>(&pl->h_tab), std::max<size_t>(bytes, 1));
    if (e != cudaSuccess) st = fail_cuda(e, "plan slice table");
    else std::memcpy(pl->h_tab, p.tab.data(), bytes);
  }
  // capture one graph with the sums in grid `grid` (-1: cleared in the graph)
  auto capture = [&](int grid, int slot) -> veckm_status {
    const bool timing = c->timing;
    c->timing = false;
    c->capture_grid = grid;
    c->capture_zeroed = false;
    veckm_status r = VECKM_OK;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) {
      r = fail_cuda(ce, "stream capture");
    } else {
      if (!single_slice(p))
        ce = cudaMemcpyAsync(c->slice_tab, pl->h_tab, bytes, cudaMemcpyHostToDevice, cs);
      r = ce == cudaSuccess ? run_canvas(c, p, d_out, predict != 0, cs)
                            : fail_cuda(ce, "slice table copy");
      cudaGraph_t graph = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
      pl->graph[slot] = graph;
      if (r == VECKM_OK && ee != cudaSuccess) r = fail_cuda(ee, "stream capture");
    }
    c->capture_grid = -1;
    c->timing = timing;
    pl->kernels = c->last_launches;
    if (r == VECKM_OK) {
      ce = cudaGraphInstantiate(&pl->exec[slot], pl->graph[slot], 0);
      if (ce != cudaSuccess) r = fail_cuda(ce, "graph instantiation");
    }
    return r;
  };
  if (st == VECKM_OK && p.N > 0) {
    st = capture(0, 0);
    if (st == VECKM_OK && c->capture_zeroed) {
      pl->pingpong = true;
      pl->units = c->capture_units;
      st = capture(1, 1);
      if (st == VECKM_OK && !c->capture_zeroed) st = fail_msg(VECKM_ECUDA, "plan graphs disagree");
    } else if (st == VECKM_OK) {
      // the head does not zero a grid here: one graph that clears its own
      cudaGraphExecDestroy(pl->exec[0]);
      cudaGraphDestroy(pl->graph[0]);
      pl->exec[0] = nullptr;
      pl->graph[0] = nullptr;
      st = capture(-1, 0);
    }
  }
  if (cs) cudaStreamDestroy(cs);
  if (st != VECKM_OK) {
    for (int k = 0; k < 2; ++k) {
      if (pl->exec[k]) cudaGraphExecDestroy(pl->exec[k]);
      if (pl->graph[k]) cudaGraphDestroy(pl->graph[k]);
    }
    if (pl->h_tab) cudaFreeHost(pl->h_tab);
    delete pl;
    return st;
  }
  c->live_plans += 1;
  *out = pl;
  return VECKM_OK;
}

veckm_status veckm_plan_launch(veckm_plan *pl, void *stream) {
  if (!pl) return fail_msg(VECKM_EINVAL, "null plan");
  if (!pl->exec[0]) return VECKM_OK;  // an empty batch
  veckm_ctx *c = pl->c;
  cudaStream_t s = (cudaStream_t)stream;
  if (!pl->pingpong) {
    grids_dirty(c);  // a replay leaves sums in both grids
    const cudaError_t e = cudaGraphLaunch(pl->exec[0], s);
    return e == cudaSuccess ? VECKM_OK : fail_cuda(e, "graph launch");
  }
  int which = c->zero_grid >= 0 && c->zero_units >= pl->units ? c->zero_grid : -1;
  grids_dirty(c);
  cudaError_t e = cudaSuccess;
  if (which < 0) {
    e = cudaMemsetAsync(c->acc, 0, (size_t)pl->units * sizeof(float4), s);
    which = 0;
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(pl->exec[which], s);
  if (e != cudaSuccess) return fail_cuda(e, "graph launch");
  // the replay's head zeroed the grid its row pass wrote
  c->zero_grid = which == 0 ? 1 : 0;
  c->zero_units = pl->units;
  return VECKM_OK;
}

int veckm_plan_kernel_count(const veckm_plan *pl) { return pl ? pl->kernels : 0; }

void veckm_plan_destroy(veckm_plan *pl) {
  if (!pl) return;
  if (pl->exec[0]) cudaDeviceSynchronize();  // replays still in flight read the pinned table
  for (int k = 0; k < 2; ++k) {
    if (pl->exec[k]) cudaGraphExecDestroy(pl->exec[k]);
    if (pl->graph[k]) cudaGraphDestroy(pl->graph[k]);
  }
  if (pl->h_tab) cudaFreeHost(pl->h_tab);
  if (pl->c) pl->c->live_plans -= 1;
  delete pl;
}

}  // extern "C"
