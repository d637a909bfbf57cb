// The context behind the veckm_ctx handle of the C ABI (private to the
// library's translation units).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "veckm_internal.h"

namespace veckm {
struct HostPipe;  // pipelined host-buffer calls (host_async.cu)
constexpr int kStages = 6;  // sort, pixel sums, pool rows, counts, pool cols, gather
constexpr long long kDefaultWaitCycles = 4000000000LL;  // about 2 s at 2 GHz
}  // namespace veckm

struct veckm_ctx {
  int device = 0;
  veckm::Geometry g{};
  int hidden = 0;
  uint32_t flags = 0;
  int64_t dt_us = 0, t_span = 0;
  double sigma2 = 25.0;
  std::vector<double> T, X, Y;
  // device state
  float4 *tx = nullptr, *ty = nullptr, *sx = nullptr, *sy = nullptr, *rx = nullptr, *ry = nullptr;
  uint2 *wt = nullptr;
  uint2 *wxy = nullptr;  // X then Y frequencies in 64-bit fixed-point turns per pixel
  float *W1 = nullptr, *W1t = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;
  uint16_t *W1h = nullptr;
  uint16_t *W2h = nullptr;  // second layer of the tensor-core head (FP16, 16 x hidden)
  float4 *acc = nullptr, *hbuf = nullptr;
  // Which of the two grids (0: acc, 1: hbuf; -1: neither) is known to hold
  // zeros over its first zero_units float4, in stream order: the tensor-core
  // head zeroes the dead row-pass grid for the next call's per-pixel sums,
  // which then go there instead of clearing a grid first.
  int zero_grid = -1;
  int64_t zero_units = 0;
  // While a plan is captured: the grid (0 or 1) its sums go to without a
  // clear, the head zeroing the other one (-1: clear acc inside the graph);
  // and whether the captured head does zero it, over how many float4.
  int capture_grid = -1;
  bool capture_zeroed = false;
  int64_t capture_units = 0;
  // Side stream of the dense path, forked from and joined back to the
  // caller's stream: the clear of the pixel-sum grid (when no grid is known
  // to be zero) under the sort, and the window counts (which need only the
  // per-pixel counts) under the pixel sums and row pass.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork0 = nullptr, ev_zero = nullptr, ev_fork = nullptr, ev_join = nullptr;
  int *cnt = nullptr, *cnt_tmp = nullptr, *ncnt = nullptr, *err = nullptr;
  int *off = nullptr, *cur = nullptr, *bsum = nullptr, *total = nullptr;
  // pixel-sorted event records (grown on demand), and the bucket sort's
  // records grouped by bucket, per-tile bucket counts and bucket totals
  int2 *rec = nullptr;
  int *rpix = nullptr;
  int4 *brec = nullptr;
  int *bhist = nullptr, *btot = nullptr;
  int64_t rec_cap = 0;
  std::vector<float> hW1;  // host copy (re-encoding on precision switch)
  std::vector<float> hb1, hW2, hb2;  // host copies (kernel parameters)
  std::vector<uint2> hwt;            // host copy of wt (a kernel parameter of the D = 64 head)
  // staging for the host-buffer entry point
  void *st_buf = nullptr;
  size_t st_cap = 0;
  int *h_err = nullptr;  // pinned
  veckm::HostPipe *pipe = nullptr;  // created by the first asynchronous host call
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::vector<cudaEvent_t>> pending;
  double stage_ms[veckm::kStages] = {};
  int64_t stage_launch[veckm::kStages] = {};
  int last_launches = 0;

  // autotuned launch shapes per geometry and pooled-grid storage
  struct TuneEntry {
    int W, H;
    uint32_t acc16;
    veckm::Tune tn;
  };
  std::vector<TuneEntry> tunes;
  // batches: canvas events (grown on demand), the device slice table and a
  // pinned host copy for direct batch calls
  int16_t *cx = nullptr, *cy = nullptr;
  uint32_t *ct = nullptr;
  int64_t canvas_cap = 0;
  void *slice_tab = nullptr, *h_slice_tab = nullptr;
  size_t slice_tab_cap = 0, h_slice_tab_cap = 0;
  cudaEvent_t tab_copied = nullptr;  // the last copy out of h_slice_tab
  int live_plans = 0;                // captured graphs that use this context's buffers
  // dense pooling or direct window form (Eq. runtime): seconds per pixel of
  // the dense passes, per flow of the dense gather, per flow and window pixel
  // of the direct form, measured on GB300 (0.5 M events, 10 k flows, 640x480,
  // 17x17 window; settable with veckm_set_path_model)
  int path = VECKM_PATH_AUTO, last_path = 0;
  // bounded device waits of the tensor-core head, and the test injection
  long long wait_cycles = veckm::kDefaultWaitCycles;
  int inject = VECKM_INJECT_NONE;
  double k_pixel = 0.43e-9, k_flow_dense = 1.53e-9, k_flow_window = 0.077e-9;

  veckm::Tables tables() const { return veckm::Tables{tx, ty, sx, sy, wt, rx, ry}; }
  veckm::Tune tune_for(const veckm::Geometry &gg) const {
    for (const TuneEntry &t : tunes)
      if (t.W == gg.W && t.H == gg.H && t.acc16 == (flags & VECKM_ACC_FP16)) return t.tn;
    return veckm::Tune{};
  }
  veckm::MLP mlp() const {
    return veckm::MLP{W1,     W1t, b1, W2, b2, W1h, hidden, (flags & VECKM_MLP_FP16) ? 1 : 0, 0,
                      hb1.data(), hW2.data(), hb2.data(), W2h, wait_cycles,
                      inject == VECKM_INJECT_HEAD_STALL ? 1 : 0, hwt.data()};
  }
};

namespace veckm {
// Grows the pixel-sorted record buffers to n events (synchronises the stream
// when it reallocates); VECKM_EBUSY while captured plans hold the old ones.
veckm_status ensure_records(veckm_ctx *c, int64_t n, cudaStream_t s);
// The encoder (flow: and the perceptron) for the events ev on geometry g: a
// sensor, or a canvas of packed sensors no larger than the context's.
veckm_status run_pipeline(veckm_ctx *c, const Geometry &g, const Events &ev, const int64_t *K,
                          int64_t nK, float *out, bool flow, cudaStream_t s, const Tune &tn);
// Argument checks shared by the entry points that take events.
veckm_status check_events_args(veckm_ctx *c, const void *x, const void *y, const void *t,
                               int64_t n, const void *K, int64_t nK, const void *out);
// Waits for and frees the asynchronous host pipeline (host_async.cu).
void destroy_pipe(HostPipe *p);
// Error helpers shared by the entry points (veckm.cu).
veckm_status fail_msg(veckm_status st, const char *fmt, ...);
veckm_status fail_cuda(cudaError_t e, const char *what);
}  // namespace veckm
