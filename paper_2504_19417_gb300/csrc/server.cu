// Serving: a native request loop for event packets from many sensors.
//
// Admission: a packet's events (8 bytes each, three 256-byte aligned arrays)
// take a region of a device arena managed as a ring.  Packets leave the ring
// in the order they entered it (batches are formed first come, first served
// and complete in order on one compute stream), so a head and a tail offset
// (and whether the live region wraps past the end) describe it completely.
// A packet that does not fit is refused at once.
// The caller's thread copies an admitted packet's events host-to-device on
// the upload stream and marks it ready; a worker thread forms batches of
// ready packets in arrival order (as many as fit one canvas and the batch
// limits), runs each as one veckm_predict_batch and copies the flows back.
// Two batches can be in flight: the next one is launched while the previous
// one still runs.  The context's error word is copied out and cleared after
// each batch, so an out-of-range event is attributed to its own batch.
//
// With resident windows (window_us > 0) each sensor stream has its own
// context (its sensor size, the server's frequencies and weights) and its
// own sliding-window stream (veckm_stream: exact fixed-point per-pixel sums
// of the window's events, resident on the device) and CUDA stream, created
// with the stream's first packet.  The worker pushes each packet onto its
// sensor's window on that sensor's CUDA stream; packets of different sensors
// overlap on the device (up to kMaxInflightW), complete in any order and are
// reported as they complete, while their arena regions return to the ring in
// arrival order.  A packet's region also holds its flows.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ctx.h"

using veckm::fail_cuda;
using veckm::fail_msg;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kMaxInflight = 2;
constexpr int kMaxInflightW = 64;  // resident windows: packets in flight at once

int64_t al256(int64_t b) { return (b + 255) & ~int64_t(255); }
int64_t footprint(int64_t n) { return 2 * al256(2 * n) + al256(4 * n); }
// resident windows: the events and then the flows (8 bytes per event)
int64_t footprint_w(int64_t n) { return footprint(n) + al256(8 * n); }

struct Pkt {
  veckm_packet p{};
  int64_t off = 0, bytes = 0;  // arena region
  cudaEvent_t uploaded = nullptr;
  bool ready = false;
  Clock::time_point t_submit;
  // resident windows
  uint32_t t_hi = 0;           // the packet's last (largest) time
  int slot = 0;                // pinned error word
  cudaEvent_t start = nullptr, done = nullptr;
  veckm_status launch_st = VECKM_OK;
  bool reported = false;
};

// A sensor stream's resident state (resident windows).
struct Sensor {
  veckm_ctx *ctx = nullptr;
  veckm_stream *st = nullptr;
  cudaStream_t cs = nullptr;
  int32_t W = 0, H = 0;
};

struct Batch {
  std::vector<Pkt> pk;
  cudaEvent_t start = nullptr, done = nullptr;
  int slot = 0;
};

}  // namespace

struct veckm_server {
  veckm_ctx *ctx = nullptr;
  int device = 0;
  // arena ring
  char *arena = nullptr;
  int64_t cap = 0, head = 0, tail = 0, used = 0;
  // batch outputs and per-batch error words
  float *d_flow[kMaxInflight] = {};
  int *h_err = nullptr;  // pinned, one per slot
  int32_t max_packets = 256;
  int64_t max_events = int64_t(1) << 24;
  std::chrono::microseconds window{0};
  cudaStream_t up = nullptr, comp = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pkt> pending;
  std::deque<veckm_completion> done;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<double> lat_ms;
  std::vector<unsigned char> seen_stream;
  veckm_server_stats st{};
  Clock::time_point t_first, t_last;
  bool any = false, stop = false;
  std::thread worker;
  std::deque<Batch> inflight;  // worker thread only
  int next_slot = 0;
  // resident windows
  int32_t window_us = 0;
  int64_t window_cap = int64_t(1) << 22;
  std::mutex sensor_mu;
  std::vector<Sensor *> sensors;  // by stream id (created with a stream's first packet)
  int *h_errw = nullptr;          // pinned, one per packet in flight
  std::deque<Pkt> wf;             // worker thread only: packets in flight, launch order
  int next_wslot = 0;

  // Live packets occupy [tail, head) or, once the ring has wrapped, [tail,
  // wrap_end) and [0, head); both allocation and release go in arrival order.
  bool wrapped = false;
  int64_t wrap_end = 0;
  bool alloc(int64_t bytes, int64_t *off) {  // under mu
    if (bytes > cap) return false;
    if (used == 0) {
      head = tail = 0;
      wrapped = false;
    }
    if (!wrapped) {
      if (cap - head >= bytes) {
        *off = head;
      } else if (tail >= bytes) {  // wrap to the start of the arena
        *off = 0;
        wrap_end = head;
        wrapped = true;
      } else {
        return false;
      }
    } else {
      if (tail - head < bytes) return false;
      *off = head;
    }
    head = *off + bytes;
    used += bytes;
    return true;
  }
  void release(const Pkt &k) {  // under mu, in allocation order
    if (wrapped && k.off < tail) wrapped = false;  // the first packet after the wrap
    tail = k.off + k.bytes;
    used -= k.bytes;
    if (used == 0) {
      head = tail = 0;
      wrapped = false;
    }
  }
  cudaEvent_t take_event() {  // under mu
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }

  void retire(bool block);
  bool launch(std::vector<Pkt> &pk);
  void run();
  // resident windows
  Sensor *sensor_for(const veckm_packet *p, veckm_status *st);
  void retire_w(bool block);
  void launch_w(Pkt &k);
  void run_w();
};

// The sensor state of p's stream, created with the stream's first packet
// (caller's thread).  VECKM_EBUSY if it cannot be allocated; VECKM_EINVAL if
// the stream's sensor size changed.
Sensor *veckm_server::sensor_for(const veckm_packet *p, veckm_status *st) {
  std::lock_guard<std::mutex> lk(sensor_mu);
  Sensor *sn = sensors[p->stream_id];
  if (sn) {
    if (sn->W != p->width || sn->H != p->height) {
      *st = fail_msg(VECKM_EINVAL, "stream %d changed its sensor from %dx%d to %dx%d",
                     p->stream_id, sn->W, sn->H, p->width, p->height);
      return nullptr;
    }
    *st = VECKM_OK;
    return sn;
  }
  sn = new (std::nothrow) Sensor();
  if (!sn) {
    *st = fail_msg(VECKM_EBUSY, "host memory for a stream's state");
    return nullptr;
  }
  sn->W = p->width;
  sn->H = p->height;
  veckm_config c{};
  c.width = p->width;
  c.height = p->height;
  c.D = ctx->g.D;
  c.dx = ctx->g.dx;
  c.dy = ctx->g.dy;
  c.hidden = ctx->hidden;
  c.dt_us = ctx->dt_us;
  c.t_span_us = ctx->t_span;
  c.sigma2 = ctx->sigma2;
  c.h_T = ctx->T.data();
  c.h_X = ctx->X.data();
  c.h_Y = ctx->Y.data();
  c.h_W1 = ctx->hW1.data();
  c.h_b1 = ctx->hb1.data();
  c.h_W2 = ctx->hW2.data();
  c.h_b2 = ctx->hb2.data();
  c.flags = ctx->flags;
  veckm_status s = veckm_create(&sn->ctx, &c);
  if (s == VECKM_OK) s = veckm_stream_create(sn->ctx, window_us, window_cap, &sn->st);
  if (s == VECKM_OK && cudaStreamCreateWithFlags(&sn->cs, cudaStreamNonBlocking) != cudaSuccess)
    s = fail_msg(VECKM_ECUDA, "stream creation");
  if (s == VECKM_OK) s = veckm_autotune(sn->ctx, sn->W, sn->H, sn->cs, nullptr);
  if (s != VECKM_OK) {
    if (sn->st) veckm_stream_destroy(sn->st);
    if (sn->ctx) veckm_destroy(sn->ctx);
    if (sn->cs) cudaStreamDestroy(sn->cs);
    delete sn;
    *st = (s == VECKM_ENOMEM) ? fail_msg(VECKM_EBUSY, "no device memory for stream %d's window",
                                         p->stream_id)
                              : s;
    return nullptr;
  }
  sensors[p->stream_id] = sn;
  *st = VECKM_OK;
  return sn;
}

void veckm_server::launch_w(Pkt &k) {
  Sensor *sn = sensors[k.p.stream_id];  // created at submission
  cudaStream_t cs = sn->cs;
  char *base = arena + k.off;
  const int64_t n = k.p.n;
  const int16_t *x = reinterpret_cast<const int16_t *>(base);
  const int16_t *y = reinterpret_cast<const int16_t *>(base + al256(2 * n));
  const uint32_t *t = reinterpret_cast<const uint32_t *>(base + 2 * al256(2 * n));
  float *f = reinterpret_cast<float *>(base + footprint(n));
  k.slot = next_wslot;
  next_wslot = (next_wslot + 1) % kMaxInflightW;
  cudaEventCreate(&k.start);
  cudaEventCreate(&k.done);
  cudaStreamWaitEvent(cs, k.uploaded, 0);
  cudaEventRecord(k.start, cs);
  k.launch_st = veckm_stream_push(sn->st, x, y, t, n, k.t_hi, f, 1, cs);
  cudaMemcpyAsync(h_errw + k.slot, sn->ctx->err, sizeof(int), cudaMemcpyDeviceToHost, cs);
  cudaMemsetAsync(sn->ctx->err, 0, sizeof(int), cs);
  if (k.launch_st == VECKM_OK)
    cudaMemcpyAsync(k.p.h_flow, f, (size_t)n * 8, cudaMemcpyDeviceToHost, cs);
  cudaEventRecord(k.done, cs);
  wf.push_back(k);
}

// Reports every finished packet (in any order) and returns the arena regions
// at the front of the ring whose packets have been reported.
void veckm_server::retire_w(bool block) {
  if (block && !wf.empty()) {
    for (Pkt &k : wf)
      if (!k.reported) {
        cudaEventSynchronize(k.done);
        break;
      }
  }
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lk(mu);
  bool any_done = false;
  for (Pkt &k : wf) {
    if (k.reported || cudaEventQuery(k.done) == cudaErrorNotReady) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, k.start, k.done);
    const int w = h_errw[k.slot];
    const veckm_status status =
        k.launch_st != VECKM_OK ? k.launch_st
        : (w & veckm::ERR_TIMEOUT) ? VECKM_ETIMEOUT
        : (w & veckm::ERR_CAPACITY) ? VECKM_EBUSY
        : (w & (veckm::ERR_EVENT_RANGE | veckm::ERR_INDEX_RANGE)) ? VECKM_ERANGE : VECKM_OK;
    const double lat = std::chrono::duration<double, std::milli>(now - k.t_submit).count();
    done.push_back(veckm_completion{k.p.tag, k.p.stream_id, status, k.p.n, lat, 1});
    lat_ms.push_back(lat);
    st.gpu_busy_s += ms * 1e-3;
    st.batches += 1;
    st.completed += 1;
    st.events_completed += k.p.n;
    t_last = now;
    k.reported = true;
    any_done = true;
  }
  while (!wf.empty() && wf.front().reported) {
    Pkt &k = wf.front();
    release(k);
    ev_pool.push_back(k.uploaded);
    cudaEventDestroy(k.start);
    cudaEventDestroy(k.done);
    wf.pop_front();
  }
  if (any_done) cv_done.notify_all();
}

void veckm_server::run_w() {
  cudaSetDevice(device);
  for (;;) {
    retire_w(false);
    Pkt k;
    {
      std::unique_lock<std::mutex> lk(mu);
      const bool can_take = !pending.empty() && pending.front().ready &&
                            (int)wf.size() < kMaxInflightW;
      if (!can_take) {
        if (stop && pending.empty() && wf.empty()) break;
        if ((int)wf.size() >= kMaxInflightW) {
          lk.unlock();
          retire_w(true);
          continue;
        }
        if (!wf.empty()) {
          // packets on the device: poll them while waiting for new ones
          cv_work.wait_for(lk, std::chrono::microseconds(50));
          continue;
        }
        cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      k = pending.front();
      pending.pop_front();
    }
    launch_w(k);
  }
}

void veckm_server::retire(bool block) {
  while (!inflight.empty()) {
    Batch &b = inflight.front();
    if (block) {
      cudaEventSynchronize(b.done);
    } else if (cudaEventQuery(b.done) == cudaErrorNotReady) {
      break;
    }
    block = false;
    const Clock::time_point now = Clock::now();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b.start, b.done);
    const int w = h_err[b.slot];
    const veckm_status status =
        (w & veckm::ERR_TIMEOUT) ? VECKM_ETIMEOUT
        : (w & (veckm::ERR_EVENT_RANGE | veckm::ERR_INDEX_RANGE)) ? VECKM_ERANGE : VECKM_OK;
    {
      std::lock_guard<std::mutex> lk(mu);
      st.gpu_busy_s += ms * 1e-3;
      st.batches += 1;
      for (const Pkt &k : b.pk) {
        const double lat = std::chrono::duration<double, std::milli>(now - k.t_submit).count();
        done.push_back(veckm_completion{k.p.tag, k.p.stream_id, status, k.p.n, lat,
                                        (int32_t)b.pk.size()});
        lat_ms.push_back(lat);
        release(k);
        ev_pool.push_back(k.uploaded);
        st.completed += 1;
        st.events_completed += k.p.n;
      }
      t_last = now;
    }
    cudaEventDestroy(b.start);
    cudaEventDestroy(b.done);
    inflight.pop_front();
    cv_done.notify_all();
  }
}

bool veckm_server::launch(std::vector<Pkt> &pk) {
  Batch b;
  b.slot = next_slot;
  next_slot = (next_slot + 1) % kMaxInflight;
  cudaEventCreate(&b.start);
  cudaEventCreate(&b.done);
  std::vector<veckm_slice> sl(pk.size());
  for (size_t i = 0; i < pk.size(); ++i) {
    const Pkt &k = pk[i];
    cudaStreamWaitEvent(comp, k.uploaded, 0);
    char *base = arena + k.off;
    const int64_t n = k.p.n;
    sl[i] = veckm_slice{reinterpret_cast<int16_t *>(base),
                        reinterpret_cast<int16_t *>(base + al256(2 * n)),
                        reinterpret_cast<uint32_t *>(base + 2 * al256(2 * n)), n, k.p.t_ref_us,
                        k.p.width, k.p.height};
  }
  cudaEventRecord(b.start, comp);
  veckm_status s = veckm_predict_batch(ctx, sl.data(), (int32_t)sl.size(), d_flow[b.slot], comp);
  cudaMemcpyAsync(h_err + b.slot, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, comp);
  cudaMemsetAsync(ctx->err, 0, sizeof(int), comp);
  if (s == VECKM_OK) {
    int64_t off = 0;
    for (const Pkt &k : pk) {
      cudaMemcpyAsync(k.p.h_flow, d_flow[b.slot] + 2 * off, (size_t)k.p.n * 8,
                      cudaMemcpyDeviceToHost, comp);
      off += k.p.n;
    }
  }
  cudaEventRecord(b.done, comp);
  if (s != VECKM_OK) {
    // report the whole batch as failed once the stream reaches this point;
    // earlier batches leave the ring first
    cudaEventSynchronize(b.done);
    while (!inflight.empty()) retire(true);
    std::lock_guard<std::mutex> lk(mu);
    const Clock::time_point now = Clock::now();
    for (const Pkt &k : pk) {
      done.push_back(veckm_completion{k.p.tag, k.p.stream_id, s, k.p.n,
                                      std::chrono::duration<double, std::milli>(now - k.t_submit).count(),
                                      (int32_t)pk.size()});
      release(k);
      ev_pool.push_back(k.uploaded);
      st.completed += 1;
    }
    cudaEventDestroy(b.start);
    cudaEventDestroy(b.done);
    cv_done.notify_all();
    return false;
  }
  b.pk = std::move(pk);
  inflight.push_back(std::move(b));
  return true;
}

void veckm_server::run() {
  cudaSetDevice(device);
  const int W = ctx->g.W, H = ctx->g.H, gx = ctx->g.dx, gy = ctx->g.dy;
  std::vector<int32_t> ws, hs, ox, oy;
  for (;;) {
    retire(false);
    std::vector<Pkt> pk;
    {
      std::unique_lock<std::mutex> lk(mu);
      const bool can_take = !pending.empty() && pending.front().ready &&
                            (int)inflight.size() < kMaxInflight;
      if (!can_take) {
        if (stop && pending.empty() && inflight.empty()) break;
        if (!inflight.empty()) {
          lk.unlock();
          retire(true);
          continue;
        }
        cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      if (window.count() > 0) {  // wait for a fuller batch, up to the window
        int64_t ev = 0, np = 0;
        for (const Pkt &k : pending) {
          ev += k.p.n;
          np += 1;
        }
        const Clock::time_point due = pending.front().t_submit + window;
        if (!stop && np < max_packets && ev < max_events && Clock::now() < due) {
          cv_work.wait_until(lk, due);
          continue;
        }
      }
      // arrival order, while ready and within the batch limits and one canvas
      int64_t events = 0;
      ws.clear();
      hs.clear();
      while (!pending.empty() && pending.front().ready && (int32_t)pk.size() < max_packets &&
             events + pending.front().p.n <= max_events) {
        ws.push_back(pending.front().p.width);
        hs.push_back(pending.front().p.height);
        ox.resize(ws.size());
        oy.resize(ws.size());
        int32_t cw = 0, ch = 0;
        if (!pk.empty() && (veckm_canvas_layout((int32_t)ws.size(), ws.data(), hs.data(), gx, gy,
                                                W, ox.data(), oy.data(), &cw, &ch) != VECKM_OK ||
                            ch > H))
          break;
        events += pending.front().p.n;
        pk.push_back(pending.front());
        pending.pop_front();
      }
    }
    launch(pk);
  }
}

extern "C" {

veckm_status veckm_server_create(const veckm_server_config *cfg, veckm_server **out) {
  if (!cfg || !out) return fail_msg(VECKM_EINVAL, "null argument");
  *out = nullptr;
  if (cfg->arena_bytes < 0 || cfg->max_batch_packets < 0 || cfg->max_batch_events < 0 ||
      cfg->max_batch_events > VECKM_MAX_EVENTS || cfg->window_us < 0 ||
      cfg->window_capacity < 0 || cfg->window_capacity > VECKM_MAX_EVENTS)
    return fail_msg(VECKM_EINVAL, "bad server limits");
  veckm_server *s = new (std::nothrow) veckm_server();
  if (!s) return fail_msg(VECKM_ENOMEM, "host allocation");
  if (veckm_status st = veckm_create(&s->ctx, &cfg->model)) {
    delete s;
    return st;
  }
  s->device = s->ctx->device;
  if (cfg->max_batch_packets > 0) s->max_packets = cfg->max_batch_packets;
  if (cfg->max_batch_events > 0) s->max_events = cfg->max_batch_events;
  s->window = std::chrono::microseconds(std::max(0, cfg->batch_window_us));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kMaxInflight && e == cudaSuccess; ++i)
    e = veckm::dev_malloc(reinterpret_cast<void **>(&s->d_flow[i]), (size_t)s->max_events * 8);
  if (e == cudaSuccess) e = veckm::host_malloc(reinterpret_cast<void **>(&s->h_err), kMaxInflight * sizeof(int));
  int64_t arena = cfg->arena_bytes;
  if (e == cudaSuccess && arena == 0) {
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    arena = (int64_t)(free_b / 4) & ~int64_t(255);
  }
  if (e == cudaSuccess) e = veckm::dev_malloc(reinterpret_cast<void **>(&s->arena), (size_t)std::max<int64_t>(arena, 256));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->comp, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    for (float *f : s->d_flow) if (f) cudaFree(f);
    if (s->h_err) cudaFreeHost(s->h_err);
    if (s->arena) cudaFree(s->arena);
    if (s->up) cudaStreamDestroy(s->up);
    if (s->comp) cudaStreamDestroy(s->comp);
    veckm_destroy(s->ctx);
    delete s;
    return fail_cuda(e, "server buffers");
  }
  s->cap = std::max<int64_t>(arena, 256);
  s->seen_stream.assign(65536, 0);
  s->window_us = cfg->window_us;
  if (cfg->window_capacity > 0) s->window_cap = cfg->window_capacity;
  if (s->window_us > 0) {
    s->sensors.assign(65536, nullptr);
    if (veckm::host_malloc(reinterpret_cast<void **>(&s->h_errw), kMaxInflightW * sizeof(int)) !=
        cudaSuccess) {
      veckm_server_destroy(s);
      return fail_msg(VECKM_ENOMEM, "server error words");
    }
    s->worker = std::thread([s] { s->run_w(); });
  } else {
    s->worker = std::thread([s] { s->run(); });
  }
  *out = s;
  return VECKM_OK;
}

veckm_status veckm_server_submit(veckm_server *s, const veckm_packet *p) {
  if (!s || !p) return fail_msg(VECKM_EINVAL, "null argument");
  if (p->n < 1 || p->n > VECKM_MAX_EVENTS) return fail_msg(VECKM_EINVAL, "packet size %lld", (long long)p->n);
  if (!p->h_x || !p->h_y || !p->h_t || !p->h_flow) return fail_msg(VECKM_EINVAL, "null packet buffer");
  if (p->stream_id < 0 || p->stream_id > 65535) return fail_msg(VECKM_EINVAL, "stream id %d", p->stream_id);
  if (p->width < 1 || p->height < 1 || p->width > s->ctx->g.W || p->height > s->ctx->g.H)
    return fail_msg(VECKM_EINVAL, "packet sensor %dx%d outside the %dx%d canvas", p->width,
                    p->height, s->ctx->g.W, s->ctx->g.H);
  if (s->window_us == 0 && p->n > s->max_events)
    return fail_msg(VECKM_EINVAL, "packet larger than a batch");
  if (s->window_us > 0 && p->n > s->window_cap)
    return fail_msg(VECKM_EINVAL, "packet larger than a stream's window capacity");
  const Clock::time_point now = Clock::now();
  const int64_t bytes = s->window_us > 0 ? footprint_w(p->n) : footprint(p->n);
  if (s->window_us > 0) {
    // the stream's resident state (created with its first packet); no room
    // for it refuses the packet like a full arena
    veckm_status sst;
    if (!s->sensor_for(p, &sst)) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.submitted += 1;
      if (sst == VECKM_EBUSY) s->st.refused += 1;
      return sst;
    }
  }
  Pkt *k = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.submitted += 1;
    if (!s->any) {
      s->any = true;
      s->t_first = now;
    }
    if (!s->seen_stream[p->stream_id]) {
      s->seen_stream[p->stream_id] = 1;
      s->st.streams += 1;
    }
    int64_t off = 0;
    if (s->stop || !s->alloc(bytes, &off)) {
      s->st.refused += 1;
      return fail_msg(VECKM_EBUSY, "no room for %lld events in the device arena", (long long)p->n);
    }
    s->st.admitted += 1;
    Pkt q;
    q.p = *p;
    q.off = off;
    q.bytes = bytes;
    q.uploaded = s->take_event();
    q.t_submit = now;
    q.t_hi = p->h_t[p->n - 1];  // resident windows: packets come sorted by time
    s->pending.push_back(q);
    k = &s->pending.back();  // deque: stable while the worker skips packets not ready
  }
  // the copies: outside the lock (the worker does not take a packet until ready)
  char *base = s->arena + k->off;
  const int64_t n = p->n;
  cudaError_t e = cudaMemcpyAsync(base, p->h_x, (size_t)n * 2, cudaMemcpyHostToDevice, s->up);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + al256(2 * n), p->h_y, (size_t)n * 2, cudaMemcpyHostToDevice, s->up);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + 2 * al256(2 * n), p->h_t, (size_t)n * 4, cudaMemcpyHostToDevice, s->up);
  if (e == cudaSuccess) e = cudaEventRecord(k->uploaded, s->up);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    k->ready = true;
  }
  s->cv_work.notify_one();
  return e == cudaSuccess ? VECKM_OK : fail_cuda(e, "packet upload");
}

int32_t veckm_server_poll(veckm_server *s, veckm_completion *out, int32_t max, int32_t wait_ms) {
  if (!s || (max > 0 && !out)) return VECKM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [s] { return !s->done.empty(); });
  int32_t k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  return k;
}

veckm_status veckm_server_drain(veckm_server *s) {
  if (!s) return fail_msg(VECKM_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [s] { return s->st.completed >= s->st.admitted; });
  return VECKM_OK;
}

veckm_status veckm_server_get_stats(veckm_server *s, veckm_server_stats *out) {
  if (!s || !out) return fail_msg(VECKM_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  std::vector<double> v = s->lat_ms;
  if (!v.empty()) {
    auto pct = [&v](double q) {
      const size_t i = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + (ptrdiff_t)i, v.end());
      return v[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = *std::max_element(v.begin(), v.end());
  }
  out->wall_s = s->any ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
  return VECKM_OK;
}

void veckm_server_destroy(veckm_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaStreamSynchronize(s->up);
  cudaStreamSynchronize(s->comp);
  for (Sensor *sn : s->sensors) {
    if (!sn) continue;
    cudaStreamSynchronize(sn->cs);
    veckm_stream_destroy(sn->st);
    veckm_destroy(sn->ctx);
    cudaStreamDestroy(sn->cs);
    delete sn;
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  for (float *f : s->d_flow) if (f) cudaFree(f);
  if (s->h_err) cudaFreeHost(s->h_err);
  if (s->h_errw) cudaFreeHost(s->h_errw);
  if (s->arena) cudaFree(s->arena);
  cudaStreamDestroy(s->up);
  cudaStreamDestroy(s->comp);
  veckm_destroy(s->ctx);
  delete s;
}

}  // extern "C"
