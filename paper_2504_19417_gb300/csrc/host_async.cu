// Pipelined predictions from host buffers.  Two staging slots per context;
// a call's uploads run on an upload stream, its encoder and perceptron on a
// compute stream (so calls still run one after another on the device), and
// its flows come back on a download stream.  The upload of one call and the
// download of the previous one therefore overlap the computation between
// them (the two directions of the host link run at once; one shared copy
// stream would queue each upload behind the previous call's download, which
// waits for that call's computation).  The context's error word is copied out and cleared after each
// call's computation, so every ticket gets its own status.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "ctx.h"

namespace veckm {

struct HostPipe {
  struct Slot {
    void *buf = nullptr;
    size_t cap = 0;
    cudaEvent_t up = nullptr, done = nullptr, down = nullptr;
    int *h_err = nullptr;  // pinned
    int64_t ticket = -1;   // in flight, or -1
  };
  cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
  Slot slot[2];
  int64_t next = 0;
  // statuses of the last tickets that completed without being waited for
  static constexpr int kKeep = 64;
  int64_t done_ticket[kKeep];
  veckm_status done_status[kKeep];
  HostPipe() {
    for (int i = 0; i < kKeep; ++i) done_ticket[i] = -1;
  }
};

void destroy_pipe(HostPipe *p) {
  if (!p) return;
  cudaStream_t ss[] = {p->up, p->comp, p->down};
  for (cudaStream_t x : ss)
    if (x) cudaStreamSynchronize(x);
  for (auto &s : p->slot) {
    if (s.buf) cudaFree(s.buf);
    if (s.h_err) cudaFreeHost(s.h_err);
    cudaEvent_t evs[] = {s.up, s.done, s.down};
    for (cudaEvent_t e : evs)
      if (e) cudaEventDestroy(e);
  }
  for (cudaStream_t x : ss)
    if (x) cudaStreamDestroy(x);
  delete p;
}

namespace {

veckm_status status_of(int w) {
  if (w & ERR_TIMEOUT) return fail_msg(VECKM_ETIMEOUT, "a bounded device wait ran out");
  if (w & ERR_CAPACITY) return fail_msg(VECKM_EBUSY, "a device capacity was exceeded");
  if (w & (ERR_EVENT_RANGE | ERR_INDEX_RANGE))
    return fail_msg(VECKM_ERANGE, "event outside the sensor or time span, or index in K outside [0, n)");
  return VECKM_OK;
}

// Waits for the slot's call, records its status, frees the slot.
veckm_status retire(HostPipe *p, HostPipe::Slot &s) {
  if (s.ticket < 0) return VECKM_OK;
  const cudaError_t e = cudaEventSynchronize(s.down);
  const veckm_status st = e != cudaSuccess ? fail_cuda(e, "asynchronous prediction") : status_of(*s.h_err);
  const int k = (int)(s.ticket % HostPipe::kKeep);
  p->done_ticket[k] = s.ticket;
  p->done_status[k] = st;
  s.ticket = -1;
  return st;
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace veckm

using namespace veckm;

extern "C" {

veckm_status veckm_predict_host_async(veckm_ctx *c, const int16_t *hx, const int16_t *hy,
                                      const uint32_t *ht, int64_t n, uint32_t t_ref,
                                      const int64_t *hK, int64_t nK, float *hflow,
                                      int64_t *ticket) {
  if (!ticket) return fail_msg(VECKM_EINVAL, "null ticket");
  veckm_status st = check_events_args(c, hx, hy, ht, n, hK, nK, hflow);
  if (st) return st;
  if (!c->pipe) {
    HostPipe *p = new (std::nothrow) HostPipe();
    if (!p) return fail_msg(VECKM_ENOMEM, "host allocation");
    cudaError_t e = cudaStreamCreateWithFlags(&p->up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->down, cudaStreamNonBlocking);
    for (auto &s : p->slot) {
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.up, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.down, cudaEventDisableTiming);
      if (e == cudaSuccess) e = host_malloc(reinterpret_cast<void **>(&s.h_err), sizeof(int));
    }
    if (e != cudaSuccess) {
      destroy_pipe(p);
      return fail_cuda(e, "host pipeline");
    }
    c->pipe = p;
  }
  HostPipe *p = c->pipe;
  const int64_t k = p->next;
  HostPipe::Slot &s = p->slot[k & 1];
  retire(p, s);  // the call two back used this slot
  const size_t bx = al256((size_t)n * 2), bt = al256((size_t)n * 4),
               bk = hK ? al256((size_t)nK * 8) : 0, bf = al256((size_t)nK * 8);
  const size_t need = 2 * bx + bt + bk + bf;
  cudaError_t e = cudaSuccess;
  if (need > s.cap) {
    if (s.buf) cudaFree(s.buf);
    s.buf = nullptr;
    s.cap = 0;
    e = dev_malloc(reinterpret_cast<void **>(&s.buf), std::max<size_t>(need, 256));
    if (e != cudaSuccess) return fail_cuda(e, "staging buffers");
    s.cap = need;
  }
  char *b = static_cast<char *>(s.buf);
  int16_t *dx = (int16_t *)b;
  int16_t *dy = (int16_t *)(b + bx);
  uint32_t *dt = (uint32_t *)(b + 2 * bx);
  int64_t *dK = hK ? (int64_t *)(b + 2 * bx + bt) : nullptr;
  float *df = (float *)(b + 2 * bx + bt + bk);
  if (n > 0) {
    e = cudaMemcpyAsync(dx, hx, (size_t)n * 2, cudaMemcpyHostToDevice, p->up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, hy, (size_t)n * 2, cudaMemcpyHostToDevice, p->up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt, ht, (size_t)n * 4, cudaMemcpyHostToDevice, p->up);
  }
  if (e == cudaSuccess && hK && nK > 0)
    e = cudaMemcpyAsync(dK, hK, (size_t)nK * 8, cudaMemcpyHostToDevice, p->up);
  if (e == cudaSuccess) e = cudaEventRecord(s.up, p->up);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->comp, s.up, 0);
  if (e != cudaSuccess) return fail_cuda(e, "host-to-device copy");
  st = veckm_predict(c, dx, dy, dt, n, t_ref, dK, nK, df, p->comp);
  if (st) return st;
  e = cudaMemcpyAsync(s.h_err, c->err, sizeof(int), cudaMemcpyDeviceToHost, p->comp);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), p->comp);
  if (e == cudaSuccess) e = cudaEventRecord(s.done, p->comp);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->down, s.done, 0);
  if (e == cudaSuccess && nK > 0)
    e = cudaMemcpyAsync(hflow, df, (size_t)nK * 8, cudaMemcpyDeviceToHost, p->down);
  if (e == cudaSuccess) e = cudaEventRecord(s.down, p->down);
  if (e != cudaSuccess) return fail_cuda(e, "device-to-host copy");
  s.ticket = k;
  p->next = k + 1;
  *ticket = k;
  return VECKM_OK;
}

veckm_status veckm_host_wait(veckm_ctx *c, int64_t ticket) {
  if (!c || !c->pipe || ticket < 0 || ticket >= c->pipe->next)
    return fail_msg(VECKM_EINVAL, "unknown ticket");
  HostPipe *p = c->pipe;
  HostPipe::Slot &s = p->slot[ticket & 1];
  if (s.ticket == ticket) return retire(p, s);
  const int k = (int)(ticket % HostPipe::kKeep);
  if (p->done_ticket[k] == ticket) return p->done_status[k];
  return fail_msg(VECKM_EINVAL, "ticket %lld is too old to report", (long long)ticket);
}

}  // extern "C"
