// veckm_encode_noalloc: the encoding of veckm_encode for callers that must not
// allocate device memory while they run.
//
// veckm_encode keeps its pixel-sorted event records in context buffers that
// grow (cudaMalloc, after a stream synchronisation) whenever a call brings
// more events than any call before.  Some callers cannot allow that: a loop
// with a real-time budget (an allocation and the synchronisation before it
// take an unbounded time), or a process that reserves all of a device's
// memory up front for its own allocator, after which cudaMalloc fails.  This
// entry point instead takes the per-event records from one fixed array in
// device memory that the library declares at file scope, so a call never
// allocates: it only launches kernels and clears context buffers with
// cudaMemsetAsync.
//
// The array holds up to kNoAllocMaxEvents events (12 bytes each, 12 MiB in
// all); every GPU that loads the library keeps it for the life of the
// process.  All calls, from every context on a device, share it: calls that
// may overlap on the GPU (two streams, two host threads) race on it and
// must be serialised by the caller.
//
// The array's device address is looked up with cudaGetSymbolAddress by the
// first call on a device (with that device current) and kept per device,
// together with the identity of the CUDA context it belongs to; a device
// reset (cudaDeviceReset) ends that context, and the next call looks the
// address up again.  The first call on a device should therefore come before
// any stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "veckm_internal.h"

namespace {

constexpr int64_t kNoAllocMaxEvents = (int64_t)1 << 20;
constexpr size_t kRecordBytes = (size_t)kNoAllocMaxEvents * (sizeof(int2) + sizeof(int));

// Records of one call: (t - t_ref, event index) pairs, then the pixel of each.
// Every call overwrites what it reads, so nothing here needs clearing.
static __device__ __align__(256) unsigned char g_noalloc_records[kRecordBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mutex;
// per device: the device address of g_noalloc_records and the id of the CUDA
// context it was looked up in (0: not looked up yet)
void *g_records_addr[kMaxDevices] = {};
unsigned long long g_records_ctx[kMaxDevices] = {};

// The id of the current CUDA context (unique for the life of the process),
// through the driver's cuCtxGetCurrent and cuCtxGetId, reached by their
// runtime entry points so that the library need not link the driver; false
// if they are unavailable.
bool current_context_id(unsigned long long *id) {
  using GetCurrent = int (*)(void **);
  using GetId = int (*)(void *, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  }
  void *ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

// The host-side name g_noalloc_records is only a stand-in for the symbol; the
// device address comes from cudaGetSymbolAddress, with the device current,
// once per device and CUDA context (every call when the context's identity
// cannot be read).
cudaError_t records_on_device(int dev, void **addr) {
  std::lock_guard<std::mutex> lock(g_mutex);
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  if (!have_id || !g_records_addr[dev] || g_records_ctx[dev] != id) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_records);
    if (e != cudaSuccess) return e;
    g_records_addr[dev] = p;
    g_records_ctx[dev] = have_id ? id : 0;
  }
  *addr = g_records_addr[dev];
  return cudaSuccess;
}

}  // namespace

using namespace veckm;

extern "C" veckm_status veckm_encode_noalloc(veckm_ctx *ctx, const int16_t *d_x,
                                             const int16_t *d_y, const uint32_t *d_t, int64_t n,
                                             uint32_t t_ref_us, const int64_t *d_K, int64_t nK,
                                             float *d_emb, void *stream) {
  CtxView c;
  if (!ctx_view(ctx, &c)) return report(VECKM_EINVAL, "null context");
  if (n < 0 || nK < 0) return report(VECKM_EINVAL, "negative size");
  if (n > kNoAllocMaxEvents)
    return report(VECKM_EINVAL,
                  "veckm_encode_noalloc takes at most 1048576 events per call "
                  "(its static record array); use veckm_encode for larger slices");
  if (nK > VECKM_MAX_EVENTS)
    return report(VECKM_EINVAL, "more than 2^30 requested events in one call");
  if (n > 0 && (!d_x || !d_y || !d_t)) return report(VECKM_EINVAL, "null event buffer");
  if (!d_K && nK != n && nK != 0) return report(VECKM_EINVAL, "K is NULL but nK != n");
  if (nK > 0 && !d_emb) return report(VECKM_EINVAL, "null output buffer");
  if (nK > 0 && n == 0) return report(VECKM_EINVAL, "nK > 0 with an empty slice");
  if (nK == 0) return VECKM_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return report(VECKM_ECUDA, "no usable current device");
  void *base = nullptr;
  if (records_on_device(dev, &base) != cudaSuccess)
    return report(VECKM_ECUDA, "cudaGetSymbolAddress failed for the static record array");
  int2 *rec = reinterpret_cast<int2 *>(base);
  int *rpix = reinterpret_cast<int *>(rec + kNoAllocMaxEvents);

  cudaStream_t s = (cudaStream_t)stream;
  grids_dirty(ctx);  // both grids are written below
  const Geometry &g = c.g;
  const Events ev{d_x, d_y, d_t, n, t_ref_us, (uint32_t)c.t_span};
  const size_t P = (size_t)g.W * g.H;
  if (cudaMemsetAsync(c.cnt, 0, P * sizeof(int), s) != cudaSuccess ||
      launch_hist(ev, g, c.cnt, c.err, nullptr, s) < 0 ||
      launch_scan(g, c.cnt, c.bsum, c.off, c.cur, c.total, s) < 0 ||
      launch_place(ev, g, c.cur, rec, rpix, s) < 0 ||
      launch_pixsum(g, c.tb, c.off + P, rec, rpix, n, c.acc, s) < 0 ||
      launch_pool_rows(g, c.tb, c.acc, c.hbuf, s, c.tn) < 0 ||
      launch_pool_cols(g, c.tb, c.hbuf, c.acc, s, c.tn) < 0 ||
      launch_counts(g, c.cnt, c.cnt_tmp, c.ncnt, s) < 0 ||
      launch_gather_emb(ev, d_K, nK, g, c.tb, c.acc, c.ncnt, d_emb, c.err, s) < 0)
    return report(VECKM_ECUDA, cudaGetErrorString(cudaGetLastError()));
  return VECKM_OK;
}
