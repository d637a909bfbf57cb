// Sliding-window streams: a per-stream resident accumulator over the last
// `window` microseconds of a sensor's events.
//
// The accumulation of Algorithm 1 (PixelEmbed, PixelCount) is linear in the
// events, so a window that slides is kept up to date by adding the events of
// each new packet and subtracting the events that leave the window.  To keep
// that exact over any number of packets the per-pixel sums are held in 64-bit
// fixed point: each component v of an event's FP32 phase exp(i t T_d/dt)
// becomes the integer v * 2^32 (exact for |v| >= 2^-8, where the FP32 spacing
// is at least 2^-32; smaller components lose their bits below 2^-32, under
// 2.4e-10), and integer addition is exact and independent of order.  An event
// adds and later subtracts the same integers, so after any sequence of
// packets the accumulator equals, bit for bit, the one built from the
// window's events alone.  Counts are exact int32.
//
// The stream's valid events live in a device ring (x, y, t; t in absolute
// microseconds), kept in time order: an event is accepted only if its time is
// at least that of every event accepted before it, in earlier packets (the
// stream's last accepted time) and earlier in its own packet (the running
// maximum over the packet's in-range events before it), so the ring's times
// ascend whatever order the events come in.  A packet is pushed with its end
// time t_hi (every event has t <= t_hi; t_hi never goes back); the window is
// then [t_hi - window, t_hi].  A push, in stream order:
//   1. flag the packet's valid events (inside the sensor and the window, not
//      earlier than an event accepted before them) and scan the flags: the
//      valid events' places in the ring;
//   2. find the first ring event still in the window (a 32-way search by one
//      warp) and how many valid events fit the ring after the expiry;
//   3. subtract the events that left;
//   4. append the valid events that fit (K[i] = an event's ring slot, or -1:
//      its output row is zeroed and the error word set);
//   5. add them;
//   6. convert the pixels whose sums changed to the stream's FP32 grid and
//      run the pooling and the gather (and perceptron) for the packet's
//      events.
// Nothing is copied to the host: a push never synchronises.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "chain.cuh"
#include "ctx.h"
#include "check.cuh"
#include "phase.cuh"

namespace veckm {
namespace {

struct RingState {
  long long head;      // events appended so far (ring position = index mod capacity)
  long long tail;      // first event still in the window
  long long tail_old;  // the tail before the current push
  long long head_old;  // the head before the current push
  long long app;       // events of the current packet that fit the ring
  unsigned t_last;     // time of the last accepted event (0 before the first)
};

__device__ __forceinline__ void red_add_s64(long long *p, long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)v) : "memory");
}

// 1a. events of the packet inside the sensor and [t_lo, t_hi]; tkey holds
// their times (0 for the others), whose running maximum decides the order
__global__ void k_ring_flags(const int16_t *__restrict__ x, const int16_t *__restrict__ y,
                             const uint32_t *__restrict__ t, long long n, int W, int H,
                             uint32_t t_lo, uint32_t t_hi, int *__restrict__ flag,
                             unsigned *__restrict__ tkey, int *err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int xi = x[i], yi = y[i];
  const uint32_t ti = t[i];
  const bool ok = xi >= 0 && xi < W && yi >= 0 && yi < H && ti >= t_lo && ti <= t_hi;
  if (!ok) atomicOr(err, ERR_EVENT_RANGE);
  flag[i] = ok ? 1 : 0;
  tkey[i] = ok ? ti : 0u;
}

// 1b. exclusive running maximum of tkey in blocks of kMaxBlock: per block
// its maximum (reduce), the exclusive maximum over the blocks before each
// (top, one CTA), then per event the maximum over the in-range events before
// it; an in-range event earlier than that, or than the stream's last accepted
// time, is out of order and not accepted.
constexpr int kMaxThreads = 256;
constexpr int kMaxPer = 4;
constexpr int kMaxBlock = kMaxThreads * kMaxPer;

// exclusive maximum of v over the threads before this one (0 for the first),
// and the block's maximum in *total
__device__ __forceinline__ unsigned block_excl_max(unsigned v, unsigned *s_warp, unsigned &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned m = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl = max(incl, m);
  }
  unsigned excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = 0u;
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
    unsigned wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned m = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi = max(wi, m);
    }
    unsigned we = __shfl_up_sync(0xffffffffu, wi, 1);
    if (lane == 0) we = 0u;
    s_warp[lane] = we;  // maximum over the warps before
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  total = s_warp[32];
  const unsigned r = max(s_warp[warp], excl);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kMaxThreads) k_tmax_reduce(const unsigned *__restrict__ tkey,
                                                             long long n,
                                                             unsigned *__restrict__ bmax) {
  __shared__ unsigned s_warp[33];
  chain_wait();
  const long long b0 = (long long)blockIdx.x * kMaxBlock + threadIdx.x * kMaxPer;
  unsigned v = 0;
#pragma unroll
  for (int i = 0; i < kMaxPer; ++i)
    if (b0 + i < n) v = max(v, tkey[b0 + i]);
  unsigned total;
  block_excl_max(v, s_warp, total);
  if (threadIdx.x == 0) bmax[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kMaxThreads) k_tmax_top(unsigned *__restrict__ bmax, int nb) {
  __shared__ unsigned s_warp[33];
  chain_wait();
  unsigned carry = 0;
  for (int base = 0; base < nb; base += kMaxThreads) {
    const int i = base + threadIdx.x;
    const unsigned v = i < nb ? bmax[i] : 0u;
    unsigned tot;
    const unsigned ex = block_excl_max(v, s_warp, tot);
    if (i < nb) bmax[i] = max(carry, ex);
    carry = max(carry, tot);
  }
}

__global__ void __launch_bounds__(kMaxThreads) k_tmax_order(const unsigned *__restrict__ tkey,
                                                            long long n,
                                                            const unsigned *__restrict__ bmax,
                                                            const RingState *st,
                                                            int *__restrict__ flag, int *err) {
  __shared__ unsigned s_warp[33];
  chain_wait();
  const long long b0 = (long long)blockIdx.x * kMaxBlock + threadIdx.x * kMaxPer;
  unsigned k[kMaxPer];
  unsigned v = 0;
#pragma unroll
  for (int i = 0; i < kMaxPer; ++i) {
    k[i] = b0 + i < n ? tkey[b0 + i] : 0u;
    v = max(v, k[i]);
  }
  unsigned total;
  unsigned run = max(max(block_excl_max(v, s_warp, total), bmax[blockIdx.x]), st->t_last);
  bool bad = false;
#pragma unroll
  for (int i = 0; i < kMaxPer; ++i) {
    if (b0 + i < n && flag[b0 + i] && k[i] < run) {
      flag[b0 + i] = 0;
      bad = true;
    }
    run = max(run, k[i]);
  }
  if (bad) atomicOr(err, ERR_EVENT_RANGE);
}

// 2. new tail: the first ring event with t >= t_lo (ring events ascend in
// t); then how many of the `*nvalid` valid packet events fit the ring
__global__ void k_ring_tail(RingState *st, const uint32_t *__restrict__ rt, long long cap,
                            uint32_t t_lo, const int *__restrict__ nvalid) {
  chain_wait();
  const long long n = nvalid ? *nvalid : 0;
  const int lane = threadIdx.x & 31;
  const long long head = st->head, tail0 = st->tail;
  long long lo = tail0, hi = head;
  // 32-way search with the warp: lane j probes lo + j * step; the first
  // probe at or after t_lo bounds the answer (the ring's times ascend) to
  // the step before it, so each round divides the range by 32
  while (lo < hi) {
    const long long step = (hi - lo + 31) / 32;
    const long long pos = lo + (long long)lane * step;
    const bool ge = pos >= hi || rt[pos % cap] >= t_lo;
    const unsigned m = __ballot_sync(0xffffffffu, ge);
    if (m == 0) {  // every probe before t_lo (all 32 inside the range)
      lo += 31 * step + 1;
      continue;
    }
    const int f = __ffs(m) - 1;
    const long long nhi = lo + (long long)f * step < hi ? lo + (long long)f * step : hi;
    if (f > 0) lo += (long long)(f - 1) * step + 1;
    hi = nhi;
  }
  if (lane == 0) {
    st->tail_old = tail0;
    st->tail = lo;
    st->head_old = head;
    const long long room = cap - (head - lo);
    st->app = n < room ? n : room;
  }
}

// 3./5. subtract (sign -1: ring events [tail_old, tail)) or add (+1: the
// appended events [head_old, head_old + app)) their fixed-point phases and
// counts.  One warp per event, lanes over units (channels 2u, 2u+1).
template <int DV>
__global__ void __launch_bounds__(256)
    k_ring_apply(const RingState *st, int sign,
                 const int16_t *__restrict__ rx, const int16_t *__restrict__ ry,
                 const uint32_t *__restrict__ rt, long long cap, int W, int U, long long npx,
                 const uint2 *__restrict__ wt, long long *__restrict__ acc64,
                 int *__restrict__ cnt, uint8_t *__restrict__ dirty) {
  chain_wait();
  const int lane = threadIdx.x & 31;
  const long long first = sign < 0 ? st->tail_old : st->head_old;
  const long long count = sign < 0 ? st->tail - st->tail_old : st->app;
  uint2 w[DV][2];
#pragma unroll
  for (int v = 0; v < DV; ++v) {
    const int u = lane + 32 * v;
    w[v][0] = __ldg(wt + 2 * u);
    w[v][1] = __ldg(wt + 2 * u + 1);
  }
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long j = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < count;
       j += nw) {
    const long long pos = (first + j) % cap;
    const int p = ry[pos] * W + rx[pos];
    if (!VK_CHECK(p >= 0 && p < npx)) continue;  // the ring holds on-sensor events only
    const uint32_t t = rt[pos];
    long long *dst = acc64 + (size_t)p * 4 * U;
#pragma unroll
    for (int v = 0; v < DV; ++v) {
      const int u = lane + 32 * v;
      const float4 ph = time_phase2(t, w[v][0], w[v][1]);  // (re, im) of channels 2u, 2u+1
      const float sc = 4294967296.0f * (float)sign;         // exact: a power of two
      red_add_s64(dst + 4 * u + 0, (long long)(ph.x * sc));
      red_add_s64(dst + 4 * u + 1, (long long)(ph.y * sc));
      red_add_s64(dst + 4 * u + 2, (long long)(ph.z * sc));
      red_add_s64(dst + 4 * u + 3, (long long)(ph.w * sc));
    }
    if (lane == 0) {
      atomicAdd(cnt + p, sign);
      dirty[p] = 1;
    }
  }
}

// 4. append valid event i (place off[i] among the valid ones) at ring
// position head + off[i] if it fits; K[i] = its ring slot, else -1 (an
// index outside the ring: the gather writes zeros for it)
__global__ void k_ring_append(const RingState *st, const int16_t *__restrict__ x,
                              const int16_t *__restrict__ y, const uint32_t *__restrict__ t,
                              long long n, const int *__restrict__ flag,
                              const int *__restrict__ off, int16_t *__restrict__ rx,
                              int16_t *__restrict__ ry, uint32_t *__restrict__ rt, long long cap,
                              int64_t *__restrict__ K, int *err) {
  chain_wait();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!flag[i]) {
    K[i] = -1;
    return;
  }
  if (off[i] >= st->app) {  // the window would hold more events than the ring
    atomicOr(err, ERR_CAPACITY);
    K[i] = -1;
    return;
  }
  const long long r = (st->head_old + off[i]) % cap;
  rx[r] = x[i];
  ry[r] = y[i];
  rt[r] = t[i];
  K[i] = r;
}

// the ring's times ascend, so the last appended event holds the largest
// accepted time
__global__ void k_ring_advance(RingState *st, const uint32_t *__restrict__ rt, long long cap) {
  chain_wait();
  if (threadIdx.x != 0) return;
  st->head = st->head_old + st->app;
  if (st->app > 0) st->t_last = rt[(st->head - 1) % cap];
}

// 6. the stream's FP32 grid for the pixels whose sums changed since the last
// push (marked by k_ring_apply): a warp takes 32 pixels, ballots their marks
// and converts each marked pixel with all lanes (rounding each 64-bit sum to
// the nearest FP32), then clears the marks.  An unchanged sum converts to the
// same FP32 value, so unmarked pixels keep their previous conversion.
__global__ void __launch_bounds__(256) k_fixed_to_float_dirty(const long long *__restrict__ acc64,
                                                              float4 *__restrict__ acc,
                                                              uint8_t *__restrict__ dirty,
                                                              long long P, int U) {
  chain_wait();
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  const float s = 2.3283064365386963e-10f;  // 2^-32
  for (long long p0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
       p0 < P; p0 += nw * 32) {
    const long long pl = p0 + lane;
    const bool mark = pl < P && dirty[pl] != 0;
    unsigned m = __ballot_sync(0xffffffffu, mark);
    if (mark) dirty[pl] = 0;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const long long p = p0 + b;
      for (int u = lane; u < U; u += 32) {
        const size_t i = (size_t)p * U + u;
        const longlong2 a = reinterpret_cast<const longlong2 *>(acc64)[2 * i];
        const longlong2 c = reinterpret_cast<const longlong2 *>(acc64)[2 * i + 1];
        acc[i] = make_float4(__ll2float_rn(a.x) * s, __ll2float_rn(a.y) * s,
                             __ll2float_rn(c.x) * s, __ll2float_rn(c.y) * s);
      }
    }
  }
}

}  // namespace
VK_CHECK_READER(check_read_stream)

}  // namespace veckm

using namespace veckm;

struct veckm_stream {
  veckm_ctx *c = nullptr;
  int64_t window = 0, cap = 0;
  long long *acc64 = nullptr;
  float4 *accf = nullptr;    // the window's per-pixel sums in FP32 (the row pass input)
  uint8_t *dirty = nullptr;  // pixels whose sums changed since the last conversion
  int *cnt = nullptr;
  int16_t *rx = nullptr, *ry = nullptr;
  uint32_t *rt = nullptr;
  int64_t *K = nullptr;
  RingState *st = nullptr;
  int *flag = nullptr, *off = nullptr, *cur = nullptr, *bsum = nullptr, *nvalid = nullptr;
  unsigned *tkey = nullptr, *bmax = nullptr;
  bool pushed = false;    // a packet (or an empty push) has set t_hi
  uint32_t last_t_hi = 0; // t_hi of the last push
};

extern "C" {

veckm_status veckm_stream_create(veckm_ctx *c, int64_t window_us, int64_t capacity,
                                 veckm_stream **out) {
  if (!out) return fail_msg(VECKM_EINVAL, "null output");
  *out = nullptr;
  if (!c) return fail_msg(VECKM_EINVAL, "null context");
  if (window_us < 0 || window_us > 0xffffffffLL) return fail_msg(VECKM_EINVAL, "window outside 0..2^32-1 us");
  if (capacity < 1 || capacity > VECKM_MAX_EVENTS) return fail_msg(VECKM_EINVAL, "capacity outside 1..2^30");
  veckm_stream *s = new (std::nothrow) veckm_stream();
  if (!s) return fail_msg(VECKM_ENOMEM, "host allocation");
  s->c = c;
  s->window = window_us;
  s->cap = capacity;
  const size_t P = (size_t)c->g.W * c->g.H;
  cudaError_t e = dev_malloc(reinterpret_cast<void **>(&s->acc64), P * (size_t)c->g.U * 4 * sizeof(long long));
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->accf), P * (size_t)c->g.U * sizeof(float4));
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->dirty), P);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->cnt), P * sizeof(int));
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->rx), (size_t)capacity * 2);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->ry), (size_t)capacity * 2);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->rt), (size_t)capacity * 4);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->K), (size_t)capacity * 8);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->st), sizeof(RingState));
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->flag), (size_t)capacity * 4);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->off), ((size_t)capacity + 1) * 4);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->cur), (size_t)capacity * 4);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->bsum), (size_t)scan_blocks(capacity) * 4);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->nvalid), 4);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&s->tkey), (size_t)capacity * 4);
  if (e == cudaSuccess)
    e = dev_malloc(reinterpret_cast<void **>(&s->bmax), (size_t)((capacity + kMaxBlock - 1) / kMaxBlock) * 4);
  if (e == cudaSuccess) e = cudaMemset(s->acc64, 0, P * (size_t)c->g.U * 4 * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(s->accf, 0, P * (size_t)c->g.U * sizeof(float4));
  if (e == cudaSuccess) e = cudaMemset(s->dirty, 0, P);
  if (e == cudaSuccess) e = cudaMemset(s->cnt, 0, P * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(s->st, 0, sizeof(RingState));
  if (e != cudaSuccess) {
    veckm_stream_destroy(s);
    return fail_cuda(e, "stream buffers");
  }
  *out = s;
  return VECKM_OK;
}

veckm_status veckm_stream_push(veckm_stream *s, const int16_t *d_x, const int16_t *d_y,
                               const uint32_t *d_t, int64_t n, uint32_t t_hi_us, float *d_out,
                               int32_t predict, void *stream) {
  if (!s) return fail_msg(VECKM_EINVAL, "null stream");
  if (n < 0 || n > s->cap) return fail_msg(VECKM_EINVAL, "packet of %lld events for a ring of %lld", (long long)n, (long long)s->cap);
  if (n > 0 && (!d_x || !d_y || !d_t || !d_out)) return fail_msg(VECKM_EINVAL, "null buffer");
  veckm_ctx *c = s->c;
  const Geometry &g = c->g;
  if (predict && g.D > 128 && (c->flags & (VECKM_MLP_BF16 | VECKM_MLP_FP16)))
    return fail_msg(VECKM_EUNSUPPORTED, "tensor-core perceptron supports D <= 128");
  if (s->pushed && t_hi_us < s->last_t_hi)
    return fail_msg(VECKM_EINVAL, "t_hi %u is before the previous push's %u: a window never "
                    "slides back", (unsigned)t_hi_us, (unsigned)s->last_t_hi);
  s->pushed = true;
  s->last_t_hi = t_hi_us;
  cudaStream_t cs = (cudaStream_t)stream;
  grids_dirty(c);  // the push pools through hbuf into acc
  const uint32_t t_lo = t_hi_us >= (uint64_t)s->window ? t_hi_us - (uint32_t)s->window : 0u;
  const int DV = g.U / 32;
  // The kernels of a push that follow another of its kernels are chained to
  // it (programmatic dependent launch, chain.cuh), up to the row pass; the
  // column pass follows the join with the side stream, and of the kernels
  // after it only the tensor-core head is chained.  Launch errors are read
  // back below (cudaPeekAtLastError).
  auto apply = [&](int sign) {
    const dim3 blocks(num_sms() * 8);
    const long long npx = (long long)g.W * g.H;
#define VECKM_APPLY(DV_)                                                                     \
  (void)launch_kernel(k_ring_apply<DV_>, blocks, dim3(256), 0, cs, true, s->st, sign, s->rx,    \
                      s->ry, s->rt, s->cap, g.W, g.U, npx, c->wt, s->acc64, s->cnt, s->dirty)
    switch (DV) {
      case 1: VECKM_APPLY(1); break;
      case 2: VECKM_APPLY(2); break;
      case 3: VECKM_APPLY(3); break;
      default: VECKM_APPLY(4); break;
    }
#undef VECKM_APPLY
  };
  int launches = 0;
  // 1. valid events and their places
  if (n > 0) {
    k_ring_flags<<<(unsigned)((n + 255) / 256), 256, 0, cs>>>(d_x, d_y, d_t, n, g.W, g.H, t_lo, t_hi_us, s->flag, s->tkey, c->err);
    const int nbm = (int)((n + kMaxBlock - 1) / kMaxBlock);
    (void)launch_kernel(k_tmax_reduce, dim3(nbm), dim3(kMaxThreads), 0, cs, true, s->tkey, n,
                        s->bmax);
    (void)launch_kernel(k_tmax_top, dim3(1), dim3(kMaxThreads), 0, cs, true, s->bmax, nbm);
    (void)launch_kernel(k_tmax_order, dim3(nbm), dim3(kMaxThreads), 0, cs, true, s->tkey, n,
                        s->bmax, s->st, s->flag, c->err);
    launches += 3;
    Geometry line{};
    line.W = (int)n;
    line.H = 1;
    const int r = launch_scan(line, s->flag, s->bsum, s->off, s->cur, s->nvalid, cs, true);
    if (r < 0) return fail_cuda(cudaGetLastError(), "stream scan launch");
    launches += 1 + r;
  }
  // 2-3. expire (the first kernel of a push without events keeps full order)
  (void)launch_kernel(k_ring_tail, dim3(1), dim3(32), 0, cs, n > 0, s->st, s->rt, s->cap, t_lo,
                      n > 0 ? s->nvalid : nullptr);
  apply(-1);
  launches += 2;
  // 4-5. append and add
  if (n > 0) {
    (void)launch_kernel(k_ring_append, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, cs, true,
                        s->st, d_x, d_y, d_t, n, s->flag, s->off, s->rx, s->ry, s->rt, s->cap,
                        s->K, c->err);
    apply(+1);
    launches += 2;
  }
  (void)launch_kernel(k_ring_advance, dim3(1), dim3(32), 0, cs, true, s->st, s->rt, s->cap);
  launches += 1;
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail_cuda(e, "stream update launch");
  }
  if (n == 0) {
    c->last_launches = launches;
    return VECKM_OK;
  }
  // 6. the window's grid, pooling, then the packet's outputs
  int r;
  // the window counts on the context's side stream, under the conversion and
  // the row pass; joined before the column pass (on every return once forked)
  struct Join {
    cudaStream_t s;
    cudaEvent_t ev;
    bool armed = false;
    ~Join() {
      if (armed) cudaStreamWaitEvent(s, ev, 0);
    }
  } join{cs, c->ev_join};
  {
    cudaError_t fe = cudaEventRecord(c->ev_fork, cs);
    if (fe == cudaSuccess) fe = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    if (fe != cudaSuccess) return fail_cuda(fe, "forking the window counts");
    r = launch_counts(g, s->cnt, c->cnt_tmp, c->ncnt, c->side);
    fe = cudaEventRecord(c->ev_join, c->side);
    join.armed = true;
    if (r < 0 || fe != cudaSuccess) return fail_cuda(cudaGetLastError(), "window count launch");
    launches += r;
  }
  const long long P = (long long)g.W * g.H;
  if (launch_kernel(k_fixed_to_float_dirty,
                    dim3((unsigned)std::min<long long>((P + 255) / 256, (long long)num_sms() * 8)),
                    dim3(256), 0, cs, true, s->acc64, s->accf, s->dirty, P, g.U) != cudaSuccess)
    return fail_cuda(cudaGetLastError(), "stream conversion launch");
  launches += 1;
  const Tables tb = c->tables();
  const Tune tn = c->tune_for(g);
  if ((r = launch_pool_rows(g, tb, s->accf, c->hbuf, cs, tn, nullptr, true)) < 0) return fail_cuda(cudaGetLastError(), "pooling (rows) launch");
  launches += r;
  if (join.armed) {
    cudaStreamWaitEvent(cs, c->ev_join, 0);
    join.armed = false;
  }
  const Events ev{s->rx, s->ry, s->rt, s->cap, 0u, 0xffffffffu};
  const bool tc_head = predict && (c->flags & (VECKM_MLP_BF16 | VECKM_MLP_FP16));
  const bool half_grid = tc_head && (c->flags & VECKM_ACC_FP16);
  r = half_grid ? launch_pool_cols_half(g, tb, c->hbuf, c->ncnt, c->acc, cs, tn)
      : tc_head ? launch_pool_cols_pair(g, tb, c->hbuf, c->acc, cs, tn)
                : launch_pool_cols(g, tb, c->hbuf, c->acc, cs, tn);
  if (r < 0) return fail_cuda(cudaGetLastError(), "pooling (columns) launch");
  launches += r;
  if (!predict) {
    r = launch_gather_emb(ev, s->K, n, g, tb, c->acc, c->ncnt, d_out, c->err, cs);
  } else if (c->flags & (VECKM_MLP_BF16 | VECKM_MLP_FP16)) {
    MLP m = c->mlp();
    m.pooled_half = half_grid ? 1 : 0;
    r = launch_predict_tc(ev, s->K, n, nullptr, nullptr, nullptr, g, tb, c->acc, c->ncnt, m,
                          d_out, c->err, cs, tn, nullptr, 0, nullptr, true);
  } else {
    r = launch_predict_fp32(ev, s->K, n, nullptr, nullptr, nullptr, g, tb, c->acc, c->ncnt,
                            c->mlp(), d_out, c->err, cs);
    if (r == -2) return fail_msg(VECKM_EUNSUPPORTED, "FP32 perceptron supports D <= 128");
  }
  if (r < 0) return fail_cuda(cudaGetLastError(), "gather launch");
  c->last_launches = launches + r;
  return VECKM_OK;
}

veckm_status veckm_stream_window(veckm_stream *s, int64_t *h_events, void *stream) {
  if (!s || !h_events) return fail_msg(VECKM_EINVAL, "null argument");
  RingState h{};
  cudaError_t e = cudaMemcpyAsync(&h, s->st, sizeof h, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail_cuda(e, "stream state");
  *h_events = h.head - h.tail;
  return VECKM_OK;
}

veckm_status veckm_stream_accumulator(veckm_stream *s, int64_t *h_acc, int32_t *h_cnt, void *stream) {
  if (!s || !h_acc || !h_cnt) return fail_msg(VECKM_EINVAL, "null argument");
  const size_t P = (size_t)s->c->g.W * s->c->g.H;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h_acc, s->acc64, P * (size_t)s->c->g.U * 4 * 8, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt, s->cnt, P * 4, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  return e == cudaSuccess ? VECKM_OK : fail_cuda(e, "stream accumulator copy");
}

void veckm_stream_destroy(veckm_stream *s) {
  if (!s) return;
  cudaDeviceSynchronize();
  void *ptrs[] = {s->acc64, s->accf, s->dirty, s->cnt, s->rx, s->ry, s->rt, s->K, s->st,
                  s->flag, s->off, s->cur, s->bsum, s->nvalid, s->tkey, s->bmax};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete s;
}

}  // extern "C"
