// CUDA-core kernels of the encoder: scatter (Algorithm 1, lines 7-10), the
// separable window pooling that replaces the adjacency-matrix product (lines
// 11-20, Eq. 16-17), the gather with the conjugate temporal phase and the
// division by the window count (line 21), and the plain FP32 perceptron.
//
// Layout: a pixel p = y*W + x holds D complex FP32 values interleaved
// (re, im), channel fastest; float4 unit u of a pixel holds channels 2u and
// 2u+1.  A warp covers 32 consecutive units (512 bytes) of one pixel, so every
// per-pixel access below is a fully coalesced 512-byte transaction.
//
// Phases are never evaluated with trigonometry on the device.  They are
// products of FP32 table rows that the host computed in FP64:
//   exp(i t_rel T/dt) = tt_hi[t_rel >> 6] * tt_lo[t_rel & 63]
//   exp(i x X/dx)     = tx[x],   exp(i y Y/dy) = ty[y].
//
// The pooling uses the modulation identity behind Eq. 16:
//   sum_q A[q] exp(i (q-p).w) = conj(phi(p)) * sum_q (A[q] phi(q)),
// phi(q) = exp(i q.w), so the complex 2-D window convolution becomes a
// plain box sum between a modulation and a demodulation, done as a row pass
// then a column pass.  Each box sum uses the van Herk / Gil-Werman block
// scheme (blocks of the window length L; a window is the suffix of one block
// plus the prefix of the next), so every window sum adds only values inside
// that window: no running-sum subtraction, whose cancellation next to a
// dense pixel would destroy the result of a sparse one.
#include <cuda_runtime.h>

#include <algorithm>

#include "veckm_internal.h"

namespace veckm {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// Two complex products: (a.x + i a.y)(b.x + i b.y) and (a.z + i a.w)(b.z + i b.w).
__device__ __forceinline__ float4 cmul2(float4 a, float4 b) {
  return make_float4(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x),
                     fmaf(a.z, b.z, -a.w * b.w), fmaf(a.z, b.w, a.w * b.z));
}

// a * conj(b), two complex lanes.
__device__ __forceinline__ float4 cmul2c(float4 a, float4 b) {
  return make_float4(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y),
                     fmaf(a.z, b.z, a.w * b.w), fmaf(a.w, b.z, -a.z * b.w));
}

__device__ __forceinline__ void red_add_v4(float4 *p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

__device__ __forceinline__ bool event_ok(int x, int y, uint32_t t, const Events &ev, int W, int H,
                                         uint32_t &trel) {
  trel = t - ev.t_ref;
  return x >= 0 && x < W && y >= 0 && y < H && t >= ev.t_ref && trel <= ev.t_span;
}

// exp(i t_rel T/dt) for unit u: hi row from global (L1-resident; events are
// time-sorted, so a warp reuses one hi row), lo row from shared memory.
__device__ __forceinline__ float4 time_phase(const float4 *__restrict__ tt_hi, const float4 *s_lo,
                                             uint32_t trel, int U, int u) {
  const float4 hi = __ldg(tt_hi + (size_t)(trel >> kTLoBits) * U + u);
  const float4 lo = s_lo[(trel & (kTLo - 1)) * U + u];
  return cmul2(hi, lo);
}

// ---------------------------------------------------------------------------
// Scatter: PixelEmbed[p] += exp(i t T/dt), PixelCount[p] += 1.
// One warp takes 32 consecutive events; lanes that hit the same pixel are
// grouped with __match_any_sync, the group's phases are summed in registers
// and the group issues one vector reduction per unit and one count add.
template <int DV>
__global__ void __launch_bounds__(256) k_scatter(Events ev, Geometry g, Tables tb,
                                                 float4 *__restrict__ acc, int *__restrict__ cnt,
                                                 int *__restrict__ err) {
  constexpr int U = 32 * DV;
  extern __shared__ float4 s_lo[];  // [64][U]
  for (int i = threadIdx.x; i < kTLo * U; i += blockDim.x) s_lo[i] = tb.tt_lo[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int64_t nchunks = (ev.n + 31) >> 5;
  for (int64_t c = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); c < nchunks;
       c += (int64_t)gridDim.x * wpb) {
    const int64_t k = c * 32 + lane;
    int key = -1;
    uint32_t trel = 0;
    if (k < ev.n) {
      const int x = ev.x[k], y = ev.y[k];
      if (event_ok(x, y, ev.t[k], ev, g.W, g.H, trel))
        key = y * g.W + x;
      else
        atomicOr(err, ERR_EVENT_RANGE);
    }
    const unsigned grp = __match_any_sync(kFull, key);
    const bool leader = key >= 0 && (__ffs(grp) - 1) == lane;
    unsigned todo = __ballot_sync(kFull, leader);
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      unsigned members = __shfl_sync(kFull, grp, j);
      const int pix = __shfl_sync(kFull, key, j);
      const int m_count = __popc(members);
      float4 s[DV];
#pragma unroll
      for (int v = 0; v < DV; ++v) s[v] = f4zero();
      while (members) {
        const int m = __ffs(members) - 1;
        members &= members - 1;
        const uint32_t tm = __shfl_sync(kFull, trel, m);
#pragma unroll
        for (int v = 0; v < DV; ++v) s[v] = add4(s[v], time_phase(tb.tt_hi, s_lo, tm, U, lane + 32 * v));
      }
      float4 *dst = acc + (size_t)pix * U;
#pragma unroll
      for (int v = 0; v < DV; ++v) red_add_v4(dst + lane + 32 * v, s[v]);
      if (lane == 0) atomicAdd(cnt + pix, m_count);
    }
  }
}

// ---------------------------------------------------------------------------
// Separable pooling.  One warp walks one line segment (a row segment in the
// row pass, a column segment in the column pass) with lanes over units.
// Walker state per lane lives in shared memory: L values, reused as the
// suffix sums of the current block.
enum class Pass { Rows, Cols };

template <int DV, Pass P>
__global__ void __launch_bounds__(128) k_pool_pass(const float4 *__restrict__ src,
                                                   float4 *__restrict__ dst, Geometry g, Tables tb,
                                                   int seg, int nseg) {
  constexpr int U = 32 * DV;
  extern __shared__ float4 smem[];
  const int r = (P == Pass::Rows) ? g.dx : g.dy;
  const int L = 2 * r + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4 *sv = smem + (size_t)warp * L * U;
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const int nlines = (P == Pass::Rows) ? g.H : g.W;
  const int len = (P == Pass::Rows) ? g.W : g.H;
  if (wid >= (int64_t)nlines * nseg) return;
  const int line = (int)(wid / nseg), s = (int)(wid % nseg);
  const int o0 = s * seg;
  const int nout = min(len, o0 + seg) - o0;
  const int in0 = o0 - r;
  // element pos of this line is at base + pos * stride (float4 units)
  const size_t base = (P == Pass::Rows) ? (size_t)line * g.W * U : (size_t)line * U;
  const size_t stride = (P == Pass::Rows) ? (size_t)U : (size_t)g.W * U;
  // Row pass: modulate by tx on input; demodulate by conj(tx) and modulate by
  // ty[line] on output.  Column pass: demodulate by conj(ty) on output.
  float4 fy[DV];
  if (P == Pass::Rows) {
#pragma unroll
    for (int v = 0; v < DV; ++v) fy[v] = __ldg(tb.ty + (size_t)line * U + lane + 32 * v);
  }
  auto load = [&](int i, float4(&w)[DV]) {
    const int pos = in0 + i;
    if (pos >= 0 && pos < len) {
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        const int u = lane + 32 * v;
        const float4 a = __ldg(src + base + (size_t)pos * stride + u);
        w[v] = (P == Pass::Rows) ? cmul2(a, __ldg(tb.tx + (size_t)pos * U + u)) : a;
      }
    } else {
#pragma unroll
      for (int v = 0; v < DV; ++v) w[v] = f4zero();
    }
  };
  auto emit = [&](int j, const float4(&sum)[DV]) {
    const int pos = o0 + j;
#pragma unroll
    for (int v = 0; v < DV; ++v) {
      const int u = lane + 32 * v;
      float4 o;
      if (P == Pass::Rows)
        o = cmul2(sum[v], cmul2c(fy[v], __ldg(tb.tx + (size_t)pos * U + u)));
      else
        o = cmul2c(sum[v], __ldg(tb.ty + (size_t)pos * U + u));
      dst[base + (size_t)pos * stride + u] = o;
    }
  };
  // suffix sums of input block 0
  {
    float4 run[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) run[v] = f4zero();
    for (int q = L - 1; q >= 0; --q) {
      float4 w[DV];
      load(q, w);
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        run[v] = add4(run[v], w[v]);
        sv[q * U + lane + 32 * v] = run[v];
      }
    }
  }
  const int nb = (nout + L - 1) / L;
  for (int b = 0; b < nb; ++b) {
    const int j0 = b * L;
    {
      float4 s0[DV];
#pragma unroll
      for (int v = 0; v < DV; ++v) s0[v] = sv[lane + 32 * v];
      emit(j0, s0);  // window == block b
    }
    float4 G[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) G[v] = f4zero();
    for (int q = 0; q < L; ++q) {
      float4 w[DV];
      load((b + 1) * L + q, w);
#pragma unroll
      for (int v = 0; v < DV; ++v) G[v] = add4(G[v], w[v]);
      if (q + 1 < L && j0 + q + 1 < nout) {
        float4 o[DV];
#pragma unroll
        for (int v = 0; v < DV; ++v) o[v] = add4(sv[(q + 1) * U + lane + 32 * v], G[v]);
        emit(j0 + q + 1, o);  // suffix of block b from q+1, plus prefix of block b+1 to q
      }
#pragma unroll
      for (int v = 0; v < DV; ++v) sv[q * U + lane + 32 * v] = w[v];
    }
    if (b + 1 < nb) {  // suffix sums of block b+1, in place
      float4 run[DV];
#pragma unroll
      for (int v = 0; v < DV; ++v) run[v] = f4zero();
      for (int q = L - 1; q >= 0; --q) {
#pragma unroll
        for (int v = 0; v < DV; ++v) {
          run[v] = add4(run[v], sv[q * U + lane + 32 * v]);
          sv[q * U + lane + 32 * v] = run[v];
        }
      }
    }
  }
}

// Window counts (Eq. 17): exact integer box sums, rows then columns.
__global__ void k_count_rows(const int *__restrict__ cnt, int *__restrict__ out, int W, int H,
                             int dx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)W * H) return;
  const int y = (int)(i / W), x = (int)(i % W);
  const int *row = cnt + (size_t)y * W;
  int s = 0;
  for (int a = max(0, x - dx); a <= min(W - 1, x + dx); ++a) s += row[a];
  out[i] = s;
}

__global__ void k_count_cols(const int *__restrict__ rows, int *__restrict__ out, int W, int H,
                             int dy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)W * H) return;
  const int y = (int)(i / W), x = (int)(i % W);
  int s = 0;
  for (int b = max(0, y - dy); b <= min(H - 1, y + dy); ++b) s += rows[(size_t)b * W + x];
  out[i] = s;
}

// ---------------------------------------------------------------------------
// Gather for one event: pooled[p] * conj(exp(i t T/dt)) / n_p.  Returns false
// (and zeros) for an invalid index or event.
template <int DV>
__device__ __forceinline__ bool gather_event(const Events &ev, const int64_t *__restrict__ K,
                                             int64_t nK, int64_t i, const Geometry &g,
                                             const Tables &tb, const float4 *s_lo,
                                             const float4 *__restrict__ pooled,
                                             const int *__restrict__ ncnt, int lane,
                                             float4 (&e)[DV], int *err) {
  constexpr int U = 32 * DV;
#pragma unroll
  for (int v = 0; v < DV; ++v) e[v] = f4zero();
  int64_t k = i;
  if (K) {
    k = K[i];
    if (k < 0 || k >= ev.n) {
      if (lane == 0) atomicOr(err, ERR_INDEX_RANGE);
      return false;
    }
  }
  const int x = ev.x[k], y = ev.y[k];
  uint32_t trel;
  if (!event_ok(x, y, ev.t[k], ev, g.W, g.H, trel)) return false;  // flagged by the scatter
  const int pix = y * g.W + x;
  const float inv = 1.0f / (float)__ldg(ncnt + pix);
#pragma unroll
  for (int v = 0; v < DV; ++v) {
    const int u = lane + 32 * v;
    const float4 pv = __ldg(pooled + (size_t)pix * U + u);
    const float4 ph = time_phase(tb.tt_hi, s_lo, trel, U, u);
    float4 o = cmul2c(pv, ph);
    o.x *= inv; o.y *= inv; o.z *= inv; o.w *= inv;
    e[v] = o;
  }
  return true;
}

template <int DV>
__global__ void __launch_bounds__(256) k_gather_emb(Events ev, const int64_t *__restrict__ K,
                                                    int64_t nK, Geometry g, Tables tb,
                                                    const float4 *__restrict__ pooled,
                                                    const int *__restrict__ ncnt,
                                                    float *__restrict__ emb, int *err) {
  constexpr int U = 32 * DV;
  extern __shared__ float4 s_lo[];
  for (int i = threadIdx.x; i < kTLo * U; i += blockDim.x) s_lo[i] = tb.tt_lo[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const int D = g.D;
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < nK;
       i += (int64_t)gridDim.x * wpb) {
    float4 e[DV];
    gather_event<DV>(ev, K, nK, i, g, tb, s_lo, pooled, ncnt, lane, e, err);
    float *row = emb + (size_t)i * 2 * D;
#pragma unroll
    for (int v = 0; v < DV; ++v) {
      const int u = lane + 32 * v;
      *reinterpret_cast<float2 *>(row + 2 * u) = make_float2(e[v].x, e[v].z);
      *reinterpret_cast<float2 *>(row + D + 2 * u) = make_float2(e[v].y, e[v].w);
    }
  }
}

// ---------------------------------------------------------------------------
// Plain FP32 perceptron fused with the gather.  A CTA takes 64 events: the
// 8 warps gather their rows into shared memory, then thread (eg, hg) computes
// a 4-event x 8-hidden block of the first layer from W1^T in shared memory,
// applies bias and ReLU, reduces its share of the second layer and the 16
// threads of an event group combine their partial outputs with shuffles.
constexpr int kHid = 128;
constexpr int kTM = 64;

template <int DV>
__global__ void __launch_bounds__(256) k_predict_fp32(Events ev, const int64_t *__restrict__ K,
                                                      int64_t nK, Geometry g, Tables tb,
                                                      const float4 *__restrict__ pooled,
                                                      const int *__restrict__ ncnt, MLP mlp,
                                                      float *__restrict__ flow, int *err) {
  constexpr int U = 32 * DV, IN = 4 * U, LDE = IN + 4;
  extern __shared__ float4 smem4[];
  const float4 *s_lo = tb.tt_lo;  // low time table read through L1 (shared memory holds W1^T)
  float *sW = reinterpret_cast<float *>(smem4);           // [IN][kHid]
  float *sE = sW + IN * kHid;                             // [kTM][LDE]
  float *sB1 = sE + kTM * LDE;                            // [kHid]
  float *sW2 = sB1 + kHid;                                // [2][kHid]
  for (int i = threadIdx.x; i < IN * kHid / 4; i += blockDim.x)
    reinterpret_cast<float4 *>(sW)[i] = __ldg(reinterpret_cast<const float4 *>(mlp.W1t) + i);
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    sB1[i] = mlp.b1[i];
    sW2[i] = mlp.W2[i];
    sW2[kHid + i] = mlp.W2[kHid + i];
  }
  __syncthreads();
  const float b20 = mlp.b2[0], b21 = mlp.b2[1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int eg = threadIdx.x >> 4, hg = threadIdx.x & 15;
  const int D = g.D;
  for (int64_t tile = blockIdx.x; tile * kTM < nK; tile += gridDim.x) {
    for (int rr = 0; rr < kTM / 8; ++rr) {
      const int row = warp * (kTM / 8) + rr;
      const int64_t i = tile * kTM + row;
      float4 e[DV];
      if (i < nK)
        gather_event<DV>(ev, K, nK, i, g, tb, s_lo, pooled, ncnt, lane, e, err);
      else {
#pragma unroll
        for (int v = 0; v < DV; ++v) e[v] = f4zero();
      }
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        const int u = lane + 32 * v;
        *reinterpret_cast<float2 *>(sE + row * LDE + 2 * u) = make_float2(e[v].x, e[v].z);
        *reinterpret_cast<float2 *>(sE + row * LDE + D + 2 * u) = make_float2(e[v].y, e[v].w);
      }
    }
    __syncthreads();
    float a[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[i][j] = sB1[8 * hg + j];
    const float *e0 = sE + (4 * eg) * LDE;
#pragma unroll 4
    for (int c = 0; c < IN; ++c) {
      const float4 w0 = *reinterpret_cast<const float4 *>(sW + c * kHid + 8 * hg);
      const float4 w1 = *reinterpret_cast<const float4 *>(sW + c * kHid + 8 * hg + 4);
      const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float xv = e0[i * LDE + c];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[i][j] = fmaf(xv, w[j], a[i][j]);
      }
    }
    float o[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[i][0] = 0.f;
      o[i][1] = 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float h = fmaxf(a[i][j], 0.f);
        o[i][0] = fmaf(h, sW2[8 * hg + j], o[i][0]);
        o[i][1] = fmaf(h, sW2[kHid + 8 * hg + j], o[i][1]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) o[i][c] += __shfl_xor_sync(kFull, o[i][c], off);
    if (hg == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t idx = tile * kTM + 4 * eg + i;
        if (idx < nK)
          *reinterpret_cast<float2 *>(flow + 2 * idx) = make_float2(o[i][0] + b20, o[i][1] + b21);
      }
    }
    __syncthreads();
  }
}

template <typename KernelT>
cudaError_t set_smem(KernelT k, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int DV>
int scatter_impl(const Events &ev, const Geometry &g, const Tables &tb, float4 *acc, int *cnt,
                 int *err, cudaStream_t s) {
  if (ev.n == 0) return 0;
  const size_t sm = (size_t)kTLo * 32 * DV * sizeof(float4);
  if (set_smem(k_scatter<DV>, sm) != cudaSuccess) return -1;
  const int64_t nchunks = (ev.n + 31) / 32;
  const int64_t want = (nchunks + 7) / 8;
  const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms() * 6);
  k_scatter<DV><<<grid, 256, sm, s>>>(ev, g, tb, acc, cnt, err);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <int DV, Pass P>
int pool_pass(const Geometry &g, const Tables &tb, const float4 *src, float4 *dst, cudaStream_t s) {
  const int r = (P == Pass::Rows) ? g.dx : g.dy;
  const int L = 2 * r + 1;
  const int len = (P == Pass::Rows) ? g.W : g.H;
  const int nlines = (P == Pass::Rows) ? g.H : g.W;
  const int seg = L * std::max(1, (96 + L / 2) / L);
  const int nseg = (len + seg - 1) / seg;
  const size_t per_warp = (size_t)L * 32 * DV * sizeof(float4);
  int wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (200 * 1024) / per_warp));
  const size_t sm = per_warp * wpb;
  if (set_smem(k_pool_pass<DV, P>, sm) != cudaSuccess) return -1;
  const int64_t warps = (int64_t)nlines * nseg;
  const int grid = (int)((warps + wpb - 1) / wpb);
  k_pool_pass<DV, P><<<grid, 32 * wpb, sm, s>>>(src, dst, g, tb, seg, nseg);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <int DV>
int gather_impl(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                const Tables &tb, const float4 *pooled, const int *ncnt, float *emb, int *err,
                cudaStream_t s) {
  if (nK == 0) return 0;
  const size_t sm = (size_t)kTLo * 32 * DV * sizeof(float4);
  if (set_smem(k_gather_emb<DV>, sm) != cudaSuccess) return -1;
  const int grid = (int)std::min<int64_t>((nK + 7) / 8, (int64_t)num_sms() * 8);
  k_gather_emb<DV><<<grid, 256, sm, s>>>(ev, K, nK, g, tb, pooled, ncnt, emb, err);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <int DV>
int predict_fp32_impl(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                      const Tables &tb, const float4 *pooled, const int *ncnt, const MLP &mlp,
                      float *flow, int *err, cudaStream_t s) {
  if (nK == 0) return 0;
  constexpr int U = 32 * DV, IN = 4 * U;
  const size_t sm = sizeof(float) * ((size_t)IN * kHid + (size_t)kTM * (IN + 4) + 3 * kHid);
  if (sm > 227 * 1024) return -2;  // W1^T does not fit in shared memory
  if (set_smem(k_predict_fp32<DV>, sm) != cudaSuccess) return -1;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_predict_fp32<DV>, 256, sm);
  const int64_t tiles = (nK + kTM - 1) / kTM;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * std::max(1, per_sm));
  k_predict_fp32<DV><<<grid, 256, sm, s>>>(ev, K, nK, g, tb, pooled, ncnt, mlp, flow, err);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

#define VECKM_DISPATCH_DV(U, CALL)          \
  switch ((U) / 32) {                       \
    case 1: { constexpr int DV = 1; return CALL; } \
    case 2: { constexpr int DV = 2; return CALL; } \
    case 3: { constexpr int DV = 3; return CALL; } \
    case 4: { constexpr int DV = 4; return CALL; } \
    default: return -1;                     \
  }

int launch_scatter(const Events &ev, const Geometry &g, const Tables &tb, float4 *acc, int *cnt,
                   int *err, cudaStream_t s) {
  VECKM_DISPATCH_DV(g.U, (scatter_impl<DV>(ev, g, tb, acc, cnt, err, s)));
}

int launch_pool_rows(const Geometry &g, const Tables &tb, const float4 *acc, float4 *hbuf,
                     cudaStream_t s) {
  VECKM_DISPATCH_DV(g.U, (pool_pass<DV, Pass::Rows>(g, tb, acc, hbuf, s)));
}

int launch_pool_cols(const Geometry &g, const Tables &tb, const float4 *hbuf, float4 *acc,
                     cudaStream_t s) {
  VECKM_DISPATCH_DV(g.U, (pool_pass<DV, Pass::Cols>(g, tb, hbuf, acc, s)));
}

int launch_counts(const Geometry &g, const int *cnt, int *cnt_tmp, int *ncnt, cudaStream_t s) {
  const int64_t P = (int64_t)g.W * g.H;
  const int grid = (int)((P + 255) / 256);
  k_count_rows<<<grid, 256, 0, s>>>(cnt, cnt_tmp, g.W, g.H, g.dx);
  k_count_cols<<<grid, 256, 0, s>>>(cnt_tmp, ncnt, g.W, g.H, g.dy);
  return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

int launch_gather_emb(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                      const Tables &tb, const float4 *pooled, const int *ncnt, float *emb,
                      int *err, cudaStream_t s) {
  VECKM_DISPATCH_DV(g.U, (gather_impl<DV>(ev, K, nK, g, tb, pooled, ncnt, emb, err, s)));
}

int launch_predict_fp32(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                        const Tables &tb, const float4 *pooled, const int *ncnt, const MLP &mlp,
                        float *flow, int *err, cudaStream_t s) {
  VECKM_DISPATCH_DV(g.U,
                    (predict_fp32_impl<DV>(ev, K, nK, g, tb, pooled, ncnt, mlp, flow, err, s)));
}

}  // namespace veckm
