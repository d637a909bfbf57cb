// CUDA-core kernels of the encoder.
//
// Pipeline for one slice (Algorithm 1 with the pooling reformulation of
// Eq. 13-17, Section 2.2.2):
//   1-3. sort by pixel: PixelCount[p] and a record (t - t_ref, k) for every
//                 event in its pixel's segment of a pixel-sorted order.  The
//                 bucket form (k_bucket_*, below) where the geometry and
//                 event count allow it, else:
//     1. k_hist     PixelCount[p] += 1 for every event.
//     2. k_scan_*   exclusive prefix sum of the counts: each pixel's segment.
//     3. k_place    counting-sort placement of each record into its segment.
//   4. k_pixsum   PixelEmbed[p] = sum over the segment of exp(i t T/dt), in
//                 record chunks of equal size; plain stores inside a chunk,
//                 vector reductions only for the two pixels at its ends.
//   5. k_box_pass rows, then columns: box sums over the (2dx+1) x (2dy+1)
//                 window of PixelEmbed modulated by the spatial phase
//                 exp(i (x X/dx + y Y/dy)) (row pass), demodulated by the
//                 conjugate phase of the output pixel (column pass).  Because
//                   sum_q A[q] exp(i (q-p).w) = conj(phi(p)) sum_q A[q] phi(q)
//                 with phi(q) = exp(i q.w), this equals the window sum with
//                 the precomputed spatial factors of Eq. 16.
//   6. k_count_box window counts n (Eq. 17), exact integer box sums (one tiled pass).
//   7. gather     pooled[p] * conj(exp(i t T/dt)) / n (Eq. 16), fused with the
//                 perceptron (mlp_tc.cu, or the FP32 kernel below).
//
// Layout: a pixel p = y*W + x holds D complex FP32 values interleaved
// (re, im), channel fastest; float4 unit u of a pixel holds channels 2u and
// 2u+1.  A warp covers 32 consecutive units (512 bytes) of one pixel, so every
// per-pixel access is a fully coalesced 512-byte transaction.
//
// Spatial phases are FP32 table rows computed on the host in FP64,
// exp(i x X/dx) = tx[x] and exp(i y Y/dy) = ty[y]; the temporal phase
// exp(i t T/dt) comes from exact fixed-point argument reduction (phase.cuh),
// so no trigonometric function ever sees an argument outside [-pi, pi).
// Inside a box-pass block the spatial phase advances from a table anchor by
// the exact step rows exp(i X/dx), exp(i Y/dy): in the column pass one step
// per output (at most 2*radius+1 steps, ~(2r+1) x 1.2e-7 relative error); in
// the row pass even and odd positions as two rotations by the squared step
// (at most radius+1 steps each, ~(r+1) x 2.4e-7 with the squared step's own
// rounding).
//
// Box sums use the van Herk / Gil-Werman block scheme (blocks of the window
// length L; each window is the suffix of one block plus the prefix of the
// next), so every window sum adds only values inside that window: there is
// no running-sum subtraction, whose cancellation next to a dense pixel would
// destroy the result of a sparse one.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "chain.cuh"
#include "check.cuh"
#include "phase.cuh"
#include "veckm_internal.h"

namespace veckm {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// a + b as two packed FP32x2 additions (the same roundings as add4)
__device__ __forceinline__ float4 add4x2(float4 a, float4 b) {
  uint64_t lo, hi;
  asm("add.rn.f32x2 %0, %1, %2;"
      : "=l"(lo)
      : "l"(*reinterpret_cast<const uint64_t *>(&a.x)), "l"(*reinterpret_cast<const uint64_t *>(&b.x)));
  asm("add.rn.f32x2 %0, %1, %2;"
      : "=l"(hi)
      : "l"(*reinterpret_cast<const uint64_t *>(&a.z)), "l"(*reinterpret_cast<const uint64_t *>(&b.z)));
  const float2 l = *reinterpret_cast<const float2 *>(&lo), h = *reinterpret_cast<const float2 *>(&hi);
  return make_float4(l.x, l.y, h.x, h.y);
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

__device__ __forceinline__ bool event_ok(int x, int y, uint32_t t, const Events &ev, int W, int H,
                                         uint32_t &trel) {
  trel = t - ev.t_ref;
  return x >= 0 && x < W && y >= 0 && y < H && t >= ev.t_ref && trel <= ev.t_span;
}

// fixed-point frequencies of channels 2u, 2u+1 for each unit this lane owns
template <int DV>
__device__ __forceinline__ void load_freqs(const uint2 *__restrict__ wt, int lane, uint2 (&w)[DV][2]) {
#pragma unroll
  for (int v = 0; v < DV; ++v) {
    const int u = lane + 32 * v;
    w[v][0] = __ldg(wt + 2 * u);
    w[v][1] = __ldg(wt + 2 * u + 1);
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait0() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
constexpr int kPlaceILP = 4;

// 1. counts per pixel (reductions without return value, kPlaceILP events per
// thread).  In pixel-sorted prediction an invalid event never reaches the
// perceptron, so its flow row is zeroed here (zero_flow non-null).
__global__ void __launch_bounds__(256) k_hist(Events ev, Geometry g, int *__restrict__ cnt,
                                              int *__restrict__ err, float *__restrict__ zero_flow) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k0 < ev.n; k0 += stride * 4) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t k = k0 + e * stride;
      if (k < ev.n) {
        uint32_t trel;
        const int x = ev.x[k], y = ev.y[k];
        if (event_ok(x, y, ev.t[k], ev, g.W, g.H, trel)) {
          atomicAdd(cnt + y * g.W + x, 1);
        } else {
          atomicOr(err, ERR_EVENT_RANGE);
          if (zero_flow) *reinterpret_cast<float2 *>(zero_flow + 2 * k) = make_float2(0.f, 0.f);
        }
      }
    }
  }
}

// 2. exclusive scan of P counts in blocks of kScanBlock.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanBlock = kScanThreads * kScanPer;

__device__ __forceinline__ int block_excl_scan(int v, int *s_warp, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += n;
    }
    s_warp[lane] = wi - w;  // exclusive
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  total = s_warp[32];
  const int r = s_warp[warp] + incl - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int *__restrict__ cnt, int64_t P,
                                                              int *__restrict__ bsum) {
  __shared__ int s_warp[33];
  chain_wait();
  const int64_t b0 = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
  int v = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i)
    if (b0 + i < P) v += cnt[b0 + i];
  int total;
  block_excl_scan(v, s_warp, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Exclusive scan of the block sums in place (one CTA, any number of blocks).
__global__ void __launch_bounds__(kScanThreads) k_scan_top(int *__restrict__ bsum, int nb,
                                                           int *__restrict__ total_out) {
  __shared__ int s_warp[33];
  chain_wait();
  int carry = 0;
  for (int base = 0; base < nb; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? bsum[i] : 0;
    int tot;
    const int ex = block_excl_scan(v, s_warp, tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

// off[p] = exclusive prefix, cur[p] = off[p] (placement cursors), off[P] = total.
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int *__restrict__ cnt, int64_t P,
                                                             const int *__restrict__ bsum,
                                                             int *__restrict__ off,
                                                             int *__restrict__ cur) {
  __shared__ int s_warp[33];
  chain_wait();
  const int64_t b0 = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
  int c[kScanPer];
  int v = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    c[i] = (b0 + i < P) ? cnt[b0 + i] : 0;
    v += c[i];
  }
  int total;
  int run = block_excl_scan(v, s_warp, total) + bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    if (b0 + i < P) {
      off[b0 + i] = run;
      cur[b0 + i] = run;
    }
    run += c[i];
  }
  if (b0 < P && b0 + kScanPer >= P) off[P] = run;  // the thread holding the last pixel
}

// 3. placement: rec[pos] = (t - t_ref, k), pix[pos] = p, pos taken from the
// pixel's cursor.  Each thread places kPlaceILP events whose cursor atomics
// are in flight together.

__global__ void __launch_bounds__(256) k_place(Events ev, Geometry g, int *__restrict__ cur,
                                               int2 *__restrict__ rec, int *__restrict__ pix) {
  chain_wait();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k0 < ev.n;
       k0 += stride * kPlaceILP) {
    int key[kPlaceILP], pos[kPlaceILP];
    uint32_t tr[kPlaceILP];
#pragma unroll
    for (int e = 0; e < kPlaceILP; ++e) {
      const int64_t k = k0 + e * stride;
      key[e] = -1;
      tr[e] = 0;
      if (k < ev.n) {
        const int x = ev.x[k], y = ev.y[k];
        if (event_ok(x, y, ev.t[k], ev, g.W, g.H, tr[e])) key[e] = y * g.W + x;
      }
    }
#pragma unroll
    for (int e = 0; e < kPlaceILP; ++e)
      if (key[e] >= 0) pos[e] = atomicAdd(cur + key[e], 1);
#pragma unroll
    for (int e = 0; e < kPlaceILP; ++e)
      if (key[e] >= 0 && VK_CHECK(pos[e] >= 0 && pos[e] < ev.n)) {
        rec[pos[e]] = make_int2((int)tr[e], (int)(k0 + e * stride));
        pix[pos[e]] = key[e];
      }
  }
}

// 1-3 (bucket form).  The same outputs as k_hist + scan + k_place (records
// grouped by pixel, per-pixel counts, the record total) without global
// atomics, and with coalesced writes.  Pixels are grouped into nb buckets of
// 2^shift consecutive pixels; events into tiles of consecutive indices.
//   a. k_bucket_count: per tile, events per bucket (shared-memory atomics);
//      also validates the events (error word, zeroed flows) as k_hist does.
//   b. k_bucket_scan: per bucket, exclusive prefix of its counts over tiles,
//      and the bucket's total.
//   c. k_bucket_scatter: per tile, the valid events (t - t_ref, index, pixel)
//      ranked by bucket in shared memory, then written bucket run by bucket
//      run to the buckets' regions at the tile's cursors.
//   d. k_bucket_sort: per bucket, a counting sort of its records by pixel in
//      shared memory, written out in order (buckets above kSortStage records
//      place them straight into the bucket's region instead); also writes
//      the pixel counts.  With a grid given, it also zeroes the rows of the
//      pixels at the edges of the per-pixel sums' record ranges (the sorted
//      positions c * kPixRecs and c * kPixRecs + kPixRecs - 1), the only
//      pixels those sums add into rather than store: the sums then need no
//      cleared grid.
// Records of one pixel come out in no particular order, as with k_place.
constexpr int kSortThreads = 512;
constexpr int kMaxBuckets = 1024;
constexpr int kMaxBucketShift = 15;  // 32768 pixels: a 128 KB shared histogram
constexpr int kMaxSortTiles = 4096;
constexpr int kSortILP = 8;        // events or records in flight per thread
constexpr int kSortStage = 4096;   // records a bucket sorts in shared memory
// Records per warp in the per-pixel sums (k_pixsum): measured on GB300
// against 64 to 256 and against one wave of longer ranges.
constexpr int kPixRecs = 128;

// Exclusive prefix of v[0..nb) into out[0..nb) (out may be v) and the sum in
// *total, for nb <= 2 * blockDim.x (one block; s_warp holds 33 ints).
__device__ void block_scan_small(const int *v, int nb, int *out, int *total, int *s_warp) {
  const int i0 = 2 * threadIdx.x;
  const int a = i0 < nb ? v[i0] : 0, b = i0 + 1 < nb ? v[i0 + 1] : 0;
  int tot;
  const int ex = block_excl_scan(a + b, s_warp, tot);
  if (i0 < nb) out[i0] = ex;
  if (i0 + 1 < nb) out[i0 + 1] = ex + a;
  if (total && threadIdx.x == 0) *total = tot;
}

// The events of tile blockIdx.x: x, y, t from offset k0, m of them.
struct TileEvents {
  const int16_t *x, *y;
  const uint32_t *t;
  int64_t k0;
  int m;
  __device__ TileEvents(const Events &ev, int per_tile) {
    k0 = (int64_t)blockIdx.x * per_tile;
    m = (int)(k0 + per_tile < ev.n ? per_tile : ev.n - k0);
    x = ev.x + k0;
    y = ev.y + k0;
    t = ev.t + k0;
  }
};

// bhist is tile-major: bhist[tile * nb + bucket]
__global__ void __launch_bounds__(kSortThreads, 3) k_bucket_count(Events ev, Geometry g, int shift,
                                                                  int nb, int per_tile,
                                                                  int *__restrict__ bhist,
                                                                  int *__restrict__ err,
                                                                  float *__restrict__ zero_flow) {
  __shared__ int h[kMaxBuckets];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const TileEvents te(ev, per_tile);
  // kILP events per thread and round: every load first, then the atomics
  // (fewer than the other sort kernels take, so that three blocks fit an SM
  // without spills)
  constexpr int kILP = 6;
  for (int jb = threadIdx.x; jb < te.m; jb += kILP * blockDim.x) {
    int x[kILP], y[kILP];
    uint32_t t[kILP];
#pragma unroll
    for (int e = 0; e < kILP; ++e) {
      const int j = jb + e * blockDim.x;
      x[e] = j < te.m ? te.x[j] : -1;
      y[e] = j < te.m ? te.y[j] : 0;
      t[e] = j < te.m ? te.t[j] : 0u;
    }
#pragma unroll
    for (int e = 0; e < kILP; ++e) {
      const int j = jb + e * blockDim.x;
      if (j >= te.m) continue;
      uint32_t trel;
      if (event_ok(x[e], y[e], t[e], ev, g.W, g.H, trel)) {
        const int b = (y[e] * g.W + x[e]) >> shift;
        if (VK_CHECK(b < nb)) atomicAdd(&h[b], 1);
      } else {
        atomicOr(err, ERR_EVENT_RANGE);
        if (zero_flow)
          *reinterpret_cast<float2 *>(zero_flow + 2 * (te.k0 + j)) = make_float2(0.f, 0.f);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) bhist[(size_t)blockIdx.x * nb + i] = h[i];
}

// one block per bucket (4 tiles per thread): the exclusive prefixes of its
// column of tile counts go to bpre, the bucket's total to btot
__global__ void __launch_bounds__(1024) k_bucket_scan(const int *__restrict__ bhist, int nb,
                                                      int tiles, int *__restrict__ bpre,
                                                      int *__restrict__ btot) {
  __shared__ int s_warp[33];
  chain_wait();
  const int b = blockIdx.x;
  const int i0 = 4 * threadIdx.x;
  int c[4], v = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    c[q] = i0 + q < tiles ? bhist[(size_t)(i0 + q) * nb + b] : 0;
    v += c[q];
  }
  int tot;
  int run = block_excl_scan(v, s_warp, tot);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (i0 + q < tiles) bpre[(size_t)(i0 + q) * nb + b] = run;
    run += c[q];
  }
  if (threadIdx.x == 0) btot[b] = tot;
}

// dynamic shared memory: per_tile records as three int arrays (t - t_ref,
// index, pixel) in bucket order
__global__ void __launch_bounds__(kSortThreads, 3) k_bucket_scatter(Events ev, Geometry g, int shift,
                                                                    int nb, int per_tile,
                                                                    const int *__restrict__ bhist,
                                                                    const int *__restrict__ bpre,
                                                                    const int *__restrict__ btot,
                                                                    int4 *__restrict__ brec) {
  extern __shared__ int sst[];
  int *st_t = sst, *st_k = sst + per_tile, *st_p = sst + 2 * per_tile;
  __shared__ int cur[kMaxBuckets];  // global position of this tile's first record per bucket
  __shared__ int loc[kMaxBuckets];  // offset of each bucket's run within the tile
  __shared__ int fil[kMaxBuckets];  // fill cursor of each run
  __shared__ int s_warp[33];
  chain_wait();
  const int *cnt_tile = bhist + (size_t)blockIdx.x * nb;
  block_scan_small(btot, nb, cur, nullptr, s_warp);  // bucket bases
  int nvalid;
  block_scan_small(cnt_tile, nb, loc, &nvalid, s_warp);
  if (threadIdx.x == 0) s_warp[32] = nvalid;  // block_excl_scan's slot, free again here
  __syncthreads();
  nvalid = s_warp[32];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    cur[i] += bpre[(size_t)blockIdx.x * nb + i];
    fil[i] = loc[i];
  }
  __syncthreads();
  const TileEvents te(ev, per_tile);
  // each valid event straight to its slot in its bucket's run (shared atomics)
  constexpr int kILP = kSortILP / 2;
  for (int jb = threadIdx.x; jb < te.m; jb += kILP * blockDim.x) {
    int x[kILP], y[kILP];
    uint32_t t[kILP];
#pragma unroll
    for (int e = 0; e < kILP; ++e) {
      const int j = jb + e * blockDim.x;
      x[e] = j < te.m ? te.x[j] : -1;
      y[e] = j < te.m ? te.y[j] : 0;
      t[e] = j < te.m ? te.t[j] : 0u;
    }
#pragma unroll
    for (int e = 0; e < kILP; ++e) {
      const int j = jb + e * blockDim.x;
      uint32_t trel;
      if (j < te.m && event_ok(x[e], y[e], t[e], ev, g.W, g.H, trel)) {
        const int p = y[e] * g.W + x[e];
        if (!VK_CHECK((p >> shift) < nb)) continue;
        const int d = atomicAdd(&fil[p >> shift], 1);
        if (d < per_tile) {  // always, when the counts came from the same events
          st_t[d] = (int)trel;
          st_k[d] = (int)(te.k0 + j);
          st_p[d] = p;
        }
      }
    }
  }
  __syncthreads();
  // the tile's records in bucket order: each bucket's run lands contiguously
  nvalid = nvalid < te.m ? nvalid : te.m;
  for (int d = threadIdx.x; d < nvalid; d += blockDim.x) {
    const int p = st_p[d];
    const int b = p >> shift;
    if (p < 0 || b >= nb) continue;
    const int64_t q = (int64_t)cur[b] + (d - loc[b]);
    if (VK_CHECK(q >= 0 && q < ev.n)) brec[q] = make_int4(st_t[d], st_k[d], p, 0);
  }
}

// one block per bucket (dynamic shared memory: 2^shift ints for the pixel
// histogram, then four arrays of kSortStage ints)
__global__ void __launch_bounds__(kSortThreads, 3) k_bucket_sort(const int4 *__restrict__ brec,
                                                              int shift, int nb, int64_t P,
                                                              const int *__restrict__ btot,
                                                              int *__restrict__ cnt,
                                                              int *__restrict__ total_out,
                                                              int2 *__restrict__ rec,
                                                              int *__restrict__ rpix,
                                                              float4 *__restrict__ zgrid,
                                                              int zunits) {
  extern __shared__ int hs[];
  const int width = 1 << shift;
  // staged records as three int arrays (t - t_ref, index, pixel) and each
  // record's rank among its pixel's, then the source of each output slot
  int *st_t = hs + width, *st_k = st_t + kSortStage, *st_p = st_k + kSortStage;
  int *st_r = st_p + kSortStage, *src = st_r;  // ranks, then (reused) sources
  __shared__ int s_warp[33];
  __shared__ int s_base[2];
  chain_wait();
  const int b = blockIdx.x;
  const int64_t p0 = (int64_t)b << shift;
  // this bucket's first record: the sum of the earlier buckets' totals
  {
    int v = 0;
    for (int i = threadIdx.x; i < b; i += blockDim.x) v += btot[i];
    int tot;
    block_excl_scan(v, s_warp, tot);
    if (threadIdx.x == 0) {
      s_base[0] = tot;
      s_base[1] = btot[b];
    }
  }
  for (int i = threadIdx.x; i < width; i += blockDim.x) hs[i] = 0;
  __syncthreads();
  const int base = s_base[0], nrec = s_base[1];
  const bool staged = nrec <= kSortStage;
  // histogram (and, staged, each record with its rank among its pixel's)
  constexpr int kILP = kSortILP / 2;
  for (int rb = threadIdx.x; rb < nrec; rb += kILP * blockDim.x) {
    int4 q[kILP];
#pragma unroll
    for (int e = 0; e < kILP; ++e) {
      const int r = rb + e * blockDim.x;
      q[e] = r < nrec ? brec[base + r] : make_int4(0, 0, -1, 0);
    }
#pragma unroll
    for (int e = 0; e < kILP; ++e) {
      // a record outside the bucket cannot come from the scatter; skip it
      // rather than index outside the histogram
      if (q[e].z < p0 || q[e].z - p0 >= width) continue;
      const int rank = atomicAdd(&hs[q[e].z - p0], 1);
      if (staged) {
        const int r = rb + e * blockDim.x;
        st_t[r] = q[e].x;
        st_k[r] = q[e].y;
        st_p[r] = q[e].z;
        st_r[r] = rank;
      }
    }
  }
  __syncthreads();
  // counts out; hs becomes each pixel's first slot in the bucket (exclusive prefix)
  const int per = (width + blockDim.x - 1) / blockDim.x;
  const int i0 = threadIdx.x * per;
  int v = 0;
  for (int q = 0; q < per && i0 + q < width; ++q) {
    const int c = hs[i0 + q];
    if (p0 + i0 + q < P) cnt[p0 + i0 + q] = c;
    v += c;
  }
  int tot;
  int run = block_excl_scan(v, s_warp, tot);
  for (int q = 0; q < per && i0 + q < width; ++q) {
    const int c = hs[i0 + q];
    hs[i0 + q] = run;
    run += c;
  }
  __syncthreads();
  if (staged) {
    // slot of record r: its pixel's first slot plus its rank; the ranks are
    // read by all threads before any slot is written (src reuses st_r)
    constexpr int kPer = (kSortStage + kSortThreads - 1) / kSortThreads;
    int dst[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int r = threadIdx.x + q * kSortThreads;
      const int pz = r < nrec ? st_p[r] - (int)p0 : -1;
      dst[q] = pz >= 0 && pz < width ? hs[pz] + st_r[r] : -1;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int r = threadIdx.x + q * kSortThreads;
      if (r < nrec && dst[q] >= 0 && dst[q] < nrec) src[dst[q]] = r;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nrec; d += blockDim.x) {  // in order: coalesced
      const int r = src[d];
      if (r < 0 || r >= nrec) continue;
      rec[base + d] = make_int2(st_t[r], st_k[r]);
      rpix[base + d] = st_p[r];
    }
  } else {
    for (int rb = threadIdx.x; rb < nrec; rb += kILP * blockDim.x) {
      int4 q[kILP];
#pragma unroll
      for (int e = 0; e < kILP; ++e) {
        const int r = rb + e * blockDim.x;
        q[e] = r < nrec ? brec[base + r] : make_int4(0, 0, -1, 0);
      }
#pragma unroll
      for (int e = 0; e < kILP; ++e) {
        if (q[e].z < p0 || q[e].z - p0 >= width) continue;
        const int pos = base + atomicAdd(&hs[q[e].z - p0], 1);
        rec[pos] = make_int2(q[e].x, q[e].y);
        rpix[pos] = q[e].z;
      }
    }
  }
  if (b == nb - 1 && threadIdx.x == 0) *total_out = base + nrec;
  if (zgrid && nrec > 0) {
    // rows of the pixels at range edges inside [base, base + nrec): one warp
    // per range, lanes over the row's units.  Their pixels are read back from
    // the slots just written (shared memory when staged, else this block's
    // own global writes, visible after the barrier).  A range's last pixel
    // is skipped when the next range starts with it inside this bucket (it
    // is zeroed as that range's first pixel).
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t end = (int64_t)base + nrec;
    auto pixel_at = [&](int64_t pos) -> int {
      if (staged) {
        const int r = src[pos - base];
        return r >= 0 && r < nrec ? st_p[r] : -1;
      }
      return rpix[pos];
    };
    const int64_t c0 = base / kPixRecs, c1 = (end - 1) / kPixRecs;
    for (int64_t c = c0 + warp; c <= c1; c += blockDim.x >> 5) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t pos = c * kPixRecs + (e ? kPixRecs - 1 : 0);
        if (pos < base || pos >= end) continue;
        const int p = pixel_at(pos);
        if (p < p0 || p - p0 >= width || p >= P) continue;
        if (e && pos + 1 < end && pixel_at(pos + 1) == p) continue;
        for (int u = lane; u < zunits; u += 32) zgrid[(size_t)p * zunits + u] = f4zero();
      }
    }
  }
}

// 4. per-pixel phase sums PixelEmbed[p] = sum over the pixel's records of
// exp(i t T/dt).  Work is balanced by records: warp c takes records
// [c*recs, (c+1)*recs) in pixel-sorted order, streams them in groups of 32
// (t and pixel, the next group loading while one is summed), and writes each
// pixel's sum when the pixel changes -
// a plain store for pixels that lie wholly inside its range, a vector
// reduction for the first pixel and, unless the range is the last, the last
// pixel, which may continue in a neighbouring warp's range.  Only those
// pixels must be zero beforehand (the bucket sort can zero exactly them);
// pixels without records are not written at all.

__device__ __forceinline__ void red_add_v4(float4 *p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

template <int DV>
__global__ void __launch_bounds__(256) k_pixsum(Geometry g, Tables tb, const int *__restrict__ nsorted,
                                                const int2 *__restrict__ rec,
                                                const int *__restrict__ rpix,
                                                float4 *__restrict__ acc, int recs) {
  chain_wait();
  constexpr int U = 32 * DV;
  const int lane = threadIdx.x & 31;
  const int64_t ns = *nsorted;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  uint2 w[DV][2];
  load_freqs<DV>(tb.wt, lane, w);
  for (int64_t r0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * recs;
       r0 < ns; r0 += nw * recs) {
    const int64_t r1 = r0 + recs < ns ? r0 + recs : ns;
    int sp = -1;        // pixel of the running sum
    bool first = true;  // the running pixel is the first of this range
    float4 s[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) s[v] = f4zero();
    auto write = [&](bool shared) {
      if (!VK_CHECK(sp >= 0 && (int64_t)sp < (int64_t)g.W * g.H)) return;
      float4 *dst = acc + (size_t)sp * U + lane;
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        if (shared)
          red_add_v4(dst + 32 * v, s[v]);
        else
          dst[32 * v] = s[v];
      }
    };
    // records of the next group of 32 load while this group is summed
    uint32_t tn = lane < r1 - r0 ? (uint32_t)__ldg(&rec[r0 + lane].x) : 0u;
    int pn = lane < r1 - r0 ? __ldg(rpix + r0 + lane) : 0;
    for (int64_t c = r0; c < r1; c += 32) {
      const int m = (int)(r1 - c < 32 ? r1 - c : 32);
      const uint32_t tl = tn;
      const int pl = pn;
      if (c + 32 < r1) {
        tn = lane < r1 - c - 32 ? (uint32_t)__ldg(&rec[c + 32 + lane].x) : 0u;
        pn = lane < r1 - c - 32 ? __ldg(rpix + c + 32 + lane) : 0;
      }
      // bit j: record j starts a pixel (differs from record j - 1, or from
      // the running pixel for j = 0)
      int prev = __shfl_up_sync(kFull, pl, 1);
      if (lane == 0) prev = sp;
      const unsigned starts = __ballot_sync(kFull, lane < m && pl != prev);
      auto step = [&](int j) {
        const uint32_t tj = __shfl_sync(kFull, tl, j);
        if ((starts >> j) & 1u) {
          if (sp >= 0) {
            write(first);
            first = false;
          }
          sp = __shfl_sync(kFull, pl, j);
#pragma unroll
          for (int v = 0; v < DV; ++v) s[v] = f4zero();
        }
#pragma unroll
        for (int v = 0; v < DV; ++v) s[v] = add4x2(s[v], time_phase2_packed(tj, w[v][0], w[v][1]));
      };
      if (m == 32) {
        // a full group: the record positions are known at compile time
#pragma unroll
        for (int j = 0; j < 32; ++j) step(j);
      } else {
#pragma unroll 4
        for (int j = 0; j < m; ++j) step(j);
      }
    }
    // the last range's last pixel, when it started inside the range, has no
    // other contributor
    if (sp >= 0) write(first || r1 < ns);
  }
}

// ---------------------------------------------------------------------------
// 5. box-sum pass.  One warp walks one line segment (a row segment in the row
// pass, a column segment in the column pass), lanes over units.  Input blocks
// of L pixels stream into a 3-slot per-warp ring with cp.async (two blocks in
// flight while the third is consumed); slot contents become the block's
// suffix sums in place.  Each slot also receives one phase-anchor row.
//
// Row pass: input pixel (x, y) is modulated by exp(i (x X/dx + y Y/dy)) before
// the sum; the x phase advances by the step exp(i X/dx) from an anchor table
// row loaded once per block (at most L steps from the anchor).
// Column pass: output pixel (x, y) is demodulated by the conjugate of the
// same phase, advancing in y from an anchor per output block.
enum class Pass { Rows, Cols };

// EMIT (column pass only) picks the output form: kEmitF32, the window sums
// as they are; kEmitF16N, divided by the pixel's window count n (Eq. 17; 0
// where the window is empty) and stored as FP16, unit u of a pixel = 8 bytes
// (Re 2u, Re 2u+1, Im 2u, Im 2u+1); kEmitF32P, the window sums as FP32 in the
// order (Re 2u, Re 2u+1, Im 2u, Im 2u+1), so that the real and the imaginary
// parts of a unit are register pairs for packed FP32x2 arithmetic.
// occ (row pass, window length L <= 32): per-pixel event counts; pixels with
// none are taken as zero without reading src, whose rows there may hold
// anything.
enum : int { kEmitF32 = 0, kEmitF16N = 1, kEmitF32P = 2 };
// LC: the window length 2r + 1 fixed at compile time (the launcher picks the
// instantiation that matches), so that the per-block loops unroll and their
// shared-memory loads issue ahead of the dependent sums; 0: any length.  With
// the length fixed, the suffix sums of the block being emitted are held in
// registers, so a warp's ring needs two slots instead of three (more warps
// fit on an SM).
template <int DV, Pass P, int EMIT = kEmitF32, int LC = 0>
__global__ void __launch_bounds__(128) k_box_pass(const float4 *__restrict__ src,
                                                 float4 *__restrict__ dst, Geometry g, Tables tb,
                                                 int seg, int nseg, int up,
                                                 const int *__restrict__ ncnt = nullptr,
                                                 const int *__restrict__ occ = nullptr) {
  static_assert(EMIT == kEmitF32 || P == Pass::Cols, "normalised output: column pass only");
  chain_wait();
  constexpr bool HALF = EMIT == kEmitF16N;
  constexpr bool NORM = HALF;  // divided by the window counts
  constexpr int U = 32 * DV;
  extern __shared__ float4 smem[];
  const int r = (P == Pass::Rows) ? g.dx : g.dy;
  const int L = LC > 0 ? LC : 2 * r + 1;
  constexpr int kUnroll = LC > 0 ? LC : 1;
  const int SL = (L + 1) * U;  // slot: L data rows + 1 anchor row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const int nlines = (P == Pass::Rows) ? g.H : g.W;
  const int len = (P == Pass::Rows) ? g.W : g.H;
  if (wid >= (int64_t)nlines * nseg) return;
  constexpr bool kRegS = LC > 0;         // suffix sums in registers
  constexpr int kSlots = kRegS ? 2 : 3;  // ring slots per warp
  float4 *ring = smem + (size_t)warp * kSlots * SL;
  // neighbouring warps take neighbouring lines of the same segment, so the
  // blocks in flight at one time sit side by side in memory
  const int line = (int)(wid % nlines), s = (int)(wid / nlines);
  const int o0 = s * seg;
  const int nout = min(len, o0 + seg) - o0;
  const int in0 = o0 - r;
  if (g.ncanvas > 0) {
    // a batch's canvas: only outputs some slice depends on are computed.  The
    // column pass's outputs inside a slice; the row pass's outputs in a
    // slice's columns within dy rows of it (what those column windows read).
    // Every window of a needed output reads needed values only, and van Herk
    // sums never mix in values from outside a window.
    bool need = false;
    for (int i = lane; i < g.ncanvas; i += 32) {
      const CanvasSlice &cs = g.canvas[i];
      if (P == Pass::Rows)
        need |= line >= cs.oy - g.dy && line < cs.oy + cs.H + g.dy && o0 < cs.ox + cs.W &&
                o0 + nout > cs.ox;
      else
        need |= line >= cs.ox && line < cs.ox + cs.W && o0 < cs.oy + cs.H && o0 + nout > cs.oy;
    }
    if (!__any_sync(kFull, need)) return;
  }
  // this warp's slice of each pixel: units u0 .. u0 + U - 1 of up (grids and
  // tables are [pixel][up] units; the ring holds one slice)
  const int u0 = blockIdx.y * U;
  const size_t base = ((P == Pass::Rows) ? (size_t)line * g.W * up : (size_t)line * up) + u0;
  const size_t stride = (P == Pass::Rows) ? (size_t)up : (size_t)g.W * up;
  const int nb = (nout + L - 1) / L;  // output blocks; input blocks 0..nb

  auto slot = [&](int b) { return ring + (size_t)(b % kSlots) * SL; };
  // row pass with occ: lane q holds the count of pixel q of the next block to
  // issue, loaded one block ahead of its use
  const bool use_occ = P == Pass::Rows && occ != nullptr && L <= 32;
  int occ_v = 0;
  auto load_occ = [&](int b) {
    const int pos = in0 + b * L + lane;
    occ_v = (b <= nb && lane < L && pos >= 0 && pos < len)
                ? __ldg(occ + (size_t)line * g.W + pos) : 0;
  };
  if (use_occ) load_occ(0);
  auto issue = [&](int b) {  // input block b and its anchor row -> its slot (one group)
    if (b <= nb) {
      float4 *sl = slot(b);
      unsigned on = ~0u;  // bit q: pixel q of the block is read
      if (use_occ) {
        on = __ballot_sync(kFull, occ_v != 0);
        load_occ(b + 1);
      }
#pragma unroll kUnroll
      for (int q = 0; q < L; ++q) {
        const int pos = in0 + b * L + q;
        const bool rd = pos >= 0 && pos < len && ((on >> (q & 31)) & 1u);
#pragma unroll
        for (int v = 0; v < DV; ++v) {
          const int u = lane + 32 * v;
          if (rd)
            cp_async16(sl + q * U + u, src + base + (size_t)pos * stride + u);
          else
            sl[q * U + u] = f4zero();
        }
      }
      const float4 *arow;
      if (P == Pass::Rows) {  // tx row of the block's first input column (halo rows from -dx)
        const int a = min(max(in0 + b * L, -g.dx), g.W - 1);
        arow = tb.tx + (size_t)(a + g.dx) * up + u0;
      } else {  // ty row of the output block's first row
        const int a = min(o0 + b * L, g.H - 1);
        arow = tb.ty + (size_t)a * up + u0;
      }
#pragma unroll
      for (int v = 0; v < DV; ++v) cp_async16(sl + L * U + lane + 32 * v, arow + lane + 32 * v);
    }
    cp_async_commit();
  };
  // kRegS: suffix sums of the block being emitted, and its anchor row
  float4 Sreg[kRegS ? LC : 1][DV], Areg[DV];
  auto suffix_regs = [&](const float4 *sl) {
#pragma unroll
    for (int v = 0; v < DV; ++v) {
      float4 run = f4zero();
#pragma unroll
      for (int q = (kRegS ? LC : 1) - 1; q >= 0; --q) {
        run = add4(run, sl[q * U + lane + 32 * v]);
        Sreg[q][v] = run;
      }
      Areg[v] = sl[L * U + lane + 32 * v];
    }
  };
  auto suffix = [&](float4 *sl) {
    float4 run[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) run[v] = f4zero();
#pragma unroll kUnroll
    for (int q = L - 1; q >= 0; --q) {
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        run[v] = add4(run[v], sl[q * U + lane + 32 * v]);
        sl[q * U + lane + 32 * v] = run[v];
      }
    }
  };
  // fixed factor of this line, the per-step rotation and its square (row pass)
  float4 fl[DV], st[DV], st2[DV];
#pragma unroll
  for (int v = 0; v < DV; ++v) {
    const int u = lane + 32 * v;
    if (P == Pass::Rows) {
      fl[v] = __ldg(tb.ty + (size_t)line * up + u0 + u);
      st[v] = __ldg(tb.sx + u0 + u);
    } else {
      fl[v] = __ldg(tb.tx + (size_t)(line + g.dx) * up + u0 + u);
      st[v] = __ldg(tb.sy + u0 + u);
    }
    st2[v] = cmul2(st[v], st[v]);
  }
  auto modulate = [&](float4 *sl) {  // row pass: sl[q] *= tx[x0 + q] ty[y]
    // the even and odd inputs' phases as two rotations by the squared step:
    // half as many dependent steps in each
    float4 pe[DV], po[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) {
      pe[v] = cmul2(sl[L * U + lane + 32 * v], fl[v]);
      po[v] = cmul2(pe[v], st[v]);
    }
#pragma unroll kUnroll
    for (int q = 0; q < L; q += 2) {
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        float4 *e = sl + q * U + lane + 32 * v;
        *e = cmul2(*e, pe[v]);
        pe[v] = cmul2(pe[v], st2[v]);
        if (q + 1 < L) {
          e[U] = cmul2(e[U], po[v]);
          po[v] = cmul2(po[v], st2[v]);
        }
      }
    }
  };

  // NORM: window counts of output block bb, one per lane (the reciprocal is
  // taken where they are used, a block later, so the load is not waited on)
  auto load_cnt = [&](int bb) {
    const int q = lane < L ? lane : 0;
    const int j = bb * L + q;
    return j < nout ? __ldg(ncnt + (size_t)(o0 + j) * g.W + line) : 0;
  };
  int cnt_next = NORM ? load_cnt(0) : 0;

  // Blocks stream through the ring one group ahead: with the suffix sums in
  // registers, block b + 3 goes into the slot of block b + 1 once that
  // block's suffix sums are taken; otherwise block b + 2 goes into the slot
  // block b - 1 used, at the start of iteration b.
  issue(0);
  issue(1);
  cp_async_wait1();
  if (P == Pass::Rows) modulate(slot(0));
  if constexpr (kRegS) {
    suffix_regs(slot(0));
    issue(2);
  } else {
    suffix(slot(0));
  }
  for (int b = 0; b < nb; ++b) {
    if constexpr (!kRegS) issue(b + 2);
    cp_async_wait1();  // block b+1 has landed
    const float4 *S = slot(b);  // (without kRegS) block b's suffix sums
    float4 *V = slot(b + 1);
    if (P == Pass::Rows && b + 1 <= nb) modulate(V);
    const int j0 = b * L;
    float4 dph[DV];  // column pass: phase of the next output, conj applied at emit
    if (P == Pass::Cols) {
#pragma unroll
      for (int v = 0; v < DV; ++v)
        dph[v] = cmul2(fl[v], kRegS ? Areg[v] : S[L * U + lane + 32 * v]);
    }
    float inv_lane = 0.f;  // NORM: 1/n of output j0 + lane (lanes < L), loaded a block ahead
    if (NORM) {
      inv_lane = cnt_next > 0 ? 1.0f / (float)cnt_next : 0.f;
      if (b + 1 < nb) cnt_next = load_cnt(b + 1);
    }
    auto emit = [&](int j, int qs, const float4 *G) {
      const int pos = o0 + j;
      float inv = 0.f;
      if (NORM) {
        if (L <= 32) {
          inv = __shfl_sync(kFull, inv_lane, j - j0);
        } else {  // a block longer than the warp: the count of this output itself
          const int c = __ldg(ncnt + (size_t)pos * g.W + line);
          inv = c > 0 ? 1.0f / (float)c : 0.f;
        }
      }
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        const int u = lane + 32 * v;
        float4 o;
        if constexpr (kRegS)
          o = Sreg[qs][v];
        else
          o = S[qs * U + u];
        if (G) o = add4(o, G[v]);
        if (P == Pass::Cols) {
          o = cmul2c(o, dph[v]);
          dph[v] = cmul2(dph[v], st[v]);
        }
        if (HALF) {
          const __half2 re = __floats2half2_rn(o.x * inv, o.z * inv);
          const __half2 im = __floats2half2_rn(o.y * inv, o.w * inv);
          reinterpret_cast<uint2 *>(dst)[base + (size_t)pos * stride + u] =
              make_uint2(*reinterpret_cast<const uint32_t *>(&re),
                         *reinterpret_cast<const uint32_t *>(&im));
        } else if (EMIT == kEmitF32P) {
          dst[base + (size_t)pos * stride + u] = make_float4(o.x, o.z, o.y, o.w);
        } else {
          dst[base + (size_t)pos * stride + u] = o;
        }
      }
    };
    emit(j0, 0, nullptr);  // window == block b
    float4 G[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) G[v] = f4zero();
    const int qmax = min(L - 1, nout - 1 - j0);
#pragma unroll kUnroll
    for (int q = 0; q < L - 1; ++q) {
      if (q < qmax) {
#pragma unroll
        for (int v = 0; v < DV; ++v) G[v] = add4(G[v], V[q * U + lane + 32 * v]);
        emit(j0 + q + 1, q + 1, G);  // suffix of block b from q+1, prefix of block b+1 to q
      }
    }
    if constexpr (kRegS) {
      if (b + 1 < nb) suffix_regs(V);
      issue(b + 3);  // into block b+1's slot, now read
    } else {
      if (b + 1 < nb) suffix(V);
    }
  }
  cp_async_wait0();
}

// 6. window counts (Eq. 17): exact integer box sums, rows then columns.
// Window counts in one pass: a block stages a kCountTile x kCountTile output
// tile and its halo (zeros outside the sensor, which equals clipping the
// window there) in shared memory, sums rows of 2dx+1, then columns of 2dy+1.
constexpr int kCountTile = 32;

__global__ void __launch_bounds__(256) k_count_box(const int *__restrict__ cnt,
                                                   int *__restrict__ out, int W, int H, int dx,
                                                   int dy) {
  extern __shared__ int csm[];
  const int iw = kCountTile + 2 * dx, ih = kCountTile + 2 * dy;
  int *in = csm;             // [ih][iw] counts
  int *rs = csm + iw * ih;   // [ih][kCountTile] row sums
  const int x0 = blockIdx.x * kCountTile, y0 = blockIdx.y * kCountTile;
  for (int i = threadIdx.x; i < iw * ih; i += blockDim.x) {
    const int gy = y0 - dy + i / iw, gx = x0 - dx + i % iw;
    in[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? __ldg(cnt + (size_t)gy * W + gx) : 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ih * kCountTile; i += blockDim.x) {
    const int r = i / kCountTile, c = i % kCountTile;
    const int *p = in + r * iw + c;
    int sum = 0;
    for (int a = 0; a <= 2 * dx; ++a) sum += p[a];
    rs[i] = sum;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kCountTile * kCountTile; i += blockDim.x) {
    const int r = i / kCountTile, c = i % kCountTile;
    const int gy = y0 + r, gx = x0 + c;
    if (gy >= H || gx >= W) continue;
    const int *p = rs + r * kCountTile + c;
    int sum = 0;
    for (int b = 0; b <= 2 * dy; ++b) sum += p[b * kCountTile];
    out[(size_t)gy * W + gx] = sum;
  }
}

// ---------------------------------------------------------------------------
// 7a. gather for requested events given by index (K, or all in input order):
// pooled[p] * conj(exp(i t T/dt)) / n_p.  Zeros for an invalid index or event.
template <int DV>
__device__ __forceinline__ bool gather_event(const Events &ev, const int64_t *__restrict__ K,
                                             int64_t i, const Geometry &g, const uint2 (&w)[DV][2],
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
  if (!event_ok(x, y, ev.t[k], ev, g.W, g.H, trel)) return false;  // flagged by k_hist
  const int pix = y * g.W + x;
  const float inv = 1.0f / (float)__ldg(ncnt + pix);
#pragma unroll
  for (int v = 0; v < DV; ++v) {
    const int u = lane + 32 * v;
    float4 o = cmul2c(__ldg(pooled + (size_t)pix * U + u), time_phase2(trel, w[v][0], w[v][1]));
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
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const int D = g.D;
  uint2 w[DV][2];
  load_freqs<DV>(tb.wt, lane, w);
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < nK;
       i += (int64_t)gridDim.x * wpb) {
    float4 e[DV];
    gather_event<DV>(ev, K, i, g, w, pooled, ncnt, lane, e, err);
    float *row = emb + (size_t)i * 2 * D;
#pragma unroll
    for (int v = 0; v < DV; ++v) {
      const int u = lane + 32 * v;
      *reinterpret_cast<float2 *>(row + 2 * u) = make_float2(e[v].x, e[v].z);
      *reinterpret_cast<float2 *>(row + D + 2 * u) = make_float2(e[v].y, e[v].w);
    }
  }
}

// 7b. plain FP32 perceptron fused with the gather.  A CTA takes 64 requested
// events: its 8 warps gather rows into shared memory, then thread (eg, hg)
// computes a 4-event x 8-hidden block of the first layer from W1^T in shared
// memory, applies bias and ReLU, reduces its share of the second layer, and
// the 16 threads of an event group combine partial outputs with shuffles.
// Sorted mode (rec != nullptr) walks the pixel-sorted records, so
// consecutive rows mostly share a pooled row (L1 hits).
constexpr int kHid = 128;
constexpr int kTM = 64;
constexpr int64_t kInvalidRow = (int64_t)1 << 62;  // output row whose event was invalid

template <int DV>
__global__ void __launch_bounds__(256) k_predict_fp32(Events ev, const int64_t *__restrict__ K,
                                                      int64_t nK, const int2 *__restrict__ rec,
                                                      const int *__restrict__ rpix,
                                                      const int *__restrict__ nsorted, Geometry g,
                                                      Tables tb, const float4 *__restrict__ pooled,
                                                      const int *__restrict__ ncnt, MLP mlp,
                                                      float *__restrict__ flow, int *err) {
  constexpr int U = 32 * DV, IN = 4 * U, LDE = IN + 4;
  extern __shared__ float4 smem4[];
  float *sW = reinterpret_cast<float *>(smem4);  // [IN][kHid]
  float *sE = sW + IN * kHid;                     // [kTM][LDE]
  float *sB1 = sE + kTM * LDE;                    // [kHid]
  float *sW2 = sB1 + kHid;                        // [2][kHid]
  int64_t *sK = reinterpret_cast<int64_t *>(sW2 + 2 * kHid);  // [kTM] output rows
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
  const int64_t ns = rec ? (int64_t)*nsorted : nK;
  uint2 w[DV][2];
  load_freqs<DV>(tb.wt, lane, w);
  for (int64_t tile = blockIdx.x; tile * kTM < nK; tile += gridDim.x) {
    for (int rr = 0; rr < kTM / 8; ++rr) {
      const int row = warp * (kTM / 8) + rr;
      const int64_t i = tile * kTM + row;
      float4 e[DV];
#pragma unroll
      for (int v = 0; v < DV; ++v) e[v] = f4zero();
      int64_t outk = -1;
      if (i < ns) {
        if (rec) {
          const int2 r = __ldg(rec + i);
          int p = __ldg(rpix + i);
          if (!VK_CHECK(p >= 0 && (int64_t)p < (int64_t)g.W * g.H)) p = 0;
          const float inv = 1.0f / (float)__ldg(ncnt + p);
#pragma unroll
          for (int v = 0; v < DV; ++v) {
            const int u = lane + 32 * v;
            float4 o = cmul2c(__ldg(pooled + (size_t)p * U + u),
                              time_phase2((uint32_t)r.x, w[v][0], w[v][1]));
            o.x *= inv; o.y *= inv; o.z *= inv; o.w *= inv;
            e[v] = o;
          }
          outk = r.y;
        } else {
          const bool ok = gather_event<DV>(ev, K, i, g, w, pooled, ncnt, lane, e, err);
          outk = ok ? i : (i | kInvalidRow);
        }
      }
      if (lane == 0) sK[row] = outk;
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
        const int64_t k = sK[4 * eg + i];
        if (k >= 0) {
          const bool ok = !(k & kInvalidRow);
          *reinterpret_cast<float2 *>(flow + 2 * (k & ~kInvalidRow)) =
              ok ? make_float2(o[i][0] + b20, o[i][1] + b21) : make_float2(0.f, 0.f);
        }
      }
    }
    __syncthreads();
  }
}

// Large dynamic shared memory, and a carveout that lets several CTAs share an SM.
// ---------------------------------------------------------------------------
// 8. the direct window form (the per-event window loop of Algorithm 1), for
// requests that are few next to the sensor's pixels.
//
// 8a. per-pixel phase sums written once per occupied pixel: warp c owns the
// pixels whose first record lies in [c*kPixRecs, (c+1)*kPixRecs) of the
// pixel-sorted records and sums each to its last record, past the range if
// need be.  Plain stores only, no clear: pixels without events keep whatever
// they held, and the direct form never reads them.
template <int DV>
__global__ void __launch_bounds__(256) k_pixsum_owned(Tables tb, const int *__restrict__ nsorted,
                                                      const int2 *__restrict__ rec,
                                                      const int *__restrict__ rpix,
                                                      float4 *__restrict__ acc) {
  chain_wait();
  constexpr int U = 32 * DV;
  const int lane = threadIdx.x & 31;
  const int64_t ns = *nsorted;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  uint2 w[DV][2];
  load_freqs<DV>(tb.wt, lane, w);
  for (int64_t r0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kPixRecs;
       r0 < ns; r0 += nw * kPixRecs) {
    const int64_t r1 = r0 + kPixRecs < ns ? r0 + kPixRecs : ns;
    // the first record of the range that starts a pixel (pixels ascend)
    int64_t c = r0;
    if (r0 > 0) {
      const int prev = __ldg(rpix + r0 - 1);
      for (;;) {
        const int64_t i = c + lane;
        const int pl = i < ns ? __ldg(rpix + i) : -2;
        const unsigned m = __ballot_sync(kFull, pl != prev);
        if (m) {
          c += __ffs(m) - 1;
          break;
        }
        c += 32;
      }
      if (c >= r1) continue;  // every record of the range continues an earlier pixel
    }
    int sp = -1;
    float4 s[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) s[v] = f4zero();
    auto store = [&]() {
      float4 *dst = acc + (size_t)sp * U + lane;
#pragma unroll
      for (int v = 0; v < DV; ++v) dst[32 * v] = s[v];
    };
    bool done = false;
    for (int64_t b = c; !done && b < ns; b += 32) {
      const int m = (int)(ns - b < 32 ? ns - b : 32);
      const uint32_t tl = lane < m ? (uint32_t)__ldg(&rec[b + lane].x) : 0u;
      const int pl = lane < m ? __ldg(rpix + b + lane) : 0;
      for (int j = 0; j < m; ++j) {
        const int pj = __shfl_sync(kFull, pl, j);
        const uint32_t tj = __shfl_sync(kFull, tl, j);
        if (pj != sp) {
          if (sp >= 0) store();
          if (b + j >= r1) {  // this pixel starts past the range: another warp's
            done = true;
            sp = -1;
            break;
          }
          sp = pj;
#pragma unroll
          for (int v = 0; v < DV; ++v) s[v] = f4zero();
        }
#pragma unroll
        for (int v = 0; v < DV; ++v) s[v] = add4(s[v], time_phase2(tj, w[v][0], w[v][1]));
      }
    }
    if (sp >= 0) store();  // the records ended inside this warp's last pixel
  }
}

// 8b. one warp per requested event: emb = conj(phase_t) / n * sum over the
// window of PixelEmbed[p] exp(i ((x_p - x) X/dx + (y_p - y) Y/dy)), the sum
// visiting only occupied pixels (a ballot over the counts of each window
// row), n = the window count.  FLOW: the perceptron follows in the same warp
// (W1 transposed, b1, W2 in shared memory; lane j computes hidden units
// j, j+32, j+64, j+96 from the encoding staged in shared memory).
constexpr int kDirWarps = 8;
constexpr int kDirBatch = 4;  // occupied window pixels whose loads are in flight together

template <int DV, bool FLOW>
__global__ void __launch_bounds__(32 * kDirWarps) k_direct(Events ev, const int64_t *__restrict__ K,
                                                         int64_t nK, Geometry g, Tables tb,
                                                         const float4 *__restrict__ acc,
                                                         const int *__restrict__ cnt, MLP mlp,
                                                         float *__restrict__ out, int *err) {
  constexpr int U = 32 * DV, IN = 4 * U;
  extern __shared__ float4 smem4[];
  float *sW = reinterpret_cast<float *>(smem4);   // FLOW: [IN][128] W1 transposed
  float *sE = sW + (FLOW ? IN * kHid : 0);        // [warps][IN] encoding rows
  float *sB1 = sE + kDirWarps * IN;               // [128]
  float *sW2 = sB1 + kHid;                        // [2][128]
  if (FLOW) {
    for (int i = threadIdx.x; i < IN * kHid / 4; i += blockDim.x)
      reinterpret_cast<float4 *>(sW)[i] = __ldg(reinterpret_cast<const float4 *>(mlp.W1t) + i);
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
      sB1[i] = mlp.b1[i];
      sW2[i] = mlp.W2[i];
      sW2[kHid + i] = mlp.W2[kHid + i];
    }
    __syncthreads();
  }
  chain_wait();  // the prologue above reads only the weights
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int D = 2 * U;
  uint2 w[DV][2];
  load_freqs<DV>(tb.wt, lane, w);
  const int64_t nwarps = (int64_t)gridDim.x * kDirWarps;
  for (int64_t i = (int64_t)blockIdx.x * kDirWarps + warp; i < nK; i += nwarps) {
    int64_t k = i;
    bool valid = true;
    if (K) {
      k = K[i];
      if (k < 0 || k >= ev.n) {
        valid = false;
        if (lane == 0) atomicOr(err, ERR_INDEX_RANGE);
      }
    }
    int x = 0, y = 0;
    uint32_t trel = 0;
    if (valid) {
      x = ev.x[k];
      y = ev.y[k];
      valid = event_ok(x, y, ev.t[k], ev, g.W, g.H, trel);
      if (!valid && lane == 0) atomicOr(err, ERR_EVENT_RANGE);
    }
    float4 e[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) e[v] = f4zero();
    if (valid) {
      int n = 0;
      for (int yy = max(0, y - g.dy); yy <= min(g.H - 1, y + g.dy); ++yy) {
        float4 rp[DV];  // exp(i (yy - y) Y/dy)
#pragma unroll
        for (int v = 0; v < DV; ++v) rp[v] = __ldg(tb.ry + (size_t)(yy - y + g.dy) * U + lane + 32 * v);
        for (int x0 = x - g.dx; x0 <= x + g.dx; x0 += 32) {
          const int xl = x0 + lane;
          const int c = (xl <= x + g.dx && xl >= 0 && xl < g.W) ? __ldg(cnt + (size_t)yy * g.W + xl) : 0;
          n += c;
          unsigned m = __ballot_sync(kFull, c > 0);
          // occupied pixels four at a time: every load issued before any use
          while (m) {
            int xs[kDirBatch];
#pragma unroll
            for (int q = 0; q < kDirBatch; ++q) {
              xs[q] = m ? x0 + __ffs(m) - 1 : -1;
              m &= m - 1;
            }
            float4 av[kDirBatch][DV], tv[kDirBatch][DV];
#pragma unroll
            for (int q = 0; q < kDirBatch; ++q) {
              const int xj = xs[q] >= 0 ? xs[q] : xs[0];
              const float4 *a = acc + ((size_t)yy * g.W + xj) * U + lane;
              const float4 *tr = tb.rx + (size_t)(xj - x + g.dx) * U + lane;  // exp(i (xj - x) X/dx)
#pragma unroll
              for (int v = 0; v < DV; ++v) {
                av[q][v] = __ldg(a + 32 * v);
                tv[q][v] = __ldg(tr + 32 * v);
              }
            }
#pragma unroll
            for (int q = 0; q < kDirBatch; ++q) {
              if (xs[q] < 0) break;
#pragma unroll
              for (int v = 0; v < DV; ++v) e[v] = add4(e[v], cmul2(av[q][v], cmul2(tv[q][v], rp[v])));
            }
          }
        }
      }
      n = __reduce_add_sync(kFull, n);  // >= 1: the event's own pixel
      const float inv = 1.0f / (float)n;
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        const float4 o = cmul2c(e[v], time_phase2(trel, w[v][0], w[v][1]));
        e[v] = make_float4(o.x * inv, o.y * inv, o.z * inv, o.w * inv);
      }
    }
    if (!FLOW) {
      float *row = out + (size_t)i * 2 * D;
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        const int u = lane + 32 * v;
        *reinterpret_cast<float2 *>(row + 2 * u) = make_float2(e[v].x, e[v].z);
        *reinterpret_cast<float2 *>(row + D + 2 * u) = make_float2(e[v].y, e[v].w);
      }
    } else {
      float *se = sE + warp * IN;  // [Re | Im], the perceptron's input order
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        const int u = lane + 32 * v;
        *reinterpret_cast<float2 *>(se + 2 * u) = make_float2(e[v].x, e[v].z);
        *reinterpret_cast<float2 *>(se + D + 2 * u) = make_float2(e[v].y, e[v].w);
      }
      __syncwarp();
      float h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) h[q] = sB1[lane + 32 * q];
      for (int cI = 0; cI < IN; ++cI) {
        const float ec = se[cI];
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = fmaf(sW[cI * kHid + lane + 32 * q], ec, h[q]);
      }
      float f0 = 0.f, f1 = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float a = fmaxf(h[q], 0.f);
        f0 = fmaf(sW2[lane + 32 * q], a, f0);
        f1 = fmaf(sW2[kHid + lane + 32 * q], a, f1);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        f0 += __shfl_xor_sync(kFull, f0, o);
        f1 += __shfl_xor_sync(kFull, f1, o);
      }
      if (lane == 0)
        *reinterpret_cast<float2 *>(out + 2 * i) =
            valid ? make_float2(f0 + mlp.b2[0], f1 + mlp.b2[1]) : make_float2(0.f, 0.f);
      __syncwarp();
    }
  }
}

template <typename KernelT>
cudaError_t set_smem(KernelT k, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  // without the opt-in a block may use 48 KB of static and dynamic memory together
  cudaFuncAttributes a{};
  e = cudaFuncGetAttributes(&a, reinterpret_cast<const void *>(k));
  if (e != cudaSuccess || a.sharedSizeBytes + bytes <= 48 * 1024) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int DV>
int pixsum_impl(const Geometry &g, const Tables &tb, const int *nsorted, const int2 *rec,
                const int *rpix, int64_t n, float4 *acc, cudaStream_t s, bool clear,
                bool chain) {
  const int64_t P = (int64_t)g.W * g.H;
  if (clear && cudaMemsetAsync(acc, 0, (size_t)P * g.U * sizeof(float4), s) != cudaSuccess)
    return -1;
  if (n == 0) return 0;
  const int64_t recs = kPixRecs;
  const int64_t warps = (n + recs - 1) / recs;
  const int grid = (int)std::min<int64_t>((warps + 7) / 8, (int64_t)num_sms() * 64);
  // after a clear the memset, not a kernel, comes before the launch
  return launch_kernel(k_pixsum<DV>, dim3(grid), dim3(256), 0, s, chain && !clear, g, tb, nsorted,
                       rec, rpix, acc, (int)recs) == cudaSuccess
             ? 1
             : -1;
}

// Largest dynamic shared memory a box-pass block may ask for.
constexpr size_t kBoxSmemMax = 200 * 1024;

template <int DV, Pass P, int EMIT = kEmitF32>
int box_pass(const Geometry &g, const Tables &tb, const float4 *src, float4 *dst, cudaStream_t s,
             const int *ncnt, int seg_windows, int wpb_req, const int *occ = nullptr,
             bool chain = false) {
  const int r = (P == Pass::Rows) ? g.dx : g.dy;
  const int L = 2 * r + 1;
  const int len = (P == Pass::Rows) ? g.W : g.H;
  const int nlines = (P == Pass::Rows) ? g.H : g.W;
  // a warp walks `seg` outputs of one line (a whole number of windows)
  const int seg = L * (seg_windows > 0 ? seg_windows : std::max(1, (128 + L / 2) / L));
  const int nseg = (len + seg - 1) / seg;
  // one warp per (line segment, 32-unit slice of the pixels): DV slices, so
  // the ring of a warp holds 32 units per row whatever D is
  // ring slots per warp: two where the window length has its own
  // instantiation (suffix sums in registers), else three
  const bool fixed_len = L == 21 || L == 17;
  const size_t per_warp = (size_t)(fixed_len ? 2 : 3) * (L + 1) * 32 * sizeof(float4);
  int wpb = per_warp * 2 <= 100 * 1024 ? 2 : 1;
  if (wpb_req > 0 && wpb_req <= 4 && per_warp * wpb_req <= kBoxSmemMax) wpb = wpb_req;
  const size_t sm = per_warp * wpb;
  // the windows of radius 10 and 8 have instantiations with their length fixed
  auto kern = L == 21   ? k_box_pass<1, P, EMIT, 21>
              : L == 17 ? k_box_pass<1, P, EMIT, 17>
                        : k_box_pass<1, P, EMIT, 0>;
  if (set_smem(kern, sm) != cudaSuccess) return -1;
  const int64_t warps = (int64_t)nlines * nseg;
  const dim3 grid((unsigned)((warps + wpb - 1) / wpb), DV);
  return launch_kernel(kern, grid, dim3(32 * wpb), sm, s, chain, src, dst, g, tb,
                       seg, nseg, 32 * DV, ncnt, occ) == cudaSuccess
             ? 1
             : -1;
}

template <int DV>
int pixsum_owned_impl(const Tables &tb, const int *nsorted, const int2 *rec, const int *rpix,
                      int64_t n, float4 *acc, cudaStream_t s, bool chain) {
  if (n == 0) return 0;
  const int64_t warps = (n + kPixRecs - 1) / kPixRecs;
  const int grid = (int)std::min<int64_t>((warps + 7) / 8, (int64_t)num_sms() * 64);
  return launch_kernel(k_pixsum_owned<DV>, dim3(grid), dim3(256), 0, s, chain, tb, nsorted, rec,
                       rpix, acc) == cudaSuccess
             ? 1
             : -1;
}

template <int DV, bool FLOW>
int direct_impl(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                const Tables &tb, const float4 *acc, const int *cnt, const MLP &mlp, float *out,
                int *err, cudaStream_t s, bool chain) {
  if (nK == 0) return 0;
  constexpr int IN = 128 * DV;
  const size_t sm = sizeof(float) * ((FLOW ? (size_t)IN * kHid : 0) + (size_t)kDirWarps * IN + 3 * kHid);
  auto kern = k_direct<DV, FLOW>;
  if (set_smem(kern, sm) != cudaSuccess) return -1;
  const int per_sm = std::max(1, blocks_per_sm((const void *)kern, 32 * kDirWarps, sm));
  const int64_t blocks = (nK + kDirWarps - 1) / kDirWarps;
  const int grid = (int)std::min<int64_t>(blocks, (int64_t)num_sms() * per_sm);
  return launch_kernel(kern, dim3(grid), dim3(32 * kDirWarps), sm, s, chain, ev, K, nK, g, tb, acc,
                       cnt, mlp, out, err) == cudaSuccess
             ? 1
             : -1;
}

template <int DV>
int gather_impl(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                const Tables &tb, const float4 *pooled, const int *ncnt, float *emb, int *err,
                cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((nK + 7) / 8, (int64_t)num_sms() * 8);
  k_gather_emb<DV><<<grid, 256, 0, s>>>(ev, K, nK, g, tb, pooled, ncnt, emb, err);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <int DV>
int predict_fp32_impl(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                      const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb, const float4 *pooled,
                      const int *ncnt, const MLP &mlp, float *flow, int *err, cudaStream_t s) {
  constexpr int U = 32 * DV, IN = 4 * U;
  const size_t sm = sizeof(float) * ((size_t)IN * kHid + (size_t)kTM * (IN + 4) + 3 * kHid) +
                    sizeof(int64_t) * kTM;
  if (sm > 227 * 1024) return -2;  // W1^T does not fit in shared memory
  if (set_smem(k_predict_fp32<DV>, sm) != cudaSuccess) return -1;
  const int per_sm = blocks_per_sm((const void *)k_predict_fp32<DV>, 256, sm);
  const int64_t tiles = (nK + kTM - 1) / kTM;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * std::max(1, per_sm));
  k_predict_fp32<DV><<<grid, 256, sm, s>>>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt,
                                           mlp, flow, err);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

int blocks_per_sm(const void *func, int threads, size_t smem) {
  cudaFuncAttributes a{};
  if (cudaFuncGetAttributes(&a, func) != cudaSuccess) return 1;
  int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  const size_t per_block_smem = smem + a.sharedSizeBytes + 1024;  // 1 KB reserved per CTA
  const int by_smem = (int)(smem_sm / per_block_smem);
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((a.numRegs * 32 + 255) / 256) * 256;
  const int by_regs = regs_warp > 0 ? regs_sm / (regs_warp * warps) : 32;
  const int by_thr = thr_sm / threads;
  return std::max(1, std::min(std::min(by_smem, by_regs), std::min(by_thr, 32)));
}

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

#define VECKM_DISPATCH_DV(U, CALL)                 \
  switch ((U) / 32) {                              \
    case 1: { constexpr int DV = 1; return CALL; } \
    case 2: { constexpr int DV = 2; return CALL; } \
    case 3: { constexpr int DV = 3; return CALL; } \
    case 4: { constexpr int DV = 4; return CALL; } \
    default: return -1;                            \
  }

int launch_hist(const Events &ev, const Geometry &g, int *cnt, int *err, float *zero_flow,
                cudaStream_t s) {
  if (ev.n == 0) return 0;
  const int grid = (int)std::min<int64_t>((ev.n + 1023) / 1024, (int64_t)num_sms() * 8);
  k_hist<<<grid, 256, 0, s>>>(ev, g, cnt, err, zero_flow);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int scan_blocks(int64_t P) { return (int)((P + kScanBlock - 1) / kScanBlock); }

int launch_scan(const Geometry &g, const int *cnt, int *bsum, int *off, int *cur, int *total,
                cudaStream_t s, bool chain) {
  const int64_t P = (int64_t)g.W * g.H;
  const int nb = scan_blocks(P);
  // the second and third kernels are chained to the one before them
  return launch_kernel(k_scan_reduce, dim3(nb), dim3(kScanThreads), 0, s, chain, cnt, P, bsum) ==
                     cudaSuccess &&
                 launch_kernel(k_scan_top, dim3(1), dim3(kScanThreads), 0, s, true, bsum, nb,
                               total) == cudaSuccess &&
                 launch_kernel(k_scan_apply, dim3(nb), dim3(kScanThreads), 0, s, true, cnt, P,
                               bsum, off, cur) == cudaSuccess
             ? 3
             : -1;
}

int launch_place(const Events &ev, const Geometry &g, int *cur, int2 *rec, int *pix,
                 cudaStream_t s, bool chain) {
  if (ev.n == 0) return 0;
  const int grid = (int)std::min<int64_t>((ev.n + 256 * kPlaceILP - 1) / (256 * kPlaceILP),
                                          (int64_t)num_sms() * 8);
  return launch_kernel(k_place, dim3(grid), dim3(256), 0, s, chain, ev, g, cur, rec, pix) ==
                 cudaSuccess
             ? 1
             : -1;
}

int bucket_sort_shift(int64_t P) {
  int shift = 0;
  while (((P + (1LL << shift) - 1) >> shift) > kMaxBuckets) ++shift;
  return shift <= kMaxBucketShift ? shift : -1;
}

int bucket_sort_max_buckets() { return kMaxBuckets; }

int bucket_sort_max_tiles() { return kMaxSortTiles; }

// events per tile: from one to two rounds of the block, as many as fill one
// wave of the scatter, and two for inputs that would need more than
// kMaxSortTiles tiles; 0 when even that is too many
static int64_t bucket_sort_tile(int64_t n) {
  const int64_t one = (int64_t)kSortILP * kSortThreads;
  if (n > 2 * one * kMaxSortTiles) return 0;
  // the fewest events per tile (a multiple of 512, from one to two rounds of
  // the block) that leave no second wave of the scatter (three blocks per SM)
  const int64_t slots = 3 * (int64_t)num_sms();
  int64_t t = (n + slots - 1) / slots;
  t = std::max(one, std::min(2 * one, (t + 511) / 512 * 512));
  if ((n + t - 1) / t > kMaxSortTiles) t = 2 * one;
  return t;
}

bool bucket_sort_fits(int64_t P, int64_t n) {
  return bucket_sort_shift(P) >= 0 && bucket_sort_tile(n) > 0;
}

int launch_bucket_sort(const Events &ev, const Geometry &g, int *cnt, int *total, int2 *rec,
                       int *rpix, int4 *brec, int *bhist, int *btot, int *err, float *zero_flow,
                       cudaStream_t s, float4 *zgrid) {
  const int64_t P = (int64_t)g.W * g.H;
  const int shift = bucket_sort_shift(P);
  const int64_t per_tile = bucket_sort_tile(ev.n);
  if (shift < 0 || per_tile == 0) return -1;
  const int nb = (int)((P + (1LL << shift) - 1) >> shift);
  if (ev.n == 0) {
    if (cudaMemsetAsync(cnt, 0, (size_t)P * sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(total, 0, sizeof(int), s) != cudaSuccess)
      return -1;
    return 0;
  }
  const int tiles = (int)((ev.n + per_tile - 1) / per_tile);
  const size_t scatter_sm = (size_t)per_tile * 3 * sizeof(int);
  const size_t sort_sm = (((size_t)1 << shift) + (size_t)kSortStage * 4) * sizeof(int);
  if (set_smem(k_bucket_scatter, scatter_sm) != cudaSuccess ||
      set_smem(k_bucket_sort, sort_sm) != cudaSuccess)
    return -1;
  const int scan_threads = std::min(1024, ((tiles + 3) / 4 + 31) / 32 * 32);
  // each kernel consumes the previous one's output: stop at a failed launch
  k_bucket_count<<<tiles, kSortThreads, 0, s>>>(ev, g, shift, nb, (int)per_tile, bhist, err,
                                               zero_flow);
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  int *bpre = bhist + (size_t)nb * tiles;
  // the other three are chained to the kernel before them
  if (launch_kernel(k_bucket_scan, dim3(nb), dim3(scan_threads), 0, s, true, bhist, nb, tiles,
                    bpre, btot) != cudaSuccess)
    return -1;
  if (launch_kernel(k_bucket_scatter, dim3(tiles), dim3(kSortThreads), scatter_sm, s, true, ev, g,
                    shift, nb, (int)per_tile, bhist, bpre, btot, brec) != cudaSuccess)
    return -1;
  return launch_kernel(k_bucket_sort, dim3(nb), dim3(kSortThreads), sort_sm, s, true, brec, shift,
                       nb, P, btot, cnt, total, rec, rpix, zgrid, g.U) == cudaSuccess
             ? 4
             : -1;
}

int launch_pixsum(const Geometry &g, const Tables &tb, const int *nsorted, const int2 *rec,
                  const int *rpix, int64_t n, float4 *acc, cudaStream_t s, bool clear,
                  bool chain) {
  VECKM_DISPATCH_DV(g.U, (pixsum_impl<DV>(g, tb, nsorted, rec, rpix, n, acc, s, clear, chain)));
}

int launch_pixsum_owned(const Geometry &g, const Tables &tb, const int *nsorted, const int2 *rec,
                        const int *rpix, int64_t n, float4 *acc, cudaStream_t s, bool chain) {
  VECKM_DISPATCH_DV(g.U, (pixsum_owned_impl<DV>(tb, nsorted, rec, rpix, n, acc, s, chain)));
}

int launch_direct(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                  const Tables &tb, const float4 *acc, const int *cnt, const MLP *mlp, float *out,
                  int *err, cudaStream_t s, bool chain) {
  if (mlp) {
    if (g.U > 64) return -2;  // W1 transposed in shared memory: 2D x 128 floats
    VECKM_DISPATCH_DV(g.U, (direct_impl<DV, true>(ev, K, nK, g, tb, acc, cnt, *mlp, out, err, s,
                                                  chain)));
  }
  VECKM_DISPATCH_DV(g.U, (direct_impl<DV, false>(ev, K, nK, g, tb, acc, cnt, MLP{}, out, err, s,
                                                 chain)));
}

int launch_pool_rows(const Geometry &g, const Tables &tb, const float4 *acc, float4 *hbuf,
                     cudaStream_t s, const Tune &tn, const int *occ, bool chain) {
  if (occ && 2 * g.dx + 1 > 32) return -1;  // the occupancy mask covers one warp's lanes
  VECKM_DISPATCH_DV(g.U, (box_pass<DV, Pass::Rows>(g, tb, acc, hbuf, s, nullptr, tn.rows_seg,
                                                   tn.rows_wpb, occ, chain)));
}

int launch_pool_cols(const Geometry &g, const Tables &tb, const float4 *hbuf, float4 *acc,
                     cudaStream_t s, const Tune &tn) {
  VECKM_DISPATCH_DV(g.U, (box_pass<DV, Pass::Cols>(g, tb, hbuf, acc, s, nullptr, tn.cols_seg,
                                                   tn.cols_wpb)));
}

int launch_pool_cols_half(const Geometry &g, const Tables &tb, const float4 *hbuf,
                          const int *ncnt, void *pooled16, cudaStream_t s, const Tune &tn) {
  VECKM_DISPATCH_DV(g.U, (box_pass<DV, Pass::Cols, kEmitF16N>(g, tb, hbuf,
                                                              reinterpret_cast<float4 *>(pooled16),
                                                              s, ncnt, tn.cols_seg, tn.cols_wpb)));
}

int launch_pool_cols_pair(const Geometry &g, const Tables &tb, const float4 *hbuf,
                          float4 *pooled, cudaStream_t s, const Tune &tn) {
  VECKM_DISPATCH_DV(g.U, (box_pass<DV, Pass::Cols, kEmitF32P>(g, tb, hbuf, pooled, s, nullptr,
                                                              tn.cols_seg, tn.cols_wpb)));
}

int launch_counts(const Geometry &g, const int *cnt, int *cnt_tmp, int *ncnt, cudaStream_t s) {
  (void)cnt_tmp;  // the tiled pass keeps its row sums in shared memory
  const size_t iw = kCountTile + 2 * (size_t)g.dx, ih = kCountTile + 2 * (size_t)g.dy;
  const size_t sm = (iw * ih + ih * kCountTile) * sizeof(int);
  if (set_smem(k_count_box, sm) != cudaSuccess) return -1;
  const dim3 grid((unsigned)((g.W + kCountTile - 1) / kCountTile),
                  (unsigned)((g.H + kCountTile - 1) / kCountTile));
  k_count_box<<<grid, 256, sm, s>>>(cnt, ncnt, g.W, g.H, g.dx, g.dy);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_gather_emb(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                      const Tables &tb, const float4 *pooled, const int *ncnt, float *emb,
                      int *err, cudaStream_t s) {
  if (nK == 0) return 0;
  VECKM_DISPATCH_DV(g.U, (gather_impl<DV>(ev, K, nK, g, tb, pooled, ncnt, emb, err, s)));
}

int launch_predict_fp32(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                        const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                        const float4 *pooled, const int *ncnt, const MLP &mlp, float *flow,
                        int *err, cudaStream_t s) {
  if (nK == 0) return 0;
  VECKM_DISPATCH_DV(g.U, (predict_fp32_impl<DV>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled,
                                                ncnt, mlp, flow, err, s)));
}

VK_CHECK_READER(check_read_kernels)

}  // namespace veckm
