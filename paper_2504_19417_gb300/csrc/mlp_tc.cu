// Perceptron on the 5th-generation tensor cores, fused with the gather.
//
// Warp-specialised pipeline, one CTA per SM pair of 128-event tiles in flight:
//   - 8 producer warps gather the rows of a tile, P[p] * conj(exp(i t T/dt))
//     (the pooled value at the event's pixel times the conjugate temporal
//     phase, Eq. 16), straight into shared memory as BF16 (or FP16) in the
//     K-major 128-byte-swizzled layout that tcgen05.mma reads: the tile is
//     split into K-blocks of 64 columns; in K-block kb, row m occupies the
//     128 bytes at kb * (128 rows * 128 B) + (m / 8) * 1024 + (m % 8) * 128,
//     and its 16-byte chunk c sits at chunk position c XOR (m % 8), so a warp
//     writing one row covers 32 distinct banks.  W1 is stored the same way.
//   - 1 MMA warp issues 2D/16 MMAs of shape 128 x 128 x 16 per tile into one
//     of two FP32 accumulators in tensor memory (2 x 128 columns) and commits
//     them to an mbarrier.
//   - 4 epilogue warps read the accumulator back with tcgen05.ld (warp w owns
//     TMEM lanes 32w..32w+31, one event row per thread), apply the window
//     count normalisation and b1 in one FMA (the first layer is linear, so
//     W1 (x / n) = (W1 x) / n), ReLU, and contract with the 2 x 128 second
//     layer on the CUDA cores.
// Shared tiles and accumulators are double buffered; the hand-offs are
// mbarriers (full: producers -> MMA and epilogue; mma_done: MMA -> epilogue;
// tmem_empty: epilogue -> MMA and producers).  No waiter can fall two phases
// behind a barrier (each role's next use of a buffer waits for the other
// roles' previous use), so parity waits are unambiguous.  Every wait is
// bounded: on time-out the kernel sets the error word and leaves.
//
// Requested events come either in pixel-sorted order (records of the
// counting sort: consecutive rows mostly share a pooled row; producers
// prefetch the following tile into L2) or by index (an explicit K list, or
// all events in input order).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "phase.cuh"
#include "veckm_internal.h"

namespace veckm {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kM = 128;  // events per tile (MMA M)
constexpr int kN = 128;  // hidden units (MMA N)
constexpr int kProdWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = kEpiWarps + kProdWarps;  // warp index of the MMA issuer
constexpr int kThreads = 32 * (kMmaWarp + 1);
constexpr int kRowsPerWarp = kM / kProdWarps;
constexpr int kTmemCols = 2 * kN;  // two accumulators
constexpr int64_t kInvalidRow = (int64_t)1 << 62;  // output row whose event was invalid
constexpr long long kWaitLimitCycles = 4000000000LL;  // ~2 s at 2 GHz, then give up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float4 cmul2c(float4 a, float4 b) {
  return make_float4(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y),
                     fmaf(a.z, b.z, a.w * b.w), fmaf(a.w, b.z, -a.z * b.w));
}

// Shared-memory matrix descriptor, K-major with 128-byte swizzling: start
// address, stride byte offset 1024 (next group of 8 rows), leading byte
// offset unused for this layout, fixed version bits 0b001 at 46, swizzle
// mode 2 (128B) at bits 61-63.  Every swizzle atom starts 1024-aligned.
__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16 (1) or F16 (0),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int half_kind_fp16, int M, int N) {
  const uint32_t ab = half_kind_fp16 ? 0u : 1u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack2(float a, float b, int fp16) {
  if (fp16) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
  }
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kWaitLimitCycles) return false;
  }
}

// d = a * b + c on two FP32 lanes at once (packed FP32x2, one instruction)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<const uint64_t *>(&a)), "l"(*reinterpret_cast<const uint64_t *>(&b)),
        "l"(*reinterpret_cast<const uint64_t *>(&c)));
  return *reinterpret_cast<const float2 *>(&d);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int DV, bool HALF>
__global__ void __launch_bounds__(kThreads, DV == 1 ? 2 : 1)
    k_predict_tc(Events ev, const int64_t *__restrict__ K, int64_t nK,
                 const int2 *__restrict__ rec, const int *__restrict__ rpix,
                 const int *__restrict__ nsorted, Geometry g, Tables tb,
                 const void *__restrict__ pooled_v, const int *__restrict__ ncnt, MLP mlp,
                 float *__restrict__ flow, int *err) {
  constexpr int U = 32 * DV;
  constexpr int IN = 4 * U;  // 2D, the MMA K extent
  constexpr int TILE_BYTES = kM * IN * 2;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = smem;                            // 2 x [128 x IN] half, SW128
  uint8_t *sB = smem + 2 * TILE_BYTES;           // [128 x IN] half (W1), SW128
  float *sB1 = reinterpret_cast<float *>(sB + TILE_BYTES);    // [128]
  float *sW2 = sB1 + kN;                                       // [2][128]
  float *sInv = sW2 + 2 * kN;                                  // [2][128] 1 / window count
  int64_t *sK = reinterpret_cast<int64_t *>(sInv + 2 * kM);    // [2][128] output rows
  uint64_t *bars = reinterpret_cast<uint64_t *>(sK + 2 * kM);  // full[2], done[2], empty[2]
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 6);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fp16 = mlp.half_kind;
  const int D = g.D;

  {  // W1 (already in SW128 order), b1, W2
    const uint4 *src = reinterpret_cast<const uint4 *>(mlp.W1h);
    uint4 *dst = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < TILE_BYTES / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    for (int i = tid; i < kN; i += blockDim.x) {
      sB1[i] = mlp.b1[i];
      sW2[i] = mlp.W2[i];
      sW2[kN + i] = mlp.W2[kN + i];
    }
  }
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int b) { return bar0 + 8u * b; };
  auto done_bar = [&](int b) { return bar0 + 8u * (2 + b); };
  auto empty_bar = [&](int b) { return bar0 + 8u * (4 + b); };
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full_bar(b)), "r"(kProdWarps));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done_bar(b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty_bar(b)), "r"(kEpiWarps));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int64_t ns = rec ? (int64_t)*nsorted : nK;
  const int64_t ntiles_all = (nK + kM - 1) / kM;
  const int nlocal = blockIdx.x < ntiles_all
                         ? (int)((ntiles_all - 1 - blockIdx.x) / gridDim.x + 1)
                         : 0;
  bool ok = true;

  if (warp >= kEpiWarps && warp < kMmaWarp) {
    // ------------------------------------------------------------ producers
    const int pw = warp - kEpiWarps;
    uint2 wf[DV][2];  // fixed-point frequencies of this lane's channels
#pragma unroll
    for (int v = 0; v < DV; ++v) {
      wf[v][0] = __ldg(tb.wt + 2 * (lane + 32 * v));
      wf[v][1] = __ldg(tb.wt + 2 * (lane + 32 * v) + 1);
    }
    // row metadata of tile t for this lane: pixel (-1 if none/invalid), t - t_ref, output row
    auto meta = [&](int64_t t, int &pix, uint32_t &trel, int64_t &outk) {
      const int64_t i = t * kM + pw * kRowsPerWarp + (lane & (kRowsPerWarp - 1));
      pix = -1;
      trel = 0;
      outk = -1;
      if (i >= ns) return;
      if (rec) {
        const int2 r = __ldg(rec + i);
        pix = __ldg(rpix + i);
        trel = (uint32_t)r.x;
        outk = r.y;
        return;
      }
      int64_t k = i;
      if (K) {
        k = K[i];
        if (k < 0 || k >= ev.n) {
          if (lane < kRowsPerWarp) atomicOr(err, ERR_INDEX_RANGE);
          outk = i | kInvalidRow;  // an invalid index's row gets zeros
          return;
        }
      }
      const int x = ev.x[k], y = ev.y[k];
      const uint32_t tt = ev.t[k];
      trel = tt - ev.t_ref;
      if (x >= 0 && x < g.W && y >= 0 && y < g.H && tt >= ev.t_ref && trel <= ev.t_span)
        pix = y * g.W + x;
      outk = pix >= 0 ? i : (i | kInvalidRow);  // an invalid event's row gets zeros
    };
    int m_pix;
    uint32_t m_trel;
    int64_t m_outk;
    if (nlocal > 0) meta(blockIdx.x, m_pix, m_trel, m_outk);
    for (int li = 0; li < nlocal && ok; ++li) {
      const int b = li & 1;
      const int64_t tile = blockIdx.x + (int64_t)li * gridDim.x;
      if (li >= 2 && !mbar_wait(empty_bar(b), ((li >> 1) - 1) & 1)) {
        ok = false;
        break;
      }
      if (rec) {  // L2 prefetch of this warp's rows of the tile after next
        const int64_t nt = tile + 2 * (int64_t)gridDim.x;
        const int64_t i = nt * kM + pw * kRowsPerWarp + (lane & (kRowsPerWarp - 1));
        if (i < ns) {
          const int p = __ldg(rpix + i);
          constexpr int kRowBytes = (HALF ? 8 : 16) * U;  // pooled bytes per pixel
          constexpr int kHalfLines = kRowBytes / 256;      // 128-byte lines per half row
          const char *row = reinterpret_cast<const char *>(pooled_v) + (size_t)p * kRowBytes;
#pragma unroll
          for (int l = 0; l < kHalfLines; ++l)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row + ((lane >> 4) * kHalfLines + l) * 128));
        }
      }
      // lane j < 16 holds the metadata of row pw*16 + j (loaded one tile ahead)
      const int pix = m_pix;
      const uint32_t trel = m_trel;
      const int64_t outk = m_outk;
      if (li + 1 < nlocal) meta(tile + gridDim.x, m_pix, m_trel, m_outk);
      if (lane < kRowsPerWarp) {
        sK[b * kM + pw * kRowsPerWarp + lane] = outk;
        sInv[b * kM + pw * kRowsPerWarp + lane] =
            pix < 0 ? 0.f : (HALF ? 1.f : 1.0f / (float)__ldg(ncnt + pix));
      }
      uint8_t *A = sA + b * TILE_BYTES;
      // rows whose loads are issued together: 8 x 8 bytes per lane on the FP16
      // grid, 4 x 16 bytes on the FP32 grid
      constexpr int kB = HALF ? 8 / DV : 4 / DV;
#pragma unroll
      for (int j0 = 0; j0 < kRowsPerWarp; j0 += kB) {
        // FP32 grid: float4 (re 2u, im 2u, re 2u+1, im 2u+1) per unit;
        // FP16 grid: uint2 (half2 re pair, half2 im pair), already divided by n
        float4 pv[kB][DV];
        uint2 qv[kB][DV];
        uint32_t tjs[kB];
#pragma unroll
        for (int r = 0; r < kB; ++r) {
          const int pj = __shfl_sync(kFull, pix, j0 + r);
          tjs[r] = __shfl_sync(kFull, trel, j0 + r);
#pragma unroll
          for (int v = 0; v < DV; ++v) {
            if constexpr (HALF)
              qv[r][v] = pj >= 0 ? __ldg(reinterpret_cast<const uint2 *>(pooled_v) +
                                         (size_t)pj * U + lane + 32 * v)
                                 : make_uint2(0u, 0u);
            else
              pv[r][v] = pj >= 0 ? __ldg(reinterpret_cast<const float4 *>(pooled_v) +
                                         (size_t)pj * U + lane + 32 * v)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int r = 0; r < kB; ++r) {
          const int m = pw * kRowsPerWarp + j0 + r;
          const uint32_t rowoff = (m >> 3) * 1024 + (m & 7) * 128;
#pragma unroll
          for (int v = 0; v < DV; ++v) {
            const int u = lane + 32 * v;
            const uint32_t kr = 2 * u, ki = D + 2 * u;
            const uint32_t cr = (kr >> 6) * (kM * 128) + rowoff +
                                ((((kr >> 3) & 7) ^ (m & 7)) << 4) + (kr & 7) * 2;
            const uint32_t ci = (ki >> 6) * (kM * 128) + rowoff +
                                ((((ki >> 3) & 7) ^ (m & 7)) << 4) + (ki & 7) * 2;
            const float4 ph = time_phase2(tjs[r], wf[v][0], wf[v][1]);  // (c0, s0, c1, s1)
            uint32_t wre, wim;
            if constexpr (HALF) {
              // packed half2: Re = PR C + PI S, Im = PI C - PR S (both channels at once)
              const __half2 PR = *reinterpret_cast<const __half2 *>(&qv[r][v].x);
              const __half2 PI = *reinterpret_cast<const __half2 *>(&qv[r][v].y);
              const __half2 C = __floats2half2_rn(ph.x, ph.z);
              const __half2 S = __floats2half2_rn(ph.y, ph.w);
              const __half2 ER = __hfma2(PR, C, __hmul2(PI, S));
              const __half2 EI = __hfma2(PI, C, __hneg2(__hmul2(PR, S)));
              if (fp16) {
                wre = *reinterpret_cast<const uint32_t *>(&ER);
                wim = *reinterpret_cast<const uint32_t *>(&EI);
              } else {
                const float2 fr = __half22float2(ER), fi = __half22float2(EI);
                wre = pack2(fr.x, fr.y, 0);
                wim = pack2(fi.x, fi.y, 0);
              }
            } else {
              const float4 e = cmul2c(pv[r][v], ph);
              wre = pack2(e.x, e.z, fp16);
              wim = pack2(e.y, e.w, fp16);
            }
            *reinterpret_cast<uint32_t *>(A + cr) = wre;
            *reinterpret_cast<uint32_t *>(A + ci) = wim;
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(full_bar(b));
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t idesc_bf16 = make_idesc(0, kM, kN);
    constexpr uint32_t idesc_fp16 = make_idesc(1, kM, kN);
    const uint32_t idesc = fp16 ? idesc_fp16 : idesc_bf16;
    const uint32_t sA_a = smem_u32(sA), sB_a = smem_u32(sB);
    for (int li = 0; li < nlocal && ok; ++li) {
      const int b = li & 1;
      if (!mbar_wait(full_bar(b), (li >> 1) & 1) ||
          (li >= 2 && !mbar_wait(empty_bar(b), ((li >> 1) - 1) & 1))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (lane == 0) {
        const uint32_t d_tmem = tmem + (uint32_t)(b * kN);
        const uint32_t a_base = sA_a + b * TILE_BYTES;
#pragma unroll
        for (int kk = 0; kk < IN / 16; ++kk) {
          // K-step kk: K-block kk / 4, 32-byte step kk % 4 inside the swizzle atom
          const uint32_t koff = (kk >> 2) * (kM * 128) + (kk & 3) * 32;
          const uint64_t ad = make_desc_sw128(a_base + koff);
          const uint64_t bd = make_desc_sw128(sB_a + koff);
          const uint32_t acc = kk > 0 ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                done_bar(b))
            : "memory");
      }
      __syncwarp();
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int row = warp * 32 + lane;  // TMEM lane = tile row
    const float b20 = mlp.b2[0], b21 = mlp.b2[1];
    for (int li = 0; li < nlocal && ok; ++li) {
      const int b = li & 1;
      // full: the producers' row metadata; done: the accumulator
      if (!mbar_wait(full_bar(b), (li >> 1) & 1) || !mbar_wait(done_bar(b), (li >> 1) & 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float inv = sInv[b * kM + row];
      const int64_t k = sK[b * kM + row];
      // packed FP32x2 arithmetic: even and odd columns in the two halves
      float2 o0 = make_float2(0.f, 0.f), o1 = make_float2(0.f, 0.f);
      const float2 inv2 = make_float2(inv, inv);
      const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * kN);
#pragma unroll
      for (int c0 = 0; c0 < kN; c0 += 16) {
        float h[16];
        tmem_ld16(base + c0, h);
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const float4 bb = *reinterpret_cast<const float4 *>(sB1 + c0 + j);
          const float4 w0 = *reinterpret_cast<const float4 *>(sW2 + c0 + j);
          const float4 w1 = *reinterpret_cast<const float4 *>(sW2 + kN + c0 + j);
          float2 a01 = ffma2(make_float2(h[j], h[j + 1]), inv2, make_float2(bb.x, bb.y));
          float2 a23 = ffma2(make_float2(h[j + 2], h[j + 3]), inv2, make_float2(bb.z, bb.w));
          a01.x = fmaxf(a01.x, 0.f); a01.y = fmaxf(a01.y, 0.f);
          a23.x = fmaxf(a23.x, 0.f); a23.y = fmaxf(a23.y, 0.f);
          o0 = ffma2(a01, make_float2(w0.x, w0.y), o0);
          o0 = ffma2(a23, make_float2(w0.z, w0.w), o0);
          o1 = ffma2(a01, make_float2(w1.x, w1.y), o1);
          o1 = ffma2(a23, make_float2(w1.z, w1.w), o1);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(empty_bar(b));
      if (k >= 0) {
        const bool valid = !(k & kInvalidRow);
        *reinterpret_cast<float2 *>(flow + 2 * (k & ~kInvalidRow)) =
            valid ? make_float2(o0.x + o0.y + b20, o1.x + o1.y + b21) : make_float2(0.f, 0.f);
      }
    }
  }
  if (!ok && lane == 0) atomicOr(err, ERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      // let MMAs that may still be in flight land before their TMEM is freed
      for (int b = 0; b < 2; ++b) mbar_wait(done_bar(b), 0), mbar_wait(done_bar(b), 1);
    }
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

template <int DV, bool HALF>
int predict_tc_impl(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                    const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                    const void *pooled, const int *ncnt, const MLP &mlp, float *flow, int *err,
                    cudaStream_t s) {
  if (nK == 0) return 0;
  constexpr int IN = 128 * DV;
  const size_t sm = (size_t)3 * kM * IN * 2 + sizeof(float) * (3 * kN + 2 * kM) +
                    sizeof(int64_t) * 2 * kM + 8 * 6 + 16 + 1024;  // + SW128 alignment slack
  auto kern = k_predict_tc<DV, HALF>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
          cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return -1;
  const int per_sm = std::min(blocks_per_sm((const void *)kern, kThreads, sm), 512 / kTmemCols);
  const int64_t tiles = (nK + kM - 1) / kM;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * per_sm);
  kern<<<grid, kThreads, sm, s>>>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow,
                                  err);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

int launch_predict_tc(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                      const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                      const void *pooled, const int *ncnt, const MLP &mlp, float *flow,
                      int *err, cudaStream_t s) {
  const bool h = mlp.pooled_half != 0;
  switch (g.U / 32) {
    case 1:
      return h ? predict_tc_impl<1, true>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow, err, s)
               : predict_tc_impl<1, false>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow, err, s);
    case 2:
      return h ? predict_tc_impl<2, true>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow, err, s)
               : predict_tc_impl<2, false>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow, err, s);
    default:
      return -1;  // 2D > 256 does not fit the operand tiles in shared memory
  }
}

}  // namespace veckm
