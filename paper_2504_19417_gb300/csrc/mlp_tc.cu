// Perceptron on the 5th-generation tensor cores, fused with the gather.
//
// For a tile of 128 requested events the CTA (8 warps) gathers emb_k (the
// pooled value at the event's pixel times the conjugate temporal phase over
// the window count, Eq. 16) straight into shared memory as BF16 (or FP16),
// in the K-major 128-byte-swizzled layout that tcgen05.mma reads: the tile is
// split into K-blocks of 64 columns; in K-block kb, row m occupies the 128
// bytes at kb * (128 rows * 128 B) + (m / 8) * 1024 + (m % 8) * 128, and its
// 16-byte chunk c (columns 8c..8c+7 of the block) sits at chunk position
// c XOR (m % 8).  A warp writing one row therefore covers 32 distinct banks.
// W1 is stored the same way (rows = hidden units).  One thread issues 2D/16
// MMAs of shape 128 x 128 x 16 with the FP32 accumulator in tensor memory
// (128 columns) and commits them to an mbarrier; after the bounded wait the
// warps read the accumulator back with tcgen05.ld (warp w reads lane quadrant
// w % 4, column half w / 4), add b1, apply ReLU and contract with the 2 x 128
// second layer on the CUDA cores.
//
// Requested events come either in pixel-sorted order (records from the
// counting sort: consecutive rows mostly share a pooled row; the next tile's
// rows are prefetched into L2 while this one computes) or by index (an
// explicit K list, or all events in input order).
//
// The first layer is the dense contraction [128 x 2D] x [2D x 128]; the
// second layer (128 -> 2) is too thin for the tensor cores and stays in
// registers.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "phase.cuh"
#include "veckm_internal.h"

namespace veckm {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kM = 128;    // events per tile (MMA M)
constexpr int kN = 128;    // hidden units (MMA N)
constexpr int kWarps = 8;
constexpr int kRowsPerWarp = kM / kWarps;
constexpr int kTmemCols = 128;
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

// byte offset of element (r, k) in a K-major SW128 tile of 128 rows
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)((k >> 6) * (128 * 128) + (r >> 3) * 1024 + (r & 7) * 128 +
                    ((((k >> 3) & 7) ^ (r & 7)) << 4) + (k & 7) * 2);
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

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int DV>
__global__ void __launch_bounds__(kWarps * 32, 2)
    k_predict_tc(Events ev, const int64_t *__restrict__ K, int64_t nK,
                 const int2 *__restrict__ rec, const int *__restrict__ rpix,
                 const int *__restrict__ nsorted, Geometry g,
                 Tables tb, const float4 *__restrict__ pooled, const int *__restrict__ ncnt,
                 MLP mlp, float *__restrict__ flow, int *err) {
  constexpr int U = 32 * DV;
  constexpr int IN = 4 * U;            // 2D, the MMA K extent
  constexpr int TILE_BYTES = kM * IN * 2;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = smem;                     // [128 x IN] half, SW128 layout
  uint8_t *sB = smem + TILE_BYTES;        // [128 x IN] half (W1), same layout
  float *sB1 = reinterpret_cast<float *>(sB + kN * IN * 2);  // [128]
  float *sW2 = sB1 + kN;                                      // [2][128]
  float2 *sPart = reinterpret_cast<float2 *>(sW2 + 2 * kN);   // [128] partial outputs
  int64_t *sK = reinterpret_cast<int64_t *>(sPart + kM);      // [128] output rows
  uint64_t *bar = reinterpret_cast<uint64_t *>(sK + kM);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fp16 = mlp.half_kind;
  const int D = g.D;
  uint2 wf[DV][2];  // fixed-point frequencies of this lane's channels
#pragma unroll
  for (int v = 0; v < DV; ++v) {
    wf[v][0] = __ldg(tb.wt + 2 * (lane + 32 * v));
    wf[v][1] = __ldg(tb.wt + 2 * (lane + 32 * v) + 1);
  }

  // W1 (already in SW128 order), b1, W2 into shared memory.
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(mlp.W1h);
    uint4 *dst = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < kN * IN * 2 / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    for (int i = tid; i < kN; i += blockDim.x) {
      sB1[i] = mlp.b1[i];
      sW2[i] = mlp.W2[i];
      sW2[kN + i] = mlp.W2[kN + i];
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
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
  const uint32_t bar_a = smem_u32(bar);
  const uint32_t sA_a = smem_u32(sA), sB_a = smem_u32(sB);
  constexpr uint32_t idesc_bf16 = make_idesc(0, kM, kN);
  constexpr uint32_t idesc_fp16 = make_idesc(1, kM, kN);
  const uint32_t idesc = fp16 ? idesc_fp16 : idesc_bf16;
  const float b20 = mlp.b2[0], b21 = mlp.b2[1];
  uint32_t phase = 0;
  bool timed_out = false;
  const int64_t ns = rec ? (int64_t)*nsorted : nK;
  // L2 prefetch of the next tile (sorted order): thread tid covers half of
  // row tid % 128; its pixel index is loaded one tile ahead.
  const int pf_row = tid & (kM - 1), pf_half = tid >> 7;
  auto pf_pixel = [&](int64_t t) -> int {
    const int64_t i = t * kM + pf_row;
    return (rec && i < ns) ? __ldg(rpix + i) : -1;
  };
  int pf_pix = pf_pixel((int64_t)blockIdx.x + gridDim.x);

  for (int64_t tile = blockIdx.x; tile * kM < nK; tile += gridDim.x) {
    if (rec) {
      if (pf_pix >= 0) {
        const char *row = reinterpret_cast<const char *>(pooled + (size_t)pf_pix * U);
#pragma unroll
        for (int l = 0; l < 2 * DV; ++l)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(row + (pf_half * 2 * DV + l) * 128));
      }
      const int64_t nt = tile + 2 * (int64_t)gridDim.x;
      if (tid < 12 && nt * kM < ns) {  // records (1 KB) and pixels (512 B) of the tile after
        const char *pr = tid < 8 ? reinterpret_cast<const char *>(rec + nt * kM) + tid * 128
                                 : reinterpret_cast<const char *>(rpix + nt * kM) + (tid - 8) * 128;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(pr));
      }
      pf_pix = pf_pixel(tile + 2 * (int64_t)gridDim.x);
    }
    // --- gather 16 rows per warp into sA ---------------------------------
    {
      // lane j < 16 holds the metadata of row warp*16 + j
      const int64_t i = tile * kM + warp * kRowsPerWarp + (lane & (kRowsPerWarp - 1));
      int pix = -1;
      uint32_t trel = 0;
      float inv = 0.f;
      int64_t outk = -1;
      if (i < ns) {
        if (rec) {
          const int2 r = __ldg(rec + i);
          pix = __ldg(rpix + i);
          trel = (uint32_t)r.x;
          outk = r.y;
          inv = 1.0f / (float)__ldg(ncnt + pix);
        } else {
          int64_t k = i;
          bool ok = true;
          if (K) {
            k = K[i];
            if (k < 0 || k >= ev.n) {
              if (lane < kRowsPerWarp) atomicOr(err, ERR_INDEX_RANGE);
              ok = false;
            }
          }
          if (ok) {
            const int x = ev.x[k], y = ev.y[k];
            const uint32_t t = ev.t[k];
            trel = t - ev.t_ref;
            if (x >= 0 && x < g.W && y >= 0 && y < g.H && t >= ev.t_ref && trel <= ev.t_span) {
              pix = y * g.W + x;
              inv = 1.0f / (float)__ldg(ncnt + pix);
            }
          }
          outk = pix >= 0 ? i : (i | kInvalidRow);  // an invalid event's row gets zeros
        }
      }
      if (lane < kRowsPerWarp) sK[warp * kRowsPerWarp + lane] = outk;
      // batches of rows: all pooled-row loads of a batch are issued before any
      // is used; the temporal phase is computed, not loaded
      constexpr int kB = 8 / DV;
#pragma unroll
      for (int j0 = 0; j0 < kRowsPerWarp; j0 += kB) {
        float4 pv[kB][DV];
        int pjs[kB];
#pragma unroll
        for (int r = 0; r < kB; ++r) {
          pjs[r] = __shfl_sync(kFull, pix, j0 + r);
          const int pc = pjs[r] >= 0 ? pjs[r] : 0;
#pragma unroll
          for (int v = 0; v < DV; ++v) pv[r][v] = __ldg(pooled + (size_t)pc * U + lane + 32 * v);
        }
#pragma unroll
        for (int r = 0; r < kB; ++r) {
          const int m = warp * kRowsPerWarp + j0 + r;
          const float ij = __shfl_sync(kFull, inv, j0 + r);
          const uint32_t tj = __shfl_sync(kFull, trel, j0 + r);
          const float sc = pjs[r] >= 0 ? ij : 0.f;
#pragma unroll
          for (int v = 0; v < DV; ++v) {
            const int u = lane + 32 * v;
            float4 e = cmul2c(pv[r][v], time_phase2(tj, wf[v][0], wf[v][1]));
            e.x *= sc; e.y *= sc; e.z *= sc; e.w *= sc;
            // Re of channels 2u, 2u+1 at columns k = 2u, 2u+1; Im at D + 2u, D + 2u + 1
            *reinterpret_cast<uint32_t *>(sA + sw128_off(m, 2 * u)) = pack2(e.x, e.z, fp16);
            *reinterpret_cast<uint32_t *>(sA + sw128_off(m, D + 2 * u)) = pack2(e.y, e.w, fp16);
          }
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // --- one thread issues the MMAs ------------------------------------------
    if (tid == 0) {
#pragma unroll
      for (int kk = 0; kk < IN / 16; ++kk) {
        // K-step kk: K-block kk / 4, 32-byte step kk % 4 inside the swizzle atom
        const uint32_t koff = (kk >> 2) * (kM * 128) + (kk & 3) * 32;
        const uint64_t ad = make_desc_sw128(sA_a + koff);
        const uint64_t bd = make_desc_sw128(sB_a + koff);
        const uint32_t acc = kk > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              bar_a)
          : "memory");
    }
    if (mbar_wait(bar_a, phase)) {
      phase ^= 1u;
    } else {
      if (lane == 0) atomicOr(err, ERR_TIMEOUT);
      timed_out = true;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(timed_out)) {
      timed_out = true;
      break;
    }
    // --- epilogue: bias, ReLU, second layer ----------------------------------
    {
      const int q = warp & 3, hh = warp >> 2;
      const int row = q * 32 + lane;
      float o0 = 0.f, o1 = 0.f;
      const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll
      for (int c0 = hh * (kN / 2); c0 < (hh + 1) * (kN / 2); c0 += 32) {
        float h[32];
        tmem_ld32(lane_base + c0, h);
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 bb = *reinterpret_cast<const float4 *>(sB1 + c0 + j);
          const float4 w0 = *reinterpret_cast<const float4 *>(sW2 + c0 + j);
          const float4 w1 = *reinterpret_cast<const float4 *>(sW2 + kN + c0 + j);
          const float a0 = fmaxf(h[j] + bb.x, 0.f), a1 = fmaxf(h[j + 1] + bb.y, 0.f);
          const float a2 = fmaxf(h[j + 2] + bb.z, 0.f), a3 = fmaxf(h[j + 3] + bb.w, 0.f);
          o0 = fmaf(a3, w0.w, fmaf(a2, w0.z, fmaf(a1, w0.y, fmaf(a0, w0.x, o0))));
          o1 = fmaf(a3, w1.w, fmaf(a2, w1.z, fmaf(a1, w1.y, fmaf(a0, w1.x, o1))));
        }
      }
      if (hh == 1) sPart[row] = make_float2(o0, o1);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (hh == 0) {
        const float2 pp = sPart[row];
        const int64_t k = sK[row];
        if (k >= 0) {
          const bool ok = !(k & kInvalidRow);
          *reinterpret_cast<float2 *>(flow + 2 * (k & ~kInvalidRow)) =
              ok ? make_float2(o0 + pp.x + b20, o1 + pp.y + b21) : make_float2(0.f, 0.f);
        }
      }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (timed_out) {
    // Let an MMA that may still be in flight land before freeing its TMEM.
    mbar_wait(bar_a, phase);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

template <int DV>
int predict_tc_impl(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                    const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb, const float4 *pooled,
                    const int *ncnt, const MLP &mlp, float *flow, int *err, cudaStream_t s) {
  if (nK == 0) return 0;
  constexpr int IN = 128 * DV;
  const size_t sm = (size_t)2 * kM * IN * 2 + sizeof(float) * 3 * kN + sizeof(float2) * kM +
                    sizeof(int64_t) * kM + 64 + 1024;  // + alignment slack for the SW128 atoms
  if (cudaFuncSetAttribute(k_predict_tc<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_predict_tc<DV>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return -1;
  const int per_sm = std::min(blocks_per_sm((const void *)k_predict_tc<DV>, kWarps * 32, sm),
                              512 / kTmemCols);
  const int64_t tiles = (nK + kM - 1) / kM;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * per_sm);
  k_predict_tc<DV><<<grid, kWarps * 32, sm, s>>>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled,
                                                 ncnt, mlp, flow, err);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

int launch_predict_tc(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                      const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                      const float4 *pooled, const int *ncnt, const MLP &mlp, float *flow,
                      int *err, cudaStream_t s) {
  switch (g.U / 32) {
    case 1:
      return predict_tc_impl<1>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow, err, s);
    case 2:
      return predict_tc_impl<2>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow, err, s);
    default: return -1;  // 2D > 256 does not fit two operand tiles in shared memory
  }
}

}  // namespace veckm
