// Perceptron on the 5th-generation tensor cores, fused with the gather.
//
// For a tile of 128 requested events the CTA gathers emb_k (pooled value at
// the event's pixel times the conjugate temporal phase over the window count,
// Algorithm 1 line 21) straight into shared memory as BF16 (or FP16), in the
// K-major "core matrix" layout that tcgen05.mma reads without swizzle:
// element (row m, column k) sits at byte
//     (m / 8) * SBO + (k / 8) * LBO + (m % 8) * 16 + (k % 8) * 2,
// with LBO = 128 (next 8 columns) and SBO = 16 * K (next 8 rows).  W1 is kept
// in the same layout (rows = hidden units).  One thread issues K/16 MMAs of
// shape 128 x 128 x 16 with the FP32 accumulator in tensor memory (128
// columns), commits them to an mbarrier, and after the (bounded) wait each
// warp reads its 32 accumulator lanes back with tcgen05.ld, adds b1, applies
// ReLU and contracts with the 2 x 128 second layer on the CUDA cores.
//
// The first layer is the dense contraction [128 x 2D] x [2D x 128]; the second
// layer (128 -> 2) is too thin for the tensor cores and stays in registers.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "veckm_internal.h"

namespace veckm {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kM = 128;    // events per tile (MMA M)
constexpr int kN = 128;    // hidden units (MMA N)
constexpr int kTmemCols = 128;
constexpr long long kWaitLimitCycles = 4000000000LL;  // ~2 s at 2 GHz, then give up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float4 cmul2c(float4 a, float4 b) {
  return make_float4(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y),
                     fmaf(a.z, b.z, a.w * b.w), fmaf(a.w, b.z, -a.z * b.w));
}
__device__ __forceinline__ float4 cmul2(float4 a, float4 b) {
  return make_float4(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x),
                     fmaf(a.z, b.z, -a.w * b.w), fmaf(a.z, b.w, a.w * b.z));
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // fixed 0b001 (descriptor version)
  // base offset 0, relative LBO, swizzle mode 0 (none)
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
__global__ void __launch_bounds__(128, 1)
    k_predict_tc(Events ev, const int64_t *__restrict__ K, int64_t nK, Geometry g, Tables tb,
                 const float4 *__restrict__ pooled, const int *__restrict__ ncnt, MLP mlp,
                 float *__restrict__ flow, int *err) {
  constexpr int U = 32 * DV;
  constexpr int IN = 4 * U;            // 2D, the MMA K extent
  constexpr int SBO = 16 * IN;         // bytes between 8-row groups
  constexpr int LBO = 128;             // bytes between 8-column groups
  constexpr int TILE_BYTES = kM * IN * 2;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sA = smem;                     // [128 x IN] half, core-matrix layout
  uint8_t *sB = smem + TILE_BYTES;        // [128 x IN] half (W1), same layout
  float *sB1 = reinterpret_cast<float *>(sB + kN * IN * 2);  // [128]
  float *sW2 = sB1 + kN;                                      // [2][128]
  uint64_t *bar = reinterpret_cast<uint64_t *>(sW2 + 2 * kN);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fp16 = mlp.half_kind;
  const int D = g.D;

  // W1 (already in core-matrix order), b1, W2 into shared memory.
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

  for (int64_t tile = blockIdx.x; tile * kM < nK; tile += gridDim.x) {
    // --- gather 32 rows per warp into sA ---------------------------------
    {
      const int64_t i = tile * kM + warp * 32 + lane;  // this lane's event (metadata)
      int pix = -1;
      uint32_t trel = 0;
      float inv = 0.f;
      if (i < nK) {
        int64_t k = i;
        bool ok = true;
        if (K) {
          k = K[i];
          if (k < 0 || k >= ev.n) {
            atomicOr(err, ERR_INDEX_RANGE);
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
      }
#pragma unroll 4
      for (int j = 0; j < 32; ++j) {
        const int pj = __shfl_sync(kFull, pix, j);
        const uint32_t tj = __shfl_sync(kFull, trel, j);
        const float ij = __shfl_sync(kFull, inv, j);
        const int m = warp * 32 + j;
        uint8_t *rowp = sA + (m >> 3) * SBO + (m & 7) * 16;
#pragma unroll
        for (int v = 0; v < DV; ++v) {
          const int u = lane + 32 * v;
          float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
          if (pj >= 0) {
            const float4 pv = __ldg(pooled + (size_t)pj * U + u);
            const float4 ph = cmul2(__ldg(tb.tt_hi + (size_t)(tj >> kTLoBits) * U + u),
                                    __ldg(tb.tt_lo + (size_t)(tj & (kTLo - 1)) * U + u));
            e = cmul2c(pv, ph);
            e.x *= ij; e.y *= ij; e.z *= ij; e.w *= ij;
          }
          // Re of channels 2u, 2u+1 at columns k = 2u, 2u+1; Im at D + 2u, D + 2u + 1
          const int kr = 2 * u, ki = D + 2 * u;
          *reinterpret_cast<uint32_t *>(rowp + (kr >> 3) * LBO + (kr & 7) * 2) = pack2(e.x, e.z, fp16);
          *reinterpret_cast<uint32_t *>(rowp + (ki >> 3) * LBO + (ki & 7) * 2) = pack2(e.y, e.w, fp16);
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
        const uint64_t ad = make_desc(sA_a + kk * 2 * LBO, LBO, SBO);
        const uint64_t bd = make_desc(sB_a + kk * 2 * LBO, LBO, SBO);
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
      float o0 = 0.f, o1 = 0.f;
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
      for (int c0 = 0; c0 < kN; c0 += 32) {
        float h[32];
        tmem_ld32(lane_base + c0, h);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float a = fmaxf(h[j] + sB1[c0 + j], 0.f);
          o0 = fmaf(a, sW2[c0 + j], o0);
          o1 = fmaf(a, sW2[kN + c0 + j], o1);
        }
      }
      const int64_t idx = tile * kM + warp * 32 + lane;
      if (idx < nK) *reinterpret_cast<float2 *>(flow + 2 * idx) = make_float2(o0 + b20, o1 + b21);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
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
int predict_tc_impl(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                    const Tables &tb, const float4 *pooled, const int *ncnt, const MLP &mlp,
                    float *flow, int *err, cudaStream_t s) {
  if (nK == 0) return 0;
  constexpr int IN = 128 * DV;
  const size_t sm = (size_t)2 * kM * IN * 2 + sizeof(float) * 3 * kN + 64;
  if (sm > 48 * 1024 &&
      cudaFuncSetAttribute(k_predict_tc<DV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess)
    return -1;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_predict_tc<DV>, 128, sm);
  per_sm = std::max(1, std::min(per_sm, 512 / kTmemCols));
  const int64_t tiles = (nK + kM - 1) / kM;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * per_sm);
  k_predict_tc<DV><<<grid, 128, sm, s>>>(ev, K, nK, g, tb, pooled, ncnt, mlp, flow, err);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

int launch_predict_tc(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                      const Tables &tb, const float4 *pooled, const int *ncnt, const MLP &mlp,
                      float *flow, int *err, cudaStream_t s) {
  switch (g.U / 32) {
    case 1: return predict_tc_impl<1>(ev, K, nK, g, tb, pooled, ncnt, mlp, flow, err, s);
    case 2: return predict_tc_impl<2>(ev, K, nK, g, tb, pooled, ncnt, mlp, flow, err, s);
    default: return -1;  // 2D > 256 does not fit two operand tiles in shared memory
  }
}

}  // namespace veckm
