// Perceptron on the 5th-generation tensor cores, fused with the gather.
//
// Each 128-event tile takes the first layer (Eq. 6) as one 128 x 128 x 2D
// tcgen05.mma chain (K steps of 16, FP32 accumulator in tensor memory) and
// the second layer as one 128 x 16 x 128 chain.  Warp-specialised roles:
//   - producer warps gather the rows of a tile, P[p] * conj(exp(i t T/dt))
//     (the pooled value at the event's pixel times the conjugate temporal
//     phase, Eq. 16), rounded to BF16 (or FP16), the first layer's A operand.
//     The K axis is ordered per unit u as Re(2u), Re(2u+1), Im(2u), Im(2u+1);
//     W1 is stored with its columns permuted to match.
//   - epilogue warps read the accumulator back with tcgen05.ld (TMEM lane =
//     tile row, one event row per thread), apply the window-count
//     normalisation and b1 in one FMA (the first layer is linear, so
//     W1 (x / n) = (W1 x) / n), and write ReLU(h) as FP16 pairs back into
//     the first 64 columns of the same accumulator (tcgen05.st).  The second
//     layer reads that A operand from tensor memory and B = W2 (2 x 128,
//     padded to 16 rows, FP16 in shared memory) and writes the two outputs
//     into columns 64..79 of the accumulator, which the epilogue reads back
//     (tcgen05.ld), adds b2 to, and stores.  One thread of an epilogue warp
//     issues the MMAs and commits them to mbarriers.
// Two kernels:
//   - k_predict_tm (D = 64): the producers write the A operand straight into
//     tensor memory (tcgen05.st, one event row per thread), four tiles in
//     production at once (four A slots of 64 columns) and two epilogue groups
//     with an accumulator each (2 x 128 columns): 24 warps, one CTA per SM.
//   - k_predict_tc (D = 128, whose A operand would not leave room for two
//     accumulators in tensor memory): the producers write the A operand into
//     shared memory in the K-major 128-byte-swizzled layout tcgen05.mma
//     reads; two tiles in flight; one epilogue group that issues the next
//     tile's first layer under the current tile's epilogue.
// The hand-offs are mbarriers (full: producers -> MMA; done: first layer ->
// epilogue and producers, whose operand slot is free once the first layer has
// run; stored: epilogue -> second-layer MMA; out: second-layer MMA ->
// epilogue; empty: epilogue -> next first layer into the same accumulator).
// No waiter can fall two phases behind a barrier (each role's next use of a
// buffer waits for the other roles' previous use), so parity waits are
// unambiguous.  Every wait is bounded: on time-out the kernel sets the error
// word and leaves.
//
// While they wait for accumulators, the epilogue warps can also zero a grid
// buffer for the caller (the next call's per-pixel sums): each CTA clears one
// contiguous share, a slice per tile, and on an early exit the rest of it.
//
// b1 and b2 reach the epilogue as a kernel parameter: read through the
// constant cache, they take no slots of the shared-memory pipe.
//
// Requested events come either in pixel-sorted order (records of the
// counting sort: consecutive rows mostly share a pooled row) or by index (an
// explicit K list, or all events in input order).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "check.cuh"
#include "phase.cuh"
#include "veckm_internal.h"

namespace veckm {

namespace {

constexpr int kM = 128;  // events per tile (MMA M)
constexpr int kN = 128;  // hidden units (MMA N)
constexpr int kEpiWarps = 4;
// k_predict_tc: 16 producer warps of 8 rows each (one CTA per SM: the
// operand tiles fill shared memory)
template <int DV>
struct Shape {
  static_assert(DV == 2, "k_predict_tc serves D = 128");
  static constexpr int prod = 16;
  static constexpr int rows = 128 / prod;
  static constexpr int threads = 32 * (4 + prod);
};
constexpr int kMmaWarp = 0;  // epilogue warp 0 also issues the MMAs
constexpr int kTmemCols = 2 * kN;  // two accumulators
// Second layer: N = 16 (the two outputs, padded), K = kN.  Its A operand,
// ReLU(h) as FP16 pairs, takes accumulator columns [0, kN/2); its outputs
// land in columns [kOutCol, kOutCol + 16) of the same accumulator.
constexpr int kN2 = 16;
constexpr int kOutCol = kN / 2;
constexpr int kW2Bytes = kN2 * kN * 2;  // W2 as FP16, K-major, 128-byte swizzled

// First-layer bias and second-layer bias, by value; for the D = 64 head also
// the fixed-point temporal frequencies of channels 2u, 2u+1 (wt[2u], wt[2u+1]
// as one uint4 per unit), read as constant operands of the phase arithmetic.
struct __align__(16) EpiParams {
  float b1[kN];
  float b2[2];
  uint4 wt[32];
};
// Output row codes (event counts are below 2^30): k >= 0 writes the flow of
// row k; -1 writes nothing; k <= -2 writes zeros to row -2 - k (an invalid
// event or index).
__device__ __forceinline__ int invalid_row(int i) { return -2 - i; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
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

// Waits for the phase with the given parity.  try_wait suspends the thread
// in hardware until the phase completes or the hint (ns) runs out, so a
// waiting warp takes no issue slots from the warps doing the work; the loop
// gives up after `limit` SM cycles (the context's wait limit).  Called by
// whole warps; the answer is the same for every lane (false if any lane gave
// up), so that no lane leaves a loop its warp mates stay in.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  bool done;
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000000u)
        : "memory");
    if (ok) {
      done = true;
      break;
    }
    if (clock64() - t0 > limit) {
      done = false;
      break;
    }
  }
  return __all_sync(0xffffffffu, done);
}

// Whether the phase with the given parity has completed (no waiting); the
// same answer for the whole warp (lane 0's).
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// a * b and a - b on two FP32 lanes at once (packed FP32x2, one instruction)
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<const uint64_t *>(&a)), "l"(*reinterpret_cast<const uint64_t *>(&b)));
  return *reinterpret_cast<const float2 *>(&d);
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<const uint64_t *>(&a)), "l"(*reinterpret_cast<const uint64_t *>(&b)));
  return *reinterpret_cast<const float2 *>(&d);
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

// 32 consecutive FP32 accumulator columns of this warp's 32 lanes.
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

// 16 consecutive 32-bit accumulator columns of this warp's 32 lanes (no wait).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}

// ReLU(lo), ReLU(hi) rounded to FP16 and packed (lo in the low half).
__device__ __forceinline__ uint32_t relu_f16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// Loads N consecutive ints of shared memory (16-byte aligned for N >= 4,
// 8-byte aligned for N = 2) in N / 4 vector loads (one for N = 2).
template <int N>
__device__ __forceinline__ void lds_ints(const int *p, int (&o)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const int4 v = reinterpret_cast<const int4 *>(p)[i];
      o[4 * i] = v.x, o[4 * i + 1] = v.y, o[4 * i + 2] = v.z, o[4 * i + 3] = v.w;
    }
  } else {
    static_assert(N == 2, "rows per batch: 2 or a multiple of 4");
    const int2 v = *reinterpret_cast<const int2 *>(p);
    o[0] = v.x, o[1] = v.y;
  }
}

// F16: the operands are FP16 (else BF16), fixed per launch.
template <int DV, bool HALF, bool F16>
__global__ void __launch_bounds__(Shape<DV>::threads, 1)
    k_predict_tc(Events ev, const int64_t *__restrict__ K, int64_t nK,
                 const int2 *__restrict__ rec, const int *__restrict__ rpix,
                 const int *__restrict__ nsorted, Geometry g, Tables tb,
                 const void *__restrict__ pooled_v, const int *__restrict__ ncnt, MLP mlp,
                 float *__restrict__ flow, int *err, float4 *__restrict__ zero_buf,
                 int64_t zero_units, const __grid_constant__ EpiParams ep) {
  constexpr int U = 32 * DV;
  constexpr int IN = 4 * U;  // 2D, the MMA K extent
  constexpr int TILE_BYTES = kM * IN * 2;
  constexpr int kProdWarps = Shape<DV>::prod;
  constexpr int kRowsPerWarp = Shape<DV>::rows;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = smem;                            // 2 x [128 x IN] half, SW128
  uint8_t *sB = smem + 2 * TILE_BYTES;           // [128 x IN] half (W1), SW128
  uint8_t *sW2 = sB + TILE_BYTES;                // [16 x 128] FP16 (W2 padded), SW128
  // row metadata of tile li in slot li & 3: a slot is rewritten only once the
  // tile four back has been read back in full
  float *sInv = reinterpret_cast<float *>(sW2 + kW2Bytes);    // [4][128] 1 valid, 0 not
  int *sK = reinterpret_cast<int *>(sInv + 4 * kM);            // [4][128] output row codes
  // full[2], done[2], empty[2], stored[2], out_done[2]
  uint64_t *bars = reinterpret_cast<uint64_t *>(sK + 4 * kM);
  int *sMeta = reinterpret_cast<int *>(bars + 10);  // per producer warp [2][pixels R | t R]
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sMeta + kProdWarps * 4 * kRowsPerWarp);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int fp16 = F16 ? 1 : 0;
  const long long wl = mlp.wait_cycles;

  {  // W1 and W2 (already in SW128 order)
    const uint4 *src = reinterpret_cast<const uint4 *>(mlp.W1h);
    uint4 *dst = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < TILE_BYTES / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    const uint4 *src2 = reinterpret_cast<const uint4 *>(mlp.W2h);
    uint4 *dst2 = reinterpret_cast<uint4 *>(sW2);
    for (int i = tid; i < kW2Bytes / 16; i += blockDim.x) dst2[i] = __ldg(src2 + i);
  }
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int b) { return bar0 + 8u * b; };
  auto done_bar = [&](int b) { return bar0 + 8u * (2 + b); };
  auto empty_bar = [&](int b) { return bar0 + 8u * (4 + b); };
  auto stored_bar = [&](int b) { return bar0 + 8u * (6 + b); };
  auto out_bar = [&](int b) { return bar0 + 8u * (8 + b); };
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full_bar(b)), "r"(kProdWarps));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done_bar(b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty_bar(b)), "r"(kEpiWarps));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(stored_bar(b)), "r"(kEpiWarps));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(out_bar(b)));
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
  const int ns = rec ? *nsorted : (int)nK;
  const int ntiles_all = (int)((nK + kM - 1) / kM);
  const int nlocal = (int)blockIdx.x < ntiles_all
                         ? (ntiles_all - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                         : 0;
  bool ok = true;

  if (warp >= kEpiWarps) {
    // ------------------------------------------------------------ producers
    // Warp pw fills rows pw*R .. pw*R+R-1 of every tile (R = kRowsPerWarp =
    // 8).  Lane l computes unit u = l + 32 v (channels 2u, 2u+1) of a row and stores its four
    // halves, Re(2u) Re(2u+1) Im(2u) Im(2u+1), as one 8-byte group at K
    // positions 4u..4u+3 (W1's columns are permuted to match on the host).
    const int pw = warp - kEpiWarps;
    uint2 wf[DV][2];  // fixed-point frequencies of this lane's channels
#pragma unroll
    for (int v = 0; v < DV; ++v) {
      wf[v][0] = __ldg(tb.wt + 2 * (lane + 32 * v));
      wf[v][1] = __ldg(tb.wt + 2 * (lane + 32 * v) + 1);
    }
    // Byte offset of that group for row pw*R + j: K-block u / 16 (bits 14+),
    // row group (bits 10+), row j % 8 (bits 7-9), 16-byte chunk (u / 2) % 8
    // XOR j % 8 (bits 4-6), half of the chunk u % 2 (bit 3).  For j % 8 == 0
    // that is lo[v]; for j % 8 == r it is lo[v] ^ (r * 0x90) (r into bits 7-9
    // and XOR-ed into bits 4-6), and adding a 1024-aligned tile base commutes
    // with that XOR.
    uint32_t lo[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) {
      const uint32_t u = lane + 32 * v;
      lo[v] = (u >> 4) * (kM * 128) + (uint32_t)pw * (kRowsPerWarp * 128) + (((u >> 1) & 7) << 4) +
              (u & 1) * 8;
    }
    // Row metadata of tile t for lane j < 16 (row pw*16 + j): the pixel whose
    // pooled vector is read, t - t_ref, 1 for a valid event (0 otherwise; the
    // FP32-grid path later replaces it by 1/n) and the output row (-1: none;
    // invalid_row(i): an invalid event whose flow is written as zeros).  Rows
    // past the end and invalid events read pixel 0: the MMA keeps rows apart
    // and their results are discarded.  Every load here is consumed a tile
    // later, so the warp never waits on it.
    auto meta = [&](int t, int &pix, uint32_t &trel, float &inv, int &outk) {
      const int i = t * kM + pw * kRowsPerWarp + (lane & (kRowsPerWarp - 1));
      pix = 0;
      trel = 0;
      inv = 0.f;
      outk = -1;
      if (i >= ns) return;
      if (rec) {
        const int2 r = __ldg(rec + i);
        pix = __ldg(rpix + i);
        if (!VK_CHECK(pix >= 0 && (int64_t)pix < (int64_t)g.W * g.H)) pix = 0;
        trel = (uint32_t)r.x;
        outk = r.y;
        inv = 1.f;
        return;
      }
      int64_t k = i;
      if (K) {
        k = K[i];
        if (k < 0 || k >= ev.n) {
          if (lane < kRowsPerWarp) atomicOr(err, ERR_INDEX_RANGE);
          outk = invalid_row(i);
          return;
        }
      }
      const int x = ev.x[k], y = ev.y[k];
      const uint32_t tt = ev.t[k];
      trel = tt - ev.t_ref;
      if (x >= 0 && x < g.W && y >= 0 && y < g.H && tt >= ev.t_ref && trel <= ev.t_span) {
        pix = y * g.W + x;
        outk = i;
        inv = 1.f;
      } else {
        outk = invalid_row(i);
      }
    };
    // pixels and t - t_ref of this warp's rows, two tiles: [tile parity]
    // [pixel of rows 0..R-1 | t of rows 0..R-1], so that a batch's pixels (or
    // times) come in one or two vector loads (16-byte aligned: the region
    // starts 16-byte aligned and R is 8)
    int *ms = sMeta + pw * 4 * kRowsPerWarp;
    auto ms_put = [&](int par, int pix, uint32_t trel) {
      if (lane < kRowsPerWarp) {
        ms[par * 2 * kRowsPerWarp + lane] = pix;
        ms[par * 2 * kRowsPerWarp + kRowsPerWarp + lane] = (int)trel;
      }
    };
    const uint32_t sA_a = smem_u32(sA);
    // FP16 grid: uint2 (half2 Re pair, half2 Im pair) per unit, already
    // divided by n; FP32 grid: float4 (re 2u, re 2u+1, im 2u, im 2u+1), the
    // real and imaginary pairs of packed FP32x2 arithmetic (the epilogue
    // divides by n: the first layer is linear)
    using Q = typename std::conditional<HALF, uint2, float4>::type;
    const Q *pooled = reinterpret_cast<const Q *>(pooled_v);
    // rows per batch: the loads of one batch are in flight while the previous
    // batch is computed (one batch of look-ahead, across tile boundaries)
    constexpr int kB = HALF ? 8 / DV : 4 / DV;
    constexpr int NB = kRowsPerWarp / kB;
    static_assert(NB % 2 == 0, "batches alternate between two register sets");
    Q qa[kB][DV], qb[kB][DV];
    auto issue = [&](int par, int j0, Q(&q)[kB][DV]) {
      constexpr int kC = kB < 4 ? kB : 4;  // pixels read per vector load
#pragma unroll
      for (int c = 0; c < kB; c += kC) {
        int pj[kC];
        lds_ints<kC>(ms + par * 2 * kRowsPerWarp + j0 + c, pj);
#pragma unroll
        for (int r = 0; r < kC; ++r) {
#pragma unroll
          for (int v = 0; v < DV; ++v)
            q[c + r][v] = __ldg(pooled + (size_t)pj[r] * U + lane + 32 * v);
        }
      }
    };
    auto compute = [&](int par, int j0, const Q(&q)[kB][DV], uint32_t Abuf) {
      // every t of the batch first; plain stores let the rows interleave
      int tjs[kB];
      lds_ints<kB>(ms + par * 2 * kRowsPerWarp + kRowsPerWarp + j0, tjs);
      uint8_t *Ag = sA + (Abuf - sA_a);
#pragma unroll
      for (int r = 0; r < kB; ++r) {
        const int j = j0 + r;
        const uint32_t tj = (uint32_t)tjs[r];
#pragma unroll
        for (int v = 0; v < DV; ++v) {
          // (c0, s0, c1, s1); the lean form needs a register the FP16 grid's
          // variant has no room for
          const float4 ph = HALF ? time_phase2(tj, wf[v][0], wf[v][1])
                                 : time_phase2_packed(tj, wf[v][0], wf[v][1]);
          uint32_t wre, wim;
          if constexpr (HALF) {
            // P conj(phase) in packed half2: Re = PR c + PI s, Im = PI c - PR s
            const __half2 PR = *reinterpret_cast<const __half2 *>(&q[r][v].x);
            const __half2 PI = *reinterpret_cast<const __half2 *>(&q[r][v].y);
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
            // P conj(phase) on the pairs R = (Re 2u, Re 2u+1), I = (Im 2u,
            // Im 2u+1), C = (c0, c1), S = (s0, s1): Re = R C + I S,
            // Im = I C - R S, each pair in one packed FP32x2 instruction
            const float2 R = make_float2(q[r][v].x, q[r][v].y);
            const float2 I = make_float2(q[r][v].z, q[r][v].w);
            const float2 C = make_float2(ph.x, ph.z), S = make_float2(ph.y, ph.w);
            const float2 er = ffma2(R, C, fmul2(I, S));
            const float2 ei = fsub2(fmul2(I, C), fmul2(R, S));
            wre = pack2(er.x, er.y, fp16);
            wim = pack2(ei.x, ei.y, fp16);
          }
          *reinterpret_cast<uint2 *>(Ag + ((lo[v] ^ (uint32_t)((j & 7) * 0x90)) + (j >> 3) * 1024)) =
              make_uint2(wre, wim);
        }
      }
    };
    int c_outk = -1;
    float c_inv = 0.f;
    int n_cnt = 0;  // FP32 grid: window count of this lane's row in the next tile
    if (nlocal > 0) {
      int pix;
      uint32_t trel;
      meta(blockIdx.x, pix, trel, c_inv, c_outk);
      if (!HALF && c_inv != 0.f) c_inv = 1.0f / (float)__ldg(ncnt + pix);
      ms_put(0, pix, trel);
      __syncwarp();
      issue(0, 0, qa);
    }
    for (int li = 0; li < nlocal && ok; ++li) {
      const int b = li & 1;
      const int tile = (int)blockIdx.x + li * (int)gridDim.x;
      const bool has_next = li + 1 < nlocal;
      int n_pix = 0;
      uint32_t n_trel = 0;
      float n_inv = 0.f;
      int n_outk = -1;
      if (has_next) meta(tile + (int)gridDim.x, n_pix, n_trel, n_inv, n_outk);
      // operand tile b is free once the first layer of tile li - 2 has run
      if (li >= 2 && !mbar_wait(done_bar(b), ((li >> 1) - 1) & 1, wl)) {
        ok = false;
        break;
      }
      const uint32_t Abuf = sA_a + b * TILE_BYTES;
#pragma unroll
      for (int h = 0; h < NB; ++h) {
        if (h + 1 < NB) {
          if (h & 1) issue(b, (h + 1) * kB, qa);
          else issue(b, (h + 1) * kB, qb);
        } else if (has_next) {
          __syncwarp();
          ms_put(b ^ 1, n_pix, n_trel);
          __syncwarp();
          issue(b ^ 1, 0, qa);
        }
        if (h & 1) compute(b, h * kB, qb, Abuf);
        else compute(b, h * kB, qa, Abuf);
        // FP32 grid: the window count of the next tile's row, loaded mid-tile
        // (its pixel has arrived by then) and inverted at the tile's end
        if (!HALF && h == NB / 2 - 1 && has_next && n_inv != 0.f) n_cnt = __ldg(ncnt + n_pix);
      }
      // the epilogue reads these after the first layer's done barrier
      if (lane < kRowsPerWarp) {
        sK[(li & 3) * kM + pw * kRowsPerWarp + lane] = c_outk;
        sInv[(li & 3) * kM + pw * kRowsPerWarp + lane] = c_inv;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      // (the stall injection of the error-path tests withholds this signal)
      if (lane == 0 && !mlp.inject_stall) mbar_arrive(full_bar(b));
      c_outk = n_outk;
      c_inv = (!HALF && n_inv != 0.f) ? 1.0f / (float)n_cnt : n_inv;
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // (warp kMmaWarp issues each tile's MMAs first)
    const int row = warp * 32 + lane;  // TMEM lane = tile row
    const float b20 = ep.b2[0], b21 = ep.b2[1];
    constexpr uint32_t idesc_bf16 = make_idesc(0, kM, kN);
    constexpr uint32_t idesc_fp16 = make_idesc(1, kM, kN);
    const uint32_t idesc = fp16 ? idesc_fp16 : idesc_bf16;
    constexpr uint32_t idesc2 = make_idesc(1, kM, kN2);  // second layer: FP16 x FP16
    const uint32_t sA_a = smem_u32(sA), sB_a = smem_u32(sB), sW2_a = smem_u32(sW2);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    // this CTA's share [z0, z1) of the buffer to zero, one slice per tile
    int64_t z0 = 0, z1 = 0, zstep = 0;
    if (zero_buf) {
      const int64_t per_cta = (zero_units + gridDim.x - 1) / gridDim.x;
      z0 = (int64_t)blockIdx.x * per_cta < zero_units ? (int64_t)blockIdx.x * per_cta : zero_units;
      z1 = z0 + per_cta < zero_units ? z0 + per_cta : zero_units;
      zstep = nlocal > 0 ? (z1 - z0 + nlocal - 1) / nlocal : 0;
    }
    auto zero_slice = [&](int c) {
      const int64_t a = z0 + (int64_t)c * zstep, e = a + zstep < z1 ? a + zstep : z1;
      for (int64_t u = a + row; u < e; u += kEpiWarps * 32) zero_buf[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    };
    int zeroed = 0;  // slices this thread has cleared
    // first layer of tile i into accumulator i & 1 (warp kMmaWarp)
    auto issue_l1 = [&](int i) {
      if (lane == 0) {
        const int bi = i & 1;
        const uint32_t d_tmem = tmem + (uint32_t)(bi * kN);
        const uint32_t a_base = sA_a + bi * TILE_BYTES;
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
                done_bar(bi))
            : "memory");
      }
      __syncwarp();
    };
    int early = -1;  // warp kMmaWarp: the tile whose first layer went out early
    for (int li = 0; li < nlocal && ok; ++li) {
      const int b = li & 1;
      const uint32_t par = (li >> 1) & 1;
      // the issuing warp waits for the producers' tile (full), every epilogue
      // warp for the first layer (done, which follows full): the producers
      // may fill tile li + 2 once tile li's first layer has run, so full can
      // move on before a slow epilogue warp looks at it, done cannot (tile
      // li + 2's first layer waits for every warp's read of tile li)
      if (warp == kMmaWarp && early != li && !mbar_wait(full_bar(b), par, wl)) {
        ok = false;
        break;
      }
      if (warp == kMmaWarp && early != li) {
        // accumulator b is free once all epilogue warps have read tile li - 2
        if (li >= 2 && !mbar_wait(empty_bar(b), par ^ 1, wl)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue_l1(li);
      }
      // done: the first layer's accumulator
      if (!mbar_wait(done_bar(b), par, wl)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float inv = sInv[(li & 3) * kM + row];
      const int k = sK[(li & 3) * kM + row];
      const float2 inv2 = make_float2(inv, inv);
      const uint32_t acc_t = tmem + lane_base + (uint32_t)(b * kN);
      // ReLU(h / n + b1) as FP16 pairs into columns [0, kN/2): chunk c reads
      // columns [32c, 32c + 32) and writes [16c, 16c + 16), which earlier
      // chunks (or this one) have already read
#pragma unroll
      for (int c0 = 0; c0 < kN; c0 += 32) {
        float h[32];
        tmem_ld32(acc_t + c0, h);
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 bb = *reinterpret_cast<const float4 *>(ep.b1 + c0 + j);
          const float2 a01 = ffma2(make_float2(h[j], h[j + 1]), inv2, make_float2(bb.x, bb.y));
          const float2 a23 = ffma2(make_float2(h[j + 2], h[j + 3]), inv2, make_float2(bb.z, bb.w));
          pk[j / 2] = relu_f16x2(a01.x, a01.y);
          pk[j / 2 + 1] = relu_f16x2(a23.x, a23.y);
        }
        tmem_st16(acc_t + c0 / 2, pk);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(stored_bar(b));
      if (warp == kMmaWarp) {
        // the second layer once every epilogue warp has stored its rows
        if (!mbar_wait(stored_bar(b), par, wl)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (lane == 0) {
          const uint32_t a_t = tmem + (uint32_t)(b * kN);
          const uint32_t d_t = a_t + kOutCol;
#pragma unroll
          for (int kk = 0; kk < kN / 16; ++kk) {
            // K-step kk: 8 columns of FP16 pairs; W2's K-block kk / 4, 32-byte step kk % 4
            const uint64_t bd = make_desc_sw128(sW2_a + (kk >> 2) * (kN2 * 128) + (kk & 3) * 32);
            const uint32_t acc = kk > 0 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_t),
                "r"(a_t + (uint32_t)(kk * 8)), "l"(bd), "r"(idesc2), "r"(acc)
                : "memory");
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  out_bar(b))
              : "memory");
        }
        __syncwarp();
        // the next tile's first layer goes to the tensor cores now, under the
        // rest of this tile's epilogue, if that tile is filled (its
        // accumulator, tile li - 1's, has been read back by every warp)
        const int nx = li + 1;
        if (nx < nlocal && mbar_test(full_bar(nx & 1), (nx >> 1) & 1) &&
            (nx < 2 || mbar_test(empty_bar(nx & 1), ((nx >> 1) - 1) & 1))) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          issue_l1(nx);
          early = nx;
        }
      }
      if (!mbar_wait(out_bar(b), par, wl)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t r0, r1;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                   : "=r"(r0), "=r"(r1)
                   : "r"(acc_t + kOutCol));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(empty_bar(b));
      if (k >= 0) {
        *reinterpret_cast<float2 *>(flow + 2 * (size_t)k) =
            make_float2(__uint_as_float(r0) + b20, __uint_as_float(r1) + b21);
      } else if (k <= -2) {
        *reinterpret_cast<float2 *>(flow + 2 * (size_t)(-2 - k)) = make_float2(0.f, 0.f);
      }
      if (zero_buf) zero_slice(zeroed++);
    }
    // the share is cleared in full even when a wait gave up
    if (zero_buf)
      while (zeroed < nlocal) zero_slice(zeroed++);
  }
  if (!ok && lane == 0) atomicOr(err, ERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      // let MMAs that may still be in flight land before their TMEM is freed
      for (int b = 0; b < 2; ++b) {
        mbar_wait(done_bar(b), 0, wl), mbar_wait(done_bar(b), 1, wl);
        mbar_wait(out_bar(b), 0, wl), mbar_wait(out_bar(b), 1, wl);
      }
    }
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

template <int DV, bool HALF, bool F16>
int predict_tc_impl(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                    const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                    const void *pooled, const int *ncnt, const MLP &mlp, float *flow, int *err,
                    cudaStream_t s, float4 *zero_buf, int64_t zero_units, bool *zeroed) {
  if (zeroed) *zeroed = false;
  if (nK == 0) return 0;
  constexpr int IN = 128 * DV;
  const size_t sm = (size_t)3 * kM * IN * 2 + kW2Bytes + sizeof(float) * (4 * kM) +
                    sizeof(int) * 4 * kM + 8 * 10 + sizeof(int2) * 2 * kM +
                    16 + 1024;  // + SW128 alignment slack
  auto kern = k_predict_tc<DV, HALF, F16>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
          cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return -1;
  constexpr int kThreads = Shape<DV>::threads;
  const int per_sm = std::min(blocks_per_sm((const void *)kern, kThreads, sm), 512 / kTmemCols);
  const int64_t tiles = (nK + kM - 1) / kM;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * per_sm);
  // zero the buffer only when every CTA has tiles enough to spread its share
  // over (at most kZeroPerTile float4, 128 KB, per tile)
  constexpr int64_t kZeroPerTile = 8192;
  const int64_t min_local = tiles / grid;
  const bool zero = zero_buf && zero_units > 0 &&
                    (zero_units + grid - 1) / grid <= min_local * kZeroPerTile;
  EpiParams ep;
  std::copy(mlp.hb1, mlp.hb1 + kN, ep.b1);
  ep.b2[0] = mlp.hb2[0];
  ep.b2[1] = mlp.hb2[1];
  kern<<<grid, kThreads, sm, s>>>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow,
                                  err, zero ? zero_buf : nullptr, zero ? zero_units : 0, ep);
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  if (zeroed) *zeroed = zero;
  return 1;
}

// ---------------------------------------------------------------------------
// D = 64: the first layer's A operand written straight into tensor memory.
//
// One CTA per SM of 24 warps: 16 producer warps in four groups of 4, one
// event row per thread, and 8 epilogue warps in two groups of 4.  A producer
// thread forms its row's 128 K-values (P[p] conj(exp(i t T/dt)) in the
// (Re 2u, Re 2u+1, Im 2u, Im 2u+1) order of W1's permuted columns) in chunks
// of 4 units and writes them as FP16 (or BF16) pairs into the tile's A slot
// of tensor memory (tcgen05.st, the warp's 32 lanes = its 32 rows).  Tensor
// memory: four A slots of 64 columns (tile li in slot li mod 4, filled by
// producer group li mod 4) and two accumulators of 128 columns (tile li in
// accumulator li mod 2, read back by epilogue group li mod 2, whose first
// warp issues the tile's MMAs).  The first layer reads A from tensor memory
// and W1 from shared memory; the epilogue and the second layer are as in
// k_predict_tc.  No operand tile takes shared memory, so four tiles can be in
// production at once and a producer group waits only for its own previous
// tile's first layer.
constexpr int kTmEpiGroups = 2;
constexpr int kTmACols = 64;     // A slot: 128 K values as FP16 pairs
constexpr int kTmAccBase = 256;  // accumulators after (at most four) A slots
constexpr int kTmCols = 512;
// P producer groups of 4 warps
template <int P>
struct TmShape {
  static_assert(P >= 2 && P <= 4, "A slots: P x 64 columns before the accumulators");
  static constexpr int warps = 4;  // per producer group
  static constexpr int threads = 32 * (warps * P + 4 * kTmEpiGroups);
  // Row-metadata slots: tile li in slot li mod (P + 2).  The slot of tile li
  // is rewritten at the end of tile li + P + 2's production, which starts
  // once tile li + 2's first layer has run; that was issued once every warp
  // of li's epilogue group (tile li + 2 is in the same group) had read tile
  // li back, metadata included.
  static constexpr int meta = P + 2;
  // Tile li signals full[li mod ring] (producers -> issuer) and
  // done[li mod ring] (first layer -> its epilogue group and the producer
  // group that fills the same A slot next, tile li + P).  ring = lcm(P, 2):
  // the tiles of one barrier, li and li + ring, then share both the producer
  // group and the epilogue group, so every waiter waits for each phase in
  // turn, and the phase of li + ring cannot complete before every waiter of
  // li's phase has passed it (li + ring's first layer waits for li's group
  // to have read tile li + ring - 2 back, and its producers for li + ring - P's
  // first layer).  With one barrier per A slot and P odd, consecutive phases
  // would alternate between the epilogue groups, and a group waiting for
  // every other phase could take the parity of a phase not yet completed
  // for its own.
  static constexpr int ring = P % 2 == 0 ? P : 2 * P;
  static constexpr int bars = 2 * ring + 8;
};

// The shape launched: four producer groups.  (On the 640 x 480, 2 M event
// slice, three groups of 8 warps that fill half a row each per thread ran
// 151 us and two such groups 189 us, against 149 us for this one.)
constexpr int kTmP = 4;

template <bool HALF, bool F16, int P>
__global__ void __launch_bounds__(TmShape<P>::threads, 1)
    k_predict_tm(Events ev, const int64_t *__restrict__ K, int64_t nK,
                 const int2 *__restrict__ rec, const int *__restrict__ rpix,
                 const int *__restrict__ nsorted, Geometry g, Tables tb,
                 const void *__restrict__ pooled_v, const int *__restrict__ ncnt, MLP mlp,
                 float *__restrict__ flow, int *err, float4 *__restrict__ zero_buf,
                 int64_t zero_units, const __grid_constant__ EpiParams ep) {
  constexpr int U = 32;        // units per pixel (D = 64)
  constexpr int IN = 4 * U;    // 2D, the MMA K extent
  constexpr int W1_BYTES = kN * IN * 2;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sB = smem;                       // [128 x IN] half (W1), SW128
  uint8_t *sW2 = sB + W1_BYTES;             // [16 x 128] FP16 (W2 padded), SW128
  constexpr int kMeta = TmShape<P>::meta;
  float *sInv = reinterpret_cast<float *>(sW2 + kW2Bytes);  // [kMeta][128] 1/n (or 1), 0 invalid
  int *sK = reinterpret_cast<int *>(sInv + kMeta * kM);      // [kMeta][128] output row codes
  // full[ring], done[ring], stored[2], out[2], empty[2], drain[2]
  constexpr int kRing = TmShape<P>::ring, kB = 2 * kRing;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sK + kMeta * kM);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + TmShape<P>::bars);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int fp16 = F16 ? 1 : 0;
  const long long wl = mlp.wait_cycles;
  {  // W1 and W2 (already in SW128 order)
    const uint4 *src = reinterpret_cast<const uint4 *>(mlp.W1h);
    uint4 *dst = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < W1_BYTES / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    const uint4 *src2 = reinterpret_cast<const uint4 *>(mlp.W2h);
    uint4 *dst2 = reinterpret_cast<uint4 *>(sW2);
    for (int i = tid; i < kW2Bytes / 16; i += blockDim.x) dst2[i] = __ldg(src2 + i);
  }
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int li) { return bar0 + 8u * (li % kRing); };           // of tile li
  auto done_bar = [&](int li) { return bar0 + 8u * (kRing + li % kRing); };  // of tile li
  auto stored_bar = [&](int g) { return bar0 + 8u * (kB + g); };
  auto out_bar = [&](int g) { return bar0 + 8u * (kB + 2 + g); };
  auto empty_bar = [&](int g) { return bar0 + 8u * (kB + 4 + g); };
  auto drain_bar = [&](int g) { return bar0 + 8u * (kB + 6 + g); };
  auto ring_par = [&](int li) { return (uint32_t)(li / kRing) & 1u; };  // tile li's phase parity
  if (tid == 0) {
    for (int d = 0; d < kRing; ++d) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full_bar(d)),
                   "r"(TmShape<P>::warps));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done_bar(d)));
    }
    for (int g2 = 0; g2 < 2; ++g2) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(stored_bar(g2)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(out_bar(g2)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(empty_bar(g2)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(drain_bar(g2)));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTmCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int ns = rec ? *nsorted : (int)nK;
  const int ntiles_all = (int)((nK + kM - 1) / kM);
  const int nlocal = (int)blockIdx.x < ntiles_all
                         ? (ntiles_all - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                         : 0;
  bool ok = true;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;  // this warp's TMEM lanes
  const int row = (warp & 3) * 32 + lane;                        // = tile row

  if (warp >= 4 * kTmEpiGroups) {
    // ------------------------------------------------------------ producers
    const int pg = (warp - 4 * kTmEpiGroups) / TmShape<P>::warps;  // tiles li = pg mod P, A slot pg
    using Q = typename std::conditional<HALF, uint2, float4>::type;
    const Q *pooled = reinterpret_cast<const Q *>(pooled_v);
    const uint32_t a_t = tmem + lane_base + (uint32_t)(pg * kTmACols);
    // Row metadata of local tile li: the pixel whose pooled vector is read,
    // t - t_ref, 1 for a valid event (0 otherwise) and the output row code.
    // Rows past the end and invalid events read pixel 0: the MMA keeps rows
    // apart and their results are discarded.
    auto meta = [&](int li, int &pix, uint32_t &trel, float &inv, int &outk) {
      const int i = ((int)blockIdx.x + li * (int)gridDim.x) * kM + row;
      pix = 0;
      trel = 0;
      inv = 0.f;
      outk = -1;
      if (i >= ns) return;
      if (rec) {
        const int2 r = __ldg(rec + i);
        pix = __ldg(rpix + i);
        if (!VK_CHECK(pix >= 0 && (int64_t)pix < (int64_t)g.W * g.H)) pix = 0;
        trel = (uint32_t)r.x;
        outk = r.y;
        inv = 1.f;
        return;
      }
      int64_t k = i;
      if (K) {
        k = K[i];
        if (k < 0 || k >= ev.n) {
          atomicOr(err, ERR_INDEX_RANGE);
          outk = invalid_row(i);
          return;
        }
      }
      const int x = ev.x[k], y = ev.y[k];
      const uint32_t tt = ev.t[k];
      trel = tt - ev.t_ref;
      if (x >= 0 && x < g.W && y >= 0 && y < g.H && tt >= ev.t_ref && trel <= ev.t_span) {
        pix = y * g.W + x;
        outk = i;
        inv = 1.f;
      } else {
        outk = invalid_row(i);
      }
    };
    // The row's units stream through a ring of R registers: unit u is loaded
    // R - 1 units ahead of its use, the last ones from the next tile's row
    // (32 is a multiple of R, so a tile's unit v sits in ring slot v mod R
    // whichever tile it belongs to).
    constexpr int R = HALF ? 16 : 8;
    static_assert(U % R == 0, "the ring wraps at a row's end");
    Q ring[R];
    int c_pix = 0, c_outk = -1;
    uint32_t c_trel = 0;
    float c_inv = 0.f;
    if (pg < nlocal) {
      meta(pg, c_pix, c_trel, c_inv, c_outk);
      const Q *prow = pooled + (size_t)c_pix * U;
#pragma unroll
      for (int v = 0; v < R - 1; ++v) ring[v] = __ldg(prow + v);
    }
    int c_cnt = (!HALF && pg < nlocal && c_inv != 0.f) ? __ldg(ncnt + c_pix) : 0;
    for (int li = pg; li < nlocal && ok; li += P) {
      const bool has_next = li + P < nlocal;
      int n_pix = 0, n_outk = -1;
      uint32_t n_trel = 0;
      float n_inv = 0.f;
      if (has_next) meta(li + P, n_pix, n_trel, n_inv, n_outk);
      // the A slot is free once this group's previous tile's first layer has run
      if (li >= P && !mbar_wait(done_bar(li - P), ring_par(li - P), wl)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const Q *prow = pooled + (size_t)c_pix * U;
      const Q *nrow = pooled + (size_t)n_pix * U;
      int n_cnt = 0;
      uint32_t pk[8];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        // the load R - 1 units ahead
        const int ua = u + R - 1;
        if (ua < U) ring[ua % R] = __ldg(prow + ua);
        else if (has_next) ring[ua % R] = __ldg(nrow + (ua - U));
        if (!HALF && u == U / 2 && has_next && n_inv != 0.f) n_cnt = __ldg(ncnt + n_pix);
        // the next row's pooled values into L2 a tile ahead of their loads
        // (its pixel has arrived by now)
        if (u == 8 && has_next) {
#pragma unroll
          for (int l = 0; l < (int)(U * sizeof(Q)) / 128; ++l)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(nrow) + 128 * l));
        }
        const Q q = ring[u % R];
        const uint4 w = ep.wt[u];
        const float4 ph = time_phase2_packed(c_trel, make_uint2(w.x, w.y), make_uint2(w.z, w.w));
        uint32_t wre, wim;
        if constexpr (HALF) {
          const __half2 PR = *reinterpret_cast<const __half2 *>(&q.x);
          const __half2 PI = *reinterpret_cast<const __half2 *>(&q.y);
          const __half2 C = __floats2half2_rn(ph.x, ph.z);
          const __half2 Sn = __floats2half2_rn(ph.y, ph.w);
          const __half2 ER = __hfma2(PR, C, __hmul2(PI, Sn));
          const __half2 EI = __hfma2(PI, C, __hneg2(__hmul2(PR, Sn)));
          if (fp16) {
            wre = *reinterpret_cast<const uint32_t *>(&ER);
            wim = *reinterpret_cast<const uint32_t *>(&EI);
          } else {
            const float2 fr = __half22float2(ER), fi = __half22float2(EI);
            wre = pack2(fr.x, fr.y, 0);
            wim = pack2(fi.x, fi.y, 0);
          }
        } else {
          const float2 Rr = make_float2(q.x, q.y);
          const float2 I = make_float2(q.z, q.w);
          const float2 C = make_float2(ph.x, ph.z), Sn = make_float2(ph.y, ph.w);
          const float2 er = ffma2(Rr, C, fmul2(I, Sn));
          const float2 ei = fsub2(fmul2(I, C), fmul2(Rr, Sn));
          wre = pack2(er.x, er.y, fp16);
          wim = pack2(ei.x, ei.y, fp16);
        }
        pk[2 * (u & 3)] = wre;
        pk[2 * (u & 3) + 1] = wim;
        if ((u & 3) == 3) {
          // unit u - 3 + j in columns 2(u - 3 + j) (Re pair) and 2(u - 3 + j) + 1
          // (Im pair): K = 4u' .. 4u'+3 for unit u'
          asm volatile(
              "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
                  a_t + (uint32_t)(2 * (u - 3))),
              "r"(pk[0]), "r"(pk[1]), "r"(pk[2]), "r"(pk[3]), "r"(pk[4]), "r"(pk[5]), "r"(pk[6]),
              "r"(pk[7])
              : "memory");
        }
      }
      const int msl = li % kMeta;
      sK[msl * kM + row] = c_outk;
      sInv[msl * kM + row] = (!HALF && c_inv != 0.f) ? 1.0f / (float)c_cnt : c_inv;
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      // (the stall injection of the error-path tests withholds this signal)
      if (lane == 0 && !mlp.inject_stall) mbar_arrive(full_bar(li));
      c_pix = n_pix;
      c_trel = n_trel;
      c_inv = n_inv;
      c_outk = n_outk;
      c_cnt = n_cnt;
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int grp = warp >> 2;        // tiles li = grp mod 2, accumulator grp
    const bool issuer = (warp & 3) == 0;
    const float b20 = ep.b2[0], b21 = ep.b2[1];
    constexpr uint32_t idesc_bf16 = make_idesc(0, kM, kN);
    constexpr uint32_t idesc_fp16 = make_idesc(1, kM, kN);
    const uint32_t idesc = fp16 ? idesc_fp16 : idesc_bf16;
    constexpr uint32_t idesc2 = make_idesc(1, kM, kN2);
    const uint32_t sB_a = smem_u32(sB), sW2_a = smem_u32(sW2);
    const uint32_t acc_col = (uint32_t)(kTmAccBase + grp * kN);
    // this CTA's share [z0, z1) of the buffer to zero, one slice per tile
    int64_t z0 = 0, z1 = 0, zstep = 0;
    if (zero_buf) {
      const int64_t per_cta = (zero_units + gridDim.x - 1) / gridDim.x;
      z0 = (int64_t)blockIdx.x * per_cta < zero_units ? (int64_t)blockIdx.x * per_cta : zero_units;
      z1 = z0 + per_cta < zero_units ? z0 + per_cta : zero_units;
      zstep = nlocal > 0 ? (z1 - z0 + nlocal - 1) / nlocal : 0;
    }
    auto zero_slice = [&](int c) {
      const int64_t a = z0 + (int64_t)c * zstep, e = a + zstep < z1 ? a + zstep : z1;
      for (int64_t u = a + row; u < e; u += 4 * 32) zero_buf[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    };
    int li = grp;
    for (; li < nlocal && ok; li += kTmEpiGroups) {
      const int sa = li % P;  // A slot
      const uint32_t pg2 = (li >> 1) & 1; // this group's barriers' parity
      if (issuer) {
        // the tile filled, and this group's accumulator read back (tile li - 2)
        if (!mbar_wait(full_bar(li), ring_par(li), wl) ||
            (li >= kTmEpiGroups && !mbar_wait(empty_bar(grp), pg2 ^ 1, wl))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (lane == 0) {
          const uint32_t a_tm = tmem + (uint32_t)(sa * kTmACols);
#pragma unroll
          for (int kk = 0; kk < IN / 16; ++kk) {
            const uint32_t koff = (kk >> 2) * (kM * 128) + (kk & 3) * 32;
            const uint64_t bd = make_desc_sw128(sB_a + koff);
            const uint32_t acc = kk > 0 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem +
                                                                                    acc_col),
                "r"(a_tm + (uint32_t)(kk * 8)), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  done_bar(li))
              : "memory");
        }
        __syncwarp();
      }
      // done: the first layer's accumulator (and the A slot is free)
      if (!mbar_wait(done_bar(li), ring_par(li), wl)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int msl = li % kMeta;
      const float inv = sInv[msl * kM + row];
      const int k = sK[msl * kM + row];
      const float2 inv2 = make_float2(inv, inv);
      const uint32_t acc_t = tmem + lane_base + acc_col;
      // ReLU(h / n + b1) as FP16 pairs into columns [0, kN/2): chunk c0
      // reads [c0, c0 + 32) and writes [c0/2, c0/2 + 16), already read
#pragma unroll
      for (int c0 = 0; c0 < kN; c0 += 32) {
        float h[32];
        uint32_t pk[16];
        tmem_ld32(acc_t + c0, h);
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 bb = *reinterpret_cast<const float4 *>(ep.b1 + c0 + j);
          const float2 a01 = ffma2(make_float2(h[j], h[j + 1]), inv2, make_float2(bb.x, bb.y));
          const float2 a23 = ffma2(make_float2(h[j + 2], h[j + 3]), inv2, make_float2(bb.z, bb.w));
          pk[j / 2] = relu_f16x2(a01.x, a01.y);
          pk[j / 2 + 1] = relu_f16x2(a23.x, a23.y);
        }
        tmem_st16(acc_t + c0 / 2, pk);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(stored_bar(grp));
      if (issuer) {
        if (!mbar_wait(stored_bar(grp), pg2, wl)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (lane == 0) {
          const uint32_t a2 = tmem + acc_col;
#pragma unroll
          for (int kk = 0; kk < kN / 16; ++kk) {
            const uint64_t bd = make_desc_sw128(sW2_a + (kk >> 2) * (kN2 * 128) + (kk & 3) * 32);
            const uint32_t acc = kk > 0 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(a2 +
                                                                                    kOutCol),
                "r"(a2 + (uint32_t)(kk * 8)), "l"(bd), "r"(idesc2), "r"(acc)
                : "memory");
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  out_bar(grp))
              : "memory");
        }
        __syncwarp();
      }
      if (!mbar_wait(out_bar(grp), pg2, wl)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t r0, r1;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                   : "=r"(r0), "=r"(r1)
                   : "r"(acc_t + kOutCol));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(empty_bar(grp));
      // (row codes come from this launch's metadata: k < nK, -2 - k < nK;
      // a code outside them is recorded and not written)
      if (k >= 0 && k < nK) {
        *reinterpret_cast<float2 *>(flow + 2 * (size_t)k) =
            make_float2(__uint_as_float(r0) + b20, __uint_as_float(r1) + b21);
      } else if (k <= -2 && -2 - (int64_t)k < nK) {
        *reinterpret_cast<float2 *>(flow + 2 * (size_t)(-2 - k)) = make_float2(0.f, 0.f);
      } else if (k != -1) {
        atomicOr(err, ERR_INDEX_RANGE);
      }
      if (zero_buf) zero_slice(li);
    }
    if (zero_buf)
      for (; li < nlocal; li += kTmEpiGroups) zero_slice(li);
    if (issuer) {
      // every MMA this warp issued has landed before the tensor memory is freed
      if (lane == 0)
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                drain_bar(grp))
            : "memory");
      __syncwarp();
      if (!mbar_wait(drain_bar(grp), 0, wl)) ok = false;
    }
  }
  if (!ok && lane == 0) atomicOr(err, ERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmCols));
  }
}

template <bool HALF, bool F16>
int predict_tm_impl(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                    const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                    const void *pooled, const int *ncnt, const MLP &mlp, float *flow, int *err,
                    cudaStream_t s, float4 *zero_buf, int64_t zero_units, bool *zeroed) {
  if (zeroed) *zeroed = false;
  if (nK == 0) return 0;
  constexpr int IN = 128;
  constexpr int P = kTmP;
  const size_t sm = (size_t)kN * IN * 2 + kW2Bytes +
                    (sizeof(float) + sizeof(int)) * TmShape<P>::meta * kM +
                    8 * TmShape<P>::bars + 16 + 1024;  // + SW128 alignment slack
  auto kern = k_predict_tm<HALF, F16, P>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
      cudaSuccess)
    return -1;
  const int64_t tiles = (nK + kM - 1) / kM;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms());
  constexpr int64_t kZeroPerTile = 8192;
  const int64_t min_local = tiles / grid;
  const bool zero = zero_buf && zero_units > 0 &&
                    (zero_units + grid - 1) / grid <= min_local * kZeroPerTile;
  EpiParams ep;
  std::copy(mlp.hb1, mlp.hb1 + kN, ep.b1);
  ep.b2[0] = mlp.hb2[0];
  ep.b2[1] = mlp.hb2[1];
  if (!mlp.hwt) return -1;
  for (int u = 0; u < 32; ++u)
    ep.wt[u] = make_uint4(mlp.hwt[2 * u].x, mlp.hwt[2 * u].y, mlp.hwt[2 * u + 1].x,
                          mlp.hwt[2 * u + 1].y);
  kern<<<grid, TmShape<P>::threads, sm, s>>>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow,
                                    err, zero ? zero_buf : nullptr, zero ? zero_units : 0, ep);
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  if (zeroed) *zeroed = zero;
  return 1;
}

}  // namespace

int launch_predict_tc(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                      const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                      const void *pooled, const int *ncnt, const MLP &mlp, float *flow,
                      int *err, cudaStream_t s, const Tune &tn, float4 *zero_buf,
                      int64_t zero_units, bool *zeroed) {
  const bool h = mlp.pooled_half != 0, f16 = mlp.half_kind != 0;
#define VECKM_TM(H_, F_)                                                                    \
  predict_tm_impl<H_, F_>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow, err, s, \
                          zero_buf, zero_units, zeroed)
#define VECKM_TC(H_, F_)                                                                    \
  predict_tc_impl<2, H_, F_>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow, err, \
                             s, zero_buf, zero_units, zeroed)
  if (zeroed) *zeroed = false;
  switch (g.U / 32) {
    case 1:
      if (h) return f16 ? VECKM_TM(true, true) : VECKM_TM(true, false);
      return f16 ? VECKM_TM(false, true) : VECKM_TM(false, false);
    case 2:
      if (h) return f16 ? VECKM_TC(true, true) : VECKM_TC(true, false);
      return f16 ? VECKM_TC(false, true) : VECKM_TC(false, false);
    default:
      return -1;  // 2D > 256 does not fit the operand tiles in shared memory
  }
#undef VECKM_TC
#undef VECKM_TM
}

VK_CHECK_READER(check_read_head)

}  // namespace veckm
