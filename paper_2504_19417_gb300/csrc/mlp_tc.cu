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
// The producers write the A operand straight into tensor memory (tcgen05.st,
// one event row per thread, 32 units of it): for D = 64 four tiles in
// production at once (four A slots of 64 columns, four producer groups of 4
// warps), for D = 128 two (A slots of 128 columns, two groups of 8 warps that
// each fill half a row per thread); two epilogue groups with an accumulator
// each (2 x 128 columns): 24 warps, one CTA per SM (k_predict_tm).
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

#include "chain.cuh"
#include "check.cuh"
#include "phase.cuh"
#include "veckm_internal.h"

namespace veckm {

namespace {

constexpr int kM = 128;  // events per tile (MMA M)
constexpr int kN = 128;  // hidden units (MMA N)
// Second layer: N = 16 (the two outputs, padded), K = kN.  Its A operand,
// ReLU(h) as FP16 pairs, takes accumulator columns [0, kN/2); its outputs
// land in columns [kOutCol, kOutCol + 16) of the same accumulator.
constexpr int kN2 = 16;
constexpr int kOutCol = kN / 2;
constexpr int kW2Bytes = kN2 * kN * 2;  // W2 as FP16, K-major, 128-byte swizzled

// First-layer bias and second-layer bias, by value; for the tensor-memory
// head also the fixed-point temporal frequencies of channels 2u, 2u+1
// (wt[2u], wt[2u+1] as one uint4 per unit), read as constant operands of the
// phase arithmetic.
struct __align__(16) EpiParams {
  float b1[kN];
  float b2[2];
  uint4 wt[64];
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


// F16: the operands are FP16 (else BF16), fixed per launch.
// ---------------------------------------------------------------------------
// The first layer's A operand written straight into tensor memory.
//
// One CTA per SM of 24 warps: 16 producer warps and 8 epilogue warps in two
// groups of 4.  A producer thread owns one event row of a tile (TMEM lane =
// row: the warp's 32 lanes are its 32 rows) and 32 of its units: for D = 64
// four producer groups of 4 warps, each thread a whole row; for D = 128 two
// groups of 8 warps, each thread half a row.  It forms the K-values
// P[p] conj(exp(i t T/dt)) of its units in the (Re 2u, Re 2u+1, Im 2u,
// Im 2u+1) order of W1's permuted columns, 4 units at a time, and writes them
// as FP16 (or BF16) pairs into the tile's A slot of tensor memory
// (tcgen05.st).  Tensor memory: P A slots of 2D/2 columns (tile li in slot
// li mod P, filled by producer group li mod P) in columns 0..255 and two
// accumulators of 128 columns (tile li in accumulator li mod 2, read back by
// epilogue group li mod 2, whose first warp issues the tile's MMAs).  The
// first layer reads A from tensor memory and W1 from shared memory; the
// epilogue and the second layer are as described at the top of this file.
// No operand tile takes shared memory, and a producer group waits only for
// its own previous tile's first layer.
constexpr int kTmEpiGroups = 2;
constexpr int kTmAccBase = 256;  // accumulators after the A slots
constexpr int kTmCols = 512;
// P producer groups of 4 S warps; each thread fills 32 units of its row (a
// row of D/2 = 32 S units)
template <int P, int S = 1>
struct TmShape {
  static_assert(P >= 2 && P * 64 * S <= kTmAccBase, "A slots: P x 64 S columns before the accumulators");
  static constexpr int warps = 4 * S;  // per producer group
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

// The shapes launched: D = 64 (DV = 1) four producer groups of 4 warps,
// D = 128 (DV = 2) two of 8.  (On the 640 x 480, 2 M event slice, D = 64,
// three groups of 8 warps that fill half a row each per thread ran 151 us and
// two such groups 189 us, against 149 us for four groups of 4.)
template <int DV>
constexpr int tm_groups() { return DV == 1 ? 4 : 2; }

template <bool HALF, bool F16, int DV, int P = tm_groups<DV>(), int S = DV>
__global__ void __launch_bounds__(TmShape<P, S>::threads, 1)
    k_predict_tm(Events ev, const int64_t *__restrict__ K, int64_t nK,
                 const int2 *__restrict__ rec, const int *__restrict__ rpix,
                 const int *__restrict__ nsorted, Geometry g, Tables tb,
                 const void *__restrict__ pooled_v, const int *__restrict__ ncnt, MLP mlp,
                 float *__restrict__ flow, int *err, float4 *__restrict__ zero_buf,
                 int64_t zero_units, const __grid_constant__ EpiParams ep) {
  constexpr int U = 32 * DV;   // units per pixel
  constexpr int IN = 4 * U;    // 2D, the MMA K extent
  constexpr int ACOLS = IN / 2;  // A slot: IN K values as FP16 pairs
  constexpr int W1_BYTES = kN * IN * 2;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sB = smem;                       // [128 x IN] half (W1), SW128
  uint8_t *sW2 = sB + W1_BYTES;             // [16 x 128] FP16 (W2 padded), SW128
  constexpr int kMeta = TmShape<P, S>::meta;
  float *sInv = reinterpret_cast<float *>(sW2 + kW2Bytes);  // [kMeta][128] 1/n (or 1), 0 invalid
  int *sK = reinterpret_cast<int *>(sInv + kMeta * kM);      // [kMeta][128] output row codes
  // full[ring], done[ring], stored[2], out[2], empty[2], drain[2]
  constexpr int kRing = TmShape<P, S>::ring, kB = 2 * kRing;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sK + kMeta * kM);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + TmShape<P, S>::bars);

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
                   "r"(TmShape<P, S>::warps));
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
  // the prologue above reads only the weights; the step's grids, records and
  // outputs from here on
  chain_wait();
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
    const int pw = warp - 4 * kTmEpiGroups;
    const int pg = pw / TmShape<P, S>::warps;  // tiles li = pg mod P, A slot pg
    // this thread's units [ub, ub + UT) of its row
    constexpr int UT = U / S;
    const int ub = S == 1 ? 0 : ((pw % TmShape<P, S>::warps) >> 2) * UT;
    using Q = typename std::conditional<HALF, uint2, float4>::type;
    const Q *pooled = reinterpret_cast<const Q *>(pooled_v);
    const uint32_t a_t = tmem + lane_base + (uint32_t)(pg * ACOLS + 2 * ub);
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
    // The thread's units stream through a ring of R registers: unit u is
    // loaded R - 1 units ahead of its use, the last ones from the next tile's
    // row (UT is a multiple of R, so a tile's unit v sits in ring slot v mod R
    // whichever tile it belongs to).
    constexpr int R = HALF ? 16 : 8;
    static_assert(UT % R == 0, "the ring wraps at a row's end");
    Q ring[R];
    int c_pix = 0, c_outk = -1;
    uint32_t c_trel = 0;
    float c_inv = 0.f;
    if (pg < nlocal) {
      meta(pg, c_pix, c_trel, c_inv, c_outk);
      const Q *prow = pooled + (size_t)c_pix * U + ub;
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
      const Q *prow = pooled + (size_t)c_pix * U + ub;
      const Q *nrow = pooled + (size_t)n_pix * U + ub;
      int n_cnt = 0;
      uint32_t pk[8];
#pragma unroll
      for (int u = 0; u < UT; ++u) {
        // the load R - 1 units ahead
        const int ua = u + R - 1;
        if (ua < UT) ring[ua % R] = __ldg(prow + ua);
        else if (has_next) ring[ua % R] = __ldg(nrow + (ua - UT));
        if (!HALF && u == UT / 2 && has_next && n_inv != 0.f) n_cnt = __ldg(ncnt + n_pix);
        // this thread's part of the next row's pooled values into L2 a tile
        // ahead of their loads (its pixel has arrived by now)
        if (u == 8 && has_next) {
#pragma unroll
          for (int l = 0; l < (int)(UT * sizeof(Q)) / 128; ++l)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(nrow) + 128 * l));
        }
        const Q q = ring[u % R];
        const uint4 w = ep.wt[ub + u];
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
      if (ub == 0) {
        const int msl = li % kMeta;
        sK[msl * kM + row] = c_outk;
        sInv[msl * kM + row] = (!HALF && c_inv != 0.f) ? 1.0f / (float)c_cnt : c_inv;
      }
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
          const uint32_t a_tm = tmem + (uint32_t)(sa * ACOLS);
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

template <int DV, bool HALF, bool F16>
int predict_tm_impl(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                    const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                    const void *pooled, const int *ncnt, const MLP &mlp, float *flow, int *err,
                    cudaStream_t s, float4 *zero_buf, int64_t zero_units, bool *zeroed,
                    bool chain) {
  if (zeroed) *zeroed = false;
  if (nK == 0) return 0;
  constexpr int IN = 128 * DV;
  constexpr int P = tm_groups<DV>(), S = DV;
  const size_t sm = (size_t)kN * IN * 2 + kW2Bytes +
                    (sizeof(float) + sizeof(int)) * TmShape<P, S>::meta * kM +
                    8 * TmShape<P, S>::bars + 16 + 1024;  // + SW128 alignment slack
  auto kern = k_predict_tm<HALF, F16, DV>;
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
  for (int u = 0; u < 32 * DV; ++u)
    ep.wt[u] = make_uint4(mlp.hwt[2 * u].x, mlp.hwt[2 * u].y, mlp.hwt[2 * u + 1].x,
                          mlp.hwt[2 * u + 1].y);
  if (launch_kernel(kern, dim3(grid), dim3(TmShape<P, S>::threads), sm, s, chain, ev, K, nK, rec,
                    rpix, nsorted, g, tb, pooled, ncnt, mlp, flow, err,
                    zero ? zero_buf : nullptr, zero ? zero_units : 0, ep) != cudaSuccess)
    return -1;
  if (zeroed) *zeroed = zero;
  return 1;
}

}  // namespace

int launch_predict_tc(const Events &ev, const int64_t *K, int64_t nK, const int2 *rec,
                      const int *rpix, const int *nsorted, const Geometry &g, const Tables &tb,
                      const void *pooled, const int *ncnt, const MLP &mlp, float *flow,
                      int *err, cudaStream_t s, const Tune &tn, float4 *zero_buf,
                      int64_t zero_units, bool *zeroed, bool chain) {
  (void)tn;
  const bool h = mlp.pooled_half != 0, f16 = mlp.half_kind != 0;
#define VECKM_TM(DV_, H_, F_)                                                                \
  predict_tm_impl<DV_, H_, F_>(ev, K, nK, rec, rpix, nsorted, g, tb, pooled, ncnt, mlp, flow,  \
                               err, s, zero_buf, zero_units, zeroed, chain)
#define VECKM_TM4(DV_)                                                                       \
  (h ? (f16 ? VECKM_TM(DV_, true, true) : VECKM_TM(DV_, true, false))                        \
     : (f16 ? VECKM_TM(DV_, false, true) : VECKM_TM(DV_, false, false)))
  if (zeroed) *zeroed = false;
  switch (g.U / 32) {
    case 1:
      return VECKM_TM4(1);
    case 2:
      return VECKM_TM4(2);
    default:
      return -1;  // 2D > 256: the A slots and accumulators exceed tensor memory
  }
#undef VECKM_TM4
#undef VECKM_TM
}

VK_CHECK_READER(check_read_head)

}  // namespace veckm
