// Internal declarations shared by the library's own translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/veckm.h"

namespace veckm {

// Bits of the device error word.
enum : int { ERR_EVENT_RANGE = 1, ERR_INDEX_RANGE = 2, ERR_TIMEOUT = 4 };

// Low level of the split time table: t_rel = 64 a + b.
constexpr int kTLoBits = 6;
constexpr int kTLo = 1 << kTLoBits;

// Device view of one slice's events.
struct Events {
  const int16_t *x, *y;
  const uint32_t *t;
  int64_t n;
  uint32_t t_ref;
  uint32_t t_span;  // largest accepted t - t_ref
};

// Device-side constant state of a context.  Complex values are stored as
// interleaved (re, im) FP32 with the channel index fastest; one float4 holds
// channels 2u and 2u+1 ("unit" u), so a pixel has U = D/2 units.
struct Geometry {
  int W, H, D, U, dx, dy;
};

struct Tables {
  const float4 *tx;     // [W][U]   exp(i x X/dx), x in [0, W)
  const float4 *ty;     // [H][U]   exp(i y Y/dy), y in [0, H)
  const float4 *tt_lo;  // [64][U]  exp(i b T/dt), b in [0, 64)
  const float4 *tt_hi;  // [NH][U]  exp(i 64 a T/dt), a in [0, NH)
};

struct MLP {
  const float *W1;       // [hidden][2D] FP32
  const float *W1t;      // [2D][hidden] FP32 (transposed copy for the CUDA-core path)
  const float *b1;       // [hidden]
  const float *W2;       // [2][hidden]
  const float *b2;       // [2]
  const uint16_t *W1h;   // [hidden][2D] BF16 or FP16 bits, core-matrix order for tcgen05
  int hidden;
  int half_kind;         // 0: BF16, 1: FP16 (for W1h)
};

// Launchers (kernels.cu).  Each returns the number of kernels it launched
// (or a negative cudaError_t value on a launch failure).
int launch_scatter(const Events &ev, const Geometry &g, const Tables &tb, float4 *acc, int *cnt,
                   int *err, cudaStream_t s);
// Pooling: row pass acc -> hbuf, column pass hbuf -> acc, window counts.
int launch_pool_rows(const Geometry &g, const Tables &tb, const float4 *acc, float4 *hbuf,
                     cudaStream_t s);
int launch_pool_cols(const Geometry &g, const Tables &tb, const float4 *hbuf, float4 *acc,
                     cudaStream_t s);
int launch_counts(const Geometry &g, const int *cnt, int *cnt_tmp, int *ncnt, cudaStream_t s);
int launch_gather_emb(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                      const Tables &tb, const float4 *pooled, const int *ncnt, float *emb,
                      int *err, cudaStream_t s);
int launch_predict_fp32(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                        const Tables &tb, const float4 *pooled, const int *ncnt, const MLP &mlp,
                        float *flow, int *err, cudaStream_t s);
int launch_predict_tc(const Events &ev, const int64_t *K, int64_t nK, const Geometry &g,
                      const Tables &tb, const float4 *pooled, const int *ncnt, const MLP &mlp,
                      float *flow, int *err, cudaStream_t s);

int num_sms();

}  // namespace veckm
