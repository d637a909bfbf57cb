// Kernel density read back from encodings (Lemma 1 of Section 2.2.1): for an
// encoding row e of event k and an integer offset q = (dt, dx, dy) from that
// event, g = Re((1/D) sum_d e_d conj(exp(i a_d))) with
// a_d = dt T_d / delta_t + dx X_d / delta_x + dy Y_d / delta_y.  Each term of
// a_d is reduced modulo one turn exactly: the frequencies are held as 64-bit
// fixed-point turns per microsecond or per pixel, multiplied by the integer
// offset modulo 2^64 (two's complement covers negative offsets), and the
// three fractions are added modulo 2^64 before one sine/cosine on [-pi, pi).
#include <cuda_runtime.h>

#include "ctx.h"

namespace veckm {
namespace {

__device__ __forceinline__ uint64_t w64(uint2 w) { return ((uint64_t)w.y << 32) | w.x; }

// one warp per query; lanes over channels
__global__ void __launch_bounds__(256)
    k_kde_query(const float *__restrict__ emb, int64_t nrows, int D, const int64_t *__restrict__ row,
                const int32_t *__restrict__ qt, const int32_t *__restrict__ qx,
                const int32_t *__restrict__ qy, int64_t nq, const uint2 *__restrict__ wt,
                const uint2 *__restrict__ wxy, float *__restrict__ out, int *err) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  const int64_t r = row[q];
  if (r < 0 || r >= nrows) {
    if (lane == 0) {
      atomicOr(err, ERR_INDEX_RANGE);
      out[q] = 0.f;
    }
    return;
  }
  const uint64_t dt = (uint64_t)(int64_t)qt[q], dx = (uint64_t)(int64_t)qx[q],
                 dy = (uint64_t)(int64_t)qy[q];
  const float *e = emb + (size_t)r * 2 * D;
  float s = 0.f;
  for (int d = lane; d < D; d += 32) {
    // a_d / (2 pi) + 1/2 modulo one turn, in 64-bit fixed point, plus half a
    // unit of the 23 bits kept below
    const uint64_t f = dt * w64(wt[d]) + dx * w64(wxy[d]) + dy * w64(wxy[D + d]) +
                       0x8000000000000000ull + (1ull << 40);
    // top 24 bits as the mantissa of a number in [1, 2); minus 1.5 gives the
    // angle in turns in [-1/2, 1/2), equal to a_d modulo whole turns
    const float turn = __uint_as_float(0x3f800000u | (uint32_t)(f >> 41)) - 1.5f;
    float sn, cs;
    __sincosf(turn * 6.28318530717958647692f, &sn, &cs);
    s = fmaf(e[d], cs, fmaf(e[D + d], sn, s));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[q] = s / (float)D;
}

}  // namespace
}  // namespace veckm

using namespace veckm;

extern "C" veckm_status veckm_kde_query(veckm_ctx *c, const float *d_emb, int64_t nrows,
                                        const int64_t *d_row, const int32_t *d_qt,
                                        const int32_t *d_qx, const int32_t *d_qy, int64_t nq,
                                        float *d_out, void *stream) {
  if (!c) return fail_msg(VECKM_EINVAL, "null context");
  if (nrows < 0 || nq < 0) return fail_msg(VECKM_EINVAL, "negative size");
  if (nq == 0) return VECKM_OK;
  if (!d_emb || !d_row || !d_qt || !d_qx || !d_qy || !d_out)
    return fail_msg(VECKM_EINVAL, "null buffer");
  const int64_t blocks = (nq * 32 + 255) / 256;
  if (blocks > 0x7fffffff) return fail_msg(VECKM_EINVAL, "too many queries");
  k_kde_query<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      d_emb, nrows, c->g.D, d_row, d_qt, d_qx, d_qy, nq, c->wt, c->wxy, d_out, c->err);
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail_cuda(e, "density query launch");
  }
  c->last_launches = 1;
  return VECKM_OK;
}
