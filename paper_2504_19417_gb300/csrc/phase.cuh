// Temporal phase exp(i t T_d / dt) of Algorithm 1 with exact argument reduction.
//
// The frequency of channel d is held in turns per microsecond, reduced to
// [-1/2, 1/2] and stored as a 64-bit fixed-point fraction w64 = round(w 2^64)
// (host, FP64).  For an integer timestamp t (microseconds since the slice
// start) the phase in turns, t w mod 1, is the top of the 64-bit product
// t * w64 mod 2^64, formed exactly with integer multiplies; the dropped bits
// are below 2^-32 turn.  The angle handed to the sine/cosine therefore always
// lies in [-pi, pi): no large-argument trigonometry ever happens, whatever the
// slice length.  Error budget per component: 2^-24 turn quantisation
// (3.7e-7 rad), the one rounding of x 2pi - 3pi below together with the FP32
// constants (at most 4e-7 rad), and __sincosf on [-pi, pi] (about 3.6e-7
// absolute).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace veckm {

// exp(i 2 pi t w) for one channel, w64 = (whi << 32) | wlo.
__device__ __forceinline__ float2 turn_phase(uint32_t t, uint32_t wlo, uint32_t whi) {
  // top 32 bits of t * w64 + 1/2 turn (mod 2^64), plus half a unit of the
  // 23-bit fraction kept below: fr / 2^32 = frac(t w + 1/2)
  const uint32_t fr = __umulhi(t, wlo) + t * whi + 0x80000100u;
  // x = 1.f with that fraction as mantissa; (x - 3/2) turns = frac(t w + 1/2)
  // - 1/2 lies in [-1/2, 1/2) and equals t w modulo whole turns; the angle
  // (x - 3/2) 2 pi is formed in one fused multiply-add
  const float x = __uint_as_float(0x3f800000u | (fr >> 9));
  float s, c;
  __sincosf(fmaf(x, 6.28318530717958647692f, -9.42477796076937971538f), &s, &c);
  return make_float2(c, s);
}

// The same value as turn_phase in fewer instructions: the high half of
// t * wlo and the sum in one multiply-add, and the float bits of x in one
// funnel shift of 0x7f:fr (identical integers, so an identical angle).  For
// kernels with registers to spare (it needs one more).
__device__ __forceinline__ float2 turn_phase_lean(uint32_t t, uint32_t wlo, uint32_t whi) {
  uint32_t fr;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(fr) : "r"(t), "r"(wlo), "r"(t * whi + 0x80000100u));
  const float x = __uint_as_float(__funnelshift_r(fr, 0x7fu, 9));
  float s, c;
  __sincosf(fmaf(x, 6.28318530717958647692f, -9.42477796076937971538f), &s, &c);
  return make_float2(c, s);
}

// Channels 2u and 2u+1 as one float4 (re0, im0, re1, im1); w holds their
// fixed-point frequencies (x, y = low, high words).
__device__ __forceinline__ float4 time_phase2(uint32_t t, uint2 w0, uint2 w1) {
  const float2 a = turn_phase(t, w0.x, w0.y);
  const float2 b = turn_phase(t, w1.x, w1.y);
  return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ float4 time_phase2_lean(uint32_t t, uint2 w0, uint2 w1) {
  const float2 a = turn_phase_lean(t, w0.x, w0.y);
  const float2 b = turn_phase_lean(t, w1.x, w1.y);
  return make_float4(a.x, a.y, b.x, b.y);
}

// time_phase2_lean with the two channels' angles formed in one packed
// FP32x2 fused multiply-add (the same rounding per lane, so the same angles).
__device__ __forceinline__ float4 time_phase2_packed(uint32_t t, uint2 w0, uint2 w1) {
  uint32_t f0, f1;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(f0) : "r"(t), "r"(w0.x), "r"(t * w0.y + 0x80000100u));
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(f1) : "r"(t), "r"(w1.x), "r"(t * w1.y + 0x80000100u));
  const float x0 = __uint_as_float(__funnelshift_r(f0, 0x7fu, 9));
  const float x1 = __uint_as_float(__funnelshift_r(f1, 0x7fu, 9));
  const float2 tp = make_float2(6.28318530717958647692f, 6.28318530717958647692f);
  const float2 tc = make_float2(-9.42477796076937971538f, -9.42477796076937971538f);
  const float2 x = make_float2(x0, x1);
  uint64_t a;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(a)
      : "l"(*reinterpret_cast<const uint64_t *>(&x)), "l"(*reinterpret_cast<const uint64_t *>(&tp)),
        "l"(*reinterpret_cast<const uint64_t *>(&tc)));
  const float2 ang = *reinterpret_cast<const float2 *>(&a);
  float s0, c0, s1, c1;
  __sincosf(ang.x, &s0, &c0);
  __sincosf(ang.y, &s1, &c1);
  return make_float4(c0, s0, c1, s1);
}

}  // namespace veckm
