// Conversions between FP64 and pairs of FP32 numbers by integer operations only, shared by the
// kernels that carry FP64 vectors through FP32 arithmetic.  On GB300 the FP64 pipe (and the
// conversion work that runs on it) issues at 1/64 of the FP32 rate, so these stay on the
// integer and FP32 pipes.
#pragma once
#include <cuda_runtime.h>

namespace cd {

// The same split by integer operations only (no FP64 or conversion instruction): hi = v
// truncated to 24 significant bits, lo = the next 24 of the remaining 29 (truncated), so
// hi + lo equals v to 48 bits.  Values below 2^-100 in magnitude (and their low parts below the
// FP32 normal range) are flushed to zero: far below the rounding of any sum they enter here.
__device__ __forceinline__ float2 ff_split_bits(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hi32 = (unsigned)(u >> 32), lo32 = (unsigned)u;
  const unsigned sign = hi32 & 0x80000000u;
  const int ex = (int)((hi32 >> 20) & 0x7ffu);
  const int exf = ex - 1023 + 127;
  if (exf < 28 || exf > 254) return make_float2(0.f, 0.f);
  const unsigned man = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const float h = __uint_as_float(sign | ((unsigned)exf << 23) | man);
  const unsigned r = lo32 & 0x1fffffffu;  // v - h = r 2^(ex - 1075)
  if (r == 0u) return make_float2(h, 0.f);
  const int lz = __clz(r);                // leading one at bit 31 - lz
  const int el = (31 - lz) + (ex - 1075) + 127;
  if (el <= 0) return make_float2(h, 0.f);
  const unsigned ml = (r << (lz + 1)) >> 9;  // the 23 bits after the leading one
  return make_float2(h, __uint_as_float(sign | ((unsigned)el << 23) | ml));
}
// exact FP32 -> FP64 by integer operations (zero and FP32 subnormals give zero)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0u) return 0.0;
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(ex - 127u + 1023u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// FP64 -> (hi, lo) by conversions (host-side constants and per-CTA scalars)
__device__ __forceinline__ float2 ff_split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(__dsub_rn(v, (double)h)));
}
// acc += c * x (all double-FP32)
__device__ __forceinline__ void ff_fma(float2& acc, float2 c, float2 x) {
  const float p = __fmul_rn(c.x, x.x);
  float e = __fmaf_rn(c.x, x.x, -p);
  e = __fmaf_rn(c.x, x.y, e);
  e = __fmaf_rn(c.y, x.x, e);
  const float sm = __fadd_rn(acc.x, p);
  const float bb = __fsub_rn(sm, acc.x);
  const float er = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(sm, bb)), __fsub_rn(p, bb));
  acc.y = __fadd_rn(acc.y, __fadd_rn(er, e));
  acc.x = sm;
}
__device__ __forceinline__ float2 ff_norm(float2 a) {
  const float sm = __fadd_rn(a.x, a.y);
  return make_float2(sm, __fsub_rn(a.y, __fsub_rn(sm, a.x)));
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  float2 acc = make_float2(0.f, 0.f);
  ff_fma(acc, a, b);
  return ff_norm(acc);
}
__device__ __forceinline__ double ff_to_double(float2 a) {
  return __dadd_rn(f2d_bits(a.x), f2d_bits(a.y));
}

}  // namespace cd
