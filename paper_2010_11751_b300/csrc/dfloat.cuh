// dfloat.cuh -- double-float ("float-float") arithmetic: a value is held as
// the unevaluated sum hi + lo of two FP32 numbers, which carries about 48
// significant bits, so that FP64-accurate arithmetic can run on the FP32
// pipe.  On B300 the FP64 pipe issues 2 operations per SM per clock, the FP32
// pipe about 120; conversions between FP32 and FP64 (cvt) also run at the
// FP64 rate, so FP64 <-> double-float conversions here work on the bits with
// integer operations.
//
// Published methods used (no other source):
//   two_sum       Knuth's error-free sum (TAOCP vol. 2, 4.2.2, Theorem B):
//                 s = fl(a + b) and the exact error e with a + b = s + e,
//                 for any ordering of |a|, |b|.
//   two_prod      error-free product with a fused multiply-add
//                 (Dekker 1971 / Ogita, Rump & Oishi 2005):
//                 p = fl(a b), e = fma(a, b, -p), a b = p + e exactly.
//   fast_two_sum  Dekker's sum for |a| >= |b|: s = fl(a + b), e = b - (s - a).
//
// The double-float operations below are "lazy": hi parts always go through
// the error-free transformations, lo parts are accumulated in plain FP32, and
// results are not renormalised unless asked.  Each operation then errs by
// about 2^-47 times the magnitude of its operands, which is what the lattice
// Boltzmann update needs: its tolerance is absolute, relative to the size of
// the populations, and the quantities it combines are of that size or smaller.
//
// Every function is __host__ __device__ so that the arithmetic can be run and
// checked on a CPU with the same IEEE-754 single-precision operations (the
// device uses round-to-nearest intrinsics, which are never contracted into
// fused multiply-adds; host builds must not contract either).
#pragma once
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace lbm {

struct DF {
  float hi, lo;
};

// ---- single-precision operations, rounded to nearest, never contracted ----
__host__ __device__ __forceinline__ float fadd(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float fsub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float fmul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float ffma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

// ---- bit access ----
__host__ __device__ __forceinline__ uint32_t fbits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float bitsf(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}
__host__ __device__ __forceinline__ void dwords(double d, uint32_t& hw, uint32_t& lw) {
#ifdef __CUDA_ARCH__
  hw = (uint32_t)__double2hiint(d);
  lw = (uint32_t)__double2loint(d);
#else
  uint64_t u;
  std::memcpy(&u, &d, 8);
  hw = (uint32_t)(u >> 32);
  lw = (uint32_t)u;
#endif
}
__host__ __device__ __forceinline__ double wordsd(uint32_t hw, uint32_t lw) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hw, (int)lw);
#else
  const uint64_t u = ((uint64_t)hw << 32) | lw;
  double d;
  std::memcpy(&d, &u, 8);
  return d;
#endif
}
__host__ __device__ __forceinline__ uint32_t funnel_l3(uint32_t lw, uint32_t hw) {
  // (hw << 3) | (lw >> 29)
#ifdef __CUDA_ARCH__
  return __funnelshift_l(lw, hw, 3);
#else
  return (hw << 3) | (lw >> 29);
#endif
}
__host__ __device__ __forceinline__ float u2f_rn(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(u);
#else
  return (float)u;  // round to nearest (the default mode)
#endif
}

// ---- error-free transformations ----
__host__ __device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = fadd(a, b);
  const float bb = fsub(s, a);
  const float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
  return {s, e};
}
__host__ __device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = fmul(a, b);
  return {p, ffma(a, b, -p)};
}
__host__ __device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = fadd(a, b);
  return {s, fsub(b, fsub(s, a))};
}

// ---- lazy double-float arithmetic ----
__host__ __device__ __forceinline__ DF df_add(DF a, DF b) {
  DF t = two_sum(a.hi, b.hi);
  t.lo = fadd(t.lo, fadd(a.lo, b.lo));
  return t;
}
__host__ __device__ __forceinline__ DF df_sub(DF a, DF b) {
  DF t = two_sum(a.hi, -b.hi);
  t.lo = fadd(t.lo, fsub(a.lo, b.lo));
  return t;
}
__host__ __device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
// a b, dropping a.lo b.lo
__host__ __device__ __forceinline__ DF df_mul(DF a, DF b) {
  DF t = two_prod(a.hi, b.hi);
  t.lo = ffma(a.hi, b.lo, ffma(a.lo, b.hi, t.lo));
  return t;
}
// a c for an FP32 c
__host__ __device__ __forceinline__ DF df_mulf(DF a, float c) {
  DF t = two_prod(a.hi, c);
  t.lo = ffma(a.lo, c, t.lo);
  return t;
}
// a b + c, with the hi product and the hi sum error-free
__host__ __device__ __forceinline__ DF df_fma(DF a, DF b, DF c) { return df_add(df_mul(a, b), c); }
__host__ __device__ __forceinline__ DF df_renorm(DF a) { return fast_two_sum(a.hi, a.lo); }
// 1 / a: an FP32 reciprocal refined by one Newton step in double-float,
// r = r0 + r0 (1 - a r0), with the residual 1 - a r0 formed error-free in its
// hi part (a must be normalised; |relative error| ~ 2^-46)
__host__ __device__ __forceinline__ DF df_recip(DF a) {
  const float r0 = 1.0f / a.hi;  // correctly rounded division (host and device)
  const DF p = two_prod(a.hi, r0);                        // a.hi r0 = p.hi + p.lo exactly
  const float res = fsub(fsub(fsub(1.0f, p.hi), p.lo), fmul(a.lo, r0));  // 1 - a r0, ~2^-24
  return fast_two_sum(r0, fmul(r0, res));
}

// ---- conversions between FP64 and double-float, on the bits ----
// Valid for |d| in [2^-74, 2^127]; smaller magnitudes (zero included) are
// taken as +-2^-74 (an absolute error below 5.3e-23), larger ones are not
// supported.  hi keeps the sign, exponent and leading 24 significand bits of d
// (truncated); lo is the remaining 29 bits, rounded to nearest FP32:
// |d - (hi + lo)| <= 2^-48 |d|.
__host__ __device__ __forceinline__ DF df_from_double(double d) {
  uint32_t hw, lw;
  dwords(d, hw, lw);
  const uint32_t sign = hw & 0x80000000u;
  uint32_t mag = hw & 0x7fffffffu;
  mag = mag > (uint32_t)((1023 - 74) << 20) ? mag : (uint32_t)((1023 - 74) << 20);
  lw = mag == (uint32_t)((1023 - 74) << 20) ? 0u : lw;
  // rebias the exponent (1023 -> 127) in place, then shift the top 23
  // significand bits into FP32 position
  const uint32_t hb = funnel_l3(lw, mag - (896u << 20)) | sign;
  // lo = (remaining 29 bits) x 2^(e - 52), with the sign of d
  const uint32_t scale = (hb & 0xff800000u) - (52u << 23);
  const float lo = fmul(u2f_rn(lw & 0x1fffffffu), bitsf(scale));
  return {bitsf(hb), lo};
}

// exact FP64 value of a normal FP32 number (integer operations only; zero and
// subnormals give 2^-127 or so in magnitude instead, below 1e-38)
__host__ __device__ __forceinline__ double f2d_bits(float x) {
  const uint32_t b = fbits(x);
  const uint32_t hw = (((b & 0x7fffffffu) >> 3) + (896u << 20)) | (b & 0x80000000u);
  return wordsd(hw, b << 29);
}
// nearest FP64 to hi + lo: both converted exactly, then one FP64 addition
__host__ __device__ __forceinline__ double df_to_double(DF a) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(f2d_bits(a.hi), f2d_bits(a.lo));
#else
  return f2d_bits(a.hi) + f2d_bits(a.lo);
#endif
}
// split of a host-side FP64 constant (exact-ish: rounded hi, rounded remainder)
__host__ __device__ __forceinline__ DF df_const(double d) {
  const float hi = (float)d;
  return {hi, (float)(d - (double)hi)};
}

}  // namespace lbm
