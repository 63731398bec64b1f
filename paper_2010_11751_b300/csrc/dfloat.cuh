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

// ---- conversions ----
// On B300 every conversion from or to a 64-bit type (cvt.f32.s64,
// cvt.s64.f32, cvt.f64.*) runs at the FP64 rate (measured ~2 per SM per
// clock), while 32-bit integer -> FP32 conversions and FP32 additions run at
// 32 to 64 times that, so 64-bit integers are converted in 21- and 32-bit
// pieces.
//
// 64-bit integer (|x| < 2^62) -> normalised double-float:
// x = a 2^42 + b 2^21 + c with 21-bit b, c; each piece is exact in FP32, the
// first two are summed error-free, and the result is renormalised, so
// |x - (hi + lo)| <= 2^-47 |x| and |lo| <= ulp(hi) / 2
__device__ __forceinline__ DF i64_to_df(long long x) {
  const int a = (int)(x >> 42);
  const int b = (int)((x >> 21) & 0x1fffff);
  const int c = (int)(x & 0x1fffff);
  const DF s = two_sum(fmul(__int2float_rn(a), 0x1p42f), fmul(__int2float_rn(b), 0x1p21f));
  return fast_two_sum(s.hi, fadd(s.lo, __int2float_rn(c)));
}
// double-float -> nearest 64-bit integer (each of two parts rounded to
// nearest: |error| <= 1), for |hi| < 2^53 and |lo| < 2^31: the multiple of
// 2^32 nearest to hi comes from a magic-number rounding (1.5 2^23 + v rounds v
// to an integer and holds it in its low significand bits), the rest of hi
// (exact, |r| <= 2^31) and lo from 32-bit conversions
__device__ __forceinline__ long long df_round_i64(DF y) {
  const float t = ffma(y.hi, 0x1p-32f, 12582912.0f);
  const int n = (int)(fbits(t) - 0x4b400000u);
  const float r = ffma(-fsub(t, 12582912.0f), 0x1p32f, y.hi);
  return (long long)((unsigned long long)(long long)n << 32) + (long long)__float2int_rn(r) +
         (long long)__float2int_rn(y.lo);
}
// a x 2^s for a power of two 2^s (exact while no part leaves the normal range)
__host__ __device__ __forceinline__ DF df_scale(DF a, float p2) { return {fmul(a.hi, p2), fmul(a.lo, p2)}; }
// host split of an FP64 constant: hi rounded to FP32, lo the rounded remainder
// (|d - (hi + lo)| <= 2^-48 |d|)
inline DF df_split(double d) {
  const float hi = (float)d;
  return {hi, (float)(d - (double)hi)};
}

// the FP64 relaxation rates prepared for the FP64 BGK-W2 and TRT collisions
// that run on the FP32 pipe (fx64.cuh): double-float copies (split on the
// host) and, per weight class c, the FP64 constant W_c = w t_c as a bit pattern
// with the factor that takes grid units to W_c's units in the last place
struct DFK {
  DF omc, hs, hd, pad;
  DF wt[4], wt3[4], wm3[4];
  DF wm[4];  // w- t_c (TRT antisymmetric rate times the weight)
  long long wbits[4];
  float yscale[4];
  double omc64;         // 1 - w
  double trt_a, trt_b;  // TRT: (1 - w)/2 + (1 - w-)/2 and (1 - w)/2 - (1 - w-)/2
  DF trt_bdf, pad2;     // trt_b as double-float
  DF wplus, wminus;     // the bulk couplings w+ and w- (RR, fx_rr.cuh)
};

}  // namespace lbm
