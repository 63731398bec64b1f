// fx64.cuh -- BGK-W2 and TRT collisions of FP64-stored populations with their
// arithmetic taken off the FP64 pipe.
//
// On B300 the FP64 pipe issues 2 operations per SM per clock (so do all
// conversions from or to 64-bit types); the plain FP64 BGK-W2 update needs
// ~124 FP64 operations per cell, which caps it near a fifth of the HBM
// roofline.  Here each population costs one FP64 fused multiply-add (two for
// TRT): the relaxation f_out = (1 - w) f + w E_k itself.
//
//  * Moments, exactly.  A population f_k whose sign and exponent equal those
//    of its lattice weight t_k (f_k / t_k in [0.56, 1.12] for the D3Q19 weight
//    classes 1/18 and 1/36, wider for the others) differs from t_k by an
//    integer number of t_k's units in the last place: the difference of the
//    two FP64 bit patterns.  Shifted to a grid common to the lattice (2^-58 for
//    D3Q19, 2^-60 for D3Q27: the unit in the last place of the smallest
//    weight), the deviations g_k = f_k - t_k are exact 64-bit integers, and so
//    are the density deviation rho - 1 = sum g_k and the momentum
//    j = sum c_k g_k (pair sums first, as in the FP64 operator).
//  * The equilibrium part, in double-float (dfloat.cuh): 1/rho, v = 1.5 j/rho
//    and A = rho - 1 - v.j, then per pair P = w t_c A + (e.v) q and
//    q = 3 w t_c (e.j), so that w E_k = w t_k + P +- q.  These are deviations
//    of size |g| rather than |f|, so each lazy double-float operation errs by
//    ~2^-47 |g|.
//  * w E_k as an FP64 number without FP64 arithmetic: P and q, rounded to the
//    units in the last place of the FP64 constant W_c = w t_c, are added as
//    integers to W_c's bit pattern.  If the sum leaves W_c's binade (or P, q
//    are too large for the integer rounding), w E_k is formed with FP64
//    additions instead.
//
// A cell with any population outside its weight's binade (strong
// non-equilibrium, high Mach number) is updated by the plain FP64 operator
// (the caller's fallback).  Both paths compute the update of Section 2.6 to
// within a few FP64 rounding errors; which one a cell takes depends only on
// its own populations, so every scheme (they differ only in where they load
// and store) still produces bit-identical results.
#pragma once
#include <cstring>

#include "dfloat.cuh"
#include "lattice.cuh"

namespace lbm {

// floor(log2 t) for 0 < t < 2^30
__host__ __device__ constexpr int fx_exp2_floor(double t) {
  int e = 0;
  while (t < 1.0) {
    t *= 2.0;
    --e;
  }
  while (t >= 2.0) {
    t *= 0.5;
    ++e;
  }
  return e;
}
__host__ __device__ constexpr double fx_pow2(int e) {
  double v = 1.0;
  for (; e > 0; --e) v *= 2.0;
  for (; e < 0; ++e) v *= 0.5;
  return v;
}

// exponent of the integer grid of the moments: the unit in the last place of
// the smallest weight (1/36 for D3Q19, 1/216 for D3Q27)
__host__ __device__ constexpr int fx_grid(int Q) { return Q == 19 ? -58 : -60; }

// the lattice weight of population K as an FP64 bit pattern, and the shift
// that takes its units in the last place to the grid
template <int Q, int K>
struct FxW {
  static constexpr double t = Lat<Q>::w(K);
  static constexpr int e = fx_exp2_floor(t);
  static constexpr long long mant = (long long)(t * fx_pow2(52 - e));  // in [2^52, 2^53)
  static constexpr long long bits = ((long long)(1023 + e) << 52) | (mant - (1LL << 52));
  static constexpr unsigned hi_tag = (unsigned)(1023 + e) << 20;  // sign 0 and the exponent field
  static constexpr int sh = e - 52 - fx_grid(Q);
  static_assert(sh >= 0 && sh < 8, "weight not representable on the grid");
};

// host: the class constants W_c = w t_c (= wt[c], as bit patterns) and the
// factors that take grid units to W_c's units in the last place
inline void fx_class_constants(int Q, const double (&wt)[4], DFK& k) {
  for (int c = 0; c < 4; ++c) {
    const double W = wt[c];
    static_assert(sizeof(double) == sizeof(long long), "64-bit double");
    std::memcpy(&k.wbits[c], &W, sizeof W);
    const int e = W > 0.0 ? fx_exp2_floor(W) : 0;
    k.yscale[c] = (float)fx_pow2(fx_grid(Q) + 52 - e);
  }
}

// nearest integer of a double-float (W_c's last-place units); ok stays true
// while the value is inside the range df_round_i64 handles
__device__ __forceinline__ long long fx_units(DF y, bool& ok) {
  ok = ok && fabsf(y.hi) < 0x1p52f && fabsf(y.lo) < 0x1p30f;
  return df_round_i64(y);
}

// w E = W_c + P + S q (S = +-1) as an FP64 number, from the rounded units of
// P and q; with FP64 additions where the integer route does not apply
template <int Q, int S>
__device__ __forceinline__ double fx_weq(const DFK& k_, int c, long long pi, long long qi, bool ok, const DF& P,
                                         const DF& q) {
  const long long b = k_.wbits[c] + pi + (S > 0 ? qi : -qi);
  if (ok && ((unsigned long long)(b ^ k_.wbits[c]) >> 52) == 0ull) return __longlong_as_double(b);
  const double p = __dadd_rn((double)P.hi, (double)P.lo), qq = __dadd_rn((double)q.hi, (double)q.lo);
  const double dev = __dmul_rn(S > 0 ? __dadd_rn(p, qq) : __dsub_rn(p, qq), fx_pow2(fx_grid(Q)));
  return __dadd_rn(__longlong_as_double(k_.wbits[c]), dev);
}

// false (and f untouched) when some population is outside its weight's binade
template <int Q, bool TRT_>
__device__ __forceinline__ bool collide_fx(double (&f)[Q], const DFK& k_, CellSums* cs) {
  constexpr int H = Lat<Q>::H;
  unsigned acc = 0u;
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    acc |= (unsigned)__double2hiint(f[k]) ^ FxW<Q, k>::hi_tag;
  });
  if (acc & 0xfff00000u) return false;
  // exact moments on the grid: r = rho - 1, j
  long long r, jx = 0, jy = 0, jz = 0;
  {
    auto dev = [&](auto kc) {
      constexpr int k = decltype(kc)::value;
      return (long long)((unsigned long long)(__double_as_longlong(f[k]) - FxW<Q, k>::bits) << FxW<Q, k>::sh);
    };
    r = dev(std::integral_constant<int, H>{});
    static_for<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const long long gm = dev(kc), gp = dev(std::integral_constant<int, k + H + 1>{});
      r += gp + gm;
      const long long d = gp - gm;
      constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
      if constexpr (ex == 1) jx += d;
      if constexpr (ex == -1) jx -= d;
      if constexpr (ey == 1) jy += d;
      if constexpr (ey == -1) jy -= d;
      if constexpr (ez == 1) jz += d;
      if constexpr (ez == -1) jz -= d;
    });
  }
  constexpr float GRID = (float)fx_pow2(fx_grid(Q));
  // rho = 1 + r, v = 1.5 j / rho (real units); A = r - v.j (grid units)
  const DF dr = i64_to_df(r);
  const DF Jx = i64_to_df(jx), Jy = i64_to_df(jy), Jz = i64_to_df(jz);
  const DF rho = fast_two_sum(1.0f, fmul(dr.hi, GRID));
  const DF inv15 = df_mulf(df_recip({rho.hi, fadd(rho.lo, fmul(dr.lo, GRID))}), 1.5f);
  const DF vx = df_mul(df_scale(Jx, GRID), inv15);
  const DF vy = df_mul(df_scale(Jy, GRID), inv15);
  const DF vz = df_mul(df_scale(Jz, GRID), inv15);
  const DF vj = df_add(df_add(df_mul(vx, Jx), df_mul(vy, Jy)), df_mul(vz, Jz));
  const DF A = df_sub(dr, vj);
  if (cs) {
    // FP64 sums of the state read: rho = 1 + r, kinetic energy |j|^2 / (2 rho) = v.j / 3
    cs->rho = __dadd_rn(1.0, __dmul_rn(__ll2double_rn(r), fx_pow2(fx_grid(Q))));
    cs->ke = __dmul_rn(__dadd_rn((double)vj.hi, (double)vj.lo), fx_pow2(fx_grid(Q)) / 3.0);
  }
  const double omc = k_.omc64;
  {
    const DF wtA = df_mul(k_.wt[0], A);
    bool ok = true;
    const long long pi = fx_units(df_scale(wtA, k_.yscale[0]), ok);
    f[H] = fma(omc, f[H], fx_weq<Q, 1>(k_, 0, pi, 0, ok, wtA, DF{0.0f, 0.0f}));
  }
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
    constexpr int c = Lat<Q>::norm2(k);
    // e.v and e.j (components of e are -1, 0 or 1)
    DF ev{0.0f, 0.0f}, ej{0.0f, 0.0f};
    bool first = true;
    auto add_c = [&](const DF& v, const DF& j, int sign) {
      const DF sv = sign > 0 ? v : df_neg(v), sj = sign > 0 ? j : df_neg(j);
      ev = first ? sv : df_add(ev, sv);
      ej = first ? sj : df_add(ej, sj);
      first = false;
    };
    if constexpr (ex != 0) add_c(vx, Jx, ex);
    if constexpr (ey != 0) add_c(vy, Jy, ey);
    if constexpr (ez != 0) add_c(vz, Jz, ez);
    const DF qp = df_mul(k_.wt3[c], ej);                       // 3 w t (e.j)
    const DF P = df_add(df_mul(ev, qp), df_mul(k_.wt[c], A));  // w t A + (e.v) q
    const DF q = TRT_ ? df_mul(k_.wm3[c], ej) : qp;            // antisymmetric part
    bool ok = true;
    const float ys = k_.yscale[c];
    const long long pi = fx_units(df_scale(P, ys), ok);
    const long long qi = fx_units(df_scale(q, ys), ok);
    const double Ep = fx_weq<Q, 1>(k_, c, pi, qi, ok, P, q);   // w E along +e
    const double Em = fx_weq<Q, -1>(k_, c, pi, qi, ok, P, q);  // w E along -e
    const double fp = f[k + H + 1], fm = f[k];
    if constexpr (TRT_) {
      // (1-w)/2 (f+ + f-) +- (1-w-)/2 (f+ - f-), one population at a time
      f[k + H + 1] = fma(k_.trt_a, fp, fma(k_.trt_b, fm, Ep));
      f[k] = fma(k_.trt_a, fm, fma(k_.trt_b, fp, Em));
    } else {
      f[k + H + 1] = fma(omc, fp, Ep);
      f[k] = fma(omc, fm, Em);
    }
  });
  return true;
}

}  // namespace lbm
