// fx_rr.cuh -- the recursive-regularized collision (RR) of FP64-stored
// populations with its arithmetic taken off the FP64 pipe, in the manner of
// fx64.cuh.
//
// The plain FP64 operator (collision.cuh, collide_rr) costs ~210 FP64
// operations per D3Q19 cell, which binds it to B300's FP64 pipe at a ninth of
// the HBM roofline.  Here:
//  * every population in its weight's binade (else the FP64 operator runs) is
//    t_k + g_k with g_k an exact integer on the grid of fx64.cuh, so every raw
//    moment of the deviations g is an exact 64-bit integer sum;
//  * the rest is double-float arithmetic (dfloat.cuh) on quantities that
//    vanish at rest -- density deviation, velocity, second-order
//    non-equilibrium, and the post-collision Hermite moments of order >= 1 --
//    so that each operation errs by ~2^-47 of a small number;
//  * the post-collision deviations follow from the Hermite moments by the
//    same transforms as the FP64 operator (Hermite -> monomial per axis, then
//    the inverse moment matrix, both linear): the moments of the rest state
//    (1, 0, ..., 0) are left out of the transform and their contribution,
//    the weights' raw moments, is added to the deviation moments exactly;
//  * each new population is t_k plus its deviation rounded to t_k's units in
//    the last place, assembled on t_k's bit pattern; a value that leaves t_k's
//    binade sends the cell back to the FP64 operator (its populations are
//    reloaded, as in fx64.cuh).
// Both compute the update of Section 2.6 (RR as defined by the oracle) to
// within a few FP64 roundings of the populations, and which one a cell takes
// depends on its own populations alone, so every scheme stays bit-identical.
#pragma once
#include "collision.cuh"
#include "dfloat.cuh"
#include "fx64.cuh"

namespace lbm {

// double-float number for the generic moment code of collision.cuh
struct dfn {
  DF v;
  __device__ __forceinline__ dfn() {}
  __device__ __forceinline__ dfn(DF x) : v(x) {}
  // compile-time constants only (a run-time double would cost FP64 conversions)
  __device__ __forceinline__ dfn(double d) : v{(float)d, (float)(d - (double)(float)d)} {}
  __device__ __forceinline__ dfn(int i) : v{(float)i, 0.0f} {}
};
__device__ __forceinline__ dfn operator+(dfn a, dfn b) { return dfn(df_add(a.v, b.v)); }
__device__ __forceinline__ dfn operator-(dfn a, dfn b) { return dfn(df_sub(a.v, b.v)); }
__device__ __forceinline__ dfn operator-(dfn a) { return dfn(df_neg(a.v)); }
__device__ __forceinline__ dfn operator*(dfn a, dfn b) { return dfn(df_mul(a.v, b.v)); }

// deviation g_K = f - t_K of a population in t_K's binade, on the narrow grid
template <int Q, int K>
__device__ __forceinline__ long long fx_dev_narrow(double f) {
  using W = FxW<Q, K, false>;
  return (long long)((unsigned long long)(__double_as_longlong(f) - W::bits) << W::sh);
}

// the RR collision of one cell (FxStatus, as collide_fx); cs: its FP64 sums
template <int Q>
__device__ __forceinline__ int collide_rr_fx(double (&f)[Q], const DFK& k_, CellSums* cs) {
  unsigned acc = 0u;
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    acc |= (unsigned)__double2hiint(f[k]) ^ FxW<Q, k, false>::hi_tag;
  });
  if (acc & 0xfff00000u) return FX_SKIPPED;
  constexpr float GRID = (float)fx_pow2(fx_grid(Q, false));
  // raw moments of the deviations, exact, then in double-float (real units)
  dfn M[Q];
  long long g0;
  {
    long long g[Q], G[Q];
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      g[k] = fx_dev_narrow<Q, k>(f[k]);
    });
    raw_moments<Q>(g, G);
    g0 = G[0];
    static_for<0, Q>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      M[J] = dfn(df_scale(i64_to_df(G[J]), GRID));
    });
  }
  const dfn drho = M[0];
  const dfn rho = dfn(1) + drho;
  const dfn inv = dfn(df_recip(rho.v));
#define IX(a, b, c) bidx<Q, a, b, c>
  const dfn ux = M[IX(1, 0, 0)] * inv, uy = M[IX(0, 1, 0)] * inv, uz = M[IX(0, 0, 1)] * inv;
  if (cs) {
    cs->rho = __dadd_rn(1.0, __dmul_rn(__ll2double_rn(g0), fx_pow2(fx_grid(Q, false))));
    const dfn ke = (ux * M[IX(1, 0, 0)] + uy * M[IX(0, 1, 0)] + uz * M[IX(0, 0, 1)]) * dfn(0.5);
    cs->ke = __dadd_rn((double)ke.v.hi, (double)ke.v.lo);
  }
  // second-order non-equilibrium: the normalised raw moment minus its rest
  // value (c_s^2 on the diagonal) is (M - drho c_s^2) / rho
  const dfn cs2 = dfn(1.0 / 3.0);
  const dfn nxx = (M[IX(2, 0, 0)] - drho * cs2) * inv - ux * ux;
  const dfn nyy = (M[IX(0, 2, 0)] - drho * cs2) * inv - uy * uy;
  const dfn nzz = (M[IX(0, 0, 2)] - drho * cs2) * inv - uz * uz;
  const dfn nxy = M[IX(1, 1, 0)] * inv - ux * uy;
  const dfn nxz = M[IX(1, 0, 1)] * inv - ux * uz;
  const dfn nyz = M[IX(0, 1, 1)] * inv - uy * uz;
  const dfn wplus = dfn(k_.wplus), wminus = dfn(k_.wminus), omc = dfn(k_.omc);
  const dfn axx = nxx - wplus * nxx - wminus * (nyy + nzz);
  const dfn ayy = nyy - wplus * nyy - wminus * (nxx + nzz);
  const dfn azz = nzz - wplus * nzz - wminus * (nxx + nyy);
  const dfn axy = omc * nxy, axz = omc * nxz, ayz = omc * nyz;
#undef IX
  // post-collision Hermite moments less the rest state's (1, 0, ..., 0)
  dfn X[Q];
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    constexpr int a = basis_exp(Q, J, 0), b = basis_exp(Q, J, 1), c = basis_exp(Q, J, 2);
    constexpr int o = a + b + c;
    if constexpr (o == 0) {
      X[J] = dfn(0);
    } else {
      dfn v = uprod<Q, J>(ux, uy, uz);
      if constexpr (o == 2) {
        if constexpr (a == 2) v = v + axx;
        else if constexpr (b == 2) v = v + ayy;
        else if constexpr (c == 2) v = v + azz;
        else if constexpr (a == 1 && b == 1) v = v + axy;
        else if constexpr (a == 1 && c == 1) v = v + axz;
        else v = v + ayz;
      } else if constexpr (o >= 3) {
        auto um = [&](int da, int db, int dc) {
          dfn r = dfn(1);
          for (int i = 0; i < a - da; ++i) r = r * ux;
          for (int i = 0; i < b - db; ++i) r = r * uy;
          for (int i = 0; i < c - dc; ++i) r = r * uz;
          return r;
        };
        if constexpr (a == 2) v = v + um(2, 0, 0) * axx;
        if constexpr (b == 2) v = v + um(0, 2, 0) * ayy;
        if constexpr (c == 2) v = v + um(0, 0, 2) * azz;
        if constexpr (a >= 1 && b >= 1) v = v + dfn(a * b) * um(1, 1, 0) * axy;
        if constexpr (a >= 1 && c >= 1) v = v + dfn(a * c) * um(1, 0, 1) * axz;
        if constexpr (b >= 1 && c >= 1) v = v + dfn(b * c) * um(0, 1, 1) * ayz;
      }
      X[J] = v;
    }
  });
  all_axes<Q, 3>(X, ux, uy, uz);  // Hermite -> monomial (linear)
  // raw moments of the new deviations: rho (w_J + X_J) - w_J = drho w_J + rho X_J
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    constexpr double wm = weight_moment<Q>(J);
    if constexpr (J == 0) X[J] = drho;
    else if constexpr (wm != 0.0) X[J] = drho * dfn(wm) + rho * X[J];
    else X[J] = rho * X[J];
  });
  dfn g[Q];
  populations_from_raw<Q>(X, g);
  // t_k plus the deviation rounded to t_k's units in the last place, on t_k's
  // bit pattern; every result must stay in t_k's binade
  bool ok = true;
  unsigned off = 0u;
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    using W = FxW<Q, k, false>;
    constexpr float SCALE = (float)fx_pow2(52 - W::e);
    const long long b = W::bits + fx_units(df_scale(g[k].v, SCALE), ok);
    off |= (unsigned)((b ^ W::bits) >> 32);
    f[k] = __longlong_as_double(b);
  });
  return (ok && (off & 0xfff00000u) == 0u) ? FX_DONE : FX_REDO;
}

}  // namespace lbm
