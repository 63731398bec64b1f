// fx64.cuh -- BGK-W2 and TRT collisions of FP64-stored populations with their
// arithmetic taken off the FP64 pipe.
//
// On B300 the FP64 pipe issues 2 operations per SM per clock (so do all
// conversions from or to 64-bit types); the plain FP64 BGK-W2 update needs
// ~124 FP64 operations per cell, which caps it near a fifth of the HBM
// roofline.  Here each population costs one FP64 fused multiply-add: the
// relaxation f_out = (1 - w) f + w E_k itself (for TRT, the part relaxing at
// the other rate joins w E_k).
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
//  * w E_k as an FP64 number without FP64 arithmetic: w t_c A, (e.v) q and q,
//    each rounded to the units in the last place of the FP64 constant
//    W_c = w t_c, are added as integers to W_c's bit pattern.
//
// A cell with any population outside its weight's binade (strong
// non-equilibrium, high Mach number), or one whose w E_k leaves W_c's binade,
// is updated by the plain FP64 operator instead (the caller reloads its
// populations in the second case: every scheme's step reads and writes a
// cell's slots from the same thread, so they are still in memory).
//
// Wide range (WIDE, a per-lattice mode chosen by the host for flows whose
// populations stray further from the weights, such as a Taylor-Green vortex
// at u0 = 0.05): populations in the binades next to their weights' are taken
// too (f_k / t_k in [0.28, 2.25) for the D3Q19 classes 1/18 and 1/36, [0.42,
// 3.37) on D3Q27), on a grid twice as fine (2^-59, 2^-61): the significand
// is shifted by the population's own exponent.  On D3Q27, whose W_c sit low
// in their binades, a w E_k that leaves W_c's binade for one next to it is
// moved there (rounded to nearest, ties to even, above; exact below) instead
// of sending the cell to the FP64 operator.  The wide code is larger, and
// costs the narrow flows ~2 % when compiled in, so the two are separate
// instantiations.
//
// Both paths, in either mode, compute the update of Section 2.6 to within a
// few FP64 rounding errors; which one a cell takes depends only on its own
// populations and the lattice's mode, so every scheme (they differ only in
// where they load and store) still produces bit-identical results.
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
// the smallest weight (1/36 for D3Q19, 1/216 for D3Q27); half of it in the
// wide mode, so that the binade below each weight's is on the grid too
__host__ __device__ constexpr int fx_grid(int Q, bool wide) { return (Q == 19 ? -58 : -60) - (wide ? 1 : 0); }

// the lattice weight of population K as an FP64 bit pattern, the shift that
// takes its units in the last place to the grid, and its value on the grid
template <int Q, int K, bool WIDE>
struct FxW {
  static constexpr double t = Lat<Q>::w(K);
  static constexpr int e = fx_exp2_floor(t);
  static constexpr long long mant = (long long)(t * fx_pow2(52 - e));  // in [2^52, 2^53)
  static constexpr long long bits = ((long long)(1023 + e) << 52) | (mant - (1LL << 52));
  static constexpr unsigned hi_tag = (unsigned)(1023 + e) << 20;  // sign 0 and the exponent field
  static constexpr int sh = e - 52 - fx_grid(Q, WIDE);
  static_assert(sh >= (WIDE ? 1 : 0) && sh < 8, "weight not representable on the grid");
  static constexpr long long grid = mant << sh;
};

// host: the class constants W_c = w t_c (= wt[c], as bit patterns) and the
// factors that take grid units to W_c's units in the last place
inline void fx_class_constants(int Q, bool wide, const double (&wt)[4], DFK& k) {
  for (int c = 0; c < 4; ++c) {
    const double W = wt[c];
    static_assert(sizeof(double) == sizeof(long long), "64-bit double");
    std::memcpy(&k.wbits[c], &W, sizeof W);
    const int e = W > 0.0 ? fx_exp2_floor(W) : 0;
    k.yscale[c] = (float)fx_pow2(fx_grid(Q, wide) + 52 - e);
  }
}

// wide mode: deviation f - t_K of population K on the grid, exact, when f is
// positive and in t_K's binade or one next to it; otherwise `bad` is set (and
// the value is meaningless)
template <int Q, int K>
__device__ __forceinline__ long long fx_dev_wide(double f, bool& bad) {
  using W = FxW<Q, K, true>;
  // high word relative to that of 2^(e - 1), the bottom of the binade below
  // t_K's: in [0, 3 2^20) for the three binades (a negative f has the sign
  // bit set and falls outside)
  constexpr unsigned LO = (unsigned)(1022 + W::e) << 20;
  const unsigned hi = (unsigned)__double2hiint(f) - LO;
  bad |= hi >= (3u << 20);
  // significand shifted to the grid: by sh - 1, sh or sh + 1
  const unsigned mhi = (hi & 0xfffffu) | 0x100000u;
  const unsigned long long m = ((unsigned long long)mhi << 32) | (unsigned)__double2loint(f);
  return (long long)(m << ((W::sh - 1) + ((hi >> 20) & 3u))) - W::grid;
}

// bit pattern of W_c + (the integer added to W_c's bit pattern), when that sum
// left W_c's binade by one (b: the sum as added, wexp: W_c's biased exponent):
// rounded to nearest, ties to even, in the binade above; exact in the one
// below; `ok` cleared further away
__device__ __forceinline__ long long fx_rebinade(long long b, long long wexp, bool& ok) {
  constexpr long long MASK = (1LL << 52) - 1;
  const long long d = (b >> 52) - wexp;
  const long long w = b & MASK;
  if (d == 1) {
    // b = (wexp + 1, V - 2^53): the significand V in W_c's units, halved
    const long long h = (w >> 1) + (w & (w >> 1) & 1);
    return (b & ~MASK) + h;
  }
  // d == -1: b = (wexp - 1, V) with V < 2^52 in W_c's units; the binade below
  // holds 2 V - 2^52 (needs V >= 2^51)
  ok = ok && d == -1 && w >= (1LL << 51);
  return b + w - (1LL << 52);
}

// nearest integer of a double-float (W_c's last-place units); ok stays true
// while the value is inside the range df_round_i64 handles
__device__ __forceinline__ long long fx_units(DF y, bool& ok) {
  ok = ok && fabsf(y.hi) < 0x1p52f && fabsf(y.lo) < 0x1p30f;
  return df_round_i64(y);
}

// running sums of a summing kernel's cells kept off the FP64 pipe: the density
// deviations rho - 1 and v.j (three times the kinetic energy) in grid units, as
// renormalised double-float sums, and the number of cells (mass = n + r 2^grid,
// kinetic energy = e 2^grid / 3)
struct FxSums {
  DF r, e;
  int n;
};

// add a cell's FP64 sums (the FP64 operator's: rho, kinetic energy) to s
template <int Q, bool WIDE>
__device__ __forceinline__ void fx_sums_add_f64(FxSums& s, double rho, double ke) {
  const double x = (rho - 1.0) * fx_pow2(-fx_grid(Q, WIDE));
  const double y = ke * (3.0 * fx_pow2(-fx_grid(Q, WIDE)));
  const float xh = __double2float_rn(x), yh = __double2float_rn(y);
  s.r = df_renorm(df_add(s.r, DF{xh, __double2float_rn(x - (double)xh)}));
  s.e = df_renorm(df_add(s.e, DF{yh, __double2float_rn(y - (double)yh)}));
  s.n += 1;
}

// mass and kinetic energy of the sums
template <int Q, bool WIDE>
__device__ __forceinline__ void fx_sums_f64(const FxSums& s, double& mass, double& ke) {
  mass = (double)s.n + ((double)s.r.hi + (double)s.r.lo) * fx_pow2(fx_grid(Q, WIDE));
  ke = ((double)s.e.hi + (double)s.e.lo) * (fx_pow2(fx_grid(Q, WIDE)) / 3.0);
}

// outcome of collide_fx
enum FxStatus : int {
  FX_SKIPPED = 0,  // a population out of range: f untouched, use the FP64 operator
  FX_DONE = 1,     // f holds the post-collision populations
  FX_REDO = 2      // some w E_k out of range: f is clobbered, reload it and use the FP64 operator
};

// cs: the cell's FP64 sums (CellSums), or running sums to add the cell to
// (FxSums; added unless the cell is skipped)
template <int Q, bool TRT_, bool WIDE, class S>
__device__ __forceinline__ int collide_fx(double (&f)[Q], const DFK& k_, S* cs) {
  constexpr int H = Lat<Q>::H;
  // on D3Q27 the wide mode also moves w E_k to the binades next to W_c's
  constexpr bool REBINADE = WIDE && Q == 27;
  bool bad = false;
  if constexpr (!WIDE) {
    unsigned acc = 0u;
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      acc |= (unsigned)__double2hiint(f[k]) ^ FxW<Q, k, false>::hi_tag;
    });
    if (acc & 0xfff00000u) return FX_SKIPPED;
  }
  // exact moments on the grid: r = rho - 1, j
  long long r, jx = 0, jy = 0, jz = 0;
  {
    auto dev = [&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (WIDE) return fx_dev_wide<Q, k>(f[k], bad);
      else
        return (long long)((unsigned long long)(__double_as_longlong(f[k]) - FxW<Q, k, false>::bits)
                           << FxW<Q, k, false>::sh);
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
  if constexpr (WIDE) {
    if (bad) return FX_SKIPPED;
  }
  constexpr float GRID = (float)fx_pow2(fx_grid(Q, WIDE));
  // rho = 1 + r, v = 1.5 j / rho (real units); A = r - v.j (grid units)
  const DF dr = i64_to_df(r);
  const DF rho = fast_two_sum(1.0f, fmul(dr.hi, GRID));
  const DF rho_r = {rho.hi, fadd(rho.lo, fmul(dr.lo, GRID))};
  const DF inv15 = df_mulf(df_recip(rho_r), 1.5f);
  DF vx, vy, vz, A;
  {
    const DF Jx = i64_to_df(jx), Jy = i64_to_df(jy), Jz = i64_to_df(jz);
    vx = df_mul(df_scale(Jx, GRID), inv15);
    vy = df_mul(df_scale(Jy, GRID), inv15);
    vz = df_mul(df_scale(Jz, GRID), inv15);
    const DF vj = df_add(df_add(df_mul(vx, Jx), df_mul(vy, Jy)), df_mul(vz, Jz));
    A = df_sub(dr, vj);
    if (cs) {
      // sums of the state read: rho = 1 + r, kinetic energy |j|^2 / (2 rho) = v.j / 3
      if constexpr (std::is_same<S, FxSums>::value) {
        cs->r = df_renorm(df_add(cs->r, dr));
        cs->e = df_renorm(df_add(cs->e, vj));
        cs->n += 1;
      } else {
        cs->rho = __dadd_rn(1.0, __dmul_rn(__ll2double_rn(r), fx_pow2(fx_grid(Q, WIDE))));
        cs->ke = __dmul_rn(__dadd_rn((double)vj.hi, (double)vj.lo), fx_pow2(fx_grid(Q, WIDE)) / 3.0);
      }
    }
  }
  // per weight class c (in W_c's last-place units): the bit pattern of
  // W_c + w t_c A, and 3 w t_c (e.j) = (2 w t_c rho / GRID) (e.v) -- likewise
  // 3 w- t_c (e.j) for TRT -- so that j is no longer needed.  The pairs come in
  // class order (|c|^2 = 1, 2, 3), and each class's constants are formed at
  // its first pair, so that only one class's are live at a time.
  bool ok = true;
  const DF rho2 = df_scale(rho_r, 2.0f / GRID);
  auto base_of = [&](int c) { return k_.wbits[c] + fx_units(df_scale(df_mul(k_.wt[c], A), k_.yscale[c]), ok); };
  long long base = base_of(0);
  DF kq{0.0f, 0.0f}, kqm{0.0f, 0.0f}, kbd{0.0f, 0.0f};
  // w E_k = W_c + w t_c A + (e.v) q +- q, assembled on W_c's bit pattern; the
  // high words of every result are checked against W_c's sign and exponent
  unsigned off = 0u;
  const double omc = k_.omc64;
  {
    long long b0 = base;
    if constexpr (REBINADE) {
      if ((b0 ^ k_.wbits[0]) >> 52) b0 = fx_rebinade(b0, k_.wbits[0] >> 52, ok);
    } else {
      off = (unsigned)((b0 ^ k_.wbits[0]) >> 32);
    }
    f[H] = fma(omc, f[H], __longlong_as_double(b0));
  }
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
    constexpr int c = Lat<Q>::norm2(k);
    static_assert(k == 0 || Lat<Q>::norm2(k - 1) <= c, "pairs in class order");
    if constexpr (k == 0 || Lat<Q>::norm2(k - 1) != c) {
      base = base_of(c);
      kq = df_scale(df_mul(k_.wt[c], rho2), k_.yscale[c]);
      if constexpr (TRT_) {
        kqm = df_scale(df_mul(k_.wm[c], rho2), k_.yscale[c]);
        kbd = df_scale(k_.trt_bdf, k_.yscale[c]);
      }
    }
    // e.v (components of e are -1, 0 or 1)
    DF ev{0.0f, 0.0f};
    bool first = true;
    auto add_c = [&](const DF& v, int sign) {
      const DF sv = sign > 0 ? v : df_neg(v);
      ev = first ? sv : df_add(ev, sv);
      first = false;
    };
    if constexpr (ex != 0) add_c(vx, ex);
    if constexpr (ey != 0) add_c(vy, ey);
    if constexpr (ez != 0) add_c(vz, ez);
    const DF qp = df_mul(kq, ev);                       // 3 w t (e.j), W_c units
    const long long pi = fx_units(df_mul(ev, qp), ok);  // (e.v) 3 w t (e.j)
    const double fp = f[k + H + 1], fm = f[k];
    long long qi;  // antisymmetric part, +- in the pair
    if constexpr (TRT_) {
      // (1-w)/2 (f+ + f-) +- (1-w-)/2 (f+ - f-) = (1 - w) f+- -+ b d, with
      // b = (1-w)/2 - (1-w-)/2 and d = f+ - f- = g+ - g-: the difference of the
      // two bit patterns (both in t_k's binade), exact on the grid; the
      // antisymmetric part 3 w- t (e.j) - b d is rounded once
      long long d;
      if constexpr (WIDE) {
        bool unused = false;  // both passed the range check of the moments
        d = fx_dev_wide<Q, k + H + 1>(fp, unused) - fx_dev_wide<Q, k>(fm, unused);
      } else {
        constexpr int sh = FxW<Q, k, false>::sh;
        d = (long long)((unsigned long long)(__double_as_longlong(fp) - __double_as_longlong(fm)) << sh);
      }
      qi = fx_units(df_sub(df_mul(kqm, ev), df_mul(kbd, i64_to_df(d))), ok);
    } else {
      qi = fx_units(qp, ok);
    }
    long long bp = base + pi + qi, bm = base + pi - qi;
    if constexpr (REBINADE) {
      if (((bp ^ k_.wbits[c]) >> 52) | ((bm ^ k_.wbits[c]) >> 52)) {
        const long long wexp = k_.wbits[c] >> 52;
        if ((bp ^ k_.wbits[c]) >> 52) bp = fx_rebinade(bp, wexp, ok);
        if ((bm ^ k_.wbits[c]) >> 52) bm = fx_rebinade(bm, wexp, ok);
      }
    } else {
      off |= (unsigned)((bp ^ k_.wbits[c]) >> 32) | (unsigned)((bm ^ k_.wbits[c]) >> 32);
    }
    f[k + H + 1] = fma(omc, fp, __longlong_as_double(bp));
    f[k] = fma(omc, fm, __longlong_as_double(bm));
  });
  return (ok && (off & 0xfff00000u) == 0u) ? FX_DONE : FX_REDO;
}

}  // namespace lbm
