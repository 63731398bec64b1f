// collision.cuh -- per-cell collision operators, in registers, for D3Q19/D3Q27.
//
// Collision step f_out = Omega(f) (Section 2.1).  Models (Section 2.2):
//   BGK_W2, BGK_NW4, TRT, REG, RR, RM, HM, CM, CHM, K.
// Moment-based models follow the route of Section 2.6: raw moments
// M_pqr = sum_k c_x^p c_y^q c_z^r f_k, a model-space transform, relaxation
// M* = M - w (M - M_eq) per moment (with the bulk-viscosity coupling of the
// second-order diagonal moments, w- = (w_b - w)/3, w+ = w- + w), back to raw
// moments, and populations rebuilt pairwise (f_k and f_kbar from shared even
// and odd moment sums, as in the f_0 / f_10 example of Section 2.6).
//
// Storage may be shifted (g_k = f_k - t_k, FP32/FP16 modes).  BGK_W2, TRT and
// REG work on the shifted values directly (density deviation drho = sum g);
// the moment models shift at the moment level: M(f) = M(g) + M(t), and the
// rebuilt populations are shifted back by subtracting M(t) before the
// reconstruction, so that the reconstruction only sees deviations.
#pragma once
#include "dfloat.cuh"
#include "fx64.cuh"
#include "lattice.cuh"

namespace lbm {

enum Model : int {
  BGK_W2 = 0, BGK_NW4 = 1, TRT = 2, REG = 3, RR = 4, RM = 5, HM = 6, CM = 7, CHM = 8, KUM = 9,
  // BGK-W2 in the educational form of Section 2.6 (see collide_bgk_w2_edu)
  BGK_W2_EDU = 10, BGK_W2_LOOP = 11
};
constexpr int NUM_MODELS = 12;

// relaxation parameters, prepared on the host
template <typename R>
struct CP {
  R omega;      // shear rate w
  R omc;        // 1 - w
  R wplus;      // bulk coupling w+ = w- + w
  R wminus;     // bulk coupling w- = (w_b - w) / 3
  R omega_high; // rate of moments of order >= 3
  R trt_minus;  // TRT antisymmetric rate from Lambda
  // per weight class c = |c_k|^2: w t_c, 3 w t_c and 3 w- t_c, with (1 - w)/2
  // and (1 - w-)/2 (precomputed on the host for the single-lattice kernels, so
  // that no thread spends FP64 operations on them)
  R wt[4], wt3[4], wm3[4];
  R hs, hd;
  // the FP64 rates split into double-float pairs on the host (used by the FP64
  // BGK-W2 and TRT collisions, which run on the FP32 pipe; see fx64.cuh)
  DFK dk;
};

template <int Q, int K>
inline constexpr int WCLASS = Lat<Q>::norm2(K);

// drho = rho - 1 for shifted storage (kept apart so that FP32 keeps its digits), rho otherwise
template <typename R, bool SH>
__device__ __forceinline__ void cell_sums(CellSums* cs, R drho, R ux, R uy, R uz) {
  if (cs) {
    // in FP64 with rounded intrinsics: no product here is shared with, or fused
    // into, the collision's own arithmetic
    const double rho = SH ? __dadd_rn(1.0, (double)drho) : (double)drho;
    const double x = (double)ux, y = (double)uy, z = (double)uz;
    const double u2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
    cs->rho = rho;
    cs->ke = __dmul_rn(__dmul_rn(0.5, rho), u2);
  }
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
// compile-time constants (variable templates force constant evaluation)
template <int Q, int P, int QQ, int RR_>
inline constexpr int bidx = basis_index(Q, P, QQ, RR_);
template <int Q, int K>
inline constexpr double WGT = Lat<Q>::w(K);
// acc += c * v for a compile-time integer c in {-1, 0, 1, ...}
template <int C, typename R>
__device__ __forceinline__ R addc(R acc, R v) {
  if constexpr (C == 0) return acc;
  else if constexpr (C == 1) return acc + v;
  else if constexpr (C == -1) return acc - v;
  else return acc + R(C) * v;
}

// moments of the lattice weights (rest-state equilibrium): prod_d k_p, k = (1, 0, 1/3)
template <int Q>
__host__ __device__ constexpr double weight_moment(int j) {
  double v = 1.0;
  for (int d = 0; d < 3; ++d) {
    int p = basis_exp(Q, j, d);
    v *= p == 0 ? 1.0 : (p == 1 ? 0.0 : 1.0 / 3.0);
  }
  return v;
}

// ---------------------------------------------------------------------------
// raw moments (un-normalised) of all basis elements from populations
// ---------------------------------------------------------------------------
// pair sums: s_k = f_k + f_kbar, d_k = f_kbar - f_k (kbar = k + H + 1 moves along e_k)
template <int Q, typename R>
__device__ __forceinline__ void pair_sums(const R (&f)[Q], R (&s)[Lat<Q>::H], R (&d)[Lat<Q>::H]) {
  constexpr int H = Lat<Q>::H;
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    s[k] = f[k] + f[k + H + 1];
    d[k] = f[k + H + 1] - f[k];
  });
}

template <int Q, int J, typename R>
__device__ __forceinline__ R raw_moment_pairs(const R (&s)[Lat<Q>::H], const R (&d)[Lat<Q>::H], R frest) {
  constexpr int H = Lat<Q>::H;
  constexpr bool even = (basis_order(Q, J) % 2) == 0;
  R acc = J == 0 ? frest : R(-0.0);
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int c = mono_at_e<Q>(J, k);
    if constexpr (even) acc = addc<c>(acc, s[k]);
    else acc = addc<c>(acc, d[k]);
  });
  return acc;
}

// index (0..Q-1) of the velocity (vx, vy, vz)
template <int Q>
__host__ __device__ constexpr int vel_index(int vx, int vy, int vz) {
  for (int k = 0; k < Q; ++k)
    if (Lat<Q>::c(k, 0) == vx && Lat<Q>::c(k, 1) == vy && Lat<Q>::c(k, 2) == vz) return k;
  return -1;
}

// all Q raw moments.  D3Q19: pair sums.  D3Q27: tensor-product sum
// factorisation, one axis at a time (m0 = f- + f0 + f+, m1 = f+ - f-,
// m2 = f+ + f-).
template <int Q, typename R>
__device__ __forceinline__ void raw_moments(const R (&f)[Q], R (&M)[Q]) {
  if constexpr (Q == 19) {
    R s[9], d[9];
    pair_sums<Q>(f, s, d);
    static_for<0, Q>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      M[J] = raw_moment_pairs<Q, J>(s, d, f[Lat<Q>::REST]);
    });
  } else {
    // A[ix][iy][iz], index 0,1,2 <-> velocity -1,0,+1 before, exponent 0,1,2 after
    R A[3][3][3];
    static_for<0, 27>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int ix = Lat<27>::c(k, 0) + 1, iy = Lat<27>::c(k, 1) + 1, iz = Lat<27>::c(k, 2) + 1;
      A[ix][iy][iz] = f[k];
    });
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        R m = A[0][b][c], z = A[1][b][c], p = A[2][b][c];
        R sp = p + m;
        A[0][b][c] = sp + z;
        A[1][b][c] = p - m;
        A[2][b][c] = sp;
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        R m = A[a][0][c], z = A[a][1][c], p = A[a][2][c];
        R sp = p + m;
        A[a][0][c] = sp + z;
        A[a][1][c] = p - m;
        A[a][2][c] = sp;
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        R m = A[a][b][0], z = A[a][b][1], p = A[a][b][2];
        R sp = p + m;
        A[a][b][0] = sp + z;
        A[a][b][1] = p - m;
        A[a][b][2] = sp;
      }
    static_for<0, 27>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      constexpr int p = basis_exp(27, J, 0), q = basis_exp(27, J, 1), r = basis_exp(27, J, 2);
      M[J] = A[p][q][r];
    });
  }
}

// ---------------------------------------------------------------------------
// populations from un-normalised raw moments: f = T^-1 M
// ---------------------------------------------------------------------------
template <int Q, typename R>
__device__ __forceinline__ void populations_from_raw(const R (&M)[Q], R (&f)[Q]) {
  constexpr int H = Lat<Q>::H;
  if constexpr (Q == 19) {
#define MB(p, q, r) M[bidx<19, p, q, r>]
    const R half = R(0.5), quarter = R(0.25);
    f[H] = MB(0, 0, 0) - MB(2, 0, 0) - MB(0, 2, 0) - MB(0, 0, 2) + MB(2, 2, 0) + MB(2, 0, 2) + MB(0, 2, 2);
    static_for<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int ex = Lat<19>::e(k, 0), ey = Lat<19>::e(k, 1), ez = Lat<19>::e(k, 2);
      R A, B;
      if constexpr (ey == 0 && ez == 0) {  // x axis, e = (1,0,0)
        A = half * (MB(2, 0, 0) - MB(2, 2, 0) - MB(2, 0, 2));
        B = half * (MB(1, 0, 0) - MB(1, 2, 0) - MB(1, 0, 2));
      } else if constexpr (ex == 0 && ez == 0) {  // y axis
        A = half * (MB(0, 2, 0) - MB(2, 2, 0) - MB(0, 2, 2));
        B = half * (MB(0, 1, 0) - MB(2, 1, 0) - MB(0, 1, 2));
      } else if constexpr (ex == 0 && ey == 0) {  // z axis
        A = half * (MB(0, 0, 2) - MB(2, 0, 2) - MB(0, 2, 2));
        B = half * (MB(0, 0, 1) - MB(2, 0, 1) - MB(0, 2, 1));
      } else if constexpr (ez == 0) {  // xy diagonal e = (ex, ey, 0)
        A = quarter * addc<ex * ey>(MB(2, 2, 0), MB(1, 1, 0));
        B = quarter * addc<ey>(R(ex) * MB(1, 2, 0), MB(2, 1, 0));
      } else if constexpr (ey == 0) {  // xz diagonal
        A = quarter * addc<ex * ez>(MB(2, 0, 2), MB(1, 0, 1));
        B = quarter * addc<ez>(R(ex) * MB(1, 0, 2), MB(2, 0, 1));
      } else {  // yz diagonal
        A = quarter * addc<ey * ez>(MB(0, 2, 2), MB(0, 1, 1));
        B = quarter * addc<ez>(R(ey) * MB(0, 1, 2), MB(0, 2, 1));
      }
      f[k + H + 1] = A + B;
      f[k] = A - B;
    });
#undef MB
  } else {
    // inverse of the 1-D transform per axis: f(0) = m0 - m2, f(+-1) = (m2 +- m1) / 2
    R A[3][3][3];
    static_for<0, 27>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      constexpr int p = basis_exp(27, J, 0), q = basis_exp(27, J, 1), r = basis_exp(27, J, 2);
      A[p][q][r] = M[J];
    });
    const R half = R(0.5);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        R m0 = A[0][b][c], m1 = A[1][b][c], m2 = A[2][b][c];
        A[0][b][c] = half * (m2 - m1);
        A[1][b][c] = m0 - m2;
        A[2][b][c] = half * (m2 + m1);
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        R m0 = A[a][0][c], m1 = A[a][1][c], m2 = A[a][2][c];
        A[a][0][c] = half * (m2 - m1);
        A[a][1][c] = m0 - m2;
        A[a][2][c] = half * (m2 + m1);
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        R m0 = A[a][b][0], m1 = A[a][b][1], m2 = A[a][b][2];
        A[a][b][0] = half * (m2 - m1);
        A[a][b][1] = m0 - m2;
        A[a][b][2] = half * (m2 + m1);
      }
    static_for<0, 27>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int ix = Lat<27>::c(k, 0) + 1, iy = Lat<27>::c(k, 1) + 1, iz = Lat<27>::c(k, 2) + 1;
      f[k] = A[ix][iy][iz];
    });
  }
}

// ---------------------------------------------------------------------------
// per-axis transforms of a moment vector (in place); they commute across axes
// ---------------------------------------------------------------------------
template <int Q, int AX>
__host__ __device__ constexpr int shifted_index(int j, int by) {
  int e[3] = {basis_exp(Q, j, 0), basis_exp(Q, j, 1), basis_exp(Q, j, 2)};
  e[AX] -= by;
  return basis_index(Q, e[0], e[1], e[2]);
}

// KIND 0: raw -> central (shift -u), 1: central -> raw (+u),
//      2: monomial -> Hermite (x^2 -> x^2 - cs^2), 3: Hermite -> monomial.
// Only basis elements of total order <= MAXO are transformed.
template <int Q, int AX, int KIND, typename R, int MAXO = 6>
__device__ __forceinline__ void axis_pass(R (&X)[Q], R u) {
  const R cs2 = R(1.0 / 3.0);
  // exponent 2 first (reads the old exponent-1 and exponent-0 entries)
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    if constexpr (basis_exp(Q, J, AX) == 2 && basis_order(Q, J) <= MAXO) {
      constexpr int J1 = shifted_index<Q, AX>(J, 1), J0 = shifted_index<Q, AX>(J, 2);
      if constexpr (KIND == 0) X[J] = X[J] - R(2) * u * X[J1] + u * u * X[J0];
      else if constexpr (KIND == 1) X[J] = X[J] + R(2) * u * X[J1] + u * u * X[J0];
      else if constexpr (KIND == 2) X[J] = X[J] - cs2 * X[J0];
      else X[J] = X[J] + cs2 * X[J0];
    }
  });
  if constexpr (KIND <= 1) {
    static_for<0, Q>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      if constexpr (basis_exp(Q, J, AX) == 1 && basis_order(Q, J) <= MAXO) {
        constexpr int J0 = shifted_index<Q, AX>(J, 1);
        if constexpr (KIND == 0) X[J] = X[J] - u * X[J0];
        else X[J] = X[J] + u * X[J0];
      }
    });
  }
}

template <int Q, int KIND, typename R, int MAXO = 6>
__device__ __forceinline__ void all_axes(R (&X)[Q], R ux, R uy, R uz) {
  axis_pass<Q, 0, KIND, R, MAXO>(X, ux);
  axis_pass<Q, 1, KIND, R, MAXO>(X, uy);
  axis_pass<Q, 2, KIND, R, MAXO>(X, uz);
}

// ---------------------------------------------------------------------------
// relaxation of a moment vector (normalised by rho)
// ---------------------------------------------------------------------------
// HIGH_EQ: orders >= 3 are set to their equilibrium (the omega_high = 1 case,
// where they need not have been computed)
template <int Q, typename R, bool HIGH_EQ = false>
__device__ __forceinline__ void relax(R (&X)[Q], const R (&Xeq)[Q], const CP<R>& p) {
  constexpr int jxx = basis_index(Q, 2, 0, 0), jyy = basis_index(Q, 0, 2, 0), jzz = basis_index(Q, 0, 0, 2);
  const R dx = X[jxx] - Xeq[jxx], dy = X[jyy] - Xeq[jyy], dz = X[jzz] - Xeq[jzz];
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    constexpr int o = basis_order(Q, J);
    if constexpr (o <= 1) {
      X[J] = Xeq[J];
    } else if constexpr (J == jxx) {
      X[J] = X[J] - p.wplus * dx - p.wminus * (dy + dz);
    } else if constexpr (J == jyy) {
      X[J] = X[J] - p.wplus * dy - p.wminus * (dx + dz);
    } else if constexpr (J == jzz) {
      X[J] = X[J] - p.wplus * dz - p.wminus * (dx + dy);
    } else if constexpr (o == 2) {
      X[J] = X[J] - p.omega * (X[J] - Xeq[J]);
    } else if constexpr (HIGH_EQ) {
      X[J] = Xeq[J];
    } else {
      X[J] = X[J] - p.omega_high * (X[J] - Xeq[J]);
    }
  });
}

// ---------------------------------------------------------------------------
// density and velocity through pair sums
// ---------------------------------------------------------------------------
template <int Q, typename R, bool SH>
struct Macro {
  R drho;  // sum of stored values (rho - 1 if shifted, rho otherwise)
  R rho, inv_rho, ux, uy, uz;
};

template <int Q, typename R, bool SH>
__device__ __forceinline__ Macro<Q, R, SH> macro_from_pairs(const R (&s)[Lat<Q>::H], const R (&d)[Lat<Q>::H],
                                                            R frest) {
  constexpr int H = Lat<Q>::H;
  Macro<Q, R, SH> m;
  R r = frest, jx = R(-0.0), jy = R(-0.0), jz = R(-0.0);
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    r = r + s[k];
    jx = addc<Lat<Q>::e(k, 0)>(jx, d[k]);
    jy = addc<Lat<Q>::e(k, 1)>(jy, d[k]);
    jz = addc<Lat<Q>::e(k, 2)>(jz, d[k]);
  });
  m.drho = r;
  m.rho = SH ? R(1) + r : r;
  m.inv_rho = R(1) / m.rho;
  m.ux = jx * m.inv_rho;
  m.uy = jy * m.inv_rho;
  m.uz = jz * m.inv_rho;
  return m;
}

// ---------------------------------------------------------------------------
// mass and momentum kept by the FP32 update.  A collision conserves the
// density and momentum of a cell exactly; rounded to FP32, the update of a
// slowly varying field leaves a small residual change of both that has the same
// sign step after step and piles up (Taylor-Green, 64^2, u0 0.05, omega 1.98:
// L2 velocity error 1.0e-4 after 2000 steps, against 1.2e-7 with the same FP32
// storage and FP64 arithmetic).  The realised change of every population (new
// minus old stored value) is summed into its mass m0 and momentum m, and the
// part of the update that carries them, t_k (m0 + 3 c_k.m), is taken out again
// (sum_k t_k = 1 and sum_k 3 t_k c_k c_k = I, so the corrected change carries
// neither); the error falls to ~2e-7.  Used by BGK-W2 with FP32 storage (in
// FP16 the storage rounding dominates, and the extra work slowed the staged
// step by 12 %; TRT's cavity error is 2.8e-6 without it).
// ---------------------------------------------------------------------------
template <int Q, typename R, bool ON>
struct ConservedFix {
  R m0 = R(0), mx = R(0), my = R(0), mz = R(0);
  // rest population: old value, new value (stored into fo)
  __device__ __forceinline__ void rest(R& f, R fo) {
    if constexpr (ON) m0 = m0 + (fo - f);
    f = fo;
  }
  // pair K: the member along e_K (fp -> new value op) and the one along -e_K
  template <int K>
  __device__ __forceinline__ void pair(R& fp, R op, R& fm, R om) {
    if constexpr (!ON) {
      fp = op;
      fm = om;
      return;
    }
    constexpr int ex = Lat<Q>::e(K, 0), ey = Lat<Q>::e(K, 1), ez = Lat<Q>::e(K, 2);
    const R dp = op - fp, dm = om - fm;
    m0 = m0 + (dp + dm);
    const R dd = dp - dm;
    mx = addc<ex>(mx, dd);
    my = addc<ey>(my, dd);
    mz = addc<ez>(mz, dd);
    fp = op;
    fm = om;
  }
  __device__ __forceinline__ void apply(R (&f)[Q]) {
    if constexpr (!ON) return;
    constexpr int H = Lat<Q>::H;
    f[H] = f[H] - R(WGT<Q, H>) * m0;
    static_for<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
      R em = R(-0.0);
      em = addc<ex>(em, mx);
      em = addc<ey>(em, my);
      em = addc<ez>(em, mz);
      const R a = R(WGT<Q, k>) * m0, b = R(3.0 * WGT<Q, k>) * em;
      f[k + H + 1] = f[k + H + 1] - (a + b);
      f[k] = f[k] - (a - b);
    });
  }
};

// ---------------------------------------------------------------------------
// BGK with the weighted second-order equilibrium (Section 2.6):
//   E_k = rho t_k (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2)
// written per opposite pair as E = t (A + rho(e.u)(4.5 e.u +- 3)),
// A = rho (1 - 1.5 u^2)  (shifted: A = drho - 1.5 rho u^2, giving E - t)
// ---------------------------------------------------------------------------
// KEEP: FP32 storage; the update gives back the mass and momentum its rounding
// created (ConservedFix)
template <int Q, typename R, bool SH, bool KEEP = false>
__device__ __forceinline__ void collide_bgk_w2(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  constexpr int H = Lat<Q>::H;
  R s[H], d[H];
  pair_sums<Q>(f, s, d);
  // density and momentum j = rho u
  R r = f[H], jx = R(-0.0), jy = R(-0.0), jz = R(-0.0);
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    r = r + s[k];
    jx = addc<Lat<Q>::e(k, 0)>(jx, d[k]);
    jy = addc<Lat<Q>::e(k, 1)>(jy, d[k]);
    jz = addc<Lat<Q>::e(k, 2)>(jz, d[k]);
  });
  const R rho = SH ? R(1) + r : r;
  if constexpr (std::is_same<R, double>::value) {
    // FP64 is bound by the FP64 pipe, so the update is arranged for the fewest
    // operations: with v = 1.5 u and q_k = 3 w t_k (e.j),
    //   w E_+- = w t A + (e.v) q_k +- q_k,
    // and relaxes as (1 - w) f + w E
    // (explicit fma / rounded adds: the contraction of products into sums is
    // fixed in the source, so that every kernel instantiating this update,
    // single-lattice or batched, rounds identically)
    const R inv15 = R(1.5) / rho;
    const R vx = jx * inv15, vy = jy * inv15, vz = jz * inv15;
    const R vj = fma(vx, jx, fma(vy, jy, __dmul_rn(vz, jz)));  // 1.5 |j|^2 / rho
    const R A = r - vj;  // rho (1 - 1.5 |u|^2) (shifted: minus 1)
    if (cs) {
      cs->rho = SH ? __dadd_rn(1.0, (double)r) : (double)r;
      cs->ke = __dmul_rn((double)vj, 1.0 / 3.0);
    }
    f[H] = fma(p.omc, f[H], __dmul_rn(p.wt[0], A));
    static_for<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
      constexpr int c = WCLASS<Q, k>;
      R ev = R(-0.0), ej = R(-0.0);
      ev = addc<ex>(ev, vx);
      ev = addc<ey>(ev, vy);
      ev = addc<ez>(ev, vz);
      ej = addc<ex>(ej, jx);
      ej = addc<ey>(ej, jy);
      ej = addc<ez>(ej, jz);
      const R q = __dmul_rn(p.wt3[c], ej);
      const R P = fma(ev, q, __dmul_rn(p.wt[c], A));
      f[k + H + 1] = fma(p.omc, f[k + H + 1], __dadd_rn(P, q));
      f[k] = fma(p.omc, f[k], __dsub_rn(P, q));
    });
  } else {
    // FP32 / FP16 storage: relax in non-equilibrium form f + w (E - f), which
    // keeps the rounding of the large terms out of the small non-equilibrium part
    const R inv = R(1) / rho;
    const R ux = jx * inv, uy = jy * inv, uz = jz * inv;
    // A = rho (1 - 1.5 |u|^2) = rho - 1.5 u.j  (shifted: A - 1 = drho - 1.5 u.j)
    const R uj = ux * jx + uy * jy + uz * jz;
    const R A = r - R(1.5) * uj;
    if (cs) {
      cs->rho = SH ? __dadd_rn(1.0, (double)r) : (double)r;
      cs->ke = __dmul_rn(0.5, (double)uj);
    }
    ConservedFix<Q, R, KEEP> fix;
    fix.rest(f[H], f[H] + p.omega * (R(WGT<Q, H>) * A - f[H]));
    static_for<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
      R eu = R(-0.0), ej = R(-0.0);
      eu = addc<ex>(eu, ux);
      eu = addc<ey>(eu, uy);
      eu = addc<ez>(eu, uz);
      ej = addc<ex>(ej, jx);
      ej = addc<ey>(ej, jy);
      ej = addc<ez>(ej, jz);
      // E_+- = t (A + 4.5 (e.u)(e.j) +- 3 e.j)
      const R t = R(WGT<Q, k>);
      const R S = (R(4.5) * t * eu) * ej + t * A;
      const R T = (R(3) * t) * ej;
      fix.template pair<k>(f[k + H + 1], f[k + H + 1] + p.omega * ((S + T) - f[k + H + 1]), f[k],
                           f[k] + p.omega * ((S - T) - f[k]));
    });
    fix.apply(f);
  }
}

// TRT: symmetric part relaxes with w, antisymmetric part with w- (from Lambda).
// Per opposite pair (plus member along e_k): E+ = t (A + 4.5 (e.u)(e.j)),
// E-_plus = 3 t e.j, with j = rho u and A = rho (1 - 1.5 |u|^2).
template <int Q, typename R, bool SH>
__device__ __forceinline__ void collide_trt(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  constexpr int H = Lat<Q>::H;
  R s[H], d[H];
  pair_sums<Q>(f, s, d);
  R r = f[H], jx = R(-0.0), jy = R(-0.0), jz = R(-0.0);
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    r = r + s[k];
    jx = addc<Lat<Q>::e(k, 0)>(jx, d[k]);
    jy = addc<Lat<Q>::e(k, 1)>(jy, d[k]);
    jz = addc<Lat<Q>::e(k, 2)>(jz, d[k]);
  });
  const R rho = SH ? R(1) + r : r;
  if constexpr (std::is_same<R, double>::value) {
    // fewest FP64 operations: with v = 1.5 u, w E+ = w t A + (e.v) q+ and
    // w- E-_plus = q-, where q+ = 3 w t (e.j) and q- = 3 w- t (e.j); the pair is
    // rebuilt from its symmetric and antisymmetric parts,
    //   X = (1 - w) s/2 + w E+,  Y = (1 - w-) d/2 + w- E-_plus,
    //   f_plus = X + Y,  f_minus = X - Y  (d = f_plus - f_minus, s = f_plus + f_minus)
    // (explicit fma / rounded adds, as in BGK-W2)
    const R inv15 = R(1.5) / rho;
    const R vx = jx * inv15, vy = jy * inv15, vz = jz * inv15;
    const R vj = fma(vx, jx, fma(vy, jy, __dmul_rn(vz, jz)));  // 1.5 |j|^2 / rho
    const R A = r - vj;
    if (cs) {
      cs->rho = SH ? __dadd_rn(1.0, (double)r) : (double)r;
      cs->ke = __dmul_rn((double)vj, 1.0 / 3.0);
    }
    f[H] = fma(p.omc, f[H], __dmul_rn(p.wt[0], A));
    static_for<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
      constexpr int c = WCLASS<Q, k>;
      R ev = R(-0.0), ej = R(-0.0);
      ev = addc<ex>(ev, vx);
      ev = addc<ey>(ev, vy);
      ev = addc<ez>(ev, vz);
      ej = addc<ex>(ej, jx);
      ej = addc<ey>(ej, jy);
      ej = addc<ez>(ej, jz);
      const R qp = __dmul_rn(p.wt3[c], ej);
      const R X = fma(p.hs, s[k], fma(ev, qp, __dmul_rn(p.wt[c], A)));
      const R Y = fma(p.hd, d[k], __dmul_rn(p.wm3[c], ej));
      f[k + H + 1] = X + Y;
      f[k] = X - Y;
    });
  } else {
    const R inv = R(1) / rho;
    const R ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const R uj = ux * jx + uy * jy + uz * jz;
    const R A = r - R(1.5) * uj;
    if (cs) {
      cs->rho = SH ? __dadd_rn(1.0, (double)r) : (double)r;
      cs->ke = __dmul_rn(0.5, (double)uj);
    }
    f[H] = f[H] - p.omega * (f[H] - R(WGT<Q, H>) * A);
    const R hp = R(0.5) * p.omega, hm = R(0.5) * p.trt_minus;
    static_for<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
      R eu = R(-0.0), ej = R(-0.0);
      eu = addc<ex>(eu, ux);
      eu = addc<ey>(eu, uy);
      eu = addc<ez>(eu, uz);
      ej = addc<ex>(ej, jx);
      ej = addc<ey>(ej, jy);
      ej = addc<ez>(ej, jz);
      const R Sp = (R(4.5) * eu) * ej + A;
      const R a = hp * s[k] - (p.omega * R(WGT<Q, k>)) * Sp;      // w+ (f+ - E+)
      const R b = hm * d[k] - (R(3) * p.trt_minus * R(WGT<Q, k>)) * ej;  // w- (f-_plus - E-_plus)
      f[k + H + 1] = f[k + H + 1] - a - b;
      f[k] = f[k] - a + b;
    });
  }
}

// ---------------------------------------------------------------------------
// BGK-W2 in the "educational" form of Section 2.6: density and velocity from
// regrouped partial sums (as above), then one plain loop over the first half
// of the directions that reads c_k and t_k from a table, forms E_k from its
// defining formula and the opposite equilibrium from the symmetry
// E_kbar = E_k - 6 rho t_k c_k.u, and relaxes both populations.  Nothing in
// the loop is unrolled or regrouped by hand.  ROLLED keeps the loop rolled
// (#pragma unroll 1, so f lives in local memory); otherwise the compiler
// decides.  Same equations as collide_bgk_w2, other rounding order.
// ---------------------------------------------------------------------------
template <int Q>
struct EduTable {
  int c[Q][3];
  double t[Q];
};
template <int Q>
constexpr EduTable<Q> make_edu_table() {
  EduTable<Q> T{};
  for (int k = 0; k < Q; ++k) {
    for (int d = 0; d < 3; ++d) T.c[k][d] = Lat<Q>::c(k, d);
    T.t[k] = Lat<Q>::w(k);
  }
  return T;
}
static __constant__ EduTable<19> edu_table19 = make_edu_table<19>();
static __constant__ EduTable<27> edu_table27 = make_edu_table<27>();
template <int Q>
__device__ __forceinline__ const EduTable<Q>& edu_table() {
  if constexpr (Q == 19) return edu_table19;
  else return edu_table27;
}

template <int Q, typename R, bool SH, bool ROLLED>
__device__ __forceinline__ void collide_bgk_w2_edu(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  constexpr int H = Lat<Q>::H;
  R s[H], d[H];
  pair_sums<Q>(f, s, d);
  R r = f[H], jx = R(-0.0), jy = R(-0.0), jz = R(-0.0);
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    r = r + s[k];
    jx = addc<Lat<Q>::e(k, 0)>(jx, d[k]);
    jy = addc<Lat<Q>::e(k, 1)>(jy, d[k]);
    jz = addc<Lat<Q>::e(k, 2)>(jz, d[k]);
  });
  const R rho = SH ? R(1) + r : r;
  const R ux = jx / rho, uy = jy / rho, uz = jz / rho;
  const R usq = ux * ux + uy * uy + uz * uz;
  cell_sums<R, SH>(cs, r, ux, uy, uz);
  const EduTable<Q>& T = edu_table<Q>();
  const R omega = p.omega;
  // rest population: E = rho t (1 - 1.5 |u|^2)
  {
    const R t = R(T.t[H]);
    const R E = rho * t * (R(1) - R(1.5) * usq) - (SH ? t : R(0));
    f[H] = f[H] + omega * (E - f[H]);
  }
  auto pair = [&](int k) {
    const R t = R(T.t[k]);
    const R cu = R(T.c[k][0]) * ux + R(T.c[k][1]) * uy + R(T.c[k][2]) * uz;
    const R Ek = rho * t * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
    const R Ekb = Ek - R(6) * rho * t * cu;
    const R shift = SH ? t : R(0);
    f[k] = f[k] + omega * ((Ek - shift) - f[k]);
    f[k + H + 1] = f[k + H + 1] + omega * ((Ekb - shift) - f[k + H + 1]);
  };
  if constexpr (ROLLED) {
#pragma unroll 1
    for (int k = 0; k < H; ++k) pair(k);
  } else {
    for (int k = 0; k < H; ++k) pair(k);
  }
}

// Regularized: f_out = E + (1 - w) t_k/(2 cs^4) H2_k : Pi_neq,
// Pi_neq = sum_k c c (f - E); W2 equilibrium.
template <int Q, typename R, bool SH>
__device__ __forceinline__ void collide_reg(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  constexpr int H = Lat<Q>::H;
  R s[H], d[H];
  pair_sums<Q>(f, s, d);
  const auto m = macro_from_pairs<Q, R, SH>(s, d, f[H]);
  cell_sums<R, SH>(cs, m.drho, m.ux, m.uy, m.uz);
  R pxx = R(-0.0), pyy = R(-0.0), pzz = R(-0.0), pxy = R(-0.0), pxz = R(-0.0), pyz = R(-0.0);
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
    pxx = addc<ex * ex>(pxx, s[k]);
    pyy = addc<ey * ey>(pyy, s[k]);
    pzz = addc<ez * ez>(pzz, s[k]);
    pxy = addc<ex * ey>(pxy, s[k]);
    pxz = addc<ex * ez>(pxz, s[k]);
    pyz = addc<ey * ez>(pyz, s[k]);
  });
  const R cs2 = R(1.0 / 3.0);
  // equilibrium flux rho (u u + cs2 I); shifted storage removes cs2 I from both sides
  const R iso = SH ? m.drho * cs2 : m.rho * cs2;
  const R nxx = pxx - (m.rho * m.ux * m.ux + iso);
  const R nyy = pyy - (m.rho * m.uy * m.uy + iso);
  const R nzz = pzz - (m.rho * m.uz * m.uz + iso);
  const R nxy = pxy - m.rho * m.ux * m.uy;
  const R nxz = pxz - m.rho * m.ux * m.uz;
  const R nyz = pyz - m.rho * m.uy * m.uz;
  const R tr3 = (nxx + nyy + nzz) * cs2;
  const R usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
  const R A = SH ? m.drho - R(1.5) * m.rho * usq : m.rho * (R(1) - R(1.5) * usq);
  f[H] = R(WGT<Q, H>) * (A + p.omc * R(4.5) * (-tr3));
  static_for<0, H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
    R eu = R(-0.0);
    eu = addc<ex>(eu, m.ux);
    eu = addc<ey>(eu, m.uy);
    eu = addc<ez>(eu, m.uz);
    R q = -tr3;
    q = addc<ex * ex>(q, nxx);
    q = addc<ey * ey>(q, nyy);
    q = addc<ez * ez>(q, nzz);
    q = addc<2 * ex * ey>(q, nxy);
    q = addc<2 * ex * ez>(q, nxz);
    q = addc<2 * ey * ez>(q, nyz);
    const R w = R(WGT<Q, k>);
    const R bk = m.rho * eu;
    const R neq = p.omc * R(4.5) * q;
    f[k + H + 1] = w * (bk * (R(4.5) * eu + R(3)) + A + neq);
    f[k] = w * (bk * (R(4.5) * eu - R(3)) + A + neq);
  });
}

// ---------------------------------------------------------------------------
// moment-space models
// ---------------------------------------------------------------------------
// normalised raw moments of f (from stored values, shifted or not)
template <int Q, typename R, bool SH>
struct MomState {
  R Mh[Q];  // normalised raw moments of f
  R rho, drho, ux, uy, uz;
};

// MAXO = 2: only the moments of order <= 2 are computed (from pair sums); the
// others are left at zero for the caller to overwrite
template <int Q, typename R, bool SH, int MAXO = 6>
__device__ __forceinline__ void load_moments(const R (&f)[Q], MomState<Q, R, SH>& st) {
  R M[Q];
  if constexpr (MAXO >= 6) {
    raw_moments<Q>(f, M);
  } else {
    constexpr int H = Lat<Q>::H;
    R s[H], d[H];
    pair_sums<Q>(f, s, d);
    static_for<0, Q>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      if constexpr (basis_order(Q, J) <= MAXO) M[J] = raw_moment_pairs<Q, J>(s, d, f[H]);
      else M[J] = R(0);
    });
  }
  st.drho = M[0];
  st.rho = SH ? R(1) + M[0] : M[0];
  const R inv = R(1) / st.rho;
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    constexpr double wm = weight_moment<Q>(J);
    if constexpr (J == 0) st.Mh[J] = R(1);
    else if constexpr (basis_order(Q, J) > MAXO) st.Mh[J] = R(0);
    else if constexpr (SH && wm != 0.0) st.Mh[J] = (M[J] + R(wm)) * inv;
    else st.Mh[J] = M[J] * inv;
  });
  st.ux = st.Mh[1];
  st.uy = st.Mh[2];
  st.uz = st.Mh[3];
}

// populations (shifted or not) from post-collision normalised raw moments
template <int Q, typename R, bool SH>
__device__ __forceinline__ void store_moments(const R (&Mh)[Q], const MomState<Q, R, SH>& st, R (&f)[Q]) {
  R M[Q];
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    constexpr double wm = weight_moment<Q>(J);
    if constexpr (J == 0) M[J] = st.drho;
    else if constexpr (SH && wm != 0.0) M[J] = st.rho * Mh[J] - R(wm);
    else M[J] = st.rho * Mh[J];
  });
  populations_from_raw<Q>(M, f);
}

// equilibrium raw moments of the product Maxwellian: prod m_p(u_d), m = (1, u, u^2 + cs2)
template <int Q, typename R>
__device__ __forceinline__ void eq_raw(R ux, R uy, R uz, R (&E)[Q]) {
  const R cs2 = R(1.0 / 3.0);
  const R m2x = ux * ux + cs2, m2y = uy * uy + cs2, m2z = uz * uz + cs2;
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    constexpr int p = basis_exp(Q, J, 0), q = basis_exp(Q, J, 1), r = basis_exp(Q, J, 2);
    R v = R(1);
    if constexpr (p == 1) v = ux;
    if constexpr (p == 2) v = m2x;
    if constexpr (q == 1) v = v * uy;
    if constexpr (q == 2) v = v * m2y;
    if constexpr (r == 1) v = v * uz;
    if constexpr (r == 2) v = v * m2z;
    E[J] = v;
  });
}

// Hermite equilibrium: prod u_d^p
template <int Q, int J, typename R>
__device__ __forceinline__ R uprod(R ux, R uy, R uz) {
  constexpr int p = basis_exp(Q, J, 0), q = basis_exp(Q, J, 1), r = basis_exp(Q, J, 2);
  R v = R(1);
  if constexpr (p == 1) v = ux;
  if constexpr (p == 2) v = ux * ux;
  if constexpr (q == 1) v = v * uy;
  if constexpr (q == 2) v = v * (uy * uy);
  if constexpr (r == 1) v = v * uz;
  if constexpr (r == 2) v = v * (uz * uz);
  return v;
}

template <int Q, typename R, bool SH>
__device__ __forceinline__ void collide_nw4(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  MomState<Q, R, SH> st;
  load_moments<Q, R, SH>(f, st);
  cell_sums<R, SH>(cs, st.drho, st.ux, st.uy, st.uz);
  R E[Q], feq[Q];
  eq_raw<Q>(st.ux, st.uy, st.uz, E);
  store_moments<Q, R, SH>(E, st, feq);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    f[k] = f[k] + p.omega * (feq[k] - f[k]);
  });
}

template <int Q, typename R, bool SH, bool HEQ>
__device__ __forceinline__ void collide_rm_impl(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  MomState<Q, R, SH> st;
  load_moments<Q, R, SH, HEQ ? 2 : 6>(f, st);
  cell_sums<R, SH>(cs, st.drho, st.ux, st.uy, st.uz);
  R E[Q];
  eq_raw<Q>(st.ux, st.uy, st.uz, E);
  relax<Q, R, HEQ>(st.Mh, E, p);
  store_moments<Q, R, SH>(st.Mh, st, f);
}
template <int Q, typename R, bool SH>
__device__ __forceinline__ void collide_rm(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  if (p.omega_high == R(1)) collide_rm_impl<Q, R, SH, true>(f, p, cs);
  else collide_rm_impl<Q, R, SH, false>(f, p, cs);
}

template <int Q, typename R, bool SH, bool HEQ>
__device__ __forceinline__ void collide_hm_impl(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  MomState<Q, R, SH> st;
  load_moments<Q, R, SH, HEQ ? 2 : 6>(f, st);
  cell_sums<R, SH>(cs, st.drho, st.ux, st.uy, st.uz);
  all_axes<Q, 2, R, HEQ ? 2 : 6>(st.Mh, st.ux, st.uy, st.uz);  // monomial -> Hermite
  R E[Q];
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    E[J] = uprod<Q, J>(st.ux, st.uy, st.uz);
  });
  relax<Q, R, HEQ>(st.Mh, E, p);
  all_axes<Q, 3>(st.Mh, st.ux, st.uy, st.uz);  // Hermite -> monomial
  store_moments<Q, R, SH>(st.Mh, st, f);
}
template <int Q, typename R, bool SH>
__device__ __forceinline__ void collide_hm(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  if (p.omega_high == R(1)) collide_hm_impl<Q, R, SH, true>(f, p, cs);
  else collide_hm_impl<Q, R, SH, false>(f, p, cs);
}

// central-moment equilibrium prod k_p, k = (1, 0, cs2)
template <int Q, typename R>
__device__ __forceinline__ void eq_central(R (&E)[Q]) {
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    constexpr double wm = weight_moment<Q>(J);
    E[J] = R(wm);
  });
}

template <int Q, typename R, bool SH, bool HEQ>
__device__ __forceinline__ void collide_cm_impl(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  MomState<Q, R, SH> st;
  load_moments<Q, R, SH, HEQ ? 2 : 6>(f, st);
  cell_sums<R, SH>(cs, st.drho, st.ux, st.uy, st.uz);
  const R ux = st.ux, uy = st.uy, uz = st.uz;
  all_axes<Q, 0, R, HEQ ? 2 : 6>(st.Mh, ux, uy, uz);  // raw -> central
  R E[Q];
  eq_central<Q>(E);
  relax<Q, R, HEQ>(st.Mh, E, p);
  all_axes<Q, 1>(st.Mh, ux, uy, uz);  // central -> raw
  st.Mh[1] = ux;
  st.Mh[2] = uy;
  st.Mh[3] = uz;
  store_moments<Q, R, SH>(st.Mh, st, f);
}
template <int Q, typename R, bool SH>
__device__ __forceinline__ void collide_cm(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  if (p.omega_high == R(1)) collide_cm_impl<Q, R, SH, true>(f, p, cs);
  else collide_cm_impl<Q, R, SH, false>(f, p, cs);
}

template <int Q, typename R, bool SH, bool HEQ>
__device__ __forceinline__ void collide_chm_impl(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  MomState<Q, R, SH> st;
  load_moments<Q, R, SH, HEQ ? 2 : 6>(f, st);
  cell_sums<R, SH>(cs, st.drho, st.ux, st.uy, st.uz);
  const R ux = st.ux, uy = st.uy, uz = st.uz;
  all_axes<Q, 0, R, HEQ ? 2 : 6>(st.Mh, ux, uy, uz);  // raw -> central
  all_axes<Q, 2, R, HEQ ? 2 : 6>(st.Mh, ux, uy, uz);  // central monomial -> central Hermite
  R E[Q];
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    E[J] = J == 0 ? R(1) : R(0);
  });
  relax<Q, R, HEQ>(st.Mh, E, p);
  all_axes<Q, 3>(st.Mh, ux, uy, uz);  // central Hermite -> central monomial
  all_axes<Q, 1>(st.Mh, ux, uy, uz);  // central -> raw
  st.Mh[1] = ux;
  st.Mh[2] = uy;
  st.Mh[3] = uz;
  store_moments<Q, R, SH>(st.Mh, st, f);
}
template <int Q, typename R, bool SH>
__device__ __forceinline__ void collide_chm(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  if (p.omega_high == R(1)) collide_chm_impl<Q, R, SH, true>(f, p, cs);
  else collide_chm_impl<Q, R, SH, false>(f, p, cs);
}

// cumulants of orders 4..6 from normalised central moments (lower orders
// coincide with central moments since first central moments vanish);
// FWD = true: kappa -> K, FWD = false: K -> kappa.
template <int Q, bool FWD, typename R>
__device__ __forceinline__ void cumulant_high(R (&X)[Q]) {
#define IX(p, q, r) bidx<Q, p, q, r>
  const R k200 = X[IX(2, 0, 0)], k020 = X[IX(0, 2, 0)], k002 = X[IX(0, 0, 2)];
  const R k110 = X[IX(1, 1, 0)], k101 = X[IX(1, 0, 1)], k011 = X[IX(0, 1, 1)];
  const R sg = FWD ? R(-1) : R(1);
  X[IX(2, 2, 0)] = X[IX(2, 2, 0)] + sg * (k200 * k020 + R(2) * k110 * k110);
  X[IX(2, 0, 2)] = X[IX(2, 0, 2)] + sg * (k200 * k002 + R(2) * k101 * k101);
  X[IX(0, 2, 2)] = X[IX(0, 2, 2)] + sg * (k020 * k002 + R(2) * k011 * k011);
  if constexpr (Q == 27) {
    const R k120 = X[IX(1, 2, 0)], k102 = X[IX(1, 0, 2)], k210 = X[IX(2, 1, 0)];
    const R k012 = X[IX(0, 1, 2)], k201 = X[IX(2, 0, 1)], k021 = X[IX(0, 2, 1)], k111 = X[IX(1, 1, 1)];
    // fourth order, mixed
    X[IX(2, 1, 1)] = X[IX(2, 1, 1)] + sg * (k200 * k011 + R(2) * k110 * k101);
    X[IX(1, 2, 1)] = X[IX(1, 2, 1)] + sg * (k020 * k101 + R(2) * k110 * k011);
    X[IX(1, 1, 2)] = X[IX(1, 1, 2)] + sg * (k002 * k110 + R(2) * k101 * k011);
    // fifth order: pair x triple partitions
    X[IX(2, 2, 1)] = X[IX(2, 2, 1)] + sg * (k200 * k021 + k020 * k201 + R(4) * k110 * k111 + R(2) * k101 * k120 +
                                            R(2) * k011 * k210);
    X[IX(2, 1, 2)] = X[IX(2, 1, 2)] + sg * (k200 * k012 + k002 * k210 + R(4) * k101 * k111 + R(2) * k110 * k102 +
                                            R(2) * k011 * k201);
    X[IX(1, 2, 2)] = X[IX(1, 2, 2)] + sg * (k002 * k120 + k020 * k102 + R(4) * k011 * k111 + R(2) * k101 * k021 +
                                            R(2) * k110 * k012);
    // sixth order: pair x quadruple (quadruple as cumulant), triple x triple, pair x pair x pair
    const R K220 = FWD ? X[IX(2, 2, 0)] : X[IX(2, 2, 0)] - (k200 * k020 + R(2) * k110 * k110);
    const R K202 = FWD ? X[IX(2, 0, 2)] : X[IX(2, 0, 2)] - (k200 * k002 + R(2) * k101 * k101);
    const R K022 = FWD ? X[IX(0, 2, 2)] : X[IX(0, 2, 2)] - (k020 * k002 + R(2) * k011 * k011);
    const R K211 = FWD ? X[IX(2, 1, 1)] : X[IX(2, 1, 1)] - (k200 * k011 + R(2) * k110 * k101);
    const R K121 = FWD ? X[IX(1, 2, 1)] : X[IX(1, 2, 1)] - (k020 * k101 + R(2) * k110 * k011);
    const R K112 = FWD ? X[IX(1, 1, 2)] : X[IX(1, 1, 2)] - (k002 * k110 + R(2) * k101 * k011);
    const R s24 = k200 * K022 + k020 * K202 + k002 * K220 + R(4) * (k110 * K112 + k101 * K121 + k011 * K211);
    const R s33 = R(2) * (k210 * k012 + k201 * k021 + k120 * k102) + R(4) * k111 * k111;
    const R s222 = k200 * k020 * k002 + R(2) * (k200 * k011 * k011 + k020 * k101 * k101 + k002 * k110 * k110) +
                   R(8) * k110 * k101 * k011;
    X[IX(2, 2, 2)] = X[IX(2, 2, 2)] + sg * (s24 + s33 + s222);
  }
#undef IX
}

template <int Q, typename R, bool SH, bool HEQ>
__device__ __forceinline__ void collide_k_impl(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  MomState<Q, R, SH> st;
  load_moments<Q, R, SH, HEQ ? 2 : 6>(f, st);
  cell_sums<R, SH>(cs, st.drho, st.ux, st.uy, st.uz);
  const R ux = st.ux, uy = st.uy, uz = st.uz;
  all_axes<Q, 0, R, HEQ ? 2 : 6>(st.Mh, ux, uy, uz);  // raw -> central
  if constexpr (!HEQ) cumulant_high<Q, true>(st.Mh);   // central -> cumulant (orders 4..6)
  R E[Q];
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    constexpr int o = basis_order(Q, J);
    constexpr bool diag2 = o == 2 && (basis_exp(Q, J, 0) == 2 || basis_exp(Q, J, 1) == 2 || basis_exp(Q, J, 2) == 2);
    E[J] = J == 0 ? R(1) : (diag2 ? R(1.0 / 3.0) : R(0));
  });
  relax<Q, R, HEQ>(st.Mh, E, p);
  cumulant_high<Q, false>(st.Mh);     // cumulant -> central
  all_axes<Q, 1>(st.Mh, ux, uy, uz);  // central -> raw
  st.Mh[1] = ux;
  st.Mh[2] = uy;
  st.Mh[3] = uz;
  store_moments<Q, R, SH>(st.Mh, st, f);
}
template <int Q, typename R, bool SH>
__device__ __forceinline__ void collide_k(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  if (p.omega_high == R(1)) collide_k_impl<Q, R, SH, true>(f, p, cs);
  else collide_k_impl<Q, R, SH, false>(f, p, cs);
}

// Recursive regularized (Hermite form): second-order non-equilibrium Hermite
// moments relaxed; every higher basis moment = prod u + recursion on the
// post-collision second-order non-equilibrium a2*:
//   a_pqr = C(p,2) u^(p-2,q,r) a_xx + C(q,2) ... + p q u^(p-1,q-1,r) a_xy + ...
template <int Q, typename R, bool SH>
__device__ __forceinline__ void collide_rr(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  MomState<Q, R, SH> st;
  load_moments<Q, R, SH>(f, st);
  cell_sums<R, SH>(cs, st.drho, st.ux, st.uy, st.uz);
  const R ux = st.ux, uy = st.uy, uz = st.uz;
  const R cs2 = R(1.0 / 3.0);
#define IX(a, b, c) bidx<Q, a, b, c>
  // non-equilibrium of the second-order Hermite moments
  const R nxx = st.Mh[IX(2, 0, 0)] - cs2 - ux * ux;
  const R nyy = st.Mh[IX(0, 2, 0)] - cs2 - uy * uy;
  const R nzz = st.Mh[IX(0, 0, 2)] - cs2 - uz * uz;
  const R nxy = st.Mh[IX(1, 1, 0)] - ux * uy;
  const R nxz = st.Mh[IX(1, 0, 1)] - ux * uz;
  const R nyz = st.Mh[IX(0, 1, 1)] - uy * uz;
  const R axx = nxx - p.wplus * nxx - p.wminus * (nyy + nzz);
  const R ayy = nyy - p.wplus * nyy - p.wminus * (nxx + nzz);
  const R azz = nzz - p.wplus * nzz - p.wminus * (nxx + nyy);
  const R axy = p.omc * nxy, axz = p.omc * nxz, ayz = p.omc * nyz;
#undef IX
  R X[Q];
  static_for<0, Q>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    constexpr int a = basis_exp(Q, J, 0), b = basis_exp(Q, J, 1), c = basis_exp(Q, J, 2);
    constexpr int o = a + b + c;
    R v = uprod<Q, J>(ux, uy, uz);
    if constexpr (o == 2) {
      if constexpr (a == 2) v = v + axx;
      else if constexpr (b == 2) v = v + ayy;
      else if constexpr (c == 2) v = v + azz;
      else if constexpr (a == 1 && b == 1) v = v + axy;
      else if constexpr (a == 1 && c == 1) v = v + axz;
      else v = v + ayz;
    } else if constexpr (o >= 3) {
      // u-monomial with exponents reduced by the pair's axes
      auto um = [&](int da, int db, int dc) {
        R r = R(1);
        for (int i = 0; i < a - da; ++i) r = r * ux;
        for (int i = 0; i < b - db; ++i) r = r * uy;
        for (int i = 0; i < c - dc; ++i) r = r * uz;
        return r;
      };
      R acc = R(-0.0);
      if constexpr (a == 2) acc = acc + um(2, 0, 0) * axx;
      if constexpr (b == 2) acc = acc + um(0, 2, 0) * ayy;
      if constexpr (c == 2) acc = acc + um(0, 0, 2) * azz;
      if constexpr (a >= 1 && b >= 1) acc = acc + R(a * b) * um(1, 1, 0) * axy;
      if constexpr (a >= 1 && c >= 1) acc = acc + R(a * c) * um(1, 0, 1) * axz;
      if constexpr (b >= 1 && c >= 1) acc = acc + R(b * c) * um(0, 1, 1) * ayz;
      v = v + acc;
    }
    X[J] = v;
  });
  all_axes<Q, 3>(X, ux, uy, uz);  // Hermite -> monomial
  X[0] = R(1);
  store_moments<Q, R, SH>(X, st, f);
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
// models and storage with the FP32-pipe FP64 operator of fx64.cuh (tried first;
// the operators below take the cells it declines)
template <int M, typename R, bool SH>
inline constexpr bool HAS_FX = (M == BGK_W2 || M == TRT) && std::is_same<R, double>::value && !SH;

// cs (optional): receives the cell's share of the conserved sums, computed from
// the pre-collision moments
// KEEP: FP32 storage (see ConservedFix)
template <int Q, int M, typename R, bool SH, bool KEEP = false>
__device__ __forceinline__ void collide(R (&f)[Q], const CP<R>& p, CellSums* cs = nullptr) {
  if constexpr (M == BGK_W2) collide_bgk_w2<Q, R, SH, KEEP>(f, p, cs);
  else if constexpr (M == BGK_NW4) collide_nw4<Q, R, SH>(f, p, cs);
  else if constexpr (M == TRT) collide_trt<Q, R, SH>(f, p, cs);
  else if constexpr (M == REG) collide_reg<Q, R, SH>(f, p, cs);
  else if constexpr (M == RR) collide_rr<Q, R, SH>(f, p, cs);
  else if constexpr (M == RM) collide_rm<Q, R, SH>(f, p, cs);
  else if constexpr (M == HM) collide_hm<Q, R, SH>(f, p, cs);
  else if constexpr (M == CM) collide_cm<Q, R, SH>(f, p, cs);
  else if constexpr (M == CHM) collide_chm<Q, R, SH>(f, p, cs);
  else if constexpr (M == BGK_W2_EDU) collide_bgk_w2_edu<Q, R, SH, false>(f, p, cs);
  else if constexpr (M == BGK_W2_LOOP) collide_bgk_w2_edu<Q, R, SH, true>(f, p, cs);
  else collide_k<Q, R, SH>(f, p, cs);
}

// the model's own equilibrium of (rho, u), in stored form (shifted or not);
// drho = rho - 1 for shifted storage (formed by the caller in FP64 so that the
// density deviation keeps its precision), rho otherwise
template <int Q, int M, typename R, bool SH>
__device__ __forceinline__ void equilibrium(R rho, R drho, R ux, R uy, R uz, R (&f)[Q]) {
  constexpr int H = Lat<Q>::H;
  if constexpr (M == BGK_W2 || M == TRT || M == REG || M == BGK_W2_EDU || M == BGK_W2_LOOP) {
    const R usq = ux * ux + uy * uy + uz * uz;
    const R A = SH ? drho - R(1.5) * rho * usq : rho * (R(1) - R(1.5) * usq);
    f[H] = R(WGT<Q, H>) * A;
    static_for<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      R eu = R(-0.0);
      eu = addc<Lat<Q>::e(k, 0)>(eu, ux);
      eu = addc<Lat<Q>::e(k, 1)>(eu, uy);
      eu = addc<Lat<Q>::e(k, 2)>(eu, uz);
      const R bk = rho * eu, w = R(WGT<Q, k>);
      f[k + H + 1] = w * (bk * (R(4.5) * eu + R(3)) + A);
      f[k] = w * (bk * (R(4.5) * eu - R(3)) + A);
    });
  } else {
    MomState<Q, R, SH> st;
    st.rho = rho;
    st.drho = drho;
    R E[Q];
    eq_raw<Q>(ux, uy, uz, E);
    store_moments<Q, R, SH>(E, st, f);
  }
}

}  // namespace lbm
