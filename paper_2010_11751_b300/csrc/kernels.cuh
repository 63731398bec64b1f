// kernels.cuh -- fused stream-and-collide kernels for the four memory-access
// schemes, plus the state-access kernels (macroscopic fields, canonical
// get/set, equilibrium initialisation, FP64 conserved sums, swap streaming).
//
// One thread per cell, cell index i = (x*ny + y)*nz + z (z fastest, so the
// Q population streams of the SoA layout are coalesced along z).
//
// Schemes (Section 2.3, Table 1 of the paper), with the wall term of the
// bounce-back rule  f_kbar(x, t+1) = f_out_k(x) - 6 t_k rho_w c_k.u_w
// (Section 2.1) added at the moment the reflected population is written, so
// that between steps every scheme stores an exact permutation of the
// canonical populations:
//   TWOPOP  read pop_k(x); write out_k(x + c_k), or out_kbar(x) = f_out_k + W_k
//           if x + c_k is solid.                        (Table 1, row 2Pop)
//   AA even read pop_k(x); write pop_kbar(x) = f_out_k (+ W_k if x + c_k solid).
//           The swap scheme's collision pass is this same kernel.
//   AA odd  read f_k(x) = pop_kbar(x - c_k) if x - c_k is fluid, else pop_k(x);
//           write pop_k(x + c_k) = f_out_k if fluid, else pop_kbar(x) = f_out_k + W_k.
//           (Table 1 AA rows; the pull side reads the neighbour in -c_k, the
//           only reading consistent with the even step's storage rule.)
//   ESOTWIST (Geier & Schoenherr 2017)  physical slot of label k at parity p:
//           k (p even) or kbar (p odd).  Read f_k(x) at cell x - max(c_k, 0)
//           from slot(k) (slot(kbar) if x - c_k is solid); write f_out_k to
//           slot(kbar) at cell x + min(c_k, 0).  Same kernel every step.
//   SWAP stream: for the first-half directions k, swap pop_kbar(x) with
//           pop_k(x + c_k) when both cells are fluid.   (Table 1, row Swap)
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "collision.cuh"
#include "debug.cuh"
#include "fx_rr.cuh"

namespace lbm {

enum Layout : int { SOA = 0, AOS = 1 };
enum StepKind : int { K_TWOPOP = 0, K_AA_EVEN = 1, K_AA_ODD = 2, K_ESOTWIST = 3, NUM_STEP_KINDS = 4 };
// where the canonical pre-collision populations are found
enum LoadKind : int { LD_LOCAL = 0, LD_AA_ODD = 1, LD_ET_EVEN = 2, LD_ET_ODD = 3, NUM_LOAD_KINDS = 4 };

struct KArgs {
  void* a;                // populations (current state)
  void* b;                // destination array of the two-population scheme
  const uint8_t* flags;   // classified flag bytes
  const uint32_t* nbmask; // per fluid cell: bit k set when the neighbour along c_k is solid (k < 27);
                          // NBMASK_UNIFORM: all those neighbours share the wall kind in bits 27-29
  const double* wall;     // wall term table [8][Q]: -6 t_k c_k.u_w(kind)
  int nx, ny, nz, N;
  int parity;             // time-step parity (esoteric twist slot labels)
  double omega, omc, wplus, wminus, omega_high, trt_minus;
  // per weight class c = |c|^2: w t_c, 3 w t_c, 3 w- t_c; and (1 - w)/2, (1 - w-)/2
  double wt[4], wt3[4], wm3[4], hs, hd;
  DFK dk;  // the same rates as double-float pairs (derived_dfk)
  // walls at a fraction of their links: per cell the row of qtab holding its Q
  // link fractions (-1: none), or null when the lattice has no such walls
  const int* qidx;
  const double* qtab;
  // FP64 BGK-W2 / TRT: 1 when the lattice runs the wide range of fx64.cuh
  // (a host decision per lattice; the launchers pick the kernel instantiation)
  int fx_wide;
#ifdef LBM_DEBUG
  unsigned long long* dbg;  // first failed bounds check (debug.cuh)
  size_t dbg_elems;         // populations in the array: Q N
  int dbg_qrows;            // rows of qtab
#endif
};

// rate constants derived from w and w- (on the host: the kernels' launch
// parameters and the batch member table)
template <int Q>
__host__ __device__ inline void derived_rates(double omega, double trt_minus, double (&wt)[4], double (&wt3)[4],
                                              double (&wm3)[4], double& hs, double& hd) {
  for (int c = 0; c < 4; ++c) {
    double t = 0.0;
    for (int k = 0; k < Q; ++k)
      if (Lat<Q>::norm2(k) == c) t = Lat<Q>::w(k);
    wt[c] = omega * t;
    wt3[c] = 3.0 * (omega * t);
    wm3[c] = (3.0 * trt_minus) * t;
  }
  hs = 0.5 * (1.0 - omega);
  hd = 0.5 * (1.0 - trt_minus);
}

// the FP64 rates prepared for the FP32-pipe FP64 collisions (host)
template <int Q>
inline DFK derived_dfk(double omc, const double (&wt)[4], const double (&wt3)[4], const double (&wm3)[4], double hs,
                       double hd, double wplus, double wminus, bool wide) {
  DFK k;
  k.omc = df_split(omc);
  k.hs = df_split(hs);
  k.hd = df_split(hd);
  k.pad = {0.0f, 0.0f};
  for (int c = 0; c < 4; ++c) {
    k.wt[c] = df_split(wt[c]);
    k.wt3[c] = df_split(wt3[c]);
    k.wm3[c] = df_split(wm3[c]);
    k.wm[c] = df_split(wm3[c] / 3.0);
  }
  fx_class_constants(Q, wide, wt, k);
  k.omc64 = omc;
  k.trt_a = hs + hd;
  k.trt_b = hs - hd;
  k.trt_bdf = df_split(hs - hd);
  k.wplus = df_split(wplus);
  k.wminus = df_split(wminus);
  k.pad2 = {0.0f, 0.0f};
  return k;
}

// ---------------------------------------------------------------------------
// population addressing
// ---------------------------------------------------------------------------
template <int Q, int L>
__device__ __forceinline__ size_t paddr(int k, int i, int N) {
  LBM_IF_DEBUG(if ((unsigned)i >= (unsigned)N || (unsigned)k >= (unsigned)Q) return DBG_BAD_ADDR;)
  if constexpr (L == SOA) return (size_t)k * (size_t)N + (size_t)i;
  else return (size_t)i * Q + (size_t)k;
}

// population load / store at element ad of the array at base (a: the step's
// arguments, whose bounds the debug build checks)
template <int P>
__device__ __forceinline__ typename Store<P>::R ldp(const KArgs& a, const void* base, size_t ad) {
  using S = typename Store<P>::S;
  LBM_IF_DEBUG(if (ad >= a.dbg_elems) {
    dbg_fault(a.dbg, DBG_POP_LOAD, ad);
    return typename Store<P>::R(0);
  })
  if constexpr (P == F16) return __half2float(reinterpret_cast<const __half*>(base)[ad]);
  else return Store<P>::to_r(__ldg(reinterpret_cast<const S*>(base) + ad));
}
template <int P>
__device__ __forceinline__ void stp(const KArgs& a, void* base, size_t ad, typename Store<P>::R v) {
  using S = typename Store<P>::S;
  LBM_IF_DEBUG(if (ad >= a.dbg_elems) {
    dbg_fault(a.dbg, DBG_POP_STORE, ad);
    return;
  })
  reinterpret_cast<S*>(base)[ad] = Store<P>::from_r(v);
}

// ---------------------------------------------------------------------------
// neighbour access: FAST = interior bulk cell (no wrap, no solid neighbour).
// Otherwise the cell's solid-neighbour mask tells which links bounce (a
// neighbour's flag byte is read only for those, to find its wall kind), and
// coordinates with periodic wrap are computed only for cells on a domain face.
// ---------------------------------------------------------------------------
template <bool FAST>
struct Nb {
  int i, x, y, z;
  int nx, ny, nz, sxy;
  bool edge;
  bool curved;  // some of the cell's walls sit at a fraction of their links (qidx / qtab)
  uint32_t mask;
  const uint8_t* flags;
#ifdef LBM_DEBUG
  unsigned long long* dbg;
  int ncell;
#endif
  // neighbourhood of cell i_ from its flag byte (the solid-neighbour mask is
  // read from a.nbmask for cells next to a wall)
  __device__ __forceinline__ Nb(int i_, const KArgs& a, uint8_t fl = 0)
      : i(i_), nx(a.nx), ny(a.ny), nz(a.nz), flags(a.flags) {
    LBM_IF_DEBUG(dbg = a.dbg; ncell = a.N;)
    sxy = a.ny * a.nz;
    x = y = z = 0;
    if constexpr (FAST) {
      edge = false;
      mask = 0u;
      curved = false;
    } else {
      edge = (fl & FLAG_EDGE) != 0;
      LBM_IF_DEBUG(if ((fl & FLAG_NEARWALL) && (unsigned)i >= (unsigned)a.N) {
        dbg_fault(a.dbg, DBG_MASK, (unsigned)i);
        fl = 0;
      })
      mask = (fl & FLAG_NEARWALL) ? __ldg(a.nbmask + i) : 0u;
      curved = (mask & NBMASK_CURVED) != 0u;
      mask &= ~NBMASK_CURVED;
      if (edge) {
        x = i / sxy;
        const int r = i - x * sxy;
        y = r / nz;
        z = r - y * nz;
      }
    }
  }
  // neighbourhood of cell i_ from a given solid-neighbour mask and domain-face bit
  __device__ __forceinline__ Nb(int i_, const KArgs& a, bool edge_, uint32_t mask_)
      : i(i_), nx(a.nx), ny(a.ny), nz(a.nz), flags(a.flags) {
    static_assert(!FAST, "bulk cells have neither solid neighbours nor wrap");
    LBM_IF_DEBUG(dbg = a.dbg; ncell = a.N;)
    sxy = a.ny * a.nz;
    x = y = z = 0;
    edge = edge_;
    mask = mask_;
    curved = false;
    if (edge) {
      x = i / sxy;
      const int r = i - x * sxy;
      y = r / nz;
      z = r - y * nz;
    }
  }
  // index of the cell at offset (dx, dy, dz), periodic
  template <int DX, int DY, int DZ>
  __device__ __forceinline__ int at() const {
    if constexpr (FAST) {
      return i + DX * sxy + DY * nz + DZ;
    } else {
      if (!edge) return i + DX * sxy + DY * nz + DZ;
      int xn = x + DX, yn = y + DY, zn = z + DZ;
      if constexpr (DX != 0) xn = xn < 0 ? xn + nx : (xn >= nx ? xn - nx : xn);
      if constexpr (DY != 0) yn = yn < 0 ? yn + ny : (yn >= ny ? yn - ny : yn);
      if constexpr (DZ != 0) zn = zn < 0 ? zn + nz : (zn >= nz ? zn - nz : zn);
      return (xn * ny + yn) * nz + zn;
    }
  }
  // is the neighbour along c_k solid? (from the mask alone: no memory access)
  template <int Q, int K>
  __device__ __forceinline__ bool solid() const {
    if constexpr (FAST) return false;
    else return ((mask >> K) & 1u) != 0;
  }
  // wall kind of a solid neighbour along c_k: from the mask word when all the
  // cell's solid neighbours share one kind, else from the neighbour's flag byte
  template <int Q, int K>
  __device__ __forceinline__ int kind() const {
    if (mask & NBMASK_UNIFORM) return (int)((mask >> NBMASK_KIND_SHIFT) & FLAG_KIND);
    const int j = at<Lat<Q>::c(K, 0), Lat<Q>::c(K, 1), Lat<Q>::c(K, 2)>();
    LBM_IF_DEBUG(if ((unsigned)j >= (unsigned)ncell) {
      dbg_fault(dbg, DBG_FLAG, (unsigned)j);
      return 0;
    })
    return flags[j] & FLAG_KIND;
  }
  template <int Q, int K>
  __device__ __forceinline__ int idx() const {
    return at<Lat<Q>::c(K, 0), Lat<Q>::c(K, 1), Lat<Q>::c(K, 2)>();
  }
};

// neighbourhood of a listed cell from its record (solid mask, domain-face bit
// and the wall kind of every solid neighbour, 3 bits per link: links 0..20 in
// kinds0, 21..26 in kinds1), so that no flag byte is read
struct NbRec : Nb<false> {
  unsigned long long kinds0, kinds1;
  __device__ __forceinline__ NbRec(int i_, const KArgs& a, uint32_t mask_edge, unsigned long long k0,
                                   unsigned long long k1)
      : Nb<false>(i_, a, (mask_edge >> 31) != 0u, mask_edge & 0x7fffffffu), kinds0(k0), kinds1(k1) {
    curved = (k1 >> 63) != 0ull;
  }
  template <int Q, int K>
  __device__ __forceinline__ int kind() const {
    if constexpr (K < 21) return (int)((kinds0 >> (3 * K)) & 7ull);
    else return (int)((kinds1 >> (3 * (K - 21))) & 7ull);
  }
};

template <int Q, int K>
__host__ __device__ constexpr int cpos(int d) { return Lat<Q>::c(K, d) > 0 ? Lat<Q>::c(K, d) : 0; }
template <int Q, int K>
__host__ __device__ constexpr int cneg(int d) { return Lat<Q>::c(K, d) < 0 ? Lat<Q>::c(K, d) : 0; }

template <int Q, int K, int PAR>
__host__ __device__ constexpr int et_slot(bool bounced) {
  // label K (or its opposite if the population arrives by reflection) at parity PAR
  return ((PAR == 0) != bounced) ? K : Lat<Q>::opp(K);
}

// ---------------------------------------------------------------------------
// canonical load: the pre-collision populations of cell i, for the state kind
// ---------------------------------------------------------------------------
// address of the canonical pre-collision population k of cell nb.i
template <int Q, int L, int LD, int k, class NB>
__device__ __forceinline__ size_t load_addr(const KArgs& a, const NB& nb) {
  const int N = a.N;
  constexpr int kb = Lat<Q>::opp(k);
  if constexpr (LD == LD_LOCAL || k == Lat<Q>::REST) {
    return paddr<Q, L>(k, nb.i, N);
  } else if constexpr (LD == LD_AA_ODD) {
    // f_k(x) = pop_kbar(x - c_k) if x - c_k fluid, else pop_k(x)
    if (!nb.template solid<Q, kb>()) return paddr<Q, L>(kb, nb.template idx<Q, kb>(), N);
    return paddr<Q, L>(k, nb.i, N);
  } else {
    constexpr int PAR = LD == LD_ET_EVEN ? 0 : 1;
    const int cell = nb.template at<-cpos<Q, k>(0), -cpos<Q, k>(1), -cpos<Q, k>(2)>();
    if (!nb.template solid<Q, kb>()) return paddr<Q, L>(et_slot<Q, k, PAR>(false), cell, N);
    return paddr<Q, L>(et_slot<Q, k, PAR>(true), cell, N);
  }
}

template <int Q, int P, int L, int LD, bool FAST, typename T, class NB>
__device__ __forceinline__ void load_cell(const KArgs& a, const NB& nb, const void* pop, T (&f)[Q]) {
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    f[k] = T(ldp<P>(a, pop, load_addr<Q, L, LD, k>(a, nb)));
  });
}

// canonical store (inverse of load_cell at parity 0 / local storage)
template <int Q, int P, int L, int LD, bool FAST>
__device__ __forceinline__ void store_cell_canonical(const KArgs& a, const Nb<FAST>& nb, void* pop,
                                                     const typename Store<P>::R (&f)[Q]) {
  const int N = a.N;
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int kb = Lat<Q>::opp(k);
    size_t ad;
    if constexpr (LD == LD_LOCAL || k == Lat<Q>::REST) {
      ad = paddr<Q, L>(k, nb.i, N);
    } else {
      const int cell = nb.template at<-cpos<Q, k>(0), -cpos<Q, k>(1), -cpos<Q, k>(2)>();
      ad = paddr<Q, L>(et_slot<Q, k, 0>(nb.template solid<Q, kb>()), cell, N);
    }
    stp<P>(a, pop, ad, f[k]);
  });
}

// ---------------------------------------------------------------------------
// the fused stream-and-collide step
// ---------------------------------------------------------------------------
// Only the load and store phases depend on whether the cell is a bulk cell
// (FAST) or sits next to a wall / on a domain face; the collision runs once,
// converged, between them, so a warp that mixes both kinds of cells does not
// execute the collision twice.
template <int Q, int P, int L, int SK, bool FAST>
__device__ __forceinline__ void step_load(const KArgs& a, int i, typename Store<P>::R (&f)[Q], uint8_t fl = 0) {
  constexpr int LD = SK == K_AA_ODD ? LD_AA_ODD : (SK == K_ESOTWIST ? LD_ET_EVEN : LD_LOCAL);
  const Nb<FAST> nb(i, a, fl);
  if constexpr (SK == K_ESOTWIST) {
    if (a.parity == 0) load_cell<Q, P, L, LD_ET_EVEN, FAST>(a, nb, a.a, f);
    else load_cell<Q, P, L, LD_ET_ODD, FAST>(a, nb, a.a, f);
  } else {
    load_cell<Q, P, L, LD, FAST>(a, nb, a.a, f);
  }
}

// walls at a fraction q of their links (lbm_set_link_fractions): the reflected
// population of such a link k is the linear interpolation of Bouzidi,
// Firdaouss & Lallemand (2001), with W the link's wall term:
//   q >= 1/2:  (f_out_k + W) / (2q) + (2q - 1)/(2q) f_out_kbar
//   q <  1/2:  2q f_out_k + (1 - 2q) f_k + W
// where f_k is the cell's pre-collision population k (the population that
// streamed in from x - c_k, standing for that neighbour's post-collision value,
// so that the rule stays local).  It is read again from the cell's load slot:
// no store of the cell has happened yet.  The value replaces f[k], complete with
// its wall term; the returned mask marks those links, whose store adds nothing.
// Links at q = 1/2 keep the halfway bounce-back of the store.  Shifted storage
// (f - t_k) works unchanged: the weights of each form sum to one.
template <int Q, int P, int L, int SK, class NB>
__device__ __forceinline__ uint32_t curved_links(const KArgs& a, const NB& nb, typename Store<P>::R (&f)[Q]) {
  using R = typename Store<P>::R;
  constexpr int H = Lat<Q>::H;
  if (!nb.curved) return 0u;
  const int row = __ldg(a.qidx + nb.i);
  LBM_IF_DEBUG(if ((unsigned)row >= (unsigned)a.dbg_qrows) {
    dbg_fault(a.dbg, DBG_CURVED, (unsigned)row);
    return 0u;
  })
  const double* q = a.qtab + (size_t)row * Q;
  uint32_t done = 0u;
  static_for<0, H>([&](auto kc) {
    constexpr int km = decltype(kc)::value, kp = km + H + 1;
    // both members first from the unmodified pair (a narrow gap bounces both)
    R vm = f[km], vp = f[kp];
    auto one = [&](auto Kc, R fo, R fo_opp, R& out) {
      constexpr int K = decltype(Kc)::value;
      if (!nb.template solid<Q, K>()) return;
      const double qk = __ldg(q + K);
      if (qk == 0.5) return;
      const R W = R(__ldg(a.wall + nb.template kind<Q, K>() * Q + K));
      const R tq = R(2.0 * qk);
      if (qk >= 0.5) {
        out = (fo + W) / tq + ((tq - R(1)) / tq) * fo_opp;
      } else {
        R fin;
        if constexpr (SK == K_ESOTWIST) {
          fin = a.parity == 0 ? ldp<P>(a, a.a, load_addr<Q, L, LD_ET_EVEN, K>(a, nb))
                              : ldp<P>(a, a.a, load_addr<Q, L, LD_ET_ODD, K>(a, nb));
        } else {
          constexpr int LD = SK == K_AA_ODD ? LD_AA_ODD : LD_LOCAL;
          fin = ldp<P>(a, a.a, load_addr<Q, L, LD, K>(a, nb));
        }
        out = tq * fo + (R(1) - tq) * fin + W;
      }
      done |= 1u << K;
    };
    one(std::integral_constant<int, km>{}, f[km], f[kp], vm);
    one(std::integral_constant<int, kp>{}, f[kp], f[km], vp);
    f[km] = vm;
    f[kp] = vp;
  });
  return done;
}

template <int Q, int P, int L, int SK, class NB>
__device__ __forceinline__ void step_store_nb(const KArgs& a, const NB& nb, const typename Store<P>::R (&f)[Q],
                                              uint32_t done = 0u) {
  using R = typename Store<P>::R;
  const int i = nb.i;
  const int N = a.N;
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int kb = Lat<Q>::opp(k);
    if constexpr (k == Lat<Q>::REST) {
      if constexpr (SK == K_TWOPOP) stp<P>(a, a.b, paddr<Q, L>(k, i, N), f[k]);
      else stp<P>(a, a.a, paddr<Q, L>(k, i, N), f[k]);
    } else {
      const bool bounce = nb.template solid<Q, k>();
      R v = f[k];
      if (bounce && !((done >> k) & 1u)) v = v + R(__ldg(a.wall + nb.template kind<Q, k>() * Q + k));
      if constexpr (SK == K_TWOPOP) {
        if (!bounce) stp<P>(a, a.b, paddr<Q, L>(k, nb.template idx<Q, k>(), N), v);
        else stp<P>(a, a.b, paddr<Q, L>(kb, i, N), v);
      } else if constexpr (SK == K_AA_EVEN) {
        stp<P>(a, a.a, paddr<Q, L>(kb, i, N), v);
      } else if constexpr (SK == K_AA_ODD) {
        if (!bounce) stp<P>(a, a.a, paddr<Q, L>(k, nb.template idx<Q, k>(), N), v);
        else stp<P>(a, a.a, paddr<Q, L>(kb, i, N), v);
      } else {  // esoteric twist
        const int cell = nb.template at<cneg<Q, k>(0), cneg<Q, k>(1), cneg<Q, k>(2)>();
        const int slot = a.parity == 0 ? kb : k;
        stp<P>(a, a.a, paddr<Q, L>(slot, cell, N), v);
      }
    }
  });
}

template <int Q, int P, int L, int SK, bool FAST>
__device__ __forceinline__ void step_store(const KArgs& a, int i, const typename Store<P>::R (&f)[Q],
                                           uint8_t fl = 0) {
  step_store_nb<Q, P, L, SK>(a, Nb<FAST>(i, a, fl), f);
}

// one cell update (load, collide, store); solid cells are left alone.
// The bulk-path loads (constant neighbour offsets) are issued before the cell's
// flag byte has arrived, so that a bulk cell pays one memory round trip
// instead of two.  They are issued only when every constant-offset address is
// inside the array: a bulk cell (flag byte 0) is interior, hence its index lies
// in [ny*nz + nz + 1, N - ny*nz - nz - 1), and the speculative loads of the
// other cells in that range read valid memory and are discarded or redone
// with exact addressing once the flag is known.
// Measured on B300: the early loads pay off for the kernels that read only
// their own cell (two-population, AA even / swap collision) in FP32 and FP64;
// the neighbour-pulling kernels (AA odd, esoteric twist) and FP16 storage run
// faster with the flag read first (fewer live registers).
template <int P, int SK>
__host__ __device__ constexpr bool early_loads() {
  return P != F16 && SK != K_AA_ODD && SK != K_ESOTWIST;
}

template <int P>
__device__ __forceinline__ CP<typename Store<P>::R> rates(const KArgs& a) {
  using R = typename Store<P>::R;
  CP<R> cp;
  cp.omega = R(a.omega);
  cp.omc = R(a.omc);
  cp.wplus = R(a.wplus);
  cp.wminus = R(a.wminus);
  cp.omega_high = R(a.omega_high);
  cp.trt_minus = R(a.trt_minus);
  for (int c = 0; c < 4; ++c) {
    cp.wt[c] = R(a.wt[c]);
    cp.wt3[c] = R(a.wt3[c]);
    cp.wm3[c] = R(a.wm3[c]);
  }
  cp.hs = R(a.hs);
  cp.hd = R(a.hd);
  cp.dk = a.dk;
  return cp;
}

// the collision of one cell: the FP32-pipe FP64 operator first where the model
// has one (fx64.cuh), the model's operator for the cells it declines;
// reload(f) refills f with the cell's pre-collision populations (called only
// when the first attempt had already overwritten them)
// (WIDE: the wide range of fx64.cuh)
template <int Q, int M, int P, bool WIDE = false, class Reload>
__device__ __forceinline__ void collide_cell(typename Store<P>::R (&f)[Q], const CP<typename Store<P>::R>& cp,
                                             CellSums* cs, Reload&& reload) {
  using R = typename Store<P>::R;
  if constexpr (HAS_FX<M, R, Store<P>::shifted>) {
    const int st = collide_fx<Q, M == TRT, WIDE>(f, cp.dk, cs);
    if (st == FX_DONE) return;
    if (st == FX_REDO) reload(f);
  } else if constexpr (M == RR && P == F64) {
    const int st = collide_rr_fx<Q>(f, cp.dk, cs);
    if (st == FX_DONE) return;
    if (st == FX_REDO) reload(f);
  }
  collide<Q, M, R, Store<P>::shifted, P == F32>(f, cp, cs);
}

// the collision of one cell in a summing FP64 BGK-W2 / TRT kernel: its sums of
// the state read go to the running sums fs (fx64.cuh), off the FP64 pipe
template <int Q, int M, int P, bool WIDE, class Reload>
__device__ __forceinline__ void collide_cell_fxsums(double (&f)[Q], const CP<double>& cp, FxSums& fs,
                                                    Reload&& reload) {
  static_assert(HAS_FX<M, typename Store<P>::R, Store<P>::shifted>, "FP64 BGK-W2 / TRT only");
  const int st = collide_fx<Q, M == TRT, WIDE>(f, cp.dk, &fs);
  if (st == FX_DONE) return;
  if (st == FX_REDO) {
    // the fast path has added the cell's (exact) sums already
    reload(f);
    collide<Q, M, double, false, false>(f, cp, nullptr);
    return;
  }
  CellSums cs{0.0, 0.0};
  collide<Q, M, double, false, false>(f, cp, &cs);
  fx_sums_add_f64<Q, WIDE>(fs, cs.rho, cs.ke);
}

// the cells with walls at a fraction of their links are updated by
// curved_cells_kernel, after the step kernel (the cells of one step touch
// disjoint memory, so which launch updates a cell does not matter)
__device__ __forceinline__ bool curved_cell(const KArgs& a, int i, uint8_t fl) {
  return a.qidx != nullptr && (fl & FLAG_NEARWALL) && (__ldg(a.nbmask + i) & NBMASK_CURVED);
}

// rate_fn() yields the relaxation rates; it is called just before the
// collision, so that a single-lattice kernel reads them from its launch
// parameters without holding registers across the loads
// cs (optional): receives the cell's share of the conserved sums of the state
// it reads; left untouched for a solid cell
template <int Q, int M, int P, int L, int SK, bool WIDE = false, class RateFn>
__device__ __forceinline__ void step_one(const KArgs& a, int i, RateFn&& rate_fn, CellSums* cs = nullptr) {
  using R = typename Store<P>::R;
  R f[Q];
  uint8_t fl;
  if constexpr (early_loads<P, SK>()) {
    const int reach = a.ny * a.nz + a.nz + 1;
    const bool in_range = i >= reach && i < a.N - reach;
    if (in_range) step_load<Q, P, L, SK, true>(a, i, f);
    fl = a.flags[i];
    if (fl & FLAG_KIND) return;  // solid cell: nothing to update
    if (fl != 0) {
      if (curved_cell(a, i, fl)) return;
      step_load<Q, P, L, SK, false>(a, i, f, fl);
    }
  } else {
    fl = a.flags[i];
    if (fl & FLAG_KIND) return;
    if (fl == 0) {
      step_load<Q, P, L, SK, true>(a, i, f);
    } else {
      if (curved_cell(a, i, fl)) return;
      step_load<Q, P, L, SK, false>(a, i, f, fl);
    }
  }
  const CP<R> cp = rate_fn();
  // (a reload reads the cell's slots again: every scheme's step reads and
  // writes a cell's slots from this thread only, and it has written none yet)
  collide_cell<Q, M, P, WIDE>(f, cp, cs, [&](R (&g)[Q]) {
    if (fl == 0) step_load<Q, P, L, SK, true>(a, i, g);
    else step_load<Q, P, L, SK, false>(a, i, g, fl);
  });
  if (fl == 0) step_store<Q, P, L, SK, true>(a, i, f);
  else step_store<Q, P, L, SK, false>(a, i, f, fl);
}


// FP32/FP16 kernels of the light models are bound by memory latency: capping
// registers so that six (D3Q19) or four (D3Q27) 256-thread blocks fit per SM
// measured fastest.  The moment models would spill under such caps: they keep
// the default register budget.  FP64 kernels are capped at two blocks per SM
// (<= 128 registers) so that a few warps per scheduler hide the FP64 pipe
// latency; the D3Q19 BGK-W2 and RR ones, whose collisions run mostly on the
// FP32 and integer pipes (fx64.cuh, fx_rr.cuh) and are bound by latency, at
// three (<= 80 registers, no spills: BGK-W2 10.4 -> 13.2 GLUPS for the 256^3
// cavity; TRT would spill there).
template <int Q, int M, int P>
inline constexpr int MIN_BLOCKS =
    P == F64 ? ((Q == 19 && (M == BGK_W2 || M == RR)) ? 3 : 2)
             : (!(M == BGK_W2 || M == TRT || M == REG) ? 1 : (Q == 19 ? (M == TRT ? 5 : 6) : 4));
// threads per block of the single-lattice step kernels
inline constexpr int step_threads(int P) { return P == F64 ? 256 : 128; }

// the FP64 BGK-W2 and TRT kernels come in two instantiations, the narrow and
// the wide range of fx64.cuh (WIDE), which the launchers pick by a.fx_wide
template <int M, int P>
inline constexpr bool FX_KERNELS = HAS_FX<M, typename Store<P>::R, Store<P>::shifted>;

template <int Q, int M, int P, int L, int SK, bool WIDE = false>
__global__ void __launch_bounds__(256, MIN_BLOCKS<Q, M, P>) step_kernel(KArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  step_one<Q, M, P, L, SK, WIDE>(a, i, [&] { return rates<P>(a); });
}

using StepFn = cudaError_t (*)(const KArgs&, int threads, cudaStream_t);

using StepSumFn = cudaError_t (*)(const KArgs&, int threads, double* partials, cudaStream_t);

// cells per thread of the summing step kernels.  With FP64 arithmetic the
// kernel is bound by the FP64 pipe, and every lane of the warp's shuffle tree
// adds (5 levels x 2 sums = 10 operations per thread), so four cells share one
// tree; the memory-bound FP32 and FP16 kernels keep one cell per thread.
__host__ __device__ constexpr int sum_cells_per_thread(int P) { return P == F64 ? 4 : 1; }

// a step kernel that also sums, over its block, the FP64 mass and kinetic
// energy of the fluid cells it reads (the collision's own moments), and writes
// them to partials[2 * block], partials[2 * block + 1] in a fixed order; a
// block covers sum_cells_per_thread(P) x blockDim.x consecutive cells
// the summing kernels hold four cells' sums per thread in FP64: two blocks per
// SM (<= 128 registers) keep them out of local memory
template <int Q, int M, int P>
inline constexpr int SUM_MIN_BLOCKS = P == F64 ? 2 : MIN_BLOCKS<Q, M, P>;

template <int Q, int M, int P, int L, int SK, bool WIDE = false>
__global__ void __launch_bounds__(256, SUM_MIN_BLOCKS<Q, M, P>) step_sum_kernel(KArgs a, double* partials) {
  constexpr int CPT = sum_cells_per_thread(P);
  const int base = blockIdx.x * blockDim.x * CPT + threadIdx.x;
  double m = 0.0, e = 0.0;
#pragma unroll 1
  for (int j = 0; j < CPT; ++j) {
    const int i = base + j * (int)blockDim.x;
    CellSums cs{0.0, 0.0};
    if (i < a.N) step_one<Q, M, P, L, SK, WIDE>(a, i, [&] { return rates<P>(a); }, &cs);
    if (j == 0) {
      m = cs.rho;
      e = cs.ke;
    } else {
      m += cs.rho;
      e += cs.ke;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_down_sync(0xffffffffu, m, o);
    e += __shfl_down_sync(0xffffffffu, e, o);
  }
  __shared__ double sm[8][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sm[w][0] = m;
    sm[w][1] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tm = 0.0, te = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      tm += sm[k][0];
      te += sm[k][1];
    }
    partials[2 * blockIdx.x] = tm;
    partials[2 * blockIdx.x + 1] = te;
  }
}

template <int Q, int M, int P, int L, int SK>
cudaError_t launch_step_sum(const KArgs& a, int threads, double* partials, cudaStream_t s) {
  const long long chunk = (long long)threads * sum_cells_per_thread(P);
  const int blocks = (int)((a.N + chunk - 1) / chunk);
  if constexpr (FX_KERNELS<M, P>) {
    if (a.fx_wide) {
      step_sum_kernel<Q, M, P, L, SK, true><<<blocks, threads, 0, s>>>(a, partials);
      return cudaGetLastError();
    }
  }
  step_sum_kernel<Q, M, P, L, SK><<<blocks, threads, 0, s>>>(a, partials);
  return cudaGetLastError();
}

// summing step kernels of one model (SoA; every lattice, storage and step kind)
template <int M>
StepSumFn step_sum_fn_for_model(int Q, int P, int L, int SK) {
  if (L != SOA) return nullptr;
  auto pick = [&](auto q, auto pp) -> StepSumFn {
    constexpr int QQ = decltype(q)::value, PP = decltype(pp)::value;
    switch (SK) {
      case K_TWOPOP: return &launch_step_sum<QQ, M, PP, SOA, K_TWOPOP>;
      case K_AA_EVEN: return &launch_step_sum<QQ, M, PP, SOA, K_AA_EVEN>;
      case K_AA_ODD: return &launch_step_sum<QQ, M, PP, SOA, K_AA_ODD>;
      case K_ESOTWIST: return &launch_step_sum<QQ, M, PP, SOA, K_ESOTWIST>;
      default: return nullptr;
    }
  };
  using I19 = std::integral_constant<int, 19>;
  using I27 = std::integral_constant<int, 27>;
  using PF64 = std::integral_constant<int, F64>;
  using PF32 = std::integral_constant<int, F32>;
  using PF16 = std::integral_constant<int, F16>;
  if (Q == 19) return P == F64 ? pick(I19{}, PF64{}) : (P == F32 ? pick(I19{}, PF32{}) : (P == F16 ? pick(I19{}, PF16{}) : nullptr));
  if (Q == 27) return P == F64 ? pick(I27{}, PF64{}) : (P == F32 ? pick(I27{}, PF32{}) : (P == F16 ? pick(I27{}, PF16{}) : nullptr));
  return nullptr;
}

template <int Q, int M, int P, int L, int SK>
cudaError_t launch_step(const KArgs& a, int threads, cudaStream_t s) {
  const int blocks = (a.N + threads - 1) / threads;
  if constexpr (FX_KERNELS<M, P>) {
    if (a.fx_wide) {
      step_kernel<Q, M, P, L, SK, true><<<blocks, threads, 0, s>>>(a);
      return cudaGetLastError();
    }
  }
  step_kernel<Q, M, P, L, SK><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

// one step of the cells with walls at a fraction of their links (a list of n
// cells), one thread each: load, collide, the interpolated reflections
// (curved_links), store
template <int Q, int M, int P, int L, int SK, bool WIDE = false>
__global__ void __launch_bounds__(128) curved_cells_kernel(KArgs a, const int* cells, int n) {
  using R = typename Store<P>::R;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = __ldg(cells + t);
  const uint8_t fl = a.flags[i];
  const Nb<false> nb(i, a, fl);
  R f[Q];
  auto load = [&](R (&g)[Q]) {
    if constexpr (SK == K_ESOTWIST) {
      if (a.parity == 0) load_cell<Q, P, L, LD_ET_EVEN, false>(a, nb, a.a, g);
      else load_cell<Q, P, L, LD_ET_ODD, false>(a, nb, a.a, g);
    } else {
      load_cell<Q, P, L, SK == K_AA_ODD ? LD_AA_ODD : LD_LOCAL, false>(a, nb, a.a, g);
    }
  };
  load(f);
  collide_cell<Q, M, P, WIDE>(f, rates<P>(a), nullptr, load);
  const uint32_t done = curved_links<Q, P, L, SK>(a, nb, f);
  step_store_nb<Q, P, L, SK>(a, nb, f, done);
}

template <int Q, int M, int P, int L, int SK>
cudaError_t launch_curved(const KArgs& a, const int* cells, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if constexpr (FX_KERNELS<M, P>) {
    if (a.fx_wide) {
      curved_cells_kernel<Q, M, P, L, SK, true><<<(n + 127) / 128, 128, 0, s>>>(a, cells, n);
      return cudaGetLastError();
    }
  }
  curved_cells_kernel<Q, M, P, L, SK><<<(n + 127) / 128, 128, 0, s>>>(a, cells, n);
  return cudaGetLastError();
}

using CurvedFn = cudaError_t (*)(const KArgs&, const int* cells, int n, cudaStream_t);

// one model: all lattices, storages, layouts and step kinds
template <int M>
CurvedFn curved_fn_for_model(int Q, int P, int L, int SK) {
#define LBM_CK(QQ, PP, LL)                                          \
  switch (SK) {                                                     \
    case K_TWOPOP: return &launch_curved<QQ, M, PP, LL, K_TWOPOP>;   \
    case K_AA_EVEN: return &launch_curved<QQ, M, PP, LL, K_AA_EVEN>; \
    case K_AA_ODD: return &launch_curved<QQ, M, PP, LL, K_AA_ODD>;   \
    case K_ESOTWIST: return &launch_curved<QQ, M, PP, LL, K_ESOTWIST>; \
    default: return nullptr;                                        \
  }
  if (Q == 19) {
    if (P == F64 && L == SOA) { LBM_CK(19, F64, SOA) }
    if (P == F64 && L == AOS) { LBM_CK(19, F64, AOS) }
    if (P == F32 && L == SOA) { LBM_CK(19, F32, SOA) }
    if (P == F16 && L == SOA) { LBM_CK(19, F16, SOA) }
  } else if (Q == 27) {
    if (P == F64 && L == SOA) { LBM_CK(27, F64, SOA) }
    if (P == F64 && L == AOS) { LBM_CK(27, F64, AOS) }
    if (P == F32 && L == SOA) { LBM_CK(27, F32, SOA) }
    if (P == F16 && L == SOA) { LBM_CK(27, F16, SOA) }
  }
#undef LBM_CK
  return nullptr;
}

// one model: all lattices, storages, layouts and step kinds
template <int M>
StepFn step_fn_for_model(int Q, int P, int L, int SK) {
#define LBM_SK(QQ, PP, LL)                                      \
  switch (SK) {                                                 \
    case K_TWOPOP: return &launch_step<QQ, M, PP, LL, K_TWOPOP>; \
    case K_AA_EVEN: return &launch_step<QQ, M, PP, LL, K_AA_EVEN>; \
    case K_AA_ODD: return &launch_step<QQ, M, PP, LL, K_AA_ODD>; \
    case K_ESOTWIST: return &launch_step<QQ, M, PP, LL, K_ESOTWIST>; \
    default: return nullptr;                                    \
  }
  if (Q == 19) {
    if (P == F64 && L == SOA) { LBM_SK(19, F64, SOA) }
    if (P == F64 && L == AOS) { LBM_SK(19, F64, AOS) }
    if (P == F32 && L == SOA) { LBM_SK(19, F32, SOA) }
    if (P == F16 && L == SOA) { LBM_SK(19, F16, SOA) }
  } else if (Q == 27) {
    if (P == F64 && L == SOA) { LBM_SK(27, F64, SOA) }
    if (P == F64 && L == AOS) { LBM_SK(27, F64, AOS) }
    if (P == F32 && L == SOA) { LBM_SK(27, F32, SOA) }
    if (P == F16 && L == SOA) { LBM_SK(27, F16, SOA) }
  }
#undef LBM_SK
  return nullptr;
}

}  // namespace lbm
