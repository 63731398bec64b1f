// state_kernels.cu -- kernels that read or write the lattice state in its
// canonical meaning (independent of scheme, layout and parity), the swap
// scheme's streaming pass, flag classification and the FP64 conserved sums.
#include "internal.h"
#include "kernels.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// flag classification: kind | FLAG_EDGE (domain face) | FLAG_NEARWALL
// ---------------------------------------------------------------------------
template <int Q>
__global__ void classify_kernel(const uint8_t* __restrict__ raw, uint8_t* __restrict__ out,
                                uint32_t* __restrict__ mask_out, int nx, int ny, int nz) {
  const int N = nx * ny * nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int sxy = ny * nz;
  const int x = i / sxy, r = i - x * sxy, y = r / nz, z = r - y * nz;
  uint8_t v = raw[i] & FLAG_KIND;
  if (v == 0) {
    if (x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || z == 0 || z == nz - 1) v |= FLAG_EDGE;
    uint32_t mask = 0u, kind0 = 0u;
    bool uniform = true;
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      int xn = x + Lat<Q>::c(k, 0), yn = y + Lat<Q>::c(k, 1), zn = z + Lat<Q>::c(k, 2);
      xn = xn < 0 ? xn + nx : (xn >= nx ? xn - nx : xn);
      yn = yn < 0 ? yn + ny : (yn >= ny ? yn - ny : yn);
      zn = zn < 0 ? zn + nz : (zn >= nz ? zn - nz : zn);
      const uint32_t kind = raw[(xn * ny + yn) * nz + zn] & FLAG_KIND;
      if (kind) {
        mask |= 1u << k;
        if (kind0 == 0u) kind0 = kind;
        else if (kind != kind0) uniform = false;
      }
    });
    if (mask) v |= FLAG_NEARWALL;
    // every solid neighbour of one wall kind (the common case): the kind rides in
    // the mask word, so that stores need no neighbour flag byte
    if (mask && uniform) mask |= NBMASK_UNIFORM | (kind0 << NBMASK_KIND_SHIFT);
    mask_out[i] = mask;
  } else {
    mask_out[i] = 0u;
  }
  out[i] = v;
}

cudaError_t launch_classify(int Q, const uint8_t* raw, uint8_t* out, uint32_t* mask, int nx, int ny, int nz,
                            cudaStream_t s) {
  const int N = nx * ny * nz, t = 256, b = (N + t - 1) / t;
  if (Q == 19) classify_kernel<19><<<b, t, 0, s>>>(raw, out, mask, nx, ny, nz);
  else classify_kernel<27><<<b, t, 0, s>>>(raw, out, mask, nx, ny, nz);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// canonical reads
// ---------------------------------------------------------------------------
template <int Q, int P, int L, int LD>
__device__ __forceinline__ void load_canonical_f64(const KArgs& a, int i, uint8_t fl, double (&f)[Q]) {
  typename Store<P>::R r[Q];
  if (fl == 0) load_cell<Q, P, L, LD, true>(a, Nb<true>(i, a), a.a, r);
  else load_cell<Q, P, L, LD, false>(a, Nb<false>(i, a, fl), a.a, r);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr double w = WGT<Q, k>;
    f[k] = Store<P>::shifted ? (double)r[k] + w : (double)r[k];
  });
}

template <int Q, int P, int L, int LD>
__global__ void __launch_bounds__(256) macro_kernel(KArgs a, double* rho, double* u, const double* wall_u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const uint8_t fl = a.flags[i];
  const int kind = fl & FLAG_KIND;
  double r, ux, uy, uz;
  if (kind) {
    r = 1.0;
    ux = wall_u[3 * kind];
    uy = wall_u[3 * kind + 1];
    uz = wall_u[3 * kind + 2];
  } else {
    double f[Q];
    load_canonical_f64<Q, P, L, LD>(a, i, fl, f);
    double s = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      s += f[k];
      jx = addc<Lat<Q>::c(k, 0)>(jx, f[k]);
      jy = addc<Lat<Q>::c(k, 1)>(jy, f[k]);
      jz = addc<Lat<Q>::c(k, 2)>(jz, f[k]);
    });
    r = s;
    ux = jx / s;
    uy = jy / s;
    uz = jz / s;
  }
  if (rho) rho[i] = r;
  if (u) {
    u[i] = ux;
    u[(size_t)a.N + i] = uy;
    u[2 * (size_t)a.N + i] = uz;
  }
}

template <int Q, int P, int L, int LD>
__global__ void __launch_bounds__(256) get_kernel(KArgs a, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const uint8_t fl = a.flags[i];
  double f[Q];
  if (fl & FLAG_KIND) {
#pragma unroll
    for (int k = 0; k < Q; ++k) f[k] = 0.0;
  } else {
    load_canonical_f64<Q, P, L, LD>(a, i, fl, f);
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) out[(size_t)k * a.N + i] = f[k];
}

// ---------------------------------------------------------------------------
// canonical writes (state reset to parity 0)
// ---------------------------------------------------------------------------
template <int Q, int P, int L, int LD>
__device__ __forceinline__ void store_canonical(const KArgs& a, int i, uint8_t fl,
                                                const typename Store<P>::R (&r)[Q]) {
  if (fl == 0) store_cell_canonical<Q, P, L, LD, true>(a, Nb<true>(i, a), a.a, r);
  else store_cell_canonical<Q, P, L, LD, false>(a, Nb<false>(i, a, fl), a.a, r);
}

template <int Q, int P, int L, int LD>
__global__ void __launch_bounds__(256) set_kernel(KArgs a, const double* in) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const uint8_t fl = a.flags[i];
  if (fl & FLAG_KIND) return;
  typename Store<P>::R r[Q];
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr double w = WGT<Q, k>;
    const double v = in[(size_t)k * a.N + i];
    r[k] = typename Store<P>::R(Store<P>::shifted ? v - w : v);
  });
  store_canonical<Q, P, L, LD>(a, i, fl, r);
}

template <int Q, int M, int P, int L, int LD>
__global__ void __launch_bounds__(256) init_kernel(KArgs a, const double* rho, const double* u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const uint8_t fl = a.flags[i];
  if (fl & FLAG_KIND) return;
  using R = typename Store<P>::R;
  const double rd = rho ? rho[i] : 1.0;
  const R r = R(rd), dr = R(Store<P>::shifted ? rd - 1.0 : rd);
  const R ux = u ? R(u[i]) : R(0), uy = u ? R(u[(size_t)a.N + i]) : R(0), uz = u ? R(u[2 * (size_t)a.N + i]) : R(0);
  R f[Q];
  equilibrium<Q, M, R, Store<P>::shifted>(r, dr, ux, uy, uz, f);
  store_canonical<Q, P, L, LD>(a, i, fl, f);
}

// ---------------------------------------------------------------------------
// FP64 sums of mass and kinetic energy over fluid cells (deterministic)
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int Q, int P, int L, int LD>
__global__ void __launch_bounds__(RED_THREADS) reduce_kernel(KArgs a, double* partials) {
  double m = 0.0, e = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
    const uint8_t fl = a.flags[i];
    if (fl & FLAG_KIND) continue;
    double f[Q];
    load_canonical_f64<Q, P, L, LD>(a, i, fl, f);
    double s = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      s += f[k];
      jx = addc<Lat<Q>::c(k, 0)>(jx, f[k]);
      jy = addc<Lat<Q>::c(k, 1)>(jy, f[k]);
      jz = addc<Lat<Q>::c(k, 2)>(jz, f[k]);
    });
    m += s;
    e += 0.5 * (jx * jx + jy * jy + jz * jz) / s;
  }
  __shared__ double sm[RED_THREADS / 32][2];
  m = warp_sum(m);
  e = warp_sum(e);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sm[wid][0] = m;
    sm[wid][1] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tm = 0.0, te = 0.0;
    for (int w = 0; w < RED_THREADS / 32; ++w) {
      tm += sm[w][0];
      te += sm[w][1];
    }
    partials[2 * blockIdx.x] = tm;
    partials[2 * blockIdx.x + 1] = te;
  }
}

__global__ void reduce_final_kernel(const double* partials, int n, double* out) {
  __shared__ double sm[2][32];
  double m = 0.0, e = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    m += partials[2 * i];
    e += partials[2 * i + 1];
  }
  m = warp_sum(m);
  e = warp_sum(e);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sm[0][wid] = m;
    sm[1][wid] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tm = 0.0, te = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tm += sm[0][w];
      te += sm[1][w];
    }
    out[0] = tm;
    out[1] = te;
  }
}

// ---------------------------------------------------------------------------
// swap scheme, streaming pass: pairwise swaps with fluid neighbours in c_k,
// k over the first half (the other half is handled by the neighbours)
// ---------------------------------------------------------------------------
template <int Q, int P, int L, bool FAST>
__device__ __forceinline__ void swap_cell(const KArgs& a, int i, uint8_t fl) {
  using S = typename Store<P>::S;
  S* pop = reinterpret_cast<S*>(a.a);
  const Nb<FAST> nb(i, a, fl);
  static_for<0, Lat<Q>::H>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int kb = Lat<Q>::opp(k);
    if (!nb.template solid<Q, k>()) {
      const size_t p0 = paddr<Q, L>(kb, i, a.N), p1 = paddr<Q, L>(k, nb.template idx<Q, k>(), a.N);
      LBM_IF_DEBUG(if (p0 >= a.dbg_elems || p1 >= a.dbg_elems) {
        dbg_fault(a.dbg, DBG_POP_STORE, p0 >= a.dbg_elems ? p0 : p1);
        return;
      })
      const S t0 = pop[p0], t1 = pop[p1];
      pop[p0] = t1;
      pop[p1] = t0;
    }
  });
}

template <int Q, int P, int L>
__global__ void __launch_bounds__(256) swap_stream_kernel(KArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const uint8_t fl = a.flags[i];
  if (fl == 0) swap_cell<Q, P, L, true>(a, i, fl);
  else if ((fl & FLAG_KIND) == 0) swap_cell<Q, P, L, false>(a, i, fl);
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
static inline int nblocks(int N, int t) { return (N + t - 1) / t; }

// call body(integral_constant Q, P, L) for the built (lattice, precision, layout) combinations
template <class F>
static cudaError_t dispatch_qpl(int Q, int P, int L, F&& body) {
  using std::integral_constant;
  if (Q == 19 && P == F64 && L == SOA) return body(integral_constant<int, 19>{}, integral_constant<int, F64>{}, integral_constant<int, SOA>{});
  if (Q == 19 && P == F64 && L == AOS) return body(integral_constant<int, 19>{}, integral_constant<int, F64>{}, integral_constant<int, AOS>{});
  if (Q == 19 && P == F32 && L == SOA) return body(integral_constant<int, 19>{}, integral_constant<int, F32>{}, integral_constant<int, SOA>{});
  if (Q == 19 && P == F16 && L == SOA) return body(integral_constant<int, 19>{}, integral_constant<int, F16>{}, integral_constant<int, SOA>{});
  if (Q == 27 && P == F64 && L == SOA) return body(integral_constant<int, 27>{}, integral_constant<int, F64>{}, integral_constant<int, SOA>{});
  if (Q == 27 && P == F64 && L == AOS) return body(integral_constant<int, 27>{}, integral_constant<int, F64>{}, integral_constant<int, AOS>{});
  if (Q == 27 && P == F32 && L == SOA) return body(integral_constant<int, 27>{}, integral_constant<int, F32>{}, integral_constant<int, SOA>{});
  if (Q == 27 && P == F16 && L == SOA) return body(integral_constant<int, 27>{}, integral_constant<int, F16>{}, integral_constant<int, SOA>{});
  return cudaErrorInvalidValue;
}

// call body(integral_constant LD) for a load kind
template <class F>
static cudaError_t dispatch_ld(int LD, F&& body) {
  using std::integral_constant;
  switch (LD) {
    case LD_LOCAL: return body(integral_constant<int, LD_LOCAL>{});
    case LD_AA_ODD: return body(integral_constant<int, LD_AA_ODD>{});
    case LD_ET_EVEN: return body(integral_constant<int, LD_ET_EVEN>{});
    case LD_ET_ODD: return body(integral_constant<int, LD_ET_ODD>{});
    default: return cudaErrorInvalidValue;
  }
}

#define LBM_CONSTS(q, p, l) constexpr int QQ = decltype(q)::value, PP = decltype(p)::value, LL = decltype(l)::value

cudaError_t launch_macro(int Q, int P, int L, int LD, const KArgs& a, double* rho, double* u, const double* wall_u,
                         cudaStream_t s) {
  return dispatch_qpl(Q, P, L, [&](auto q, auto p, auto l) {
    LBM_CONSTS(q, p, l);
    return dispatch_ld(LD, [&](auto ld) {
      macro_kernel<QQ, PP, LL, decltype(ld)::value><<<nblocks(a.N, 256), 256, 0, s>>>(a, rho, u, wall_u);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_get(int Q, int P, int L, int LD, const KArgs& a, double* out, cudaStream_t s) {
  return dispatch_qpl(Q, P, L, [&](auto q, auto p, auto l) {
    LBM_CONSTS(q, p, l);
    return dispatch_ld(LD, [&](auto ld) {
      get_kernel<QQ, PP, LL, decltype(ld)::value><<<nblocks(a.N, 256), 256, 0, s>>>(a, out);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_set(int Q, int P, int L, int LD, const KArgs& a, const double* in, cudaStream_t s) {
  if (LD != LD_LOCAL && LD != LD_ET_EVEN) return cudaErrorInvalidValue;
  return dispatch_qpl(Q, P, L, [&](auto q, auto p, auto l) {
    LBM_CONSTS(q, p, l);
    if (LD == LD_LOCAL) set_kernel<QQ, PP, LL, LD_LOCAL><<<nblocks(a.N, 256), 256, 0, s>>>(a, in);
    else set_kernel<QQ, PP, LL, LD_ET_EVEN><<<nblocks(a.N, 256), 256, 0, s>>>(a, in);
    return cudaGetLastError();
  });
}

cudaError_t launch_init(int Q, int P, int L, int LD, bool nw4, const KArgs& a, const double* rho, const double* u,
                        cudaStream_t s) {
  if (LD != LD_LOCAL && LD != LD_ET_EVEN) return cudaErrorInvalidValue;
  const int b = nblocks(a.N, 256);
  return dispatch_qpl(Q, P, L, [&](auto q, auto p, auto l) {
    LBM_CONSTS(q, p, l);
    if (nw4) {
      if (LD == LD_LOCAL) init_kernel<QQ, BGK_NW4, PP, LL, LD_LOCAL><<<b, 256, 0, s>>>(a, rho, u);
      else init_kernel<QQ, BGK_NW4, PP, LL, LD_ET_EVEN><<<b, 256, 0, s>>>(a, rho, u);
    } else {
      if (LD == LD_LOCAL) init_kernel<QQ, BGK_W2, PP, LL, LD_LOCAL><<<b, 256, 0, s>>>(a, rho, u);
      else init_kernel<QQ, BGK_W2, PP, LL, LD_ET_EVEN><<<b, 256, 0, s>>>(a, rho, u);
    }
    return cudaGetLastError();
  });
}

int reduce_partials_count(int N) {
  int b = nblocks(N, RED_THREADS);
  return b < 2048 ? b : 2048;
}

cudaError_t launch_reduce(int Q, int P, int L, int LD, const KArgs& a, double* partials, double* out2,
                          cudaStream_t s) {
  const int nb = reduce_partials_count(a.N);
  cudaError_t e = dispatch_qpl(Q, P, L, [&](auto q, auto p, auto l) {
    LBM_CONSTS(q, p, l);
    return dispatch_ld(LD, [&](auto ld) {
      reduce_kernel<QQ, PP, LL, decltype(ld)::value><<<nb, RED_THREADS, 0, s>>>(a, partials);
      return cudaGetLastError();
    });
  });
  if (e != cudaSuccess) return e;
  reduce_final_kernel<<<1, 1024, 0, s>>>(partials, nb, out2);
  return cudaGetLastError();
}

// the fluid cells of an FP64 state with a population outside its weight's
// binade -- those the narrow range of the FP64 BGK-W2 / TRT fast path
// (fx64.cuh) leaves to the FP64 operator -- added to *count
template <int Q, int P, int L, int LD>
__global__ void __launch_bounds__(256) fx_range_kernel(KArgs a, int* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool out = false;
  if (i < a.N) {
    const uint8_t fl = a.flags[i];
    if (!(fl & FLAG_KIND)) {
      double f[Q];
      load_canonical_f64<Q, P, L, LD>(a, i, fl, f);
      unsigned acc = 0u;
      static_for<0, Q>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        acc |= (unsigned)__double2hiint(f[k]) ^ FxW<Q, k, false>::hi_tag;
      });
      out = (acc & 0xfff00000u) != 0u;
    }
  }
  const unsigned b = __ballot_sync(0xffffffffu, out);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, __popc(b));
}

cudaError_t launch_fx_range_count(int Q, int P, int L, int LD, const KArgs& a, int* count, cudaStream_t s) {
  if (P != F64) return cudaErrorInvalidValue;
  const int blocks = (a.N + 255) / 256;
  return dispatch_qpl(Q, P, L, [&](auto q, auto p, auto l) {
    LBM_CONSTS(q, p, l);
    return dispatch_ld(LD, [&](auto ld) {
      fx_range_kernel<QQ, PP, LL, decltype(ld)::value><<<blocks, 256, 0, s>>>(a, count);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_reduce_final(const double* partials, int n, double* out, cudaStream_t s) {
  reduce_final_kernel<<<1, 1024, 0, s>>>(partials, n, out);
  return cudaGetLastError();
}

cudaError_t launch_swap_stream(int Q, int P, int L, const KArgs& a, int threads, cudaStream_t s) {
  return dispatch_qpl(Q, P, L, [&](auto q, auto p, auto l) {
    LBM_CONSTS(q, p, l);
    swap_stream_kernel<QQ, PP, LL><<<nblocks(a.N, threads), threads, 0, s>>>(a);
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
// list of the fluid cells that are not bulk cells (flag byte non-zero and not
// solid), sorted, with the offset of every tile of `tile` cells into it: one
// warp per tile counts (pass 1), then writes its cells in order (pass 2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool nonbulk_fluid(uint8_t f) { return f != 0 && (f & FLAG_KIND) == 0; }

__global__ void tile_count_kernel(const uint8_t* flags, int N, int tile, int ntiles, int* counts) {
  const int t = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (t >= ntiles) return;
  const long long b = (long long)t * tile, e = b + tile < N ? b + tile : N;
  int c = 0;
  for (long long i = b + lane; i < e; i += 32) c += nonbulk_fluid(flags[i]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) counts[t] = c;
}

__global__ void tile_fill_kernel(const uint8_t* flags, int N, int tile, int ntiles, const int* offsets, int* list) {
  const int t = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (t >= ntiles) return;
  const long long b = (long long)t * tile, e = b + tile < N ? b + tile : N;
  int at = offsets[t];
  for (long long i0 = b; i0 < e; i0 += 32) {
    const long long i = i0 + lane;
    const bool pred = i < e && nonbulk_fluid(flags[i]);
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (pred) list[at + __popc(m & ((1u << lane) - 1u))] = (int)i;
    at += __popc(m);
  }
}

cudaError_t launch_list_count(const uint8_t* flags, int N, int tile, int* counts, cudaStream_t s) {
  const int ntiles = (N + tile - 1) / tile;
  const long long threads = 32LL * ntiles;
  if (ntiles > 0) tile_count_kernel<<<(int)((threads + 255) / 256), 256, 0, s>>>(flags, N, tile, ntiles, counts);
  return cudaGetLastError();
}

cudaError_t launch_list_fill(const uint8_t* flags, int N, int tile, const int* offsets, int* list, cudaStream_t s) {
  const int ntiles = (N + tile - 1) / tile;
  const long long threads = 32LL * ntiles;
  if (ntiles > 0) tile_fill_kernel<<<(int)((threads + 255) / 256), 256, 0, s>>>(flags, N, tile, ntiles, offsets, list);
  return cudaGetLastError();
}

template <int Q>
__global__ void listed_records_kernel(KArgs a, const int* list, int n, uint32_t* mask, unsigned long long* kinds) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = list[t];
  const Nb<false> nb(i, a, a.flags[i]);
  unsigned long long k0 = 0ull, k1 = 0ull;
  static_for<0, Q>([&](auto kc) {
    constexpr int K = decltype(kc)::value;
    if constexpr (K != Lat<Q>::REST) {
      if (nb.template solid<Q, K>()) {
        const unsigned long long v = (unsigned long long)nb.template kind<Q, K>();
        if constexpr (K < 21) k0 |= v << (3 * K);
        else k1 |= v << (3 * (K - 21));
      }
    }
  });
  mask[t] = nb.mask | (nb.edge ? 0x80000000u : 0u);
  kinds[2 * (size_t)t] = k0;
  kinds[2 * (size_t)t + 1] = k1 | (nb.curved ? (1ull << 63) : 0ull);
}

__global__ void mark_curved_kernel(uint32_t* mask, const int* qidx, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const bool on = qidx != nullptr && qidx[i] >= 0;
  mask[i] = (mask[i] & ~NBMASK_CURVED) | (on ? NBMASK_CURVED : 0u);
}

cudaError_t launch_mark_curved(uint32_t* mask, const int* qidx, int N, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  mark_curved_kernel<<<(N + 255) / 256, 256, 0, s>>>(mask, qidx, N);
  return cudaGetLastError();
}

cudaError_t launch_listed_records(int Q, const KArgs& a, const int* list, int n, uint32_t* mask,
                                  unsigned long long* kinds, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int b = (n + 255) / 256;
  if (Q == 19) listed_records_kernel<19><<<b, 256, 0, s>>>(a, list, n, mask, kinds);
  else listed_records_kernel<27><<<b, 256, 0, s>>>(a, list, n, mask, kinds);
  return cudaGetLastError();
}

}  // namespace lbm
