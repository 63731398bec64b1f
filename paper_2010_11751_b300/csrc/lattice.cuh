// lattice.cuh -- compile-time D3Q19 / D3Q27 tables for the device kernels.
//
// Velocity order (the library's canonical order): the vectors whose first
// non-zero component is -1, sorted by |c|^2 then lexicographically
// (-1 < 0 < 1); then the rest vector; then the negated first half, so that
// opposite(k) = k + H + 1 for k < H = (Q-1)/2.  For D3Q19 this yields
// c_0 = (-1,0,0) = -c_10 (Section 2.6 of the paper).
//
// Everything here is constexpr so that, inside compile-time loops
// (static_for), velocity components, weights and basis exponents are
// constant expressions and fold into immediates.
#pragma once
#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_fp16.h>

namespace lbm {

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// first-half vectors (first non-zero component -1), in canonical order
//  |c|^2 = 1: 0:(-1,0,0) 1:(0,-1,0) 2:(0,0,-1)
//  |c|^2 = 2: 3:(-1,-1,0) 4:(-1,0,-1) 5:(-1,0,1) 6:(-1,1,0) 7:(0,-1,-1) 8:(0,-1,1)
//  |c|^2 = 3 (D3Q27 only): 9:(-1,-1,-1) 10:(-1,-1,1) 11:(-1,1,-1) 12:(-1,1,1)
__host__ __device__ constexpr int half_vel(int k, int d) {
  const int t[13][3] = {{-1, 0, 0},  {0, -1, 0},   {0, 0, -1},  {-1, -1, 0}, {-1, 0, -1},
                        {-1, 0, 1},  {-1, 1, 0},   {0, -1, -1}, {0, -1, 1},  {-1, -1, -1},
                        {-1, -1, 1}, {-1, 1, -1},  {-1, 1, 1}};
  return t[k][d];
}

template <int Q>
struct Lat {
  static_assert(Q == 19 || Q == 27, "D3Q19 or D3Q27");
  static constexpr int H = (Q - 1) / 2;  // number of opposite pairs
  static constexpr int REST = H;
  __host__ __device__ static constexpr int opp(int k) { return k == H ? H : (k < H ? k + H + 1 : k - H - 1); }
  __host__ __device__ static constexpr int c(int k, int d) {
    return k == H ? 0 : (k < H ? half_vel(k, d) : -half_vel(k - H - 1, d));
  }
  __host__ __device__ static constexpr int norm2(int k) {
    return c(k, 0) * c(k, 0) + c(k, 1) * c(k, 1) + c(k, 2) * c(k, 2);
  }
  // weight t_k
  __host__ __device__ static constexpr double w(int k) {
    return Q == 19 ? (norm2(k) == 0 ? 1.0 / 3.0 : (norm2(k) == 1 ? 1.0 / 18.0 : 1.0 / 36.0))
                   : (norm2(k) == 0 ? 8.0 / 27.0
                                    : (norm2(k) == 1 ? 2.0 / 27.0 : (norm2(k) == 2 ? 1.0 / 54.0 : 1.0 / 216.0)));
  }
  // positive member e_k = -c_k of pair k (k < H); its population index is k + H + 1
  __host__ __device__ static constexpr int e(int k, int d) { return -half_vel(k, d); }
};

// monomial moment basis c_x^p c_y^q c_z^r, ordered by total order
__host__ __device__ constexpr int basis_exp(int Q, int j, int d) {
  const int b27[27][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2},
                          {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 2, 0}, {1, 0, 2}, {2, 1, 0}, {0, 1, 2},
                          {2, 0, 1}, {0, 2, 1}, {1, 1, 1}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}, {2, 1, 1},
                          {1, 2, 1}, {1, 1, 2}, {2, 2, 1}, {2, 1, 2}, {1, 2, 2}, {2, 2, 2}};
  // D3Q19 basis: entries 0..15 of the D3Q27 list, then 220, 202, 022
  const int map19[19] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 17, 18, 19};
  return Q == 27 ? b27[j][d] : b27[map19[j]][d];
}

__host__ __device__ constexpr int basis_index(int Q, int p, int q, int r) {
  for (int j = 0; j < Q; ++j)
    if (basis_exp(Q, j, 0) == p && basis_exp(Q, j, 1) == q && basis_exp(Q, j, 2) == r) return j;
  return -1;
}

__host__ __device__ constexpr int basis_order(int Q, int j) {
  return basis_exp(Q, j, 0) + basis_exp(Q, j, 1) + basis_exp(Q, j, 2);
}

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

// value of basis monomial j at the positive pair velocity e_k (k < H)
template <int Q>
__host__ __device__ constexpr int mono_at_e(int j, int k) {
  return ipow_c(Lat<Q>::e(k, 0), basis_exp(Q, j, 0)) * ipow_c(Lat<Q>::e(k, 1), basis_exp(Q, j, 1)) *
         ipow_c(Lat<Q>::e(k, 2), basis_exp(Q, j, 2));
}

// one cell's share of the conserved sums (mass rho, kinetic energy rho |u|^2 / 2),
// taken from the moments a collision computes anyway; accumulated in FP64
struct CellSums {
  double rho, ke;
};

// storage types: FP64 stores f; FP32 / FP16 store the shifted g = f - t_k
enum Prec : int { F64 = 0, F32 = 1, F16 = 2 };

template <int P>
struct Store;
template <>
struct Store<F64> {
  using S = double;
  using R = double;
  static constexpr bool shifted = false;
  __device__ __forceinline__ static R to_r(S v) { return v; }
  __device__ __forceinline__ static S from_r(R v) { return v; }
};
template <>
struct Store<F32> {
  using S = float;
  using R = float;
  static constexpr bool shifted = true;
  __device__ __forceinline__ static R to_r(S v) { return v; }
  __device__ __forceinline__ static S from_r(R v) { return v; }
};
template <>
struct Store<F16> {
  using S = __half;
  using R = float;
  static constexpr bool shifted = true;
  __device__ __forceinline__ static R to_r(S v) { return __half2float(v); }
  __device__ __forceinline__ static S from_r(R v) { return __float2half_rn(v); }
};

// cell flag byte: bits 0-2 wall kind (0 = fluid); bit 6: cell on a domain face
// (neighbour indices need periodic wrap); bit 7: fluid cell with at least one
// solid neighbour.  A byte equal to 0 selects the bulk fast path.
constexpr uint8_t FLAG_KIND = 0x07;
constexpr uint8_t FLAG_EDGE = 0x40;
constexpr uint8_t FLAG_NEARWALL = 0x80;
// solid-neighbour mask word of a fluid cell: bits 0..26 one per link; bit 30
// set when every solid neighbour has the same wall kind, stored in bits 27..29
constexpr uint32_t NBMASK_UNIFORM = 1u << 30;
constexpr int NBMASK_KIND_SHIFT = 27;
// bit 31: some of the cell's walls sit at a fraction of their links
// (lbm_set_link_fractions); in the listed-cell records it is bit 63 of the
// second wall-kind word
constexpr uint32_t NBMASK_CURVED = 1u << 31;

}  // namespace lbm
