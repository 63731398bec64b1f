// batch.cuh -- one launch per time step for many independent lattices.
//
// Each member lattice keeps its own population array (AA pattern, SoA), flags,
// wall table, relaxation rates and time-step parity.  A device table of member
// descriptors and, per step parity, a block -> member map let one grid cover
// every member of that parity: a block reads its member with one load, then
// updates threads x cells-per-thread consecutive cells of that member with the
// same per-cell code as the single-lattice kernels (so a batched step is
// bit-identical to stepping the members one by one).  A time step launches the
// even-step kernel on one parity class and the odd-step kernel on the other.
#pragma once
#include "kernels.cuh"

namespace lbm {

struct __align__(16) Member {
  void* pop;
  const uint8_t* flags;
  const uint32_t* nbmask;
  const double* wall;
  int nx, ny, nz, N;
  int fx_wide;      // FP64 BGK-W2 / TRT: the member runs the wide range of fx64.cuh
  int block_begin;  // first grid block of the member (within its parity class map)
  int pad0, pad1;
  // the member's relaxation rates in both arithmetic types, derived and rounded
  // to nearest on the host exactly as a single-lattice kernel rounds its launch
  // parameters, so that no thread spends FP64 operations or conversions on them
  CP<double> rd;
  CP<float> rf;
#ifdef LBM_DEBUG
  unsigned long long* dbg;  // the member handle's fault word (debug.cuh)
#endif
};

struct BatchArgs {
  const Member* m;
  const int* block_member;  // grid block -> member index (members of one step parity)
  int cpt;                  // cells per thread
};

// register bounds of the batch kernels: milder than the single-lattice ones,
// because the member's pointers and sizes come from a table in global memory
// and live in registers (a single-lattice kernel reads them from its launch
// parameters)
// (the FP64 D3Q27 BGK-W2 and TRT batch kernels, which hold 27 populations and
// the member's addressing beside the integer and double-float state of
// fx64.cuh, take the full register file instead of spilling; the autotuner
// picks their block size)
template <int Q, int M, int P>
inline constexpr int BATCH_MIN_BLOCKS =
    P == F64 ? ((Q == 27 && (M == BGK_W2 || M == TRT)) ? 1 : 2)
             : (MIN_BLOCKS<Q, M, P> == 1 ? 1 : (Q == 19 ? 4 : 3));

// one kernel per AA step kind (SK = K_AA_EVEN or K_AA_ODD), so that each holds
// a single body; the host launches it on the members whose step parity matches
template <int Q, int M, int P, int SK>
__global__ void __launch_bounds__(256, BATCH_MIN_BLOCKS<Q, M, P>) batch_aa_kernel(BatchArgs b) {
  const int mi = __ldg(b.block_member + blockIdx.x);
  const Member* mm = b.m + mi;
  KArgs a;
  a.a = mm->pop;
  a.b = nullptr;
  a.flags = mm->flags;
  a.nbmask = mm->nbmask;
  a.wall = mm->wall;
  a.nx = mm->nx;
  a.ny = mm->ny;
  a.nz = mm->nz;
  a.N = mm->N;
  a.parity = SK == K_AA_ODD ? 1 : 0;
  a.qidx = nullptr;  // members never have walls at a fraction of their links
  a.qtab = nullptr;
#ifdef LBM_DEBUG
  a.dbg = mm->dbg;
  a.dbg_elems = (size_t)Q * (size_t)mm->N;
  a.dbg_qrows = 0;
#endif
  using R = typename Store<P>::R;
  // the member's rates, staged in shared memory once per block and read
  // from there just before each collision
  constexpr int NW = (int)(sizeof(CP<R>) / sizeof(R));
  static_assert(sizeof(CP<R>) == NW * sizeof(R), "CP holds rates only");
  __shared__ CP<R> s_cp;
  {
    const CP<R>* src;
    if constexpr (std::is_same<R, double>::value) src = &mm->rd;
    else src = &mm->rf;
    for (int w = threadIdx.x; w < NW; w += blockDim.x)
      reinterpret_cast<R*>(&s_cp)[w] = __ldg(reinterpret_cast<const R*>(src) + w);
  }
  __syncthreads();
  const int base = (blockIdx.x - mm->block_begin) * blockDim.x * b.cpt + threadIdx.x;
  // a member's cells all take its own range of the FP64 fast path (fx64.cuh),
  // as when it is stepped alone
  auto cells = [&](auto wide) {
#pragma unroll 1
    for (int j = 0; j < b.cpt; ++j) {
      const int i = base + j * blockDim.x;
      if (i < a.N) step_one<Q, M, P, SOA, SK, decltype(wide)::value>(a, i, [&] { return s_cp; });
    }
  };
  if constexpr (FX_KERNELS<M, P>) {
    if (mm->fx_wide) {
      cells(std::true_type{});
      return;
    }
  }
  cells(std::false_type{});
}

// sk: K_AA_EVEN or K_AA_ODD
using BatchFn = cudaError_t (*)(const BatchArgs&, int sk, int blocks, int threads, cudaStream_t);

template <int Q, int M, int P>
cudaError_t launch_batch(const BatchArgs& b, int sk, int blocks, int threads, cudaStream_t s) {
  if (sk == K_AA_EVEN) batch_aa_kernel<Q, M, P, K_AA_EVEN><<<blocks, threads, 0, s>>>(b);
  else batch_aa_kernel<Q, M, P, K_AA_ODD><<<blocks, threads, 0, s>>>(b);
  return cudaGetLastError();
}

template <int M>
BatchFn batch_fn_for_model(int Q, int P) {
  if (Q == 19) {
    if (P == F64) return &launch_batch<19, M, F64>;
    if (P == F32) return &launch_batch<19, M, F32>;
    if (P == F16) return &launch_batch<19, M, F16>;
  } else if (Q == 27) {
    if (P == F64) return &launch_batch<27, M, F64>;
    if (P == F32) return &launch_batch<27, M, F32>;
    if (P == F16) return &launch_batch<27, M, F16>;
  }
  return nullptr;
}

}  // namespace lbm
