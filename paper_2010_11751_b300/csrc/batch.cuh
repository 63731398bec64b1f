// batch.cuh -- one launch per time step for many independent lattices.
//
// Each member lattice keeps its own population array (AA pattern, SoA), flags,
// wall table, relaxation rates and time-step parity.  A device table of member
// descriptors and a block -> member map let one grid cover every member: a
// block reads its member with one load, then updates threads x cells-per-thread
// consecutive cells of that member with the same per-cell code as the
// single-lattice kernels (so a batched step is bit-identical to stepping the
// members one by one).
#pragma once
#include "kernels.cuh"

namespace lbm {

struct __align__(16) Member {
  void* pop;
  const uint8_t* flags;
  const uint32_t* nbmask;
  const double* wall;
  int nx, ny, nz, N;
  int parity0;      // parity of the member's step count when the batch call starts
  int block_begin;  // first grid block of the member
  int pad0, pad1;
  double omega, omc, wplus, wminus, omega_high, trt_minus;
};

struct BatchArgs {
  const Member* m;
  const int* block_member;  // grid block -> member index
  int step;                 // step index within the batch call (parity offset)
  int cpt;                  // cells per thread
};

// the batch kernel holds both AA bodies and the cells-per-thread loop; register
// caps that suit the single-lattice kernels make it spill, so it keeps the
// default register budget
template <int Q, int M, int P>
inline constexpr int BATCH_MIN_BLOCKS = 1;

template <int Q, int M, int P>
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
  a.omega = mm->omega;
  a.omc = mm->omc;
  a.wplus = mm->wplus;
  a.wminus = mm->wminus;
  a.omega_high = mm->omega_high;
  a.trt_minus = mm->trt_minus;
  const int parity = (mm->parity0 + b.step) & 1;
  a.parity = parity;
  const int base = (blockIdx.x - mm->block_begin) * blockDim.x * b.cpt + threadIdx.x;
  if (parity == 0) {
    for (int j = 0; j < b.cpt; ++j) {
      const int i = base + j * blockDim.x;
      if (i < a.N) step_one<Q, M, P, SOA, K_AA_EVEN>(a, i);
    }
  } else {
    for (int j = 0; j < b.cpt; ++j) {
      const int i = base + j * blockDim.x;
      if (i < a.N) step_one<Q, M, P, SOA, K_AA_ODD>(a, i);
    }
  }
}

using BatchFn = cudaError_t (*)(const BatchArgs&, int blocks, int threads, cudaStream_t);

template <int Q, int M, int P>
cudaError_t launch_batch(const BatchArgs& b, int blocks, int threads, cudaStream_t s) {
  batch_aa_kernel<Q, M, P><<<blocks, threads, 0, s>>>(b);
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
