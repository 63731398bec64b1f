// internal.h -- declarations shared by the library's translation units
// (launchers of the state kernels, per-model step-kernel tables).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace lbm {

struct KArgs;
struct BatchArgs;

// the staged AA kernels widen each bulk copy to 128-byte boundaries (whole L2
// lines), so population and flag arrays carry this many bytes past their end
constexpr int RUN_ALIGN_BYTES = 128;
constexpr size_t STAGE_PAD_BYTES = RUN_ALIGN_BYTES;
using StepFn = cudaError_t (*)(const KArgs&, int threads, cudaStream_t);
// step kernel that also writes per-block FP64 partial sums (mass, kinetic
// energy) of the state it reads: partials[2 b], partials[2 b + 1] for block b
using StepSumFn = cudaError_t (*)(const KArgs&, int threads, double* partials, cudaStream_t);
using BatchFn = cudaError_t (*)(const BatchArgs&, int sk, int blocks, int threads, cudaStream_t);
// the fluid cells that are not bulk cells (flag byte non-zero), sorted, with a
// record each: solid-neighbour mask | domain-face bit << 31, and the wall kind
// of every solid neighbour (3 bits per link; links 0..20 in kinds[2t], 21..26
// in kinds[2t + 1], whose bit 63 marks walls at a fraction of their links)
struct Listed {
  const int* cell = nullptr;
  const uint32_t* mask = nullptr;
  const unsigned long long* kinds = nullptr;
  int n = 0;
};
// a second stream and two events of a handle, so that a staged step can run
// its listed-cell kernel beside the staged kernel (side == nullptr: one after
// the other on the handle's stream)
struct SideStream {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
// staged AA step: bulk cells through the shared-memory tile pipeline, listed
// cells from their records; err receives the kernel's error word
// and wait_cycles bounds each wait of its copy pipeline (SM clock cycles).
// With nparts set, the step also writes *nparts pairs of FP64 partial sums
// (mass, kinetic energy) of the state it reads to partials, or, with partials
// NULL, only returns that count (nothing is launched); a configuration without
// summing kernels returns cudaErrorNotSupported for it.
using StagedFn = cudaError_t (*)(const KArgs&, int* err, long long wait_cycles, const Listed& listed,
                                 const SideStream& ss, cudaStream_t, double* partials, int* nparts);

// step kernel for (lattice, model, precision, layout, step kind); nullptr if not built
StepFn step_fn(int model, int Q, int P, int L, int SK);
// one step of the listed cells with walls at a fraction of their links, for the
// same key (run after the step kernel, which leaves those cells alone)
using CurvedFn = cudaError_t (*)(const KArgs&, const int* cells, int n, cudaStream_t);
CurvedFn curved_fn(int model, int Q, int P, int L, int SK);
// summing step kernel for the same key (SoA only); nullptr if not built
StepSumFn step_sum_fn(int model, int Q, int P, int L, int SK);
// batched AA kernel (SoA) for (lattice, model, precision); nullptr if not built
BatchFn batch_fn(int model, int Q, int P);
// staged AA step (SoA) for (lattice, model, precision, K_AA_EVEN / K_AA_ODD);
// nullptr where the one-thread-per-cell kernels are used
StagedFn staged_fn(int model, int Q, int P, int SK);

cudaError_t launch_classify(int Q, const uint8_t* raw, uint8_t* out, uint32_t* mask, int nx, int ny, int nz,
                            cudaStream_t s);
// set (qidx[i] >= 0) or clear the curved-wall bit of every cell's solid-neighbour
// mask; qidx null clears all
cudaError_t launch_mark_curved(uint32_t* mask, const int* qidx, int N, cudaStream_t s);
cudaError_t launch_macro(int Q, int P, int L, int LD, const KArgs& a, double* rho, double* u, const double* wall_u,
                         cudaStream_t s);
cudaError_t launch_get(int Q, int P, int L, int LD, const KArgs& a, double* out, cudaStream_t s);
cudaError_t launch_set(int Q, int P, int L, int LD, const KArgs& a, const double* in, cudaStream_t s);
cudaError_t launch_init(int Q, int P, int L, int LD, bool nw4, const KArgs& a, const double* rho, const double* u,
                        cudaStream_t s);
// add to *count the fluid cells of the FP64 state with a population outside its
// weight's binade (the narrow range of fx64.cuh); FP64 storage only
cudaError_t launch_fx_range_count(int Q, int P, int L, int LD, const KArgs& a, int* count, cudaStream_t s);
int reduce_partials_count(int N);
// out[0], out[1] = the sums of the n pairs of partials, in a fixed order
cudaError_t launch_reduce_final(const double* partials, int n, double* out, cudaStream_t s);
cudaError_t launch_reduce(int Q, int P, int L, int LD, const KArgs& a, double* partials, double* out2,
                          cudaStream_t s);
cudaError_t launch_swap_stream(int Q, int P, int L, const KArgs& a, int threads, cudaStream_t s);
// the fluid cells whose flag byte is non-zero, per tile of `tile` cells:
// counts[t] = their number in tile t; then, from the exclusive prefix sums
// offsets[t], their indices in ascending order into list
cudaError_t launch_list_count(const uint8_t* flags, int N, int tile, int* counts, cudaStream_t s);
cudaError_t launch_list_fill(const uint8_t* flags, int N, int tile, const int* offsets, int* list, cudaStream_t s);
// the records of the n listed cells (see Listed)
cudaError_t launch_listed_records(int Q, const KArgs& a, const int* list, int n, uint32_t* mask,
                                  unsigned long long* kinds, cudaStream_t s);
// cells per tile of the staged AA kernels of lattice Q
constexpr int staged_tile(int Q) { return Q == 19 ? 1024 : 512; }

// record the calling thread's last error text (read back by lbm_last_error) and return code
int set_error(int code, const char* msg);

}  // namespace lbm
