// internal.h -- declarations shared by the library's translation units
// (launchers of the state kernels, per-model step-kernel tables).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace lbm {

struct KArgs;
struct BatchArgs;
using StepFn = cudaError_t (*)(const KArgs&, int threads, cudaStream_t);
using BatchFn = cudaError_t (*)(const BatchArgs&, int sk, int blocks, int threads, cudaStream_t);

// step kernel for (lattice, model, precision, layout, step kind); nullptr if not built
StepFn step_fn(int model, int Q, int P, int L, int SK);
// batched AA kernel (SoA) for (lattice, model, precision); nullptr if not built
BatchFn batch_fn(int model, int Q, int P);

cudaError_t launch_classify(int Q, const uint8_t* raw, uint8_t* out, uint32_t* mask, int nx, int ny, int nz,
                            cudaStream_t s);
cudaError_t launch_macro(int Q, int P, int L, int LD, const KArgs& a, double* rho, double* u, const double* wall_u,
                         cudaStream_t s);
cudaError_t launch_get(int Q, int P, int L, int LD, const KArgs& a, double* out, cudaStream_t s);
cudaError_t launch_set(int Q, int P, int L, int LD, const KArgs& a, const double* in, cudaStream_t s);
cudaError_t launch_init(int Q, int P, int L, int LD, bool nw4, const KArgs& a, const double* rho, const double* u,
                        cudaStream_t s);
int reduce_partials_count(int N);
cudaError_t launch_reduce(int Q, int P, int L, int LD, const KArgs& a, double* partials, double* out2,
                          cudaStream_t s);
cudaError_t launch_swap_stream(int Q, int P, int L, const KArgs& a, int threads, cudaStream_t s);

// record the calling thread's last error text (read back by lbm_last_error) and return code
int set_error(int code, const char* msg);

}  // namespace lbm
