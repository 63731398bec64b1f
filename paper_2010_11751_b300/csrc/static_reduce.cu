// static_reduce.cu -- FP64 mass and kinetic-energy sums over caller-owned
// device buffers, with no allocation at all.
//
// This is a variant of the library's conserved-sums reduction (lbm_reduce)
// for callers that are not allowed to allocate device memory.  Examples are a
// host application that hands the library every buffer from its own pool, a
// real-time loop that cannot afford the implicit synchronisation of
// cudaMalloc/cudaFree, or an environment with a fixed device-memory budget.
// The caller passes the populations, the flags and the output; the per-block
// partial sums go to the fixed array below, which every GPU that loads the
// library holds until the process exits.
#include <cuda.h>  // driver types only: the two driver calls below are reached through the runtime
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "lattice.cuh"
#include "lbm.h"

namespace {

constexpr int SR_THREADS = 256;
constexpr int SR_CELLS_PER_THREAD = 8;
constexpr int SR_CELLS_PER_BLOCK = SR_THREADS * SR_CELLS_PER_THREAD;  // 2048 cells per block
constexpr int SR_MAX_BLOCKS = 16384;                                   // one partial pair per block
constexpr long long SR_MAX_CELLS = (long long)SR_MAX_BLOCKS * SR_CELLS_PER_BLOCK;  // 33,554,432
constexpr int SR_MAX_DEVICES = 64;

// 2 doubles (mass, energy) per block: 256 KiB.  Every block of the first
// kernel overwrites its own pair before the second kernel reads it, so
// nothing here needs to start at zero; the contents of the previous call are
// simply overwritten.
static __device__ __align__(256) double g_static_partials[2 * SR_MAX_BLOCKS];

__device__ __forceinline__ double warp_sum_sr(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int Q>
__global__ void __launch_bounds__(SR_THREADS) static_partials_kernel(const double* __restrict__ f,
                                                                   const uint8_t* __restrict__ flags, int N,
                                                                   double* __restrict__ partials) {
  double m = 0.0, e = 0.0;
  const int base = blockIdx.x * SR_CELLS_PER_BLOCK + threadIdx.x;
#pragma unroll
  for (int j = 0; j < SR_CELLS_PER_THREAD; ++j) {
    const int i = base + j * SR_THREADS;
    if (i >= N || (flags[i] & lbm::FLAG_KIND)) continue;
    double s = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    lbm::static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const double v = f[(size_t)k * N + i];
      s += v;
      if constexpr (lbm::Lat<Q>::c(k, 0) != 0) jx += lbm::Lat<Q>::c(k, 0) * v;
      if constexpr (lbm::Lat<Q>::c(k, 1) != 0) jy += lbm::Lat<Q>::c(k, 1) * v;
      if constexpr (lbm::Lat<Q>::c(k, 2) != 0) jz += lbm::Lat<Q>::c(k, 2) * v;
    });
    m += s;
    e += 0.5 * (jx * jx + jy * jy + jz * jz) / s;
  }
  __shared__ double sm[SR_THREADS / 32][2];
  m = warp_sum_sr(m);
  e = warp_sum_sr(e);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sm[wid][0] = m;
    sm[wid][1] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tm = 0.0, te = 0.0;
    for (int w = 0; w < SR_THREADS / 32; ++w) {
      tm += sm[w][0];
      te += sm[w][1];
    }
    partials[2 * blockIdx.x] = tm;
    partials[2 * blockIdx.x + 1] = te;
  }
}

__global__ void static_final_kernel(const double* __restrict__ partials, int nb, double* __restrict__ out) {
  __shared__ double sm[2][32];
  double m = 0.0, e = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    m += partials[2 * b];
    e += partials[2 * b + 1];
  }
  m = warp_sum_sr(m);
  e = warp_sum_sr(e);
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

// Device address of the scratch array, looked up once per device context.
// The key is the current context's unique id (cuCtxGetId), not the device
// index alone: after cudaDeviceReset the device's next primary context loads
// the library's device code again, at another address, and gets a new id.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
std::once_flag g_driver_once;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

void load_driver_entry_points() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
  fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(fn);
  cudaGetLastError();
}

// unique id of the calling thread's current context; false if there is none
// or it cannot be had (then nothing is cached and every call looks up)
bool current_context_id(unsigned long long* id) {
  std::call_once(g_driver_once, load_driver_entry_points);
  if (!g_ctx_get_current || !g_ctx_get_id) return false;
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

struct ScratchEntry {
  unsigned long long ctx_id = 0;
  double* addr = nullptr;
};
std::mutex g_static_mu;
ScratchEntry g_static_addr[SR_MAX_DEVICES];

int static_scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= SR_MAX_DEVICES) return lbm::set_error(LBM_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  unsigned long long id = 0;
  ScratchEntry& c = g_static_addr[dev];
  if (c.addr && current_context_id(&id) && id == c.ctx_id) {
    *out = c.addr;
    return LBM_OK;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
  if (e != cudaSuccess || !p)
    return lbm::set_error(LBM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch array failed");
  // the lookup made the device's context current if it was not yet
  if (current_context_id(&id)) {
    c.ctx_id = id;
    c.addr = static_cast<double*>(p);
  } else {
    c = ScratchEntry{};
  }
  *out = static_cast<double*>(p);
  return LBM_OK;
}

// device memory of device `dev`, or managed memory
bool device_accessible(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" LBM_API int lbm_conserved_sums_static(int lattice, int N, const double* f, const uint8_t* flags,
                                                 double* out, void* stream) {
  if (lattice != 19 && lattice != 27) return lbm::set_error(LBM_ERR_INVALID_ARG, "lattice must be 19 or 27");
  if (!f || !flags || !out) return lbm::set_error(LBM_ERR_INVALID_ARG, "f, flags and out must not be NULL");
  if (N < 1 || (long long)N > SR_MAX_CELLS)
    return lbm::set_error(LBM_ERR_INVALID_ARG,
                          "N must be in [1, 33554432]: the fixed scratch holds partial sums for 16384 blocks "
                          "of 2048 cells");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lbm::set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
  if (!device_accessible(f, dev) || !device_accessible(flags, dev) || !device_accessible(out, dev))
    return lbm::set_error(LBM_ERR_INVALID_ARG,
                          "f, flags and out must be device memory of the current device (or managed memory)");
  cudaStream_t s = (cudaStream_t)stream;
  int sdev = -1;
  e = cudaStreamGetDevice(s, &sdev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return lbm::set_error(LBM_ERR_INVALID_ARG, "stream is not a valid CUDA stream");
  }
  if (sdev != dev) return lbm::set_error(LBM_ERR_INVALID_ARG, "stream belongs to another device than the current one");
  double* partials = nullptr;
  int rc = static_scratch_address(dev, &partials);
  if (rc != LBM_OK) return rc;
  const int nb = (N + SR_CELLS_PER_BLOCK - 1) / SR_CELLS_PER_BLOCK;
  if (lattice == 19) static_partials_kernel<19><<<nb, SR_THREADS, 0, s>>>(f, flags, N, partials);
  else static_partials_kernel<27><<<nb, SR_THREADS, 0, s>>>(f, flags, N, partials);
  static_final_kernel<<<1, 1024, 0, s>>>(partials, nb, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return lbm::set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}
