// handle.h -- the lattice handle behind lbm_t (shared by the single-lattice
// API and the batch scheduler).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.cuh"
#include "lbm.h"

struct lbm_s {
  int Q = 19, nx = 0, ny = 0, nz = 0, N = 0;
  int scheme = LBM_TWOPOP, model = lbm::BGK_W2, layout = lbm::SOA, prec = lbm::F64;
  double omega = 1.0, omega_bulk = 1.0, omega_high = 1.0, lambda = 0.25;
  bool bulk_follows = true;
  double wall_u[8][3] = {};
  double wall_table[8 * 27] = {};
  cudaStream_t stream = nullptr;
  uint8_t* d_flags = nullptr;
  uint32_t* d_nbmask = nullptr;  // solid-neighbour bit mask per cell
  void* d_pop[2] = {nullptr, nullptr};
  int npop = 1;
  int cur = 0;
  long long steps = 0;
  bool populated = false;
  double* d_wall = nullptr;   // [8][Q] wall terms
  double* d_wallu = nullptr;  // [8][3] wall velocities
  bool wall_dirty = true;
  double* d_partials = nullptr;
  int partials = 0;
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
  int threads = 256;
  lbm::StepFn fns[lbm::NUM_STEP_KINDS] = {};
  lbm::StagedFn sfns[2] = {};  // staged AA even / odd steps, or null (one-thread-per-cell kernels)
  lbm::StepSumFn sumfns[lbm::NUM_STEP_KINDS] = {};  // summing step kernels (SoA), or null
  double* d_sum_partials = nullptr;                 // their per-block partial sums
  size_t sum_partials_cap = 0;                      // doubles allocated there
  int* d_err = nullptr;        // [0] error word of the staged kernels, [1] scratch counter
  // range of the FP64 BGK-W2 / TRT fast path (fx64.cuh): LBM_PARAM_FX_RANGE
  // (0 auto, 1 narrow, 2 wide) and the range in use
  int fx_mode = 0;
  bool fx_wide = false;
  long long nfluid = 0;        // fluid cells (flag 0)
  long long wait_cycles = 1LL << 32;  // bound of each staged-pipeline wait (SM clock cycles)
  // fluid cells with a non-zero flag byte (staged steps), sorted, and their records
  int* d_list = nullptr;
  uint32_t* d_list_mask = nullptr;
  unsigned long long* d_list_kinds = nullptr;
  int* d_tile_off = nullptr;   // per-tile offsets, only while the list is built
  int nlist = -1;              // number of listed cells; -1 until the list is built
  lbm::SideStream side;        // for the staged steps' listed-cell kernel
  // walls at a fraction of their links (lbm_set_link_fractions): per cell its row
  // of d_qtab ([rows][Q] link fractions) or -1; both null when there are none
  int* d_qidx = nullptr;
  double* d_qtab = nullptr;
  int qrows = 0;
  int* d_qcells = nullptr;  // those cells, updated by the curved-cell kernel after each step kernel
  int nqcells = 0;
  lbm::CurvedFn cfns[lbm::NUM_STEP_KINDS] = {};
};

namespace lbm {
// make a handle ready to be stepped: populations written (rest equilibrium if
// never written) and the wall table on the device; returns LBM_OK or an error
int handle_prepare(lbm_s* h);
// relaxation rates of the handle in FP64 and rounded to nearest in FP32: the
// values the step kernels compute with in either arithmetic type
void handle_rates(const lbm_s* h, CP<double>* rd, CP<float>* rf);
}  // namespace lbm
