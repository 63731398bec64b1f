// debug.cuh -- bounds checks of the LBM_DEBUG build (liblbm_debug.so).
//
// The library built with -DLBM_DEBUG checks, in every step and state kernel,
// each population load and store against the Q N populations of the array,
// each cell index (own cell, neighbour, flag byte, solid-neighbour mask word)
// against [0, N), each bulk copy of the staged kernels against the array's
// extent plus its STAGE_PAD_BYTES of padding, and each read of a staged run
// against the run held in shared memory.  A failed check records the first
// fault of the handle in a 64-bit device word (kind in bits 56..63, the
// offending element or byte index below) and skips the access (a skipped
// load yields 0, a skipped copy arrives on its barrier without bytes): the
// kernel neither traps nor touches memory outside the arrays.  The padding of
// the population and flag arrays is filled with a canary byte at allocation;
// lbm_debug_check reads the fault word and verifies the canaries.
//
// In the release build every macro here expands to nothing and the kernels
// are unchanged.
#pragma once
#include <cstdint>

namespace lbm {

enum DebugKind : unsigned {
  DBG_NONE = 0,
  DBG_POP_LOAD = 1,    // population load outside [0, Q N)
  DBG_POP_STORE = 2,   // population store outside [0, Q N)
  DBG_CELL = 3,        // neighbour or own cell index outside [0, N)
  DBG_FLAG = 4,        // flag byte read outside [0, N)
  DBG_MASK = 5,        // solid-neighbour mask read outside [0, N)
  DBG_COPY_POP = 6,    // staged bulk copy of populations past the padded array
  DBG_COPY_FLAGS = 7,  // staged bulk copy of flag bytes past the padded array
  DBG_STAGE_READ = 8,  // read of a staged run outside the run in shared memory
  DBG_CURVED = 9,      // link-fraction row outside the table
  DBG_PAD = 10,        // a canary byte of the padding was overwritten (host check)
};

// canary byte of the padding past the population and flag arrays
constexpr unsigned char DEBUG_CANARY = 0xA5;

#ifdef LBM_DEBUG
// record (kind, index) in *w unless an earlier fault is there
__device__ __forceinline__ void dbg_fault(unsigned long long* w, unsigned kind, unsigned long long index) {
  if (w) atomicCAS(w, 0ull, ((unsigned long long)kind << 56) | (index & ((1ull << 56) - 1)));
}
// cell index sentinel: an address computed from an out-of-range cell
constexpr size_t DBG_BAD_ADDR = ~size_t(0);
#define LBM_IF_DEBUG(...) __VA_ARGS__
#else
#define LBM_IF_DEBUG(...)
#endif

}  // namespace lbm
