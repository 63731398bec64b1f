// staged.cuh -- AA-pattern step of FP16-stored populations (SoA) whose reads
// are staged in shared memory by bulk asynchronous copies.
//
// A persistent block walks over tiles of TILE consecutive cells.  For each
// tile a producer warp issues, per population label k, one bulk copy
// (cp.async.bulk, completion counted on an mbarrier) of the contiguous run of
// the source array that the tile's bulk cells read: for the even AA step the
// cells' own slot k; for the odd step slot k-bar of the cells x - c_k, a run
// shifted by the constant offset c_k . (ny nz, nz, 1).  With STAGES buffers in
// flight per block, the bytes a multiprocessor has outstanding no longer
// depend on how many loads its threads can hold in registers, which is what
// limits the one-thread-per-cell kernels with 2-byte populations.
//
// The copies are whole 128-byte units (the run is widened to the enclosing
// 128-byte boundaries), so the population and flag arrays carry 128 bytes of
// padding past their end.  The staged kernel updates the bulk cells (flag
// byte 0), reading their populations from shared memory.  The other fluid
// cells (next to a wall or on a domain face: 1.2 % at 512^3) are updated
// by a one-thread-per-cell kernel on the global-memory path, on a second stream
// beside the staged kernel (the two touch disjoint cells), from a
// sorted list with a record per cell built once per lattice (solid-neighbour
// mask, domain-face bit, wall kinds of the solid neighbours), so that each
// waits on two memory round trips (record, then populations) and reads no
// flag byte.  Updating those cells while the bulk copies stream was measured
// 1.5 to 5 times slower in every form tried (inline in the consumer loop, by
// extra warps inside the stage pipeline, or by extra warps beside it, paced
// to the tile being staged or not): their scattered loads queue behind the
// bulk copies that keep HBM busy, taking ~18 us for a tile's dozen cells, and
// inside the pipeline they hold back the release of whole stages.  Stores go
// straight to global memory.  Every cell is updated exactly as by the
// one-thread-per-cell kernels (same loads, collision and stores; the cells of
// one AA step touch disjoint memory), so the results are bit-identical to
// theirs.
//
// Warp roles: warp 0 is the producer (lane k issues the copy of label k, lane
// Q the copy of the tile's flag bytes); warps 1..CW consume.  Each stage has
// a `full` barrier (Q + 1 producer arrivals plus the copied bytes) and an
// `empty` barrier (one arrival per consumer warp once it has read the stage),
// so no block-wide barrier is taken inside the tile loop.
//
// Every wait of the pipeline (consumers on `full`, the producer on `empty`) is
// bounded by `wait_cycles` SM clock cycles (set by the host; about 2 s unless
// changed); on a timeout the thread records an error code in *err and leaves
// the loop.  Whether its loop ended normally or on a timeout, the producer
// then waits (bounded by the default ~2 s, whatever wait_cycles is) until the
// copies of the last STAGES stages it issued have landed, so that no block
// exits while a bulk copy is still writing into its shared memory -- even
// when its consumer warps gave up early.
#pragma once
#include "internal.h"
#include "kernels.cuh"

namespace lbm {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
// default bound of a wait, in SM clock cycles (about 2 s at 2 GHz)
constexpr long long WAIT_CYCLES_DEFAULT = 1LL << 32;
// wait for the phase with parity `phase` to complete; false once `bound`
// cycles have passed without it
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase,
                                                  long long bound = WAIT_CYCLES_DEFAULT) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase))
    if (clock64() - t0 > bound) return false;
  return true;
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// error codes written to *err by the staged kernels
constexpr int STAGE_ERR_TIMEOUT = 1;


template <int Q, int P, int TILE, int STAGES>
struct StageLayout {
  static constexpr int ES = (int)sizeof(typename Store<P>::S);  // bytes per stored population
  static constexpr int ALIGN = RUN_ALIGN_BYTES / ES;             // elements per alignment unit
  static_assert(TILE % 16 == 0, "TILE must be a multiple of 16 cells");
  static_assert(Q + 1 <= 32, "one producer lane per label plus one for the flags");
  static constexpr int SEG = TILE + 2 * ALIGN;  // elements per staged run
  static constexpr int SEG_BYTES = SEG * ES;
  static constexpr int STAGE_BYTES = Q * SEG_BYTES + TILE;  // runs, then the tile's flag bytes
  // head: full[STAGES], empty[STAGES] barriers, then the run offsets [STAGES][Q]
  static constexpr int HEAD = 128 * ((STAGES * 16 + STAGES * Q * 4 + 127) / 128);
  static constexpr int BYTES = HEAD + STAGES * STAGE_BYTES;
};

// label k of the step kind reads population array `pop` at cell i - off
template <int Q, int SK>
__device__ __forceinline__ void stage_src(int k, int sxy, int nz, int& pop, int& off) {
  pop = k;
  off = 0;
  if constexpr (SK == K_AA_ODD) {
    static_for<0, Q>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      if (k == K && K != Lat<Q>::REST) {
        pop = Lat<Q>::opp(K);
        off = Lat<Q>::c(K, 0) * sxy + Lat<Q>::c(K, 1) * nz + Lat<Q>::c(K, 2);
      }
    });
  }
}

// producer lane `lane` stages its part of tile `tile` into buffer `st`:
// lanes 0..Q-1 one population run each, lane Q the flag bytes; every one of
// these Q + 1 lanes arrives once on full[st]
template <int Q, int P, int SK, int TILE, int STAGES>
__device__ __forceinline__ void stage_issue_lane(const KArgs& a, unsigned char* smem, int tile, int st, int lane) {
  using G = StageLayout<Q, P, TILE, STAGES>;
  const uint32_t full = smem_addr(smem + 8 * st);
  int* s_off = reinterpret_cast<int*>(smem + 16 * STAGES) + st * Q;
  unsigned char* buf = smem + G::HEAD + st * G::STAGE_BYTES;
  const long long N = a.N;
  const long long base = (long long)tile * TILE;
  const int cnt = (int)(N - base < TILE ? N - base : TILE);
  if (lane < Q) {
    int pk, off;
    stage_src<Q, SK>(lane, a.ny * a.nz, a.nz, pk, off);
    const long long p0 = (long long)pk * N;
    const long long start = p0 + base - off;
    // only bulk cells read the run, and their sources lie inside population pk
    long long lo = start > p0 ? start : p0;
    long long hi = start + cnt < p0 + N ? start + cnt : p0 + N;
    if (hi > lo) {
      lo &= ~(long long)(G::ALIGN - 1);
      hi = (hi + G::ALIGN - 1) & ~(long long)(G::ALIGN - 1);
      LBM_IF_DEBUG(if (lo < 0 || hi > (long long)Q * N + (long long)(STAGE_PAD_BYTES / G::ES) ||
                       hi - lo > G::SEG) {
        dbg_fault(a.dbg, DBG_COPY_POP, (unsigned long long)(hi * G::ES));
        s_off[lane] = 0;
        mbar_arrive(full);
        return;
      })
      const uint32_t bytes = (uint32_t)((hi - lo) * G::ES);
      s_off[lane] = (int)(start - lo);
      mbar_arrive_expect_tx(full, bytes);
      bulk_copy_g2s(smem_addr(buf + lane * G::SEG_BYTES),
                    static_cast<const unsigned char*>(a.a) + lo * G::ES, bytes, full);
    } else {
      s_off[lane] = 0;  // no bulk cell of the tile reads this label
      mbar_arrive(full);
    }
  } else if (lane == Q) {
    const uint32_t fbytes = (uint32_t)((cnt + 15) & ~15);
    LBM_IF_DEBUG(if (base + fbytes > N + (long long)STAGE_PAD_BYTES || fbytes > (uint32_t)TILE) {
      dbg_fault(a.dbg, DBG_COPY_FLAGS, (unsigned long long)(base + fbytes));
      mbar_arrive(full);
      return;
    })
    mbar_arrive_expect_tx(full, fbytes);
    bulk_copy_g2s(smem_addr(buf + Q * G::SEG_BYTES), a.flags + base, fbytes, full);
  }
}

// blocks per SM the register budget is sized for: two for the light models
// (FP64: four for D3Q19 and three for D3Q27, as many as their stages fit in
// shared memory), one for the moment models.  The budget decides whether the
// listed-cell kernel, running beside on a second stream, finds room on the
// SMs: at 112 registers per thread (two 9-warp D3Q19 FP64 blocks) it found
// none and the FP64 step ran 22 % slower than at 96.
template <int Q, int M, int P>
inline constexpr int STAGED_BLOCKS =
    P == F64 ? (Q == 19 ? 4 : 3) : ((M == BGK_W2 || M == TRT || M == REG) ? 2 : 1);
// registers per thread for that many blocks of CW + 1 warps (a multiple of 8,
// at most 255), given as an explicit cap; the FP16 light-model kernels are held
// to 96 (two 9-warp blocks would allow 112), which leaves the listed-cell
// kernel room beside them (512^3 cavity, D3Q19 BGK-W2: 57.1 -> 60.2 GLUPS,
// TRT 53.2 -> 59.0)
template <int Q, int M, int P, int CW>
inline constexpr int STAGED_REGS =
    (P == F16 && (M == BGK_W2 || M == TRT || M == REG))
        ? 96
        : ((65536 / (STAGED_BLOCKS<Q, M, P> * 32 * (1 + CW))) / 8 * 8 > 255
               ? 255
               : (65536 / (STAGED_BLOCKS<Q, M, P> * 32 * (1 + CW))) / 8 * 8);

// one producer warp and CW consumer warps per block.  SUMS: every consumer warp
// also sums, in FP64, the mass and kinetic energy of the bulk cells it updates
// (from the moments its collisions compute) and writes them to
// partials[2 w], partials[2 w + 1] with w = blockIdx.x * CW + its index -- a
// fixed assignment of cells to warps (the grid and its tile order are fixed),
// so the sums are reproducible
// (WIDE: the wide range of the FP64 BGK-W2 / TRT collision, fx64.cuh)
template <int Q, int M, int P, int SK, int TILE, int STAGES, int CW, bool SUMS, bool WIDE = false>
__global__ void __maxnreg__((STAGED_REGS<Q, M, P, CW>))
    staged_aa_kernel(KArgs a, int ntiles, int* err, long long wait_cycles, double* partials) {
  using G = StageLayout<Q, P, TILE, STAGES>;
  using R = typename Store<P>::R;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_addr(smem + 8 * s), Q + 1);             // full
      mbar_init(smem_addr(smem + 8 * (STAGES + s)), CW);     // empty
    }
    fence_proxy_async_smem();
  }
  __syncthreads();
  if (warp == 0) {
    // producer; `it` counts the stages issued
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int st = it % STAGES;
      if (it >= STAGES) {
        // wait until every consumer warp has released the previous use of st
        // (the whole warp takes one decision, so that no lane issues a copy
        // after the others have stopped)
        const uint32_t ph = (uint32_t)((it / STAGES - 1) & 1);
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(smem_addr(smem + 8 * (STAGES + st)), ph, wait_cycles))) {
          if (lane == 0) atomicOr(err, STAGE_ERR_TIMEOUT);
          break;
        }
      }
      stage_issue_lane<Q, P, SK, TILE, STAGES>(a, smem, tile, st, lane);
    }
    // drain: stage j (of the last STAGES issued) has had one use since its
    // previous release, so its `full` phase of parity (j / STAGES) & 1 is the
    // one that completes when stage j's copies have landed (already complete
    // when the consumers took it)
    if (lane == 0) {
      for (int j = it > STAGES ? it - STAGES : 0; j < it; ++j)
        if (!mbar_wait_bounded(smem_addr(smem + 8 * (j % STAGES)), (uint32_t)((j / STAGES) & 1)))
          atomicOr(err, STAGE_ERR_TIMEOUT);
    }
    return;
  }
  // consumers: the bulk cells of each tile, from the staged runs
  const CP<R> cp = rates<P>(a);
  const int ct = threadIdx.x - 32;
  // summing variants (FP64 BGK-W2 / TRT): the sums of the cells this thread
  // updates, kept on the FP32 pipe (fx64.cuh)
  FxSums fs{{0.0f, 0.0f}, {0.0f, 0.0f}, 0};
  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int st = it % STAGES;
    const uint32_t full = smem_addr(smem + 8 * st);
    // one decision per warp: a warp leaves whole, never with some lanes still
    // due at the __syncwarp below
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(full, (uint32_t)((it / STAGES) & 1), wait_cycles))) {
      if (lane == 0) atomicOr(err, STAGE_ERR_TIMEOUT);
      return;
    }
    const int* s_off = reinterpret_cast<const int*>(smem + 16 * STAGES) + st * Q;
    const unsigned char* buf = smem + G::HEAD + st * G::STAGE_BYTES;
    const uint8_t* sflags = buf + Q * G::SEG_BYTES;
    const int base = tile * TILE;
    const int cnt = a.N - base < TILE ? a.N - base : TILE;
    for (int c = ct; c < cnt; c += 32 * CW) {
      if (sflags[c] != 0) continue;  // solid, or a listed cell
      R f[Q];
      auto fetch = [&](R (&g)[Q]) {
        static_for<0, Q>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          const auto* run = reinterpret_cast<const typename Store<P>::S*>(buf + k * G::SEG_BYTES);
          LBM_IF_DEBUG(if ((unsigned)(s_off[k] + c) >= (unsigned)G::SEG) {
            dbg_fault(a.dbg, DBG_STAGE_READ, (unsigned)(s_off[k] + c));
            g[k] = R(0);
            return;
          })
          g[k] = Store<P>::to_r(run[s_off[k] + c]);
        });
      };
      fetch(f);
      if constexpr (SUMS) {
        if constexpr (FX_KERNELS<M, P>) {
          collide_cell_fxsums<Q, M, P, WIDE>(f, cp, fs, fetch);  // a reload reads the stage again
        } else {
          // RR: the cell's FP64 sums, added to the running sums
          CellSums cs{0.0, 0.0};
          collide_cell<Q, M, P, WIDE>(f, cp, &cs, fetch);
          fx_sums_add_f64<Q, WIDE>(fs, cs.rho, cs.ke);
        }
      } else {
        collide_cell<Q, M, P, WIDE>(f, cp, nullptr, fetch);
      }
      step_store<Q, P, SOA, SK, true>(a, base + c, f);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_addr(smem + 8 * (STAGES + st)));  // release stage st
  }
  if constexpr (SUMS) {
    double msum, esum;
    fx_sums_f64<Q, WIDE>(fs, msum, esum);
    for (int o = 16; o > 0; o >>= 1) {
      msum += __shfl_down_sync(0xffffffffu, msum, o);
      esum += __shfl_down_sync(0xffffffffu, esum, o);
    }
    if (lane == 0) {
      const int w = blockIdx.x * CW + (warp - 1);
      partials[2 * w] = msum;
      partials[2 * w + 1] = esum;
    }
  }
}

// the listed cells, one thread each, from their records.  SUMS: each 128-thread
// block writes the FP64 mass and kinetic energy of its cells to
// partials[2 b], partials[2 b + 1] (warp trees, then the four warps in order)
template <int Q, int M, int P, int SK, bool SUMS, bool WIDE = false>
__global__ void __launch_bounds__(128) listed_cells_kernel(KArgs a, Listed listed, double* partials) {
  using R = typename Store<P>::R;
  constexpr int LD = SK == K_AA_ODD ? LD_AA_ODD : LD_LOCAL;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  CellSums cs{0.0, 0.0};
  if (t < listed.n) {
    const NbRec nb(__ldg(listed.cell + t), a, __ldg(listed.mask + t), __ldg(listed.kinds + 2 * (size_t)t),
                   __ldg(listed.kinds + 2 * (size_t)t + 1));
    R f[Q];
    load_cell<Q, P, SOA, LD, false>(a, nb, a.a, f);
    const CP<R> cp = rates<P>(a);
    collide_cell<Q, M, P, WIDE>(f, cp, SUMS ? &cs : nullptr,
                          [&](R (&g)[Q]) { load_cell<Q, P, SOA, LD, false>(a, nb, a.a, g); });
    const uint32_t done = curved_links<Q, P, SOA, SK>(a, nb, f);
    step_store_nb<Q, P, SOA, SK>(a, nb, f, done);
  }
  if constexpr (SUMS) {
    double m = cs.rho, e = cs.ke;
    for (int o = 16; o > 0; o >>= 1) {
      m += __shfl_down_sync(0xffffffffu, m, o);
      e += __shfl_down_sync(0xffffffffu, e, o);
    }
    __shared__ double sm[4][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
      sm[w][0] = m;
      sm[w][1] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      partials[2 * blockIdx.x] = ((sm[0][0] + sm[1][0]) + sm[2][0]) + sm[3][0];
      partials[2 * blockIdx.x + 1] = ((sm[0][1] + sm[1][1]) + sm[2][1]) + sm[3][1];
    }
  }
}

// tile shape per lattice and storage: TILE cells, STAGES buffers, CW consumer warps
template <int Q, int P>
struct StagedShape {
  static constexpr int TILE = staged_tile(Q);
  static constexpr int STAGES = 2;
  static constexpr int CW = 8;
};
// FP64: 8-byte populations make a stage of 1024 cells 160 KB.  128-cell tiles
// (one cell per consumer thread), two stages and four 5-warp blocks per SM
// measured fastest for D3Q19 (256^3 cavity: 17.6 GLUPS, against 17.4 for
// 256-cell tiles, 16.1 for three stages and 15.2 for 64-cell tiles); D3Q27
// runs three such blocks.
template <>
struct StagedShape<19, F64> {
  static constexpr int TILE = 128;
  static constexpr int STAGES = 2;
  static constexpr int CW = 4;
};
template <>
struct StagedShape<27, F64> {
  static constexpr int TILE = 128;
  static constexpr int STAGES = 2;
  static constexpr int CW = 4;
};

// one AA step (SK = K_AA_EVEN or K_AA_ODD) of the whole lattice: the staged
// kernel over the bulk cells, then the listed-cell kernel; with nparts, the
// summing variants (FP64 only), whose partial sums follow each other in
// partials: the staged kernel's warps, then the listed kernel's blocks
template <int Q, int M, int P, int SK>
cudaError_t launch_staged_step(const KArgs& a, int* err, long long wait_cycles, const Listed& listed,
                               const SideStream& ss, cudaStream_t s, double* partials, int* nparts) {
  using Sh = StagedShape<Q, P>;
  using G = StageLayout<Q, P, Sh::TILE, Sh::STAGES>;
  constexpr int threads = 32 * (1 + Sh::CW);
  constexpr bool can_sum = P == F64;
  if (nparts && !can_sum) return cudaErrorNotSupported;
  constexpr bool fx = FX_KERNELS<M, P>;
  auto kern_n = staged_aa_kernel<Q, M, P, SK, Sh::TILE, Sh::STAGES, Sh::CW, false>;
  auto kern_sum_n = staged_aa_kernel<Q, M, P, SK, Sh::TILE, Sh::STAGES, Sh::CW, can_sum>;
  auto kern_w = staged_aa_kernel<Q, M, P, SK, Sh::TILE, Sh::STAGES, Sh::CW, false, fx>;
  auto kern_sum_w = staged_aa_kernel<Q, M, P, SK, Sh::TILE, Sh::STAGES, Sh::CW, can_sum, fx>;
  // blocks of the persistent grid: resident blocks per SM x SMs (set once)
  static const int grid = [&] {
    for (auto k : {kern_n, kern_sum_n, kern_w, kern_sum_w})
      if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G::BYTES) != cudaSuccess) return 0;
    auto kern = kern_n;
    int occ = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, G::BYTES) != cudaSuccess) return 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return (occ > 0 ? occ : 1) * sms;
  }();
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  const int ntiles = (a.N + Sh::TILE - 1) / Sh::TILE;
  const int blocks = ntiles < grid ? ntiles : grid;
  const int lblocks = (listed.n + 127) / 128;
  if (nparts) {
    *nparts = blocks * Sh::CW + (listed.n > 0 ? lblocks : 0);
    if (!partials) return cudaSuccess;
  }
  // the two kernels update disjoint cells: with a side stream, the listed-cell
  // kernel runs beside the staged kernel (fork after the previous step, join
  // before the next)
  const bool side = ss.side && listed.n > 0;
  cudaError_t e = cudaSuccess;
  if (side) {
    e = cudaEventRecord(ss.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss.side, ss.fork, 0);
    if (e != cudaSuccess) return e;
  }
  const bool wide = fx && a.fx_wide;
  if (ntiles > 0) {
    if (nparts) (wide ? kern_sum_w : kern_sum_n)<<<blocks, threads, G::BYTES, s>>>(a, ntiles, err, wait_cycles, partials);
    else (wide ? kern_w : kern_n)<<<blocks, threads, G::BYTES, s>>>(a, ntiles, err, wait_cycles, nullptr);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || listed.n <= 0) return e;
  cudaStream_t ls = side ? ss.side : s;
  auto lk_n = listed_cells_kernel<Q, M, P, SK, false>;
  auto lk_sum_n = listed_cells_kernel<Q, M, P, SK, can_sum>;
  auto lk_w = listed_cells_kernel<Q, M, P, SK, false, fx>;
  auto lk_sum_w = listed_cells_kernel<Q, M, P, SK, can_sum, fx>;
  if (nparts) (wide ? lk_sum_w : lk_sum_n)<<<lblocks, 128, 0, ls>>>(a, listed, partials + 2 * blocks * Sh::CW);
  else (wide ? lk_w : lk_n)<<<lblocks, 128, 0, ls>>>(a, listed, nullptr);
  e = cudaGetLastError();
  if (e == cudaSuccess && side) {
    e = cudaEventRecord(ss.join, ss.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ss.join, 0);
  }
  return e;
}

// staged AA step of one model (SoA) for FP16 storage, and for FP64 BGK-W2, TRT
// and D3Q27 RR; nullptr elsewhere.  FP16 populations are where it pays most:
// 2-byte loads leave the one-thread-per-cell kernels short of bytes in flight.
// The FP64 BGK-W2, TRT and RR collisions (fx64.cuh, fx_rr.cuh) keep ~80
// registers per thread busy for 1100 to 4300 instructions per cell, so the
// one-thread-per-cell kernels hold too few loads in flight to cover HBM
// latency; staged, the copies are in flight while the consumers compute.  D3Q19
// RR is bound by instruction issue: staged (three 5-warp blocks per SM, as its
// registers allow) it ran at 8.4 GLUPS against 10.1 for the one-thread-per-cell
// kernel's 24 warps per SM, so it keeps that kernel.  FP32 keeps the
// one-thread-per-cell kernels (they run near the HBM roof), as do the other FP64
// moment models (FP64-pipe bound).
template <int M>
StagedFn staged_fn_for_model(int Q, int P, int SK) {
  constexpr bool fx = M == BGK_W2 || M == TRT || M == RR;
  constexpr bool fx19 = M == BGK_W2 || M == TRT;
  auto pick = [&](auto q, auto pp) -> StagedFn {
    constexpr int QQ = decltype(q)::value, PP = decltype(pp)::value;
    if (SK == K_AA_EVEN) return &launch_staged_step<QQ, M, PP, K_AA_EVEN>;
    if (SK == K_AA_ODD) return &launch_staged_step<QQ, M, PP, K_AA_ODD>;
    return nullptr;
  };
  using I19 = std::integral_constant<int, 19>;
  using I27 = std::integral_constant<int, 27>;
  if (P == F16) return Q == 19 ? pick(I19{}, std::integral_constant<int, F16>{})
                               : (Q == 27 ? pick(I27{}, std::integral_constant<int, F16>{}) : nullptr);
  if constexpr (fx) {
    if (P == F64) {
      if (Q == 27) return pick(I27{}, std::integral_constant<int, F64>{});
      if constexpr (fx19) {
        if (Q == 19) return pick(I19{}, std::integral_constant<int, F64>{});
      }
    }
  }
  return nullptr;
}

}  // namespace lbm
