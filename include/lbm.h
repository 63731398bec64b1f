/*
 * lbm.h -- C ABI of the B300 (sm_103a) lattice Boltzmann stream-and-collide
 * library liblbm.so.
 *
 * Method: Latt, Coreixas & Beny, "Cross-platform programming model for
 * many-core lattice Boltzmann simulation", arXiv:2010.11751.
 *   - one time iteration = collision f_out = Omega(f) followed by streaming
 *     f_k(x + c_k, t+1) = f_out_k(x, t)  (Section 2.1, collision/streaming eqs.)
 *   - walls: link-wise bounce-back with momentum exchange,
 *     f_kbar(x, t+1) = f_out_k(x, t) - 6 t_k rho_w c_k.u_w, rho_w = 1
 *     (Section 2.1, momentum-exchange equation)
 *   - memory-access schemes: double population, swap, AA-pattern
 *     (Section 2.3, Table 1) and the esoteric twist (Geier & Schoenherr 2017)
 *   - layouts: structure-of-arrays pop[Q][N], array-of-structures pop[N][Q]
 *     (Section 2.3, end)
 *   - collision models of Section 2.2 / Section 2.6.
 *
 * Conventions common to every call
 *   - Every function returns LBM_OK (0) or a negative LBM_ERR_* code; the
 *     text of the last error of the calling thread is lbm_last_error().
 *   - Cell index i = (x*ny + y)*nz + z (z fastest), N = nx*ny*nz.
 *   - Canonical population order k = 0..Q-1: the velocities whose first
 *     non-zero component is -1, sorted by |c|^2 then lexicographically
 *     (-1 < 0 < 1); then the rest velocity; then the negated first half.
 *     opposite(k) = k + (Q+1)/2 for k < (Q-1)/2.  For D3Q19 this gives
 *     c_0 = (-1,0,0) = -c_10 as in Section 2.6.
 *   - Canonical population arrays are FP64, [Q][N] (SoA), independent of the
 *     handle's scheme, layout, precision and time-step parity.
 *   - Flag field: uint8 per cell; 0 = fluid, 1 = resting bounce-back wall,
 *     2..7 = moving wall with the velocity set by lbm_set_wall_velocity.
 *     The box is periodic in every axis; closed domains carry explicit wall
 *     layers.  Solid cells read back as f = 0, rho = 1, u = wall velocity.
 *   - Pointer arguments marked "host or device" may point to host memory
 *     (pageable or pinned) or to device memory of the handle's GPU; the
 *     library detects which with cudaPointerGetAttributes.  Host transfers
 *     are synchronous with respect to the handle's stream.
 *   - All device work is enqueued on the handle's stream (default: the legacy
 *     default stream).  lbm_step does not synchronise.  Handles are not
 *     thread-safe: one host thread at a time per handle.
 *   - The library owns every device buffer it allocates; caller buffers stay
 *     the caller's.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

/* largest lattice, nx*ny*nz cells (2^31 - 2^22) */
#define LBM_MAX_CELLS 2143289344LL

/* ---- status codes ---- */
#define LBM_OK 0
#define LBM_ERR_INVALID_ARG (-1) /* bad enum, bad size, NULL pointer, n < 0 */
#define LBM_ERR_OOM (-2)         /* request does not fit in free device memory */
#define LBM_ERR_STATE (-3)       /* call not allowed in the handle's current state */
#define LBM_ERR_DIVERGED (-4)    /* non-finite mass or energy detected */
#define LBM_ERR_TIMEOUT (-5)     /* a bounded device wait gave up */
#define LBM_ERR_CUDA (-6)        /* a CUDA runtime call failed */
#define LBM_ERR_UNSUPPORTED (-7) /* combination not built (see lbm_supported) */

/* ---- lattices ---- */
#define LBM_D3Q19 19
#define LBM_D3Q27 27

/* ---- memory-access schemes (Section 2.3, Table 1) ---- */
#define LBM_TWOPOP 0   /* double population: read pop, write out at x+c_k; swap arrays */
#define LBM_SWAP 1     /* collide (store to opposite slot), then 9 (13) pairwise swaps */
#define LBM_AA 2       /* AA-pattern: local step / pull-collide-push step, alternating */
#define LBM_ESOTWIST 3 /* esoteric twist: one in-place kernel, slot labels swap each step */

/* ---- collision models (Section 2.2) ---- */
#define LBM_BGK_W2 0  /* BGK, second-order weighted equilibrium (Section 2.6) */
#define LBM_BGK_NW4 1 /* BGK, non-weighted product-Maxwellian equilibrium */
#define LBM_TRT 2     /* two-relaxation-time, magic parameter Lambda */
#define LBM_REG 3     /* regularized (second-order Hermite projection) */
#define LBM_RR 4      /* recursive regularized, Hermite-moment form */
#define LBM_RM 5      /* raw-moment multi-relaxation (Section 2.6 relaxation law) */
#define LBM_HM 6      /* Hermite-moment multi-relaxation */
#define LBM_CM 7      /* central-moment multi-relaxation */
#define LBM_CHM 8     /* central-Hermite-moment multi-relaxation */
#define LBM_K 9       /* cumulant */
/* BGK-W2 again, in the "educational" form of Section 2.6 (one plain loop over
 * the directions with tabulated c_k, t_k; only the density and velocity sums
 * regrouped), for the unrolled-versus-educational comparison of Section 4:
 * loops as the compiler chooses to compile them, or kept rolled. */
#define LBM_BGK_W2_EDU 10
#define LBM_BGK_W2_LOOP 11

/* ---- layouts (Section 2.3) ---- */
#define LBM_SOA 0 /* pop[Q][N] */
#define LBM_AOS 1 /* pop[N][Q] */

/* ---- storage precision ---- */
#define LBM_F64 0 /* populations f stored in FP64, FP64 arithmetic */
#define LBM_F32 1 /* shifted populations f - t_k stored in FP32, FP32 arithmetic */
#define LBM_F16 2 /* shifted populations f - t_k stored in FP16, FP32 arithmetic */

/* ---- relaxation parameters (Section 2.6) ---- */
#define LBM_PARAM_OMEGA 0      /* omega_nu, shear rate; nu = (1/omega - 1/2)/3 */
#define LBM_PARAM_OMEGA_BULK 1 /* omega_nu_b of the bulk coupling; default: follows omega */
#define LBM_PARAM_OMEGA_HIGH 2 /* rate of moments of order >= 3; default 1 */
#define LBM_PARAM_TRT_LAMBDA 3 /* TRT magic parameter; default 1/4 */
/* Bound, in SM clock cycles, of each wait in the copy pipeline of the staged
 * AA steps (FP16 SoA storage; see lbm_step); default 2^32, about 2 s at
 * 2 GHz.  Integer values in [1, 2^40].  A bound far below a copy's latency
 * (a few hundred cycles) makes the waits give up, which is how the
 * LBM_ERR_TIMEOUT path is exercised: the step's results are then undefined and
 * the handle reports LBM_ERR_TIMEOUT from then on.  Before a block of the
 * staged kernel exits, it always waits for its own copies in flight with the
 * default bound, whatever this value is. */
#define LBM_PARAM_WAIT_CYCLES 4
/* Range of the FP64 BGK-W2 and TRT fast path (collision arithmetic on the
 * FP32 and integer pipes, exact integer moments; cells outside the range take
 * the plain FP64 operator).  1: narrow -- populations in their weights'
 * binades; 2: wide -- also the binades next to them, for faster flows (a
 * Taylor-Green vortex at u0 = 0.05 runs ~3x faster), at ~2 % extra cost for
 * flows that stay near the weights; 0 (default): auto -- after every state
 * write (lbm_init_equilibrium with rho or u, lbm_set_populations) the
 * library counts the fluid cells with a population outside its weight's
 * binade and picks wide when they exceed 1 %; those calls then synchronise
 * the stream.  Either range matches the FP64 oracle within 1e-12; results
 * are bit-identical across schemes and layouts for a given range, but a
 * lattice resumed from lbm_set_populations may pick another range than the
 * run it was saved from (set 1 or 2 explicitly for bit-exact resumption).
 * No effect on other models and storage precisions. */
#define LBM_PARAM_FX_RANGE 5

typedef struct lbm_s* lbm_t;

/* Create a lattice.  lattice: 19 or 27; nx, ny, nz >= 1 with N <= LBM_MAX_CELLS;
 * scheme: LBM_TWOPOP..LBM_ESOTWIST; collision: LBM_BGK_W2..LBM_BGK_W2_LOOP;
 * omega in (0, 2); flags: host array of N bytes (copied).  Layout SoA and
 * precision FP64 unless changed before the populations are first written.
 * Device memory for the populations is reserved at the first call that
 * writes them; LBM_ERR_OOM if it would not fit. */
LBM_API int lbm_create(lbm_t* out, int lattice, int nx, int ny, int nz, int scheme, int collision, double omega,
               const uint8_t* flags);

/* Change layout / precision.  Only before populations are first written
 * (lbm_init_equilibrium, lbm_set_populations or lbm_step), else LBM_ERR_STATE.
 * LBM_ERR_UNSUPPORTED for combinations that are not built (see lbm_supported). */
LBM_API int lbm_set_layout(lbm_t h, int layout);
LBM_API int lbm_set_precision(lbm_t h, int precision);

/* Velocity of moving-wall kind flag (2..7); rho_w = 1.  Takes effect at the
 * next step. */
LBM_API int lbm_set_wall_velocity(lbm_t h, int flag, double ux, double uy, double uz);

/* Walls at a fraction of their links: the extension of link-wise bounce-back
 * to curved walls that Section 1 points to, kept local to the wall cell.
 * q: host, FP64 [Q][N] canonical; for every fluid cell i and link k whose
 * neighbour x + c_k is solid, q[k*N + i] in (0, 1] is the fraction of the
 * link from x at which the wall lies (1/2: the halfway bounce-back of Section
 * 2.1); entries of other links are ignored.  The reflected population of a
 * link with q != 1/2 is the linear interpolation of Bouzidi, Firdaouss &
 * Lallemand (2001), W being the link's wall term -6 t_k rho_w c_k.u_w:
 *   q >= 1/2:  f_kbar(x, t+1) = [f_out_k(x) + W] / (2q) + (2q - 1)/(2q) f_out_kbar(x)
 *   q <  1/2:  f_kbar(x, t+1) = 2q f_out_k(x) + (1 - 2q) f_k(x, t) + W
 * with the cell's pre-collision f_k(x, t) standing for the neighbour's
 * post-collision f_out_k(x - c_k) (the same value one step earlier).  The
 * array is copied; the library keeps a per-cell index (4 bytes per cell) and
 * the Q fractions of each cell with a link at q != 1/2, counted by
 * lbm_device_bytes.  q NULL removes them (halfway walls again).  Takes effect
 * at the next step; waits for the handle's stream.  LBM_ERR_INVALID_ARG for a
 * NULL handle or a fraction outside (0, 1] on a wall link; a handle with such
 * walls cannot join a batch (LBM_ERR_UNSUPPORTED from lbm_batch_add). */
LBM_API int lbm_set_link_fractions(lbm_t h, const double* q);

/* Set LBM_PARAM_*.  omega and omega_bulk in (0, 2), omega_high in (0, 2],
 * lambda > 0, wait_cycles an integer in [1, 2^40], fx range 0, 1 or 2.
 * Takes effect at the next step. */
LBM_API int lbm_set_param(lbm_t h, int key, double value);

/* All device work of this handle goes to this cudaStream_t (NULL: legacy default).
 * The staged AA steps of FP16 SoA storage also run a kernel on a stream of the
 * handle's own, forked from and joined back to this one by events, so that
 * work enqueued here later still follows the whole step. */
LBM_API int lbm_set_stream(lbm_t h, void* stream);

/* f = the collision model's own equilibrium of (rho, u) on every fluid cell.
 * rho: N doubles, u: 3*N doubles (ux[N], uy[N], uz[N]); host or device.
 * Either may be NULL: rho = 1, u = 0.  Resets the time-step parity. */
LBM_API int lbm_init_equilibrium(lbm_t h, const double* rho, const double* u);

/* Enqueue n >= 0 time iterations on the handle's stream; asynchronous.  If
 * the populations were never written, they are first set to the equilibrium
 * at rho = 1, u = 0.  The first AA step of an FP16 SoA handle also builds
 * (once, synchronously) the list of cells next to a wall or on a domain face
 * that its staged steps update separately.  The staged steps wait on their
 * shared-memory copies with a ~2 s bound; a wait that gives up is reported by
 * the next lbm_reduce or host lbm_get_populations as LBM_ERR_TIMEOUT. */
LBM_API int lbm_step(lbm_t h, int n);

/* lbm_reduce followed by lbm_step(h, n), in fewer passes over memory: the
 * FP64 mass and energy (as lbm_reduce defines them) of the state the call
 * starts from, computed by the first of the n steps from the moments its
 * collision forms anyway (for n = 0 it is lbm_reduce).  Handles without such a
 * kernel (AoS layout, the staged FP16 AA steps) run the reduction, then the
 * steps.  The sums agree with lbm_reduce's up to FP64 summation order; FP32
 * and FP16 storage form each cell's share in FP32.  Synchronises the stream;
 * errors as lbm_reduce. */
LBM_API int lbm_step_sums(lbm_t h, int n, double* mass, double* energy);

/* lbm_step_sums without the wait (no counterpart in the paper): enqueues the
 * same work (n >= 1 steps; the sums of the state the call starts from) and
 * returns at once.  out: 2 doubles {mass, energy}, device memory or
 * page-locked host memory (cudaHostAlloc / cudaHostRegister), written when
 * the handle's stream reaches the copy; pageable host memory is rejected with
 * LBM_ERR_INVALID_ARG.  A caller that keeps one call in flight while it reads
 * the previous call's sums keeps the GPU busy.  Divergence shows as non-finite
 * sums; a staged-wait timeout is reported by the next synchronous call
 * (lbm_reduce, lbm_step_sums, lbm_get_populations to the host). */
LBM_API int lbm_step_sums_async(lbm_t h, int n, double* out);

/* rho[N] and u[3*N] (FP64) of the current pre-collision state; host or device.
 * Either may be NULL.  Synchronises the handle's stream for host outputs. */
LBM_API int lbm_macroscopic(lbm_t h, double* rho, double* u);

/* Canonical populations f[Q*N] (FP64, [Q][N]); host or device.  Shifted
 * storage is un-shifted (f = stored + t_k).  Solid cells read 0.  With a host
 * buffer: synchronises the stream and returns LBM_ERR_TIMEOUT if a staged
 * step gave up waiting (see lbm_step). */
LBM_API int lbm_get_populations(lbm_t h, double* f);

/* Load canonical populations f[Q*N]; host or device.  Solid-cell entries are
 * ignored.  Resets the time-step parity. */
LBM_API int lbm_set_populations(lbm_t h, const double* f);

/* FP64 sums over fluid cells: mass = sum rho, energy = sum rho |u|^2 / 2.
 * Host outputs; synchronises the stream.  LBM_ERR_TIMEOUT if a staged step
 * gave up waiting (see lbm_step); else LBM_ERR_DIVERGED if either sum is not
 * finite (the outputs are still written). */
LBM_API int lbm_reduce(lbm_t h, double* mass, double* energy);

/* Number of time iterations taken since the populations were last written. */
LBM_API int lbm_steps_done(lbm_t h, long long* steps);

/* Device bytes the handle holds (populations, flags, tables, scratch). */
LBM_API int lbm_device_bytes(lbm_t h, size_t* bytes);

/* Algorithmic bytes moved per cell update by the handle's step (populations
 * read + written + the 1-byte cell flag), for roofline accounting. */
LBM_API int lbm_bytes_per_cell_update(lbm_t h, double* bytes);

/* Number of kernel launches one time step of the handle makes (*n >= 1):
 * 1 for the one-thread-per-cell kernels; 2 for swap (collision, then the
 * streaming pass) and for the staged AA steps of SoA storage in FP16 (every
 * model) and in FP64 (BGK-W2 and TRT, and RR on D3Q27): the
 * shared-memory-staged kernel over the bulk cells, then the kernel over the
 * cells next to a wall or on a domain face, if there are any.  May build the latter's cell list (device memory it
 * owns; see lbm_device_bytes). */
LBM_API int lbm_kernels_per_step(lbm_t h, int* n);

/* Bounds checks (no counterpart in the paper; a test and debugging aid).
 * liblbm_debug.so, built from the same sources with -DLBM_DEBUG (collision
 * models BGK-W2, TRT and K only), checks in every kernel each population load
 * and store against the array's Q N populations, each own or neighbour cell
 * index and flag / mask read against [0, N), each bulk copy of the staged
 * steps against the array plus its 128 bytes of padding, and each read of a
 * staged run against the run in shared memory.  A failed check records the
 * handle's first fault and skips the access (a skipped load reads 0); nothing
 * traps.  The padding past the population and flag arrays holds canary bytes
 * (0xA5) in that build.
 *   Synchronises the handle's streams, then *fault = 0 when no check failed
 *   and every canary is intact; else kind << 56 | index: kind 1 population
 *   load, 2 population store (index: element), 3 cell, 4 flag read, 5 mask
 *   read (index: cell), 6 staged population copy, 7 staged flag copy (index:
 *   end of the copy), 8 staged run read (index in the run), 9 link-fraction
 *   row, 10 canary (array 0 / 1 populations, 2 flags, in bits 32..39; byte of
 *   the padding below).  The device fault word is cleared by the read.
 * liblbm.so has no checks: it sets *fault = 0 and returns
 * LBM_ERR_UNSUPPORTED. */
LBM_API int lbm_debug_check(lbm_t h, unsigned long long* fault);

/* Free everything the handle owns.  NULL is accepted. */
LBM_API int lbm_destroy(lbm_t h);

/* 1 if (lattice, scheme, collision, layout, precision) is built, else 0. */
LBM_API int lbm_supported(int lattice, int scheme, int collision, int layout, int precision);

/* Text of the calling thread's last error ("" if none). */
LBM_API const char* lbm_last_error(void);

/* ======================================================================
 * Batched stepping of many independent lattices: one kernel launch per time
 * step covers every member (no counterpart in the paper; the paper steps one
 * lattice).  Members must share lattice, collision model and precision and
 * use the AA pattern with the SoA layout.  They keep their own memory,
 * parameters and time-step parity; a batched step is bit-identical to
 * stepping each member alone.  Work runs on the batch stream (by default an
 * internal stream that orders with the legacy default stream); members on
 * other streams are synchronised before each batch call.  A member must not
 * be stepped or read on its own while a batch call may still be running:
 * call lbm_batch_sync first.
 * ====================================================================== */
typedef struct lbm_batch_s* lbm_batch_t;

LBM_API int lbm_batch_create(lbm_batch_t* out);
/* Add a handle; LBM_ERR_INVALID_ARG if it does not match the first member. */
LBM_API int lbm_batch_add(lbm_batch_t b, lbm_t h);
/* Remove a handle (waits for the batch stream). */
LBM_API int lbm_batch_remove(lbm_batch_t b, lbm_t h);
/* Threads per block (32..256, multiple of 32) and cells per thread (1, 2, 4);
 * 0 selects the defaults (256, 1). */
LBM_API int lbm_batch_set_launch(lbm_batch_t b, int threads_per_block, int cells_per_thread);
/* Time every (threads, cells-per-thread) shape in {32,64,128,256} x {1,2,4}
 * on the batch as it stands (CUDA events on the batch stream) and keep the
 * fastest.  The trial steps advance the members (6 steps per shape).  The
 * choice is cached per (lattice, collision, precision, size class =
 * floor(log2(mean member cells))) for the process; a cached choice is reused
 * without trials.  Outputs may be NULL. */
LBM_API int lbm_batch_autotune(lbm_batch_t b, int* threads_per_block, int* cells_per_thread);
/* Advance every member by n >= 0 steps, one launch per step; with
 * use_graph != 0 the n launches are captured once into a CUDA graph and
 * replayed by later calls with the same n and membership.  Asynchronous. */
LBM_API int lbm_batch_step(lbm_batch_t b, int n, int use_graph);
/* Launch the batch's steps on a caller's stream (NULL: the batch's own blocking stream).  A
 * change of stream first waits for the steps already enqueued on the previous one; a member's
 * work on its own stream, or on the legacy default stream, is waited for when the membership
 * changes.  LBM_ERR_INVALID_ARG for a NULL batch, LBM_ERR_CUDA on a failed wait. */
LBM_API int lbm_batch_set_stream(lbm_batch_t b, void* stream);
LBM_API int lbm_batch_sync(lbm_batch_t b);
LBM_API int lbm_batch_size(lbm_batch_t b, int* members, long long* cells);
LBM_API int lbm_batch_destroy(lbm_batch_t b);

/* FP64 conserved sums over caller-owned device buffers, without allocating.
 * No counterpart in the paper: this exists for callers that cannot let the
 * library call cudaMalloc -- an application that hands out every device
 * buffer from its own pool, a real-time loop that cannot take the implicit
 * synchronisation of cudaMalloc/cudaFree, or an environment with a fixed
 * device-memory budget.  It computes what lbm_reduce computes, from
 * canonical populations instead of a handle.
 *   lattice: 19 or 27.  N: cells, 1 <= N <= 33,554,432 (larger N is rejected
 *   with LBM_ERR_INVALID_ARG: the fixed scratch holds partial sums for 16,384
 *   blocks of 2,048 cells).  f: device pointer, FP64 canonical populations
 *   [Q][N].  flags: device pointer, one byte per cell, 0 = fluid, 1..7 =
 *   solid (solid cells are skipped).  out: device pointer to 2 doubles,
 *   receives {sum rho, sum rho |u|^2 / 2} over fluid cells.  stream: a
 *   cudaStream_t of the current device, or NULL.  Asynchronous: out is
 *   written when the stream reaches the kernels.
 * Scratch: a 256 KiB array in device global memory, fixed in the library
 * image, which every GPU that loads the library keeps until the process
 * exits.  Its address is looked up (cudaGetSymbolAddress) on the first call
 * made in each device context, with that device current, and kept for that
 * context (keyed by the context's unique id, so that a context made again
 * after cudaDeviceReset is looked up afresh); make the first call on a device
 * before any stream capture.  All calls share the array: calls whose kernels
 * overlap on the GPU (different streams, or concurrent host threads) race
 * and must be serialised by the caller.  No cudaMalloc, cudaFree or
 * allocating routine is called.  Pointers that are not device memory of the
 * current device (or managed memory), and a stream of another device, are
 * rejected with LBM_ERR_INVALID_ARG before any kernel runs; the sizes of the
 * buffers cannot be checked here and are the caller's to get right. */
LBM_API int lbm_conserved_sums_static(int lattice, int N, const double* f, const uint8_t* flags, double* out,
                                      void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
