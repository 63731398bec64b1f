// api.cu -- host side of the C ABI declared in include/lbm.h.
//
// A handle owns its device buffers (classified flags, one or two population
// arrays, the wall-term table, reduction partials and a staging buffer for
// host transfers) and enqueues every kernel on its stream.  The time-step
// parity and, for the two-population scheme, the current array are host
// state; step kernels are looked up once per (model, lattice, precision,
// layout, step kind) from the compiled tables.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "handle.h"
#include "internal.h"
#include "kernels.cuh"
#include "lbm.h"

using namespace lbm;

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(call)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

size_t elem_size(int prec) { return prec == F64 ? 8 : (prec == F32 ? 4 : 2); }

template <int Q>
void fill_wall_table(const double (&wall_u)[8][3], double* out) {
  // W[kind][k] = -6 t_k rho_w c_k.u_w(kind), rho_w = 1 (Section 2.1)
  for (int fl = 0; fl < 8; ++fl)
    for (int k = 0; k < Q; ++k) {
      const double cu = Lat<Q>::c(k, 0) * wall_u[fl][0] + Lat<Q>::c(k, 1) * wall_u[fl][1] +
                        Lat<Q>::c(k, 2) * wall_u[fl][2];
      out[fl * Q + k] = fl <= 1 ? 0.0 : -6.0 * Lat<Q>::w(k) * 1.0 * cu;
    }
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
}  // namespace

int lbm::set_error(int code, const char* msg) { return fail(code, msg); }


namespace {

size_t pop_bytes(const lbm_s* h) { return (size_t)h->Q * (size_t)h->N * elem_size(h->prec); }

int resolve_kernels(lbm_s* h) {
  for (int sk = 0; sk < NUM_STEP_KINDS; ++sk) h->fns[sk] = step_fn(h->model, h->Q, h->prec, h->layout, sk);
  if (!h->fns[K_TWOPOP]) return fail(LBM_ERR_UNSUPPORTED, "combination of lattice, model, precision and layout is not built");
  const bool staged = h->scheme == LBM_AA && h->layout == SOA;
  h->sfns[0] = staged ? staged_fn(h->model, h->Q, h->prec, K_AA_EVEN) : nullptr;
  h->sfns[1] = staged ? staged_fn(h->model, h->Q, h->prec, K_AA_ODD) : nullptr;
  for (int sk = 0; sk < NUM_STEP_KINDS; ++sk) h->sumfns[sk] = step_sum_fn(h->model, h->Q, h->prec, h->layout, sk);
  for (int sk = 0; sk < NUM_STEP_KINDS; ++sk) h->cfns[sk] = curved_fn(h->model, h->Q, h->prec, h->layout, sk);
  return LBM_OK;
}

KArgs make_args(const lbm_s* h);

// sorted list of the fluid cells with a non-zero flag byte and its per-tile
// offsets, built once per handle before the first staged step (the flags never
// change after lbm_create)
int ensure_nonbulk_list(lbm_s* h) {
  if (h->nlist >= 0) return LBM_OK;
  const int tile = staged_tile(h->Q);
  const int ntiles = (h->N + tile - 1) / tile;
  std::vector<int> off((size_t)ntiles + 1, 0);
  LBM_CUDA(cudaMalloc(&h->d_tile_off, sizeof(int) * ((size_t)ntiles + 1)));
  LBM_CUDA(launch_list_count(h->d_flags, h->N, tile, h->d_tile_off, h->stream));
  LBM_CUDA(cudaMemcpyAsync(off.data(), h->d_tile_off, sizeof(int) * (size_t)ntiles, cudaMemcpyDeviceToHost,
                           h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  long long run = 0;
  for (int t = 0; t < ntiles; ++t) {
    const int c = off[t];
    off[t] = (int)run;
    run += c;
  }
  off[ntiles] = (int)run;
  LBM_CUDA(cudaMemcpyAsync(h->d_tile_off, off.data(), sizeof(int) * ((size_t)ntiles + 1), cudaMemcpyHostToDevice,
                           h->stream));
  if (run > 0) {
    LBM_CUDA(cudaMalloc(&h->d_list, sizeof(int) * (size_t)run));
    LBM_CUDA(cudaMalloc(&h->d_list_mask, sizeof(uint32_t) * (size_t)run));
    LBM_CUDA(cudaMalloc(&h->d_list_kinds, 2 * sizeof(unsigned long long) * (size_t)run));
    LBM_CUDA(launch_list_fill(h->d_flags, h->N, tile, h->d_tile_off, h->d_list, h->stream));
    LBM_CUDA(launch_listed_records(h->Q, make_args(h), h->d_list, (int)run, h->d_list_mask, h->d_list_kinds,
                                   h->stream));
  }
  LBM_CUDA(cudaStreamSynchronize(h->stream));  // `off` is read by the copy above
  LBM_CUDA(cudaFree(h->d_tile_off));           // only needed to sort the list
  h->d_tile_off = nullptr;
  h->nlist = (int)run;
  if (run > 0 && !h->side.side) {
    LBM_CUDA(cudaStreamCreateWithFlags(&h->side.side, cudaStreamNonBlocking));
    LBM_CUDA(cudaEventCreateWithFlags(&h->side.fork, cudaEventDisableTiming));
    LBM_CUDA(cudaEventCreateWithFlags(&h->side.join, cudaEventDisableTiming));
  }
  return LBM_OK;
}

// LBM_ERR_TIMEOUT if a staged kernel recorded a bounded wait that gave up
// (reads the device error word; the caller has synchronised the stream)
int check_device_error(lbm_s* h) {
  int w = 0;
  LBM_CUDA(cudaMemcpy(&w, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (w != 0) return fail(LBM_ERR_TIMEOUT, "a staged step kernel gave up waiting for its staged copies");
  return LBM_OK;
}

int ensure_alloc(lbm_s* h) {
  if (h->d_pop[0]) return LBM_OK;
  const size_t need = pop_bytes(h) * (size_t)h->npop;
  size_t freeb = 0, total = 0;
  LBM_CUDA(cudaMemGetInfo(&freeb, &total));
  if (need + (size_t(256) << 20) > freeb)
    return fail(LBM_ERR_OOM, "populations need " + std::to_string(need >> 20) + " MiB, " +
                                 std::to_string(freeb >> 20) + " MiB free");
  for (int a = 0; a < h->npop; ++a) {
    // the staged kernels copy whole 128-byte units, up to STAGE_PAD_BYTES past the end
    LBM_CUDA(cudaMalloc(&h->d_pop[a], pop_bytes(h) + STAGE_PAD_BYTES));
    LBM_CUDA(cudaMemsetAsync(h->d_pop[a], 0, pop_bytes(h) + STAGE_PAD_BYTES, h->stream));
    // bounds-checked build: the padding holds canary bytes that no kernel may write
    LBM_IF_DEBUG(LBM_CUDA(cudaMemsetAsync(static_cast<unsigned char*>(h->d_pop[a]) + pop_bytes(h), DEBUG_CANARY,
                                          STAGE_PAD_BYTES, h->stream));)
  }
  return LBM_OK;
}

int ensure_stage(lbm_s* h, size_t bytes) {
  if (h->stage_bytes >= bytes) return LBM_OK;
  if (h->d_stage) {
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    LBM_CUDA(cudaFree(h->d_stage));
    h->d_stage = nullptr;
    h->stage_bytes = 0;
  }
  LBM_CUDA(cudaMalloc(&h->d_stage, bytes));
  h->stage_bytes = bytes;
  return LBM_OK;
}

int upload_wall(lbm_s* h) {
  if (!h->wall_dirty) return LBM_OK;
  if (h->Q == 19) fill_wall_table<19>(h->wall_u, h->wall_table);
  else fill_wall_table<27>(h->wall_u, h->wall_table);
  LBM_CUDA(cudaMemcpyAsync(h->d_wall, h->wall_table, sizeof(double) * 8 * h->Q, cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA(cudaMemcpyAsync(h->d_wallu, h->wall_u, sizeof(double) * 24, cudaMemcpyHostToDevice, h->stream));
  // the host tables are members of the handle and outlive the copies
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  h->wall_dirty = false;
  return LBM_OK;
}

#ifdef LBM_DEBUG
// the 64-bit fault word of the bounds-checked build (after the staged error
// word and the scratch counter)
unsigned long long* debug_word(const lbm_s* h) { return reinterpret_cast<unsigned long long*>(h->d_err + 2); }
#endif

KArgs make_args(const lbm_s* h) {
  KArgs a;
  a.a = h->d_pop[h->cur];
  a.b = h->npop > 1 ? h->d_pop[1 - h->cur] : nullptr;
  a.flags = h->d_flags;
  a.nbmask = h->d_nbmask;
  a.wall = h->d_wall;
  a.qidx = h->d_qidx;
  a.qtab = h->d_qtab;
  a.nx = h->nx;
  a.ny = h->ny;
  a.nz = h->nz;
  a.N = h->N;
  a.parity = (int)(h->steps & 1);
#ifdef LBM_DEBUG
  a.dbg = debug_word(h);
  a.dbg_elems = (size_t)h->Q * (size_t)h->N;
  a.dbg_qrows = h->qrows;
#endif
  const double w = h->omega, wb = h->bulk_follows ? h->omega : h->omega_bulk;
  a.omega = w;
  a.omc = 1.0 - w;
  a.wminus = (wb - w) / 3.0;
  a.wplus = a.wminus + w;
  a.omega_high = h->omega_high;
  a.trt_minus = 1.0 / (0.5 + h->lambda / (1.0 / w - 0.5));
  a.fx_wide = h->fx_wide ? 1 : 0;
  if (h->Q == 19) {
    derived_rates<19>(w, a.trt_minus, a.wt, a.wt3, a.wm3, a.hs, a.hd);
    a.dk = derived_dfk<19>(a.omc, a.wt, a.wt3, a.wm3, a.hs, a.hd, a.wplus, a.wminus, h->fx_wide);
  } else {
    derived_rates<27>(w, a.trt_minus, a.wt, a.wt3, a.wm3, a.hs, a.hd);
    a.dk = derived_dfk<27>(a.omc, a.wt, a.wt3, a.wm3, a.hs, a.hd, a.wplus, a.wminus, h->fx_wide);
  }
  return a;
}

int load_kind(const lbm_s* h) {
  const bool odd = (h->steps & 1) != 0;
  switch (h->scheme) {
    case LBM_AA: return odd ? LD_AA_ODD : LD_LOCAL;
    case LBM_ESOTWIST: return odd ? LD_ET_ODD : LD_ET_EVEN;
    default: return LD_LOCAL;
  }
}

int store_kind(const lbm_s* h) { return h->scheme == LBM_ESOTWIST ? LD_ET_EVEN : LD_LOCAL; }

bool nw4_equilibrium(int model) {
  return !(model == BGK_W2 || model == TRT || model == REG || model == BGK_W2_EDU || model == BGK_W2_LOOP);
}

int reset_populations(lbm_s* h) {
  int rc = ensure_alloc(h);
  if (rc) return rc;
  h->cur = 0;
  h->steps = 0;
  for (int a = 0; a < h->npop; ++a) LBM_CUDA(cudaMemsetAsync(h->d_pop[a], 0, pop_bytes(h), h->stream));
  return upload_wall(h);
}

// range of the FP64 BGK-W2 / TRT fast path (fx64.cuh) for the state just
// written: forced by LBM_PARAM_FX_RANGE, or, in auto mode, wide when more than
// 1 % of the fluid cells have a population outside its weight's binade (each
// would take the FP64 operator in the narrow range).  Auto mode synchronises
// the stream to read the count.
int decide_fx_range(lbm_s* h, bool rest = false) {
  const bool fx = h->prec == F64 && (h->model == BGK_W2 || h->model == TRT);
  if (!fx || h->fx_mode != 0) {
    h->fx_wide = fx && h->fx_mode == 2;
    return LBM_OK;
  }
  if (!h->populated || rest) {
    h->fx_wide = false;  // the rest state: every population equals its weight
    return LBM_OK;
  }
  int* count = h->d_err + 1;
  LBM_CUDA(cudaMemsetAsync(count, 0, sizeof(int), h->stream));
  const KArgs a = make_args(h);
  LBM_CUDA(launch_fx_range_count(h->Q, h->prec, h->layout, load_kind(h), a, count, h->stream));
  int n = 0;
  LBM_CUDA(cudaMemcpyAsync(&n, count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  h->fx_wide = (long long)n * 100 > h->nfluid;
  return LBM_OK;
}

int init_eq_device(lbm_s* h, const double* rho, const double* u) {
  int rc = reset_populations(h);
  if (rc) return rc;
  KArgs a = make_args(h);
  LBM_CUDA(launch_init(h->Q, h->prec, h->layout, store_kind(h), nw4_equilibrium(h->model), a, rho, u, h->stream));
  h->populated = true;
  return decide_fx_range(h, !rho && !u);
}

int valid_omega(double w) { return std::isfinite(w) && w > 0.0 && w < 2.0; }

}  // namespace

int lbm::handle_prepare(lbm_s* h) {
  if (!h->populated) {
    int rc = init_eq_device(h, nullptr, nullptr);
    if (rc) return rc;
  }
  return upload_wall(h);
}

void lbm::handle_rates(const lbm_s* h, CP<double>* rd, CP<float>* rf) {
  const KArgs a = make_args(h);
  rd->omega = a.omega;
  rd->omc = a.omc;
  rd->wplus = a.wplus;
  rd->wminus = a.wminus;
  rd->omega_high = a.omega_high;
  rd->trt_minus = a.trt_minus;
  for (int c = 0; c < 4; ++c) {
    rd->wt[c] = a.wt[c];
    rd->wt3[c] = a.wt3[c];
    rd->wm3[c] = a.wm3[c];
  }
  rd->hs = a.hs;
  rd->hd = a.hd;
  rd->dk = a.dk;
  // host conversion rounds to nearest, as the kernels' conversion of their parameters does
  rf->omega = (float)rd->omega;
  rf->omc = (float)rd->omc;
  rf->wplus = (float)rd->wplus;
  rf->wminus = (float)rd->wminus;
  rf->omega_high = (float)rd->omega_high;
  rf->trt_minus = (float)rd->trt_minus;
  for (int c = 0; c < 4; ++c) {
    rf->wt[c] = (float)rd->wt[c];
    rf->wt3[c] = (float)rd->wt3[c];
    rf->wm3[c] = (float)rd->wm3[c];
  }
  rf->hs = (float)rd->hs;
  rf->hd = (float)rd->hd;
  rf->dk = rd->dk;
}

extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

int lbm_supported(int lattice, int scheme, int collision, int layout, int precision) {
  if (lattice != 19 && lattice != 27) return 0;
  if (scheme < LBM_TWOPOP || scheme > LBM_ESOTWIST) return 0;
  if (collision < 0 || collision >= NUM_MODELS) return 0;
  if (layout != LBM_SOA && layout != LBM_AOS) return 0;
  if (precision < LBM_F64 || precision > LBM_F16) return 0;
  return step_fn(collision, lattice, precision, layout, K_TWOPOP) != nullptr ? 1 : 0;
}

int lbm_create(lbm_t* out, int lattice, int nx, int ny, int nz, int scheme, int collision, double omega,
               const uint8_t* flags) {
  if (!out) return fail(LBM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (lattice != 19 && lattice != 27) return fail(LBM_ERR_INVALID_ARG, "lattice must be 19 or 27");
  if (nx < 1 || ny < 1 || nz < 1) return fail(LBM_ERR_INVALID_ARG, "dimensions must be >= 1");
  const long long N = (long long)nx * ny * nz;
  // cell indices are 32-bit; the headroom keeps one-thread-per-cell indices of
  // the last block and grid-stride loop indices from overflowing
  if (N > LBM_MAX_CELLS) return fail(LBM_ERR_INVALID_ARG, "nx*ny*nz must be <= 2^31 - 2^22");
  if (scheme < LBM_TWOPOP || scheme > LBM_ESOTWIST) return fail(LBM_ERR_INVALID_ARG, "unknown scheme");
  if (collision < 0 || collision >= NUM_MODELS) return fail(LBM_ERR_INVALID_ARG, "unknown collision model");
  if (!valid_omega(omega)) return fail(LBM_ERR_INVALID_ARG, "omega must be in (0, 2)");
  if (!flags) return fail(LBM_ERR_INVALID_ARG, "flags is NULL");
  for (long long i = 0; i < N; ++i)
    if (flags[i] > 7) return fail(LBM_ERR_INVALID_ARG, "flag values must be 0..7");
  long long nfluid = 0;
  for (long long i = 0; i < N; ++i) nfluid += flags[i] == 0;

  lbm_s* h = new lbm_s();
  h->Q = lattice;
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->N = (int)N;
  h->nfluid = nfluid;
  h->scheme = scheme;
  h->model = collision;
  h->omega = omega;
  h->npop = scheme == LBM_TWOPOP ? 2 : 1;
  h->threads = step_threads(h->prec);
  int rc = resolve_kernels(h);
  if (rc) {
    delete h;
    return rc;
  }
  uint8_t* raw = nullptr;
  cudaError_t e = cudaMalloc(&h->d_flags, N + STAGE_PAD_BYTES);  // padded as the populations
  if (e == cudaSuccess) e = cudaMemset(h->d_flags, 0, N + STAGE_PAD_BYTES);
  LBM_IF_DEBUG(if (e == cudaSuccess) e = cudaMemset(h->d_flags + N, DEBUG_CANARY, STAGE_PAD_BYTES);)
  // [0] staged-kernel error word, [1] scratch counter, [2..3] the 64-bit fault
  // word of the bounds-checked build
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_nbmask, sizeof(uint32_t) * N);
  if (e == cudaSuccess) e = cudaMalloc(&raw, N);
  if (e == cudaSuccess) e = cudaMemcpy(raw, flags, N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_classify(lattice, raw, h->d_flags, h->d_nbmask, nx, ny, nz, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (raw) cudaFree(raw);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_wall, sizeof(double) * 8 * 27);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_wallu, sizeof(double) * 24);
  if (e == cudaSuccess) {
    h->partials = reduce_partials_count(h->N);
    e = cudaMalloc(&h->d_partials, sizeof(double) * (2 * h->partials + 2));
  }
  if (e != cudaSuccess) {
    lbm_destroy(h);
    return cuda_fail(e, "lbm_create");
  }
  *out = h;
  return LBM_OK;
}

int lbm_set_layout(lbm_t h, int layout) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  if (layout != LBM_SOA && layout != LBM_AOS) return fail(LBM_ERR_INVALID_ARG, "unknown layout");
  if (h->populated) return fail(LBM_ERR_STATE, "layout can only change before populations are written");
  if (!lbm_supported(h->Q, h->scheme, h->model, layout, h->prec))
    return fail(LBM_ERR_UNSUPPORTED, "layout not built for this precision (AoS is FP64 only)");
  for (int a = 0; a < 2; ++a)
    if (h->d_pop[a]) {
      cudaFree(h->d_pop[a]);
      h->d_pop[a] = nullptr;
    }
  h->layout = layout;
  return resolve_kernels(h);
}

int lbm_set_precision(lbm_t h, int precision) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  if (precision < LBM_F64 || precision > LBM_F16) return fail(LBM_ERR_INVALID_ARG, "unknown precision");
  if (h->populated) return fail(LBM_ERR_STATE, "precision can only change before populations are written");
  if (!lbm_supported(h->Q, h->scheme, h->model, h->layout, precision))
    return fail(LBM_ERR_UNSUPPORTED, "precision not built for this layout (FP32/FP16 are SoA only)");
  for (int a = 0; a < 2; ++a)
    if (h->d_pop[a]) {
      cudaFree(h->d_pop[a]);
      h->d_pop[a] = nullptr;
    }
  h->prec = precision;
  h->threads = step_threads(h->prec);
  return resolve_kernels(h);
}

int lbm_set_wall_velocity(lbm_t h, int flag, double ux, double uy, double uz) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  if (flag < 2 || flag > 7) return fail(LBM_ERR_INVALID_ARG, "moving-wall flags are 2..7");
  if (!std::isfinite(ux) || !std::isfinite(uy) || !std::isfinite(uz))
    return fail(LBM_ERR_INVALID_ARG, "wall velocity must be finite");
  h->wall_u[flag][0] = ux;
  h->wall_u[flag][1] = uy;
  h->wall_u[flag][2] = uz;
  h->wall_dirty = true;
  return LBM_OK;
}

int lbm_set_link_fractions(lbm_t h, const double* q) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  const int Q = h->Q, N = h->N;
  std::vector<int> qidx, cells;
  std::vector<double> rows;
  if (q) {
    // the classified flag bytes: wall kind in bits 0..2
    std::vector<uint8_t> fl((size_t)N);
    LBM_CUDA(cudaMemcpyAsync(fl.data(), h->d_flags, (size_t)N, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    int cv[27][3];
    for (int k = 0; k < Q; ++k)
      for (int d = 0; d < 3; ++d) cv[k][d] = Q == 19 ? Lat<19>::c(k, d) : Lat<27>::c(k, d);
    qidx.assign((size_t)N, -1);
    cells.clear();
    const int sxy = h->ny * h->nz;
    for (int i = 0; i < N; ++i) {
      if (fl[(size_t)i] & FLAG_KIND) continue;
      const int x = i / sxy, y = (i / h->nz) % h->ny, z = i % h->nz;
      bool curved = false;
      for (int k = 0; k < Q; ++k) {
        const int xn = (x + cv[k][0] + h->nx) % h->nx, yn = (y + cv[k][1] + h->ny) % h->ny,
                  zn = (z + cv[k][2] + h->nz) % h->nz;
        if (!(fl[(size_t)((xn * h->ny + yn) * h->nz + zn)] & FLAG_KIND)) continue;
        const double v = q[(size_t)k * N + i];
        if (!(v > 0.0 && v <= 1.0))
          return fail(LBM_ERR_INVALID_ARG, "link fraction of cell " + std::to_string(i) + ", link " +
                                               std::to_string(k) + " is not in (0, 1]");
        if (v != 0.5) curved = true;
      }
      if (!curved) continue;
      qidx[(size_t)i] = (int)(rows.size() / Q);
      cells.push_back(i);
      for (int k = 0; k < Q; ++k) rows.push_back(q[(size_t)k * N + i]);
    }
  }
  // replace the tables (the previous steps must be done with them)
  const bool had = h->nqcells > 0;
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (h->d_qidx) LBM_CUDA(cudaFree(h->d_qidx));
  if (h->d_qtab) LBM_CUDA(cudaFree(h->d_qtab));
  if (h->d_qcells) LBM_CUDA(cudaFree(h->d_qcells));
  h->d_qidx = nullptr;
  h->d_qtab = nullptr;
  h->d_qcells = nullptr;
  h->qrows = 0;
  h->nqcells = 0;
  if (!rows.empty()) {
    LBM_CUDA(cudaMalloc(&h->d_qidx, sizeof(int) * (size_t)N));
    LBM_CUDA(cudaMalloc(&h->d_qtab, sizeof(double) * rows.size()));
    LBM_CUDA(cudaMalloc(&h->d_qcells, sizeof(int) * cells.size()));
    LBM_CUDA(cudaMemcpyAsync(h->d_qidx, qidx.data(), sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(cudaMemcpyAsync(h->d_qtab, rows.data(), sizeof(double) * rows.size(), cudaMemcpyHostToDevice,
                             h->stream));
    LBM_CUDA(cudaMemcpyAsync(h->d_qcells, cells.data(), sizeof(int) * cells.size(), cudaMemcpyHostToDevice,
                             h->stream));
    h->qrows = (int)(rows.size() / Q);
    h->nqcells = (int)cells.size();
  }
  LBM_CUDA(launch_mark_curved(h->d_nbmask, h->d_qidx, N, h->stream));
  // the listed-cell records carry the mark: build them again at the next staged step
  if (h->nlist >= 0 && (had || h->nqcells > 0)) {
    if (h->d_list) LBM_CUDA(cudaFree(h->d_list));
    if (h->d_list_mask) LBM_CUDA(cudaFree(h->d_list_mask));
    if (h->d_list_kinds) LBM_CUDA(cudaFree(h->d_list_kinds));
    h->d_list = nullptr;
    h->d_list_mask = nullptr;
    h->d_list_kinds = nullptr;
    h->nlist = -1;
  }
  LBM_CUDA(cudaStreamSynchronize(h->stream));  // the host tables above are freed on return
  return LBM_OK;
}

int lbm_set_param(lbm_t h, int key, double v) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  switch (key) {
    case LBM_PARAM_OMEGA:
      if (!valid_omega(v)) return fail(LBM_ERR_INVALID_ARG, "omega must be in (0, 2)");
      h->omega = v;
      return LBM_OK;
    case LBM_PARAM_OMEGA_BULK:
      if (!valid_omega(v)) return fail(LBM_ERR_INVALID_ARG, "omega_bulk must be in (0, 2)");
      h->omega_bulk = v;
      h->bulk_follows = false;
      return LBM_OK;
    case LBM_PARAM_OMEGA_HIGH:
      if (!(std::isfinite(v) && v > 0.0 && v <= 2.0)) return fail(LBM_ERR_INVALID_ARG, "omega_high must be in (0, 2]");
      h->omega_high = v;
      return LBM_OK;
    case LBM_PARAM_TRT_LAMBDA:
      if (!(std::isfinite(v) && v > 0.0)) return fail(LBM_ERR_INVALID_ARG, "lambda must be > 0");
      h->lambda = v;
      return LBM_OK;
    case LBM_PARAM_WAIT_CYCLES:
      if (!(std::isfinite(v) && v >= 1.0 && v <= 1099511627776.0))
        return fail(LBM_ERR_INVALID_ARG, "wait_cycles must be in [1, 2^40]");
      h->wait_cycles = (long long)v;
      return LBM_OK;
    case LBM_PARAM_FX_RANGE:
      if (!(v == 0.0 || v == 1.0 || v == 2.0)) return fail(LBM_ERR_INVALID_ARG, "fx range must be 0, 1 or 2");
      h->fx_mode = (int)v;
      return decide_fx_range(h);
    default:
      return fail(LBM_ERR_INVALID_ARG, "unknown parameter key");
  }
}

int lbm_set_stream(lbm_t h, void* stream) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  h->stream = (cudaStream_t)stream;
  return LBM_OK;
}

int lbm_init_equilibrium(lbm_t h, const double* rho, const double* u) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  const size_t N = (size_t)h->N;
  const bool dev_r = !rho || is_device_pointer(rho), dev_u = !u || is_device_pointer(u);
  if (dev_r && dev_u) return init_eq_device(h, rho, u);
  int rc = ensure_stage(h, sizeof(double) * 4 * N);
  if (rc) return rc;
  double* st = (double*)h->d_stage;
  const double* dr = rho;
  const double* du = u;
  if (rho && !dev_r) {
    LBM_CUDA(cudaMemcpyAsync(st, rho, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    dr = st;
  }
  if (u && !dev_u) {
    LBM_CUDA(cudaMemcpyAsync(st + N, u, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, h->stream));
    du = st + N;
  }
  return init_eq_device(h, dr, du);
}

namespace {
// blocks of the handle's summing step kernel (one pair of partial sums each)
int sum_blocks(const lbm_s* h) {
  const long long chunk = (long long)h->threads * sum_cells_per_thread(h->prec);
  return (int)((h->N + chunk - 1) / chunk);
}

// step kind of the handle's next step
int next_step_kind(const lbm_s* h) {
  switch (h->scheme) {
    case LBM_TWOPOP: return K_TWOPOP;
    case LBM_AA: return (h->steps & 1) ? K_AA_ODD : K_AA_EVEN;
    case LBM_SWAP: return K_AA_EVEN;
    default: return K_ESOTWIST;
  }
}

Listed listed_of(const lbm_s* h) {
  Listed listed;
  listed.cell = h->d_list;
  listed.mask = h->d_list_mask;
  listed.kinds = h->d_list_kinds;
  listed.n = h->nlist;
  return listed;
}

// pairs of partial sums a summing step of the handle writes: its summing step
// kernel's blocks, or the staged step's (0 if neither exists)
int step_sum_parts(lbm_s* h, int* nparts) {
  *nparts = 0;
  const bool staged = h->scheme == LBM_AA && h->sfns[(int)(h->steps & 1)];
  if (staged) {
    int rc = ensure_nonbulk_list(h);
    if (rc) return rc;
    const cudaError_t e = h->sfns[(int)(h->steps & 1)](make_args(h), h->d_err, h->wait_cycles, listed_of(h),
                                                       h->side, h->stream, nullptr, nparts);
    if (e == cudaErrorNotSupported) *nparts = 0;
    else if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
  }
  // the summing step kernels leave the cells with walls at a fraction of their
  // links (and their sums) to the curved-cell kernel: reduce separately then
  if (h->sumfns[next_step_kind(h)] && h->nqcells == 0) *nparts = sum_blocks(h);
  return LBM_OK;
}

// enqueue one time step; with sum_partials, the step's kernel also writes the
// per-block FP64 sums of the state it reads (returns the number of blocks in
// *nparts), and the caller guarantees that a summing kernel exists
int enqueue_step(lbm_s* h, double* sum_partials = nullptr, int* nparts = nullptr) {
  KArgs a = make_args(h);
  cudaError_t e = cudaSuccess;
  auto kernel = [&](int sk) {
    cudaError_t r;
    if (sum_partials) {
      *nparts = sum_blocks(h);
      r = h->sumfns[sk](a, h->threads, sum_partials, h->stream);
    } else {
      r = h->fns[sk](a, h->threads, h->stream);
    }
    // the cells with walls at a fraction of their links, which the step kernel left alone
    if (r == cudaSuccess && h->nqcells > 0) r = h->cfns[sk](a, h->d_qcells, h->nqcells, h->stream);
    return r;
  };
  switch (h->scheme) {
    case LBM_TWOPOP:
      e = kernel(K_TWOPOP);
      h->cur ^= 1;
      break;
    case LBM_AA: {
      const int odd = (int)(h->steps & 1);
      if (h->sfns[odd]) {
        const int rc = ensure_nonbulk_list(h);
        if (rc) return rc;
        e = h->sfns[odd](a, h->d_err, h->wait_cycles, listed_of(h), h->side, h->stream, sum_partials,
                         sum_partials ? nparts : nullptr);
      } else {
        e = kernel(odd ? K_AA_ODD : K_AA_EVEN);
      }
      break;
    }
    case LBM_SWAP:
      e = kernel(K_AA_EVEN);
      if (e == cudaSuccess) e = launch_swap_stream(h->Q, h->prec, h->layout, a, h->threads, h->stream);
      break;
    case LBM_ESOTWIST:
      e = kernel(K_ESOTWIST);
      break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
  ++h->steps;
  return LBM_OK;
}

}  // namespace

int lbm_step(lbm_t h, int n) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0) return fail(LBM_ERR_INVALID_ARG, "n must be >= 0");
  if (!h->populated) {
    int rc = init_eq_device(h, nullptr, nullptr);
    if (rc) return rc;
  }
  int rc = upload_wall(h);
  if (rc) return rc;
  for (int s = 0; s < n; ++s) {
    rc = enqueue_step(h);
    if (rc) return rc;
  }
  return LBM_OK;
}

}  // extern "C"

namespace {
// enqueue lbm_step_sums' work on the handle's stream: the sums of the current
// state land in the two doubles at *out2 (device memory of the handle)
int enqueue_step_sums(lbm_s* h, int n, double** out2) {
  if (!h->populated) {
    int rc = init_eq_device(h, nullptr, nullptr);
    if (rc) return rc;
  }
  int rc = upload_wall(h);
  if (rc) return rc;
  *out2 = h->d_partials + 2 * h->partials;
  int parts = 0;
  rc = step_sum_parts(h, &parts);
  if (rc) return rc;
  if (parts == 0) {
    // no summing kernel for this configuration: the reduction kernel reads the
    // state first, then the steps run
    KArgs a = make_args(h);
    LBM_CUDA(launch_reduce(h->Q, h->prec, h->layout, load_kind(h), a, h->d_partials, *out2, h->stream));
    return lbm_step(h, n);
  }
  const size_t need = 2 * (size_t)parts;
  if (h->sum_partials_cap < need) {
    if (h->d_sum_partials) {
      LBM_CUDA(cudaStreamSynchronize(h->stream));
      LBM_CUDA(cudaFree(h->d_sum_partials));
      h->d_sum_partials = nullptr;
      h->sum_partials_cap = 0;
    }
    LBM_CUDA(cudaMalloc(&h->d_sum_partials, sizeof(double) * need));
    h->sum_partials_cap = need;
  }
  int nparts = 0;
  rc = enqueue_step(h, h->d_sum_partials, &nparts);
  if (rc) return rc;
  LBM_CUDA(launch_reduce_final(h->d_sum_partials, nparts, *out2, h->stream));
  return lbm_step(h, n - 1);
}
}  // namespace

extern "C" {

int lbm_step_sums(lbm_t h, int n, double* mass, double* energy) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0) return fail(LBM_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return lbm_reduce(h, mass, energy);
  double* out2 = nullptr;
  int rc = enqueue_step_sums(h, n, &out2);
  if (rc) return rc;
  double r[2];
  LBM_CUDA(cudaMemcpyAsync(r, out2, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (mass) *mass = r[0];
  if (energy) *energy = r[1];
  rc = check_device_error(h);
  if (rc) return rc;
  if (!std::isfinite(r[0]) || !std::isfinite(r[1])) return fail(LBM_ERR_DIVERGED, "mass or energy is not finite");
  return LBM_OK;
}

int lbm_step_sums_async(lbm_t h, int n, double* out) {
  if (!h || !out) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
  if (n < 1) return fail(LBM_ERR_INVALID_ARG, "n must be >= 1");
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, out) != cudaSuccess) {
    cudaGetLastError();
    return fail(LBM_ERR_INVALID_ARG, "out must be device memory or page-locked host memory");
  }
  if (at.type == cudaMemoryTypeUnregistered)
    return fail(LBM_ERR_INVALID_ARG, "out must be device memory or page-locked host memory");
  double* out2 = nullptr;
  int rc = enqueue_step_sums(h, n, &out2);
  if (rc) return rc;
  LBM_CUDA(cudaMemcpyAsync(out, out2, 2 * sizeof(double), cudaMemcpyDefault, h->stream));
  return LBM_OK;
}

int lbm_macroscopic(lbm_t h, double* rho, double* u) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  if (!h->populated) return fail(LBM_ERR_STATE, "populations were never written");
  int rc = upload_wall(h);
  if (rc) return rc;
  const size_t N = (size_t)h->N;
  const bool dev_r = !rho || is_device_pointer(rho), dev_u = !u || is_device_pointer(u);
  double* dr = rho;
  double* du = u;
  if (!dev_r || !dev_u) {
    rc = ensure_stage(h, sizeof(double) * 4 * N);
    if (rc) return rc;
    if (!dev_r) dr = (double*)h->d_stage;
    if (!dev_u) du = (double*)h->d_stage + N;
  }
  KArgs a = make_args(h);
  LBM_CUDA(launch_macro(h->Q, h->prec, h->layout, load_kind(h), a, dr, du, h->d_wallu, h->stream));
  if (!dev_r) LBM_CUDA(cudaMemcpyAsync(rho, dr, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
  if (!dev_u) LBM_CUDA(cudaMemcpyAsync(u, du, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, h->stream));
  if (!dev_r || !dev_u) LBM_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_get_populations(lbm_t h, double* f) {
  if (!h || !f) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
  if (!h->populated) return fail(LBM_ERR_STATE, "populations were never written");
  const size_t bytes = sizeof(double) * (size_t)h->Q * (size_t)h->N;
  const bool dev = is_device_pointer(f);
  double* dst = f;
  if (!dev) {
    int rc = ensure_stage(h, bytes);
    if (rc) return rc;
    dst = (double*)h->d_stage;
  }
  KArgs a = make_args(h);
  LBM_CUDA(launch_get(h->Q, h->prec, h->layout, load_kind(h), a, dst, h->stream));
  if (!dev) {
    LBM_CUDA(cudaMemcpyAsync(f, dst, bytes, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    return check_device_error(h);
  }
  return LBM_OK;
}

int lbm_set_populations(lbm_t h, const double* f) {
  if (!h || !f) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
  const size_t bytes = sizeof(double) * (size_t)h->Q * (size_t)h->N;
  const double* src = f;
  int rc;
  if (!is_device_pointer(f)) {
    rc = ensure_stage(h, bytes);
    if (rc) return rc;
    LBM_CUDA(cudaMemcpyAsync(h->d_stage, f, bytes, cudaMemcpyHostToDevice, h->stream));
    src = (const double*)h->d_stage;
  }
  rc = reset_populations(h);
  if (rc) return rc;
  KArgs a = make_args(h);
  LBM_CUDA(launch_set(h->Q, h->prec, h->layout, store_kind(h), a, src, h->stream));
  h->populated = true;
  return decide_fx_range(h);
}

int lbm_reduce(lbm_t h, double* mass, double* energy) {
  if (!h) return fail(LBM_ERR_INVALID_ARG, "handle is NULL");
  if (!h->populated) return fail(LBM_ERR_STATE, "populations were never written");
  KArgs a = make_args(h);
  double* out2 = h->d_partials + 2 * h->partials;
  LBM_CUDA(launch_reduce(h->Q, h->prec, h->layout, load_kind(h), a, h->d_partials, out2, h->stream));
  double r[2];
  LBM_CUDA(cudaMemcpyAsync(r, out2, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (mass) *mass = r[0];
  if (energy) *energy = r[1];
  const int rc = check_device_error(h);
  if (rc) return rc;
  if (!std::isfinite(r[0]) || !std::isfinite(r[1])) return fail(LBM_ERR_DIVERGED, "mass or energy is not finite");
  return LBM_OK;
}

int lbm_steps_done(lbm_t h, long long* steps) {
  if (!h || !steps) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
  *steps = h->steps;
  return LBM_OK;
}

int lbm_device_bytes(lbm_t h, size_t* bytes) {
  if (!h || !bytes) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
  size_t b = (size_t)h->N * (1 + sizeof(uint32_t)) + STAGE_PAD_BYTES +
             sizeof(double) * (8 * 27 + 24 + 2 * h->partials + 2 + h->sum_partials_cap) + h->stage_bytes +
             4 * sizeof(int) +
             (h->nlist > 0 ? (sizeof(int) + sizeof(uint32_t) + 2 * sizeof(unsigned long long)) * (size_t)h->nlist : 0) +
             (h->d_qidx ? sizeof(int) * ((size_t)h->N + h->nqcells) + sizeof(double) * (size_t)h->qrows * h->Q : 0);
  for (int a = 0; a < 2; ++a)
    if (h->d_pop[a]) b += pop_bytes(h) + STAGE_PAD_BYTES;
  *bytes = b;
  return LBM_OK;
}

int lbm_bytes_per_cell_update(lbm_t h, double* bytes) {
  if (!h || !bytes) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
  const double pops = (double)h->Q * (double)elem_size(h->prec);
  // two-population, AA and esoteric twist read and write every population once;
  // swap reads and writes them twice (collision pass, then streaming pass)
  *bytes = h->scheme == LBM_SWAP ? 4.0 * pops + 2.0 : 2.0 * pops + 1.0;
  return LBM_OK;
}

int lbm_kernels_per_step(lbm_t h, int* n) {
  if (!h || !n) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
  int k = 1;
  if (h->scheme == LBM_SWAP) {
    k = 2;
  } else if (h->scheme == LBM_AA && h->sfns[0]) {
    const int rc = ensure_nonbulk_list(h);
    if (rc) return rc;
    k = h->nlist > 0 ? 2 : 1;
  }
  *n = k;
  return LBM_OK;
}

int lbm_debug_check(lbm_t h, unsigned long long* fault) {
  if (!h || !fault) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
#ifndef LBM_DEBUG
  *fault = 0;
  return fail(LBM_ERR_UNSUPPORTED, "this library is built without bounds checks; liblbm_debug.so has them");
#else
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (h->side.side) LBM_CUDA(cudaStreamSynchronize(h->side.side));
  unsigned long long w = 0;
  LBM_CUDA(cudaMemcpy(&w, debug_word(h), sizeof(w), cudaMemcpyDeviceToHost));
  if (w != 0) LBM_CUDA(cudaMemset(debug_word(h), 0, sizeof(w)));
  // canaries of the padding past the population arrays (index 0, 1) and the flags (2)
  unsigned char pad[STAGE_PAD_BYTES];
  for (int a = 0; a < 3 && w == 0; ++a) {
    const unsigned char* p = a < 2 ? (h->d_pop[a] ? static_cast<const unsigned char*>(h->d_pop[a]) + pop_bytes(h)
                                                 : nullptr)
                                   : h->d_flags + h->N;
    if (!p) continue;
    LBM_CUDA(cudaMemcpy(pad, p, STAGE_PAD_BYTES, cudaMemcpyDeviceToHost));
    for (size_t b = 0; b < STAGE_PAD_BYTES; ++b)
      if (pad[b] != DEBUG_CANARY) {
        w = ((unsigned long long)DBG_PAD << 56) | ((unsigned long long)a << 32) | b;
        break;
      }
  }
  *fault = w;
  return LBM_OK;
#endif
}

int lbm_destroy(lbm_t h) {
  if (!h) return LBM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (int a = 0; a < 2; ++a)
    if (h->d_pop[a]) cudaFree(h->d_pop[a]);
  if (h->d_flags) cudaFree(h->d_flags);
  if (h->d_nbmask) cudaFree(h->d_nbmask);
  if (h->d_wall) cudaFree(h->d_wall);
  if (h->d_wallu) cudaFree(h->d_wallu);
  if (h->d_partials) cudaFree(h->d_partials);
  if (h->d_stage) cudaFree(h->d_stage);
  if (h->d_err) cudaFree(h->d_err);
  if (h->side.side) {
    cudaStreamSynchronize(h->side.side);
    cudaStreamDestroy(h->side.side);
  }
  if (h->side.fork) cudaEventDestroy(h->side.fork);
  if (h->side.join) cudaEventDestroy(h->side.join);
  if (h->d_sum_partials) cudaFree(h->d_sum_partials);
  if (h->d_list) cudaFree(h->d_list);
  if (h->d_tile_off) cudaFree(h->d_tile_off);
  if (h->d_list_mask) cudaFree(h->d_list_mask);
  if (h->d_list_kinds) cudaFree(h->d_list_kinds);
  if (h->d_qidx) cudaFree(h->d_qidx);
  if (h->d_qtab) cudaFree(h->d_qtab);
  if (h->d_qcells) cudaFree(h->d_qcells);
  delete h;
  return LBM_OK;
}

}  // extern "C"
