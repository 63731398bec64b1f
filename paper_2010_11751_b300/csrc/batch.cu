// batch.cu -- host side of the batched stepping API (lbm_batch_*).
//
// A batch schedules member handles (same lattice, collision and precision,
// AA pattern, SoA) with one kernel launch per time step covering all of them.
// Per call, the member table (pointers, sizes, rates) is uploaded; members are
// split by step parity into two classes, each with its own block -> member
// map, rebuilt only when the membership, the launch shape or the split
// changes (a uniform parity flip just swaps the two classes).  With use_graph, the n launches of a call are
// captured once into a CUDA graph and replayed while nothing changes.  The
// autotuner times every (threads per block, cells per thread) pair on the
// batch itself and caches the winner per (lattice, model, precision, size
// class).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "batch.cuh"
#include "handle.h"
#include "internal.h"
#include "lbm.h"

using namespace lbm;

struct lbm_batch_s {
  std::vector<lbm_s*> members;
  int Q = 0, model = -1, prec = -1;
  int threads = 256, cpt = 1;
  cudaStream_t user_stream = nullptr;
  cudaStream_t own_stream = nullptr;  // capture needs a non-legacy stream
  std::vector<Member> h_members;
  Member* d_members = nullptr;
  int cap_members = 0;
  // per parity class c (members whose step count had parity c when the maps were
  // built): block -> member map on the device and its number of blocks
  std::vector<int> h_map[2];
  int* d_map[2] = {nullptr, nullptr};
  int cap_map[2] = {0, 0};
  int blocks[2] = {0, 0};
  std::vector<int> map_parity;  // each member's step parity when the maps were built
  bool map_dirty = true;
  cudaGraphExec_t gexec = nullptr;
  int graph_n = 0;
  int graph_e0 = 0;
  BatchFn fn = nullptr;
};

namespace {

int bfail(int code, const char* msg) { return set_error(code, msg); }

#define BCUDA(call)                                                   \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return set_error(LBM_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

cudaStream_t bstream(lbm_batch_s* b) { return b->user_stream ? b->user_stream : b->own_stream; }

void drop_graph(lbm_batch_s* b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  b->graph_n = 0;
}

int rebuild_map(lbm_batch_s* b) {
  const int chunk = b->threads * b->cpt;
  const size_t n = b->members.size();
  b->h_members.resize(n);
  b->map_parity.resize(n);
  for (int c = 0; c < 2; ++c) {
    b->h_map[c].clear();
    int blocks = 0;
    for (size_t m = 0; m < n; ++m) {
      const int par = (int)(b->members[m]->steps & 1);
      b->map_parity[m] = par;
      if (par != c) continue;
      const int nb = (b->members[m]->N + chunk - 1) / chunk;
      b->h_members[m].block_begin = blocks;
      b->h_map[c].insert(b->h_map[c].end(), nb, (int)m);
      blocks += nb;
    }
    if (blocks > b->cap_map[c]) {
      if (b->d_map[c]) BCUDA(cudaFree(b->d_map[c]));
      b->d_map[c] = nullptr;
      BCUDA(cudaMalloc(&b->d_map[c], sizeof(int) * std::max(blocks, 1)));
      b->cap_map[c] = blocks;
    }
    if (blocks)
      BCUDA(cudaMemcpyAsync(b->d_map[c], b->h_map[c].data(), sizeof(int) * blocks, cudaMemcpyHostToDevice,
                            bstream(b)));
    b->blocks[c] = blocks;
  }
  BCUDA(cudaStreamSynchronize(bstream(b)));
  b->map_dirty = false;
  drop_graph(b);
  return LBM_OK;
}

// which map holds the members of current parity 0: 0 or 1 (-1: the split changed)
int parity_class_of_even(const lbm_batch_s* b) {
  bool same = true, flipped = true;
  for (size_t m = 0; m < b->members.size(); ++m) {
    const int par = (int)(b->members[m]->steps & 1);
    same = same && par == b->map_parity[m];
    flipped = flipped && par != b->map_parity[m];
  }
  if (same) return 0;
  if (flipped) return 1;
  return -1;
}

int upload_members(lbm_batch_s* b) {
  const int n = (int)b->members.size();
  for (int m = 0; m < n; ++m) {
    lbm_s* h = b->members[m];
    int rc = handle_prepare(h);
    if (rc) return rc;
    // work the member enqueued on its own stream (or on the legacy default stream, which a
    // caller's non-blocking stream does not order with) must be done first
    if (h->stream != bstream(b)) BCUDA(cudaStreamSynchronize(h->stream));
    Member& d = b->h_members[m];
    d.pop = h->d_pop[0];
    d.flags = h->d_flags;
    d.nbmask = h->d_nbmask;
    d.wall = h->d_wall;
    d.nx = h->nx;
    d.ny = h->ny;
    d.nz = h->nz;
    d.N = h->N;
    handle_rates(h, &d.rd, &d.rf);
    d.fx_wide = h->fx_wide ? 1 : 0;
    LBM_IF_DEBUG(d.dbg = reinterpret_cast<unsigned long long*>(h->d_err + 2);)
  }
  if (n > b->cap_members) {
    if (b->d_members) BCUDA(cudaFree(b->d_members));
    b->d_members = nullptr;
    BCUDA(cudaMalloc(&b->d_members, sizeof(Member) * n));
    b->cap_members = n;
    drop_graph(b);
  }
  BCUDA(cudaMemcpyAsync(b->d_members, b->h_members.data(), sizeof(Member) * n, cudaMemcpyHostToDevice, bstream(b)));
  return LBM_OK;
}

// n steps; e0 = map class holding the members whose parity is 0 at the first step
cudaError_t launch_steps(lbm_batch_s* b, int n, int e0, cudaStream_t s) {
  BatchArgs a;
  a.m = b->d_members;
  a.cpt = b->cpt;
  for (int st = 0; st < n; ++st) {
    const int ce = (e0 + st) & 1;  // class taking an even (local) step now
    for (int c = 0; c < 2; ++c) {
      if (!b->blocks[c]) continue;
      a.block_member = b->d_map[c];
      cudaError_t e = b->fn(a, c == ce ? K_AA_EVEN : K_AA_ODD, b->blocks[c], b->threads, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

int run_steps(lbm_batch_s* b, int n, bool use_graph) {
  if (b->members.empty() || n == 0) return LBM_OK;
  int rc;
  if (!b->map_dirty && parity_class_of_even(b) < 0) b->map_dirty = true;
  if (b->map_dirty) {
    rc = rebuild_map(b);
    if (rc) return rc;
  }
  const int e0 = parity_class_of_even(b);
  rc = upload_members(b);
  if (rc) return rc;
  cudaStream_t s = bstream(b);
  if (!use_graph) {
    BCUDA(launch_steps(b, n, e0, s));
  } else {
    if (!b->gexec || b->graph_n != n || b->graph_e0 != e0) {
      drop_graph(b);
      cudaGraph_t g = nullptr;
      BCUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = launch_steps(b, n, e0, s);
      cudaError_t e2 = cudaStreamEndCapture(s, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return set_error(LBM_ERR_CUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      e = cudaGraphInstantiate(&b->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
      b->graph_n = n;
      b->graph_e0 = e0;
    }
    BCUDA(cudaGraphLaunch(b->gexec, s));
  }
  for (lbm_s* h : b->members) h->steps += n;
  return LBM_OK;
}

// process-wide autotuning cache: (Q, model, precision, size class) -> (threads, cpt)
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;

int size_class(const lbm_batch_s* b) {
  long long cells = 0;
  for (lbm_s* h : b->members) cells += h->N;
  const double avg = b->members.empty() ? 1.0 : (double)cells / b->members.size();
  return (int)std::floor(std::log2(std::max(avg, 1.0)));
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch_t* out) {
  if (!out) return bfail(LBM_ERR_INVALID_ARG, "out is NULL");
  lbm_batch_s* b = new lbm_batch_s();
  // a blocking stream: it orders with the legacy default stream, on which
  // member handles run unless they were given a stream of their own
  cudaError_t e = cudaStreamCreate(&b->own_stream);
  if (e != cudaSuccess) {
    delete b;
    return set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_add(lbm_batch_t b, lbm_t h) {
  if (!b || !h) return bfail(LBM_ERR_INVALID_ARG, "NULL argument");
  if (h->scheme != LBM_AA || h->layout != LBM_SOA)
    return bfail(LBM_ERR_INVALID_ARG, "batch members must use the AA pattern and the SoA layout");
  if (std::find(b->members.begin(), b->members.end(), h) != b->members.end())
    return bfail(LBM_ERR_INVALID_ARG, "handle is already in the batch");
  if (h->d_qidx) return bfail(LBM_ERR_UNSUPPORTED, "batch members cannot have walls at a fraction of their links");
  if (!b->members.empty() && (h->Q != b->Q || h->model != b->model || h->prec != b->prec))
    return bfail(LBM_ERR_INVALID_ARG, "batch members must share lattice, collision model and precision");
  if (b->members.empty()) {
    BatchFn fn = batch_fn(h->model, h->Q, h->prec);
    if (!fn) return bfail(LBM_ERR_UNSUPPORTED, "no batched kernel for this combination");
    b->Q = h->Q;
    b->model = h->model;
    b->prec = h->prec;
    b->fn = fn;
  }
  b->members.push_back(h);
  b->map_dirty = true;
  return LBM_OK;
}

int lbm_batch_remove(lbm_batch_t b, lbm_t h) {
  if (!b || !h) return bfail(LBM_ERR_INVALID_ARG, "NULL argument");
  auto it = std::find(b->members.begin(), b->members.end(), h);
  if (it == b->members.end()) return bfail(LBM_ERR_INVALID_ARG, "handle is not in the batch");
  // the member's work must be finished before the caller uses it alone
  BCUDA(cudaStreamSynchronize(bstream(b)));
  b->members.erase(it);
  b->map_dirty = true;
  return LBM_OK;
}

int lbm_batch_set_launch(lbm_batch_t b, int threads, int cpt) {
  if (!b) return bfail(LBM_ERR_INVALID_ARG, "batch is NULL");
  if (threads == 0) threads = 256;
  if (cpt == 0) cpt = 1;
  if (threads < 32 || threads > 256 || threads % 32) return bfail(LBM_ERR_INVALID_ARG, "threads must be 32..256, multiple of 32");
  if (cpt != 1 && cpt != 2 && cpt != 4) return bfail(LBM_ERR_INVALID_ARG, "cells per thread must be 1, 2 or 4");
  if (threads != b->threads || cpt != b->cpt) {
    b->threads = threads;
    b->cpt = cpt;
    b->map_dirty = true;
  }
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch_t b, int* threads_out, int* cpt_out) {
  if (!b) return bfail(LBM_ERR_INVALID_ARG, "batch is NULL");
  if (b->members.empty()) return bfail(LBM_ERR_STATE, "batch is empty");
  const auto key = std::make_tuple(b->Q, b->model, b->prec, size_class(b));
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      int rc = lbm_batch_set_launch(b, it->second.first, it->second.second);
      if (threads_out) *threads_out = b->threads;
      if (cpt_out) *cpt_out = b->cpt;
      return rc;
    }
  }
  cudaEvent_t e0, e1;
  BCUDA(cudaEventCreate(&e0));
  BCUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bt = 256, bc = 1;
  const int shapes_t[4] = {32, 64, 128, 256};
  const int shapes_c[3] = {1, 2, 4};
  int rc = LBM_OK;
  for (int ti = 0; ti < 4 && rc == LBM_OK; ++ti)
    for (int ci = 0; ci < 3 && rc == LBM_OK; ++ci) {
      rc = lbm_batch_set_launch(b, shapes_t[ti], shapes_c[ci]);
      if (rc) break;
      rc = run_steps(b, 2, false);  // warm-up (rebuilds the map)
      if (rc) break;
      cudaStream_t s = bstream(b);
      cudaEventRecord(e0, s);
      rc = run_steps(b, 4, false);
      cudaEventRecord(e1, s);
      if (rc) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bt = shapes_t[ti];
        bc = shapes_c[ci];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = {bt, bc};
  }
  rc = lbm_batch_set_launch(b, bt, bc);
  if (threads_out) *threads_out = bt;
  if (cpt_out) *cpt_out = bc;
  return rc;
}

int lbm_batch_step(lbm_batch_t b, int n, int use_graph) {
  if (!b) return bfail(LBM_ERR_INVALID_ARG, "batch is NULL");
  if (n < 0) return bfail(LBM_ERR_INVALID_ARG, "n must be >= 0");
  return run_steps(b, n, use_graph != 0);
}

int lbm_batch_set_stream(lbm_batch_t b, void* stream) {
  if (!b) return bfail(LBM_ERR_INVALID_ARG, "batch is NULL");
  if ((cudaStream_t)stream != b->user_stream) {
    // the steps already enqueued on the old stream finish before any on the new one starts
    BCUDA(cudaStreamSynchronize(bstream(b)));
    drop_graph(b);
  }
  b->user_stream = (cudaStream_t)stream;
  return LBM_OK;
}

int lbm_batch_size(lbm_batch_t b, int* members, long long* cells) {
  if (!b) return bfail(LBM_ERR_INVALID_ARG, "batch is NULL");
  long long c = 0;
  for (lbm_s* h : b->members) c += h->N;
  if (members) *members = (int)b->members.size();
  if (cells) *cells = c;
  return LBM_OK;
}

int lbm_batch_sync(lbm_batch_t b) {
  if (!b) return bfail(LBM_ERR_INVALID_ARG, "batch is NULL");
  BCUDA(cudaStreamSynchronize(bstream(b)));
  return LBM_OK;
}

int lbm_batch_destroy(lbm_batch_t b) {
  if (!b) return LBM_OK;
  cudaStreamSynchronize(bstream(b));
  drop_graph(b);
  if (b->d_members) cudaFree(b->d_members);
  for (int c = 0; c < 2; ++c)
    if (b->d_map[c]) cudaFree(b->d_map[c]);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
  return LBM_OK;
}

}  // extern "C"
