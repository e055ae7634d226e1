// hpcg_ctx.h -- host-side handle of the MG-PCG library (hpcg_handle), shared by
// the host translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "hpcg.h"
#include "hpcg_internal.cuh"

using namespace hpcg;

// ---------------------------------------------------------------------------
// error plumbing
extern char g_last_cuda_error[256];
extern std::atomic<long> g_launches;
int cuda_fail(cudaError_t e, const char *what);
#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)
#define CKL(what)                                         \
  do {                                                    \
    g_launches.fetch_add(1, std::memory_order_relaxed);   \
    cudaError_t e_ = cudaGetLastError();                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);    \
  } while (0)
#define TRY(x)              \
  do {                      \
    int rc_ = (x);          \
    if (rc_ != HPCG_OK) return rc_; \
  } while (0)

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
struct LevelData {
  std::vector<Inst> inst;  // host copy
  LevelTab tab{};
  long n = 0;
  // workspace offsets (bytes)
  size_t o_tab = 0, o_r = 0, o_z = 0, o_r32 = 0, o_z32 = 0, o_kap = 0, o_invd = 0, o_kap32 = 0, o_invd32 = 0, o_zq = 0, o_ze = 0;
  long nlines = 0;  // x-lines over all instances (sum of ny * nz)
  bool even_nx = false;  // every instance's lines have an even length (x pairs move as vectors)
  bool planes = false;   // block-floating-point smoother runs grouped by plane parity (k_gs_planes_bfp)
  // device pointers (valid once a workspace is bound)
  double *r = nullptr, *z = nullptr, *kap = nullptr, *invd = nullptr;
  float *r32 = nullptr, *z32 = nullptr, *kap32 = nullptr, *invd32 = nullptr;
  long long *zq = nullptr;  // block-floating-point z: mantissas [n]
  int *ze = nullptr;        // and one exponent per x-line [nlines]
};

struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  const void *key[4] = {nullptr, nullptr, nullptr, nullptr};
  long kernels = 0;
};

struct hpcg_ctx {
  int batch = 0;  // 0: single grid, 1: batch of grids
  hpcg_options opt{};
  int levels = 0;
  int count = 1;
  bool has_kappa = false;
  const double *kappa_pending = nullptr;
  LevelData lv[kMaxLevels];
  // workspace
  char *ws = nullptr;
  size_t ws_bytes = 0, need = 0;
  bool ws_owned = false;
  bool ready = false;
  size_t o_st = 0, o_hist = 0, o_part = 0, o_out = 0, o_cg = 0;
  size_t npart = 0;
  CgState *st = nullptr;
  double *hist = nullptr, *part = nullptr, *dout = nullptr;
  double *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_ap = nullptr;
  // multi-RHS region (sized by opt.max_rhs)
  size_t o_multi = 0, multi_bytes = 0;
  cudaStream_t cap = nullptr;
  GraphCache g_iter;
  hpcg_ctx *multi = nullptr;  // internal batch of max_rhs copies of the grid (hpcg_pcg_solve_multi)
  int multi_R = 0;
  bool tuned = false;
  bool use_bfp = false;  // the FP64 V-cycle keeps z in block floating point (hpcg_options.block_fp)
  // persistent tail of the V-cycle (levels tail_first..levels-1 in one cooperative launch)
  int tail_first = -1;        // -1: no tail
  bool tail_ok = true;        // cleared if a cooperative launch is refused
  int tail_grid = 0;
  long long wait_limit = 2000000000LL;  // clock cycles a grid barrier may wait (about 1 s)
  size_t o_tail = 0, o_sync = 0;        // TailPlan[2] (FP64, FP32); {barrier count, generation, error, -, batch all-done flag}
  // cluster kernel of the block-floating-point V-cycle's coarse end (levels bfp_tail_first..levels-1)
  int bfp_tail_first = -1;  // -1: none
  int bfp_tail_ok = -1;     // -1: not checked yet; 0: the GPU cannot run the cluster
  size_t o_tail_bfp = 0;    // BfpTailPlan
  int fin_cluster_ok = -1;  // -1: not checked yet; 1: per-line reductions finalise in a cluster (k_finalize_lines)
  // tolerance solves: two pinned flag slots and their events for the host's
  // one-iteration-lag poll of the convergence flag (made once per handle)
  int *poll_flags = nullptr;
  cudaEvent_t poll_ev[2] = {nullptr, nullptr};
  int device = 0;
  std::mutex mu;
};

struct hpcg_ctx;
int red_blocks(long n);
int grid_for(long n);
int ensure_ready(hpcg_ctx *h, cudaStream_t s);
