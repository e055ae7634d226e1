// hpcg_core.cu -- host driver of the GB300 MG-PCG library: handle, workspace,
// V-cycle (Listing 1) and preconditioned CG (Section II-C) enqueueing, CUDA
// graph capture of one CG iteration, and the C-ABI entry points of hpcg.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <utility>
#include <mutex>
#include <vector>

#include "hpcg.h"
#include "hpcg_ctx.h"
#include "hpcg_kernels.cuh"
#include "hpcg_lines.cuh"
#include "hpcg_tail.cuh"
#include "hpcg_fixed.cuh"
#include "hpcg_bfp.cuh"
#include "hpcg_spmv.cuh"

using namespace hpcg;

// Kernel launch with programmatic dependent launch allowed: the kernel may be
// scheduled while its predecessor in the stream still runs; every kernel of
// this library starts with griddepcontrol.wait (pdl_enter), so it reads its
// inputs only after the predecessor has finished.
static thread_local bool t_pdl = true;  // set per call from the handle's option

// Per-phase timing of one CG iteration (hpcg_profile_iteration): an event is
// recorded after every kernel group; the time between two events belongs to
// the group the later one closes.  Outside a profiling call prof_mark is a no-op.
enum ProfKind { PK_SMOOTH = 0, PK_RESTRICT, PK_PROLONG, PK_TAIL, PK_SPMV, PK_DOT, PK_UPDATE, PK_FINALIZE, PK_CONVERT, PK_COUNT };
struct Prof {
  cudaStream_t s;
  std::vector<cudaEvent_t> ev;
  std::vector<int> tag;  // kind * 16 + level
};
static thread_local Prof *t_prof = nullptr;
static void prof_mark(int kind, int level) {
  if (!t_prof) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, t_prof->s);
  t_prof->ev.push_back(e);
  t_prof->tag.push_back(kind * 16 + level);
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = t_pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// error plumbing (declared in hpcg_ctx.h)
char g_last_cuda_error[256] = "no error";
std::atomic<long> g_launches{0};

int cuda_fail(cudaError_t e, const char *what) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", what, cudaGetErrorString(e));
  return HPCG_ERR_CUDA;
}

// ---------------------------------------------------------------------------
static int validate_dims(int nx, int ny, int nz, int levels) {
  if (levels < 1 || levels > kMaxLevels) return HPCG_ERR_INVALID_ARG;
  const int div = 1 << (levels - 1);
  if (nx < 2 || ny < 2 || nz < 2) return HPCG_ERR_INVALID_ARG;
  if (nx % div || ny % div || nz % div) return HPCG_ERR_INVALID_ARG;
  if (nx / div < 2 || ny / div < 2 || nz / div < 2) return HPCG_ERR_INVALID_ARG;
  if ((double)nx * ny * nz > 2.0e9) return HPCG_ERR_INVALID_ARG;  // int32 row indices of the maps
  return HPCG_OK;
}

int red_blocks(long n) {
  long b = (n + (long)kRedThreads * kRedItems - 1) / ((long)kRedThreads * kRedItems);
  if (b < 1) b = 1;
  if (b > kMaxRedBlocksPerInst) b = kMaxRedBlocksPerInst;
  return (int)b;
}

static int nch_supported(int need) {
  static const int avail[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16};
  for (int a : avail)
    if (a >= need) return a;
  return 0;
}

static void set_line_prefixes(LevelData &L) {
  int br = 0, bl = 0, po = 0;
  for (Inst &g : L.inst) {
    g.poff = po;
    po += g.ny * g.nz;
    g.blk_row = br;
    g.nrow = row_blocks(g.ny, g.nz, L.tab.row_lpc, L.tab.row_zc);
    g.blk_line = bl;
    g.nline = line_blocks(g.ny, g.nz, L.tab.line_lpc, L.tab.line_zc);
    br += g.nrow;
    bl += g.nline;
  }
  L.tab.nblk_row = br;
  L.tab.nblk_line = bl;
}

// Launch shape of the line kernels of a level: the largest z-chunk (longest
// reuse of plane sums) and lines per block that still give at least two blocks
// per SM over all instances (152 SMs), else the shape with the most blocks.
static void choose_line_params(LevelData &L) {
  int nxm = 0;
  for (const Inst &g : L.inst) nxm = std::max(nxm, g.nx);
  L.tab.nch = nch_supported((nxm + 31) / 32);
  // colour-step kernels hold each line split by x parity: ceil(nx/2) per parity
  {
    const int need = (((nxm + 1) / 2) + 31) / 32;
    static const int avail2[] = {1, 2, 3, 4, 5, 6, 8};
    L.tab.nch2 = 0;
    for (int a : avail2)
      if (a >= need) {
        L.tab.nch2 = a;
        break;
      }
    if (L.tab.nch2 == 0) L.tab.nch = 0;  // lines too long for the registers: one-thread-per-row kernels
  }
  const int target = 2 * 152;
  auto pick = [&](bool lines_of_class, int *lpc_out, int *zc_out) {
    static const int lpcs[] = {8, 4, 2, 1};
    static const int zcs[] = {16, 8, 4, 2, 1};
    int best_lpc = 1, best_zc = 1;
    long best_blocks = -1;
    for (int zc : zcs)
      for (int lpc : lpcs) {
        long blocks = 0;
        for (const Inst &g : L.inst)
          blocks += lines_of_class ? line_blocks(g.ny, g.nz, lpc, zc) : row_blocks(g.ny, g.nz, lpc, zc);
        if (blocks >= target && lpc >= 2) {
          *lpc_out = lpc;
          *zc_out = zc;
          return;
        }
        if (blocks > best_blocks) {
          best_blocks = blocks;
          best_lpc = lpc;
          best_zc = zc;
        }
      }
    *lpc_out = best_lpc;
    *zc_out = best_zc;
  };
  pick(false, &L.tab.row_lpc, &L.tab.row_zc);
  pick(true, &L.tab.line_lpc, &L.tab.line_zc);
  set_line_prefixes(L);
}

// Builds the instance tables and the workspace layout.
static void plan(hpcg_ctx *h, const std::vector<int> &dims) {
  h->count = (int)dims.size() / 3;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  for (int l = 0; l < h->levels; ++l) {
    LevelData &L = h->lv[l];
    L.inst.resize(h->count);
    long rows = 0;
    int bf = 0, bh = 0, br = 0;
    for (int i = 0; i < h->count; ++i) {
      Inst &g = L.inst[i];
      g.nx = dims[3 * i] >> l;
      g.ny = dims[3 * i + 1] >> l;
      g.nz = dims[3 * i + 2] >> l;
      g.n = (long)g.nx * g.ny * g.nz;
      g.off = rows;
      g.blk_full = bf;
      g.blk_half = bh;
      g.blk_red = br;
      g.nred = red_blocks(g.n);
      g.poff = 0;
      rows += g.n;
      bf += tiles_of(g.nx, g.ny, g.nz);
      bh += tiles_of(half_up(g.nx), half_up(g.ny), half_up(g.nz));
      br += g.nred;
    }
    L.n = rows;
    L.nlines = 0;
    L.even_nx = true;
    for (const Inst &g : L.inst) {
      L.nlines += (long)g.ny * g.nz;
      L.even_nx = L.even_nx && (g.nx % 2) == 0;
    }
    L.tab.count = h->count;
    L.tab.nblk_full = bf;
    L.tab.nblk_half = bh;
    L.tab.nblk_red = br;
    L.tab.n = rows;
    choose_line_params(L);
  }
  for (int l = 0; l < h->levels; ++l) h->lv[l].o_tab = take(sizeof(Inst) * h->count);
  h->o_st = take(sizeof(CgState) * h->count);
  h->o_hist = take(sizeof(double) * (size_t)kHistoryCap * h->count);
  const LevelData &L0 = h->lv[0];
  // partial sums: enough for any launch shape the autotuner may pick (one line per block at most)
  long max_row_blocks = 0;
  for (const Inst &g : L0.inst) max_row_blocks += (long)g.ny * g.nz;
  h->npart = (size_t)std::max(std::max((long)std::max(L0.tab.nblk_full, L0.tab.nblk_red), max_row_blocks), (long)kRawDotBlocks) + 64;
  h->o_part = take(sizeof(double) * h->npart);
  h->o_out = take(sizeof(double) * (h->count + 64));
  h->o_tail = take(2 * sizeof(TailPlan));
  h->o_tail_bfp = take(sizeof(BfpTailPlan));
  h->o_sync = take(64);
  const long n0 = L0.n;
  h->o_cg = take(sizeof(double) * 4 * (size_t)n0);
  const bool mixed = h->opt.precision == HPCG_MIXED;
  for (int l = 0; l < h->levels; ++l) {
    LevelData &L = h->lv[l];
    if (l > 0) {
      L.o_r = take(sizeof(double) * L.n);
      L.o_z = take(sizeof(double) * L.n);
    }
    if (mixed) {
      L.o_r32 = take(sizeof(float) * L.n);
      L.o_z32 = take(sizeof(float) * L.n);
    } else if (h->opt.block_fp) {
      L.o_zq = take(sizeof(long long) * L.n);
      L.o_ze = take(sizeof(int) * L.nlines);
    }
    if (h->batch == 0) {  // a diagonal field can be bound to a single-grid handle
      L.o_kap = take(sizeof(double) * L.n);
      L.o_invd = take(sizeof(double) * L.n);
      L.o_kap32 = take(sizeof(float) * L.n);
      L.o_invd32 = take(sizeof(float) * L.n);
    }
  }
  h->multi_bytes = 0;
  if (h->opt.max_rhs > 0 && h->batch == 0) {
    // multi-RHS solves run as a batch of copies of this grid whose workspace
    // is this region (sized for max_rhs copies)
    hpcg_ctx tmp;
    tmp.opt = h->opt;
    tmp.opt.max_rhs = 0;
    tmp.batch = 1;
    tmp.levels = h->levels;
    std::vector<int> rep;
    for (int k = 0; k < h->opt.max_rhs; ++k) rep.insert(rep.end(), dims.begin(), dims.begin() + 3);
    plan(&tmp, rep);
    h->multi_bytes = tmp.need;
    h->o_multi = take(h->multi_bytes);
  }
  h->need = off;
}

static int build_tail_plans(hpcg_ctx *h);
static int bind(hpcg_ctx *h, char *ws, size_t bytes, bool owned) {
  if (bytes < h->need) return HPCG_ERR_NO_WORKSPACE;
  if (((uintptr_t)ws & 255) != 0) return HPCG_ERR_INVALID_ARG;
  if (h->ws_owned && h->ws && h->ws != ws) cudaFree(h->ws);
  h->ws = ws;
  h->ws_bytes = bytes;
  h->ws_owned = owned;
  CK(cudaGetDevice(&h->device));
  for (int l = 0; l < h->levels; ++l) {
    LevelData &L = h->lv[l];
    L.tab.inst = (const Inst *)(ws + L.o_tab);
    CK(cudaMemcpy((void *)L.tab.inst, L.inst.data(), sizeof(Inst) * h->count, cudaMemcpyHostToDevice));
    L.r = l > 0 ? (double *)(ws + L.o_r) : nullptr;
    L.z = l > 0 ? (double *)(ws + L.o_z) : nullptr;
    L.r32 = h->opt.precision == HPCG_MIXED ? (float *)(ws + L.o_r32) : nullptr;
    L.z32 = h->opt.precision == HPCG_MIXED ? (float *)(ws + L.o_z32) : nullptr;
    const bool bfp_space = h->opt.precision != HPCG_MIXED && h->opt.block_fp;
    L.zq = bfp_space ? (long long *)(ws + L.o_zq) : nullptr;
    L.ze = bfp_space ? (int *)(ws + L.o_ze) : nullptr;
    if (h->batch == 0) {
      L.kap = (double *)(ws + L.o_kap);
      L.invd = (double *)(ws + L.o_invd);
      L.kap32 = (float *)(ws + L.o_kap32);
      L.invd32 = (float *)(ws + L.o_invd32);
    }
  }
  h->st = (CgState *)(ws + h->o_st);
  h->hist = (double *)(ws + h->o_hist);
  h->part = (double *)(ws + h->o_part);
  h->dout = (double *)(ws + h->o_out);
  const long n0 = h->lv[0].n;
  h->cg_r = (double *)(ws + h->o_cg);
  h->cg_z = h->cg_r + n0;
  h->cg_p = h->cg_z + n0;
  h->cg_ap = h->cg_p + n0;
  if (h->g_iter.exec) {
    cudaGraphExecDestroy(h->g_iter.exec);
    h->g_iter = GraphCache{};
  }
  if (h->multi) {  // its workspace was a region of the previous one
    hpcg_destroy(h->multi);
    h->multi = nullptr;
    h->multi_R = 0;
  }
  h->ready = true;
  CK(cudaMemset(ws + h->o_sync, 0, 64));
  return build_tail_plans(h);
}

static int set_kappa_impl(hpcg_ctx *h, const double *kappa, cudaStream_t s);
static int autotune_impl(hpcg_ctx *h, int *shapes, cudaStream_t s);
static int build_tail_plans(hpcg_ctx *h);

int ensure_ready(hpcg_ctx *h, cudaStream_t s) {
  t_pdl = h->opt.pdl != 0;
  if (!h->ready) {
    char *p = nullptr;
    cudaError_t e = cudaMalloc(&p, h->need);
    if (e != cudaSuccess) {
      cuda_fail(e, "cudaMalloc(workspace)");
      return HPCG_ERR_OUT_OF_MEMORY;
    }
    TRY(bind(h, p, h->need, true));
  }
  if (h->kappa_pending) {
    const double *k = h->kappa_pending;
    h->kappa_pending = nullptr;
    TRY(set_kappa_impl(h, k, s));
  }
  if (h->opt.autotune && !h->tuned) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) TRY(autotune_impl(h, nullptr, s));
  }
  return HPCG_OK;
}

int grid_for(long n) {
  long b = (n + 255) / 256;
  if (b > 152L * 16) b = 152L * 16;
  if (b < 1) b = 1;
  return (int)b;
}

static int set_kappa_impl(hpcg_ctx *h, const double *kappa, cudaStream_t s) {
  if (h->batch) return HPCG_ERR_UNSUPPORTED;
  if (!kappa) {
    h->has_kappa = false;
    return build_tail_plans(h);
  }
  LevelData &L0 = h->lv[0];
  CK(cudaMemcpyAsync(L0.kap, kappa, sizeof(double) * L0.n, cudaMemcpyDeviceToDevice, s));
  for (int l = 0; l < h->levels; ++l) {
    LevelData &L = h->lv[l];
    if (l > 0) {
      const Inst &f = h->lv[l - 1].inst[0];
      const Inst &c = L.inst[0];
      launch_k(k_inject_kappa, grid_for(c.n), 256, 0, s, f.nx, f.ny, c.nx, c.ny, c.nz, h->lv[l - 1].kap, L.kap);
      CKL("k_inject_kappa");
    }
    launch_k(k_kappa_derived, grid_for(L.n), 256, 0, s, L.n, L.kap, L.invd, L.kap32, L.invd32);
    CKL("k_kappa_derived");
  }
  h->has_kappa = true;
  return build_tail_plans(h);
}

// ---------------------------------------------------------------------------
static std::vector<int> phase_sequence(int sweeps, int symmetric);

// Runs of one line class (see enqueue_smoother) of a smoother application.
static int make_runs(int sweeps, int symmetric, TailRun *out, int cap) {
  const std::vector<int> seq = phase_sequence(sweeps, symmetric);
  int nr = 0;
  size_t i = 0;
  while (i < seq.size()) {
    size_t j = i + 1;
    while (j < seq.size() && (seq[j] >> 1) == (seq[i] >> 1)) ++j;
    if (nr >= cap) return -1;
    out[nr].cls = (signed char)(seq[i] >> 1);
    out[nr].pa = (signed char)(seq[i] & 1);
    out[nr].steps = (signed char)(j - i);
    out[nr].pad = 0;
    ++nr;
    i = j;
  }
  return nr;
}

// Chooses the levels of the persistent tail (small levels whose lines fit one
// 32-wide chunk per parity) and writes the FP64 and FP32 tail plans.
static int build_bfp_tail(hpcg_ctx *h);
static int build_fp64_tail(hpcg_ctx *h);
static int build_tail_plans(hpcg_ctx *h) {
  TRY(build_fp64_tail(h));
  return build_bfp_tail(h);
}

// The block-floating-point coarse end (k_vcycle_tail_bfp): the levels from
// `first` down with at most kBfpTailRows rows and one 64-point chunk per x
// parity, if this GPU can run a cluster of kBfpTailCtas blocks.
static int build_bfp_tail(hpcg_ctx *h) {
  h->bfp_tail_first = -1;
  if (!h->use_bfp || !h->opt.cluster_tail || h->levels < 2) return HPCG_OK;
  int first = h->levels;
  for (int l = h->levels - 1; l >= 1; --l) {
    const LevelData &L = h->lv[l];
    if (L.tab.nch2 != 1 || L.n > kBfpTailRows) break;
    first = l;
  }
  if (first >= h->levels) return HPCG_OK;
  if (h->bfp_tail_ok < 0) {
    int nclusters = 0;
    cudaError_t e = cudaFuncSetAttribute(k_vcycle_tail_bfp<1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(kBfpTailCtas);
      cfg.blockDim = dim3(32, kBfpTailWarps);
      cudaLaunchAttribute a[1];
      a[0].id = cudaLaunchAttributeClusterDimension;
      a[0].val.clusterDim.x = kBfpTailCtas;
      a[0].val.clusterDim.y = 1;
      a[0].val.clusterDim.z = 1;
      cfg.attrs = a;
      cfg.numAttrs = 1;
      e = cudaOccupancyMaxActiveClusters(&nclusters, k_vcycle_tail_bfp<1>, &cfg);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      nclusters = 0;
    }
    h->bfp_tail_ok = nclusters > 0 ? 1 : 0;
  }
  if (!h->bfp_tail_ok) return HPCG_OK;
  BfpTailPlan P;
  memset(&P, 0, sizeof(P));
  P.first = first;
  P.last = h->levels - 1;
  P.count = h->count;
  for (int l = first; l < h->levels; ++l) {
    const LevelData &L = h->lv[l];
    BfpTailLevel &T = P.lv[l];
    const bool coarsest = l == h->levels - 1;
    T.tab = L.tab.inst;
    T.g1 = L.inst[0];
    T.r = L.r;
    T.zq = L.zq;
    T.ze = L.ze;
    T.invd = h->has_kappa ? L.invd : nullptr;
    T.kap = h->has_kappa ? L.kap : nullptr;
    T.rnext = coarsest ? nullptr : h->lv[l + 1].r;
    T.tabnext = coarsest ? nullptr : h->lv[l + 1].tab.inst;
    T.lpc = L.tab.line_lpc;
    T.zc = L.tab.line_zc;
    T.nblk_line = L.tab.nblk_line;
    T.nlines = (int)L.nlines;
    T.npre = make_runs(coarsest ? 1 : h->opt.pre_sweeps, 1, T.pre, kTailRuns);
    T.npost = coarsest ? 0 : make_runs(h->opt.post_sweeps, 1, T.post, kTailRuns);
    if (T.npre < 0 || T.npost < 0) return HPCG_OK;  // too many runs: no tail
  }
  CK(cudaMemcpy(h->ws + h->o_tail_bfp, &P, sizeof(P), cudaMemcpyHostToDevice));
  h->bfp_tail_first = first;
  return HPCG_OK;
}

static int build_fp64_tail(hpcg_ctx *h) {
  h->tail_first = -1;
  if (!h->tail_ok || !h->opt.persistent || h->levels < 2) return HPCG_OK;
  int first = h->levels;
  for (int l = h->levels - 1; l >= 1; --l) {
    const LevelTab &t = h->lv[l].tab;
    if (t.nch == 0 || t.nch2 != 1 || h->lv[l].n > 50000) break;
    first = l;
  }
  if (first >= h->levels) return HPCG_OK;
  for (int prec = 0; prec < 2; ++prec) {
    if (prec == 1 && h->opt.precision != HPCG_MIXED) continue;
    TailPlan P;
    memset(&P, 0, sizeof(P));
    P.first = first;
    P.last = h->levels - 1;
    P.count = h->count;
    for (int l = first; l < h->levels; ++l) {
      const LevelData &L = h->lv[l];
      TailLevel &T = P.lv[l];
      T.tab = L.tab.inst;
      T.r = prec == 0 ? (void *)L.r : (void *)L.r32;
      T.z = prec == 0 ? (void *)L.z : (void *)L.z32;
      T.invd = h->has_kappa ? (prec == 0 ? (const void *)L.invd : (const void *)L.invd32) : nullptr;
      T.kap = h->has_kappa ? (prec == 0 ? (const void *)L.kap : (const void *)L.kap32) : nullptr;
      T.lpc = L.tab.line_lpc;
      T.zc = L.tab.line_zc;
      T.nvb = L.tab.nblk_line;
      const bool coarsest = l == h->levels - 1;
      T.npre = make_runs(coarsest ? 1 : h->opt.pre_sweeps, h->opt.symmetric, T.pre, kTailRuns);
      T.npost = coarsest ? 0 : make_runs(h->opt.post_sweeps, h->opt.symmetric, T.post, kTailRuns);
      if (T.npre < 0 || T.npost < 0) return HPCG_OK;  // too many runs: no tail
      const TailRun last = T.pre[T.npre - 1];
      const int last_parity = (last.steps & 1) ? last.pa : 1 - last.pa;
      T.fuse = (!coarsest && last.cls == 0 && last_parity == 0) ? 1 : 0;
    }
    CK(cudaMemcpy(h->ws + h->o_tail + prec * sizeof(TailPlan), &P, sizeof(P), cudaMemcpyHostToDevice));
  }
  int dev = 0, sms = 0, occ = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_vcycle_tail<double>, 32 * kTailThreadsY, 0));
  int occ32 = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, k_vcycle_tail<float>, 32 * kTailThreadsY, 0));
  occ = std::min(occ, occ32);
  if (occ < 1) return HPCG_OK;
  // just enough blocks to take the largest phase in one round (fewer blocks
  // make every grid barrier cheaper), one per SM at most so all are resident
  int need = 1;
  for (int l = first; l < h->levels; ++l) {
    const LevelTab &t = h->lv[l].tab;
    const int vpb = std::max(1, kTailThreadsY / t.line_lpc);
    need = std::max(need, (t.nblk_line + vpb - 1) / vpb);
  }
  h->tail_grid = std::min(sms, need);
  h->tail_first = first;
  return HPCG_OK;
}

// Launches the tail for precision T (0: FP64 plan, 1: FP32 plan) as a cooperative kernel.
// stage_level >= 0: only that stage of that level (hpcg_mg_stage).
template <typename T>
static int enqueue_tail(hpcg_ctx *h, cudaStream_t s, const CgState *st, int stage_level = -1, int stage = 0) {
  unsigned *bar = (unsigned *)(h->ws + h->o_sync);
  int *err = (int *)(bar + 2);
  const TailPlan *plan = (const TailPlan *)(h->ws + h->o_tail + (sizeof(T) == 4 ? sizeof(TailPlan) : 0));
  CK(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(h->tail_grid);
  cfg.blockDim = dim3(32, kTailThreadsY);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_vcycle_tail<T>, plan, bar, err, h->wait_limit, const_cast<CgState *>(st), stage_level, stage);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (e != cudaSuccess) return cuda_fail(e, "k_vcycle_tail (cooperative launch)");
  return HPCG_OK;
}

static int reset_error_word(hpcg_ctx *h, cudaStream_t s) {
  CK(cudaMemsetAsync(h->ws + h->o_sync + 2 * sizeof(unsigned), 0, sizeof(int), s));
  return HPCG_OK;
}

// ---------------------------------------------------------------------------
// Smoother phase sequence: colours 0..7 (then 7..0 when symmetric) per sweep.
// A colour step recomputed right after the same colour's step returns the same
// bits (its inputs are r and the other colours, which did not change), so
// consecutive repeats are dropped.
static std::vector<int> phase_sequence(int sweeps, int symmetric) {
  std::vector<int> seq;
  for (int s = 0; s < sweeps; ++s) {
    for (int k = 0; k < 8; ++k) seq.push_back(k);
    if (symmetric)
      for (int k = 7; k >= 0; --k) seq.push_back(k);
  }
  std::vector<int> out;
  for (int k : seq)
    if (out.empty() || out.back() != k) out.push_back(k);
  return out;
}

template <typename T>
static const T *kap_of(const LevelData &L, bool has);
template <>
const double *kap_of<double>(const LevelData &L, bool has) { return has ? L.kap : nullptr; }
template <>
const float *kap_of<float>(const LevelData &L, bool has) { return has ? L.kap32 : nullptr; }
template <typename T>
static const T *invd_of(const LevelData &L, bool has);
template <>
const double *invd_of<double>(const LevelData &L, bool has) { return has ? L.invd : nullptr; }
template <>
const float *invd_of<float>(const LevelData &L, bool has) { return has ? L.invd32 : nullptr; }

template <typename T>
static int enqueue_zero(hpcg_ctx *h, int l, T *v, cudaStream_t s, const CgState *st) {
  const LevelData &L = h->lv[l];
  launch_k(k_zero_inst<T>, L.tab.nblk_red, kRedThreads, 0, s, L.tab.inst, h->count, v, st);
  CKL("k_zero_inst");
  return HPCG_OK;
}

template <typename T, int NCH>
static void launch_gs_lines(const LevelData &L, int count, int py, int pz, int pa, int steps, int vmask, const T *r, T *z, const T *invd,
                            const CgState *st, const Inst *tabc, T *rc, const T *kap, cudaStream_t s, bool fixed) {
  const dim3 grid(L.tab.nblk_line), block(32, L.tab.line_lpc);
  if constexpr (sizeof(T) == 8) {
    if (fixed && NCH <= 6) {  // longer lines would spill registers: plain FP64 sums
      launch_k(k_gs_lines_fx<NCH>, grid, block, 0, s, L.tab.inst, count, L.tab.line_lpc, L.tab.line_zc, py, pz, pa, steps, vmask, r, z, invd,
                                                st, tabc, rc, kap);
      return;
    }
  }
  if (L.even_nx && ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(z)) & (2 * sizeof(T) - 1)) == 0) {  // x pairs as vectors
    launch_k(k_gs_lines<T, NCH, true>, grid, block, 0, s, L.tab.inst, count, L.tab.line_lpc, L.tab.line_zc, py, pz, pa, steps, vmask, r, z,
             invd, st, tabc, rc, kap);
    return;
  }
  launch_k(k_gs_lines<T, NCH>, grid, block, 0, s, L.tab.inst, count, L.tab.line_lpc, L.tab.line_zc, py, pz, pa, steps, vmask, r, z, invd, st,
                                            tabc, rc, kap);
}

// `steps` colour steps on the lines of class (py, pz), alternating x parity
// from pa.  vmask: line classes holding valid z (others count as zero).  rc
// (nullable, class (0,0) runs ending on even x): fused residual + injection
// into level l+1.
template <typename T>
static int enqueue_line_steps(hpcg_ctx *h, int l, int py, int pz, int pa, int steps, const T *r, T *z, cudaStream_t s,
                              const CgState *st, int vmask = 0xF, T *rc = nullptr) {
  const LevelData &L = h->lv[l];
  const T *invd = invd_of<T>(L, h->has_kappa);
  const T *kap = kap_of<T>(L, h->has_kappa);
  const Inst *tabc = rc ? h->lv[l + 1].tab.inst : nullptr;
  switch (L.tab.nch ? L.tab.nch2 : 0) {
#define HPCG_GS_CASE(N) \
  case N: launch_gs_lines<T, N>(L, h->count, py, pz, pa, steps, vmask, r, z, invd, st, tabc, rc, kap, s, h->opt.fixed_point != 0); break;
    HPCG_GS_CASE(1) HPCG_GS_CASE(2) HPCG_GS_CASE(3) HPCG_GS_CASE(4) HPCG_GS_CASE(5) HPCG_GS_CASE(6)
    HPCG_GS_CASE(8)
#undef HPCG_GS_CASE
    default: {
      // lines longer than the register window: one launch per colour step
      // (callers zero z first and restrict separately on this path)
      if (rc || vmask != 0xF) return HPCG_ERR_UNSUPPORTED;
      for (int k = 0; k < steps; ++k) {
        const int px = (k & 1) ? 1 - pa : pa;
        launch_k(k_gs_color<T>, L.tab.nblk_half, dim3(kTileX, kTileY), 0, s, L.tab.inst, h->count, px, py, pz, r, z, invd, st);
        CKL("k_gs_color");
      }
      return HPCG_OK;
    }
  }
  CKL("k_gs_lines");
  return HPCG_OK;
}

template <typename T>
static int enqueue_colour(hpcg_ctx *h, int l, int k, const T *r, T *z, cudaStream_t s, const CgState *st) {
  return enqueue_line_steps<T>(h, l, (k >> 1) & 1, (k >> 2) & 1, k & 1, 1, r, z, s, st);
}

// The smoother's colour sequence grouped into runs of one line class: the
// colours 2m, 2m+1 of a run share (y, z) parities and alternate in x parity.
// from_zero: z holds no valid values yet (it counts as zero; nothing needs to
// be cleared first).  rc (nullable): restrict the residual into it, fused into
// the last run when that run is class (0,0) ending on even x; *fused tells
// whether that happened.
template <typename T>
static int enqueue_smoother(hpcg_ctx *h, int l, const T *r, T *z, int sweeps, cudaStream_t s, const CgState *st,
                            bool from_zero = false, T *rc = nullptr, bool *fused = nullptr) {
  const std::vector<int> seq = phase_sequence(sweeps, h->opt.symmetric);
  const bool lines = h->lv[l].tab.nch > 0;
  if (fused) *fused = false;
  if (from_zero && !lines) TRY(enqueue_zero<T>(h, l, z, s, st));
  int vmask = (from_zero && lines) ? 0 : 0xF;
  size_t i = 0;
  while (i < seq.size()) {
    size_t j = i + 1;
    while (j < seq.size() && (seq[j] >> 1) == (seq[i] >> 1)) ++j;
    const int k = seq[i];
    const int steps = (int)(j - i);
    const int cls = k >> 1;
    const int last_parity = (steps & 1) ? (k & 1) : 1 - (k & 1);
    T *rc_here = nullptr;
    if (rc && lines && j == seq.size() && cls == 0 && last_parity == 0) {
      rc_here = rc;
      if (fused) *fused = true;
    }
    TRY(enqueue_line_steps<T>(h, l, cls & 1, (cls >> 1) & 1, k & 1, steps, r, z, s, st, vmask, rc_here));
    vmask |= 1 << cls;
    i = j;
  }
  prof_mark(PK_SMOOTH, l);  // one event per smoother application: its runs keep their launch overlap
  return HPCG_OK;
}

// y = A x (Mode 0) or y = b - A x (Mode 1) on level l; optional p.Ap partials
// (then finalize with stencil mode 2).
template <typename T, int N, int Mode>
static void launch_spmv_lines(hpcg_ctx *h, const LevelData &L, const T *x, const T *b, T *y, const T *kap, double *partials,
                              const CgState *st, cudaStream_t s) {
  const dim3 blk(32, L.tab.row_lpc);
  if constexpr (sizeof(T) == 8 && N <= 6) {  // lines of up to 192 points: each plane staged once per block
    if (h->opt.fixed_point && L.tab.row_lpc <= kSpmvMaxLpc) {
      // a batch: each block takes the register window of its instance's lines
      auto kern = (h->count > 1 && N > 1) ? k_spmv_stage_fx_batch<N, Mode> : k_spmv_stage_fx<N, Mode>;
      // opt in to more than 48 KB of dynamic shared memory, once per device and kernel
      static std::atomic<unsigned long long> smem_set[2] = {{0}, {0}};
      const int which = kern == k_spmv_stage_fx<N, Mode> ? 0 : 1;
      const unsigned long long bit = 1ULL << (h->device & 63);
      if (!(smem_set[which].load(std::memory_order_relaxed) & bit)) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spmv_stage_smem<N>(kSpmvMaxLpc));
        smem_set[which].fetch_or(bit);
      }
      const int vec16 = L.even_nx && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
      launch_k(kern, L.tab.nblk_row, blk, spmv_stage_smem<N>(L.tab.row_lpc), s, L.tab.inst, h->count, L.tab.row_lpc, L.tab.row_zc, x, b, y,
               kap, partials, st, vec16);
      return;
    }
  }
  if constexpr (sizeof(T) == 8 && N <= 8) {
    if (h->opt.fixed_point) {
      launch_k(k_spmv_lines_fx<N, Mode>, L.tab.nblk_row, blk, 0, s, L.tab.inst, h->count, L.tab.row_lpc, L.tab.row_zc, x, b, y, kap, partials,
                                                              st);
      return;
    }
  }
  launch_k(k_spmv_lines<T, N, Mode>, L.tab.nblk_row, blk, 0, s, L.tab.inst, h->count, L.tab.row_lpc, L.tab.row_zc, x, b, y, kap, partials, st);
}

template <typename T, int Mode>
static int enqueue_spmv(hpcg_ctx *h, int l, const T *x, const T *b, T *y, const T *kap, double *partials, const CgState *st,
                        cudaStream_t s) {
  const LevelData &L = h->lv[l];
  switch (L.tab.nch) {
#define HPCG_SP_CASE(N)                                                          \
  case N:                                                                        \
    launch_spmv_lines<T, N, Mode>(h, L, x, b, y, kap, partials, st, s);          \
    break;
    HPCG_SP_CASE(1) HPCG_SP_CASE(2) HPCG_SP_CASE(3) HPCG_SP_CASE(4) HPCG_SP_CASE(5) HPCG_SP_CASE(6)
    HPCG_SP_CASE(7) HPCG_SP_CASE(8) HPCG_SP_CASE(10) HPCG_SP_CASE(12) HPCG_SP_CASE(16)
#undef HPCG_SP_CASE
    default:  // lines longer than the register window: one thread per row (partials per 32x8 tile)
      launch_k(k_spmv<T, Mode>, L.tab.nblk_full, dim3(kTileX, kTileY), 0, s, L.tab.inst, h->count, x, b, y, kap, partials, st);
      break;
  }
  CKL("k_spmv_lines");
  return HPCG_OK;
}

template <typename T>
static int enqueue_restrict(hpcg_ctx *h, int l, const T *r, const T *z, T *rc, cudaStream_t s, const CgState *st) {
  const LevelData &F = h->lv[l], &C = h->lv[l + 1];
  launch_k(k_restrict_residual<T>, C.tab.nblk_full, dim3(kTileX, kTileY), 0, s, F.tab.inst, C.tab.inst, h->count, r, z, rc,
                                                                          kap_of<T>(F, h->has_kappa), st);
  CKL("k_restrict_residual");
  prof_mark(PK_RESTRICT, l);
  return HPCG_OK;
}

template <typename T>
static int enqueue_prolong(hpcg_ctx *h, int l, const T *zc, T *z, cudaStream_t s, const CgState *st) {
  const LevelData &F = h->lv[l], &C = h->lv[l + 1];
  launch_k(k_prolong_add<T>, C.tab.nblk_full, dim3(kTileX, kTileY), 0, s, F.tab.inst, C.tab.inst, h->count, zc, z, st);
  CKL("k_prolong_add");
  prof_mark(PK_PROLONG, l);
  return HPCG_OK;
}


// ---------------------------------------------------------------------------
// The FP64 V-cycle with z in block floating point (hpcg_bfp.cuh): the same
// runs, restriction and refinement as enqueue_vcycle_t, on the level arrays
// zq (mantissas) and ze (line exponents).
template <int NC>
static void launch_gs_bfp(const LevelData &L, int count, int py, int pz, int pa, int steps, int vmask, const double *r, const double *invd,
                          const CgState *st, const Inst *tabc, double *rc, const double *kap, double *zout, double *dpart,
                          const LevelData *C, cudaStream_t s, bool split, bool refine_only) {
  if constexpr (NC >= 2 && NC <= 4) {
    // lines of 2-4 chunks: one warp per 64-point chunk (k_gs_lines_bfp_split;
    // steps == 0 there is the refinement alone)
    if (split && L.tab.line_lpc <= kBfpSplitMaxLines) {
      launch_k(k_gs_lines_bfp_split<NC>, dim3(L.tab.nblk_line), dim3(32, NC * L.tab.line_lpc), 0, s, L.tab.inst, count, L.tab.line_lpc,
               L.tab.line_zc, py, pz, pa, steps, vmask, r, L.zq, L.ze, invd, st, tabc, rc, kap, zout, dpart,
               C ? (const long long *)C->zq : nullptr, C ? (const int *)C->ze : nullptr, C ? C->tab.inst : nullptr, L.inst[0]);
      return;
    }
  }
  if constexpr (NC == 2 || NC == 3) {
    if (count > 1 && !refine_only) {  // a batch: each block takes the register window of its instance's lines
      launch_k(k_gs_lines_bfp_batch<NC>, dim3(L.tab.nblk_line), dim3(32, L.tab.line_lpc), 0, s, L.tab.inst, count, L.tab.line_lpc,
               L.tab.line_zc, py, pz, pa, steps, vmask, r, L.zq, L.ze, invd, st, tabc, rc, kap, zout, dpart,
               C ? (const long long *)C->zq : nullptr, C ? (const int *)C->ze : nullptr, C ? C->tab.inst : nullptr, L.inst[0]);
      return;
    }
  }
  if (refine_only) {  // hpcg_mg_stage: the fused refinement alone
    launch_k(k_gs_lines_bfp_refine<NC>, dim3(L.tab.nblk_line), dim3(32, L.tab.line_lpc), 0, s, L.tab.inst, count, L.tab.line_lpc,
             L.tab.line_zc, py, pz, pa, steps, vmask, r, L.zq, L.ze, invd, st, tabc, rc, kap, zout, dpart,
             C ? (const long long *)C->zq : nullptr, C ? (const int *)C->ze : nullptr, C ? C->tab.inst : nullptr, L.inst[0]);
    return;
  }
  launch_k(k_gs_lines_bfp<NC>, dim3(L.tab.nblk_line), dim3(32, L.tab.line_lpc), 0, s, L.tab.inst, count, L.tab.line_lpc, L.tab.line_zc, py,
           pz, pa, steps, vmask, r, L.zq, L.ze, invd, st, tabc, rc, kap, zout, dpart, C ? (const long long *)C->zq : nullptr,
           C ? (const int *)C->ze : nullptr, C ? C->tab.inst : nullptr, L.inst[0]);
}

// prolong (nullable): refine from this coarser level, fused into the run (a
// class (0,0) run of a post-smoother).
static int enqueue_line_steps_bfp(hpcg_ctx *h, int l, int py, int pz, int pa, int steps, const double *r, cudaStream_t s,
                                  const CgState *st, int vmask, double *rc, double *zout, double *dpart = nullptr,
                                  const LevelData *prolong = nullptr) {
  const LevelData &L = h->lv[l];
  const double *invd = invd_of<double>(L, h->has_kappa);
  const double *kap = kap_of<double>(L, h->has_kappa);
  const Inst *tabc = rc ? h->lv[l + 1].tab.inst : nullptr;
  switch (L.tab.nch2) {
#define HPCG_BFP_CASE(N) \
  case N: launch_gs_bfp<N>(L, h->count, py, pz, pa, steps, vmask, r, invd, st, tabc, rc, kap, zout, dpart, prolong, s, h->opt.bfp_split != 0, \
                           steps == 0); \
    break;
    HPCG_BFP_CASE(1) HPCG_BFP_CASE(2) HPCG_BFP_CASE(3) HPCG_BFP_CASE(4) HPCG_BFP_CASE(5) HPCG_BFP_CASE(6)
#undef HPCG_BFP_CASE
    default: return HPCG_ERR_UNSUPPORTED;
  }
  CKL("k_gs_lines_bfp");
  return HPCG_OK;
}

// Runs R (one z parity pz) of level l in one launch of k_gs_planes_bfp.
static int enqueue_planes_bfp(hpcg_ctx *h, int l, int pz, const PlaneRuns &R, const double *r, cudaStream_t s, const CgState *st) {
  const LevelData &L = h->lv[l];
  const LevelData *C = l + 1 < h->levels ? &h->lv[l + 1] : nullptr;
  const double *invd = invd_of<double>(L, h->has_kappa);
  const double *kap = kap_of<double>(L, h->has_kappa);
  const Inst &g = L.inst[0];
  const dim3 grid((unsigned)((g.nz - pz + 1) / 2)), block(32, kPlaneWarps);
  const Inst *tabc = C ? C->tab.inst : nullptr;
  const long long *zqc = C ? (const long long *)C->zq : nullptr;
  const int *zec = C ? (const int *)C->ze : nullptr;
  switch (L.tab.nch2) {
#define HPCG_PL_CASE(N) \
  case N: launch_k(k_gs_planes_bfp<N>, grid, block, 0, s, L.tab.inst, h->count, R, r, L.zq, L.ze, invd, st, tabc, kap, zqc, zec, tabc, g); break;
    HPCG_PL_CASE(1) HPCG_PL_CASE(2) HPCG_PL_CASE(3) HPCG_PL_CASE(4) HPCG_PL_CASE(5) HPCG_PL_CASE(6)
#undef HPCG_PL_CASE
    default: return HPCG_ERR_UNSUPPORTED;
  }
  CKL("k_gs_planes_bfp");
  return HPCG_OK;
}

// Whether level l's block-floating-point runs may be grouped by plane parity.
static bool planes_apply(const hpcg_ctx *h, int l) {
  const LevelData &L = h->lv[l];
  const bool split = h->opt.bfp_split && L.tab.nch2 >= 2 && L.tab.nch2 <= 4 && L.tab.line_lpc <= kBfpSplitMaxLines;
  return h->use_bfp && h->count == 1 && !split && L.tab.nch2 >= 1 && L.tab.nch2 <= 6;
}

// One smoother application (`sweeps` symmetric sweeps) on level l, grouped
// into runs as in enqueue_smoother.  rc (nullable): residual + injection
// fused into the last run, which for the symmetric smoother is class (0,0)
// ending on even x.  zout (nullable): the FP64 z, written by the last run of
// every line class; with dpart also the per-line partials of r.z.  refine:
// the refinement from level l+1 (Listing 1's z <- z + refine(z_c)) is fused
// into the first run, which for the symmetric smoother is class (0,0): the
// lines that hold every injected point.
static int enqueue_smoother_bfp(hpcg_ctx *h, int l, const double *r, int sweeps, cudaStream_t s, const CgState *st, bool from_zero,
                                double *rc, double *zout, double *dpart = nullptr, bool refine = false) {
  const std::vector<int> seq = phase_sequence(sweeps, 1);
  std::vector<std::pair<int, int>> runs;  // (first colour, steps)
  for (size_t i = 0; i < seq.size();) {
    size_t j = i + 1;
    while (j < seq.size() && (seq[j] >> 1) == (seq[i] >> 1)) ++j;
    runs.push_back({seq[i], (int)(j - i)});
    i = j;
  }
  int vmask = from_zero ? 0 : 0xF;
  const bool planes = h->lv[l].planes;
  PlaneRuns group{};  // runs of one plane parity waiting for their launch (planes)
  int group_pz = -1;
  for (size_t i = 0; i < runs.size(); ++i) {
    const int k = runs[i].first, steps = runs[i].second, cls = k >> 1;
    bool last_of_class = true;
    for (size_t j = i + 1; j < runs.size(); ++j) last_of_class = last_of_class && (runs[j].first >> 1) != cls;
    const int last_parity = (steps & 1) ? (k & 1) : 1 - (k & 1);
    double *rc_here = (rc && i + 1 == runs.size()) ? rc : nullptr;
    if (steps < 2 || (rc_here && (cls != 0 || last_parity != 0))) return HPCG_ERR_UNSUPPORTED;
    const bool refine_here = refine && i == 0;
    if (refine_here && cls != 0) return HPCG_ERR_UNSUPPORTED;
    if (planes) {
      const int pz = (cls >> 1) & 1;
      if (group.nruns > 0 && (pz != group_pz || group.nruns == kPlaneMaxRuns)) {
        TRY(enqueue_planes_bfp(h, l, group_pz, group, r, s, st));
        group = PlaneRuns{};
      }
      if (group.nruns == 0) {
        group.vmask = vmask;
        group_pz = pz;
      }
      PlaneRun &u = group.run[group.nruns++];
      u.cls = cls;
      u.pa = k & 1;
      u.steps = steps;
      u.refine = refine_here ? 1 : 0;
      u.rc = rc_here;
      u.zout = last_of_class ? zout : nullptr;
      u.dpart = last_of_class ? dpart : nullptr;
    } else {
      TRY(enqueue_line_steps_bfp(h, l, cls & 1, (cls >> 1) & 1, k & 1, steps, r, s, st, vmask, rc_here, last_of_class ? zout : nullptr,
                                 last_of_class ? dpart : nullptr, refine_here ? &h->lv[l + 1] : nullptr));
    }
    vmask |= 1 << cls;
  }
  if (planes && group.nruns > 0) TRY(enqueue_planes_bfp(h, l, group_pz, group, r, s, st));
  prof_mark(PK_SMOOTH, l);  // one event per smoother application: its runs keep their launch overlap
  return HPCG_OK;
}


// Levels bfp_tail_first..L-1 of the V-cycle in one cluster launch.
static int enqueue_tail_bfp(hpcg_ctx *h, cudaStream_t s, const CgState *st, int stage_level = -1, int stage = 0) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kBfpTailCtas);
  cfg.blockDim = dim3(32, kBfpTailWarps);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kBfpTailCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_vcycle_tail_bfp<1>, (const BfpTailPlan *)(h->ws + h->o_tail_bfp), st, stage_level, stage);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (e != cudaSuccess) return cuda_fail(e, "k_vcycle_tail_bfp (cluster launch)");
  prof_mark(PK_TAIL, h->bfp_tail_first);
  return HPCG_OK;
}

// Listing 1 on levels 0..L-1: r is the finest right-hand side (FP64), z the
// FP64 result on the finest level; rz (nullable): per-line partials of r.z.
static int enqueue_vcycle_bfp(hpcg_ctx *h, const double *r, double *z, cudaStream_t s, const CgState *st, double *rz) {
  const int L = h->levels;
  const int first = h->bfp_tail_first > 0 ? h->bfp_tail_first : L;  // levels from `first` run in the cluster kernel
  for (int l = 0; l < first; ++l) {
    const bool coarsest = l == L - 1;
    TRY(enqueue_smoother_bfp(h, l, l == 0 ? r : h->lv[l].r, coarsest ? 1 : h->opt.pre_sweeps, s, st, true,
                             coarsest ? nullptr : h->lv[l + 1].r, (coarsest && l == 0) ? z : nullptr, (coarsest && l == 0) ? rz : nullptr));
    if (coarsest) break;
  }
  if (first < L) TRY(enqueue_tail_bfp(h, s, st));
  for (int l = (first < L ? first : L - 1) - 1; l >= 0; --l) {
    // z <- z + refine(z_c), fused into the post-smoother's first run, then post-smoothing
    TRY(enqueue_smoother_bfp(h, l, l == 0 ? r : h->lv[l].r, h->opt.post_sweeps, s, st, false, nullptr, l == 0 ? z : nullptr,
                             l == 0 ? rz : nullptr, true));
  }
  return HPCG_OK;
}

// Listing 1 on levels 0..L-1; rl[l], zl[l] are the level vectors in precision T.
template <typename T>
static int enqueue_vcycle_t(hpcg_ctx *h, T *const *rl, T *const *zl, cudaStream_t s, const CgState *st) {
  const int L = h->levels;
  if (h->tail_first > 0) {
    const int first = h->tail_first;
    for (int l = 0; l < first; ++l) {
      bool fused = false;
      TRY(enqueue_smoother<T>(h, l, rl[l], zl[l], h->opt.pre_sweeps, s, st, true, rl[l + 1], &fused));
      if (!fused) TRY(enqueue_restrict<T>(h, l, rl[l], zl[l], rl[l + 1], s, st));
    }
    TRY(enqueue_tail<T>(h, s, st));  // levels first..L-1 and back up to `first`
    prof_mark(PK_TAIL, first);
    for (int l = first - 1; l >= 0; --l) {
      TRY(enqueue_prolong<T>(h, l, zl[l + 1], zl[l], s, st));
      TRY(enqueue_smoother<T>(h, l, rl[l], zl[l], h->opt.post_sweeps, s, st));
    }
    return HPCG_OK;
  }
  for (int l = 0; l < L; ++l) {
    // z <- 0 and pre-smoothing; on the way down the residual restriction
    // r_c <- restrict(r - A z) is fused into the smoother's last run when it
    // can be, else it is its own launch
    bool fused = false;
    TRY(enqueue_smoother<T>(h, l, rl[l], zl[l], l == L - 1 ? 1 : h->opt.pre_sweeps, s, st, true,
                            l == L - 1 ? nullptr : rl[l + 1], &fused));
    if (l == L - 1) break;  // coarsest: return
    if (!fused) TRY(enqueue_restrict<T>(h, l, rl[l], zl[l], rl[l + 1], s, st));
  }
  for (int l = L - 2; l >= 0; --l) {
    TRY(enqueue_prolong<T>(h, l, zl[l + 1], zl[l], s, st));                     // z <- z + refine(z_c)
    TRY(enqueue_smoother<T>(h, l, rl[l], zl[l], h->opt.post_sweeps, s, st));    // post-smoothing
  }
  return HPCG_OK;
}

// ---------------------------------------------------------------------------
// One stage of Listing 1 on one level (hpcg_mg_stage): exactly the launches
// the V-cycle above issues for that stage, on the handle's level vectors, so
// that the stages run in V-cycle order reproduce hpcg_mg_vcycle bit for bit.
enum VStore { VS_BFP = 0, VS_F64 = 1, VS_F32 = 2 };
static int vstore_of(const hpcg_ctx *h) {
  if (h->opt.precision == HPCG_MIXED) return VS_F32;
  return h->use_bfp ? VS_BFP : VS_F64;
}

template <typename T>
static int enqueue_stage_t(hpcg_ctx *h, int l, int stage, T *const *rl, T *const *zl, cudaStream_t s) {
  const bool coarsest = l == h->levels - 1;
  if (h->tail_first > 0 && l >= h->tail_first) return enqueue_tail<T>(h, s, nullptr, l, stage);
  if (stage == HPCG_STAGE_PRE) {
    bool fused = false;
    TRY(enqueue_smoother<T>(h, l, rl[l], zl[l], coarsest ? 1 : h->opt.pre_sweeps, s, nullptr, true, coarsest ? nullptr : rl[l + 1],
                            &fused));
    if (!coarsest && !fused) TRY(enqueue_restrict<T>(h, l, rl[l], zl[l], rl[l + 1], s, nullptr));
    return HPCG_OK;
  }
  TRY(enqueue_prolong<T>(h, l, zl[l + 1], zl[l], s, nullptr));
  if (stage == HPCG_STAGE_POST) TRY(enqueue_smoother<T>(h, l, rl[l], zl[l], h->opt.post_sweeps, s, nullptr));
  return HPCG_OK;
}

static int enqueue_stage(hpcg_ctx *h, int l, int stage, const double *r0, double *z0, cudaStream_t s) {
  const bool coarsest = l == h->levels - 1;
  const int vs = vstore_of(h);
  if (vs == VS_BFP) {
    if (h->bfp_tail_first > 0 && l >= h->bfp_tail_first) return enqueue_tail_bfp(h, s, nullptr, l, stage);
    const double *r = l == 0 ? r0 : h->lv[l].r;
    if (stage == HPCG_STAGE_PRE)
      return enqueue_smoother_bfp(h, l, r, coarsest ? 1 : h->opt.pre_sweeps, s, nullptr, true, coarsest ? nullptr : h->lv[l + 1].r,
                                  (coarsest && l == 0) ? z0 : nullptr);
    if (stage == HPCG_STAGE_REFINE)  // the refinement of the post-smoother's first run (class (0,0)), without its colour steps
      return enqueue_line_steps_bfp(h, l, 0, 0, 0, 0, r, s, nullptr, 0xF, nullptr, nullptr, nullptr, &h->lv[l + 1]);
    return enqueue_smoother_bfp(h, l, r, h->opt.post_sweeps, s, nullptr, false, nullptr, l == 0 ? z0 : nullptr, nullptr, true);
  }
  if (vs == VS_F64) {
    double *rl[kMaxLevels], *zl[kMaxLevels];
    rl[0] = const_cast<double *>(r0);
    zl[0] = z0;
    for (int k = 1; k < h->levels; ++k) {
      rl[k] = h->lv[k].r;
      zl[k] = h->lv[k].z;
    }
    return enqueue_stage_t<double>(h, l, stage, rl, zl, s);
  }
  float *rl[kMaxLevels], *zl[kMaxLevels];
  for (int k = 0; k < h->levels; ++k) {
    rl[k] = h->lv[k].r32;
    zl[k] = h->lv[k].z32;
  }
  const LevelData &L0 = h->lv[0];
  if (l == 0 && stage != HPCG_STAGE_REFINE) {  // the FP32 copy of r, as the V-cycle makes it
    launch_k(k_convert<double, float>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, r0, L0.r32, (const CgState *)nullptr);
    CKL("k_convert");
  }
  TRY(enqueue_stage_t<float>(h, l, stage, rl, zl, s));
  if (l == 0 && stage == HPCG_STAGE_POST) {
    launch_k(k_convert<float, double>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, L0.z32, z0, (const CgState *)nullptr);
    CKL("k_convert");
  }
  return HPCG_OK;
}

// Level vectors between the caller's FP64 buffers and the handle's storage
// (to_user: storage -> v).  which: 0 = r, 1 = z.
static int copy_level_vector(hpcg_ctx *h, int l, int which, double *v, bool to_user, cudaStream_t s) {
  LevelData &L = h->lv[l];
  const int vs = vstore_of(h);
  if (vs == VS_F32) {
    float *f = which == 0 ? L.r32 : L.z32;
    if (to_user)
      launch_k(k_convert<float, double>, L.tab.nblk_red, kRedThreads, 0, s, L.tab.inst, h->count, (const float *)f, v,
               (const CgState *)nullptr);
    else
      launch_k(k_convert<double, float>, L.tab.nblk_red, kRedThreads, 0, s, L.tab.inst, h->count, (const double *)v, f,
               (const CgState *)nullptr);
    CKL("k_convert");
    return HPCG_OK;
  }
  if (which == 1 && vs == VS_BFP) {
    const dim3 grid((unsigned)((L.nlines + 7) / 8)), block(32, 8);
    if (to_user)
      launch_k(k_bfp_to_double, grid, block, 0, s, L.tab.inst, h->count, L.nlines, (const long long *)L.zq, (const int *)L.ze, v);
    else
      launch_k(k_bfp_from_double, grid, block, 0, s, L.tab.inst, h->count, L.nlines, (const double *)v, L.zq, L.ze);
    CKL("k_bfp_convert");
    return HPCG_OK;
  }
  double *d = which == 0 ? L.r : L.z;
  if (to_user)
    CK(cudaMemcpyAsync(v, d, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemcpyAsync(d, v, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, s));
  return HPCG_OK;
}

static int level_vectors(hpcg_ctx *h, int level, double *r_dev, double *z_dev, bool to_user, cudaStream_t s) {
  if (level == 0 && r_dev) return HPCG_ERR_INVALID_ARG;                      // the finest r is the caller's own
  if (level == 0 && z_dev && vstore_of(h) == VS_F64) return HPCG_ERR_UNSUPPORTED;  // the finest z is the caller's z
  TRY(ensure_ready(h, s));
  if (r_dev) TRY(copy_level_vector(h, level, 0, r_dev, to_user, s));
  if (z_dev) TRY(copy_level_vector(h, level, 1, z_dev, to_user, s));
  return HPCG_OK;
}

// z = M r on level-0 FP64 vectors, in the handle's precision.  r32_current:
// the FP32 copy of r (level-0 r32) is already up to date (the CG update wrote it).
// rz (nullable) and *rz_done: the block-floating-point V-cycle also writes the
// per-line partials of r.z into rz, and says so.
static int enqueue_vcycle(hpcg_ctx *h, const double *r, double *z, cudaStream_t s, const CgState *st, bool r32_current = false,
                          bool keep_z32 = false, double *rz = nullptr, bool *rz_done = nullptr) {
  if (rz_done) *rz_done = false;
  if (h->opt.precision == HPCG_MIXED) {
    const LevelData &L0 = h->lv[0];
    if (!r32_current) {
      launch_k(k_convert<double, float>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, r, L0.r32, st);
      CKL("k_convert");
      prof_mark(PK_CONVERT, 0);
    }
    float *rl[kMaxLevels], *zl[kMaxLevels];
    for (int l = 0; l < h->levels; ++l) {
      rl[l] = h->lv[l].r32;
      zl[l] = h->lv[l].z32;
    }
    TRY(enqueue_vcycle_t<float>(h, rl, zl, s, st));
    if (!keep_z32) {
      launch_k(k_convert<float, double>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, L0.z32, z, st);
      CKL("k_convert");
      prof_mark(PK_CONVERT, 0);
    }
    return HPCG_OK;
  }
  if (h->use_bfp && h->tail_first <= 0 && ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(z)) & 15) == 0) {
    TRY(enqueue_vcycle_bfp(h, r, z, s, st, rz));
    if (rz_done) *rz_done = rz != nullptr;
    return HPCG_OK;
  }
  double *rl[kMaxLevels], *zl[kMaxLevels];
  rl[0] = const_cast<double *>(r);
  zl[0] = z;
  for (int l = 1; l < h->levels; ++l) {
    rl[l] = h->lv[l].r;
    zl[l] = h->lv[l].z;
  }
  return enqueue_vcycle_t<double>(h, rl, zl, s, st);
}

// Finalisation of a reduction with one partial per x-line of the finest
// level: across a cluster of kFinCluster blocks per instance when the GPU can
// run it, else in one block per instance (k_finalize, stencil 2).
template <int Kind>
static int enqueue_finalize_lines(hpcg_ctx *h, cudaStream_t s) {
  const LevelData &L0 = h->lv[0];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kFinCluster * h->count);
  cfg.blockDim = dim3(kRedThreads);
  cfg.stream = s;
  cudaLaunchAttribute a[1];
  a[0].id = cudaLaunchAttributeClusterDimension;
  a[0].val.clusterDim.x = kFinCluster;
  a[0].val.clusterDim.y = 1;
  a[0].val.clusterDim.z = 1;
  cfg.attrs = a;
  cfg.numAttrs = 1;
  if (h->fin_cluster_ok < 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_finalize_lines<Kind>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    h->fin_cluster_ok = n > 0 ? 1 : 0;
  }
  if (h->fin_cluster_ok) {
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_finalize_lines<Kind>, (const Inst *)L0.tab.inst, h->count, (const double *)h->part,
                                             h->st, h->hist);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (e != cudaSuccess) return cuda_fail(e, "k_finalize_lines (cluster launch)");
    return HPCG_OK;
  }
  launch_k(k_finalize<Kind>, h->count, kFinThreads, 0, s, L0.tab.inst, h->count, h->part, 2, h->st, h->hist, nullptr);
  CKL("k_finalize");
  return HPCG_OK;
}

// ---------------------------------------------------------------------------
// PCG (Section II-C), HPCG iteration order; every kernel is gated per instance
// by the device-side `done` flag, so iterations enqueued after convergence are
// no-ops and the host may run ahead of the device.  Each iteration's
// x += alpha p is deferred to the next iteration's p update (which reads the
// same old p); a solve ends with the pending one (enqueue_x_pending), and a
// mixed-precision residual replacement applies it before forming b - A x.
static int enqueue_pcg_init(hpcg_ctx *h, const double *b, double *x, int max_iters, double tol, cudaStream_t s) {
  std::vector<CgState> init(h->count);
  for (auto &c : init) {
    memset(&c, 0, sizeof(c));
    c.first = 1;
    c.tol = tol;
    c.max_iters = max_iters;
    c.mixed = h->opt.precision == HPCG_MIXED;
    c.restart_every = c.mixed && h->opt.restart_every > 0 ? h->opt.restart_every : 0;
    c.status = HPCG_OK;
  }
  CK(cudaMemcpyAsync(h->st, init.data(), sizeof(CgState) * h->count, cudaMemcpyHostToDevice, s));
  const LevelData &L0 = h->lv[0];
  // r = b - A x
  TRY((enqueue_spmv<double, 1>(h, 0, x, b, h->cg_r, h->has_kappa ? L0.kap : nullptr, nullptr, nullptr, s)));
  launch_k(k_dot_partial<double>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, h->cg_r, h->cg_r, h->part, h->st);
  CKL("k_dot_partial");
  launch_k(k_finalize<FIN_NORM0>, h->count, kRedThreads, 0, s, L0.tab.inst, h->count, h->part, 0, h->st, h->hist, nullptr);
  CKL("k_finalize<NORM0>");
  if (h->opt.precision == HPCG_MIXED) {  // FP32 copy of the initial residual for the preconditioner
    launch_k(k_convert<double, float>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, (const double *)h->cg_r, L0.r32,
             (const CgState *)nullptr);
    CKL("k_convert");
  }
  return HPCG_OK;
}

static int enqueue_pcg_iter(hpcg_ctx *h, const double *b, double *x, cudaStream_t s) {
  const LevelData &L0 = h->lv[0];
  const double *kap = h->has_kappa ? L0.kap : nullptr;
  const bool mixed = h->opt.precision == HPCG_MIXED;
  if (mixed) {
    launch_k(k_update_x_restart, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, (const double *)h->cg_p, x,
             (const CgState *)h->st);
    CKL("k_update_x_restart");
    launch_k(k_restart_residual, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, x, b, h->cg_r, L0.r32, kap, h->st);
    CKL("k_restart_residual");
    prof_mark(PK_UPDATE, 0);
  }
  // z = M r; mixed precision leaves z in FP32 (level-0 z32), which the dot and
  // the p update read directly (r32 is kept current by the CG updates)
  // (the block-floating-point V-cycle also leaves the per-line partials of r.z)
  bool rz_fused = false;
  TRY(enqueue_vcycle(h, h->cg_r, h->cg_z, s, h->st, mixed, mixed, h->part, &rz_fused));
  if (rz_fused) {
    TRY(enqueue_finalize_lines<FIN_RTZ>(h, s));
  } else {
    if (mixed)
      launch_k(k_dot_partial<float>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, h->cg_r, (const float *)L0.z32, h->part,
               h->st);
    else
      launch_k(k_dot_partial<double>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, h->cg_r, (const double *)h->cg_z,
               h->part, h->st);
    CKL("k_dot_partial");
    prof_mark(PK_DOT, 0);
    launch_k(k_finalize<FIN_RTZ>, h->count, kRedThreads, 0, s, L0.tab.inst, h->count, h->part, 0, h->st, h->hist, nullptr);
    CKL("k_finalize<RTZ>");
  }
  prof_mark(PK_FINALIZE, 0);
  if (mixed)
    launch_k(k_update_p<float>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, (const float *)L0.z32, h->cg_p, x, h->st);
  else
    launch_k(k_update_p<double>, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, (const double *)h->cg_z, h->cg_p, x,
             h->st);  // with the previous iteration's x += alpha p
  CKL("k_update_p");
  prof_mark(PK_UPDATE, 0);
  TRY((enqueue_spmv<double, 0>(h, 0, h->cg_p, nullptr, h->cg_ap, kap, h->part, h->st, s)));  // Ap, p.Ap partials
  prof_mark(PK_SPMV, 0);
  if (L0.tab.nch) {
    TRY(enqueue_finalize_lines<FIN_PAP>(h, s));
  } else {
    launch_k(k_finalize<FIN_PAP>, h->count, kFinThreads, 0, s, L0.tab.inst, h->count, h->part, 1, h->st, h->hist, nullptr);
    CKL("k_finalize<PAP>");
  }
  prof_mark(PK_FINALIZE, 0);
  launch_k(k_update_xr, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, h->cg_p, h->cg_ap, (double *)nullptr, h->cg_r,
           mixed ? L0.r32 : nullptr, h->part, h->st);
  CKL("k_update_xr");
  prof_mark(PK_UPDATE, 0);
  launch_k(k_finalize<FIN_NORM>, h->count, kRedThreads, 0, s, L0.tab.inst, h->count, h->part, 0, h->st, h->hist, nullptr);
  CKL("k_finalize<NORM>");
  prof_mark(PK_FINALIZE, 0);
  return HPCG_OK;
}

// Captures one CG iteration into a graph (cached per (b, x)).
static int get_iter_graph(hpcg_ctx *h, const double *b, double *x, cudaGraphExec_t *out, long *kernels) {
  GraphCache &g = h->g_iter;
  if (g.exec && g.key[0] == b && g.key[1] == x) {
    *out = g.exec;
    *kernels = g.kernels;
    return HPCG_OK;
  }
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  long nk = 0;
  for (int attempt = 0;; ++attempt) {
    cudaGraph_t graph = nullptr;
    const long before = g_launches.load();
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_pcg_iter(h, b, x, h->cap);
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    nk = g_launches.load() - before;
    g_launches.fetch_sub(nk);  // counted again at every replay
    if (rc == HPCG_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc == HPCG_OK && e == cudaSuccess) break;
    cudaGetLastError();
    if (attempt == 0 && h->tail_first > 0) {
      // a cooperative launch the capture refused: fall back to one launch per step
      h->tail_ok = false;
      TRY(build_tail_plans(h));
      continue;
    }
    if (rc != HPCG_OK) return rc;
    return cuda_fail(e, "iteration graph capture");
  }
  g.key[0] = b;
  g.key[1] = x;
  g.kernels = nk;
  *out = g.exec;
  *kernels = nk;
  return HPCG_OK;
}

// The last x += alpha p of every instance: the iterations defer it to the next
// iteration's p update, so a solve ends with it.
static int enqueue_x_pending(hpcg_ctx *h, double *x, cudaStream_t s) {
  const LevelData &L0 = h->lv[0];
  launch_k(k_update_x_pending, L0.tab.nblk_red, kRedThreads, 0, s, L0.tab.inst, h->count, (const double *)h->cg_p, x,
           (const CgState *)h->st);
  CKL("k_update_x_pending");
  return HPCG_OK;
}

// flag[0] = 1 once every instance of a batch has finished its solve (the
// batch's convergence flag, polled by the host like a single grid's done).
__global__ void k_all_done(const CgState *__restrict__ st, int count, int *flag) {
  pdl_enter();
  int ok = 1;
  for (int i = threadIdx.x; i < count; i += blockDim.x) ok &= st[i].done != 0;
  ok = __syncthreads_and(ok);
  if (threadIdx.x == 0) *flag = ok;
}

// The pinned flag slots and events of the convergence poll, made on the
// first tolerance solve of the handle (cudaMallocHost synchronises the device).
static int ensure_poll(hpcg_ctx *h) {
  if (!h->poll_flags) CK(cudaMallocHost(&h->poll_flags, sizeof(int) * 2));
  for (int k = 0; k < 2; ++k)
    if (!h->poll_ev[k]) CK(cudaEventCreateWithFlags(&h->poll_ev[k], cudaEventDisableTiming));
  return HPCG_OK;
}

static int run_pcg(hpcg_ctx *h, const double *b, double *x, int max_iters, double tol, hpcg_stats *stats, cudaStream_t s) {
  if (max_iters < 0 || max_iters > kHistoryCap) return HPCG_ERR_INVALID_ARG;
  TRY(reset_error_word(h, s));
  TRY(enqueue_pcg_init(h, b, x, max_iters, tol, s));
  cudaGraphExec_t exec;
  long nk = 0;
  TRY(get_iter_graph(h, b, x, &exec, &nk));
  const int every = h->opt.check_every > 0 ? h->opt.check_every : 1;
  std::vector<CgState> hs(h->count);
  if (tol > 0.0) TRY(ensure_poll(h));
  int *const all_done = (int *)(h->ws + h->o_sync + 16);  // batches: every instance done
  int rc = HPCG_OK;
  int pending = -1;  // slot whose flag copy is in flight
  for (int it = 0; it < max_iters; ++it) {
    cudaError_t e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaGraphLaunch");
      break;
    }
    g_launches.fetch_add(nk);
    if (tol > 0.0 && ((it + 1) % every == 0)) {
      // the host reads the flag of the iteration before this one while the GPU
      // runs this one (one iteration of lag; iterations enqueued after
      // convergence are no-ops on the device): a single grid's done, or the
      // all-done flag of a batch
      const int slot = it & 1;
      const int *flag = &h->st[0].done;
      if (h->count > 1) {
        e = launch_k(k_all_done, dim3(1), dim3(256), 0, s, (const CgState *)h->st, h->count, all_done);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        flag = all_done;
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->poll_flags + slot, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaEventRecord(h->poll_ev[slot], s);
      if (e == cudaSuccess && pending >= 0) e = cudaEventSynchronize(h->poll_ev[pending]);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "convergence flag poll");
        break;
      }
      if (pending >= 0 && h->poll_flags[pending]) break;
      pending = slot;
    }
  }
  if (rc == HPCG_OK) rc = enqueue_x_pending(h, x, s);
  if (rc == HPCG_OK) {
    cudaError_t e = cudaMemcpyAsync(hs.data(), h->st, sizeof(CgState) * h->count, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "stats copy");
  }
  if (rc != HPCG_OK) return rc;
  int worst = HPCG_OK;
  for (int i = 0; i < h->count; ++i) {
    const CgState &c = hs[i];
    int st = c.status;
    if (st == HPCG_OK && tol > 0.0 && !c.converged) st = HPCG_ERR_NOT_CONVERGED;
    if (stats) {
      hpcg_stats &o = stats[i];
      o.iters = c.iter;
      o.restarts = c.restarts;
      o.converged = c.converged;
      o.status = st;
      o.rel_res = c.normr0 > 0 ? c.normr / c.normr0 : 0.0;
      if (o.history && o.history_cap > 0 && c.iter > 0) {
        int m = c.iter < o.history_cap ? c.iter : o.history_cap;
        CK(cudaMemcpy(o.history, h->hist + (size_t)i * kHistoryCap, sizeof(double) * m, cudaMemcpyDeviceToHost));
      }
    }
    if (st == HPCG_ERR_TIMEOUT || (st == HPCG_ERR_BREAKDOWN && worst != HPCG_ERR_TIMEOUT)) worst = st;
    else if (st != HPCG_OK && worst == HPCG_OK) worst = st;
  }
  int err = 0;
  CK(cudaMemcpy(&err, h->ws + h->o_sync + 2 * sizeof(unsigned), sizeof(int), cudaMemcpyDeviceToHost));
  if (err) worst = HPCG_ERR_TIMEOUT;
  return worst;
}

// ---------------------------------------------------------------------------
// Launch-shape autotuner: for every level, times each candidate (lines per
// block, planes per block) of the SpMV line kernel and of the colour-pair line
// kernel on the level's own vectors and keeps the fastest.  The shape changes
// only how lines are grouped into blocks, never the arithmetic of a row.
static int time_shape(hpcg_ctx *h, int l, bool rows, int lpc, int zc, cudaStream_t s, float *ms) {
  LevelData &L = h->lv[l];
  if (rows) {
    L.tab.row_lpc = lpc;
    L.tab.row_zc = zc;
  } else {
    L.tab.line_lpc = lpc;
    L.tab.line_zc = zc;
  }
  set_line_prefixes(L);
  CK(cudaMemcpyAsync((void *)L.tab.inst, L.inst.data(), sizeof(Inst) * h->count, cudaMemcpyHostToDevice, s));
  double *a = l == 0 ? h->cg_r : L.r;
  double *b = l == 0 ? h->cg_z : L.z;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = HPCG_OK;
  const int reps = 6;
  for (int it = 0; it <= reps && rc == HPCG_OK; ++it) {
    if (it == 1) cudaEventRecord(e0, s);
    if (rows)
      rc = enqueue_spmv<double, 0>(h, l, a, nullptr, b, nullptr, nullptr, nullptr, s);
    else if (h->opt.precision == HPCG_MIXED)  // the V-cycle runs the FP32 kernel
      rc = enqueue_line_steps<float>(h, l, 0, 0, 0, 2, L.r32, L.z32, s, nullptr);
    else if (h->use_bfp)  // ... or the block-floating-point one
      rc = enqueue_line_steps_bfp(h, l, 0, 0, 0, 2, a, s, nullptr, 0xF, nullptr, nullptr);
    else
      rc = enqueue_line_steps<double>(h, l, 0, 0, 0, 2, a, b, s, nullptr);
  }
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HPCG_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
  *ms = t / reps;
  return HPCG_OK;
}

// One block-floating-point smoother application on level l (from z = 0, as
// the pre-smoother), timed over a few repetitions.
static int time_smoother_bfp(hpcg_ctx *h, int l, const double *r, cudaStream_t s, float *ms) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = HPCG_OK;
  const int reps = 4;
  for (int it = 0; it <= reps && rc == HPCG_OK; ++it) {
    if (it == 1) cudaEventRecord(e0, s);
    rc = enqueue_smoother_bfp(h, l, r, 1, s, nullptr, true, nullptr, nullptr);
  }
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HPCG_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
  *ms = t / reps;
  return HPCG_OK;
}

static int autotune_impl(hpcg_ctx *h, int *shapes, cudaStream_t s) {
  static const int lpcs[] = {1, 2, 4, 8};
  static const int zcs[] = {1, 2, 4, 8, 16};
  for (int l = 0; l < h->levels; ++l) {
    LevelData &L = h->lv[l];
    if (L.tab.nch == 0) continue;
    double *a = l == 0 ? h->cg_r : L.r;
    double *b = l == 0 ? h->cg_z : L.z;
    CK(cudaMemsetAsync(a, 0, sizeof(double) * L.n, s));
    CK(cudaMemsetAsync(b, 0, sizeof(double) * L.n, s));
    if (h->opt.precision == HPCG_MIXED) {
      CK(cudaMemsetAsync(L.r32, 0, sizeof(float) * L.n, s));
      CK(cudaMemsetAsync(L.z32, 0, sizeof(float) * L.n, s));
    }
    if (h->use_bfp)  // valid (zero) lines and exponents to time on
      TRY(enqueue_smoother_bfp(h, l, a, 1, s, nullptr, true, nullptr, nullptr));
    for (int pass = 0; pass < 2; ++pass) {
      const bool rows = pass == 0;
      float best = 1e30f;
      int bl = rows ? L.tab.row_lpc : L.tab.line_lpc, bz = rows ? L.tab.row_zc : L.tab.line_zc;
      for (int zc : zcs)
        for (int lpc : lpcs) {
          float ms = 0.f;
          TRY(time_shape(h, l, rows, lpc, zc, s, &ms));
          if (ms < best) {
            best = ms;
            bl = lpc;
            bz = zc;
          }
        }
      if (rows) {
        L.tab.row_lpc = bl;
        L.tab.row_zc = bz;
      } else {
        L.tab.line_lpc = bl;
        L.tab.line_zc = bz;
      }
      set_line_prefixes(L);
    }
    CK(cudaMemcpyAsync((void *)L.tab.inst, L.inst.data(), sizeof(Inst) * h->count, cudaMemcpyHostToDevice, s));
    if (h->opt.fuse_planes == 0 && planes_apply(h, l)) {  // one smoother application with and without grouped runs
      float ms[2] = {0.f, 0.f};
      for (int fused = 0; fused < 2; ++fused) {
        L.planes = fused != 0;
        TRY(time_smoother_bfp(h, l, a, s, &ms[fused]));
      }
      L.planes = ms[1] < ms[0];
    }
  }
  CK(cudaStreamSynchronize(s));
  // partial-sum buffers are sized by the largest launch: keep within them
  const size_t need_part = (size_t)std::max(std::max(h->lv[0].tab.nblk_full, h->lv[0].tab.nblk_red), h->lv[0].tab.nblk_row) + 64;
  if (need_part > h->npart) return HPCG_ERR_NO_WORKSPACE;
  if (shapes)
    for (int l = 0; l < h->levels; ++l) {
      shapes[4 * l + 0] = h->lv[l].tab.row_lpc;
      shapes[4 * l + 1] = h->lv[l].tab.row_zc;
      shapes[4 * l + 2] = h->lv[l].tab.line_lpc;
      shapes[4 * l + 3] = h->lv[l].tab.line_zc;
    }
  if (h->g_iter.exec) {  // captured with the previous block counts
    cudaGraphExecDestroy(h->g_iter.exec);
    h->g_iter = GraphCache{};
  }
  h->tuned = true;
  return build_tail_plans(h);
}

// ---------------------------------------------------------------------------
// C ABI
extern "C" {

int hpcg_profile_iteration(hpcg_handle h, const double *b_dev, double *x_dev, double *ms_host, int cap, void *stream) {
  if (!h || !b_dev || !x_dev || !ms_host) return HPCG_ERR_INVALID_ARG;
  const int L = h->levels;
  if (cap < 3 * L + 7) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  TRY(reset_error_word(h, s));
  TRY(enqueue_pcg_init(h, b_dev, x_dev, 2, 0.0, s));
  // one warm-up iteration (caches, clocks), then the timed one
  TRY(enqueue_pcg_iter(h, b_dev, x_dev, s));
  Prof prof;
  prof.s = s;
  t_prof = &prof;
  prof_mark(PK_COUNT, 0);  // start
  int rc = enqueue_pcg_iter(h, b_dev, x_dev, s);
  t_prof = nullptr;
  if (rc == HPCG_OK) rc = enqueue_x_pending(h, x_dev, s);
  cudaError_t e = cudaStreamSynchronize(s);
  for (int i = 0; i < 3 * L + 7; ++i) ms_host[i] = 0.0;
  if (rc == HPCG_OK && e == cudaSuccess) {
    for (size_t i = 1; i < prof.ev.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, prof.ev[i - 1], prof.ev[i]);
      const int kind = prof.tag[i] / 16, lev = prof.tag[i] % 16;
      double *slot = nullptr;
      switch (kind) {
        case PK_SMOOTH: slot = &ms_host[lev]; break;
        case PK_RESTRICT: slot = &ms_host[L + lev]; break;
        case PK_PROLONG: slot = &ms_host[2 * L + lev]; break;
        case PK_TAIL: slot = &ms_host[3 * L]; break;
        case PK_SPMV: slot = &ms_host[3 * L + 1]; break;
        case PK_DOT: slot = &ms_host[3 * L + 2]; break;
        case PK_UPDATE: slot = &ms_host[3 * L + 3]; break;
        case PK_FINALIZE: slot = &ms_host[3 * L + 4]; break;
        case PK_CONVERT: slot = &ms_host[3 * L + 5]; break;
        default: break;
      }
      if (slot) *slot += ms;
      ms_host[3 * L + 6] += ms;
    }
  }
  for (cudaEvent_t ev : prof.ev) cudaEventDestroy(ev);
  if (rc != HPCG_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "profile synchronize");
  return HPCG_OK;
}

int hpcg_set_wait_limit(hpcg_handle h, long long cycles) {
  if (!h || cycles < 0) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  h->wait_limit = cycles;
  if (h->g_iter.exec) {  // the limit is a kernel argument of the captured graph
    cudaGraphExecDestroy(h->g_iter.exec);
    h->g_iter = GraphCache{};
  }
  return HPCG_OK;
}

int hpcg_device_status(hpcg_handle h, int *status_out) {
  if (!h || !status_out) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  *status_out = HPCG_OK;
  if (!h->ready) return HPCG_OK;
  CK(cudaDeviceSynchronize());
  int err = 0;
  CK(cudaMemcpy(&err, h->ws + h->o_sync + 2 * sizeof(unsigned), sizeof(int), cudaMemcpyDeviceToHost));
  *status_out = err ? HPCG_ERR_TIMEOUT : HPCG_OK;
  return HPCG_OK;
}

int hpcg_persistent_levels(hpcg_handle h, int *first_level) {
  if (!h || !first_level) return HPCG_ERR_INVALID_ARG;
  *first_level = h->tail_first;
  return HPCG_OK;
}

int hpcg_set_launch_shapes(hpcg_handle h, const int *shapes_host) {
  if (!h || !shapes_host) return HPCG_ERR_INVALID_ARG;
  for (int l = 0; l < h->levels; ++l)
    for (int k = 0; k < 4; ++k) {
      const int v = shapes_host[4 * l + k];
      if (v < 1 || v > ((k & 1) ? 64 : 8)) return HPCG_ERR_INVALID_ARG;
    }
  std::lock_guard<std::mutex> lk(h->mu);
  for (int l = 0; l < h->levels; ++l) {
    LevelData &L = h->lv[l];
    L.tab.row_lpc = shapes_host[4 * l + 0];
    L.tab.row_zc = shapes_host[4 * l + 1];
    L.tab.line_lpc = shapes_host[4 * l + 2];
    L.tab.line_zc = shapes_host[4 * l + 3];
    set_line_prefixes(L);
    if (h->ready) CK(cudaMemcpy((void *)L.tab.inst, L.inst.data(), sizeof(Inst) * h->count, cudaMemcpyHostToDevice));
  }
  if (h->g_iter.exec) {
    cudaGraphExecDestroy(h->g_iter.exec);
    h->g_iter = GraphCache{};
  }
  h->tuned = true;
  return h->ready ? build_tail_plans(h) : HPCG_OK;
}

int hpcg_autotune(hpcg_handle h, int *shapes_host, void *stream) {
  if (!h) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const int tune = h->opt.autotune;
  h->opt.autotune = 0;  // ensure_ready must not tune on its own here
  int rc = ensure_ready(h, s);
  h->opt.autotune = tune;
  if (rc != HPCG_OK) return rc;
  return autotune_impl(h, shapes_host, s);
}

int hpcg_options_default(hpcg_options *opt, int nx, int ny, int nz) {
  if (!opt) return HPCG_ERR_INVALID_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->nx = nx;
  opt->ny = ny;
  opt->nz = nz;
  opt->levels = 4;
  opt->precision = HPCG_FP64;
  opt->pre_sweeps = 1;
  opt->post_sweeps = 1;
  opt->symmetric = 1;
  opt->check_every = 1;
  opt->max_rhs = 0;
  opt->autotune = 1;
  opt->fixed_point = 1;
  opt->pdl = 1;
  opt->persistent = 0;
  opt->block_fp = 1;
  opt->cluster_tail = 0;
  opt->restart_every = 0;
  opt->bfp_split = 0;
  opt->fuse_planes = 0;
  return HPCG_OK;
}

static int make_handle(const hpcg_options *opt, const std::vector<int> &dims, int batch, hpcg_handle *out) {
  hpcg_ctx *h = new hpcg_ctx();
  h->opt = *opt;
  h->batch = batch;
  h->levels = opt->levels;
  plan(h, dims);
  // block floating point needs the colour-pair line kernels on every level
  // (lines of at most 6 x 64 points), even line lengths (its kernels move
  // x pairs as 16-byte vectors) and a smoother whose last run restricts
  bool bfp = opt->block_fp && opt->precision == HPCG_FP64 && opt->fixed_point && opt->symmetric && !opt->persistent;
  for (int l = 0; l < h->levels; ++l) {
    bfp = bfp && h->lv[l].tab.nch > 0 && h->lv[l].tab.nch2 >= 1 && h->lv[l].tab.nch2 <= 6;
    for (const Inst &g : h->lv[l].inst) bfp = bfp && (g.nx % 2) == 0;
  }
  h->use_bfp = bfp;
  for (int l = 0; l < h->levels; ++l) h->lv[l].planes = opt->fuse_planes > 0 && planes_apply(h, l);
  *out = h;
  return HPCG_OK;
}

int hpcg_setup_ex(const hpcg_options *opt, const double *kappa_dev, hpcg_handle *out) {
  if (!opt || !out) return HPCG_ERR_INVALID_ARG;
  TRY(validate_dims(opt->nx, opt->ny, opt->nz, opt->levels));
  if (opt->precision != HPCG_FP64 && opt->precision != HPCG_MIXED) return HPCG_ERR_INVALID_ARG;
  if (opt->pre_sweeps < 1 || opt->post_sweeps < 1 || opt->pre_sweeps > 16 || opt->post_sweeps > 16) return HPCG_ERR_INVALID_ARG;
  if (opt->max_rhs < 0 || opt->max_rhs > 64) return HPCG_ERR_INVALID_ARG;
  std::vector<int> dims = {opt->nx, opt->ny, opt->nz};
  TRY(make_handle(opt, dims, 0, out));
  (*out)->kappa_pending = kappa_dev;
  return HPCG_OK;
}

int hpcg_setup(int nx, int ny, int nz, int levels, hpcg_handle *out) {
  hpcg_options o;
  hpcg_options_default(&o, nx, ny, nz);
  o.levels = levels;
  return hpcg_setup_ex(&o, nullptr, out);
}

int hpcg_setup_batch(int count, const int *dims_host, int levels, int precision, hpcg_handle *out) {
  if (count < 1 || count > 4096 || !dims_host || !out) return HPCG_ERR_INVALID_ARG;
  if (precision != HPCG_FP64 && precision != HPCG_MIXED) return HPCG_ERR_INVALID_ARG;
  std::vector<int> dims(dims_host, dims_host + 3 * count);
  for (int i = 0; i < count; ++i) TRY(validate_dims(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], levels));
  hpcg_options o;
  hpcg_options_default(&o, dims[0], dims[1], dims[2]);
  o.levels = levels;
  o.precision = precision;
  o.check_every = 4;
  return make_handle(&o, dims, 1, out);
}

int hpcg_batch_offsets(hpcg_handle h, long *offsets_host) {
  if (!h || !offsets_host) return HPCG_ERR_INVALID_ARG;
  for (int i = 0; i < h->count; ++i) offsets_host[i] = h->lv[0].inst[i].off;
  offsets_host[h->count] = h->lv[0].n;
  return HPCG_OK;
}

int hpcg_set_kappa(hpcg_handle h, const double *kappa_dev, void *stream) {
  if (!h) return HPCG_ERR_INVALID_ARG;
  if (h->batch) return HPCG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(h->mu);
  h->kappa_pending = nullptr;
  TRY(ensure_ready(h, (cudaStream_t)stream));
  if (h->g_iter.exec) {  // kernels captured with or without kappa: recapture
    cudaGraphExecDestroy(h->g_iter.exec);
    h->g_iter = GraphCache{};
  }
  return set_kappa_impl(h, kappa_dev, (cudaStream_t)stream);
}

int hpcg_destroy(hpcg_handle h) {
  if (!h) return HPCG_ERR_INVALID_ARG;
  if (h->ready) cudaDeviceSynchronize();
  if (h->g_iter.exec) cudaGraphExecDestroy(h->g_iter.exec);
  for (cudaEvent_t e : h->poll_ev)
    if (e) cudaEventDestroy(e);
  if (h->poll_flags) cudaFreeHost(h->poll_flags);
  if (h->multi) hpcg_destroy(h->multi);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->ws_owned && h->ws) cudaFree(h->ws);
  delete h;
  return HPCG_OK;
}

int hpcg_workspace_bytes(hpcg_handle h, size_t *bytes) {
  if (!h || !bytes) return HPCG_ERR_INVALID_ARG;
  *bytes = h->need;
  return HPCG_OK;
}

int hpcg_bind_workspace(hpcg_handle h, void *dev, size_t bytes) {
  if (!h || !dev) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  return bind(h, (char *)dev, bytes, false);
}

int hpcg_level_dims(hpcg_handle h, int level, int *dims_host) {
  if (!h || !dims_host || level < 0 || level >= h->levels) return HPCG_ERR_INVALID_ARG;
  const Inst &g = h->lv[level].inst[0];
  dims_host[0] = g.nx;
  dims_host[1] = g.ny;
  dims_host[2] = g.nz;
  return HPCG_OK;
}

int hpcg_get_colors(hpcg_handle h, int level, int *colors_dev, void *stream) {
  if (!h || !colors_dev || level < 0 || level >= h->levels) return HPCG_ERR_INVALID_ARG;
  const Inst &g = h->lv[level].inst[0];
  launch_k(k_colors, grid_for(g.n), 256, 0, (cudaStream_t)stream, g.nx, g.ny, g.nz, colors_dev);
  CKL("k_colors");
  return HPCG_OK;
}

int hpcg_get_f2c(hpcg_handle h, int level, int *f2c_dev, void *stream) {
  if (!h || !f2c_dev || level < 0 || level >= h->levels - 1) return HPCG_ERR_INVALID_ARG;
  const Inst &f = h->lv[level].inst[0], &c = h->lv[level + 1].inst[0];
  launch_k(k_f2c, grid_for(c.n), 256, 0, (cudaStream_t)stream, f.nx, f.ny, c.nx, c.ny, c.nz, f2c_dev);
  CKL("k_f2c");
  return HPCG_OK;
}

int hpcg_get_row_nnz(hpcg_handle h, int level, int *nnz_dev, void *stream) {
  if (!h || !nnz_dev || level < 0 || level >= h->levels) return HPCG_ERR_INVALID_ARG;
  const Inst &g = h->lv[level].inst[0];
  launch_k(k_row_nnz, grid_for(g.n), 256, 0, (cudaStream_t)stream, g.nx, g.ny, g.nz, nnz_dev);
  CKL("k_row_nnz");
  return HPCG_OK;
}

int hpcg_get_rhs(hpcg_handle h, double *b_dev, void *stream) {
  if (!h || !b_dev) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  for (int i = 0; i < h->count; ++i) {
    const Inst &g = h->lv[0].inst[i];
    launch_k(k_rhs_ones, grid_for(g.n), 256, 0, s, g.nx, g.ny, g.nz, h->has_kappa ? h->lv[0].kap : nullptr, b_dev + g.off);
    CKL("k_rhs_ones");
  }
  return HPCG_OK;
}

int hpcg_spmv(hpcg_handle h, int level, const double *x_dev, double *y_dev, void *stream) {
  if (!h || !x_dev || !y_dev || level < 0 || level >= h->levels) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  const LevelData &L = h->lv[level];
  TRY((enqueue_spmv<double, 0>(h, level, x_dev, nullptr, y_dev, h->has_kappa ? L.kap : nullptr, nullptr, nullptr, s)));
  return HPCG_OK;
}

int hpcg_rbgs_color(hpcg_handle h, int level, int color, const double *r_dev, double *z_dev, void *stream) {
  if (!h || !r_dev || !z_dev || level < 0 || level >= h->levels || color < 0 || color > 7) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  return enqueue_colour<double>(h, level, color, r_dev, z_dev, s, nullptr);
}

int hpcg_rbgs(hpcg_handle h, int level, const double *r_dev, double *z_dev, void *stream) {
  if (!h || !r_dev || !z_dev || level < 0 || level >= h->levels) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  return enqueue_smoother<double>(h, level, r_dev, z_dev, 1, s, nullptr);
}

int hpcg_restrict_residual(hpcg_handle h, int level, const double *r_dev, const double *z_dev, double *rc_dev, void *stream) {
  if (!h || !r_dev || !z_dev || !rc_dev || level < 0 || level >= h->levels - 1) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  return enqueue_restrict<double>(h, level, r_dev, z_dev, rc_dev, s, nullptr);
}

int hpcg_prolong_add(hpcg_handle h, int level, const double *zc_dev, double *z_dev, void *stream) {
  if (!h || !zc_dev || !z_dev || level < 0 || level >= h->levels - 1) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  return enqueue_prolong<double>(h, level, zc_dev, z_dev, s, nullptr);
}

int hpcg_mg_vcycle(hpcg_handle h, const double *r_dev, double *z_dev, void *stream) {
  if (!h || !r_dev || !z_dev || r_dev == z_dev) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  TRY(reset_error_word(h, s));
  return enqueue_vcycle(h, r_dev, z_dev, s, nullptr);
}

int hpcg_mg_stage(hpcg_handle h, int level, int stage, const double *r0_dev, double *z0_dev, void *stream) {
  if (!h || level < 0 || level >= h->levels) return HPCG_ERR_INVALID_ARG;
  if (stage != HPCG_STAGE_PRE && stage != HPCG_STAGE_REFINE && stage != HPCG_STAGE_POST) return HPCG_ERR_INVALID_ARG;
  if (stage != HPCG_STAGE_PRE && level == h->levels - 1) return HPCG_ERR_INVALID_ARG;  // the coarsest level has no coarser one
  if (level == 0 && (!r0_dev || !z0_dev || (const void *)r0_dev == (const void *)z0_dev)) return HPCG_ERR_INVALID_ARG;
  if (level == 0 && vstore_of(h) == VS_BFP && ((reinterpret_cast<uintptr_t>(r0_dev) | reinterpret_cast<uintptr_t>(z0_dev)) & 15) != 0)
    return HPCG_ERR_INVALID_ARG;  // hpcg_mg_vcycle would take the FP64-storage path for these
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  TRY(reset_error_word(h, s));
  return enqueue_stage(h, level, stage, r0_dev, z0_dev, s);
}

int hpcg_get_level_vectors(hpcg_handle h, int level, double *r_dev, double *z_dev, void *stream) {
  if (!h || level < 0 || level >= h->levels || (r_dev && r_dev == z_dev)) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  return level_vectors(h, level, r_dev, z_dev, true, (cudaStream_t)stream);
}

int hpcg_set_level_vectors(hpcg_handle h, int level, const double *r_dev, const double *z_dev, void *stream) {
  if (!h || level < 0 || level >= h->levels || (r_dev && r_dev == z_dev)) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  return level_vectors(h, level, const_cast<double *>(r_dev), const_cast<double *>(z_dev), false, (cudaStream_t)stream);
}

int hpcg_dot(hpcg_handle h, long n, const double *a_dev, const double *b_dev, double *out_dev, void *stream) {
  if (!h || !out_dev || n < 0 || (n > 0 && (!a_dev || !b_dev))) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  launch_k(k_dot_raw, kRawDotBlocks, kRedThreads, 0, s, n, a_dev, b_dev, h->part);
  CKL("k_dot_raw");
  launch_k(k_sum_raw, 1, kRedThreads, 0, s, kRawDotBlocks, h->part, out_dev);
  CKL("k_sum_raw");
  return HPCG_OK;
}

int hpcg_waxpby(hpcg_handle h, long n, double alpha, const double *x_dev, double beta, const double *y_dev, double *w_dev,
                void *stream) {
  if (!h || n < 0) return HPCG_ERR_INVALID_ARG;
  if (n == 0) return HPCG_OK;
  if (!x_dev || !y_dev || !w_dev) return HPCG_ERR_INVALID_ARG;
  launch_k(k_waxpby, grid_for(n), 256, 0, (cudaStream_t)stream, n, alpha, x_dev, beta, y_dev, w_dev);
  CKL("k_waxpby");
  return HPCG_OK;
}

int hpcg_pcg_solve(hpcg_handle h, const double *b_dev, double *x_dev, int max_iters, double rel_tol, hpcg_stats *stats,
                   void *stream) {
  if (!h || !b_dev || !x_dev || h->batch) return h && h->batch ? HPCG_ERR_UNSUPPORTED : HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  return run_pcg(h, b_dev, x_dev, max_iters, rel_tol, stats, s);
}

int hpcg_pcg_solve_multi(hpcg_handle h, int nrhs, const double *B_dev, double *X_dev, int max_iters, double rel_tol,
                         hpcg_stats *stats, void *stream) {
  if (!h || !B_dev || !X_dev || nrhs < 1 || nrhs > 64) return HPCG_ERR_INVALID_ARG;
  if (h->batch) return HPCG_ERR_UNSUPPORTED;
  if (nrhs > h->opt.max_rhs) return HPCG_ERR_NO_WORKSPACE;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  if (h->has_kappa) return HPCG_ERR_UNSUPPORTED;  // the copies carry no diagonal field
  if (!h->multi || h->multi_R != nrhs) {
    if (h->multi) hpcg_destroy(h->multi);
    h->multi = nullptr;
    std::vector<int> rep;
    const Inst &g = h->lv[0].inst[0];
    for (int k = 0; k < nrhs; ++k) rep.insert(rep.end(), {g.nx, g.ny, g.nz});
    hpcg_options o = h->opt;
    o.max_rhs = 0;
    hpcg_handle m = nullptr;
    TRY(make_handle(&o, rep, 1, &m));
    int rc = bind(m, h->ws + h->o_multi, h->multi_bytes, false);
    if (rc != HPCG_OK) {
      delete m;
      return rc;
    }
    h->multi = m;
    h->multi_R = nrhs;
  }
  std::lock_guard<std::mutex> lk2(h->multi->mu);
  TRY(ensure_ready(h->multi, s));
  // the [nrhs][n] arrays are exactly the batch's concatenated vectors
  return run_pcg(h->multi, B_dev, X_dev, max_iters, rel_tol, stats, s);
}

int hpcg_pcg_solve_batch(hpcg_handle h, const double *b_dev, double *x_dev, int max_iters, double rel_tol, hpcg_stats *stats,
                         void *stream) {
  if (!h || !b_dev || !x_dev) return HPCG_ERR_INVALID_ARG;
  if (!h->batch) return HPCG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  return run_pcg(h, b_dev, x_dev, max_iters, rel_tol, stats, s);
}

int hpcg_pcg_backward(hpcg_handle h, const double *x_dev, const double *grad_x_dev, double *grad_b_dev, double *grad_kappa_dev,
                      int max_iters, double rel_tol, hpcg_stats *stats, void *stream) {
  if (!h || !x_dev || !grad_x_dev || !grad_b_dev) return HPCG_ERR_INVALID_ARG;
  if (grad_b_dev == x_dev || grad_b_dev == grad_x_dev) return HPCG_ERR_INVALID_ARG;
  if (h->batch) return HPCG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  TRY(ensure_ready(h, s));
  const long n = h->lv[0].n;
  CK(cudaMemsetAsync(grad_b_dev, 0, sizeof(double) * n, s));  // lambda_0 = 0
  int rc = run_pcg(h, grad_x_dev, grad_b_dev, max_iters, rel_tol, stats, s);  // A lambda = grad_x
  if (rc != HPCG_OK && rc != HPCG_ERR_NOT_CONVERGED) return rc;
  if (grad_kappa_dev) {
    launch_k(k_grad_kappa, grid_for(n), 256, 0, s, n, grad_b_dev, x_dev, grad_kappa_dev);
    CKL("k_grad_kappa");
  }
  return rc;
}

const char *hpcg_strerror(int status) {
  switch (status) {
    case HPCG_OK: return "ok";
    case HPCG_ERR_INVALID_ARG: return "invalid argument";
    case HPCG_ERR_CUDA: return "CUDA error";
    case HPCG_ERR_BREAKDOWN: return "CG breakdown (p.Ap <= 0 or non-finite scalar)";
    case HPCG_ERR_NOT_CONVERGED: return "tolerance not reached within max_iters";
    case HPCG_ERR_TIMEOUT: return "bounded device wait timed out";
    case HPCG_ERR_NO_WORKSPACE: return "workspace too small";
    case HPCG_ERR_OUT_OF_MEMORY: return "device allocation failed";
    case HPCG_ERR_UNSUPPORTED: return "unsupported for this handle";
    default: return "unknown status";
  }
}

const char *hpcg_last_cuda_error(void) { return g_last_cuda_error; }

int hpcg_bounds_status(long long *count_host, long long *first_host, int reset) {
  if (!count_host || !first_host) return HPCG_ERR_INVALID_ARG;
#ifdef HPCG_BOUNDS_CHECK
  BoundsWord w;
  CK(cudaMemcpyFromSymbol(&w, g_bounds, sizeof(w)));
  *count_host = (long long)w.count;
  first_host[0] = w.first ? (long long)((w.first - 1) >> 40) : -1;                 // source line of the first violation
  first_host[1] = w.first ? (long long)((w.first - 1) & ((1ULL << 40) - 1)) : -1;  // its index (low 40 bits)
  if (reset) {
    const BoundsWord zero = {0, 0};
    CK(cudaMemcpyToSymbol(g_bounds, &zero, sizeof(zero)));
  }
  return HPCG_OK;
#else
  (void)reset;
  *count_host = 0;
  first_host[0] = first_host[1] = -1;
  return HPCG_ERR_UNSUPPORTED;
#endif
}
long hpcg_launch_count(void) { return g_launches.load(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free V-cycle.
//
// Some callers cannot allocate device memory at the point where they need a
// preconditioner application: code running while a CUDA graph is being
// captured under a strict allocator, plug-ins living inside a host
// application that owns every device allocation, or real-time loops that
// forbid allocation after start-up.  hpcg_mg_vcycle_noalloc serves them: it
// takes only the input r and the output z, and keeps everything else (the
// level tables and the coarse-level vectors r_l, z_l of levels 1..L-1) in the
// fixed device array below, which every GPU that loads this library holds
// until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HPCG_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name only stands for the symbol, so its device address is looked up once per
// device, with that device current, by cudaGetSymbolAddress.
static void *g_noalloc_base[64];
static std::mutex g_noalloc_mu;

static int noalloc_base(void **out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return HPCG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void *p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_base[dev] = p;
  }
  *out = g_noalloc_base[dev];
  return HPCG_OK;
}

// Writes the one-instance level tables of an nx x ny x nz hierarchy.
__global__ void k_noalloc_tables(int nx, int ny, int nz, int levels, Inst *__restrict__ tabs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int l = 0; l < levels; ++l) {
    Inst g;
    g.nx = nx >> l;
    g.ny = ny >> l;
    g.nz = nz >> l;
    g.n = (long)g.nx * g.ny * g.nz;
    g.off = 0;
    g.blk_full = 0;
    g.blk_half = 0;
    g.blk_red = 0;
    g.blk_row = g.nrow = g.blk_line = g.nline = 0;
    long b = (g.n + (long)kRedThreads * kRedItems - 1) / ((long)kRedThreads * kRedItems);
    g.nred = (int)(b < 1 ? 1 : (b > kMaxRedBlocksPerInst ? kMaxRedBlocksPerInst : b));
    g.poff = 0;
    tabs[l] = g;
  }
}

// The array's layout for one hierarchy: the level tables, then r_l and z_l of
// every coarse level (byte offsets); returns the bytes used.
static size_t noalloc_layout(int nx, int ny, int nz, int levels, size_t *off_r, size_t *off_z) {
  size_t need = align256(sizeof(Inst) * kMaxLevels);
  for (int l = 1; l < levels; ++l) {
    const size_t nl = (size_t)(nx >> l) * (size_t)(ny >> l) * (size_t)(nz >> l);
    off_r[l] = need;
    need = align256(need + sizeof(double) * nl);
    off_z[l] = need;
    need = align256(need + sizeof(double) * nl);
  }
  return need;
}

extern "C" int hpcg_mg_vcycle_noalloc(int nx, int ny, int nz, int levels, const double *r_dev, double *z_dev, void *stream) {
  if (!r_dev || !z_dev || r_dev == z_dev) return HPCG_ERR_INVALID_ARG;
  TRY(validate_dims(nx, ny, nz, levels));
  size_t off_r[kMaxLevels] = {0}, off_z[kMaxLevels] = {0};
  const size_t need = noalloc_layout(nx, ny, nz, levels, off_r, off_z);
  if (need > (size_t)HPCG_NOALLOC_SCRATCH_BYTES) return HPCG_ERR_NO_WORKSPACE;
  void *base_v = nullptr;
  TRY(noalloc_base(&base_v));
  char *base = (char *)base_v;
  cudaStream_t s = (cudaStream_t)stream;
  Inst *tabs = (Inst *)base;
  k_noalloc_tables<<<1, 32, 0, s>>>(nx, ny, nz, levels, tabs);
  CKL("k_noalloc_tables");
  double *rl[kMaxLevels], *zl[kMaxLevels];
  int nfull[kMaxLevels], nhalf[kMaxLevels], nred[kMaxLevels];
  for (int l = 0; l < levels; ++l) {
    const int a = nx >> l, b = ny >> l, c = nz >> l;
    nfull[l] = tiles_of(a, b, c);
    nhalf[l] = tiles_of(half_up(a), half_up(b), half_up(c));
    nred[l] = red_blocks((long)a * b * c);
    rl[l] = l == 0 ? const_cast<double *>(r_dev) : (double *)(base + off_r[l]);
    zl[l] = l == 0 ? z_dev : (double *)(base + off_z[l]);
  }
  // one symmetric smoother application: colours 0..7 then 6..0 (the repeat of
  // colour 7 returns the same bits and is left out, as in hpcg_mg_vcycle)
  static const int kSeq[15] = {0, 1, 2, 3, 4, 5, 6, 7, 6, 5, 4, 3, 2, 1, 0};
  const dim3 blk(kTileX, kTileY);
  for (int l = 0; l < levels; ++l) {
    k_zero_inst<double><<<nred[l], kRedThreads, 0, s>>>(tabs + l, 1, zl[l], nullptr);
    CKL("k_zero_inst");
    for (int k : kSeq) {
      k_gs_color<double><<<nhalf[l], blk, 0, s>>>(tabs + l, 1, k & 1, (k >> 1) & 1, (k >> 2) & 1, rl[l], zl[l], nullptr, nullptr);
      CKL("k_gs_color");
    }
    if (l == levels - 1) break;
    k_restrict_residual<double><<<nfull[l + 1], blk, 0, s>>>(tabs + l, tabs + l + 1, 1, rl[l], zl[l], rl[l + 1], nullptr, nullptr);
    CKL("k_restrict_residual");
  }
  for (int l = levels - 2; l >= 0; --l) {
    k_prolong_add<double><<<nfull[l + 1], blk, 0, s>>>(tabs + l, tabs + l + 1, 1, zl[l + 1], zl[l], nullptr);
    CKL("k_prolong_add");
    for (int k : kSeq) {
      k_gs_color<double><<<nhalf[l], blk, 0, s>>>(tabs + l, 1, k & 1, (k >> 1) & 1, (k >> 2) & 1, rl[l], zl[l], nullptr, nullptr);
      CKL("k_gs_color");
    }
  }
  return HPCG_OK;
}

// Copies r_l and z_l of coarse level `level` of the last allocation-free
// V-cycle on an nx x ny x nz hierarchy out of the array (device-to-device
// copies on `stream`, nothing allocated); for checking the coarse levels.
extern "C" int hpcg_noalloc_level_vectors(int nx, int ny, int nz, int levels, int level, double *r_dev, double *z_dev, void *stream) {
  TRY(validate_dims(nx, ny, nz, levels));
  if (level < 1 || level >= levels || (!r_dev && !z_dev)) return HPCG_ERR_INVALID_ARG;
  size_t off_r[kMaxLevels] = {0}, off_z[kMaxLevels] = {0};
  if (noalloc_layout(nx, ny, nz, levels, off_r, off_z) > (size_t)HPCG_NOALLOC_SCRATCH_BYTES) return HPCG_ERR_NO_WORKSPACE;
  void *base_v = nullptr;
  TRY(noalloc_base(&base_v));
  const char *base = (const char *)base_v;
  const size_t bytes = sizeof(double) * (size_t)(nx >> level) * (size_t)(ny >> level) * (size_t)(nz >> level);
  cudaStream_t s = (cudaStream_t)stream;
  if (r_dev) CK(cudaMemcpyAsync(r_dev, base + off_r[level], bytes, cudaMemcpyDeviceToDevice, s));
  if (z_dev) CK(cudaMemcpyAsync(z_dev, base + off_z[level], bytes, cudaMemcpyDeviceToDevice, s));
  return HPCG_OK;
}
