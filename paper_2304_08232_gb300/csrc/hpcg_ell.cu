// hpcg_ell.cu -- the operator materialised as a sliced-ELL matrix whose rows
// are grouped by colour, P^T A P (Section III-A), with the MG-PCG of
// Listing 1 and Section II-C on it.
//
// The matrix-free kernels of the rest of the library find the rows of a
// colour by parity arithmetic and need no matrix.  This engine stores A the
// way a general sparse code would: 27 slots per row (8 to 27 used, the rest
// padding with value 0 and the row's own column), in slices of 32 rows laid
// out slot-major inside the slice so that a warp reads one slot of its 32
// rows with one coalesced load.  With colour grouping (the permutation P of
// Section III-A) the rows of colour k are the contiguous range
// [cstart[k], cstart[k+1]) and a colour phase reads a contiguous run of
// slices; in natural order a colour phase masks every row and touches every
// slice.  Both orders run the same per-row arithmetic, so they give the same
// bits after the permutation is undone.
//
// Row numbering inside colour k = (px, py, pz): the rows of that colour in
// increasing natural index, i.e. (xh, yh, zh) = (x >> 1, y >> 1, z >> 1) with
// index xh + cx (yh + cy zh), cx and cy the colour's counts along x and y.
// Slot order inside a row: the row's nonzeros in ascending natural column
// index, the order of the CRS rows of Section II-B.
//
// EXACT instances form each product and sum with separate IEEE operations
// (no fused multiply-add), from 0.0 in slot order, and the colour update as
// (r - s + z d) / d with the diagonal inside s (Listing 3); these match a
// plain sequential CRS evaluation bit for bit.  The default instances fuse
// the multiply-adds.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "hpcg.h"
#include "hpcg_ctx.h"
#include "hpcg_ell.cuh"

using namespace hpcg_ell;

// ---------------------------------------------------------------------------
struct EllLevel {
  EllGeom g;
  long nslices;
  int *col = nullptr;
  void *val = nullptr;  // double or __nv_bfloat16 slots (hpcg_ell_ctx::bf16)
  double *diag = nullptr;
  int *perm = nullptr;
  int *f2c = nullptr;   // to the next coarser level (all levels but the last)
  double *r = nullptr;  // level vectors of the coarse levels (stored order)
  double *z = nullptr;
};

struct hpcg_ell_ctx {
  int levels;
  int sorted;
  int exact;
  int bf16;  // operator values stored in BF16 (exact for 26, -1 and 0)
  EllLevel lv[kEllMaxLevels];
  // CG work vectors on level 0 (stored order) and scalars
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *ap = nullptr;
  double *part = nullptr, *hist = nullptr;
  EllCg *st = nullptr;
  int hist_cap = 0;
  size_t bytes = 0;
  std::vector<void *> allocs;
  std::mutex mu;
};

static int ell_alloc(hpcg_ell_ctx *h, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (sliced-ELL operator)");
  h->allocs.push_back(*p);
  h->bytes += bytes;
  return HPCG_OK;
}

static void ell_free(hpcg_ell_ctx *h) {
  for (void *p : h->allocs) cudaFree(p);
  h->allocs.clear();
}

static int ell_build(hpcg_ell_ctx *h, int nx, int ny, int nz) {
  for (int l = 0; l < h->levels; ++l) {
    EllLevel &L = h->lv[l];
    EllGeom &g = L.g;
    g.nx = nx >> l;
    g.ny = ny >> l;
    g.nz = nz >> l;
    g.sorted = h->sorted;
    g.n = (long)g.nx * g.ny * g.nz;
    g.cstart[0] = 0;
    for (int c = 0; c < 8; ++c) {
      const long cnt = h->sorted ? (long)count_par(g.nx, c & 1) * count_par(g.ny, (c >> 1) & 1) * count_par(g.nz, c >> 2) : 0;
      g.cstart[c + 1] = g.cstart[c] + cnt;
    }
    if (!h->sorted)
      for (int c = 0; c <= 8; ++c) g.cstart[c] = 0;
    L.nslices = (g.n + kSlice - 1) / kSlice;
    const size_t slots = (size_t)L.nslices * kEllW * kSlice;
    TRY(ell_alloc(h, (void **)&L.col, slots * sizeof(int)));
    TRY(ell_alloc(h, (void **)&L.val, slots * (h->bf16 ? sizeof(__nv_bfloat16) : sizeof(double))));
    TRY(ell_alloc(h, (void **)&L.diag, g.n * sizeof(double)));
    TRY(ell_alloc(h, (void **)&L.perm, g.n * sizeof(int)));
    if (l > 0) {
      TRY(ell_alloc(h, (void **)&L.r, g.n * sizeof(double)));
      TRY(ell_alloc(h, (void **)&L.z, g.n * sizeof(double)));
    }
    const long rows = L.nslices * kSlice;
    if (h->bf16)
      k_ell_build<__nv_bfloat16><<<blocks_for(rows), kEllThreads>>>(g, rows, L.col, (__nv_bfloat16 *)L.val, L.diag, L.perm);
    else
      k_ell_build<double><<<blocks_for(rows), kEllThreads>>>(g, rows, L.col, (double *)L.val, L.diag, L.perm);
    CKL("k_ell_build");
  }
  for (int l = 0; l + 1 < h->levels; ++l) {
    EllLevel &L = h->lv[l];
    const EllGeom &gc = h->lv[l + 1].g;
    TRY(ell_alloc(h, (void **)&L.f2c, gc.n * sizeof(int)));
    k_ell_f2c<<<blocks_for(gc.n), kEllThreads>>>(L.g, gc, L.f2c);
    CKL("k_ell_f2c");
  }
  const long n = h->lv[0].g.n;
  for (double **v : {&h->b, &h->x, &h->r, &h->z, &h->p, &h->ap}) TRY(ell_alloc(h, (void **)v, n * sizeof(double)));
  TRY(ell_alloc(h, (void **)&h->part, kEllDotBlocks * sizeof(double)));
  TRY(ell_alloc(h, (void **)&h->st, sizeof(EllCg)));
  CK(cudaDeviceSynchronize());
  return HPCG_OK;
}

// ---------------------------------------------------------------------------
// enqueue helpers (stored order)

// Calls f with the (EXACT, value type) instance the handle uses:
// f(std::integral_constant<bool, EXACT>, (const TV *)values).
template <typename F>
static void ell_dispatch(const hpcg_ell_ctx *h, const void *val, F &&f) {
  if (h->bf16) {
    if (h->exact)
      f(std::true_type{}, (const __nv_bfloat16 *)val);
    else
      f(std::false_type{}, (const __nv_bfloat16 *)val);
  } else {
    if (h->exact)
      f(std::true_type{}, (const double *)val);
    else
      f(std::false_type{}, (const double *)val);
  }
}
static int ell_spmv(hpcg_ell_ctx *h, int l, const double *x, double *y, cudaStream_t s) {
  const EllLevel &L = h->lv[l];
  ell_dispatch(h, L.val, [&](auto ex, auto val) {
    k_ell_spmv<decltype(ex)::value><<<blocks_for(L.g.n), kEllThreads, 0, s>>>(L.g.n, L.col, val, x, y);
  });
  CKL("k_ell_spmv");
  return HPCG_OK;
}

static int ell_colour(hpcg_ell_ctx *h, int l, int k, const double *r, double *z, cudaStream_t s) {
  const EllLevel &L = h->lv[l];
  long p0 = 0, p1 = L.g.n;
  int mask = k;
  if (h->sorted) {
    p0 = L.g.cstart[k];
    p1 = L.g.cstart[k + 1];
    mask = -1;
  }
  if (p1 <= p0) return HPCG_OK;
  ell_dispatch(h, L.val, [&](auto ex, auto val) {
    k_ell_gs<decltype(ex)::value><<<blocks_for(p1 - p0), kEllThreads, 0, s>>>(p0, p1, mask, L.g, L.col, val, L.diag, r, z);
  });
  CKL("k_ell_gs");
  return HPCG_OK;
}

// one symmetric smoother application: colours 0..7 then 7..0
static int ell_smoother(hpcg_ell_ctx *h, int l, const double *r, double *z, cudaStream_t s) {
  for (int k = 0; k < 8; ++k) TRY(ell_colour(h, l, k, r, z, s));
  for (int k = 7; k >= 0; --k) TRY(ell_colour(h, l, k, r, z, s));
  return HPCG_OK;
}

static int ell_fill(long n, double v, double *a, cudaStream_t s) {
  if (n <= 0) return HPCG_OK;
  k_ell_fill<<<blocks_for(n), kEllThreads, 0, s>>>(n, v, a);
  CKL("k_ell_fill");
  return HPCG_OK;
}

// Listing 1 from level l: z <- 0, pre-smoother, and on a level with a coarser
// one the injected residual, the coarse solve, refinement and post-smoother
static int ell_mg(hpcg_ell_ctx *h, int l, const double *r, double *z, cudaStream_t s) {
  const EllLevel &L = h->lv[l];
  TRY(ell_fill(L.g.n, 0.0, z, s));
  TRY(ell_smoother(h, l, r, z, s));
  if (l == h->levels - 1) return HPCG_OK;
  EllLevel &C = h->lv[l + 1];
  ell_dispatch(h, L.val, [&](auto ex, auto val) {
    k_ell_restrict<decltype(ex)::value><<<blocks_for(C.g.n), kEllThreads, 0, s>>>(C.g.n, L.f2c, L.col, val, r, z, C.r);
  });
  CKL("k_ell_restrict");
  TRY(ell_mg(h, l + 1, C.r, C.z, s));
  k_ell_prolong<<<blocks_for(C.g.n), kEllThreads, 0, s>>>(C.g.n, L.f2c, C.z, z);
  CKL("k_ell_prolong");
  TRY(ell_smoother(h, l, r, z, s));
  return HPCG_OK;
}

static int ell_dot(hpcg_ell_ctx *h, const double *a, const double *b, int kind, int k, cudaStream_t s) {
  const long n = h->lv[0].g.n;
  k_ell_dot<<<kEllDotBlocks, kEllThreads, 0, s>>>(n, a, b, h->part);
  CKL("k_ell_dot");
  k_ell_scalar<<<1, kEllThreads, 0, s>>>(kind, h->part, kEllDotBlocks, h->st, h->hist, k);
  CKL("k_ell_scalar");
  return HPCG_OK;
}

static int ell_check_level(const hpcg_ell_ctx *h, int l) { return (l < 0 || l >= h->levels) ? HPCG_ERR_INVALID_ARG : HPCG_OK; }

// ---------------------------------------------------------------------------
// C ABI
extern "C" {

int hpcg_ell_setup(int nx, int ny, int nz, int levels, int colour_sorted, int exact, int bf16_values, hpcg_ell_handle *out) {
  if (!out) return HPCG_ERR_INVALID_ARG;
  *out = nullptr;
  if (levels < 1 || levels > kEllMaxLevels) return HPCG_ERR_INVALID_ARG;
  const int div = 1 << (levels - 1);
  if (nx < 2 || ny < 2 || nz < 2 || nx % div || ny % div || nz % div) return HPCG_ERR_INVALID_ARG;
  if (nx / div < 2 || ny / div < 2 || nz / div < 2) return HPCG_ERR_INVALID_ARG;
  if ((double)nx * ny * nz > 2.0e9) return HPCG_ERR_INVALID_ARG;  // int32 column indices
  hpcg_ell_ctx *h = new hpcg_ell_ctx();
  h->levels = levels;
  h->sorted = colour_sorted ? 1 : 0;
  h->exact = exact ? 1 : 0;
  h->bf16 = bf16_values ? 1 : 0;
  const int rc = ell_build(h, nx, ny, nz);
  if (rc != HPCG_OK) {
    ell_free(h);
    delete h;
    return rc;
  }
  *out = h;
  return HPCG_OK;
}

int hpcg_ell_destroy(hpcg_ell_handle h) {
  if (!h) return HPCG_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  ell_free(h);
  if (h->hist) cudaFree(h->hist);
  delete h;
  return HPCG_OK;
}

int hpcg_ell_bytes(hpcg_ell_handle h, size_t *bytes) {
  if (!h || !bytes) return HPCG_ERR_INVALID_ARG;
  *bytes = h->bytes;
  return HPCG_OK;
}

int hpcg_ell_level_info(hpcg_ell_handle h, int level, long *info_host) {
  if (!h || !info_host) return HPCG_ERR_INVALID_ARG;
  TRY(ell_check_level(h, level));
  const EllLevel &L = h->lv[level];
  info_host[0] = L.g.n;
  info_host[1] = L.nslices;
  for (int c = 0; c <= 8; ++c) info_host[2 + c] = L.g.cstart[c];
  return HPCG_OK;
}

int hpcg_ell_permutation(hpcg_ell_handle h, int level, int *perm_dev, void *stream) {
  if (!h || !perm_dev) return HPCG_ERR_INVALID_ARG;
  TRY(ell_check_level(h, level));
  const EllLevel &L = h->lv[level];
  CK(cudaMemcpyAsync(perm_dev, L.perm, L.g.n * sizeof(int), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return HPCG_OK;
}

int hpcg_ell_matrix(hpcg_ell_handle h, int level, int *col_dev, double *val_dev, void *stream) {
  if (!h || !col_dev || !val_dev) return HPCG_ERR_INVALID_ARG;
  TRY(ell_check_level(h, level));
  const EllLevel &L = h->lv[level];
  const size_t slots = (size_t)L.nslices * kEllW * kSlice;
  CK(cudaMemcpyAsync(col_dev, L.col, slots * sizeof(int), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  if (h->bf16) {
    k_ell_widen<__nv_bfloat16><<<blocks_for((long)slots), kEllThreads, 0, (cudaStream_t)stream>>>((long)slots, (const __nv_bfloat16 *)L.val,
                                                                                                   val_dev);
    CKL("k_ell_widen");
  } else {
    CK(cudaMemcpyAsync(val_dev, L.val, slots * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  }
  return HPCG_OK;
}

int hpcg_ell_permute(hpcg_ell_handle h, int level, int to_stored, const double *src_dev, double *dst_dev, void *stream) {
  if (!h || !src_dev || !dst_dev || src_dev == dst_dev) return HPCG_ERR_INVALID_ARG;
  TRY(ell_check_level(h, level));
  const EllLevel &L = h->lv[level];
  k_ell_permute<<<blocks_for(L.g.n), kEllThreads, 0, (cudaStream_t)stream>>>(L.g.n, to_stored ? 1 : 0, L.perm, src_dev, dst_dev);
  CKL("k_ell_permute");
  return HPCG_OK;
}

int hpcg_ell_spmv(hpcg_ell_handle h, int level, const double *x_dev, double *y_dev, void *stream) {
  if (!h || !x_dev || !y_dev || x_dev == y_dev) return HPCG_ERR_INVALID_ARG;
  TRY(ell_check_level(h, level));
  std::lock_guard<std::mutex> lk(h->mu);
  return ell_spmv(h, level, x_dev, y_dev, (cudaStream_t)stream);
}

int hpcg_ell_rbgs_color(hpcg_ell_handle h, int level, int color, const double *r_dev, double *z_dev, void *stream) {
  if (!h || !r_dev || !z_dev || color < 0 || color > 7) return HPCG_ERR_INVALID_ARG;
  TRY(ell_check_level(h, level));
  std::lock_guard<std::mutex> lk(h->mu);
  return ell_colour(h, level, color, r_dev, z_dev, (cudaStream_t)stream);
}

int hpcg_ell_rbgs(hpcg_ell_handle h, int level, const double *r_dev, double *z_dev, void *stream) {
  if (!h || !r_dev || !z_dev) return HPCG_ERR_INVALID_ARG;
  TRY(ell_check_level(h, level));
  std::lock_guard<std::mutex> lk(h->mu);
  return ell_smoother(h, level, r_dev, z_dev, (cudaStream_t)stream);
}

int hpcg_ell_mg_vcycle(hpcg_ell_handle h, const double *r_dev, double *z_dev, void *stream) {
  if (!h || !r_dev || !z_dev || r_dev == z_dev) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  return ell_mg(h, 0, r_dev, z_dev, (cudaStream_t)stream);
}

int hpcg_ell_pcg_solve(hpcg_ell_handle h, const double *b_dev, double *x_dev, int max_iters, double rel_tol, hpcg_stats *stats,
                       void *stream) {
  if (!h || !b_dev || !x_dev || max_iters < 0) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const EllLevel &L0 = h->lv[0];
  const long n = L0.g.n;
  if (max_iters > h->hist_cap) {
    if (h->hist) {
      cudaFree(h->hist);
      h->hist = nullptr;
    }
    CK(cudaMalloc(&h->hist, (size_t)(max_iters > 0 ? max_iters : 1) * sizeof(double)));
    h->hist_cap = max_iters;
  }
  const unsigned nb = blocks_for(n);
  // natural -> stored order; r0 = b - A x0
  k_ell_permute<<<nb, kEllThreads, 0, s>>>(n, 1, L0.perm, b_dev, h->b);
  CKL("k_ell_permute");
  k_ell_permute<<<nb, kEllThreads, 0, s>>>(n, 1, L0.perm, x_dev, h->x);
  CKL("k_ell_permute");
  TRY(ell_spmv(h, 0, h->x, h->ap, s));
  k_ell_axpby<<<nb, kEllThreads, 0, s>>>(n, 1.0, h->b, -1.0, h->ap, h->r);
  CKL("k_ell_axpby");
  TRY(ell_dot(h, h->r, h->r, ES_NORM0, 0, s));
  EllCg host_st;
  CK(cudaMemcpyAsync(&host_st, h->st, sizeof(EllCg), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int k = 0;
  bool converged = host_st.normr0 == 0.0;
  double rel = 0.0;
  if (!converged) {
    for (k = 1; k <= max_iters; ++k) {
      TRY(ell_mg(h, 0, h->r, h->z, s));
      TRY(ell_dot(h, h->r, h->z, k == 1 ? ES_RTZ_FIRST : ES_RTZ, 0, s));
      k_ell_update_p<<<nb, kEllThreads, 0, s>>>(n, k == 1, h->z, h->p, h->st);
      CKL("k_ell_update_p");
      TRY(ell_spmv(h, 0, h->p, h->ap, s));
      TRY(ell_dot(h, h->p, h->ap, ES_PAP, 0, s));
      k_ell_update_xr<<<nb, kEllThreads, 0, s>>>(n, h->p, h->ap, h->x, h->r, h->st);
      CKL("k_ell_update_xr");
      TRY(ell_dot(h, h->r, h->r, ES_NORM, k - 1, s));
      if (rel_tol > 0.0) {
        CK(cudaMemcpyAsync(&rel, h->hist + (k - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!(rel == rel)) break;  // NaN: breakdown
        if (rel <= rel_tol) {
          converged = true;
          break;
        }
      }
    }
    if (k > max_iters) k = max_iters;
  }
  k_ell_permute<<<nb, kEllThreads, 0, s>>>(n, 0, L0.perm, h->x, x_dev);
  CKL("k_ell_permute");
  std::vector<double> hist((size_t)(k > 0 ? k : 1), 0.0);
  if (k > 0) CK(cudaMemcpyAsync(hist.data(), h->hist, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  rel = k > 0 ? hist[k - 1] : 0.0;
  if (rel_tol > 0.0 && k > 0 && rel <= rel_tol) converged = true;
  int status = HPCG_OK;
  if (!(rel == rel)) status = HPCG_ERR_BREAKDOWN;
  else if (rel_tol > 0.0 && !converged) status = HPCG_ERR_NOT_CONVERGED;
  if (stats) {
    stats->iters = k;
    stats->restarts = 0;
    stats->converged = converged ? 1 : 0;
    stats->status = status;
    stats->rel_res = rel;
    if (stats->history && stats->history_cap > 0) {
      const int m = k < stats->history_cap ? k : stats->history_cap;
      for (int i = 0; i < m; ++i) stats->history[i] = hist[i];
    }
  }
  return status;
}

}  // extern "C"
