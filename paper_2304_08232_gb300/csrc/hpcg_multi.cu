// hpcg_multi.cu -- many right-hand sides on one grid in one solve
// (hpcg_pcg_solve_multi).
//
// Layout: the R systems share the grid, so their vectors are interleaved,
// v[i*R + k] for row i and right-hand side k.  Each neighbour access of the
// matrix-free 27-point stencil then reads R consecutive values, i.e. a warp
// reads whole 256-byte rows of the interleaved array.  Every kernel is the
// FP64 counterpart of a single-RHS kernel (same arithmetic per (row, rhs)),
// CG scalars live per right-hand side in CgState[R], and each right-hand side
// stops on its own: once converged its updates are frozen.
#include <cuda_runtime.h>
#include <string.h>

#include <vector>

#include "hpcg_ctx.h"
#include "hpcg_device.cuh"

namespace {

constexpr int kMThreads = 256;    // threads of a multi-RHS block: R x (256 / R)
constexpr int kMGrid = 1184;      // fixed grid (8 x 148) of the reductions and stencils: deterministic partials

struct MGeo {
  int nx, ny, nz;
  long n;
};

__device__ __forceinline__ double nbr_sum26_m(const double *__restrict__ v, int R, int k, int x, int y, int z, int nx, int ny, int nz) {
  double s = 0.0;
  const long sxy = (long)nx * ny;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    const int zz = z + dz;
    if (zz < 0 || zz >= nz) continue;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = y + dy;
      if (yy < 0 || yy >= ny) continue;
      const long base = (long)zz * sxy + (long)yy * nx;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx;
        if (xx < 0 || xx >= nx) continue;
        if (dx == 0 && dy == 0 && dz == 0) continue;
        s += __ldg(v + (base + xx) * R + k);
      }
    }
  }
  return s;
}

// per-RHS block reduction: thread t holds a value for rhs t % R; result for
// rhs k (< R) is written to out[k] by thread k; fixed order
__device__ __forceinline__ void block_sum_rhs(double v, int R, double *sh, double *out) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  if (t < R) {
    double s = 0.0;
    for (int m = t; m < (int)blockDim.x; m += R) s += sh[m];
    out[t] = s;
  }
  __syncthreads();
}

// y = A x (Mode 0) / y = b - A x (Mode 1); optional partials of x.y per rhs
template <int Mode>
__global__ void __launch_bounds__(kMThreads) km_spmv(MGeo g, int R, const double *__restrict__ x, const double *__restrict__ b,
                                                     double *__restrict__ y, double *__restrict__ partials) {
  __shared__ double sh[kMThreads];
  const int k = threadIdx.x % R;
  const int rpb = blockDim.x / R;
  double acc = 0.0;
  for (long row = (long)blockIdx.x * rpb + threadIdx.x / R; row < g.n; row += (long)gridDim.x * rpb) {
    const int xx = (int)(row % g.nx), yy = (int)((row / g.nx) % g.ny), zz = (int)(row / ((long)g.nx * g.ny));
    const long gi = row * R + k;
    const double xi = x[gi];
    const double ax = 26.0 * xi - nbr_sum26_m(x, R, k, xx, yy, zz, g.nx, g.ny, g.nz);
    const double out = Mode == 0 ? ax : b[gi] - ax;
    y[gi] = out;
    acc += xi * out;
  }
  if (partials) block_sum_rhs(acc, R, sh, partials + (long)blockIdx.x * R);
}

// one colour step of red-black Gauss-Seidel for every rhs
__global__ void __launch_bounds__(kMThreads) km_gs_color(MGeo g, int R, int px, int py, int pz, const double *__restrict__ r,
                                                         double *__restrict__ z) {
  const int k = threadIdx.x % R;
  const int rpb = blockDim.x / R;
  const int cx = (g.nx - px + 1) / 2, cy = (g.ny - py + 1) / 2, cz = (g.nz - pz + 1) / 2;
  const long cnt = (long)cx * cy * cz;
  for (long q = (long)blockIdx.x * rpb + threadIdx.x / R; q < cnt; q += (long)gridDim.x * rpb) {
    const int xx = 2 * (int)(q % cx) + px, yy = 2 * (int)((q / cx) % cy) + py, zz = 2 * (int)(q / ((long)cx * cy)) + pz;
    const long row = xx + (long)g.nx * (yy + (long)g.ny * zz);
    const double s = r[row * R + k] + nbr_sum26_m(z, R, k, xx, yy, zz, g.nx, g.ny, g.nz);
    z[row * R + k] = s * (1.0 / 26.0);
  }
}

// rc[c] = r[f(c)] - (A z)[f(c)] for every rhs
__global__ void __launch_bounds__(kMThreads) km_restrict(MGeo f, MGeo c, int R, const double *__restrict__ r,
                                                         const double *__restrict__ z, double *__restrict__ rc) {
  const int k = threadIdx.x % R;
  const int rpb = blockDim.x / R;
  for (long q = (long)blockIdx.x * rpb + threadIdx.x / R; q < c.n; q += (long)gridDim.x * rpb) {
    const int xc = (int)(q % c.nx), yc = (int)((q / c.nx) % c.ny), zc = (int)(q / ((long)c.nx * c.ny));
    const int xf = 2 * xc, yf = 2 * yc, zf = 2 * zc;
    const long rowf = xf + (long)f.nx * (yf + (long)f.ny * zf);
    const double az = 26.0 * z[rowf * R + k] - nbr_sum26_m(z, R, k, xf, yf, zf, f.nx, f.ny, f.nz);
    rc[q * R + k] = r[rowf * R + k] - az;
  }
}

// z[f(c)] += zc[c] for every rhs
__global__ void __launch_bounds__(kMThreads) km_prolong(MGeo f, MGeo c, int R, const double *__restrict__ zc, double *__restrict__ z) {
  const int k = threadIdx.x % R;
  const int rpb = blockDim.x / R;
  for (long q = (long)blockIdx.x * rpb + threadIdx.x / R; q < c.n; q += (long)gridDim.x * rpb) {
    const int xc = (int)(q % c.nx), yc = (int)((q / c.nx) % c.ny), zc_ = (int)(q / ((long)c.nx * c.ny));
    const long rowf = 2L * xc + (long)f.nx * (2L * yc + (long)f.ny * 2L * zc_);
    z[rowf * R + k] += zc[q * R + k];
  }
}

// per-rhs partials of a.b
__global__ void __launch_bounds__(kMThreads) km_dot(long n, int R, const double *__restrict__ a, const double *__restrict__ b,
                                                    double *__restrict__ partials) {
  __shared__ double sh[kMThreads];
  const int k = threadIdx.x % R;
  const int rpb = blockDim.x / R;
  double acc = 0.0;
  for (long row = (long)blockIdx.x * rpb + threadIdx.x / R; row < n; row += (long)gridDim.x * rpb) acc += a[row * R + k] * b[row * R + k];
  block_sum_rhs(acc, R, sh, partials + (long)blockIdx.x * R);
}

// one block per rhs: fixed-order sum of its partials, then the CG scalar update
template <int Kind>
__global__ void __launch_bounds__(kRedThreads) km_finalize(int R, int nblk, const double *__restrict__ partials, CgState *__restrict__ st,
                                                           double *__restrict__ hist) {
  __shared__ double sh[kRedThreads / 32];
  const int k = blockIdx.x;
  if (st[k].done) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partials[(long)b * R + k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) fin_apply<Kind>(st[k], s, hist + (long)k * kHistoryCap);
}

__global__ void __launch_bounds__(kMThreads) km_update_p(long n, int R, const double *__restrict__ zv, double *__restrict__ p,
                                                         const CgState *__restrict__ st) {
  const int k = threadIdx.x % R;
  const int rpb = blockDim.x / R;
  const CgState &c = st[k];
  if (c.done) return;
  const bool first = c.first;
  const double beta = c.beta;
  for (long row = (long)blockIdx.x * rpb + threadIdx.x / R; row < n; row += (long)gridDim.x * rpb) {
    const long gi = row * R + k;
    p[gi] = first ? zv[gi] : zv[gi] + beta * p[gi];
  }
}

__global__ void __launch_bounds__(kMThreads) km_update_xr(long n, int R, const double *__restrict__ p, const double *__restrict__ ap,
                                                          double *__restrict__ x, double *__restrict__ r, double *__restrict__ partials,
                                                          const CgState *__restrict__ st) {
  __shared__ double sh[kMThreads];
  const int k = threadIdx.x % R;
  const int rpb = blockDim.x / R;
  const CgState &c = st[k];
  double acc = 0.0;
  if (!c.done) {
    const double alpha = c.alpha;
    for (long row = (long)blockIdx.x * rpb + threadIdx.x / R; row < n; row += (long)gridDim.x * rpb) {
      const long gi = row * R + k;
      x[gi] = x[gi] + alpha * p[gi];
      const double rn = r[gi] - alpha * ap[gi];
      r[gi] = rn;
      acc += rn * rn;
    }
  }
  block_sum_rhs(acc, R, sh, partials + (long)blockIdx.x * R);
}

// dst[i*R + k] = src[k*n + i] and back, through a 32x33 shared tile
__global__ void km_interleave(long n, int R, const double *__restrict__ src, double *__restrict__ dst) {
  __shared__ double t[32][33];
  const long i0 = (long)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int k = k0 + j;
    const long i = i0 + threadIdx.x;
    t[j][threadIdx.x] = (k < R && i < n) ? src[(long)k * n + i] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const long i = i0 + j;
    const int k = k0 + threadIdx.x;
    if (k < R && i < n) dst[i * R + k] = t[threadIdx.x][j];
  }
}

__global__ void km_deinterleave(long n, int R, const double *__restrict__ src, double *__restrict__ dst) {
  __shared__ double t[32][33];
  const long i0 = (long)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const long i = i0 + j;
    const int k = k0 + threadIdx.x;
    t[j][threadIdx.x] = (k < R && i < n) ? src[i * R + k] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int k = k0 + j;
    const long i = i0 + threadIdx.x;
    if (k < R && i < n) dst[(long)k * n + i] = t[threadIdx.x][j];
  }
}

#define CKM(what)                                         \
  do {                                                    \
    g_launches.fetch_add(1, std::memory_order_relaxed);   \
    cudaError_t e_ = cudaGetLastError();                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);    \
  } while (0)

struct MultiBufs {
  double *X, *B, *r, *z, *p, *ap;
  double *lr[kMaxLevels], *lz[kMaxLevels];
  double *part;
  CgState *st;
  double *hist;
  MGeo geo[kMaxLevels];
  int levels, R;
};

static MultiBufs carve(hpcg_ctx *h, int R) {
  MultiBufs m{};
  char *base = h->ws + h->o_multi;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *p = base + off;
    off = align256(off + bytes);
    return p;
  };
  const long n0 = h->lv[0].n;
  m.X = (double *)take(sizeof(double) * n0 * R);
  m.B = (double *)take(sizeof(double) * n0 * R);
  m.r = (double *)take(sizeof(double) * n0 * R);
  m.z = (double *)take(sizeof(double) * n0 * R);
  m.p = (double *)take(sizeof(double) * n0 * R);
  m.ap = (double *)take(sizeof(double) * n0 * R);
  m.levels = h->levels;
  m.R = R;
  for (int l = 0; l < h->levels; ++l) {
    const Inst &g = h->lv[l].inst[0];
    m.geo[l] = MGeo{g.nx, g.ny, g.nz, g.n};
    if (l == 0) {
      m.lr[0] = m.r;
      m.lz[0] = m.z;
    } else {
      m.lr[l] = (double *)take(sizeof(double) * g.n * R);
      m.lz[l] = (double *)take(sizeof(double) * g.n * R);
    }
  }
  m.part = (double *)take(sizeof(double) * (size_t)kMGrid * R);
  m.st = (CgState *)take(sizeof(CgState) * R);
  m.hist = (double *)take(sizeof(double) * (size_t)kHistoryCap * R);
  return m;
}

static int mgrid(long rows, int R) {
  const int rpb = kMThreads / R;
  long b = (rows + rpb - 1) / rpb;
  if (b > kMGrid) b = kMGrid;
  return (int)(b < 1 ? 1 : b);
}

static int enqueue_vcycle_m(const MultiBufs &m, cudaStream_t s, int symmetric) {
  const int R = m.R, bt = (kMThreads / R) * R;
  std::vector<int> seq;
  for (int k = 0; k < 8; ++k) seq.push_back(k);
  if (symmetric)
    for (int k = 6; k >= 0; --k) seq.push_back(k);  // colour 7 repeated right after itself returns the same bits
  for (int l = 0; l < m.levels; ++l) {
    cudaMemsetAsync(m.lz[l], 0, sizeof(double) * m.geo[l].n * R, s);
    for (int k : seq) {
      km_gs_color<<<mgrid((m.geo[l].n + 7) / 8, R), bt, 0, s>>>(m.geo[l], R, k & 1, (k >> 1) & 1, (k >> 2) & 1, m.lr[l], m.lz[l]);
      CKM("km_gs_color");
    }
    if (l == m.levels - 1) break;
    km_restrict<<<mgrid(m.geo[l + 1].n, R), bt, 0, s>>>(m.geo[l], m.geo[l + 1], R, m.lr[l], m.lz[l], m.lr[l + 1]);
    CKM("km_restrict");
  }
  for (int l = m.levels - 2; l >= 0; --l) {
    km_prolong<<<mgrid(m.geo[l + 1].n, R), bt, 0, s>>>(m.geo[l], m.geo[l + 1], R, m.lz[l + 1], m.lz[l]);
    CKM("km_prolong");
    for (int k : seq) {
      km_gs_color<<<mgrid((m.geo[l].n + 7) / 8, R), bt, 0, s>>>(m.geo[l], R, k & 1, (k >> 1) & 1, (k >> 2) & 1, m.lr[l], m.lz[l]);
      CKM("km_gs_color");
    }
  }
  return HPCG_OK;
}

static int enqueue_iter_m(const MultiBufs &m, cudaStream_t s, int symmetric) {
  const int R = m.R, bt = (kMThreads / R) * R;
  const MGeo g = m.geo[0];
  const int G = mgrid(g.n, R);
  int rc = enqueue_vcycle_m(m, s, symmetric);
  if (rc != HPCG_OK) return rc;
  km_dot<<<G, bt, 0, s>>>(g.n, R, m.r, m.z, m.part);
  CKM("km_dot");
  km_finalize<FIN_RTZ><<<R, kRedThreads, 0, s>>>(R, G, m.part, m.st, m.hist);
  CKM("km_finalize<RTZ>");
  km_update_p<<<G, bt, 0, s>>>(g.n, R, m.z, m.p, m.st);
  CKM("km_update_p");
  km_spmv<0><<<G, bt, 0, s>>>(g, R, m.p, nullptr, m.ap, m.part);
  CKM("km_spmv");
  km_finalize<FIN_PAP><<<R, kRedThreads, 0, s>>>(R, G, m.part, m.st, m.hist);
  CKM("km_finalize<PAP>");
  km_update_xr<<<G, bt, 0, s>>>(g.n, R, m.p, m.ap, m.X, m.r, m.part, m.st);
  CKM("km_update_xr");
  km_finalize<FIN_NORM><<<R, kRedThreads, 0, s>>>(R, G, m.part, m.st, m.hist);
  CKM("km_finalize<NORM>");
  return HPCG_OK;
}

}  // namespace

extern "C" int hpcg_pcg_solve_multi(hpcg_handle h, int nrhs, const double *B_dev, double *X_dev, int max_iters, double rel_tol,
                                    hpcg_stats *stats, void *stream) {
  if (!h || !B_dev || !X_dev || nrhs < 1 || nrhs > 64) return HPCG_ERR_INVALID_ARG;
  if (h->batch) return HPCG_ERR_UNSUPPORTED;
  if (nrhs > h->opt.max_rhs) return HPCG_ERR_NO_WORKSPACE;
  if (max_iters < 0 || max_iters > kHistoryCap) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ready(h, s);
  if (rc != HPCG_OK) return rc;
  if (h->has_kappa) return HPCG_ERR_UNSUPPORTED;  // the multi-RHS kernels carry no diagonal field
  const int R = nrhs;
  MultiBufs m = carve(h, R);
  const long n = m.geo[0].n;
  const int bt = (kMThreads / R) * R;
  const int G = mgrid(n, R);
  // interleave the caller's [R][n] arrays
  dim3 tb(32, 8), tg((unsigned)((n + 31) / 32), (unsigned)((R + 31) / 32));
  km_interleave<<<tg, tb, 0, s>>>(n, R, B_dev, m.B);
  CKM("km_interleave");
  km_interleave<<<tg, tb, 0, s>>>(n, R, X_dev, m.X);
  CKM("km_interleave");
  std::vector<CgState> init(R);
  for (auto &c : init) {
    memset(&c, 0, sizeof(c));
    c.first = 1;
    c.tol = rel_tol;
    c.max_iters = max_iters;
  }
  if (cudaMemcpyAsync(m.st, init.data(), sizeof(CgState) * R, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "state upload");
  km_spmv<1><<<G, bt, 0, s>>>(m.geo[0], R, m.X, m.B, m.r, nullptr);  // r = B - A X
  CKM("km_spmv(residual)");
  km_dot<<<G, bt, 0, s>>>(n, R, m.r, m.r, m.part);
  CKM("km_dot");
  km_finalize<FIN_NORM0><<<R, kRedThreads, 0, s>>>(R, G, m.part, m.st, m.hist);
  CKM("km_finalize<NORM0>");
  // one CG iteration as a graph (cached per R)
  GraphCache &gc = h->g_multi;
  if (!(gc.exec && gc.key[0] == (const void *)(long)R)) {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    gc = GraphCache{};
    if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "capture stream");
    cudaGraph_t graph;
    const long before = g_launches.load();
    cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    rc = enqueue_iter_m(m, h->cap, h->opt.symmetric);
    e = cudaStreamEndCapture(h->cap, &graph);
    if (rc != HPCG_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    gc.kernels = g_launches.load() - before;
    g_launches.fetch_sub(gc.kernels);
    e = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    gc.key[0] = (const void *)(long)R;
  }
  const int every = h->opt.check_every > 0 ? h->opt.check_every : 1;
  std::vector<CgState> hs(R);
  for (int it = 0; it < max_iters; ++it) {
    cudaError_t e = cudaGraphLaunch(gc.exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    g_launches.fetch_add(gc.kernels);
    if (rel_tol > 0.0 && (it + 1) % every == 0) {
      if (cudaMemcpyAsync(hs.data(), m.st, sizeof(CgState) * R, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "state poll");
      bool all = true;
      for (auto &c : hs) all = all && c.done;
      if (all) break;
    }
  }
  km_deinterleave<<<tg, tb, 0, s>>>(n, R, m.X, X_dev);
  CKM("km_deinterleave");
  if (cudaMemcpyAsync(hs.data(), m.st, sizeof(CgState) * R, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "stats copy");
  int worst = HPCG_OK;
  for (int k = 0; k < R; ++k) {
    const CgState &c = hs[k];
    int st = c.status;
    if (st == HPCG_OK && rel_tol > 0.0 && !c.converged) st = HPCG_ERR_NOT_CONVERGED;
    if (stats) {
      hpcg_stats &o = stats[k];
      o.iters = c.iter;
      o.restarts = 0;
      o.converged = c.converged;
      o.status = st;
      o.rel_res = c.normr0 > 0 ? c.normr / c.normr0 : 0.0;
      if (o.history && o.history_cap > 0 && c.iter > 0) {
        const int mm = c.iter < o.history_cap ? c.iter : o.history_cap;
        if (cudaMemcpy(o.history, m.hist + (size_t)k * kHistoryCap, sizeof(double) * mm, cudaMemcpyDeviceToHost) != cudaSuccess)
          return cuda_fail(cudaGetLastError(), "history copy");
      }
    }
    if (st == HPCG_ERR_BREAKDOWN) worst = st;
    else if (st != HPCG_OK && worst == HPCG_OK) worst = st;
  }
  return worst;
}
