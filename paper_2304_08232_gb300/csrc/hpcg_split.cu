// hpcg_split.cu -- one grid split into two sub-domains along z, each with
// its own rows, its own copy of the neighbour's boundary plane (the halo) and
// colour-aware halo exchange, run on one GPU.
//
// The distributed layout of the reference implementation (the data
// distribution section of the paper) gives every node a box of the grid and
// the 2D halos of its neighbours; the multigrid smoother then exchanges,
// after each colour, only the halo values of that colour (the paper's
// description of the reference's colour-aware exchange).  Here the two boxes
// are the slabs z < nz/2 and z >= nz/2 of every level, each a sliced-ELL
// matrix over its own rows (grouped by colour, P^T A P) whose columns index
// [own rows | halo rows]; the halo rows are the neighbour's boundary plane,
// grouped by colour.  The "ranks" are launched one after the other on one
// stream, and an exchange is a gather kernel that reads the neighbour's
// vector (the copy an interconnect would make); nothing waits on anything.
//
// Exchanges:
//  - after colour phase k of a smoother: the halo rows of colour k;
//  - after refinement: colour 0 (the injected points have even x, y and z);
//  - before an SpMV (and of a vector entering a level call): the whole halo.
// Restriction and refinement stay inside a slab: the fine point (2xc, 2yc,
// 2zc) of a coarse point of slab d lies in fine slab d.
// Every row's arithmetic is that of hpcg_ell.cu with the same slot order
// (ascending natural column), so the level calls give the same bits as the
// whole-grid engine; only the dot products, summed per slab and then over the
// slabs, round differently.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "hpcg.h"
#include "hpcg_ctx.h"
#include "hpcg_ell.cuh"

using namespace hpcg_ell;

namespace {

constexpr int kDomains = 2;

// halo[h] = from[src[h]] for h in [0, cnt)
__global__ void __launch_bounds__(kEllThreads) k_split_exchange(long cnt, const int *__restrict__ src, const double *__restrict__ from,
                                                                double *__restrict__ halo) {
  const long h = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (h < cnt) halo[h] = from[src[h]];
}

// natural -> local (dst[p] = src[map[p]]) or local -> natural (dst[map[p]] = src[p])
__global__ void __launch_bounds__(kEllThreads) k_split_permute(long cnt, int to_local, const int *__restrict__ map,
                                                               const double *__restrict__ src, double *__restrict__ dst) {
  const long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (p >= cnt) return;
  if (to_local)
    dst[p] = src[map[p]];
  else
    dst[map[p]] = src[p];
}

struct SplitDom {
  int z0 = 0, z1 = 0;     // global z range [z0, z1)
  long nloc = 0, nhalo = 0;
  long nslices = 0;
  long cstart[9] = {};    // own rows of colour k: [cstart[k], cstart[k+1])
  long hstart[9] = {};    // halo rows of colour k: local [nloc + hstart[k], nloc + hstart[k+1])
  int *col = nullptr;     // slots (columns local: own rows, then halo rows)
  double *val = nullptr;
  double *diag = nullptr;
  int *perm = nullptr;    // own row -> natural index
  int *src = nullptr;     // halo row -> own row of the other slab
  int *f2c = nullptr;     // coarse own row -> fine own row (levels but the last)
  double *r = nullptr;    // level vectors: r [nloc], z [nloc + nhalo]
  double *z = nullptr;
  double *t = nullptr;    // level-call scratch [nloc + nhalo]
};

struct SplitLevel {
  int nx = 0, ny = 0, nz = 0;
  long n = 0;
  SplitDom d[kDomains];
};

inline unsigned nblk(long n) { return (unsigned)((n + kEllThreads - 1) / kEllThreads); }
inline int colour_of(int x, int y, int z) { return (x & 1) + 2 * (y & 1) + 4 * (z & 1); }

}  // namespace

struct hpcg_split_ctx {
  int levels = 0;
  int exact = 0;
  SplitLevel lv[kEllMaxLevels];
  double *b[kDomains] = {}, *x[kDomains] = {}, *r[kDomains] = {}, *z[kDomains] = {}, *p[kDomains] = {}, *ap[kDomains] = {};
  double *part = nullptr;
  EllCg *st = nullptr;
  double *hist = nullptr;
  int hist_cap = 0;
  long exchanged = 0;   // halo values copied since setup
  long exchanges = 0;   // exchange steps (one per colour step, refinement or full halo) since setup
  size_t bytes = 0;
  std::vector<void *> allocs;
  std::mutex mu;
};

static int sp_alloc(hpcg_split_ctx *h, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (split operator)");
  h->allocs.push_back(*p);
  h->bytes += bytes;
  return HPCG_OK;
}

template <typename T>
static int sp_upload(hpcg_split_ctx *h, T **dst, const std::vector<T> &v) {
  TRY(sp_alloc(h, (void **)dst, v.size() * sizeof(T)));
  if (!v.empty()) CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HPCG_OK;
}

// Host construction of one level: own and halo rows of both slabs, their
// matrices with local columns, the exchange sources and the injection maps.
static int sp_build_level(hpcg_split_ctx *h, int l, int nx, int ny, int nz) {
  SplitLevel &L = h->lv[l];
  L.nx = nx;
  L.ny = ny;
  L.nz = nz;
  L.n = (long)nx * ny * nz;
  std::vector<int> lmap[kDomains], hperm[kDomains];  // natural -> local index; halo row -> natural index
  for (int d = 0; d < kDomains; ++d) {
    SplitDom &D = L.d[d];
    D.z0 = d * nz / kDomains;
    D.z1 = (d + 1) * nz / kDomains;
    lmap[d].assign(L.n, -1);
    std::vector<int> perm;
    perm.reserve((size_t)nx * ny * (D.z1 - D.z0));
    for (int c = 0; c < 8; ++c) {  // own rows grouped by colour, natural order inside
      D.cstart[c] = (long)perm.size();
      for (int z = D.z0; z < D.z1; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x)
            if (colour_of(x, y, z) == c) {
              const long g = x + (long)nx * (y + (long)ny * z);
              lmap[d][g] = (int)perm.size();
              perm.push_back((int)g);
            }
    }
    D.cstart[8] = D.nloc = (long)perm.size();
    const int zh = d == 0 ? D.z1 : D.z0 - 1;  // the neighbour's boundary plane
    for (int c = 0; c < 8; ++c) {
      D.hstart[c] = (long)hperm[d].size();
      if (zh < 0 || zh >= nz) continue;
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
          if (colour_of(x, y, zh) == c) {
            const long g = x + (long)nx * (y + (long)ny * zh);
            lmap[d][g] = (int)(D.nloc + (long)hperm[d].size());
            hperm[d].push_back((int)g);
          }
    }
    D.hstart[8] = D.nhalo = (long)hperm[d].size();
    // matrix over own rows, columns in ascending natural index
    D.nslices = (D.nloc + kSlice - 1) / kSlice;
    const size_t slots = (size_t)D.nslices * kEllW * kSlice;
    std::vector<int> col(slots, 0);
    std::vector<double> val(slots, 0.0);
    for (long p = 0; p < D.nloc; ++p) {
      const long g = perm[p];
      const int x = (int)(g % nx), y = (int)((g / nx) % ny), z = (int)(g / ((long)nx * ny));
      int s = 0;
      for (int dz = -1; dz <= 1; ++dz) {
        const int zz = z + dz;
        if (zz < 0 || zz >= nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
          const int yy = y + dy;
          if (yy < 0 || yy >= ny) continue;
          for (int dx = -1; dx <= 1; ++dx) {
            const int xx = x + dx;
            if (xx < 0 || xx >= nx) continue;
            const long j = xx + (long)nx * (yy + (long)ny * zz);
            const int lj = lmap[d][j];
            if (lj < 0) return HPCG_ERR_INVALID_ARG;  // a neighbour outside the slab and its halo: cannot happen
            const size_t a = ((size_t)(p >> 5) * kEllW + s) * kSlice + (p & 31);
            col[a] = lj;
            val[a] = (dx == 0 && dy == 0 && dz == 0) ? 26.0 : -1.0;
            ++s;
          }
        }
      }
      for (; s < kEllW; ++s) col[((size_t)(p >> 5) * kEllW + s) * kSlice + (p & 31)] = (int)p;
    }
    TRY(sp_upload(h, &D.col, col));
    TRY(sp_upload(h, &D.val, val));
    TRY(sp_upload(h, &D.perm, perm));
    TRY(sp_upload(h, &D.diag, std::vector<double>(D.nloc, 26.0)));
    TRY(sp_alloc(h, (void **)&D.r, D.nloc * sizeof(double)));
    TRY(sp_alloc(h, (void **)&D.z, (D.nloc + D.nhalo) * sizeof(double)));
    TRY(sp_alloc(h, (void **)&D.t, (D.nloc + D.nhalo) * sizeof(double)));
  }
  // exchange sources, once both slabs are numbered: the neighbour's own row of each halo row
  for (int d = 0; d < kDomains; ++d) {
    SplitDom &D = L.d[d];
    const int o = 1 - d;
    std::vector<int> src((size_t)D.nhalo);
    for (long hh = 0; hh < D.nhalo; ++hh) {
      const long g = hperm[d][hh];
      const int lo = lmap[o][g];
      if (lo < 0 || lo >= L.d[o].nloc) return HPCG_ERR_INVALID_ARG;  // halo point not owned by the neighbour: cannot happen
      src[hh] = lo;
    }
    TRY(sp_upload(h, &D.src, src));
  }
  // injection maps of the finer level l-1 into this level, slab by slab
  if (l > 0) {
    SplitLevel &F = h->lv[l - 1];
    for (int d = 0; d < kDomains; ++d) {
      std::vector<int> cperm((size_t)L.d[d].nloc);
      CK(cudaMemcpy(cperm.data(), L.d[d].perm, cperm.size() * sizeof(int), cudaMemcpyDeviceToHost));
      std::vector<int> fperm((size_t)F.d[d].nloc);
      CK(cudaMemcpy(fperm.data(), F.d[d].perm, fperm.size() * sizeof(int), cudaMemcpyDeviceToHost));
      std::vector<int> floc((size_t)F.n, -1);
      for (long p = 0; p < F.d[d].nloc; ++p) floc[fperm[p]] = (int)p;
      std::vector<int> f2c(cperm.size());
      for (size_t pc = 0; pc < cperm.size(); ++pc) {
        const long g = cperm[pc];
        const int x = (int)(g % nx), y = (int)((g / nx) % ny), z = (int)(g / ((long)nx * ny));
        const long gf = 2 * x + (long)F.nx * (2 * y + (long)F.ny * 2 * z);
        if (floc[gf] < 0) return HPCG_ERR_INVALID_ARG;  // injected point outside the fine slab: cannot happen
        f2c[pc] = floc[gf];
      }
      TRY(sp_upload(h, &F.d[d].f2c, f2c));
    }
  }
  return HPCG_OK;
}

// ---------------------------------------------------------------------------
// enqueue helpers

// halo rows of colours [c0, c1) of every slab from its neighbour's vector;
// v[d] has nloc + nhalo entries
static int sp_exchange(hpcg_split_ctx *h, int l, double *const v[kDomains], int c0, int c1, cudaStream_t s) {
  SplitLevel &L = h->lv[l];
  for (int d = 0; d < kDomains; ++d) {
    const SplitDom &D = L.d[d];
    const long a = D.hstart[c0], b = D.hstart[c1];
    if (b <= a) continue;
    k_split_exchange<<<nblk(b - a), kEllThreads, 0, s>>>(b - a, D.src + a, v[1 - d], v[d] + D.nloc + a);
    CKL("k_split_exchange");
    h->exchanged += b - a;
  }
  h->exchanges += 1;
  return HPCG_OK;
}

static int sp_spmv(hpcg_split_ctx *h, int l, double *const x[kDomains], double *const y[kDomains], cudaStream_t s) {
  TRY(sp_exchange(h, l, x, 0, 8, s));
  for (int d = 0; d < kDomains; ++d) {
    const SplitDom &D = h->lv[l].d[d];
    if (h->exact)
      k_ell_spmv<true, double><<<nblk(D.nloc), kEllThreads, 0, s>>>(D.nloc, D.col, D.val, x[d], y[d]);
    else
      k_ell_spmv<false, double><<<nblk(D.nloc), kEllThreads, 0, s>>>(D.nloc, D.col, D.val, x[d], y[d]);
    CKL("k_ell_spmv");
  }
  return HPCG_OK;
}

// one symmetric smoother application; z's halo must be current on entry
static int sp_smoother(hpcg_split_ctx *h, int l, double *const r[kDomains], double *const z[kDomains], cudaStream_t s) {
  const EllGeom none = {};
  for (int it = 0; it < 16; ++it) {
    const int k = it < 8 ? it : 15 - it;
    for (int d = 0; d < kDomains; ++d) {
      const SplitDom &D = h->lv[l].d[d];
      const long p0 = D.cstart[k], p1 = D.cstart[k + 1];
      if (p1 <= p0) continue;
      if (h->exact)
        k_ell_gs<true, double><<<nblk(p1 - p0), kEllThreads, 0, s>>>(p0, p1, -1, none, D.col, D.val, D.diag, r[d], z[d]);
      else
        k_ell_gs<false, double><<<nblk(p1 - p0), kEllThreads, 0, s>>>(p0, p1, -1, none, D.col, D.val, D.diag, r[d], z[d]);
      CKL("k_ell_gs");
    }
    TRY(sp_exchange(h, l, z, k, k + 1, s));  // the values of colour k just updated
  }
  return HPCG_OK;
}

// Listing 1 from level l on both slabs
static int sp_mg(hpcg_split_ctx *h, int l, double *const r[kDomains], double *const z[kDomains], cudaStream_t s) {
  SplitLevel &L = h->lv[l];
  for (int d = 0; d < kDomains; ++d) {
    const long m = L.d[d].nloc + L.d[d].nhalo;
    k_ell_fill<<<nblk(m), kEllThreads, 0, s>>>(m, 0.0, z[d]);
    CKL("k_ell_fill");
  }
  TRY(sp_smoother(h, l, r, z, s));
  if (l == h->levels - 1) return HPCG_OK;
  SplitLevel &C = h->lv[l + 1];
  double *rc[kDomains], *zc[kDomains];
  for (int d = 0; d < kDomains; ++d) {
    const SplitDom &D = L.d[d];
    const long nc = C.d[d].nloc;
    rc[d] = C.d[d].r;
    zc[d] = C.d[d].z;
    if (h->exact)
      k_ell_restrict<true, double><<<nblk(nc), kEllThreads, 0, s>>>(nc, D.f2c, D.col, D.val, r[d], z[d], rc[d]);
    else
      k_ell_restrict<false, double><<<nblk(nc), kEllThreads, 0, s>>>(nc, D.f2c, D.col, D.val, r[d], z[d], rc[d]);
    CKL("k_ell_restrict");
  }
  TRY(sp_mg(h, l + 1, rc, zc, s));
  for (int d = 0; d < kDomains; ++d) {
    const long nc = C.d[d].nloc;
    k_ell_prolong<<<nblk(nc), kEllThreads, 0, s>>>(nc, L.d[d].f2c, zc[d], z[d]);
    CKL("k_ell_prolong");
  }
  TRY(sp_exchange(h, l, z, 0, 1, s));  // refinement changed only colour-0 points
  TRY(sp_smoother(h, l, r, z, s));
  return HPCG_OK;
}

// a . b over both slabs' own rows into the CG scalar `kind`
static int sp_dot(hpcg_split_ctx *h, double *const a[kDomains], double *const b[kDomains], int kind, int k, cudaStream_t s) {
  for (int d = 0; d < kDomains; ++d) {
    const long n = h->lv[0].d[d].nloc;
    k_ell_dot<<<kEllDotBlocks, kEllThreads, 0, s>>>(n, a[d], b[d], h->part + d * kEllDotBlocks);
    CKL("k_ell_dot");
  }
  k_ell_scalar<<<1, kEllThreads, 0, s>>>(kind, h->part, kDomains * kEllDotBlocks, h->st, h->hist, k);
  CKL("k_ell_scalar");
  return HPCG_OK;
}

static int sp_permute(hpcg_split_ctx *h, int l, int to_local, const double *nat_in, double *const loc[kDomains], double *nat_out,
                      cudaStream_t s) {
  for (int d = 0; d < kDomains; ++d) {
    const SplitDom &D = h->lv[l].d[d];
    if (to_local)
      k_split_permute<<<nblk(D.nloc), kEllThreads, 0, s>>>(D.nloc, 1, D.perm, nat_in, loc[d]);
    else
      k_split_permute<<<nblk(D.nloc), kEllThreads, 0, s>>>(D.nloc, 0, D.perm, loc[d], nat_out);
    CKL("k_split_permute");
  }
  return HPCG_OK;
}

static void sp_free(hpcg_split_ctx *h) {
  for (void *p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->hist) cudaFree(h->hist);
  h->hist = nullptr;
}

// ---------------------------------------------------------------------------
extern "C" {

int hpcg_split_setup(int nx, int ny, int nz, int levels, int exact, hpcg_split_handle *out) {
  if (!out) return HPCG_ERR_INVALID_ARG;
  *out = nullptr;
  if (levels < 1 || levels > kEllMaxLevels) return HPCG_ERR_INVALID_ARG;
  const int div = 1 << (levels - 1);
  if (nx < 2 || ny < 2 || nz < 2 || nx % div || ny % div || nz % (2 * div)) return HPCG_ERR_INVALID_ARG;
  if (nx / div < 2 || ny / div < 2 || nz / div < 2) return HPCG_ERR_INVALID_ARG;
  if ((double)nx * ny * nz > 2.0e9) return HPCG_ERR_INVALID_ARG;
  hpcg_split_ctx *h = new hpcg_split_ctx();
  h->levels = levels;
  h->exact = exact ? 1 : 0;
  int rc = HPCG_OK;
  for (int l = 0; l < levels && rc == HPCG_OK; ++l) rc = sp_build_level(h, l, nx >> l, ny >> l, nz >> l);
  for (int d = 0; d < kDomains && rc == HPCG_OK; ++d) {
    const long own = h->lv[0].d[d].nloc, all = own + h->lv[0].d[d].nhalo;
    for (auto v : {&h->b[d], &h->r[d], &h->ap[d]})
      if (rc == HPCG_OK) rc = sp_alloc(h, (void **)v, own * sizeof(double));
    for (auto v : {&h->x[d], &h->z[d], &h->p[d]})
      if (rc == HPCG_OK) rc = sp_alloc(h, (void **)v, all * sizeof(double));
  }
  if (rc == HPCG_OK) rc = sp_alloc(h, (void **)&h->part, kDomains * kEllDotBlocks * sizeof(double));
  if (rc == HPCG_OK) rc = sp_alloc(h, (void **)&h->st, sizeof(EllCg));
  if (rc != HPCG_OK) {
    sp_free(h);
    delete h;
    return rc;
  }
  *out = h;
  return HPCG_OK;
}

int hpcg_split_destroy(hpcg_split_handle h) {
  if (!h) return HPCG_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  sp_free(h);
  delete h;
  return HPCG_OK;
}

int hpcg_split_info(hpcg_split_handle h, int level, int domain, long *info_host) {
  if (!h || !info_host || level < 0 || level >= h->levels || domain < 0 || domain >= kDomains) return HPCG_ERR_INVALID_ARG;
  const SplitDom &D = h->lv[level].d[domain];
  info_host[0] = D.z0;
  info_host[1] = D.z1;
  info_host[2] = D.nloc;
  info_host[3] = D.nhalo;
  for (int c = 0; c <= 8; ++c) info_host[4 + c] = D.cstart[c];
  for (int c = 0; c <= 8; ++c) info_host[13 + c] = D.hstart[c];
  return HPCG_OK;
}

int hpcg_split_exchange_count(hpcg_split_handle h, long *values_host, long *steps_host) {
  if (!h || !values_host || !steps_host) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  *values_host = h->exchanged;
  *steps_host = h->exchanges;
  return HPCG_OK;
}

int hpcg_split_spmv(hpcg_split_handle h, int level, const double *x_dev, double *y_dev, void *stream) {
  if (!h || !x_dev || !y_dev || x_dev == y_dev || level < 0 || level >= h->levels) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  SplitLevel &L = h->lv[level];
  double *xl[kDomains] = {L.d[0].t, L.d[1].t}, *yl[kDomains] = {L.d[0].r, L.d[1].r};
  TRY(sp_permute(h, level, 1, x_dev, xl, nullptr, s));
  TRY(sp_spmv(h, level, xl, yl, s));
  return sp_permute(h, level, 0, nullptr, yl, y_dev, s);
}

int hpcg_split_rbgs(hpcg_split_handle h, int level, const double *r_dev, double *z_dev, void *stream) {
  if (!h || !r_dev || !z_dev || r_dev == z_dev || level < 0 || level >= h->levels) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  SplitLevel &L = h->lv[level];
  double *rl[kDomains] = {L.d[0].r, L.d[1].r}, *zl[kDomains] = {L.d[0].t, L.d[1].t};
  TRY(sp_permute(h, level, 1, r_dev, rl, nullptr, s));
  TRY(sp_permute(h, level, 1, z_dev, zl, nullptr, s));
  TRY(sp_exchange(h, level, zl, 0, 8, s));
  TRY(sp_smoother(h, level, rl, zl, s));
  return sp_permute(h, level, 0, nullptr, zl, z_dev, s);
}

int hpcg_split_mg_vcycle(hpcg_split_handle h, const double *r_dev, double *z_dev, void *stream) {
  if (!h || !r_dev || !z_dev || r_dev == z_dev) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  SplitLevel &L = h->lv[0];
  double *rl[kDomains] = {L.d[0].r, L.d[1].r}, *zl[kDomains] = {L.d[0].t, L.d[1].t};
  TRY(sp_permute(h, 0, 1, r_dev, rl, nullptr, s));
  TRY(sp_mg(h, 0, rl, zl, s));
  return sp_permute(h, 0, 0, nullptr, zl, z_dev, s);
}

int hpcg_split_pcg_solve(hpcg_split_handle h, const double *b_dev, double *x_dev, int max_iters, double rel_tol, hpcg_stats *stats,
                         void *stream) {
  if (!h || !b_dev || !x_dev || max_iters < 0) return HPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t s = (cudaStream_t)stream;
  if (max_iters > h->hist_cap) {
    if (h->hist) {
      cudaFree(h->hist);
      h->hist = nullptr;
    }
    CK(cudaMalloc(&h->hist, (size_t)(max_iters > 0 ? max_iters : 1) * sizeof(double)));
    h->hist_cap = max_iters;
  }
  double *const *b = h->b, *const *x = h->x, *const *r = h->r, *const *z = h->z, *const *p = h->p, *const *ap = h->ap;
  TRY(sp_permute(h, 0, 1, b_dev, b, nullptr, s));
  TRY(sp_permute(h, 0, 1, x_dev, x, nullptr, s));
  TRY(sp_spmv(h, 0, x, ap, s));  // exchanges x's halo first
  for (int d = 0; d < kDomains; ++d) {
    const long n = h->lv[0].d[d].nloc;
    k_ell_axpby<<<nblk(n), kEllThreads, 0, s>>>(n, 1.0, b[d], -1.0, ap[d], r[d]);
    CKL("k_ell_axpby");
  }
  TRY(sp_dot(h, r, r, ES_NORM0, 0, s));
  EllCg host_st;
  CK(cudaMemcpyAsync(&host_st, h->st, sizeof(EllCg), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int k = 0;
  bool converged = host_st.normr0 == 0.0;
  double rel = 0.0;
  if (!converged) {
    for (k = 1; k <= max_iters; ++k) {
      TRY(sp_mg(h, 0, r, z, s));
      TRY(sp_dot(h, r, z, k == 1 ? ES_RTZ_FIRST : ES_RTZ, 0, s));
      for (int d = 0; d < kDomains; ++d) {
        const long n = h->lv[0].d[d].nloc;
        k_ell_update_p<<<nblk(n), kEllThreads, 0, s>>>(n, k == 1, z[d], p[d], h->st);
        CKL("k_ell_update_p");
      }
      TRY(sp_spmv(h, 0, p, ap, s));  // exchanges p's halo first
      TRY(sp_dot(h, p, ap, ES_PAP, 0, s));
      for (int d = 0; d < kDomains; ++d) {
        const long n = h->lv[0].d[d].nloc;
        k_ell_update_xr<<<nblk(n), kEllThreads, 0, s>>>(n, p[d], ap[d], x[d], r[d], h->st);
        CKL("k_ell_update_xr");
      }
      TRY(sp_dot(h, r, r, ES_NORM, k - 1, s));
      if (rel_tol > 0.0) {
        CK(cudaMemcpyAsync(&rel, h->hist + (k - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!(rel == rel)) break;
        if (rel <= rel_tol) {
          converged = true;
          break;
        }
      }
    }
    if (k > max_iters) k = max_iters;
  }
  TRY(sp_permute(h, 0, 0, nullptr, x, x_dev, s));
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
