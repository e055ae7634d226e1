// hpcg_ell.cuh -- device code of the materialised (sliced-ELL) operator:
// the slot layout, the row kernels (SpMV, colour phase, injected residual,
// refinement) and the CG kernels with fixed-grid reductions.  Used by the
// whole-grid engine (hpcg_ell.cu) and the two-sub-domain engine
// (hpcg_split.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

namespace hpcg_ell {

constexpr int kEllW = 27;             // slots per row
constexpr int kSlice = 32;            // rows per slice
constexpr int kEllThreads = 256;      // threads per block of the row kernels
constexpr int kEllDotBlocks = 608;    // fixed grid of the dot products (4 per SM of 152), fixed summation order
constexpr int kEllMaxLevels = 8;

struct EllGeom {
  int nx, ny, nz;
  int sorted;       // 1: rows grouped by colour; 0: natural order
  long n;
  long cstart[9];   // sorted: rows of colour k at [cstart[k], cstart[k+1])
};

__host__ __device__ __forceinline__ int count_par(int n, int par) { return (n - par + 1) >> 1; }

// stored index of grid point (x, y, z)
__device__ __forceinline__ long ell_index(const EllGeom &g, int x, int y, int z) {
  if (!g.sorted) return x + (long)g.nx * (y + (long)g.ny * z);
  const int px = x & 1, py = y & 1, pz = z & 1;
  const long cx = count_par(g.nx, px), cy = count_par(g.ny, py);
  return g.cstart[px + 2 * py + 4 * pz] + (x >> 1) + cx * ((y >> 1) + cy * (long)(z >> 1));
}

// grid point of stored row p
__device__ __forceinline__ void ell_coords(const EllGeom &g, long p, int &x, int &y, int &z) {
  if (!g.sorted) {
    x = (int)(p % g.nx);
    y = (int)((p / g.nx) % g.ny);
    z = (int)(p / ((long)g.nx * g.ny));
    return;
  }
  int c = 0;
  while (c < 7 && p >= g.cstart[c + 1]) ++c;
  const int px = c & 1, py = (c >> 1) & 1, pz = c >> 2;
  const long cx = count_par(g.nx, px), cy = count_par(g.ny, py);
  const long k = p - g.cstart[c];
  x = 2 * (int)(k % cx) + px;
  y = 2 * (int)((k / cx) % cy) + py;
  z = 2 * (int)(k / (cx * cy)) + pz;
}

// address of slot s of stored row p
__device__ __forceinline__ long slot_of(long p, int s) { return ((p >> 5) * kEllW + s) * kSlice + (p & 31); }

// Stored operator values: FP64, or BF16 (the values 26, -1 and 0 are exact in
// BF16, so a BF16 matrix gives the same products as an FP64 one).  A BF16 value
// is widened to FP64 on the integer pipe by moving its sign, exponent and
// 7 mantissa bits into the FP64 fields (a conversion instruction would occupy
// the FP64 pipe, which the products already fill); this covers zero and the
// normal numbers, the values the operator stores.
__device__ __forceinline__ double ell_val(const double *p) { return __ldg(p); }
__device__ __forceinline__ double ell_val(const __nv_bfloat16 *p) {
  const unsigned int u = __ldg(reinterpret_cast<const unsigned short *>(p));
  const unsigned int e = (u >> 7) & 0xFFu;
  const unsigned long long bits = ((unsigned long long)(u >> 15) << 63) | ((unsigned long long)(e + 1023u - 127u) << 52) |
                                  ((unsigned long long)(u & 0x7Fu) << 45);
  return e == 0u ? 0.0 : __longlong_as_double((long long)bits);
}
__device__ __forceinline__ void ell_set(double *p, double v) { *p = v; }
__device__ __forceinline__ void ell_set(__nv_bfloat16 *p, double v) { *p = __float2bfloat16_rn((float)v); }

__device__ __forceinline__ long gtid() { return blockIdx.x * (long)blockDim.x + threadIdx.x; }

// One thread per stored row (padding rows of the last slice included): the
// row's slots, the diagonal and the natural index.
template <typename TV>
__global__ void k_ell_build(EllGeom g, long nrows_padded, int *__restrict__ col, TV *__restrict__ val, double *__restrict__ diag,
                            int *__restrict__ perm) {
  const long p = gtid();
  if (p >= nrows_padded) return;
  if (p >= g.n) {
    for (int s = 0; s < kEllW; ++s) {
      col[slot_of(p, s)] = 0;
      ell_set(val + slot_of(p, s), 0.0);
    }
    return;
  }
  int x, y, z;
  ell_coords(g, p, x, y, z);
  perm[p] = (int)(x + (long)g.nx * (y + (long)g.ny * z));
  diag[p] = 26.0;
  int s = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int zz = z + dz;
    if (zz < 0 || zz >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = y + dy;
      if (yy < 0 || yy >= g.ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx;
        if (xx < 0 || xx >= g.nx) continue;
        const bool self = dx == 0 && dy == 0 && dz == 0;
        col[slot_of(p, s)] = (int)ell_index(g, xx, yy, zz);
        ell_set(val + slot_of(p, s), self ? 26.0 : -1.0);
        ++s;
      }
    }
  }
  for (; s < kEllW; ++s) {
    col[slot_of(p, s)] = (int)p;
    ell_set(val + slot_of(p, s), 0.0);
  }
}

// f2c[pc]: stored fine row of the fine point (2 xc, 2 yc, 2 zc) injected into
// stored coarse row pc (Section II-F)
static __global__ void k_ell_f2c(EllGeom gf, EllGeom gc, int *__restrict__ f2c) {
  const long pc = gtid();
  if (pc >= gc.n) return;
  int x, y, z;
  ell_coords(gc, pc, x, y, z);
  f2c[pc] = (int)ell_index(gf, 2 * x, 2 * y, 2 * z);
}

// sum over the slots of row p of val * v[col]
template <bool EXACT, typename TV>
__device__ __forceinline__ double row_sum(long p, const int *__restrict__ col, const TV *__restrict__ val, const double *__restrict__ v) {
  const long base = ((p >> 5) * kEllW) * kSlice + (p & 31);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kEllW; ++k) {
    const double a = ell_val(val + base + k * kSlice);
    const double b = v[__ldg(col + base + k * kSlice)];
    s = EXACT ? __dadd_rn(s, __dmul_rn(a, b)) : fma(a, b, s);
  }
  return s;
}

template <bool EXACT, typename TV>
__global__ void __launch_bounds__(kEllThreads) k_ell_spmv(long n, const int *__restrict__ col, const TV *__restrict__ val,
                                                          const double *__restrict__ x, double *__restrict__ y) {
  const long p = gtid();
  if (p < n) y[p] = row_sum<EXACT>(p, col, val, x);
}

// One colour phase (Listings 2 and 3) over stored rows [p0, p1): rows of
// colour k (all of them when the rows are grouped; mask >= 0 tests the colour
// of each row in natural order).  Rows of one colour have no neighbour of
// their colour, so they update independently.
template <bool EXACT, typename TV>
__global__ void __launch_bounds__(kEllThreads) k_ell_gs(long p0, long p1, int mask, EllGeom g, const int *__restrict__ col,
                                                        const TV *__restrict__ val, const double *__restrict__ diag,
                                                        const double *__restrict__ r, double *__restrict__ z) {
  const long p = p0 + gtid();
  if (p >= p1) return;
  if (mask >= 0) {
    const int x = (int)(p % g.nx), y = (int)((p / g.nx) % g.ny), zz = (int)(p / ((long)g.nx * g.ny));
    if ((x & 1) + 2 * (y & 1) + 4 * (zz & 1) != mask) return;
  }
  const double s = row_sum<EXACT>(p, col, val, z);
  const double d = diag[p];
  const double v = EXACT ? __dadd_rn(__dsub_rn(r[p], s), __dmul_rn(z[p], d)) : fma(z[p], d, r[p] - s);
  z[p] = v / d;
}

// rc = injection of r - A z (Section II-F), only at the injected rows
template <bool EXACT, typename TV>
__global__ void __launch_bounds__(kEllThreads) k_ell_restrict(long nc, const int *__restrict__ f2c, const int *__restrict__ col,
                                                              const TV *__restrict__ val, const double *__restrict__ r,
                                                              const double *__restrict__ z, double *__restrict__ rc) {
  const long pc = gtid();
  if (pc >= nc) return;
  const long pf = f2c[pc];
  rc[pc] = EXACT ? __dsub_rn(r[pf], row_sum<true>(pf, col, val, z)) : r[pf] - row_sum<false>(pf, col, val, z);
}

// z[f2c] += zc (refinement, the transpose of injection)
static __global__ void __launch_bounds__(kEllThreads) k_ell_prolong(long nc, const int *__restrict__ f2c, const double *__restrict__ zc,
                                                             double *__restrict__ z) {
  const long pc = gtid();
  if (pc >= nc) return;
  const long pf = f2c[pc];
  z[pf] = __dadd_rn(z[pf], zc[pc]);
}

template <typename TV>
__global__ void k_ell_widen(long n, const TV *__restrict__ v, double *__restrict__ out) {
  const long i = gtid();
  if (i < n) out[i] = ell_val(v + i);
}

static __global__ void k_ell_fill(long n, double v, double *__restrict__ a) {
  const long i = gtid();
  if (i < n) a[i] = v;
}

// dst[p] = src[perm[p]] (natural -> stored) or dst[perm[p]] = src[p] (stored -> natural)
static __global__ void k_ell_permute(long n, int to_stored, const int *__restrict__ perm, const double *__restrict__ src, double *__restrict__ dst) {
  const long p = gtid();
  if (p >= n) return;
  if (to_stored)
    dst[p] = src[perm[p]];
  else
    dst[perm[p]] = src[p];
}

// ---------------------------------------------------------------------------
// CG on the stored order: scalars stay on the device.
struct EllCg {
  double rtz, normr0, alpha, beta;
};

__device__ __forceinline__ double ell_block_sum(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  __syncthreads();
  return s;
}

// fixed-grid partial sums of a . b (one per block)
static __global__ void __launch_bounds__(kEllThreads) k_ell_dot(long n, const double *__restrict__ a, const double *__restrict__ b,
                                                         double *__restrict__ part) {
  __shared__ double sh[kEllThreads / 32];
  double s = 0.0;
  for (long i = gtid(); i < n; i += (long)gridDim.x * blockDim.x) s = fma(a[i], b[i], s);
  s = ell_block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

enum EllScalar { ES_NORM0 = 0, ES_RTZ_FIRST, ES_RTZ, ES_PAP, ES_NORM };

// one block: the partials in a fixed order, then the CG scalar of `kind`
// (cnt partials: kEllDotBlocks per sub-domain)
static __global__ void __launch_bounds__(kEllThreads) k_ell_scalar(int kind, const double *__restrict__ part, int cnt, EllCg *__restrict__ st,
                                                            double *__restrict__ hist, int k) {
  __shared__ double sh[kEllThreads / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) v += part[i];
  const double s = ell_block_sum(v, sh);
  if (threadIdx.x != 0) return;
  switch (kind) {
    case ES_NORM0: st->normr0 = sqrt(s); break;
    case ES_RTZ_FIRST: st->rtz = s; break;
    case ES_RTZ: st->beta = s / st->rtz; st->rtz = s; break;
    case ES_PAP: st->alpha = st->rtz / s; break;
    default: hist[k] = sqrt(s) / st->normr0; break;
  }
}

// w = a x + b y with host scalars
static __global__ void __launch_bounds__(kEllThreads) k_ell_axpby(long n, double a, const double *__restrict__ x, double b,
                                                           const double *__restrict__ y, double *__restrict__ w) {
  const long i = gtid();
  if (i < n) w[i] = __dadd_rn(__dmul_rn(a, x[i]), __dmul_rn(b, y[i]));
}

// p = z (first iteration) or z + beta p
static __global__ void __launch_bounds__(kEllThreads) k_ell_update_p(long n, int first, const double *__restrict__ z, double *__restrict__ p,
                                                              const EllCg *__restrict__ st) {
  const long i = gtid();
  if (i >= n) return;
  p[i] = first ? z[i] : __dadd_rn(z[i], __dmul_rn(st->beta, p[i]));
}

// x += alpha p; r -= alpha Ap
static __global__ void __launch_bounds__(kEllThreads) k_ell_update_xr(long n, const double *__restrict__ p, const double *__restrict__ ap,
                                                               double *__restrict__ x, double *__restrict__ r, const EllCg *__restrict__ st) {
  const long i = gtid();
  if (i >= n) return;
  const double alpha = st->alpha;
  x[i] = __dadd_rn(x[i], __dmul_rn(alpha, p[i]));
  r[i] = __dsub_rn(r[i], __dmul_rn(alpha, ap[i]));
}

static inline unsigned blocks_for(long n) { return (unsigned)((n + kEllThreads - 1) / kEllThreads); }

}  // namespace hpcg_ell
