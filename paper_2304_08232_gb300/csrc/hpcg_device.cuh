// hpcg_device.cuh -- inline device helpers shared by the kernel files:
// matrix-free neighbour sums of the 27-point operator (Sections II-B/C) and
// deterministic block reductions.
#pragma once
#include "hpcg_internal.cuh"

namespace hpcg {

// Bounds-checking build (compiled with -DHPCG_BOUNDS_CHECK): before each group
// of global accesses, the kernels of the default FP64 path check the index
// range they are about to touch against the extent of its array (an
// instance's rows, its x-lines, the next level's rows), and on a miss count
// the violation, remember the first one (source line and index) in a device
// word and skip the access; nothing traps.  hpcg_bounds_status reads the
// word.  In the normal build HPCG_IN is the constant true and every check
// compiles away.
#ifdef HPCG_BOUNDS_CHECK
struct BoundsWord {
  unsigned long long count;
  unsigned long long first;  // (source line << 40) | (index & (2^40 - 1)), + 1 so that 0 means none
};
static __device__ BoundsWord g_bounds;  // one per translation unit (the kernels of hpcg_core.cu use this one)
static __device__ __noinline__ bool bounds_fail(long first, int line) {
  atomicAdd(&g_bounds.count, 1ULL);
  atomicCAS(&g_bounds.first, 0ULL, (((unsigned long long)line << 40) | ((unsigned long long)first & ((1ULL << 40) - 1))) + 1ULL);
  return false;
}
// [first, first + len) inside [lo, hi)?
static __device__ __forceinline__ bool bounds_ok(long first, long len, long lo, long hi, int line) {
  return (first >= lo && first + len <= hi) ? true : bounds_fail(first, line);
}
#define HPCG_IN(first, len, lo, hi) ::hpcg::bounds_ok((long)(first), (long)(len), (long)(lo), (long)(hi), __LINE__)
#else
#define HPCG_IN(first, len, lo, hi) true
#endif

// Programmatic dependent launch: wait until the preceding kernel has finished
// and its writes are visible.  Blocks signal their dependents implicitly when
// they exit, so the next kernel is launched as this one drains instead of
// after its completion is processed (an explicit early signal measured slower:
// it places the next grid's first wave while this one still runs).  Without
// the launch attribute: a no-op.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Sum of the 26 neighbours of (x,y,z) that lie inside the grid, in ascending
// column order.  v points at the grid's first row.
template <typename T>
__device__ __forceinline__ T nbr_sum26(const T *__restrict__ v, int x, int y, int z, int nx, int ny, int nz) {
  T s = T(0);
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
        s += __ldg(v + base + xx);
      }
    }
  }
  return s;
}

template <typename T>
__device__ __forceinline__ T diag_of(const T *__restrict__ kap, long gi) {
  return kap ? T(26) + kap[gi] : T(26);
}

template <typename T>
__device__ __forceinline__ T inv_diag_of(const T *__restrict__ invd, long gi) {
  return invd ? invd[gi] : T(1) / T(26);
}

constexpr unsigned kFull = 0xffffffffu;

// Exact 64-bit fixed point for sums of FP64 values (used by the line kernels
// of hpcg_fixed.cuh, hpcg_bfp.cuh and hpcg_spmv.cuh, and by the reductions
// below): q(v) = trunc(v * 2^(1080 - E)) for a value whose biased exponent is
// at most E, so |q| < 2^58 and 32 such terms sum below 2^63 exactly.
constexpr int kFxMinE = 64, kFxMaxE = 2000;

__device__ __forceinline__ int fx_exp(double v) { return (__double2hiint(v) >> 20) & 0x7FF; }

// q(v) for a value whose biased exponent is at most E (E in [kFxMinE, kFxMaxE]).
__device__ __forceinline__ long long fx_of(double v, int E) {
  const int hi = __double2hiint(v);
  const unsigned lo = (unsigned)__double2loint(v);
  const int e = (hi >> 20) & 0x7FF;
  const unsigned long long m = ((unsigned long long)((unsigned)(hi & 0xFFFFF) | 0x100000u) << 32) | lo;
  unsigned long long q;
  // |v| = m 2^(e-1075); q = m 2^(e-E+5) = (m << 5) >> (E - e); shifts of 64 or
  // more give 0 (zeros and denormals have e = 0 and E >= 64)
  asm("shr.b64 %0, %1, %2;" : "=l"(q) : "l"(m << 5), "r"((unsigned)(E - e)));
  const long long s = (long long)(hi >> 31);
  return ((long long)q ^ s) - s;
}

// q 2^(E-1080) as FP64, rounded to nearest (ties to even), built from the
// bits of q on the integer pipe: an int64 -> double conversion instruction
// occupies the FP64 pipe for several of its issue slots on this GPU.
// E in [kFxMinE, kFxMaxE] keeps the result a normal number.
__device__ __forceinline__ double fx_to_double(long long q, int E) {
  const unsigned long long sign = (unsigned long long)q & 0x8000000000000000ULL;
  const unsigned long long a = q < 0 ? 0ULL - (unsigned long long)q : (unsigned long long)q;  // |q| < 2^63
  const int lz = __clzll(a);                                  // >= 1 for a != 0
  const unsigned long long m = a << lz;                        // leading one at bit 63
  const unsigned long long mant = m >> 11;                     // 53 significant bits
  const unsigned long long rbit = (m >> 10) & 1ULL;            // first dropped bit
  const unsigned long long sticky = (m & 0x3FFULL) != 0ULL;    // any further dropped bit
  const unsigned long long up = rbit & (sticky | (mant & 1ULL));
  // |value| = m 2^(E - 1080 - lz); biased exponent of the leading one: E + 6 - lz.
  // A carry out of the mantissa rounding moves into the exponent field.
  const unsigned long long bits = ((unsigned long long)(E + 6 - lz) << 52) + (mant - (1ULL << 52)) + up;
  return a == 0ULL ? 0.0 : __longlong_as_double((long long)(bits | sign));
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Sum of one FP64 value per lane of a warp (the per-line partials of r.z and
// p.Ap), valid in lane 0, on the integer pipe: every value in fixed point at
// the warp's largest biased exponent E (|q| < 2^58, 32 terms below 2^63), an
// exact int64 tree, one rounding.  Each term loses under 2^-58 of the largest
// value, as close as an FP64 tree gets, and the result does not depend on
// the order of the additions.  It keeps the five FP64 adds per line off the
// narrow FP64 pipe (one FP64 CG iteration at 192^3: 1.56 M FP64-pipe warp
// instructions instead of about 1.75 M).  A warp holding huge or non-finite
// values (E > kFxMaxE) sums in FP64, so NaN and Inf propagate.
__device__ __forceinline__ double warp_sum_fx(double v) {
  const int e = warp_max(fx_exp(v));
  if (e > kFxMaxE) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
  }
  const int E = max(e, kFxMinE);
  long long q = fx_of(v, E);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q += __shfl_down_sync(kFull, q, o);
  return fx_to_double(q, E);
}

// Deterministic block sum (exact integer tree over each warp's lanes, warps
// added in a fixed order); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh) {
  v = warp_sum_fx(v);
  const int lane = threadIdx.x & 31;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
  if ((tid & 31) == 0) sh[warp] = v;
  (void)lane;
  __syncthreads();
  double s = 0.0;
  if (tid == 0)
    for (int w = 0; w < nwarps; ++w) s += sh[w];
  __syncthreads();
  return s;
}

// Fixed-order sum of partials[first .. first+cnt) inside one block; valid in
// thread 0.  Thread t sums elements t + k*blockDim in eight interleaved
// accumulators (independent load/add chains), combined in a fixed order.
__device__ __forceinline__ double sum_partials(const double *__restrict__ partials, int first, int cnt, double *sh) {
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 0.0;
  const int bd = blockDim.x;
  int k = threadIdx.x;
  for (; k + 7 * bd < cnt; k += 8 * bd) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] += partials[first + k + j * bd];
  }
#pragma unroll
  for (int j = 0; j < 7; ++j)
    if (k + j * bd < cnt) a[j] += partials[first + k + j * bd];
  return block_sum(((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])), sh);
}

enum FinKind { FIN_NORM0 = 0, FIN_RTZ = 1, FIN_PAP = 2, FIN_NORM = 3, FIN_OUT = 4 };

// CG scalar update of one instance from a finished reduction s (thread 0 only):
//  FIN_NORM0: normr0 = sqrt(s)            (start of the solve)
//  FIN_RTZ:   rtz' = s; beta = rtz'/rtz   (after z = M r)
//  FIN_PAP:   alpha = rtz / s             (after Ap = A p; breakdown check; x += alpha p pending)
//  FIN_NORM:  normr = sqrt(s); history; convergence and stall tests
// hist points at this instance's history row (nullable).
template <int Kind>
__device__ __forceinline__ void fin_apply(CgState &c, double s, double *hist) {
  if (Kind == FIN_NORM0) {
    c.normr0 = sqrt(s);
    c.normr = c.normr0;
    c.best = c.normr0;
    if (!(c.normr0 > 0.0) || !isfinite(c.normr0)) {
      c.done = 1;
      c.converged = (c.normr0 == 0.0);
      c.status = (c.normr0 == 0.0) ? HPCG_OK : HPCG_ERR_BREAKDOWN;
    }
  } else if (Kind == FIN_RTZ) {
    if (c.restart) {
      c.first = 1;
      c.restart = 0;
      c.restarts += 1;
      c.xpend = 0;  // applied before the residual was replaced (k_update_x_restart)
    }
    if (c.first) {
      c.beta = 0.0;
    } else {
      c.beta = s / c.rtz;
    }
    c.rtz = s;
    if (!isfinite(s)) {
      c.done = 1;
      c.status = HPCG_ERR_BREAKDOWN;
    }
  } else if (Kind == FIN_PAP) {
    c.pAp = s;
    if (!(s > 0.0) || !isfinite(s)) {
      c.done = 1;
      c.status = HPCG_ERR_BREAKDOWN;
      c.alpha = 0.0;
      c.xpend = 0;
    } else {
      c.alpha = c.rtz / s;
      c.xpend = 1;
    }
    c.first = 0;
  } else if (Kind == FIN_NORM) {
    c.normr = sqrt(s);
    const double rel = c.normr / c.normr0;
    if (hist && c.iter < kHistoryCap) hist[c.iter] = rel;
    c.iter += 1;
    if (!isfinite(rel)) {
      c.done = 1;
      c.status = HPCG_ERR_BREAKDOWN;
    } else if (c.tol > 0.0 && rel <= c.tol) {
      c.done = 1;
      c.converged = 1;
    } else if (c.iter >= c.max_iters) {
      c.done = 1;
    } else if (c.mixed) {
      // stall test of the mixed-precision outer loop: no 1% progress over the
      // best residual for 3 iterations -> replace r by b - A x next iteration
      if (c.normr < 0.99 * c.best) {
        c.best = c.normr;
        c.stall = 0;
      } else if (++c.stall >= 3) {
        c.restart = 1;
        c.stall = 0;
        c.best = c.normr;
      }
      if (c.restart_every > 0 && c.iter % c.restart_every == 0) c.restart = 1;  // periodic replacement
    }
  }
}

}  // namespace hpcg
