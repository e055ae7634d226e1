// hpcg_spmv.cuh -- the FP64 SpMV y = A x (Section II-C's spmv, matrix-free)
// with each plane's x-lines staged once per block in shared memory.
//
// A x = (27 + kappa) x - S, where S is the 27-point box sum of x (the operator
// is 26 + kappa on the diagonal and -1 on every neighbour).  S is summed
// exactly in 64-bit fixed point on the integer pipe, as in k_spmv_lines_fx,
// but every value is converted to fixed point once instead of once per warp
// that needs it: a block of lpc warps owns the x-lines y0 .. y0+lpc-1 and
// marches through its zc planes; at each plane step every warp loads its own
// line of the next plane (the first and last warp also the lines y0-1 and
// y0+lpc beside the block), takes the line's largest biased exponent e_L and
// stores q = trunc(v 2^(1080 - e_L)), |q| < 2^58, in shared memory.  A line's
// plane sum aligns the three staged lines y-1, y, y+1 to their largest
// exponent; the box sum adds three plane sums (z-1, z, z+1) at their largest
// exponent E and then three columns (x-1, x, x+1).  Shifts only shrink
// values, so the 27 terms stay below 2^58 at E and sum below 2^63 exactly.
// Without kappa, 27 x - S is formed at scale E + 1 and converted once; with
// kappa (27 + kappa) x - S is formed in FP64.  Every scale is a function of
// the line maxima alone, so the result does not depend on the launch shape.
// Each truncation or alignment drops less than one unit at its scale, so S is
// within a few units of 2^(E - 1080), a few 2^-58 of the largest term.
//
// Shared memory is a ring of four plane buffers (plane p in buffer
// (p - z0 + 1) mod 4).  While the block computes plane zz, the raw FP64 lines
// of plane zz + 2 are in flight into the buffer of plane zz - 2 (cp.async:
// each warp copies its own line, the first and last warp also the lines
// beside the block), the lines of plane zz + 1 have arrived and each warp
// converts its own line in place (its copies are its own, so a warp-level
// wait suffices), and plane zz's buffer still holds the own line's mantissas
// for 27 x.  One block barrier per plane step (__syncthreads_or, which also
// tells every warp whether any line converted in that step was huge or not
// finite) orders the conversions before the plane sums and every read of a
// buffer before its next fill.  A block that meets such a line finishes its
// planes with FP64 sums read from global memory, so NaN and Inf propagate.
#pragma once
#include "hpcg_bfp.cuh"

namespace hpcg {

constexpr int kSpmvMaxLpc = 8;  // lines (warps) per block: the launch-shape autotuner's largest

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Starts the copy of line yl of plane zp into a shared-memory slot (zeros
// outside the grid, stored directly); vec16: the line starts on a 16-byte
// boundary and has an even length, so it moves in 16-byte pieces.  The copies
// also fill L1 (.ca), where the own line's FP64 values are read again for the
// x . y partials.
template <int NC>
__device__ __forceinline__ void spmv_fetch_line(const double *__restrict__ xg, int nx, int ny, int nz, long sxy, int zp, int yl, int lane,
                                                bool vec16, long long *__restrict__ slot) {
  if (zp < 0 || zp >= nz || yl < 0 || yl >= ny || !HPCG_IN((long)zp * sxy + (long)yl * nx, nx, 0, (long)nz * sxy)) {
#pragma unroll
    for (int c = 0; c < NC; ++c) slot[lane + 32 * c] = 0;
    return;
  }
  const double *l = xg + (long)zp * sxy + (long)yl * nx;
  if (vec16) {
#pragma unroll
    for (int c = 0; c < (NC + 1) / 2; ++c) {
      const int xx = 2 * (lane + 32 * c);
      if (xx < nx) cp_async16(slot + xx, l + xx);
    }
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int xx = lane + 32 * c;
      if (xx < nx) cp_async8(slot + xx, l + xx);
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {  // the padding of the slot past the line's end reads as zero
    const int xx = lane + 32 * c;
    if (xx >= nx) slot[xx] = 0;
  }
}

// Converts the raw line in a slot in place to fixed point at the line's
// largest exponent (|q| < 2^58) and records that exponent.  Returns true for
// a line beyond the fixed-point range (the slot then holds zeros).
template <int NC>
__device__ __forceinline__ bool spmv_convert_line(long long *__restrict__ slot, int *__restrict__ se, int lane) {
  double v[NC];
  int e = kFxMinE;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    v[c] = __longlong_as_double(slot[lane + 32 * c]);
    e = max(e, fx_exp(v[c]));
  }
  e = warp_max(e);
  const bool bad = e > kFxMaxE;  // huge, Inf or NaN (biased exponent 2047)
#pragma unroll
  for (int c = 0; c < NC; ++c) slot[lane + 32 * c] = bad ? 0LL : fx_of(v[c], e);
  if (lane == 0) *se = e;
  return bad;
}

// Sum of the staged lines in slots w, w+1, w+2 (lines y-1, y, y+1 of a plane)
// at their largest exponent, which it returns.
template <int NC>
__device__ __forceinline__ int spmv_plane_sum(const long long *__restrict__ buf, const int *__restrict__ se, int w, int lane,
                                              long long (&t)[NC]) {
  const int ea = se[w], eb = se[w + 1], ed = se[w + 2];
  const int et = max(max(ea, eb), ed);
  const long long *la = buf + w * 32 * NC;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int i = lane + 32 * c;
    t[c] = (shr_q(la[i], et - ea) + shr_q(la[32 * NC + i], et - eb)) + shr_q(la[64 * NC + i], et - ed);
  }
  return et;
}

// Dynamic shared memory of one block: four plane buffers of lpc + 2 line
// slots, and their line exponents.
template <int NC>
__host__ __device__ constexpr size_t spmv_stage_smem(int lpc) {
  return (size_t)4 * (lpc + 2) * 32 * NC * sizeof(long long) + (size_t)4 * (lpc + 2) * sizeof(int);
}

// The work of one block (instance ii).
template <int NC, int Mode>
__device__ __forceinline__ void spmv_stage_block(const Inst *__restrict__ tab, int count, int ii, int lpc, int zc, const double *__restrict__ x,
                                                 const double *__restrict__ b, double *__restrict__ y, const double *__restrict__ kap,
                                                 double *__restrict__ partials, const CgState *__restrict__ st, int vec16,
                                                 long long *__restrict__ smem_spmv) {
  const int nslot = lpc + 2;
  const int bstride = nslot * 32 * NC;  // one plane buffer
  long long *const sq = smem_spmv;
  int *const se = reinterpret_cast<int *>(smem_spmv + 4 * bstride);  // [4][nslot]
  const int blk = blockIdx.x;
  const Inst g = tab[ii];
  const int w = threadIdx.y, lane = threadIdx.x;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nby = (ny + lpc - 1) / lpc;
  const int lb = blk - g.blk_row;
  const int y0 = (lb % nby) * lpc;
  const int yy = y0 + w;
  const int z0 = (lb / nby) * zc;
  const int z1 = min(z0 + zc, nz);
  const long sxy = (long)nx * ny;
  const double *xg = x + g.off;
  const bool own = yy < ny;
  if (st && st[ii].done) {  // the whole block: a block belongs to one instance
    if (partials && own && lane == 0)
      for (int zz = z0; zz < z1; ++zz) partials[g.poff + (long)zz * ny + yy] = 0.0;
    return;
  }
  if (z0 >= z1) return;  // the whole block

  // plane zp into buffer bf: every warp copies its own line, the first and
  // last warp also the lines beside the block (one commit group per call)
  auto fetch = [&](int zp, int bf) {
    long long *buf = sq + bf * bstride;
    spmv_fetch_line<NC>(xg, nx, ny, nz, sxy, zp, yy, lane, vec16 != 0, buf + (w + 1) * 32 * NC);
    if (w == 0) spmv_fetch_line<NC>(xg, nx, ny, nz, sxy, zp, y0 - 1, lane, vec16 != 0, buf);
    if (w == lpc - 1) spmv_fetch_line<NC>(xg, nx, ny, nz, sxy, zp, y0 + lpc, lane, vec16 != 0, buf + (lpc + 1) * 32 * NC);
    cp_async_commit();
  };
  // the lines this warp fetched into buffer bf, converted in place
  auto convert = [&](int bf) -> bool {
    long long *buf = sq + bf * bstride;
    int *e = se + bf * nslot;
    bool bad = spmv_convert_line<NC>(buf + (w + 1) * 32 * NC, e + w + 1, lane);
    if (w == 0) bad |= spmv_convert_line<NC>(buf, e, lane);
    if (w == lpc - 1) bad |= spmv_convert_line<NC>(buf + (lpc + 1) * 32 * NC, e + lpc + 1, lane);
    return bad;
  };
  // writes row (yy, zz) from ax = (27 + kappa) x - S: the output and the
  // line's partial of x . y
  auto emit = [&](int zz, double (&ax)[NC]) {
    const long rowbase = (long)zz * sxy + (long)yy * nx;
    if (!(HPCG_IN(rowbase, nx, 0, g.n) && HPCG_IN((long)zz * ny + yy, 1, 0, (long)ny * nz))) return;  // the whole warp
    double dotv = 0.0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int xx = lane + 32 * c;
      if (xx < nx) {
        const long gi = g.off + rowbase + xx;
        const double out = Mode == 0 ? ax[c] : b[gi] - ax[c];
        y[gi] = out;
        if (partials) dotv += xg[rowbase + xx] * out;
      }
    }
    if (partials) {  // exact tree over the lanes of this line, on the integer pipe
      dotv = warp_sum_fx(dotv);
      if (lane == 0) partials[g.poff + (long)zz * ny + yy] = dotv;
    }
  };
  // rows zfrom .. z1-1 with FP64 sums from global memory (a staged line was
  // huge or not finite); every warp of the block arrives here at the same
  // plane step and no barrier follows (copies still in flight are drained)
  auto fp64_rows = [&](int zfrom) {
    cp_async_wait<0>();
    if (!own) return;
    for (int zz = zfrom; zz < z1; ++zz) {
      if (!HPCG_IN((long)zz * sxy + (long)yy * nx, nx, 0, g.n)) continue;
      double t0[NC], t1[NC], t2[NC], u[NC], ul[NC], ur[NC], ax[NC];
      tsum<double, NC>(xg, nx, ny, nz, yy, zz - 1, lane, t0);
      tsum<double, NC>(xg, nx, ny, nz, yy, zz, lane, t1);
      tsum<double, NC>(xg, nx, ny, nz, yy, zz + 1, lane, t2);
#pragma unroll
      for (int c = 0; c < NC; ++c) u[c] = (t0[c] + t1[c]) + t2[c];
      line_neighbours<double, NC>(u, ul, ur, lane);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xx = lane + 32 * c;
        const long gi = g.off + (long)zz * sxy + (long)yy * nx + xx;
        ax[c] = xx < nx ? (kap ? 27.0 + kap[gi] : 27.0) * xg[gi - g.off] - ((ul[c] + u[c]) + ur[c]) : 0.0;
      }
      emit(zz, ax);
    }
  };

  // prologue: planes z0 - 1 and z0 (buffers 0, 1), plane z0 + 1 in flight (2)
  fetch(z0 - 1, 0);
  fetch(z0, 1);
  fetch(z0 + 1, 2);
  long long T0[NC], T1[NC];
  cp_async_wait<2>();
  __syncwarp();
  if (__syncthreads_or(convert(0))) return fp64_rows(z0);
  int e0 = spmv_plane_sum<NC>(sq, se, w, lane, T0);
  cp_async_wait<1>();
  __syncwarp();
  if (__syncthreads_or(convert(1))) return fp64_rows(z0);
  int e1 = spmv_plane_sum<NC>(sq + bstride, se + nslot, w, lane, T1);
  int bc = 1;  // buffer of plane zz
  for (int zz = z0; zz < z1; ++zz) {
    const int bn = bc == 3 ? 0 : bc + 1;  // plane zz + 1 (arrived or arriving)
    const int bf = bn == 3 ? 0 : bn + 1;  // plane zz + 2 goes into the buffer of plane zz - 2
    fetch(zz + 2, bf);
    cp_async_wait<1>();  // everything but the group just committed: plane zz + 1 is here
    __syncwarp();
    if (__syncthreads_or(convert(bn))) return fp64_rows(zz);
    long long T2[NC];
    const int e2 = spmv_plane_sum<NC>(sq + bn * bstride, se + bn * nslot, w, lane, T2);
    if (own && HPCG_IN((long)zz * sxy + (long)yy * nx, nx, 0, g.n)) {  // kappa and x are read at the own row
      const int E = max(max(e0, e1), e2);
      long long u[NC], ul[NC], ur[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) u[c] = (shr_q(T0[c], E - e0) + shr_q(T1[c], E - e1)) + shr_q(T2[c], E - e2);
      line_neighbours_i<NC>(u, ul, ur, lane);
      const long long *oq = sq + bc * bstride + (w + 1) * 32 * NC;  // the own line of plane zz
      const int eo = se[bc * nslot + w + 1];                          // at or below E
      double ax[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const long long S = (ul[c] + u[c]) + ur[c];
        const int xx = lane + 32 * c;
        if (!kap)  // 27 x - S exactly at scale E + 1 (both terms below 2^62 there), one rounding
          ax[c] = fx_to_double(27 * shr_q(oq[lane + 32 * c], E + 1 - eo) - (S >> 1), E + 1);
        else
          ax[c] = xx < nx ? (27.0 + kap[g.off + (long)zz * sxy + (long)yy * nx + xx]) * xg[(long)zz * sxy + (long)yy * nx + xx] -
                                fx_to_double(S, E)
                          : 0.0;
      }
      emit(zz, ax);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T0[c] = T1[c];
      T1[c] = T2[c];
    }
    e0 = e1;
    e1 = e2;
    bc = bn;
  }
  cp_async_wait<0>();  // the last fetch (beyond the block's planes) lands before the block ends
}

template <int NC, int Mode>
__global__ void __launch_bounds__(32 * kSpmvMaxLpc) k_spmv_stage_fx(const Inst *__restrict__ tab, int count, int lpc, int zc,
                                                                     const double *__restrict__ x, const double *__restrict__ b,
                                                                     double *__restrict__ y, const double *__restrict__ kap,
                                                                     double *__restrict__ partials, const CgState *__restrict__ st,
                                                                     int vec16) {
  pdl_enter();
  extern __shared__ __align__(16) long long smem_spmv[];
  const int ii = count == 1 ? 0 : find_inst<3>(tab, count, blockIdx.x);
  spmv_stage_block<NC, Mode>(tab, count, ii, lpc, zc, x, b, y, kap, partials, st, vec16, smem_spmv);
}

// The same for a batch whose instances have x-lines of different lengths:
// each block (one instance) takes the narrowest register window that holds
// its lines (the launch's shared memory, sized for the widest, holds it).
// Same arithmetic per line, so the same bits as k_spmv_stage_fx.
template <int NC, int Mode>
__global__ void __launch_bounds__(32 * kSpmvMaxLpc) k_spmv_stage_fx_batch(const Inst *__restrict__ tab, int count, int lpc, int zc,
                                                                           const double *__restrict__ x, const double *__restrict__ b,
                                                                           double *__restrict__ y, const double *__restrict__ kap,
                                                                           double *__restrict__ partials, const CgState *__restrict__ st,
                                                                           int vec16) {
  pdl_enter();
  extern __shared__ __align__(16) long long smem_spmv[];
  const int ii = find_inst<3>(tab, count, blockIdx.x);
  const int nxi = tab[ii].nx;
  if (nxi <= 32) return spmv_stage_block<1, Mode>(tab, count, ii, lpc, zc, x, b, y, kap, partials, st, vec16, smem_spmv);
  if constexpr (NC > 2) {
    if (nxi <= 64) return spmv_stage_block<2, Mode>(tab, count, ii, lpc, zc, x, b, y, kap, partials, st, vec16, smem_spmv);
  }
  if constexpr (NC > 3) {
    if (nxi <= 96) return spmv_stage_block<3, Mode>(tab, count, ii, lpc, zc, x, b, y, kap, partials, st, vec16, smem_spmv);
  }
  spmv_stage_block<NC, Mode>(tab, count, ii, lpc, zc, x, b, y, kap, partials, st, vec16, smem_spmv);
}

}  // namespace hpcg
