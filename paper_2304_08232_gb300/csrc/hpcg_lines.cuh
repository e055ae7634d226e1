// hpcg_lines.cuh -- x-line kernels of the 27-point operator (FP64 path and
// FP32 preconditioner).
//
// One warp owns one x-line (fixed y, z); lane l holds x = l + 32c for
// c < NCH.  Neighbour values along x come from warp shuffles, the other
// eight lines of the 3x3 (y, z) neighbourhood from global memory (each line
// read whole, coalesced).  Sums are separable: line sums over y, then over z
// while the warp marches through its z-planes (reusing the previous plane's
// sum), then over x.
//
// Colour steps (Section III-A, Listings 2/3) come in pairs: colours 2m and
// 2m+1 differ only in x parity, i.e. they update the even and the odd points
// of the same lines (y and z of fixed parities).  Every neighbour of such a
// line that is not on the line itself lies on a line of another parity class,
// which the pair does not change.  So the kernel forms that off-line part P(x)
// once and then performs the colour steps one after the other along the line:
// first the points of x parity `pa`, then the other parity with the new
// values, and for a third step the first parity again.  Each step is the
// update of Eq. 1, z_i <- (r_i + sum_{j != i} z_j) / A_ii.
#pragma once
#include "hpcg_device.cuh"

namespace hpcg {

constexpr unsigned kFull = 0xffffffffu;

// vl[c] = v at x-1, vr[c] = v at x+1, for x = lane + 32c; zero past both ends
// of the 32*NCH window (values at x >= nx must already be zero).
template <typename T, int NCH>
__device__ __forceinline__ void line_neighbours(const T (&v)[NCH], T (&vl)[NCH], T (&vr)[NCH], int lane) {
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const T up = __shfl_up_sync(kFull, v[c], 1);
    const T prev_last = __shfl_sync(kFull, c > 0 ? v[c > 0 ? c - 1 : 0] : T(0), 31);
    vl[c] = lane == 0 ? (c > 0 ? prev_last : T(0)) : up;
    const T dn = __shfl_down_sync(kFull, v[c], 1);
    const T next_first = __shfl_sync(kFull, c + 1 < NCH ? v[c + 1 < NCH ? c + 1 : c] : T(0), 0);
    vr[c] = lane == 31 ? (c + 1 < NCH ? next_first : T(0)) : dn;
  }
}

// Sum over y-1, y, y+1 of line (., y, zz) of the grid at zg (zero outside).
template <typename T, int NCH>
__device__ __forceinline__ void tsum(const T *__restrict__ zg, int nx, int ny, int nz, int y, int zz, int lane, T (&t)[NCH]) {
  const bool zin = zz >= 0 && zz < nz;
  const long sxy = (long)nx * ny;
  const T *lm = zg + (long)zz * sxy + (long)(y - 1) * nx;
  const T *l0 = lm + nx;
  const T *lp = l0 + nx;
  const bool ym = y - 1 >= 0, yp = y + 1 < ny;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int x = lane + 32 * c;
    T s = T(0);
    if (zin && x < nx) {
      const T a = ym ? __ldg(lm + x) : T(0);
      const T b = __ldg(l0 + x);
      const T d = yp ? __ldg(lp + x) : T(0);
      s = (a + b) + d;
    }
    t[c] = s;
  }
}

// Colour steps on the lines of class (py, pz): `steps` alternating x parities
// starting with `pa`.  Block = 32 x lpc threads (lpc lines), zc updated planes
// per block.  Reads z of the 3x3 line neighbourhood, writes z on its own lines.
template <typename T, int NCH>
__global__ void __launch_bounds__(256) k_gs_lines(const Inst *__restrict__ tab, int count, int lpc, int zc, int py, int pz, int pa,
                                                  int steps, const T *__restrict__ r, T *__restrict__ z, const T *__restrict__ invd,
                                                  const CgState *__restrict__ st) {
  const int blk = blockIdx.x;
  const int ii = find_inst<4>(tab, count, blk);
  const Inst g = tab[ii];
  if (st && st[ii].done) return;
  const int cy = (g.ny - py + 1) / 2, cz = (g.nz - pz + 1) / 2;
  const int nby = (half_up(g.ny) + lpc - 1) / lpc;
  const int lb = blk - g.blk_line;
  const int j = (lb % nby) * lpc + threadIdx.y;
  const int m0 = (lb / nby) * zc;
  const int m1 = min(m0 + zc, cz);
  if (j >= cy || m0 >= m1) return;  // whole warp
  const int lane = threadIdx.x;
  const int y = 2 * j + py;
  const int nx = g.nx;
  const long sxy = (long)nx * g.ny;
  T *zg = z + g.off;
  const T *rg = r + g.off;
  const bool ym = y - 1 >= 0, yp = y + 1 < g.ny;
  T tprev[NCH];
  tsum<T, NCH>(zg, nx, g.ny, g.nz, y, 2 * m0 + pz - 1, lane, tprev);
  for (int m = m0; m < m1; ++m) {
    const int zz = 2 * m + pz;
    T tnext[NCH], P[NCH];
    tsum<T, NCH>(zg, nx, g.ny, g.nz, y, zz + 1, lane, tnext);
    {
      T cc[NCH], cl[NCH], cr[NCH];
      const T *lm = zg + (long)zz * sxy + (long)(y - 1) * nx;
      const T *lp = lm + 2 * nx;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int x = lane + 32 * c;
        T v = T(0);
        if (x < nx) v = (ym ? __ldg(lm + x) : T(0)) + (yp ? __ldg(lp + x) : T(0));
        cc[c] = (tprev[c] + tnext[c]) + v;  // off-line column sum at x
      }
      line_neighbours<T, NCH>(cc, cl, cr, lane);
#pragma unroll
      for (int c = 0; c < NCH; ++c) P[c] = (cl[c] + cc[c]) + cr[c];
    }
    const long rowbase = (long)zz * sxy + (long)y * nx;
    T own[NCH], rr[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const int x = lane + 32 * c;
      own[c] = x < nx ? zg[rowbase + x] : T(0);
      rr[c] = x < nx ? rg[rowbase + x] : T(0);
    }
    for (int s = 0; s < steps; ++s) {
      const int q = (s & 1) ? 1 - pa : pa;
      T ol[NCH], orr[NCH];
      line_neighbours<T, NCH>(own, ol, orr, lane);
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int x = lane + 32 * c;
        if (x < nx && (x & 1) == q) {
          const T id = invd ? invd[g.off + rowbase + x] : T(1) / T(26);
          own[c] = (((rr[c] + P[c]) + ol[c]) + orr[c]) * id;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const int x = lane + 32 * c;
      if (x < nx && (steps > 1 || (x & 1) == pa)) zg[rowbase + x] = own[c];
    }
#pragma unroll
    for (int c = 0; c < NCH; ++c) tprev[c] = tnext[c];
  }
}

// y = A x (Mode 0) or y = b - A x (Mode 1) over every x-line; A x = (27 + kappa) x - S
// with S the 27-point box sum.  Block = 32 x lpc threads (lpc consecutive lines
// in y), zc consecutive planes.  Optional partials of x.y per block.
template <typename T, int NCH, int Mode>
__global__ void __launch_bounds__(256) k_spmv_lines(const Inst *__restrict__ tab, int count, int lpc, int zc, const T *__restrict__ x,
                                                    const T *__restrict__ b, T *__restrict__ y, const T *__restrict__ kap,
                                                    double *__restrict__ partials, const CgState *__restrict__ st) {
  __shared__ double sh[8];
  const int blk = blockIdx.x;
  const int ii = find_inst<3>(tab, count, blk);
  const Inst g = tab[ii];
  const bool skip = st && st[ii].done;
  const int nby = (g.ny + lpc - 1) / lpc;
  const int lb = blk - g.blk_row;
  const int yy = (lb % nby) * lpc + threadIdx.y;
  const int z0 = (lb / nby) * zc;
  const int z1 = min(z0 + zc, g.nz);
  const int lane = threadIdx.x;
  const int nx = g.nx;
  const long sxy = (long)nx * g.ny;
  const T *xg = x + g.off;
  double dotv = 0.0;
  if (!skip && yy < g.ny && z0 < z1) {
    T t0[NCH], t1[NCH];
    tsum<T, NCH>(xg, nx, g.ny, g.nz, yy, z0 - 1, lane, t0);
    tsum<T, NCH>(xg, nx, g.ny, g.nz, yy, z0, lane, t1);
    for (int zz = z0; zz < z1; ++zz) {
      T t2[NCH], u[NCH], ul[NCH], ur[NCH];
      tsum<T, NCH>(xg, nx, g.ny, g.nz, yy, zz + 1, lane, t2);
#pragma unroll
      for (int c = 0; c < NCH; ++c) u[c] = (t0[c] + t1[c]) + t2[c];
      line_neighbours<T, NCH>(u, ul, ur, lane);
      const long rowbase = (long)zz * sxy + (long)yy * nx;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int xx = lane + 32 * c;
        if (xx < nx) {
          const T s = (ul[c] + u[c]) + ur[c];
          const T xi = xg[rowbase + xx];
          const long gi = g.off + rowbase + xx;
          const T d1 = kap ? T(27) + kap[gi] : T(27);
          const T ax = d1 * xi - s;
          const T out = Mode == 0 ? ax : b[gi] - ax;
          y[gi] = out;
          if (partials) dotv += (double)xi * (double)out;
        }
      }
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        t0[c] = t1[c];
        t1[c] = t2[c];
      }
    }
  }
  if (partials) {
    // fixed-order block sum over (lane, line)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dotv += __shfl_down_sync(kFull, dotv, o);
    if (lane == 0) sh[threadIdx.y] = dotv;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)blockDim.y; ++w) s += sh[w];
      partials[blk] = s;
    }
  }
}

}  // namespace hpcg
