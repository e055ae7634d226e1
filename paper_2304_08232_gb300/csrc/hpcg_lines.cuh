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
#include <type_traits>
#include "hpcg_device.cuh"

namespace hpcg {


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

// Loads of z and r.  Kernels launched once per step read lines no one writes
// during the launch, through the read-only path (COH = false).  The persistent
// tail kernel reads lines other blocks wrote earlier in the same launch, so it
// loads at L2 (COH = true), which the grid barrier's fences keep coherent.
template <bool COH, typename T>
__device__ __forceinline__ T ld_line(const T *p) {
  if (COH) return __ldcg(p);
  return __ldg(p);
}

// The values at x and x + 1 of a line (x even, line length even, so the pair
// is aligned to its size) in one vector load.
template <bool COH, typename T>
__device__ __forceinline__ void ld_pair(const T *p, T &e, T &o) {
  using V = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  const V v = ld_line<COH>(reinterpret_cast<const V *>(p));
  e = v.x;
  o = v.y;
}

// Line class of line (y, z): its y and z parities, (y & 1) + 2 (z & 1).
__device__ __forceinline__ int line_class(int y, int z) { return (y & 1) + 2 * (z & 1); }

// Sum over y-1, y, y+1 of line (., y, zz) of the grid at zg (zero outside).
// Lines whose class bit is clear in vmask hold no valid data yet and count as
// zero (smoothing from z = 0 without clearing z first).
template <typename T, int NCH>
__device__ __forceinline__ void tsum(const T *__restrict__ zg, int nx, int ny, int nz, int y, int zz, int lane, T (&t)[NCH],
                                     int vmask = 0xF) {
  const bool zin = zz >= 0 && zz < nz;
  const long sxy = (long)nx * ny;
  const T *lm = zg + (long)zz * sxy + (long)(y - 1) * nx;
  const T *l0 = lm + nx;
  const T *lp = l0 + nx;
  const bool ym = y - 1 >= 0 && ((vmask >> line_class(y + 1, zz)) & 1);  // y-1 and y+1 share a class
  const bool yp = y + 1 < ny && ((vmask >> line_class(y + 1, zz)) & 1);
  const bool y0 = (vmask >> line_class(y, zz)) & 1;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int x = lane + 32 * c;
    T s = T(0);
    if (zin && x < nx) {
      const T a = ym ? __ldg(lm + x) : T(0);
      const T b = y0 ? __ldg(l0 + x) : T(0);
      const T d = yp ? __ldg(lp + x) : T(0);
      s = (a + b) + d;
    }
    t[c] = s;
  }
}

// Parity-split registers of a line: lane l holds E[c] = v(x = 2k) and
// O[c] = v(x = 2k + 1) for k = l + 32c, so that a colour step (one x parity)
// keeps all 32 lanes busy.  Neighbours along x: for even x = 2k they are
// O[k-1] and O[k]; for odd x = 2k+1 they are E[k] and E[k+1].
template <typename T, int NC>
__device__ __forceinline__ void prev_of(const T (&v)[NC], T (&out)[NC], int lane) {  // out[k] = v[k-1]
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T up = __shfl_up_sync(kFull, v[c], 1);
    const T last = __shfl_sync(kFull, v[c > 0 ? c - 1 : 0], 31);
    out[c] = lane == 0 ? (c > 0 ? last : T(0)) : up;
  }
}
template <typename T, int NC>
__device__ __forceinline__ void next_of(const T (&v)[NC], T (&out)[NC], int lane) {  // out[k] = v[k+1]
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T dn = __shfl_down_sync(kFull, v[c], 1);
    const T first = __shfl_sync(kFull, v[c + 1 < NC ? c + 1 : c], 0);
    out[c] = lane == 31 ? (c + 1 < NC ? first : T(0)) : dn;
  }
}

// Sum over y-1, y, y+1 of line (., y, zz) at even (te) and odd (to) x.
template <typename T, int NC, bool COH, bool PAIR = false>
__device__ __forceinline__ void tsum2(const T *__restrict__ zg, int nx, int ny, int nz, int y, int zz, int lane, T (&te)[NC],
                                      T (&to)[NC], int vmask) {
  const bool zin = zz >= 0 && zz < nz;
  const long sxy = (long)nx * ny;
  const T *lm = zg + (long)zz * sxy + (long)(y - 1) * nx;
  const T *l0 = lm + nx;
  const T *lp = l0 + nx;
  const bool ym = zin && y - 1 >= 0 && ((vmask >> line_class(y + 1, zz)) & 1);
  const bool yp = zin && y + 1 < ny && ((vmask >> line_class(y + 1, zz)) & 1);
  const bool y0 = zin && ((vmask >> line_class(y, zz)) & 1);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int xe = 2 * (lane + 32 * c), xo = xe + 1;
    T se = T(0), so = T(0);
    if (PAIR) {
      if (xe < nx) {
        T ae = T(0), ao = T(0), be = T(0), bo = T(0), de = T(0), d_o = T(0);
        if (ym) ld_pair<COH>(lm + xe, ae, ao);
        if (y0) ld_pair<COH>(l0 + xe, be, bo);
        if (yp) ld_pair<COH>(lp + xe, de, d_o);
        se = (ae + be) + de;
        so = (ao + bo) + d_o;
      }
    } else {
      if (xe < nx)
        se = ((ym ? ld_line<COH>(lm + xe) : T(0)) + (y0 ? ld_line<COH>(l0 + xe) : T(0))) + (yp ? ld_line<COH>(lp + xe) : T(0));
      if (xo < nx)
        so = ((ym ? ld_line<COH>(lm + xo) : T(0)) + (y0 ? ld_line<COH>(l0 + xo) : T(0))) + (yp ? ld_line<COH>(lp + xo) : T(0));
    }
    te[c] = se;
    to[c] = so;
  }
}

// Colour steps on the lines of class (py, pz): `steps` alternating x parities
// starting with `pa`.  Block = 32 x lpc threads (lpc lines), zc updated planes
// per block.  Reads z of the 3x3 line neighbourhood, writes z on its own lines.
//
// vmask: line classes whose z values are valid; the others count as zero (the
// first forward sweep from z = 0).  rc (nullable): fused residual + injection
// (Listing 1's residual and restriction) after the last step, for a run on class (0, 0) that
// ends on even x: every injected fine row (2xc, 2yc, 2zc) lies on these lines,
// its neighbour sum is P + z(x-1) + z(x+1) with values final for this
// smoother application, so rc[c] = r - (A_ii z - that sum) is formed here.
// PAIR: every line has an even length, so x pairs move as one vector.
template <typename T, int NC, bool COH = false, bool PAIR = false>
__device__ __forceinline__ void gs_lines_vblock(int blk, int wy, const Inst *__restrict__ tab, int count, int lpc, int zc, int py, int pz,
                                                int pa, int steps, int vmask, const T *__restrict__ r, T *__restrict__ z,
                                                const T *__restrict__ invd, const CgState *__restrict__ st,
                                                const Inst *__restrict__ tabc, T *__restrict__ rc, const T *__restrict__ kap) {
  const int ii = find_inst<4>(tab, count, blk);
  const Inst g = tab[ii];
  if (st && st[ii].done) return;
  const int cy = (g.ny - py + 1) / 2, cz = (g.nz - pz + 1) / 2;
  const int nby = (half_up(g.ny) + lpc - 1) / lpc;
  const int lb = blk - g.blk_line;
  const int j = (lb % nby) * lpc + wy;
  const int m0 = (lb / nby) * zc;
  const int m1 = min(m0 + zc, cz);
  if (j >= cy || m0 >= m1) return;  // whole warp
  const int lane = threadIdx.x;
  const int y = 2 * j + py;
  const int nx = g.nx;
  const long sxy = (long)nx * g.ny;
  T *zg = z + g.off;
  const T *rg = r + g.off;
  const int cls_v = line_class(y + 1, pz);  // lines (y +- 1, zz)
  const bool ym = y - 1 >= 0 && ((vmask >> cls_v) & 1), yp = y + 1 < g.ny && ((vmask >> cls_v) & 1);
  const bool own_valid = (vmask >> line_class(y, pz)) & 1;
  T tpe[NC], tpo[NC];
  tsum2<T, NC, COH, PAIR>(zg, nx, g.ny, g.nz, y, 2 * m0 + pz - 1, lane, tpe, tpo, vmask);
  for (int m = m0; m < m1; ++m) {
    const int zz = 2 * m + pz;
    T tne[NC], tno[NC], PE[NC], PO[NC];
    tsum2<T, NC, COH, PAIR>(zg, nx, g.ny, g.nz, y, zz + 1, lane, tne, tno, vmask);
    const long rowbase = (long)zz * sxy + (long)y * nx;
    T E[NC], O[NC], rE[NC], rO[NC];
    if (PAIR) {  // own line and right-hand side, issued with the neighbours' loads
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 2 * (lane + 32 * c);
        E[c] = O[c] = rE[c] = rO[c] = T(0);
        if (xe < nx) {
          if (own_valid) {
            if (COH)
              ld_pair<true>(zg + rowbase + xe, E[c], O[c]);
            else
              ld_pair<false>(zg + rowbase + xe, E[c], O[c]);  // own line: this warp alone writes it
          }
          ld_pair<COH>(rg + rowbase + xe, rE[c], rO[c]);
        }
      }
    }
    {
      T ce[NC], co[NC], sh[NC];
      const T *lm = zg + (long)zz * sxy + (long)(y - 1) * nx;
      const T *lp = lm + 2 * nx;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 2 * (lane + 32 * c), xo = xe + 1;
        T ve = T(0), vo = T(0);
        if (PAIR) {
          if (xe < nx) {
            T ae = T(0), ao = T(0), de = T(0), d_o = T(0);
            if (ym) ld_pair<COH>(lm + xe, ae, ao);
            if (yp) ld_pair<COH>(lp + xe, de, d_o);
            ve = ae + de;
            vo = ao + d_o;
          }
        } else {
          if (xe < nx) ve = (ym ? ld_line<COH>(lm + xe) : T(0)) + (yp ? ld_line<COH>(lp + xe) : T(0));
          if (xo < nx) vo = (ym ? ld_line<COH>(lm + xo) : T(0)) + (yp ? ld_line<COH>(lp + xo) : T(0));
        }
        ce[c] = (tpe[c] + tne[c]) + ve;  // off-line column sums at x
        co[c] = (tpo[c] + tno[c]) + vo;
      }
      prev_of<T, NC>(co, sh, lane);  // cc(x-1) at even x
#pragma unroll
      for (int c = 0; c < NC; ++c) PE[c] = (sh[c] + ce[c]) + co[c];
      next_of<T, NC>(ce, sh, lane);  // cc(x+1) at odd x
#pragma unroll
      for (int c = 0; c < NC; ++c) PO[c] = (ce[c] + co[c]) + sh[c];
    }
    if (!PAIR) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 2 * (lane + 32 * c), xo = xe + 1;
        E[c] = (xe < nx && own_valid) ? (COH ? __ldcg(zg + rowbase + xe) : zg[rowbase + xe]) : T(0);
        O[c] = (xo < nx && own_valid) ? (COH ? __ldcg(zg + rowbase + xo) : zg[rowbase + xo]) : T(0);
        rE[c] = xe < nx ? (COH ? __ldcg(rg + rowbase + xe) : rg[rowbase + xe]) : T(0);
        rO[c] = xo < nx ? (COH ? __ldcg(rg + rowbase + xo) : rg[rowbase + xo]) : T(0);
      }
    }
    T nb[NC];  // neighbours along x of the parity updated last
    for (int s = 0; s < steps; ++s) {
      const int q = (s & 1) ? 1 - pa : pa;
      if (q == 0) {
        prev_of<T, NC>(O, nb, lane);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int xe = 2 * (lane + 32 * c);
          if (xe < nx) {
            const T id = invd ? invd[g.off + rowbase + xe] : T(1) / T(26);
            E[c] = (((rE[c] + PE[c]) + nb[c]) + O[c]) * id;
          }
        }
      } else {
        next_of<T, NC>(E, nb, lane);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int xo = 2 * (lane + 32 * c) + 1;
          if (xo < nx) {
            const T id = invd ? invd[g.off + rowbase + xo] : T(1) / T(26);
            O[c] = (((rO[c] + PO[c]) + E[c]) + nb[c]) * id;
          }
        }
      }
    }
    const bool write_e = steps > 1 || !own_valid || pa == 0;
    const bool write_o = steps > 1 || !own_valid || pa == 1;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int xe = 2 * (lane + 32 * c), xo = xe + 1;
      if (PAIR && write_e && write_o) {
        using V = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
        if (xe < nx) *reinterpret_cast<V *>(zg + rowbase + xe) = V{E[c], O[c]};
      } else {
        if (write_e && xe < nx) zg[rowbase + xe] = E[c];
        if (write_o && xo < nx) zg[rowbase + xo] = O[c];
      }
    }
    if (rc) {
      // the last step updated even x; nb holds its (unchanged) left odd neighbours
      const Inst gc = tabc[ii];
      const long cbase = gc.off + (long)(zz >> 1) * gc.nx * gc.ny + (long)(y >> 1) * gc.nx;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 2 * (lane + 32 * c);
        if (xe < nx) {
          const T d = kap ? T(26) + kap[g.off + rowbase + xe] : T(26);
          const T nbs = (PE[c] + nb[c]) + O[c];
          rc[cbase + (xe >> 1)] = rE[c] - (d * E[c] - nbs);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      tpe[c] = tne[c];
      tpo[c] = tno[c];
    }
  }
}

template <typename T, int NC, bool PAIR = false>
__global__ void __launch_bounds__(256) k_gs_lines(const Inst *__restrict__ tab, int count, int lpc, int zc, int py, int pz, int pa,
                                                  int steps, int vmask, const T *__restrict__ r, T *__restrict__ z,
                                                  const T *__restrict__ invd, const CgState *__restrict__ st, const Inst *__restrict__ tabc,
                                                  T *__restrict__ rc, const T *__restrict__ kap) {
  pdl_enter();
  gs_lines_vblock<T, NC, false, PAIR>(blockIdx.x, threadIdx.y, tab, count, lpc, zc, py, pz, pa, steps, vmask, r, z, invd, st, tabc, rc,
                                      kap);
}

// y = A x (Mode 0) or y = b - A x (Mode 1) over every x-line; A x = (27 + kappa) x - S
// with S the 27-point box sum.  Block = 32 x lpc threads (lpc consecutive lines
// in y), zc consecutive planes.  Optional partials of x.y, one per x-line
// (index poff + z ny + y), so the reduction does not depend on the launch shape.
template <typename T, int NCH, int Mode>
__global__ void __launch_bounds__(256) k_spmv_lines(const Inst *__restrict__ tab, int count, int lpc, int zc, const T *__restrict__ x,
                                                    const T *__restrict__ b, T *__restrict__ y, const T *__restrict__ kap,
                                                    double *__restrict__ partials, const CgState *__restrict__ st) {
  pdl_enter();
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
      double dotv = 0.0;
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
      if (partials) {  // fixed shuffle tree over the lanes of this line
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dotv += __shfl_down_sync(kFull, dotv, o);
        if (lane == 0) partials[g.poff + (long)zz * g.ny + yy] = dotv;
      }
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        t0[c] = t1[c];
        t1[c] = t2[c];
      }
    }
  }
  if (skip && partials) {
    // a converged instance still owns its partial slots: zero them
    if (yy < g.ny)
      for (int zz = z0 + 0; zz < z1; ++zz)
        if (lane == 0) partials[g.poff + (long)zz * g.ny + yy] = 0.0;
  }
}

}  // namespace hpcg
