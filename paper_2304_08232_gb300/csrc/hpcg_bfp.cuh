// hpcg_bfp.cuh -- the FP64 V-cycle with its level vectors z held in block
// floating point: a 64-bit integer mantissa per point and one exponent per
// x-line.
//
// The colour-pair kernel of hpcg_fixed.cuh spends most of its integer
// instructions turning the FP64 values it loads into fixed point, about five
// conversions per updated point.  Here z stays in that form between kernels:
// point i of line L holds q_i with value q_i 2^(e_L - 1080), |q_i| < 2^58, so
// that a kernel only aligns whole lines to a common exponent (one shift per
// value, by an amount that is the same across the warp) before adding them
// exactly.  Each colour step's sum r + sum_{j != i} z_j is formed exactly at
// a scale S of the whole line, and the new value costs one rounding: the
// division by A_ii = 26 through an integer multiplier, or a multiply by
// 1 / A_ii in FP64 when kappa is set, at scale S - 3 (at least 2^-56 of the
// step's largest term).  The line is then stored with its exponent lowered
// until its largest mantissa has bit 57 set (an exact shift), so exponents
// follow the data from run to run instead of the sums' bounds.
//
// Every exponent is a function of the data alone (the lines summed, the
// right-hand side, the own line), never of how lines and planes are grouped
// into blocks, so results do not depend on the launch shape.  A line whose
// values are non-finite or beyond 2^977 gets the exponent kBfpNaN and reads as
// NaN from then on, so non-finite input still ends in a NaN result.
//
// Only the V-cycle uses this form: the right-hand sides r stay FP64, and the
// finest level's z is written back in FP64 by the last run that touches each
// line class (the final-touch runs of the last post-smoother).
#pragma once
#include "hpcg_fixed.cuh"
#include "hpcg_tail.cuh"

namespace hpcg {

constexpr int kBfpNaN = 2047;  // exponent of a line that reads as NaN

// Arithmetic right shift by d >= 0 (amounts of 64 or more give the sign).
__device__ __forceinline__ long long shr_q(long long v, int d) {
  long long r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"((unsigned)d));
  return r;
}

__device__ __forceinline__ double bfp_nan() { return __longlong_as_double(0x7ff8000000000000LL); }

// Mantissa pairs (x = 2k, 2k+1 for k = lane + 32c) of one line; nx is even,
// so a pair is either inside the line or past its end.
template <int NC, bool COH = false>
__device__ __forceinline__ void ld_pairs_q(const long long *__restrict__ line, bool ok, int nx, int lane, long long (&e)[NC],
                                           long long (&o)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int xe = 64 * c + 2 * lane;
    if (ok && xe < nx) {
      const longlong2 v = ld_line<COH>(reinterpret_cast<const longlong2 *>(line + xe));
      e[c] = v.x;
      o[c] = v.y;
    } else {
      e[c] = 0;
      o[c] = 0;
    }
  }
}
template <int NC, bool COH = false>
__device__ __forceinline__ void ld_pairs_d(const double *__restrict__ line, int nx, int lane, double (&e)[NC], double (&o)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int xe = 64 * c + 2 * lane;
    if (xe < nx) {
      const double2 v = ld_line<COH>(reinterpret_cast<const double2 *>(line + xe));
      e[c] = v.x;
      o[c] = v.y;
    } else {
      e[c] = 0.0;
      o[c] = 0.0;
    }
  }
}

// Sum over lines y-1, y, y+1 of plane zz (those with ok set), at the largest
// exponent of the three; returns that exponent.
// nrows, nlines: the instance's rows and x-lines (the extents the
// bounds-checking build checks the three lines against).
template <int NC, bool COH = false>
__device__ __forceinline__ int bfp_plane_sum(const long long *__restrict__ qg, const int *__restrict__ eg, int nx, int ny, long sxy, int y,
                                             int zz, bool oka, bool okb, bool okd, int lane, long long (&te)[NC], long long (&to)[NC],
                                             long nrows, long nlines) {
  const long li = (long)zz * ny + y;
  const long row0 = (long)zz * sxy + (long)(y - 1) * nx;
  oka = oka && HPCG_IN(li - 1, 1, 0, nlines) && HPCG_IN(row0, nx, 0, nrows);
  okb = okb && HPCG_IN(li, 1, 0, nlines) && HPCG_IN(row0 + nx, nx, 0, nrows);
  okd = okd && HPCG_IN(li + 1, 1, 0, nlines) && HPCG_IN(row0 + 2 * nx, nx, 0, nrows);
  const int ea = oka ? ld_line<COH>(eg + li - 1) : kFxMinE;
  const int eb = okb ? ld_line<COH>(eg + li) : kFxMinE;
  const int ed = okd ? ld_line<COH>(eg + li + 1) : kFxMinE;
  const int et = max(max(ea, eb), ed);
  const long long *la = qg + (long)zz * sxy + (long)(y - 1) * nx;
  long long ae[NC], ao[NC], be[NC], bo[NC], de[NC], d_o[NC];
  ld_pairs_q<NC, COH>(la, oka, nx, lane, ae, ao);
  ld_pairs_q<NC, COH>(la + nx, okb, nx, lane, be, bo);
  ld_pairs_q<NC, COH>(la + 2 * nx, okd, nx, lane, de, d_o);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    te[c] = (shr_q(ae[c], et - ea) + shr_q(be[c], et - eb)) + shr_q(de[c], et - ed);
    to[c] = (shr_q(ao[c], et - ea) + shr_q(bo[c], et - eb)) + shr_q(d_o[c], et - ed);
  }
  return et;
}

// First row of coarse line (y/2, zz/2) of coarse instance table entry gc.
__device__ __forceinline__ long gc_base_of(const Inst &gc, int zz, int y) {
  return gc.off + (long)(zz >> 1) * gc.nx * gc.ny + (long)(y >> 1) * gc.nx;
}

// New value of a colour step from its exact sum t (scale S), stored at scale
// sout: t / 26 with four guard bits from the integer multiplier, rounded to
// nearest at S - 3 (8 t / 26 = 4 t / 13 is never halfway between integers,
// so the nearest is unique); with kappa, t * (1 / A_ii) in FP64 converted at
// sout.  |t| < 2^58 at S (the colour steps' scale bound), so t + 13 2^56 is
// positive and one unsigned multiply-high divides it; that offset is exactly
// 2^58 units at S - 3 (13 2^56 * 8/26), taken off the quotient.  (The offset
// touches only the high word, as does 2^58.)
__device__ __forceinline__ long long bfp_new_value(long long t, int S, int sout, const double *__restrict__ invd, long gi) {
  if (!invd) {
    constexpr unsigned long long kOff = 13ULL << 56, kOffQ = 1ULL << 58;
    const unsigned long long u = (unsigned long long)t + kOff;
    return (long long)(((__umul64hi(u, kDiv26) + 1ULL) >> 1) - kOffQ);
  }
  return fx_of(fx_to_double(t, S) * invd[gi], sout);
}

// Colour-pair runs of the V-cycle on the block-floating-point z (see
// k_gs_lines / k_gs_lines_fx for the run structure): `steps` >= 2 colour
// steps on the lines of class (py, pz), x parity pa first.  vmask: classes
// holding valid z (others read as zero).  rc (nullable): fused residual +
// injection into the FP64 right-hand side of level l+1 (runs of class (0,0)
// ending on even x).  zout (nullable): FP64 copy of the updated lines; with
// dpart, also the per-line partial sums of r.z (at [line], as the SpMV's p.Ap).
// zqc, zec, tabcp (nullable): the next coarser level's z and table, whose
// refinement into these (class (0,0)) lines is fused into this run.
// The work of block `blk` (warp wy of it) of a launch of k_gs_lines_bfp; COH:
// load with L2-coherent loads (data written earlier in the same launch).
// g1: the grid when count == 1 (a kernel parameter, so that a single grid's
// launch does not wait for a table load before its first data loads).
// REFINE_ONLY: stop after the fused refinement and store the refined line
// (hpcg_mg_stage's refinement stage; the V-cycle's kernels never set it).
template <int NC, bool COH, bool REFINE_ONLY = false>
__device__ __forceinline__ void gs_bfp_block(int blk, int wy, const Inst *__restrict__ tab, const Inst &g1, int count, int lpc, int zc,
                                             int py, int pz, int pa, int steps, int vmask, const double *__restrict__ r,
                                             long long *__restrict__ zq, int *__restrict__ ze, const double *__restrict__ invd,
                                             const CgState *__restrict__ st, const Inst *__restrict__ tabc, double *__restrict__ rc,
                                             const double *__restrict__ kap, double *__restrict__ zout, double *__restrict__ dpart,
                                             const long long *__restrict__ zqc, const int *__restrict__ zec,
                                             const Inst *__restrict__ tabcp) {
  const int ii = count == 1 ? 0 : find_inst<4>(tab, count, blk);
  const Inst g = count == 1 ? g1 : tab[ii];
  const int done = st ? ld_line<COH>(&st[ii].done) : 0;  // tested once the first loads are issued
  const int cy = (g.ny - py + 1) / 2, cz = (g.nz - pz + 1) / 2;
  const int nby = (half_up(g.ny) + lpc - 1) / lpc;
  const int lb = blk - g.blk_line;
  const int j = (lb % nby) * lpc + wy;
  const int m0 = (lb / nby) * zc;
  const int m1 = min(m0 + zc, cz);
  if (j >= cy || m0 >= m1) return;  // whole warp
  const int lane = threadIdx.x;
  const int y = 2 * j + py;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long sxy = (long)nx * ny;
  long long *qg = zq + g.off;
  int *eg = ze + g.poff;  // exponent of line (y, z) at eg[z ny + y]
  const double *rg = r + g.off;
  const bool vy = (vmask >> line_class(y + 1, pz)) & 1;  // lines (y +- 1, z) of the updated planes
  const bool ym = y - 1 >= 0 && vy, yp = y + 1 < ny && vy;
  const bool own_valid = (vmask >> line_class(y, pz)) & 1;
  const bool vyo = (vmask >> line_class(y + 1, pz + 1)) & 1;  // lines (y +- 1, z +- 1)
  const bool vy0 = (vmask >> line_class(y, pz + 1)) & 1;      // line (y, z +- 1)

  long long tpe[NC], tpo[NC];  // plane sum of the plane below the current one, at exponent Ec
  int Ec;
  {
    const int zz = 2 * m0 + pz - 1;
    const bool zin = zz >= 0;
    Ec = bfp_plane_sum<NC, COH>(qg, eg, nx, ny, sxy, y, zz, zin && y - 1 >= 0 && vyo, zin && vy0, zin && y + 1 < ny && vyo, lane, tpe,
                                tpo, g.n, (long)ny * nz);
  }
  if (done) return;  // converged instance: nothing changes
  for (int m = m0; m < m1; ++m) {
    const int zz = 2 * m + pz;
    const bool zin = zz + 1 < nz;
    long long te[NC], to[NC];
    const int et = bfp_plane_sum<NC, COH>(qg, eg, nx, ny, sxy, y, zz + 1, zin && y - 1 >= 0 && vyo, zin && vy0, zin && y + 1 < ny && vyo,
                                          lane, te, to, g.n, (long)ny * nz);
    const long li = (long)zz * ny + y;
    const long rowbase = (long)zz * sxy + (long)y * nx;
    // the own line (z, r, the FP64 copy, kappa fields, its exponent and r.z
    // partial) and the lines beside it, against the instance's extents
    if (!(HPCG_IN(rowbase, nx, 0, g.n) && HPCG_IN(li, 1, 0, (long)ny * nz))) continue;
    const bool ymc = ym && HPCG_IN(rowbase - nx, nx, 0, g.n) && HPCG_IN(li - 1, 1, 0, (long)ny * nz);
    const bool ypc = yp && HPCG_IN(rowbase + nx, nx, 0, g.n) && HPCG_IN(li + 1, 1, 0, (long)ny * nz);
    const int eu = ymc ? ld_line<COH>(eg + li - 1) : kFxMinE;
    const int ew = ypc ? ld_line<COH>(eg + li + 1) : kFxMinE;
    int eo = own_valid ? (COH ? __ldcg(eg + li) : eg[li]) : kFxMinE;
    long long ue[NC], uo[NC], we[NC], wo[NC], qe[NC], qo[NC];
    ld_pairs_q<NC, COH>(qg + rowbase - nx, ymc, nx, lane, ue, uo);
    ld_pairs_q<NC, COH>(qg + rowbase + nx, ypc, nx, lane, we, wo);
    if (own_valid && COH) {
      ld_pairs_q<NC, true>(qg + rowbase, true, nx, lane, qe, qo);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) {  // own line: written only by this warp
        const int xe = 64 * c + 2 * lane;
        const longlong2 v = (own_valid && xe < nx) ? *reinterpret_cast<const longlong2 *>(qg + rowbase + xe) : make_longlong2(0, 0);
        qe[c] = v.x;
        qo[c] = v.y;
      }
    }
    if (zqc) {
      // refinement z <- z + R^T z_c fused into this run (the first of the
      // post-smoother, on class (0,0) lines): coarse line (y/2, zz/2) adds to
      // the even x of this line, which moves to exponent max(e_f, e_c) + 1
      // (the arithmetic of prolong_bfp_line, in registers)
      const Inst gc = tabcp[ii];
      const long lic = (long)(zz >> 1) * gc.ny + (y >> 1);
      if (!(HPCG_IN(gc.off + lic * gc.nx, (nx + 1) / 2, gc.off, gc.off + gc.n) &&
            HPCG_IN(gc.poff + lic, 1, gc.poff, gc.poff + (long)gc.ny * gc.nz)))
        continue;
      const int e_c = ld_line<COH>(zec + gc.poff + lic);
      const int Sp = max(eo, e_c) + 1;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 64 * c + 2 * lane;
        const long long cv = xe < nx ? ld_line<COH>(zqc + gc.off + lic * gc.nx + (xe >> 1)) : 0;
        qe[c] = shr_q(qe[c], Sp - eo) + shr_q(cv, Sp - e_c);
        qo[c] = shr_q(qo[c], Sp - eo);
      }
      eo = (eo > kFxMaxE || e_c > kFxMaxE) ? kBfpNaN : Sp;
      if constexpr (REFINE_ONLY) {  // store the refined line at its exponent
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int xe = 64 * c + 2 * lane;
          if (xe < nx)
            *reinterpret_cast<longlong2 *>(qg + rowbase + xe) = eo == kBfpNaN ? make_longlong2(0, 0) : make_longlong2(qe[c], qo[c]);
        }
        if (lane == 0) eg[li] = eo;
        continue;  // the plane sums carried to the next plane are not needed without colour steps
      }
    }
    double rE[NC], rO[NC];
    ld_pairs_d<NC, COH>(rg + rowbase, nx, lane, rE, rO);
    // off-line sums: column sums at x (both planes beside + the two lines beside), then over x-1..x+1
    const int E = max(max(Ec, et), max(eu, ew));
    long long PE[NC], PO[NC];
    {
      long long ce[NC], co[NC], sh[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        ce[c] = (shr_q(tpe[c], E - Ec) + shr_q(te[c], E - et)) + (shr_q(ue[c], E - eu) + shr_q(we[c], E - ew));
        co[c] = (shr_q(tpo[c], E - Ec) + shr_q(to[c], E - et)) + (shr_q(uo[c], E - eu) + shr_q(wo[c], E - ew));
      }
      prev_of_i<NC>(co, sh, lane);  // column x-1 of an even x
#pragma unroll
      for (int c = 0; c < NC; ++c) PE[c] = (sh[c] + ce[c]) + co[c];
      next_of_i<NC>(ce, sh, lane);  // column x+1 of an odd x
#pragma unroll
      for (int c = 0; c < NC; ++c) PO[c] = (ce[c] + co[c]) + sh[c];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      tpe[c] = te[c];
      tpo[c] = to[c];
    }
    Ec = et;
    // the scale of the colour steps: every term below 2^56 there (r, the own
    // line, P whose 24 terms sum below 2^62.6 at E), with 3 more bits per
    // doubling of |1 / A_ii| above 1/2 (kappa), so that up to three steps of
    // new values stay below 2^58
    int er = kFxMinE;
#pragma unroll
    for (int c = 0; c < NC; ++c) er = max(er, max(fx_exp(rE[c]), fx_exp(rO[c])));
    er = warp_max(er);
    int idx = 0;
    if (invd) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 64 * c + 2 * lane;
        if (xe < nx) idx = max(idx, max(fx_exp(invd[g.off + rowbase + xe]), fx_exp(invd[g.off + rowbase + xe + 1])));
      }
      idx = warp_max(idx);
    }
    const int S = max(E + 5, max(er, eo)) + 2 + 3 * max(0, idx - 1021);
    const int sout = (invd && idx > 1018) ? S : S - 3;
    const bool bad = E > kFxMaxE || er > kFxMaxE || eo > kFxMaxE || S > kFxMaxE + 8;  // the same in every lane
    if (bad) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 64 * c + 2 * lane;
        if (xe < nx) {
          *reinterpret_cast<longlong2 *>(qg + rowbase + xe) = make_longlong2(0, 0);
          if (zout) *reinterpret_cast<double2 *>(zout + g.off + rowbase + xe) = make_double2(bfp_nan(), bfp_nan());
        }
      }
      if (lane == 0) eg[li] = kBfpNaN;
      if (zout && dpart && lane == 0) dpart[g.poff + li] = bfp_nan();
      if (rc) {
        const Inst gc = tabc[ii];
        const long cbase = gc.off + (long)(zz >> 1) * gc.nx * gc.ny + (long)(y >> 1) * gc.nx;
        if (HPCG_IN(cbase, (nx + 1) / 2, gc.off, gc.off + gc.n)) {
#pragma unroll
          for (int c = 0; c < NC; ++c)
            if (64 * c + 2 * lane < nx) rc[cbase + 32 * c + lane] = bfp_nan();
        }
      }
      continue;
    }
    long long re[NC], ro[NC], oE[NC], oO[NC], sE[NC], sO[NC], nb[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      re[c] = fx_of(rE[c], S) + shr_q(PE[c], S - E);
      ro[c] = fx_of(rO[c], S) + shr_q(PO[c], S - E);
      oE[c] = shr_q(qe[c], S - eo);
      oO[c] = shr_q(qo[c], S - eo);
      sE[c] = 0;
      sO[c] = 0;
    }
    const int down = S - sout;  // 3, or 0 with a large |1 / A_ii|
    for (int s = 0; s < steps; ++s) {
      const int q = (s & 1) ? 1 - pa : pa;
      if (q == 0) {
        prev_of_i<NC>(oO, nb, lane);  // O at x - 1 of every even x
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int xe = 64 * c + 2 * lane;
          if (xe < nx) {
            sE[c] = bfp_new_value((re[c] + nb[c]) + oO[c], S, sout, invd, g.off + rowbase + xe);
            oE[c] = shr_q(sE[c], down);
          }
        }
      } else {
        next_of_i<NC>(oE, nb, lane);  // E at x + 1 of every odd x
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int xo = 64 * c + 2 * lane + 1;
          if (xo < nx) {
            sO[c] = bfp_new_value((ro[c] + oE[c]) + nb[c], S, sout, invd, g.off + rowbase + xo);
            oO[c] = shr_q(sO[c], down);
          }
        }
      }
    }
    // Stored exponent: the new values are far below the scale bound sout they
    // were rounded at, so shift them up until the line's largest |q| reaches
    // bit 57 (exact).  The exponent then follows the data, and the next run's
    // scales, derived from its neighbours' exponents, stay tight.
    unsigned long long mag = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      mag |= sE[c] < 0 ? 0ULL - (unsigned long long)sE[c] : (unsigned long long)sE[c];
      mag |= sO[c] < 0 ? 0ULL - (unsigned long long)sO[c] : (unsigned long long)sO[c];
    }
    const unsigned mhi = __reduce_or_sync(kFull, (unsigned)(mag >> 32)), mlo = __reduce_or_sync(kFull, (unsigned)mag);
    const int lz = mhi ? __clz(mhi) : 32 + __clz(mlo);  // 64 for an all-zero line
    const int up = min(max(lz - 6, 0), sout - kFxMinE);
    double rz = 0.0;  // r.z over the line (FP64 output runs)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int xe = 64 * c + 2 * lane;
      if (xe < nx) {
        *reinterpret_cast<longlong2 *>(qg + rowbase + xe) =
            make_longlong2((long long)((unsigned long long)sE[c] << up), (long long)((unsigned long long)sO[c] << up));
        if (zout) {
          const double ze_ = fx_to_double(sE[c], sout), zo_ = fx_to_double(sO[c], sout);
          *reinterpret_cast<double2 *>(zout + g.off + rowbase + xe) = make_double2(ze_, zo_);
          rz += rE[c] * ze_ + rO[c] * zo_;
        }
      }
    }
    if (lane == 0) eg[li] = sout - up;
    if (zout && dpart) {  // per-line partial of r.z, exact tree on the integer pipe
      rz = warp_sum_fx(rz);
      if (lane == 0) dpart[g.poff + li] = rz;
    }
    if (rc && HPCG_IN(gc_base_of(tabc[ii], zz, y), (nx + 1) / 2, tabc[ii].off, tabc[ii].off + tabc[ii].n)) {
      // r - A z at the even points from the final values, exactly
      const Inst gc = tabc[ii];
      const long cbase = gc.off + (long)(zz >> 1) * gc.nx * gc.ny + (long)(y >> 1) * gc.nx;
      prev_of_i<NC>(oO, nb, lane);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 64 * c + 2 * lane;
        if (xe < nx) {
          const long long t = (re[c] + nb[c]) + oO[c];  // r + sum of the neighbours, scale S
          double res;
          if (!kap)  // 26 E at scale S - 3 is 13 E at S - 2; t at S is 4 t at S - 2
            res = fx_to_double(4 * t - 13 * sE[c], S - 2);
          else
            res = fx_to_double(t, S) - (26.0 + kap[g.off + rowbase + xe]) * fx_to_double(sE[c], sout);
          rc[cbase + 32 * c + lane] = res;
        }
      }
    }
  }
}

template <int NC>
__global__ void __launch_bounds__(256) k_gs_lines_bfp(const Inst *__restrict__ tab, int count, int lpc, int zc, int py, int pz, int pa,
                                                      int steps, int vmask, const double *__restrict__ r, long long *__restrict__ zq,
                                                      int *__restrict__ ze, const double *__restrict__ invd, const CgState *__restrict__ st,
                                                      const Inst *__restrict__ tabc, double *__restrict__ rc,
                                                      const double *__restrict__ kap, double *__restrict__ zout, double *__restrict__ dpart,
                                                      const long long *__restrict__ zqc, const int *__restrict__ zec,
                                                      const Inst *__restrict__ tabcp, const Inst g1) {
  pdl_enter();
  gs_bfp_block<NC, false>(blockIdx.x, threadIdx.y, tab, g1, count, lpc, zc, py, pz, pa, steps, vmask, r, zq, ze, invd, st, tabc, rc, kap,
                          zout, dpart, zqc, zec, tabcp);
}

// The same runs for a batch whose instances have x-lines of different lengths:
// each block belongs to one instance and takes the narrowest register window
// that holds that instance's lines (a launch sized for the widest line would
// leave most lanes of a short line idle).  Same arithmetic per line, so the
// same bits as k_gs_lines_bfp.
template <int NC>
__global__ void __launch_bounds__(256) k_gs_lines_bfp_batch(const Inst *__restrict__ tab, int count, int lpc, int zc, int py, int pz, int pa,
                                                            int steps, int vmask, const double *__restrict__ r, long long *__restrict__ zq,
                                                            int *__restrict__ ze, const double *__restrict__ invd,
                                                            const CgState *__restrict__ st, const Inst *__restrict__ tabc,
                                                            double *__restrict__ rc, const double *__restrict__ kap, double *__restrict__ zout,
                                                            double *__restrict__ dpart, const long long *__restrict__ zqc,
                                                            const int *__restrict__ zec, const Inst *__restrict__ tabcp, const Inst g1) {
  pdl_enter();
  const int nxi = tab[find_inst<4>(tab, count, blockIdx.x)].nx;
  if (nxi <= 64) {
    gs_bfp_block<1, false>(blockIdx.x, threadIdx.y, tab, g1, count, lpc, zc, py, pz, pa, steps, vmask, r, zq, ze, invd, st, tabc, rc, kap,
                           zout, dpart, zqc, zec, tabcp);
    return;
  }
  if constexpr (NC > 2) {
    if (nxi <= 128) {
      gs_bfp_block<2, false>(blockIdx.x, threadIdx.y, tab, g1, count, lpc, zc, py, pz, pa, steps, vmask, r, zq, ze, invd, st, tabc, rc,
                             kap, zout, dpart, zqc, zec, tabcp);
      return;
    }
  }
  gs_bfp_block<NC, false>(blockIdx.x, threadIdx.y, tab, g1, count, lpc, zc, py, pz, pa, steps, vmask, r, zq, ze, invd, st, tabc, rc, kap,
                          zout, dpart, zqc, zec, tabcp);
}

// The refinement fused into a post-smoother's first run, alone: the same
// block work as k_gs_lines_bfp (same launch shape and arguments), stopping
// once the refined class (0,0) line is stored (hpcg_mg_stage).
template <int NC>
__global__ void __launch_bounds__(256) k_gs_lines_bfp_refine(const Inst *__restrict__ tab, int count, int lpc, int zc, int py, int pz, int pa,
                                                             int steps, int vmask, const double *__restrict__ r, long long *__restrict__ zq,
                                                             int *__restrict__ ze, const double *__restrict__ invd,
                                                             const CgState *__restrict__ st, const Inst *__restrict__ tabc,
                                                             double *__restrict__ rc, const double *__restrict__ kap, double *__restrict__ zout,
                                                             double *__restrict__ dpart, const long long *__restrict__ zqc,
                                                             const int *__restrict__ zec, const Inst *__restrict__ tabcp, const Inst g1) {
  pdl_enter();
  gs_bfp_block<NC, false, true>(blockIdx.x, threadIdx.y, tab, g1, count, lpc, zc, py, pz, pa, steps, vmask, r, zq, ze, invd, st, tabc, rc,
                                kap, zout, dpart, zqc, zec, tabcp);
}

// ---------------------------------------------------------------------------
// Consecutive colour-pair runs whose line classes share the z parity pz (a
// symmetric sweep's runs in class order are [0 1], [2 3 2], [1 0]) in one
// launch.  A run on class (py, pz) reads, besides its own lines, the lines
// of the other y parity in its own planes and the lines of the planes
// between (parity 1 - pz), which no run of the group writes; so one block
// per plane of parity pz takes every line of that plane, run after run with
// a block barrier between runs, and no block reads what another block of the
// launch writes.  Each run is gs_bfp_block on virtual blocks of one plane
// (zc = 1) with L2-coherent loads (the lines written by the run before, by
// other warps of the block): the same arithmetic per line as one launch per
// run, so the same bits.  It saves a launch per run and reads the planes of
// parity 1 - pz once per group instead of once per run, but a block then
// takes a whole plane (no plane sum carried along z, loads through L2 only,
// one block per SM): one launch per run measured faster at every grid size,
// and the autotuner keeps the faster form per level.
struct PlaneRun {
  int cls, pa, steps, refine;  // refine: the coarser level's z is refined into this (class (0,0)) run
  double *rc;                  // fused residual + injection into the coarser level, or null
  double *zout, *dpart;        // FP64 z and per-line r.z partials (a class's last run), or null
};
constexpr int kPlaneMaxRuns = 3;
struct PlaneRuns {
  PlaneRun run[kPlaneMaxRuns];
  int nruns, vmask;  // vmask: line classes holding valid z before the first run
};
constexpr int kPlaneWarps = 16;  // warps (lines at a time) of a plane block

template <int NC>
__global__ void __launch_bounds__(32 * kPlaneWarps, 1)
    k_gs_planes_bfp(const Inst *__restrict__ tab, int count, const PlaneRuns R, const double *__restrict__ r, long long *__restrict__ zq,
                    int *__restrict__ ze, const double *__restrict__ invd, const CgState *__restrict__ st, const Inst *__restrict__ tabc,
                    const double *__restrict__ kap, const long long *__restrict__ zqc, const int *__restrict__ zec,
                    const Inst *__restrict__ tabcp, const Inst g1) {
  pdl_enter();
  const int nby = (half_up(g1.ny) + kPlaneWarps - 1) / kPlaneWarps;  // virtual blocks of kPlaneWarps lines per plane
  int vmask = R.vmask;
  for (int k = 0; k < R.nruns; ++k) {
    const PlaneRun &u = R.run[k];
    for (int yb = 0; yb < nby; ++yb)
      gs_bfp_block<NC, true>((int)blockIdx.x * nby + yb, threadIdx.y, tab, g1, count, kPlaneWarps, 1, u.cls & 1, (u.cls >> 1) & 1, u.pa,
                             u.steps, vmask, r, zq, ze, invd, st, u.rc ? tabc : nullptr, u.rc, kap, u.zout, u.dpart,
                             u.refine ? zqc : nullptr, u.refine ? zec : nullptr, u.refine ? tabcp : nullptr);
    vmask |= 1 << u.cls;
    __syncthreads();  // this run's lines are written before the next run reads them
  }
}

// ---------------------------------------------------------------------------
// The same colour-pair runs with each x-line split over W warps, one 64-point
// chunk each (x in [64k, 64k + 64), the lane holding the pair x = 64k + 2 lane,
// + 1).  One warp per line holds W pairs per lane (122 registers at W = 3: two
// 8-warp blocks per SM, each warp mostly waiting on its loads); one pair per
// lane needs far fewer registers, so more warps wait at a time.  What the
// one-warp kernel moves between chunks inside a warp goes through shared
// memory here: the column sums beside each chunk boundary, the line's largest
// exponents of r and 1 / A_ii, the value beside the boundary before each
// colour step, the OR of the magnitudes that sets the stored exponent, and
// the chunk partials of r.z (summed in chunk order, so that partial differs in
// rounding from the one-warp kernel's; z, its exponents and the restricted
// residual are the same bits).
//
// Every warp of a block passes the same sequence of block barriers (one after
// the column sums, one per colour step, one for the magnitudes, one for the
// r.z partials when they are asked for): the only early exits (no planes,
// converged instance) hold for the whole block, and lines past the grid's
// edge or with non-finite values skip loads, arithmetic and stores between
// barriers, never a barrier.
constexpr int kBfpSplitMaxLines = 8;  // lines per block (the autotuner's largest)

template <int W>
__global__ void __launch_bounds__(1024)
    k_gs_lines_bfp_split(const Inst *__restrict__ tab, int count, int lpc, int zc, int py, int pz, int pa, int steps, int vmask,
                         const double *__restrict__ r, long long *__restrict__ zq, int *__restrict__ ze, const double *__restrict__ invd,
                         const CgState *__restrict__ st, const Inst *__restrict__ tabc, double *__restrict__ rc,
                         const double *__restrict__ kap, double *__restrict__ zout, double *__restrict__ dpart,
                         const long long *__restrict__ zqc, const int *__restrict__ zec, const Inst *__restrict__ tabcp, const Inst g1) {
  pdl_enter();
  __shared__ long long s_ce[kBfpSplitMaxLines][W], s_co[kBfpSplitMaxLines][W];  // a chunk's first ce, last co
  __shared__ int s_er[kBfpSplitMaxLines][W], s_id[kBfpSplitMaxLines][W];         // a chunk's largest r and 1/A_ii exponents
  __shared__ long long s_o[kBfpSplitMaxLines][W], s_e[kBfpSplitMaxLines][W];     // a chunk's last odd, first even value
  __shared__ unsigned s_mhi[kBfpSplitMaxLines][W], s_mlo[kBfpSplitMaxLines][W];
  __shared__ double s_rz[kBfpSplitMaxLines][W];
  const int lane = threadIdx.x;
  const int k = threadIdx.y % W;   // chunk of the line
  const int wy = threadIdx.y / W;  // line of the block
  const int blk = blockIdx.x;
  const int ii = count == 1 ? 0 : find_inst<4>(tab, count, blk);
  const Inst g = count == 1 ? g1 : tab[ii];
  const int cy = (g.ny - py + 1) / 2, cz = (g.nz - pz + 1) / 2;
  const int nby = (half_up(g.ny) + lpc - 1) / lpc;
  const int lb = blk - g.blk_line;
  const int j = (lb % nby) * lpc + wy;
  const int m0 = (lb / nby) * zc;
  const int m1 = min(m0 + zc, cz);
  if (m0 >= m1) return;           // the whole block
  if (st && st[ii].done) return;  // the whole block: a block belongs to one instance
  const bool lok = j < cy;        // this line lies inside the grid
  const int y = lok ? 2 * j + py : py;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long sxy = (long)nx * ny;
  long long *qg = zq + g.off;
  int *eg = ze + g.poff;
  const double *rg = r + g.off;
  const int xe = 64 * k + 2 * lane;  // this lane's pair
  const bool xin = lok && xe < nx;
  const bool vy = (vmask >> line_class(y + 1, pz)) & 1;
  const bool ym = lok && y - 1 >= 0 && vy, yp = lok && y + 1 < ny && vy;
  const bool own_valid = lok && ((vmask >> line_class(y, pz)) & 1);
  const bool vyo = (vmask >> line_class(y + 1, pz + 1)) & 1;
  const bool vy0 = (vmask >> line_class(y, pz + 1)) & 1;
  auto ldq = [&](const long long *line, bool ok, long long &e, long long &o) {
    if (ok && xin) {
      const longlong2 v = __ldg(reinterpret_cast<const longlong2 *>(line + xe));
      e = v.x;
      o = v.y;
    } else {
      e = 0;
      o = 0;
    }
  };
  // sum over lines y-1, y, y+1 of plane zz at the largest of their exponents
  auto plane = [&](int zz, long long &te, long long &to) -> int {
    const bool zin = lok && zz >= 0 && zz < nz;
    const bool oka = zin && y - 1 >= 0 && vyo, okb = zin && vy0, okd = zin && y + 1 < ny && vyo;
    const long li = (long)zz * ny + y;
    const int ea = oka ? __ldg(eg + li - 1) : kFxMinE;
    const int eb = okb ? __ldg(eg + li) : kFxMinE;
    const int ed = okd ? __ldg(eg + li + 1) : kFxMinE;
    const int et = max(max(ea, eb), ed);
    const long long *la = qg + (long)zz * sxy + (long)(y - 1) * nx;
    long long ae, ao, be, bo, de, d_o;
    ldq(la, oka, ae, ao);
    ldq(la + nx, okb, be, bo);
    ldq(la + 2 * nx, okd, de, d_o);
    te = (shr_q(ae, et - ea) + shr_q(be, et - eb)) + shr_q(de, et - ed);
    to = (shr_q(ao, et - ea) + shr_q(bo, et - eb)) + shr_q(d_o, et - ed);
    return et;
  };
  long long tpe, tpo;
  int Ec = plane(2 * m0 + pz - 1, tpe, tpo);
  for (int m = m0; m < m1; ++m) {
    const int zz = 2 * m + pz;
    long long te, to;
    const int et = plane(zz + 1, te, to);
    const long li = (long)zz * ny + y;
    const long rowbase = (long)zz * sxy + (long)y * nx;
    const int eu = ym ? __ldg(eg + li - 1) : kFxMinE;
    const int ew = yp ? __ldg(eg + li + 1) : kFxMinE;
    int eo = own_valid ? eg[li] : kFxMinE;
    long long ue, uo, we, wo, qe = 0, qo = 0;
    ldq(qg + rowbase - nx, ym, ue, uo);
    ldq(qg + rowbase + nx, yp, we, wo);
    if (own_valid && xin) {  // own line: written only by this warp
      const longlong2 v = *reinterpret_cast<const longlong2 *>(qg + rowbase + xe);
      qe = v.x;
      qo = v.y;
    }
    if (zqc && lok) {  // refinement fused into this run (see gs_bfp_block)
      const Inst gc = tabcp[ii];
      const long lic = (long)(zz >> 1) * gc.ny + (y >> 1);
      const int e_c = __ldg(zec + gc.poff + lic);
      const int Sp = max(eo, e_c) + 1;
      const long long cv = xin ? __ldg(zqc + gc.off + lic * gc.nx + (xe >> 1)) : 0;
      qe = shr_q(qe, Sp - eo) + shr_q(cv, Sp - e_c);
      qo = shr_q(qo, Sp - eo);
      eo = (eo > kFxMaxE || e_c > kFxMaxE) ? kBfpNaN : Sp;
    }
    if (steps == 0) {  // refinement alone (hpcg_mg_stage), the same for every warp of the block: no barrier is skipped unevenly
      if (zqc && xin)
        *reinterpret_cast<longlong2 *>(qg + rowbase + xe) = eo == kBfpNaN ? make_longlong2(0, 0) : make_longlong2(qe, qo);
      if (zqc && lok && k == 0 && lane == 0) eg[li] = eo;
      continue;
    }
    double rE = 0.0, rO = 0.0;
    if (xin) {
      const double2 v = __ldg(reinterpret_cast<const double2 *>(rg + rowbase + xe));
      rE = v.x;
      rO = v.y;
    }
    const int E = max(max(Ec, et), max(eu, ew));
    const long long ce = (shr_q(tpe, E - Ec) + shr_q(te, E - et)) + (shr_q(ue, E - eu) + shr_q(we, E - ew));
    const long long co = (shr_q(tpo, E - Ec) + shr_q(to, E - et)) + (shr_q(uo, E - eu) + shr_q(wo, E - ew));
    tpe = te;
    tpo = to;
    Ec = et;
    int erc = max(kFxMinE, max(fx_exp(rE), fx_exp(rO)));
    erc = warp_max(erc);
    int idc = 0;
    if (invd) {
      if (xin) idc = max(fx_exp(invd[g.off + rowbase + xe]), fx_exp(invd[g.off + rowbase + xe + 1]));
      idc = warp_max(idc);
    }
    if (lane == 0) {
      s_ce[wy][k] = ce;
      s_er[wy][k] = erc;
      s_id[wy][k] = idc;
    }
    if (lane == 31) s_co[wy][k] = co;
    __syncthreads();
    int er = s_er[wy][0], idx = s_id[wy][0];
#pragma unroll
    for (int kk = 1; kk < W; ++kk) {
      er = max(er, s_er[wy][kk]);
      idx = max(idx, s_id[wy][kk]);
    }
    long long PE, PO;
    {
      long long sh = __shfl_up_sync(kFull, co, 1);
      if (lane == 0) sh = k > 0 ? s_co[wy][k - 1] : 0LL;  // column x-1 of an even x
      PE = (sh + ce) + co;
      sh = __shfl_down_sync(kFull, ce, 1);
      if (lane == 31) sh = k + 1 < W ? s_ce[wy][k + 1] : 0LL;  // column x+1 of an odd x
      PO = (ce + co) + sh;
    }
    const int S = max(E + 5, max(er, eo)) + 2 + 3 * max(0, idx - 1021);
    const int sout = (invd && idx > 1018) ? S : S - 3;
    const bool bad = E > kFxMaxE || er > kFxMaxE || eo > kFxMaxE || S > kFxMaxE + 8;  // the same for the whole line
    const bool act = lok && !bad;
    long long re = 0, ro = 0, oE = 0, oO = 0, sE = 0, sO = 0, nbl = 0;
    if (act) {
      re = fx_of(rE, S) + shr_q(PE, S - E);
      ro = fx_of(rO, S) + shr_q(PO, S - E);
      oE = shr_q(qe, S - eo);
      oO = shr_q(qo, S - eo);
    }
    const int down = S - sout;
    for (int s = 0; s < steps; ++s) {
      const int q = (s & 1) ? 1 - pa : pa;
      if (q == 0) {
        if (lane == 31) s_o[wy][k] = oO;
        __syncthreads();
        long long nb = __shfl_up_sync(kFull, oO, 1);
        if (lane == 0) nb = k > 0 ? s_o[wy][k - 1] : 0LL;  // O at x - 1 of this even x
        nbl = nb;
        if (act && xe < nx) {
          sE = bfp_new_value((re + nb) + oO, S, sout, invd, g.off + rowbase + xe);
          oE = shr_q(sE, down);
        }
      } else {
        if (lane == 0) s_e[wy][k] = oE;
        __syncthreads();
        long long nb = __shfl_down_sync(kFull, oE, 1);
        if (lane == 31) nb = k + 1 < W ? s_e[wy][k + 1] : 0LL;  // E at x + 1 of this odd x
        if (act && xe + 1 < nx) {
          sO = bfp_new_value((ro + oE) + nb, S, sout, invd, g.off + rowbase + xe + 1);
          oO = shr_q(sO, down);
        }
      }
    }
    // stored exponent: the line's largest |q| moved up to bit 57 (see gs_bfp_block)
    const unsigned long long mag = (sE < 0 ? 0ULL - (unsigned long long)sE : (unsigned long long)sE) |
                                   (sO < 0 ? 0ULL - (unsigned long long)sO : (unsigned long long)sO);
    const unsigned chi = __reduce_or_sync(kFull, (unsigned)(mag >> 32)), clo = __reduce_or_sync(kFull, (unsigned)mag);
    if (lane == 0) {
      s_mhi[wy][k] = chi;
      s_mlo[wy][k] = clo;
    }
    __syncthreads();
    unsigned mhi = 0, mlo = 0;
#pragma unroll
    for (int kk = 0; kk < W; ++kk) {
      mhi |= s_mhi[wy][kk];
      mlo |= s_mlo[wy][kk];
    }
    const int lz = mhi ? __clz(mhi) : 32 + __clz(mlo);
    const int up = min(max(lz - 6, 0), sout - kFxMinE);
    double rz = 0.0;
    if (lok && bad) {
      if (xin) {
        *reinterpret_cast<longlong2 *>(qg + rowbase + xe) = make_longlong2(0, 0);
        if (zout) *reinterpret_cast<double2 *>(zout + g.off + rowbase + xe) = make_double2(bfp_nan(), bfp_nan());
      }
      if (k == 0 && lane == 0) eg[li] = kBfpNaN;
      if (rc && xin) {
        const Inst gc = tabc[ii];
        rc[gc.off + (long)(zz >> 1) * gc.nx * gc.ny + (long)(y >> 1) * gc.nx + (xe >> 1)] = bfp_nan();
      }
      rz = bfp_nan();
    } else if (act) {
      if (xin) {
        *reinterpret_cast<longlong2 *>(qg + rowbase + xe) =
            make_longlong2((long long)((unsigned long long)sE << up), (long long)((unsigned long long)sO << up));
        if (zout) {
          const double ze_ = fx_to_double(sE, sout), zo_ = fx_to_double(sO, sout);
          *reinterpret_cast<double2 *>(zout + g.off + rowbase + xe) = make_double2(ze_, zo_);
          rz = rE * ze_ + rO * zo_;
        }
      }
      if (k == 0 && lane == 0) eg[li] = sout - up;
      if (rc && xin) {  // r - A z at the even points (the run ends on even x: nbl is the final O at x - 1)
        const Inst gc = tabc[ii];
        const long cbase = gc.off + (long)(zz >> 1) * gc.nx * gc.ny + (long)(y >> 1) * gc.nx;
        const long long t = (re + nbl) + oO;
        double res;
        if (!kap)
          res = fx_to_double(4 * t - 13 * sE, S - 2);
        else
          res = fx_to_double(t, S) - (26.0 + kap[g.off + rowbase + xe]) * fx_to_double(sE, sout);
        rc[cbase + (xe >> 1)] = res;
      }
    }
    if (zout && dpart) {  // per-line partial of r.z: lanes by a fixed shuffle tree, then chunks in order
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rz += __shfl_down_sync(kFull, rz, o);
      if (lane == 0) s_rz[wy][k] = rz;
      __syncthreads();
      if (lok && k == 0 && lane == 0) {
        double tot = s_rz[wy][0];
#pragma unroll
        for (int kk = 1; kk < W; ++kk) tot += s_rz[wy][kk];
        dpart[g.poff + li] = tot;
      }
    }
  }
}

// Refinement z_f <- z_f + R^T z_c on the block-floating-point vectors for
// coarse line wl (all instances' lines numbered in order), which feeds the
// even points of fine line (2 yc, 2 zc).  The fine line moves to exponent
// max(e_f, e_c) + 1, which keeps the sums below 2^58.  (The cluster kernel's
// refinement step; the per-launch V-cycle does the same inside the first
// post-smoother run.)
template <bool COH>
__device__ __forceinline__ void prolong_bfp_line(int wl, int lane, const Inst *__restrict__ tabf, const Inst *__restrict__ tabc, int count,
                                                 const long long *__restrict__ qc, const int *__restrict__ ec, long long *__restrict__ qf,
                                                 int *__restrict__ ef, const CgState *__restrict__ st) {
  const int ii = find_inst<5>(tabc, count, wl);
  if (st && st[ii].done) return;
  const Inst gc = tabc[ii], gf = tabf[ii];
  const int li = wl - gc.poff;
  const int yc = li % gc.ny, zc = li / gc.ny;
  const int yf = 2 * yc, zf = 2 * zc;
  const long lf = (long)zf * gf.ny + yf;
  const int e_f = COH ? __ldcg(ef + gf.poff + lf) : ef[gf.poff + lf];
  const int e_c = ld_line<COH>(ec + gc.poff + li);
  const bool bad = e_f > kFxMaxE || e_c > kFxMaxE;
  const int S = max(e_f, e_c) + 1;
  long long *fl = qf + gf.off + lf * gf.nx;
  const long long *cl = qc + gc.off + (long)li * gc.nx;
  for (int xe = 2 * lane; xe < gf.nx; xe += 64) {
    const longlong2 v = COH ? __ldcg(reinterpret_cast<const longlong2 *>(fl + xe)) : *reinterpret_cast<const longlong2 *>(fl + xe);
    const long long c = ld_line<COH>(cl + (xe >> 1));
    *reinterpret_cast<longlong2 *>(fl + xe) =
        bad ? make_longlong2(0, 0) : make_longlong2(shr_q(v.x, S - e_f) + shr_q(c, S - e_c), shr_q(v.y, S - e_f));
  }
  if (lane == 0) ef[gf.poff + lf] = bad ? kBfpNaN : S;
}


// ---------------------------------------------------------------------------
// The coarse end of the V-cycle in one launch of one thread-block cluster.
//
// On the smallest levels every run is a few microseconds of work, and one
// launch per run costs more than the work.  Here the levels first..last (at
// most kBfpTailRows rows each, one 64-point chunk per line) run their
// pre-smoothers (restriction fused into each level's last run), the coarsest
// level's smoother, then refinement and post-smoothers back up to `first`,
// inside one kernel whose kBfpTailCtas blocks form one cluster.  Runs are
// separated by the cluster's hardware barrier (release/acquire at cluster
// scope); data written earlier in the launch is read with L2-coherent loads.
// Every block executes the same barrier sequence, so the barrier always
// completes.  The arithmetic is that of k_gs_lines_bfp / prolong_bfp_line, so
// the results are the same bits as one launch per run.
constexpr int kBfpTailCtas = 16;
constexpr int kBfpTailWarps = 16;  // warps per block of the cluster kernel
constexpr long kBfpTailRows = 32768;

struct BfpTailLevel {
  const Inst *tab;
  Inst g1;                        // tab[0] (used when the handle has one grid)
  const double *r;                // right-hand side of the level (FP64)
  long long *zq;                  // block-floating-point z
  int *ze;
  const double *invd, *kap;       // kappa fields, or null
  double *rnext;                  // right-hand side of level + 1 (fused restriction), null on the coarsest
  const Inst *tabnext;
  int lpc, zc, nblk_line, nlines;  // colour-line launch shape and its blocks; x-lines of the level
  int npre, npost;
  TailRun pre[kTailRuns], post[kTailRuns];
};

struct BfpTailPlan {
  int first, last, count, pad;
  BfpTailLevel lv[kMaxLevels];
};

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int NC>
__device__ __forceinline__ void bfp_tail_runs(const BfpTailPlan &P, int l, const TailRun *runs, int nruns, bool from_zero, bool fuse,
                                              const CgState *st) {
  const BfpTailLevel &L = P.lv[l];
  int vmask = from_zero ? 0 : 0xF;
  const int vpb = kBfpTailWarps / L.lpc;  // virtual blocks per block step
  const int w = threadIdx.y;
  for (int k = 0; k < nruns; ++k) {
    const TailRun run = runs[k];
    double *rc = (fuse && k == nruns - 1) ? L.rnext : nullptr;
    if (w < vpb * L.lpc) {
      for (int base = blockIdx.x * vpb; base < L.nblk_line; base += gridDim.x * vpb) {
        const int vb = base + w / L.lpc;
        if (vb < L.nblk_line)
          gs_bfp_block<NC, true>(vb, w % L.lpc, L.tab, L.g1, P.count, L.lpc, L.zc, run.cls & 1, (run.cls >> 1) & 1, run.pa, run.steps,
                                 vmask, L.r, L.zq, L.ze, L.invd, st, rc ? L.tabnext : nullptr, rc, L.kap, nullptr, nullptr, nullptr,
                                 nullptr, nullptr);
      }
    }
    vmask |= 1 << run.cls;
    cluster_barrier();
  }
}

// Refinement of level l from level l+1 over every line of the coarse level.
__device__ __forceinline__ void bfp_tail_refine(const BfpTailPlan &P, int l, const CgState *st) {
  const BfpTailLevel &F = P.lv[l], &C = P.lv[l + 1];
  const int nw = gridDim.x * blockDim.y;
  for (int wl = blockIdx.x * blockDim.y + threadIdx.y; wl < C.nlines; wl += nw)
    prolong_bfp_line<true>(wl, threadIdx.x, F.tab, C.tab, P.count, C.zq, C.ze, F.zq, F.ze, st);
}

// stage_level < 0: the whole coarse end (levels first..last down, then back
// up to first).  Otherwise only stage `stage` (HPCG_STAGE_PRE / _REFINE /
// _POST of hpcg_mg_stage) of level stage_level, with the same arithmetic.
template <int NC>
__global__ void __launch_bounds__(32 * kBfpTailWarps) k_vcycle_tail_bfp(const BfpTailPlan *__restrict__ plan,
                                                                         const CgState *__restrict__ st, int stage_level, int stage) {
  pdl_enter();
  const BfpTailPlan &P = *plan;
  if (stage_level >= 0) {
    const int l = stage_level;
    if (stage == HPCG_STAGE_PRE) {
      bfp_tail_runs<NC>(P, l, P.lv[l].pre, P.lv[l].npre, true, l < P.last, st);
    } else {
      bfp_tail_refine(P, l, st);
      if (stage == HPCG_STAGE_POST) {
        cluster_barrier();
        bfp_tail_runs<NC>(P, l, P.lv[l].post, P.lv[l].npost, false, false, st);
      }
    }
    return;
  }
  for (int l = P.first; l <= P.last; ++l) bfp_tail_runs<NC>(P, l, P.lv[l].pre, P.lv[l].npre, true, l < P.last, st);
  for (int l = P.last - 1; l >= P.first; --l) {
    bfp_tail_refine(P, l, st);
    cluster_barrier();
    bfp_tail_runs<NC>(P, l, P.lv[l].post, P.lv[l].npost, false, false, st);
  }
}

// ---------------------------------------------------------------------------
// Level vectors into and out of block floating point, for inspection and for
// stage-by-stage checks of the V-cycle (hpcg_get_level_vectors,
// hpcg_set_level_vectors).  One warp per x-line of every instance of a level
// (`nlines` lines in all, numbered as the exponents are).

__global__ void __launch_bounds__(256) k_bfp_to_double(const Inst *__restrict__ tab, int count, long nlines, const long long *__restrict__ zq,
                                                       const int *__restrict__ ze, double *__restrict__ out) {
  const long wl = (long)blockIdx.x * blockDim.y + threadIdx.y;
  if (wl >= nlines) return;
  const int ii = count == 1 ? 0 : find_inst<5>(tab, count, (int)wl);
  const Inst g = tab[ii];
  const long base = g.off + (wl - g.poff) * g.nx;  // row of x = 0 on line (y, z): x + nx (y + ny z)
  const int e = ze[wl];
  for (int x = threadIdx.x; x < g.nx; x += 32) out[base + x] = e == kBfpNaN ? bfp_nan() : fx_to_double(zq[base + x], e);
}

// Each line gets the largest biased exponent of its values (at least
// kFxMinE) as its exponent and every value is truncated at that scale
// (|q| < 2^58, the largest with bit 57 set, as the colour runs store lines);
// a line holding a non-finite value or one beyond the range of the fixed-point
// sums reads as NaN.
__global__ void __launch_bounds__(256) k_bfp_from_double(const Inst *__restrict__ tab, int count, long nlines, const double *__restrict__ in,
                                                         long long *__restrict__ zq, int *__restrict__ ze) {
  const long wl = (long)blockIdx.x * blockDim.y + threadIdx.y;
  if (wl >= nlines) return;
  const int ii = count == 1 ? 0 : find_inst<5>(tab, count, (int)wl);
  const Inst g = tab[ii];
  const long base = g.off + (wl - g.poff) * g.nx;
  int emax = kFxMinE;
  for (int x = threadIdx.x; x < g.nx; x += 32) emax = max(emax, fx_exp(in[base + x]));
  emax = warp_max(emax);
  const bool bad = emax > kFxMaxE;  // includes Inf and NaN (biased exponent 2047)
  for (int x = threadIdx.x; x < g.nx; x += 32) zq[base + x] = bad ? 0LL : fx_of(in[base + x], emax);
  if (threadIdx.x == 0) ze[wl] = bad ? kBfpNaN : emax;
}

}  // namespace hpcg
