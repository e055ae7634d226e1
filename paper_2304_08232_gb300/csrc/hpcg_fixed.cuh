// hpcg_fixed.cuh -- FP64 line kernels whose neighbour sums run on the integer
// pipe in exact fixed point.
//
// On this GPU an FP64 add issues at 2 per SM per clock while 64-bit integer
// adds issue at about 64 (128 32-bit ops).  The colour-pair and SpMV line
// kernels spend most of their FP64 instructions summing neighbour values
// whose coefficients are all 1 (the off-diagonal entries are -1).  Here every
// value summed in one line-plane step is first mapped to a 64-bit integer
// against a common exponent bound E of that step,
//     q(v) = trunc(v * 2^(1080 - E)),  |v| < 2^(E - 1022)  =>  |q| < 2^58,
// the sums are formed exactly in int64 (at most 27 terms: |sum| < 2^63), and
// the result is converted back once (round to nearest, then an exact power-of-
// two scale).  E is the largest biased exponent among the values of the step
// (so |q| < 2^58 and 24 terms sum below 2^63); truncating each term costs at
// most 2^-5 ulp of the largest value, so a 24-term sum is within one ulp of it:
// tighter than the FP64 summation it replaces.  E is raised to at least 64, so
// values below 2^-1016 in magnitude count as zero (an absolute error under
// 1e-305); a warp whose step holds huge (E > 2000) or non-finite values
// continues with FP64 sums, so NaN and Inf still propagate.  The colour-step
// update (r + sum) / A_ii stays in FP64 (on this GPU the integer pipe, not
// the FP64 pipe, limits these kernels).  Without kappa the SpMV's 27 x - S is
// formed in fixed point too: its only rounding is the final conversion, and
// it issues no FP64 instruction.
#pragma once
#include "hpcg_lines.cuh"

namespace hpcg {

template <int NC>
__device__ __forceinline__ void prev_of_i(const long long (&v)[NC], long long (&out)[NC], int lane) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const long long up = __shfl_up_sync(kFull, v[c], 1);
    const long long last = __shfl_sync(kFull, v[c > 0 ? c - 1 : 0], 31);
    out[c] = lane == 0 ? (c > 0 ? last : 0LL) : up;
  }
}
template <int NC>
__device__ __forceinline__ void next_of_i(const long long (&v)[NC], long long (&out)[NC], int lane) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const long long dn = __shfl_down_sync(kFull, v[c], 1);
    const long long first = __shfl_sync(kFull, v[c + 1 < NC ? c + 1 : c], 0);
    out[c] = lane == 31 ? (c + 1 < NC ? first : 0LL) : dn;
  }
}

// Raw values of one x-line (parity split), zero where absent or invalid.
template <int NC>
__device__ __forceinline__ void load_line(const double *__restrict__ line, bool ok, int nx, int lane, double (&e)[NC], double (&o)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int xe = 2 * (lane + 32 * c), xo = xe + 1;
    e[c] = (ok && xe < nx) ? __ldg(line + xe) : 0.0;
    o[c] = (ok && xo < nx) ? __ldg(line + xo) : 0.0;
  }
}

// A read-only load the compiler may not merge with an earlier one: the
// fixed-point kernels read each value twice (exponent pass, conversion pass)
// rather than keep it in a register between the passes.
__device__ __forceinline__ double ld_nc_again(const double *p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

template <int NC>
__device__ __forceinline__ int max_exp3(const double (&a)[NC], const double (&b)[NC], int m) {
#pragma unroll
  for (int c = 0; c < NC; ++c) m = max(m, max(fx_exp(a[c]), fx_exp(b[c])));
  return m;
}

// The own line's values (E_ at even x, O_ at odd x; zero where the line holds
// no valid data yet) and the right-hand side there.
template <int NC>
__device__ __forceinline__ void load_own(const double *__restrict__ zg, const double *__restrict__ rg, long rowbase, int nx, int lane,
                                         bool own_valid, double (&E_)[NC], double (&O_)[NC], double (&rE)[NC], double (&rO)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int xe = 2 * (lane + 32 * c), xo = xe + 1;
    E_[c] = (xe < nx && own_valid) ? zg[rowbase + xe] : 0.0;
    O_[c] = (xo < nx && own_valid) ? zg[rowbase + xo] : 0.0;
    rE[c] = xe < nx ? rg[rowbase + xe] : 0.0;
    rO[c] = xo < nx ? rg[rowbase + xo] : 0.0;
  }
}

// Colour steps along the own line (FP64), the stores, and the fused
// residual + injection: the part of k_gs_lines after the off-line sums.
// E_, O_, rE, rO hold the own line as load_own reads it.
template <int NC>
__device__ __forceinline__ void pair_steps(const Inst &g, int ii, int zz, int y, int lane, int pa, int steps, bool own_valid,
                                           const double (&PE)[NC], const double (&PO)[NC], double (&E_)[NC], double (&O_)[NC],
                                           const double (&rE)[NC], const double (&rO)[NC], double *__restrict__ zg,
                                           const double *__restrict__ invd, const Inst *__restrict__ tabc, double *__restrict__ rc,
                                           const double *__restrict__ kap) {
  const int nx = g.nx;
  const long rowbase = (long)zz * nx * g.ny + (long)y * nx;
  double nb[NC];
  for (int s = 0; s < steps; ++s) {
    const int q = (s & 1) ? 1 - pa : pa;
    if (q == 0) {
      prev_of<double, NC>(O_, nb, lane);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 2 * (lane + 32 * c);
        if (xe < nx) {
          const double id = invd ? invd[g.off + rowbase + xe] : 1.0 / 26.0;
          E_[c] = (((rE[c] + PE[c]) + nb[c]) + O_[c]) * id;
        }
      }
    } else {
      next_of<double, NC>(E_, nb, lane);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xo = 2 * (lane + 32 * c) + 1;
        if (xo < nx) {
          const double id = invd ? invd[g.off + rowbase + xo] : 1.0 / 26.0;
          O_[c] = (((rO[c] + PO[c]) + E_[c]) + nb[c]) * id;
        }
      }
    }
  }
  const bool write_e = steps > 1 || !own_valid || pa == 0;
  const bool write_o = steps > 1 || !own_valid || pa == 1;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int xe = 2 * (lane + 32 * c), xo = xe + 1;
    if (write_e && xe < nx) zg[rowbase + xe] = E_[c];
    if (write_o && xo < nx) zg[rowbase + xo] = O_[c];
  }
  if (rc) {
    const Inst gc = tabc[ii];
    const long cbase = gc.off + (long)(zz >> 1) * gc.nx * gc.ny + (long)(y >> 1) * gc.nx;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int xe = 2 * (lane + 32 * c);
      if (xe < nx) {
        const double d = kap ? 26.0 + kap[g.off + rowbase + xe] : 26.0;
        const double nbs = (PE[c] + nb[c]) + O_[c];
        rc[cbase + (xe >> 1)] = rE[c] - (d * E_[c] - nbs);
      }
    }
  }
}

template <int NC>
__device__ __forceinline__ void pair_update(const Inst &g, int ii, int zz, int y, int lane, int pa, int steps, bool own_valid,
                                            const double (&PE)[NC], const double (&PO)[NC], const double *__restrict__ rg,
                                            double *__restrict__ zg, const double *__restrict__ invd, const Inst *__restrict__ tabc,
                                            double *__restrict__ rc, const double *__restrict__ kap) {
  double E_[NC], O_[NC], rE[NC], rO[NC];
  load_own<NC>(zg, rg, (long)zz * g.nx * g.ny + (long)y * g.nx, g.nx, lane, own_valid, E_, O_, rE, rO);
  pair_steps<NC>(g, ii, zz, y, lane, pa, steps, own_valid, PE, PO, E_, O_, rE, rO, zg, invd, tabc, rc, kap);
}

// Arithmetic right shift that saturates for shifts of 64 or more.
__device__ __forceinline__ long long shr_fx(long long v, int d) { return d < 64 ? v >> d : (v < 0 ? -1LL : 0LL); }

// ceil(2^68 / 26): for 0 <= a < 2^64, floor(a * kDiv26 / 2^64) equals a * 16/26
// to within one unit (the multiplier's relative excess is below 2^-63).
constexpr unsigned long long kDiv26 = 11351842506898185610ULL;

template <int NC>
__device__ __forceinline__ void prev_of_int(const int (&v)[NC], int (&out)[NC], int lane) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int up = __shfl_up_sync(kFull, v[c], 1);
    const int last = __shfl_sync(kFull, v[c > 0 ? c - 1 : 0], 31);
    out[c] = lane == 0 ? (c > 0 ? last : v[c]) : up;
  }
}
template <int NC>
__device__ __forceinline__ void next_of_int(const int (&v)[NC], int (&out)[NC], int lane) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int dn = __shfl_down_sync(kFull, v[c], 1);
    const int first = __shfl_sync(kFull, v[c + 1 < NC ? c + 1 : c], 0);
    out[c] = lane == 31 ? (c + 1 < NC ? first : v[c]) : dn;
  }
}

// Colour-pair kernel (see k_gs_lines) with the off-line sums in fixed point.
// Every lane scales each of its 32-wide chunks (the x pair 2k, 2k+1) on its
// own, so only one chunk's raw values are live at a time.  Each plane sum T
// (over y-1..y+1) is kept at the scale of its own three lines; a step adds T
// below, T above and the two lines beside at the largest scale of the four,
// and the x-window sum aligns the three columns it adds to their largest
// scale.  Every scale depends only on the values summed, never on how planes
// are grouped into blocks, so results do not depend on the launch shape.
template <int NC>
__global__ void __launch_bounds__(256) k_gs_lines_fx(const Inst *__restrict__ tab, int count, int lpc, int zc, int py, int pz, int pa,
                                                     int steps, int vmask, const double *__restrict__ r, double *__restrict__ z,
                                                     const double *__restrict__ invd, const CgState *__restrict__ st,
                                                     const Inst *__restrict__ tabc, double *__restrict__ rc,
                                                     const double *__restrict__ kap) {
  pdl_enter();
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
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long sxy = (long)nx * ny;
  double *zg = z + g.off;
  const double *rg = r + g.off;
  const bool vy = (vmask >> line_class(y + 1, pz)) & 1;       // lines (y +- 1, z) of the updated planes
  const bool ym = y - 1 >= 0 && vy, yp = y + 1 < ny && vy;
  const bool own_valid = (vmask >> line_class(y, pz)) & 1;
  const bool vyo = (vmask >> line_class(y + 1, pz + 1)) & 1;  // lines (y +- 1, z +- 1)
  const bool vy0 = (vmask >> line_class(y, pz + 1)) & 1;      // line (y, z +- 1)

  int m = m0;
  long long tpe[NC], tpo[NC];  // fixed-point plane sums of the plane below the current one
  int Ec[NC];                  // their per-chunk scale
  bool fixed;
  {
    const int zz = 2 * m0 + pz - 1;
    const bool zin = zz >= 0;
    const double *la = zg + (long)zz * sxy + (long)(y - 1) * nx;
    const bool oka = zin && y - 1 >= 0 && vyo, okb = zin && vy0, okd = zin && y + 1 < ny && vyo;
    bool bad = false;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int xe = 64 * c + 2 * lane, xo = xe + 1;
      const bool ie = xe < nx, io = xo < nx;
      const double ae = (oka && ie) ? __ldg(la + xe) : 0.0, ao = (oka && io) ? __ldg(la + xo) : 0.0;
      const double be = (okb && ie) ? __ldg(la + nx + xe) : 0.0, bo = (okb && io) ? __ldg(la + nx + xo) : 0.0;
      const double de = (okd && ie) ? __ldg(la + 2 * nx + xe) : 0.0, d_o = (okd && io) ? __ldg(la + 2 * nx + xo) : 0.0;
      const int e = max(max(max(fx_exp(ae), fx_exp(ao)), max(fx_exp(be), fx_exp(bo))), max(max(fx_exp(de), fx_exp(d_o)), kFxMinE));
      bad |= e > kFxMaxE;
      Ec[c] = e;
      tpe[c] = (fx_of(ae, e) + fx_of(be, e)) + fx_of(de, e);
      tpo[c] = (fx_of(ao, e) + fx_of(bo, e)) + fx_of(d_o, e);
    }
    fixed = !__any_sync(kFull, bad);
  }
  if (fixed) {
    for (; m < m1; ++m) {
      const int zz = 2 * m + pz;
      const bool zin = zz + 1 < nz;
      const double *la = zg + (long)(zz + 1) * sxy + (long)(y - 1) * nx;
      const double *vm = zg + (long)zz * sxy + (long)(y - 1) * nx;
      const bool oka = zin && y - 1 >= 0 && vyo, okb = zin && vy0, okd = zin && y + 1 < ny && vyo;
      long long ce[NC], co[NC], nte[NC], nto[NC];
      int En[NC], Et[NC];
      bool bad = false;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 64 * c + 2 * lane, xo = xe + 1;
        const bool ie = xe < nx, io = xo < nx;
        const double ae = (oka && ie) ? __ldg(la + xe) : 0.0, ao = (oka && io) ? __ldg(la + xo) : 0.0;
        const double be = (okb && ie) ? __ldg(la + nx + xe) : 0.0, bo = (okb && io) ? __ldg(la + nx + xo) : 0.0;
        const double de = (okd && ie) ? __ldg(la + 2 * nx + xe) : 0.0, d_o = (okd && io) ? __ldg(la + 2 * nx + xo) : 0.0;
        const double ue = (ym && ie) ? __ldg(vm + xe) : 0.0, uo = (ym && io) ? __ldg(vm + xo) : 0.0;
        const double we = (yp && ie) ? __ldg(vm + 2 * nx + xe) : 0.0, wo = (yp && io) ? __ldg(vm + 2 * nx + xo) : 0.0;
        // plane sum above at the scale of its own three lines
        const int et = max(max(max(max(fx_exp(ae), fx_exp(ao)), max(fx_exp(be), fx_exp(bo))), max(fx_exp(de), fx_exp(d_o))), kFxMinE);
        // the step's scale: both plane sums and the two lines beside
        const int e = max(max(et, Ec[c]), max(max(fx_exp(ue), fx_exp(uo)), max(fx_exp(we), fx_exp(wo))));
        bad |= e > kFxMaxE;
        const long long te = (fx_of(ae, et) + fx_of(be, et)) + fx_of(de, et);
        const long long to = (fx_of(ao, et) + fx_of(bo, et)) + fx_of(d_o, et);
        ce[c] = (shr_fx(tpe[c], e - Ec[c]) + shr_fx(te, e - et)) + (fx_of(ue, e) + fx_of(we, e));  // off-line column sums at x
        co[c] = (shr_fx(tpo[c], e - Ec[c]) + shr_fx(to, e - et)) + (fx_of(uo, e) + fx_of(wo, e));
        nte[c] = te;
        nto[c] = to;
        En[c] = e;
        Et[c] = et;
      }
      if (__any_sync(kFull, bad)) {  // huge or non-finite values: FP64 from this plane on
        fixed = false;
        break;
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        tpe[c] = nte[c];
        tpo[c] = nto[c];
        Ec[c] = Et[c];
      }
      long long PEf[NC], POf[NC];
      int Ee[NC], Eo[NC];
      {
        long long sh[NC];
        int Es[NC];
        prev_of_i<NC>(co, sh, lane);  // column x-1 of an even x
        prev_of_int<NC>(En, Es, lane);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int E3 = max(Es[c], En[c]);
          PEf[c] = (shr_fx(sh[c], E3 - Es[c]) + shr_fx(ce[c], E3 - En[c])) + shr_fx(co[c], E3 - En[c]);
          Ee[c] = E3;
        }
        next_of_i<NC>(ce, sh, lane);  // column x+1 of an odd x
        next_of_int<NC>(En, Es, lane);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int E3 = max(Es[c], En[c]);
          POf[c] = (shr_fx(ce[c], E3 - En[c]) + shr_fx(co[c], E3 - En[c])) + shr_fx(sh[c], E3 - Es[c]);
          Eo[c] = E3;
        }
      }
      {
        double PE[NC], PO[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          PE[c] = fx_to_double(PEf[c], Ee[c]);
          PO[c] = fx_to_double(POf[c], Eo[c]);
        }
        pair_update<NC>(g, ii, zz, y, lane, pa, steps, own_valid, PE, PO, rg, zg, invd, tabc, rc, kap);
      }
    }
  }
  // FP64 sums for the remaining planes (rare: huge or non-finite values)
  if (m < m1) {
    double tdpe[NC], tdpo[NC];
    tsum2<double, NC, false>(zg, nx, ny, nz, y, 2 * m + pz - 1, lane, tdpe, tdpo, vmask);
    for (; m < m1; ++m) {
      const int zz = 2 * m + pz;
      double tne[NC], tno[NC], PE[NC], PO[NC], ce[NC], co[NC], sh[NC];
      tsum2<double, NC, false>(zg, nx, ny, nz, y, zz + 1, lane, tne, tno, vmask);
      const double *lm = zg + (long)zz * sxy + (long)(y - 1) * nx;
      const double *lp = lm + 2 * nx;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int xe = 2 * (lane + 32 * c), xo = xe + 1;
        double ve = 0.0, vo = 0.0;
        if (xe < nx) ve = (ym ? __ldg(lm + xe) : 0.0) + (yp ? __ldg(lp + xe) : 0.0);
        if (xo < nx) vo = (ym ? __ldg(lm + xo) : 0.0) + (yp ? __ldg(lp + xo) : 0.0);
        ce[c] = (tdpe[c] + tne[c]) + ve;
        co[c] = (tdpo[c] + tno[c]) + vo;
      }
      prev_of<double, NC>(co, sh, lane);
#pragma unroll
      for (int c = 0; c < NC; ++c) PE[c] = (sh[c] + ce[c]) + co[c];
      next_of<double, NC>(ce, sh, lane);
#pragma unroll
      for (int c = 0; c < NC; ++c) PO[c] = (ce[c] + co[c]) + sh[c];
      pair_update<NC>(g, ii, zz, y, lane, pa, steps, own_valid, PE, PO, rg, zg, invd, tabc, rc, kap);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        tdpe[c] = tne[c];
        tdpo[c] = tno[c];
      }
    }
  }
}

// Raw values of one x-line, x = lane + 32c (SpMV layout), zero where absent.
template <int NC>
__device__ __forceinline__ void load_row(const double *__restrict__ line, bool ok, int nx, int lane, double (&v)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int x = lane + 32 * c;
    v[c] = (ok && x < nx) ? __ldg(line + x) : 0.0;
  }
}

// Row layout (x = lane + 32c) versions of the two passes.
template <int NC>
__device__ __forceinline__ int row_max_exp(const double *__restrict__ line, bool ok, int nx, int lane, int m) {
  if (!ok) return m;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int x = lane + 32 * c;
    if (x < nx) m = max(m, fx_exp(ld_nc_again(line + x)));
  }
  return m;
}
template <int NC>
__device__ __forceinline__ void row_add_fx(const double *__restrict__ line, bool ok, int nx, int lane, int E, long long (&acc)[NC]) {
  if (!ok) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int x = lane + 32 * c;
    if (x < nx) acc[c] += fx_of(ld_nc_again(line + x), E);
  }
}

template <int NC>
__device__ __forceinline__ int max_exp_row(const double (&a)[NC], int m) {
#pragma unroll
  for (int c = 0; c < NC; ++c) m = max(m, fx_exp(a[c]));
  return m;
}

template <int NC>
__device__ __forceinline__ void line_neighbours_i(const long long (&v)[NC], long long (&vl)[NC], long long (&vr)[NC], int lane) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const long long up = __shfl_up_sync(kFull, v[c], 1);
    const long long prev_last = __shfl_sync(kFull, v[c > 0 ? c - 1 : 0], 31);
    vl[c] = lane == 0 ? (c > 0 ? prev_last : 0LL) : up;
    const long long dn = __shfl_down_sync(kFull, v[c], 1);
    const long long next_first = __shfl_sync(kFull, v[c + 1 < NC ? c + 1 : c], 0);
    vr[c] = lane == 31 ? (c + 1 < NC ? next_first : 0LL) : dn;
  }
}

// y = A x (Mode 0) or y = b - A x (Mode 1) over every x-line (see
// k_spmv_lines): A x = (27 + kappa) x - S with the 27-point box sum S formed
// exactly in fixed point (plane sums over y, then over z, then over x).
template <int NC, int Mode>
__global__ void __launch_bounds__(256) k_spmv_lines_fx(const Inst *__restrict__ tab, int count, int lpc, int zc, const double *__restrict__ x,
                                                       const double *__restrict__ b, double *__restrict__ y, const double *__restrict__ kap,
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
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long sxy = (long)nx * ny;
  const double *xg = x + g.off;
  if (skip) {
    if (partials && yy < ny && lane == 0)
      for (int zz = z0; zz < z1; ++zz) partials[g.poff + (long)zz * ny + yy] = 0.0;
    return;
  }
  if (yy >= ny || z0 >= z1) return;
  const bool ym = yy - 1 >= 0, yp = yy + 1 < ny;
  // plane sums over y-1..y+1 of planes z0-1 and z0; each plane sum in fixed
  // point at the scale of its own three lines (e0, e1), so that the result
  // does not depend on how planes are grouped into blocks
  long long t0[NC], t1[NC];
  double d0[NC], d1[NC];  // the same in FP64 once a warp leaves the fixed point
  int e0, e1;
  bool fixed;
  {
    const double *l = xg + (long)(z0 - 1) * sxy + (long)(yy - 1) * nx;
    const bool za = z0 - 1 >= 0;
    int e = row_max_exp<NC>(l, za && ym, nx, lane, 0);
    e = row_max_exp<NC>(l + nx, za, nx, lane, e);
    e = row_max_exp<NC>(l + 2 * nx, za && yp, nx, lane, e);
    e0 = max(warp_max(e), kFxMinE);
    e = row_max_exp<NC>(l + sxy, ym, nx, lane, 0);
    e = row_max_exp<NC>(l + sxy + nx, true, nx, lane, e);
    e = row_max_exp<NC>(l + sxy + 2 * nx, yp, nx, lane, e);
    e1 = max(warp_max(e), kFxMinE);
    fixed = e0 <= kFxMaxE && e1 <= kFxMaxE;
    if (fixed) {
#pragma unroll
      for (int c = 0; c < NC; ++c) t0[c] = t1[c] = 0;
      row_add_fx<NC>(l, za && ym, nx, lane, e0, t0);
      row_add_fx<NC>(l + nx, za, nx, lane, e0, t0);
      row_add_fx<NC>(l + 2 * nx, za && yp, nx, lane, e0, t0);
      row_add_fx<NC>(l + sxy, ym, nx, lane, e1, t1);
      row_add_fx<NC>(l + sxy + nx, true, nx, lane, e1, t1);
      row_add_fx<NC>(l + sxy + 2 * nx, yp, nx, lane, e1, t1);
    } else {
      tsum<double, NC>(xg, nx, ny, nz, yy, z0 - 1, lane, d0);
      tsum<double, NC>(xg, nx, ny, nz, yy, z0, lane, d1);
    }
  }
  for (int zz = z0; zz < z1; ++zz) {
    const double *l = xg + (long)(zz + 1) * sxy + (long)(yy - 1) * nx;
    const bool zin = zz + 1 < nz;
    double S[NC];
    long long Sf[NC];  // the box sums in fixed point at scale SE while the warp stays fixed
    int SE = 0;
    bool sfix = false;
    if (fixed) {
      int e = row_max_exp<NC>(l, zin && ym, nx, lane, 0);
      e = row_max_exp<NC>(l + nx, zin, nx, lane, e);
      e = row_max_exp<NC>(l + 2 * nx, zin && yp, nx, lane, e);
      const int e2 = max(warp_max(e), kFxMinE);
      if (e2 > kFxMaxE) {  // huge or non-finite values: FP64 from here on
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          d0[c] = fx_to_double(t0[c], e0);
          d1[c] = fx_to_double(t1[c], e1);
        }
        fixed = false;
      } else {
        const int E = max(max(e0, e1), e2);
        long long u[NC], t2[NC], ul[NC], ur[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) t2[c] = 0;
        row_add_fx<NC>(l, zin && ym, nx, lane, e2, t2);
        row_add_fx<NC>(l + nx, zin, nx, lane, e2, t2);
        row_add_fx<NC>(l + 2 * nx, zin && yp, nx, lane, e2, t2);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          u[c] = (shr_fx(t0[c], E - e0) + shr_fx(t1[c], E - e1)) + shr_fx(t2[c], E - e2);
          t0[c] = t1[c];
          t1[c] = t2[c];
        }
        e0 = e1;
        e1 = e2;
        line_neighbours_i<NC>(u, ul, ur, lane);
#pragma unroll
        for (int c = 0; c < NC; ++c) Sf[c] = (ul[c] + u[c]) + ur[c];
        SE = E;
        sfix = true;
      }
    }
    if (!fixed) {
      double t2[NC], u[NC], ul[NC], ur[NC];
      tsum<double, NC>(xg, nx, ny, nz, yy, zz + 1, lane, t2);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        u[c] = (d0[c] + d1[c]) + t2[c];
        d0[c] = d1[c];
        d1[c] = t2[c];
      }
      line_neighbours<double, NC>(u, ul, ur, lane);
#pragma unroll
      for (int c = 0; c < NC; ++c) S[c] = (ul[c] + u[c]) + ur[c];
    }
    const long rowbase = (long)zz * sxy + (long)yy * nx;
    double dotv = 0.0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int xx = lane + 32 * c;
      if (xx < nx) {
        const double xi = xg[rowbase + xx];
        const long gi = g.off + rowbase + xx;
        double ax;
        if (sfix && !kap) {
          // 27 x - S exactly at scale SE + 1 (|27 x| and |S| < 27 2^57 there), one rounding
          ax = fx_to_double(27 * fx_of(xi, SE + 1) - (Sf[c] >> 1), SE + 1);
        } else {
          const double d1 = kap ? 27.0 + kap[gi] : 27.0;
          ax = d1 * xi - (sfix ? fx_to_double(Sf[c], SE) : S[c]);
        }
        const double out = Mode == 0 ? ax : b[gi] - ax;
        y[gi] = out;
        if (partials) dotv += xi * out;
      }
    }
    if (partials) {  // fixed shuffle tree over the lanes of this line
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dotv += __shfl_down_sync(kFull, dotv, o);
      if (lane == 0) partials[g.poff + (long)zz * ny + yy] = dotv;
    }
  }
}

}  // namespace hpcg
