// hpcg_tail.cuh -- the coarse end of the V-cycle (Listing 1 on the smallest
// levels) in one persistent cooperative launch.
//
// On the small levels every colour-pair run is a few microseconds of work, so
// one kernel launch per run would be dominated by launch latency.  The tail
// kernel instead runs, for levels first..last, the pre-smoother runs (with the
// residual injection fused into each level's last run), the coarsest level's
// smoother, then the refinement + post-smoother runs back up, all in one
// launch.  Phases are separated by a grid-wide barrier; every block takes the
// virtual blocks (line groups) of a phase round-robin.  The launch is
// cooperative, so all blocks are resident and the barrier cannot deadlock.
// Every wait is bounded: after `limit` clock cycles a block records a timeout
// in *err, marks every instance's CG state done with HPCG_ERR_TIMEOUT and
// leaves; the other blocks see *err and leave too.
#pragma once
#include "hpcg_lines.cuh"

namespace hpcg {

constexpr int kTailRuns = 40;
constexpr int kTailThreadsY = 8;  // warps per block of the tail kernel

struct TailRun {
  signed char cls, pa, steps, pad;
};

struct TailLevel {
  const Inst *tab;      // device instance table of the level
  void *r, *z;          // level vectors in the tail's precision
  const void *invd, *kap;
  int lpc, zc, nvb;     // colour-line launch shape and its virtual blocks (all instances)
  int npre, npost;
  int fuse;             // 1: the last pre run (class (0,0), even x last) restricts into level+1
  TailRun pre[kTailRuns], post[kTailRuns];
};

struct TailPlan {
  int first, last, count, pad;
  TailLevel lv[kMaxLevels];
};

// Release-add and acquire-load at GPU scope (PTX memory model): the arrival
// publishes every write the block made before the preceding __syncthreads,
// the acquiring load makes the other blocks' published writes visible.
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier with a bounded wait on a monotonic arrival counter: the k-th
// barrier of the launch is passed once the counter reaches k * gridDim.x
// (`target` counts this block's barriers).  Returns false when the wait ran
// out here or another block reported an error.
__device__ __forceinline__ bool tail_barrier(unsigned *count, unsigned &target, int *err, long long limit, CgState *st, int ninst) {
  __shared__ int ok;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    ok = 1;
    red_release_add(count, 1u);
    const volatile int *ve = err;
    const long long t0 = clock64();
    while (ld_acquire(count) < target) {
      if (*ve != 0) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > limit) {
        atomicExch(err, 1);
        if (st)
          for (int i = 0; i < ninst; ++i) {
            st[i].done = 1;
            st[i].status = HPCG_ERR_TIMEOUT;
          }
        ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// Runs the colour-pair runs of one smoother application on level L; blocks
// take the level's virtual blocks round-robin, warps the lines of a block.
template <typename T>
__device__ __forceinline__ bool tail_runs(const TailPlan &P, int l, const TailRun *runs, int nruns, bool from_zero, bool fuse,
                                          unsigned *bar, unsigned &target, int *err, long long limit, CgState *st) {
  const TailLevel &L = P.lv[l];
  int vmask = from_zero ? 0 : 0xF;
  const int vpb = kTailThreadsY / L.lpc;  // virtual blocks per block step
  const int w = threadIdx.y;
  for (int k = 0; k < nruns; ++k) {
    const TailRun run = runs[k];
    T *rc = (fuse && k == nruns - 1) ? (T *)P.lv[l + 1].r : nullptr;
    const Inst *tabc = rc ? P.lv[l + 1].tab : nullptr;
    if (w < vpb * L.lpc) {
      for (int base = blockIdx.x * vpb; base < L.nvb; base += gridDim.x * vpb) {
        const int vb = base + w / L.lpc;
        if (vb < L.nvb)
          gs_lines_vblock<T, 1, true>(vb, w % L.lpc, L.tab, P.count, L.lpc, L.zc, run.cls & 1, (run.cls >> 1) & 1, run.pa, run.steps,
                                vmask, (const T *)L.r, (T *)L.z, (const T *)L.invd, st, tabc, rc, (const T *)L.kap);
      }
    }
    vmask |= 1 << run.cls;
    if (!tail_barrier(bar, target, err, limit, st, P.count)) return false;
  }
  return true;
}

// Refinement + correction of level l from level l+1, every instance.
template <typename T>
__device__ __forceinline__ void tail_prolong(const TailPlan &P, int l, const CgState *st) {
  const TailLevel &F = P.lv[l], &C = P.lv[l + 1];
  const long nthr = (long)gridDim.x * blockDim.x * blockDim.y;
  const long tid = (long)blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * blockDim.x + threadIdx.x;
  for (int ii = 0; ii < P.count; ++ii) {
    if (st && st[ii].done) continue;
    const Inst f = F.tab[ii], c = C.tab[ii];
    for (long q = tid; q < c.n; q += nthr) {
      const int xc = (int)(q % c.nx), yc = (int)((q / c.nx) % c.ny), zc = (int)(q / ((long)c.nx * c.ny));
      const long lf = 2L * xc + (long)f.nx * (2L * yc + (long)f.ny * 2L * zc);
      T *zf = (T *)F.z + f.off + lf;
      *zf = __ldcg(zf) + __ldcg((const T *)C.z + c.off + q);
    }
  }
}

// Residual + injection as its own phase (when it cannot be fused: forward-only smoother).
template <typename T>
__device__ __forceinline__ void tail_restrict(const TailPlan &P, int l, const CgState *st) {
  const TailLevel &F = P.lv[l], &C = P.lv[l + 1];
  const long nthr = (long)gridDim.x * blockDim.x * blockDim.y;
  const long tid = (long)blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * blockDim.x + threadIdx.x;
  for (int ii = 0; ii < P.count; ++ii) {
    if (st && st[ii].done) continue;
    const Inst f = F.tab[ii], c = C.tab[ii];
    const T *zg = (const T *)F.z + f.off;
    for (long q = tid; q < c.n; q += nthr) {
      const int xc = (int)(q % c.nx), yc = (int)((q / c.nx) % c.ny), zc = (int)(q / ((long)c.nx * c.ny));
      const int xf = 2 * xc, yf = 2 * yc, zf = 2 * zc;
      const long lf = xf + (long)f.nx * (yf + (long)f.ny * zf);
      const T d = F.kap ? T(26) + ((const T *)F.kap)[f.off + lf] : T(26);
      T nb = T(0);  // 26 neighbours, ascending column order, coherent loads
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int xx = xf + dx, yy = yf + dy, zz = zf + dz;
            if ((dx | dy | dz) == 0 || xx < 0 || yy < 0 || zz < 0 || xx >= f.nx || yy >= f.ny || zz >= f.nz) continue;
            nb += __ldcg(zg + xx + (long)f.nx * (yy + (long)f.ny * zz));
          }
      const T az = d * __ldcg(zg + lf) - nb;
      ((T *)C.r)[c.off + q] = __ldcg((const T *)F.r + f.off + lf) - az;
    }
  }
}

// stage_level < 0: the whole coarse end (levels first..last down, then back
// up to first).  Otherwise only stage `stage` (HPCG_STAGE_PRE / _REFINE /
// _POST of hpcg_mg_stage) of level stage_level, with the same arithmetic.
template <typename T>
__global__ void __launch_bounds__(32 * kTailThreadsY) k_vcycle_tail(const TailPlan *__restrict__ plan, unsigned *bar, int *err,
                                                                     long long limit, CgState *st, int stage_level, int stage) {
  const TailPlan &P = *plan;
  unsigned target = 0;
  if (stage_level >= 0) {
    const int l = stage_level;
    const TailLevel &L = P.lv[l];
    if (stage == HPCG_STAGE_PRE) {
      if (!tail_runs<T>(P, l, L.pre, L.npre, true, L.fuse != 0 && l < P.last, bar, target, err, limit, st)) return;
      if (l < P.last && !L.fuse) tail_restrict<T>(P, l, st);
    } else {
      tail_prolong<T>(P, l, st);
      if (stage == HPCG_STAGE_POST) {
        if (!tail_barrier(bar, target, err, limit, st, P.count)) return;
        tail_runs<T>(P, l, L.post, L.npost, false, false, bar, target, err, limit, st);
      }
    }
    return;
  }
  for (int l = P.first; l <= P.last; ++l) {
    const TailLevel &L = P.lv[l];
    if (!tail_runs<T>(P, l, L.pre, L.npre, true, L.fuse != 0 && l < P.last, bar, target, err, limit, st)) return;
    if (l < P.last && !L.fuse) {
      tail_restrict<T>(P, l, st);
      if (!tail_barrier(bar, target, err, limit, st, P.count)) return;
    }
  }
  for (int l = P.last - 1; l >= P.first; --l) {
    tail_prolong<T>(P, l, st);
    if (!tail_barrier(bar, target, err, limit, st, P.count)) return;
    if (!tail_runs<T>(P, l, P.lv[l].post, P.lv[l].npost, false, false, bar, target, err, limit, st)) return;
  }
}

}  // namespace hpcg
