// hpcg_internal.cuh -- device-side data structures shared by the kernels and
// the host driver of the GB300 MG-PCG library.
//
// Layout in HBM: every level of every instance stores its vectors in natural
// row order i = x + nx*(y + ny*z); the vectors of all instances of one level
// are concatenated (Inst::off is the first row of an instance), so that one
// kernel launch covers the same step of every instance of a batch.  A
// single-instance handle is a batch of one.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hpcg.h"

namespace hpcg {

constexpr int kMaxLevels = 8;
constexpr int kTileX = 32;       // threads of a block along x (one warp)
constexpr int kTileY = 8;        // warps of a block along y
constexpr int kBlock = kTileX * kTileY;
constexpr int kRedThreads = 256; // threads of a reduction block
constexpr int kFinThreads = 1024; // threads of a finalize block (one per instance)
constexpr int kRedItems = 8;     // elements per thread per reduction block (before the block strides)
constexpr int kMaxRedBlocksPerInst = 2432;  // 16 per SM of 152; a fixed cap keeps reductions deterministic
constexpr int kHistoryCap = 8192;
constexpr int kRawDotBlocks = 304;  // fixed grid of the plain dot product (2 x 152 SMs)

// One grid (one level of one instance).
struct Inst {
  int nx, ny, nz;
  int blk_full;   // first block of this grid in a launch over all rows (32x8 tiles per z-plane)
  int blk_half;   // first block in a launch over one colour class (half lattice)
  int blk_red;    // first block in a reduction launch
  int nred;       // reduction blocks of this grid
  int blk_row;    // first block in a line launch over every x-line (one warp per line)
  int nrow;       // blocks of this grid in that launch
  int blk_line;   // first block in a line launch over the lines of one colour-line class
  int nline;      // blocks of this grid in that launch
  int poff;       // first per-line partial sum of this grid (prefix of ny * nz)
  long off;       // first row of this grid in the level's concatenated vectors
  long n;         // rows
};

// Per-level launch description (host copy; `inst` points to the device table).
struct LevelTab {
  const Inst *inst;  // device array [count]
  int count;
  int nblk_full, nblk_half, nblk_red, nblk_row, nblk_line;
  int row_lpc, row_zc;    // line launch over all lines: lines (warps) per block, z-planes per block
  int line_lpc, line_zc;  // line launch over one line class: lines per block, updated planes per block
  int nch;                // 32-wide x chunks per line (ceil(max nx / 32)); 0 = line kernels unavailable
  int nch2;               // 32-wide chunks per x parity (ceil(ceil(max nx / 2) / 32)) of the colour-step kernels
  long n;                 // rows over all instances
};

// Blocks of a line launch over every x-line of an nx x ny x nz grid.
__host__ __device__ inline int row_blocks(int ny, int nz, int lpc, int zc) {
  return ((ny + lpc - 1) / lpc) * ((nz + zc - 1) / zc);
}
// Blocks of a line launch over the lines of one colour-line class (y, z of fixed parities).
__host__ __device__ inline int line_blocks(int ny, int nz, int lpc, int zc) {
  const int hy = (ny + 1) / 2, hz = (nz + 1) / 2;
  return ((hy + lpc - 1) / lpc) * ((hz + zc - 1) / zc);
}

// Device-resident CG scalars of one instance.
struct CgState {
  double rtz, pAp, alpha, beta, normr, normr0, best, tol;
  double hist_prev[3];
  int iter, done, status, first, restart, restarts, stall, max_iters;
  int converged, mixed;
  int xpend;  // x += alpha p of this alpha is still to be applied (deferred to the next p update)
  int restart_every;  // mixed precision: residual replacement every this many iterations (0: on stalls only)
};

// Blocks of a 32x8-tiled launch over an nx x ny x nz box, one z-plane per tile row.
__host__ __device__ inline int tiles_of(int nx, int ny, int nz) {
  return ((nx + kTileX - 1) / kTileX) * ((ny + kTileY - 1) / kTileY) * nz;
}
__host__ __device__ inline int half_up(int v) { return (v + 1) / 2; }

// Finds the instance that owns global block `b` (prefix `which` in the table;
// Which = 5: the instance owning global x-line `b` of a level);
// tables hold at most a few hundred entries, a binary search is uniform per block.
template <int Which>
__device__ inline int find_inst(const Inst *__restrict__ tab, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    int start = Which == 0 ? tab[mid].blk_full
                : Which == 1 ? tab[mid].blk_half
                : Which == 2 ? tab[mid].blk_red
                : Which == 3 ? tab[mid].blk_row
                : Which == 4 ? tab[mid].blk_line
                             : tab[mid].poff;
    if (start <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace hpcg
