/*
 * hpcg.h -- C ABI of the GB300 (sm_103a) multigrid-preconditioned CG library
 * for the HPCG 27-point operator, following Scolari & Yzelman, "Effective
 * implementation of the High Performance Conjugate Gradient benchmark on
 * GraphBLAS" (arXiv 2304.08232).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid rows are numbered i = x + nx*(y + ny*z) (x fastest); every vector
 *    argument is a dense array of one value per row in that order.
 *  - Pointers named *_dev are DEVICE pointers on the handle's GPU; pointers
 *    named *_host are host pointers.  The caller owns every buffer it passes
 *    and keeps it alive until the stream has finished the call's work.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous with respect to the host unless stated otherwise.
 *  - Every call returns an hpcg_status; HPCG_OK == 0.  A non-zero status
 *    leaves caller buffers in an unspecified state unless stated otherwise.
 *    hpcg_strerror() turns a status into text.
 *  - The operator is matrix-free: diagonal 26 (+ kappa_i when a diagonal field
 *    is bound), -1 to every other grid point within distance one in each
 *    coordinate (Dirichlet boundary, no ghost rows), Sections II-B and II-C.
 *  - Colour classes (Section III-A, greedy colouring, eight colours on this
 *    grid) are color_i = (x&1) + 2(y&1) + 4(z&1); coarse level l+1 has each
 *    dimension halved and coarse row c = (xc,yc,zc) is injected from fine row
 *    (2xc, 2yc, 2zc) (Section II-F, straight injection).
 */
#ifndef HPCG_GB300_H
#define HPCG_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hpcg_ctx *hpcg_handle;

typedef enum {
  HPCG_OK = 0,
  HPCG_ERR_INVALID_ARG = 1,   /* null pointer, bad level, dimension < 2 or not divisible by 2^(levels-1) */
  HPCG_ERR_CUDA = 2,          /* a CUDA runtime call failed; the text is in hpcg_last_cuda_error() */
  HPCG_ERR_BREAKDOWN = 3,     /* CG breakdown: p.Ap <= 0, or a NaN/Inf scalar */
  HPCG_ERR_NOT_CONVERGED = 4, /* tolerance not met within max_iters; x and stats are still valid */
  HPCG_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out; the kernel returned early */
  HPCG_ERR_NO_WORKSPACE = 6,  /* bound workspace smaller than hpcg_workspace_bytes() */
  HPCG_ERR_OUT_OF_MEMORY = 7, /* cudaMalloc of an internally owned workspace failed */
  HPCG_ERR_UNSUPPORTED = 8    /* the call does not apply to this handle's kind */
} hpcg_status;

typedef enum {
  HPCG_FP64 = 0,  /* every step in FP64 */
  HPCG_MIXED = 1  /* MG preconditioner in FP32 (operator values -1 and 26 are exact
                     in BF16 and are compile-time constants of the matrix-free
                     kernels; a kappa diagonal is kept in FP32); the outer residual,
                     dot products and solution update stay in FP64 */
} hpcg_precision;

typedef struct {
  int nx, ny, nz;   /* finest grid */
  int levels;       /* MG levels including the finest, 1..8 (Listing 1; HPCG uses 4) */
  int precision;    /* hpcg_precision of the preconditioner */
  int pre_sweeps;   /* smoother applications before the coarse correction (default 1) */
  int post_sweeps;  /* smoother applications after it (default 1) */
  int symmetric;    /* 1: forward colours 0..7 then backward 7..0 (default); 0: forward only */
  int check_every;  /* tolerance solves: host looks at the device convergence flag every
                       this many iterations (default 1; work after convergence is skipped
                       on the device, so a larger value only costs idle launches) */
  int max_rhs;      /* largest nrhs of hpcg_pcg_solve_multi the workspace is sized for (default 0) */
  int autotune;     /* 1 (default): the first compute call times candidate launch shapes of the
                       line kernels on every level and keeps the fastest (hpcg_autotune) */
  int fixed_point;  /* 1 (default): FP64 colour steps and SpMV sum neighbour values exactly in
                       64-bit fixed point on the integer pipe (at least as accurate as FP64
                       summation; FP64 is used for steps with huge or non-finite values);
                       0: plain FP64 sums */
  int pdl;          /* 1 (default): kernels are launched with programmatic dependent launch, so
                       a kernel is scheduled while its predecessor finishes; 0: plain launches */
  int persistent;   /* 1: the smallest levels of the V-cycle run in one persistent cooperative
                       kernel (hpcg_persistent_levels); 0 (default): one launch per step, which
                       measured faster on one 192^3 grid (graph launches beat grid barriers) */
  int block_fp;     /* 1 (default): inside the FP64 V-cycle (with fixed_point, the symmetric
                       smoother, no persistent kernel, grids up to 384 points along x) the level
                       vectors z are kept as 64-bit integer mantissas with one exponent per x-line,
                       so colour steps add exactly without converting each value they load; each
                       new value is rounded once, at an absolute 2^-56 of the largest term of its
                       colour step (its line's and the neighbouring lines' values: 53 bits for
                       values of the line's typical size, zero for values far below their
                       neighbourhood's), and non-finite values end as NaN; r and the result z
                       stay FP64.  0: the FP64 V-cycle keeps z in FP64 */
  int cluster_tail; /* 1: with block_fp, the levels of at most 32768 rows whose x-lines fit 64
                       points run in one launch of a 16-block thread-block cluster, runs separated
                       by the cluster barrier instead of kernel boundaries (same bits as one launch
                       per run); 0 (default): one launch per run on every level, which measured
                       faster on one 192^3 grid (16 SMs do the coarse runs slower than launches) */
  int restart_every; /* mixed precision: also replace the recurrence residual by b - A x (FP64) after
                        every this many iterations, besides the stall rule (no 1% progress in 3
                        iterations); 0 (default): on stalls only */
  int bfp_split;     /* with block_fp: levels whose x-lines have 65-256 points run their colour steps
                        with one warp per 64-point chunk of a line (neighbours across chunks through
                        shared memory; same z bits, r.z partials summed chunk by chunk); 0 (default):
                        one warp per line */
  int fuse_planes;   /* with block_fp, one grid: the colour-pair runs of a smoother application whose
                        line classes share their z parity ([0 1], [2 3 2], [1 0]) run in one launch,
                        one block per plane of that parity and a block barrier between runs (same
                        bits; the planes between are read once per group instead of once per run).
                        0 (default): the autotuner times each level both ways and keeps the faster
                        (one launch per run measured faster at every size from 128^3 to
                        384 x 1024 x 1024); 1: always; -1: never */
} hpcg_options;

typedef struct {
  int iters;          /* CG iterations run */
  int restarts;       /* residual replacements r = b - A x (mixed precision) */
  int converged;      /* 1 if ||r||/||r0|| <= rel_tol was reached */
  int status;         /* hpcg_status of the solve */
  double rel_res;     /* final recurrence residual ||r_k||/||r_0|| */
  double *history;    /* host, caller-owned, may be NULL: ||r_k||/||r_0|| for k = 1..iters */
  int history_cap;    /* capacity of history in doubles */
} hpcg_stats;

/* Fills *opt with defaults for an nx x ny x nz grid with 4 levels, FP64. */
int hpcg_options_default(hpcg_options *opt, int nx, int ny, int nz);

/* Builds a hierarchy handle (Section II-B input generation, Listing 1 levels).
 * Allocates no device memory: bind a workspace (below) or let the first compute
 * call allocate one it owns.  Errors: INVALID_ARG for null out, levels outside
 * 1..8, a dimension < 2 on the coarsest level or not divisible by 2^(levels-1). */
int hpcg_setup(int nx, int ny, int nz, int levels, hpcg_handle *out);

/* As hpcg_setup with explicit options.  kappa_dev (nullable, device, n doubles)
 * is a per-row diagonal field: A_ii = 26 + kappa_i; the values are copied into
 * the workspace on the first compute call (or by hpcg_set_kappa), coarse levels
 * take kappa at their injected fine rows. */
int hpcg_setup_ex(const hpcg_options *opt, const double *kappa_dev, hpcg_handle *out);

/* Replaces the diagonal field (device, n doubles; NULL removes it).  Needs a
 * workspace; runs on `stream`. */
int hpcg_set_kappa(hpcg_handle h, const double *kappa_dev, void *stream);

/* Frees the handle and any workspace it allocated itself (not a bound one).
 * Synchronises the device first. */
int hpcg_destroy(hpcg_handle h);

/* Bytes of device workspace the handle needs (all levels' vectors, CG vectors,
 * reduction partials, device scalars, residual history). */
int hpcg_workspace_bytes(hpcg_handle h, size_t *bytes);

/* Binds caller-owned device memory (>= hpcg_workspace_bytes, 256-byte aligned)
 * as the workspace; the library then allocates nothing.  The memory must stay
 * valid until hpcg_destroy or another bind.  Errors: NO_WORKSPACE if too small. */
int hpcg_bind_workspace(hpcg_handle h, void *dev, size_t bytes);

/* Dimensions of MG level `level` (0 = finest) into dims_host[3]. */
int hpcg_level_dims(hpcg_handle h, int level, int *dims_host);

/* --- setup maps, written by GPU kernels into caller device buffers --------- */
/* Colour of every row of `level` (Section III-A), int32 [n_level]. */
int hpcg_get_colors(hpcg_handle h, int level, int *colors_dev, void *stream);
/* Injection map of `level` -> level+1: f2c[c] = fine row of coarse row c,
 * int32 [n_{level+1}] (Section II-F). INVALID_ARG on the coarsest level. */
int hpcg_get_f2c(hpcg_handle h, int level, int *f2c_dev, void *stream);
/* Nonzeros of every row (8..27), int32 [n_level] (Section II-C). */
int hpcg_get_row_nnz(hpcg_handle h, int level, int *nnz_dev, void *stream);
/* HPCG right-hand side b = A * ones (exact solution ones), FP64 [n_0]. */
int hpcg_get_rhs(hpcg_handle h, double *b_dev, void *stream);

/* --- single steps of the hot path -------------------------------------------- */
/* y = A_level x (spmv, Section II-C); FP64 [n_level]; x and y must not overlap. */
int hpcg_spmv(hpcg_handle h, int level, const double *x_dev, double *y_dev, void *stream);

/* One colour step of the red-black Gauss-Seidel pass (Listings 2 and 3): every
 * row i of colour `color` gets z_i <- (r_i - sum_{j != i} A_ij z_j) / A_ii, in
 * place on z; FP64 [n_level]. */
int hpcg_rbgs_color(hpcg_handle h, int level, int color, const double *r_dev, double *z_dev, void *stream);

/* One smoother application on `level`: colours 0..7, then (symmetric option)
 * 7..0, in place on z (the smoother that replaces SGS, Sections II-E, III-A). */
int hpcg_rbgs(hpcg_handle h, int level, const double *r_dev, double *z_dev, void *stream);

/* Fused residual and restriction (Listing 1's residual and restriction, Section II-F):
 * rc[c] = r[f2c[c]] - (A_level z)[f2c[c]]; r, z FP64 [n_level], rc [n_{level+1}]. */
int hpcg_restrict_residual(hpcg_handle h, int level, const double *r_dev, const double *z_dev, double *rc_dev, void *stream);

/* Refinement and correction (Listing 1's coarse correction): z[f2c[c]] += zc[c]; others unchanged. */
int hpcg_prolong_add(hpcg_handle h, int level, const double *zc_dev, double *z_dev, void *stream);

/* z = M r: one V-cycle of Listing 1 from z = 0 on all levels, in the handle's
 * precision; FP64 [n_0] in and out; r and z must not overlap. */
int hpcg_mg_vcycle(hpcg_handle h, const double *r_dev, double *z_dev, void *stream);

/* --- the V-cycle stage by stage, and its level vectors ------------------------ */
/* Listing 1 on level l is: z_l <- 0 and pre-smoothing; on a non-coarsest level
 * the residual restricted by injection into the next level's right-hand side,
 * r_{l+1} <- R (r_l - A_l z_l) (Section II-F); the recursion; then z_l <- z_l +
 * R^T z_{l+1} (refinement and correction) and post-smoothing.  These calls run
 * one such stage on one level with the launches hpcg_mg_vcycle itself issues
 * for it (restriction and refinement fused into smoother runs where the
 * V-cycle fuses them; the coarse end's single-launch kernel when
 * hpcg_options.cluster_tail or .persistent put the level there), on the level
 * vectors the handle keeps, so that running PRE on levels 0..L-1 and then
 * POST on levels L-2..0 reproduces hpcg_mg_vcycle bit for bit.  Their purpose
 * is to observe and drive the coarse levels, whose effect on the V-cycle's
 * output is otherwise hidden (with this smoother and injection the coarse
 * correction lands on points that the post-smoother recomputes first).
 *
 * Stages (level < L-1 for REFINE and POST):
 *   HPCG_STAGE_PRE:    z_l <- 0, pre-smoothing (one application on the coarsest
 *                      level), and on a non-coarsest level r_{l+1} <- R (r_l - A_l z_l).
 *   HPCG_STAGE_REFINE: z_l <- z_l + R^T z_{l+1} alone.
 *   HPCG_STAGE_POST:   z_l <- z_l + R^T z_{l+1}, then post-smoothing.
 * Level vectors: r_l and z_l for l >= 1 live in the handle's workspace; on
 * level 0 r_0 is r0_dev (FP64 [n_0], caller's) and z_0 is z0_dev with block_fp
 * off, else the workspace's (block floating point, or FP32 in mixed
 * precision) with z0_dev receiving the FP64 result of POST (and of PRE when
 * levels == 1).  r0_dev and z0_dev are required on level 0 (distinct; 16-byte
 * aligned with block_fp) and ignored on other levels.  Errors: INVALID_ARG for
 * a level or stage out of range or missing level-0 vectors. */
typedef enum { HPCG_STAGE_PRE = 0, HPCG_STAGE_REFINE = 1, HPCG_STAGE_POST = 2 } hpcg_stage;
int hpcg_mg_stage(hpcg_handle h, int level, int stage, const double *r0_dev, double *z0_dev, void *stream);

/* Copies level `level`'s right-hand side r_l and iterate z_l, as the last
 * V-cycle or stage on this handle left them, into caller device buffers of
 * n_level FP64 values (either pointer may be NULL).  Block-floating-point z is
 * converted exactly (each value is its mantissa times the line's power of
 * two), FP32 vectors are widened.  Level 0: r_dev must be NULL (r_0 is the
 * caller's), and z_0 exists only with block_fp or mixed precision
 * (UNSUPPORTED otherwise). */
int hpcg_get_level_vectors(hpcg_handle h, int level, double *r_dev, double *z_dev, void *stream);
/* Writes r_l and/or z_l of `level` (same rules).  Block floating point stores
 * each x-line at the largest exponent of its values, truncating every value
 * to 58 bits below that line's largest power of two; mixed precision rounds
 * to FP32.  hpcg_get_level_vectors returns the stored values. */
int hpcg_set_level_vectors(hpcg_handle h, int level, const double *r_dev, const double *z_dev, void *stream);

/* out_dev[0] = a . b over n FP64 values, deterministic fixed-order reduction. */
int hpcg_dot(hpcg_handle h, long n, const double *a_dev, const double *b_dev, double *out_dev, void *stream);

/* w = alpha x + beta y over n FP64 values (waxpby, Section II-C); w may alias x or y. */
int hpcg_waxpby(hpcg_handle h, long n, double alpha, const double *x_dev, double beta, const double *y_dev, double *w_dev, void *stream);

/* --- solves -------------------------------------------------------------------- */
/* Preconditioned CG (Section II-C) with the MG preconditioner, HPCG iteration
 * order.  x_dev holds x0 on entry and the solution on exit.  rel_tol <= 0 runs
 * exactly max_iters iterations; otherwise stops once ||r_k||/||r_0|| <= rel_tol.
 * Mixed precision replaces r by b - A x in FP64 when the residual stalls for 3
 * iterations.  Blocks the host until the solve is done (it reads back the
 * statistics); stats (nullable) is filled.  Returns NOT_CONVERGED (x valid) if
 * rel_tol > 0 was not reached, BREAKDOWN if p.Ap <= 0 or NaN. */
int hpcg_pcg_solve(hpcg_handle h, const double *b_dev, double *x_dev, int max_iters, double rel_tol,
                   hpcg_stats *stats, void *stream);

/* Backward of the differentiable solve x = A(kappa)^{-1} b: solves the adjoint
 * A lambda = grad_x (A is symmetric) with the same MG-PCG from lambda = 0, then
 * grad_b = lambda and, if grad_kappa_dev is not NULL, grad_kappa_i = -lambda_i x_i
 * (the diagonal of -lambda x^T, since dA/dkappa_i = e_i e_i^T).  All FP64 [n_0].
 * grad_b_dev receives lambda and must not alias x_dev or grad_x_dev. */
int hpcg_pcg_backward(hpcg_handle h, const double *x_dev, const double *grad_x_dev, double *grad_b_dev,
                      double *grad_kappa_dev, int max_iters, double rel_tol, hpcg_stats *stats, void *stream);

/* --- batched forms -------------------------------------------------------------- */
/* nrhs right-hand sides on the handle's grid in one multi-RHS solve; B and X are
 * FP64 [nrhs][n_0] (each RHS contiguous); X holds the initial guesses.  Every
 * RHS stops on its own at rel_tol (its updates are frozen after convergence).
 * stats (nullable) is an array of nrhs records.  nrhs in 1..64. */
int hpcg_pcg_solve_multi(hpcg_handle h, int nrhs, const double *B_dev, double *X_dev, int max_iters,
                         double rel_tol, hpcg_stats *stats, void *stream);

/* A batch of `count` independent grids (dims_host: 3*count ints, nx ny nz per
 * instance), each with its own `levels`-level hierarchy, solved together.
 * Vectors of the batch are the instances' vectors concatenated in order. */
int hpcg_setup_batch(int count, const int *dims_host, int levels, int precision, hpcg_handle *out);

/* Row offset of every instance in the concatenated vectors, int64 [count+1]. */
int hpcg_batch_offsets(hpcg_handle h, long *offsets_host);

/* Solves every instance of a batch handle; b, x concatenated FP64; stats
 * (nullable) is an array of `count` records.  Each instance stops on its own. */
int hpcg_pcg_solve_batch(hpcg_handle h, const double *b_dev, double *x_dev, int max_iters, double rel_tol,
                         hpcg_stats *stats, void *stream);

/* --- per-level time breakdown -------------------------------------------------------------- */
/* The paper's instrument (Section V-C, Figs. 4-7): time of the smoother and of
 * restriction/refinement per MG level, and of the CG kernels, for one CG
 * iteration.  Starts a solve of A x = b from x_dev (two iterations are run:
 * one warm-up, one timed with CUDA events between kernel groups, launched one
 * by one rather than as a graph), so x_dev is changed.  ms_host (cap >=
 * 3*levels + 7 doubles) receives: smoother ms per level (restriction fused into
 * the smoother's last run counts here), separate restriction ms per level,
 * refinement ms per level, persistent coarse kernel ms, SpMV ms, dot products
 * ms, vector updates ms, scalar finalisation ms, precision conversions ms, and
 * the total.  Synchronises `stream`. */
int hpcg_profile_iteration(hpcg_handle h, const double *b_dev, double *x_dev, double *ms_host, int cap, void *stream);

/* --- launch-shape autotuner ------------------------------------------------------------ */
/* Times candidate launch shapes (x-lines per block, z-planes per block) of the
 * SpMV and colour-step line kernels on every level of the handle and keeps the
 * fastest; results stay bit-identical whatever the shape.  Synchronises
 * `stream`; must not be called while `stream` is being captured.  Runs once on
 * the first compute call when hpcg_options.autotune is set.  shapes_host
 * (nullable) receives 4 ints per level: row lines, row planes, colour-line
 * lines, colour-line planes. */
int hpcg_autotune(hpcg_handle h, int *shapes_host, void *stream);

/* Sets the launch shapes (same 4 ints per level as hpcg_autotune reports, each
 * lines-per-block in 1..8 and planes-per-block in 1..64) instead of tuning, so
 * that a run can be repeated with the same launches (profiling).  Marks the
 * handle as tuned.  Errors: INVALID_ARG for a null pointer or a value out of
 * range. */
int hpcg_set_launch_shapes(hpcg_handle h, const int *shapes_host);

/* --- persistent coarse levels and bounded waits ----------------------------------------- */
/* The smallest levels of the V-cycle (those whose x-lines fit one 32-wide chunk
 * per parity, up to 50,000 rows over all instances) run in one persistent
 * cooperative kernel whose phases are separated by grid barriers.  Every
 * barrier wait is bounded by a number of SM clock cycles (default 2e9, about
 * one second); a wait that runs out makes the kernel record HPCG_ERR_TIMEOUT,
 * mark every instance's solve as finished and return, leaving the context
 * usable.  hpcg_set_wait_limit changes the bound (0 makes any wait time out:
 * a host-side way to exercise the error path).  Not part of the paper. */
int hpcg_set_wait_limit(hpcg_handle h, long long cycles);
/* Synchronises the device and reports HPCG_ERR_TIMEOUT in *status_out if a
 * bounded wait of the handle's kernels ran out since the last solve or
 * V-cycle started, HPCG_OK otherwise. */
int hpcg_device_status(hpcg_handle h, int *status_out);
/* First level run by the persistent kernel, or -1 when every level uses one
 * launch per step. */
int hpcg_persistent_levels(hpcg_handle h, int *first_level);

/* --- allocation-free V-cycle ---------------------------------------------------------- */
/* No counterpart in the paper: a convenience for callers that cannot allocate
 * device memory when they need the preconditioner (for example code running
 * during a CUDA graph capture under a strict allocator, plug-ins inside a host
 * application that owns all device allocations, or real-time loops that forbid
 * allocation after start-up).
 *
 * z = M r for an nx x ny x nz grid with `levels` levels, exactly the FP64
 * V-cycle of hpcg_mg_vcycle with default options (one symmetric smoother
 * application before and after each coarse correction, no kappa field), but
 * without a handle: r_dev and z_dev (FP64 [nx*ny*nz], device, caller-owned, not
 * overlapping) are the only buffers it touches besides a fixed device array of
 * HPCG_NOALLOC_SCRATCH_BYTES inside the library, which holds the level tables
 * and the coarse-level vectors.  That array is static: every GPU that loads the
 * library keeps it until the process exits, and the call itself allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 *  - Size limit: the coarse levels need 16 bytes per coarse row (sum over levels
 *    1..levels-1 of (nx>>l)(ny>>l)(nz>>l)) plus under 4 KiB of tables and alignment
 *    padding; larger problems
 *    are rejected with HPCG_ERR_NO_WORKSPACE before any GPU work.  192^3 with 4
 *    levels fits.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the one array and leaves its contents behind; the
 *    V-cycle zeroes each coarse correction itself before use, so stale contents
 *    never leak into a result.  Calls whose GPU work overlaps (different
 *    streams, or host threads without ordering) race on the array: serialise
 *    them on one stream.
 * Errors: INVALID_ARG for null or identical pointers and for the size rules of
 * hpcg_setup; NO_WORKSPACE beyond the size limit; CUDA for a failed launch. */
#define HPCG_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int hpcg_mg_vcycle_noalloc(int nx, int ny, int nz, int levels, const double *r_dev, double *z_dev, void *stream);
/* For checking the allocation-free V-cycle's coarse levels (no counterpart in
 * the paper either): copies r_l and z_l (FP64, (nx>>l)(ny>>l)(nz>>l) values,
 * either pointer may be NULL) of coarse level `level` (1..levels-1) as the
 * last hpcg_mg_vcycle_noalloc on the same hierarchy left them in the shared
 * array, with device-to-device copies on `stream`; allocates nothing.
 * Errors: INVALID_ARG for the size rules, a level out of range or two null
 * pointers; NO_WORKSPACE beyond the array's size. */
int hpcg_noalloc_level_vectors(int nx, int ny, int nz, int levels, int level, double *r_dev, double *z_dev, void *stream);

/* --- materialised operator, rows grouped by colour (P^T A P) --------------------- */
/* Section III-A: rows of one colour can be stored contiguously by permuting the
 * system, P^T A P, so that each colour phase of the smoother reads a contiguous
 * range.  This engine stores the 27-point operator of every level as a
 * sliced-ELL matrix (FP64 values, int32 columns, 27 slots per row of which 8 to
 * 27 are used, slices of 32 rows stored slot-major) and runs the SpMV, the
 * colour phases, the injected residual, refinement, the V-cycle of Listing 1
 * and PCG on it.  It exists beside the matrix-free kernels above to compare
 * storage schemes; it has no kappa field, no mixed precision and no batches.
 *
 * Stored order: with colour_sorted = 1 the rows of colour k (color_i =
 * (x&1) + 2(y&1) + 4(z&1), the greedy colouring) are the range
 * [cstart[k], cstart[k+1]) and inside it in increasing natural index; with
 * colour_sorted = 0 the stored order is the natural order and a colour phase
 * tests the colour of every row.  Slots of a row hold its nonzeros in
 * ascending natural column index; unused slots hold value 0 and the row's own
 * column.  Vectors passed to the level calls below are in STORED order;
 * hpcg_ell_permute converts.
 *
 * exact = 1: every product and sum is a separate IEEE operation (no fused
 * multiply-add), sums start from 0.0 in slot order, and the colour update is
 * (r_i - s_i + z_i d_i) / d_i with s_i including the diagonal (Listing 3), so
 * the level calls reproduce a plain sequential CRS evaluation bit for bit;
 * exact = 0 (faster) fuses the multiply-adds.  bf16_values = 1 stores the
 * values in BF16 (2 bytes instead of 8 per slot): 26, -1 and 0 are exact there,
 * so every result is the same, bit for bit, as with FP64 values.
 *
 * Memory: hpcg_ell_setup allocates (cudaMalloc) about 12 * 27 bytes per row for
 * the matrix (6 * 27 with BF16 values) plus vectors and maps, on the current
 * device (3.1 GB at 192^3 with 4 levels and FP64 values); hpcg_ell_bytes
 * reports the total.  Calls are ordered on `stream`;
 * the handle serialises host threads.
 * Errors: INVALID_ARG for null or aliased pointers, a level or colour out of
 * range, and the grid rules of hpcg_setup; CUDA when an allocation or launch
 * fails. */
typedef struct hpcg_ell_ctx *hpcg_ell_handle;
int hpcg_ell_setup(int nx, int ny, int nz, int levels, int colour_sorted, int exact, int bf16_values, hpcg_ell_handle *out);
int hpcg_ell_destroy(hpcg_ell_handle h);
int hpcg_ell_bytes(hpcg_ell_handle h, size_t *bytes);
/* info_host[0] = rows, [1] = slices of 32 rows, [2..10] = cstart[0..8] (all zero when not sorted). */
int hpcg_ell_level_info(hpcg_ell_handle h, int level, long *info_host);
/* perm_dev[p] (int32 [n], device) = natural row index of stored row p. */
int hpcg_ell_permutation(hpcg_ell_handle h, int level, int *perm_dev, void *stream);
/* Copies the slices: slot s of stored row p at ((p/32)*27 + s)*32 + p%32 of
 * col_dev (int32) and val_dev (FP64, widened from BF16 storage), each of
 * slices*27*32 entries. */
int hpcg_ell_matrix(hpcg_ell_handle h, int level, int *col_dev, double *val_dev, void *stream);
/* to_stored = 1: dst[p] = src[perm[p]]; 0: dst[perm[p]] = src[p] (FP64 [n], distinct buffers). */
int hpcg_ell_permute(hpcg_ell_handle h, int level, int to_stored, const double *src_dev, double *dst_dev, void *stream);
/* y = A x on `level` (stored order, x and y distinct). */
int hpcg_ell_spmv(hpcg_ell_handle h, int level, const double *x_dev, double *y_dev, void *stream);
/* One colour phase (Listings 2 and 3): rows of colour `color` updated in place in z. */
int hpcg_ell_rbgs_color(hpcg_ell_handle h, int level, int color, const double *r_dev, double *z_dev, void *stream);
/* One symmetric smoother application: colours 0..7, then 7..0, in place in z. */
int hpcg_ell_rbgs(hpcg_ell_handle h, int level, const double *r_dev, double *z_dev, void *stream);
/* z = M r on level 0 (Listing 1, stored order; z starts from 0 on every level). */
int hpcg_ell_mg_vcycle(hpcg_ell_handle h, const double *r_dev, double *z_dev, void *stream);
/* PCG as hpcg_pcg_solve (FP64, b and x in NATURAL order, x holds x0 on entry);
 * the host reads the residual after every iteration when rel_tol > 0. */
int hpcg_ell_pcg_solve(hpcg_ell_handle h, const double *b_dev, double *x_dev, int max_iters, double rel_tol, hpcg_stats *stats,
                       void *stream);

/* --- two sub-domains with colour-aware halo exchange ---------------------------- */
/* The data distribution of the reference implementation (the paper's section on
 * distributed execution) gives each node a box of the grid plus the boundary
 * planes of its neighbours (halos), and the reference's smoother exchanges,
 * after each colour, only the halo values of that colour.  This engine splits
 * every level into the slabs z < nz/2 and z >= nz/2, each with its own rows
 * (a sliced-ELL matrix grouped by colour, as hpcg_ell_*, whose columns index
 * [own rows | halo rows]) and a copy of the neighbour's boundary plane, and runs
 * the two slabs on one GPU one after the other on `stream`; an exchange is a
 * device-to-device gather from the neighbour's vector.  Exchanges: after colour
 * phase k the halo rows of colour k; after refinement colour 0 (the injected
 * points); before an SpMV the whole halo.  The level calls give the same values
 * as hpcg_ell_* on the whole grid (bit for bit with exact = 1); dot products sum
 * per slab, then over the slabs.  Vectors are in NATURAL order.
 *
 * Grid rules: those of hpcg_setup, and nz divisible by 2^levels (each slab keeps
 * at least one plane on the coarsest level).  hpcg_split_setup builds the maps
 * on the host and allocates the matrices with cudaMalloc (about the size of
 * hpcg_ell_setup's).
 * Errors: INVALID_ARG for null or aliased pointers, a level or slab out of
 * range, or the grid rules; CUDA when an allocation or launch fails. */
typedef struct hpcg_split_ctx *hpcg_split_handle;
int hpcg_split_setup(int nx, int ny, int nz, int levels, int exact, hpcg_split_handle *out);
int hpcg_split_destroy(hpcg_split_handle h);
/* info_host[0..1] = the slab's z range [z0, z1); [2] own rows; [3] halo rows;
 * [4..12] own rows' colour starts; [13..21] halo rows' colour starts. */
int hpcg_split_info(hpcg_split_handle h, int level, int domain, long *info_host);
/* Halo values copied and exchange steps since setup (host counters). */
int hpcg_split_exchange_count(hpcg_split_handle h, long *values_host, long *steps_host);
/* y = A x on `level`. */
int hpcg_split_spmv(hpcg_split_handle h, int level, const double *x_dev, double *y_dev, void *stream);
/* One symmetric smoother application (colours 0..7, 7..0) from z, in place. */
int hpcg_split_rbgs(hpcg_split_handle h, int level, const double *r_dev, double *z_dev, void *stream);
/* z = M r (Listing 1). */
int hpcg_split_mg_vcycle(hpcg_split_handle h, const double *r_dev, double *z_dev, void *stream);
/* PCG as hpcg_pcg_solve (FP64; x holds x0 on entry). */
int hpcg_split_pcg_solve(hpcg_split_handle h, const double *b_dev, double *x_dev, int max_iters, double rel_tol,
                         hpcg_stats *stats, void *stream);

/* --- measurement aid ------------------------------------------------------------------ */
/* Not part of the paper: the FP64 fused multiply-add issue rate of the current
 * GPU, the denominator of the FP64 term of a binding roofline (on this GPU the
 * FP64 pipe is narrow enough to bind some kernels before memory does).  Launches
 * `blocks` blocks of 256 threads, each thread 8 independent chains of `iters`
 * dependent FMAs (one untimed warm-up launch, then one launch timed with CUDA
 * events on `stream`); sink_dev (device, blocks*256 doubles, caller-owned)
 * receives each thread's sum so that no FMA is optimised away.  *ms_host gets
 * the timed launch's milliseconds and *fma_host the FMA instructions it
 * executed per thread summed over threads (divide by 32 for warp-level
 * instructions).  Synchronises `stream`.  Errors: INVALID_ARG for a
 * non-positive count or null pointer; CUDA for a failed launch. */
int hpcg_probe_fp64_rate(int blocks, int iters, double *sink_dev, double *ms_host, double *fma_host, void *stream);

/* Diagnostic, not part of the paper: the int64 -> FP64 conversion that the
 * fixed-point and block-floating-point kernels build on the integer pipe,
 * out_dev[i] = q_i 2^(E_i - 1080) rounded to nearest (ties to even), beside
 * ref_dev[i] = CUDA's round-to-nearest __ll2double_rn(q_i) scaled exactly by
 * 2^(E_i - 1080), for n pairs (device arrays: q int64 with |q_i| < 2^63, E int32
 * in [64, 2000], outputs FP64).  The two agree bit for bit when the kernels'
 * conversion is right.  Errors: INVALID_ARG for n < 0 or a null pointer. */
int hpcg_fx_to_double_check(long n, const long long *q_dev, const int *e_dev, double *out_dev, double *ref_dev, void *stream);

/* --- diagnostics ------------------------------------------------------------------ */
/* Bounds-checking build (not part of the paper; the library compiled with
 * -DHPCG_BOUNDS_CHECK, paper_2304_08232_gb300/build.py build_checked): the
 * kernels of the default FP64 path (colour-pair runs in block floating point,
 * the staged SpMV, the CG updates, dot products and reductions, the level-vector
 * conversions) check every index range they touch against its array's extent;
 * a miss is counted, the first one recorded, and the access skipped (nothing
 * traps).  Synchronises with the device (a symbol copy).  *count_host receives
 * the violations since the last reset, first_host[0..1] the source line of the
 * first one and its index (-1, -1 if none); reset != 0 clears the record.
 * Returns UNSUPPORTED from the normal build (count 0). */
int hpcg_bounds_status(long long *count_host, long long *first_host, int reset);
const char *hpcg_strerror(int status);
/* Text of the last CUDA error seen by the library in this process (thread-unsafe). */
const char *hpcg_last_cuda_error(void);
/* Number of kernel launches the library has issued in this process. */
long hpcg_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* HPCG_GB300_H */
