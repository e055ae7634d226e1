/*
 * hpcg_oracle.c -- plain, slow, FP64 CPU oracle for the HPCG-on-GraphBLAS hot
 * path (Scolari & Yzelman, "Effective implementation of the High Performance
 * Conjugate Gradient benchmark on GraphBLAS").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code with the CUDA library.
 *
 * Style: single-threaded, explicit loops, double precision, compiled with
 * -ffp-contract=off so that every a*b+c is two roundings.  The rows of one
 * SpMV and of one colour step are independent, so their loops carry OpenMP
 * pragmas: a plain build ignores them; a build with -fopenmp (the CPU
 * baseline on all host cores, the parallelisation of the reference code that
 * the paper compares against: one parallel loop per colour) computes the same
 * bits, since every row's arithmetic is unchanged.  Dot products stay
 * sequential.  The operator is
 * stored explicitly in CRS (Section III-A keeps A in a sparse matrix and the
 * diagonal in its own vector A_diag), rows in natural order
 * i = x + nx*(y + ny*z), each row's nonzeros in ascending column index.
 *
 * Every function names the passage of the paper it follows.  Readings where
 * the paper is silent (right-hand side, symmetric sweep, coarse operators, CG
 * recurrence) are listed beside the function that takes them.
 *
 * Parity pins live in tests/test_oracle_*.py (closed forms, Kronecker
 * structure, dense triangular Gauss-Seidel, dense direct solves).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_LEVELS 8

typedef struct {
  int nx, ny, nz;
  long n, nnz;
  long *row_ptr; /* n+1 */
  int *col;      /* nnz */
  double *val;   /* nnz */
  double *diag;  /* n: A_diag (Section III-A, Listing 3) */
  int *color;    /* n: greedy colour of each row (Section III-A) */
  int ncolors;
  int *f2c;      /* n of the next coarser level: fine row injected into each coarse row; NULL on the coarsest */
  /* working vectors of this level for the V-cycle (Listing 1) */
  double *r, *z, *f, *tmp;
} orc_level;

typedef struct {
  int levels;
  int symmetric; /* 1: forward colours then backward colours (default); 0: forward only */
  orc_level lv[ORC_MAX_LEVELS];
} orc_problem;

/* ------------------------------------------------------------------------ */
/* Input generation (Section II-B; 27-point heat-diffusion stencil, Sec. II-C:
 * "8 to 27 nonzeroes per row").  Row i couples to every grid point whose
 * coordinates differ from its own by at most one in each direction and that
 * lies inside the grid (no ghost points).  Diagonal 26 (+ kappa_i for the
 * diagonal-coefficient field of the differentiable form), off-diagonal -1.
 * Entries are emitted with dz outermost, dx innermost, i.e. in ascending
 * column index.  Returns the number of entries (8..27). */
int orc_row_entries(int nx, int ny, int nz, const double *kappa, long i, int *cols, double *vals) {
  int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
  int cnt = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int zz = z + dz;
    if (zz < 0 || zz >= nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int yy = y + dy;
      if (yy < 0 || yy >= ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        int xx = x + dx;
        if (xx < 0 || xx >= nx) continue;
        long j = xx + (long)nx * (yy + (long)ny * zz);
        cols[cnt] = (int)j;
        if (j == i)
          vals[cnt] = 26.0 + (kappa ? kappa[i] : 0.0);
        else
          vals[cnt] = -1.0;
        ++cnt;
      }
    }
  }
  return cnt;
}

/* Build the CRS arrays of one level by calling the row generator in order. */
static int build_level(orc_level *L, int nx, int ny, int nz, const double *kappa) {
  L->nx = nx; L->ny = ny; L->nz = nz;
  L->n = (long)nx * ny * nz;
  L->row_ptr = (long *)malloc(sizeof(long) * (L->n + 1));
  /* nonzeros: at most 27 per row; shrink later is unnecessary for an oracle */
  L->col = (int *)malloc(sizeof(int) * 27 * L->n);
  L->val = (double *)malloc(sizeof(double) * 27 * L->n);
  L->diag = (double *)malloc(sizeof(double) * L->n);
  if (!L->row_ptr || !L->col || !L->val || !L->diag) return -1;
  long k = 0;
  L->row_ptr[0] = 0;
  for (long i = 0; i < L->n; ++i) {
    int cnt = orc_row_entries(nx, ny, nz, kappa, i, L->col + k, L->val + k);
    /* A_diag: the diagonal kept in its own vector (Section III-A). */
    for (int e = 0; e < cnt; ++e)
      if (L->col[k + e] == i) L->diag[i] = L->val[k + e];
    k += cnt;
    L->row_ptr[i + 1] = k;
  }
  L->nnz = k;
  return 0;
}

/* Greedy colouring (Section III-A): rows are visited in increasing index; each
 * row takes the smallest colour that no already-coloured row it directly
 * depends on (a nonzero A_ij, j != i) carries. */
static void greedy_color(orc_level *L) {
  L->color = (int *)malloc(sizeof(int) * L->n);
  for (long i = 0; i < L->n; ++i) L->color[i] = -1;
  int maxc = 0;
  for (long i = 0; i < L->n; ++i) {
    int used[64];
    memset(used, 0, sizeof(used));
    for (long k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) {
      long j = L->col[k];
      if (j != i && L->color[j] >= 0 && L->color[j] < 64) used[L->color[j]] = 1;
    }
    int c = 0;
    while (used[c]) ++c;
    L->color[i] = c;
    if (c + 1 > maxc) maxc = c + 1;
  }
  L->ncolors = maxc;
}

/* Straight injection (Section II-F): coarse point (xc,yc,zc) takes the fine
 * value at the lowest corner (2xc,2yc,2zc) of its octet.  Returns a new array
 * of ncx*ncy*ncz fine-row indices. */
static int *make_f2c(int nfx, int nfy, int ncx, int ncy, int ncz) {
  int *f2c = (int *)malloc(sizeof(int) * (long)ncx * ncy * ncz);
  for (int zc = 0; zc < ncz; ++zc)
    for (int yc = 0; yc < ncy; ++yc)
      for (int xc = 0; xc < ncx; ++xc) {
        long c = xc + (long)ncx * (yc + (long)ncy * zc);
        long f = 2L * xc + (long)nfx * (2L * yc + (long)nfy * 2L * zc);
        f2c[c] = (int)f;
      }
  return f2c;
}

void orc_free(orc_problem *p);

/* Builds the hierarchy.  Coarse operators: the paper does not say how
 * mg_level.A is formed for coarser levels (Listing 1); this oracle regenerates
 * the same 27-point stencil on the halved grid, and, when a diagonal field
 * kappa is present, gives each coarse row the kappa of its injected fine row.
 * Each dimension must be divisible by 2^(levels-1) and >= 2 on the coarsest
 * level.  Returns NULL on invalid sizes. */
orc_problem *orc_create(int nx, int ny, int nz, int levels, const double *kappa) {
  if (levels < 1 || levels > ORC_MAX_LEVELS) return NULL;
  int div = 1 << (levels - 1);
  if (nx < 2 || ny < 2 || nz < 2) return NULL;
  if (nx % div || ny % div || nz % div) return NULL;
  if (nx / div < 2 || ny / div < 2 || nz / div < 2) return NULL;
  orc_problem *p = (orc_problem *)calloc(1, sizeof(orc_problem));
  p->levels = levels;
  p->symmetric = 1;
  double *kap = NULL; /* kappa of the level being built */
  if (kappa) {
    long n0 = (long)nx * ny * nz;
    kap = (double *)malloc(sizeof(double) * n0);
    memcpy(kap, kappa, sizeof(double) * n0);
  }
  for (int l = 0; l < levels; ++l) {
    int sx = nx >> l, sy = ny >> l, sz = nz >> l;
    if (l > 0) {
      orc_level *F = &p->lv[l - 1];
      F->f2c = make_f2c(F->nx, F->ny, sx, sy, sz);
      if (kap) {
        long nc = (long)sx * sy * sz;
        double *kc = (double *)malloc(sizeof(double) * nc);
        for (long c = 0; c < nc; ++c) kc[c] = kap[F->f2c[c]];
        free(kap);
        kap = kc;
      }
    }
    orc_level *L = &p->lv[l];
    if (build_level(L, sx, sy, sz, kap) != 0) { free(kap); orc_free(p); return NULL; }
    greedy_color(L);
    L->r = (double *)calloc(L->n, sizeof(double));
    L->z = (double *)calloc(L->n, sizeof(double));
    L->f = (double *)calloc(L->n, sizeof(double));
    L->tmp = (double *)calloc(L->n, sizeof(double));
  }
  free(kap);
  return p;
}

void orc_free(orc_problem *p) {
  if (!p) return;
  for (int l = 0; l < ORC_MAX_LEVELS; ++l) {
    orc_level *L = &p->lv[l];
    free(L->row_ptr); free(L->col); free(L->val); free(L->diag); free(L->color); free(L->f2c);
    free(L->r); free(L->z); free(L->f); free(L->tmp);
  }
  free(p);
}

void orc_set_symmetric(orc_problem *p, int symmetric) { p->symmetric = symmetric; }
/* Threads the parallel loops use: 1 in the plain build. */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
int orc_levels(const orc_problem *p) { return p->levels; }
long orc_level_n(const orc_problem *p, int l) { return p->lv[l].n; }
long orc_level_nnz(const orc_problem *p, int l) { return p->lv[l].nnz; }
int orc_level_ncolors(const orc_problem *p, int l) { return p->lv[l].ncolors; }
void orc_level_dims(const orc_problem *p, int l, int *d) { d[0] = p->lv[l].nx; d[1] = p->lv[l].ny; d[2] = p->lv[l].nz; }

void orc_export_csr(const orc_problem *p, int l, long *row_ptr, int *col, double *val) {
  const orc_level *L = &p->lv[l];
  memcpy(row_ptr, L->row_ptr, sizeof(long) * (L->n + 1));
  memcpy(col, L->col, sizeof(int) * L->nnz);
  memcpy(val, L->val, sizeof(double) * L->nnz);
}
void orc_export_colors(const orc_problem *p, int l, int *out) { memcpy(out, p->lv[l].color, sizeof(int) * p->lv[l].n); }
void orc_export_diag(const orc_problem *p, int l, double *out) { memcpy(out, p->lv[l].diag, sizeof(double) * p->lv[l].n); }
void orc_export_row_nnz(const orc_problem *p, int l, int *out) {
  const orc_level *L = &p->lv[l];
  for (long i = 0; i < L->n; ++i) out[i] = (int)(L->row_ptr[i + 1] - L->row_ptr[i]);
}
/* f2c of level l maps level l+1 rows to level l rows; l must not be the coarsest */
void orc_export_f2c(const orc_problem *p, int l, int *out) { memcpy(out, p->lv[l].f2c, sizeof(int) * p->lv[l + 1].n); }
/* The right-hand side (which = 0) or result (which = 1) that the last orc_mg
 * call left on coarse level l >= 1: the restricted residual r_c that Listing 1
 * hands to the coarser level, and the z_c that level returned. */
void orc_export_coarse(const orc_problem *p, int l, int which, double *out) {
  memcpy(out, which ? p->lv[l].z : p->lv[l].r, sizeof(double) * p->lv[l].n);
}

/* ------------------------------------------------------------------------ */
/* spmv / mxv (Section II-C): y_i = sum_j A_ij x_j, left to right over the
 * row's entries in ascending column order. */
void orc_spmv(const orc_problem *p, int l, const double *x, double *y) {
  const orc_level *L = &p->lv[l];
#pragma omp parallel for schedule(static)
  for (long i = 0; i < L->n; ++i) {
    double s = 0.0;
    for (long k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) s += L->val[k] * x[L->col[k]];
    y[i] = s;
  }
}

/* Same product for a list of rows only, generating each row on the fly; used to
 * check sampled outputs of grids too large to hold in CRS. */
void orc_spmv_rows(int nx, int ny, int nz, const double *kappa, long nrows, const long *rows, const double *x, double *y) {
  int cols[27];
  double vals[27];
  for (long t = 0; t < nrows; ++t) {
    int cnt = orc_row_entries(nx, ny, nz, kappa, rows[t], cols, vals);
    double s = 0.0;
    for (int e = 0; e < cnt; ++e) s += vals[e] * x[cols[e]];
    y[t] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* One colour step of the red-black (multi-colour) Gauss-Seidel pass
 * (Listings 2 and 3): a masked mxv forms tmp_i = sum_j A_ij z_j for every row i
 * of colour k (the sum includes the diagonal term), then every such row is
 * updated as z_i <- (r_i - tmp_i + z_i * d_i) / d_i. */
void orc_rbgs_color_step(const orc_problem *p, int l, int k, const double *r, double *z) {
  const orc_level *L = &p->lv[l];
  double *tmp = L->tmp;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < L->n; ++i) {
    if (L->color[i] != k) continue;
    double s = 0.0;
    for (long e = L->row_ptr[i]; e < L->row_ptr[i + 1]; ++e) s += L->val[e] * z[L->col[e]];
    tmp[i] = s;
  }
#pragma omp parallel for schedule(static)
  for (long i = 0; i < L->n; ++i) {
    if (L->color[i] != k) continue;
    double d = L->diag[i];
    double v = r[i] - tmp[i] + z[i] * d;
    z[i] = v / d;
  }
}

/* One smoother application.  The paper's listings show the forward pass
 * (colours 0..c-1, Listing 3's loop bound); the smoother it replaces, SGS
 * (Section II-E), follows the forward sweep by a backward sweep, and the
 * replacement must keep the preconditioner symmetric.  Reading used here: one
 * application = forward colours 0..c-1 then backward colours c-1..0.  With
 * symmetric == 0 only the forward pass runs (ablation). */
void orc_rbgs(const orc_problem *p, int l, const double *r, double *z) {
  const orc_level *L = &p->lv[l];
  for (int k = 0; k < L->ncolors; ++k) orc_rbgs_color_step(p, l, k, r, z);
  if (p->symmetric)
    for (int k = L->ncolors - 1; k >= 0; --k) orc_rbgs_color_step(p, l, k, r, z);
}

/* Restriction by injection (Section II-F, III-B): rc[c] = v[f2c[c]]. */
void orc_restrict(const orc_problem *p, int l, const double *v, double *rc) {
  const orc_level *F = &p->lv[l];
  long nc = p->lv[l + 1].n;
  for (long c = 0; c < nc; ++c) rc[c] = v[F->f2c[c]];
}

/* Refinement = transpose of injection (Section II-F, III-B): adds the coarse
 * value at the injected fine point and zero elsewhere: z[f2c[c]] += zc[c]. */
void orc_prolong_add(const orc_problem *p, int l, const double *zc, double *z) {
  const orc_level *F = &p->lv[l];
  long nc = p->lv[l + 1].n;
  for (long c = 0; c < nc; ++c) z[F->f2c[c]] = z[F->f2c[c]] + zc[c];
}

/* The MG preconditioner, Listing 1, recursively from level l.  z holds the
 * initial guess on entry (the caller zeroes it: Listing 1 starts every level
 * from z = 0) and the result on exit.  One smoother application before and
 * one after the coarse correction; on the coarsest level one application and
 * return. */
void orc_mg(const orc_problem *p, int l, const double *r, double *z) {
  const orc_level *L = &p->lv[l];
  orc_rbgs(p, l, r, z);                       /* pre-smoothing */
  if (l == p->levels - 1) return;             /* coarsest level */
  orc_spmv(p, l, z, L->f);                    /* f <- A z */
  for (long i = 0; i < L->n; ++i) L->tmp[i] = r[i] - L->f[i];
  const orc_level *C = &p->lv[l + 1];
  orc_restrict(p, l, L->tmp, C->r);           /* r_c <- restrict(r - f) */
  for (long c = 0; c < C->n; ++c) C->z[c] = 0.0; /* z_c <- 0 */
  orc_mg(p, l + 1, C->r, C->z);               /* z_c <- MG(coarser, z_c, r_c) */
  orc_prolong_add(p, l, C->z, z);             /* z <- z + refine(z_c) */
  orc_rbgs(p, l, r, z);                       /* post-smoothing */
}

/* Top-level preconditioner application z = M r (z starts from 0). */
void orc_mg_apply(const orc_problem *p, const double *r, double *z) {
  for (long i = 0; i < p->lv[0].n; ++i) z[i] = 0.0;
  orc_mg(p, 0, r, z);
}

/* ------------------------------------------------------------------------ */
static double dot(long n, const double *a, const double *b) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Preconditioned CG (Section II-C), in HPCG's iteration order:
 *   r = b - A x;  ||r0|| = ||r||
 *   for k = 1..max_iters:
 *     z = M r
 *     if k == 1: p = z, rtz = r.z   else: rtz' = r.z, beta = rtz'/rtz, p = z + beta p
 *     Ap = A p;  alpha = rtz / (p.Ap)
 *     x = x + alpha p;  r = r - alpha Ap
 *     hist[k-1] = ||r|| / ||r0||;  stop if <= tol
 * The paper states only "until the residual is smaller than a threshold or a
 * fixed number of iterations"; the relative 2-norm test is the reading used.
 * With precond == 0, z = r (plain CG).  x holds x0 on entry.
 * Returns the number of iterations run; hist needs max_iters entries. */
int orc_pcg(const orc_problem *p, const double *b, double *x, int max_iters, double tol, int precond, double *hist) {
  long n = p->lv[0].n;
  double *r = (double *)malloc(sizeof(double) * n);
  double *z = (double *)malloc(sizeof(double) * n);
  double *pp = (double *)malloc(sizeof(double) * n);
  double *Ap = (double *)malloc(sizeof(double) * n);
  orc_spmv(p, 0, x, Ap);
  for (long i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
  double normr0 = sqrt(dot(n, r, r));
  double rtz = 0.0;
  int k = 0;
  if (normr0 == 0.0) goto done;
  for (k = 1; k <= max_iters; ++k) {
    if (precond)
      orc_mg_apply(p, r, z);
    else
      for (long i = 0; i < n; ++i) z[i] = r[i];
    if (k == 1) {
      for (long i = 0; i < n; ++i) pp[i] = z[i];
      rtz = dot(n, r, z);
    } else {
      double rtz_new = dot(n, r, z);
      double beta = rtz_new / rtz;
      rtz = rtz_new;
      for (long i = 0; i < n; ++i) pp[i] = z[i] + beta * pp[i];
    }
    orc_spmv(p, 0, pp, Ap);
    double alpha = rtz / dot(n, pp, Ap);
    for (long i = 0; i < n; ++i) x[i] = x[i] + alpha * pp[i];
    for (long i = 0; i < n; ++i) r[i] = r[i] - alpha * Ap[i];
    double rel = sqrt(dot(n, r, r)) / normr0;
    if (hist) hist[k - 1] = rel;
    if (rel <= tol) break;
  }
  if (k > max_iters) k = max_iters;
done:
  free(r); free(z); free(pp); free(Ap);
  return k;
}
