/*
 * gk_oracle.c -- sequential CPU oracle (test infrastructure only; see the
 * header).  Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC.
 *
 * Each function states the passage of arXiv:2006.16852 (or the textbook
 * definition the paper cites) that it follows.  Nothing here is blocked,
 * fused or reordered beyond what the definition says.
 */
#include "gk_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Sparse matrix-vector product                                              */
/* ------------------------------------------------------------------------ */

/* Section 4.2: the simple apply x = A b and the advanced apply
 * x = alpha*A*b + beta*x, with "simple = advanced(alpha=1, beta=0)".
 * Row sum: s = 0; for k in increasing order, s = fma(a_ik, b_k, s).
 * beta == 0 does not read the old output (BLAS convention), so a NaN there
 * does not propagate; otherwise the result is fma(beta, y_old, alpha*s). */
/* Rows are independent and each row's sum runs in increasing k whatever
 * thread takes the row, so splitting the rows over threads (OpenMP, static
 * chunks) leaves every result bit unchanged; the dot products and the
 * solvers' vector steps stay sequential. */
void or_csr_spmv(int64_t n_rows, const int32_t* rowptr, const int32_t* col, const double* val,
                 const double* x, double alpha, double beta, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_rows; ++i) {
    double s = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s = fma(val[k], x[col[k]], s);
    double as = alpha * s;
    y[i] = (beta == 0.0) ? as : fma(beta, y[i], as);
  }
}

/* Threads the row loops of the SpMVs may use (<= 0: all the host's cores);
 * returns the number they will use.  1 when built without OpenMP. */
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n <= 0) n = omp_get_num_procs();
  omp_set_num_threads(n);
  return n;
#else
  (void)n;
  return 1;
#endif
}

/* Error-free transformations (Ogita, Rump, Oishi, "Accurate sum and dot
 * product", SIAM J. Sci. Comput. 26(6), 2005): TwoSum (Knuth) and
 * TwoProduct via fma; Dot2 accumulates the rounding errors separately and is
 * as accurate as a dot product computed in twice the working precision. */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}

static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}

void or_csr_spmv_dot2(int64_t n_rows, const int32_t* rowptr, const int32_t* col, const double* val,
                      const double* x, double* y_acc, double* abs_ax) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_rows; ++i) {
    double p = 0.0, s = 0.0, bound = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      double h, r, q;
      two_prod(val[k], x[col[k]], &h, &r);
      two_sum(p, h, &p, &q);
      s += q + r;
      bound += fabs(val[k]) * fabs(x[col[k]]);
    }
    y_acc[i] = p + s;
    abs_ax[i] = bound;
  }
}

/* ------------------------------------------------------------------------ */
/* Dense vector kernels (the scale / add_scaled / dot of Section 4.2)        */
/* ------------------------------------------------------------------------ */

double or_dot(int64_t n, const double* x, const double* y) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

double or_norm2(int64_t n, const double* x) { return sqrt(or_dot(n, x, x)); }

/* ------------------------------------------------------------------------ */
/* Jacobi preconditioners (Section 3.2; block inversion by Gauss-Jordan     */
/* elimination with pivoting, Section 7.5)                                    */
/* ------------------------------------------------------------------------ */

/* Diagonal entry a_ii of a CSR row, or 0 with *found = 0 when absent. */
static double diag_entry(const int32_t* rowptr, const int32_t* col, const double* val, int64_t i,
                         int* found) {
  for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    if (col[k] == i) {
      *found = 1;
      return val[k];
    }
  }
  *found = 0;
  return 0.0;
}

/* Scalar Jacobi, Section 3.2 ("diagonal scaling"): M = diag(A). */
int or_jacobi_scalar(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     double* dinv) {
  for (int64_t i = 0; i < n; ++i) {
    int found;
    double d = diag_entry(rowptr, col, val, i, &found);
    if (!found || d == 0.0) return OR_ERR_SINGULAR;
    dinv[i] = 1.0 / d;
  }
  return OR_OK;
}

int64_t or_block_jacobi_size(int64_t n, int32_t bs) {
  if (bs <= 0) return 0;
  int64_t full = n / bs, last = n % bs;
  return full * (int64_t)bs * bs + last * last;
}

/* Block-Jacobi generate, Sections 3.2 and 7.5: diagonal block D_k holds the
 * entries of A in rows and columns [k*bs, min((k+1)*bs, n)); it is inverted
 * by Gauss-Jordan elimination on the augmented matrix [D_k | I] with partial
 * (row) pivoting.  Pivot: the largest |entry| in the column at or below the
 * diagonal, the lowest row on ties.  Pivot row scaled by its reciprocal;
 * every other row eliminated with w_ij = fma(-w_ik, w_kj, w_ij). */
int or_block_jacobi_generate(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                             int32_t bs, double* blocks, int64_t* bad_block) {
  if (bs <= 0) return OR_ERR_ARG;
  int64_t nblocks = (n + bs - 1) / bs;
  double* w = (double*)malloc(sizeof(double) * (size_t)bs * 2 * bs);
  if (!w) return OR_ERR_ARG;
  int64_t off = 0;
  for (int64_t b = 0; b < nblocks; ++b) {
    int64_t r0 = b * bs;
    int64_t m = (r0 + bs <= n) ? bs : n - r0;
    int64_t wd = 2 * m; /* row stride of the augmented matrix */
    memset(w, 0, sizeof(double) * (size_t)m * wd);
    for (int64_t i = 0; i < m; ++i) {
      for (int64_t k = rowptr[r0 + i]; k < rowptr[r0 + i + 1]; ++k) {
        int64_t c = col[k];
        if (c >= r0 && c < r0 + m) w[i * wd + (c - r0)] = val[k];
      }
      w[i * wd + m + i] = 1.0;
    }
    for (int64_t k = 0; k < m; ++k) {
      int64_t piv = k;
      double best = fabs(w[k * wd + k]);
      for (int64_t i = k + 1; i < m; ++i) {
        double a = fabs(w[i * wd + k]);
        if (a > best) {
          best = a;
          piv = i;
        }
      }
      if (best == 0.0) {
        free(w);
        if (bad_block) *bad_block = b;
        return OR_ERR_SINGULAR;
      }
      if (piv != k) {
        for (int64_t j = 0; j < wd; ++j) {
          double t = w[k * wd + j];
          w[k * wd + j] = w[piv * wd + j];
          w[piv * wd + j] = t;
        }
      }
      double rcp = 1.0 / w[k * wd + k];
      for (int64_t j = 0; j < wd; ++j) w[k * wd + j] = w[k * wd + j] * rcp;
      for (int64_t i = 0; i < m; ++i) {
        if (i == k) continue;
        double f = w[i * wd + k];
        for (int64_t j = 0; j < wd; ++j) w[i * wd + j] = fma(-f, w[k * wd + j], w[i * wd + j]);
      }
    }
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < m; ++j) blocks[off + i * m + j] = w[i * wd + m + j];
    off += m * m;
  }
  free(w);
  return OR_OK;
}

/* z = M^{-1} r.  Block case: z_i = sum_j (D_k^{-1})_{ij} r_j, a dense
 * row-major matvec per block with the sum in increasing j via fma. */
void or_precond_apply(int64_t n, const or_precond* P, const double* r, double* z) {
  if (!P || P->kind == OR_PREC_NONE) {
    for (int64_t i = 0; i < n; ++i) z[i] = r[i];
    return;
  }
  if (P->kind == OR_PREC_SCALAR_JACOBI) {
    for (int64_t i = 0; i < n; ++i) z[i] = P->dinv[i] * r[i];
    return;
  }
  int64_t bs = P->block_size;
  int64_t off = 0;
  for (int64_t r0 = 0; r0 < n; r0 += bs) {
    int64_t m = (r0 + bs <= n) ? bs : n - r0;
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < m; ++j) s = fma(P->blocks[off + i * m + j], r[r0 + j], s);
      z[r0 + i] = s;
    }
    off += m * m;
  }
}

/* ------------------------------------------------------------------------ */
/* Hybrid ELL + COO split                                                     */
/* ------------------------------------------------------------------------ */

/* Brute force over every candidate width K = 0 .. max row length. */
int64_t or_hyb_width(int64_t n_rows, const int32_t* rowptr, int64_t vt, int64_t it) {
  int64_t maxlen = 0;
  for (int64_t i = 0; i < n_rows; ++i) {
    int64_t l = rowptr[i + 1] - rowptr[i];
    if (l > maxlen) maxlen = l;
  }
  int64_t bestk = 0, bestcost = -1;
  for (int64_t K = 0; K <= maxlen; ++K) {
    int64_t coo = 0;
    for (int64_t i = 0; i < n_rows; ++i) {
      int64_t l = rowptr[i + 1] - rowptr[i];
      if (l > K) coo += l - K;
    }
    int64_t cost = K * n_rows * (vt + it) + coo * (vt + 2 * it);
    if (bestcost < 0 || cost < bestcost) {
      bestcost = cost;
      bestk = K;
    }
  }
  return bestk;
}

/* ------------------------------------------------------------------------ */
/* Krylov solvers                                                             */
/* ------------------------------------------------------------------------ */

static int is_finite(double v) { return isfinite(v) != 0; }

/* r = b - A x, with A x by the ordered row sum of or_csr_spmv. */
static void residual(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const double* b, const double* x, double* r) {
  or_csr_spmv(n, rowptr, col, val, x, 1.0, 0.0, r);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
}

/* Stopping criteria of Section 2.5, combined by logical OR (Listing 1):
 * ResidualNormReduction first, then Iteration.  A non-finite residual norm
 * ends the solve (it can neither converge nor recover). */
static int check_stop(double rnorm, double tol_abs, int64_t k, int64_t max_iters) {
  if (!is_finite(rnorm)) return OR_STOP_NAN;
  if (rnorm <= tol_abs) return OR_STOP_CONVERGED;
  if (k >= max_iters) return OR_STOP_MAX_ITERS;
  return OR_STOP_NONE;
}

static void finish(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                   const double* b, const double* x, double ref, double rnorm, or_status* st,
                   double* work) {
  residual(n, rowptr, col, val, b, x, work);
  st->spmvs += 1;
  st->rel_res = rnorm / ref;
  st->rel_res_true = or_norm2(n, work) / ref;
  st->ref_norm = ref;
}

/* Preconditioned CG (the CG of Section 3.1, Listing 1; the textbook
 * algorithm of Saad, "Iterative Methods for Sparse Linear Systems", which the
 * paper cites).  With M the preconditioner:
 *   r = b - A x;  z = M^{-1} r;  p = z;  rho = r.z
 *   repeat: q = A p;  sigma = p.q;  alpha = rho / sigma
 *           x = x + alpha p;  r = r - alpha q
 *           z = M^{-1} r;  rho' = r.z;  beta = rho' / rho;  p = z + beta p
 * sigma <= 0 (or not finite) on a nonzero p is a breakdown. */
int or_cg(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
          const or_precond* P, const double* b, double* x, const or_criteria* crit,
          or_status* st, double* res_hist) {
  if (n < 0 || !crit || !st) return OR_ERR_ARG;
  memset(st, 0, sizeof(*st));
  double* r = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  if (!r || !z || !p || !q) {
    free(r); free(z); free(p); free(q);
    return OR_ERR_ARG;
  }
  residual(n, rowptr, col, val, b, x, r);
  st->spmvs = 1;
  double bnorm = or_norm2(n, b);
  double rnorm = or_norm2(n, r);
  double ref = crit->rel_to_b ? bnorm : rnorm;
  if (ref == 0.0) ref = 1.0; /* b = 0 (or r_0 = 0): absolute criterion */
  double tol = crit->reduction_factor * ref;
  or_precond_apply(n, P, r, z);
  for (int64_t i = 0; i < n; ++i) p[i] = z[i];
  double rho = or_dot(n, r, z);
  int64_t k = 0;
  int stop;
  if (res_hist) res_hist[0] = rnorm / ref;
  while ((stop = check_stop(rnorm, tol, k, crit->max_iters)) == OR_STOP_NONE) {
    or_csr_spmv(n, rowptr, col, val, p, 1.0, 0.0, q);
    st->spmvs += 1;
    double sigma = or_dot(n, p, q);
    if (!is_finite(sigma)) { stop = OR_STOP_NAN; break; }
    if (sigma <= 0.0) { stop = OR_STOP_BREAKDOWN; break; }
    double alpha = rho / sigma;
    for (int64_t i = 0; i < n; ++i) x[i] = fma(alpha, p[i], x[i]);
    for (int64_t i = 0; i < n; ++i) r[i] = fma(-alpha, q[i], r[i]);
    k += 1;
    rnorm = or_norm2(n, r);
    if (res_hist) res_hist[k] = rnorm / ref;
    or_precond_apply(n, P, r, z);
    double rho_new = or_dot(n, r, z);
    double beta = rho_new / rho;
    for (int64_t i = 0; i < n; ++i) p[i] = fma(beta, p[i], z[i]);
    rho = rho_new;
  }
  st->iters = k;
  st->stop_reason = stop;
  finish(n, rowptr, col, val, b, x, ref, rnorm, st, q);
  free(r); free(z); free(p); free(q);
  return OR_OK;
}

/* Preconditioned BiCGSTAB (Section 3.1, Listing 3; van der Vorst 1992 in the
 * form of Barrett et al., "Templates for the Solution of Linear Systems",
 * 1994), shadow residual r^ = r_0:
 *   rho = r^.r;  beta = (rho/rho_prev)(alpha/omega);  p = r + beta (p - omega v)
 *   p^ = M^{-1} p;  v = A p^;  alpha = rho / (r^.v);  s = r - alpha v
 *   if ||s|| meets the criterion: x = x + alpha p^ and stop (half step)
 *   s^ = M^{-1} s;  t = A s^;  omega = (t.s)/(t.t)
 *   x = x + alpha p^ + omega s^;  r = s - omega t
 * rho = 0, r^.v = 0, t.t = 0 or omega = 0 are breakdowns.  A half-step exit
 * counts as one iteration. */
int or_bicgstab(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                const or_precond* P, const double* b, double* x, const or_criteria* crit,
                or_status* st, double* res_hist) {
  if (n < 0 || !crit || !st) return OR_ERR_ARG;
  memset(st, 0, sizeof(*st));
  size_t sz = sizeof(double) * (size_t)(n + 1);
  double *r = malloc(sz), *rh = malloc(sz), *p = malloc(sz), *v = malloc(sz), *ph = malloc(sz),
         *s = malloc(sz), *sh = malloc(sz), *t = malloc(sz);
  if (!r || !rh || !p || !v || !ph || !s || !sh || !t) {
    free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(t);
    return OR_ERR_ARG;
  }
  residual(n, rowptr, col, val, b, x, r);
  st->spmvs = 1;
  double bnorm = or_norm2(n, b);
  double rnorm = or_norm2(n, r);
  double ref = crit->rel_to_b ? bnorm : rnorm;
  if (ref == 0.0) ref = 1.0;
  double tol = crit->reduction_factor * ref;
  for (int64_t i = 0; i < n; ++i) {
    rh[i] = r[i];
    p[i] = 0.0;
    v[i] = 0.0;
  }
  double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  int64_t k = 0;
  int stop;
  if (res_hist) res_hist[0] = rnorm / ref;
  while ((stop = check_stop(rnorm, tol, k, crit->max_iters)) == OR_STOP_NONE) {
    double rho = or_dot(n, rh, r);
    if (!is_finite(rho)) { stop = OR_STOP_NAN; break; }
    if (rho == 0.0) { stop = OR_STOP_BREAKDOWN; break; }
    double beta = (rho / rho_prev) * (alpha / omega);
    for (int64_t i = 0; i < n; ++i) p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]);
    or_precond_apply(n, P, p, ph);
    or_csr_spmv(n, rowptr, col, val, ph, 1.0, 0.0, v);
    st->spmvs += 1;
    double rhv = or_dot(n, rh, v);
    if (!is_finite(rhv)) { stop = OR_STOP_NAN; break; }
    if (rhv == 0.0) { stop = OR_STOP_BREAKDOWN; break; }
    alpha = rho / rhv;
    for (int64_t i = 0; i < n; ++i) s[i] = fma(-alpha, v[i], r[i]);
    double snorm = or_norm2(n, s);
    if (is_finite(snorm) && snorm <= tol) {
      for (int64_t i = 0; i < n; ++i) x[i] = fma(alpha, ph[i], x[i]);
      for (int64_t i = 0; i < n; ++i) r[i] = s[i];
      k += 1;
      rnorm = snorm;
      if (res_hist) res_hist[k] = rnorm / ref;
      stop = OR_STOP_CONVERGED;
      break;
    }
    or_precond_apply(n, P, s, sh);
    or_csr_spmv(n, rowptr, col, val, sh, 1.0, 0.0, t);
    st->spmvs += 1;
    double tt = or_dot(n, t, t);
    double ts = or_dot(n, t, s);
    if (!is_finite(tt) || !is_finite(ts)) { stop = OR_STOP_NAN; break; }
    if (tt == 0.0) { stop = OR_STOP_BREAKDOWN; break; }
    omega = ts / tt;
    for (int64_t i = 0; i < n; ++i) x[i] = fma(omega, sh[i], fma(alpha, ph[i], x[i]));
    for (int64_t i = 0; i < n; ++i) r[i] = fma(-omega, t[i], s[i]);
    rho_prev = rho;
    k += 1;
    rnorm = or_norm2(n, r);
    if (res_hist) res_hist[k] = rnorm / ref;
    if (omega == 0.0) {
      stop = check_stop(rnorm, tol, k, crit->max_iters);
      if (stop == OR_STOP_NONE) stop = OR_STOP_BREAKDOWN;
      break;
    }
  }
  st->iters = k;
  st->stop_reason = stop;
  finish(n, rowptr, col, val, b, x, ref, rnorm, st, t);
  free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(t);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Mixed precision: adaptive block storage and iterative refinement         */
/* ------------------------------------------------------------------------ */

void or_block_jacobi_precision(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                               int32_t bs, const double* blocks, uint8_t* prec, double* kappa) {
  int64_t off = 0, b = 0;
  for (int64_t r0 = 0; r0 < n; r0 += bs, ++b) {
    int64_t m = (r0 + bs <= n) ? bs : n - r0;
    double na = 0.0, ni = 0.0;
    for (int64_t j = 0; j < m; ++j) {
      /* column j of D: |a_{r0+i, r0+j}| summed over i in increasing order */
      double cs = 0.0;
      for (int64_t i = 0; i < m; ++i) {
        double a = 0.0;
        for (int64_t k = rowptr[r0 + i]; k < rowptr[r0 + i + 1]; ++k)
          if (col[k] == r0 + j) a = fabs(val[k]);
        cs += a;
      }
      if (cs > na) na = cs;
      /* column j of D^{-1} (blocks are row-major here) */
      double ci = 0.0;
      for (int64_t i = 0; i < m; ++i) ci += fabs(blocks[off + i * m + j]);
      if (ci > ni) ni = ci;
    }
    double k1 = na * ni;
    if (kappa) kappa[b] = k1;
    prec[b] = (k1 <= 1e-2 * 2048.0) ? 0 : 1;
    off += m * m;
  }
}

typedef struct {
  int32_t kind, bs;
  float* dinv;      /* scalar Jacobi */
  float* blocks;    /* block Jacobi, row-major, values as stored (rounded), scaled */
  float* scale;     /* per block: 2^e */
} or_precond32;

static void precond32_apply(int64_t n, const or_precond32* P, const float* r, float* z) {
  if (P->kind == OR_PREC_NONE) {
    for (int64_t i = 0; i < n; ++i) z[i] = r[i];
  } else if (P->kind == OR_PREC_SCALAR_JACOBI) {
    for (int64_t i = 0; i < n; ++i) z[i] = P->dinv[i] * r[i];
  } else {
    int64_t bs = P->bs, off = 0, b = 0;
    for (int64_t r0 = 0; r0 < n; r0 += bs, ++b) {
      int64_t m = (r0 + bs <= n) ? bs : n - r0;
      for (int64_t i = 0; i < m; ++i) {
        float s = 0.0f;
        for (int64_t j = 0; j < m; ++j) s = fmaf(P->blocks[off + i * m + j], r[r0 + j], s);
        z[r0 + i] = s * P->scale[b];
      }
      off += m * m;
    }
  }
}

static float dotf(int64_t n, const float* x, const float* y) {
  float s = 0.0f;
  for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

int or_ir_cg(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
             const or_precond* P, const double* b, double* x, const or_criteria* crit,
             double inner_reduction, int64_t inner_max, or_status* st, int64_t* outer) {
  if (n < 0 || !crit || !st) return OR_ERR_ARG;
  memset(st, 0, sizeof(*st));
  int64_t nnz = rowptr[n];
  size_t fz = sizeof(float) * (size_t)(n + 1);
  float *val32 = malloc(sizeof(float) * (size_t)(nnz + 1)), *r = malloc(fz), *p = malloc(fz), *q = malloc(fz),
        *z = malloc(fz), *d = malloc(fz);
  double* r64 = malloc(sizeof(double) * (size_t)(n + 1));
  or_precond32 P32 = {OR_PREC_NONE, 1, NULL, NULL, NULL};
  for (int64_t k = 0; k < nnz; ++k) val32[k] = (float)val[k];
  if (P && P->kind == OR_PREC_SCALAR_JACOBI) {
    P32.kind = OR_PREC_SCALAR_JACOBI;
    P32.dinv = malloc(fz);
    for (int64_t i = 0; i < n; ++i) P32.dinv[i] = (float)P->dinv[i];
  } else if (P && P->kind == OR_PREC_BLOCK_JACOBI) {
    int64_t bs = P->block_size, nb = (n + bs - 1) / bs, total = or_block_jacobi_size(n, (int32_t)bs);
    uint8_t* prec = malloc((size_t)nb + 1);
    P32.kind = OR_PREC_BLOCK_JACOBI;
    P32.bs = (int32_t)bs;
    P32.blocks = malloc(sizeof(float) * (size_t)(total + 1));
    P32.scale = malloc(sizeof(float) * (size_t)(nb + 1));
    or_block_jacobi_precision(n, rowptr, col, val, (int32_t)bs, P->blocks, prec, NULL);
    int64_t off = 0, blk = 0;
    for (int64_t r0 = 0; r0 < n; r0 += bs, ++blk) {
      int64_t m = (r0 + bs <= n) ? bs : n - r0;
      double vmax = 0.0;
      for (int64_t e = 0; e < m * m; ++e) vmax = fmax(vmax, fabs(P->blocks[off + e]));
      int ex = 0;
      if (vmax > 0.0) frexp(vmax, &ex);
      double sc = ldexp(1.0, -ex);
      P32.scale[blk] = (float)ldexp(1.0, ex);
      for (int64_t e = 0; e < m * m; ++e) {
        double v = P->blocks[off + e] * sc;
        P32.blocks[off + e] = prec[blk] == 0 ? (float)(_Float16)v : (float)v;
      }
      off += m * m;
    }
    free(prec);
  }
  double bnorm = or_norm2(n, b), ref = 0.0, tol = 0.0, rnorm = 0.0;
  int stop = OR_STOP_NONE;
  int64_t k_total = 0, steps = 0;
  for (;;) {
    residual(n, rowptr, col, val, b, x, r64);
    st->spmvs += 1;
    rnorm = or_norm2(n, r64);
    if (steps == 0) {
      ref = crit->rel_to_b ? bnorm : rnorm;
      if (ref == 0.0) ref = 1.0;
      tol = crit->reduction_factor * ref;
    }
    stop = check_stop(rnorm, tol, k_total, crit->max_iters);
    if (stop != OR_STOP_NONE || steps >= 200) {
      if (stop == OR_STOP_NONE) stop = OR_STOP_MAX_ITERS;
      break;
    }
    /* inner CG in float on A d = r / ||r|| */
    double inv = 1.0 / rnorm;
    for (int64_t i = 0; i < n; ++i) {
      r[i] = (float)(r64[i] * inv);
      d[i] = 0.0f;
    }
    precond32_apply(n, &P32, r, z);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    float rho = dotf(n, r, z);
    double rr0 = dotf(n, r, r);
    /* the last inner solve only needs the reduction that is still missing */
    double red = fmax(inner_reduction, 0.5 * tol / rnorm);
    double tol2 = red * red * rr0;
    int64_t it = 0;
    int broke = 0;
    while (it < inner_max) {
      for (int64_t i = 0; i < n; ++i) {
        float s = 0.0f;
        for (int64_t kk = rowptr[i]; kk < rowptr[i + 1]; ++kk) s = fmaf(val32[kk], p[col[kk]], s);
        q[i] = s;
      }
      float sigma = dotf(n, p, q);
      if (!isfinite(sigma) || sigma <= 0.0f) { broke = 1; break; }
      float alpha = (float)((double)rho / (double)sigma);
      for (int64_t i = 0; i < n; ++i) d[i] = fmaf(alpha, p[i], d[i]);
      for (int64_t i = 0; i < n; ++i) r[i] = fmaf(-alpha, q[i], r[i]);
      it += 1;
      precond32_apply(n, &P32, r, z);
      float rz = dotf(n, r, z);
      float rr = dotf(n, r, r);
      if (!isfinite(rz) || !isfinite(rr)) { broke = 1; break; }
      if ((double)rr <= tol2) break;
      float beta = (float)((double)rz / (double)rho);
      for (int64_t i = 0; i < n; ++i) p[i] = fmaf(beta, p[i], z[i]);
      rho = rz;
    }
    for (int64_t i = 0; i < n; ++i) x[i] = fma(rnorm, (double)d[i], x[i]);
    k_total += it;
    st->spmvs += it;
    steps += 1;
    if (it == 0 || (broke && it <= 1)) { stop = OR_STOP_BREAKDOWN; break; }
  }
  st->iters = k_total;
  st->stop_reason = stop;
  st->rel_res = rnorm / ref;
  st->rel_res_true = rnorm / ref;
  st->ref_norm = ref;
  if (outer) *outer = steps;
  free(val32); free(r); free(p); free(q); free(z); free(d); free(r64);
  free(P32.dinv); free(P32.blocks); free(P32.scale);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Single-precision CG and BiCGSTAB (the batched FP32 solves)                */
/* ------------------------------------------------------------------------ */

/* Float copies of A's values, b and x_0, and the scalar Jacobi inverse in
 * float (1 / (float) a_ii).  OR_ERR_SINGULAR when a diagonal is missing or 0. */
static int f32_setup(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     int32_t jacobi, const double* b, const double* x, float* val32, float* b32,
                     float* x32, float* dinv) {
  int64_t nnz = rowptr[n];
  for (int64_t k = 0; k < nnz; ++k) val32[k] = (float)val[k];
  for (int64_t i = 0; i < n; ++i) {
    b32[i] = (float)b[i];
    x32[i] = (float)x[i];
  }
  if (!jacobi) return OR_OK;
  for (int64_t i = 0; i < n; ++i) {
    float d = 0.0f;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i) d = val32[k];
    if (d == 0.0f) return OR_ERR_SINGULAR;
    dinv[i] = 1.0f / d;
  }
  return OR_OK;
}

/* y = A x in float: ordered row sums by fmaf. */
static void spmvf(int64_t n, const int32_t* rowptr, const int32_t* col, const float* val32,
                  const float* x, float* y) {
  for (int64_t i = 0; i < n; ++i) {
    float s = 0.0f;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s = fmaf(val32[k], x[col[k]], s);
    y[i] = s;
  }
}

static void jacf(int64_t n, int32_t jacobi, const float* dinv, const float* r, float* z) {
  for (int64_t i = 0; i < n; ++i) z[i] = jacobi ? dinv[i] * r[i] : r[i];
}

int or_cg_f32(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, int32_t jacobi,
              const double* b, double* x, const or_criteria* crit, or_status* st) {
  if (n < 0 || !crit || !st) return OR_ERR_ARG;
  memset(st, 0, sizeof(*st));
  size_t fz = sizeof(float) * (size_t)(n + 1);
  float *a32 = malloc(sizeof(float) * (size_t)(rowptr[n] + 1)), *b32 = malloc(fz), *x32 = malloc(fz),
        *dinv = malloc(fz), *r = malloc(fz), *z = malloc(fz), *p = malloc(fz), *q = malloc(fz);
  double* work = malloc(sizeof(double) * (size_t)(n + 1));
  int rc = f32_setup(n, rowptr, col, val, jacobi, b, x, a32, b32, x32, dinv);
  if (rc == OR_OK) {
    spmvf(n, rowptr, col, a32, x32, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b32[i] - q[i];
    st->spmvs = 1;
    double bnorm = sqrt((double)dotf(n, b32, b32));
    double rnorm = sqrt((double)dotf(n, r, r));
    double ref = crit->rel_to_b ? bnorm : rnorm;
    if (ref == 0.0) ref = 1.0;
    double tol = crit->reduction_factor * ref;
    jacf(n, jacobi, dinv, r, z);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    float rho = dotf(n, r, z);
    int64_t k = 0;
    int stop;
    while ((stop = check_stop(rnorm, tol, k, crit->max_iters)) == OR_STOP_NONE) {
      spmvf(n, rowptr, col, a32, p, q);
      st->spmvs += 1;
      float sigma = dotf(n, p, q);
      if (!isfinite(sigma)) { stop = OR_STOP_NAN; break; }
      if (sigma <= 0.0f) { stop = OR_STOP_BREAKDOWN; break; }
      float alpha = rho / sigma;
      for (int64_t i = 0; i < n; ++i) x32[i] = fmaf(alpha, p[i], x32[i]);
      for (int64_t i = 0; i < n; ++i) r[i] = fmaf(-alpha, q[i], r[i]);
      k += 1;
      rnorm = sqrt((double)dotf(n, r, r));
      jacf(n, jacobi, dinv, r, z);
      float rho_new = dotf(n, r, z);
      float beta = rho_new / rho;
      for (int64_t i = 0; i < n; ++i) p[i] = fmaf(beta, p[i], z[i]);
      rho = rho_new;
    }
    for (int64_t i = 0; i < n; ++i) x[i] = (double)x32[i];
    st->iters = k;
    st->stop_reason = stop;
    finish(n, rowptr, col, val, b, x, ref, rnorm, st, work);
  }
  free(a32); free(b32); free(x32); free(dinv); free(r); free(z); free(p); free(q); free(work);
  return rc;
}

int or_bicgstab_f32(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, int32_t jacobi,
                    const double* b, double* x, const or_criteria* crit, or_status* st) {
  if (n < 0 || !crit || !st) return OR_ERR_ARG;
  memset(st, 0, sizeof(*st));
  size_t fz = sizeof(float) * (size_t)(n + 1);
  float *a32 = malloc(sizeof(float) * (size_t)(rowptr[n] + 1)), *b32 = malloc(fz), *x32 = malloc(fz),
        *dinv = malloc(fz), *r = malloc(fz), *rh = malloc(fz), *p = malloc(fz), *v = malloc(fz),
        *ph = malloc(fz), *s = malloc(fz), *sh = malloc(fz), *t = malloc(fz);
  double* work = malloc(sizeof(double) * (size_t)(n + 1));
  int rc = f32_setup(n, rowptr, col, val, jacobi, b, x, a32, b32, x32, dinv);
  if (rc == OR_OK) {
    spmvf(n, rowptr, col, a32, x32, t);
    for (int64_t i = 0; i < n; ++i) r[i] = b32[i] - t[i];
    st->spmvs = 1;
    double bnorm = sqrt((double)dotf(n, b32, b32));
    double rnorm = sqrt((double)dotf(n, r, r));
    double ref = crit->rel_to_b ? bnorm : rnorm;
    if (ref == 0.0) ref = 1.0;
    double tol = crit->reduction_factor * ref;
    for (int64_t i = 0; i < n; ++i) {
      rh[i] = r[i];
      p[i] = 0.0f;
      v[i] = 0.0f;
    }
    float rho_prev = 1.0f, alpha = 1.0f, omega = 1.0f;
    int64_t k = 0;
    int stop, restarts = 0;
    /* Breakdown of the Lanczos part (rho = r^.r or r^.v exactly zero in
     * single precision, where r^ has become orthogonal to the Krylov
     * residuals to within float rounding): restart from the current iterate
     * with r^ = r, p = v = 0 and rho_prev = alpha = omega = 1 -- the remedy
     * the Templates book (Barrett et al. 1994) gives for this breakdown -- at
     * most OR_F32_RESTARTS times, then report the breakdown. */
#define OR_F32_RESTARTS 4
#define F32_RESTART_OR_STOP()                                       \
  if (restarts < OR_F32_RESTARTS) {                                 \
    restarts += 1;                                                  \
    for (int64_t i = 0; i < n; ++i) {                               \
      rh[i] = r[i];                                                 \
      p[i] = 0.0f;                                                  \
      v[i] = 0.0f;                                                  \
    }                                                               \
    rho_prev = 1.0f;                                                \
    alpha = 1.0f;                                                   \
    omega = 1.0f;                                                   \
    continue;                                                       \
  }                                                                 \
  stop = OR_STOP_BREAKDOWN;                                         \
  break
    while ((stop = check_stop(rnorm, tol, k, crit->max_iters)) == OR_STOP_NONE) {
      float rho = dotf(n, rh, r);
      if (!isfinite(rho)) { stop = OR_STOP_NAN; break; }
      if (rho == 0.0f) { F32_RESTART_OR_STOP(); }
      float beta = (rho / rho_prev) * (alpha / omega);
      for (int64_t i = 0; i < n; ++i) p[i] = fmaf(beta, fmaf(-omega, v[i], p[i]), r[i]);
      jacf(n, jacobi, dinv, p, ph);
      spmvf(n, rowptr, col, a32, ph, v);
      st->spmvs += 1;
      float rhv = dotf(n, rh, v);
      if (!isfinite(rhv)) { stop = OR_STOP_NAN; break; }
      if (rhv == 0.0f) { F32_RESTART_OR_STOP(); }
      alpha = rho / rhv;
      for (int64_t i = 0; i < n; ++i) s[i] = fmaf(-alpha, v[i], r[i]);
      double snorm = sqrt((double)dotf(n, s, s));
      if (isfinite(snorm) && snorm <= tol) {
        for (int64_t i = 0; i < n; ++i) x32[i] = fmaf(alpha, ph[i], x32[i]);
        for (int64_t i = 0; i < n; ++i) r[i] = s[i];
        k += 1;
        rnorm = snorm;
        stop = OR_STOP_CONVERGED;
        break;
      }
      jacf(n, jacobi, dinv, s, sh);
      spmvf(n, rowptr, col, a32, sh, t);
      st->spmvs += 1;
      float tt = dotf(n, t, t);
      float ts = dotf(n, t, s);
      if (!isfinite(tt) || !isfinite(ts)) { stop = OR_STOP_NAN; break; }
      if (tt == 0.0f) { stop = OR_STOP_BREAKDOWN; break; }
      omega = ts / tt;
      for (int64_t i = 0; i < n; ++i) x32[i] = fmaf(omega, sh[i], fmaf(alpha, ph[i], x32[i]));
      for (int64_t i = 0; i < n; ++i) r[i] = fmaf(-omega, t[i], s[i]);
      rho_prev = rho;
      k += 1;
      rnorm = sqrt((double)dotf(n, r, r));
      if (omega == 0.0f) {
        stop = check_stop(rnorm, tol, k, crit->max_iters);
        if (stop == OR_STOP_NONE) stop = OR_STOP_BREAKDOWN;
        break;
      }
    }
#undef F32_RESTART_OR_STOP
    for (int64_t i = 0; i < n; ++i) x[i] = (double)x32[i];
    st->iters = k;
    st->stop_reason = stop;
    finish(n, rowptr, col, val, b, x, ref, rnorm, st, work);
  }
  free(a32); free(b32); free(x32); free(dinv); free(r); free(rh); free(p); free(v); free(ph); free(s);
  free(sh); free(t); free(work);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* CGS, FCG and restarted GMRES (the rest of Section 3.1's Krylov family)    */
/* ------------------------------------------------------------------------ */

/* Preconditioned CGS (Sonneveld 1989, in the form of Barrett et al.,
 * "Templates", 1994), shadow residual r^ = r_0:
 *   rho = r^.r;  first step: u = r, p = u;  else beta = rho / rho_prev,
 *   u = r + beta q, p = u + beta (q + beta p)
 *   p^ = M^{-1} p;  v^ = A p^;  alpha = rho / (r^.v^);  q = u - alpha v^
 *   u^ = M^{-1} (u + q);  x = x + alpha u^;  q^ = A u^;  r = r - alpha q^
 * rho = 0 or r^.v^ = 0 are breakdowns. */
int or_cgs(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const or_precond* P,
           const double* b, double* x, const or_criteria* crit, or_status* st, double* res_hist) {
  if (n < 0 || !crit || !st) return OR_ERR_ARG;
  memset(st, 0, sizeof(*st));
  size_t sz = sizeof(double) * (size_t)(n + 1);
  double *r = malloc(sz), *rh = malloc(sz), *u = malloc(sz), *p = malloc(sz), *q = malloc(sz),
         *ph = malloc(sz), *vh = malloc(sz), *uh = malloc(sz), *t = malloc(sz);
  residual(n, rowptr, col, val, b, x, r);
  st->spmvs = 1;
  double bnorm = or_norm2(n, b), rnorm = or_norm2(n, r);
  double ref = crit->rel_to_b ? bnorm : rnorm;
  if (ref == 0.0) ref = 1.0;
  double tol = crit->reduction_factor * ref;
  for (int64_t i = 0; i < n; ++i) {
    rh[i] = r[i];
    q[i] = 0.0;
    p[i] = 0.0;
  }
  double rho_prev = 1.0;
  int64_t k = 0;
  int stop;
  if (res_hist) res_hist[0] = rnorm / ref;
  while ((stop = check_stop(rnorm, tol, k, crit->max_iters)) == OR_STOP_NONE) {
    double rho = or_dot(n, rh, r);
    if (!is_finite(rho)) { stop = OR_STOP_NAN; break; }
    if (rho == 0.0) { stop = OR_STOP_BREAKDOWN; break; }
    if (k == 0) {
      for (int64_t i = 0; i < n; ++i) {
        u[i] = r[i];
        p[i] = u[i];
      }
    } else {
      double beta = rho / rho_prev;
      for (int64_t i = 0; i < n; ++i) {
        u[i] = fma(beta, q[i], r[i]);
        p[i] = fma(beta, fma(beta, p[i], q[i]), u[i]);
      }
    }
    or_precond_apply(n, P, p, ph);
    or_csr_spmv(n, rowptr, col, val, ph, 1.0, 0.0, vh);
    st->spmvs += 1;
    double rv = or_dot(n, rh, vh);
    if (!is_finite(rv)) { stop = OR_STOP_NAN; break; }
    if (rv == 0.0) { stop = OR_STOP_BREAKDOWN; break; }
    double alpha = rho / rv;
    for (int64_t i = 0; i < n; ++i) {
      q[i] = fma(-alpha, vh[i], u[i]);
      t[i] = u[i] + q[i];
    }
    or_precond_apply(n, P, t, uh);
    for (int64_t i = 0; i < n; ++i) x[i] = fma(alpha, uh[i], x[i]);
    or_csr_spmv(n, rowptr, col, val, uh, 1.0, 0.0, t);
    st->spmvs += 1;
    for (int64_t i = 0; i < n; ++i) r[i] = fma(-alpha, t[i], r[i]);
    rho_prev = rho;
    k += 1;
    rnorm = or_norm2(n, r);
    if (res_hist) res_hist[k] = rnorm / ref;
  }
  st->iters = k;
  st->stop_reason = stop;
  finish(n, rowptr, col, val, b, x, ref, rnorm, st, t);
  free(r); free(rh); free(u); free(p); free(q); free(ph); free(vh); free(uh); free(t);
  return OR_OK;
}

/* Flexible CG (Notay 2000; the Polak-Ribiere form of beta):
 *   as CG, but beta = z_{k+1}.(r_{k+1} - r_k) / (r_k.z_k), with
 *   r_{k+1} - r_k = -alpha q.  For a fixed SPD preconditioner it equals CG in
 *   exact arithmetic; it tolerates a preconditioner that varies. */
int or_fcg(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const or_precond* P,
           const double* b, double* x, const or_criteria* crit, or_status* st, double* res_hist) {
  if (n < 0 || !crit || !st) return OR_ERR_ARG;
  memset(st, 0, sizeof(*st));
  size_t sz = sizeof(double) * (size_t)(n + 1);
  double *r = malloc(sz), *z = malloc(sz), *p = malloc(sz), *q = malloc(sz), *t = malloc(sz);
  residual(n, rowptr, col, val, b, x, r);
  st->spmvs = 1;
  double bnorm = or_norm2(n, b), rnorm = or_norm2(n, r);
  double ref = crit->rel_to_b ? bnorm : rnorm;
  if (ref == 0.0) ref = 1.0;
  double tol = crit->reduction_factor * ref;
  or_precond_apply(n, P, r, z);
  for (int64_t i = 0; i < n; ++i) p[i] = z[i];
  double rho = or_dot(n, r, z);
  int64_t k = 0;
  int stop;
  if (res_hist) res_hist[0] = rnorm / ref;
  while ((stop = check_stop(rnorm, tol, k, crit->max_iters)) == OR_STOP_NONE) {
    or_csr_spmv(n, rowptr, col, val, p, 1.0, 0.0, q);
    st->spmvs += 1;
    double sigma = or_dot(n, p, q);
    if (!is_finite(sigma)) { stop = OR_STOP_NAN; break; }
    if (sigma <= 0.0) { stop = OR_STOP_BREAKDOWN; break; }
    double alpha = rho / sigma;
    for (int64_t i = 0; i < n; ++i) x[i] = fma(alpha, p[i], x[i]);
    for (int64_t i = 0; i < n; ++i) r[i] = fma(-alpha, q[i], r[i]);
    k += 1;
    rnorm = or_norm2(n, r);
    if (res_hist) res_hist[k] = rnorm / ref;
    or_precond_apply(n, P, r, z);
    for (int64_t i = 0; i < n; ++i) t[i] = -alpha * q[i];
    double rho_t = or_dot(n, z, t);
    double rho_new = or_dot(n, r, z);
    double beta = rho_t / rho;
    for (int64_t i = 0; i < n; ++i) p[i] = fma(beta, p[i], z[i]);
    rho = rho_new;
  }
  st->iters = k;
  st->stop_reason = stop;
  finish(n, rowptr, col, val, b, x, ref, rnorm, st, q);
  free(r); free(z); free(p); free(q); free(t);
  return OR_OK;
}

/* Restarted GMRES(m) (Saad and Schultz 1986) with right preconditioning:
 * the Arnoldi process on A M^{-1} with modified Gram-Schmidt, Givens
 * rotations on the Hessenberg matrix, the residual estimate |g_{j+1}| as the
 * criterion's norm after every step, and at the end of a cycle (m steps or
 * the criterion met) x = x + M^{-1} V y with y from H y = g; the next cycle
 * starts from the true residual.  One Arnoldi step counts as one iteration.
 * A zero h_{j+1,j} (lucky breakdown) ends the cycle. */
int or_gmres(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const or_precond* P,
             const double* b, double* x, const or_criteria* crit, int32_t m, or_status* st, double* res_hist) {
  if (n < 0 || !crit || !st || m < 1) return OR_ERR_ARG;
  memset(st, 0, sizeof(*st));
  size_t sz = sizeof(double) * (size_t)(n + 1);
  double* V = malloc(sz * (size_t)(m + 1));
  double *w = malloc(sz), *z = malloc(sz), *r = malloc(sz);
  double* H = calloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* H[i * m + j] */
  double *cs = malloc(sizeof(double) * (size_t)m), *sn = malloc(sizeof(double) * (size_t)m);
  double *g = malloc(sizeof(double) * (size_t)(m + 1)), *y = malloc(sizeof(double) * (size_t)m);
  residual(n, rowptr, col, val, b, x, r);
  st->spmvs = 1;
  double bnorm = or_norm2(n, b), rnorm = or_norm2(n, r);
  double ref = crit->rel_to_b ? bnorm : rnorm;
  if (ref == 0.0) ref = 1.0;
  double tol = crit->reduction_factor * ref;
  int64_t k = 0;
  int stop = OR_STOP_NONE;
  if (res_hist) res_hist[0] = rnorm / ref;
  while ((stop = check_stop(rnorm, tol, k, crit->max_iters)) == OR_STOP_NONE) {
    /* one cycle */
    double beta = rnorm;
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int j = 0, steps = 0;
    int cycle_stop = 0;
    for (j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * (size_t)(n + 1);
      double* vn = V + (size_t)(j + 1) * (size_t)(n + 1);
      or_precond_apply(n, P, vj, z);
      or_csr_spmv(n, rowptr, col, val, z, 1.0, 0.0, w);
      st->spmvs += 1;
      for (int i = 0; i <= j; ++i) {
        double* vi = V + (size_t)i * (size_t)(n + 1);
        double h = or_dot(n, w, vi);
        H[i * m + j] = h;
        for (int64_t l = 0; l < n; ++l) w[l] = fma(-h, vi[l], w[l]);
      }
      double hn = or_norm2(n, w);
      H[(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (int64_t l = 0; l < n; ++l) vn[l] = w[l] / hn;
      /* previous rotations on column j, then a new one for (j, j+1) */
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double d = hypot(a, c);
      cs[j] = d != 0.0 ? a / d : 1.0;
      sn[j] = d != 0.0 ? c / d : 0.0;
      H[j * m + j] = d;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k += 1;
      steps = j + 1;
      rnorm = fabs(g[j + 1]);
      if (res_hist) res_hist[k] = rnorm / ref;
      if (check_stop(rnorm, tol, k, crit->max_iters) != OR_STOP_NONE || hn == 0.0) {
        cycle_stop = 1;
        break;
      }
    }
    (void)cycle_stop;
    /* y = H^{-1} g (upper triangular, steps x steps), x += M^{-1} V y */
    for (int i = steps - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < steps; ++l) s = fma(-H[i * m + l], y[l], s);
      y[i] = s / H[i * m + i];
    }
    for (int64_t l = 0; l < n; ++l) {
      double s = 0.0;
      for (int i = 0; i < steps; ++i) s = fma(V[(size_t)i * (size_t)(n + 1) + l], y[i], s);
      w[l] = s;
    }
    or_precond_apply(n, P, w, z);
    for (int64_t l = 0; l < n; ++l) x[l] += z[l];
    residual(n, rowptr, col, val, b, x, r);
    st->spmvs += 1;
    rnorm = or_norm2(n, r);
    if (!is_finite(rnorm)) { stop = OR_STOP_NAN; break; }
  }
  st->iters = k;
  st->stop_reason = stop;
  finish(n, rowptr, col, val, b, x, ref, rnorm, st, w);
  free(V); free(w); free(z); free(r); free(H); free(cs); free(sn); free(g); free(y);
  return OR_OK;
}
