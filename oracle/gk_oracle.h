/*
 * gk_oracle.h -- plain, slow CPU oracle for the sparse
 * linear-operator hot path of "Ginkgo: A Modern Linear Operator Algebra
 * Framework for High Performance Computing" (arXiv:2006.16852).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only the tests, the smoke check and the benchmark's
 * CPU baseline do.  It shares no code, header, table or helper with the CUDA
 * path.
 *
 * Everything is sequential except the row loops of the two SpMVs, which
 * OpenMP may split over threads (static chunks): each row's sum is still
 * formed in increasing k by one thread, so no result depends on the thread
 * count.
 *
 * Conventions: FP64 values, int32 column indices and row pointers, int64
 * sizes.  Every floating-point step is written in the order the definition
 * or algorithm states; the library is compiled with -ffp-contract=off so
 * that the only fused multiply-adds are the explicit fma() calls.
 *
 * Parity status: every function below is pinned by the CPU tests against
 * brute force, closed forms or invariants (tests/test_oracle_*.py).
 */
#ifndef GK_ORACLE_H
#define GK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes shared by the oracle's own functions */
#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_SINGULAR 2

/* stop reasons (criteria of Section 2.5) */
#define OR_STOP_NONE 0
#define OR_STOP_CONVERGED 1
#define OR_STOP_MAX_ITERS 2
#define OR_STOP_BREAKDOWN 3
#define OR_STOP_NAN 4

/* preconditioner kinds (Section 3.2) */
#define OR_PREC_NONE 0
#define OR_PREC_SCALAR_JACOBI 1
#define OR_PREC_BLOCK_JACOBI 2

typedef struct {
  int64_t max_iters;        /* Iteration criterion (Listing 8): stop once k >= max_iters        */
  double reduction_factor;  /* ResidualNormReduction: stop once ||r_k|| <= factor * ref        */
  int32_t rel_to_b;         /* ref = ||b|| if nonzero, else ||r_0||                          */
} or_criteria;

typedef struct {
  int64_t iters;         /* iterations performed                                 */
  int64_t spmvs;         /* matrix applications, including the initial residual  */
  double rel_res;        /* recurred ||r|| / ref at exit                           */
  double rel_res_true;   /* ||b - A x|| / ref recomputed at exit                  */
  double ref_norm;       /* ref used by the criterion                            */
  int32_t stop_reason;   /* OR_STOP_*                                            */
  int32_t pad_;
} or_status;

typedef struct {
  int32_t kind;            /* OR_PREC_*                                            */
  int32_t block_size;      /* block size for OR_PREC_BLOCK_JACOBI                  */
  const double* dinv;      /* scalar: n inverse diagonal entries                   */
  const double* blocks;    /* block: inverse blocks, row-major, concatenated       */
} or_precond;

/* x = alpha*A*b + beta*x (Section 4.2, simple and advanced apply). */
void or_csr_spmv(int64_t n_rows, const int32_t* rowptr, const int32_t* col, const double* val,
                 const double* x, double alpha, double beta, double* y);

/* Threads the SpMV row loops use (OpenMP, static chunks; results are the
 * same for any count).  n <= 0: all the host's cores.  Returns the count in
 * effect, 1 without OpenMP. */
int or_set_threads(int n);

/* Accurate row sums by Dot2 (Ogita, Rump, Oishi 2005) and the bound (|A||x|)_i. */
void or_csr_spmv_dot2(int64_t n_rows, const int32_t* rowptr, const int32_t* col, const double* val,
                      const double* x, double* y_acc, double* abs_ax);

/* Plain dot product and 2-norm: sum in increasing index order. */
double or_dot(int64_t n, const double* x, const double* y);
double or_norm2(int64_t n, const double* x);

/* Scalar Jacobi: dinv_i = 1 / a_ii.  OR_ERR_SINGULAR if a diagonal is missing or zero. */
int or_jacobi_scalar(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     double* dinv);

/* Number of doubles the block-Jacobi inverse blocks occupy for (n, bs). */
int64_t or_block_jacobi_size(int64_t n, int32_t bs);

/* Block-Jacobi generate: contiguous blocks of bs rows (last one shorter), each
 * diagonal block inverted by Gauss-Jordan elimination with partial pivoting.
 * Blocks are written row-major and concatenated.  On a zero pivot returns
 * OR_ERR_SINGULAR and stores the failing block index in *bad_block. */
int or_block_jacobi_generate(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                             int32_t bs, double* blocks, int64_t* bad_block);

/* z = M^{-1} r for the given preconditioner (scalar, block, or copy). */
void or_precond_apply(int64_t n, const or_precond* P, const double* r, double* z);

/* Width K of the ELL part of the hybrid format: the smallest K minimising
 * K*n*(vt+it) + nnz_coo(K)*(vt+2*it), nnz_coo(K) = sum_i max(0, len_i - K). */
int64_t or_hyb_width(int64_t n_rows, const int32_t* rowptr, int64_t vt, int64_t it);

/* Preconditioned conjugate gradients (Section 3.1, Listing 1). x holds x_0 on
 * entry and the solution on exit.  res_hist (nullable, max_iters+1 entries)
 * receives the recurred relative residual of every iterate. */
int or_cg(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
          const or_precond* P, const double* b, double* x, const or_criteria* crit,
          or_status* st, double* res_hist);

/* Preconditioned BiCGSTAB (Section 3.1, Listing 3). */
int or_bicgstab(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                const or_precond* P, const double* b, double* x, const or_criteria* crit,
                or_status* st, double* res_hist);

/* Adaptive-precision block Jacobi (Section 3.2): for every inverse block,
 * kappa_1 = ||D||_1 ||D^{-1}||_1 (column sums in increasing row order, the
 * maximum over columns) and the storage precision: 0 = FP16 when
 * kappa_1 * 2^-11 <= 1e-2, else 1 = FP32.  kappa may be NULL. */
void or_block_jacobi_precision(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                               int32_t bs, const double* blocks, uint8_t* prec, double* kappa);

/* Iterative refinement with a lower-precision CG inner solver (Sections
 * 2.2.3 and 3.1): outer r = b - A x, ||r|| and the criteria in FP64; inner CG
 * on A d = r / ||r|| with float matrix values, float vectors and float
 * accumulation, stopped when ||r_inner|| <= red * ||r_inner,0|| with
 * red = max(inner_reduction, tol / (2 ||r||)) -- the reduction still missing --
 * or after inner_max iterations; then x = x + ||r|| d.  The inner
 * preconditioner is the float copy of P: scalar Jacobi, or block Jacobi
 * with each block stored in FP16 or float by or_block_jacobi_precision and
 * scaled by the power of two that puts its largest magnitude in [0.5, 1).
 * st->iters counts inner iterations, *outer the refinement steps. */
int or_ir_cg(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
             const or_precond* P, const double* b, double* x, const or_criteria* crit,
             double inner_reduction, int64_t inner_max, or_status* st, int64_t* outer);

/* Preconditioned CGS (Section 3.1; Sonneveld 1989, Templates form). */
int or_cgs(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const or_precond* P,
           const double* b, double* x, const or_criteria* crit, or_status* st, double* res_hist);

/* Flexible CG (Section 3.1; Notay 2000): beta = z_{k+1}.(r_{k+1} - r_k) / rho_k. */
int or_fcg(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const or_precond* P,
           const double* b, double* x, const or_criteria* crit, or_status* st, double* res_hist);

/* Restarted GMRES(m) with right preconditioning (Section 3.1; Saad and
 * Schultz 1986): modified Gram-Schmidt Arnoldi, Givens rotations, the
 * rotated residual |g_{j+1}| as the criterion's norm after every Arnoldi step
 * (one iteration each); every cycle ends with x += M^{-1} V y and restarts
 * from the true residual, which the criterion is checked on again. */
int or_gmres(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const or_precond* P,
             const double* b, double* x, const or_criteria* crit, int32_t m, or_status* st, double* res_hist);

/* CG and BiCGSTAB in single precision (the batched FP32 solves): the steps of
 * or_cg and or_bicgstab with float matrix values, float b, x, vectors and
 * float sums (in increasing index order), norms sqrt((double) sum); scalar
 * Jacobi (1 / (float) a_ii) if jacobi != 0, else none.  x is FP64 in memory
 * (rounded to float on entry); rel_res_true is computed in FP64 on exit.
 * OR_ERR_SINGULAR if jacobi and a diagonal entry is missing or zero. */
int or_cg_f32(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, int32_t jacobi,
              const double* b, double* x, const or_criteria* crit, or_status* st);
/* or_bicgstab_f32 restarts (r^ = r, p = v = 0, rho_prev = alpha = omega = 1;
 * the iteration count continues) when rho or r^.v is exactly zero before
 * convergence, at most 4 times; then it reports OR_STOP_BREAKDOWN. */
int or_bicgstab_f32(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, int32_t jacobi,
                    const double* b, double* x, const or_criteria* crit, or_status* st);

#ifdef __cplusplus
}
#endif
#endif
