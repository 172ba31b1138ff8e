/*
 * gk.h -- C ABI of the GB300 sparse linear-operator library.
 *
 * The calls follow the linear-operator statement of arXiv:2006.16852
 * (Ginkgo): every object is an operator L with apply(b, x): x = L(b)
 * (Section 2.2.2); solvers S_A and preconditioners P_A are produced from the
 * system operator L_A by generate() (Section 2.2.3); the simple apply
 * x = A b and the advanced apply x = alpha A b + beta x are both provided
 * (Section 4.2); iterations stop on combined criteria (Section 2.5).
 *
 * Conventions shared by every call
 *  - Return value: GK_OK (0) or a GK_ERR_* code; the thread-local message of
 *    the last failure is returned by gk_last_error().  No call throws.
 *  - Values are FP64 (gk_dtype GK_F64), indices int32, sizes int64.
 *  - Vector arguments are plain pointers to n contiguous doubles.  They may
 *    be device memory (cudaMalloc, torch CUDA tensors, managed memory) or
 *    host memory (pinned or pageable).  Host vectors are staged through a
 *    library-owned device buffer; a call given a host output returns only
 *    after the result is back in host memory.
 *  - Ownership mirrors the paper's lend/share/give (Section 2.4): vectors
 *    are lent for the duration of the call; gk_matrix_create_csr copies the
 *    caller's CSR arrays into library-owned storage; solvers and
 *    preconditioners share ownership of the matrix (and preconditioner) they
 *    were generated from, so the caller may destroy its handles in any order.
 *  - stream is a cudaStream_t (NULL = the legacy default stream).  All device
 *    work is enqueued on it.  gk_apply/gk_apply_adv/gk_precond_apply with
 *    device vectors are asynchronous; gk_solve returns after the solve has
 *    finished and its status has been read back.
 *  - Calls on one handle must not overlap in time on different streams: each
 *    handle owns its reduction scratch.
 *  - The device current at creation time owns a handle; calls switch to it.
 */
#ifndef GK_H
#define GK_H

#include <stdint.h>

#if defined(__GNUC__)
#define GK_API __attribute__((visibility("default")))
#else
#define GK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define GK_OK 0
#define GK_ERR_ARG 1         /* null handle/pointer, negative size, bad enum        */
#define GK_ERR_DIM 2         /* operator and vector sizes do not conform (Sec. 4.2) */
#define GK_ERR_DTYPE 3       /* value type not supported                            */
#define GK_ERR_NOT_DEVICE 4  /* pointer from another device                         */
#define GK_ERR_CSR 5         /* rowptr not monotone / columns unsorted, repeated or */
                             /* out of range                                        */
#define GK_ERR_FORMAT 6      /* format refused (ELL padding over 8x nnz)            */
#define GK_ERR_SINGULAR 7    /* zero/missing diagonal or singular diagonal block    */
#define GK_ERR_UNSUPPORTED 8 /* combination not built                               */
#define GK_ERR_CUDA 9        /* CUDA runtime error (message in gk_last_error)       */
#define GK_ERR_ALLOC 10      /* device allocation failed                            */
#define GK_ERR_TIMEOUT 11    /* a device-side wait exceeded its iteration limit     */

/* ---- enums -------------------------------------------------------------- */
#define GK_F64 0
#define GK_F32 1

/* Storage formats of the system matrix. */
#define GK_CSR 0        /* CSR, rows binned by length: rows of up to 256 entries sorted
                           by length into slices of 32 (a copy stored column-major,
                           one thread per row), longer rows cut into pieces of up to
                           512 consecutive entries, one warp per piece                  */
#define GK_CSR_MERGE 1  /* CSR, merge-path split of rows+nonzeros into equal tiles      */
#define GK_ELL 2        /* ELLPACK, column-major, padded to the longest row             */
#define GK_HYB 3        /* hybrid: ELL part of width K plus the overflow of longer rows
                           in COO form (row, column, value; sorted by row, then
                           column); K minimises K*n_rows*12 + overflow*16 bytes,
                           the smallest such K on ties                                   */
#define GK_AUTO 4       /* GK_CSR when at least 75 % of its slots (length-sorted slices,
                           warp and block rows) hold stored entries, else GK_CSR_MERGE */

#define GK_CG 0
#define GK_BICGSTAB 1
#define GK_IR_CG 2       /* FP64 iterative refinement around an FP32 CG inner solver */
#define GK_FCG 3         /* flexible CG (Polak-Ribiere beta)                          */
#define GK_CGS 4         /* conjugate gradient squared                                */
#define GK_GMRES 5       /* restarted GMRES, right preconditioning                    */

/* Stop reasons (the stopping_status of Section 2.5). */
#define GK_STOP_NONE 0
#define GK_STOP_CONVERGED 1  /* ||r_k|| <= reduction_factor * ref                       */
#define GK_STOP_MAX_ITERS 2  /* k >= max_iters (Iteration criterion)                    */
#define GK_STOP_BREAKDOWN 3  /* p.Ap <= 0 (CG, FCG); rho, r^.v, t.t or omega zero         */
                             /* (BiCGSTAB); r^.r or r^.v^ zero (CGS)                     */
#define GK_STOP_NAN 4        /* a residual norm or a reduction became NaN/Inf           */
#define GK_STOP_TIME 5       /* time_limit_s exceeded (Time criterion)                  */

typedef struct gk_matrix_s* gk_matrix;
typedef struct gk_precond_s* gk_precond;
typedef struct gk_solver_s* gk_solver;

/* Combined stopping criteria (Section 2.5, Listing 1): the first one met
 * stops the iteration.  ResidualNormReduction: ||r_k||_2 <= reduction_factor
 * * ref with ref = ||b||_2 if rel_to_b != 0, else ||r_0||_2.  Iteration:
 * k >= max_iters.  Time: wall time > time_limit_s (<= 0 disables it).
 * check_every <= 0 runs the whole solve as one CUDA graph whose loop is
 * controlled on the device (the criteria, Time included, are evaluated by
 * the GPU after every iteration); check_every > 0 instead launches the
 * iterations from the host and reads the stop flag back after every
 * check_every iterations.  check_every == 0 (the default) additionally lets
 * GK_CG and GK_BICGSTAB without a preconditioner or with scalar Jacobi and
 * without a Time criterion run as ONE launch: a 16-CTA thread-block cluster
 * (the vectors the SpMVs read in distributed shared memory, the phases
 * separated by cluster barriers) up to 32,768 rows for GK_CG and 16,384 rows
 * for GK_BICGSTAB; and, for GK_CG from 32,769 to 262,144 rows when no row
 * has more than 64 entries, a cooperative grid of one CTA per SM (grid-wide
 * barriers in global memory).  check_every < 0 always takes the graph. */
typedef struct {
  int64_t max_iters;        /* GK_IR_CG: limit on the total of inner iterations      */
  double reduction_factor;
  int32_t rel_to_b;
  int32_t check_every;
  double time_limit_s;
  /* GK_IR_CG only: each inner solve stops once its residual is reduced by
   * max(inner_reduction, tol / (2 ||r||)) (inner_reduction <= 0: 1e-5) or
   * after inner_max_iters iterations (<= 0: max_iters). */
  double inner_reduction;
  int32_t inner_max_iters;
  /* GK_GMRES only: the restart length m, Arnoldi vectors kept per cycle
   * (<= 0: 30; at most 128). */
  int32_t krylov_dim;
} gk_criteria;

/* Convergence record of one solve (the Convergence logger of Section 2.6). */
typedef struct {
  int64_t iters;        /* iterations performed (a BiCGSTAB half step counts as one) */
  int64_t spmvs;        /* matrix applications including the initial residual and    */
                        /* the final true-residual check                             */
  double rel_res;       /* recurred ||r_k|| / ref at exit                             */
  double rel_res_true;  /* ||b - A x|| / ref recomputed at exit                       */
  double ref_norm;      /* ref used by the residual criterion                         */
  int32_t stop_reason;  /* GK_STOP_*                                                  */
  int32_t device_error; /* nonzero if a device-side wait timed out                    */
  int64_t outer_iters;  /* GK_IR_CG: refinement steps (FP64 residuals); else 0        */
  int32_t form;         /* how the iteration ran: GK_FORM_*                           */
  int32_t idle_iters;   /* iterations whose kernels were launched after the stop and  */
                        /* did nothing: a graph's loop body runs whole passes of CG   */
                        /* iterations (GK_IR_CG: of inner iterations), a host loop    */
                        /* whole groups of check_every                                */
} gk_status;

#define GK_FORM_GRAPH 0    /* one CUDA graph, loop controlled on the device            */
#define GK_FORM_HOST 1     /* iterations launched from the host (check_every > 0)      */
#define GK_FORM_CLUSTER 2  /* one launch of a 16-CTA thread-block cluster (small CG  */
                           /* and BiCGSTAB)                                           */
#define GK_FORM_GRID 3     /* one cooperative launch, grid-wide barriers (mid-size CG) */

/* What a solver was built into. */
typedef struct {
  int32_t kind;             /* GK_CG, GK_BICGSTAB, GK_IR_CG, GK_FCG, GK_CGS,      */
                            /* GK_GMRES                                            */
  int32_t inner_format;     /* GK_IR_CG: storage of the FP32 operator copy (GK_ELL */
                            /* for ELL/HYB matrices, else GK_CSR)                  */
  int64_t n;
  int64_t inner_fp16_blocks; /* GK_IR_CG + block Jacobi: blocks stored in FP16   */
  int64_t inner_fp32_blocks; /* ... and in FP32                                  */
  int64_t device_bytes;
} gk_solver_info;

typedef struct {
  int64_t n_rows, n_cols, nnz;
  int32_t format;          /* the format actually built (GK_AUTO resolved)     */
  int32_t dtype;
  int64_t ell_width;       /* K for ELL/HYB, else 0                            */
  int64_t tail_rows;       /* HYB: rows with more than K entries               */
  int64_t tail_nnz;        /* HYB: entries stored outside the ELL part          */
  int64_t short_items;     /* GK_CSR: warp items of up to 32 short rows         */
  int64_t long_rows;       /* GK_CSR: rows of more than 256 entries (in pieces) */
  int64_t tiles;           /* GK_CSR_MERGE: merge-path tiles                    */
  int64_t device_bytes;    /* bytes of library-owned device storage             */
  int64_t spmv_bytes;      /* algorithmic bytes of one simple apply: the stored */
                           /* operator (CSR: nnz*12 + (n_rows+1)*4; ELL:        */
                           /* nnz*12; HYB: ELL entries*12 + COO entries*16),    */
                           /* x read once (n_cols*8), y written (n_rows*8)      */
  int64_t split_rows;      /* GK_CSR: rows of more than 512 entries, whose      */
                           /* pieces a second kernel adds (2 launches / apply)  */
} gk_matrix_info;

/* ---- errors ------------------------------------------------------------- */
/* Message of the last failing call on this thread ("" if none).  The string
 * is owned by the library and valid until the next call on this thread. */
GK_API const char* gk_last_error(void);
GK_API int32_t gk_version(void);

/* ---- matrices (the CSR LinOp of Section 2.2.4) --------------------------- */
/* Builds a library-owned copy of the n_rows x n_cols CSR matrix
 * (rowptr[n_rows+1], col[nnz], val[nnz]; any of them host or device memory)
 * in the requested format.  Columns must be sorted and unique within each
 * row and in [0, n_cols); rowptr[0] = 0, nondecreasing, rowptr[n_rows] = nnz.
 * Violations return GK_ERR_CSR.  GK_ELL is refused (GK_ERR_FORMAT) when its
 * padded size exceeds 8 * nnz + n_rows slots.  On success *out owns the copy. */
GK_API int gk_matrix_create_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* rowptr,
                         const int32_t* col, const void* val, int32_t dtype, int32_t format,
                         void* stream, gk_matrix* out);
GK_API int gk_matrix_get_info(gk_matrix A, gk_matrix_info* info);
GK_API int gk_matrix_destroy(gk_matrix A);

/* Simple apply, Section 4.2: x = A b (b has n_cols entries, x n_rows).
 * Row sums accumulate with one fused multiply-add per stored entry. */
GK_API int gk_apply(gk_matrix A, const void* b, void* x, void* stream);

/* Advanced apply, Section 4.2: x = alpha A b + beta x.  beta == 0 does not
 * read x (BLAS convention), so gk_apply == gk_apply_adv(1, A, b, 0, x). */
GK_API int gk_apply_adv(double alpha, gk_matrix A, const void* b, double beta, void* x, void* stream);

/* x = A b and result[0] = u . x in one pass: the SpMV with the fused dot
 * product every Krylov iteration uses (Section 7.4 on fusing the reductions
 * of Krylov solvers into the kernels that produce their operands).  A square;
 * b, x, u, result: device memory; the sum's order is fixed (per-row products
 * accumulated per thread, then the block and grid reductions of gk_dot), so
 * the result is reproducible run to run.  Calls on one matrix must be ordered
 * (they share the matrix's reduction scratch). */
GK_API int gk_apply_dot(gk_matrix A, const double* b, double* x, const double* u, double* result, void* stream);

/* ---- preconditioners (Section 3.2) -------------------------------------- */
/* Jacobi preconditioner P_A = M^{-1} generated from A (square).
 * block_size 1: scalar Jacobi, M = diag(A).  block_size 2..32: block Jacobi
 * on contiguous blocks of block_size rows (the last one shorter), each
 * diagonal block inverted by Gauss-Jordan elimination with partial pivoting
 * (Section 7.5).  A zero/missing diagonal or a singular block returns
 * GK_ERR_SINGULAR.  The inverse diagonal or blocks are allocated on `stream`
 * from the device's default stream-ordered memory pool (the library lets the
 * pool keep up to 8 GB of freed memory for reuse, so repeated generations do
 * not map memory again); the call returns after the generation has
 * finished (it reads back the error check). */
GK_API int gk_precond_generate(gk_matrix A, int32_t block_size, void* stream, gk_precond* out);

/* z = M^{-1} r (the preconditioner as a LinOp). */
GK_API int gk_precond_apply(gk_precond P, const void* r, void* z, void* stream);

/* Copies the inverse diagonal blocks, row-major and concatenated (block k
 * holds m_k*m_k doubles, m_k = block_size except for the last block), into
 * host memory out[n_out].  For block_size 1 this is 1/a_ii.  n_out must be
 * at least the total size. */
GK_API int gk_precond_get_blocks(gk_precond P, double* out, int64_t n_out, void* stream);
GK_API int gk_precond_destroy(gk_precond P);

/* ---- solvers (Section 3.1) ---------------------------------------------- */
/* S_A = generate(A): a Krylov solver operator bound to A -- CG, BiCGSTAB,
 * FCG, CGS or restarted GMRES (Section 3.1) -- optionally preconditioned by
 * P (NULL for none), stopping on *crit.
 * GK_FCG: CG with beta = z_{k+1}.(r_{k+1} - r_k) / (r_k.z_k) (Notay's
 * flexible CG; equal to CG for a fixed preconditioner in exact arithmetic).
 * GK_CGS: Sonneveld's CGS in the Templates form with r^ = r_0 (two SpMVs per
 * iteration; breakdown when r^.r or r^.v^ vanishes).
 * GK_GMRES: GMRES(m), m = crit->krylov_dim, right-preconditioned (A M^{-1}),
 * Arnoldi with classical Gram-Schmidt applied twice, Givens rotations; an
 * Arnoldi step is one iteration and its rotated residual |g_{j+1}| is the
 * norm the criteria see; every cycle ends with x += M^{-1} V y and a fresh
 * true residual.
 * GK_IR_CG is the iterative refinement of Sections 2.2.3 and 3.1 with a
 * CG inner solver run in lower precision: the outer loop computes r = b - A x,
 * its norm and the update x += d in FP64; the inner solve of A d = r runs on
 * an FP32 copy of A with FP32 vectors and FP32 accumulation, preconditioned
 * by an FP32 copy of P (scalar Jacobi) or by P's inverse blocks stored per
 * block in FP16 or FP32 chosen by the block's condition number kappa_1
 * (Section 3.2's adaptive-precision block Jacobi: FP16 when
 * kappa_1 * 2^-11 <= 1e-2, each block scaled by a power of two). */
GK_API int gk_solver_generate(gk_matrix A, gk_precond P, int32_t kind, const gk_criteria* crit,
                       gk_solver* out);

/* x = S_A(b): x holds the initial guess on entry and the solution on exit
 * (Section 2.1).  *st (nullable) receives the convergence record.
 * Non-convergence is not an error: GK_OK is returned and st->stop_reason
 * says which criterion ended the iteration. */
GK_API int gk_solve(gk_solver S, const void* b, void* x, gk_status* st, void* stream);
GK_API int gk_solver_destroy(gk_solver S);
GK_API int gk_solver_get_info(gk_solver S, gk_solver_info* info);

/* ---- batched small systems ------------------------------------------------ */
/* Many independent square systems (the per-right-hand-side / per-system
 * stopping status of Section 2.5 taken to independent matrices), stored as
 * one block-diagonal CSR matrix: system s owns rows and columns
 * [sys_ptr[s], sys_ptr[s+1]) and each of its rows may reference only those
 * columns, in increasing order without repeats (else GK_ERR_CSR).  Systems
 * of 1 to 4096 rows are supported (GK_ERR_UNSUPPORTED beyond).  dtype GK_F64
 * solves in FP64; GK_F32 stores the values in FP32 and solves in FP32 (b and
 * x stay FP64 in memory).
 * gk_batch_create: sys_ptr is a host array of n_sys+1 offsets starting at 0;
 * rowptr (n_rows+1), col and val (nnz) may be host or device memory and are
 * copied.  The handle owns its device memory; calls on one handle must be
 * ordered (they share a schedule counter and a status array). */
typedef struct gk_batch_s* gk_batch;

typedef struct {
  int32_t iters;        /* iterations (GK_IR_CG: inner iterations, all steps)  */
  int32_t stop_reason;  /* GK_STOP_* per system                              */
  double rel_res;       /* recurred ||r|| / ||b|| (or / ||r_0||) at exit;
                           GK_IR_CG: the last FP64 residual                  */
  int32_t outer_iters;  /* GK_IR_CG: refinement steps; else 0                */
  int32_t reserved_;
} gk_batch_status;

GK_API int gk_batch_create(int64_t n_sys, const int64_t* sys_ptr, int64_t nnz, const int32_t* rowptr,
                           const int32_t* col, const double* val, int32_t dtype, void* stream, gk_batch* out);

/* Size classes: class c holds the systems of 16*2^c + 1 to 32*2^c rows
 * (class 0: 1 to 32 rows, ..., class 7: 2049 to 4096 rows). */
#define GK_BATCH_CLASSES 8

/* Solves every system with CG or BiCGSTAB (kind), scalar Jacobi if
 * jacobi != 0, in one CUDA graph launch.  kind GK_IR_CG (FP64 batches
 * only) is the iterative refinement of gk_solver_generate per system: FP64
 * residual, criteria and update on the FP64 values, FP32 CG corrections on
 * an FP32 copy with the FP64 inverse diagonal rounded to FP32, inner stop
 * by crit->inner_reduction / inner_max_iters as for gk_solve, at most 200
 * refinement steps; it reaches FP64 residuals with FP32 inner work.  In
 * every kind: each size class is one persistent
 * kernel (the classes run side by side as independent graph branches); a
 * thread block holds one system at a time with its vectors in shared memory
 * and takes the class's systems in decreasing size.  Each system's result
 * depends only on the system, b, x_0 and its class's block size -- not on its
 * neighbours, the schedule or the run.  b and x are device arrays of n_rows
 * doubles laid out like the rows; x holds the initial guesses and receives
 * the solutions.  st (host, nullable) receives n_sys records (the call then
 * waits for the stream).  crit: max_iters, reduction_factor and rel_to_b
 * apply to every system; the other fields are ignored.  When a class's
 * largest system does not fit in one block's shared memory (BiCGSTAB with
 * Jacobi in FP64 above about 3500 rows) GK_ERR_UNSUPPORTED is returned. */
GK_API int gk_batch_solve(gk_batch B, int32_t kind, int32_t jacobi, const gk_criteria* crit, const void* b,
                          void* x, gk_batch_status* st, void* stream);

/* The autotuner: for (kind, jacobi), times every non-empty class alone at
 * block sizes 32 (one warp per system), 64, 128 and 256, solving for b from
 * x = 0 into a workspace of the handle, and keeps the fastest size per class
 * for later gk_batch_solve calls.  threads (nullable, GK_BATCH_CLASSES
 * entries) receives the chosen sizes (0 for empty classes); times_ms
 * (nullable, GK_BATCH_CLASSES * 4 entries, class-major) the measured times,
 * -1 where a size does not fit or the class is empty.  Waits for the stream. */
GK_API int gk_batch_autotune(gk_batch B, int32_t kind, int32_t jacobi, const gk_criteria* crit, const void* b,
                             int32_t* threads, double* times_ms, void* stream);

/* Sets the block size per class for (kind, jacobi): GK_BATCH_CLASSES entries
 * of 32, 64, 128, 256, or 0 for the built-in default (32 up to 64 rows, 64
 * up to 512, else 128).  GK_ERR_ARG for any other value. */
GK_API int gk_batch_set_threads(gk_batch B, int32_t kind, int32_t jacobi, const int32_t* threads);

/* Per class (GK_BATCH_CLASSES entries each, all nullable): systems in the
 * class, rows of its largest system, and the block size (kind, jacobi) will
 * run it with (0 for empty classes). */
GK_API int gk_batch_get_info(gk_batch B, int32_t kind, int32_t jacobi, int32_t* counts, int32_t* nmax,
                             int32_t* threads);
GK_API int gk_batch_destroy(gk_batch B);

/* ---- learned warm start -------------------------------------------------- */
/* Not in the paper: a convolutional network that predicts the initial guess
 * x0 of a variable-coefficient diffusion solve on an H x W grid (natural
 * row-major ordering) from the log-coefficient field g (one value per grid
 * point) and the right-hand side b; zero-start CG remains the reference the
 * prediction is judged against.  Six 3x3 convolutions with dilations
 * dilations[0..5] and zero padding, channels 2 -> 32 -> 32 -> 32 -> 32 -> 32
 * -> 1, ReLU between layers.  Input (B, 2, H, W) float = [g, b / rms(b)];
 * output (B, 1, H, W) float = x / (rms(b) * out_scale).  Parameters: one
 * float vector, per layer the weights (out, in, 3, 3) then the biases.
 * Training runs in FP32 (deterministic reductions, Adam with beta1 0.9,
 * beta2 0.999, eps 1e-8); inference in BF16 (weights, biases, activations)
 * with FP32 products and sums.  All array arguments are device memory unless
 * said otherwise; calls on one handle must be ordered (shared scratch). */
typedef struct gk_wsnet_s* gk_wsnet;

/* batch_max: largest batch of the training / forward calls; dilations: 6
 * values in 1..64.  GK_ERR_UNSUPPORTED when a gradient kernel's shared
 * memory (about 4 * (32 W + 96 (W + 2 d)) bytes) exceeds the device's. */
GK_API int gk_wsnet_create(int32_t H, int32_t W, int32_t batch_max, const int32_t* dilations, gk_wsnet* out);
GK_API int gk_wsnet_num_params(gk_wsnet N, int64_t* n);
/* params: host or device floats; resets Adam's moments and step count. */
GK_API int gk_wsnet_set_params(gk_wsnet N, const float* params, void* stream);
GK_API int gk_wsnet_get_params(gk_wsnet N, float* params, void* stream);
/* Training loss: 0 (default) the mean squared error over all outputs; 1 the
 * energy norm (1 / N) sum_p e_p (A e)_p of e = output - target, with A the
 * 5-point variable-coefficient operator of each sample (cell coefficients
 * exp(input channel 0), faces the harmonic mean of the two cells, a boundary
 * face the cell's own coefficient) -- the norm CG's error decreases in. */
GK_API int gk_wsnet_set_loss(gk_wsnet N, int32_t kind);
/* FP32 forward of B inputs x (B, 2, H, W) into y (B, 1, H, W). */
GK_API int gk_wsnet_forward(gk_wsnet N, int32_t B, const float* x, float* y, void* stream);
/* The training loss against target (B, 1, H, W) and its gradient for every
 * parameter, without an update; loss and grads: host or device,
 * nullable.  Waits for the stream. */
GK_API int gk_wsnet_gradients(gk_wsnet N, int32_t B, const float* x, const float* target, float* loss,
                              float* grads, void* stream);
/* One Adam step on the batch; loss (host or device, nullable) receives the
 * batch loss before the step (asynchronously: synchronize the stream before
 * reading a host value). */
GK_API int gk_wsnet_train_step(gk_wsnet N, int32_t B, const float* x, const float* target, float lr,
                               float* loss, void* stream);
/* BF16 inference of B inputs into y (B, 1, H, W) float.  The four 32 -> 32
 * layers run on the tensor cores (tcgen05.mma, BF16 operands, FP32
 * accumulator in tensor memory), the first and last layer on the CUDA cores
 * with FP32 sums; activations between layers are BF16.  Asynchronous: a
 * device-side wait that gave up is reported by gk_wsnet_check. */
GK_API int gk_wsnet_infer_bf16(gk_wsnet N, int32_t B, const float* x, float* y, void* stream);
/* Waits for the stream; GK_ERR_TIMEOUT (and the flag cleared) if a
 * tensor-core completion wait of an inference since the last check gave up
 * (its outputs are then incomplete), else GK_OK. */
GK_API int gk_wsnet_check(gk_wsnet N, void* stream);
/* Network input of one problem from FP64 g and b (H W each) into feat
 * (2 H W floats) and, when x (FP64 solution) is given, the training target
 * x / (rms(b) * out_scale) into target (H W floats). */
GK_API int gk_wsnet_features(gk_wsnet N, const double* g, const double* b, const double* x, double out_scale,
                             float* feat, float* target, void* stream);
/* The warm start of one problem: features, BF16 inference, x0 = prediction
 * * rms(b) * out_scale in FP64; when A (nullable) is given, x0 is then scaled
 * by alpha = (x0 . b) / (x0 . A x0), the multiple of the prediction closest to
 * the solution in the A-norm (for SPD A never farther than x = 0). */
GK_API int gk_wsnet_warm_start(gk_wsnet N, gk_matrix A, const double* g, const double* b, double out_scale,
                               double* x0, void* stream);
GK_API int gk_wsnet_destroy(gk_wsnet N);

/* ---- reductions ---------------------------------------------------------- */
/* result[0] = sum_i x_i y_i in FP64 with a fixed, run-to-run reproducible
 * reduction order (per-block trees, then one block over the block partials;
 * Section 7.4 stresses the weight of such global reductions in Krylov
 * solvers).  x, y, result: device memory of the current device.  The library
 * keeps one reduction workspace per device, so gk_dot calls on one device
 * must be ordered (issued to one stream, or synchronized). */
GK_API int gk_dot(int64_t n, const double* x, const double* y, double* result, void* stream);

/* result[0] = sum_k v[k] * x[c[k]] over k < n: the SpMV's work per stored
 * entry (an index and a value streamed, x gathered, one fused multiply-add)
 * without its row structure.  Not in the paper: it measures the ceiling that
 * the SpMV kernels of a matrix with scattered columns are held against (the
 * same (c, v) stream as the matrix's CSR arrays).  c, v, x, result: device
 * memory of the current device; an index outside [0, n_x) contributes 0.
 * Terms are summed per thread (threads take k, k + T, ... with T the
 * launch's threads), then by the block and grid reductions of gk_dot, so the
 * result is reproducible run to run.  One workspace per device: calls on one
 * device must be ordered. */
GK_API int gk_gather_dot(int64_t n, const int32_t* c, const double* v, const double* x, int64_t n_x,
                         double* result, void* stream);

/* *tflops = the rate, in TFLOP/s, at which the current device retires FP64
 * fused multiply-adds (2 flops each), measured: a kernel of 8 independent
 * FMA chains per thread, 8 blocks of 256 threads per SM, iters FMAs per
 * chain, timed with CUDA events on stream after one warm-up launch.  Not in
 * the paper: the SpMV and Krylov kernels issue one FP64 FMA per stored entry
 * and several per row, and on a GPU whose FP64 rate is low next to its
 * memory bandwidth that rate is a roofline of its own, reported beside the
 * HBM one.  Synchronous (waits for the measurement); allocates nothing but
 * two events.  iters >= 1 (about 20,000 gives a launch of a few ms). */
GK_API int gk_fp64_rate(int64_t iters, double* tflops, void* stream);

/* gk_dot without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- for example
 * code whose GPU memory is entirely reserved by another allocator (a
 * framework's caching pool sized to the whole device), or a host application
 * that forbids libraries from owning device allocations -- whereas gk_dot
 * allocates its reduction workspace on its first call on each device.
 *   - Scratch: a static device array inside the library holding 1024 block
 *     partial sums plus one counter (about 8 KB); every GPU that loads the
 *     library keeps it until the process exits.  The reduction uses 4 blocks
 *     per SM, so GPUs with more than 256 SMs are rejected with
 *     GK_ERR_UNSUPPORTED.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - The scratch is shared by every call on a device and keeps the last
 *     call's contents; each call clears the counter on its stream before the
 *     kernel.  Calls that overlap on the GPU (different streams, no ordering)
 *     race on it: order them.
 *   - Result, order of summation and arguments as gk_dot. */
GK_API int gk_dot_noalloc(int64_t n, const double* x, const double* y, double* result, void* stream);

/* ---- failure detection --------------------------------------------------- */
/* Exercises the failure path of the library's bounded device-side waits (not
 * in the paper).  Every wait on the GPU -- a thread block waiting for its
 * bulk copies, the cooperative-grid solver's barriers, the tensor-core
 * completions -- gives up after about 2 s, sets a device error bit and lets
 * the kernel return, so a stalled wait ends the call with GK_ERR_TIMEOUT (or
 * gk_status.device_error) instead of hanging the GPU.  This call launches one
 * warp that waits, through the same code, on a barrier phase that nothing
 * completes; it returns after the wait has given up (about 2 s at the
 * maximum SM clock) with *err_out = the device error word: 1 when the wait
 * timed out as designed.  The device stays usable afterwards.  Synchronous
 * on stream; allocates and frees 4 bytes of device memory. */
GK_API int gk_wait_selftest(int32_t* err_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GK_H */
