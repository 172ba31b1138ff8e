// gk_internal.h -- host/device declarations shared by the library's
// translation units: handle structures, the device solver state, the SpMV
// epilogue descriptor and the launchers.
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gk.h"

namespace gk {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);

#define GK_TRY_CUDA(call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ::gk::cuda_error(e_, #call); \
  } while (0)

#define GK_TRY(call)            \
  do {                          \
    int rc_ = (call);           \
    if (rc_ != GK_OK) return rc_; \
  } while (0)

// Device allocation that records its size in *counter (may be null).
int dalloc(void** p, size_t bytes, int64_t* counter);
template <class T>
int dalloc_n(T** p, size_t n, int64_t* counter) {
  return dalloc(reinterpret_cast<void**>(p), n * sizeof(T), counter);
}
void dfree(void* p);
// Stream-ordered allocation on s from the device's default memory pool (which
// keeps up to 8 GB of freed memory for reuse); dfree releases it.
int dalloc_async(void** p, size_t bytes, int64_t* counter, cudaStream_t s);
template <class T>
int dalloc_async_n(T** p, size_t n, int64_t* counter, cudaStream_t s) {
  return dalloc_async(reinterpret_cast<void**>(p), n * sizeof(T), counter, s);
}

// Number of SMs of the current device (cached per device).
int sm_count();
int current_device();

// Lets kernel `fn` use `smem` bytes of dynamic shared memory and asks for
// the largest shared-memory carveout, so that as many of its blocks fit an
// SM as its shared memory allows (with the default carveout the occupancy
// query and the launch may settle for fewer).
int set_smem(const void* fn, size_t smem);
template <typename F>
int set_smem(F* fn, size_t smem) {
  return set_smem(reinterpret_cast<const void*>(fn), smem);
}

// Launches kern<<<grid, block, smem, s>>>(args...) with programmatic stream
// serialization: the grid may start while the previous kernel in the stream
// drains (its launch overlaps that kernel's tail instead of following it);
// the kernel must call pdl_wait() before reading what the previous kernel
// wrote.  In a captured graph the dependency becomes a programmatic edge.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Makes `dev` current for the lifetime of the guard, then restores the
// caller's device.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// ---------------------------------------------------------------------------
// device-side solver state (one per solver handle; also used by gk_dot)
// ---------------------------------------------------------------------------
struct SolverState {
  double rho, rho_prev, alpha, beta, omega;
  double factor, ref, tol;   // residual criterion: ||r|| <= tol = factor * ref
  double rnorm, snorm;       // last recurred ||r||, ||s|| (BiCGSTAB)
  double bnorm, rnorm0;
  double red[2];             // raw sums of the last reduction (diagnostics)
  double true_rr;            // ||b - A x||^2 of the final check
  long long iter, max_iters, spmvs;
  long long iter_guard;      // iterations the device-side loop has run
  long long outer;           // iterative refinement: outer steps taken
  unsigned long long t_start_ns, time_limit_ns;
  int stop;                  // GK_STOP_*
  int half;                  // BiCGSTAB: converged at the half step
  int rel_to_b;
  int err;                   // device error bits (kErrTimeout)
};

// What the last block of a reduction does with the sums.
enum Fin : int {
  FIN_NONE = 0,
  FIN_SETUP_RESID,  // sums = (||r0||^2, ||b||^2): set ref and tol
  FIN_CG_START,     // sums = (r.z): rho; check the criteria at k = 0
  FIN_CG_SIGMA,     // sums = (p.q): alpha = rho / sigma
  FIN_CG_ITER,      // sums = (r.z, r.r): k += 1, criteria, beta
  FIN_BI_START,     // sums = (r^.r): criteria at k = 0, first rho and beta
  FIN_BI_RHV,       // sums = (r^.v): alpha
  FIN_BI_S,         // sums = (s.s): half-step test
  FIN_BI_OMEGA,     // sums = (s.t, t.t): omega
  FIN_BI_ITER,      // sums = (r^.r, r.r): k += 1, criteria, next rho/beta
  FIN_TRUE_RESID,   // sums = (||b - A x||^2, -): store
  FIN_IR_RESID,     // sums = (||b - A x||^2, ||b||^2): outer criteria of refinement
  FIN_FCG_ITER,     // sums = (r.z, r.r, z.q): k += 1, criteria, flexible beta
  FIN_CGS_START,    // sums = (r^.r): criteria at k = 0, first rho
  FIN_CGS_ALPHA,    // sums = (r^.v^): alpha
  FIN_CGS_ITER,     // sums = (r^.r, r.r): k += 1, criteria, next rho and beta
  FIN_GMRES_RESID,  // sums = (||b - A x||^2, -): the true residual after a GMRES cycle
};

// ---------------------------------------------------------------------------
// SpMV epilogue: what happens to each finished row sum s_i
// ---------------------------------------------------------------------------
enum EpiMode : int {
  EPI_COPY = 4,   // y_i = s_i (alpha = 1, beta = 0: no FP64 work beyond the row sum)
  EPI_PLAIN = 0,  // y_i = alpha s_i (beta == 0) or fma(beta, y_i, alpha s_i)
  EPI_RESID = 1,  // y_i = u_i - s_i (u = b): sums (y.y, u.u)
  EPI_DOT = 2,    // y_i = s_i: sums (u.y)
  EPI_DOT2 = 3,   // y_i = s_i: sums (u.y, y.y)
};

struct Epi {
  int mode = EPI_PLAIN;
  int fin = FIN_NONE;
  double alpha = 1.0, beta = 0.0;
  int beta_zero = 1;          // beta == 0, decided on the host (no FP64 compare per row)
  const double* u = nullptr;
  double* y = nullptr;
  SolverState* st = nullptr;  // scalars the reduction feeds
  int skip_mode = 0;          // 0 never skip, 1 skip if st->stop, 2 if st->stop || st->half
  double* partials = nullptr; // reduction scratch (>= grid * 2 doubles)
  unsigned int* counter = nullptr;
  int* err = nullptr;         // device error word for bounded waits
};

// ---------------------------------------------------------------------------
// matrix handle
// ---------------------------------------------------------------------------
// Iterations of CG (and of the refinement's inner CG) per pass of a solve
// graph's loop body.
constexpr int kGraphUnroll = 4;

constexpr int kMergeThreads = 256;
constexpr int kMergeItems = 8;  // merge-path items (row ends + nonzeros) per lane
constexpr int kMergeTile = 32 * kMergeItems;  // items per warp tile
// GK_CSR: rows of up to kSliceMaxLen entries go to length-sorted slices of 32
// rows; longer rows are cut into pieces of at most kPieceLen consecutive
// entries, each summed by one warp.
constexpr int kSliceMaxLen = 256;
constexpr int kPieceLen = 512;
constexpr int kSliceThreads = 256;
constexpr int kEllThreads = 256;
// GK_HYB's COO overflow: each lane sums kCooPerLane consecutive entries, a
// warp takes a chunk of kCooChunk.
constexpr int kCooPerLane = 8;
constexpr int kCooChunk = 32 * kCooPerLane;
constexpr int kCooThreads = 256;
// Blocks of the merge-path fix-up launch; reduction scratch holds
// 2 * (max grid + kFixupMaxGrid) doubles.
constexpr int kFixupMaxGrid = 64;

struct MergePlan {
  int64_t n_rows = 0, nnz = 0, n_tiles = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  int32_t* tile_i = nullptr;  // [n_tiles + 1] merge coordinates of tile starts
  int32_t* tile_j = nullptr;
  // per-apply scratch: partial sums of rows cut by tile boundaries (per
  // tile: the part of its first row when that row began in an earlier tile
  // and ends in this one; the part of the row left open at its end)
  double* head_val = nullptr;
  double* carry_val = nullptr;
  int grid = 0;
};

struct Matrix {
  std::atomic<int> refs{1};
  int device = 0;
  int64_t n_rows = 0, n_cols = 0, nnz = 0;
  int format = GK_CSR;
  int64_t device_bytes = 0;
  // CSR copy (every format keeps it)
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  std::vector<int32_t> h_rowptr;  // host copy of the row pointers (planning)
  // GK_CSR: rows sorted by decreasing length.  Rows of <= kSliceMaxLen
  // entries in slices of 32 rows, each slice column-major (entry k of lane l
  // at sl_off[c] + 32 k + l) and padded to its longest row with column -1;
  // the rest by length: mid rows (warp per row), big rows (block per row).
  int32_t* sl_perm = nullptr;   // [n_sell] the row of each slice lane
  int64_t* sl_off = nullptr;    // [n_slices + 1]
  int32_t* sl_col = nullptr;
  double* sl_val = nullptr;
  int64_t n_sell = 0, n_slices = 0, sl_entries = 0;
  // rows longer than kSliceMaxLen (n_long of them), cut into pieces of at
  // most kPieceLen consecutive entries, longest first: {row, first entry,
  // end entry, slot}; slot is -1 when the row is a single piece (its warp
  // finishes it), else the piece's partial-sum slot in pc_sum.  Rows of
  // several pieces (lr_row, their slots lr_off[i] .. lr_off[i + 1]) are
  // finished by a second launch that adds their pieces in order.
  int4* pc = nullptr;
  int64_t n_pc = 0, n_long = 0;
  int32_t* lr_row = nullptr;
  int32_t* lr_off = nullptr;
  int64_t n_lr = 0;
  double* pc_sum = nullptr;
  int grid_sl = 0;        // persistent grid of the epilogues with reductions
  int grid_sl_plain = 0;  // ... of the plain applies (more blocks per SM)
  // GK_CSR_MERGE
  MergePlan merge;
  // GK_ELL / GK_HYB
  int64_t K = 0, ld = 0;
  int32_t* ell_col = nullptr;
  double* ell_val = nullptr;
  int grid_ell = 0;
  // GK_HYB overflow ("tail"): the entries of rows longer than K beyond their
  // first K, in COO form sorted by (row, column): tail_row / tail_col /
  // tail_val (the same entries are also addressed row-compressed through
  // tail_rowptr, which the FP32 copy of the refinement uses).  Arrays are
  // padded to whole chunks of kCooChunk entries.
  int64_t m_tail = 0, tail_nnz = 0;
  int32_t* tail_rows = nullptr;
  int32_t* tail_rowptr = nullptr;
  int32_t* tail_row = nullptr;   // [tail_nnz] global row of each entry
  int32_t* tail_col = nullptr;
  double* tail_val = nullptr;
  int32_t* tail_slot = nullptr;  // [n_rows] index into tail_sum or -1
  double* tail_sum = nullptr;    // [m_tail]
  int64_t coo_chunks = 0;        // chunks of kCooChunk entries
  int32_t* coo_first = nullptr;  // [coo_chunks] first / last row of each chunk
  int32_t* coo_last = nullptr;
  double* coo_head = nullptr;    // [coo_chunks] partial sums of those rows in the chunk
  double* coo_tail = nullptr;
  int grid_coo = 0;
  // scratch of gk_apply / precond generation
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  int* err = nullptr;
  SolverState* dot_st = nullptr;  // gk_apply_dot: receives the fused sum
  int* h_flag = nullptr;          // pinned host words of the preconditioner generation's error check
  double* stage_in = nullptr;   // host-vector staging
  double* stage_out = nullptr;
  int max_grid = 0;             // partials hold max_grid * 2 doubles
};

void matrix_release(Matrix* A);

// Enqueue y = op(A x) with the epilogue e on stream s.  x has n_cols entries.
int spmv_launch(const Matrix& A, const double* x, const Epi& e, cudaStream_t s);

// Grid size used by SpMV launches of this matrix (for scratch sizing).
int spmv_max_grid(const Matrix& A);
// Persistent grid sizes of the SpMV kernels for a given amount of work.
int merge_grid(int64_t n_tiles);
int coo_grid(int64_t n_chunks);
int sliced_grid(int64_t warp_items, bool plain);
int ell_grid(int64_t n_rows);

// Format construction (matrix.cu).
int build_merge_plan(MergePlan& P, int64_t n_rows, int64_t nnz, const int32_t* rowptr,
                     const int32_t* col, const double* val, int64_t* bytes, cudaStream_t s);

// ---------------------------------------------------------------------------
// vector arguments (host or device)
// ---------------------------------------------------------------------------
struct VecArg {
  const void* user = nullptr;
  double* dev = nullptr;  // device pointer the kernels use
  bool staged = false;    // user pointer is host memory
};
// Classifies p with one pointer query: device memory of `device` is used in
// place; host memory is staged through *staging (allocated on first use,
// n doubles, size added to *bytes) and copied in when copy_in.
int vec_in(VecArg& v, const void* p, int64_t n, double** staging, int64_t* bytes, bool copy_in, int device,
           cudaStream_t s);
// For staged outputs: copies back and synchronizes s.
int vec_out(VecArg& v, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// preconditioner handle
// ---------------------------------------------------------------------------
struct Precond {
  std::atomic<int> refs{1};
  int device = 0;
  Matrix* A = nullptr;
  int64_t n = 0;
  int bs = 1;
  int64_t nblocks = 0;
  double* dinv = nullptr;    // scalar Jacobi: 1/a_ii
  double* blocks = nullptr;  // block Jacobi: inverse blocks, each row-major
  int64_t block_elems = 0;
  double* stage_in = nullptr;
  double* stage_out = nullptr;
  int64_t device_bytes = 0;
};

void precond_release(Precond* P);

enum PrecKind : int { PREC_NONE = 0, PREC_SCALAR = 1, PREC_BLOCK = 2 };

struct IrData;
struct GmresData;

// Solver handle.
struct Solver {
  std::atomic<int> refs{1};
  int device = 0;
  Matrix* A = nullptr;
  Precond* P = nullptr;
  int kind = GK_CG;
  int pk = PREC_NONE;
  gk_criteria crit{};
  int64_t n = 0;
  int64_t device_bytes = 0;
  double *b = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
  double *rh = nullptr, *ph = nullptr, *s = nullptr, *sh = nullptr, *t = nullptr;
  SolverState* st = nullptr;
  SolverState* h_st = nullptr;  // pinned
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  int grid_vec = 1;
  cudaStream_t cs = nullptr;  // capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  IrData* ir = nullptr;  // GK_IR_CG: the FP32 inner solver
  int64_t ir_idle = 0;   // GK_IR_CG: inner iterations launched after the inner stops (last solve)
  GmresData* gm = nullptr;  // GK_GMRES: Arnoldi basis and Hessenberg state
  int cl_lg = -1;           // GK_CG / GK_BICGSTAB small-system form: rows per CTA = 2^cl_lg (-1: none)
  int cl_rpt = 1;           // ... rows per thread
  bool cl_stage = false;    // ... the CTA's rows of the matrix staged in shared memory
  int cl_nnz = 0;           // ... room for that many entries
  size_t cl_smem = 0;       // ... dynamic shared memory per CTA
  int gr_grid = 0;          // GK_CG mid-size form: CTAs of the cooperative launch (0: not available)
  int gr_rpt = 1, gr_rows = 0;
  bool gr_stage = false;            // its CTAs' rows of the matrix staged in shared memory
  int gr_nnz = 0;
  size_t gr_smem = 0;
  double* gr_part = nullptr;        // its per-CTA partial sums
  unsigned int* gr_sync = nullptr;  // its barrier words
};

// Mixed-precision iterative refinement (mixed.cu).
int ir_generate(Solver* S);
int ir_solve(Solver* S, cudaStream_t s);
void ir_release(IrData* ir);

// CG of a small system in one thread-block cluster (cluster_cg.cu): the plan
// (sets cl_lg >= 0 when the form applies and a 16-CTA cluster can run) and
// the solve (one launch; the state is left as the graph form leaves it
// before its final true-residual check).
int cluster_cg_plan(Solver* S);
int cluster_cg_solve(Solver* S, cudaStream_t s);

// CG of a mid-size system (32,769 .. 262,144 rows, rows of at most 64
// entries) in one cooperative launch with grid-wide barriers (grid_cg.cu).
int grid_cg_plan(Solver* S);
int grid_cg_solve(Solver* S, cudaStream_t s);

// Restarted GMRES (gmres.cu).
int gmres_generate(Solver* S);
int gmres_solve(Solver* S, cudaStream_t s);
void gmres_release(GmresData* d);


// z = M^{-1} r as a standalone launch.
int precond_apply_launch(const Precond* P, const double* r, double* z, cudaStream_t s);

}  // namespace gk

// The opaque C handles are the C++ objects themselves.
inline gk::Matrix* as_matrix(gk_matrix h) { return reinterpret_cast<gk::Matrix*>(h); }
inline gk::Precond* as_precond(gk_precond h) { return reinterpret_cast<gk::Precond*>(h); }
