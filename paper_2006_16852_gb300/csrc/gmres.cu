// gmres.cu -- restarted GMRES(m) (Section 3.1's Krylov family; Saad and
// Schultz 1986) with right preconditioning, A M^{-1} u = b, x = M^{-1} u.
//
// One cycle: V_0 = r / ||r||, g = ||r|| e_1; for j = 0 .. m-1 an Arnoldi
// step w = A M^{-1} V_j orthogonalised against V_0..V_j by classical
// Gram-Schmidt applied twice (each pass: all the dot products in one launch,
// then one update launch), h_{j+1,j} = ||w||, V_{j+1} = w / h_{j+1,j}, the
// previous Givens rotations applied to the new column of H and a new one
// that zeroes h_{j+1,j}; |g_{j+1}| is the residual norm the criteria see.
// The cycle ends when the criteria are met, after m steps, or when
// h_{j+1,j} = 0; then y = H^{-1} g, x += M^{-1} V y and r = b - A x is
// recomputed (its norm is checked again at the start of the next cycle).
// Each cycle is one CUDA graph whose Arnoldi steps sit in a conditional
// WHILE node; the host reads the stop flag once per cycle.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "gk_device.cuh"
#include "gk_internal.h"
#include "precond_device.cuh"
#include "solver_state.cuh"

namespace gk {

constexpr int kGmresMaxDim = 128;
constexpr int kGmresThreads = 256;

struct GmresState {
  double H[(kGmresMaxDim + 1) * kGmresMaxDim];  // H[i * m + j]
  double cs[kGmresMaxDim], sn[kGmresMaxDim];
  double g[kGmresMaxDim + 1], y[kGmresMaxDim];
  double hn;   // ||w|| of the current step
  int j;       // current Arnoldi step
  int steps;   // steps taken in this cycle
  int end;     // the cycle ends after this step
  int pass;    // Gram-Schmidt pass (0, 1)
};

struct GmresData {
  int m = 30;
  int64_t ldv = 0;         // stride between Arnoldi vectors
  double* V = nullptr;     // (m + 1) * ldv
  double* w = nullptr;
  double* z = nullptr;     // M^{-1} V_j, then V y
  double* dot_part = nullptr;  // (m + 1) x dot_grid partial dot products
  int dot_grid = 1;
  GmresState* gs = nullptr;
  double* part = nullptr;  // norm reduction partials
  unsigned int* counter = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int64_t bytes = 0;
};

namespace {

struct GmArgs {
  int n;
  int m;
  int64_t ldv;
  double* V;
  double* w;
  double* z;
  double* x;
  const double* r;
  const double* dinv;
  const double* blocks;
  int bs, nblocks;
  GmresState* gs;
  SolverState* st;
  double* dot_part;
  int dot_grid;
  double* part;
  unsigned int* counter;
  cudaGraphConditionalHandle cond;
};

#define GM_FOR_ROWS(i) \
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x)

#define GM_FOR_BLOCK_LANES(L)                                                                    \
  const int lane_ = threadIdx.x & 31;                                                           \
  const int bpw_ = 32 / a.bs;                                                                   \
  const int nw_ = (gridDim.x * blockDim.x) >> 5;                                                 \
  for (int w_ = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w_ * bpw_ < a.nblocks; w_ += nw_) \
    for (BjLane L = bj_lane(w_ * bpw_, lane_, a.bs, a.n, a.nblocks), *once_ = &L; once_; once_ = nullptr)

// The true residual r and its norm are known: V_0 = r / ||r||, g = ||r|| e_1.
__global__ void __launch_bounds__(kGmresThreads) gm_begin_kernel(GmArgs a) {
  const double beta = a.st->rnorm;
  const double inv = 1.0 / beta;
  GM_FOR_ROWS(i) a.V[i] = a.r[i] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    GmresState* s = a.gs;
    for (int k = 0; k <= a.m; ++k) s->g[k] = 0.0;
    s->g[0] = beta;
    s->j = 0;
    s->steps = 0;
    s->end = 0;
  }
}

// z = M^{-1} V_j (a copy without a preconditioner, so that the SpMV that
// follows always reads z).
template <int PK, int BS>
__global__ void __launch_bounds__(kGmresThreads) gm_precond_kernel(GmArgs a) {
  const double* v = a.V + static_cast<int64_t>(a.gs->j) * a.ldv;
  if (PK == PREC_BLOCK) {
    GM_FOR_BLOCK_LANES(L) {
      const double rv = L.active ? v[L.row] : 0.0;
      const double zz = bj_apply_lane<BS>(a.blocks, L, a.bs, rv);
      if (L.active) a.z[L.row] = zz;
    }
  } else {
    GM_FOR_ROWS(i) a.z[i] = PK == PREC_SCALAR ? a.dinv[i] * v[i] : v[i];
  }
}

// Partial sums of V_i . w for i <= j: block (bx, i) sums the rows of its
// grid-stride share; one block row of the grid per Arnoldi vector.
__global__ void __launch_bounds__(kGmresThreads) gm_dots_kernel(GmArgs a) {
  __shared__ double scratch[kRedScratch];
  const int i = blockIdx.y;
  if (i > a.gs->j) return;
  const double* v = a.V + static_cast<int64_t>(i) * a.ldv;
  double sum[1] = {0.0};
  GM_FOR_ROWS(r) sum[0] = fma(v[r], a.w[r], sum[0]);
  block_sum<1, double>(sum, scratch);
  if (threadIdx.x == 0) a.dot_part[static_cast<int64_t>(i) * a.dot_grid + blockIdx.x] = sum[0];
}

// h_i = sum of the partials in block order; H(i, j) += h_i (the first pass
// sets it).  One thread per i.
__global__ void gm_collect_kernel(GmArgs a) {
  GmresState* s = a.gs;
  const int j = s->j;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    double h = 0.0;
    for (int b = 0; b < a.dot_grid; ++b) h += a.dot_part[static_cast<int64_t>(i) * a.dot_grid + b];
    a.dot_part[static_cast<int64_t>(a.m + 1) * a.dot_grid + i] = h;  // this pass's coefficients
    if (s->pass == 0) s->H[i * a.m + j] = h;
    else s->H[i * a.m + j] += h;
  }
}

// w -= sum_{i <= j} h_i V_i; on the second pass also ||w||^2 (the last block
// stores ||w|| and advances the pass counter).
__global__ void __launch_bounds__(kGmresThreads) gm_orth_kernel(GmArgs a) {
  __shared__ double scratch[kRedScratch];
  __shared__ double hs[kGmresMaxDim + 1];
  GmresState* s = a.gs;
  const int j = s->j;
  const bool last = s->pass == 1;
  const double* h = a.dot_part + static_cast<int64_t>(a.m + 1) * a.dot_grid;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  double nn[1] = {0.0};
  GM_FOR_ROWS(r) {
    double wv = a.w[r];
    for (int i = 0; i <= j; ++i) wv = fma(-hs[i], a.V[static_cast<int64_t>(i) * a.ldv + r], wv);
    a.w[r] = wv;
    nn[0] = fma(wv, wv, nn[0]);
  }
  double tot[1];
  const bool lastblk = grid_sum<1, double>(nn, a.part, a.counter, scratch, tot);
  if (lastblk && threadIdx.x == 0) {
    if (last) s->hn = sqrt(tot[0]);
    s->pass = last ? 0 : 1;
  }
}

// h_{j+1,j} = ||w||; Givens rotations; residual estimate and criteria;
// whether the cycle goes on (re-arms the WHILE node).
__global__ void gm_step_kernel(GmArgs a) {
  GmresState* s = a.gs;
  SolverState* st = a.st;
  const int m = a.m, j = s->j;
  double* H = s->H;
  const double hn = s->hn;
  H[(j + 1) * m + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double x0 = H[i * m + j], x1 = H[(i + 1) * m + j];
    H[i * m + j] = s->cs[i] * x0 + s->sn[i] * x1;
    H[(i + 1) * m + j] = -s->sn[i] * x0 + s->cs[i] * x1;
  }
  const double x0 = H[j * m + j], x1 = H[(j + 1) * m + j];
  const double d = hypot(x0, x1);
  s->cs[j] = d != 0.0 ? x0 / d : 1.0;
  s->sn[j] = d != 0.0 ? x1 / d : 0.0;
  H[j * m + j] = d;
  H[(j + 1) * m + j] = 0.0;
  s->g[j + 1] = -s->sn[j] * s->g[j];
  s->g[j] = s->cs[j] * s->g[j];
  st->iter += 1;
  st->spmvs += 1;
  st->iter_guard += 1;
  st->rnorm = fabs(s->g[j + 1]);
  const int stop = check_stop(st, st->rnorm, st->iter);
  s->steps = j + 1;
  s->end = (stop != GK_STOP_NONE || j + 1 >= m || hn == 0.0 || !isfinite(hn)) ? 1 : 0;
  if (!isfinite(hn) || !isfinite(st->rnorm)) st->stop = GK_STOP_NAN;
  cudaGraphSetConditional(a.cond, s->end ? 0u : 1u);
}

// V_{j+1} = w / h_{j+1,j} unless the cycle ends; then j += 1.
__global__ void __launch_bounds__(kGmresThreads) gm_next_kernel(GmArgs a) {
  GmresState* s = a.gs;
  if (!s->end) {
    const double inv = 1.0 / s->hn;
    double* vn = a.V + static_cast<int64_t>(s->j + 1) * a.ldv;
    GM_FOR_ROWS(i) vn[i] = a.w[i] * inv;
  }
}

__global__ void gm_advance_kernel(GmArgs a) {
  if (!a.gs->end) a.gs->j += 1;
}

// y = H^{-1} g (back substitution over the steps taken).
__global__ void gm_solve_kernel(GmArgs a) {
  GmresState* s = a.gs;
  const int m = a.m, k = s->steps;
  for (int i = k - 1; i >= 0; --i) {
    double v = s->g[i];
    for (int l = i + 1; l < k; ++l) v = fma(-s->H[i * m + l], s->y[l], v);
    s->y[i] = v / s->H[i * m + i];
  }
}

// z = V y.
__global__ void __launch_bounds__(kGmresThreads) gm_combine_kernel(GmArgs a) {
  __shared__ double ys[kGmresMaxDim];
  const int k = a.gs->steps;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = a.gs->y[i];
  __syncthreads();
  GM_FOR_ROWS(r) {
    double v = 0.0;
    for (int i = 0; i < k; ++i) v = fma(a.V[static_cast<int64_t>(i) * a.ldv + r], ys[i], v);
    a.z[r] = v;
  }
}

// x += M^{-1} z.
template <int PK, int BS>
__global__ void __launch_bounds__(kGmresThreads) gm_update_kernel(GmArgs a) {
  if (PK == PREC_BLOCK) {
    GM_FOR_BLOCK_LANES(L) {
      const double zv = L.active ? a.z[L.row] : 0.0;
      const double u = bj_apply_lane<BS>(a.blocks, L, a.bs, zv);
      if (L.active) a.x[L.row] += u;
    }
  } else {
    GM_FOR_ROWS(i) a.x[i] += PK == PREC_SCALAR ? a.dinv[i] * a.z[i] : a.z[i];
  }
}

// Criteria at the start of a cycle on the true residual.
__global__ void gm_check_kernel(SolverState* st) {
  if (st->stop == GK_STOP_NONE) st->stop = check_stop(st, st->rnorm, st->iter);
}

#undef GM_FOR_ROWS
#undef GM_FOR_BLOCK_LANES

GmArgs gm_args(const Solver& S, const GmresData& d) {
  GmArgs a;
  a.n = static_cast<int>(S.n);
  a.m = d.m;
  a.ldv = d.ldv;
  a.V = d.V;
  a.w = d.w;
  a.z = d.z;
  a.x = S.x;
  a.r = S.r;
  a.dinv = S.P ? S.P->dinv : nullptr;
  a.blocks = S.P ? S.P->blocks : nullptr;
  a.bs = S.P ? S.P->bs : 1;
  a.nblocks = S.P ? static_cast<int>(S.P->nblocks) : 0;
  a.gs = d.gs;
  a.st = S.st;
  a.dot_part = d.dot_part;
  a.dot_grid = d.dot_grid;
  a.part = d.part;
  a.counter = d.counter;
  a.cond = d.cond;
  return a;
}

int gm_grid(const Solver& S) {
  const int64_t units = (S.pk == PREC_BLOCK) ? ((S.P->nblocks + (32 / S.P->bs) - 1) / (32 / S.P->bs)) * 32 : S.n;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((units + kGmresThreads - 1) / kGmresThreads,
                                                                  8 * sm_count())));
}

#define GM_LAUNCH_PK(kern, grid, s, args)                                                    \
  do {                                                                                      \
    if (S.pk == PREC_BLOCK) {                                                               \
      switch (S.P->bs) {                                                                    \
        case 4: kern<PREC_BLOCK, 4><<<grid, kGmresThreads, 0, s>>>(args); break;           \
        case 8: kern<PREC_BLOCK, 8><<<grid, kGmresThreads, 0, s>>>(args); break;           \
        case 16: kern<PREC_BLOCK, 16><<<grid, kGmresThreads, 0, s>>>(args); break;         \
        case 32: kern<PREC_BLOCK, 32><<<grid, kGmresThreads, 0, s>>>(args); break;         \
        default: kern<PREC_BLOCK, 0><<<grid, kGmresThreads, 0, s>>>(args); break;          \
      }                                                                                     \
    } else if (S.pk == PREC_SCALAR) {                                                       \
      kern<PREC_SCALAR, 0><<<grid, kGmresThreads, 0, s>>>(args);                            \
    } else {                                                                                \
      kern<PREC_NONE, 0><<<grid, kGmresThreads, 0, s>>>(args);                              \
    }                                                                                       \
    GK_TRY_CUDA(cudaGetLastError());                                                        \
  } while (0)

Epi gm_epi(const Solver& S, int mode, const double* u, double* y, int fin) {
  Epi e;
  e.mode = mode;
  e.fin = fin;
  e.u = u;
  e.y = y;
  e.st = S.st;
  e.skip_mode = 0;
  e.partials = S.partials;
  e.counter = S.counter;
  e.err = &S.st->err;
  return e;
}

// One Arnoldi step (the WHILE body).
int gm_enqueue_step(const Solver& S, const GmresData& d, const GmArgs& a, cudaStream_t s) {
  const int grid = gm_grid(S);
  GM_LAUNCH_PK(gm_precond_kernel, grid, s, a);
  GK_TRY(spmv_launch(*S.A, d.z, gm_epi(S, EPI_COPY, nullptr, d.w, FIN_NONE), s));
  for (int pass = 0; pass < 2; ++pass) {
    gm_dots_kernel<<<dim3(d.dot_grid, d.m + 1), kGmresThreads, 0, s>>>(a);
    GK_TRY_CUDA(cudaGetLastError());
    gm_collect_kernel<<<1, 128, 0, s>>>(a);
    GK_TRY_CUDA(cudaGetLastError());
    gm_orth_kernel<<<d.dot_grid, kGmresThreads, 0, s>>>(a);
    GK_TRY_CUDA(cudaGetLastError());
  }
  gm_step_kernel<<<1, 1, 0, s>>>(a);
  GK_TRY_CUDA(cudaGetLastError());
  gm_next_kernel<<<grid, kGmresThreads, 0, s>>>(a);
  GK_TRY_CUDA(cudaGetLastError());
  gm_advance_kernel<<<1, 1, 0, s>>>(a);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

// A cycle: begin -> WHILE { Arnoldi step } -> y -> x += M^{-1} V y -> r = b - A x.
int gm_build_graph(Solver& S, GmresData& d) {
  if (!d.cs) GK_TRY_CUDA(cudaStreamCreateWithFlags(&d.cs, cudaStreamNonBlocking));
  GK_TRY_CUDA(cudaGraphCreate(&d.graph, 0));
  GK_TRY_CUDA(cudaGraphConditionalHandleCreate(&d.cond, d.graph, 1, cudaGraphCondAssignDefault));
  const GmArgs a = gm_args(S, d);
  const int grid = gm_grid(S);
  GK_TRY_CUDA(cudaStreamBeginCaptureToGraph(d.cs, d.graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int rc = GK_OK;
  cudaGraph_t body = nullptr;
  do {
    gm_begin_kernel<<<grid, kGmresThreads, 0, d.cs>>>(a);
    cudaError_t e = cudaGetLastError();
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(d.cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = d.cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, d.graph, deps, nullptr, ndeps, &np);
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(d.cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) {
      rc = cuda_error(e, "GMRES graph");
      break;
    }
    body = np.conditional.phGraph_out[0];
    gm_solve_kernel<<<1, 1, 0, d.cs>>>(a);
    gm_combine_kernel<<<grid, kGmresThreads, 0, d.cs>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = cuda_error(e, "GMRES graph");
      break;
    }
    GM_LAUNCH_PK(gm_update_kernel, grid, d.cs, a);
    rc = spmv_launch(*S.A, S.x, gm_epi(S, EPI_RESID, S.b, S.r, FIN_GMRES_RESID), d.cs);
  } while (false);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(d.cs, &captured);
  if (rc != GK_OK) return rc;
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture (GMRES)");
  GK_TRY_CUDA(cudaStreamBeginCaptureToGraph(d.cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  rc = gm_enqueue_step(S, d, a, d.cs);
  e = cudaStreamEndCapture(d.cs, &captured);
  if (rc != GK_OK) return rc;
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture (GMRES step)");
  GK_TRY_CUDA(cudaGraphInstantiate(&d.exec, d.graph, 0));
  return GK_OK;
}

__global__ void gm_init_kernel(SolverState* st, double factor, long long max_iters, int rel_to_b,
                               unsigned long long time_limit_ns) {
  SolverState z;
  memset(&z, 0, sizeof(z));
  z.factor = factor;
  z.max_iters = max_iters;
  z.rel_to_b = rel_to_b;
  z.time_limit_ns = time_limit_ns;
  *st = z;
}

}  // namespace

int gmres_generate(Solver* S) {
  std::unique_ptr<GmresData> hold(new GmresData);
  GmresData* d = hold.get();
  const int m = S->crit.krylov_dim > 0 ? S->crit.krylov_dim : 30;
  if (m > kGmresMaxDim) return set_error(GK_ERR_ARG, "GMRES: krylov_dim %d (at most %d)", m, kGmresMaxDim);
  d->m = m;
  d->ldv = (S->n + 31) / 32 * 32;
  d->dot_grid = std::max(1, std::min<int>(2 * sm_count(), static_cast<int>((S->n + kGmresThreads - 1) / kGmresThreads)));
  int64_t* by = &d->bytes;
  int rc = GK_OK;
  do {
    if ((rc = dalloc_n(&d->V, static_cast<size_t>((m + 1) * d->ldv), by)) ||
        (rc = dalloc_n(&d->w, static_cast<size_t>(d->ldv), by)) || (rc = dalloc_n(&d->z, static_cast<size_t>(d->ldv), by)) ||
        (rc = dalloc_n(&d->dot_part, static_cast<size_t>((m + 2) * d->dot_grid + m + 2), by)) ||
        (rc = dalloc_n(&d->gs, 1, by)) || (rc = dalloc_n(&d->part, static_cast<size_t>(d->dot_grid + 2), by)) ||
        (rc = dalloc_n(&d->counter, 1, by)))
      break;
    cudaError_t e = cudaMemset(d->counter, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(d->gs, 0, sizeof(GmresState));
    if (e != cudaSuccess) rc = cuda_error(e, "GMRES allocation");
  } while (false);
  if (rc != GK_OK) {
    gmres_release(hold.release());
    return rc;
  }
  S->device_bytes += d->bytes;
  S->gm = hold.release();
  return GK_OK;
}

int gmres_solve(Solver* S, cudaStream_t s) {
  GmresData& d = *S->gm;
  if (!d.exec) GK_TRY(gm_build_graph(*S, d));
  const gk_criteria& c = S->crit;
  const unsigned long long tl = c.time_limit_s > 0 ? static_cast<unsigned long long>(c.time_limit_s * 1e9) : 0ull;
  gm_init_kernel<<<1, 1, 0, s>>>(S->st, c.reduction_factor, static_cast<long long>(c.max_iters), c.rel_to_b, tl);
  GK_TRY_CUDA(cudaGetLastError());
  GK_TRY(spmv_launch(*S->A, S->x, gm_epi(*S, EPI_RESID, S->b, S->r, FIN_SETUP_RESID), s));
  // at most max_iters / 1 + 2 cycles (every cycle takes at least one step)
  for (int64_t cyc = 0; cyc <= c.max_iters + 2; ++cyc) {
    gm_check_kernel<<<1, 1, 0, s>>>(S->st);
    GK_TRY_CUDA(cudaGetLastError());
    GK_TRY_CUDA(cudaMemcpyAsync(S->h_st, S->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    GK_TRY_CUDA(cudaStreamSynchronize(s));
    if (S->h_st->stop != GK_STOP_NONE) break;
    GK_TRY_CUDA(cudaGraphLaunch(d.exec, s));
  }
  // the true residual of the result, as the other solvers report it
  return spmv_launch(*S->A, S->x, gm_epi(*S, EPI_RESID, S->b, d.w, FIN_TRUE_RESID), s);
}

void gmres_release(GmresData* d) {
  if (!d) return;
  if (d->exec) cudaGraphExecDestroy(d->exec);
  if (d->graph) cudaGraphDestroy(d->graph);
  if (d->cs) cudaStreamDestroy(d->cs);
  for (void* p : {static_cast<void*>(d->V), static_cast<void*>(d->w), static_cast<void*>(d->z),
                  static_cast<void*>(d->dot_part), static_cast<void*>(d->gs), static_cast<void*>(d->part),
                  static_cast<void*>(d->counter)})
    dfree(p);
  delete d;
}

}  // namespace gk
