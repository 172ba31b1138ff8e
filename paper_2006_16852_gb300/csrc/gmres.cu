// gmres.cu -- restarted GMRES(m) (Section 3.1's Krylov family; Saad and
// Schultz 1986) with right preconditioning, A M^{-1} u = b, x = M^{-1} u.
//
// One cycle: V_0 = r / ||r||, g = ||r|| e_1; for j = 0 .. m-1 an Arnoldi
// step w = A M^{-1} V_j orthogonalised against V_0..V_j by classical
// Gram-Schmidt applied twice (each pass: all the dot products in one launch
// whose last block also sums them, then one update launch), h_{j+1,j} =
// ||w||, V_{j+1} = w / h_{j+1,j} (with M^{-1} V_{j+1} for the next step in
// the same pass), the previous Givens rotations applied to the new column
// of H and a new one that zeroes h_{j+1,j}; |g_{j+1}| is the residual norm
// the criteria see.  On a GB300 the 4 (j+1) n FP64 multiply-adds of the two
// passes, not the bytes, bound a step.
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
constexpr int kDotThreads = 256;  // the dot-product sweep

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
  double* dot_part = nullptr;  // (m + 1) x dot_grid partial dot products, then m + 1 coefficients
  int dot_grid = 1;            // blocks of the dot-product launch
  int grid = 1;                // blocks of the orthogonalisation launch
  GmresState* gs = nullptr;
  double* part = nullptr;  // norm reduction partials
  unsigned int* counter = nullptr;   // [0] norm reduction, [1] dot products
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
  double* coef;  // this pass's coefficients h_i (after the (m + 1) x dot_grid partials)
  double* part;
  unsigned int* counter;
  unsigned int* dcounter;
  cudaGraphConditionalHandle cond;
  int host;  // 1: host-driven steps (no conditional node; a step after the cycle's end does nothing)
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

// h_i = V_i . w for every i <= j in one sweep: chunks of 8 vectors, each
// chunk's FP64 partial sums per block (w is re-read per chunk, from L2); the
// last block to arrive sums the block partials of every i in block order
// (warp k takes i = k, k + 8, ...: lane l adds partials l, l + 32, ... into
// four interleaved sums so that four loads are in flight, then the four
// sums and one butterfly) and stores this pass's coefficients and H(i, j)
// (the first pass sets it, the second adds).
__global__ void __launch_bounds__(kDotThreads) gm_dots_kernel(GmArgs a) {
  __shared__ double scratch[8 * kDotThreads];
  __shared__ unsigned int s_last;
  GmresState* s = a.gs;
  if (a.host && s->end) return;
  const int j = s->j;
  const int G = gridDim.x;
  for (int c0 = 0; c0 <= j; c0 += 8) {
    double acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.0;
    GM_FOR_ROWS(r) {
      const double wr = a.w[r];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (c0 + k <= j) acc[k] = fma(a.V[static_cast<int64_t>(c0 + k) * a.ldv + r], wr, acc[k]);
    }
    // block sums of the 8 values, warp k summing value k (lane l adds
    // threads l, l + 32, ... in order, then one butterfly): block_sum's
    // order, but eight warps share the slow FP64 adds instead of one
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) scratch[k * kDotThreads + threadIdx.x] = acc[k];
    __syncthreads();
    const int wk = threadIdx.x >> 5, lk = threadIdx.x & 31;
    if (wk < 8 && c0 + wk <= j) {
      double v = scratch[wk * kDotThreads + lk];
      for (int u = lk + 32; u < kDotThreads; u += 32) v += scratch[wk * kDotThreads + u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lk == 0) a.dot_part[static_cast<int64_t>(c0 + wk) * G + blockIdx.x] = v;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(a.dcounter, 1u);
    s_last = (t == static_cast<unsigned int>(G) - 1u) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i <= j; i += kDotThreads / 32) {
    const double* p = a.dot_part + static_cast<int64_t>(i) * G;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int b = lane;
    for (; b + 96 < G; b += 128) {
      v0 += __ldcg(p + b);
      v1 += __ldcg(p + b + 32);
      v2 += __ldcg(p + b + 64);
      v3 += __ldcg(p + b + 96);
    }
    for (; b < G; b += 32) v0 += __ldcg(p + b);
    double v = (v0 + v1) + (v2 + v3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
      a.coef[i] = v;
      if (s->pass == 0) s->H[i * a.m + j] = v;
      else s->H[i * a.m + j] += v;
    }
  }
  if (threadIdx.x == 0) *a.dcounter = 0u;
}

// w -= sum_{i <= j} h_i V_i; on the second pass also ||w||^2 (the last block
// stores ||w|| and advances the pass counter).
__global__ void __launch_bounds__(kGmresThreads) gm_orth_kernel(GmArgs a) {
  __shared__ double scratch[kRedScratch];
  __shared__ double hs[kGmresMaxDim + 1];
  GmresState* s = a.gs;
  if (a.host && s->end) return;
  const int j = s->j;
  const bool last = s->pass == 1;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) hs[i] = a.coef[i];
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
// whether the cycle goes on (re-arms the WHILE node).  One warp: column j
// of H and the previous rotations are staged in shared memory by all lanes,
// lane 0 applies the rotations there, all lanes write the column back.
__global__ void __launch_bounds__(32) gm_step_kernel(GmArgs a) {
  __shared__ double col[kGmresMaxDim + 1], cs[kGmresMaxDim], sn[kGmresMaxDim];
  GmresState* s = a.gs;
  if (a.host && s->end) return;
  SolverState* st = a.st;
  const int m = a.m, j = s->j, lane = threadIdx.x;
  double* H = s->H;
  for (int i = lane; i <= j; i += 32) col[i] = H[i * m + j];
  for (int i = lane; i < j; i += 32) {
    cs[i] = s->cs[i];
    sn[i] = s->sn[i];
  }
  __syncwarp();
  if (lane == 0) {
    const double hn = s->hn;
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double x0 = col[i], x1 = col[i + 1];
      col[i] = cs[i] * x0 + sn[i] * x1;
      col[i + 1] = -sn[i] * x0 + cs[i] * x1;
    }
    const double x0 = col[j], x1 = col[j + 1];
    const double d = hypot(x0, x1);
    const double c = d != 0.0 ? x0 / d : 1.0, sj = d != 0.0 ? x1 / d : 0.0;
    s->cs[j] = c;
    s->sn[j] = sj;
    col[j] = d;
    col[j + 1] = 0.0;
    const double gj = s->g[j];
    s->g[j + 1] = -sj * gj;
    s->g[j] = c * gj;
    st->iter += 1;
    st->spmvs += 1;
    st->iter_guard += 1;
    st->rnorm = fabs(s->g[j + 1]);
    const int stop = check_stop(st, st->rnorm, st->iter);
    s->steps = j + 1;
    s->end = (stop != GK_STOP_NONE || j + 1 >= m || hn == 0.0 || !isfinite(hn)) ? 1 : 0;
    if (!isfinite(hn) || !isfinite(st->rnorm)) st->stop = GK_STOP_NAN;
    if (!s->end) s->j = j + 1;
    if (!a.host) cudaGraphSetConditional(a.cond, s->end ? 0u : 1u);
  }
  __syncwarp();
  for (int i = lane; i <= j + 1; i += 32) H[i * m + j] = col[i];
}

// Unless the cycle ends: V_{j+1} = w / h_{j+1,j} and z = M^{-1} V_{j+1}
// for the next step (the step kernel has advanced j already).
template <int PK, int BS>
__global__ void __launch_bounds__(kGmresThreads) gm_next_kernel(GmArgs a) {
  GmresState* s = a.gs;
  if (s->end) return;
  const double inv = 1.0 / s->hn;
  double* vn = a.V + static_cast<int64_t>(s->j) * a.ldv;
  if (PK == PREC_BLOCK) {
    GM_FOR_BLOCK_LANES(L) {
      const double v = L.active ? a.w[L.row] * inv : 0.0;
      if (L.active) vn[L.row] = v;
      const double zz = bj_apply_lane<BS>(a.blocks, L, a.bs, v);
      if (L.active) a.z[L.row] = zz;
    }
  } else {
    GM_FOR_ROWS(i) {
      const double v = a.w[i] * inv;
      vn[i] = v;
      a.z[i] = PK == PREC_SCALAR ? a.dinv[i] * v : v;
    }
  }
}

// y = H^{-1} g (back substitution over the steps taken): the block stages
// the k x k upper triangle and g in shared memory (dynamic, k * k + k
// doubles), thread 0 substitutes row by row from there.
__global__ void __launch_bounds__(256) gm_solve_kernel(GmArgs a) {
  extern __shared__ double sh[];
  GmresState* s = a.gs;
  const int m = a.m, k = s->steps;
  double* hk = sh;          // hk[i * k + l] = H(i, l)
  double* gy = sh + k * k;  // g, then y
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    const int i = idx / k, l = idx - (idx / k) * k;
    hk[idx] = l >= i ? s->H[i * m + l] : 0.0;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) gy[i] = s->g[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double v = gy[i];
      for (int l = i + 1; l < k; ++l) v = fma(-hk[i * k + l], gy[l], v);
      gy[i] = v / hk[i * k + i];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) s->y[i] = gy[i];
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
  a.coef = d.dot_part + static_cast<int64_t>(d.m + 1) * d.dot_grid;
  a.part = d.part;
  a.counter = d.counter;
  a.dcounter = d.counter + 1;
  a.cond = d.cond;
  a.host = 0;
  return a;
}

size_t gm_solve_smem(const GmresData& d) { return sizeof(double) * (static_cast<size_t>(d.m) * d.m + d.m); }

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

// One Arnoldi step (the WHILE body); z = M^{-1} V_j is ready on entry.
int gm_enqueue_step(const Solver& S, const GmresData& d, const GmArgs& a, cudaStream_t s) {
  const int grid = gm_grid(S);
  GK_TRY(spmv_launch(*S.A, d.z, gm_epi(S, EPI_COPY, nullptr, d.w, FIN_NONE), s));
  for (int pass = 0; pass < 2; ++pass) {
    gm_dots_kernel<<<d.dot_grid, kDotThreads, 0, s>>>(a);
    GK_TRY_CUDA(cudaGetLastError());
    gm_orth_kernel<<<d.grid, kGmresThreads, 0, s>>>(a);
    GK_TRY_CUDA(cudaGetLastError());
  }
  gm_step_kernel<<<1, 32, 0, s>>>(a);
  GK_TRY_CUDA(cudaGetLastError());
  GM_LAUNCH_PK(gm_next_kernel, grid, s, a);
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
    if (e == cudaSuccess) {
      rc = [&]() -> int {
        GM_LAUNCH_PK(gm_precond_kernel, grid, d.cs, a);
        return GK_OK;
      }();
      if (rc != GK_OK) break;
    }
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
    gm_solve_kernel<<<1, 256, gm_solve_smem(d), d.cs>>>(a);
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
  d->grid = std::max(1, std::min<int>(4 * sm_count(), static_cast<int>((S->n + kGmresThreads - 1) / kGmresThreads)));
  d->dot_grid = std::max(1, std::min<int>(4 * sm_count(), static_cast<int>((S->n + kDotThreads - 1) / kDotThreads)));
  int64_t* by = &d->bytes;
  int rc = GK_OK;
  do {
    if ((rc = dalloc_n(&d->V, static_cast<size_t>((m + 1) * d->ldv), by)) ||
        (rc = dalloc_n(&d->w, static_cast<size_t>(d->ldv), by)) || (rc = dalloc_n(&d->z, static_cast<size_t>(d->ldv), by)) ||
        (rc = dalloc_n(&d->dot_part, static_cast<size_t>((m + 1) * d->dot_grid + m + 2), by)) ||
        (rc = dalloc_n(&d->gs, 1, by)) || (rc = dalloc_n(&d->part, static_cast<size_t>(d->grid + 2), by)) ||
        (rc = dalloc_n(&d->counter, 2, by)))
      break;
    if ((rc = set_smem(gm_solve_kernel, gm_solve_smem(*d))) != GK_OK) break;
    cudaError_t e = cudaMemset(d->counter, 0, 2 * sizeof(unsigned int));
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

// A cycle launched kernel by kernel (check_every > 0): the Arnoldi steps in
// groups of check_every, each group followed by a read of the cycle's end
// flag; the same kernels as the graph, for profilers that cannot see
// kernels under a conditional node.
int gm_host_cycle(Solver& S, GmresData& d, cudaStream_t s) {
  GmArgs a = gm_args(S, d);
  a.host = 1;
  const int grid = gm_grid(S);
  gm_begin_kernel<<<grid, kGmresThreads, 0, s>>>(a);
  GK_TRY_CUDA(cudaGetLastError());
  GM_LAUNCH_PK(gm_precond_kernel, grid, s, a);
  const int every = std::max(1, S.crit.check_every);
  for (int done = 0; done < d.m;) {
    for (int k = 0; k < every && done < d.m; ++k, ++done) GK_TRY(gm_enqueue_step(S, d, a, s));
    int end = 0;
    GK_TRY_CUDA(cudaMemcpyAsync(&end, &d.gs->end, sizeof(int), cudaMemcpyDeviceToHost, s));
    GK_TRY_CUDA(cudaStreamSynchronize(s));
    if (end) break;
  }
  gm_solve_kernel<<<1, 256, gm_solve_smem(d), s>>>(a);
  gm_combine_kernel<<<grid, kGmresThreads, 0, s>>>(a);
  GK_TRY_CUDA(cudaGetLastError());
  GM_LAUNCH_PK(gm_update_kernel, grid, s, a);
  return spmv_launch(*S.A, S.x, gm_epi(S, EPI_RESID, S.b, S.r, FIN_GMRES_RESID), s);
}

int gmres_solve(Solver* S, cudaStream_t s) {
  GmresData& d = *S->gm;
  const bool host = S->crit.check_every > 0;
  if (!host && !d.exec) GK_TRY(gm_build_graph(*S, d));
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
    if (host) GK_TRY(gm_host_cycle(*S, d, s));
    else GK_TRY_CUDA(cudaGraphLaunch(d.exec, s));
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
