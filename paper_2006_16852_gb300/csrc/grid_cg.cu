// grid_cg.cu -- the whole preconditioned CG solve (Section 3.1, criteria of
// Section 2.5) of a mid-size system in ONE cooperative launch: one CTA per
// SM, every CTA resident for the whole solve, the phases separated by
// grid-wide barriers in global memory.
//
// Between 32,768 rows (the cluster form's limit) and a few hundred thousand,
// an iteration of the graph form is still bound by launch and reduction
// latency (~20 us for three launches) rather than by its bytes or FP64
// work.  Here an iteration is two grid barriers plus the work spread over
// all 152 SMs.
//
// Rows: CTA b owns rows [b R, (b + 1) R), thread t the CTA's rows t, t + 256,
// ...; x, r, q and the Jacobi diagonal of a row stay in the owning thread's
// registers, and r is mirrored in global memory (L2) with the direction
// vectors, because the SpMV reads them at arbitrary columns.  An iteration:
//   p = z + beta p_prev, formed at every gathered column by the reader
//       exactly as by the row's owner (no barrier between the direction
//       update and the SpMV); q = A p (CSR rows, each summed in increasing
//       column order as the oracle's ordered SpMV), sigma = p.q -> barrier
//   alpha = rho / sigma; x += alpha p; r -= alpha q; z = M^{-1} r;
//   rho' = r.z, ||r||^2                                     -> barrier
//   criteria; beta = rho' / rho
// A reduction: each CTA's sum (fixed butterflies) is stored in its slot, the
// barrier, then every CTA adds all the slots in one fixed order -- all CTAs
// hold bit-identical totals and take identical stop decisions, so they pass
// the same number of barriers.  Every barrier wait is bounded: a wait that
// gives up sets the error bit and an abort flag that ends every other
// CTA's waits at once, so the launch always returns.
#include <algorithm>
#include <vector>

#include "gk_device.cuh"
#include "gk_internal.h"
#include "solver_state.cuh"

namespace gk {
namespace {

constexpr int kGrThreads = 256;
constexpr int kGrMaxRpt = 8;
constexpr int64_t kGrMinRows = 32769;    // below: the cluster form
constexpr int64_t kGrMaxRows = 262144;   // above: the graph form's SpMV kernels win
constexpr int kGrMaxRowLen = 64;         // one thread per row: no long rows

struct GridArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const double* b;
  double* x;
  double* p;   // x0, then the direction vectors p_k (k even)
  double* p2;  // the direction vectors p_k (k odd)
  double* r;   // the residual, mirrored for the gathers of the SpMV
  const double* dinv;
  SolverState* st;
  double* part;        // [4 slots][grid][2] CTA partial sums
  unsigned int* sync;  // [0] arrivals, [1] generation, [2] abort
  int n;
  int rows_per_cta;
  int stage_nnz;  // STAGE: room for this many entries of the CTA's rows in shared memory
};

// Grid barrier (thread 0 of every CTA arrives; the last arrival resets the
// count and advances the generation).  Returns false if the solve is being
// aborted (this or another CTA's wait gave up).
__device__ __forceinline__ bool grid_barrier(const GridArgs& a, unsigned int& gen, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vsync = a.sync;
    __threadfence();
    const unsigned int g0 = gen;
    if (atomicAdd(a.sync, 1u) == gridDim.x - 1) {
      atomicExch(a.sync, 0u);
      __threadfence();
      atomicAdd(a.sync + 1, 1u);
    } else {
      const long long t0 = clock64();
      for (uint32_t i = 0;; ++i) {
        if (vsync[1] != g0) break;
        if (vsync[2] != 0u) {
          ok = 0;
          break;
        }
        if (i > kMaxPolls || clock64() - t0 > kMaxWaitCycles) {
          atomicOr(&a.st->err, kErrTimeout);
          atomicExch(a.sync + 2, 1u);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    gen = g0 + 1;
    if (vsync[2] != 0u) ok = 0;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// The iteration's scalars, derived by thread 0 of each CTA.
struct GrScalars {
  double rho, alpha, beta, rnorm, rnorm0, bnorm, ref, tol;
  long long iter, spmvs;
  int stop;
};

// Sum of v over the grid: CTA sum by butterflies, stored in the slot, the
// barrier, then all CTA sums added by every CTA in the same order (thread j
// takes CTAs j, j + 256, ...; then butterflies); thread 0 runs post(totals),
// deriving the iteration's scalars into shared memory once per CTA instead
// of in every warp (FP64 divisions and square roots are long), and the
// closing barrier publishes them.
template <int K, typename Post>
__device__ __forceinline__ bool grid_total(const GridArgs& a, int slot, double (&v)[K], double (*wsum)[2],
                                           Post post, unsigned int& gen, int* s_ok) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum<K, double>(v);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) wsum[warp][k] = v[k];
  }
  __syncthreads();
  double* slots = a.part + static_cast<int64_t>(slot) * gridDim.x * 2;
  if (warp == 0) {
    double s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = lane < kGrThreads / 32 ? wsum[lane][k] : 0.0;
#pragma unroll
    for (int o = kGrThreads / 64; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) slots[blockIdx.x * 2 + k] = s[k];
    }
  }
  if (!grid_barrier(a, gen, s_ok)) return false;
  double s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0.0;
  for (int j = threadIdx.x; j < static_cast<int>(gridDim.x); j += kGrThreads) {
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] += __ldcg(slots + j * 2 + k);
  }
  warp_sum<K, double>(s);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) wsum[warp][k] = s[k];
  }
  __syncthreads();
  if (warp == 0) {
    double u[K];
#pragma unroll
    for (int k = 0; k < K; ++k) u[k] = lane < kGrThreads / 32 ? wsum[lane][k] : 0.0;
#pragma unroll
    for (int o = kGrThreads / 64; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) u[k] += __shfl_xor_sync(0xffffffffu, u[k], o);
    }
    if (lane == 0) post(u);
  }
  __syncthreads();
  return true;
}

// STAGE: the CTA's rows of the matrix are copied to shared memory once (one
// gather round trip per row instead of three dependent ones).
template <int PK, int RPT, bool STAGE>
__global__ void __launch_bounds__(kGrThreads) cg_grid_kernel(GridArgs a) {
  extern __shared__ double s_val[];  // STAGE: values, then row pointers and columns
  __shared__ double wsum[kGrThreads / 32][2];
  __shared__ GrScalars sc;
  __shared__ int s_ok;
  const int t = threadIdx.x;
  const int row0 = blockIdx.x * a.rows_per_cta;
  const int R = a.rows_per_cta;
  int32_t* s_rp = reinterpret_cast<int32_t*>(s_val + a.stage_nnz);
  int32_t* s_col = s_rp + R + 1;
  if (STAGE) {
    const int first = min(row0, a.n), rows_here = max(0, min(R, a.n - row0));
    const int e0 = __ldg(a.rowptr + first);
    for (int l = t; l <= R; l += kGrThreads) s_rp[l] = __ldg(a.rowptr + first + min(l, rows_here)) - e0;
    const int ne = __ldg(a.rowptr + first + rows_here) - e0;
    for (int k = t; k < ne; k += kGrThreads) {
      s_col[k] = __ldg(a.col + e0 + k);
      s_val[k] = __ldg(a.val + e0 + k);
    }
  }
  SolverState* st = a.st;
  const double factor = st->factor;
  const long long max_iters = st->max_iters;
  const int rel_to_b = st->rel_to_b;
  unsigned int gen = 0;

  double x[RPT], r[RPT], d[RPT];
  bool own[RPT];
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int l = t + u * kGrThreads;
    const int i = row0 + l;
    own[u] = l < a.rows_per_cta && i < a.n;
    x[u] = own[u] ? a.x[i] : 0.0;
    d[u] = (PK == PREC_SCALAR && own[u]) ? __ldg(a.dinv + i) : 1.0;
    if (own[u]) a.p[i] = x[u];
  }
  // sum_k val_k v(col_k) in increasing k, v read through `value`
  auto row_apply = [&](int i, auto value) {
    double s = 0.0;
    const int l = i - row0;
    int k = STAGE ? s_rp[l] : __ldg(a.rowptr + i);
    const int k1 = STAGE ? s_rp[l + 1] : __ldg(a.rowptr + i + 1);
    for (; k + 4 <= k1; k += 4) {
      int c[4];
      double v[4], pv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = STAGE ? s_col[k + u] : __ldg(a.col + k + u);
        v[u] = STAGE ? s_val[k + u] : __ldg(a.val + k + u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) pv[u] = value(c[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) s = fma(v[u], pv[u], s);
    }
    for (; k < k1; ++k) s = fma(STAGE ? s_val[k] : __ldg(a.val + k), value(STAGE ? s_col[k] : __ldg(a.col + k)), s);
    return s;
  };
  auto criteria = [&](double rn, double tol, long long k) {
    if (!isfinite(rn)) return GK_STOP_NAN;
    if (rn <= tol) return GK_STOP_CONVERGED;
    if (k >= max_iters) return GK_STOP_MAX_ITERS;
    return GK_STOP_NONE;
  };
  if (t == 0) {
    sc.rnorm0 = sc.bnorm = sc.rnorm = sc.rho = sc.tol = 0.0;
    sc.ref = sc.alpha = 1.0;
    sc.beta = 0.0;
    sc.iter = 0;
    sc.spmvs = 1;
    sc.stop = GK_STOP_NONE;
  }
  bool ok = grid_barrier(a, gen, &s_ok);  // x0 everywhere (in the first p buffer)
  if (ok) {
    double v[2] = {0.0, 0.0};
    auto x0_at = [&](int c) { return __ldcg(a.p + c); };
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      if (!own[u]) continue;
      const int i = row0 + t + u * kGrThreads;
      const double bi = a.b[i];
      r[u] = bi - row_apply(i, x0_at);
      a.r[i] = r[u];
      v[0] = fma(r[u], r[u], v[0]);
      v[1] = fma(bi, bi, v[1]);
    }
    ok = grid_total<2>(a, 0, v, wsum, [&](const double* tt) {
      sc.rnorm0 = sqrt(tt[0]);
      sc.bnorm = sqrt(tt[1]);
      double ref = rel_to_b ? sc.bnorm : sc.rnorm0;
      if (ref == 0.0) ref = 1.0;
      sc.ref = ref;
      sc.tol = factor * ref;
      sc.rnorm = sc.rnorm0;
    }, gen, &s_ok);
  }
  if (ok) {
    double v[1] = {0.0};
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      if (!own[u]) continue;
      const double z = PK == PREC_SCALAR ? d[u] * r[u] : r[u];
      v[0] = fma(r[u], z, v[0]);
    }
    ok = grid_total<1>(a, 1, v, wsum, [&](const double* tt) {
      sc.rho = tt[0];
      sc.stop = criteria(sc.rnorm, sc.tol, 0);
    }, gen, &s_ok);
  }
  // Iteration k reads p_{k-1} from buffer (k+1) % 2 and r_k from a.r (both
  // complete since the previous barrier), forms p_k = z_k + beta p_{k-1} at
  // every gathered column exactly as its owner does, and the owner stores
  // p_k in buffer k % 2, which nobody reads before the next iteration.
  // Two barriers per iteration.
  double* pbuf[2] = {a.p, a.p2};
  for (long long k = 0; ok && sc.stop == GK_STOP_NONE; ++k) {
    const double* pold = pbuf[(k + 1) & 1];
    double* pnew = pbuf[k & 1];
    const bool first = k == 0;
    const double beta = sc.beta;
    auto p_at = [&](int c) {
      const double rc = __ldcg(a.r + c);
      const double z = PK == PREC_SCALAR ? __ldg(a.dinv + c) * rc : rc;
      return first ? z : fma(beta, __ldcg(pold + c), z);
    };
    double q[RPT], pl[RPT];
    double v[1] = {0.0};
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      q[u] = 0.0;
      pl[u] = 0.0;
      if (!own[u]) continue;
      const int i = row0 + t + u * kGrThreads;
      const double z = PK == PREC_SCALAR ? d[u] * r[u] : r[u];
      pl[u] = first ? z : fma(beta, __ldcg(pold + i), z);
      pnew[i] = pl[u];
      q[u] = row_apply(i, p_at);
      v[0] = fma(pl[u], q[u], v[0]);
    }
    if (!(ok = grid_total<1>(a, 2, v, wsum, [&](const double* tt) {
          sc.spmvs += 1;
          const double sigma = tt[0];
          if (!isfinite(sigma)) sc.stop = GK_STOP_NAN;
          else if (sigma <= 0.0) sc.stop = GK_STOP_BREAKDOWN;
          else sc.alpha = sc.rho / sigma;
        }, gen, &s_ok)))
      break;
    if (sc.stop != GK_STOP_NONE) break;
    const double alpha = sc.alpha;
    double w[2] = {0.0, 0.0};
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      if (!own[u]) continue;
      const int i = row0 + t + u * kGrThreads;
      x[u] = fma(alpha, pl[u], x[u]);
      r[u] = fma(-alpha, q[u], r[u]);
      a.r[i] = r[u];
      const double z = PK == PREC_SCALAR ? d[u] * r[u] : r[u];
      w[0] = fma(r[u], z, w[0]);
      w[1] = fma(r[u], r[u], w[1]);
    }
    if (!(ok = grid_total<2>(a, 3, w, wsum, [&](const double* tt) {
          sc.iter += 1;
          sc.rnorm = sqrt(tt[1]);
          sc.stop = criteria(sc.rnorm, sc.tol, sc.iter);
          sc.beta = tt[0] / sc.rho;
          sc.rho = tt[0];
        }, gen, &s_ok)))
      break;
  }
#pragma unroll
  for (int u = 0; u < RPT; ++u)
    if (own[u]) a.x[row0 + t + u * kGrThreads] = x[u];
  if (blockIdx.x == 0 && t == 0) {
    st->rnorm = sc.rnorm;
    st->rnorm0 = sc.rnorm0;
    st->bnorm = sc.bnorm;
    st->ref = sc.ref;
    st->tol = sc.tol;
    st->rho = sc.rho;
    st->alpha = sc.alpha;
    st->beta = sc.beta;
    st->iter = sc.iter;
    st->iter_guard = sc.iter;
    st->spmvs = sc.spmvs;
    st->stop = ok ? sc.stop : GK_STOP_NAN;
  }
}

using GrKernel = void (*)(GridArgs);

template <int PK, bool STAGE>
GrKernel pick_rpt(int rpt) {
  switch (rpt) {
    case 1: return cg_grid_kernel<PK, 1, STAGE>;
    case 2: return cg_grid_kernel<PK, 2, STAGE>;
    case 4: return cg_grid_kernel<PK, 4, STAGE>;
    default: return cg_grid_kernel<PK, 8, STAGE>;
  }
}

GrKernel pick(int pk, int rpt, bool stage) {
  if (pk == PREC_SCALAR) return stage ? pick_rpt<PREC_SCALAR, true>(rpt) : pick_rpt<PREC_SCALAR, false>(rpt);
  return stage ? pick_rpt<PREC_NONE, true>(rpt) : pick_rpt<PREC_NONE, false>(rpt);
}

// Shared memory a CTA's rows take when staged, at most this much.
constexpr size_t kGrStageMax = 160 * 1024;

}  // namespace

int grid_cg_plan(Solver* S) {
  S->gr_grid = 0;
  if (S->kind != GK_CG || S->pk == PREC_BLOCK) return GK_OK;
  const int64_t n = S->n;
  if (n < kGrMinRows || n > kGrMaxRows) return GK_OK;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, S->device) != cudaSuccess || !coop) {
    cudaGetLastError();
    return GK_OK;
  }
  // longest row (one thread per row)
  std::vector<int32_t> rp(static_cast<size_t>(n) + 1);
  GK_TRY_CUDA(cudaMemcpy(rp.data(), S->A->rowptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost));
  int32_t longest = 0;
  for (int64_t i = 0; i < n; ++i) longest = std::max(longest, rp[i + 1] - rp[i]);
  if (longest > kGrMaxRowLen) return GK_OK;
  const int G = sm_count();
  const int64_t per_cta = (n + G - 1) / G;
  int rpt = 1;
  while (static_cast<int64_t>(rpt) * kGrThreads < per_cta) rpt *= 2;
  if (rpt > kGrMaxRpt) return GK_OK;
  int64_t most = 0;
  for (int c = 0; c < G; ++c) {
    const int64_t lo = std::min<int64_t>(c * per_cta, n), hi = std::min<int64_t>((c + 1) * per_cta, n);
    most = std::max<int64_t>(most, rp[hi] - rp[lo]);
  }
  const size_t smem = 12 * static_cast<size_t>(most) + 4 * static_cast<size_t>(per_cta + 1);
  const bool stage = smem <= kGrStageMax;
  GrKernel k = pick(S->pk, rpt, stage);
  if (stage && set_smem(k, smem) != GK_OK) return GK_OK;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kGrThreads, stage ? smem : 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return GK_OK;
  }
  GK_TRY(dalloc_n(&S->gr_part, static_cast<size_t>(4) * G * 2, &S->device_bytes));
  GK_TRY(dalloc_n(&S->gr_sync, 4, &S->device_bytes));
  S->gr_grid = G;
  S->gr_rpt = rpt;
  S->gr_rows = static_cast<int>(per_cta);
  S->gr_stage = stage;
  S->gr_nnz = stage ? static_cast<int>(most) : 0;
  S->gr_smem = stage ? smem : 0;
  return GK_OK;
}

int grid_cg_solve(Solver* S, cudaStream_t s) {
  GridArgs a;
  a.rowptr = S->A->rowptr;
  a.col = S->A->col;
  a.val = S->A->val;
  a.b = S->b;
  a.x = S->x;
  a.p = S->p;
  a.p2 = S->q;
  a.r = S->r;
  a.dinv = S->P ? S->P->dinv : nullptr;
  a.st = S->st;
  a.part = S->gr_part;
  a.sync = S->gr_sync;
  a.n = static_cast<int>(S->n);
  a.rows_per_cta = S->gr_rows;
  a.stage_nnz = S->gr_nnz;
  GK_TRY_CUDA(cudaMemsetAsync(S->gr_sync, 0, 4 * sizeof(unsigned int), s));
  void* args[] = {&a};
  GK_TRY_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(pick(S->pk, S->gr_rpt, S->gr_stage)),
                                          dim3(S->gr_grid), dim3(kGrThreads), args, S->gr_smem, s));
  return GK_OK;
}

}  // namespace gk
