// cluster_cg.cu -- the whole preconditioned CG (and, below, BiCGSTAB) solve
// (Section 3.1, with the criteria of Section 2.5) of a small system in ONE
// launch: a thread-block cluster of 16 CTAs on 16 SMs, the vector the SpMV
// reads (CG's search direction p) distributed over the CTAs' shared memory
// and read across the cluster (distributed shared memory), the other
// vectors in registers of the thread that owns the row, and the cluster's
// hardware barrier between the phases.
//
// Small systems are latency-bound: the graph form spends a few microseconds
// per kernel launch and per grid-wide reduction, three times per iteration,
// while the arithmetic of a 4,096-row iteration is about 40,000 FP64
// multiply-adds.  Here an iteration costs three cluster barriers and the
// FP64 work spread over 16 SMs.
//
// Rows: CTA c owns rows [c L, (c + 1) L), L = 2^lg >= n / 16; thread t owns
// the CTA's rows t, t + 256, ..., (RPT of them).  An iteration:
//   q = A p (CSR, each row summed in increasing column order as the oracle's
//       ordered SpMV), sigma = p.q                                -> barrier
//   alpha = rho / sigma; x += alpha p; r -= alpha q; z = M^{-1} r;
//   rho' = r.z, ||r||^2                                           -> barrier
//   criteria; beta = rho' / rho; p = z + beta p                   -> barrier
// Every reduction: a fixed per-thread order, fixed butterflies within the
// CTA, then the 16 CTA partials added in one fixed butterfly by every CTA --
// all CTAs get bit-identical totals, so their stop decisions (and barrier
// counts) agree.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "gk_device.cuh"
#include "gk_internal.h"
#include "solver_state.cuh"

namespace cg = cooperative_groups;

namespace gk {
namespace {

constexpr int kClCtas = 16;
constexpr int kClThreads = 256;
// rows per thread: n <= 16 * 256 * 8 = 32,768.  The FP64 work of an
// iteration grows with n / 16 per SM here but with n / 152 in the graph form:
// measured (before the matrix staging and the one-thread scalars) 7.1 us per
// iteration at n = 4,096 (graph 21.7 us), but ~29 us at n = 65,536 (graph
// ~23 us); 32,768 rows is below the crossing.
constexpr int kClMaxRpt = 8;

struct ClusterArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const double* b;
  double* x;
  const double* dinv;
  SolverState* st;
  int n;
  int lg;         // rows per CTA = 2^lg
  int stage_nnz;  // STAGE: room for this many entries of the CTA's rows in shared memory
};

// The iteration's scalars, derived by thread 0 and read by the block.
struct ClScalars {
  double rho, alpha, beta, rnorm, rnorm0, bnorm, ref, tol;
  long long iter, spmvs;
  int stop;
};

// Partial sums published by each CTA (one slot per phase, so that a slot is
// never rewritten before every CTA has read it: between the read of a slot
// and its next write lies a barrier that the reader passes only after it).
struct ClSlots {
  double setup[2];  // ||r0||^2, ||b||^2
  double start[1];  // r.z
  double sigma[1];  // p.q
  double iter[2];   // r.z, r.r
};

// Sum of v over the cluster: a butterfly in every warp (all warps at once),
// the 8 warp sums in a 3-level butterfly in warp 0, the CTA's sum published
// in `slot`, the cluster barrier, then the 16 CTA sums in a 4-level
// butterfly over lanes 0..15 -- 12 dependent FP64 adds in all, which on this
// GPU's slow FP64 pipe is what a reduction costs.  Thread 0 alone then runs
// post(totals), which derives the iteration's scalars into shared memory
// (divisions and square roots cost dozens of FP64 instructions: done by
// every warp they took half the FP64 pipe's time); the closing barrier
// publishes them to the block.
template <int K, typename Post>
__device__ __forceinline__ void cluster_total(cg::cluster_group& cl, double (&v)[K], double (*wsum)[K],
                                              double* slot, Post post) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum<K, double>(v);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) wsum[warp][k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
    double s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = lane < kClThreads / 32 ? wsum[lane][k] : 0.0;
#pragma unroll
    for (int o = kClThreads / 64; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) slot[k] = s[k];
    }
  }
  cl.sync();
  if (warp == 0) {
    // lane q < 16 reads CTA q's sum; every CTA adds the same values in the
    // same order
    const double* rs = cl.map_shared_rank(slot, lane & (kClCtas - 1));
    double s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = rs[k];
#pragma unroll
    for (int o = kClCtas / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    }
    if (lane == 0) post(s);
  }
  __syncthreads();
}

// The CTA's rows of the matrix in shared memory: row pointers relative to
// the CTA's first entry (L + 1 ints), columns and values (stage_nnz each).
struct ClStaged {
  const int32_t* rp;
  const int32_t* col;
  const double* val;
};

__device__ __forceinline__ ClStaged cl_stage_rows(const ClusterArgs& a, int row0, int L, double* s_val) {
  int32_t* s_rp = reinterpret_cast<int32_t*>(s_val + a.stage_nnz);
  int32_t* s_col = s_rp + L + 1;
  const int first = min(row0, a.n), rows_here = max(0, min(L, a.n - row0));
  const int e0 = __ldg(a.rowptr + first);
  for (int l = threadIdx.x; l <= L; l += kClThreads) s_rp[l] = __ldg(a.rowptr + first + min(l, rows_here)) - e0;
  const int ne = __ldg(a.rowptr + first + rows_here) - e0;
  for (int k = threadIdx.x; k < ne; k += kClThreads) {
    s_col[k] = __ldg(a.col + e0 + k);
    s_val[k] = __ldg(a.val + e0 + k);
  }
  return ClStaged{s_rp, s_col, s_val};
}

// sum_k val_k v(col_k) over row i in increasing k, v read through gather;
// entries in groups of 4 so that their loads are in flight together.
template <bool STAGE, typename Gather>
__device__ __forceinline__ double cl_row_apply(const ClusterArgs& a, const ClStaged& sr, int i, int row0,
                                               Gather gather) {
  double s = 0.0;
  const int l = i - row0;
  int k = STAGE ? sr.rp[l] : __ldg(a.rowptr + i);
  const int k1 = STAGE ? sr.rp[l + 1] : __ldg(a.rowptr + i + 1);
  for (; k + 4 <= k1; k += 4) {
    int c[4];
    double v[4], pv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c[u] = STAGE ? sr.col[k + u] : __ldg(a.col + k + u);
      v[u] = STAGE ? sr.val[k + u] : __ldg(a.val + k + u);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) pv[u] = gather(c[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) s = fma(v[u], pv[u], s);
  }
  for (; k < k1; ++k) s = fma(STAGE ? sr.val[k] : __ldg(a.val + k), gather(STAGE ? sr.col[k] : __ldg(a.col + k)), s);
  return s;
}

// STAGE: the CTA's rows of the matrix (row pointers, columns, values) are
// copied to shared memory once, so that an SpMV row costs one gather round
// trip instead of three dependent L2 round trips.
template <int PK, int RPT, bool STAGE>
__global__ void __launch_bounds__(kClThreads) cg_cluster_kernel(ClusterArgs a) {
  extern __shared__ double p_loc[];  // this CTA's slice of p (2^lg values), then the staged rows
  __shared__ double* p_of[kClCtas];  // every CTA's slice, as seen from here
  __shared__ ClSlots slots;
  __shared__ double wsum[kClThreads / 32][2];
  __shared__ ClScalars sc;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  const int t = threadIdx.x;
  const int L = 1 << a.lg;
  const int mask = L - 1;
  if (t < kClCtas) p_of[t] = cl.map_shared_rank(p_loc, t);
  const int row0 = rank * L;
  SolverState* st = a.st;
  const double factor = st->factor;
  const long long max_iters = st->max_iters;
  const int rel_to_b = st->rel_to_b;
  ClStaged sr{};
  if (STAGE) sr = cl_stage_rows(a, row0, L, p_loc + L);

  double x[RPT], r[RPT], d[RPT];
  bool own[RPT];
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int l = t + u * kClThreads;
    const int i = row0 + l;
    own[u] = l < L && i < a.n;
    x[u] = own[u] ? a.x[i] : 0.0;
    d[u] = (PK == PREC_SCALAR && own[u]) ? a.dinv[i] : 1.0;
    if (l < L) p_loc[l] = x[u];
  }
  cl.sync();  // p = x0 everywhere (and the staged rows complete)

  // q_i = sum_k val_k p[col_k] (p read across the cluster; the CTA's own
  // slice directly)
  auto gather = [&](int c) {
    const int o = c >> a.lg;
    return o == rank ? p_loc[c & mask] : p_of[o][c & mask];
  };
  auto row_apply = [&](int i) { return cl_row_apply<STAGE>(a, sr, i, row0, gather); };

  // r0 = b - A x0; ||r0||, ||b||: the reference and the tolerance
  {
    double v[2] = {0.0, 0.0};
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      if (!own[u]) continue;
      const int i = row0 + t + u * kClThreads;
      const double bi = a.b[i];
      r[u] = bi - row_apply(i);
      v[0] = fma(r[u], r[u], v[0]);
      v[1] = fma(bi, bi, v[1]);
    }
    cluster_total<2>(cl, v, wsum, slots.setup, [&](const double* tt) {
      sc.rnorm0 = sqrt(tt[0]);
      sc.bnorm = sqrt(tt[1]);
      double ref = rel_to_b ? sc.bnorm : sc.rnorm0;
      if (ref == 0.0) ref = 1.0;
      sc.ref = ref;
      sc.tol = factor * ref;
      sc.rnorm = sc.rnorm0;
      sc.iter = 0;
      sc.spmvs = 1;
      sc.alpha = 1.0;
      sc.beta = 0.0;
    });
  }
  // the criteria (thread 0), in the order of check_stop; no Time criterion
  // here: this form is chosen only without one
  auto criteria = [&](double rn, long long k) {
    if (!isfinite(rn)) return GK_STOP_NAN;
    if (rn <= sc.tol) return GK_STOP_CONVERGED;
    if (k >= max_iters) return GK_STOP_MAX_ITERS;
    return GK_STOP_NONE;
  };
  // z0 = M^{-1} r0, p0 = z0, rho = r0.z0
  {
    double v[1] = {0.0};
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int l = t + u * kClThreads;
      if (!own[u]) continue;
      const double z = PK == PREC_SCALAR ? d[u] * r[u] : r[u];
      p_loc[l] = z;
      v[0] = fma(r[u], z, v[0]);
    }
    cluster_total<1>(cl, v, reinterpret_cast<double(*)[1]>(&wsum[0][0]), slots.start, [&](const double* tt) {
      sc.rho = tt[0];
      sc.stop = criteria(sc.rnorm, 0);
    });
  }
  while (sc.stop == GK_STOP_NONE) {
    double q[RPT];
    {
      double v[1] = {0.0};
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        q[u] = 0.0;
        if (!own[u]) continue;
        const int l = t + u * kClThreads;
        q[u] = row_apply(row0 + l);
        v[0] = fma(p_loc[l], q[u], v[0]);
      }
      cluster_total<1>(cl, v, reinterpret_cast<double(*)[1]>(&wsum[0][0]), slots.sigma, [&](const double* tt) {
        sc.spmvs += 1;
        const double sigma = tt[0];
        if (!isfinite(sigma)) sc.stop = GK_STOP_NAN;
        else if (sigma <= 0.0) sc.stop = GK_STOP_BREAKDOWN;
        else sc.alpha = sc.rho / sigma;
      });
    }
    if (sc.stop != GK_STOP_NONE) break;
    const double alpha = sc.alpha;
    {
      double v[2] = {0.0, 0.0};
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        if (!own[u]) continue;
        const int l = t + u * kClThreads;
        x[u] = fma(alpha, p_loc[l], x[u]);
        r[u] = fma(-alpha, q[u], r[u]);
        const double z = PK == PREC_SCALAR ? d[u] * r[u] : r[u];
        v[0] = fma(r[u], z, v[0]);
        v[1] = fma(r[u], r[u], v[1]);
      }
      cluster_total<2>(cl, v, wsum, slots.iter, [&](const double* tt) {
        sc.iter += 1;
        sc.rnorm = sqrt(tt[1]);
        sc.stop = criteria(sc.rnorm, sc.iter);
        sc.beta = tt[0] / sc.rho;
        sc.rho = tt[0];
      });
    }
    if (sc.stop != GK_STOP_NONE) break;
    const double beta = sc.beta;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      if (!own[u]) continue;
      const int l = t + u * kClThreads;
      const double z = PK == PREC_SCALAR ? d[u] * r[u] : r[u];
      p_loc[l] = fma(beta, p_loc[l], z);
    }
    cl.sync();  // the new p everywhere before the next SpMV
  }
#pragma unroll
  for (int u = 0; u < RPT; ++u)
    if (own[u]) a.x[row0 + t + u * kClThreads] = x[u];
  if (rank == 0 && t == 0) {
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
    st->stop = sc.stop;
  }
  // no CTA may leave while others can still read its shared memory
  cl.sync();
}

// ---- BiCGSTAB (the Templates form of Section 3.1's BiCGSTAB, as the graph
// form computes it) -----------------------------------------------------

struct BiScalars {
  double rho, rho_prev, alpha, omega, beta, rnorm, snorm, rnorm0, bnorm, ref, tol;
  long long iter, spmvs;
  int stop, half;
};

struct BiSlots {
  double setup[2];  // ||r0||^2, ||b||^2
  double start[1];  // r^.r
  double rhv[1];    // r^.v
  double ss[1];     // s.s
  double om[2];     // s.t, t.t
  double it[2];     // r^.r, r.r
};

// rows per thread at most 4 here (10 vectors per row live in registers):
// n <= 16 * 256 * 4 = 16,384
constexpr int kBiMaxRpt = 4;

// An iteration, five cluster barriers: p = r + beta (p - omega v) and
// p^ = M^{-1} p (p^ published); v = A p^ with r^.v -> alpha; s = r - alpha v
// with ||s|| (s^ = M^{-1} s published by the same barrier; half-step exit
// when ||s|| meets the criterion); t = A s^ with s.t, t.t -> omega;
// x += alpha p^ + omega s^, r = s - omega t with r^.r, ||r|| -> the criteria
// and the next rho and beta.  p^ and s^ live in shared memory (read across
// the cluster by the SpMVs), the other vectors in the owner's registers.
template <int PK, int RPT, bool STAGE>
__global__ void __launch_bounds__(kClThreads) bicg_cluster_kernel(ClusterArgs a) {
  extern __shared__ double dyn[];  // p^ slice (L), s^ slice (L), then the staged rows
  __shared__ double* ph_of[kClCtas];
  __shared__ double* sh_of[kClCtas];
  __shared__ BiSlots slots;
  __shared__ double wsum[kClThreads / 32][2];
  __shared__ BiScalars sc;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  const int t = threadIdx.x;
  const int L = 1 << a.lg;
  const int mask = L - 1;
  double* ph_loc = dyn;
  double* sh_loc = dyn + L;
  if (t < kClCtas) {
    ph_of[t] = cl.map_shared_rank(ph_loc, t);
    sh_of[t] = cl.map_shared_rank(sh_loc, t);
  }
  const int row0 = rank * L;
  SolverState* st = a.st;
  const double factor = st->factor;
  const long long max_iters = st->max_iters;
  const int rel_to_b = st->rel_to_b;
  ClStaged sr{};
  if (STAGE) sr = cl_stage_rows(a, row0, L, dyn + 2 * L);
  double x[RPT], r[RPT], rh[RPT], p[RPT], v[RPT], s_[RPT], d[RPT], ph[RPT], sh[RPT];
  bool own[RPT];
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int l = t + u * kClThreads;
    const int i = row0 + l;
    own[u] = l < L && i < a.n;
    x[u] = own[u] ? a.x[i] : 0.0;
    d[u] = (PK == PREC_SCALAR && own[u]) ? a.dinv[i] : 1.0;
    r[u] = rh[u] = p[u] = v[u] = s_[u] = ph[u] = sh[u] = 0.0;
    if (l < L) ph_loc[l] = x[u];
  }
  cl.sync();  // x0 everywhere (in the p^ slices) and the staged rows complete
  auto at = [&](double* const* of, const double* loc) {
    return [=](int c) {
      const int o = c >> a.lg;
      return o == rank ? loc[c & mask] : of[o][c & mask];
    };
  };
  auto criteria = [&](double rn, long long k) {
    if (!isfinite(rn)) return GK_STOP_NAN;
    if (rn <= sc.tol) return GK_STOP_CONVERGED;
    if (k >= max_iters) return GK_STOP_MAX_ITERS;
    return GK_STOP_NONE;
  };
  // a fresh rho = r^.r either fails (NaN, zero) or yields the next beta
  auto new_rho = [&](double rho) {
    if (!isfinite(rho)) sc.stop = GK_STOP_NAN;
    else if (rho == 0.0) sc.stop = GK_STOP_BREAKDOWN;
    else {
      sc.beta = (rho / sc.rho_prev) * (sc.alpha / sc.omega);
      sc.rho = rho;
    }
  };
  {
    double w[2] = {0.0, 0.0};
    const auto x0_at = at(ph_of, ph_loc);
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      if (!own[u]) continue;
      const int i = row0 + t + u * kClThreads;
      const double bi = a.b[i];
      r[u] = bi - cl_row_apply<STAGE>(a, sr, i, row0, x0_at);
      w[0] = fma(r[u], r[u], w[0]);
      w[1] = fma(bi, bi, w[1]);
    }
    cluster_total<2>(cl, w, wsum, slots.setup, [&](const double* tt) {
      sc.rnorm0 = sqrt(tt[0]);
      sc.bnorm = sqrt(tt[1]);
      double ref = rel_to_b ? sc.bnorm : sc.rnorm0;
      if (ref == 0.0) ref = 1.0;
      sc.ref = ref;
      sc.tol = factor * ref;
      sc.rnorm = sc.rnorm0;
      sc.iter = 0;
      sc.spmvs = 1;
      sc.rho = 0.0;
      sc.rho_prev = sc.alpha = sc.omega = 1.0;
      sc.beta = 0.0;
      sc.snorm = 0.0;
      sc.half = 0;
      sc.stop = GK_STOP_NONE;
    });
  }
  {
    // r^ = r0, p = v = 0, rho = r^.r; the criteria at k = 0
    double w[1] = {0.0};
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      if (!own[u]) continue;
      rh[u] = r[u];
      w[0] = fma(r[u], r[u], w[0]);
    }
    cluster_total<1>(cl, w, reinterpret_cast<double(*)[1]>(&wsum[0][0]), slots.start, [&](const double* tt) {
      sc.stop = criteria(sc.rnorm, 0);
      if (sc.stop == GK_STOP_NONE) new_rho(tt[0]);
    });
  }
  const auto ph_at = at(ph_of, ph_loc);
  const auto sh_at = at(sh_of, sh_loc);
  while (sc.stop == GK_STOP_NONE) {
    const double beta = sc.beta, omega0 = sc.omega;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      if (!own[u]) continue;
      p[u] = fma(beta, fma(-omega0, v[u], p[u]), r[u]);
      ph[u] = PK == PREC_SCALAR ? d[u] * p[u] : p[u];
      ph_loc[t + u * kClThreads] = ph[u];
    }
    cl.sync();  // p^ everywhere
    {
      double w[1] = {0.0};
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        if (!own[u]) continue;
        v[u] = cl_row_apply<STAGE>(a, sr, row0 + t + u * kClThreads, row0, ph_at);
        w[0] = fma(rh[u], v[u], w[0]);
      }
      cluster_total<1>(cl, w, reinterpret_cast<double(*)[1]>(&wsum[0][0]), slots.rhv, [&](const double* tt) {
        sc.spmvs += 1;
        const double rhv = tt[0];
        if (!isfinite(rhv)) sc.stop = GK_STOP_NAN;
        else if (rhv == 0.0) sc.stop = GK_STOP_BREAKDOWN;
        else sc.alpha = sc.rho / rhv;
      });
    }
    if (sc.stop != GK_STOP_NONE) break;
    const double alpha = sc.alpha;
    {
      double w[1] = {0.0};
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        if (!own[u]) continue;
        s_[u] = fma(-alpha, v[u], r[u]);
        w[0] = fma(s_[u], s_[u], w[0]);
        sh[u] = PK == PREC_SCALAR ? d[u] * s_[u] : s_[u];
        sh_loc[t + u * kClThreads] = sh[u];
      }
      // the reduction's cluster barrier also publishes s^
      cluster_total<1>(cl, w, reinterpret_cast<double(*)[1]>(&wsum[0][0]), slots.ss, [&](const double* tt) {
        sc.snorm = sqrt(tt[0]);
        if (isfinite(sc.snorm) && sc.snorm <= sc.tol) {
          sc.half = 1;
          sc.iter += 1;
          sc.rnorm = sc.snorm;
          sc.stop = GK_STOP_CONVERGED;
        }
      });
    }
    if (sc.half) {
      // converged at the half step: x += alpha p^, r = s
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        if (!own[u]) continue;
        x[u] = fma(alpha, ph[u], x[u]);
        r[u] = s_[u];
      }
      break;
    }
    double tv[RPT];
    {
      double w[2] = {0.0, 0.0};
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        tv[u] = 0.0;
        if (!own[u]) continue;
        tv[u] = cl_row_apply<STAGE>(a, sr, row0 + t + u * kClThreads, row0, sh_at);
        w[0] = fma(s_[u], tv[u], w[0]);
        w[1] = fma(tv[u], tv[u], w[1]);
      }
      cluster_total<2>(cl, w, wsum, slots.om, [&](const double* tt) {
        sc.spmvs += 1;
        const double ts = tt[0], ttv = tt[1];
        if (!isfinite(ttv) || !isfinite(ts)) sc.stop = GK_STOP_NAN;
        else if (ttv == 0.0) sc.stop = GK_STOP_BREAKDOWN;
        else sc.omega = ts / ttv;
      });
    }
    if (sc.stop != GK_STOP_NONE) break;
    const double omega = sc.omega;
    {
      double w[2] = {0.0, 0.0};
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        if (!own[u]) continue;
        x[u] = fma(omega, sh[u], fma(alpha, ph[u], x[u]));
        r[u] = fma(-omega, tv[u], s_[u]);
        w[0] = fma(rh[u], r[u], w[0]);
        w[1] = fma(r[u], r[u], w[1]);
      }
      cluster_total<2>(cl, w, wsum, slots.it, [&](const double* tt) {
        sc.iter += 1;
        sc.rho_prev = sc.rho;
        sc.rnorm = sqrt(tt[1]);
        int stop = criteria(sc.rnorm, sc.iter);
        if (stop == GK_STOP_NONE && sc.omega == 0.0) stop = GK_STOP_BREAKDOWN;
        sc.stop = stop;
        if (stop == GK_STOP_NONE) new_rho(tt[0]);
      });
    }
  }
#pragma unroll
  for (int u = 0; u < RPT; ++u)
    if (own[u]) a.x[row0 + t + u * kClThreads] = x[u];
  if (rank == 0 && t == 0) {
    st->rnorm = sc.rnorm;
    st->snorm = sc.snorm;
    st->rnorm0 = sc.rnorm0;
    st->bnorm = sc.bnorm;
    st->ref = sc.ref;
    st->tol = sc.tol;
    st->rho = sc.rho;
    st->rho_prev = sc.rho_prev;
    st->alpha = sc.alpha;
    st->omega = sc.omega;
    st->beta = sc.beta;
    st->half = sc.half;
    st->iter = sc.iter;
    st->iter_guard = sc.iter;
    st->spmvs = sc.spmvs;
    st->stop = sc.stop;
  }
  cl.sync();  // no CTA leaves while others can still read its shared memory
}

using ClKernel = void (*)(ClusterArgs);

template <int PK, bool STAGE>
ClKernel pick_rpt(int kind, int rpt) {
  if (kind == GK_BICGSTAB) {
    switch (rpt) {
      case 1: return bicg_cluster_kernel<PK, 1, STAGE>;
      case 2: return bicg_cluster_kernel<PK, 2, STAGE>;
      default: return bicg_cluster_kernel<PK, 4, STAGE>;
    }
  }
  switch (rpt) {
    case 1: return cg_cluster_kernel<PK, 1, STAGE>;
    case 2: return cg_cluster_kernel<PK, 2, STAGE>;
    case 4: return cg_cluster_kernel<PK, 4, STAGE>;
    default: return cg_cluster_kernel<PK, 8, STAGE>;
  }
}

ClKernel pick(int kind, int pk, int rpt, bool stage) {
  if (pk == PREC_SCALAR)
    return stage ? pick_rpt<PREC_SCALAR, true>(kind, rpt) : pick_rpt<PREC_SCALAR, false>(kind, rpt);
  return stage ? pick_rpt<PREC_NONE, true>(kind, rpt) : pick_rpt<PREC_NONE, false>(kind, rpt);
}

cudaLaunchConfig_t launch_config(size_t smem, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClCtas, 1, 1);
  cfg.blockDim = dim3(kClThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Shared memory a CTA's rows take when staged, at most this much.
constexpr size_t kClStageMax = 160 * 1024;

}  // namespace

int cluster_cg_plan(Solver* S) {
  S->cl_lg = -1;
  if ((S->kind != GK_CG && S->kind != GK_BICGSTAB) || S->pk == PREC_BLOCK) return GK_OK;
  const int64_t n = S->n;
  const int max_rpt = S->kind == GK_BICGSTAB ? kBiMaxRpt : kClMaxRpt;
  if (n < 1 || n > static_cast<int64_t>(kClCtas) * kClThreads * max_rpt) return GK_OK;
  int lg = 0;
  while ((static_cast<int64_t>(kClCtas) << lg) < n) ++lg;
  const int rpt = std::max(1, (1 << lg) / kClThreads);
  // the most entries any CTA's rows hold: stage them if they fit
  std::vector<int32_t> rp(static_cast<size_t>(n) + 1);
  GK_TRY_CUDA(cudaMemcpy(rp.data(), S->A->rowptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost));
  int64_t most = 0;
  for (int c = 0; c < kClCtas; ++c) {
    const int64_t lo = std::min<int64_t>(static_cast<int64_t>(c) << lg, n);
    const int64_t hi = std::min<int64_t>(static_cast<int64_t>(c + 1) << lg, n);
    most = std::max<int64_t>(most, rp[hi] - rp[lo]);
  }
  const size_t L = size_t(1) << lg;
  const size_t staged = 12 * static_cast<size_t>(most) + 4 * (L + 1);
  const bool stage = staged <= kClStageMax;
  const size_t slices = S->kind == GK_BICGSTAB ? 2 : 1;  // p (CG); p^ and s^ (BiCGSTAB)
  const size_t smem = 8 * L * slices + (stage ? staged : 0);
  ClKernel k = pick(S->kind, S->pk, rpt, stage);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      set_smem(k, smem) != GK_OK) {
    cudaGetLastError();
    return GK_OK;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = launch_config(smem, nullptr, attr);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return GK_OK;
  }
  S->cl_lg = lg;
  S->cl_rpt = rpt;
  S->cl_stage = stage;
  S->cl_nnz = stage ? static_cast<int>(most) : 0;
  S->cl_smem = smem;
  return GK_OK;
}

int cluster_cg_solve(Solver* S, cudaStream_t s) {
  ClusterArgs a;
  a.rowptr = S->A->rowptr;
  a.col = S->A->col;
  a.val = S->A->val;
  a.b = S->b;
  a.x = S->x;
  a.dinv = S->P ? S->P->dinv : nullptr;
  a.st = S->st;
  a.n = static_cast<int>(S->n);
  a.lg = S->cl_lg;
  a.stage_nnz = S->cl_nnz;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = launch_config(S->cl_smem, s, attr);
  GK_TRY_CUDA(cudaLaunchKernelEx(&cfg, pick(S->kind, S->pk, S->cl_rpt, S->cl_stage), a));
  return GK_OK;
}

}  // namespace gk
