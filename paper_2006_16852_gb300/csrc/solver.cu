// solver.cu -- the Krylov solver operators S_A (Section 3.1): preconditioned
// CG (Listing 1), BiCGSTAB (Listing 3), flexible CG and CGS, generated from
// a matrix, an optional Jacobi preconditioner and combined stopping criteria
// (Section 2.5).  Restarted GMRES lives in gmres.cu.
//
// One iteration is a few fused kernels: each SpMV carries the dot product
// that follows it, and each vector update carries the preconditioner apply
// and the next dot products, so an iteration crosses HBM as few times as
// possible.  All scalars (alpha, beta, omega, norms, the stop flag) live in
// a device-side SolverState and are produced by the last block of each
// fixed-order reduction; the host never reads them inside the loop.  The
// whole solve is one CUDA graph whose iteration body sits in a conditional
// WHILE node that the last kernel of each iteration re-arms.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>

#include "gk_device.cuh"
#include "gk_internal.h"
#include "precond_device.cuh"
#include "solver_state.cuh"

namespace gk {

namespace {

constexpr int kVecThreads = 256;

struct VecArgs {
  int n;
  const double* dinv;
  const double* blocks;
  int bs, nblocks;
  const double* b;
  double *x, *r, *p, *q, *z;        // CG (q doubles as BiCGSTAB's v)
  double *rh, *ph, *s, *sh, *t;     // BiCGSTAB; CGS: s = u, sh = u^, t = v^ then q^
  SolverState* st;
  double* partials;
  unsigned int* counter;
  cudaGraphConditionalHandle cond;
  int use_cond;
};

// Re-arms (or ends) the conditional WHILE loop.  Called by exactly one
// thread per iteration.  A guard ends the loop if it ever runs more than
// max_iters + 2 times.
__device__ __forceinline__ void loop_control(const VecArgs& a) {
  SolverState* st = a.st;
  st->iter_guard += 1;
  if (st->stop == GK_STOP_NONE && st->iter_guard > st->max_iters + 2) {
    st->stop = GK_STOP_MAX_ITERS;
    st->err |= 2;
  }
  if (a.use_cond) cudaGraphSetConditional(a.cond, st->stop == GK_STOP_NONE ? 1u : 0u);
}

__global__ void solver_init_kernel(SolverState* st, double factor, long long max_iters, int rel_to_b,
                                   unsigned long long time_limit_ns) {
  SolverState z;
  memset(&z, 0, sizeof(z));
  z.rho_prev = 1.0;
  z.alpha = 1.0;
  z.omega = 1.0;
  z.factor = factor;
  z.max_iters = max_iters;
  z.rel_to_b = rel_to_b;
  z.time_limit_ns = time_limit_ns;
  *st = z;
}

// Grid-stride loop over rows for the scalar/no preconditioner kernels, or
// warp groups of whole diagonal blocks for block Jacobi.
#define FOR_ROWS(i)                                                                    \
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x)

#define FOR_BLOCK_LANES(L)                                                               \
  const int lane_ = threadIdx.x & 31;                                                    \
  const int bpw_ = 32 / a.bs;                                                            \
  const int nw_ = (gridDim.x * blockDim.x) >> 5;                                          \
  for (int w_ = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w_ * bpw_ < a.nblocks; w_ += nw_) \
    for (BjLane L = bj_lane(w_ * bpw_, lane_, a.bs, a.n, a.nblocks), *once_ = &L; once_; once_ = nullptr)

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

// Scalar-Jacobi / unpreconditioned vector kernels run at 8 blocks of 256
// threads per SM (32 registers) with 128-bit loads of row pairs; the
// block-Jacobi variants keep the default register budget.
template <int PK>
struct VecMinBlocks {
  static constexpr int value = PK == PREC_BLOCK ? 1 : 8;
};

// Grid-stride loop over row pairs (2 i2, 2 i2 + 1).
#define FOR_PAIRS(i2) \
  for (int i2 = blockIdx.x * blockDim.x + threadIdx.x; 2 * i2 < a.n; i2 += gridDim.x * blockDim.x)

__device__ __forceinline__ void reduce_finalize(const VecArgs& a, double s0, double s1, int fin,
                                                double* scratch, bool control) {
  double v[2] = {s0, s1}, out[2];
  if (grid_sum<2>(v, a.partials, a.counter, scratch, out) && threadIdx.x == 0) {
    finalize(fin, out, a.st);
    if (control) loop_control(a);
  }
}

// scratch: >= 3 * blockDim.x doubles.
__device__ __forceinline__ void reduce_finalize3(const VecArgs& a, double s0, double s1, double s2, int fin,
                                                 double* scratch) {
  double v[3] = {s0, s1, s2}, out[3];
  if (grid_sum<3>(v, a.partials, a.counter, scratch, out) && threadIdx.x == 0) finalize(fin, out, a.st);
}

// ---- CG --------------------------------------------------------------------

// z = M^{-1} r, p = z, rho = r.z; criteria at k = 0.
template <int PK, int BS = 0>
__global__ void __launch_bounds__(kVecThreads) cg_start_kernel(VecArgs a) {
  pdl_wait();
  __shared__ double scratch[kRedScratch];
  double rz = 0.0;
  if (PK == PREC_BLOCK) {
    FOR_BLOCK_LANES(L) {
      const double rm = L.active ? a.r[L.row] : 0.0;
      const double zz = bj_apply_lane<BS>(a.blocks, L, a.bs, rm);
      if (L.active) {
        a.p[L.row] = zz;
        rz = fma(rm, zz, rz);
      }
    }
  } else {
    FOR_ROWS(i) {
      const double rv = a.r[i];
      const double zv = (PK == PREC_SCALAR) ? a.dinv[i] * rv : rv;
      a.p[i] = zv;
      rz = fma(rv, zv, rz);
    }
  }
  reduce_finalize(a, rz, 0.0, FIN_CG_START, scratch, false);
}

// x += alpha p; r -= alpha q; z = M^{-1} r; (r.z, r.r); k += 1 and criteria.
// FLEX (flexible CG): also z.q, for beta = -alpha z.q / rho.
template <int PK, int BS, bool FLEX>
__device__ __forceinline__ void cg_update_body(const VecArgs& a, double* scratch) {
  if (a.st->stop) return;
  const double alpha = a.st->alpha;
  double rz = 0.0, rr = 0.0, zq = 0.0;
  if (PK == PREC_BLOCK) {
    FOR_BLOCK_LANES(L) {
      double rn = 0.0;
      if (L.active) {
        a.x[L.row] = fma(alpha, a.p[L.row], a.x[L.row]);
        rn = fma(-alpha, a.q[L.row], a.r[L.row]);
        a.r[L.row] = rn;
      }
      const double zz = bj_apply_lane<BS>(a.blocks, L, a.bs, rn);
      if (L.active) {
        a.z[L.row] = zz;
        rz = fma(rn, zz, rz);
        rr = fma(rn, rn, rr);
        if (FLEX) zq = fma(zz, a.q[L.row], zq);
      }
    }
  } else {
    FOR_PAIRS(i2) {
      const int i = 2 * i2;
      if (i + 1 < a.n) {
        const double2 xv = ld2(a.x + i), pv = ld2(a.p + i), qv = ld2(a.q + i), rv = ld2(a.r + i);
        st2(a.x + i, fma(alpha, pv.x, xv.x), fma(alpha, pv.y, xv.y));
        const double r0 = fma(-alpha, qv.x, rv.x), r1 = fma(-alpha, qv.y, rv.y);
        st2(a.r + i, r0, r1);
        rr = fma(r0, r0, rr);
        rr = fma(r1, r1, rr);
        if (PK == PREC_SCALAR) {
          // z = D^{-1} r is kept for the direction step, which then reads
          // z and p instead of r, D^{-1} and p (the same bytes, one FP64
          // multiply per row fewer)
          const double2 d = ld2(a.dinv + i);
          const double z0 = d.x * r0, z1 = d.y * r1;
          st2(a.z + i, z0, z1);
          rz = fma(r0, z0, rz);
          rz = fma(r1, z1, rz);
          if (FLEX) {
            zq = fma(z0, qv.x, zq);
            zq = fma(z1, qv.y, zq);
          }
        } else if (FLEX) {
          zq = fma(r0, qv.x, zq);
          zq = fma(r1, qv.y, zq);
        }
      } else {
        a.x[i] = fma(alpha, a.p[i], a.x[i]);
        const double rn = fma(-alpha, a.q[i], a.r[i]);
        a.r[i] = rn;
        rr = fma(rn, rn, rr);
        const double zn = PK == PREC_SCALAR ? a.dinv[i] * rn : rn;
        if (PK == PREC_SCALAR) {
          a.z[i] = zn;
          rz = fma(rn, zn, rz);
        }
        if (FLEX) zq = fma(zn, a.q[i], zq);
      }
    }
    if (PK == PREC_NONE) rz = rr;
  }
  if (FLEX) reduce_finalize3(a, rz, rr, zq, FIN_FCG_ITER, scratch);
  else reduce_finalize(a, rz, rr, FIN_CG_ITER, scratch, false);
}

// Prologue of CG's update step, run while the SpMV ahead of it may still be
// running: the lines of x, p and r (and of the preconditioner) that the
// thread reads first, into L2.  q, the SpMV's output, is read only after
// pdl_wait().
template <int PK, int BS>
__device__ __forceinline__ void cg_update_prefetch(const VecArgs& a) {
  const int lane = threadIdx.x & 31;
  if (PK == PREC_BLOCK) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int bpw = 32 / a.bs;
    if (w * bpw < a.nblocks) {
      const BjLane L = bj_lane(w * bpw, lane, a.bs, a.n, a.nblocks);
      if (L.active) {
        if ((lane & 15) == 0) {
          prefetch_l2(a.x + L.row);
          prefetch_l2(a.p + L.row);
          prefetch_l2(a.r + L.row);
        }
        prefetch_l2(a.blocks + static_cast<int64_t>(L.blk) * a.bs * a.bs + static_cast<int64_t>(L.i) * L.m);
      }
    }
  } else {
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i < a.n && (lane & 7) == 0) {
      prefetch_l2(a.x + i);
      prefetch_l2(a.p + i);
      prefetch_l2(a.r + i);
      if (PK == PREC_SCALAR) prefetch_l2(a.dinv + i);
    }
  }
}

template <int PK, int BS = 0>
__global__ void __launch_bounds__(kVecThreads, VecMinBlocks<PK>::value) cg_update_kernel(VecArgs a) {
  cg_update_prefetch<PK, BS>(a);
  pdl_wait();
  pdl_launch_dependents();
  __shared__ double scratch[kRedScratch];
  cg_update_body<PK, BS, false>(a, scratch);
}

template <int PK, int BS = 0>
__global__ void __launch_bounds__(kVecThreads, VecMinBlocks<PK>::value) fcg_update_kernel(VecArgs a) {
  pdl_wait();
  __shared__ double scratch[3 * kVecThreads];  // a three-value block reduction
  cg_update_body<PK, BS, true>(a, scratch);
}

// p = z + beta p; ends the iteration (loop control).
template <int PK>
__global__ void __launch_bounds__(kVecThreads, 8) cg_direction_kernel(VecArgs a) {
  {
    // prologue: p and the diagonal, which the running update step does not
    // write, into L2
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i < a.n && (threadIdx.x & 7) == 0) prefetch_l2(a.p + i);
  }
  pdl_wait();
  pdl_launch_dependents();
  if (blockIdx.x == 0 && threadIdx.x == 0) loop_control(a);
  if (a.st->stop) return;
  const double beta = a.st->beta;
  FOR_PAIRS(i2) {
    const int i = 2 * i2;
    if (i + 1 < a.n) {
      const double2 zv = PK == PREC_NONE ? ld2(a.r + i) : ld2(a.z + i);
      const double2 pv = ld2(a.p + i);
      st2(a.p + i, fma(beta, pv.x, zv.x), fma(beta, pv.y, zv.y));
    } else {
      const double zv = PK == PREC_NONE ? a.r[i] : a.z[i];
      a.p[i] = fma(beta, a.p[i], zv);
    }
  }
}

// ---- BiCGSTAB --------------------------------------------------------------

// r^ = r_0, p = v = 0, rho = r^.r; criteria at k = 0.
__global__ void __launch_bounds__(kVecThreads) bicg_start_kernel(VecArgs a) {
  pdl_wait();
  __shared__ double scratch[kRedScratch];
  double rho = 0.0;
  FOR_ROWS(i) {
    const double rv = a.r[i];
    a.rh[i] = rv;
    a.p[i] = 0.0;
    a.q[i] = 0.0;
    rho = fma(rv, rv, rho);
  }
  reduce_finalize(a, rho, 0.0, FIN_BI_START, scratch, false);
}

// p = r + beta (p - omega v); p^ = M^{-1} p.
template <int PK, int BS = 0>
__global__ void __launch_bounds__(kVecThreads) bicg_dir_kernel(VecArgs a) {
  pdl_wait();
  if (a.st->stop) return;
  const double beta = a.st->beta, omega = a.st->omega;
  if (PK == PREC_BLOCK) {
    FOR_BLOCK_LANES(L) {
      double pn = 0.0;
      if (L.active) {
        pn = fma(beta, fma(-omega, a.q[L.row], a.p[L.row]), a.r[L.row]);
        a.p[L.row] = pn;
      }
      const double zz = bj_apply_lane<BS>(a.blocks, L, a.bs, pn);
      if (L.active) a.ph[L.row] = zz;
    }
  } else {
    FOR_ROWS(i) {
      const double pn = fma(beta, fma(-omega, a.q[i], a.p[i]), a.r[i]);
      a.p[i] = pn;
      if (PK == PREC_SCALAR) a.ph[i] = a.dinv[i] * pn;
    }
  }
}

// s = r - alpha v; s^ = M^{-1} s; ||s||^2 (half-step test).
template <int PK, int BS = 0>
__global__ void __launch_bounds__(kVecThreads) bicg_s_kernel(VecArgs a) {
  pdl_wait();
  __shared__ double scratch[kRedScratch];
  if (a.st->stop) return;
  const double alpha = a.st->alpha;
  double ss = 0.0;
  if (PK == PREC_BLOCK) {
    FOR_BLOCK_LANES(L) {
      double sn = 0.0;
      if (L.active) {
        sn = fma(-alpha, a.q[L.row], a.r[L.row]);
        a.s[L.row] = sn;
        ss = fma(sn, sn, ss);
      }
      const double zz = bj_apply_lane<BS>(a.blocks, L, a.bs, sn);
      if (L.active) a.sh[L.row] = zz;
    }
  } else {
    FOR_ROWS(i) {
      const double sn = fma(-alpha, a.q[i], a.r[i]);
      a.s[i] = sn;
      ss = fma(sn, sn, ss);
      if (PK == PREC_SCALAR) a.sh[i] = a.dinv[i] * sn;
    }
  }
  reduce_finalize(a, ss, 0.0, FIN_BI_S, scratch, false);
}

// x += alpha p^ + omega s^; r = s - omega t; (r^.r, r.r); k += 1, criteria,
// next rho and beta; ends the iteration.  After a half-step exit only
// x += alpha p^ and r = s.
__global__ void __launch_bounds__(kVecThreads) bicg_update_kernel(VecArgs a) {
  pdl_wait();
  __shared__ double scratch[kRedScratch];
  if (a.st->stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) loop_control(a);
    return;
  }
  const double alpha = a.st->alpha, omega = a.st->omega;
  const bool half = a.st->half != 0;
  double rho = 0.0, rr = 0.0;
  FOR_ROWS(i) {
    if (half) {
      a.x[i] = fma(alpha, a.ph[i], a.x[i]);
      a.r[i] = a.s[i];
    } else {
      a.x[i] = fma(omega, a.sh[i], fma(alpha, a.ph[i], a.x[i]));
      const double rn = fma(-omega, a.t[i], a.s[i]);
      a.r[i] = rn;
      rho = fma(a.rh[i], rn, rho);
      rr = fma(rn, rn, rr);
    }
  }
  reduce_finalize(a, rho, rr, FIN_BI_ITER, scratch, true);
}

// ---- CGS ---------------------------------------------------------------------

// r^ = r_0, p = q = 0, rho = r^.r; criteria at k = 0.
__global__ void __launch_bounds__(kVecThreads) cgs_start_kernel(VecArgs a) {
  pdl_wait();
  __shared__ double scratch[kRedScratch];
  double rho = 0.0;
  FOR_ROWS(i) {
    const double rv = a.r[i];
    a.rh[i] = rv;
    a.p[i] = 0.0;
    a.q[i] = 0.0;
    rho = fma(rv, rv, rho);
  }
  reduce_finalize(a, rho, 0.0, FIN_CGS_START, scratch, false);
}

// u = r (first step) or r + beta q; p = u (first step) or u + beta (q + beta p);
// p^ = M^{-1} p.
template <int PK, int BS = 0>
__global__ void __launch_bounds__(kVecThreads) cgs_dir_kernel(VecArgs a) {
  pdl_wait();
  if (a.st->stop) return;
  const bool first = a.st->iter == 0;
  const double beta = a.st->beta;
  if (PK == PREC_BLOCK) {
    FOR_BLOCK_LANES(L) {
      double pn = 0.0;
      if (L.active) {
        const double rv = a.r[L.row];
        const double un = first ? rv : fma(beta, a.q[L.row], rv);
        pn = first ? un : fma(beta, fma(beta, a.p[L.row], a.q[L.row]), un);
        a.s[L.row] = un;
        a.p[L.row] = pn;
      }
      const double zz = bj_apply_lane<BS>(a.blocks, L, a.bs, pn);
      if (L.active) a.ph[L.row] = zz;
    }
  } else {
    FOR_ROWS(i) {
      const double rv = a.r[i];
      const double un = first ? rv : fma(beta, a.q[i], rv);
      const double pn = first ? un : fma(beta, fma(beta, a.p[i], a.q[i]), un);
      a.s[i] = un;
      a.p[i] = pn;
      if (PK == PREC_SCALAR) a.ph[i] = a.dinv[i] * pn;
    }
  }
}

// q = u - alpha v^; u^ = M^{-1} (u + q); x += alpha u^.
template <int PK, int BS = 0>
__global__ void __launch_bounds__(kVecThreads) cgs_q_kernel(VecArgs a) {
  pdl_wait();
  if (a.st->stop) return;
  const double alpha = a.st->alpha;
  if (PK == PREC_BLOCK) {
    FOR_BLOCK_LANES(L) {
      double w = 0.0;
      if (L.active) {
        const double qn = fma(-alpha, a.t[L.row], a.s[L.row]);
        a.q[L.row] = qn;
        w = a.s[L.row] + qn;
      }
      const double uh = bj_apply_lane<BS>(a.blocks, L, a.bs, w);
      if (L.active) {
        a.sh[L.row] = uh;
        a.x[L.row] = fma(alpha, uh, a.x[L.row]);
      }
    }
  } else {
    FOR_ROWS(i) {
      const double qn = fma(-alpha, a.t[i], a.s[i]);
      a.q[i] = qn;
      const double w = a.s[i] + qn;
      const double uh = PK == PREC_SCALAR ? a.dinv[i] * w : w;
      a.sh[i] = uh;
      a.x[i] = fma(alpha, uh, a.x[i]);
    }
  }
}

// r -= alpha q^; (r^.r, r.r); k += 1, criteria, next rho and beta; ends the
// iteration.
__global__ void __launch_bounds__(kVecThreads) cgs_update_kernel(VecArgs a) {
  pdl_wait();
  __shared__ double scratch[kRedScratch];
  if (a.st->stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) loop_control(a);
    return;
  }
  const double alpha = a.st->alpha;
  double rho = 0.0, rr = 0.0;
  FOR_ROWS(i) {
    const double rn = fma(-alpha, a.t[i], a.r[i]);
    a.r[i] = rn;
    rho = fma(a.rh[i], rn, rho);
    rr = fma(rn, rn, rr);
  }
  reduce_finalize(a, rho, rr, FIN_CGS_ITER, scratch, true);
}

#undef FOR_ROWS
#undef FOR_PAIRS
#undef FOR_BLOCK_LANES

}  // namespace



namespace {

void solver_release(Solver* S) {
  if (!S) return;
  if (S->refs.fetch_sub(1) != 1) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  if (S->exec) cudaGraphExecDestroy(S->exec);
  if (S->graph) cudaGraphDestroy(S->graph);
  if (S->cs) cudaStreamDestroy(S->cs);
  for (double* v : {S->b, S->x, S->r, S->p, S->q, S->z, S->rh, S->ph, S->s, S->sh, S->t}) dfree(v);
  dfree(S->st);
  dfree(S->partials);
  dfree(S->counter);
  dfree(S->gr_part);
  dfree(S->gr_sync);
  if (S->h_st) cudaFreeHost(S->h_st);
  ir_release(S->ir);
  gmres_release(S->gm);
  precond_release(S->P);
  matrix_release(S->A);
  if (prev >= 0) cudaSetDevice(prev);
  delete S;
}

struct SolverDeleter {
  void operator()(Solver* s) const { solver_release(s); }
};

VecArgs vec_args(const Solver& S, int use_cond) {
  VecArgs a;
  a.n = static_cast<int>(S.n);
  a.dinv = S.P ? S.P->dinv : nullptr;
  a.blocks = S.P ? S.P->blocks : nullptr;
  a.bs = S.P ? S.P->bs : 1;
  a.nblocks = S.P ? static_cast<int>(S.P->nblocks) : 0;
  a.b = S.b;
  a.x = S.x;
  a.r = S.r;
  a.p = S.p;
  a.q = S.q;
  a.z = S.z;
  a.rh = S.rh;
  a.s = S.s;
  // without a preconditioner p^ = p and s^ = s
  a.ph = S.ph ? S.ph : S.p;
  a.sh = S.sh ? S.sh : S.s;
  a.t = S.t;
  a.st = S.st;
  a.partials = S.partials;
  a.counter = S.counter;
  a.cond = S.cond;
  a.use_cond = use_cond;
  return a;
}

int vec_grid(const Solver& S) {
  const int64_t units = (S.pk == PREC_BLOCK)
                            ? ((S.P->nblocks + (32 / S.P->bs) - 1) / (32 / S.P->bs)) * 32
                            : S.n;
  const int64_t g = (units + kVecThreads - 1) / kVecThreads;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, 8 * sm_count())));
}

Epi spmv_epi(const Solver& S, int mode, const double* u, double* y, int fin, int skip_mode) {
  Epi e;
  e.mode = mode;
  e.fin = fin;
  e.u = u;
  e.y = y;
  e.st = S.st;
  e.skip_mode = skip_mode;
  e.partials = S.partials;
  e.counter = S.counter;
  e.err = &S.st->err;
  return e;
}

// As LAUNCH_PK for kernels that apply block Jacobi: the block size becomes
// a template argument where a vectorised apply is compiled for it.
#define LAUNCH_PK_BS(kern, grid, s, args)                                                       \
  do {                                                                                          \
    if (S.pk == PREC_BLOCK) {                                                                   \
      switch (S.P->bs) {                                                                        \
        case 4: launch_pdl(kern<PREC_BLOCK, 4>, grid, kVecThreads, 0, s, args); break;                 \
        case 8: launch_pdl(kern<PREC_BLOCK, 8>, grid, kVecThreads, 0, s, args); break;                 \
        case 16: launch_pdl(kern<PREC_BLOCK, 16>, grid, kVecThreads, 0, s, args); break;               \
        case 32: launch_pdl(kern<PREC_BLOCK, 32>, grid, kVecThreads, 0, s, args); break;               \
        default: launch_pdl(kern<PREC_BLOCK, 0>, grid, kVecThreads, 0, s, args); break;                \
      }                                                                                         \
    } else if (S.pk == PREC_SCALAR) {                                                           \
      launch_pdl(kern<PREC_SCALAR, 0>, grid, kVecThreads, 0, s, args);                                  \
    } else {                                                                                    \
      launch_pdl(kern<PREC_NONE, 0>, grid, kVecThreads, 0, s, args);                                    \
    }                                                                                           \
    GK_TRY_CUDA(cudaGetLastError());                                                            \
  } while (0)

#define LAUNCH_PK(kern, grid, s, args)                                                          \
  do {                                                                                          \
    if (S.pk == PREC_BLOCK) launch_pdl(kern<PREC_BLOCK>, grid, kVecThreads, 0, s, args);               \
    else if (S.pk == PREC_SCALAR) launch_pdl(kern<PREC_SCALAR>, grid, kVecThreads, 0, s, args);        \
    else launch_pdl(kern<PREC_NONE>, grid, kVecThreads, 0, s, args);                                    \
    GK_TRY_CUDA(cudaGetLastError());                                                            \
  } while (0)

int enqueue_setup(const Solver& S, cudaStream_t s, const VecArgs& a) {
  const gk_criteria& c = S.crit;
  unsigned long long tl = c.time_limit_s > 0 ? static_cast<unsigned long long>(c.time_limit_s * 1e9) : 0ull;
  solver_init_kernel<<<1, 1, 0, s>>>(S.st, c.reduction_factor, static_cast<long long>(c.max_iters),
                                     c.rel_to_b, tl);
  GK_TRY_CUDA(cudaGetLastError());
  GK_TRY(spmv_launch(*S.A, S.x, spmv_epi(S, EPI_RESID, S.b, S.r, FIN_SETUP_RESID, 0), s));
  if (S.kind == GK_CG || S.kind == GK_FCG) {
    LAUNCH_PK_BS(cg_start_kernel, S.grid_vec, s, a);
  } else if (S.kind == GK_CGS) {
    launch_pdl(cgs_start_kernel, S.grid_vec, kVecThreads, 0, s, a);
    GK_TRY_CUDA(cudaGetLastError());
  } else {
    launch_pdl(bicg_start_kernel, S.grid_vec, kVecThreads, 0, s, a);
    GK_TRY_CUDA(cudaGetLastError());
  }
  return GK_OK;
}

int enqueue_iteration(const Solver& S, cudaStream_t s, const VecArgs& a) {
  if (S.kind == GK_CG || S.kind == GK_FCG) {
    GK_TRY(spmv_launch(*S.A, S.p, spmv_epi(S, EPI_DOT, S.p, S.q, FIN_CG_SIGMA, 1), s));
    if (S.kind == GK_CG) LAUNCH_PK_BS(cg_update_kernel, S.grid_vec, s, a);
    else LAUNCH_PK_BS(fcg_update_kernel, S.grid_vec, s, a);
    LAUNCH_PK(cg_direction_kernel, S.grid_vec, s, a);
  } else if (S.kind == GK_CGS) {
    const double* ph = (S.pk == PREC_NONE) ? S.p : S.ph;
    LAUNCH_PK_BS(cgs_dir_kernel, S.grid_vec, s, a);
    GK_TRY(spmv_launch(*S.A, ph, spmv_epi(S, EPI_DOT, S.rh, S.t, FIN_CGS_ALPHA, 1), s));
    LAUNCH_PK_BS(cgs_q_kernel, S.grid_vec, s, a);
    GK_TRY(spmv_launch(*S.A, S.sh, spmv_epi(S, EPI_COPY, nullptr, S.t, FIN_NONE, 1), s));
    launch_pdl(cgs_update_kernel, S.grid_vec, kVecThreads, 0, s, a);
    GK_TRY_CUDA(cudaGetLastError());
  } else {
    const double* ph = (S.pk == PREC_NONE) ? S.p : S.ph;
    const double* sh = (S.pk == PREC_NONE) ? S.s : S.sh;
    LAUNCH_PK_BS(bicg_dir_kernel, S.grid_vec, s, a);
    GK_TRY(spmv_launch(*S.A, ph, spmv_epi(S, EPI_DOT, S.rh, S.q, FIN_BI_RHV, 1), s));
    LAUNCH_PK_BS(bicg_s_kernel, S.grid_vec, s, a);
    GK_TRY(spmv_launch(*S.A, sh, spmv_epi(S, EPI_DOT2, S.s, S.t, FIN_BI_OMEGA, 2), s));
    launch_pdl(bicg_update_kernel, S.grid_vec, kVecThreads, 0, s, a);
    GK_TRY_CUDA(cudaGetLastError());
  }
  return GK_OK;
}

int enqueue_final(const Solver& S, cudaStream_t s) {
  double* scratch = (S.kind == GK_CG || S.kind == GK_FCG) ? S.q : S.t;
  return spmv_launch(*S.A, S.x, spmv_epi(S, EPI_RESID, S.b, scratch, FIN_TRUE_RESID, 0), s);
}

#undef LAUNCH_PK

// The whole solve as one graph: setup -> WHILE(cond) { iteration } -> final.
int build_graph(Solver& S) {
  if (!S.cs) GK_TRY_CUDA(cudaStreamCreateWithFlags(&S.cs, cudaStreamNonBlocking));
  GK_TRY_CUDA(cudaGraphCreate(&S.graph, 0));
  GK_TRY_CUDA(cudaGraphConditionalHandleCreate(&S.cond, S.graph, 1, cudaGraphCondAssignDefault));
  VecArgs a = vec_args(S, 1);
  GK_TRY_CUDA(cudaStreamBeginCaptureToGraph(S.cs, S.graph, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_setup(S, S.cs, a);
  cudaGraph_t body = nullptr;
  if (rc == GK_OK) {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(S.cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = S.cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, S.graph, deps, nullptr, ndeps, &np);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(S.cs, &cnode, nullptr, 1,
                                                                   cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) rc = cuda_error(e, "adding the conditional loop node");
    else body = np.conditional.phGraph_out[0];
  }
  if (rc == GK_OK) rc = enqueue_final(S, S.cs);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(S.cs, &captured);
  if (rc != GK_OK) return rc;
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  GK_TRY_CUDA(cudaStreamBeginCaptureToGraph(S.cs, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
  // CG and FCG: kGraphUnroll iterations per pass of the loop body, so that
  // three iterations in four skip the loop's turn-around (about 7 us on a
  // GB300, with no programmatic edge across it).  The kernels of an
  // iteration after the stop do nothing.
  const int passes = (S.kind == GK_CG || S.kind == GK_FCG) ? kGraphUnroll : 1;
  rc = enqueue_iteration(S, S.cs, a);
  for (int u = 1; u < passes && rc == GK_OK; ++u) rc = enqueue_iteration(S, S.cs, a);
  e = cudaStreamEndCapture(S.cs, &captured);
  if (rc != GK_OK) return rc;
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture (body)");
  GK_TRY_CUDA(cudaGraphInstantiate(&S.exec, S.graph, 0));
  return GK_OK;
}

int alloc_vec(double** v, int64_t n, int64_t* bytes) {
  return dalloc_n(v, static_cast<size_t>(std::max<int64_t>(n, 1)), bytes);
}

}  // namespace

}  // namespace gk

using namespace gk;

extern "C" int gk_solver_generate(gk_matrix hA, gk_precond hP, int32_t kind, const gk_criteria* crit,
                                  gk_solver* out) {
  if (!out) return set_error(GK_ERR_ARG, "gk_solver_generate: out is NULL");
  *out = nullptr;
  Matrix* A = as_matrix(hA);
  Precond* P = as_precond(hP);
  if (!A || !crit) return set_error(GK_ERR_ARG, "gk_solver_generate: NULL matrix or criteria");
  if (kind != GK_CG && kind != GK_BICGSTAB && kind != GK_IR_CG && kind != GK_FCG && kind != GK_CGS &&
      kind != GK_GMRES)
    return set_error(GK_ERR_ARG, "unknown solver kind %d", kind);
  if (A->n_rows != A->n_cols) return set_error(GK_ERR_DIM, "gk_solver_generate: matrix is not square");
  if (P && P->n != A->n_rows) return set_error(GK_ERR_DIM, "preconditioner size %lld != %lld",
                                               (long long)P->n, (long long)A->n_rows);
  if (crit->max_iters < 0 || !(crit->reduction_factor >= 0.0))
    return set_error(GK_ERR_ARG, "gk_solver_generate: bad criteria");
  int prev = current_device();
  if (prev != A->device) cudaSetDevice(A->device);
  std::unique_ptr<Solver, SolverDeleter> hold(new Solver);
  Solver* S = hold.get();
  S->device = A->device;
  A->refs.fetch_add(1);
  S->A = A;
  if (P) {
    P->refs.fetch_add(1);
    S->P = P;
    S->pk = (P->bs == 1) ? PREC_SCALAR : PREC_BLOCK;
  }
  S->kind = kind;
  S->crit = *crit;
  S->n = A->n_rows;
  int64_t* by = &S->device_bytes;
  int rc = GK_OK;
  do {
    if ((rc = alloc_vec(&S->b, S->n, by)) || (rc = alloc_vec(&S->x, S->n, by)) ||
        (rc = alloc_vec(&S->r, S->n, by)) || (rc = alloc_vec(&S->p, S->n, by)) ||
        (rc = alloc_vec(&S->q, S->n, by)))
      break;
    if ((kind == GK_CG || kind == GK_FCG) && S->pk != PREC_NONE && (rc = alloc_vec(&S->z, S->n, by))) break;
    if (kind == GK_CGS) {
      if ((rc = alloc_vec(&S->rh, S->n, by)) || (rc = alloc_vec(&S->s, S->n, by)) ||
          (rc = alloc_vec(&S->t, S->n, by)) || (rc = alloc_vec(&S->sh, S->n, by)))
        break;
      if (S->pk != PREC_NONE && (rc = alloc_vec(&S->ph, S->n, by))) break;
    }
    if (kind == GK_BICGSTAB) {
      if ((rc = alloc_vec(&S->rh, S->n, by)) || (rc = alloc_vec(&S->s, S->n, by)) ||
          (rc = alloc_vec(&S->t, S->n, by)))
        break;
      if (S->pk != PREC_NONE && ((rc = alloc_vec(&S->ph, S->n, by)) || (rc = alloc_vec(&S->sh, S->n, by))))
        break;
    }
    if ((rc = dalloc_n(&S->st, 1, by))) break;
    S->grid_vec = vec_grid(*S);
    const int pg = std::max(S->grid_vec, spmv_max_grid(*A));
    if ((rc = dalloc_n(&S->partials, static_cast<size_t>(3 * (pg + kFixupMaxGrid)), by)) ||
        (rc = dalloc_n(&S->counter, 1, by)))
      break;
    cudaError_t e = cudaMemset(S->counter, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(S->st, 0, sizeof(SolverState));
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_st, sizeof(SolverState));
    if (e != cudaSuccess) {
      rc = cuda_error(e, "solver allocation");
      break;
    }
    if (kind == GK_IR_CG && (rc = ir_generate(S))) break;
    if (kind == GK_GMRES && (rc = gmres_generate(S))) break;
    if ((kind == GK_CG || kind == GK_BICGSTAB) && (rc = cluster_cg_plan(S))) break;
    if (kind == GK_CG && S->cl_lg < 0 && (rc = grid_cg_plan(S))) break;
  } while (false);
  if (prev != A->device) cudaSetDevice(prev);
  if (rc != GK_OK) return rc;
  *out = reinterpret_cast<gk_solver>(hold.release());
  return GK_OK;
}

extern "C" int gk_solve(gk_solver h, const void* b, void* x, gk_status* status, void* stream) {
  Solver* S = reinterpret_cast<Solver*>(h);
  if (!S) return set_error(GK_ERR_ARG, "gk_solve: NULL solver");
  if (S->n > 0 && (!b || !x)) return set_error(GK_ERR_ARG, "gk_solve: NULL vector");
  int prev = current_device();
  if (prev != S->device) cudaSetDevice(S->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = GK_OK;
  int form = S->crit.check_every > 0 ? GK_FORM_HOST : GK_FORM_GRAPH;
  int64_t launched = -1;  // iterations launched, where more than were done
  do {
    if (S->n == 0) {
      if (status) {
        memset(status, 0, sizeof(*status));
        status->stop_reason = GK_STOP_CONVERGED;
      }
      break;
    }
    const size_t vb = sizeof(double) * static_cast<size_t>(S->n);
    cudaError_t e = cudaMemcpyAsync(S->b, b, vb, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->x, x, vb, cudaMemcpyDefault, s);
    if (e != cudaSuccess) {
      rc = cuda_error(e, "gk_solve: copying b and x");
      break;
    }
    if (S->kind == GK_IR_CG) {
      if ((rc = ir_solve(S, s))) break;
    } else if (S->kind == GK_GMRES) {
      if ((rc = gmres_solve(S, s))) break;
    } else if ((S->kind == GK_CG || S->kind == GK_BICGSTAB) && S->cl_lg >= 0 && S->crit.check_every == 0 &&
               !(S->crit.time_limit_s > 0)) {
      // small system: the whole iteration in one thread-block cluster
      const gk_criteria& c = S->crit;
      solver_init_kernel<<<1, 1, 0, s>>>(S->st, c.reduction_factor, static_cast<long long>(c.max_iters), c.rel_to_b,
                                         0ull);
      e = cudaGetLastError();
      if (e != cudaSuccess) {
        rc = cuda_error(e, "gk_solve: state init");
        break;
      }
      if ((rc = cluster_cg_solve(S, s))) break;
      if ((rc = enqueue_final(*S, s))) break;
      form = GK_FORM_CLUSTER;
    } else if (S->kind == GK_CG && S->gr_grid > 0 && S->crit.check_every == 0 && !(S->crit.time_limit_s > 0)) {
      // mid-size system: the whole iteration in one cooperative launch
      const gk_criteria& c = S->crit;
      solver_init_kernel<<<1, 1, 0, s>>>(S->st, c.reduction_factor, static_cast<long long>(c.max_iters), c.rel_to_b,
                                         0ull);
      e = cudaGetLastError();
      if (e != cudaSuccess) {
        rc = cuda_error(e, "gk_solve: state init");
        break;
      }
      if ((rc = grid_cg_solve(S, s))) break;
      if ((rc = enqueue_final(*S, s))) break;
      form = GK_FORM_GRID;
    } else if (S->crit.check_every > 0) {
      // host-driven loop: groups of check_every iterations, then a status read
      VecArgs a = vec_args(*S, 0);
      if ((rc = enqueue_setup(*S, s, a))) break;
      const auto t0 = std::chrono::steady_clock::now();
      int64_t done = 0;
      for (;;) {
        for (int i = 0; i < S->crit.check_every && rc == GK_OK; ++i) rc = enqueue_iteration(*S, s, a);
        if (rc) break;
        done += S->crit.check_every;
        e = cudaMemcpyAsync(S->h_st, S->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
          rc = cuda_error(e, "gk_solve: status read");
          break;
        }
        if (S->h_st->stop != GK_STOP_NONE) break;
        if (S->crit.time_limit_s > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >
                S->crit.time_limit_s) {
          int tstop = GK_STOP_TIME;
          cudaMemcpyAsync(&S->st->stop, &tstop, sizeof(int), cudaMemcpyHostToDevice, s);
          break;
        }
        if (done > S->crit.max_iters + 2) break;
      }
      if (rc) break;
      launched = done;
      if ((rc = enqueue_final(*S, s))) break;
    } else {
      if (!S->exec && (rc = build_graph(*S))) break;
      e = cudaGraphLaunch(S->exec, s);
      if (e != cudaSuccess) {
        rc = cuda_error(e, "gk_solve: cudaGraphLaunch");
        break;
      }
    }
    e = cudaMemcpyAsync(x, S->x, vb, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->h_st, S->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = cuda_error(e, "gk_solve: reading the result");
      break;
    }
    const SolverState& H = *S->h_st;
    if (status) {
      status->iters = H.iter;
      status->spmvs = H.spmvs;
      status->ref_norm = H.ref;
      status->rel_res = H.rnorm / H.ref;
      status->rel_res_true = sqrt(H.true_rr) / H.ref;
      status->stop_reason = H.stop;
      status->device_error = H.err;
      status->outer_iters = H.outer;
      status->form = form;
      int64_t idle = 0;
      if (S->kind == GK_IR_CG) {
        idle = S->ir_idle;
      } else if (launched >= 0) {
        idle = launched - H.iter;
      } else if (form == GK_FORM_GRAPH && (S->kind == GK_CG || S->kind == GK_FCG)) {
        idle = kGraphUnroll * std::max<int64_t>(1, (H.iter + kGraphUnroll - 1) / kGraphUnroll) - H.iter;
      }
      status->idle_iters = static_cast<int32_t>(std::max<int64_t>(idle, 0));
    }
    if (H.err & kErrTimeout) rc = set_error(GK_ERR_TIMEOUT, "gk_solve: a device-side wait timed out");
  } while (false);
  if (prev != S->device) cudaSetDevice(prev);
  return rc;
}

extern "C" int gk_solver_destroy(gk_solver h) {
  if (!h) return set_error(GK_ERR_ARG, "gk_solver_destroy: NULL handle");
  solver_release(reinterpret_cast<Solver*>(h));
  return GK_OK;
}
