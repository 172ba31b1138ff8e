// solver_state.cuh -- device-side scalar steps of the Krylov solvers, run by
// one thread of the last block of each fused reduction.  The order of the
// criteria and breakdown tests follows the CPU reference of Section 3.1:
// criteria of Section 2.5 (residual reduction, then iteration count, then
// time), NaN first.
#pragma once

#include <cmath>

#include "gk_internal.h"

namespace gk {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int check_stop(const SolverState* st, double rnorm, long long k) {
  if (!isfinite(rnorm)) return GK_STOP_NAN;
  if (rnorm <= st->tol) return GK_STOP_CONVERGED;
  if (k >= st->max_iters) return GK_STOP_MAX_ITERS;
  if (st->time_limit_ns && global_ns() - st->t_start_ns > st->time_limit_ns) return GK_STOP_TIME;
  return GK_STOP_NONE;
}

// BiCGSTAB: a fresh rho = r^.r either fails (NaN, zero) or yields the next beta.
__device__ __forceinline__ void bicg_new_rho(SolverState* st, double rho) {
  if (!isfinite(rho)) {
    st->stop = GK_STOP_NAN;
  } else if (rho == 0.0) {
    st->stop = GK_STOP_BREAKDOWN;
  } else {
    st->beta = (rho / st->rho_prev) * (st->alpha / st->omega);
    st->rho = rho;
  }
}

// s: the sums of the reduction (two, or three for FIN_FCG_ITER).
__device__ __forceinline__ void finalize(int fin, const double* s, SolverState* st) {
  st->red[0] = s[0];
  st->red[1] = s[1];
  switch (fin) {
    case FIN_SETUP_RESID: {
      st->spmvs += 1;
      st->t_start_ns = global_ns();
      double rn = sqrt(s[0]);
      double bn = sqrt(s[1]);
      st->rnorm = rn;
      st->rnorm0 = rn;
      st->bnorm = bn;
      double ref = st->rel_to_b ? bn : rn;
      if (ref == 0.0) ref = 1.0;
      st->ref = ref;
      st->tol = st->factor * ref;
      break;
    }
    case FIN_CG_START:
      st->rho = s[0];
      st->stop = check_stop(st, st->rnorm, 0);
      break;
    case FIN_CG_SIGMA: {
      st->spmvs += 1;
      double sigma = s[0];
      if (!isfinite(sigma)) st->stop = GK_STOP_NAN;
      else if (sigma <= 0.0) st->stop = GK_STOP_BREAKDOWN;
      else st->alpha = st->rho / sigma;
      break;
    }
    case FIN_CG_ITER: {
      st->iter += 1;
      st->rnorm = sqrt(s[1]);
      st->stop = check_stop(st, st->rnorm, st->iter);
      st->beta = s[0] / st->rho;
      st->rho = s[0];
      break;
    }
    case FIN_BI_START:
      st->stop = check_stop(st, st->rnorm, 0);
      if (st->stop == GK_STOP_NONE) bicg_new_rho(st, s[0]);
      break;
    case FIN_BI_RHV: {
      st->spmvs += 1;
      double rhv = s[0];
      if (!isfinite(rhv)) st->stop = GK_STOP_NAN;
      else if (rhv == 0.0) st->stop = GK_STOP_BREAKDOWN;
      else st->alpha = st->rho / rhv;
      break;
    }
    case FIN_BI_S: {
      double sn = sqrt(s[0]);
      st->snorm = sn;
      if (isfinite(sn) && sn <= st->tol) st->half = 1;
      break;
    }
    case FIN_BI_OMEGA: {
      st->spmvs += 1;
      double ts = s[0], tt = s[1];
      if (!isfinite(tt) || !isfinite(ts)) st->stop = GK_STOP_NAN;
      else if (tt == 0.0) st->stop = GK_STOP_BREAKDOWN;
      else st->omega = ts / tt;
      break;
    }
    case FIN_BI_ITER: {
      st->iter += 1;
      if (st->half) {
        st->rnorm = st->snorm;
        st->stop = GK_STOP_CONVERGED;
        break;
      }
      st->rho_prev = st->rho;
      st->rnorm = sqrt(s[1]);
      int stop = check_stop(st, st->rnorm, st->iter);
      if (stop == GK_STOP_NONE && st->omega == 0.0) stop = GK_STOP_BREAKDOWN;
      st->stop = stop;
      if (stop == GK_STOP_NONE) bicg_new_rho(st, s[0]);
      break;
    }
    case FIN_FCG_ITER: {
      // beta = z_{k+1}.(r_{k+1} - r_k) / rho_k with r_{k+1} - r_k = -alpha q
      st->iter += 1;
      st->rnorm = sqrt(s[1]);
      st->stop = check_stop(st, st->rnorm, st->iter);
      st->beta = (-st->alpha * s[2]) / st->rho;
      st->rho = s[0];
      break;
    }
    case FIN_CGS_START:
      st->stop = check_stop(st, st->rnorm, 0);
      if (st->stop == GK_STOP_NONE) {
        if (!isfinite(s[0])) st->stop = GK_STOP_NAN;
        else if (s[0] == 0.0) st->stop = GK_STOP_BREAKDOWN;
        else st->rho = s[0];
      }
      break;
    case FIN_CGS_ALPHA: {
      st->spmvs += 1;
      const double rv = s[0];
      if (!isfinite(rv)) st->stop = GK_STOP_NAN;
      else if (rv == 0.0) st->stop = GK_STOP_BREAKDOWN;
      else st->alpha = st->rho / rv;
      break;
    }
    case FIN_CGS_ITER: {
      st->spmvs += 1;
      st->iter += 1;
      st->rnorm = sqrt(s[1]);
      st->stop = check_stop(st, st->rnorm, st->iter);
      if (st->stop == GK_STOP_NONE) {
        const double rho = s[0];
        if (!isfinite(rho)) {
          st->stop = GK_STOP_NAN;
        } else if (rho == 0.0) {
          st->stop = GK_STOP_BREAKDOWN;
        } else {
          st->beta = rho / st->rho;
          st->rho_prev = st->rho;
          st->rho = rho;
        }
      }
      break;
    }
    case FIN_GMRES_RESID:
      st->spmvs += 1;
      st->rnorm = sqrt(s[0]);
      st->true_rr = s[0];
      break;
    case FIN_TRUE_RESID:
      st->spmvs += 1;
      st->true_rr = s[0];
      break;
    case FIN_IR_RESID: {
      // iterative refinement: r = b - A x in FP64 after every inner solve
      st->spmvs += 1;
      const double rn = sqrt(s[0]);
      if (st->outer == 0) {
        st->t_start_ns = global_ns();
        st->bnorm = sqrt(s[1]);
        st->rnorm0 = rn;
        double ref = st->rel_to_b ? st->bnorm : rn;
        if (ref == 0.0) ref = 1.0;
        st->ref = ref;
        st->tol = st->factor * ref;
      }
      st->rnorm = rn;
      st->true_rr = s[0];
      st->stop = check_stop(st, rn, st->iter);
      break;
    }
    default:
      break;
  }
}

}  // namespace gk
