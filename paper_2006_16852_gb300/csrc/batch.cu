// batch.cu -- many small independent systems solved in one graph launch.
//
// The stopping status of Section 2.5 is kept per right-hand side; here it is
// kept per independent system.  One thread block owns one system at a time:
// its vectors live in shared memory, its matrix is read through the L1/L2
// caches (it stays there across the system's iterations), dot
// products are fixed-order block reductions, and the block takes its next
// system from an atomic counter over the systems sorted by decreasing size,
// so the longest solves start first.  CG and BiCGSTAB follow the steps of
// the large-system solvers (Section 3.1).
//
// Systems are grouped in size classes (rows in (16*2^c, 32*2^c]); each class
// is one persistent kernel whose shared memory is sized for the class's
// largest system and whose block size (32 = one warp per system, 64, 128 or
// 256) is picked per class by gk_batch_autotune.  The class kernels are
// independent branches of one CUDA graph, so the hardware runs them side by
// side and a class's tail overlaps the others' work.
//
// Storage: each system is kept as its own column-major ELL block (width =
// its longest row, entries of a row in CSR order, padding entries value 0
// and the row's own column) with 16-bit local column indices, so a warp's
// k-th entries are one contiguous load and an entry costs 10 bytes in FP64
// (6 in FP32) instead of CSR's 12.
#include <algorithm>
#include <type_traits>
#include <climits>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "gk_device.cuh"
#include "gk_internal.h"

namespace gk {

constexpr int kBatchMaxRows = 4096;
constexpr int kBatchClasses = GK_BATCH_CLASSES;
constexpr int kBatchCandidates[4] = {32, 64, 128, 256};

namespace {

struct BatchClass {
  int k0 = 0;     // first position in the size order
  int count = 0;  // systems in the class
  int nmax = 0;   // rows of its largest system
};

struct BatchArgs {
  const int32_t* sys_ptr;
  const int32_t* order;
  const int32_t* ell_off;   // per system: first ELL entry
  const int32_t* ell_w;     // per system: ELL width
  const uint16_t* ell_col;  // local column indices
  const void* ell_val;      // values in the solve precision
  const float* ell_val32;   // FP32 copy of FP64 values (refinement inner solves)
  const double* b;
  double* x;
  gk_batch_status* st;
  unsigned int* next;  // this class's counter
  long long max_iters;
  double factor;
  double inner_red;          // refinement: inner reduction target
  long long inner_max;       // refinement: inner iteration limit
  int rel_to_b;
  int k0, count, nmax;
};

constexpr int kBatchMaxOuter = 200;  // refinement steps per system
constexpr int kBicgRestarts = 4;     // FP32 BiCGSTAB restarts after a breakdown, per system

// ---------------------------------------------------------------------------
// Reductions.  The totals of K per-thread values are formed in a fixed order
// (block_sum: warp 0 over the block; one warp: an xor butterfly, which leaves
// the same bits in every lane), then f(totals, out) derives the step's
// scalars -- divisions, square roots, breakdown tests -- on the thread(s)
// holding the totals, and out[] reaches every thread through shared memory.
// ---------------------------------------------------------------------------
template <bool WARP, int K, int S, typename T, typename F>
__device__ __forceinline__ void reduce(T (&v)[K], T* red, double* sc, double (&out)[S], F f) {
  if (WARP) {
    warp_sum<K, T>(v);
    f(v, out);
  } else {
    block_sum<K, T>(v, red);
    if (threadIdx.x == 0) {
      f(v, out);
#pragma unroll
      for (int s = 0; s < S; ++s) sc[s] = out[s];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) out[s] = sc[s];
  }
}

// One system's matrix: n rows, ELL width w, entry (k, i) at k * n + i.
template <typename T>
struct SysMat {
  const T* __restrict__ val;
  const uint16_t* __restrict__ col;
  int n, w;
};

template <typename T>
__device__ __forceinline__ SysMat<T> sys_mat(const BatchArgs& a, int sys, int n) {
  const int off = a.ell_off[sys];
  return SysMat<T>{static_cast<const T*>(a.ell_val) + off, a.ell_col + off, n, a.ell_w[sys]};
}

// Q = A P (P in shared memory).  Row sums in CSR order; a padding entry
// adds 0 * P[i].
template <typename T>
__device__ __forceinline__ void sys_spmv(const SysMat<T>& m, const T* P, T* Q) {
  for (int i = threadIdx.x; i < m.n; i += blockDim.x) {
    T s = T(0);
#pragma unroll 5
    for (int k = 0; k < m.w; ++k) s = fma(__ldg(m.val + k * m.n + i), P[__ldg(m.col + k * m.n + i)], s);
    Q[i] = s;
  }
}

__device__ __forceinline__ int sys_check(double rnorm, double tol, long long k, long long max_iters) {
  if (!isfinite(rnorm)) return GK_STOP_NAN;
  if (rnorm <= tol) return GK_STOP_CONVERGED;
  if (k >= max_iters) return GK_STOP_MAX_ITERS;
  return GK_STOP_NONE;
}

// D = 1 / diag(A) for the system (1 where the diagonal is missing or zero).
// A row's stored entries precede its padding, so the first entry in the
// row's own column is the diagonal when there is one.
template <typename T>
__device__ __forceinline__ void sys_jacobi(const SysMat<T>& m, T* D) {
  for (int i = threadIdx.x; i < m.n; i += blockDim.x) {
    T d = T(0);
    for (int k = 0; k < m.w; ++k)
      if (m.col[k * m.n + i] == i) {
        d = m.val[k * m.n + i];
        break;
      }
    D[i] = (d != T(0)) ? T(1) / d : T(1);
  }
}

template <typename T>
__device__ __forceinline__ void sys_finish(const BatchArgs& a, const T* X, int sys, int r0, int n, long long it,
                                           int stop, double rnorm, double ref) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) a.x[r0 + i] = static_cast<double>(X[i]);
  if (threadIdx.x == 0 && a.st) {
    a.st[sys].iters = static_cast<int32_t>(it);
    a.st[sys].stop_reason = stop;
    a.st[sys].rel_res = rnorm / ref;
    a.st[sys].outer_iters = 0;
  }
}

// Initial residual r = b - A x into R (and RH if given; A x staged in Q);
// returns ||r_0|| and the reference norm of the criterion.
template <typename T, bool WARP>
__device__ __forceinline__ void sys_start(const BatchArgs& a, const SysMat<T>& m, T* red, double* sc, int r0,
                                          int n, const T* X, T* R, T* Q, T* RH, double& rnorm, double& ref) {
  sys_spmv<T>(m, X, Q);
  T s2[2] = {T(0), T(0)};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T bi = static_cast<T>(a.b[r0 + i]);
    const T ri = bi - Q[i];
    R[i] = ri;
    if (RH) RH[i] = ri;
    s2[0] = fma(ri, ri, s2[0]);
    s2[1] = fma(bi, bi, s2[1]);
  }
  double o[2];
  const int rel_to_b = a.rel_to_b;
  reduce<WARP>(s2, red, sc, o, [&](T(&t)[2], double(&out)[2]) {
    const double rn = sqrt(static_cast<double>(t[0]));
    const double rf = rel_to_b ? sqrt(static_cast<double>(t[1])) : rn;
    out[0] = rn;
    out[1] = rf == 0.0 ? 1.0 : rf;
  });
  rnorm = o[0];
  ref = o[1];
}

// CG keeps x, r, p, q = A p and, with Jacobi, the inverse diagonal; between
// the residual update and the direction update q holds z = M^-1 r.
template <typename T, bool JAC, bool WARP>
__device__ void cg_system(const BatchArgs& a, T* V, T* red, double* sc, int sys, int r0, int n) {
  const SysMat<T> m = sys_mat<T>(a, sys, n);
  const int nm = a.nmax;
  T *X = V, *R = V + nm, *P = V + 2 * nm, *Q = V + 3 * nm, *D = V + 4 * nm;
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[i] = static_cast<T>(a.x[r0 + i]);
  if (JAC) sys_jacobi<T>(m, D);
  __syncthreads();
  double rnorm, ref;
  sys_start<T, WARP>(a, m, red, sc, r0, n, X, R, Q, nullptr, rnorm, ref);
  const double tol = a.factor * ref;
  T rho;
  {
    T v[1] = {T(0)};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const T z = JAC ? D[i] * R[i] : R[i];
      P[i] = z;
      v[0] = fma(R[i], z, v[0]);
    }
    double o[1];
    reduce<WARP>(v, red, sc, o, [](T(&t)[1], double(&out)[1]) { out[0] = static_cast<double>(t[0]); });
    rho = static_cast<T>(o[0]);
  }
  long long it = 0;
  int stop = sys_check(rnorm, tol, 0, a.max_iters);
  while (stop == GK_STOP_NONE) {
    sys_spmv<T>(m, P, Q);
    T sg[1] = {T(0)};
    for (int i = threadIdx.x; i < n; i += blockDim.x) sg[0] = fma(P[i], Q[i], sg[0]);
    double oa[2];
    reduce<WARP>(sg, red, sc, oa, [&](T(&t)[1], double(&out)[2]) {
      const T sigma = t[0];
      int code = GK_STOP_NONE;
      if (!isfinite(static_cast<double>(sigma))) code = GK_STOP_NAN;
      else if (sigma <= T(0)) code = GK_STOP_BREAKDOWN;
      out[0] = code == GK_STOP_NONE ? static_cast<double>(rho / sigma) : 0.0;
      out[1] = code;
    });
    if (oa[1] != 0.0) {
      stop = static_cast<int>(oa[1]);
      break;
    }
    const T alpha = static_cast<T>(oa[0]);
    T v[2] = {T(0), T(0)};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      X[i] = fma(alpha, P[i], X[i]);
      const T rn = fma(-alpha, Q[i], R[i]);
      R[i] = rn;
      const T z = JAC ? D[i] * rn : rn;
      if (JAC) Q[i] = z;
      v[0] = fma(rn, z, v[0]);
      v[1] = fma(rn, rn, v[1]);
    }
    double ob[3];
    reduce<WARP>(v, red, sc, ob, [&](T(&t)[2], double(&out)[3]) {
      out[0] = sqrt(static_cast<double>(t[1]));
      out[1] = static_cast<double>(t[0] / rho);
      out[2] = static_cast<double>(t[0]);
    });
    ++it;
    rnorm = ob[0];
    stop = sys_check(rnorm, tol, it, a.max_iters);
    if (stop != GK_STOP_NONE) break;
    const T beta = static_cast<T>(ob[1]);
    rho = static_cast<T>(ob[2]);
    const T* Z = JAC ? Q : R;
    for (int i = threadIdx.x; i < n; i += blockDim.x) P[i] = fma(beta, P[i], Z[i]);
    __syncthreads();
  }
  __syncthreads();
  sys_finish<T>(a, X, sys, r0, n, it, stop, rnorm, ref);
}

// BiCGSTAB keeps x, r (overwritten by s, then by the next r), the shadow
// residual, p, v = A p^, t = A s^ and, with Jacobi, the inverse diagonal and
// one vector for p^ (then s^): the x update by alpha p^ is done before s^
// overwrites p^, which leaves the rounding of every step as written.
template <typename T, bool JAC, bool WARP>
__device__ void bicg_system(const BatchArgs& a, T* V, T* red, double* sc, int sys, int r0, int n) {
  const SysMat<T> m = sys_mat<T>(a, sys, n);
  const int nm = a.nmax;
  T *X = V, *R = V + nm, *RH = V + 2 * nm, *P = V + 3 * nm, *W = V + 4 * nm, *TT = V + 5 * nm;
  T* H = JAC ? V + 6 * nm : nullptr;
  T* D = JAC ? V + 7 * nm : nullptr;
  const T* PH = JAC ? H : P;  // p^ = M^-1 p
  const T* SH = JAC ? H : R;  // s^ = M^-1 s (s lives in R)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    X[i] = static_cast<T>(a.x[r0 + i]);
    P[i] = T(0);
  }
  if (JAC) sys_jacobi<T>(m, D);
  __syncthreads();
  double rnorm, ref;
  sys_start<T, WARP>(a, m, red, sc, r0, n, X, R, W, RH, rnorm, ref);
  for (int i = threadIdx.x; i < n; i += blockDim.x) W[i] = T(0);
  const double tol = a.factor * ref;
  T rho_prev = T(1), alpha = T(1), omega = T(1);
  long long it = 0;
  int stop = sys_check(rnorm, tol, 0, a.max_iters);
  // FP32: a breakdown of the Lanczos part (rho or r^.v exactly zero, r^
  // orthogonal to the Krylov residuals to within float rounding) restarts
  // from the current iterate with r^ = r, p = v = 0, rho_prev = alpha =
  // omega = 1, at most kBicgRestarts times (the iteration count continues).
  int restarts = 0;
  auto restart = [&]() -> bool {
    if (!std::is_same<T, float>::value || restarts >= kBicgRestarts) return false;
    ++restarts;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      RH[i] = R[i];
      P[i] = T(0);
      W[i] = T(0);
    }
    rho_prev = T(1);
    alpha = T(1);
    omega = T(1);
    __syncthreads();
    return true;
  };
  while (stop == GK_STOP_NONE) {
    T rv[1] = {T(0)};
    for (int i = threadIdx.x; i < n; i += blockDim.x) rv[0] = fma(RH[i], R[i], rv[0]);
    double o1[3];
    reduce<WARP>(rv, red, sc, o1, [&](T(&t)[1], double(&out)[3]) {
      const T rho = t[0];
      int code = GK_STOP_NONE;
      if (!isfinite(static_cast<double>(rho))) code = GK_STOP_NAN;
      else if (rho == T(0)) code = GK_STOP_BREAKDOWN;
      out[0] = static_cast<double>(rho);
      out[1] = code == GK_STOP_NONE ? static_cast<double>((rho / rho_prev) * (alpha / omega)) : 0.0;
      out[2] = code;
    });
    if (o1[2] != 0.0) {
      if (static_cast<int>(o1[2]) == GK_STOP_BREAKDOWN && restart()) continue;
      stop = static_cast<int>(o1[2]);
      break;
    }
    const T rho = static_cast<T>(o1[0]), beta = static_cast<T>(o1[1]);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const T pn = fma(beta, fma(-omega, W[i], P[i]), R[i]);
      P[i] = pn;
      if (JAC) H[i] = D[i] * pn;
    }
    __syncthreads();
    sys_spmv<T>(m, PH, W);
    T hv[1] = {T(0)};
    for (int i = threadIdx.x; i < n; i += blockDim.x) hv[0] = fma(RH[i], W[i], hv[0]);
    double o2[2];
    reduce<WARP>(hv, red, sc, o2, [&](T(&t)[1], double(&out)[2]) {
      int code = GK_STOP_NONE;
      if (!isfinite(static_cast<double>(t[0]))) code = GK_STOP_NAN;
      else if (t[0] == T(0)) code = GK_STOP_BREAKDOWN;
      out[0] = code == GK_STOP_NONE ? static_cast<double>(rho / t[0]) : 0.0;
      out[1] = code;
    });
    if (o2[1] != 0.0) {
      if (static_cast<int>(o2[1]) == GK_STOP_BREAKDOWN && restart()) continue;
      stop = static_cast<int>(o2[1]);
      break;
    }
    alpha = static_cast<T>(o2[0]);
    T ss[1] = {T(0)};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      X[i] = fma(alpha, PH[i], X[i]);
      const T sn = fma(-alpha, W[i], R[i]);
      R[i] = sn;
      if (JAC) H[i] = D[i] * sn;
      ss[0] = fma(sn, sn, ss[0]);
    }
    double o3[1];
    reduce<WARP>(ss, red, sc, o3, [](T(&t)[1], double(&out)[1]) { out[0] = sqrt(static_cast<double>(t[0])); });
    const double snorm = o3[0];
    if (isfinite(snorm) && snorm <= tol) {
      ++it;
      rnorm = snorm;
      stop = GK_STOP_CONVERGED;
      break;
    }
    sys_spmv<T>(m, SH, TT);
    T tw[2] = {T(0), T(0)};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      tw[0] = fma(TT[i], R[i], tw[0]);
      tw[1] = fma(TT[i], TT[i], tw[1]);
    }
    double o4[2];
    reduce<WARP>(tw, red, sc, o4, [](T(&t)[2], double(&out)[2]) {
      int code = GK_STOP_NONE;
      if (!isfinite(static_cast<double>(t[0])) || !isfinite(static_cast<double>(t[1]))) code = GK_STOP_NAN;
      else if (t[1] == T(0)) code = GK_STOP_BREAKDOWN;
      out[0] = code == GK_STOP_NONE ? static_cast<double>(t[0] / t[1]) : 0.0;
      out[1] = code;
    });
    if (o4[1] != 0.0) {
      stop = static_cast<int>(o4[1]);
      break;
    }
    omega = static_cast<T>(o4[0]);
    T rr[1] = {T(0)};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      X[i] = fma(omega, SH[i], X[i]);
      const T rn = fma(-omega, TT[i], R[i]);
      R[i] = rn;
      rr[0] = fma(rn, rn, rr[0]);
    }
    double o5[1];
    reduce<WARP>(rr, red, sc, o5, [](T(&t)[1], double(&out)[1]) { out[0] = sqrt(static_cast<double>(t[0])); });
    rho_prev = rho;
    ++it;
    rnorm = o5[0];
    stop = sys_check(rnorm, tol, it, a.max_iters);
    if (stop == GK_STOP_NONE && omega == T(0)) stop = GK_STOP_BREAKDOWN;
  }
  __syncthreads();
  sys_finish<T>(a, X, sys, r0, n, it, stop, rnorm, ref);
}

// Iterative refinement (Sections 2.2.3 and 3.1) per system: the residual
// r = b - A x, its norm, the criteria and the update x = x + ||r|| d in FP64
// on the FP64 values; the correction d from CG in FP32 on the FP32 copy of A
// (FP32 vectors and sums) for A d = r / ||r||, stopped once its residual is
// reduced by max(inner_reduction, tol / (2 ||r||)) or after inner_max
// iterations.  Jacobi: the FP64 inverse diagonal rounded to FP32.
// Shared memory: x and r in FP64, then r, p, q (z between the updates), d
// and the inverse diagonal in FP32.
template <bool JAC, bool WARP>
__device__ void ir_system(const BatchArgs& a, unsigned char* smem, double* redd, double* sc, int sys, int r0,
                          int n) {
  const SysMat<double> m64 = sys_mat<double>(a, sys, n);
  const SysMat<float> m32{a.ell_val32 + a.ell_off[sys], m64.col, n, m64.w};
  const int nm = a.nmax;
  double* X = reinterpret_cast<double*>(smem);
  double* R64 = X + nm;
  float* R = reinterpret_cast<float*>(R64 + nm);
  float *P = R + nm, *Q = R + 2 * nm, *DX = R + 3 * nm, *D = R + 4 * nm;
  float* redf = reinterpret_cast<float*>(redd);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    X[i] = a.x[r0 + i];
    if (JAC) {
      double d = 0.0;
      for (int k = 0; k < m64.w; ++k)
        if (m64.col[k * n + i] == i) {
          d = m64.val[k * n + i];
          break;
        }
      D[i] = d != 0.0 ? static_cast<float>(1.0 / d) : 1.0f;
    }
  }
  __syncthreads();
  long long k_total = 0;
  int steps = 0, stop = GK_STOP_NONE;
  double rnorm = 0.0, ref = 1.0, tol = 0.0;
  const int rel_to_b = a.rel_to_b;
  for (;;) {
    // FP64 residual and its norm (and ||b|| on the first step)
    sys_spmv<double>(m64, X, R64);
    double s2[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double bi = a.b[r0 + i];
      const double ri = bi - R64[i];
      R64[i] = ri;
      s2[0] = fma(ri, ri, s2[0]);
      s2[1] = fma(bi, bi, s2[1]);
    }
    double o[3];
    const bool first = steps == 0;
    const double ref_prev = ref;
    reduce<WARP>(s2, redd, sc, o, [&](double(&t)[2], double(&out)[3]) {
      const double rn = sqrt(t[0]);
      double rf = ref_prev;
      if (first) {
        rf = rel_to_b ? sqrt(t[1]) : rn;
        if (rf == 0.0) rf = 1.0;
      }
      out[0] = rn;
      out[1] = rf;
      out[2] = 1.0 / rn;
    });
    rnorm = o[0];
    ref = o[1];
    const double inv = o[2];
    if (first) tol = a.factor * ref;
    stop = sys_check(rnorm, tol, k_total, a.max_iters);
    if (stop != GK_STOP_NONE || steps >= kBatchMaxOuter) {
      if (stop == GK_STOP_NONE) stop = GK_STOP_MAX_ITERS;
      break;
    }
    // FP32 inner CG on A d = r / ||r|| from d = 0
    float v2[2] = {0.0f, 0.0f};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float ri = static_cast<float>(R64[i] * inv);
      R[i] = ri;
      DX[i] = 0.0f;
      const float z = JAC ? D[i] * ri : ri;
      P[i] = z;
      v2[0] = fmaf(ri, z, v2[0]);
      v2[1] = fmaf(ri, ri, v2[1]);
    }
    double oi[2];
    const double inner_red = a.inner_red;
    reduce<WARP>(v2, redf, sc, oi, [&](float(&t)[2], double(&out)[2]) {
      const double red = fmax(inner_red, 0.5 * tol / rnorm);
      out[0] = static_cast<double>(t[0]);
      out[1] = red * red * static_cast<double>(t[1]);
    });
    float rho = static_cast<float>(oi[0]);
    const double tol2 = oi[1];
    long long it = 0;
    bool broke = false;
    while (it < a.inner_max) {
      sys_spmv<float>(m32, P, Q);
      float sg[1] = {0.0f};
      for (int i = threadIdx.x; i < n; i += blockDim.x) sg[0] = fmaf(P[i], Q[i], sg[0]);
      double oa[2];
      reduce<WARP>(sg, redf, sc, oa, [&](float(&t)[1], double(&out)[2]) {
        const float sigma = t[0];
        const bool bad = !isfinite(sigma) || sigma <= 0.0f;
        out[0] = bad ? 0.0 : static_cast<double>(static_cast<float>(static_cast<double>(rho) / sigma));
        out[1] = bad ? 1.0 : 0.0;
      });
      if (oa[1] != 0.0) {
        broke = true;
        break;
      }
      const float alpha = static_cast<float>(oa[0]);
      float v[2] = {0.0f, 0.0f};
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        DX[i] = fmaf(alpha, P[i], DX[i]);
        const float rn = fmaf(-alpha, Q[i], R[i]);
        R[i] = rn;
        const float z = JAC ? D[i] * rn : rn;
        if (JAC) Q[i] = z;
        v[0] = fmaf(rn, z, v[0]);
        v[1] = fmaf(rn, rn, v[1]);
      }
      double ob[3];
      reduce<WARP>(v, redf, sc, ob, [&](float(&t)[2], double(&out)[3]) {
        // out[2]: 0 go on, 1 broke (not finite), 2 inner target reached
        const bool bad = !isfinite(t[0]) || !isfinite(t[1]);
        out[0] = static_cast<double>(t[0]);
        out[1] = bad ? 0.0 : static_cast<double>(static_cast<float>(static_cast<double>(t[0]) / rho));
        out[2] = bad ? 1.0 : (static_cast<double>(t[1]) <= tol2 ? 2.0 : 0.0);
      });
      ++it;
      if (ob[2] == 1.0) {
        broke = true;
        break;
      }
      if (ob[2] == 2.0) break;
      const float beta = static_cast<float>(ob[1]);
      rho = static_cast<float>(ob[0]);
      const float* Z = JAC ? Q : R;
      for (int i = threadIdx.x; i < n; i += blockDim.x) P[i] = fmaf(beta, P[i], Z[i]);
      __syncthreads();
    }
    // x = x + ||r|| d in FP64
    for (int i = threadIdx.x; i < n; i += blockDim.x) X[i] = fma(rnorm, static_cast<double>(DX[i]), X[i]);
    __syncthreads();
    k_total += it;
    ++steps;
    if (it == 0 || (broke && it <= 1)) {
      stop = GK_STOP_BREAKDOWN;
      break;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) a.x[r0 + i] = X[i];
  if (threadIdx.x == 0 && a.st) {
    a.st[sys].iters = static_cast<int32_t>(k_total);
    a.st[sys].stop_reason = stop;
    a.st[sys].rel_res = rnorm / ref;
    a.st[sys].outer_iters = steps;
  }
}

// Shared-memory bytes per row a block keeps for one system.
__host__ __device__ constexpr int batch_row_bytes(int kind, bool jac, int el) {
  return kind == GK_CG ? el * (jac ? 5 : 4)
                       : (kind == GK_BICGSTAB ? el * (jac ? 8 : 6) : 16 + 4 * (jac ? 5 : 4));
}

// Offset of the reduction scratch (16-byte aligned) behind the vectors.
__host__ __device__ constexpr size_t batch_red_offset(int kind, bool jac, int el, int nmax) {
  return (static_cast<size_t>(batch_row_bytes(kind, jac, el)) * nmax + 15) / 16 * 16;
}


template <typename T, int KIND, bool JAC, bool WARP>
__global__ void __launch_bounds__(256) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char bsm[];
  __shared__ double s_sc[4];
  __shared__ int s_k;
  T* V = reinterpret_cast<T*>(bsm);
  unsigned char* redp = bsm + batch_red_offset(KIND, JAC, static_cast<int>(sizeof(T)), a.nmax);
  T* red = reinterpret_cast<T*>(redp);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_k = static_cast<int>(atomicAdd(a.next, 1u));
    __syncthreads();
    const int k = s_k;
    if (k >= a.count) break;
    const int sys = a.order[a.k0 + k];
    const int r0 = a.sys_ptr[sys], n = a.sys_ptr[sys + 1] - r0;
    if constexpr (KIND == GK_CG) cg_system<T, JAC, WARP>(a, V, red, s_sc, sys, r0, n);
    else if constexpr (KIND == GK_BICGSTAB) bicg_system<T, JAC, WARP>(a, V, red, s_sc, sys, r0, n);
    else ir_system<JAC, WARP>(a, bsm, reinterpret_cast<double*>(redp), s_sc, sys, r0, n);
  }
}

__global__ void batch_validate_kernel(const int32_t* sys_ptr, const int32_t* rowptr, const int32_t* col, int n_sys,
                                      int* bad) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sys; s += gridDim.x * blockDim.x) {
    const int r0 = sys_ptr[s], r1 = sys_ptr[s + 1];
    for (int r = r0; r < r1; ++r) {
      int prev = -1;
      for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
        const int c = col[k];
        if (c < r0 || c >= r1 || c <= prev) {
          atomicMin(bad, r);
          break;
        }
        prev = c;
      }
    }
  }
}

// Column-major ELL block of every system (one thread block per system,
// grid-stride over systems); values converted to the solve precision.
template <typename T>
__global__ void batch_ell_kernel(const int32_t* sys_ptr, const int32_t* rowptr, const int32_t* col,
                                 const double* val, const int32_t* ell_off, const int32_t* ell_w, int n_sys,
                                 T* ev, uint16_t* ec) {
  for (int s = blockIdx.x; s < n_sys; s += gridDim.x) {
    const int r0 = sys_ptr[s], n = sys_ptr[s + 1] - r0, w = ell_w[s];
    T* v = ev + ell_off[s];
    uint16_t* c = ec + ell_off[s];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int k0 = rowptr[r0 + i], len = rowptr[r0 + i + 1] - k0;
      for (int k = 0; k < w; ++k) {
        const bool real = k < len;
        v[k * n + i] = real ? static_cast<T>(val[k0 + k]) : T(0);
        c[k * n + i] = static_cast<uint16_t>(real ? col[k0 + k] - r0 : i);
      }
    }
  }
}

using BatchFn = void (*)(BatchArgs);

template <typename T, int KIND, bool JAC>
BatchFn pick_w(bool warp) {
  return warp ? batch_kernel<T, KIND, JAC, true> : batch_kernel<T, KIND, JAC, false>;
}

template <typename T>
BatchFn pick_t(int kind, bool jac, bool warp) {
  if (kind == GK_CG) return jac ? pick_w<T, GK_CG, true>(warp) : pick_w<T, GK_CG, false>(warp);
  return jac ? pick_w<T, GK_BICGSTAB, true>(warp) : pick_w<T, GK_BICGSTAB, false>(warp);
}

BatchFn pick_kernel(int dtype, int kind, bool jac, int threads) {
  const bool warp = threads == 32;
  if (kind == GK_IR_CG) return jac ? pick_w<double, GK_IR_CG, true>(warp) : pick_w<double, GK_IR_CG, false>(warp);
  return dtype == GK_F32 ? pick_t<float>(kind, jac, warp) : pick_t<double>(kind, jac, warp);
}

// Block size a class runs with before (or without) autotuning.
int default_threads(int c) { return c <= 1 ? 32 : (c <= 4 ? 64 : 128); }

}  // namespace

struct Batch {
  int device = 0;
  int64_t n_sys = 0, n_rows = 0, nnz = 0;
  int dtype = GK_F64;
  int nmax = 0;
  BatchClass cls[kBatchClasses];
  int64_t ell_entries = 0;
  int32_t* sys_ptr = nullptr;
  int32_t* order = nullptr;
  int32_t* ell_off = nullptr;
  int32_t* ell_w = nullptr;
  uint16_t* ell_col = nullptr;
  void* ell_val = nullptr;
  float* ell_val32 = nullptr;  // FP64 batches: FP32 copy for refinement
  unsigned int* next = nullptr;  // one counter per class
  gk_batch_status* st = nullptr;
  double* xtune = nullptr;
  int threads[3][2][kBatchClasses] = {};  // [kind][jacobi][class]; 0 = default
  int64_t device_bytes = 0;
  cudaGraphExec_t exec = nullptr;  // graph of the last configuration solved
  uint64_t key[8 + kBatchClasses] = {};
};

namespace {

struct ClassPlan {
  BatchFn fn = nullptr;
  int threads = 0, grid = 0;
  size_t smem = 0;
};

int class_threads(const Batch& B, int kind, int jac, int c) {
  const int t = B.threads[kind][jac ? 1 : 0][c];
  return t > 0 ? t : default_threads(c);
}

// Kernel, shared memory and persistent grid for one class at one block size
// (no launch; GK_ERR_UNSUPPORTED if the class's vectors do not fit).
int plan_class(const Batch& B, int kind, int jac, int c, int threads, ClassPlan* p) {
  const BatchClass& k = B.cls[c];
  const size_t el = B.dtype == GK_F32 ? 4 : 8;
  p->threads = threads;
  const int elk = kind == GK_IR_CG ? 8 : static_cast<int>(el);
  p->smem = batch_red_offset(kind, jac != 0, elk, k.nmax) + 16 * static_cast<size_t>(threads) + 16;
  p->fn = pick_kernel(B.dtype, kind, jac != 0, threads);
  int smem_max = 0;
  GK_TRY_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, B.device));
  if (p->smem + 64 > static_cast<size_t>(smem_max))
    return set_error(GK_ERR_UNSUPPORTED, "batch: a %d-row system needs %zu bytes of shared memory (max %d)", k.nmax,
                     p->smem, smem_max);
  GK_TRY(set_smem(reinterpret_cast<const void*>(p->fn), p->smem));
  int per_sm = 0;
  GK_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->fn, threads, p->smem));
  if (per_sm < 1) return set_error(GK_ERR_UNSUPPORTED, "batch: no block of %d threads fits an SM", threads);
  p->grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(per_sm) * sm_count(), k.count));
  return GK_OK;
}

BatchArgs class_args(const Batch& B, const gk_criteria& c, const double* b, double* x, int cl) {
  BatchArgs a;
  a.sys_ptr = B.sys_ptr;
  a.order = B.order;
  a.ell_off = B.ell_off;
  a.ell_w = B.ell_w;
  a.ell_col = B.ell_col;
  a.ell_val = B.ell_val;
  a.ell_val32 = B.ell_val32;
  a.b = b;
  a.x = x;
  a.st = B.st;
  a.next = B.next + cl;
  a.max_iters = c.max_iters;
  a.factor = c.reduction_factor;
  a.rel_to_b = c.rel_to_b;
  a.inner_red = c.inner_reduction > 0 ? c.inner_reduction : 1e-5;
  a.inner_max = c.inner_max_iters > 0 ? c.inner_max_iters : std::max<int64_t>(c.max_iters, 1);
  a.k0 = B.cls[cl].k0;
  a.count = B.cls[cl].count;
  a.nmax = B.cls[cl].nmax;
  return a;
}

int launch_class(const ClassPlan& p, const BatchArgs& a, cudaStream_t s) {
  p.fn<<<p.grid, p.threads, p.smem, s>>>(a);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

void batch_release(Batch* B) {
  if (!B) return;
  const int prev = current_device();
  cudaSetDevice(B->device);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  void* ptrs[] = {B->sys_ptr, B->order,  B->ell_off, B->ell_w, B->ell_col, B->ell_val,
                  B->ell_val32, B->next, B->st,     B->xtune};
  for (void* p : ptrs) dfree(p);
  cudaSetDevice(prev);
  delete B;
}

struct BatchDeleter {
  void operator()(Batch* b) const { batch_release(b); }
};

int check_kind(int32_t kind) {
  if (kind != GK_CG && kind != GK_BICGSTAB && kind != GK_IR_CG)
    return set_error(GK_ERR_ARG, "batch: kind must be GK_CG, GK_BICGSTAB or GK_IR_CG");
  return GK_OK;
}

int check_kind(const Batch& B, int32_t kind) {
  GK_TRY(check_kind(kind));
  if (kind == GK_IR_CG && B.dtype != GK_F64)
    return set_error(GK_ERR_ARG, "batch: GK_IR_CG needs an FP64 batch (its residuals use the FP64 values)");
  return GK_OK;
}

// Records, on capture stream cs, a reset of the class counters followed by
// the class kernels as independent branches joined back into cs.
int capture_solve(const Batch& B, const ClassPlan* plan, const BatchArgs* args, cudaStream_t cs) {
  cudaStream_t side[kBatchClasses] = {};
  cudaEvent_t fork = nullptr, join[kBatchClasses] = {};
  int rc = GK_OK;
  cudaError_t e = cudaMemsetAsync(B.next, 0, sizeof(unsigned int) * kBatchClasses, cs);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(fork, cs);
  for (int c = kBatchClasses - 1; c >= 0 && e == cudaSuccess && rc == GK_OK; --c) {
    if (!B.cls[c].count) continue;
    e = cudaStreamCreateWithFlags(&side[c], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[c], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side[c], fork, 0);
    if (e != cudaSuccess) break;
    rc = launch_class(plan[c], args[c], side[c]);
    // join the branch back even after a failed launch, so the capture can end
    const cudaError_t e2 = cudaEventRecord(join[c], side[c]);
    e = e2 == cudaSuccess ? cudaStreamWaitEvent(cs, join[c], 0) : e2;
  }
  if (rc == GK_OK && e != cudaSuccess) rc = cuda_error(e, "batch graph");
  for (int c = 0; c < kBatchClasses; ++c) {
    if (join[c]) cudaEventDestroy(join[c]);
    if (side[c]) cudaStreamDestroy(side[c]);
  }
  if (fork) cudaEventDestroy(fork);
  return rc;
}

}  // namespace

}  // namespace gk

using namespace gk;

extern "C" int gk_batch_create(int64_t n_sys, const int64_t* sys_ptr, int64_t nnz, const int32_t* rowptr,
                               const int32_t* col, const double* val, int32_t dtype, void* stream, gk_batch* out) {
  if (!out) return set_error(GK_ERR_ARG, "gk_batch_create: out is NULL");
  *out = nullptr;
  if (n_sys <= 0 || !sys_ptr || !rowptr || nnz < 0 || (nnz > 0 && (!col || !val)))
    return set_error(GK_ERR_ARG, "gk_batch_create: bad argument");
  if (dtype != GK_F64 && dtype != GK_F32) return set_error(GK_ERR_DTYPE, "gk_batch_create: dtype %d", dtype);
  if (nnz > INT32_MAX - 16 || n_sys > INT32_MAX - 16)
    return set_error(GK_ERR_ARG, "gk_batch_create: sizes exceed int32 indexing");
  std::vector<int64_t> sp(sys_ptr, sys_ptr + n_sys + 1);
  if (sp[0] != 0) return set_error(GK_ERR_CSR, "gk_batch_create: sys_ptr[0] != 0");
  int nmax = 0;
  for (int64_t s = 0; s < n_sys; ++s) {
    const int64_t m = sp[s + 1] - sp[s];
    if (m <= 0) return set_error(GK_ERR_CSR, "gk_batch_create: system %lld is empty", (long long)s);
    if (m > kBatchMaxRows)
      return set_error(GK_ERR_UNSUPPORTED, "gk_batch_create: system %lld has %lld rows (max %d)", (long long)s,
                       (long long)m, kBatchMaxRows);
    nmax = std::max<int>(nmax, static_cast<int>(m));
  }
  const int64_t n_rows = sp[n_sys];
  if (n_rows > INT32_MAX - 16) return set_error(GK_ERR_ARG, "gk_batch_create: too many rows");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::unique_ptr<Batch, BatchDeleter> hold(new Batch);
  Batch* B = hold.get();
  B->device = current_device();
  B->n_sys = n_sys;
  B->n_rows = n_rows;
  B->nnz = nnz;
  B->dtype = dtype;
  B->nmax = nmax;
  int64_t* by = &B->device_bytes;
  std::vector<int32_t> sp32(sp.begin(), sp.end());
  std::vector<int32_t> order(static_cast<size_t>(n_sys));
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return sp[a + 1] - sp[a] > sp[b + 1] - sp[b]; });
  for (int64_t k = 0; k < n_sys; ++k) {
    const int m = static_cast<int>(sp[order[k] + 1] - sp[order[k]]);
    int c = 0;
    while (m > (32 << c)) ++c;
    BatchClass& cl = B->cls[c];
    if (cl.count == 0) {
      cl.k0 = static_cast<int>(k);
      cl.nmax = m;  // decreasing order: the class's first system is its largest
    }
    ++cl.count;
  }
  GK_TRY(dalloc_n(&B->sys_ptr, sp32.size(), by));
  GK_TRY(dalloc_n(&B->order, order.size(), by));
  GK_TRY(dalloc_n(&B->next, kBatchClasses, by));
  GK_TRY(dalloc_n(&B->st, static_cast<size_t>(n_sys), by));
  GK_TRY_CUDA(cudaMemcpyAsync(B->sys_ptr, sp32.data(), sizeof(int32_t) * sp32.size(), cudaMemcpyHostToDevice, s));
  GK_TRY_CUDA(cudaMemcpyAsync(B->order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, s));
  // the caller's CSR, staged on the device for validation and conversion
  // (freed on every return path)
  struct Staging {
    int32_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    ~Staging() {
      dfree(rowptr);
      dfree(col);
      dfree(val);
    }
  } d;
  int64_t staged_bytes = 0;
  GK_TRY(dalloc_n(&d.rowptr, static_cast<size_t>(n_rows + 1), &staged_bytes));
  GK_TRY(dalloc_n(&d.col, static_cast<size_t>(std::max<int64_t>(nnz, 1)), &staged_bytes));
  GK_TRY(dalloc_n(&d.val, static_cast<size_t>(std::max<int64_t>(nnz, 1)), &staged_bytes));
  GK_TRY_CUDA(cudaMemcpyAsync(d.rowptr, rowptr, sizeof(int32_t) * (n_rows + 1), cudaMemcpyDefault, s));
  if (nnz > 0) {
    GK_TRY_CUDA(cudaMemcpyAsync(d.col, col, sizeof(int32_t) * nnz, cudaMemcpyDefault, s));
    GK_TRY_CUDA(cudaMemcpyAsync(d.val, val, sizeof(double) * nnz, cudaMemcpyDefault, s));
  }
  std::vector<int32_t> hrp(static_cast<size_t>(n_rows + 1));
  GK_TRY_CUDA(cudaMemcpyAsync(hrp.data(), d.rowptr, sizeof(int32_t) * hrp.size(), cudaMemcpyDeviceToHost, s));
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  if (hrp[0] != 0 || hrp[n_rows] != nnz) return set_error(GK_ERR_CSR, "gk_batch_create: rowptr does not span nnz");
  for (int64_t i = 0; i < n_rows; ++i)
    if (hrp[i + 1] < hrp[i]) return set_error(GK_ERR_CSR, "gk_batch_create: rowptr decreases at %lld", (long long)i);
  int* bad = reinterpret_cast<int*>(B->next);
  const int bad_init = INT_MAX;
  int badh = INT_MAX;
  GK_TRY_CUDA(cudaMemcpyAsync(bad, &bad_init, sizeof(int), cudaMemcpyHostToDevice, s));
  batch_validate_kernel<<<static_cast<int>(std::min<int64_t>((n_sys + 255) / 256, 4096)), 256, 0, s>>>(
      B->sys_ptr, d.rowptr, d.col, static_cast<int>(n_sys), bad);
  GK_TRY_CUDA(cudaGetLastError());
  GK_TRY_CUDA(cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  if (badh != INT_MAX)
    return set_error(GK_ERR_CSR, "gk_batch_create: row %d leaves its system, or its columns are unsorted/repeated",
                     badh);
  // per-system ELL widths and offsets
  std::vector<int32_t> ew(static_cast<size_t>(n_sys)), eo(static_cast<size_t>(n_sys) + 1);
  int64_t total = 0;
  for (int64_t q = 0; q < n_sys; ++q) {
    int w = 0;
    for (int64_t r = sp[q]; r < sp[q + 1]; ++r) w = std::max(w, hrp[r + 1] - hrp[r]);
    ew[q] = w;
    eo[q] = static_cast<int32_t>(total);
    total += static_cast<int64_t>(w) * (sp[q + 1] - sp[q]);
    if (total > INT32_MAX - 16) return set_error(GK_ERR_UNSUPPORTED, "gk_batch_create: ELL storage exceeds 2^31");
  }
  eo[n_sys] = static_cast<int32_t>(total);
  B->ell_entries = total;
  GK_TRY(dalloc_n(&B->ell_off, eo.size(), by));
  GK_TRY(dalloc_n(&B->ell_w, ew.size(), by));
  GK_TRY(dalloc_n(&B->ell_col, static_cast<size_t>(std::max<int64_t>(total, 1)), by));
  GK_TRY(dalloc(&B->ell_val, static_cast<size_t>(std::max<int64_t>(total, 1)) * (dtype == GK_F32 ? 4 : 8), by));
  GK_TRY_CUDA(cudaMemcpyAsync(B->ell_off, eo.data(), sizeof(int32_t) * eo.size(), cudaMemcpyHostToDevice, s));
  GK_TRY_CUDA(cudaMemcpyAsync(B->ell_w, ew.data(), sizeof(int32_t) * ew.size(), cudaMemcpyHostToDevice, s));
  const int eg = static_cast<int>(std::min<int64_t>(n_sys, 16 * sm_count()));
  if (dtype == GK_F32)
    batch_ell_kernel<float><<<eg, 128, 0, s>>>(B->sys_ptr, d.rowptr, d.col, d.val, B->ell_off, B->ell_w,
                                               static_cast<int>(n_sys), static_cast<float*>(B->ell_val), B->ell_col);
  else
    batch_ell_kernel<double><<<eg, 128, 0, s>>>(B->sys_ptr, d.rowptr, d.col, d.val, B->ell_off, B->ell_w,
                                                static_cast<int>(n_sys), static_cast<double*>(B->ell_val),
                                                B->ell_col);
  GK_TRY_CUDA(cudaGetLastError());
  if (dtype == GK_F64) {
    GK_TRY(dalloc_n(&B->ell_val32, static_cast<size_t>(std::max<int64_t>(total, 1)), by));
    batch_ell_kernel<float><<<eg, 128, 0, s>>>(B->sys_ptr, d.rowptr, d.col, d.val, B->ell_off, B->ell_w,
                                               static_cast<int>(n_sys), B->ell_val32, B->ell_col);
    GK_TRY_CUDA(cudaGetLastError());
  }
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  *out = reinterpret_cast<gk_batch>(hold.release());
  return GK_OK;
}

extern "C" int gk_batch_solve(gk_batch h, int32_t kind, int32_t jacobi, const gk_criteria* crit, const void* b,
                              void* x, gk_batch_status* st, void* stream) {
  Batch* B = reinterpret_cast<Batch*>(h);
  if (!B || !crit || !b || !x) return set_error(GK_ERR_ARG, "gk_batch_solve: NULL argument");
  GK_TRY(check_kind(*B, kind));
  const int prev = current_device();
  if (prev != B->device) cudaSetDevice(B->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = GK_OK;
  do {
    uint64_t key[8 + kBatchClasses];
    memset(key, 0, sizeof(key));
    key[0] = static_cast<uint64_t>(kind);
    key[1] = static_cast<uint64_t>(jacobi != 0);
    key[2] = reinterpret_cast<uint64_t>(b);
    key[3] = reinterpret_cast<uint64_t>(x);
    key[4] = static_cast<uint64_t>(crit->max_iters);
    memcpy(&key[5], &crit->reduction_factor, sizeof(double));
    key[6] = static_cast<uint64_t>(crit->rel_to_b);
    memcpy(&key[7], &crit->inner_reduction, sizeof(double));
    key[7] ^= static_cast<uint64_t>(static_cast<uint32_t>(crit->inner_max_iters)) * 0x9E3779B97F4A7C15ull;
    for (int c = 0; c < kBatchClasses; ++c) key[8 + c] = static_cast<uint64_t>(class_threads(*B, kind, jacobi, c));
    if (!B->exec || memcmp(key, B->key, sizeof(key)) != 0) {
      if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
      }
      ClassPlan plan[kBatchClasses];
      BatchArgs args[kBatchClasses];
      for (int c = 0; c < kBatchClasses && rc == GK_OK; ++c) {
        if (!B->cls[c].count) continue;
        rc = plan_class(*B, kind, jacobi, c, class_threads(*B, kind, jacobi, c), &plan[c]);
        args[c] = class_args(*B, *crit, static_cast<const double*>(b), static_cast<double*>(x), c);
      }
      if (rc != GK_OK) break;
      cudaStream_t cs = nullptr;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        rc = cuda_error(e, "batch graph");
        if (cs) cudaStreamDestroy(cs);
        break;
      }
      rc = capture_solve(*B, plan, args, cs);
      e = cudaStreamEndCapture(cs, &g);
      if (rc == GK_OK && e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (rc != GK_OK) break;
      if (e != cudaSuccess) {
        rc = cuda_error(e, "batch graph");
        B->exec = nullptr;
        break;
      }
      memcpy(B->key, key, sizeof(key));
    }
    cudaError_t e = cudaGraphLaunch(B->exec, s);
    if (e != cudaSuccess) {
      rc = cuda_error(e, "gk_batch_solve: graph launch");
      break;
    }
    if (st) {
      e = cudaMemcpyAsync(st, B->st, sizeof(gk_batch_status) * B->n_sys, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) rc = cuda_error(e, "gk_batch_solve: status");
    }
  } while (false);
  if (prev != B->device) cudaSetDevice(prev);
  return rc;
}

extern "C" int gk_batch_set_threads(gk_batch h, int32_t kind, int32_t jacobi, const int32_t* threads) {
  Batch* B = reinterpret_cast<Batch*>(h);
  if (!B || !threads) return set_error(GK_ERR_ARG, "gk_batch_set_threads: NULL argument");
  GK_TRY(check_kind(kind));
  for (int c = 0; c < kBatchClasses; ++c) {
    const int t = threads[c];
    if (t != 0 && t != 32 && t != 64 && t != 128 && t != 256)
      return set_error(GK_ERR_ARG, "gk_batch_set_threads: block size %d (0, 32, 64, 128 or 256)", t);
  }
  for (int c = 0; c < kBatchClasses; ++c) B->threads[kind][jacobi ? 1 : 0][c] = threads[c];
  return GK_OK;
}

extern "C" int gk_batch_get_info(gk_batch h, int32_t kind, int32_t jacobi, int32_t* counts, int32_t* nmax,
                                 int32_t* threads) {
  Batch* B = reinterpret_cast<Batch*>(h);
  if (!B) return set_error(GK_ERR_ARG, "gk_batch_get_info: NULL handle");
  GK_TRY(check_kind(kind));
  for (int c = 0; c < kBatchClasses; ++c) {
    if (counts) counts[c] = B->cls[c].count;
    if (nmax) nmax[c] = B->cls[c].nmax;
    if (threads) threads[c] = B->cls[c].count ? class_threads(*B, kind, jacobi, c) : 0;
  }
  return GK_OK;
}

extern "C" int gk_batch_autotune(gk_batch h, int32_t kind, int32_t jacobi, const gk_criteria* crit, const void* b,
                                 int32_t* threads, double* times_ms, void* stream) {
  Batch* B = reinterpret_cast<Batch*>(h);
  if (!B || !crit || !b) return set_error(GK_ERR_ARG, "gk_batch_autotune: NULL argument");
  GK_TRY(check_kind(*B, kind));
  const int prev = current_device();
  if (prev != B->device) cudaSetDevice(B->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = GK_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int chosen[kBatchClasses] = {};
  do {
    if (!B->xtune && (rc = dalloc_n(&B->xtune, static_cast<size_t>(B->n_rows), &B->device_bytes))) break;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
      rc = cuda_error(e, "events");
      break;
    }
    for (int c = 0; c < kBatchClasses && rc == GK_OK; ++c) {
      if (times_ms)
        for (int j = 0; j < 4; ++j) times_ms[c * 4 + j] = -1.0;
      if (!B->cls[c].count) continue;
      BatchArgs a = class_args(*B, *crit, static_cast<const double*>(b), B->xtune, c);
      a.st = nullptr;
      float best_ms = 0.0f;
      for (int j = 0; j < 4 && rc == GK_OK; ++j) {
        ClassPlan p;
        rc = plan_class(*B, kind, jacobi, c, kBatchCandidates[j], &p);
        if (rc == GK_ERR_UNSUPPORTED) {  // this block size does not fit: skip it
          rc = GK_OK;
          continue;
        }
        if (rc != GK_OK) break;
        float ms = -1.0f;
        for (int rep = 0; rep < 2 && rc == GK_OK; ++rep) {  // the first run warms the caches
          e = cudaMemsetAsync(B->xtune, 0, sizeof(double) * B->n_rows, s);
          if (e == cudaSuccess) e = cudaMemsetAsync(B->next + c, 0, sizeof(unsigned int), s);
          if (e == cudaSuccess) e = cudaEventRecord(e0, s);
          if (e != cudaSuccess) {
            rc = cuda_error(e, "autotune");
            break;
          }
          rc = launch_class(p, a, s);
          if (rc != GK_OK) break;
          e = cudaEventRecord(e1, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) rc = cuda_error(e, "autotune timing");
        }
        if (rc != GK_OK) break;
        if (times_ms) times_ms[c * 4 + j] = ms;
        if (chosen[c] == 0 || ms < best_ms) {
          chosen[c] = kBatchCandidates[j];
          best_ms = ms;
        }
      }
      if (rc == GK_OK && chosen[c] == 0)
        rc = set_error(GK_ERR_UNSUPPORTED, "gk_batch_autotune: class %d fits no block size", c);
    }
    if (rc != GK_OK) break;
    for (int c = 0; c < kBatchClasses; ++c) {
      B->threads[kind][jacobi ? 1 : 0][c] = chosen[c];
      if (threads) threads[c] = chosen[c];
    }
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (prev != B->device) cudaSetDevice(prev);
  return rc;
}

extern "C" int gk_batch_destroy(gk_batch h) {
  if (!h) return set_error(GK_ERR_ARG, "gk_batch_destroy: NULL handle");
  batch_release(reinterpret_cast<Batch*>(h));
  return GK_OK;
}
