// mixed.cu -- mixed-precision iterative refinement (GK_IR_CG).
//
// The paper builds iterative refinement from an outer fixed-point iteration
// and an inner solver given as a factory (Sections 2.2.3 and 3.1), and lets
// block-Jacobi store each inverted diagonal block in the precision its
// condition number allows (Section 3.2, "adaptive precision").  Here:
//   outer (FP64):  r = b - A x and ||r|| (FP64 SpMV), criteria, x += ||r|| d
//   inner (FP32):  CG on A d = r / ||r|| with an FP32 copy of A, FP32
//                  vectors and FP32 accumulation, stopped after a relative
//                  reduction max(inner_reduction, tol / (2 ||r||));
//   preconditioner of the inner solve: FP32 copy of scalar Jacobi, or the
//                  FP64 block-Jacobi inverses re-stored per block in FP16
//                  (kappa_1 * 2^-11 <= 1e-2) or FP32, each block scaled by a
//                  power of two so its largest entry lies in [0.5, 1).
// On this GPU the inner solve is bound by HBM alone (FP32 FMAs are ~60x
// faster than FP64 ones, and an FP32 entry moves 8 instead of 12 bytes).
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "gk_device.cuh"
#include "gk_internal.h"
#include "precond_device.cuh"
#include "solver_state.cuh"

namespace gk {

struct InnerState {
  double rho, alpha, beta, rr0, tol2;
  double red[2];
  long long it, max_it;
  long long d_it;  // the iteration whose d += alpha p the direction step has applied
  int done;
  int breakdown;
};

struct IrData {
  int fmt = GK_CSR;  // GK_ELL: FP32 copy of the ELL part (+ HYB overflow as CSR); GK_CSR: CSR copy
  float* val32 = nullptr;
  float* ell_val32 = nullptr;
  float* tail_val32 = nullptr;
  float* tail_sum32 = nullptr;
  int lpr = 32, tail_lpr = 32;
  float *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *d = nullptr;
  float* dinv = nullptr;
  __half* blk16 = nullptr;
  float* blk32 = nullptr;
  uint8_t* prec = nullptr;
  float* bscale = nullptr;
  int64_t n16 = 0, n32 = 0;
  InnerState* ist = nullptr;
  float* partials = nullptr;
  unsigned int* counter = nullptr;
  int grid = 1;
  double inner_red = 1e-5;
  long long inner_max = 0;
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int64_t bytes = 0;
};

namespace {

constexpr int kIrThreads = 256;
constexpr int kMaxOuter = 200;
constexpr double kFp16KappaMax = 1e-2 * 2048.0;  // kappa_1 * 2^-11 <= 1e-2

__global__ void to_float_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = static_cast<float>(in[i]);
}

// --------------------------------------------------------------------------
// adaptive-precision block storage
// --------------------------------------------------------------------------

// One warp per block: kappa_1 = ||D||_1 ||D^{-1}||_1 (column sums in
// increasing row order, maximum over columns), the storage precision, the
// power-of-two scale, and the scaled copy (row-major like the FP64 blocks:
// entry (i, j) at i * m + j, so that a lane reads its row with vector loads).
__global__ void __launch_bounds__(128) bj_adapt_kernel(const int32_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ col,
                                                       const double* __restrict__ val,
                                                       const double* __restrict__ inv, int n, int bs,
                                                       int nblocks, __half* blk16, float* blk32, uint8_t* prec,
                                                       float* bscale) {
  __shared__ double tile[4][32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double(*T)[33] = tile[w];
  for (int blk = blockIdx.x * 4 + w; blk < nblocks; blk += gridDim.x * 4) {
    const int r0 = blk * bs;
    const int m = min(bs, n - r0);
    const int64_t off = static_cast<int64_t>(blk) * bs * bs;
    for (int j = 0; j < 32; ++j) T[lane][j] = 0.0;
    __syncwarp();
    if (lane < m) {
      for (int k = rowptr[r0 + lane]; k < rowptr[r0 + lane + 1]; ++k) {
        const int c = col[k];
        if (c >= r0 && c < r0 + m) T[lane][c - r0] = fabs(val[k]);
      }
    }
    __syncwarp();
    double na = 0.0, ni = 0.0, vmax = 0.0;
    if (lane < m) {
      for (int i = 0; i < m; ++i) na += T[i][lane];
      for (int i = 0; i < m; ++i) {  // column `lane` of the row-major inverse
        const double v = fabs(inv[off + static_cast<int64_t>(i) * m + lane]);
        ni += v;
        vmax = fmax(vmax, v);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      na = fmax(na, __shfl_xor_sync(0xffffffffu, na, o));
      ni = fmax(ni, __shfl_xor_sync(0xffffffffu, ni, o));
      vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    const bool half = na * ni <= kFp16KappaMax;
    int e = 0;
    if (vmax > 0.0) frexp(vmax, &e);  // vmax = f * 2^e, f in [0.5, 1)
    const double sc = ldexp(1.0, -e);
    if (lane == 0) {
      prec[blk] = half ? 0 : 1;
      bscale[blk] = static_cast<float>(ldexp(1.0, e));
    }
    for (int idx = lane; idx < m * m; idx += 32) {  // row-major in and out
      const double v = inv[off + idx] * sc;
      if (half) blk16[off + idx] = __double2half(v);
      else blk32[off + idx] = static_cast<float>(v);
    }
    __syncwarp();
  }
}

// z_i = bscale * sum_j D'(i, j) r_j for the lane's block (FP32 arithmetic,
// increasing j).  BS > 0: the block size known at compile time -- a full
// block's row is fetched with 16-byte (FP32) or 8/16-byte (FP16) loads, all
// issued before the sum; BS = 0: any block size, one load per entry.  The
// loads may diverge; the shuffles that hand r_j around are executed by every
// lane of the warp.
template <int BS>
__device__ __forceinline__ float bj_apply32(const IrData& a, const BjLane& L, int bs, float r_mine) {
  if constexpr (BS == 0) {
    float z = 0.0f;
    const int64_t off = static_cast<int64_t>(L.blk) * bs * bs + static_cast<int64_t>(L.i) * L.m;
    const bool h = L.active && a.prec[L.blk] == 0;
    for (int j = 0; j < bs; ++j) {
      const float rj = __shfl_sync(0xffffffffu, r_mine, (L.base + j) & 31);
      if (L.active && j < L.m) {
        const float dv = h ? __half2float(a.blk16[off + j]) : a.blk32[off + j];
        z = fmaf(dv, rj, z);
      }
    }
    return L.active ? z * a.bscale[L.blk] : 0.0f;
  } else {
    float dv[BS];
#pragma unroll
    for (int j = 0; j < BS; ++j) dv[j] = 0.0f;
    if (L.active) {
      const int64_t off = static_cast<int64_t>(L.blk) * BS * BS + static_cast<int64_t>(L.i) * L.m;
      const bool h = a.prec[L.blk] == 0;
      if (L.m == BS && h && BS % 8 == 0) {
        const uint4* src = reinterpret_cast<const uint4*>(a.blk16 + off);
#pragma unroll
        for (int k = 0; k < BS / 8; ++k) {
          const uint4 u = __ldg(src + k);
          const unsigned int w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[q]));
            dv[8 * k + 2 * q] = f.x;
            dv[8 * k + 2 * q + 1] = f.y;
          }
        }
      } else if (L.m == BS && !h && BS % 4 == 0) {
        const float4* src = reinterpret_cast<const float4*>(a.blk32 + off);
#pragma unroll
        for (int k = 0; k < BS / 4; ++k) {
          const float4 f = __ldg(src + k);
          dv[4 * k] = f.x;
          dv[4 * k + 1] = f.y;
          dv[4 * k + 2] = f.z;
          dv[4 * k + 3] = f.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < BS; ++j)
          if (j < L.m) dv[j] = h ? __half2float(a.blk16[off + j]) : a.blk32[off + j];
      }
    }
    float z = 0.0f;
#pragma unroll
    for (int j = 0; j < BS; ++j) {
      const float rj = __shfl_sync(0xffffffffu, r_mine, (L.base + j) & 31);
      if (j < L.m) z = fmaf(dv[j], rj, z);
    }
    return L.active ? z * a.bscale[L.blk] : 0.0f;
  }
}

// --------------------------------------------------------------------------
// FP32 SpMV q = A p with sigma = p.q -> alpha = rho / sigma
// --------------------------------------------------------------------------

struct IrArgs {
  int n;
  // operator
  const int32_t* rowptr;
  const int32_t* col;
  const int32_t* ell_col;
  int64_t ld;
  int K;
  const int32_t* tail_rowptr;
  const int32_t* tail_slot;
  int m_tail;
  // preconditioner
  int bs, nblocks;
  // outer (FP64) vectors and state
  double* x;
  const double* r64;
  SolverState* st;
  cudaGraphConditionalHandle cond;
  int use_cond;  // 0: launched from the host (no graph loop to re-arm)
};

__device__ __forceinline__ void inner_alpha(InnerState* ist, float sigma) {
  if (!isfinite(sigma) || sigma <= 0.0f) {
    ist->done = 1;
    ist->breakdown = 1;
  } else {
    ist->alpha = ist->rho / static_cast<double>(sigma);
  }
}

struct Ell32 {
  const int32_t* col;
  const float* val;
  int64_t ld;
  int K;
  int n;
  const int32_t* tail_slot;
  const float* tail_sum;
  InnerState* ist;
  float* partials;
  unsigned int* counter;
};

template <bool TAIL, bool DOT>
__global__ void __launch_bounds__(kIrThreads, 8) ir_spmv_ell_kernel(Ell32 a, const float* __restrict__ x,
                                                                     float* __restrict__ y) {
  pdl_wait();
  __shared__ float scratch[kRedScratch];
  if (a.ist->done) return;
  float a0 = 0.0f;
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < a.n; row += stride) {
    const int32_t* cp = a.col + row;
    const float* vp = a.val + row;
    float s = 0.0f;
    int j = 0;
    for (; j + 4 <= a.K; j += 4) {
      int cc[4];
      float vv[4], xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) cc[u] = __ldcs(cp + (j + u) * a.ld);
#pragma unroll
      for (int u = 0; u < 4; ++u) vv[u] = __ldcs(vp + (j + u) * a.ld);
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = cc[u] >= 0 ? __ldg(x + cc[u]) : 0.0f;
#pragma unroll
      for (int u = 0; u < 4; ++u) s = fmaf(vv[u], xv[u], s);
    }
    for (; j < a.K; ++j) {
      const int c = __ldcs(cp + j * a.ld);
      if (c >= 0) s = fmaf(__ldcs(vp + j * a.ld), __ldg(x + c), s);
    }
    if (TAIL) {
      const int t = __ldg(a.tail_slot + row);
      if (t >= 0) s += __ldcg(a.tail_sum + t);
    }
    y[row] = s;
    if (DOT) a0 = fmaf(x[row], s, a0);
  }
  if (DOT) {
    float v[1] = {a0}, out[1];
    if (grid_sum<1, float>(v, a.partials, a.counter, scratch, out) && threadIdx.x == 0) inner_alpha(a.ist, out[0]);
  }
}

// Sub-warp of LPR lanes per row; FP32 shuffles are cheap, so a short xor
// tree per row is fine here.
template <int LPR, bool DOT>
__global__ void __launch_bounds__(kIrThreads, 8) ir_spmv_csr_kernel(const int32_t* __restrict__ rowptr,
                                                                     const int32_t* __restrict__ col,
                                                                     const float* __restrict__ val, int n,
                                                                     IrData d, const float* __restrict__ x,
                                                                     float* __restrict__ y) {
  pdl_wait();
  __shared__ float scratch[kRedScratch];
  if (d.ist->done) return;
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31, sub = lane % LPR, grp = lane / LPR;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  float a0 = 0.0f;
  for (int base = gw * RPW; base < n; base += nw * RPW) {
    const int row = base + grp;
    float s = 0.0f;
    if (row < n) {
      const int k1 = __ldg(rowptr + row + 1);
      for (int k = __ldg(rowptr + row) + sub; k < k1; k += LPR) s = fmaf(__ldcs(val + k), __ldg(x + __ldcs(col + k)), s);
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (row < n && sub == 0) {
      y[row] = s;
      if (DOT) a0 = fmaf(x[row], s, a0);
    }
  }
  if (DOT) {
    float v[1] = {a0}, out[1];
    if (grid_sum<1, float>(v, d.partials, d.counter, scratch, out) && threadIdx.x == 0) inner_alpha(d.ist, out[0]);
  }
}

// --------------------------------------------------------------------------
// inner CG vector kernels (FP32) and the outer update
// --------------------------------------------------------------------------

#define IR_FOR_ROWS(i) for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x)
#define IR_FOR_BLOCK_LANES(L)                                                                        \
  const int lane_ = threadIdx.x & 31;                                                                \
  const int bpw_ = 32 / a.bs;                                                                        \
  const int nw_ = (gridDim.x * blockDim.x) >> 5;                                                      \
  for (int w_ = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w_ * bpw_ < a.nblocks; w_ += nw_)      \
    for (BjLane L = bj_lane(w_ * bpw_, lane_, a.bs, a.n, a.nblocks), *once_ = &L; once_; once_ = nullptr)

// r = r64 / ||r64||, d = 0, z = M^{-1} r, p = z, rho = r.z, rr0 = r.r.
template <int PK, int BS>
__global__ void __launch_bounds__(kIrThreads) ir_start_kernel(IrArgs a, IrData d) {
  pdl_wait();
  __shared__ float scratch[kRedScratch];
  const double inv = 1.0 / a.st->rnorm;
  float rz = 0.0f, rr = 0.0f;
  if (PK == PREC_BLOCK) {
    IR_FOR_BLOCK_LANES(L) {
      float rv = 0.0f;
      if (L.active) {
        rv = static_cast<float>(a.r64[L.row] * inv);
        d.r[L.row] = rv;
        d.d[L.row] = 0.0f;
      }
      const float zz = bj_apply32<BS>(d, L, a.bs, rv);
      if (L.active) {
        d.p[L.row] = zz;
        rz = fmaf(rv, zz, rz);
        rr = fmaf(rv, rv, rr);
      }
    }
  } else {
    IR_FOR_ROWS(i) {
      const float rv = static_cast<float>(a.r64[i] * inv);
      d.r[i] = rv;
      d.d[i] = 0.0f;
      const float zv = (PK == PREC_SCALAR) ? d.dinv[i] * rv : rv;
      d.p[i] = zv;
      rz = fmaf(rv, zv, rz);
      rr = fmaf(rv, rv, rr);
    }
  }
  float v[2] = {rz, rr}, out[2];
  if (grid_sum<2, float>(v, d.partials, d.counter, scratch, out) && threadIdx.x == 0) {
    InnerState* s = d.ist;
    s->rho = out[0];
    s->rr0 = out[1];
    // the last inner solve only needs the reduction that is still missing
    const double red = fmax(d.inner_red, 0.5 * a.st->tol / a.st->rnorm);
    s->tol2 = red * red * static_cast<double>(out[1]);
    s->it = 0;
    s->d_it = 0;
    s->max_it = d.inner_max;
    s->breakdown = 0;
    s->done = (out[1] > 0.0f && isfinite(out[1])) ? 0 : 1;
  }
}

// Where d += alpha p happens: with block Jacobi the update kernel is bound
// by its block apply, so d's update goes to the direction kernel, which reads
// p anyway (block-Jacobi refinement on the 27-point matrix 32.9 -> 30.8 ms);
// otherwise it stays in the update kernel (moving it there measured slower).
template <int PK>
struct DInDirection {
  static constexpr bool value = PK == PREC_BLOCK;
};

// [d += alpha p;] r -= alpha q; z = M^{-1} r; (r.z, r.r); inner criteria.
// When the direction kernel updates d, it must know whether this
// iteration's update ran: block 0 first records the iteration count the
// direction kernel last caught up with (before any early return), and the
// finalize raises the count past it only if the update runs.
template <int PK, int BS>
__global__ void __launch_bounds__(kIrThreads) ir_update_kernel(IrArgs a, IrData d) {
  pdl_wait();
  __shared__ float scratch[kRedScratch];
  if (blockIdx.x == 0 && threadIdx.x == 0) d.ist->d_it = d.ist->it;
  if (d.ist->done) return;
  const float alpha = static_cast<float>(d.ist->alpha);
  float rz = 0.0f, rr = 0.0f;
  if (PK == PREC_BLOCK) {
    IR_FOR_BLOCK_LANES(L) {
      float rn = 0.0f;
      if (L.active) {
        if (!DInDirection<PK>::value) d.d[L.row] = fmaf(alpha, d.p[L.row], d.d[L.row]);
        rn = fmaf(-alpha, d.q[L.row], d.r[L.row]);
        d.r[L.row] = rn;
      }
      const float zz = bj_apply32<BS>(d, L, a.bs, rn);
      if (L.active) {
        d.z[L.row] = zz;
        rz = fmaf(rn, zz, rz);
        rr = fmaf(rn, rn, rr);
      }
    }
  } else {
    IR_FOR_ROWS(i) {
      if (!DInDirection<PK>::value) d.d[i] = fmaf(alpha, d.p[i], d.d[i]);
      const float rn = fmaf(-alpha, d.q[i], d.r[i]);
      d.r[i] = rn;
      rr = fmaf(rn, rn, rr);
      if (PK == PREC_SCALAR) rz = fmaf(rn, d.dinv[i] * rn, rz);
    }
    if (PK == PREC_NONE) rz = rr;
  }
  float v[2] = {rz, rr}, out[2];
  if (grid_sum<2, float>(v, d.partials, d.counter, scratch, out) && threadIdx.x == 0) {
    InnerState* s = d.ist;
    s->it += 1;
    const double rrd = out[1];
    if (!isfinite(out[0]) || !isfinite(out[1])) {
      s->done = 1;
      s->breakdown = 1;
    } else if (rrd <= s->tol2 || s->it >= s->max_it) {
      s->done = 1;
    }
    s->beta = static_cast<double>(out[0]) / s->rho;
    s->rho = out[0];
  }
}

// [d += alpha p if this iteration's update ran (it past d_it),] then
// p = z + beta p unless the inner solve is done; re-arms the inner loop.
template <int PK>
__global__ void __launch_bounds__(kIrThreads) ir_direction_kernel(IrArgs a, IrData d) {
  pdl_wait();
  const InnerState* s = d.ist;
  const bool dup = DInDirection<PK>::value && s->it > s->d_it;
  const bool pup = !s->done;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool more = !s->done && s->it < s->max_it + 2;
    if (a.use_cond) cudaGraphSetConditional(a.cond, more ? 1u : 0u);
  }
  if (!dup && !pup) return;
  const float alpha = static_cast<float>(s->alpha), beta = static_cast<float>(s->beta);
  IR_FOR_ROWS(i) {
    const float pv = d.p[i];
    if (dup) d.d[i] = fmaf(alpha, pv, d.d[i]);
    if (pup) {
      float zv;
      if (PK == PREC_BLOCK) zv = d.z[i];
      else if (PK == PREC_SCALAR) zv = d.dinv[i] * d.r[i];
      else zv = d.r[i];
      d.p[i] = fmaf(beta, pv, zv);
    }
  }
}

// x += ||r|| d in FP64; bookkeeping of the outer step.
__global__ void __launch_bounds__(kIrThreads) ir_apply_kernel(IrArgs a, IrData d) {
  const double scale = a.st->rnorm;
  IR_FOR_ROWS(i) a.x[i] = fma(scale, static_cast<double>(d.d[i]), a.x[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    SolverState* st = a.st;
    const InnerState* s = d.ist;
    st->outer += 1;
    st->iter += s->it;
    st->spmvs += s->it;
    if (s->it == 0 || (s->breakdown && s->it <= 1)) st->stop = GK_STOP_BREAKDOWN;
  }
}

__global__ void ir_init_kernel(SolverState* st, double factor, long long max_iters, int rel_to_b,
                               unsigned long long time_limit_ns) {
  SolverState z;
  memset(&z, 0, sizeof(z));
  z.factor = factor;
  z.max_iters = max_iters;
  z.rel_to_b = rel_to_b;
  z.time_limit_ns = time_limit_ns;
  *st = z;
}

#undef IR_FOR_ROWS
#undef IR_FOR_BLOCK_LANES

IrArgs ir_args(const Solver& S, const IrData& d) {
  IrArgs a;
  const Matrix& A = *S.A;
  a.n = static_cast<int>(S.n);
  a.rowptr = A.rowptr;
  a.col = A.col;
  a.ell_col = A.ell_col;
  a.ld = A.ld;
  a.K = static_cast<int>(A.K);
  a.tail_rowptr = A.tail_rowptr;
  a.tail_slot = A.tail_slot;
  a.m_tail = static_cast<int>(A.m_tail);
  a.bs = S.P ? S.P->bs : 1;
  a.nblocks = S.P ? static_cast<int>(S.P->nblocks) : 0;
  a.x = S.x;
  a.r64 = S.r;
  a.st = S.st;
  a.cond = d.cond;
  a.use_cond = 1;
  return a;
}

int lanes_per_row(double mean) {
  int l = 1;
  while (l < 32 && l < mean * 0.5) l <<= 1;
  return l;
}

template <bool DOT>
void launch_csr32(int lpr, int grid, cudaStream_t s, const int32_t* rowptr, const int32_t* col, const float* val,
                  int n, const IrData& d, const float* x, float* y) {
  switch (lpr) {
    case 1: launch_pdl(ir_spmv_csr_kernel<1, DOT>, grid, kIrThreads, 0, s, rowptr, col, val, n, d, x, y); break;
    case 2: launch_pdl(ir_spmv_csr_kernel<2, DOT>, grid, kIrThreads, 0, s, rowptr, col, val, n, d, x, y); break;
    case 4: launch_pdl(ir_spmv_csr_kernel<4, DOT>, grid, kIrThreads, 0, s, rowptr, col, val, n, d, x, y); break;
    case 8: launch_pdl(ir_spmv_csr_kernel<8, DOT>, grid, kIrThreads, 0, s, rowptr, col, val, n, d, x, y); break;
    case 16: launch_pdl(ir_spmv_csr_kernel<16, DOT>, grid, kIrThreads, 0, s, rowptr, col, val, n, d, x, y); break;
    default: launch_pdl(ir_spmv_csr_kernel<32, DOT>, grid, kIrThreads, 0, s, rowptr, col, val, n, d, x, y); break;
  }
}

// q = A32 p with sigma = p.q (-> alpha).
int ir_spmv(const Solver& S, const IrData& d, const IrArgs& a, cudaStream_t s) {
  const Matrix& A = *S.A;
  if (d.fmt == GK_ELL) {
    const bool tail = A.format == GK_HYB && A.m_tail > 0;
    const Ell32 e32{A.ell_col, d.ell_val32, A.ld, static_cast<int>(A.K), a.n, A.tail_slot, d.tail_sum32,
                    d.ist, d.partials, d.counter};
    if (tail) {
      launch_csr32<false>(d.tail_lpr, d.grid, s, A.tail_rowptr, A.tail_col, d.tail_val32,
                          static_cast<int>(A.m_tail), d, d.p, d.tail_sum32);
      launch_pdl(ir_spmv_ell_kernel<true, true>, d.grid, kIrThreads, 0, s, e32, d.p, d.q);
    } else {
      launch_pdl(ir_spmv_ell_kernel<false, true>, d.grid, kIrThreads, 0, s, e32, d.p, d.q);
    }
  } else {
    launch_csr32<true>(d.lpr, d.grid, s, A.rowptr, A.col, d.val32, a.n, d, d.p, d.q);
  }
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

// Block-Jacobi kernels with the block size as a template argument where it
// is one of the common sizes (vectorised, unrolled apply), else generic.
#define IR_LAUNCH_BS(kern, bs, grid, s, a, d)                                      \
  do {                                                                             \
    switch (bs) {                                                                  \
      case 4: launch_pdl(kern<PREC_BLOCK, 4>, grid, kIrThreads, 0, s, a, d); break;       \
      case 8: launch_pdl(kern<PREC_BLOCK, 8>, grid, kIrThreads, 0, s, a, d); break;       \
      case 16: launch_pdl(kern<PREC_BLOCK, 16>, grid, kIrThreads, 0, s, a, d); break;     \
      case 32: launch_pdl(kern<PREC_BLOCK, 32>, grid, kIrThreads, 0, s, a, d); break;     \
      default: launch_pdl(kern<PREC_BLOCK, 0>, grid, kIrThreads, 0, s, a, d); break;      \
    }                                                                              \
  } while (0)


// The inner solve and the update of x as one graph:
// start -> WHILE(cond) { SpMV; update; direction } -> apply.
int ir_enqueue_start(const Solver& S, const IrData& d, const IrArgs& a, cudaStream_t s) {
  if (S.pk == PREC_BLOCK) IR_LAUNCH_BS(ir_start_kernel, a.bs, d.grid, s, a, d);
  else if (S.pk == PREC_SCALAR) launch_pdl(ir_start_kernel<PREC_SCALAR, 0>, d.grid, kIrThreads, 0, s, a, d);
  else launch_pdl(ir_start_kernel<PREC_NONE, 0>, d.grid, kIrThreads, 0, s, a, d);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

// One inner CG iteration: FP32 SpMV (with p.q), update, direction.
int ir_enqueue_inner(const Solver& S, const IrData& d, const IrArgs& a, cudaStream_t s) {
  GK_TRY(ir_spmv(S, d, a, s));
  if (S.pk == PREC_BLOCK) {
    IR_LAUNCH_BS(ir_update_kernel, a.bs, d.grid, s, a, d);
    launch_pdl(ir_direction_kernel<PREC_BLOCK>, d.grid, kIrThreads, 0, s, a, d);
  } else if (S.pk == PREC_SCALAR) {
    launch_pdl(ir_update_kernel<PREC_SCALAR, 0>, d.grid, kIrThreads, 0, s, a, d);
    launch_pdl(ir_direction_kernel<PREC_SCALAR>, d.grid, kIrThreads, 0, s, a, d);
  } else {
    launch_pdl(ir_update_kernel<PREC_NONE, 0>, d.grid, kIrThreads, 0, s, a, d);
    launch_pdl(ir_direction_kernel<PREC_NONE>, d.grid, kIrThreads, 0, s, a, d);
  }
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

int ir_build_graph(Solver& S, IrData& d) {
  if (!d.cs) GK_TRY_CUDA(cudaStreamCreateWithFlags(&d.cs, cudaStreamNonBlocking));
  GK_TRY_CUDA(cudaGraphCreate(&d.graph, 0));
  GK_TRY_CUDA(cudaGraphConditionalHandleCreate(&d.cond, d.graph, 1, cudaGraphCondAssignDefault));
  const IrArgs a = ir_args(S, d);
  GK_TRY_CUDA(cudaStreamBeginCaptureToGraph(d.cs, d.graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int rc = GK_OK;
  do {
    rc = ir_enqueue_start(S, d, a, d.cs);
    if (rc != GK_OK) break;
    cudaError_t e = cudaSuccess;
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
      rc = cuda_error(e, "refinement graph");
      break;
    }
    ir_apply_kernel<<<d.grid, kIrThreads, 0, d.cs>>>(a, d);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = cuda_error(e, "refinement graph");
      break;
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(d.cs, &captured);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    cudaGraph_t body = np.conditional.phGraph_out[0];
    GK_TRY_CUDA(cudaStreamBeginCaptureToGraph(d.cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    // kGraphUnroll inner iterations per pass of the body (those after the
    // inner stop do nothing): fewer turn-arounds of the loop
    int brc = GK_OK;
    for (int u = 0; u < kGraphUnroll && brc == GK_OK; ++u) brc = ir_enqueue_inner(S, d, a, d.cs);
    e = cudaStreamEndCapture(d.cs, &captured);
    if (brc != GK_OK) return brc;
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture (inner body)");
    GK_TRY_CUDA(cudaGraphInstantiate(&d.exec, d.graph, 0));
    return GK_OK;
  } while (false);
  cudaGraph_t g2 = nullptr;
  cudaStreamEndCapture(d.cs, &g2);
  return rc;
}

int fgrid(int64_t n) {
  const int64_t g = (n + kIrThreads - 1) / kIrThreads;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, 8 * sm_count())));
}

}  // namespace

void ir_release(IrData* d) {
  if (!d) return;
  if (d->exec) cudaGraphExecDestroy(d->exec);
  if (d->graph) cudaGraphDestroy(d->graph);
  if (d->cs) cudaStreamDestroy(d->cs);
  void* ptrs[] = {d->val32, d->ell_val32, d->tail_val32, d->tail_sum32, d->r, d->p, d->q, d->z, d->d,
                  d->dinv, d->blk16, d->blk32, d->prec, d->bscale, d->ist, d->partials, d->counter};
  for (void* p : ptrs) dfree(p);
  delete d;
}

int ir_generate(Solver* S) {
  IrData* d = new IrData;
  S->ir = d;
  const Matrix& A = *S->A;
  const int64_t n = S->n;
  int64_t* by = &d->bytes;
  cudaStream_t s = nullptr;
  d->inner_red = S->crit.inner_reduction > 0 ? S->crit.inner_reduction : 1e-5;
  d->inner_max = S->crit.inner_max_iters > 0 ? S->crit.inner_max_iters : std::max<int64_t>(S->crit.max_iters, 1);
  d->grid = fgrid(n);
  // FP32 operator copy
  if (A.format == GK_ELL || A.format == GK_HYB) {
    d->fmt = GK_ELL;
    const int64_t slots = std::max<int64_t>(A.K * A.ld, 1);
    GK_TRY(dalloc_n(&d->ell_val32, static_cast<size_t>(slots), by));
    to_float_kernel<<<fgrid(slots), kIrThreads, 0, s>>>(A.ell_val, d->ell_val32, A.K * A.ld);
    if (A.format == GK_HYB && A.m_tail > 0) {
      GK_TRY(dalloc_n(&d->tail_val32, static_cast<size_t>(A.tail_nnz + 1), by));
      GK_TRY(dalloc_n(&d->tail_sum32, static_cast<size_t>(A.m_tail + 1), by));
      to_float_kernel<<<fgrid(A.tail_nnz), kIrThreads, 0, s>>>(A.tail_val, d->tail_val32, A.tail_nnz);
      d->tail_lpr = lanes_per_row(static_cast<double>(A.tail_nnz) / static_cast<double>(A.m_tail));
    }
  } else {
    d->fmt = GK_CSR;
    GK_TRY(dalloc_n(&d->val32, static_cast<size_t>(A.nnz + 1), by));
    to_float_kernel<<<fgrid(A.nnz), kIrThreads, 0, s>>>(A.val, d->val32, A.nnz);
    d->lpr = lanes_per_row(n > 0 ? static_cast<double>(A.nnz) / static_cast<double>(n) : 1.0);
  }
  GK_TRY_CUDA(cudaGetLastError());
  // inner vectors
  for (float** v : {&d->r, &d->p, &d->q, &d->d}) GK_TRY(dalloc_n(v, static_cast<size_t>(n + 1), by));
  // preconditioner copy
  if (S->pk == PREC_SCALAR) {
    GK_TRY(dalloc_n(&d->dinv, static_cast<size_t>(n + 1), by));
    to_float_kernel<<<fgrid(n), kIrThreads, 0, s>>>(S->P->dinv, d->dinv, n);
    GK_TRY_CUDA(cudaGetLastError());
  } else if (S->pk == PREC_BLOCK) {
    const Precond& P = *S->P;
    GK_TRY(dalloc_n(&d->z, static_cast<size_t>(n + 1), by));
    const size_t el = static_cast<size_t>(std::max<int64_t>(P.block_elems, 1));
    GK_TRY(dalloc_n(&d->blk16, el, by));
    GK_TRY(dalloc_n(&d->blk32, el, by));
    GK_TRY(dalloc_n(&d->prec, static_cast<size_t>(P.nblocks + 1), by));
    GK_TRY(dalloc_n(&d->bscale, static_cast<size_t>(P.nblocks + 1), by));
    if (P.nblocks > 0) {
      const int64_t g = std::min<int64_t>((P.nblocks + 3) / 4, 16 * static_cast<int64_t>(sm_count()));
      bj_adapt_kernel<<<static_cast<int>(g), 128, 0, s>>>(A.rowptr, A.col, A.val, P.blocks, static_cast<int>(n),
                                                           P.bs, static_cast<int>(P.nblocks), d->blk16, d->blk32,
                                                           d->prec, d->bscale);
      GK_TRY_CUDA(cudaGetLastError());
      std::vector<uint8_t> h(static_cast<size_t>(P.nblocks));
      GK_TRY_CUDA(cudaMemcpy(h.data(), d->prec, h.size(), cudaMemcpyDeviceToHost));
      for (uint8_t v : h) (v == 0 ? d->n16 : d->n32) += 1;
    }
  }
  GK_TRY(dalloc_n(&d->ist, 1, by));
  GK_TRY(dalloc_n(&d->partials, static_cast<size_t>(2 * d->grid + 2), by));
  GK_TRY(dalloc_n(&d->counter, 1, by));
  GK_TRY_CUDA(cudaMemset(d->counter, 0, sizeof(unsigned int)));
  GK_TRY_CUDA(cudaMemset(d->ist, 0, sizeof(InnerState)));
  GK_TRY_CUDA(cudaDeviceSynchronize());
  S->device_bytes += d->bytes;
  return GK_OK;
}

int ir_solve(Solver* S, cudaStream_t s) {
  IrData& d = *S->ir;
  const bool host_loop = S->crit.check_every > 0;
  if (!host_loop && !d.exec) GK_TRY(ir_build_graph(*S, d));
  const gk_criteria& c = S->crit;
  const unsigned long long tl = c.time_limit_s > 0 ? static_cast<unsigned long long>(c.time_limit_s * 1e9) : 0ull;
  ir_init_kernel<<<1, 1, 0, s>>>(S->st, c.reduction_factor, static_cast<long long>(c.max_iters), c.rel_to_b, tl);
  GK_TRY_CUDA(cudaGetLastError());
  Epi e;
  e.mode = EPI_RESID;
  e.fin = FIN_IR_RESID;
  e.u = S->b;
  e.y = S->r;
  e.st = S->st;
  e.skip_mode = 0;
  e.partials = S->partials;
  e.counter = S->counter;
  e.err = &S->st->err;
  // inner iterations launched beyond those done: whole passes of the graph's
  // loop body, or whole groups of check_every in the host loop
  S->ir_idle = 0;
  long long prev_iter = 0;
  int64_t launched = -1;  // by the inner solve just finished
  for (int outer = 0;; ++outer) {
    GK_TRY(spmv_launch(*S->A, S->x, e, s));
    GK_TRY_CUDA(cudaMemcpyAsync(S->h_st, S->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    GK_TRY_CUDA(cudaStreamSynchronize(s));
    if (outer > 0) {
      const int64_t inner = S->h_st->iter - prev_iter;
      if (launched < 0) launched = kGraphUnroll * std::max<int64_t>(1, (inner + kGraphUnroll - 1) / kGraphUnroll);
      S->ir_idle += std::max<int64_t>(launched - inner, 0);
    }
    prev_iter = S->h_st->iter;
    launched = -1;
    if (S->h_st->stop != GK_STOP_NONE) break;
    if (outer >= kMaxOuter) {
      const int stop = GK_STOP_MAX_ITERS;
      GK_TRY_CUDA(cudaMemcpyAsync(&S->st->stop, &stop, sizeof(int), cudaMemcpyHostToDevice, s));
      break;
    }
    if (!host_loop) {
      GK_TRY_CUDA(cudaGraphLaunch(d.exec, s));
      continue;
    }
    // the inner solve launched from the host, its state read every
    // check_every iterations (same kernels as the graph's loop body)
    IrArgs a = ir_args(*S, d);
    a.use_cond = 0;
    GK_TRY(ir_enqueue_start(*S, d, a, s));
    int64_t done = 0;
    for (;;) {
      for (int i = 0; i < S->crit.check_every; ++i) GK_TRY(ir_enqueue_inner(*S, d, a, s));
      done += S->crit.check_every;
      InnerState h;
      GK_TRY_CUDA(cudaMemcpyAsync(&h, d.ist, sizeof(InnerState), cudaMemcpyDeviceToHost, s));
      GK_TRY_CUDA(cudaStreamSynchronize(s));
      if (h.done || h.it >= h.max_it + 2 || done > h.max_it + 2) break;
    }
    launched = done;
    ir_apply_kernel<<<d.grid, kIrThreads, 0, s>>>(a, d);
    GK_TRY_CUDA(cudaGetLastError());
  }
  return GK_OK;
}

}  // namespace gk

using namespace gk;

extern "C" int gk_solver_get_info(gk_solver h, gk_solver_info* info) {
  Solver* S = reinterpret_cast<Solver*>(h);
  if (!S || !info) return set_error(GK_ERR_ARG, "gk_solver_get_info: NULL argument");
  memset(info, 0, sizeof(*info));
  info->kind = S->kind;
  info->n = S->n;
  info->device_bytes = S->device_bytes;
  if (S->ir) {
    info->inner_format = S->ir->fmt;
    info->inner_fp16_blocks = S->ir->n16;
    info->inner_fp32_blocks = S->ir->n32;
  }
  return GK_OK;
}
