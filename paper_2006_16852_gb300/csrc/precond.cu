// precond.cu -- Jacobi preconditioners (Section 3.2): scalar diagonal scaling
// and block Jacobi whose diagonal blocks are inverted by Gauss-Jordan
// elimination with partial pivoting (Section 7.5): one thread per block, in
// registers, up to block size 8 (after a row-parallel extraction); one lane
// group of a warp per block, in shared memory, above.
#include <algorithm>
#include <climits>
#include <memory>

#include "gk_device.cuh"
#include "gk_internal.h"
#include "precond_device.cuh"

namespace gk {

namespace {

// First index k in [lo, hi) with col[k] >= c (hi if none); the columns of a
// row are sorted.
__device__ __forceinline__ int lower_col(const int32_t* __restrict__ col, int lo, int hi, int c) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(col + mid) < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Narrows [lo, hi) to at most P entries while keeping the first index k with
// col[k] >= c inside [lo, hi] (the columns of a row are sorted).  Each round
// probes P evenly spaced positions whose loads are independent, so a round
// costs one memory latency and shrinks the range about P + 1 times (a
// binary search pays one latency per halving).
template <int P>
__device__ __forceinline__ void narrow_col(const int32_t* __restrict__ col, int& lo, int& hi, int c) {
  while (hi - lo > P) {
    const int step = (hi - lo) / (P + 1);
    int below = 0;  // the probes are sorted: those below c are a prefix
#pragma unroll
    for (int j = 0; j < P; ++j) below += __ldg(col + lo + (j + 1) * step) < c ? 1 : 0;
    const int nlo = below > 0 ? lo + below * step + 1 : lo;
    if (below < P) hi = lo + (below + 1) * step;
    lo = nlo;
  }
}

constexpr int kNarrow = 8;  // probes per round of narrow_col

__global__ void jacobi_scalar_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                     const double* __restrict__ val, int n, double* dinv, int* bad) {
  const int stride = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    double d = 0.0;
    const int k1 = __ldg(rowptr + r + 1);
    int lo = __ldg(rowptr + r), hi = k1;
    narrow_col<kNarrow>(col, lo, hi, r);
    // the diagonal, if present, is the entry at the first index >= lo with
    // column >= r, which lies in [lo, hi]: the window's columns loaded together
    int at = -1;
#pragma unroll
    for (int j = 0; j <= kNarrow; ++j)
      if (lo + j <= hi && lo + j < k1 && __ldg(col + lo + j) == r) at = lo + j;
    const bool found = at >= 0;
    if (found) d = __ldg(val + at);
    if (!found || d == 0.0) {
      atomicMin(bad, r);
      dinv[r] = 0.0;
    } else {
      dinv[r] = 1.0 / d;
    }
  }
}

// Pivot key of a candidate |w|: the magnitude's bit pattern, which orders
// like |w| for every non-NaN value.  A NaN candidate never wins (-1), and a
// NaN on the diagonal is never displaced (the largest key): the strict
// comparison "a > best" of the elimination takes no NaN.
__device__ __forceinline__ long long piv_key(double w, bool diag) {
  const long long b = __double_as_longlong(w) & 0x7fffffffffffffffll;
  if (b > 0x7ff0000000000000ll) return diag ? 0x7fffffffffffffffll : -1ll;
  return b;
}

// Small blocks (bs <= 8) in two launches.
//
// bj_extract_kernel: one thread per row writes that row of its dense
// diagonal block (row-major, zeros where A has no entry) into the output
// array: its entries inside the block are a contiguous run of the sorted
// columns, found by a binary search for the first column >= the block's
// first row.  Few registers, full occupancy: the searches' load latency is
// hidden by other warps.
template <int BT>
__global__ void __launch_bounds__(256) bj_extract_kernel(const int32_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col,
                                                         const double* __restrict__ val, int n, int bs,
                                                         double* blocks) {
  const int stride = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const int blk = r / bs, i = r - blk * bs, r0 = blk * bs;
    const int m = min(bs, n - r0);
    const int k1 = __ldg(rowptr + r + 1);
    int lo = __ldg(rowptr + r), hi = k1;
    narrow_col<kNarrow>(col, lo, hi, r0);
    // the run inside the block starts at an index in [lo, hi] and holds at
    // most m entries: the window [lo, min(hi + m, k1)) covers it.  Its
    // columns are loaded together; s counts those left of the block.
    const int kend = min(hi + m, k1);
    int s = 0, cnt = 0;
#pragma unroll
    for (int j = 0; j < kNarrow + BT; ++j) {
      const int c = lo + j < kend ? __ldg(col + lo + j) - r0 : m;
      s += c < 0 ? 1 : 0;
      cnt += (c >= 0 && c < m) ? 1 : 0;
    }
    // the run [lo + s, lo + s + cnt): columns (again, from L1) and values
    int cc[BT];
#pragma unroll
    for (int j = 0; j < BT; ++j) cc[j] = j < cnt ? __ldg(col + lo + s + j) - r0 : BT;
    double vv[BT];
#pragma unroll
    for (int j = 0; j < BT; ++j) vv[j] = j < cnt ? __ldg(val + lo + s + j) : 0.0;
    // the row of the dense block: zeros, then the entries at their columns
    // (the same 8 * m bytes, merged in L2 before they reach memory)
    double* out = blocks + static_cast<int64_t>(blk) * bs * bs + static_cast<int64_t>(i) * m;
#pragma unroll
    for (int j = 0; j < BT; ++j)
      if (j < m) out[j] = 0.0;
#pragma unroll
    for (int j = 0; j < BT; ++j)
      if (cc[j] < m) out[cc[j]] = vv[j];
  }
}

// bj_invert_kernel: one thread per diagonal block, the block in registers
// (BT = 2, 4 or 8: the largest block this instantiation takes).  A thread
// block takes kBjRegThreads consecutive blocks: they are one contiguous run
// of the output array, loaded and stored coalesced through shared memory
// (element-major, block-minor, odd stride) and inverted in place there.
// The elimination is the Gauss-Jordan of [D | I] with partial pivoting,
// stored in place: once column k of the left half is eliminated it holds
// nothing (the unit vector e_k), so its registers take the right-half
// column that becomes non-zero at step k -- the identity column of the row
// that is pivot row k (orig[k]).  Every stored entry receives exactly the
// operations of the augmented elimination (the pivot row scaled by the
// reciprocal of the pivot, w_ij = fma(-w_ik, w_kj, w_ij) for the other
// rows); the only operations left out act on entries that are structurally
// zero and leave them zero.  Rows are exchanged by selects with static
// register indices (the pivot row index is data, the loop indices are not).
// The FP64 pipe bounds this kernel: about bs^3 fused multiply-adds and bs
// divisions per block, each with all 32 lanes of a warp busy.
constexpr int kBjRegThreads = 128;
constexpr int kBjLds = kBjRegThreads + 1;

// a / d for 0 <= a < 2^16 and 1 <= d <= 64 through a float reciprocal:
// (a + 0.5) / d lies at least 1/128 from an integer and the float product
// errs by under 2^-7 of that, so the truncation is exact (an integer division
// would cost tens of instructions per element).
__device__ __forceinline__ int div_small(int a, float inv_d) {
  return static_cast<int>((static_cast<float>(a) + 0.5f) * inv_d);
}

template <int BT>
__global__ void __launch_bounds__(kBjRegThreads) bj_invert_kernel(int n, int bs, int nblocks, double* blocks,
                                                                  int* bad) {
  extern __shared__ double S[];  // [BT * BT][kBjLds]
  const int bs2 = bs * bs;
  const int last_m = n - (nblocks - 1) * bs;
  const float inv_bs2 = 1.0f / static_cast<float>(bs2), inv_bs = 1.0f / static_cast<float>(bs);
  const float inv_last = 1.0f / static_cast<float>(last_m);
  for (int blk0 = blockIdx.x * kBjRegThreads; blk0 < nblocks; blk0 += gridDim.x * kBjRegThreads) {
    const int nb = min(kBjRegThreads, nblocks - blk0);
    const int64_t base = static_cast<int64_t>(blk0) * bs2;
    const int len = (nb - 1) * bs2 + (blk0 + nb == nblocks ? last_m * last_m : bs2);  // <= 128 * 64
    __syncthreads();  // the previous run's stores have read S
    for (int o = threadIdx.x; o < len; o += kBjRegThreads) {
      const int b = div_small(o, inv_bs2), e = o - b * bs2;
      const bool lastb = blk0 + b == nblocks - 1;
      const int mb = lastb ? last_m : bs;
      const int i = div_small(e, lastb ? inv_last : inv_bs), j = e - i * mb;
      S[(i * BT + j) * kBjLds + b] = __ldcs(blocks + base + o);
    }
    __syncthreads();
    const int b = threadIdx.x;
    if (b < nb) {
      const int blk = blk0 + b;
      const int m = min(bs, n - blk * bs);
      double A[BT][BT];
      int orig[BT];
#pragma unroll
      for (int i = 0; i < BT; ++i) {
        orig[i] = i;
#pragma unroll
        for (int j = 0; j < BT; ++j) A[i][j] = (i < m && j < m) ? S[(i * BT + j) * kBjLds + b] : 0.0;
      }
      bool singular = false;
#pragma unroll
      for (int k = 0; k < BT; ++k) {
        if (k < m && !singular) {
          // pivot: largest |A[i][k]|, i in [k, m), lowest row on ties
          long long best = piv_key(A[k][k], true);
          int piv = k;
#pragma unroll
          for (int i = k + 1; i < BT; ++i) {
            const long long a = piv_key(A[i][k], false);
            if (i < m && a > best) {
              best = a;
              piv = i;
            }
          }
          if (best == 0) {
            singular = true;
          } else {
#pragma unroll
            for (int i = k + 1; i < BT; ++i) {
              const bool sw = i == piv;
#pragma unroll
              for (int j = 0; j < BT; ++j) {
                const double t = A[k][j];
                A[k][j] = sw ? A[i][j] : t;
                A[i][j] = sw ? t : A[i][j];
              }
              const int t = orig[k];
              orig[k] = sw ? orig[i] : t;
              orig[i] = sw ? t : orig[i];
            }
            const double rcp = 1.0 / A[k][k];
#pragma unroll
            for (int j = 0; j < BT; ++j)
              if (j != k) A[k][j] = A[k][j] * rcp;
            A[k][k] = rcp;  // right-half column orig[k]: 1 * rcp
#pragma unroll
            for (int i = 0; i < BT; ++i) {
              if (i != k && i < m) {
                const double f = A[i][k];
#pragma unroll
                for (int j = 0; j < BT; ++j)
                  if (j != k) A[i][j] = fma(-f, A[k][j], A[i][j]);
                A[i][k] = fma(-f, rcp, 0.0);
              }
            }
          }
        }
      }
      if (singular) atomicMin(bad, blk);
      // inverse(i, orig[k]) = A[i][k]
#pragma unroll
      for (int i = 0; i < BT; ++i)
#pragma unroll
        for (int k = 0; k < BT; ++k)
          if (i < m && k < m) S[(i * BT + orig[k]) * kBjLds + b] = A[i][k];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < len; o += kBjRegThreads) {
      const int bb = div_small(o, inv_bs2), e = o - bb * bs2;
      const bool lastb = blk0 + bb == nblocks - 1;
      const int mb = lastb ? last_m : bs;
      const int i = div_small(e, lastb ? inv_last : inv_bs), j = e - i * mb;
      blocks[base + o] = S[(i * BT + j) * kBjLds + bb];
    }
  }
}

// Gauss-Jordan inversion of the diagonal blocks on the augmented matrices
// [D | I] held in shared memory (block sizes above 8).  A warp inverts 32/GW blocks at once, one
// group of GW lanes (GW = the next power of two >= the block size) per
// block, lane i owning row i; each block's tile has an odd row stride
// (2 GW + 1 doubles) so column accesses are conflict-free.
// Pivot: largest |entry| in column k at or below row k, lowest row on ties
// (xor butterfly over piv_key inside the group).  The pivot row is scaled by the
// reciprocal of the pivot and every other row i is updated
// w_ij = fma(-w_ik, w_kj, w_ij).  Columns left of and at k are never read
// again once step k is done, so only columns j > k are updated: the right
// half (the inverse) receives exactly the operations of the full elimination.
constexpr int kBjWarps = 4;

template <int GW>
__global__ void __launch_bounds__(kBjWarps * 32) bj_generate_kernel(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const double* __restrict__ val,
    int n, int bs, int nblocks, double* blocks, int* bad) {
  extern __shared__ double bj_smem[];
  constexpr int G = 32 / GW;
  constexpr int LD = 2 * GW + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / GW, i = lane - grp * GW;
  double* W = bj_smem + (warp * G + grp) * GW * LD;
  const int step_blocks = gridDim.x * kBjWarps * G;
  for (int blk0 = (blockIdx.x * kBjWarps + warp) * G; blk0 < nblocks; blk0 += step_blocks) {
    const int blk = blk0 + grp;
    const int r0 = blk * bs;
    const int m = blk < nblocks ? min(bs, n - r0) : 0;
    const int wd = 2 * m;
    for (int idx = i; idx < GW * LD; idx += GW) W[idx] = 0.0;
    __syncwarp();
    if (i < m) {
      // the row's entries inside the block: a contiguous run of the sorted
      // columns, found by a binary search for the first column >= r0
      const int r = r0 + i;
      const int k1 = __ldg(rowptr + r + 1);
      for (int k = lower_col(col, __ldg(rowptr + r), k1, r0); k < k1; ++k) {
        const int c = __ldg(col + k) - r0;
        if (c >= m) break;
        W[i * LD + c] = __ldg(val + k);
      }
      W[i * LD + m + i] = 1.0;
    }
    __syncwarp();
    bool singular = false;
    for (int k = 0; k < bs; ++k) {
      const bool live = k < m && !singular;
      long long a = (live && i >= k && i < m) ? piv_key(W[i * LD + k], i == k) : -2ll;
      int idx = i;
#pragma unroll
      for (int o = GW / 2; o > 0; o >>= 1) {
        const long long a2 = __shfl_xor_sync(0xffffffffu, a, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (a2 > a || (a2 == a && i2 < idx)) {
          a = a2;
          idx = i2;
        }
      }
      if (live && a == 0) singular = true;
      const bool work = live && !singular;
      const int piv = idx;
      __syncwarp();
      if (work && piv != k) {
        for (int j = k + i; j < wd; j += GW) {
          const double t = W[k * LD + j];
          W[k * LD + j] = W[piv * LD + j];
          W[piv * LD + j] = t;
        }
      }
      __syncwarp();
      const double rcp = work ? 1.0 / W[k * LD + k] : 0.0;
      __syncwarp();
      if (work)
        for (int j = k + 1 + i; j < wd; j += GW) W[k * LD + j] = W[k * LD + j] * rcp;
      __syncwarp();
      if (work && i < m && i != k) {
        const double f = W[i * LD + k];
        for (int j = k + 1; j < wd; ++j) W[i * LD + j] = fma(-f, W[k * LD + j], W[i * LD + j]);
      }
      __syncwarp();
    }
    if (singular && i == 0) atomicMin(bad, blk);
    const int64_t off = static_cast<int64_t>(blk) * bs * bs;
    for (int e = i; e < m * m; e += GW) {  // row-major: e = ii * m + j
      const int ii = e / m, j = e - ii * m;
      blocks[off + e] = W[ii * LD + m + j];
    }
    __syncwarp();
  }
}

template <int GW>
int launch_bj_generate(const Matrix* A, int n, int bs, int nblocks, double* blocks, int* bad, cudaStream_t s) {
  const size_t smem = sizeof(double) * static_cast<size_t>(kBjWarps) * 32 * (2 * GW + 1);
  GK_TRY(set_smem(bj_generate_kernel<GW>, smem));
  const int64_t warps = (nblocks + (32 / GW) - 1) / (32 / GW);
  const int64_t g = std::min<int64_t>((warps + kBjWarps - 1) / kBjWarps, 16 * static_cast<int64_t>(sm_count()));
  bj_generate_kernel<GW><<<static_cast<int>(std::max<int64_t>(g, 1)), kBjWarps * 32, smem, s>>>(
      A->rowptr, A->col, A->val, n, bs, nblocks, blocks, bad);
  return GK_OK;
}

template <int BT>
int launch_bj_generate_reg(const Matrix* A, int n, int bs, int nblocks, double* blocks, int* bad,
                           cudaStream_t s) {
  const int64_t ge = std::min<int64_t>((n + 255) / 256, 16 * static_cast<int64_t>(sm_count()));
  bj_extract_kernel<BT><<<static_cast<int>(std::max<int64_t>(ge, 1)), 256, 0, s>>>(A->rowptr, A->col, A->val, n,
                                                                                   bs, blocks);
  const size_t smem = sizeof(double) * BT * BT * kBjLds;
  GK_TRY(set_smem(bj_invert_kernel<BT>, smem));
  // resident blocks per SM: registers allow 8 at block sizes up to 4 (64 per
  // thread), 2 at 8 (190 per thread); the grid is capped at 8 and 4
  const int64_t g = std::min<int64_t>((nblocks + kBjRegThreads - 1) / kBjRegThreads,
                                      (BT <= 4 ? 8 : 4) * static_cast<int64_t>(sm_count()));
  bj_invert_kernel<BT><<<static_cast<int>(std::max<int64_t>(g, 1)), kBjRegThreads, smem, s>>>(n, bs, nblocks,
                                                                                               blocks, bad);
  return GK_OK;
}

int bj_generate(const Matrix* A, int n, int bs, int nblocks, double* blocks, int* bad, cudaStream_t s) {
  if (bs <= 2) return launch_bj_generate_reg<2>(A, n, bs, nblocks, blocks, bad, s);
  if (bs <= 4) return launch_bj_generate_reg<4>(A, n, bs, nblocks, blocks, bad, s);
  if (bs <= 8) return launch_bj_generate_reg<8>(A, n, bs, nblocks, blocks, bad, s);
  if (bs <= 16) return launch_bj_generate<16>(A, n, bs, nblocks, blocks, bad, s);
  return launch_bj_generate<32>(A, n, bs, nblocks, blocks, bad, s);
}

__global__ void scalar_apply_kernel(const double* __restrict__ dinv, const double* __restrict__ r, double* z,
                                    int64_t n) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    z[i] = dinv[i] * r[i];
}

template <int BS>
__global__ void bj_apply_kernel(const double* __restrict__ blocks, int n, int bs, int nblocks,
                                const double* __restrict__ r, double* z) {
  const int lane = threadIdx.x & 31;
  const int bpw = 32 / bs;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * bpw < nblocks; w += nw) {
    const BjLane L = bj_lane(w * bpw, lane, bs, n, nblocks);
    const double rm = L.active ? r[L.row] : 0.0;
    const double zz = bj_apply_lane<BS>(blocks, L, bs, rm);
    if (L.active) z[L.row] = zz;
  }
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, 8 * sm_count())));
}

struct PrecondDeleter {
  void operator()(Precond* p) const { precond_release(p); }
};

}  // namespace

int64_t bj_total_elems(int64_t n, int bs) {
  if (n == 0) return 0;
  int64_t full = n / bs, last = n % bs;
  return full * bs * bs + last * last;
}

void precond_release(Precond* P) {
  if (!P) return;
  if (P->refs.fetch_sub(1) != 1) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  dfree(P->dinv);
  dfree(P->blocks);
  dfree(P->stage_in);
  dfree(P->stage_out);
  matrix_release(P->A);
  if (prev >= 0) cudaSetDevice(prev);
  delete P;
}

int precond_apply_launch(const Precond* P, const double* r, double* z, cudaStream_t s) {
  if (P->n == 0) return GK_OK;
  if (P->bs == 1) {
    scalar_apply_kernel<<<grid_for(P->n, 256), 256, 0, s>>>(P->dinv, r, z, P->n);
  } else {
    const int bpw = 32 / P->bs;
    const int64_t warps = (P->nblocks + bpw - 1) / bpw;
#define GK_BJ_APPLY(BS)                                                                                   \
  bj_apply_kernel<BS><<<grid_for(warps * 32, 256), 256, 0, s>>>(P->blocks, static_cast<int>(P->n), P->bs, \
                                                                static_cast<int>(P->nblocks), r, z)
    GK_BJ_DISPATCH(P->bs, GK_BJ_APPLY);
#undef GK_BJ_APPLY
  }
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

}  // namespace gk

using namespace gk;

extern "C" int gk_precond_generate(gk_matrix h, int32_t block_size, void* stream, gk_precond* out) {
  if (!out) return set_error(GK_ERR_ARG, "gk_precond_generate: out is NULL");
  *out = nullptr;
  Matrix* A = as_matrix(h);
  if (!A) return set_error(GK_ERR_ARG, "gk_precond_generate: NULL matrix");
  if (A->n_rows != A->n_cols) return set_error(GK_ERR_DIM, "gk_precond_generate: matrix is not square");
  if (block_size < 1 || block_size > 32)
    return set_error(GK_ERR_ARG, "gk_precond_generate: block_size %d not in [1, 32]", block_size);
  int prev = current_device();
  if (prev != A->device) cudaSetDevice(A->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::unique_ptr<Precond, PrecondDeleter> hold(new Precond);
  Precond* P = hold.get();
  P->device = A->device;
  A->refs.fetch_add(1);
  P->A = A;
  P->n = A->n_rows;
  P->bs = block_size;
  int rc = GK_OK;
  do {
    // the error word: INT_MAX in, the smallest failing row or block out,
    // through pinned host words (asynchronous copies, no staging)
    if (!A->h_flag && cudaMallocHost(&A->h_flag, 2 * sizeof(int)) != cudaSuccess) {
      A->h_flag = nullptr;
      rc = cuda_error(cudaGetLastError(), "cudaMallocHost");
      break;
    }
    A->h_flag[0] = INT_MAX;
    if (cudaMemcpyAsync(A->err + 1, A->h_flag, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      rc = cuda_error(cudaGetLastError(), "cudaMemcpyAsync");
      break;
    }
    if (block_size == 1) {
      P->nblocks = P->n;
      if ((rc = dalloc_async_n(&P->dinv, static_cast<size_t>(std::max<int64_t>(P->n, 1)), &P->device_bytes, s)))
        break;
      if (P->n > 0)
        jacobi_scalar_kernel<<<grid_for(P->n, 256), 256, 0, s>>>(A->rowptr, A->col, A->val,
                                                                  static_cast<int>(P->n), P->dinv, A->err + 1);
    } else {
      P->nblocks = (P->n + block_size - 1) / block_size;
      P->block_elems = bj_total_elems(P->n, block_size);
      if ((rc = dalloc_async_n(&P->blocks, static_cast<size_t>(std::max<int64_t>(P->block_elems, 1)),
                               &P->device_bytes, s)))
        break;
      if (P->nblocks > 0)
        bj_generate(A, static_cast<int>(P->n), block_size, static_cast<int>(P->nblocks), P->blocks, A->err + 1, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = cuda_error(e, "Jacobi generate launch");
      break;
    }
    if (cudaMemcpyAsync(A->h_flag + 1, A->err + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = cuda_error(cudaGetLastError(), "Jacobi generate");
      break;
    }
    const int bad = A->h_flag[1];
    if (bad != INT_MAX) {
      rc = block_size == 1 ? set_error(GK_ERR_SINGULAR, "zero or missing diagonal in row %d", bad)
                           : set_error(GK_ERR_SINGULAR, "diagonal block %d is singular", bad);
      break;
    }
  } while (false);
  if (prev != A->device) cudaSetDevice(prev);
  if (rc != GK_OK) return rc;
  *out = reinterpret_cast<gk_precond>(hold.release());
  return GK_OK;
}

extern "C" int gk_precond_apply(gk_precond h, const void* r, void* z, void* stream) {
  Precond* P = as_precond(h);
  if (!P) return set_error(GK_ERR_ARG, "gk_precond_apply: NULL preconditioner");
  if (r == z && P->n > 0) return set_error(GK_ERR_ARG, "gk_precond_apply: r and z must not alias");
  int prev = current_device();
  if (prev != P->device) cudaSetDevice(P->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = GK_OK;
  do {
    VecArg vr, vz;
    if ((rc = vec_in(vr, r, P->n, &P->stage_in, &P->device_bytes, true, P->device, s))) break;
    if ((rc = vec_in(vz, z, P->n, &P->stage_out, &P->device_bytes, false, P->device, s))) break;
    if ((rc = precond_apply_launch(P, vr.dev, vz.dev, s))) break;
    rc = vec_out(vz, P->n, s);
  } while (false);
  if (prev != P->device) cudaSetDevice(prev);
  return rc;
}

extern "C" int gk_precond_get_blocks(gk_precond h, double* out, int64_t n_out, void* stream) {
  Precond* P = as_precond(h);
  if (!P || !out) return set_error(GK_ERR_ARG, "gk_precond_get_blocks: NULL argument");
  const int64_t total = P->bs == 1 ? P->n : P->block_elems;
  if (n_out < total) return set_error(GK_ERR_DIM, "gk_precond_get_blocks: need %lld doubles", (long long)total);
  if (total == 0) return GK_OK;
  int prev = current_device();
  if (prev != P->device) cudaSetDevice(P->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = GK_OK;
  do {
    // the device layout is the exported one: row-major blocks, concatenated
    const double* src = P->bs == 1 ? P->dinv : P->blocks;
    if (cudaMemcpyAsync(out, src, sizeof(double) * total, cudaMemcpyDefault, s) != cudaSuccess) {
      rc = cuda_error(cudaGetLastError(), "cudaMemcpyAsync");
      break;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = cuda_error(cudaGetLastError(), "sync");
  } while (false);
  if (prev != P->device) cudaSetDevice(prev);
  return rc;
}

extern "C" int gk_precond_destroy(gk_precond h) {
  if (!h) return set_error(GK_ERR_ARG, "gk_precond_destroy: NULL handle");
  precond_release(as_precond(h));
  return GK_OK;
}
