// spmv.cu -- sparse matrix-vector products y = op(A x) for the four storage
// formats (Section 4.2's simple and advanced apply), each with a fused
// epilogue that can also produce the dot products a Krylov step needs.
//
// FP64 throughput shapes every kernel here: the GPU retires about two FP64
// fused multiply-adds per SM per clock, barely more than the ~1.9 nonzeros
// per SM per clock that HBM delivers for 12-byte (value + index) entries.  So
// each stored entry costs exactly one DFMA, warps keep all 32 lanes busy in
// the DFMA loops, and reductions of partial sums are kept off the
// per-nonzero path.
#include <algorithm>
#include <cstdio>

#include "gk_device.cuh"
#include "gk_internal.h"
#include "solver_state.cuh"

namespace gk {

// ---------------------------------------------------------------------------
// epilogue
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool epi_skip(const Epi& e) {
  if (e.st == nullptr || e.skip_mode == 0) return false;
  const volatile int* f = &e.st->stop;
  if (f[0] != 0) return true;
  return e.skip_mode == 2 && f[1] != 0;  // f[1] is st->half
}

__device__ __forceinline__ void epi_row(const Epi& e, int row, double s, double& a0, double& a1) {
  switch (e.mode) {
    case EPI_COPY:
      e.y[row] = s;
      break;
    case EPI_PLAIN: {
      double as = e.alpha * s;
      e.y[row] = e.beta_zero ? as : fma(e.beta, e.y[row], as);
      break;
    }
    case EPI_RESID: {
      double b = e.u[row];
      double r = b - s;
      e.y[row] = r;
      a0 = fma(r, r, a0);
      a1 = fma(b, b, a1);
      break;
    }
    case EPI_DOT:
      e.y[row] = s;
      a0 = fma(e.u[row], s, a0);
      break;
    default:  // EPI_DOT2
      e.y[row] = s;
      a0 = fma(e.u[row], s, a0);
      a1 = fma(s, s, a1);
      break;
  }
}

// The same epilogue with the mode fixed at compile time (used where register
// pressure matters: the ELL kernel runs at full occupancy only within 32
// registers per thread).
template <int MODE>
__device__ __forceinline__ void epi_row_t(const Epi& e, int row, double s, double& a0, double& a1) {
  if (MODE == EPI_COPY) {
    e.y[row] = s;
  } else if (MODE == EPI_PLAIN) {
    double as = e.alpha * s;
    e.y[row] = e.beta_zero ? as : fma(e.beta, e.y[row], as);
  } else if (MODE == EPI_RESID) {
    double b = e.u[row];
    double r = b - s;
    e.y[row] = r;
    a0 = fma(r, r, a0);
    a1 = fma(b, b, a1);
  } else if (MODE == EPI_DOT) {
    e.y[row] = s;
    a0 = fma(e.u[row], s, a0);
  } else {
    e.y[row] = s;
    a0 = fma(e.u[row], s, a0);
    a1 = fma(s, s, a1);
  }
}

// Grid-wide reduction of (a0, a1) and the scalar step that consumes it.
__device__ __forceinline__ void epi_finish(const Epi& e, double a0, double a1, double* scratch) {
  if (e.mode == EPI_PLAIN || e.mode == EPI_COPY) return;
  double v[2] = {a0, a1}, out[2];
  if (grid_sum<2>(v, e.partials, e.counter, scratch, out)) {
    if (threadIdx.x == 0 && e.st) finalize(e.fin, out, e.st);
  }
}

// Out-of-line copy for kernels whose row loop must stay within a tight
// register budget.
__device__ __noinline__ void epi_finish_ool(const Epi& e, double a0, double a1, double* scratch) {
  epi_finish(e, a0, a1, scratch);
}

// Block partials only; a later launch finishes the reduction.
__device__ __forceinline__ void epi_partial(const Epi& e, double a0, double a1, double* scratch) {
  if (e.mode == EPI_PLAIN || e.mode == EPI_COPY) return;
  double v[2] = {a0, a1};
  block_sum<2>(v, scratch);
  if (threadIdx.x == 0) {
    e.partials[2 * blockIdx.x] = v[0];
    e.partials[2 * blockIdx.x + 1] = v[1];
  }
}

// ---------------------------------------------------------------------------
// GK_CSR: rows binned by length.  The plan sorts the rows by decreasing
// length.  Rows of up to kSliceMaxLen entries form slices of 32 consecutive
// (in that order) rows stored column-major and padded to the slice's longest
// row -- so neighbouring lanes have nearly equal work and their loads of
// values and indices are coalesced; each lane sums its row sequentially in
// CSR order, bit-identical to the CPU reference.  Longer rows are cut into
// pieces of at most kPieceLen consecutive entries, each summed by one warp
// (coalesced loads, xor butterfly), so that no row holds up the launch: a
// row of one piece is finished by its warp, the pieces of longer rows are
// added in order by a second launch (spmv_long_fixup_kernel).
// Values and indices are streamed (read once, evict first) so that the
// gathered vector keeps the caches (27-point matrix: 135.9 -> 116.5 us).
// ---------------------------------------------------------------------------

// Gathers a lane keeps in flight in the slice loop: 8 for the plain applies
// and the fused dot of CG's SpMV (within 40 registers at 6 blocks per SM), 4
// for the two-accumulator epilogues.
template <int MODE>
struct EllBatchOf {
  static constexpr int value = (MODE == EPI_COPY || MODE == EPI_PLAIN || MODE == EPI_DOT) ? 8 : 4;
};
// Strides of 32 entries a lane keeps in flight in a piece of a long row: 8
// for CG's fused dot (40 registers), 4 for the plain applies, whose
// 32-register build slows down with 8.
template <int MODE>
struct MidBatchOf {
  static constexpr int value = MODE == EPI_DOT ? 8 : 4;
};

struct SliceArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const int32_t* perm;
  const int64_t* off;
  const int32_t* scol;
  const double* sval;
  int n_sell, n_slices;
  const int4* pc;        // pieces of the long rows: {row, k0, k1, slot}
  int n_pc;
  const int32_t* lr_row;  // rows of several pieces and their slots
  const int32_t* lr_off;
  int n_lr;
  double* pc_sum;         // [slots] the pieces' sums
  const double* x;
};

// Blocks per SM the sliced kernel is compiled for: 8 (32 registers, 64
// warps: the gathers' latency is what the warps hide; power-law matrix
// 174 -> 163 us) for the plain applies, 6 (40 registers) for the
// epilogues with reductions, whose 32-register build measured slower inside
// CG (45.7 -> 49.9 ms on the 27-point matrix) or spilled.
template <int MODE>
struct SliceMinBlocks {
  static constexpr int value = (MODE == EPI_COPY || MODE == EPI_PLAIN) ? 8 : 6;
};

template <int MODE>
__global__ void __launch_bounds__(kSliceThreads, SliceMinBlocks<MODE>::value) spmv_sliced_kernel(SliceArgs a,
                                                                                                Epi e) {
  pdl_wait();
  constexpr int B = EllBatchOf<MODE>::value;
  __shared__ double red_scratch[kRedScratch];
  if (epi_skip(e)) return;
  double a0 = 0.0, a1 = 0.0;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n_items = a.n_pc + a.n_slices;
  for (int it = gw; it < n_items; it += nw) {
    if (it < a.n_pc) {
      const int4 pc = __ldg(a.pc + it);
      const int k0 = pc.y, k1 = pc.z;
      constexpr int MB = MidBatchOf<MODE>::value;
      double s = 0.0;
      int k = k0 + lane;
      for (; k + 32 * (MB - 1) < k1; k += 32 * MB) {
        int cc[MB];
        double vv[MB], xv[MB];
#pragma unroll
        for (int u = 0; u < MB; ++u) cc[u] = __ldcs(a.col + k + 32 * u);
#pragma unroll
        for (int u = 0; u < MB; ++u) vv[u] = __ldcs(a.val + k + 32 * u);
#pragma unroll
        for (int u = 0; u < MB; ++u) xv[u] = __ldg(a.x + cc[u]);
#pragma unroll
        for (int u = 0; u < MB; ++u) s = fma(vv[u], xv[u], s);
      }
#pragma unroll
      for (int g = 0; g < MB / 4; ++g, k += 128) {  // fewer than MB strides of 32 left: guarded batches of 4
        int cc[4];
        double vv[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool in = k + 32 * u < k1;
          cc[u] = in ? __ldcs(a.col + k + 32 * u) : -1;
          vv[u] = in ? __ldcs(a.val + k + 32 * u) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = cc[u] >= 0 ? __ldg(a.x + cc[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (cc[u] >= 0) s = fma(vv[u], xv[u], s);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        if (pc.w < 0) epi_row_t<MODE>(e, pc.x, s, a0, a1);
        else a.pc_sum[pc.w] = s;
      }
    } else {
      const int c = it - a.n_pc;
      const int base = c * 32 + lane;
      const int64_t o0 = __ldg(a.off + c);
      const int L = static_cast<int>((__ldg(a.off + c + 1) - o0) >> 5);
      const int32_t* cp = a.scol + o0 + lane;
      const double* vp = a.sval + o0 + lane;
      double s = 0.0;
      int j = 0;
      for (; j + B <= L; j += B) {
        int cc[B];
        double vv[B], xv[B];
#pragma unroll
        for (int u = 0; u < B; ++u) cc[u] = __ldcs(cp + (j + u) * 32);
#pragma unroll
        for (int u = 0; u < B; ++u) vv[u] = __ldcs(vp + (j + u) * 32);
#pragma unroll
        for (int u = 0; u < B; ++u) xv[u] = cc[u] >= 0 ? __ldg(a.x + cc[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < B; ++u)
          if (cc[u] >= 0) s = fma(vv[u], xv[u], s);
      }
      // the last L mod B slots in guarded batches of 4 (a round of loads
      // per 4 slots, not per slot), still summed in slot order
      for (; j < L; j += 4) {
        int cc[4];
        double vv[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool in = j + u < L;
          cc[u] = in ? __ldcs(cp + (j + u) * 32) : -1;
          vv[u] = in ? __ldcs(vp + (j + u) * 32) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = cc[u] >= 0 ? __ldg(a.x + cc[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (cc[u] >= 0) s = fma(vv[u], xv[u], s);
      }
      if (base < a.n_sell) epi_row_t<MODE>(e, __ldg(a.perm + base), s, a0, a1);
    }
  }
  if (MODE != EPI_COPY && MODE != EPI_PLAIN) {
    if (a.n_lr > 0) epi_partial(e, a0, a1, red_scratch);  // the fix-up launch finishes the sum
    else epi_finish(e, a0, a1, red_scratch);
  }
}

// Rows of several pieces (one warp each, all rows in parallel): the pieces'
// sums added in order (lane-strided, then an xor butterfly: a fixed order),
// then the epilogue; then the epilogue's reduction, the main launch's block
// partials folded into this launch's fixed-order grid sum, whose block
// partials live after the main launch's.
template <int MODE>
__global__ void __launch_bounds__(256) spmv_long_fixup_kernel(SliceArgs a, Epi e, int main_grid) {
  __shared__ double red_scratch[kRedScratch];
  pdl_wait();
  if (epi_skip(e)) return;
  double a0 = 0.0, a1 = 0.0;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int w = gw; w < a.n_lr; w += nw) {
    const int o0 = __ldg(a.lr_off + w), o1 = __ldg(a.lr_off + w + 1);
    double s = 0.0;
    for (int o = o0 + lane; o < o1; o += 32) s += __ldcg(a.pc_sum + o);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) epi_row_t<MODE>(e, __ldg(a.lr_row + w), s, a0, a1);
  }
  if (MODE == EPI_COPY || MODE == EPI_PLAIN) return;
  const int stride = gridDim.x * blockDim.x;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  for (int b = gt; b < main_grid; b += stride) {
    a0 += __ldcg(e.partials + 2 * b);
    a1 += __ldcg(e.partials + 2 * b + 1);
  }
  double v[2] = {a0, a1}, out[2];
  if (grid_sum<2>(v, e.partials + 2 * main_grid, e.counter, red_scratch, out) && threadIdx.x == 0 && e.st)
    finalize(e.fin, out, e.st);
}

// ---------------------------------------------------------------------------
// GK_ELL (and the ELL part of GK_HYB): column-major slots, one row per
// thread, padding slots carry column -1 and are skipped.  Rows with an
// overflow in the HYB tail add its precomputed partial sum.
// ---------------------------------------------------------------------------

struct EllArgs {
  const int32_t* col;
  const double* val;
  int64_t ld;
  int K;
  int n_rows;
  const double* x;
  const int32_t* tail_slot;
  const double* tail_sum;
};

// 8 blocks of 256 threads per SM (32 registers): full occupancy is what hides
// the latency of the gathers (measured: 6 blocks/SM ran 10-25 % slower).
// Values and indices are read once: streaming loads (evict first), so that
// they do not push the gathered vector out of the caches (measured 131.5 ->
// 123.5 us on the 27-point matrix).
// The reduction epilogues carry two accumulators and a second vector through
// the loop; they issue their gathers in batches of 4 instead of 8 so that
// they, too, fit 32 registers and keep 8 blocks per SM.
template <int MODE>
struct EllBatch {
  static constexpr int value = (MODE == EPI_COPY || MODE == EPI_PLAIN) ? 8 : 4;
};

// Slots of its first row a thread prefetches into L2 before the previous
// kernel has finished (the matrix is not written by any kernel of a solve).
constexpr int kEllPrefetchSlots = 8;

template <int MODE, bool TAIL>
__global__ void __launch_bounds__(kEllThreads, 8) spmv_ell_kernel(EllArgs a, Epi e) {
  {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    if (row < a.n_rows && (lane & 15) == 0) {
      const int kp = min(a.K, kEllPrefetchSlots);
      for (int j = 0; j < kp; ++j) {
        if (lane == 0) prefetch_l2(a.col + row + j * a.ld);
        prefetch_l2(a.val + row + j * a.ld);
      }
    }
  }
  pdl_wait();
  pdl_launch_dependents();
  constexpr int B = EllBatch<MODE>::value;
  __shared__ double red_scratch[kRedScratch];
  if (epi_skip(e)) return;
  double a0 = 0.0, a1 = 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < a.n_rows; row += stride) {
    double s = 0.0;
    const int32_t* cp = a.col + row;
    const double* vp = a.val + row;
    int j = 0;
    for (; j + B <= a.K; j += B) {
      int cc[B];
      double xv[B], vv[B];
#pragma unroll
      for (int u = 0; u < B; ++u) cc[u] = __ldcs(cp + (j + u) * a.ld);
#pragma unroll
      for (int u = 0; u < B; ++u) vv[u] = __ldcs(vp + (j + u) * a.ld);
#pragma unroll
      for (int u = 0; u < B; ++u) xv[u] = cc[u] >= 0 ? __ldg(a.x + cc[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < B; ++u)
        if (cc[u] >= 0) s = fma(vv[u], xv[u], s);
    }
    for (; j < a.K; j += 4) {
      int cc[4];
      double xv[4], vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cc[u] = (j + u < a.K) ? __ldcs(cp + (j + u) * a.ld) : -1;
        vv[u] = cc[u] >= 0 ? __ldcs(vp + (j + u) * a.ld) : 0.0;
        xv[u] = cc[u] >= 0 ? __ldg(a.x + cc[u]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (cc[u] >= 0) s = fma(vv[u], xv[u], s);
    }
    if (TAIL) {
      const int t = __ldg(a.tail_slot + row);
      if (t >= 0) s += __ldcg(a.tail_sum + t);
    }
    epi_row_t<MODE>(e, row, s, a0, a1);
  }
  if (MODE != EPI_COPY && MODE != EPI_PLAIN) epi_finish(e, a0, a1, red_scratch);
}

template <bool TAIL>
void launch_ell_t(int grid, cudaStream_t s, const EllArgs& a, const Epi& e) {
  switch (e.mode) {
    case EPI_COPY: launch_pdl(spmv_ell_kernel<EPI_COPY, TAIL>, grid, kEllThreads, 0, s, a, e); break;
    case EPI_PLAIN: launch_pdl(spmv_ell_kernel<EPI_PLAIN, TAIL>, grid, kEllThreads, 0, s, a, e); break;
    case EPI_RESID: launch_pdl(spmv_ell_kernel<EPI_RESID, TAIL>, grid, kEllThreads, 0, s, a, e); break;
    case EPI_DOT: launch_pdl(spmv_ell_kernel<EPI_DOT, TAIL>, grid, kEllThreads, 0, s, a, e); break;
    default: launch_pdl(spmv_ell_kernel<EPI_DOT2, TAIL>, grid, kEllThreads, 0, s, a, e); break;
  }
}

// ---------------------------------------------------------------------------
// GK_CSR_MERGE: merge-path SpMV.  The sequence of n_rows row ends and nnz
// entries (row r's end follows its last entry) is cut into tiles of
// kMergeTile items, one tile per warp at a time, kMergeItems consecutive
// items per lane, so every lane does the same amount of work whatever the
// row lengths.  A lane finds its start on the merge path by a binary search
// over the tile's row pointers (staged in shared memory), loads its (at most
// kMergeItems) entries and walks its items: a row whose end it meets is
// complete if the row began in the lane, else it is the lane's head.  Heads
// are joined to the lanes before them by a segmented inclusive scan over the
// warp (shuffles, fixed tree order); a row that began in an earlier tile
// leaves the tile's part in a per-tile partial sum, and a one-thread-per-tile
// fix-up launch adds the parts from earlier tiles (the tile's last open row
// leaves its part as well).  No thread-block barrier: warps are independent.
// ---------------------------------------------------------------------------

// Steps of a segmented inclusive warp scan that suffice when the lanes in
// `open` (bit l: lane l adds the value of lane l - 1) form chains of at most
// L consecutive lanes: ceil(log2(L + 1)).  A lane's sum is final once its
// chain is resolved, so stopping there changes no bit, and each FP64 add
// saved is a warp instruction of the (slow) FP64 pipe saved.
__device__ __forceinline__ int scan_steps(unsigned int open) {
  int L = 0;
  for (unsigned int x = open; x; x &= x << 1) ++L;
  return 32 - __clz(L);
}

constexpr int kMergeStage = kMergeTile + 8;  // staged row pointers per warp
constexpr int kMergeWarps = kMergeThreads / 32;

struct MergeArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const int32_t* tile_i;
  const int32_t* tile_j;
  double* c_head;  // per tile: its part of its first row, when that row began earlier and ends here
  double* c_tail;  // per tile: its part of the row left open at its end
  int n_rows;
  int nnz;
  int n_tiles;
  const double* x;
};

__global__ void __launch_bounds__(kMergeThreads) spmv_merge_kernel(MergeArgs a, Epi e) {
  __shared__ int32_t s_rp[kMergeWarps][kMergeStage];
  __shared__ double red_scratch[kRedScratch];
  pdl_wait();
  if (epi_skip(e)) return;
  constexpr int E = kMergeItems;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* rp = s_rp[wib];
  const int total = a.n_rows + a.nnz;
  double a0 = 0.0, a1 = 0.0;
  for (int t = blockIdx.x * kMergeWarps + wib; t < a.n_tiles; t += gridDim.x * kMergeWarps) {
    const int ti = __ldg(a.tile_i + t), tj = __ldg(a.tile_j + t);
    const int ti1 = __ldg(a.tile_i + t + 1), tj1 = __ldg(a.tile_j + t + 1);
    const int d0 = t * kMergeTile, d1 = min(d0 + kMergeTile, total);
    // row pointers rowptr[ti .. min(ti1 + 1, n_rows)] (at most kMergeTile + 2)
    const int nrp = min(ti1 + 1, a.n_rows) - ti + 1;
    __syncwarp();
    for (int q = lane; q < nrp; q += 32) rp[q] = __ldg(a.rowptr + ti + q);
    __syncwarp();
#define RPW(r) rp[(r) - ti]
    // the lane's start (row, k) on the merge path; inactive lanes sit at the tile end
    const int dl = d0 + lane * E;
    const bool active = dl < d1;
    int row = ti1, k = tj1;
    if (active) {
      int lo = max(ti, dl - tj1), hi = min(ti1, dl - tj);
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (RPW(mid + 1) <= dl - mid - 1) lo = mid + 1;
        else hi = mid;
      }
      row = lo;
      k = dl - lo;
    }
    int row_end = __shfl_down_sync(0xffffffffu, row, 1);
    int k_end = __shfl_down_sync(0xffffffffu, k, 1);
    if (lane == 31) {
      row_end = ti1;
      k_end = tj1;
    }
    const int cnt = active ? k_end - k : 0;
    double vv[E], xv[E];
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const bool in = u < cnt;
      vv[u] = in ? __ldcs(a.val + k + u) : 0.0;
      xv[u] = in ? __ldg(a.x + __ldcs(a.col + k + u)) : 0.0;
    }
    // walk: a row end met before entry kk (rowptr[cur + 1] <= kk) ends row cur
    const bool mid_start = active && k > RPW(row);
    int cur = row;
    int nxt = (active && cur < a.n_rows) ? RPW(cur + 1) : 0x7fffffff;
    bool emitted = false;
    int head_row = -1;
    double head = 0.0, sum = 0.0;
#pragma unroll
    for (int u = 0; u < E; ++u) {
      if (u < cnt) {
        while (k + u >= nxt) {
          if (!emitted && mid_start) {
            head_row = cur;
            head = sum;
          } else {
            epi_row(e, cur, sum, a0, a1);
          }
          emitted = true;
          ++cur;
          nxt = cur < a.n_rows ? RPW(cur + 1) : 0x7fffffff;
          sum = 0.0;
        }
        sum = fma(vv[u], xv[u], sum);
      }
    }
    if (active) {
      while (cur < row_end) {
        if (!emitted && mid_start) {
          head_row = cur;
          head = sum;
        } else {
          epi_row(e, cur, sum, a0, a1);
        }
        emitted = true;
        ++cur;
        sum = 0.0;
      }
    }
    // segmented inclusive scan of the lanes' open sums: a lane that met no
    // row end and began inside a row continues the lane before it
    double S = sum;
    int open = (lane > 0 && active && !emitted && mid_start) ? 1 : 0;
    const int steps = scan_steps(__ballot_sync(0xffffffffu, open));
    for (int d = 1; d < (1 << steps); d <<= 1) {
      const double Sp = __shfl_up_sync(0xffffffffu, S, d);
      const int op = __shfl_up_sync(0xffffffffu, open, d);
      if (lane >= d && open) {
        S = Sp + S;
        open = op;
      }
    }
    const double S_prev = __shfl_up_sync(0xffffffffu, S, 1);
    if (head_row >= 0) {
      const double v = lane > 0 ? S_prev + head : head;
      if (head_row == ti && tj > RPW(ti)) a.c_head[t] = v;  // began in an earlier tile
      else epi_row(e, head_row, v, a0, a1);
    }
    if (active && lane == (d1 - d0 - 1) / E) a.c_tail[t] = S;
#undef RPW
  }
  epi_partial(e, a0, a1, red_scratch);
}

// Rows that began in an earlier tile and end in tile t (one thread per tile,
// all tiles in parallel): the tile's part plus the open parts of the tiles
// before it, back to the tile where the row began; then the epilogue's
// reduction: the main launch's block partials are folded into this launch's
// own fixed-order grid sum, whose block partials live after the main launch's.
__global__ void __launch_bounds__(256) spmv_merge_fixup_kernel(MergeArgs a, Epi e, int main_grid) {
  __shared__ double red_scratch[kRedScratch];
  pdl_wait();
  if (epi_skip(e)) return;
  double a0 = 0.0, a1 = 0.0;
  const int stride = gridDim.x * blockDim.x;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  for (int t = gt; t < a.n_tiles; t += stride) {
    const int f = __ldg(a.tile_i + t);
    if (t == 0 || !(__ldg(a.tile_j + t) > __ldg(a.rowptr + f)) || !(__ldg(a.tile_i + t + 1) > f)) continue;
    double v = a.c_head[t];
    const int rf = __ldg(a.rowptr + f);
    for (int u = t - 1; u >= 0; --u) {
      v += a.c_tail[u];
      if (!(u > 0 && __ldg(a.tile_i + u) == f && __ldg(a.tile_j + u) > rf)) break;
    }
    epi_row(e, f, v, a0, a1);
  }
  if (e.mode == EPI_PLAIN || e.mode == EPI_COPY) return;
  for (int b = gt; b < main_grid; b += stride) {
    a0 += __ldcg(e.partials + 2 * b);
    a1 += __ldcg(e.partials + 2 * b + 1);
  }
  double v[2] = {a0, a1}, out[2];
  if (grid_sum<2>(v, e.partials + 2 * main_grid, e.counter, red_scratch, out) && threadIdx.x == 0 && e.st)
    finalize(e.fin, out, e.st);
}

// ---------------------------------------------------------------------------
// GK_HYB overflow in COO form: entries (row, column, value) sorted by (row,
// column), a row index per entry (the COO SpMV of the paper's solver
// evaluation).  The entries are cut into chunks of kCooChunk; a warp takes a
// chunk and each lane kCooPerLane consecutive entries, so the work per warp
// does not depend on the row lengths.  A lane sums its runs of equal row in
// entry order (fma); runs that cross lanes are joined by a segmented
// inclusive scan over the warp (shuffles, fixed tree order); rows that cross
// chunks are finished by a one-thread-per-chunk fix-up launch from each
// chunk's partial sums of its first and last row.  The results are the
// overflow sums of the tail rows (indexed by the row's tail slot), which the
// ELL kernel then adds to its row sums.  Padding entries past nnz are never
// summed; the arrays are allocated in whole chunks so that every lane's
// 16-byte loads stay inside them.
// ---------------------------------------------------------------------------

struct CooArgs {
  const int32_t* row;
  const int32_t* col;
  const double* val;
  int nnz;
  int n_chunks;
  const int32_t* slot;  // [n_rows] tail slot of each row
  double* out;          // [m_tail] overflow sum of each tail row
  int32_t* c_first;     // per chunk: its first and last row and their partial sums
  int32_t* c_last;
  double* c_head;
  double* c_tail;
  const double* x;
};

__global__ void __launch_bounds__(kCooThreads) spmv_coo_kernel(CooArgs a, Epi e) {
  pdl_wait();
  constexpr int E = kCooPerLane;
  if (epi_skip(e)) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < a.n_chunks; c += nw) {
    const int c0 = c * kCooChunk;
    const int e0 = c0 + lane * E;
    int rr[E], cc[E];
    double vv[E], xv[E];
    {
      const int4* rp = reinterpret_cast<const int4*>(a.row + e0);
      const int4* cp = reinterpret_cast<const int4*>(a.col + e0);
      const double2* vp = reinterpret_cast<const double2*>(a.val + e0);
#pragma unroll
      for (int h = 0; h < E / 4; ++h) {
        const int4 r4 = __ldcs(rp + h), c4 = __ldcs(cp + h);
        rr[4 * h] = r4.x; rr[4 * h + 1] = r4.y; rr[4 * h + 2] = r4.z; rr[4 * h + 3] = r4.w;
        cc[4 * h] = c4.x; cc[4 * h + 1] = c4.y; cc[4 * h + 2] = c4.z; cc[4 * h + 3] = c4.w;
      }
#pragma unroll
      for (int h = 0; h < E / 2; ++h) {
        const double2 v2 = __ldcs(vp + h);
        vv[2 * h] = v2.x;
        vv[2 * h + 1] = v2.y;
      }
    }
#pragma unroll
    for (int u = 0; u < E; ++u) xv[u] = (e0 + u < a.nnz) ? __ldg(a.x + cc[u]) : 0.0;
    // the lane's runs: the first (head), whole rows in between (written
    // here), the last (tail)
    int first = -1, cur = -1;
    double head = 0.0, sum = 0.0;
#pragma unroll
    for (int u = 0; u < E; ++u) {
      if (e0 + u < a.nnz) {
        if (rr[u] != cur) {
          if (cur >= 0) {
            if (cur == first) head = sum;
            else a.out[__ldg(a.slot + cur)] = sum;
          }
          if (first < 0) first = rr[u];
          cur = rr[u];
          sum = 0.0;
        }
        sum = fma(vv[u], xv[u], sum);
      }
    }
    const int last = cur;
    if (first == last) head = sum;
    // segmented inclusive scan of the tails over the lanes: a lane that is a
    // single run of the previous lane's last row adds the scan before it
    const int prev_last = __shfl_up_sync(0xffffffffu, last, 1);
    double S = sum;
    int open = (lane > 0 && first >= 0 && first == last && prev_last == first) ? 1 : 0;
    const int steps = scan_steps(__ballot_sync(0xffffffffu, open));
    for (int d = 1; d < (1 << steps); d <<= 1) {
      const double Sp = __shfl_up_sync(0xffffffffu, S, d);
      const int op = __shfl_up_sync(0xffffffffu, open, d);
      if (lane >= d && open) {
        S = Sp + S;
        open = op;
      }
    }
    const double S_prev = __shfl_up_sync(0xffffffffu, S, 1);
    const int next_first = __shfl_down_sync(0xffffffffu, first, 1);
    const int chunk_first = __shfl_sync(0xffffffffu, first, 0);
    int before = -1;
    if (lane == 0 && c0 > 0) before = __ldg(a.row + c0 - 1);
    before = __shfl_sync(0xffffffffu, before, 0);
    const bool head_open = before == chunk_first;  // the chunk's first row began in an earlier chunk
    const int nvalid = min(32, (a.nnz - c0 + E - 1) / E);
    if (lane < nvalid) {
      // a row that ends in this lane (and is not the chunk's last row) is
      // complete unless it began in an earlier chunk
      if (first != last) {
        const double v = ((lane > 0 && prev_last == first) ? S_prev : 0.0) + head;
        if (head_open && first == chunk_first) a.c_head[c] = v;
        else a.out[__ldg(a.slot + first)] = v;
      }
      if (lane < nvalid - 1) {
        if (next_first != last) {
          if (head_open && last == chunk_first) a.c_head[c] = S;
          else a.out[__ldg(a.slot + last)] = S;
        }
      } else {
        a.c_first[c] = chunk_first;
        a.c_last[c] = last;
        a.c_tail[c] = S;
      }
    }
  }
}

// Rows that cross chunk boundaries, one thread per chunk: the chunk's first
// row if it began in an earlier chunk and ends inside this one, and the
// chunk's last row if it ends with this chunk; each sums its pieces from
// this chunk back to the chunk where it began.
__global__ void __launch_bounds__(256) spmv_coo_fixup_kernel(CooArgs a, Epi e) {
  pdl_wait();
  if (epi_skip(e)) return;
  const int stride = gridDim.x * blockDim.x;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.n_chunks; c += stride) {
    const int f = a.c_first[c], l = a.c_last[c];
    if (c > 0 && f != l && a.c_last[c - 1] == f) {
      double v = a.c_head[c];
      for (int u = c - 1; u >= 0; --u) {
        v += a.c_tail[u];
        if (!(a.c_first[u] == f && u > 0 && a.c_last[u - 1] == f)) break;
      }
      a.out[__ldg(a.slot + f)] = v;
    }
    if (c == a.n_chunks - 1 || a.c_first[c + 1] != l) {
      double v = a.c_tail[c];
      for (int u = c; u > 0 && a.c_first[u] == l && a.c_last[u - 1] == l; --u) v += a.c_tail[u - 1];
      a.out[__ldg(a.slot + l)] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

namespace {

struct KernelGrids {
  int bin = 0, ell = 0, merge = 0;
};

int occupancy_grid(const void* fn, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * sm_count();
}

MergeArgs merge_args(const MergePlan& P, const double* x) {
  MergeArgs m;
  m.rowptr = P.rowptr;
  m.col = P.col;
  m.val = P.val;
  m.tile_i = P.tile_i;
  m.tile_j = P.tile_j;
  m.c_head = P.head_val;
  m.c_tail = P.carry_val;
  m.n_rows = static_cast<int>(P.n_rows);
  m.nnz = static_cast<int>(P.nnz);
  m.n_tiles = static_cast<int>(P.n_tiles);
  m.x = x;
  return m;
}

int launch_merge(const MergePlan& P, const double* x, const Epi& e, cudaStream_t s) {
  if (P.n_tiles == 0) return GK_OK;
  MergeArgs m = merge_args(P, x);
  launch_pdl(spmv_merge_kernel, P.grid, kMergeThreads, 0, s, m, e);
  GK_TRY_CUDA(cudaGetLastError());
  const int fg = static_cast<int>(std::min<int64_t>(kFixupMaxGrid, (P.n_tiles + 255) / 256));
  launch_pdl(spmv_merge_fixup_kernel, fg, 256, 0, s, m, e, P.grid);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

}  // namespace

int merge_grid(int64_t n_tiles) {
  int g = occupancy_grid(reinterpret_cast<const void*>(spmv_merge_kernel), kMergeThreads, 0);
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, (n_tiles + kMergeWarps - 1) / kMergeWarps)));
}

int sliced_grid(int64_t warp_items, bool plain) {
  const void* fn = plain ? reinterpret_cast<const void*>(spmv_sliced_kernel<EPI_COPY>)
                         : reinterpret_cast<const void*>(spmv_sliced_kernel<EPI_RESID>);
  int g = occupancy_grid(fn, kSliceThreads, 0);
  int64_t need = (warp_items + kSliceThreads / 32 - 1) / (kSliceThreads / 32);
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, need)));
}

int ell_grid(int64_t n_rows) {
  int g = occupancy_grid(reinterpret_cast<const void*>(spmv_ell_kernel<EPI_COPY, false>), kEllThreads, 0);
  int64_t need = (n_rows + kEllThreads - 1) / kEllThreads;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, need)));
}

int coo_grid(int64_t n_chunks) {
  int g = occupancy_grid(reinterpret_cast<const void*>(spmv_coo_kernel), kCooThreads, 0);
  int64_t need = (n_chunks + kCooThreads / 32 - 1) / (kCooThreads / 32);
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, need)));
}

namespace {

int launch_coo(const Matrix& A, const double* x, const Epi& e, cudaStream_t s) {
  if (A.coo_chunks == 0) return GK_OK;
  CooArgs c{A.tail_row, A.tail_col, A.tail_val, static_cast<int>(A.tail_nnz), static_cast<int>(A.coo_chunks),
            A.tail_slot, A.tail_sum, A.coo_first, A.coo_last, A.coo_head, A.coo_tail, x};
  launch_pdl(spmv_coo_kernel, A.grid_coo, kCooThreads, 0, s, c, e);
  GK_TRY_CUDA(cudaGetLastError());
  const int fg = static_cast<int>(std::min<int64_t>(4 * sm_count(), (A.coo_chunks + 255) / 256));
  launch_pdl(spmv_coo_fixup_kernel, fg, 256, 0, s, c, e);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

}  // namespace

int spmv_max_grid(const Matrix& A) {
  return std::max({A.grid_sl, A.grid_sl_plain, A.grid_ell, A.merge.grid, 1});
}

int spmv_launch(const Matrix& A, const double* x, const Epi& e, cudaStream_t s) {
  if (A.n_rows == 0) return GK_OK;
  switch (A.format) {
    case GK_CSR: {
      SliceArgs b{A.rowptr, A.col, A.val, A.sl_perm, A.sl_off, A.sl_col, A.sl_val, static_cast<int>(A.n_sell),
                  static_cast<int>(A.n_slices), A.pc, static_cast<int>(A.n_pc), A.lr_row, A.lr_off,
                  static_cast<int>(A.n_lr), A.pc_sum, x};
      const bool plain = e.mode == EPI_COPY || e.mode == EPI_PLAIN;
      const int g = plain ? A.grid_sl_plain : A.grid_sl;
      switch (e.mode) {
        case EPI_COPY: launch_pdl(spmv_sliced_kernel<EPI_COPY>, g, kSliceThreads, 0, s, b, e); break;
        case EPI_PLAIN: launch_pdl(spmv_sliced_kernel<EPI_PLAIN>, g, kSliceThreads, 0, s, b, e); break;
        case EPI_RESID: launch_pdl(spmv_sliced_kernel<EPI_RESID>, g, kSliceThreads, 0, s, b, e); break;
        case EPI_DOT: launch_pdl(spmv_sliced_kernel<EPI_DOT>, g, kSliceThreads, 0, s, b, e); break;
        default: launch_pdl(spmv_sliced_kernel<EPI_DOT2>, g, kSliceThreads, 0, s, b, e); break;
      }
      GK_TRY_CUDA(cudaGetLastError());
      if (A.n_lr > 0) {
        const int fg = static_cast<int>(std::min<int64_t>(kFixupMaxGrid, (A.n_lr + 7) / 8));
        switch (e.mode) {
          case EPI_COPY: launch_pdl(spmv_long_fixup_kernel<EPI_COPY>, fg, 256, 0, s, b, e, g); break;
          case EPI_PLAIN: launch_pdl(spmv_long_fixup_kernel<EPI_PLAIN>, fg, 256, 0, s, b, e, g); break;
          case EPI_RESID: launch_pdl(spmv_long_fixup_kernel<EPI_RESID>, fg, 256, 0, s, b, e, g); break;
          case EPI_DOT: launch_pdl(spmv_long_fixup_kernel<EPI_DOT>, fg, 256, 0, s, b, e, g); break;
          default: launch_pdl(spmv_long_fixup_kernel<EPI_DOT2>, fg, 256, 0, s, b, e, g); break;
        }
        GK_TRY_CUDA(cudaGetLastError());
      }
      return GK_OK;
    }
    case GK_CSR_MERGE:
      return launch_merge(A.merge, x, e, s);
    case GK_ELL:
    case GK_HYB: {
      if (A.format == GK_HYB && A.m_tail > 0) {
        Epi te;
        te.mode = EPI_COPY;
        te.y = A.tail_sum;
        te.st = e.st;
        te.skip_mode = e.skip_mode;
        te.err = e.err;
        GK_TRY(launch_coo(A, x, te, s));
      }
      const bool tail = A.format == GK_HYB && A.m_tail > 0;
      EllArgs ea{A.ell_col, A.ell_val, A.ld, static_cast<int>(A.K), static_cast<int>(A.n_rows), x,
                 tail ? A.tail_slot : nullptr, A.tail_sum};
      if (tail) launch_ell_t<true>(A.grid_ell, s, ea, e);
      else launch_ell_t<false>(A.grid_ell, s, ea, e);
      GK_TRY_CUDA(cudaGetLastError());
      return GK_OK;
    }
    default:
      return set_error(GK_ERR_UNSUPPORTED, "unknown format %d", A.format);
  }
}

}  // namespace gk
