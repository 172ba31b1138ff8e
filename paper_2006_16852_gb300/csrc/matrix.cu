// matrix.cu -- creation of the CSR operator (Section 2.2.4: "objects A ... are
// LinOp objects that store their data as matrices in CSR") and of its
// GPU-side storage formats: row-length bins, merge-path tiles, ELL and the
// hybrid ELL + overflow split.  The caller's arrays are copied into
// library-owned storage (the "give"/copy ownership of Section 2.4).
#include <algorithm>
#include <climits>
#include <memory>
#include <vector>

#include "gk_device.cuh"
#include "gk_internal.h"

namespace gk {

namespace {

// Index arrays are padded so that 16-byte bulk copies rounded up to a
// multiple of four elements never read past the allocation.
inline int64_t padded(int64_t n) { return ((n + 3) & ~int64_t(3)) + 8; }

__global__ void validate_csr_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                    int n_rows, int n_cols, int* bad_row) {
  const int stride = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += stride) {
    const int k0 = rowptr[r], k1 = rowptr[r + 1];
    int prev = -1;
    for (int k = k0; k < k1; ++k) {
      const int c = col[k];
      if (c < 0 || c >= n_cols || c <= prev) {
        atomicMin(bad_row, r);
        break;
      }
      prev = c;
    }
  }
}

// Merge-path coordinates (rows consumed, nonzeros consumed) of every tile
// start: the largest i with rowptr[i] + i <= d such that the i-th row end
// precedes the diagonal d.
__global__ void merge_plan_kernel(const int32_t* __restrict__ rowptr, int n_rows, int nnz, int n_tiles,
                                  int32_t* tile_i, int32_t* tile_j) {
  const int stride = gridDim.x * blockDim.x;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= n_tiles; t += stride) {
    const long long dl = min(static_cast<long long>(t) * kMergeTile, static_cast<long long>(n_rows) + nnz);
    const int d = static_cast<int>(dl);
    int lo = max(0, d - nnz), hi = min(d, n_rows);
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (rowptr[mid + 1] <= d - mid - 1) lo = mid + 1;
      else hi = mid;
    }
    tile_i[t] = lo;
    tile_j[t] = d - lo;
  }
}

// ELL (column-major, ld rows per slot column) and, for HYB, the overflow of
// rows longer than K as COO entries (row, column, value) in row order.
__global__ void ell_fill_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, int n_rows, int K, int64_t ld,
                                int32_t* ell_col, double* ell_val, const int32_t* __restrict__ tail_slot,
                                const int32_t* __restrict__ tail_rowptr, int32_t* tail_row, int32_t* tail_col,
                                double* tail_val) {
  const int stride = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += stride) {
    const int k0 = rowptr[r], len = rowptr[r + 1] - k0;
    for (int j = 0; j < K; ++j) {
      const int64_t o = static_cast<int64_t>(j) * ld + r;
      if (j < len) {
        ell_col[o] = col[k0 + j];
        ell_val[o] = val[k0 + j];
      } else {
        ell_col[o] = -1;
        ell_val[o] = 0.0;
      }
    }
    if (len > K && tail_slot) {
      const int base = tail_rowptr[tail_slot[r]];
      for (int j = K; j < len; ++j) {
        tail_row[base + j - K] = r;
        tail_col[base + j - K] = col[k0 + j];
        tail_val[base + j - K] = val[k0 + j];
      }
    }
  }
}

template <class T>
int upload(T** dst, const std::vector<T>& src, int64_t pad_to, int64_t* bytes, cudaStream_t s) {
  int64_t n = std::max<int64_t>(pad_to, static_cast<int64_t>(src.size()));
  GK_TRY(dalloc_n(dst, static_cast<size_t>(std::max<int64_t>(n, 1)), bytes));
  GK_TRY_CUDA(cudaMemsetAsync(*dst, 0, sizeof(T) * std::max<int64_t>(n, 1), s));
  if (!src.empty())
    GK_TRY_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
  return GK_OK;
}

int grid1d(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, 65535)));
}

struct MatrixDeleter {
  void operator()(Matrix* m) const { matrix_release(m); }
};

// Fill the length-sorted slices: one thread per (slice, lane); entry k of
// the lane's row at off[c] + 32 k + lane, padding with column -1 and 0.
__global__ void slice_fill_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, const int32_t* __restrict__ perm,
                                  const int64_t* __restrict__ off, int64_t n_slices, int64_t n_sell,
                                  int32_t* __restrict__ scol, double* __restrict__ sval) {
  const int64_t total = n_slices * 32;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = t >> 5;
    const int lane = static_cast<int>(t & 31);
    const int64_t o0 = off[c];
    const int L = static_cast<int>((off[c + 1] - o0) >> 5);
    const int row = t < n_sell ? perm[t] : -1;
    const int k0 = row >= 0 ? rowptr[row] : 0;
    const int len = row >= 0 ? rowptr[row + 1] - k0 : 0;
    for (int k = 0; k < L; ++k) {
      const int64_t d = o0 + 32 * static_cast<int64_t>(k) + lane;
      scol[d] = k < len ? col[k0 + k] : -1;
      sval[d] = k < len ? val[k0 + k] : 0.0;
    }
  }
}

// Stored entries over the DFMA lane slots the GK_CSR kernel issues (slices:
// 32 x their longest row; a long row 32 x ceil(len / 32) plus a butterfly
// per piece).
double sliced_efficiency(const std::vector<int32_t>& rp, int64_t n) {
  std::vector<int64_t> cnt(kSliceMaxLen + 1, 0);
  double slots = 0.0, nnz = static_cast<double>(rp[n]);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t len = rp[i + 1] - rp[i];
    if (len <= kSliceMaxLen) cnt[len] += 1;
    else slots += 32.0 * ((len + 31) / 32) + 160.0 * ((len + kPieceLen - 1) / kPieceLen);
  }
  int64_t in_slice = 0;  // rows placed so far, longest first
  for (int64_t L = kSliceMaxLen; L >= 0; --L) {
    for (int64_t r = 0; r < cnt[L]; ++r, ++in_slice)
      if ((in_slice & 31) == 0) slots += 32.0 * static_cast<double>(L);
  }
  return slots > 0 ? nnz / slots : 1.0;
}

}  // namespace

int build_merge_plan(MergePlan& P, int64_t n_rows, int64_t nnz, const int32_t* rowptr,
                     const int32_t* col, const double* val, int64_t* bytes, cudaStream_t s) {
  P.n_rows = n_rows;
  P.nnz = nnz;
  P.rowptr = rowptr;
  P.col = col;
  P.val = val;
  P.n_tiles = (n_rows + nnz + kMergeTile - 1) / kMergeTile;
  const size_t nt = static_cast<size_t>(std::max<int64_t>(P.n_tiles, 1));
  GK_TRY(dalloc_n(&P.tile_i, nt + 1, bytes));
  GK_TRY(dalloc_n(&P.tile_j, nt + 1, bytes));
  GK_TRY(dalloc_n(&P.head_val, nt, bytes));
  GK_TRY(dalloc_n(&P.carry_val, nt, bytes));
  if (P.n_tiles > 0) {
    merge_plan_kernel<<<grid1d(P.n_tiles + 1, 256), 256, 0, s>>>(
        rowptr, static_cast<int>(n_rows), static_cast<int>(nnz), static_cast<int>(P.n_tiles), P.tile_i,
        P.tile_j);
    GK_TRY_CUDA(cudaGetLastError());
  }
  P.grid = merge_grid(P.n_tiles);
  return GK_OK;
}

void matrix_release(Matrix* A) {
  if (!A) return;
  if (A->refs.fetch_sub(1) != 1) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(A->device);
  void* ptrs[] = {A->rowptr, A->col, A->val, A->sl_perm, A->sl_off, A->sl_col, A->sl_val, A->pc, A->lr_row, A->lr_off, A->pc_sum,
                  A->merge.tile_i, A->merge.tile_j, A->merge.head_val, A->merge.carry_val, A->ell_col,
                  A->ell_val,
                  A->tail_rows, A->tail_rowptr, A->tail_row, A->tail_col, A->tail_val, A->tail_slot,
                  A->tail_sum, A->coo_first, A->coo_last, A->coo_head, A->coo_tail, A->partials, A->counter,
                  A->err, A->dot_st, A->stage_in, A->stage_out};
  for (void* p : ptrs) dfree(p);
  if (A->h_flag) cudaFreeHost(A->h_flag);
  if (prev >= 0) cudaSetDevice(prev);
  delete A;
}

}  // namespace gk

using namespace gk;

extern "C" int gk_matrix_create_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* rowptr,
                                    const int32_t* col, const void* val, int32_t dtype, int32_t format,
                                    void* stream, gk_matrix* out) {
  if (!out) return set_error(GK_ERR_ARG, "gk_matrix_create_csr: out is NULL");
  *out = nullptr;
  if (n_rows < 0 || n_cols < 0 || nnz < 0)
    return set_error(GK_ERR_ARG, "gk_matrix_create_csr: negative size");
  if (nnz > INT32_MAX - 64 || n_rows > INT32_MAX - 64 || n_cols > INT32_MAX ||
      n_rows + nnz > static_cast<int64_t>(INT32_MAX) - 4 * kMergeTile)
    return set_error(GK_ERR_ARG, "gk_matrix_create_csr: sizes exceed int32 indexing");
  if (!rowptr || (nnz > 0 && (!col || !val)))
    return set_error(GK_ERR_ARG, "gk_matrix_create_csr: NULL array");
  if (dtype == GK_F32)
    return set_error(GK_ERR_UNSUPPORTED, "gk_matrix_create_csr: FP32 storage is not built");
  if (dtype != GK_F64) return set_error(GK_ERR_DTYPE, "gk_matrix_create_csr: unknown dtype %d", dtype);
  if (format < GK_CSR || format > GK_AUTO)
    return set_error(GK_ERR_ARG, "gk_matrix_create_csr: unknown format %d", format);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  std::unique_ptr<Matrix, MatrixDeleter> hold(new Matrix);
  Matrix* A = hold.get();
  A->device = current_device();
  A->n_rows = n_rows;
  A->n_cols = n_cols;
  A->nnz = nnz;
  int64_t* bytes = &A->device_bytes;

  // ---- library-owned CSR copy ------------------------------------------------
  GK_TRY(dalloc_n(&A->rowptr, padded(n_rows + 1), bytes));
  GK_TRY(dalloc_n(&A->col, padded(nnz), bytes));
  GK_TRY(dalloc_n(&A->val, padded(nnz), bytes));
  GK_TRY_CUDA(cudaMemsetAsync(A->rowptr, 0, sizeof(int32_t) * padded(n_rows + 1), s));
  GK_TRY_CUDA(cudaMemsetAsync(A->col, 0, sizeof(int32_t) * padded(nnz), s));
  GK_TRY_CUDA(cudaMemsetAsync(A->val, 0, sizeof(double) * padded(nnz), s));
  GK_TRY_CUDA(cudaMemcpyAsync(A->rowptr, rowptr, sizeof(int32_t) * (n_rows + 1), cudaMemcpyDefault, s));
  if (nnz > 0) {
    GK_TRY_CUDA(cudaMemcpyAsync(A->col, col, sizeof(int32_t) * nnz, cudaMemcpyDefault, s));
    GK_TRY_CUDA(cudaMemcpyAsync(A->val, val, sizeof(double) * nnz, cudaMemcpyDefault, s));
  }
  A->h_rowptr.resize(static_cast<size_t>(n_rows + 1));
  GK_TRY_CUDA(cudaMemcpyAsync(A->h_rowptr.data(), A->rowptr, sizeof(int32_t) * (n_rows + 1),
                              cudaMemcpyDeviceToHost, s));
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  const std::vector<int32_t>& rp = A->h_rowptr;
  if (rp[0] != 0) return set_error(GK_ERR_CSR, "rowptr[0] = %d, expected 0", rp[0]);
  for (int64_t i = 0; i < n_rows; ++i)
    if (rp[i + 1] < rp[i]) return set_error(GK_ERR_CSR, "rowptr decreases at row %lld", (long long)i);
  if (rp[n_rows] != nnz)
    return set_error(GK_ERR_CSR, "rowptr[n_rows] = %d, expected nnz = %lld", rp[n_rows], (long long)nnz);

  GK_TRY(dalloc_n(&A->counter, 4, bytes));
  GK_TRY(dalloc_n(&A->err, 4, bytes));
  GK_TRY_CUDA(cudaMemsetAsync(A->counter, 0, 4 * sizeof(unsigned int), s));
  if (n_rows > 0) {
    int bad_init = INT_MAX, bad = INT_MAX;
    GK_TRY_CUDA(cudaMemcpyAsync(A->err, &bad_init, sizeof(int), cudaMemcpyHostToDevice, s));
    validate_csr_kernel<<<grid1d(n_rows, 256), 256, 0, s>>>(A->rowptr, A->col, static_cast<int>(n_rows),
                                                             static_cast<int>(n_cols), A->err);
    GK_TRY_CUDA(cudaGetLastError());
    GK_TRY_CUDA(cudaMemcpyAsync(&bad, A->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GK_TRY_CUDA(cudaStreamSynchronize(s));
    if (bad != INT_MAX)
      return set_error(GK_ERR_CSR, "row %d: column index out of range, unsorted or repeated", bad);
  }
  GK_TRY_CUDA(cudaMemsetAsync(A->err, 0, 4 * sizeof(int), s));

  // ---- format ------------------------------------------------------------------
  int fmt = format;
  if (fmt == GK_AUTO) fmt = (sliced_efficiency(rp, n_rows) >= 0.75) ? GK_CSR : GK_CSR_MERGE;
  A->format = fmt;
  if (fmt == GK_CSR) {
    // counting sort by decreasing length (ties: increasing row index)
    std::vector<int64_t> cnt(kSliceMaxLen + 2, 0);
    std::vector<int32_t> longr;
    for (int64_t i = 0; i < n_rows; ++i) {
      const int64_t len = rp[i + 1] - rp[i];
      if (len <= kSliceMaxLen) cnt[kSliceMaxLen - len + 1] += 1;
      else longr.push_back(static_cast<int32_t>(i));
    }
    for (int64_t L = 1; L <= kSliceMaxLen + 1; ++L) cnt[L] += cnt[L - 1];
    const int64_t n_sell = cnt[kSliceMaxLen + 1];
    std::vector<int32_t> perm(static_cast<size_t>(n_sell));
    for (int64_t i = 0; i < n_rows; ++i) {
      const int64_t len = rp[i + 1] - rp[i];
      if (len <= kSliceMaxLen) perm[cnt[kSliceMaxLen - len]++] = static_cast<int32_t>(i);
    }
    auto by_len = [&](int32_t x, int32_t y) {
      const int64_t lx = rp[x + 1] - rp[x], ly = rp[y + 1] - rp[y];
      return lx != ly ? lx > ly : x < y;
    };
    std::sort(longr.begin(), longr.end(), by_len);
    // long rows in pieces of kPieceLen consecutive entries (the last one
    // shorter), longest first (ties: row, then position)
    std::vector<int4> pc;
    std::vector<int32_t> lr_row, lr_off(1, 0);
    int32_t n_slot = 0;
    for (const int32_t r : longr) {
      const int32_t k0 = rp[r], k1 = rp[r + 1];
      const bool split = k1 - k0 > kPieceLen;
      for (int32_t k = k0; k < k1; k += kPieceLen)
        pc.push_back(make_int4(r, k, std::min(k1, k + kPieceLen), split ? n_slot++ : -1));
      if (split) {
        lr_row.push_back(r);
        lr_off.push_back(n_slot);
      }
    }
    std::stable_sort(pc.begin(), pc.end(), [](const int4& u, const int4& v) { return u.z - u.y > v.z - v.y; });
    const int64_t n_slices = (n_sell + 31) / 32;
    std::vector<int64_t> off(static_cast<size_t>(n_slices + 1), 0);
    for (int64_t c = 0; c < n_slices; ++c) {
      const int32_t r = perm[static_cast<size_t>(c * 32)];  // the slice's longest row
      off[c + 1] = off[c] + 32 * static_cast<int64_t>(rp[r + 1] - rp[r]);
    }
    A->n_sell = n_sell;
    A->n_slices = n_slices;
    A->sl_entries = off[n_slices];
    A->n_long = static_cast<int64_t>(longr.size());
    A->n_pc = static_cast<int64_t>(pc.size());
    A->n_lr = static_cast<int64_t>(lr_row.size());
    GK_TRY(upload(&A->sl_perm, perm, 0, bytes, s));
    GK_TRY(upload(&A->sl_off, off, 0, bytes, s));
    GK_TRY(upload(&A->pc, pc, 0, bytes, s));
    GK_TRY(upload(&A->lr_row, lr_row, 0, bytes, s));
    GK_TRY(upload(&A->lr_off, lr_off, 0, bytes, s));
    GK_TRY(dalloc_n(&A->pc_sum, static_cast<size_t>(std::max<int32_t>(n_slot, 1)), bytes));
    GK_TRY(dalloc_n(&A->sl_col, static_cast<size_t>(std::max<int64_t>(A->sl_entries, 1)), bytes));
    GK_TRY(dalloc_n(&A->sl_val, static_cast<size_t>(std::max<int64_t>(A->sl_entries, 1)), bytes));
    if (n_slices > 0) {
      slice_fill_kernel<<<grid1d(n_slices * 32, 256), 256, 0, s>>>(A->rowptr, A->col, A->val, A->sl_perm,
                                                                   A->sl_off, n_slices, n_sell, A->sl_col,
                                                                   A->sl_val);
      GK_TRY_CUDA(cudaGetLastError());
    }
    A->grid_sl = sliced_grid(A->n_pc + A->n_slices, false);
    A->grid_sl_plain = sliced_grid(A->n_pc + A->n_slices, true);
  } else if (fmt == GK_CSR_MERGE) {
    GK_TRY(build_merge_plan(A->merge, n_rows, nnz, A->rowptr, A->col, A->val, bytes, s));
  } else {  // GK_ELL, GK_HYB
    int64_t maxlen = 0;
    for (int64_t i = 0; i < n_rows; ++i) maxlen = std::max<int64_t>(maxlen, rp[i + 1] - rp[i]);
    int64_t K = maxlen;
    if (fmt == GK_ELL) {
      if (K * n_rows > 8 * nnz + n_rows)
        return set_error(GK_ERR_FORMAT,
                         "ELL would hold %lld slots for %lld entries (longest row %lld); use GK_HYB",
                         (long long)(K * n_rows), (long long)nnz, (long long)K);
    } else {
      // smallest K minimising K*n*(8+4) + overflow*(8+2*4), from the
      // histogram of row lengths
      std::vector<int64_t> hist(static_cast<size_t>(maxlen + 2), 0);
      for (int64_t i = 0; i < n_rows; ++i) hist[rp[i + 1] - rp[i]] += 1;
      // gt[k] = #rows longer than k, over[k] = sum max(0, len - k)
      std::vector<int64_t> over(static_cast<size_t>(maxlen + 2), 0), gt(static_cast<size_t>(maxlen + 2), 0);
      for (int64_t k = maxlen - 1; k >= 0; --k) {
        gt[k] = gt[k + 1] + hist[k + 1];
        over[k] = over[k + 1] + gt[k];
      }
      int64_t bestK = 0, bestc = -1;
      for (int64_t k = 0; k <= maxlen; ++k) {
        int64_t c = k * n_rows * 12 + over[k] * 16;
        if (bestc < 0 || c < bestc) {
          bestc = c;
          bestK = k;
        }
      }
      K = bestK;
    }
    A->K = K;
    A->ld = ((n_rows + 31) / 32) * 32;
    GK_TRY(dalloc_n(&A->ell_col, static_cast<size_t>(std::max<int64_t>(K * A->ld, 1)), bytes));
    GK_TRY(dalloc_n(&A->ell_val, static_cast<size_t>(std::max<int64_t>(K * A->ld, 1)), bytes));
    if (fmt == GK_HYB) {
      std::vector<int32_t> slot(static_cast<size_t>(n_rows), -1), trows, trp(1, 0);
      for (int64_t i = 0; i < n_rows; ++i) {
        int64_t len = rp[i + 1] - rp[i];
        if (len > K) {
          slot[i] = static_cast<int32_t>(trows.size());
          trows.push_back(static_cast<int32_t>(i));
          trp.push_back(trp.back() + static_cast<int32_t>(len - K));
        }
      }
      A->m_tail = static_cast<int64_t>(trows.size());
      A->tail_nnz = trp.back();
      // COO arrays in whole chunks (each lane's 16-byte loads stay inside)
      A->coo_chunks = (A->tail_nnz + kCooChunk - 1) / kCooChunk;
      const int64_t coo_n = std::max<int64_t>(A->coo_chunks * kCooChunk, padded(A->tail_nnz));
      GK_TRY(upload(&A->tail_slot, slot, 0, bytes, s));
      GK_TRY(upload(&A->tail_rows, trows, 0, bytes, s));
      GK_TRY(upload(&A->tail_rowptr, trp, padded(A->m_tail + 1), bytes, s));
      GK_TRY(dalloc_n(&A->tail_row, static_cast<size_t>(coo_n), bytes));
      GK_TRY(dalloc_n(&A->tail_col, static_cast<size_t>(coo_n), bytes));
      GK_TRY(dalloc_n(&A->tail_val, static_cast<size_t>(coo_n), bytes));
      GK_TRY(dalloc_n(&A->tail_sum, static_cast<size_t>(std::max<int64_t>(A->m_tail, 1)), bytes));
      GK_TRY_CUDA(cudaMemsetAsync(A->tail_row, 0, sizeof(int32_t) * coo_n, s));
      GK_TRY_CUDA(cudaMemsetAsync(A->tail_col, 0, sizeof(int32_t) * coo_n, s));
      GK_TRY_CUDA(cudaMemsetAsync(A->tail_val, 0, sizeof(double) * coo_n, s));
      const size_t nc = static_cast<size_t>(std::max<int64_t>(A->coo_chunks, 1));
      GK_TRY(dalloc_n(&A->coo_first, nc, bytes));
      GK_TRY(dalloc_n(&A->coo_last, nc, bytes));
      GK_TRY(dalloc_n(&A->coo_head, nc, bytes));
      GK_TRY(dalloc_n(&A->coo_tail, nc, bytes));
      A->grid_coo = coo_grid(A->coo_chunks);
    }
    if (n_rows > 0) {
      ell_fill_kernel<<<grid1d(n_rows, 256), 256, 0, s>>>(
          A->rowptr, A->col, A->val, static_cast<int>(n_rows), static_cast<int>(K), A->ld, A->ell_col,
          A->ell_val, fmt == GK_HYB ? A->tail_slot : nullptr, A->tail_rowptr, A->tail_row, A->tail_col,
          A->tail_val);
      GK_TRY_CUDA(cudaGetLastError());
    }
    A->grid_ell = ell_grid(n_rows);
  }
  A->max_grid = std::max(spmv_max_grid(*A), 4 * sm_count());
  GK_TRY(dalloc_n(&A->partials, static_cast<size_t>(2 * (A->max_grid + kFixupMaxGrid)), bytes));
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  *out = reinterpret_cast<gk_matrix>(hold.release());
  return GK_OK;
}

extern "C" int gk_matrix_get_info(gk_matrix h, gk_matrix_info* info) {
  Matrix* A = as_matrix(h);
  if (!A || !info) return set_error(GK_ERR_ARG, "gk_matrix_get_info: NULL argument");
  info->n_rows = A->n_rows;
  info->n_cols = A->n_cols;
  info->nnz = A->nnz;
  info->format = A->format;
  info->dtype = GK_F64;
  info->ell_width = (A->format == GK_ELL || A->format == GK_HYB) ? A->K : 0;
  info->tail_rows = A->m_tail;
  info->tail_nnz = A->tail_nnz;
  info->short_items = A->n_slices;
  info->long_rows = A->n_long;
  info->split_rows = A->n_lr;
  info->tiles = A->merge.n_tiles;
  info->device_bytes = A->device_bytes;
  // the stored operator once (CSR: values, indices, row pointers; ELL: the
  // entries' values and indices; HYB: ELL entries + COO entries with their
  // row index), x read once, y written once
  int64_t mat = A->nnz * 12 + (A->n_rows + 1) * 4;
  if (A->format == GK_ELL) mat = A->nnz * 12;
  if (A->format == GK_HYB) mat = (A->nnz - A->tail_nnz) * 12 + A->tail_nnz * 16;
  info->spmv_bytes = mat + A->n_cols * 8 + A->n_rows * 8;
  return GK_OK;
}

extern "C" int gk_matrix_destroy(gk_matrix h) {
  if (!h) return set_error(GK_ERR_ARG, "gk_matrix_destroy: NULL handle");
  matrix_release(as_matrix(h));
  return GK_OK;
}
