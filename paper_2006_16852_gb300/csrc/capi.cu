// capi.cu -- error reporting, allocation helpers, host/device vector
// arguments, the apply calls (Section 4.2) and the reproducible dot product.
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "gk_device.cuh"
#include "gk_internal.h"

namespace gk {

namespace {
thread_local std::string g_last_error;
}

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error so later calls can proceed
  return set_error(e == cudaErrorMemoryAllocation ? GK_ERR_ALLOC : GK_ERR_CUDA, "%s: %s (%s)", what,
                   cudaGetErrorString(e), cudaGetErrorName(e));
}

int dalloc(void** p, size_t bytes, int64_t* counter) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(GK_ERR_ALLOC, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  if (counter) *counter += static_cast<int64_t>(bytes);
  return GK_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

namespace {
std::mutex g_pool_mu;
bool g_pool_ready[64] = {};
}  // namespace

int dalloc_async(void** p, size_t bytes, int64_t* counter, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  const int dev = current_device();
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool_ready[dev]) {
      // keep up to 8 GB of freed memory in this process's default pool of the
      // device instead of returning it at the next synchronization
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = 8ull << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
      cudaGetLastError();
      g_pool_ready[dev] = true;
    }
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(GK_ERR_ALLOC, "cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  if (counter) *counter += static_cast<int64_t>(bytes);
  return GK_OK;
}

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return d;
}

int set_smem(const void* fn, size_t smem) {
  GK_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  GK_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   static_cast<int>(cudaSharedmemCarveoutMaxShared)));
  return GK_OK;
}

int sm_count() {
  static int cache[64] = {};
  int d = current_device();
  if (d >= 0 && d < 64 && cache[d]) return cache[d];
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    v = 1;
  }
  if (d >= 0 && d < 64) cache[d] = v;
  return v;
}

int vec_in(VecArg& v, const void* p, int64_t n, double** staging, int64_t* bytes, bool copy_in, int device,
           cudaStream_t s) {
  v.user = p;
  v.staged = false;
  v.dev = nullptr;
  if (n == 0) return GK_OK;
  if (!p) return set_error(GK_ERR_ARG, "NULL vector");
  if (reinterpret_cast<uintptr_t>(p) % 8 != 0) return set_error(GK_ERR_ARG, "vector not 8-byte aligned");
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    at.type = cudaMemoryTypeUnregistered;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    if (at.type == cudaMemoryTypeDevice && at.device != device)
      return set_error(GK_ERR_NOT_DEVICE, "vector lives on device %d, operator on device %d", at.device,
                       device);
    v.dev = static_cast<double*>(const_cast<void*>(p));
    return GK_OK;
  }
  if (!*staging) GK_TRY(dalloc_n(staging, static_cast<size_t>(n + 1), bytes));
  v.staged = true;
  v.dev = *staging;
  if (copy_in)
    GK_TRY_CUDA(cudaMemcpyAsync(*staging, p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  return GK_OK;
}

int vec_out(VecArg& v, int64_t n, cudaStream_t s) {
  if (!v.staged || n == 0) return GK_OK;
  GK_TRY_CUDA(cudaMemcpyAsync(const_cast<void*>(v.user), v.dev, sizeof(double) * n, cudaMemcpyDeviceToHost,
                              s));
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  return GK_OK;
}

namespace {

// True for host memory (pinned or pageable).
bool is_host(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// Deterministic dot product: per-thread fma accumulation over a grid-stride
// range, then the fixed-order grid reduction.
__global__ void __launch_bounds__(256) dot_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                  int64_t n, double* partials, unsigned int* counter,
                                                  double* result) {
  __shared__ double scratch[kRedScratch];
  double a[1] = {0.0};
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    a[0] = fma(__ldg(x + i), __ldg(y + i), a[0]);
  double out[1];
  if (grid_sum<1>(a, partials, counter, scratch, out) && threadIdx.x == 0) result[0] = out[0];
}

// Gathered dot product sum_k v_k x_{c_k} over a stream of (c_k, v_k) pairs:
// the SpMV's per-entry work (a streamed index and value, a gathered x, one
// fma) without its row structure.  Each thread takes entries k = g, g + T,
// ... (coalesced, streamed), kGatherBatch gathers in flight; 8 blocks of 256
// threads per SM within 32 registers.  An index outside [0, n_x) contributes
// 0 (checked per entry; the SpMV kernels rely on the validation at matrix
// creation instead).
constexpr int kGatherBatch = 8;

__global__ void __launch_bounds__(256, 8) gather_dot_kernel(const int32_t* __restrict__ c,
                                                            const double* __restrict__ v,
                                                            const double* __restrict__ x, int64_t n,
                                                            uint32_t n_x, double* partials,
                                                            unsigned int* counter, double* result) {
  __shared__ double scratch[kRedScratch];
  double a[1] = {0.0};
  const int64_t T = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; k + (kGatherBatch - 1) * T < n; k += kGatherBatch * T) {
    int cc[kGatherBatch];
    double vv[kGatherBatch], xv[kGatherBatch];
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u) cc[u] = __ldcs(c + k + u * T);
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u) vv[u] = __ldcs(v + k + u * T);
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u) xv[u] = static_cast<uint32_t>(cc[u]) < n_x ? __ldg(x + cc[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u) a[0] = fma(vv[u], xv[u], a[0]);
  }
  for (; k < n; k += T) {
    const int ck = __ldcs(c + k);
    a[0] = fma(__ldcs(v + k), static_cast<uint32_t>(ck) < n_x ? __ldg(x + ck) : 0.0, a[0]);
  }
  double out[1];
  if (grid_sum<1>(a, partials, counter, scratch, out) && threadIdx.x == 0) result[0] = out[0];
}

struct DotWorkspace {
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  int grid = 0;
};
std::mutex g_dot_mu;
DotWorkspace g_dot_ws[64];
DotWorkspace g_gather_ws[64];

}  // namespace

int dot_grid() { return 4 * sm_count(); }

}  // namespace gk

using namespace gk;

extern "C" const char* gk_last_error(void) { return gk::g_last_error.c_str(); }

extern "C" int32_t gk_version(void) { return 100; }

extern "C" int gk_apply_adv(double alpha, gk_matrix h, const void* b, double beta, void* x, void* stream) {
  Matrix* A = as_matrix(h);
  if (!A) return set_error(GK_ERR_ARG, "gk_apply: NULL matrix");
  if (b == x && A->n_rows > 0) return set_error(GK_ERR_ARG, "gk_apply: b and x must not alias");
  DeviceGuard g(A->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (A->n_rows == 0) return GK_OK;
  VecArg vb, vx;
  GK_TRY(vec_in(vb, b, A->n_cols, &A->stage_in, &A->device_bytes, true, A->device, s));
  GK_TRY(vec_in(vx, x, A->n_rows, &A->stage_out, &A->device_bytes, beta != 0.0, A->device, s));
  Epi e;
  e.mode = (alpha == 1.0 && beta == 0.0) ? EPI_COPY : EPI_PLAIN;
  e.alpha = alpha;
  e.beta = beta;
  e.beta_zero = beta == 0.0 ? 1 : 0;
  e.y = vx.dev;
  e.err = A->err;
  GK_TRY(spmv_launch(*A, vb.dev, e, s));
  return vec_out(vx, A->n_rows, s);
}

extern "C" int gk_apply(gk_matrix h, const void* b, void* x, void* stream) {
  return gk_apply_adv(1.0, h, b, 0.0, x, stream);
}

extern "C" int gk_apply_dot(gk_matrix h, const double* b, double* x, const double* u, double* result,
                            void* stream) {
  Matrix* A = as_matrix(h);
  if (!A || !b || !x || !u || !result) return set_error(GK_ERR_ARG, "gk_apply_dot: NULL argument");
  if (b == x) return set_error(GK_ERR_ARG, "gk_apply_dot: b and x must not alias");
  if (is_host(b) || is_host(x) || is_host(u) || is_host(result))
    return set_error(GK_ERR_NOT_DEVICE, "gk_apply_dot: vectors and result must be device memory");
  if (A->n_rows != A->n_cols) return set_error(GK_ERR_DIM, "gk_apply_dot: matrix is not square");
  DeviceGuard g(A->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!A->dot_st) {
    GK_TRY(dalloc_n(&A->dot_st, 1, &A->device_bytes));
    GK_TRY_CUDA(cudaMemsetAsync(A->dot_st, 0, sizeof(SolverState), s));
  }
  if (A->n_rows == 0) {
    GK_TRY_CUDA(cudaMemsetAsync(result, 0, sizeof(double), s));
    return GK_OK;
  }
  // the SpMV's EPI_DOT epilogue of the Krylov steps: x = A b and u.x in one
  // pass, the fixed-order sum left in dot_st->red[0] by the last block
  Epi e;
  e.mode = EPI_DOT;
  e.fin = FIN_NONE;
  e.u = u;
  e.y = x;
  e.st = A->dot_st;
  e.skip_mode = 0;
  e.partials = A->partials;
  e.counter = A->counter;
  e.err = A->err;
  GK_TRY(spmv_launch(*A, b, e, s));
  GK_TRY_CUDA(cudaMemcpyAsync(result, &A->dot_st->red[0], sizeof(double), cudaMemcpyDeviceToDevice, s));
  return GK_OK;
}

extern "C" int gk_dot(int64_t n, const double* x, const double* y, double* result, void* stream) {
  if (n < 0 || !result || (n > 0 && (!x || !y))) return set_error(GK_ERR_ARG, "gk_dot: bad argument");
  if (is_host(x) || is_host(y) || is_host(result))
    return set_error(GK_ERR_NOT_DEVICE, "gk_dot: x, y and result must be device memory");
  int dev = current_device();
  if (dev < 0 || dev >= 64) return set_error(GK_ERR_UNSUPPORTED, "gk_dot: device index %d", dev);
  DotWorkspace* ws;
  {
    std::lock_guard<std::mutex> lock(g_dot_mu);
    ws = &g_dot_ws[dev];
    if (!ws->partials) {
      ws->grid = dot_grid();
      GK_TRY(dalloc_n(&ws->partials, static_cast<size_t>(ws->grid), nullptr));
      GK_TRY(dalloc_n(&ws->counter, 1, nullptr));
      GK_TRY_CUDA(cudaMemset(ws->counter, 0, sizeof(unsigned int)));
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dot_kernel<<<ws->grid, 256, 0, s>>>(x, y, n, ws->partials, ws->counter, result);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

extern "C" int gk_gather_dot(int64_t n, const int32_t* c, const double* v, const double* x, int64_t n_x,
                             double* result, void* stream) {
  if (n < 0 || n_x < 0 || n_x > 0x7fffffff || !result || (n > 0 && (!c || !v || !x)))
    return set_error(GK_ERR_ARG, "gk_gather_dot: bad argument");
  if (is_host(c) || is_host(v) || is_host(x) || is_host(result))
    return set_error(GK_ERR_NOT_DEVICE, "gk_gather_dot: c, v, x and result must be device memory");
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return set_error(GK_ERR_UNSUPPORTED, "gk_gather_dot: device index %d", dev);
  DotWorkspace* ws;
  {
    std::lock_guard<std::mutex> lock(g_dot_mu);
    ws = &g_gather_ws[dev];
    if (!ws->partials) {
      ws->grid = 8 * sm_count();
      GK_TRY(dalloc_n(&ws->partials, static_cast<size_t>(ws->grid), nullptr));
      GK_TRY(dalloc_n(&ws->counter, 1, nullptr));
      GK_TRY_CUDA(cudaMemset(ws->counter, 0, sizeof(unsigned int)));
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gather_dot_kernel<<<ws->grid, 256, 0, s>>>(c, v, x, n, static_cast<uint32_t>(n_x), ws->partials, ws->counter,
                                             result);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

// ---------------------------------------------------------------------------
// gk_dot_noalloc: gk_dot for callers that cannot allocate device memory.  The
// reduction scratch (one partial sum per block, then the arrival counter) is
// a file-scope device array instead of a cudaMalloc'd workspace.  Its host
// address is looked up once per device with cudaGetSymbolAddress (the host
// name of the array is only a stand-in and must never reach a kernel).
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxBlocks = 1024;
// [0, kNoAllocMaxBlocks): block partials; the next 8 bytes: the counter.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 32];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {};

}  // namespace

extern "C" int gk_dot_noalloc(int64_t n, const double* x, const double* y, double* result, void* stream) {
  if (n < 0 || !result || (n > 0 && (!x || !y))) return set_error(GK_ERR_ARG, "gk_dot_noalloc: bad argument");
  if (is_host(x) || is_host(y) || is_host(result))
    return set_error(GK_ERR_NOT_DEVICE, "gk_dot_noalloc: x, y and result must be device memory");
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return set_error(GK_ERR_UNSUPPORTED, "gk_dot_noalloc: device index %d", dev);
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_error(e, "gk_dot_noalloc: cudaGetSymbolAddress");
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  const int grid = dot_grid();
  if (grid > kNoAllocMaxBlocks)
    return set_error(GK_ERR_UNSUPPORTED,
                     "gk_dot_noalloc: the reduction needs %d block partials, the static scratch holds %d "
                     "(GPUs with more than %d SMs are not supported)",
                     grid, kNoAllocMaxBlocks, kNoAllocMaxBlocks / 4);
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNoAllocMaxBlocks);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GK_TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
  dot_kernel<<<grid, 256, 0, s>>>(x, y, n, scratch, counter, result);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

// ---------------------------------------------------------------------------
// gk_wait_selftest: the failure path of the bounded device-side waits.  One
// warp waits, with the same mbar_wait every bulk-copy consumer uses, on an
// mbarrier phase that nothing completes (one expected arrival, none made, no
// copy issued).  The wait gives up at its clock limit, sets kErrTimeout in
// the error word and the kernel returns, so the context stays usable.
// ---------------------------------------------------------------------------
namespace gk {

__global__ void __launch_bounds__(32) wait_selftest_kernel(int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  const bool ok = mbar_wait(&bar, 0u, threadIdx.x == 0 ? err : nullptr);
  if (threadIdx.x == 0 && ok) atomicOr(err, 2);  // the phase completed: not expected
}

}  // namespace gk

extern "C" int gk_wait_selftest(int32_t* err_out, void* stream) {
  if (!err_out) return set_error(GK_ERR_ARG, "gk_wait_selftest: err_out is null");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d = nullptr;
  GK_TRY_CUDA(cudaMalloc(&d, sizeof(int)));
  int h = -1;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_error(e, "gk_wait_selftest");
  *err_out = h;
  return GK_OK;
}

// ---------------------------------------------------------------------------
// gk_fp64_rate: the rate at which this GPU retires FP64 fused multiply-adds,
// measured (the SpMV and Krylov kernels issue one per stored entry and a few
// per row; on this GPU that rate, not HBM, is often what bounds them).
// ---------------------------------------------------------------------------
namespace gk {
namespace {

constexpr int kRateChains = 8;  // independent FMA chains per thread
__device__ double g_rate_sink;  // written only if a result is impossible: keeps the chains live

__global__ void __launch_bounds__(256) fp64_rate_kernel(int64_t iters, double b, double c) {
  double a[kRateChains];
#pragma unroll
  for (int k = 0; k < kRateChains; ++k) a[k] = 1e-3 * threadIdx.x + k;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kRateChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kRateChains; ++k) s += a[k];
  if (s == -1.0) g_rate_sink = s;
}

}  // namespace
}  // namespace gk

extern "C" int gk_fp64_rate(int64_t iters, double* tflops, void* stream) {
  if (!tflops || iters < 1) return set_error(GK_ERR_ARG, "gk_fp64_rate: bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = 8 * sm_count();  // 8 blocks of 256 threads: every SM full
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fp64_rate_kernel<<<grid, 256, 0, s>>>(1, 0.999999, 1e-6);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    fp64_rate_kernel<<<grid, 256, 0, s>>>(iters, 0.999999, 1e-6);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_error(e, "gk_fp64_rate");
  const double flops = 2.0 * static_cast<double>(iters) * kRateChains * 256.0 * grid;
  *tflops = ms > 0.0f ? flops / (static_cast<double>(ms) * 1e-3) / 1e12 : 0.0;
  return GK_OK;
}
