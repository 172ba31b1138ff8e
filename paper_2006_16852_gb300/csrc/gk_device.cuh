// gk_device.cuh -- device-side building blocks shared by the kernels:
// bulk asynchronous copies (TMA, cp.async.bulk) into shared memory completed
// on an mbarrier, bounded waits, and the fixed-order FP64 grid reduction.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gk {

// Device error word bits (SolverState::err / Workspace::err).
constexpr int kErrTimeout = 1;

// A wait gives up after this many failed polls (each try_wait may suspend the
// thread for a hardware-defined interval); the wall-clock limit below is the
// binding one in practice.
constexpr uint32_t kMaxPolls = 1u << 26;
// ~2 s at the 2.07 GHz maximum SM clock.
constexpr long long kMaxWaitCycles = 4000000000LL;

// Programmatic dependent launch: a kernel launched with launch_pdl (below)
// may be scheduled while the kernel before it in the stream is still
// finishing; its threads call pdl_wait() before touching anything that
// kernel produced (it returns once that grid has completed and its memory
// operations are visible; in a kernel launched without the attribute it
// returns at once).  Every kernel that launch_pdl starts calls it first, so
// the stream's order holds transitively.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Lets the next kernel of the stream (if launched with launch_pdl) be
// scheduled before this grid has finished: its blocks take the SM slots that
// this grid's blocks free, run their prologue and wait in pdl_wait() until
// this grid has completed.  Called after pdl_wait(), so a kernel's dependents
// never start before the kernel ahead of it has completed, and a prologue may
// touch anything but this grid's output.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Brings the line holding *p into L2 (a hint: no data comes back and L1 is
// not involved, so a prologue's prefetch cannot observe a stale copy).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared (both 16-byte aligned, bytes % 16 == 0),
// completing `bytes` transactions on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`.  Returns false (and sets
// kErrTimeout in *err) if the limit is reached.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  for (uint32_t i = 0; i < kMaxPolls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > kMaxWaitCycles) break;
  }
  if (err) atomicOr(err, kErrTimeout);
  return false;
}

// ---------------------------------------------------------------------------
// Fixed-order FP64 reductions.  A block sums its threads' values in one warp
// (block_sum below); the grid sums per-block partials in the last block to
// arrive (an integer ticket decides which block that is, the order of the sum
// does not depend on it).  The result is identical from run to run for a
// fixed grid and block shape.
// ---------------------------------------------------------------------------

// Shared scratch (doubles) a reduction of up to two values over a block of up
// to 256 threads needs.
constexpr int kRedScratch = 512;

template <int K, typename T>
__device__ __forceinline__ void warp_sum(T (&v)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
}

// Sum over the block; the result is valid in thread 0.  Per-thread values go
// to shared memory and warp 0 alone adds them (lane l sums threads l, l+32,
// ... in order, then one xor butterfly): an FP64 add tree in every warp would
// cost the (slow) FP64 pipe about three times as much.
// scratch: >= K * blockDim.x doubles; blockDim.x a multiple of 32, <= 1024.
template <int K, typename T>
__device__ __forceinline__ void block_sum(T (&v)[K], T* scratch) {
  const int nt = blockDim.x;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) scratch[k * nt + threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
    T w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      w[k] = scratch[k * nt + threadIdx.x];
      for (int t = threadIdx.x + 32; t < nt; t += 32) w[k] += scratch[k * nt + t];
    }
    warp_sum<K, T>(w);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = w[k];
    }
  }
}

// Grid-wide sum.  Every block calls it with its threads' values; returns true
// in exactly one block (the last to arrive), where thread 0 holds the totals
// in out[].  partials: >= gridDim.x*K doubles; counter: zero on entry, reset
// to zero by the last block.
template <int K, typename T>
__device__ __forceinline__ bool grid_sum(T (&v)[K], T* partials, unsigned int* counter, T* scratch,
                                         T (&out)[K]) {
  __shared__ unsigned int s_last;
  block_sum<K, T>(v, scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[blockIdx.x * K + k] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  T w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = T(0);
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] += __ldcg(partials + b * K + k);
  }
  block_sum<K, T>(w, scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = w[k];
    *counter = 0u;
  }
  return true;
}

}  // namespace gk
