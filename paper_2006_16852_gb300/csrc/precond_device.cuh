// precond_device.cuh -- device pieces of the Jacobi preconditioners shared by
// the standalone apply and the fused Krylov steps.
#pragma once

#include "gk_internal.h"

namespace gk {

// Block-Jacobi lane mapping: a warp serves bpw = 32 / bs blocks; lane l works
// on row (l % bs) of block (warp_block0 + l / bs).
struct BjLane {
  int blk;     // block index
  int i;       // row inside the block
  int m;       // rows of this block (bs, or fewer for the last block)
  int base;    // first lane of this block's lane group
  int row;     // global row
  bool active;
};

__device__ __forceinline__ BjLane bj_lane(int warp_block0, int lane, int bs, int n, int nblocks) {
  BjLane L;
  const int bpw = 32 / bs;
  const int sub = lane / bs;
  L.i = lane - sub * bs;
  L.blk = warp_block0 + sub;
  L.base = sub * bs;
  L.m = 0;
  L.row = 0;
  L.active = false;
  if (sub < bpw && L.blk < nblocks) {
    const int r0 = L.blk * bs;
    L.m = min(bs, n - r0);
    L.row = r0 + L.i;
    L.active = L.i < L.m;
  }
  return L;
}

// z_i = sum_j Dinv(i, j) r_j for the lane's block, with the r_j held by the
// lanes of the block's group; blocks are stored row-major (entry (i, j) at
// i * m + j), block k at offset k * bs * bs.  Sum in increasing j via fma,
// the order of the CPU reference.  BS > 0: the block size known at compile
// time -- a full block's row is fetched with 16-byte loads, all issued before
// the sum; BS = 0: any block size.  The loads may diverge; every lane of the
// warp executes the shuffles.
template <int BS>
__device__ __forceinline__ double bj_apply_lane(const double* __restrict__ blocks, const BjLane& L, int bs,
                                                double r_mine) {
  if constexpr (BS == 0) {
    double z = 0.0;
    const int64_t off = static_cast<int64_t>(L.blk) * bs * bs + static_cast<int64_t>(L.i) * L.m;
    for (int j = 0; j < bs; ++j) {
      const double rj = __shfl_sync(0xffffffffu, r_mine, (L.base + j) & 31);
      if (L.active && j < L.m) z = fma(__ldg(blocks + off + j), rj, z);
    }
    return z;
  } else {
    double dv[BS];
#pragma unroll
    for (int j = 0; j < BS; ++j) dv[j] = 0.0;
    if (L.active) {
      const int64_t off = static_cast<int64_t>(L.blk) * BS * BS + static_cast<int64_t>(L.i) * L.m;
      if (L.m == BS && BS % 2 == 0) {
        const double2* src = reinterpret_cast<const double2*>(blocks + off);
#pragma unroll
        for (int k = 0; k < BS / 2; ++k) {
          const double2 v = __ldg(src + k);
          dv[2 * k] = v.x;
          dv[2 * k + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < BS; ++j)
          if (j < L.m) dv[j] = __ldg(blocks + off + j);
      }
    }
    double z = 0.0;
#pragma unroll
    for (int j = 0; j < BS; ++j) {
      const double rj = __shfl_sync(0xffffffffu, r_mine, (L.base + j) & 31);
      if (L.active && j < L.m) z = fma(dv[j], rj, z);
    }
    return z;
  }
}

// Calls body<BS>() with BS = bs for the block sizes that have a compiled,
// vectorised apply, else BS = 0.
#define GK_BJ_DISPATCH(bs, CALL) \
  do {                           \
    switch (bs) {                \
      case 4: CALL(4); break;    \
      case 8: CALL(8); break;    \
      case 16: CALL(16); break;  \
      case 32: CALL(32); break;  \
      default: CALL(0); break;   \
    }                            \
  } while (0)

}  // namespace gk
