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
// lanes of the block's group; blocks are stored column-major, block k at
// offset k * bs * bs.  Sum in increasing j via fma, the order of the CPU
// reference.  Every lane of the warp must call it.
__device__ __forceinline__ double bj_apply_lane(const double* __restrict__ blocks, const BjLane& L, int bs,
                                                double r_mine) {
  double z = 0.0;
  const int64_t off = static_cast<int64_t>(L.blk) * bs * bs;
  for (int j = 0; j < bs; ++j) {
    const double rj = __shfl_sync(0xffffffffu, r_mine, (L.base + j) & 31);
    if (L.active && j < L.m) z = fma(__ldg(blocks + off + static_cast<int64_t>(j) * L.m + L.i), rj, z);
  }
  return z;
}

}  // namespace gk
