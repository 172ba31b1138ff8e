// wsnet.cu -- the learned warm start: a small convolutional network that
// predicts the initial guess x0 of a variable-coefficient diffusion solve
// from the log-coefficient field g and the right-hand side b, trained on
// solutions the library's own solver produced.  Not in the paper: it extends
// the method, and plain zero-start CG stays the reference it is judged by.
//
// Network: six 3x3 convolutions with dilations d_l and zero padding,
// channels 2 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU between layers.
// Input (B, 2, H, W) = [g, b / rms(b)]; output (B, 1, H, W) =
// x / (rms(b) * out_scale).  Activations are NCHW.
//
// Training (FP32, deterministic): forward, mean-squared-error loss, backward
// (data gradients as a forward convolution with flipped, transposed weights;
// weight gradients as per-block partial sums reduced in a fixed order), Adam.
// Inference: weights, biases and activations in BF16, products formed in FP32
// (exact for BF16 operands) and summed in FP32; the four 32 -> 32 layers run
// on the tensor cores (tcgen05.mma, accumulator in tensor memory).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "gk_device.cuh"
#include "gk_internal.h"

namespace gk {
namespace {

constexpr int kLayers = 6;
constexpr int kCh[kLayers + 1] = {2, 32, 32, 32, 32, 32, 1};
constexpr int kConvThreads = 256;
constexpr int kWgradRows = 4;  // image rows per weight-gradient block

__device__ __forceinline__ float to_f(float v) { return v; }
template <typename T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }

enum ConvMode { CONV_LINEAR = 0, CONV_RELU = 1, CONV_MASK = 2 };

// y[b, o, p] = epilogue(sum_{c, ky, kx} w[o, c, ky, kx] x[b, c, p + d (ky-1, kx-1)])
// One thread per output pixel computes all COUT channels; the weights sit in
// shared memory as [c * 9 + tap][o] (o padded to a multiple of 4) and are
// read as float4 broadcasts.  Sum order: c, then ky, then kx, then + bias.
// CONV_MASK (data gradient): no bias, result * (mask[b, o, p] > 0).
template <int CIN, int COUT, int MODE, typename TI, typename TW, typename TO>
__global__ void __launch_bounds__(kConvThreads) conv_fwd_kernel(const TI* __restrict__ x, const TW* __restrict__ w,
                                                                const TW* __restrict__ bias, int H, int W, int dil,
                                                                TO* __restrict__ y, const float* __restrict__ mask) {
  constexpr int CO4 = (COUT + 3) / 4 * 4;
  __shared__ __align__(16) float ws[CIN * 9 * CO4];
  __shared__ float bs[CO4];
  for (int idx = threadIdx.x; idx < CIN * 9 * CO4; idx += blockDim.x) {
    const int ct = idx / CO4, o = idx - ct * CO4;
    ws[idx] = o < COUT ? to_f(w[o * CIN * 9 + ct]) : 0.0f;
  }
  for (int o = threadIdx.x; o < CO4; o += blockDim.x) bs[o] = (MODE != CONV_MASK && o < COUT) ? to_f(bias[o]) : 0.0f;
  __syncthreads();
  const int HW = H * W;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  const int b = blockIdx.y;
  const int i = p / W, j = p - (p / W) * W;
  float acc[CO4];
#pragma unroll
  for (int o = 0; o < CO4; ++o) acc[o] = 0.0f;
  const TI* xb = x + static_cast<int64_t>(b) * CIN * HW;
  for (int c = 0; c < CIN; ++c) {
    const TI* xc = xb + static_cast<int64_t>(c) * HW;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int ii = i + dil * (ky - 1);
      const bool rok = ii >= 0 && ii < H;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int jj = j + dil * (kx - 1);
        const float v = (rok && jj >= 0 && jj < W) ? to_f(xc[ii * W + jj]) : 0.0f;
        const float4* wr = reinterpret_cast<const float4*>(ws + (c * 9 + ky * 3 + kx) * CO4);
#pragma unroll
        for (int q = 0; q < CO4 / 4; ++q) {
          const float4 wv = wr[q];
          acc[4 * q] = fmaf(wv.x, v, acc[4 * q]);
          acc[4 * q + 1] = fmaf(wv.y, v, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(wv.z, v, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(wv.w, v, acc[4 * q + 3]);
        }
      }
    }
  }
  const int64_t ob = static_cast<int64_t>(b) * COUT * HW + p;
#pragma unroll
  for (int o = 0; o < COUT; ++o) {
    float r = acc[o];
    if (MODE == CONV_MASK) {
      r = mask[ob + static_cast<int64_t>(o) * HW] > 0.0f ? r : 0.0f;
    } else {
      r += bs[o];
      if (MODE == CONV_RELU) r = fmaxf(r, 0.0f);
    }
    y[ob + static_cast<int64_t>(o) * HW] = from_f<TO>(r);
  }
}

// Partial weight and bias gradients of one layer over kWgradRows image rows
// of one sample:  dw[o, c, tap] += sum_x dy[b, o, y, x] x[b, c, y + d (ky-1), x + d (kx-1)],
// dbias[o] += sum_x dy[b, o, y, x].  A thread owns CO_T output channels of one
// input channel for one residue class of x (XSPLIT classes); the sums (slot
// = block, STRIDE = COUT * CIN * 9 + COUT floats in the parameter layout)
// of the block's residue classes are summed first (in class order, through
// shared memory) and the block writes one slot; the slots are summed in a
// fixed order by wgrad_chunk_kernel and wgrad_final_kernel.
template <int CIN, int COUT>
struct WgradShape {
  static constexpr int CO_T = COUT >= 4 ? 4 : 1;
  static constexpr int NG = CIN * (COUT / CO_T);
  static constexpr int XSPLIT = kConvThreads / NG;
  static constexpr int STRIDE = COUT * CIN * 9 + COUT;
  static_assert(NG * XSPLIT == kConvThreads, "thread mapping");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) conv_wgrad_kernel(const float* __restrict__ x,
                                                                  const float* __restrict__ dy, int H, int W,
                                                                  int dil, float* __restrict__ partials) {
  using S = WgradShape<CIN, COUT>;
  extern __shared__ float sm[];
  const int DS = W | 1;                  // odd row strides: conflict-free
  const int XS = (W + 2 * dil) | 1;
  float* dys = sm;                       // [COUT][DS]
  float* xs = dys + COUT * DS;           // [3][CIN][XS], x position p stored at p + dil
  const int t = threadIdx.x;
  const int g = t / S::XSPLIT, s = t - (t / S::XSPLIT) * S::XSPLIT;
  const int ci = g / (COUT / S::CO_T), co0 = (g - ci * (COUT / S::CO_T)) * S::CO_T;
  const int b = blockIdx.y;
  const int y0 = blockIdx.x * kWgradRows;
  const int HW = H * W;
  float acc[S::CO_T][9], dacc[S::CO_T];
#pragma unroll
  for (int k = 0; k < S::CO_T; ++k) {
    dacc[k] = 0.0f;
#pragma unroll
    for (int tp = 0; tp < 9; ++tp) acc[k][tp] = 0.0f;
  }
  for (int yy = y0; yy < min(y0 + kWgradRows, H); ++yy) {
    __syncthreads();
    for (int idx = t; idx < COUT * W; idx += kConvThreads) {
      const int o = idx / W, xx = idx - o * W;
      dys[o * DS + xx] = dy[(static_cast<int64_t>(b) * COUT + o) * HW + yy * W + xx];
    }
    const int XW = W + 2 * dil;
    for (int idx = t; idx < 3 * CIN * XW; idx += kConvThreads) {
      const int row = idx / XW, q = idx - row * XW;
      const int ky = row / CIN, c = row - ky * CIN;
      const int iy = yy + dil * (ky - 1), ix = q - dil;
      float v = 0.0f;
      if (iy >= 0 && iy < H && ix >= 0 && ix < W) v = x[(static_cast<int64_t>(b) * CIN + c) * HW + iy * W + ix];
      xs[row * XS + q] = v;
    }
    __syncthreads();
    for (int xx = s; xx < W; xx += S::XSPLIT) {
      float d[S::CO_T];
#pragma unroll
      for (int k = 0; k < S::CO_T; ++k) d[k] = dys[(co0 + k) * DS + xx];
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const float* xr = xs + (ky * CIN + ci) * XS + xx;
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const float v = xr[dil * kx];
#pragma unroll
          for (int k = 0; k < S::CO_T; ++k) acc[k][ky * 3 + kx] = fmaf(d[k], v, acc[k][ky * 3 + kx]);
        }
      }
      if (ci == 0) {
#pragma unroll
        for (int k = 0; k < S::CO_T; ++k) dacc[k] += d[k];
      }
    }
  }
  __syncthreads();  // the staging area becomes the class reduction buffer
  float* rs = sm + static_cast<int64_t>(s) * S::STRIDE;
#pragma unroll
  for (int k = 0; k < S::CO_T; ++k) {
#pragma unroll
    for (int tp = 0; tp < 9; ++tp) rs[((co0 + k) * CIN + ci) * 9 + tp] = acc[k][tp];
    if (ci == 0) rs[COUT * CIN * 9 + co0 + k] = dacc[k];
  }
  __syncthreads();
  float* out = partials + (static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x) * S::STRIDE;
  for (int e = t; e < S::STRIDE; e += kConvThreads) {
    float sum = 0.0f;
#pragma unroll
    for (int c = 0; c < S::XSPLIT; ++c) sum += sm[c * S::STRIDE + e];
    out[e] = sum;
  }
}

// Slot sums in two fixed-order passes: chunk[ch][e] = sum of the slots
// [ch * per, (ch + 1) * per) in order; grads[e] = sum of the chunks in order.
constexpr int kReduceChunks = 32;

__global__ void wgrad_chunk_kernel(const float* __restrict__ partials, int64_t nslots, int stride, int64_t per,
                                   float* __restrict__ chunk) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ch = blockIdx.y;
  if (e >= stride) return;
  float sum = 0.0f;
  const int64_t s1 = min(nslots, (ch + 1) * per);
  for (int64_t sl = ch * per; sl < s1; ++sl) sum += partials[sl * stride + e];
  chunk[static_cast<int64_t>(ch) * stride + e] = sum;
}

__global__ void wgrad_final_kernel(const float* __restrict__ chunk, int nch, int stride, float* __restrict__ grads) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= stride) return;
  float sum = 0.0f;
  for (int ch = 0; ch < nch; ++ch) sum += chunk[static_cast<int64_t>(ch) * stride + e];
  grads[e] = sum;
}

// Flipped, transposed weights of one layer for its data gradient:
// wf[c, o, ky, kx] = w[o, c, 2 - ky, 2 - kx].
__global__ void flip_kernel(const float* __restrict__ w, int cin, int cout, float* __restrict__ wf) {
  const int n = cin * cout * 9;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int tp = idx % 9, oc = idx / 9;
    const int c = oc / cout, o = oc - c * cout;  // idx indexes wf as [c][o][tap]
    wf[idx] = w[(o * cin + c) * 9 + (8 - tp)];
  }
}

// Mean squared error: dout = 2 (out - t) / N; per-block partial sums of
// (out - t)^2 (fixed order), the last block adds them in order into *loss.
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ out, const float* __restrict__ tgt,
                                                  int64_t n, float* __restrict__ dout, float* partials,
                                                  unsigned int* counter, float* loss) {
  __shared__ float scratch[kRedScratch];
  float sq = 0.0f;
  const float sc = 2.0f / static_cast<float>(n);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float d = out[i] - tgt[i];
    dout[i] = sc * d;
    sq = fmaf(d, d, sq);
  }
  float v[1] = {sq}, tot[1];
  if (grid_sum<1, float>(v, partials, counter, scratch, tot) && threadIdx.x == 0) *loss = tot[0] / static_cast<float>(n);
}

// Energy-norm loss L = (1 / N) sum_p e_p (A e)_p, e = out - target, with A
// the 5-point variable-coefficient operator of the sample (cell coefficients
// exp(g), g = input channel 0; faces the harmonic mean of the two cells, a
// boundary face the cell's own coefficient).  dout = 2 A e / N (A is
// symmetric).  Per-block partial sums of e.(A e), reduced like mse_kernel.
__device__ __forceinline__ float face(float ca, float cb) { return 2.0f * ca * cb / (ca + cb); }

__global__ void __launch_bounds__(256) energy_kernel(const float* __restrict__ out, const float* __restrict__ tgt,
                                                     const float* __restrict__ feat, int B, int H, int W,
                                                     float* __restrict__ dout, float* partials,
                                                     unsigned int* counter, float* loss) {
  __shared__ float scratch[kRedScratch];
  const int64_t HW = static_cast<int64_t>(H) * W, n = B * HW;
  const float sc = 2.0f / static_cast<float>(n);
  float acc = 0.0f;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < n;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t b = q / HW, p = q - b * HW;
    const int i = static_cast<int>(p / W), j = static_cast<int>(p - (p / W) * W);
    const float* g = feat + b * 2 * HW;  // channel 0 of sample b
    const float* e0 = out + b * HW;
    const float* t0 = tgt + b * HW;
    const float c = expf(g[p]);
    const float e = e0[p] - t0[p];
    float diag = 0.0f, off = 0.0f;
    const int di[4] = {-1, 0, 0, 1}, dj[4] = {0, -1, 1, 0};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ii = i + di[k], jj = j + dj[k];
      if (ii >= 0 && ii < H && jj >= 0 && jj < W) {
        const int64_t pn = static_cast<int64_t>(ii) * W + jj;
        const float f = face(c, expf(g[pn]));
        diag += f;
        off = fmaf(f, e0[pn] - t0[pn], off);
      } else {
        diag += c;
      }
    }
    const float ae = fmaf(diag, e, -off);
    dout[q] = sc * ae;
    acc = fmaf(e, ae, acc);
  }
  float v[1] = {acc}, tot[1];
  if (grid_sum<1, float>(v, partials, counter, scratch, tot) && threadIdx.x == 0) *loss = tot[0] / static_cast<float>(n);
}

// Adam (Kingma and Ba, 2015), step t >= 1.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int64_t n) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

// rms of b (fixed-order reduction): the last block stores it.
__global__ void __launch_bounds__(256) rms_kernel(const double* __restrict__ b, int64_t n, double* partials,
                                                  unsigned int* counter, double* rms) {
  __shared__ double scratch[kRedScratch];
  double s = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    s = fma(b[i], b[i], s);
  double v[1] = {s}, tot[1];
  if (grid_sum<1, double>(v, partials, counter, scratch, tot) && threadIdx.x == 0) {
    const double r = sqrt(tot[0] / static_cast<double>(n));
    *rms = r > 0.0 ? r : 1.0;
  }
}

// Network input [g, b / rms(b)] in FP32 and, when x is given, the target
// x / (rms(b) * out_scale).
__global__ void features_kernel(const double* __restrict__ g, const double* __restrict__ b,
                                const double* __restrict__ x, const double* __restrict__ rms, double out_scale,
                                int64_t n, float* __restrict__ feat, float* __restrict__ tgt) {
  const double inv = 1.0 / *rms;
  const double tinv = 1.0 / (*rms * out_scale);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    feat[i] = static_cast<float>(g[i]);
    feat[n + i] = static_cast<float>(b[i] * inv);
    if (x) tgt[i] = static_cast<float>(x[i] * tinv);
  }
}

// x0 = y * rms(b) * out_scale in FP64.
__global__ void scale_out_kernel(const float* __restrict__ y, const double* __restrict__ rms, double out_scale,
                                 int64_t n, double* __restrict__ x0) {
  const double sc = *rms * out_scale;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x0[i] = static_cast<double>(y[i]) * sc;
}

// Galerkin scaling of the prediction: (x0.b, x0.A x0) -> x0 *= alpha with
// alpha = (x0.b) / (x0.A x0) (the multiple of x0 closest to the solution in
// the A-norm, so never farther than x = 0 for SPD A).  Sums first (last
// block stores alpha), the scaling in a second launch.
__global__ void __launch_bounds__(256) galerkin_sums_kernel(const double* __restrict__ x0,
                                                            const double* __restrict__ b,
                                                            const double* __restrict__ ax0, int64_t n,
                                                            double* partials, unsigned int* counter,
                                                            double* alpha) {
  __shared__ double scratch[kRedScratch];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    s0 = fma(x0[i], b[i], s0);
    s1 = fma(x0[i], ax0[i], s1);
  }
  double v[2] = {s0, s1}, tot[2];
  if (grid_sum<2, double>(v, partials, counter, scratch, tot) && threadIdx.x == 0)
    *alpha = (tot[1] > 0.0 && isfinite(tot[0] / tot[1])) ? tot[0] / tot[1] : 0.0;
}

__global__ void scale_kernel(double* __restrict__ x0, const double* __restrict__ alpha, int64_t n) {
  const double a = *alpha;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x0[i] *= a;
}

// ---------------------------------------------------------------------------
// BF16 inference on the tensor cores.  Activations are NHWC BF16 between the
// layers (a pixel's 32 channels are 64 contiguous bytes).  The 32 -> 32
// layers run as an implicit GEMM on tcgen05: a tile is 128 consecutive
// pixels of one image row (M = 128), N = 32 output channels, K = 9 taps x 32
// input channels, issued as 18 MMAs of K = 16 (BF16 operands, FP32
// accumulator in tensor memory).  For each kernel row ky the block stages
// the input row y + d (ky - 1) from x0 - d to x0 + 127 + d once (zeros
// outside the image); the three taps kx of that row are the same staged
// window read from slot kx d on, so the MMA's A operand is the window with a
// start address shifted by kx d rows.  Operands are K-major without
// swizzling: a core matrix is 8 rows x 16 bytes (8 channels); rows of a
// matrix are 16 bytes apart and its 8-channel chunks LBO bytes apart.  The
// first layer (2 input channels, K = 18 padded to 32) runs on the tensor
// cores too (conv_first_tc_kernel); the last (1 output channel) has no GEMM
// worth the name and runs on the CUDA cores, reading NHWC.
// ---------------------------------------------------------------------------

constexpr int kTcThreads = 128;                 // 4 warps: one TMEM lane quarter each
constexpr int kTcTile = 128;                    // pixels per tile (MMA M)
constexpr int kTcStripMax = 16;                 // output rows per work item (a strip), at most
constexpr int kTcMaxDil = 64;                   // largest dilation (gk_wsnet_create checks it)
constexpr uint32_t kTcChunkB = 32 * 16;         // bytes between 8-channel chunks of a tap's weights
constexpr int kTcPacked = 9 * 4 * 32 * 8;       // packed BF16 weights of one 32 -> 32 layer
constexpr int kTcMidLayers = kLayers - 2;

// 16-byte asynchronous global -> shared copy through L1 (cp.async); the
// bytes past src_bytes (0 or 16) are zero-filled, and with src_bytes 0
// nothing is read from src.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
// Waits for all of this thread's cp.async copies.
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared memory of a block: this header, then the ring of three staged
// input rows, [row slot][chunk][pixel slot][8 channels], win = 128 + 2 dil
// pixel slots per chunk: sized per layer, so that layers of small dilation
// fit more blocks per SM.
struct TcSmem {
  __nv_bfloat16 b[kTcPacked];           // [tap][chunk][out][8 channels]
  float bias[32];
  uint64_t bar;
  uint32_t tmem;
};
constexpr size_t kTcAOffset = (sizeof(TcSmem) + 127) / 128 * 128;
constexpr size_t tc_smem_bytes(int dil) { return kTcAOffset + 3 * 4 * static_cast<size_t>(kTcTile + 2 * dil) * 16; }
// ... and the folded last layer's weights after the ring (conv_tc_kernel<true>)
constexpr size_t kTcLastBytes = 9 * 32 * sizeof(float);

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits
// 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 =
// 0), N / 8 in bits 17-22, M / 16 in bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory matrix descriptor: start address / 16 (bits 0-13), leading
// (K-direction) byte offset / 16 (bits 16-29), stride (M/N-direction) byte
// offset / 16 (bits 32-45), the fixed version bits 46-48 = 0b001, no
// swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
         (static_cast<uint64_t>(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of the warp's 32 TMEM lanes (lane = pixel).
__device__ __forceinline__ void tc_load32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return l | (h << 16);
}

// One 32 -> 32 layer with ReLU: x, y NHWC BF16 (B, H, W, 32); wp the packed
// weights [tap][chunk][out][8]; bias BF16.  Persistent over tiles; err gets
// kErrTimeout if an MMA completion wait gives up.
// LAST: this is the network's last 32 -> 32 layer and the 32 -> 1 layer
// after it is folded into its epilogue: since that layer has one output
// channel, its output is y(p) = b + sum over taps of t_tap(p + offset_tap)
// with t_tap(q) = sum over channels of w[tap][c] h(q)[c]; the epilogue
// rounds h to BF16 (the value the unfused form stores) and writes the nine
// t_tap(q) as FP32 planes T[tap][pixel] to y, and conv_last_sum_kernel adds
// them up.  The 64-byte activation is then never written nor read back.
template <bool LAST>
__global__ void __launch_bounds__(kTcThreads) conv_tc_kernel(const __nv_bfloat16* __restrict__ x,
                                                             const __nv_bfloat16* __restrict__ wp,
                                                             const __nv_bfloat16* __restrict__ bias, int B, int H,
                                                             int W, int dil, int strip,
                                                             const __nv_bfloat16* __restrict__ w_last,
                                                             __nv_bfloat16* __restrict__ y, int* err) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(tc_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int i = t; i < kTcPacked / 8; i += kTcThreads)
    reinterpret_cast<uint4*>(S.b)[i] = __ldg(reinterpret_cast<const uint4*>(wp) + i);
  if (t < 32) S.bias[t] = __bfloat162float(bias[t]);
  // LAST: the 32 -> 1 layer's weights [tap][channel], after the ring
  float* const w_last_s =
      reinterpret_cast<float*>(tc_raw + kTcAOffset + 3 * 4 * static_cast<size_t>(kTcTile + 2 * dil) * 16);
  if (LAST)
    for (int i = t; i < 9 * 32; i += kTcThreads) w_last_s[i] = __bfloat162float(w_last[(i & 31) * 9 + (i >> 5)]);
  if (t == 0) {
    mbar_init(&S.bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&S.tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const int64_t n_pix = static_cast<int64_t>(B) * H * W;  // LAST: the T planes' stride
  const int nslot = kTcTile + 2 * dil;              // pixel slots of a staged row
  const uint32_t chunk_a = static_cast<uint32_t>(nslot) * 16;  // bytes between its 8-channel chunks
  uint4* const ring = reinterpret_cast<uint4*>(tc_raw + kTcAOffset);
  const uint32_t a_base = smem_u32(ring), b_base = smem_u32(S.b);
  const int tiles_x = (W + kTcTile - 1) / kTcTile;
  // Work items are strips: the output rows y0, y0 + dil, ..., of one image
  // and one 128-pixel column range (at most `strip` of them).  Output row
  // y_k reads input rows y_k - dil, y_k and y_k + dil, so consecutive rows of
  // a strip share two of their three input rows: a ring of three staged rows
  // holds them, and each tile after a strip's first stages one new row,
  // while the tile before it is read back.
  const int per_class = (H + dil - 1) / dil;             // rows of the fullest residue class
  const int chunks = (per_class + strip - 1) / strip;
  const int n_strips = B * tiles_x * dil * chunks;
  uint32_t phase = 0;
  bool pending = false;  // an MMA group whose completion was not observed
  // Stages input row ys of image img (zeros outside the image) for the
  // column range starting at x0 into ring slot q, with asynchronous 16-byte
  // copies: nothing passes through registers, so all of a row's copies are
  // in flight at once.
  auto stage = [&](int64_t img, int ys, int x0, int q) {
    for (int sl = t; sl < nslot; sl += kTcThreads) {
      const int xs = x0 - dil + sl;
      const bool in = ys >= 0 && ys < H && xs >= 0 && xs < W;
      const uint4* src = in ? reinterpret_cast<const uint4*>(x + (img + static_cast<int64_t>(ys) * W + xs) * 32)
                            : reinterpret_cast<const uint4*>(x);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        cp_async16(ring + (q * 4 + c) * nslot + sl, src + c, in ? 16u : 0u);
    }
  };
  bool failed = false;
  for (int item = blockIdx.x; item < n_strips && !failed; item += gridDim.x) {
    int rest = item;
    const int ch = rest % chunks;
    rest /= chunks;
    const int cls = rest % dil;
    rest /= dil;
    const int xt = rest % tiles_x;
    const int b = rest / tiles_x;
    const int x0 = xt * kTcTile;
    const int64_t img = static_cast<int64_t>(b) * H * W;  // first pixel of this sample
    const int y0 = cls + ch * strip * dil;                 // first output row of the strip
    if (y0 >= H) continue;
    const int nrow = min(strip, (H - 1 - y0) / dil + 1);
    // input row m of the strip (m = -1 .. nrow) is y0 + m * dil, in slot (m + 1) % 3
    stage(img, y0 - dil, x0, 0);
    stage(img, y0, x0, 1);
    stage(img, y0 + dil, x0, 2);
    for (int k = 0; k < nrow; ++k) {
      const int yy = y0 + k * dil;
      cp_async_wait_all();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // staged rows -> tensor core reads
      tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc_fence_after();
        uint32_t acc = 0;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
          const int q = (k + ky) % 3;  // slot of input row k - 1 + ky
#pragma unroll
          for (int kx = 0; kx < 3; ++kx)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint32_t aa = a_base + ((q * 4 + 2 * h) * nslot + kx * dil) * 16;
              const uint32_t bb = b_base + ((ky * 3 + kx) * 4 + 2 * h) * kTcChunkB;
              tc_mma(tmem, tc_desc(aa, chunk_a, 128), tc_desc(bb, kTcChunkB, 128), acc);
              acc = 1;
            }
        }
        tc_commit(&S.bar);
      }
      pending = true;
      const bool ok = __syncthreads_and(mbar_wait(&S.bar, phase, err));
      if (!ok) {
        failed = true;
        break;
      }
      pending = false;
      phase ^= 1u;
      // the MMAs have read the ring: input row k + 2 goes into the slot of
      // row k - 1 while this tile's accumulator is read back and stored
      if (k + 1 < nrow) stage(img, yy + 2 * dil, x0, k % 3);
      tc_fence_after();
      float v[32];
      tc_load32(tmem + (static_cast<uint32_t>(warp * 32) << 16), v);
      const int px = x0 + warp * 32 + lane;
      if (px < W && LAST) {
        float h[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) h[c] = __bfloat162float(__float2bfloat16_rn(fmaxf(v[c] + S.bias[c], 0.0f)));
        float* T = reinterpret_cast<float*>(y) + img + static_cast<int64_t>(yy) * W + px;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          float tt = 0.0f;
#pragma unroll
          for (int c = 0; c < 32; ++c) tt = fmaf(w_last_s[tap * 32 + c], h[c], tt);
          T[tap * n_pix] = tt;
        }
      } else if (px < W) {
        uint4* dst = reinterpret_cast<uint4*>(y + (img + static_cast<int64_t>(yy) * W + px) * 32);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float o[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) o[e] = fmaxf(v[c * 8 + e] + S.bias[c * 8 + e], 0.0f);
          dst[c] = make_uint4(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]), pack_bf16x2(o[4], o[5]),
                              pack_bf16x2(o[6], o[7]));
        }
      }
    }
    // the next strip's first rows overwrite every slot: all reads of this
    // strip's last tile are done (its MMAs completed above), and the
    // barrier at the next tile's start orders the copies after them
  }
  cp_async_wait_all();  // no copy of this block is left in flight at exit
  // an MMA whose completion was not seen is waited for once more (bounded)
  // before its accumulator's tensor memory is released
  if (pending) mbar_wait(&S.bar, phase, err);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
  }
}

// The first layer (2 -> 32, ReLU) on the tensor cores: an implicit GEMM
// with K = 2 channels x 9 taps = 18, padded with zeros to 32 (two MMAs of
// K = 16).  A tile is 128 pixels of one image row (M = 128): each thread
// gathers its pixel's 18 input values (BF16 NCHW; zeros outside the image)
// into the A tile, K-major without swizzle like conv_tc_kernel's operands
// (8-value chunks 128 x 16 bytes apart); the block packs the 32 x 18
// weights the same way once ([chunk][out][8], zero-padded); the epilogue is
// conv_tc_kernel's (bias, ReLU, BF16 NHWC).  (A CUDA-core form, one thread
// per pixel, was bound by its 576 FP32 fused multiply-adds per pixel.)
constexpr int kTcFirstChunkA = kTcTile * 16;  // bytes between the A tile's 8-value chunks

struct TcFirstSmem {
  __nv_bfloat16 a[4 * kTcTile * 8];  // [chunk][pixel][8 values of k]
  __nv_bfloat16 b[4 * 32 * 8];       // [chunk][out][8 values of k]
  float bias[32];
  uint64_t bar;
  uint32_t tmem;
};

__global__ void __launch_bounds__(kTcThreads) conv_first_tc_kernel(const __nv_bfloat16* __restrict__ x,
                                                                   const __nv_bfloat16* __restrict__ w,
                                                                   const __nv_bfloat16* __restrict__ bias, int B,
                                                                   int H, int W, int dil,
                                                                   __nv_bfloat16* __restrict__ y, int* err) {
  __shared__ __align__(1024) TcFirstSmem S;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  // weights [chunk j][out n][e] = w[n][8 j + e] (k = channel * 9 + tap), zero past k = 17
  for (int i = t; i < 4 * 32 * 8; i += kTcThreads) {
    const int e = i & 7, n = (i >> 3) & 31, j = i >> 8;
    const int k = 8 * j + e;
    S.b[i] = k < 18 ? w[n * 18 + k] : __float2bfloat16_rn(0.0f);
  }
  if (t < 32) S.bias[t] = __bfloat162float(bias[t]);
  if (t == 0) {
    mbar_init(&S.bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&S.tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t a_base = smem_u32(S.a), b_base = smem_u32(S.b);
  const int tiles_x = (W + kTcTile - 1) / kTcTile;
  const int n_tiles = B * H * tiles_x;
  const int64_t HW = static_cast<int64_t>(H) * W;
  uint32_t phase = 0;
  bool pending = false;  // an MMA group whose completion was not observed
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int row = tile / tiles_x;  // b * H + yy
    const int x0 = (tile - row * tiles_x) * kTcTile;
    const int yy = row % H;
    const int b = row / H;
    const int px = x0 + t;  // this thread's pixel
    const __nv_bfloat16* xb = x + static_cast<int64_t>(b) * 2 * HW;
    __align__(16) __nv_bfloat16 v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __float2bfloat16_rn(0.0f);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const int ii = yy + dil * (ky - 1), jj = px + dil * (kx - 1);
          if (px < W && ii >= 0 && ii < H && jj >= 0 && jj < W)
            v[c * 9 + ky * 3 + kx] = xb[c * HW + static_cast<int64_t>(ii) * W + jj];
        }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      reinterpret_cast<uint4*>(S.a)[j * kTcTile + t] = *reinterpret_cast<const uint4*>(v + 8 * j);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (int h = 0; h < 2; ++h)
        tc_mma(tmem, tc_desc(a_base + 2 * h * kTcFirstChunkA, kTcFirstChunkA, 128),
               tc_desc(b_base + 2 * h * kTcChunkB, kTcChunkB, 128), h);
      tc_commit(&S.bar);
    }
    pending = true;
    const bool ok = __syncthreads_and(mbar_wait(&S.bar, phase, err));
    if (!ok) break;
    pending = false;
    phase ^= 1u;
    tc_fence_after();
    float acc[32];
    tc_load32(tmem + (static_cast<uint32_t>(warp * 32) << 16), acc);
    const int po = x0 + warp * 32 + lane;  // TMEM lane = pixel
    if (po < W) {
      uint4* dst = reinterpret_cast<uint4*>(y + (static_cast<int64_t>(b) * HW + static_cast<int64_t>(yy) * W + po) * 32);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) o[e] = fmaxf(acc[c * 8 + e] + S.bias[c * 8 + e], 0.0f);
        dst[c] = make_uint4(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]), pack_bf16x2(o[4], o[5]),
                            pack_bf16x2(o[6], o[7]));
      }
    }
  }
  // an MMA whose completion was not seen is waited for once more (bounded)
  // before its accumulator's tensor memory is released
  if (pending) mbar_wait(&S.bar, phase, err);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
  }
}

// Packs the 32 -> 32 layers' FP32 weights (out, in, 3, 3) into the MMA's B
// layout [tap][chunk][out][8 channels], rounded to BF16.
__global__ void pack_tc_kernel(const float* __restrict__ p, int64_t off0, int64_t stride,
                               __nv_bfloat16* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kTcMidLayers * kTcPacked) return;
  const int l = i / kTcPacked, r = i - l * kTcPacked;
  const int e = r & 7, o = (r >> 3) & 31, kc = (r >> 8) & 3, tap = r >> 10;
  const int c = kc * 8 + e;
  out[i] = __float2bfloat16_rn(p[off0 + l * stride + (o * 32 + c) * 9 + tap]);
}

// The last layer (32 -> 1, linear), second half: y(p) = b + sum over the
// nine taps of T[tap][p + offset_tap] (zero outside the image), the planes
// the last 32 -> 32 layer's epilogue wrote (conv_tc_kernel<true>); taps in
// (ky, kx) order.  y FP32 (B, 1, H, W).
__global__ void __launch_bounds__(256) conv_last_sum_kernel(const float* __restrict__ T,
                                                            const __nv_bfloat16* __restrict__ bias, int B, int H,
                                                            int W, int dil, float* __restrict__ y) {
  const int HW = H * W;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  const int b = blockIdx.y;
  const int i = p / W, j = p - i * W;
  const int64_t n_pix = static_cast<int64_t>(B) * HW;
  const float* Tb = T + static_cast<int64_t>(b) * HW;
  float acc = __bfloat162float(bias[0]);
#pragma unroll
  for (int ky = 0; ky < 3; ++ky)
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      const int ii = i + dil * (ky - 1), jj = j + dil * (kx - 1);
      if (ii >= 0 && ii < H && jj >= 0 && jj < W) acc += __ldg(Tb + (ky * 3 + kx) * n_pix + ii * W + jj);
    }
  y[static_cast<int64_t>(b) * HW + p] = acc;
}

int ew_grid(int64_t n) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * sm_count())));
}

}  // namespace

struct WsNet {
  int device = 0;
  int H = 0, W = 0, Bmax = 0;
  int dil[kLayers] = {};
  int64_t off_w[kLayers] = {}, off_b[kLayers] = {};
  int64_t nparams = 0;
  int step = 0;
  int loss_kind = 0;  // 0 mean squared error, 1 energy norm
  int64_t device_bytes = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // flat FP32 master, gradient, Adam moments
  float* wflip = nullptr;                                          // flipped weights (same offsets)
  __nv_bfloat16* pbf = nullptr;                                    // BF16 copy for inference
  bool bf_stale = true;
  float* act[kLayers + 1] = {};  // act[0] unused (the caller's input); act[l + 1] = layer l output
  float* dbuf[2] = {};           // data-gradient ping-pong
  __nv_bfloat16* hbf[3] = {};    // inference: input copy (NCHW) + ping-pong activations (NHWC)
  __nv_bfloat16* wtc = nullptr;  // the 32 -> 32 layers' weights in the tensor-core layout
  int* err = nullptr;            // device-side wait that gave up (kErrTimeout)
  int tc_smem_sm = 0, tc_reserved = 0;  // shared memory per SM and reserved per block
  float* partials = nullptr;
  int64_t partial_floats = 0;
  float* chunk = nullptr;  // kReduceChunks x the largest stride
  float* red = nullptr;
  unsigned int* counter = nullptr;
  double* dred = nullptr;
  unsigned int* dcounter = nullptr;
  double* scal = nullptr;  // [0] rms(b), [1] alpha
  float* feat = nullptr;   // one problem's input (2 H W) and output (H W)
  double* ax = nullptr;    // A x0 (warm start with projection)
  int64_t ax_n = 0;
};

namespace {

void wsnet_release(WsNet* N) {
  if (!N) return;
  const int prev = current_device();
  cudaSetDevice(N->device);
  void* ptrs[] = {N->p,      N->g,      N->m,        N->v,     N->wflip,   N->pbf,  N->dbuf[0],
                  N->dbuf[1], N->hbf[0], N->hbf[1],   N->hbf[2], N->partials, N->chunk, N->red,
                  N->counter, N->dred,   N->dcounter, N->scal,  N->feat,     N->ax,      N->wtc, N->err};
  for (void* q : ptrs) dfree(q);
  for (int l = 1; l <= kLayers; ++l) dfree(N->act[l]);
  cudaSetDevice(prev);
  delete N;
}

struct WsDeleter {
  void operator()(WsNet* n) const { wsnet_release(n); }
};

template <int CIN, int COUT, int MODE, typename TI, typename TW, typename TO>
int launch_conv(const TI* x, const TW* w, const TW* bias, int B, int H, int W, int dil, TO* y, const float* mask,
                cudaStream_t s) {
  const dim3 grid((H * W + kConvThreads - 1) / kConvThreads, B);
  conv_fwd_kernel<CIN, COUT, MODE, TI, TW, TO><<<grid, kConvThreads, 0, s>>>(x, w, bias, H, W, dil, y, mask);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

template <typename TI, typename TW, typename TO>
int forward_layer(int l, const TI* x, const TW* w, const TW* bias, int B, int H, int W, int dil, TO* y,
                  cudaStream_t s) {
  if (l == 0) return launch_conv<2, 32, CONV_RELU>(x, w, bias, B, H, W, dil, y, nullptr, s);
  if (l < kLayers - 1) return launch_conv<32, 32, CONV_RELU>(x, w, bias, B, H, W, dil, y, nullptr, s);
  return launch_conv<32, 1, CONV_LINEAR>(x, w, bias, B, H, W, dil, y, nullptr, s);
}

size_t wgrad_smem(int cin, int cout, int W, int dil) {
  const int co_t = cout >= 4 ? 4 : 1;
  const size_t xsplit = kConvThreads / (cin * (cout / co_t));
  const size_t staging = static_cast<size_t>(cout) * (W | 1) + 3 * static_cast<size_t>(cin) * ((W + 2 * dil) | 1);
  const size_t classes = xsplit * (static_cast<size_t>(cout) * cin * 9 + cout);
  return sizeof(float) * std::max(staging, classes);
}

template <int CIN, int COUT>
int launch_wgrad(const WsNet& N, const float* x, const float* dy, int B, int dil, float* grads, cudaStream_t s) {
  using S = WgradShape<CIN, COUT>;
  const size_t smem = wgrad_smem(CIN, COUT, N.W, dil);
  GK_TRY(set_smem(conv_wgrad_kernel<CIN, COUT>, smem));
  const dim3 grid((N.H + kWgradRows - 1) / kWgradRows, B);
  const int64_t nslots = static_cast<int64_t>(grid.x) * grid.y;
  if (nslots * S::STRIDE > N.partial_floats) return set_error(GK_ERR_UNSUPPORTED, "wsnet: gradient scratch too small");
  conv_wgrad_kernel<CIN, COUT><<<grid, kConvThreads, smem, s>>>(x, dy, N.H, N.W, dil, N.partials);
  GK_TRY_CUDA(cudaGetLastError());
  const int nch = static_cast<int>(std::min<int64_t>(kReduceChunks, nslots));
  const int64_t per = (nslots + nch - 1) / nch;
  wgrad_chunk_kernel<<<dim3((S::STRIDE + 255) / 256, nch), 256, 0, s>>>(N.partials, nslots, S::STRIDE, per, N.chunk);
  GK_TRY_CUDA(cudaGetLastError());
  wgrad_final_kernel<<<(S::STRIDE + 255) / 256, 256, 0, s>>>(N.chunk, nch, S::STRIDE, grads);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

int check_batch(const WsNet* N, int32_t B) {
  if (!N) return set_error(GK_ERR_ARG, "wsnet: NULL handle");
  if (B < 1 || B > N->Bmax) return set_error(GK_ERR_DIM, "wsnet: batch %d outside 1..%d", B, N->Bmax);
  return GK_OK;
}

// FP32 forward of a batch into N.act[1..6].
int forward_f32(WsNet& N, int B, const float* x, cudaStream_t s) {
  const float* in = x;
  for (int l = 0; l < kLayers; ++l) {
    GK_TRY((forward_layer<float, float, float>(l, in, N.p + N.off_w[l], N.p + N.off_b[l], B, N.H, N.W, N.dil[l],
                                               N.act[l + 1], s)));
    in = N.act[l + 1];
  }
  return GK_OK;
}

// Loss (into N.red[0], device) and gradients (into N.g) of a batch.
int gradients(WsNet& N, int B, const float* x, const float* target, cudaStream_t s) {
  GK_TRY(forward_f32(N, B, x, s));
  const int64_t nout = static_cast<int64_t>(B) * N.H * N.W;
  float* dout = N.dbuf[0];
  if (N.loss_kind == 1)
    energy_kernel<<<ew_grid(nout), 256, 0, s>>>(N.act[kLayers], target, x, B, N.H, N.W, dout, N.red + 2, N.counter,
                                                N.red);
  else
    mse_kernel<<<ew_grid(nout), 256, 0, s>>>(N.act[kLayers], target, nout, dout, N.red + 2, N.counter, N.red);
  GK_TRY_CUDA(cudaGetLastError());
  for (int l = 0; l < kLayers; ++l) {
    flip_kernel<<<ew_grid(kCh[l] * kCh[l + 1] * 9), 256, 0, s>>>(N.p + N.off_w[l], kCh[l], kCh[l + 1],
                                                                  N.wflip + N.off_w[l]);
    GK_TRY_CUDA(cudaGetLastError());
  }
  const float* gcur = dout;
  int pp = 0;
  for (int l = kLayers - 1; l >= 0; --l) {
    const float* xin = l == 0 ? x : N.act[l];
    float* gw = N.g + N.off_w[l];  // the bias gradient follows the weights
    if (l == 0) GK_TRY((launch_wgrad<2, 32>(N, xin, gcur, B, N.dil[l], gw, s)));
    else if (l < kLayers - 1) GK_TRY((launch_wgrad<32, 32>(N, xin, gcur, B, N.dil[l], gw, s)));
    else GK_TRY((launch_wgrad<32, 1>(N, xin, gcur, B, N.dil[l], gw, s)));
    if (l == 0) break;
    float* gnext = N.dbuf[1 - pp];
    // data gradient of layer l, masked by the ReLU of layer l - 1 (its output act[l])
    if (l == kLayers - 1)
      GK_TRY((launch_conv<1, 32, CONV_MASK, float, float, float>(gcur, N.wflip + N.off_w[l], nullptr, B, N.H, N.W,
                                                                 N.dil[l], gnext, N.act[l], s)));
    else
      GK_TRY((launch_conv<32, 32, CONV_MASK, float, float, float>(gcur, N.wflip + N.off_w[l], nullptr, B, N.H,
                                                                  N.W, N.dil[l], gnext, N.act[l], s)));
    gcur = gnext;
    pp = 1 - pp;
  }
  return GK_OK;
}

int infer_bf16(WsNet& N, int B, const float* x, float* y, cudaStream_t s) {
  if (N.bf_stale) {
    to_bf16_kernel<<<ew_grid(N.nparams), 256, 0, s>>>(N.p, N.pbf, N.nparams);
    GK_TRY_CUDA(cudaGetLastError());
    pack_tc_kernel<<<(kTcMidLayers * kTcPacked + 255) / 256, 256, 0, s>>>(N.p, N.off_w[1], N.off_w[2] - N.off_w[1],
                                                                          N.wtc);
    GK_TRY_CUDA(cudaGetLastError());
    N.bf_stale = false;
  }
  const int64_t nin = static_cast<int64_t>(B) * 2 * N.H * N.W;
  to_bf16_kernel<<<ew_grid(nin), 256, 0, s>>>(x, N.hbf[0], nin);
  GK_TRY_CUDA(cudaGetLastError());
  const dim3 pg((N.H * N.W + 255) / 256, B);
  const int64_t tiles = static_cast<int64_t>(B) * N.H * ((N.W + kTcTile - 1) / kTcTile);
  conv_first_tc_kernel<<<static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(tiles, 8 * sm_count()))),
                         kTcThreads, 0, s>>>(N.hbf[0], N.pbf + N.off_w[0], N.pbf + N.off_b[0], B, N.H, N.W,
                                             N.dil[0], N.hbf[1], N.err);
  GK_TRY_CUDA(cudaGetLastError());
  const __nv_bfloat16* in = N.hbf[1];
  for (int l = 1; l < kLayers - 1; ++l) {
    __nv_bfloat16* out = N.hbf[1 + (l & 1)];
    // resident blocks per SM: shared memory is the limit (registers, warps
    // and the 512 tensor-memory columns allow 16 blocks of 32 columns), and
    // it depends on the dilation through the staged rows' width
    const size_t smem = tc_smem_bytes(N.dil[l]) + (l == kLayers - 2 ? kTcLastBytes : 0);
    int per_sm = std::max(1, std::min(16, static_cast<int>(static_cast<size_t>(N.tc_smem_sm) / (smem + N.tc_reserved))));
    // small batches keep three blocks per SM (the count the widest rows
    // allow): more blocks would shorten every block's strips, and each strip
    // stages two rows more than it computes
    if (tiles < 16 * 3 * static_cast<int64_t>(sm_count())) per_sm = std::min(per_sm, 3);
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(tiles, int64_t(per_sm) * sm_count())));
    // strips as long as the work still gives every resident CTA about four
    // of them (a batch of one image runs single rows, each staging its
    // three input rows; large batches reuse rows along strips of up to 16),
    // then evened out over the rows of a residue class
    const int target = static_cast<int>(
        std::max<int64_t>(1, std::min<int64_t>(kTcStripMax, tiles / (4 * static_cast<int64_t>(grid)))));
    const int per_class = (N.H + N.dil[l] - 1) / N.dil[l];
    const int n_chunks = (per_class + target - 1) / target;
    const int strip = (per_class + n_chunks - 1) / n_chunks;
    // the last 32 -> 32 layer also folds in the 32 -> 1 layer: it writes the
    // nine tap planes (36 bytes per pixel, within the 64 of the buffer)
    if (l == kLayers - 2)
      conv_tc_kernel<true><<<grid, kTcThreads, smem, s>>>(in, N.wtc + (l - 1) * kTcPacked, N.pbf + N.off_b[l], B,
                                                          N.H, N.W, N.dil[l], strip, N.pbf + N.off_w[kLayers - 1],
                                                          out, N.err);
    else
      conv_tc_kernel<false><<<grid, kTcThreads, smem, s>>>(in, N.wtc + (l - 1) * kTcPacked, N.pbf + N.off_b[l], B,
                                                           N.H, N.W, N.dil[l], strip, nullptr, out, N.err);
    GK_TRY_CUDA(cudaGetLastError());
    in = out;
  }
  conv_last_sum_kernel<<<pg, 256, 0, s>>>(reinterpret_cast<const float*>(in), N.pbf + N.off_b[kLayers - 1], B, N.H,
                                          N.W, N.dil[kLayers - 1], y);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

}  // namespace
}  // namespace gk

using namespace gk;

extern "C" int gk_wsnet_create(int32_t H, int32_t W, int32_t batch_max, const int32_t* dilations, gk_wsnet* out) {
  if (!out || !dilations) return set_error(GK_ERR_ARG, "gk_wsnet_create: NULL argument");
  *out = nullptr;
  if (H < 1 || W < 1 || batch_max < 1 || static_cast<int64_t>(H) * W > (1 << 26))
    return set_error(GK_ERR_DIM, "gk_wsnet_create: H %d, W %d, batch %d", H, W, batch_max);
  std::unique_ptr<WsNet, WsDeleter> hold(new WsNet);
  WsNet* N = hold.get();
  N->device = current_device();
  N->H = H;
  N->W = W;
  N->Bmax = batch_max;
  int64_t off = 0;
  for (int l = 0; l < kLayers; ++l) {
    N->dil[l] = dilations[l];
    if (dilations[l] < 1 || dilations[l] > kTcMaxDil)
      return set_error(GK_ERR_ARG, "gk_wsnet_create: dilation %d outside 1..64", dilations[l]);
    N->off_w[l] = off;
    off += static_cast<int64_t>(kCh[l]) * kCh[l + 1] * 9;
    N->off_b[l] = off;
    off += kCh[l + 1];
  }
  N->nparams = off;
  int smem_max = 0;
  GK_TRY_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, N->device));
  for (int l = 0; l < kLayers; ++l)
    if (wgrad_smem(kCh[l], kCh[l + 1], W, N->dil[l]) > static_cast<size_t>(smem_max))
      return set_error(GK_ERR_UNSUPPORTED, "gk_wsnet_create: width %d with dilation %d needs too much shared memory",
                       W, N->dil[l]);
  int64_t* by = &N->device_bytes;
  const size_t np = static_cast<size_t>(off);
  for (float** q : {&N->p, &N->g, &N->m, &N->v, &N->wflip}) GK_TRY(dalloc_n(q, np, by));
  GK_TRY(dalloc_n(&N->pbf, np, by));
  const size_t img = static_cast<size_t>(H) * W;
  const size_t big = static_cast<size_t>(batch_max) * 32 * img;
  for (int l = 1; l <= kLayers; ++l)
    GK_TRY(dalloc_n(&N->act[l], l < kLayers ? big : static_cast<size_t>(batch_max) * img, by));
  for (float** q : {&N->dbuf[0], &N->dbuf[1]}) GK_TRY(dalloc_n(q, big, by));
  GK_TRY(dalloc_n(&N->hbf[0], static_cast<size_t>(batch_max) * 2 * img, by));
  GK_TRY(dalloc_n(&N->hbf[1], big, by));
  GK_TRY(dalloc_n(&N->hbf[2], big, by));
  GK_TRY(dalloc_n(&N->wtc, static_cast<size_t>(kTcMidLayers) * kTcPacked, by));
  GK_TRY(dalloc_n(&N->err, 1, by));
  GK_TRY_CUDA(cudaMemset(N->err, 0, sizeof(int)));
  GK_TRY(set_smem(conv_tc_kernel<false>, tc_smem_bytes(kTcMaxDil)));
  GK_TRY(set_smem(conv_tc_kernel<true>, tc_smem_bytes(kTcMaxDil) + kTcLastBytes));
  // the grid of each layer is sized from its shared-memory footprint (the
  // occupancy query has been seen to report 1 for this kernel where 3 fit)
  GK_TRY_CUDA(cudaDeviceGetAttribute(&N->tc_smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, N->device));
  GK_TRY_CUDA(cudaDeviceGetAttribute(&N->tc_reserved, cudaDevAttrReservedSharedMemoryPerBlock, N->device));
  // weight-gradient slots: the largest layer's count
  int64_t pf = 0;
  const int64_t blocks = static_cast<int64_t>((H + kWgradRows - 1) / kWgradRows) * batch_max;
  pf = std::max<int64_t>(pf, blocks * WgradShape<2, 32>::STRIDE);
  pf = std::max<int64_t>(pf, blocks * WgradShape<32, 32>::STRIDE);
  pf = std::max<int64_t>(pf, blocks * WgradShape<32, 1>::STRIDE);
  N->partial_floats = pf;
  GK_TRY(dalloc_n(&N->partials, static_cast<size_t>(pf), by));
  GK_TRY(dalloc_n(&N->chunk, static_cast<size_t>(kReduceChunks) * WgradShape<32, 32>::STRIDE, by));
  const int rg = 8 * sm_count() + 8;
  GK_TRY(dalloc_n(&N->red, static_cast<size_t>(rg + 4), by));
  GK_TRY(dalloc_n(&N->counter, 1, by));
  GK_TRY(dalloc_n(&N->dred, static_cast<size_t>(2 * rg + 4), by));
  GK_TRY(dalloc_n(&N->dcounter, 1, by));
  GK_TRY(dalloc_n(&N->scal, 4, by));
  GK_TRY(dalloc_n(&N->feat, 3 * img, by));
  GK_TRY_CUDA(cudaMemset(N->counter, 0, sizeof(unsigned int)));
  GK_TRY_CUDA(cudaMemset(N->dcounter, 0, sizeof(unsigned int)));
  GK_TRY_CUDA(cudaMemset(N->m, 0, np * sizeof(float)));
  GK_TRY_CUDA(cudaMemset(N->v, 0, np * sizeof(float)));
  GK_TRY_CUDA(cudaMemset(N->p, 0, np * sizeof(float)));
  GK_TRY_CUDA(cudaDeviceSynchronize());
  *out = reinterpret_cast<gk_wsnet>(hold.release());
  return GK_OK;
}

extern "C" int gk_wsnet_num_params(gk_wsnet h, int64_t* n) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  if (!N || !n) return set_error(GK_ERR_ARG, "gk_wsnet_num_params: NULL argument");
  *n = N->nparams;
  return GK_OK;
}

extern "C" int gk_wsnet_set_params(gk_wsnet h, const float* params, void* stream) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  if (!N || !params) return set_error(GK_ERR_ARG, "gk_wsnet_set_params: NULL argument");
  DeviceGuard dg(N->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GK_TRY_CUDA(cudaMemcpyAsync(N->p, params, sizeof(float) * N->nparams, cudaMemcpyDefault, s));
  GK_TRY_CUDA(cudaMemsetAsync(N->m, 0, sizeof(float) * N->nparams, s));
  GK_TRY_CUDA(cudaMemsetAsync(N->v, 0, sizeof(float) * N->nparams, s));
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  N->step = 0;
  N->bf_stale = true;
  return GK_OK;
}

extern "C" int gk_wsnet_set_loss(gk_wsnet h, int32_t kind) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  if (!N) return set_error(GK_ERR_ARG, "gk_wsnet_set_loss: NULL handle");
  if (kind != 0 && kind != 1) return set_error(GK_ERR_ARG, "gk_wsnet_set_loss: kind %d (0 or 1)", kind);
  N->loss_kind = kind;
  return GK_OK;
}

extern "C" int gk_wsnet_get_params(gk_wsnet h, float* params, void* stream) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  if (!N || !params) return set_error(GK_ERR_ARG, "gk_wsnet_get_params: NULL argument");
  DeviceGuard dg(N->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GK_TRY_CUDA(cudaMemcpyAsync(params, N->p, sizeof(float) * N->nparams, cudaMemcpyDefault, s));
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  return GK_OK;
}

extern "C" int gk_wsnet_forward(gk_wsnet h, int32_t B, const float* x, float* y, void* stream) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  GK_TRY(check_batch(N, B));
  if (!x || !y) return set_error(GK_ERR_ARG, "gk_wsnet_forward: NULL argument");
  DeviceGuard dg(N->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GK_TRY(forward_f32(*N, B, x, s));
  GK_TRY_CUDA(cudaMemcpyAsync(y, N->act[kLayers], sizeof(float) * B * N->H * N->W, cudaMemcpyDeviceToDevice, s));
  return GK_OK;
}

extern "C" int gk_wsnet_gradients(gk_wsnet h, int32_t B, const float* x, const float* target, float* loss,
                                  float* grads, void* stream) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  GK_TRY(check_batch(N, B));
  if (!x || !target) return set_error(GK_ERR_ARG, "gk_wsnet_gradients: NULL argument");
  DeviceGuard dg(N->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GK_TRY(gradients(*N, B, x, target, s));
  if (grads) GK_TRY_CUDA(cudaMemcpyAsync(grads, N->g, sizeof(float) * N->nparams, cudaMemcpyDefault, s));
  if (loss) GK_TRY_CUDA(cudaMemcpyAsync(loss, N->red, sizeof(float), cudaMemcpyDefault, s));
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  return GK_OK;
}

extern "C" int gk_wsnet_train_step(gk_wsnet h, int32_t B, const float* x, const float* target, float lr,
                                   float* loss, void* stream) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  GK_TRY(check_batch(N, B));
  if (!x || !target) return set_error(GK_ERR_ARG, "gk_wsnet_train_step: NULL argument");
  if (!(lr > 0.0f)) return set_error(GK_ERR_ARG, "gk_wsnet_train_step: learning rate %g", lr);
  DeviceGuard dg(N->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GK_TRY(gradients(*N, B, x, target, s));
  N->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, static_cast<float>(N->step)), c2 = 1.0f - powf(b2, static_cast<float>(N->step));
  adam_kernel<<<ew_grid(N->nparams), 256, 0, s>>>(N->p, N->g, N->m, N->v, N->nparams, lr, b1, b2, 1e-8f, c1, c2);
  GK_TRY_CUDA(cudaGetLastError());
  N->bf_stale = true;
  if (loss) GK_TRY_CUDA(cudaMemcpyAsync(loss, N->red, sizeof(float), cudaMemcpyDefault, s));
  return GK_OK;
}

extern "C" int gk_wsnet_infer_bf16(gk_wsnet h, int32_t B, const float* x, float* y, void* stream) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  GK_TRY(check_batch(N, B));
  if (!x || !y) return set_error(GK_ERR_ARG, "gk_wsnet_infer_bf16: NULL argument");
  DeviceGuard dg(N->device);
  return infer_bf16(*N, B, x, y, static_cast<cudaStream_t>(stream));
}

extern "C" int gk_wsnet_check(gk_wsnet h, void* stream) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  if (!N) return set_error(GK_ERR_ARG, "gk_wsnet_check: NULL handle");
  DeviceGuard dg(N->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int e = 0;
  GK_TRY_CUDA(cudaMemcpyAsync(&e, N->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GK_TRY_CUDA(cudaStreamSynchronize(s));
  if (e != 0) {
    GK_TRY_CUDA(cudaMemsetAsync(N->err, 0, sizeof(int), s));
    GK_TRY_CUDA(cudaStreamSynchronize(s));
    return set_error(GK_ERR_TIMEOUT, "gk_wsnet_check: a tensor-core completion wait gave up");
  }
  return GK_OK;
}

extern "C" int gk_wsnet_features(gk_wsnet h, const double* g, const double* b, const double* x, double out_scale,
                                 float* feat, float* target, void* stream) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  if (!N || !g || !b || !feat || (x && !target)) return set_error(GK_ERR_ARG, "gk_wsnet_features: NULL argument");
  if (!(out_scale > 0.0)) return set_error(GK_ERR_ARG, "gk_wsnet_features: out_scale must be positive");
  DeviceGuard dg(N->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = static_cast<int64_t>(N->H) * N->W;
  rms_kernel<<<ew_grid(n), 256, 0, s>>>(b, n, N->dred + 4, N->dcounter, N->scal);
  GK_TRY_CUDA(cudaGetLastError());
  features_kernel<<<ew_grid(n), 256, 0, s>>>(g, b, x, N->scal, out_scale, n, feat, target);
  GK_TRY_CUDA(cudaGetLastError());
  return GK_OK;
}

extern "C" int gk_wsnet_warm_start(gk_wsnet h, gk_matrix A, const double* g, const double* b, double out_scale,
                                   double* x0, void* stream) {
  WsNet* N = reinterpret_cast<WsNet*>(h);
  if (!N || !g || !b || !x0) return set_error(GK_ERR_ARG, "gk_wsnet_warm_start: NULL argument");
  if (!(out_scale > 0.0)) return set_error(GK_ERR_ARG, "gk_wsnet_warm_start: out_scale must be positive");
  DeviceGuard dg(N->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = static_cast<int64_t>(N->H) * N->W;
  Matrix* M = A ? as_matrix(A) : nullptr;
  if (M && (M->n_rows != n || M->n_cols != n))
    return set_error(GK_ERR_DIM, "gk_wsnet_warm_start: matrix is %lld x %lld, the grid has %lld points",
                     (long long)M->n_rows, (long long)M->n_cols, (long long)n);
  rms_kernel<<<ew_grid(n), 256, 0, s>>>(b, n, N->dred + 4, N->dcounter, N->scal);
  GK_TRY_CUDA(cudaGetLastError());
  features_kernel<<<ew_grid(n), 256, 0, s>>>(g, b, nullptr, N->scal, out_scale, n, N->feat, nullptr);
  GK_TRY_CUDA(cudaGetLastError());
  float* y = N->feat + 2 * n;
  GK_TRY(infer_bf16(*N, 1, N->feat, y, s));
  scale_out_kernel<<<ew_grid(n), 256, 0, s>>>(y, N->scal, out_scale, n, x0);
  GK_TRY_CUDA(cudaGetLastError());
  if (M) {
    if (N->ax_n < n) {
      dfree(N->ax);
      N->ax = nullptr;
      GK_TRY(dalloc_n(&N->ax, static_cast<size_t>(n), &N->device_bytes));
      N->ax_n = n;
    }
    Epi e;
    e.mode = EPI_COPY;
    e.y = N->ax;
    e.err = M->err;
    GK_TRY(spmv_launch(*M, x0, e, s));
    galerkin_sums_kernel<<<ew_grid(n), 256, 0, s>>>(x0, b, N->ax, n, N->dred + 4, N->dcounter, N->scal + 1);
    GK_TRY_CUDA(cudaGetLastError());
    scale_kernel<<<ew_grid(n), 256, 0, s>>>(x0, N->scal + 1, n);
    GK_TRY_CUDA(cudaGetLastError());
  }
  return GK_OK;
}

extern "C" int gk_wsnet_destroy(gk_wsnet h) {
  if (!h) return set_error(GK_ERR_ARG, "gk_wsnet_destroy: NULL handle");
  wsnet_release(reinterpret_cast<WsNet*>(h));
  return GK_OK;
}
