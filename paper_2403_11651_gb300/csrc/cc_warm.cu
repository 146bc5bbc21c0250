// Warm-start predictor: image -> latent pyramid (levels 0 .. 4), trained on latents the
// encoder reached.  Four 3x3 stride-2 convolutions with 32 channels and ReLU (zero
// padding 1) give levels 1 .. 4 through 1x1 convolutions; a 3x3 stride-1 convolution of
// the image gives level 0; levels 5 and 6 start at 0.  Loss: the sum over the predicted
// levels of each level's mean squared error.  Every reduction runs in a fixed order.
//
// Convolution: out[co][y][x] = b[co] + sum_{ci, ky, kx} w[co][ci][ky][kx]
//                                        * in[ci][s y + ky - 1][s x + kx - 1]  (0 outside).
//
// The three 32-to-32-channel convolutions (conv 2 .. 4, four fifths of the multiply-adds)
// run on the tensor cores with BF16 operands and FP32 accumulation: their inputs, weights
// and output gradients are rounded to BF16 (to nearest, ties to even) as they are staged,
// in the forward pass, the input gradient and the weight gradient alike.  Conv 1 (3 input
// channels), the heads, the loss and Adam stay in FP32 on the CUDA cores.  Activations of
// conv 1 .. 4 are stored pixel-major (32 floats per pixel).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cc_internal.cuh"
#include "cc_tc16.cuh"
#include "../../include/coolchic.h"

namespace cc {
namespace {

constexpr int kWCh = 32;

struct WarmLayout {
  int c_w[5], c_b[5];     // conv i = 1 .. 4 (index i); 0 unused
  int h_w[5], h_b[5];     // heads 1 .. 4 (1x1) and 0 (3x3 on the image)
  int total;
};

WarmLayout warm_layout() {
  WarmLayout L;
  int k = 0;
  L.c_w[0] = L.c_b[0] = -1;
  L.c_w[1] = k; k += kWCh * 3 * 9; L.c_b[1] = k; k += kWCh;
  for (int i = 2; i <= 4; ++i) { L.c_w[i] = k; k += kWCh * kWCh * 9; L.c_b[i] = k; k += kWCh; }
  for (int i = 1; i <= 4; ++i) { L.h_w[i] = k; k += kWCh; L.h_b[i] = k; k += 1; }
  L.h_w[0] = k; k += 3 * 9; L.h_b[0] = k; k += 1;
  L.total = k;
  return L;
}

__global__ void __launch_bounds__(256) k_wconv(const float* __restrict__ in, int Ci, int Hi, int Wi,
                                               const float* __restrict__ w, const float* __restrict__ b,
                                               float* __restrict__ out, int Co, int Ho, int Wo,
                                               int s, int relu) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)Co * Ho * Wo) return;
  const int co = (int)(q / ((long long)Ho * Wo));
  const int r = (int)(q - (long long)co * Ho * Wo), y = r / Wo, x = r - y * Wo;
  float acc = b[co];
  for (int ci = 0; ci < Ci; ++ci) {
    const float* wp = w + ((long long)co * Ci + ci) * 9;
    const float* ip = in + (long long)ci * Hi * Wi;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int iy = s * y + ky - 1;
      if (iy < 0 || iy >= Hi) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int ix = s * x + kx - 1;
        if (ix >= 0 && ix < Wi) acc = fmaf(wp[ky * 3 + kx], ip[(long long)iy * Wi + ix], acc);
      }
    }
  }
  out[q] = relu ? fmaxf(acc, 0.f) : acc;
}

// squared error of the predicted levels 0 .. 4 in one grid: block b belongs to the level
// l with first[l] <= b < first[l + 1]; d/dpred = 2 diff / n_l and a per-block partial sum of
// diff^2 / n_l in float-float arithmetic (fixed order)
struct LossLevels {
  int first[6];        // first block of each level, first[5] = total
  long long off[5];    // level offsets in flat latent order
  int n[5];
};
__global__ void __launch_bounds__(256) k_wloss(LossLevels lv, const float* __restrict__ pred,
                                               const float* __restrict__ target,
                                               float* __restrict__ dpred,
                                               float2* __restrict__ part) {
  int l = 0;
#pragma unroll
  for (int k = 1; k < 5; ++k) l = (int)blockIdx.x >= lv.first[k] ? k : l;
  const int n = lv.n[l];
  const int p = ((int)blockIdx.x - lv.first[l]) * blockDim.x + threadIdx.x;
  float e = 0.f;
  if (p < n) {
    const long long q = lv.off[l] + p;
    const float d = pred[q] - target[q];
    dpred[q] = 2.f * d / (float)n;
    e = d * d / (float)n;
  }
  __shared__ float2 red[256];
  red[threadIdx.x] = make_float2(e, 0.f);
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] = ff_add(red[threadIdx.x], red[threadIdx.x + st]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Adam state kept on the device so that a training step replays as one graph: the step
// count t (the update about to be taken is step t + 1), the learning rate, and the bias
// corrections of step s, (1 / (1 - 0.9^s), 1 / sqrt(1 - 0.999^s)) computed in FP64 on the
// host and rounded to float, for s < kWBcSteps (both are 1.0f beyond: 0.999^s < 2^-47).
constexpr int kWBcSteps = 32768;
struct WarmAdam {
  long long t;
  float lr;
  float2 bc[kWBcSteps];
};

__global__ void __launch_bounds__(256) k_wadam(float* p, float* m, float* v, const float* g, int n,
                                               const WarmAdam* ad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long s = ad->t + 1;
  const float2 bc = s < kWBcSteps ? ad->bc[s] : make_float2(1.f, 1.f);
  const float gi = g[i];
  m[i] = 0.9f * m[i] + 0.1f * gi;
  v[i] = 0.999f * v[i] + 0.001f * gi * gi;
  p[i] -= ad->lr * (m[i] * bc.x) / (sqrtf(v[i]) * bc.y + 1e-8f);
}

__global__ void k_wadam_advance(WarmAdam* ad) { ad->t += 1; }

int blocks(long long n) { return (int)((n + 255) / 256); }

// ------------------------------------------------------------ pixel-major FP32 layers

// conv 1 (3 -> 32, stride 2) with ReLU, pixel-major output, and head 1 on its output:
// one thread per output pixel, the weights staged in shared memory
__global__ void __launch_bounds__(256) k_wc1_fwd(const float* __restrict__ x, int H, int W,
                                                 const float* __restrict__ w,
                                                 const float* __restrict__ b,
                                                 const float* __restrict__ hw,
                                                 const float* __restrict__ hb,
                                                 float* __restrict__ act, int Ho, int Wo,
                                                 float* __restrict__ pred) {
  __shared__ float s_w[kWCh * 27], s_b[kWCh], s_h[kWCh];
  for (int i = threadIdx.x; i < kWCh * 27; i += blockDim.x) s_w[i] = w[i];
  if (threadIdx.x < kWCh) {
    s_b[threadIdx.x] = b[threadIdx.x];
    s_h[threadIdx.x] = hw[threadIdx.x];
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ho * Wo) return;
  const int oy = p / Wo, ox = p - oy * Wo;
  float v[27];
#pragma unroll
  for (int ci = 0; ci < 3; ++ci)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int iy = 2 * oy + ky - 1, ix = 2 * ox + kx - 1;
        v[ci * 9 + ky * 3 + kx] = iy >= 0 && iy < H && ix >= 0 && ix < W
                                      ? x[(long long)ci * H * W + (long long)iy * W + ix] : 0.f;
      }
  float h = hb[0];
  float4* out = reinterpret_cast<float4*>(act + (long long)p * kWCh);
#pragma unroll 1
  for (int c4 = 0; c4 < kWCh / 4; ++c4) {
    float o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int co = 4 * c4 + e;
      float a = s_b[co];
#pragma unroll
      for (int k = 0; k < 27; ++k) a = fmaf(s_w[co * 27 + k], v[k], a);
      o[e] = fmaxf(a, 0.f);
      h = fmaf(s_h[co], o[e], h);
    }
    out[c4] = make_float4(o[0], o[1], o[2], o[3]);
  }
  pred[p] = h;
}

// gradient of the top activation (conv 4's output) from head 4 alone, through its ReLU:
// da[q][c] = [act[q][c] > 0] hw[c] dpred[q]
__global__ void __launch_bounds__(256) k_whead_top(const float* __restrict__ act,
                                                   const float* __restrict__ hw,
                                                   const float* __restrict__ dpred, int n,
                                                   float* __restrict__ da) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)n * kWCh) return;
  const int c = (int)(q % kWCh);
  da[q] = act[q] > 0.f ? hw[c] * dpred[q / kWCh] : 0.f;
}

// Weight gradients that are sums over many pixels are taken in two steps: per-block
// partial sums over a range of kWPix pixels (fixed order inside the block), then
// k_wsum_parts sums the blocks in block order.
constexpr int kWPix = 256;
constexpr int kWPix1 = 64;    // conv 1: eight pixels per thread

// conv 1: block b covers output pixels [b kWPix1, (b + 1) kWPix1); thread (co = t % 32,
// g = t / 32) sums the pixels g, g + 8, ... of the range; part[b][co][k]: k < 27 the
// weight w[co][ci][tap] (k = ci * 9 + tap), k = 27 the bias
__global__ void __launch_bounds__(256) k_wc1_wgrad_part(const float* __restrict__ dact, int Ho,
                                                        int Wo, const float* __restrict__ x,
                                                        int H, int W, float* __restrict__ part) {
  const int co = threadIdx.x & 31, g = threadIdx.x >> 5;
  float acc[28];
#pragma unroll
  for (int k = 0; k < 28; ++k) acc[k] = 0.f;
  const int p1 = min(Ho * Wo, (blockIdx.x + 1) * kWPix1);
  for (int p = blockIdx.x * kWPix1 + g; p < p1; p += 8) {
    const int oy = p / Wo, ox = p - oy * Wo;
    const float d = dact[(long long)p * kWCh + co];
    acc[27] += d;
#pragma unroll
    for (int ci = 0; ci < 3; ++ci)
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const int iy = 2 * oy + ky - 1, ix = 2 * ox + kx - 1;
          const float v = iy >= 0 && iy < H && ix >= 0 && ix < W
                              ? __ldg(x + (long long)ci * H * W + (long long)iy * W + ix) : 0.f;
          acc[ci * 9 + ky * 3 + kx] = fmaf(d, v, acc[ci * 9 + ky * 3 + kx]);
        }
  }
  __shared__ float red[8][kWCh * 28 + 1];
#pragma unroll
  for (int k = 0; k < 28; ++k) red[g][co * 28 + k] = acc[k];
  __syncthreads();
  for (int j = threadIdx.x; j < kWCh * 28; j += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q][j];
    part[(long long)blockIdx.x * kWCh * 28 + j] = t;
  }
}

// head 0 (3x3, 3 -> 1, stride 1, on the image): block b covers pixels
// [b kWPix, (b + 1) kWPix), one per thread; part[b][k]: k < 27 the weight, 27 the bias
__global__ void __launch_bounds__(256) k_whead0_wgrad_part(const float* __restrict__ dpred,
                                                           const float* __restrict__ x, int H,
                                                           int W, float* __restrict__ part) {
  float acc[28];
#pragma unroll
  for (int k = 0; k < 28; ++k) acc[k] = 0.f;
  const int p1 = min(H * W, (blockIdx.x + 1) * kWPix);
  for (int p = blockIdx.x * kWPix + threadIdx.x; p < p1; p += blockDim.x) {
    const int y = p / W, xx = p - y * W;
    const float d = dpred[p];
    acc[27] += d;
#pragma unroll
    for (int ci = 0; ci < 3; ++ci)
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const int iy = y + ky - 1, ix = xx + kx - 1;
          const float v = iy >= 0 && iy < H && ix >= 0 && ix < W
                              ? __ldg(x + (long long)ci * H * W + (long long)iy * W + ix) : 0.f;
          acc[ci * 9 + ky * 3 + kx] = fmaf(d, v, acc[ci * 9 + ky * 3 + kx]);
        }
  }
  __shared__ float red[28][257];
#pragma unroll
  for (int k = 0; k < 28; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
#pragma unroll
      for (int k = 0; k < 28; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 28) part[(long long)blockIdx.x * 28 + threadIdx.x] = red[threadIdx.x][0];
}

// the 1x1 heads of levels 1 .. 4 on their pixel-major activations, in one grid: block b
// belongs to level i + 1 with first[i] <= b < first[i + 1] and covers that level's pixels
// [(b - first[i]) kWPix, ...); part[b][c]: c < 32 sum_p act[p][c] dpred[p], c = 32 the sum
// of dpred
struct HeadLevels {
  const float* act[4];
  const float* dpred[4];
  int n[4];
  int first[5];
};
__global__ void __launch_bounds__(256) k_whead_wgrad_part(HeadLevels hl, float* __restrict__ part) {
  int i = 0;
#pragma unroll
  for (int k = 1; k < 4; ++k) i = (int)blockIdx.x >= hl.first[k] ? k : i;
  const float* act = hl.act[i];
  const float* dpred = hl.dpred[i];
  const int n = hl.n[i], b = (int)blockIdx.x - hl.first[i];
  const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
  float aw = 0.f, ab = 0.f;
  const int p1 = min(n, (b + 1) * kWPix);
  for (int p = b * kWPix + g; p < p1; p += 8) {
    const float d = dpred[p];
    aw = fmaf(act[(long long)p * kWCh + c], d, aw);
    ab += d;
  }
  __shared__ float red[8][kWCh + 1];
  red[g][c] = aw;
  if (c == 0) red[g][kWCh] = ab;
  __syncthreads();
  if (threadIdx.x <= kWCh) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
    part[(long long)blockIdx.x * (kWCh + 1) + threadIdx.x] = t;
  }
}

// sum of part[b][j] over blocks b in [b0, b1) by one warp: lane l adds the blocks
// b0 + l, b0 + l + 32, ... (eight loads in flight), then the lanes are added in a fixed
// tree; the result is in lane 0
__device__ __forceinline__ float warp_col_sum(const float* __restrict__ part, int ncols, int j,
                                              int b0, int b1) {
  const int lane = threadIdx.x & 31;
  float t = 0.f;
  for (int b = b0 + lane; b < b1; b += 32 * 8) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int bb = b + 32 * q;
      v[q] = bb < b1 ? part[(long long)bb * ncols + j] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) t += v[q];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  return t;
}

// the heads' gradients: out[33 i + c] = the sum over level i + 1's blocks of part[b][c]
// (heads 1 .. 4 are consecutive [w (32), b] groups of the flat parameters); one warp per
// output
__global__ void __launch_bounds__(256) k_whead_wsum(HeadLevels hl, const float* __restrict__ part,
                                                    float* __restrict__ out) {
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= 4 * (kWCh + 1)) return;
  const int i = j / (kWCh + 1), c = j - i * (kWCh + 1);
  const float t = warp_col_sum(part, kWCh + 1, c, hl.first[i], hl.first[i + 1]);
  if ((threadIdx.x & 31) == 0) out[j] = t;
}

// the sum over blocks of part[b][j], j < ncols, one warp per column (warp_col_sum); column
// j goes to dw[j] when j % per < per - 1 (index (j / per) * (per - 1) + j % per), else to
// db[j / per]
__global__ void __launch_bounds__(256) k_wsum_parts(const float* __restrict__ part, int nblocks,
                                                    int ncols, int per, float* __restrict__ dw,
                                                    float* __restrict__ db) {
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= ncols) return;
  const float t = warp_col_sum(part, ncols, j, 0, nblocks);
  if ((threadIdx.x & 31) != 0) return;
  const int r = j / per, k = j - r * per;
  if (k < per - 1) dw[r * (per - 1) + k] = t; else db[r] = t;
}

// the loss: the per-block partials of every level summed over 256 lanes and a tree, in a
// fixed order (one block of 256 threads)
__global__ void __launch_bounds__(256) k_wloss_sum(const float2* __restrict__ part, int n,
                                                   double* __restrict__ loss) {
  float2 a = make_float2(0.f, 0.f);
  for (int i = threadIdx.x; i < n; i += 256) a = ff_add(a, part[i]);
  __shared__ float2 red[256];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] = ff_add(red[threadIdx.x], red[threadIdx.x + st]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (double)red[0].x + (double)red[0].y;
}

// ------------------------------------------------------------ BF16 tensor-core layers
//
// Implicit GEMM over tiles of 128 pixels, one per thread and one row of the accumulator
// each.  K = 288 = 9 taps x 32 channels, k = tap * 32 + channel with tap = 3 ky + kx.
// Operands are K-major core-matrix tiles in shared memory: row r, K index k at byte
// (r / 8) * kTcRG + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.  18 MMAs of K = 16
// (M = 128, N = 32) accumulate in 32 tensor-memory columns.
constexpr int kTcK = 9 * kWCh;            // 288
constexpr int kTcRG = (kTcK / 8) * 128;   // bytes between 8-row groups: 4608
constexpr int kTcABytes = 16 * kTcRG;     // 128 rows
constexpr int kTcBBytes = 4 * kTcRG;      // 32 rows
constexpr int kTcSmem = kTcABytes + kTcBBytes + 64;
constexpr long long kTcWaitBudget = 1ll << 30;   // SM clocks (about half a second)

struct TcConv {
  const float* in;      // pixel-major input (Hi x Wi x 32) or, for the input gradient,
                        // the output gradient (Ho x Wo x 32)
  const float* b;       // conv bias
  int Hi, Wi, Ho, Wo;
  float* out;           // forward: pixel-major activation; input gradient: dact of the input
  // forward: the head on the output; input gradient: the head of the input's level and the
  // input activation (ReLU mask)
  const float* hw;
  const float* hb;
  float* pred;          // forward
  const float* dpred;   // input gradient
  const float* act_in;  // input gradient
  int* fault;           // set when the MMA wait gives up
  const uint8_t* wimg;  // the layer's B operand image (k_wtc_prep), kTcBBytes
};

// stage 8 BF16 values (16 bytes) at row r, chunk kc of a K-major tile
__device__ __forceinline__ void tc_put(uint8_t* tile, int r, int kc, const float (&v)[8]) {
  *reinterpret_cast<uint4*>(tile + (r >> 3) * kTcRG + kc * 128 + (r & 7) * 16) = pack_bf16x8(v);
}

// The B operands of conv 2 .. 4 as BF16 images in the staged K-major layout, made once
// per pass from the parameters; a CTA copies its layer's image into shared memory with one
// bulk copy.  Image 2 (i - 2) is conv i's forward B: row n = output channel co,
// k = tap * 32 + ci -> w[co][ci][tap]; image 2 (i - 2) + 1 its input-gradient B: row n =
// input channel ci, k = tap * 32 + co -> w[co][ci][tap].  Grid: one block per image.
struct WImgArgs {
  const float* w[3];   // conv 2 .. 4 weights (flat parameter layout)
  uint8_t* img;        // 6 images of kTcBBytes
};
__global__ void __launch_bounds__(256) k_wtc_prep(WImgArgs a) {
  const int im = blockIdx.x, dgrad = im & 1;
  const float* __restrict__ w = a.w[im >> 1];
  uint8_t* dst = a.img + (size_t)im * kTcBBytes;
  for (int c = threadIdx.x; c < kWCh * (kTcK / 8); c += blockDim.x) {
    const int n = c / (kTcK / 8), kc = c - n * (kTcK / 8);
    const int tap = kc >> 2, j0 = (kc & 3) * 8;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = j0 + e;   // ci (forward) or co (input gradient)
      v[e] = dgrad ? w[(j * kWCh + n) * 9 + tap] : w[(n * kWCh + j) * 9 + tap];
    }
    tc_put(dst, n, kc, v);
  }
}

// one-dimensional bulk copy (TMA) of `bytes` from global to shared memory, completing the
// transaction bytes on mbar; addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      :: "r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mbar) : "memory");
}

// one thread issues the 18 MMAs of a tile and commits them to the barrier
__device__ __forceinline__ void tile_mma(uint32_t sA, uint32_t sB, uint32_t tmem, uint32_t bar) {
  constexpr uint32_t idesc = tc16_idesc(128, kWCh, false, false);
  tc_fence_after();
#pragma unroll 1
  for (int kk = 0; kk < kTcK / 16; ++kk)
    tc16_mma(tmem, tc16_desc(sA + kk * 256, 128, kTcRG), tc16_desc(sB + kk * 256, 128, kTcRG),
             idesc, kk > 0 ? 1u : 0u);
  tc_commit(bar);
}

// Forward of conv 2 .. 4 (stride 2): act_out = ReLU(conv(in) + b), pixel-major, and the head
// of its level: pred[p] = hb + sum_c hw[c] act_out[p][c].  One tile of 128 output pixels per
// CTA of 128 threads.
template <bool DGRAD>
__global__ void __launch_bounds__(128) k_wtc_conv(TcConv a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + kTcABytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kTcABytes + kTcBBytes);
  uint64_t* wbar = bar + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kTcABytes + kTcBBytes + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc_alloc(smem_u32(tslot), 32);
  if (tid == 0) {
    mbar_init(smem_u32(bar), 1);
    mbar_init(smem_u32(wbar), 1);
    mbar_expect_tx(smem_u32(wbar), kTcBBytes);
    bulk_load(smem_u32(sB), a.wimg, kTcBBytes, smem_u32(wbar));
  }
  // A: row m = this thread's pixel
  const int nq = DGRAD ? a.Hi * a.Wi : a.Ho * a.Wo;   // pixels of the result
  const int q = blockIdx.x * 128 + tid;
  const bool valid = q < nq;
  if (!DGRAD) {
    const int oy = valid ? q / a.Wo : 0, ox = valid ? q - oy * a.Wo : 0;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int iy = 2 * oy + tap / 3 - 1, ix = 2 * ox + tap % 3 - 1;
      const bool in = valid && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
      const float4* src = reinterpret_cast<const float4*>(
          a.in + (in ? ((long long)iy * a.Wi + ix) * kWCh : 0));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float v[8];
        const float4 u0 = in ? __ldg(src + 2 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 u1 = in ? __ldg(src + 2 * j + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
        v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
        tc_put(sA, tid, tap * 4 + j, v);
      }
    }
  } else {
    // input pixel (iy, ix) receives tap (ky, kx) of output (oy, ox) when 2 oy + ky - 1 = iy
    const int iy = valid ? q / a.Wi : 0, ix = valid ? q - iy * a.Wi : 0;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int ty = iy + 1 - tap / 3, tx = ix + 1 - tap % 3;
      const int oy = ty >> 1, ox = tx >> 1;
      const bool in = valid && ty >= 0 && tx >= 0 && !(ty & 1) && !(tx & 1) && oy < a.Ho &&
                      ox < a.Wo;
      const float4* src = reinterpret_cast<const float4*>(
          a.in + (in ? ((long long)oy * a.Wo + ox) * kWCh : 0));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float v[8];
        const float4 u0 = in ? __ldg(src + 2 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 u1 = in ? __ldg(src + 2 * j + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
        v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
        tc_put(sA, tid, tap * 4 + j, v);
      }
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // the weights' bulk copy: waited for by the thread that issues the MMAs
  bool wok = true;
  if (tid == 0) {
    wok = mbar_wait(smem_u32(wbar), 0, kTcWaitBudget);
    if (wok) tile_mma(smem_u32(sA), smem_u32(sB), tmem, smem_u32(bar));
  }
  if (__syncthreads_or(wok ? 0 : 1)) {
    // no MMA was issued: report; the copy gets another bounded wait before the CTA leaves
    if (tid == 0) {
      atomicExch(a.fault, 1);
      mbar_wait(smem_u32(wbar), 0, kTcWaitBudget);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 32);
    return;
  }
  const bool ok = mbar_wait(smem_u32(bar), 0, kTcWaitBudget);
  tc_fence_after();
  if (__syncthreads_or(ok ? 0 : 1)) {
    // report, and give the MMAs another bounded wait before the columns are freed
    if (tid == 0) atomicExch(a.fault, 1);
    mbar_wait(smem_u32(bar), 0, kTcWaitBudget);
  } else {
    float acc[32];
    tc_ld_row<32>(tmem + ((uint32_t)(warp * 32) << 16), acc);
    if (valid) {
      float4* out = reinterpret_cast<float4*>(a.out + (long long)q * kWCh);
      if (!DGRAD) {
        float h = a.hb[0];
#pragma unroll
        for (int c = 0; c < kWCh; ++c) {
          acc[c] = fmaxf(acc[c] + a.b[c], 0.f);
          h = fmaf(a.hw[c], acc[c], h);
        }
#pragma unroll
        for (int c4 = 0; c4 < kWCh / 4; ++c4)
          out[c4] = make_float4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2], acc[4 * c4 + 3]);
        a.pred[q] = h;
      } else {
        // add the gradient the input's head sends, then the input's ReLU
        const float g = a.dpred[q];
        const float4* ain = reinterpret_cast<const float4*>(a.act_in + (long long)q * kWCh);
#pragma unroll
        for (int c4 = 0; c4 < kWCh / 4; ++c4) {
          const float4 m = __ldg(ain + c4);
          float r[4];
          const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = 4 * c4 + e;
            r[e] = mv[e] > 0.f ? fmaf(a.hw[c], g, acc[c]) : 0.f;
          }
          out[c4] = make_float4(r[0], r[1], r[2], r[3]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 32);
}

// Weight gradient of conv 2 .. 4: dW^T[k][co] = sum_p im2col(in)[p][k] dout[p][co] with
// k = tap * 32 + ci, and db[co] = sum_p dout[p][co] as row k = 288 (a column of ones in
// the staged input).  Both operands are read MN-major: the staged input tile (rows = pixels,
// 48 chunks of 8 k per row; K of the MMA = pixels) and the output-gradient tile (rows =
// pixels, 4 chunks of 8 channels).  Three accumulators of 128 rows of k (M = 128, N = 32)
// over the CTA's tiles; then each CTA writes its 289 x 32 partial sums.
constexpr int kWgChunks = 48;                 // k = 0 .. 383 (rows 289 .. 383 are zero)
constexpr int kWgRG = kWgChunks * 128;        // 6144 bytes between 8-pixel groups
constexpr int kWgABytes = 16 * kWgRG;         // 98304
constexpr int kWgDRG = 4 * 128;               // 512
constexpr int kWgDBytes = 16 * kWgDRG;        // 8192
// the MMAs' reads stay inside the allocation under either assignment of the descriptor's
// two offsets
constexpr int kWgSmem = 190 * 1024;
constexpr int kWgRows = kTcK + 1;             // 289

__global__ void __launch_bounds__(128) k_wtc_wgrad(const float* __restrict__ in, int Hi, int Wi,
                                                   const float* __restrict__ dout, int Ho, int Wo,
                                                   float* __restrict__ part, int* fault) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sD = smem + kWgABytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kWgABytes + kWgDBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kWgABytes + kWgDBytes + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc_alloc(smem_u32(tslot), 128);
  if (tid == 0) mbar_init(smem_u32(bar), 1);
  // chunks 36 .. 47 of every row: the ones column (k = 288) and zeros
  {
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int kc = 37; kc < kWgChunks; ++kc)
      *reinterpret_cast<uint4*>(sA + (tid >> 3) * kWgRG + kc * 128 + (tid & 7) * 16) =
          pack_bf16x8(v);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int n = Ho * Wo, n_tiles = (n + 127) / 128;
  constexpr uint32_t idesc = tc16_idesc(128, kWCh, true, true);
  int phase = 0;
  bool ok = true;
  bool first = true;
  for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
    const int p = t * 128 + tid;
    const bool valid = p < n;
    const int oy = valid ? p / Wo : 0, ox = valid ? p - oy * Wo : 0;
    uint8_t* rowA = sA + (tid >> 3) * kWgRG + (tid & 7) * 16;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int iy = 2 * oy + tap / 3 - 1, ix = 2 * ox + tap % 3 - 1;
      const bool inb = valid && iy >= 0 && iy < Hi && ix >= 0 && ix < Wi;
      const float4* src = reinterpret_cast<const float4*>(
          in + (inb ? ((long long)iy * Wi + ix) * kWCh : 0));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float v[8];
        const float4 u0 = inb ? __ldg(src + 2 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 u1 = inb ? __ldg(src + 2 * j + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
        v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
        *reinterpret_cast<uint4*>(rowA + (tap * 4 + j) * 128) = pack_bf16x8(v);
      }
    }
    {
      float v[8] = {valid ? 1.f : 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      *reinterpret_cast<uint4*>(rowA + 36 * 128) = pack_bf16x8(v);
    }
    const float4* dsrc = reinterpret_cast<const float4*>(dout + (valid ? (long long)p * kWCh : 0));
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float v[8];
      const float4 u0 = valid ? __ldg(dsrc + 2 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 u1 = valid ? __ldg(dsrc + 2 * j + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
      v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
      v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
      *reinterpret_cast<uint4*>(sD + (tid >> 3) * kWgDRG + j * 128 + (tid & 7) * 16) =
          pack_bf16x8(v);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), d0 = smem_u32(sD);
#pragma unroll 1
      for (int mt = 0; mt < 3; ++mt)
#pragma unroll 1
        for (int s = 0; s < 8; ++s)
          tc16_mma(tmem + mt * 32, tc16_desc(a0 + mt * 2048 + s * 2 * kWgRG, kWgRG, 128),
                   tc16_desc(d0 + s * 2 * kWgDRG, kWgDRG, 128), idesc,
                   (first && s == 0) ? 0u : 1u);
      tc_commit(smem_u32(bar));
    }
    first = false;
    // the tiles are restaged only after the MMAs have read them
    ok = mbar_wait(smem_u32(bar), (uint32_t)phase, kTcWaitBudget);
    phase ^= 1;
    tc_fence_after();
    if (__syncthreads_or(ok ? 0 : 1)) ok = false;
  }
  if (!ok) {
    // report, and give the MMAs another bounded wait before the columns are freed
    if (tid == 0) atomicExch(fault, 1);
    mbar_wait(smem_u32(bar), (uint32_t)(phase ^ 1), kTcWaitBudget);
  } else {
    // row k = mt * 128 + tid of the three accumulators (zero when the CTA had no tile)
#pragma unroll 1
    for (int mt = 0; mt < 3; ++mt) {
      float acc[32];
      tc_ld_row<32>(tmem + mt * 32 + ((uint32_t)(warp * 32) << 16), acc);
      const int k = mt * 128 + tid;
      if (k < kWgRows) {
        float* dst = part + ((long long)blockIdx.x * kWgRows + k) * kWCh;
#pragma unroll
        for (int c = 0; c < kWCh; ++c) dst[c] = first ? 0.f : acc[c];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 128);
}

// sum of the wgrad kernel's per-CTA partials in CTA order (eight loads in flight per
// thread) into the flat gradient: dw[co][ci][tap] from row tap * 32 + ci, db[co] from row 288
__global__ void __launch_bounds__(256) k_wtc_wreduce(const float* __restrict__ part, int ctas,
                                                     float* __restrict__ dw,
                                                     float* __restrict__ db) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // row * 32 + co
  if (i >= kWgRows * kWCh) return;
  float t = 0.f;
  for (int c0 = 0; c0 < ctas; c0 += 8) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      v[q] = c0 + q < ctas ? part[(long long)(c0 + q) * kWgRows * kWCh + i] : 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += v[q];
  }
  const int k = i / kWCh, co = i - k * kWCh;
  if (k < kTcK) {
    const int tap = k / kWCh, ci = k - tap * kWCh;
    dw[(co * kWCh + ci) * 9 + tap] = t;
  } else {
    db[co] = t;
  }
}



}  // namespace
}  // namespace cc

using namespace cc;

struct cc_warm {
  int H = 0, W = 0, dev = 0;
  cudaStream_t st = nullptr;
  Geo geo;
  WarmLayout L;
  int h[5], w[5];          // activation sizes: level l = conv l output (l = 1 .. 4), 0 = image
  void* mem = nullptr;
  float *params, *grads, *m, *v;
  float *x, *act[5], *dact[5], *pred, *dpred, *target;
  uint8_t* img;
  float2* part;
  int n_part = 0;
  double* loss;             // the last loss (device)
  float* wpart;             // per-CTA partials of a tensor-core weight gradient
  int wg_ctas = 0;
  int* fault;               // a tensor-core wait gave up
  uint8_t* wimg;            // BF16 B-operand images of conv 2 .. 4 (k_wtc_prep)
  WarmAdam* adam;           // device
  float lr = -1.f;          // the learning rate in adam->lr
  cudaGraphExec_t pass = nullptr;     // image to planar, forward, loss, gradients
  cudaGraphExec_t update = nullptr;   // Adam and the step count
};

namespace {

thread_local char w_err[256] = "";

int wfail(cudaError_t e, const char* what) {
  snprintf(w_err, sizeof(w_err), "%s: %s", what, cudaGetErrorString(e));
  cc::set_error_text(w_err);
  return CC_ECUDA;
}

#define WCK(call)                                          \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return wfail(e_, #call);        \
  } while (0)

TcConv tc_args(cc_warm* c, int i) {
  TcConv a{};
  a.b = c->params + c->L.c_b[i];
  a.Hi = c->h[i - 1]; a.Wi = c->w[i - 1];
  a.Ho = c->h[i]; a.Wo = c->w[i];
  a.fault = c->fault;
  a.wimg = c->wimg + (size_t)2 * (i - 2) * kTcBBytes;   // forward; + kTcBBytes: input gradient
  return a;
}

// offsets of the latent levels in flat latent order
void level_offsets(const Geo& g, long long (&fo)[kLevels]) {
  long long o = 0;
  for (int l = 0; l < kLevels; ++l) { fo[l] = o; o += (long long)g.h[l] * g.w[l]; }
}

// forward: image (already planar in x) -> act[1..4] (pixel-major), pred (flat latent order;
// levels 5, 6 = 0)
int warm_forward(cc_warm* c) {
  const WarmLayout& L = c->L;
  float* P = c->params;
  const Geo& g = c->geo;
  // levels 5 and 6 of pred stay 0 (zeroed at creation, never written)
  long long fo[kLevels];
  level_offsets(g, fo);
  // level 0: 3x3 stride 1 on the image
  k_wconv<<<blocks((long long)c->H * c->W), 256, 0, c->st>>>(c->x, 3, c->H, c->W, P + L.h_w[0],
                                                             P + L.h_b[0], c->pred + fo[0], 1,
                                                             c->H, c->W, 1, 0);
  // the tensor-core layers' weights as BF16 operand images
  {
    WImgArgs wa;
    for (int i = 2; i <= 4; ++i) wa.w[i - 2] = P + L.c_w[i];
    wa.img = c->wimg;
    k_wtc_prep<<<6, 256, 0, c->st>>>(wa);
  }
  // conv 1 (FP32) and head 1
  k_wc1_fwd<<<blocks((long long)c->h[1] * c->w[1]), 256, 0, c->st>>>(
      c->x, c->H, c->W, P + L.c_w[1], P + L.c_b[1], P + L.h_w[1], P + L.h_b[1], c->act[1],
      c->h[1], c->w[1], c->pred + fo[1]);
  // conv 2 .. 4 on the tensor cores, each with its head
  for (int i = 2; i <= 4; ++i) {
    TcConv a = tc_args(c, i);
    a.in = c->act[i - 1];
    a.out = c->act[i];
    a.hw = P + L.h_w[i];
    a.hb = P + L.h_b[i];
    a.pred = c->pred + fo[i];
    const int n = c->h[i] * c->w[i];
    k_wtc_conv<false><<<(n + 127) / 128, 128, kTcSmem, c->st>>>(a);
  }
  WCK(cudaGetLastError());
  return CC_OK;
}

// loss into c->loss (device) and the gradients into c->grads, for targets (flat latent
// order, device)
int warm_backward(cc_warm* c, const float* target) {
  const WarmLayout& L = c->L;
  const Geo& g = c->geo;
  float* P = c->params;
  float* G = c->grads;
  long long fo[kLevels];
  level_offsets(g, fo);
  LossLevels lv;
  lv.first[0] = 0;
  for (int l = 0; l <= 4; ++l) {
    lv.n[l] = g.h[l] * g.w[l];
    lv.off[l] = fo[l];
    lv.first[l + 1] = lv.first[l] + blocks(lv.n[l]);
  }
  k_wloss<<<lv.first[5], 256, 0, c->st>>>(lv, c->pred, target, c->dpred, c->part);
  k_wloss_sum<<<1, 256, 0, c->st>>>(c->part, lv.first[5], c->loss);
  // level 0 head (3x3 on the image): weight gradient only
  {
    const int nbk = (c->H * c->W + kWPix - 1) / kWPix;
    k_whead0_wgrad_part<<<nbk, 256, 0, c->st>>>(c->dpred + fo[0], c->x, c->H, c->W, c->wpart);
    k_wsum_parts<<<(28 + 7) / 8, 256, 0, c->st>>>(c->wpart, nbk, 28, 28, G + L.h_w[0],
                                               G + L.h_b[0]);
  }
  // heads 1 .. 4 (after head 0's sums have read c->wpart: same stream)
  {
    HeadLevels hl;
    hl.first[0] = 0;
    for (int i = 1; i <= 4; ++i) {
      hl.act[i - 1] = c->act[i];
      hl.dpred[i - 1] = c->dpred + fo[i];
      hl.n[i - 1] = c->h[i] * c->w[i];
      hl.first[i] = hl.first[i - 1] + (hl.n[i - 1] + kWPix - 1) / kWPix;
    }
    k_whead_wgrad_part<<<hl.first[4], 256, 0, c->st>>>(hl, c->wpart);
    k_whead_wsum<<<(4 * (kWCh + 1) + 7) / 8, 256, 0, c->st>>>(hl, c->wpart, G + L.h_w[1]);
  }
  // conv 4's output gradient comes from head 4 only
  {
    const int n = c->h[4] * c->w[4];
    k_whead_top<<<blocks((long long)n * kWCh), 256, 0, c->st>>>(c->act[4], P + L.h_w[4],
                                                                c->dpred + fo[4], n, c->dact[4]);
  }
  for (int i = 4; i >= 2; --i) {
    // weight gradient of conv i
    const int n = c->h[i] * c->w[i];
    const int ctas = std::min(c->wg_ctas, (n + 127) / 128);
    k_wtc_wgrad<<<ctas, 128, kWgSmem, c->st>>>(c->act[i - 1], c->h[i - 1], c->w[i - 1],
                                               c->dact[i], c->h[i], c->w[i], c->wpart, c->fault);
    k_wtc_wreduce<<<blocks((long long)kWgRows * kWCh), 256, 0, c->st>>>(c->wpart, ctas,
                                                                        G + L.c_w[i],
                                                                        G + L.c_b[i]);
    // input gradient of conv i, with head i - 1's gradient and the ReLU of its input
    TcConv a = tc_args(c, i);
    a.in = c->dact[i];
    a.out = c->dact[i - 1];
    a.hw = P + L.h_w[i - 1];
    a.dpred = c->dpred + fo[i - 1];
    a.act_in = c->act[i - 1];
    a.wimg += kTcBBytes;
    const int ni = c->h[i - 1] * c->w[i - 1];
    k_wtc_conv<true><<<(ni + 127) / 128, 128, kTcSmem, c->st>>>(a);
  }
  // conv 1's weight gradient (its input, the image, needs none)
  {
    const int nbk = (c->h[1] * c->w[1] + kWPix1 - 1) / kWPix1;
    k_wc1_wgrad_part<<<nbk, 256, 0, c->st>>>(c->dact[1], c->h[1], c->w[1], c->x, c->H, c->W,
                                             c->wpart);
    k_wsum_parts<<<(kWCh * 28 + 7) / 8, 256, 0, c->st>>>(c->wpart, nbk, kWCh * 28, 28,
                                                            G + L.c_w[1], G + L.c_b[1]);
  }
  WCK(cudaGetLastError());
  return CC_OK;
}

// Adam on the parameters with the device state, then the step count
int warm_adam(cc_warm* c) {
  k_wadam<<<blocks(c->L.total), 256, 0, c->st>>>(c->params, c->m, c->v, c->grads, c->L.total,
                                                  c->adam);
  k_wadam_advance<<<1, 1, 0, c->st>>>(c->adam);
  WCK(cudaGetLastError());
  return CC_OK;
}

int warm_image(cc_warm* c, const uint8_t* rgb);
int warm_planar(cc_warm* c);

// capture what fn enqueues on c->st as a graph (on a stream of its own)
template <typename F>
int capture(cc_warm* c, F fn, cudaGraphExec_t* out) {
  cudaStream_t cs;
  WCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t keep = c->st;
  c->st = cs;
  cudaGraph_t g = nullptr;
  int e = CC_OK;
  cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    e = fn();
    const cudaError_t ce2 = cudaStreamEndCapture(cs, &g);
    if (ce == cudaSuccess) ce = ce2;
  }
  c->st = keep;
  if (ce == cudaSuccess && e == CC_OK) ce = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e) return e;
  if (ce != cudaSuccess) return wfail(ce, "predictor graph capture");
  return CC_OK;
}

// A training step's forward pass, loss and gradients from the predictor's image and
// target buffers, as one graph (captured on first use); lr goes to the device state when it
// changes.  The Adam update is the graph c->update.
int train_graph(cc_warm* c, float lr) {
  if (!c->pass) {
    int e = capture(c, [&] {
      int r = warm_planar(c);
      if (!r) r = warm_forward(c);
      if (!r) r = warm_backward(c, c->target);
      return r;
    }, &c->pass);
    if (!e) e = capture(c, [&] { return warm_adam(c); }, &c->update);
    if (e) return e;
  }
  if (lr != c->lr) {
    WCK(cudaMemcpyAsync(&c->adam->lr, &lr, sizeof(float), cudaMemcpyHostToDevice, c->st));
    WCK(cudaStreamSynchronize(c->st));
    c->lr = lr;
  }
  WCK(cudaGraphLaunch(c->pass, c->st));
  return CC_OK;
}

// the last loss (synchronises); CC_ETIMEOUT if a tensor-core wait gave up
int read_loss(cc_warm* c, double* loss) {
  double l = 0.0;
  int f = 0;
  WCK(cudaMemcpyAsync(&l, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  WCK(cudaMemcpyAsync(&f, c->fault, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  WCK(cudaStreamSynchronize(c->st));
  if (loss) *loss = l;
  if (f) {
    cc::set_error_text("a tensor-core wait of the warm-start predictor gave up");
    return CC_ETIMEOUT;
  }
  return std::isfinite(l) ? CC_OK : CC_ENONFINITE;
}

int warm_planar(cc_warm* c) {
  WCK(image_to_planar(c->img, c->x, c->H, c->W, c->st));
  return CC_OK;
}

int warm_image(cc_warm* c, const uint8_t* rgb) {
  WCK(cudaMemcpyAsync(c->img, rgb, (size_t)3 * c->H * c->W, cudaMemcpyDefault, c->st));
  return warm_planar(c);
}

}  // namespace

extern "C" {

int cc_warm_param_count(int* n) {
  if (!n) return CC_EINVAL;
  *n = warm_layout().total;
  return CC_OK;
}

int cc_warm_create(int H, int W, const float* params, void* stream, cc_warm** out) {
  if (!out || !params || H < 16 || W < 16 || H > 16384 || W > 16384) return CC_EINVAL;
  *out = nullptr;
  cc_warm* c = new cc_warm();
  c->H = H; c->W = W;
  c->L = warm_layout();
  c->st = (cudaStream_t)stream;
  cudaGetDevice(&c->dev);
  // the library's latent geometry (level l: ceil(H / 2^l) x ceil(W / 2^l))
  for (int l = 0; l < kLevels; ++l) {
    c->geo.h[l] = (H + (1 << l) - 1) >> l;
    c->geo.w[l] = (W + (1 << l) - 1) >> l;
  }
  c->geo.n_lat = 0;
  for (int l = 0; l < kLevels; ++l) c->geo.n_lat += c->geo.h[l] * c->geo.w[l];
  c->h[0] = H; c->w[0] = W;
  for (int i = 1; i <= 4; ++i) { c->h[i] = (c->h[i - 1] + 1) / 2; c->w[i] = (c->w[i - 1] + 1) / 2; }
  c->n_part = 0;
  for (int l = 0; l <= 4; ++l) c->n_part += blocks((long long)c->geo.h[l] * c->geo.w[l]);
  // one allocation
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t at = off; off = (off + bytes + 255) & ~(size_t)255; return at; };
  const size_t NP = (size_t)c->L.total * sizeof(float);
  const size_t o_p = take(NP), o_g = take(NP), o_m = take(NP), o_v = take(NP);
  const size_t o_x = take((size_t)3 * H * W * sizeof(float));
  size_t o_a[5] = {0}, o_d[5] = {0};
  for (int i = 1; i <= 4; ++i) {
    o_a[i] = take((size_t)kWCh * c->h[i] * c->w[i] * sizeof(float));
    o_d[i] = take((size_t)kWCh * c->h[i] * c->w[i] * sizeof(float));
  }
  const size_t o_pred = take((size_t)c->geo.n_lat * sizeof(float));
  const size_t o_dpred = take((size_t)c->geo.n_lat * sizeof(float));
  const size_t o_tgt = take((size_t)c->geo.n_lat * sizeof(float));
  const size_t o_img = take((size_t)3 * H * W);
  const size_t o_part = take((size_t)c->n_part * sizeof(float2));
  const size_t o_loss = take(sizeof(double));
  const size_t o_adam = take(sizeof(WarmAdam));
  const size_t o_wimg = take((size_t)6 * kTcBBytes);
  const size_t o_fault = take(sizeof(int));
  c->wg_ctas = 64;
  // partial sums: the tensor-core weight gradients', conv 1's, head 0's and the heads'
  const size_t nb1 = ((size_t)c->h[1] * c->w[1] + kWPix1 - 1) / kWPix1;
  const size_t nb0 = ((size_t)H * W + kWPix - 1) / kWPix;
  size_t nbh = 0;   // blocks of the heads' partial sums, levels 1 .. 4
  for (int i = 1; i <= 4; ++i) nbh += ((size_t)c->h[i] * c->w[i] + kWPix - 1) / kWPix;
  const size_t wpart_floats = std::max({(size_t)c->wg_ctas * kWgRows * kWCh, nb1 * kWCh * 28,
                                        nb0 * 28, nbh * (kWCh + 1)});
  const size_t o_wpart = take(wpart_floats * sizeof(float));
  cudaError_t e = cudaMalloc(&c->mem, off);
  if (e != cudaSuccess) { delete c; return CC_ENOMEM; }
  char* b = (char*)c->mem;
  c->params = (float*)(b + o_p); c->grads = (float*)(b + o_g);
  c->m = (float*)(b + o_m); c->v = (float*)(b + o_v);
  c->x = (float*)(b + o_x);
  c->act[0] = c->dact[0] = nullptr;
  for (int i = 1; i <= 4; ++i) { c->act[i] = (float*)(b + o_a[i]); c->dact[i] = (float*)(b + o_d[i]); }
  c->pred = (float*)(b + o_pred); c->dpred = (float*)(b + o_dpred);
  c->target = (float*)(b + o_tgt);
  c->img = (uint8_t*)(b + o_img); c->part = (float2*)(b + o_part);
  c->loss = (double*)(b + o_loss); c->fault = (int*)(b + o_fault);
  c->adam = (WarmAdam*)(b + o_adam);
  c->wimg = (uint8_t*)(b + o_wimg);
  c->wpart = (float*)(b + o_wpart);
  if ((e = cudaFuncSetAttribute(k_wtc_conv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kTcSmem)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_wtc_conv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kTcSmem)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_wtc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kWgSmem)) != cudaSuccess) {
    cudaFree(c->mem);
    delete c;
    return wfail(e, "warm-start predictor kernel attributes");
  }
  std::vector<WarmAdam> ad(1);
  ad[0].t = 0;
  ad[0].lr = 0.f;
  ad[0].bc[0] = make_float2(1.f, 1.f);
  for (int k = 1; k < kWBcSteps; ++k)
    ad[0].bc[k] = make_float2((float)(1.0 / (1.0 - std::pow(0.9, (double)k))),
                              (float)(1.0 / std::sqrt(1.0 - std::pow(0.999, (double)k))));
  if ((e = cudaMemsetAsync(c->mem, 0, off, c->st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->params, params, NP, cudaMemcpyDefault, c->st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->adam, ad.data(), sizeof(WarmAdam), cudaMemcpyHostToDevice,
                           c->st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->st)) != cudaSuccess) {
    cudaFree(c->mem);
    delete c;
    return wfail(e, "warm-start predictor set-up");
  }
  *out = c;
  return CC_OK;
}

int cc_warm_predict(cc_warm* c, const uint8_t* rgb_hwc, float* latents_out) {
  if (!c || !rgb_hwc || !latents_out) return CC_EINVAL;
  WCK(cudaSetDevice(c->dev));
  int e = warm_image(c, rgb_hwc);
  if (!e) e = warm_forward(c);
  if (e) return e;
  WCK(cudaMemcpyAsync(latents_out, c->pred, (size_t)c->geo.n_lat * sizeof(float),
                      cudaMemcpyDefault, c->st));
  WCK(cudaStreamSynchronize(c->st));
  return CC_OK;
}

int cc_warm_loss_grad(cc_warm* c, const uint8_t* rgb_hwc, const float* target, double* loss,
                      float* grads_out) {
  if (!c || !rgb_hwc || !target) return CC_EINVAL;
  WCK(cudaSetDevice(c->dev));
  // the target may be host memory: staged on the device before the loss kernels read it
  WCK(cudaMemcpyAsync(c->target, target, (size_t)c->geo.n_lat * sizeof(float),
                      cudaMemcpyDefault, c->st));
  int e = warm_image(c, rgb_hwc);
  if (!e) e = warm_forward(c);
  if (!e) e = warm_backward(c, c->target);
  if (!e) e = read_loss(c, loss);
  if (e) return e;
  if (grads_out) {
    WCK(cudaMemcpyAsync(grads_out, c->grads, (size_t)c->L.total * sizeof(float),
                        cudaMemcpyDefault, c->st));
    WCK(cudaStreamSynchronize(c->st));
  }
  return CC_OK;
}

int cc_warm_train_step(cc_warm* c, const uint8_t* rgb_hwc, const float* target, float lr,
                       double* loss) {
  if (!c || !rgb_hwc || !target) return CC_EINVAL;
  WCK(cudaSetDevice(c->dev));
  WCK(cudaMemcpyAsync(c->target, target, (size_t)c->geo.n_lat * sizeof(float),
                      cudaMemcpyDefault, c->st));
  WCK(cudaMemcpyAsync(c->img, rgb_hwc, (size_t)3 * c->H * c->W, cudaMemcpyDefault, c->st));
  int e = train_graph(c, lr);
  if (!e && loss) {
    cudaPointerAttributes pa{};
    WCK(cudaPointerGetAttributes(&pa, loss));
    if (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) {
      // a device destination: the loss is copied on the stream, no synchronisation
      WCK(cudaMemcpyAsync(loss, c->loss, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    } else {
      // a host destination: synchronise, and take no step on a non-finite loss
      e = read_loss(c, loss);
    }
  }
  if (e) return e;
  WCK(cudaGraphLaunch(c->update, c->st));
  return CC_OK;
}

int cc_warm_get_params(cc_warm* c, float* out) {
  if (!c || !out) return CC_EINVAL;
  WCK(cudaMemcpyAsync(out, c->params, (size_t)c->L.total * sizeof(float), cudaMemcpyDefault, c->st));
  WCK(cudaStreamSynchronize(c->st));
  return CC_OK;
}

int cc_warm_set_params(cc_warm* c, const float* params) {
  if (!c || !params) return CC_EINVAL;
  WCK(cudaMemcpyAsync(c->params, params, (size_t)c->L.total * sizeof(float), cudaMemcpyDefault, c->st));
  WCK(cudaStreamSynchronize(c->st));
  return CC_OK;
}

void cc_warm_free(cc_warm* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->pass) cudaGraphExecDestroy(c->pass);
  if (c->update) cudaGraphExecDestroy(c->update);
  if (c->mem) cudaFree(c->mem);
  delete c;
}

}  // extern "C"
