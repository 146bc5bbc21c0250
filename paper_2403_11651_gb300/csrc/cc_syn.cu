// Upsampling f_upsilon and synthesis f_theta (Sec. II "Decoding" item iii, Table 1),
// the distortion term of eq. (1), and their adjoints.
//
// Upsampling: level l >= 1 reaches full resolution through l stride-2 k x k transposed
// convolutions ("1-1-TConv-k") with its filter; inputs are read clamp-to-edge and the
// output of each step is cropped to the next level's size.  In polyphase form every
// output takes (k/2)^2 taps: b[j] = sum over u = j + c (mod 2) of f[u] a[clamp((j+c-u)/2)],
// c = k/2 - 1, along both axes.  The planes of every step are kept in HBM (7.6 floats per
// pixel in total) so that the adjoint can read its inputs back.
//
// Synthesis per pixel: 7-C-Conv-1 + ReLU, C-3-Conv-1 + ReLU, then 3-3-ConvR-3 layers
// h <- h + act(conv3x3(h) + b) with replicate padding, act = ReLU except in the last layer.
// Weights come from __constant__ banks refreshed before every pass.  All parameter
// gradients are per-CTA partial sums written in a fixed order (no atomics).
#include "cc_internal.cuh"

namespace cc {

constexpr int kMaxC = 40;
constexpr int k3x3 = 84;                  // floats per 3x3 layer (W 3x3x3x3, b 3)
constexpr int kSyn1x1Base = 2 * k3x3;     // 1x1 layers follow two reserved 3x3 slots
constexpr int kSynBank = (kSyn1x1Base + 12 * kMaxC + 4 + 3) & ~3;
// Constant bank of the synthesis and upsampling kernels, filled by one device-to-device
// copy of an image built on the device before every pass.  Layout of `syn`:
// [3x3 layer 0 | 3x3 layer 1 | W_a^T (7 x C) | b_a (C) | W_b (3 x C) | b_b], the 1x1
// weights laid out so that those of hidden channels 2m and 2m + 1 are adjacent.  `synb`
// is a second copy read by backward passes only: with one copy the compiler keeps every
// weight used by both a forward and a backward loop in a register between the two uses.
struct __align__(16) SynBank {
  float syn[kSynBank];
  float synb[kSynBank];
  float up[(kLevels - 1) * 64];
};
__constant__ SynBank c_synbank;
#define c_syn c_synbank.syn
#define c_synb c_synbank.synb
#define c_up c_synbank.up

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

template <int T>
__device__ __forceinline__ float block_sum(float v, float* s_tmp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < T / 32; ++k) t += s_tmp[k];
  }
  __syncthreads();
  return t;
}

// ------------------------------------------------------------------ upsampling

struct UpFwdArgs {
  const float* src[kLevels - 1];
  float* dst[kLevels - 1];
  int fidx[kLevels - 1];
  int sh, sw, dh, dw;
};

// One thread per 2x2 output quad (2t + py, 2s + px): along each axis output 2t + p reads
// the inputs t + d, d in [p - K/4, p + K/4 - 1], with tap u = p - 2d + K/2 - 1, so the
// quad needs a (K/2 + 1)^2 input patch and every tap index is a compile-time constant.
template <int K>
__global__ void __launch_bounds__(256) k_up_fwd(UpFwdArgs a) {
  pdl_wait();
  pdl_trigger();
  constexpr int c = K / 2 - 1;
  constexpr int R = K / 4;          // patch rows t - R .. t + R
  constexpr int P = 2 * R + 1;
  const int li = blockIdx.y;
  const float* __restrict__ src = a.src[li];
  float* __restrict__ dst = a.dst[li];
  float f[K * K];
  const int fb = a.fidx[li] * K * K;
#pragma unroll
  for (int u = 0; u < K * K; ++u) f[u] = c_up[fb + u];
  const int qh = (a.dh + 1) >> 1, qw = (a.dw + 1) >> 1;
  const int n = qh * qw;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int t = q / qw, sx = q - t * qw;
    int col[P];
#pragma unroll
    for (int d = 0; d < P; ++d) col[d] = clampi(sx - R + d, 0, a.sw - 1);
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int dy = 0; dy < P; ++dy) {
      const float* row = src + clampi(t - R + dy, 0, a.sh - 1) * a.sw;
      float v[P];
#pragma unroll
      for (int d = 0; d < P; ++d) v[d] = __ldg(row + col[d]);
#pragma unroll
      for (int py = 0; py < 2; ++py) {
        const int uy = py - 2 * (dy - R) + c;
        if (uy < 0 || uy >= K) continue;   // compile-time
#pragma unroll
        for (int px = 0; px < 2; ++px)
#pragma unroll
          for (int dx = 0; dx < P; ++dx) {
            const int ux = px - 2 * (dx - R) + c;
            if (ux < 0 || ux >= K) continue;   // compile-time
            acc[py][px] = fmaf(f[uy * K + ux], v[dx], acc[py][px]);
          }
      }
    }
#pragma unroll
    for (int py = 0; py < 2; ++py)
#pragma unroll
      for (int px = 0; px < 2; ++px) {
        const int oy = 2 * t + py, ox = 2 * sx + px;
        if (oy < a.dh && ox < a.dw) dst[oy * a.dw + ox] = acc[py][px];
      }
  }
}

struct UpBwdArgs {
  const float* dout[kLevels - 1];   // gradient at resolution j
  const float* in[kLevels - 1];     // forward input at resolution j+1
  float* din[kLevels - 1];          // gradient at resolution j+1
  int fidx[kLevels - 1];
  int lev[kLevels - 1];
  int sh, sw, dh, dw;
  int tiles_x, tiles;               // input tiles of kUpTY x kUpTX
  float* part;                      // [gridDim.x][kLevels][K*K] of this step
};

constexpr int kUpTY = 16, kUpTX = 32;

// Shared-memory tile of one adjoint step.  Positions v of the input, real or virtual
// (beyond an edge, folding onto it through the clamp), read the outputs 2v - c + u.  A
// tile of kUpTY x kUpTX real inputs together with R = K/4 virtual positions on each side
// reads DR output rows; their columns are kept as two parity planes (even / odd offset
// from the tile's first column) so that lanes with consecutive inputs read consecutive
// words.  A holds the forward input at the tile's positions (clamped at the virtual ones).
template <int K>
struct UpBwdShape {
  static constexpr int c = K / 2 - 1, R = K / 4, H = K / 2;
  static constexpr int DR = 2 * kUpTY + 4 * R + K - 2;
  static constexpr int DW = kUpTX + 2 * R + H - 1;
  static constexpr int DS = DW | 1;
  static constexpr int AR = kUpTY + 2 * R, AW = kUpTX + 2 * R;
  static constexpr int AS = AW + 1;
  static constexpr int G = 2 * K, NW = 256 / G;   // filter-gradient lanes per worker, workers
};

// Adjoint of one step over tiles of the input plane.
//  din[i] = sum over positions v folding onto i of sum_u f[u] dout[2v - c + u]
//  dF[u]  = sum over positions v of in[clamp(v)] dout[2v - c + u]
// with outputs outside the plane counting as zero.  Each thread computes din at two
// vertically adjacent inputs (rows of their windows overlap), then, as one of 2K lanes
// of a row worker, the K/2 filter-gradient taps (uy, px + 2k) along one row of positions,
// each loaded output feeding K/2 taps through a sliding window.  Filter-gradient
// partials stay in registers over the CTA's tiles and are summed in a fixed order.
template <int K>
__global__ void __launch_bounds__(256, 2) k_up_bwd(UpBwdArgs a) {
  pdl_wait();
  pdl_trigger();
  using S = UpBwdShape<K>;
  constexpr int c = S::c, R = S::R, H = S::H, KK = K * K;
  __shared__ float s_d[2][S::DR][S::DS];
  __shared__ float s_a[S::AR][S::AS];
  __shared__ float s_red[S::NW][KK];
  const int li = blockIdx.y;
  const float* __restrict__ dout = a.dout[li];
  const float* __restrict__ in = a.in[li];
  float* __restrict__ din = a.din[li];
  float f[KK];
  const int fb = a.fidx[li] * KK;
#pragma unroll
  for (int u = 0; u < KK; ++u) f[u] = c_up[fb + u];
  const int tid = threadIdx.x;
  // input-gradient role: column tx, rows 2 ty and 2 ty + 1 of the tile
  const int tx = tid & 31, ty = tid >> 5;
  // filter-gradient role: taps (uy, px + 2k), row worker w
  const int gi = tid % S::G, w = tid / S::G;
  const int fuy = gi >> 1, fpx = gi & 1;
  float acc[H];
#pragma unroll
  for (int k = 0; k < H; ++k) acc[k] = 0.f;
  const int vymax = (a.dh - 1 + c) >> 1, vxmax = (a.dw - 1 + c) >> 1;
  for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x) {
    const int y0 = (tile / a.tiles_x) * kUpTY, x0 = (tile % a.tiles_x) * kUpTX;
    const int rb = 2 * (y0 - R) - c, cb = 2 * (x0 - R) - c;
    // every load of a thread is issued before the first is used (fixed trip counts,
    // unrolled): on the small grids of the coarse steps this latency is the kernel's time
    {
      constexpr int ND = S::DR * 2 * S::DW, KD = (ND + 255) / 256;
      constexpr int NA = S::AR * S::AW, KA = (NA + 255) / 256;
      float vd[KD], va[KA];
#pragma unroll
      for (int k = 0; k < KD; ++k) {
        const int i = tid + 256 * k;
        const int r = i / (2 * S::DW), cc2 = i - r * (2 * S::DW);
        const int oy = rb + r, ox = cb + cc2;
        vd[k] = (i < ND && oy >= 0 && oy < a.dh && ox >= 0 && ox < a.dw)
                    ? __ldg(dout + (size_t)oy * a.dw + ox) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        const int i = tid + 256 * k;
        const int r = i / S::AW, m = i - r * S::AW;
        const int vy = clampi(y0 - R + r, 0, a.sh - 1), vx = clampi(x0 - R + m, 0, a.sw - 1);
        va[k] = i < NA ? __ldg(in + (size_t)vy * a.sw + vx) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < KD; ++k) {
        const int i = tid + 256 * k;
        const int r = i / (2 * S::DW), cc2 = i - r * (2 * S::DW);
        if (i < ND) s_d[cc2 & 1][r][cc2 >> 1] = vd[k];
      }
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        const int i = tid + 256 * k;
        const int r = i / S::AW, m = i - r * S::AW;
        if (i < NA) s_a[r][m] = va[k];
      }
    }
    __syncthreads();
    // ---- input gradient at (iy, ix) and (iy + 1, ix)
    {
      const int iy = y0 + 2 * ty, ix = x0 + tx;
      const int r0 = 2 * (2 * ty + R), m0 = tx + R;
      float g0 = 0.f, g1 = 0.f;
#pragma unroll
      for (int rr = 0; rr < K + 2; ++rr) {
        float q[K];
#pragma unroll
        for (int ux = 0; ux < K; ++ux) q[ux] = s_d[ux & 1][r0 + rr][m0 + (ux >> 1)];
        if (rr < K) {
#pragma unroll
          for (int ux = 0; ux < K; ++ux) g0 = fmaf(f[rr * K + ux], q[ux], g0);
        }
        if (rr >= 2) {
#pragma unroll
          for (int ux = 0; ux < K; ++ux) g1 = fmaf(f[(rr - 2) * K + ux], q[ux], g1);
        }
      }
      // virtual positions beyond an edge fold onto the border inputs
      if (ix < a.sw) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int py = iy + e;
          if (py >= a.sh) break;
          const int vy0 = py == 0 ? -R : py, vy1 = py == a.sh - 1 ? vymax : py;
          const int vx0 = ix == 0 ? -R : ix, vx1 = ix == a.sw - 1 ? vxmax : ix;
          float g = e ? g1 : g0;
          if (vy0 != vy1 || vx0 != vx1) {
            for (int vy = vy0; vy <= vy1; ++vy)
              for (int vx = vx0; vx <= vx1; ++vx) {
                if (vy == py && vx == ix) continue;
                const int rr0 = 2 * (vy - y0 + R), mm0 = vx - x0 + R;
#pragma unroll
                for (int uy = 0; uy < K; ++uy)
#pragma unroll
                  for (int ux = 0; ux < K; ++ux)
                    g = fmaf(f[uy * K + ux], s_d[ux & 1][rr0 + uy][mm0 + (ux >> 1)], g);
              }
          }
          din[(size_t)py * a.sw + ix] = g;
        }
      }
    }
    // ---- filter gradient over the positions this tile owns
    {
      const int ry0 = y0 == 0 ? -R : y0;
      const int ry1 = y0 + kUpTY >= a.sh ? vymax : y0 + kUpTY - 1;
      const int cx0 = x0 == 0 ? -R : x0;
      const int cx1 = x0 + kUpTX >= a.sw ? vxmax : x0 + kUpTX - 1;
      const int m_lo = cx0 - x0 + R, m_hi = cx1 - x0 + R;   // inclusive, in [0, AW)
      for (int vy = ry0 + w; vy <= ry1; vy += S::NW) {
        const float* drow = &s_d[fpx][2 * (vy - y0 + R) + fuy][0];
        const float* arow = &s_a[vy - y0 + R][0];
        float q[H];
#pragma unroll
        for (int k = 0; k < H - 1; ++k) q[k] = drow[m_lo + k];
        int m = m_lo;
        for (; m + H - 1 <= m_hi; m += H) {
#pragma unroll
          for (int s = 0; s < H; ++s) {
            // window q[(s + k) % H] holds drow[m + s + k]
            q[(s + H - 1) % H] = drow[m + s + H - 1];
            const float av = arow[m + s];
#pragma unroll
            for (int k = 0; k < H; ++k) acc[k] = fmaf(av, q[(s + k) % H], acc[k]);
          }
        }
        for (; m <= m_hi; ++m) {
          const float av = arow[m];
#pragma unroll
          for (int k = 0; k < H; ++k) acc[k] = fmaf(av, drow[m + k], acc[k]);
        }
      }
    }
    __syncthreads();
  }
  // per-CTA filter gradient: row workers summed in order
#pragma unroll
  for (int k = 0; k < H; ++k) s_red[w][fuy * K + fpx + 2 * k] = acc[k];
  __syncthreads();
  for (int u = tid; u < KK; u += 256) {
    float t = 0.f;
#pragma unroll
    for (int r = 0; r < S::NW; ++r) t += s_red[r][u];
    a.part[((long long)blockIdx.x * kLevels + a.lev[li]) * KK + u] = t;
  }
}

template <int K>
static cudaError_t up_forward_k(const Arch& ar, const Geo& g, const float* yhat,
                                const UpPlan& up, int ctas, cudaStream_t st) {
  for (int j = kLevels - 2; j >= 0; --j) {
    UpFwdArgs a;
    int n = 0;
    for (int l = j + 1; l < kLevels; ++l, ++n) {
      a.src[n] = (l == j + 1) ? yhat + g.off[l] : up.plane[l][j + 1];
      a.dst[n] = up.plane[l][j];
      a.fidx[n] = ar.per_level ? l - 1 : 0;
    }
    a.sh = g.h[j + 1]; a.sw = g.w[j + 1]; a.dh = g.h[j]; a.dw = g.w[j];
    // about three resident waves in total, so that each thread loads its level's filter
    // once for several quads
    const int tot = ((a.dh + 1) / 2) * ((a.dw + 1) / 2);
    const int need = (tot + 255) / 256, cap = (3 * ctas) / n > 1 ? (3 * ctas) / n : 1;
    cudaError_t e = launch_k(k_up_fwd<K>, dim3(need < cap ? need : cap, n), dim3(256), 0, st, a);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t up_forward(const Arch& a, const Geo& g, const float* yhat, const UpPlan& up,
                       int ctas, cudaStream_t st) {
  if (a.K == 8) return up_forward_k<8>(a, g, yhat, up, ctas, st);
  if (a.K == 4) return up_forward_k<4>(a, g, yhat, up, ctas, st);
  return cudaErrorInvalidValue;
}

template <int K>
static cudaError_t up_backward_k(const Arch& ar, const Geo& g, const float* yhat,
                                 const UpPlan& up, float* gsyn, float* part_up, int grid,
                                 cudaStream_t st) {
  for (int j = 0; j < kLevels - 1; ++j) {
    UpBwdArgs a;
    int n = 0;
    for (int l = j + 1; l < kLevels; ++l, ++n) {
      a.dout[n] = up.dplane[l][j];
      a.in[n] = (l == j + 1) ? yhat + g.off[l] : up.plane[l][j + 1];
      a.din[n] = (l == j + 1) ? gsyn + g.off[l] : up.dplane[l][j + 1];
      a.fidx[n] = ar.per_level ? l - 1 : 0;
      a.lev[n] = l;
    }
    a.sh = g.h[j + 1]; a.sw = g.w[j + 1]; a.dh = g.h[j]; a.dw = g.w[j];
    // rows [j * grid, j * grid + grid) belong to this step
    a.part = part_up + (long long)j * grid * kLevels * K * K;
    // one CTA per input tile and level, at most `grid` per level (a CTA then loops over
    // several tiles); the part rows of CTAs that are not launched stay zero from the
    // context set-up
    a.tiles_x = (a.sw + kUpTX - 1) / kUpTX;
    a.tiles = a.tiles_x * ((a.sh + kUpTY - 1) / kUpTY);
    const int nb = a.tiles < grid ? a.tiles : grid;
    cudaError_t e = launch_k(k_up_bwd<K>, dim3(nb, n), dim3(256), 0, st, a);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t up_backward(const Arch& a, const Geo& g, const float* yhat, const UpPlan& up,
                        float* gsyn, float* part_up, int grid, cudaStream_t st) {
  if (a.K == 8) return up_backward_k<8>(a, g, yhat, up, gsyn, part_up, grid, st);
  if (a.K == 4) return up_backward_k<4>(a, g, yhat, up, gsyn, part_up, grid, st);
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ 3x3 residual layers
//
// The synthesis kernels work on tiles of kSTY x kSTX pixels, one pixel per thread, with
// a one-pixel halo of the 3-channel planes they gather staged in shared memory (rows of
// kSHX floats, channels kSHS floats apart: the 27 taps of one pixel fall in distinct
// banks).  Loads are replicate-clamped at the image border, which is the padding of the
// forward convolution.  With NR layers (ReLU on all but the last, which is linear):
//   forward : 1x1 stack -> h_0; layers 0 .. NR-2 (k_conv3_fwd); layer NR-1 with the
//             distortion, dL/dx_hat and the layer's weight gradient (k_conv3_last), since
//             the pre-activation gradient of a linear layer is its output gradient;
//   backward: (NR = 2) layer 1's input gradient, layer 0's pre-activation gradient and
//             weight gradient (k_conv3_mid); layer 0's input gradient inside the 1x1
//             backward (k_syn1x1_bwd).
// Per-CTA partial sums of weight gradients and distortion are written in a fixed order.

constexpr int kSTY = 8, kSTX = 32;            // synthesis tile, kSTY * kSTX = 256 threads
constexpr int kSHX = 35;                       // halo row stride (kSTX + 2 used)
constexpr int kSHS = 361;                      // halo channel stride ((kSTY + 2) rows used)
constexpr int kSHR = kSTY + 2;

struct SynTileGeo {
  int H, W, ntx, n_tiles;
};

__device__ __forceinline__ void tile_xy(const SynTileGeo& t, int tile, int& y0, int& x0) {
  const int ty = tile / t.ntx;
  y0 = ty * kSTY;
  x0 = (tile - ty * t.ntx) * kSTX;
}

// A thread's share of a halo tile load: elements i = threadIdx.x + 256 k of the
// 3 x (kSTY + 2 HALO) x (kSTX + 2 HALO) region around a tile, with their shared-memory
// index (rows RS floats apart, channels CS) and their offset from the tile's first pixel
// in a [3][H][W] plane set, computed once per kernel.  Tiles whose region lies inside the
// image load at base + offset; border tiles clamp each coordinate (replicate padding).  The
// values pass through registers so that a kernel can issue the next tile's loads before
// it computes the current one.
template <int HALO, int RS, int CS>
struct HaloPlanT {
  static constexpr int R = kSTY + 2 * HALO, C = kSTX + 2 * HALO, N = 3 * R * C;
  static constexpr int K = (N + 255) / 256;
  static_assert(C <= RS && R * RS <= CS, "halo region does not fit its layout");
  int sidx[K];   // -1: no element for this thread
  int goff[K];
  int H, W;
  __device__ __forceinline__ void init(int H_, int W_) {
    H = H_;
    W = W_;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = threadIdx.x + 256 * k;
      const int ci = i / (R * C), rc = i - ci * (R * C);
      const int r = rc / C, c = rc - r * C;
      sidx[k] = i < N ? ci * CS + r * RS + c : -1;
      goff[k] = ci * H * W + (r - HALO) * W + (c - HALO);
    }
  }
  __device__ __forceinline__ void load(float (&v)[K], const float* __restrict__ h, int y0,
                                       int x0) const {
    if (y0 >= HALO && x0 >= HALO && y0 + kSTY + HALO <= H && x0 + kSTX + HALO <= W) {
      const float* base = h + y0 * W + x0;
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = sidx[k] >= 0 ? __ldg(base + goff[k]) : 0.f;
      return;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = threadIdx.x + 256 * k;
      const int ci = i / (R * C), rc = i - ci * (R * C);
      const int r = rc / C, c = rc - r * C;
      const int gy = clampi(y0 - HALO + r, 0, H - 1), gx = clampi(x0 - HALO + c, 0, W - 1);
      v[k] = sidx[k] >= 0 ? __ldg(h + ci * H * W + gy * W + gx) : 0.f;
    }
  }
  __device__ __forceinline__ void store(float* s, const float (&v)[K]) const {
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (sidx[k] >= 0) s[sidx[k]] = v[k];
  }
};
using HaloPlan = HaloPlanT<1, kSHX, kSHS>;
constexpr int kHaloK = HaloPlan::K;

// the 27 inputs of pixel (ty, tx) of the tile: v[ci * 9 + (dy + 1) * 3 + dx + 1]
__device__ __forceinline__ void gather_halo(float (&v)[27], const float* s, int ty, int tx) {
#pragma unroll
  for (int ci = 0; ci < 3; ++ci)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx)
        v[ci * 9 + dy * 3 + dx] = s[ci * kSHS + (ty + dy) * kSHX + tx + dx];
}

template <int I>
__device__ __forceinline__ void conv_z(float (&z)[3], const float (&v)[27]) {
  constexpr int Wo = I * k3x3;
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    float s = c_syn[Wo + 81 + o];
#pragma unroll
    for (int k = 0; k < 27; ++k) s = fmaf(c_syn[Wo + o * 27 + k], v[k], s);
    z[o] = s;
  }
}

// Adjoint of layer I at pixel (y, x) = tile (ty, tx): sum over the outputs p and taps whose
// replicate-clamped read landed on (y, x) of W[o][ci][tap] dz[o][p].  s_dz holds dz over
// the tile and its halo; inside the image only p = (y, x) - tap qualify.
template <int I>
__device__ __forceinline__ void conv_adjoint(float (&acc)[3], const float* s_dz, int ty, int tx,
                                             int y, int x, int y0, int x0, int H, int W) {
  constexpr int Wo = I * k3x3;
  if (y > 0 && x > 0 && y < H - 1 && x < W - 1) {
#pragma unroll
    for (int ci = 0; ci < 3; ++ci)
#pragma unroll
      for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx)
            acc[ci] = fmaf(c_synb[Wo + o * 27 + ci * 9 + (dy + 1) * 3 + (dx + 1)],
                           s_dz[o * kSHS + (ty + 1 - dy) * kSHX + tx + 1 - dx], acc[ci]);
    return;
  }
  for (int dy = -1; dy <= 1; ++dy)
    for (int py = y - dy - 1; py <= y - dy + 1; ++py) {
      if (py < 0 || py >= H || clampi(py + dy, 0, H - 1) != y) continue;
      for (int dx = -1; dx <= 1; ++dx)
        for (int px = x - dx - 1; px <= x - dx + 1; ++px) {
          if (px < 0 || px >= W || clampi(px + dx, 0, W - 1) != x) continue;
          const float* d = s_dz + (py - y0 + 1) * kSHX + (px - x0 + 1);
#pragma unroll
          for (int o = 0; o < 3; ++o)
#pragma unroll
            for (int ci = 0; ci < 3; ++ci)
              acc[ci] = fmaf(c_synb[Wo + o * 27 + ci * 9 + (dy + 1) * 3 + (dx + 1)],
                             d[o * kSHS], acc[ci]);
        }
    }
}

// Weight-gradient partial of one 3x3 layer over a tile.  Thread t < 255 owns input
// channel ci = t / 85 and the pixels q = t % 85 + 85 j of the tile; it adds the 27 products
// dz[o][q] h[ci][q + tap] (o < 3, 9 taps) and the bias terms dz[o][q] into registers that
// persist over the CTA's tiles.  s_dz: [3][256], s_h: the layer input's halo tile.
// s_h points at the tap (-1, -1) of the tile's first pixel in a layout of rows RS and
// channels CS floats apart (the one-pixel halo tile by default).
constexpr int kWG = 85;                        // pixel groups per channel
template <int RS = kSHX, int CS = kSHS>
__device__ __forceinline__ void conv_wgrad(float (&acc)[30], const float* s_dz, const float* s_h) {
  const int t = threadIdx.x;
  if (t >= 3 * kWG) return;
  const int ci = t / kWG;
  for (int q = t - ci * kWG; q < 256; q += kWG) {
    const float* hh = s_h + ci * CS + (q >> 5) * RS + (q & 31);
    float hv[9];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) hv[dy * 3 + dx] = hh[dy * RS + dx];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float d = s_dz[o * 256 + q];
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[o * 9 + k] = fmaf(d, hv[k], acc[o * 9 + k]);
      acc[27 + o] += d;
    }
  }
}

// Per-CTA sum of conv_wgrad's registers in a fixed order: s_red holds kWG x 84 floats
// (it may alias the tiles, which are dead by then).
__device__ __forceinline__ void conv_wgrad_store(const float (&acc)[30], float* s_red, float* part) {
  const int t = threadIdx.x;
  __syncthreads();
  if (t < 3 * kWG) {
    const int ci = t / kWG, g = t - ci * kWG;
    float* row = s_red + g * 84;
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
      for (int k = 0; k < 9; ++k) row[o * 27 + ci * 9 + k] = acc[o * 9 + k];
    if (ci == 0) {
#pragma unroll
      for (int o = 0; o < 3; ++o) row[81 + o] = acc[27 + o];
    }
  }
  __syncthreads();
  if (t < 84) {
    float sum = 0.f;
    for (int g = 0; g < kWG; ++g) sum += s_red[g * 84 + t];
    part[(long long)blockIdx.x * 84 + t] = sum;
  }
}

struct ConvArgs {
  SynTileGeo t;
  const float* hin;    // [3][HW] layer input
  float* hout;         // [3][HW] layer output
  const float* x;      // [3][HW] image (last layer)
  float* dxhat;        // [3][HW] dL/dx_hat (last layer)
  const float* g;      // [3][HW] output gradient of layer 1 (= its pre-activation gradient)
  float* dh;           // [3][HW] gradient of layer 1's input
  float* dz;           // [3][HW] pre-activation gradient of layer 0
  float* part;         // per-CTA partials (84 per CTA)
  float* part_d;       // per-CTA distortion partials (last layer)
  float dscale;        // 2 / (3 H W)
};

// Layer I (not the last): h_out = h_in + ReLU(conv(h_in) + b).
template <int I>
__global__ void __launch_bounds__(256) k_conv3_fwd(ConvArgs a) {
  pdl_wait();
  pdl_trigger();
  __shared__ float s_h[3 * kSHS];
  const int HW = a.t.H * a.t.W;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  HaloPlan hp;
  hp.init(a.t.H, a.t.W);
  float nv[kHaloK];
  if (blockIdx.x < a.t.n_tiles) {
    int y0, x0;
    tile_xy(a.t, blockIdx.x, y0, x0);
    hp.load(nv, a.hin, y0, x0);
  }
  for (int tile = blockIdx.x; tile < a.t.n_tiles; tile += gridDim.x) {
    int y0, x0;
    tile_xy(a.t, tile, y0, x0);
    hp.store(s_h, nv);
    __syncthreads();
    if (tile + (int)gridDim.x < a.t.n_tiles) {
      int ny0, nx0;
      tile_xy(a.t, tile + gridDim.x, ny0, nx0);
      hp.load(nv, a.hin, ny0, nx0);
    }
    const int y = y0 + ty, x = x0 + tx;
    if (y < a.t.H && x < a.t.W) {
      float v[27], z[3];
      gather_halo(v, s_h, ty, tx);
      conv_z<I>(z, v);
#pragma unroll
      for (int o = 0; o < 3; ++o) a.hout[o * HW + y * a.t.W + x] = v[o * 9 + 4] + fmaxf(z[o], 0.f);
    }
    __syncthreads();
  }
}

// Last layer I (linear): x_hat = h_in + conv(h_in) + b, the distortion partial sum of
// (x_hat - x)^2, dL/dx_hat = 2 (x_hat - x) / (3HW), and the layer's weight gradient.
template <int I>
__global__ void __launch_bounds__(256, 3) k_conv3_last(ConvArgs a) {
  pdl_wait();
  pdl_trigger();
  __shared__ float s_all[kWG * 84];   // halo tile + dz, then the reduction
  __shared__ float s_tmp[8];
  float* s_h = s_all;
  float* s_dz = s_all + 3 * kSHS;
  const int HW = a.t.H * a.t.W;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float dsum = 0.f;
  float wacc[30];
#pragma unroll
  for (int k = 0; k < 30; ++k) wacc[k] = 0.f;
  HaloPlan hp;
  hp.init(a.t.H, a.t.W);
  float nv[kHaloK];
  if (blockIdx.x < a.t.n_tiles) {
    int y0, x0;
    tile_xy(a.t, blockIdx.x, y0, x0);
    hp.load(nv, a.hin, y0, x0);
  }
  for (int tile = blockIdx.x; tile < a.t.n_tiles; tile += gridDim.x) {
    int y0, x0;
    tile_xy(a.t, tile, y0, x0);
    hp.store(s_h, nv);
    __syncthreads();
    if (tile + (int)gridDim.x < a.t.n_tiles) {
      int ny0, nx0;
      tile_xy(a.t, tile + gridDim.x, ny0, nx0);
      hp.load(nv, a.hin, ny0, nx0);
    }
    const int y = y0 + ty, x = x0 + tx;
    const bool valid = y < a.t.H && x < a.t.W;
    float v[27], z[3];
    gather_halo(v, s_h, ty, tx);
    conv_z<I>(z, v);
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      float g = 0.f;
      if (valid) {
        const int p = o * HW + y * a.t.W + x;
        const float out = v[o * 9 + 4] + z[o];
        a.hout[p] = out;
        const float d = out - __ldg(a.x + p);
        dsum = fmaf(d, d, dsum);
        g = d * a.dscale;
        a.dxhat[p] = g;
      }
      s_dz[o * 256 + threadIdx.x] = g;
    }
    __syncthreads();
    conv_wgrad(wacc, s_dz, s_h);
    __syncthreads();
  }
  const float t = block_sum<256>(dsum, s_tmp);
  if (threadIdx.x == 0) a.part_d[blockIdx.x] = t;
  conv_wgrad_store(wacc, s_all, a.part);
}

// NR = 2: gradient of layer 1's input, dh = g + conv_1^T(g) (layer 1 is linear, so g is
// also its pre-activation gradient); layer 0's pre-activation gradient dz = [z_0 > 0] dh
// with z_0 recomputed from h_0; layer 0's weight gradient.
__global__ void __launch_bounds__(256, 3) k_conv3_mid(ConvArgs a) {
  pdl_wait();
  pdl_trigger();
  __shared__ float s_all[kWG * 84];   // two halo tiles + dz, then the reduction
  float* s_g = s_all;
  float* s_h = s_all + 3 * kSHS;
  float* s_dz = s_all + 6 * kSHS;
  const int HW = a.t.H * a.t.W;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float wacc[30];
#pragma unroll
  for (int k = 0; k < 30; ++k) wacc[k] = 0.f;
  HaloPlan hp;
  hp.init(a.t.H, a.t.W);
  float nvg[kHaloK], nvh[kHaloK];
  if (blockIdx.x < a.t.n_tiles) {
    int y0, x0;
    tile_xy(a.t, blockIdx.x, y0, x0);
    hp.load(nvg, a.g, y0, x0);
    hp.load(nvh, a.hin, y0, x0);
  }
  for (int tile = blockIdx.x; tile < a.t.n_tiles; tile += gridDim.x) {
    int y0, x0;
    tile_xy(a.t, tile, y0, x0);
    hp.store(s_g, nvg);
    hp.store(s_h, nvh);
    __syncthreads();
    if (tile + (int)gridDim.x < a.t.n_tiles) {
      int ny0, nx0;
      tile_xy(a.t, tile + gridDim.x, ny0, nx0);
      hp.load(nvg, a.g, ny0, nx0);
      hp.load(nvh, a.hin, ny0, nx0);
    }
    const int y = y0 + ty, x = x0 + tx;
    const bool valid = y < a.t.H && x < a.t.W;
    float dz[3] = {0.f, 0.f, 0.f};
    if (valid) {
      float dh[3];
#pragma unroll
      for (int ci = 0; ci < 3; ++ci) dh[ci] = s_g[ci * kSHS + (ty + 1) * kSHX + tx + 1];
      conv_adjoint<1>(dh, s_g, ty, tx, y, x, y0, x0, a.t.H, a.t.W);
      float v[27], z[3];
      gather_halo(v, s_h, ty, tx);
      conv_z<0>(z, v);
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        const int p = o * HW + y * a.t.W + x;
        dz[o] = z[o] > 0.f ? dh[o] : 0.f;
        a.dh[p] = dh[o];
        a.dz[p] = dz[o];
      }
    }
#pragma unroll
    for (int o = 0; o < 3; ++o) s_dz[o * 256 + threadIdx.x] = dz[o];
    __syncthreads();
    conv_wgrad(wacc, s_dz, s_h);
    __syncthreads();
  }
  conv_wgrad_store(wacc, s_all, a.part);
}

// NR = 2 in a pass with gradients: the three 3x3 kernels above in one.  On 8 x 32 tiles,
// from h_0 staged with a 3-pixel halo and x with a 1-pixel halo (replicate-clamped):
//   A: h_1 = h_0 + ReLU(conv_0(h_0) + b_0) on the tile and a 2-pixel halo, and the sign of
//      layer 0's pre-activation z_0 on the tile;
//   B: x_hat = h_1 + conv_1(h_1) + b_1 and g = dL/dx_hat = 2 (x_hat - x) / (3HW) on the tile
//      and a 1-pixel halo (the halo's g is recomputed, not read back); x_hat, g and the
//      distortion partial of the tile;
//   C: on the tile, layer 1's weight gradient (g (x) h_1), its input gradient
//      dh = g + conv_1^T(g), layer 0's pre-activation gradient dz = [z_0 > 0] dh and weight
//      gradient (dz (x) h_0).  dh and dz go to HBM for the 1x1 backward.
// A halo position is computed at its clamped pixel, so that it holds what the replicate
// padding of the next layer reads.  Neither h_1 nor the halo's g leaves the CTA.
constexpr int kP3X = kSTX + 7, kP3S = (kSTY + 6) * kP3X + 1;   // h_0 with a 3-pixel halo
constexpr int kP2X = kSTX + 5, kP2S = (kSTY + 4) * kP2X + 1;   // h_1 with a 2-pixel halo
struct PairSmem {
  static constexpr int H0 = 0, H1 = H0 + 3 * kP3S, G = H1 + 3 * kP2S, X = G + 3 * kSHS,
                       DZ1 = X + 3 * kSHS, DZ0 = DZ1 + 768, M0 = DZ0 + 768, END = M0 + 768;
  static constexpr int FLOATS = END > kWG * 84 ? END : kWG * 84;
};

// Element i = threadIdx.x + 256 k of the 3 x (kSTY + 2 HALO) x (kSTX + 2 HALO) region around
// a tile, clamped to the image, without per-thread index tables (register budget).
template <int HALO, int RS, int CS>
struct HaloLoad {
  static constexpr int R = kSTY + 2 * HALO, C = kSTX + 2 * HALO, N = 3 * R * C;
  static constexpr int K = (N + 255) / 256;
  static_assert(C <= RS && R * RS <= CS, "halo region does not fit its layout");
  static __device__ __forceinline__ void load(float (&v)[K], const float* __restrict__ h,
                                              int y0, int x0, int H, int W) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = threadIdx.x + 256 * k;
      const int ci = i / (R * C), rc = i - ci * (R * C);
      const int r = rc / C, c = rc - r * C;
      const int gy = clampi(y0 - HALO + r, 0, H - 1), gx = clampi(x0 - HALO + c, 0, W - 1);
      // past the region (i >= N) the address stays inside the three planes
      v[k] = i < N ? __ldg(h + (ci < 3 ? ci : 2) * H * W + gy * W + gx) : 0.f;
    }
  }
  static __device__ __forceinline__ void store(float* s, const float (&v)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = threadIdx.x + 256 * k;
      const int ci = i / (R * C), rc = i - ci * (R * C);
      const int r = rc / C, c = rc - r * C;
      if (i < N) s[ci * CS + r * RS + c] = v[k];
    }
  }
};

// the 27 inputs of a 3x3 layer at a pixel whose clamped tap rows and columns are rr, cc in
// a staged layout of rows RS and channels CS floats apart
template <int RS, int CS>
__device__ __forceinline__ void gather_at(float (&v)[27], const float* s, const int (&rr)[3],
                                          const int (&cc)[3]) {
#pragma unroll
  for (int ci = 0; ci < 3; ++ci)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx)
        v[ci * 9 + dy * 3 + dx] = s[ci * CS + rr[dy] * RS + cc[dx]];
}

__global__ void __launch_bounds__(256, 2) k_conv3_pair(ConvArgs a) {
  pdl_wait();
  pdl_trigger();
  using L3 = HaloLoad<3, kP3X, kP3S>;
  using L1 = HaloLoad<1, kSHX, kSHS>;
  __shared__ float s_all[PairSmem::FLOATS];
  __shared__ float s_tmp[8];
  float* s_h0 = s_all + PairSmem::H0;
  float* s_h1 = s_all + PairSmem::H1;
  float* s_g = s_all + PairSmem::G;
  float* s_x = s_all + PairSmem::X;
  float* s_dz1 = s_all + PairSmem::DZ1;
  float* s_dz0 = s_all + PairSmem::DZ0;
  float* s_m0 = s_all + PairSmem::M0;
  const int H = a.t.H, W = a.t.W, HW = H * W;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float dsum = 0.f;
  float w1[30], w0[30];
#pragma unroll
  for (int k = 0; k < 30; ++k) w1[k] = w0[k] = 0.f;
  float n3[L3::K], n1[L1::K];
  if (blockIdx.x < a.t.n_tiles) {
    int y0, x0;
    tile_xy(a.t, blockIdx.x, y0, x0);
    L3::load(n3, a.hin, y0, x0, H, W);
    L1::load(n1, a.x, y0, x0, H, W);
  }
  for (int tile = blockIdx.x; tile < a.t.n_tiles; tile += gridDim.x) {
    int y0, x0;
    tile_xy(a.t, tile, y0, x0);
    L3::store(s_h0, n3);
    L1::store(s_x, n1);
    __syncthreads();
    if (tile + (int)gridDim.x < a.t.n_tiles) {
      int ny0, nx0;
      tile_xy(a.t, tile + gridDim.x, ny0, nx0);
      L3::load(n3, a.hin, ny0, nx0, H, W);
      L1::load(n1, a.x, ny0, nx0, H, W);
    }
    // A: h_1 over the tile and a 2-pixel halo
    for (int i = threadIdx.x; i < (kSTY + 4) * (kSTX + 4); i += 256) {
      const int r = i / (kSTX + 4), c = i - r * (kSTX + 4);
      const int py = clampi(y0 - 2 + r, 0, H - 1), px = clampi(x0 - 2 + c, 0, W - 1);
      int rr[3], cc[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        rr[d] = clampi(py + d - 1, 0, H - 1) - (y0 - 3);
        cc[d] = clampi(px + d - 1, 0, W - 1) - (x0 - 3);
      }
      float v[27], z[3];
      gather_at<kP3X, kP3S>(v, s_h0, rr, cc);
      conv_z<0>(z, v);
#pragma unroll
      for (int o = 0; o < 3; ++o) s_h1[o * kP2S + r * kP2X + c] = v[o * 9 + 4] + fmaxf(z[o], 0.f);
      const int qy = r - 2, qx = c - 2;
      if ((unsigned)qy < (unsigned)kSTY && (unsigned)qx < (unsigned)kSTX) {
#pragma unroll
        for (int o = 0; o < 3; ++o) s_m0[o * 256 + qy * kSTX + qx] = z[o] > 0.f ? 1.f : 0.f;
      }
    }
    __syncthreads();
    // B: x_hat and g over the tile and a 1-pixel halo
    for (int i = threadIdx.x; i < (kSTY + 2) * (kSTX + 2); i += 256) {
      const int r = i / (kSTX + 2), c = i - r * (kSTX + 2);
      const int py = clampi(y0 - 1 + r, 0, H - 1), px = clampi(x0 - 1 + c, 0, W - 1);
      int rr[3], cc[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        rr[d] = clampi(py + d - 1, 0, H - 1) - (y0 - 2);
        cc[d] = clampi(px + d - 1, 0, W - 1) - (x0 - 2);
      }
      float v[27], z[3];
      gather_at<kP2X, kP2S>(v, s_h1, rr, cc);
      conv_z<1>(z, v);
      const int qy = r - 1, qx = c - 1;
      const bool in_tile = (unsigned)qy < (unsigned)kSTY && (unsigned)qx < (unsigned)kSTX;
      const bool valid = in_tile && y0 + qy < H && x0 + qx < W;
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        const float xh = v[o * 9 + 4] + z[o];
        const float d = xh - s_x[o * kSHS + r * kSHX + c];
        const float g = d * a.dscale;
        s_g[o * kSHS + r * kSHX + c] = g;
        if (in_tile) s_dz1[o * 256 + qy * kSTX + qx] = valid ? g : 0.f;
        if (valid) {
          const int p = o * HW + (y0 + qy) * W + x0 + qx;
          a.hout[p] = xh;
          a.dxhat[p] = g;
          dsum = fmaf(d, d, dsum);
        }
      }
    }
    __syncthreads();
    // C: layer 1's weight gradient, its input gradient, layer 0's pre-activation gradient
    conv_wgrad<kP2X, kP2S>(w1, s_dz1, s_h1 + kP2X + 1);
    {
      const int y = y0 + ty, x = x0 + tx;
      float dz[3] = {0.f, 0.f, 0.f};
      if (y < H && x < W) {
        float dh[3];
#pragma unroll
        for (int ci = 0; ci < 3; ++ci) dh[ci] = s_g[ci * kSHS + (ty + 1) * kSHX + tx + 1];
        conv_adjoint<1>(dh, s_g, ty, tx, y, x, y0, x0, H, W);
#pragma unroll
        for (int o = 0; o < 3; ++o) {
          dz[o] = s_m0[o * 256 + threadIdx.x] > 0.f ? dh[o] : 0.f;
          const int p = o * HW + y * W + x;
          a.dh[p] = dh[o];
          a.dz[p] = dz[o];
        }
      }
#pragma unroll
      for (int o = 0; o < 3; ++o) s_dz0[o * 256 + threadIdx.x] = dz[o];
    }
    __syncthreads();
    conv_wgrad<kP3X, kP3S>(w0, s_dz0, s_h0 + 2 * kP3X + 2);
    __syncthreads();
  }
  const float t = block_sum<256>(dsum, s_tmp);
  if (threadIdx.x == 0) a.part_d[blockIdx.x] = t;
  conv_wgrad_store(w1, s_all, a.part + (size_t)gridDim.x * 84);
  conv_wgrad_store(w0, s_all, a.part);
}

// ------------------------------------------------------------------ synthesis 1x1 layers

struct Syn1x1Args {
  const float* feat[kLevels];   // level-0 latents, then the upsampled planes of l = 1..6
  float* h2;                    // [3][HW] output of the C-3 layer (written forward, read backward)
  const float* dhout;           // [3][HW] output gradient of 3x3 layer 0 (backward)
  const float* dz0;             // [3][HW] its pre-activation gradient (backward)
  float* dfeat[kLevels];        // gradient of each feature plane
  float* part;                  // [gridDim.x][11C + 3]
  int HW;
  SynTileGeo t;
};

// The 1x1 layers run on packed FP32 pairs over the hidden channel: the bank holds W_a
// transposed (7 x C) and W_b row-major (3 x C), so that the weights of channels 2m and
// 2m + 1 are adjacent.  z_1 and dL/dh_1 are exact per channel; z_2 and dL/df sum the even
// and the odd channels separately and add the two halves at the end.
template <int C>
struct Syn1x1W {
  static constexpr int WAT = kSyn1x1Base, BA = WAT + 7 * C, WBR = BA + C, BB = WBR + 3 * C;
  static constexpr int M = C / 2;   // channel pairs
};

// Two pixels per thread (p and p + 256 of the block's 512), so that every weight pair
// loaded from the bank serves both.
template <int C>
__global__ void __launch_bounds__(256) k_syn1x1_fwd(Syn1x1Args a) {
  pdl_wait();
  pdl_trigger();
  using Wt = Syn1x1W<C>;
  constexpr int M = Wt::M;
  const float2* wa = reinterpret_cast<const float2*>(c_syn + Wt::WAT);   // [7][M]
  const float2* ba = reinterpret_cast<const float2*>(c_syn + Wt::BA);    // [M]
  const float2* wb = reinterpret_cast<const float2*>(c_syn + Wt::WBR);   // [3][M]
  for (int p0 = blockIdx.x * 512 + threadIdx.x; p0 < a.HW; p0 += gridDim.x * 512) {
    const int p1 = p0 + 256;
    const bool v1 = p1 < a.HW;
    float2 fa[kLevels], fb[kLevels];
#pragma unroll
    for (int k = 0; k < kLevels; ++k) {
      const float u = __ldg(a.feat[k] + p0), v = v1 ? __ldg(a.feat[k] + p1) : 0.f;
      fa[k] = make_float2(u, u);
      fb[k] = make_float2(v, v);
    }
    float2 za2[3], zb2[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) za2[j] = zb2[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float2 za = ba[m], zb = za;
#pragma unroll
      for (int k = 0; k < kLevels; ++k) {
        const float2 w = wa[k * M + m];
        za = __ffma2_rn(w, fa[k], za);
        zb = __ffma2_rn(w, fb[k], zb);
      }
      const float2 ha = make_float2(fmaxf(za.x, 0.f), fmaxf(za.y, 0.f));
      const float2 hb = make_float2(fmaxf(zb.x, 0.f), fmaxf(zb.y, 0.f));
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float2 w = wb[j * M + m];
        za2[j] = __ffma2_rn(w, ha, za2[j]);
        zb2[j] = __ffma2_rn(w, hb, zb2[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float bj = c_syn[Wt::BB + j];
      a.h2[j * a.HW + p0] = fmaxf(bj + (za2[j].x + za2[j].y), 0.f);
      if (v1) a.h2[j * a.HW + p1] = fmaxf(bj + (zb2[j].x + zb2[j].y), 0.f);
    }
  }
}

// Backward tile shapes.  Weight gradients from the staged rows: [dW_a | db_a] in 4 x 8
// blocks (channels c..c+3 x [f, 1]) by the first kTA threads, [dW_b | db_b] in 3 x 4 blocks
// (outputs x channels h..h+3 of [h_1, 1]) by the others, so that every warp runs one kind.
constexpr int kTA = 160;
template <int C>
struct Syn1x1Shape {
  static constexpr int T = kPixTile;
  static constexpr int SZ = C + 4;   // stride of dz1 and [h1, 1] rows
  static constexpr int SF = 12;      // stride of [f, 1] rows
  static constexpr int SD = 4;       // stride of [dz2, 0] rows
  static constexpr int NUA = C / 4;          // 4 x 8 blocks of [dW_a | db_a]
  static constexpr int NUB = (C + 4) / 4;    // 3 x 4 blocks of [dW_b | db_b]
  static constexpr int GA = kTA / NUA;       // pixel groups of the A blocks
  static constexpr int GB = (T - kTA) / NUB; // and of the B blocks
  static constexpr int GM = GA > GB ? GA : GB;
  static constexpr int NP = 11 * C + 3;
  static constexpr int tile_floats = T * (2 * SZ + SF + SD);
  static constexpr int halo_floats = 3 * kSHS;   // dz of 3x3 layer 0 over the tile + halo
  static constexpr int smem_floats =
      tile_floats + halo_floats > GM * NP ? tile_floats + halo_floats : GM * NP;
};

template <int C>
__global__ void __launch_bounds__(256, 2) k_syn1x1_bwd(Syn1x1Args a) {
  pdl_wait();
  pdl_trigger();
  using Sh = Syn1x1Shape<C>;
  using Wt = Syn1x1W<C>;
  constexpr int T = Sh::T, SZ = Sh::SZ, SF = Sh::SF, SD = Sh::SD, M = Wt::M;
  constexpr int NUA = Sh::NUA, NUB = Sh::NUB, GA = Sh::GA, GB = Sh::GB, NP = Sh::NP;
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  float* s_dz1 = sm;               // [T][SZ]
  float* s_h1 = s_dz1 + T * SZ;    // [T][SZ]  (h1, 1, 0, 0, 0)
  float* s_f = s_h1 + T * SZ;      // [T][SF]  (f0..f6, 1, 0...)
  float* s_dz2 = s_f + T * SF;     // [T][SD]  (dz2, 0)
  float* s_halo = s_dz2 + T * SD;  // 3 x kSHS

  const int tid = threadIdx.x;
  const bool is_a = tid < kTA;
  const int unit = is_a ? tid % NUA : (tid - kTA) % NUB;
  const int grp = is_a ? tid / NUA : (tid - kTA) / NUB;
  const bool worker = is_a ? grp < GA : grp < GB;
  // A blocks: acc[r][kk] = (dW[c0 + r][2kk], dW[c0 + r][2kk + 1]); B blocks use r < 3, kk < 2
  float2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[r][k] = make_float2(0.f, 0.f);

  const float2* wa = reinterpret_cast<const float2*>(c_syn + Wt::WAT);
  const float2* ba = reinterpret_cast<const float2*>(c_syn + Wt::BA);
  const float2* wb = reinterpret_cast<const float2*>(c_syn + Wt::WBR);
  const int tx = tid & 31, ty = tid >> 5;
  HaloPlan hp;
  hp.init(a.t.H, a.t.W);
  float nv[kHaloK];
  if (blockIdx.x < a.t.n_tiles) {
    int y0, x0;
    tile_xy(a.t, blockIdx.x, y0, x0);
    hp.load(nv, a.dz0, y0, x0);
  }
  for (int tile = blockIdx.x; tile < a.t.n_tiles; tile += gridDim.x) {
    int y0, x0;
    tile_xy(a.t, tile, y0, x0);
    hp.store(s_halo, nv);
    __syncthreads();
    if (tile + (int)gridDim.x < a.t.n_tiles) {
      int ny0, nx0;
      tile_xy(a.t, tile + gridDim.x, ny0, nx0);
      hp.load(nv, a.dz0, ny0, nx0);
    }
    const int y = y0 + ty, x = x0 + tx;
    const bool valid = y < a.t.H && x < a.t.W;
    const int p = valid ? y * a.t.W + x : 0;
    float f[kLevels];
#pragma unroll
    for (int k = 0; k < kLevels; ++k) f[k] = valid ? __ldg(a.feat[k] + p) : 0.f;
    // gradient of h2: output gradient of 3x3 layer 0 plus its input-gradient stencil
    float dh2[3] = {0.f, 0.f, 0.f};
    if (valid) {
#pragma unroll
      for (int j = 0; j < 3; ++j) dh2[j] = __ldg(a.dhout + j * a.HW + p);
      conv_adjoint<0>(dh2, s_halo, ty, tx, y, x, y0, x0, a.t.H, a.t.W);
    }
    // dz2 = [h2 > 0] dh2: the ReLU mask of the C-3 layer from the forward's stored output
    float dz2[3] = {0.f, 0.f, 0.f};
    if (valid) {
#pragma unroll
      for (int j = 0; j < 3; ++j) dz2[j] = __ldg(a.h2 + j * a.HW + p) > 0.f ? dh2[j] : 0.f;
    }
    *reinterpret_cast<float4*>(s_dz2 + tid * SD) = make_float4(dz2[0], dz2[1], dz2[2], 0.f);
    // One loop over the hidden channel pairs: recompute z1 and h1 = ReLU(z1), then
    // dh1 = W_b^T dz2, dz1 = [z1 > 0] dh1 and df += W_a^T dz1, each W_a pair loaded once for
    // both of its uses; h1 and dz1 go to the staged rows of the weight gradient.
    float2 fd[kLevels];
#pragma unroll
    for (int k = 0; k < kLevels; ++k) fd[k] = make_float2(f[k], f[k]);
    const float2 g0 = make_float2(dz2[0], dz2[0]), g1 = make_float2(dz2[1], dz2[1]),
                 g2 = make_float2(dz2[2], dz2[2]);
    float2 dfp[kLevels];
#pragma unroll
    for (int k = 0; k < kLevels; ++k) dfp[k] = make_float2(0.f, 0.f);
    float* hrow = s_h1 + tid * SZ;
    float* zrow = s_dz1 + tid * SZ;
#pragma unroll
    for (int m = 0; m < M; m += 2) {
      float2 hh[2], dd[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float2 w[kLevels];
#pragma unroll
        for (int k = 0; k < kLevels; ++k) w[k] = wa[k * M + m + u];
        float2 z = ba[m + u];
#pragma unroll
        for (int k = 0; k < kLevels; ++k) z = __ffma2_rn(w[k], fd[k], z);
        const float2 h = make_float2(fmaxf(z.x, 0.f), fmaxf(z.y, 0.f));
        float2 dh = __fmul2_rn(wb[m + u], g0);
        dh = __ffma2_rn(wb[M + m + u], g1, dh);
        dh = __ffma2_rn(wb[2 * M + m + u], g2, dh);
        const float2 dz = make_float2(h.x > 0.f ? dh.x : 0.f, h.y > 0.f ? dh.y : 0.f);
#pragma unroll
        for (int k = 0; k < kLevels; ++k) dfp[k] = __ffma2_rn(w[k], dz, dfp[k]);
        hh[u] = h;
        dd[u] = dz;
      }
      *reinterpret_cast<float4*>(hrow + 2 * m) =
          valid ? make_float4(hh[0].x, hh[0].y, hh[1].x, hh[1].y) : make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(zrow + 2 * m) = make_float4(dd[0].x, dd[0].y, dd[1].x, dd[1].y);
    }
    *reinterpret_cast<float4*>(hrow + C) = make_float4(valid ? 1.f : 0.f, 0.f, 0.f, 0.f);
    float* frow = s_f + tid * SF;
#pragma unroll
    for (int k = 0; k < kLevels; ++k) frow[k] = f[k];
    frow[7] = valid ? 1.f : 0.f;
    if (valid) {
#pragma unroll
      for (int k = 0; k < kLevels; ++k) a.dfeat[k][p] = dfp[k].x + dfp[k].y;
    }
    __syncthreads();
    if (worker) {
      if (is_a) {   // rows c = 4 unit .. +3 of [dW_a | db_a]
        const int c0 = unit * 4;
        for (int q = grp; q < T; q += GA) {
          const float4 dz = *reinterpret_cast<const float4*>(s_dz1 + q * SZ + c0);
          const float4 f0 = *reinterpret_cast<const float4*>(s_f + q * SF);
          const float4 f1 = *reinterpret_cast<const float4*>(s_f + q * SF + 4);
          const float dv[4] = {dz.x, dz.y, dz.z, dz.w};
          const float2 fp[4] = {make_float2(f0.x, f0.y), make_float2(f0.z, f0.w),
                                make_float2(f1.x, f1.y), make_float2(f1.z, f1.w)};
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 4; ++k)
              acc[r][k] = __ffma2_rn(make_float2(dv[r], dv[r]), fp[k], acc[r][k]);
        }
      } else {      // cols 4 unit .. +3 of [dW_b | db_b]
        const int h0 = unit * 4;
        for (int q = grp; q < T; q += GB) {
          const float4 dz = *reinterpret_cast<const float4*>(s_dz2 + q * SD);
          const float4 hv = *reinterpret_cast<const float4*>(s_h1 + q * SZ + h0);
          const float dv[3] = {dz.x, dz.y, dz.z};
          const float2 hp[2] = {make_float2(hv.x, hv.y), make_float2(hv.z, hv.w)};
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 2; ++k)
              acc[r][k] = __ffma2_rn(make_float2(dv[r], dv[r]), hp[k], acc[r][k]);
        }
      }
    }
    __syncthreads();
  }
  // partial layout: W_a (C x 7), b_a (C), W_b (3 x C), b_b (3); groups summed in order
  float* red = sm;
  if (worker) {
    float* mine = red + grp * NP;
    if (is_a) {
      const int c0 = unit * 4;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int k = 0; k < 7; ++k) mine[(c0 + r) * 7 + k] = (k & 1) ? acc[r][k >> 1].y : acc[r][k >> 1].x;
        mine[7 * C + c0 + r] = acc[r][3].y;
      }
    } else {
      const int h0 = unit * 4;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int col = h0 + k;
          const float v = (k & 1) ? acc[r][k >> 1].y : acc[r][k >> 1].x;
          if (col < C) mine[8 * C + r * C + col] = v;
          else if (col == C) mine[11 * C + r] = v;
        }
    }
  }
  __syncthreads();
  for (int j = tid; j < NP; j += T) {
    const int ng = j < 8 * C ? GA : GB;
    float t = 0.f;
    for (int g = 0; g < ng; ++g) t += red[g * NP + j];
    a.part[(long long)blockIdx.x * NP + j] = t;
  }
}

// ------------------------------------------------------------------ drivers

template <int C>
static cudaError_t syn1x1_fwd_t(const Syn1x1Args& a, cudaStream_t st) {
  return launch_k(k_syn1x1_fwd<C>, dim3((a.HW + 511) / 512), dim3(256), 0, st, a);
}

template <int C>
static cudaError_t syn1x1_bwd_t(const Syn1x1Args& a, int grid, cudaStream_t st) {
  const size_t smem = (size_t)Syn1x1Shape<C>::smem_floats * sizeof(float);
  return launch_k(k_syn1x1_bwd<C>, dim3(grid), dim3(kPixTile), smem, st, a);
}

template <int C>
static cudaError_t syn_prepare_t() {
  return cudaFuncSetAttribute(k_syn1x1_bwd<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(Syn1x1Shape<C>::smem_floats * sizeof(float)));
}

cudaError_t syn_prepare(const Arch& a) {
  switch (a.C) {
    case 8: return syn_prepare_t<8>();
    case 16: return syn_prepare_t<16>();
    case 40: return syn_prepare_t<40>();
    default: return cudaErrorInvalidValue;
  }
}

static Syn1x1Args make_1x1(const Geo& g, const float* yhat, const UpPlan& up) {
  Syn1x1Args s{};
  s.feat[0] = yhat + g.off[0];
  for (int l = 1; l < kLevels; ++l) s.feat[l] = up.plane[l][0];
  s.HW = g.H * g.W;
  return s;
}

int syn1x1_partial_cols(const Arch& a) { return 11 * a.C + 3; }

static SynTileGeo tile_geo(const Geo& g) {
  SynTileGeo t;
  t.H = g.H;
  t.W = g.W;
  t.ntx = (g.W + kSTX - 1) / kSTX;
  t.n_tiles = t.ntx * ((g.H + kSTY - 1) / kSTY);
  return t;
}

int syn_tile_count(const Geo& g) { return tile_geo(g).n_tiles; }

cudaError_t syn_forward(const Arch& ar, const Geo& g, const float* yhat, const UpPlan& up,
                        const float* x, float* hbuf, float* dxhat, float* part_d,
                        float* part_conv, int grid, cudaStream_t st, float* dh, float* dz) {
  const int HW = g.H * g.W;
  Syn1x1Args s = make_1x1(g, yhat, up);
  s.h2 = hbuf;
  cudaError_t e;
  switch (ar.C) {
    case 8: e = syn1x1_fwd_t<8>(s, st); break;
    case 16: e = syn1x1_fwd_t<16>(s, st); break;
    case 40: e = syn1x1_fwd_t<40>(s, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  ConvArgs c{};
  c.t = tile_geo(g);
  c.x = x;
  c.dxhat = dxhat;
  c.part_d = part_d;
  c.part = part_conv + (size_t)(ar.NR - 1) * grid * 84;
  c.dscale = 2.0f / (3.0f * (float)HW);
  c.hin = hbuf;
  c.hout = hbuf + (size_t)3 * HW;
  if (ar.NR == 1) return launch_k(k_conv3_last<0>, dim3(grid), dim3(256), 0, st, c);
  if (dh && dz) {
    c.hout = hbuf + (size_t)6 * HW;
    c.dh = dh;
    c.dz = dz;
    c.part = part_conv;
    return launch_k(k_conv3_pair, dim3(grid), dim3(256), 0, st, c);
  }
  if ((e = launch_k(k_conv3_fwd<0>, dim3(grid), dim3(256), 0, st, c)) != cudaSuccess) return e;
  c.hin = hbuf + (size_t)3 * HW;
  c.hout = hbuf + (size_t)6 * HW;
  return launch_k(k_conv3_last<1>, dim3(grid), dim3(256), 0, st, c);
}

// dhbuf holds NR + 1 gradient planes-of-3: dhbuf[NR] = dL/dx_hat (written by the forward).
cudaError_t syn_backward(const Arch& ar, const Geo& g, const float* yhat, const UpPlan& up,
                         float* hbuf, float* dhbuf, float* dz, float* gsyn, float* part_conv,
                         float* part_syn, int grid, cudaStream_t st, bool convs_done) {
  const int HW = g.H * g.W;
  const float* dxhat = dhbuf + (size_t)ar.NR * 3 * HW;
  Syn1x1Args s = make_1x1(g, yhat, up);
  s.t = tile_geo(g);
  if (ar.NR == 2) {
    ConvArgs c{};
    c.t = s.t;
    c.g = dxhat;
    c.hin = hbuf;
    c.dh = dhbuf + (size_t)3 * HW;
    c.dz = dz;
    c.part = part_conv;
    if (!convs_done) {
      cudaError_t e = launch_k(k_conv3_mid, dim3(grid), dim3(256), 0, st, c);
      if (e != cudaSuccess) return e;
    }
    s.dhout = c.dh;
    s.dz0 = dz;
  } else {
    // one linear layer: its output gradient is also its pre-activation gradient
    s.dhout = dxhat;
    s.dz0 = dxhat;
  }
  s.h2 = hbuf;
  s.dfeat[0] = gsyn + g.off[0];
  for (int l = 1; l < kLevels; ++l) s.dfeat[l] = up.dplane[l][0];
  s.part = part_syn;
  switch (ar.C) {
    case 8: return syn1x1_bwd_t<8>(s, grid, st);
    case 16: return syn1x1_bwd_t<16>(s, grid, st);
    case 40: return syn1x1_bwd_t<40>(s, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void k_planar_to_hwc(const float* __restrict__ xh, float* __restrict__ out, int HW) {
  pdl_wait();
  pdl_trigger();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) out[p * 3 + c] = xh[c * HW + p];
  }
}

cudaError_t syn_decode(const Arch& a, const Geo& g, const float* hbuf_last, float* out_hwc,
                       cudaStream_t st) {
  (void)a;
  const int HW = g.H * g.W;
  return launch_k(k_planar_to_hwc, dim3((HW + 255) / 256 < 2048 ? (HW + 255) / 256 : 2048),
                  dim3(256), 0, st, hbuf_last, out_hwc, HW);
}

// Bank image from the flat parameters (synthesis section: W_a, b_a, W_b, b_b, then the 3x3
// layers; upsampling filters).
__global__ void k_syn_image(const float* __restrict__ syn, int C, int NR,
                            const float* __restrict__ filters, int n_filt, SynBank* img) {
  pdl_wait();
  pdl_trigger();
  const int n3 = NR * k3x3;
  const float* p1 = syn;                   // W_a (C x 7), b_a, W_b (3 x C), b_b
  const float* p3 = syn + 11 * C + 3;      // 3x3 layers
  for (int i = threadIdx.x; i < kSynBank; i += blockDim.x) {
    float v = 0.f;
    if (i < n3) {
      v = p3[i];
    } else if (i >= kSyn1x1Base) {
      const int r = i - kSyn1x1Base;
      if (r < 7 * C) {
        v = p1[(r % C) * 7 + r / C];        // W_a^T
      } else if (r < 11 * C + 3) {
        v = p1[r];                          // b_a, W_b, b_b as in the parameters
      }
    }
    img->syn[i] = v;
    img->synb[i] = v;
  }
  for (int i = threadIdx.x; i < (kLevels - 1) * 64; i += blockDim.x)
    img->up[i] = i < n_filt ? filters[i] : 0.f;
}

size_t syn_image_bytes() { return sizeof(SynBank); }

cudaError_t syn_build_image(const float* d_params, const Layout& lay, const Arch& a,
                            void* d_image, cudaStream_t st) {
  k_syn_image<<<1, 256, 0, st>>>(d_params + lay.syn0, a.C, a.NR, d_params + lay.up0,
                                 lay.n_up * a.K * a.K, (SynBank*)d_image);
  return cudaGetLastError();
}

cudaError_t syn_copy_bank(const void* d_image, cudaStream_t st) {
  return cudaMemcpyToSymbolAsync(c_synbank, d_image, sizeof(SynBank), 0,
                                 cudaMemcpyDeviceToDevice, st);
}

cudaError_t syn_upload(const float* d_params, const Layout& lay, const Arch& a, void* d_image,
                       cudaStream_t st) {
  cudaError_t e = syn_build_image(d_params, lay, a, d_image, st);
  return e != cudaSuccess ? e : syn_copy_bank(d_image, st);
}

int syn_image_weight_floats() { return (int)(sizeof(SynBank) / sizeof(float)); }

}  // namespace cc
