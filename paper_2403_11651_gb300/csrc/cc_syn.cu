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
// [3x3 layer 0 | 3x3 layer 1 | W_a (C x 7) | b_a (C) | W_b^T (C x 4, 4th column 0) | b_b],
// W_b transposed so that the three weights of one hidden channel are adjacent.  `synb`
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
  float* part;                      // [gridDim.x][kLevels][K*K] of this step
};

// Adjoint of one step.  Thread per input position i: it gathers every output that read
// i, directly or through the clamp (virtual positions beyond the border fold onto the
// edge), giving dL/d in[i] = sum f[u] dout[o] and the filter gradient in[i] * dout[o].
// Inputs whose 8 x 8 output window lies inside the plane take a branch-free path.
template <int K>
__global__ void __launch_bounds__(128) k_up_bwd(UpBwdArgs a) {
  constexpr int c = K / 2 - 1;
  constexpr int KK = K * K;
  const int li = blockIdx.y;
  const float* __restrict__ dout = a.dout[li];
  const float* __restrict__ in = a.in[li];
  float* __restrict__ din = a.din[li];
  float f[KK];
  const int fb = a.fidx[li] * KK;
#pragma unroll
  for (int u = 0; u < KK; ++u) f[u] = c_up[fb + u];
  float facc[KK];
#pragma unroll
  for (int u = 0; u < KK; ++u) facc[u] = 0.f;
  const int n = a.sh * a.sw;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int iy = p / a.sw, ix = p - iy * a.sw;
    const float xin = __ldg(in + p);
    // virtual input positions folding onto (iy, ix) through the clamp: just (iy, ix)
    // inside the plane, up to K/4 more beyond an edge
    const int vy0 = iy == 0 ? -(K / 4) : iy;
    const int vy1 = iy == a.sh - 1 ? (a.dh - 1 + c) >> 1 : iy;
    const int vx0 = ix == 0 ? -(K / 4) : ix;
    const int vx1 = ix == a.sw - 1 ? (a.dw - 1 + c) >> 1 : ix;
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    for (int vy = vy0; vy <= vy1; ++vy) {
      int roff[K];
      uint32_t rok = 0;
#pragma unroll
      for (int uy = 0; uy < K; ++uy) {
        const int oy = 2 * vy - c + uy;
        rok |= (oy >= 0 && oy < a.dh ? 1u : 0u) << uy;
        roff[uy] = clampi(oy, 0, a.dh - 1) * a.dw;
      }
      for (int vx = vx0; vx <= vx1; ++vx) {
        int col[K];
        uint32_t cok = 0;
#pragma unroll
        for (int ux = 0; ux < K; ++ux) {
          const int ox = 2 * vx - c + ux;
          cok |= (ox >= 0 && ox < a.dw ? 1u : 0u) << ux;
          col[ux] = clampi(ox, 0, a.dw - 1);
        }
        // every read is inside the plane; reads of outputs beyond it count as zero
#pragma unroll
        for (int uy = 0; uy < K; ++uy) {
          const float* row = dout + roff[uy];
          const bool ry = (rok >> uy) & 1u;
#pragma unroll
          for (int ux = 0; ux < K; ++ux) {
            float gv = __ldg(row + col[ux]);
            gv = (ry && ((cok >> ux) & 1u)) ? gv : 0.f;
            g[ux & 3] = fmaf(f[uy * K + ux], gv, g[ux & 3]);
            facc[uy * K + ux] = fmaf(xin, gv, facc[uy * K + ux]);
          }
        }
      }
    }
    din[p] = (g[0] + g[1]) + (g[2] + g[3]);
  }
  // per-CTA filter gradient: warp sums, then warps in order
  __shared__ float s_w[4][KK];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < KK; ++u) {
    float v = facc[u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[wid][u] = v;
  }
  __syncthreads();
  for (int u = threadIdx.x; u < KK; u += blockDim.x) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w][u];
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
    k_up_fwd<K><<<dim3(need < cap ? need : cap, n), 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
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
    // rows [j * grid, j * grid + grid) belong to this step; only as many CTAs as there is
    // work for are launched, the rows of the others stay zero from the context set-up
    a.part = part_up + (long long)j * grid * kLevels * K * K;
    // 128-thread CTAs, about two resident per SM in total (grid = 2 x SMs): each thread
    // loads its filter once and handles many inputs before the per-CTA reduction
    const int need = (a.sh * a.sw + 127) / 128, cap = grid / n > 1 ? grid / n : 1;
    k_up_bwd<K><<<dim3(need < cap ? need : cap, n), 128, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
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

// ------------------------------------------------------------------ synthesis 1x1 layers

struct Syn1x1Args {
  const float* feat[kLevels];   // level-0 latents, then the upsampled planes of l = 1..6
  const float* dh2;             // [3][HW] gradient of the C-3 layer output
  float* h2;                    // [3][HW]
  float* dfeat[kLevels];        // gradient of each feature plane
  float* part;                  // [gridDim.x][11C + 3]
  int HW;
};

template <int C>
__global__ void __launch_bounds__(256) k_syn1x1_fwd(Syn1x1Args a) {
  constexpr int WA = kSyn1x1Base, BA = WA + 7 * C, WB = BA + C, BB = WB + 4 * C;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.HW; p += gridDim.x * blockDim.x) {
    float f[kLevels];
#pragma unroll
    for (int k = 0; k < kLevels; ++k) f[k] = __ldg(a.feat[k] + p);
    float z2[3] = {c_syn[BB], c_syn[BB + 1], c_syn[BB + 2]};
#pragma unroll
    for (int o = 0; o < C; ++o) {
      float z = c_syn[BA + o];
#pragma unroll
      for (int k = 0; k < kLevels; ++k) z = fmaf(c_syn[WA + o * kLevels + k], f[k], z);
      const float h1 = fmaxf(z, 0.f);
#pragma unroll
      for (int j = 0; j < 3; ++j) z2[j] = fmaf(c_syn[WB + o * 4 + j], h1, z2[j]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) a.h2[j * a.HW + p] = fmaxf(z2[j], 0.f);
  }
}

template <int C>
struct Syn1x1Shape {
  static constexpr int T = kPixTile;
  static constexpr int SZ = C + 4;   // stride of dz1 and [h1, 1] rows
  static constexpr int SF = 12;      // stride of [f, 1] rows
  static constexpr int SD = 4;       // stride of [dz2, 0] rows
  static constexpr int NUA = C / 4;          // 4x8 blocks of [dW_a | db_a]
  static constexpr int NUB = (C + 4) / 4;    // 4x4 blocks of [dW_b | db_b] (row 3 unused)
  static constexpr int NU = NUA + NUB;
  static constexpr int G = T / NU;
  static constexpr int NP = 11 * C + 3;
  static constexpr int tile_floats = T * (2 * SZ + SF + SD);
  static constexpr int smem_floats = tile_floats > G * NP ? tile_floats : G * NP;
};

template <int C>
__global__ void __launch_bounds__(256, 2) k_syn1x1_bwd(Syn1x1Args a) {
  using Sh = Syn1x1Shape<C>;
  constexpr int T = Sh::T, SZ = Sh::SZ, SF = Sh::SF, SD = Sh::SD;
  constexpr int NUA = Sh::NUA, NU = Sh::NU, G = Sh::G, NP = Sh::NP;
  constexpr int WA = kSyn1x1Base, BA = WA + 7 * C, WB = BA + C, BB = WB + 4 * C;
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  float* s_dz1 = sm;               // [T][SZ]
  float* s_h1 = s_dz1 + T * SZ;    // [T][SZ]  (h1, 1, 0, 0, 0)
  float* s_f = s_h1 + T * SZ;      // [T][SF]  (f0..f6, 1, 0...)
  float* s_dz2 = s_f + T * SF;     // [T][SD]  (dz2, 0)

  const int tid = threadIdx.x;
  const bool worker = tid < G * NU;
  const int unit = tid % NU, grp = tid / NU;
  float acc[4][8];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[r][k] = 0.f;

  const int n_tiles = (a.HW + T - 1) / T;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int p = tile * T + tid;
    const bool valid = p < a.HW;
    float f[kLevels];
#pragma unroll
    for (int k = 0; k < kLevels; ++k) f[k] = valid ? __ldg(a.feat[k] + p) : 0.f;
    float dh2[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) dh2[j] = valid ? __ldg(a.dh2 + j * a.HW + p) : 0.f;
    // recompute z1, h1, z2
    float z2[3] = {c_syn[BB], c_syn[BB + 1], c_syn[BB + 2]};
    float h1[C];
#pragma unroll
    for (int o = 0; o < C; ++o) {
      float z = c_syn[BA + o];
#pragma unroll
      for (int k = 0; k < kLevels; ++k) z = fmaf(c_syn[WA + o * kLevels + k], f[k], z);
      h1[o] = fmaxf(z, 0.f);
#pragma unroll
      for (int j = 0; j < 3; ++j) z2[j] = fmaf(c_syn[WB + o * 4 + j], h1[o], z2[j]);
    }
    float* hrow = s_h1 + tid * SZ;
#pragma unroll
    for (int o = 0; o < C; o += 4)
      *reinterpret_cast<float4*>(hrow + o) = valid ? make_float4(h1[o], h1[o + 1], h1[o + 2], h1[o + 3])
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(hrow + C) = make_float4(valid ? 1.f : 0.f, 0.f, 0.f, 0.f);
    float dz2[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) dz2[j] = z2[j] > 0.f ? dh2[j] : 0.f;
    *reinterpret_cast<float4*>(s_dz2 + tid * SD) = make_float4(dz2[0], dz2[1], dz2[2], 0.f);
    float df[kLevels];
#pragma unroll
    for (int k = 0; k < kLevels; ++k) df[k] = 0.f;
#pragma unroll
    for (int o = 0; o < C; ++o) {
      float dh1 = 0.f;
#pragma unroll
      for (int j = 0; j < 3; ++j) dh1 = fmaf(c_synb[WB + o * 4 + j], dz2[j], dh1);
      h1[o] = h1[o] > 0.f ? dh1 : 0.f;    // now dz1 (relu'(z1) = [h1 > 0])
#pragma unroll
      for (int k = 0; k < kLevels; ++k) df[k] = fmaf(c_synb[WA + o * kLevels + k], h1[o], df[k]);
    }
    float* zrow = s_dz1 + tid * SZ;
#pragma unroll
    for (int o = 0; o < C; o += 4)
      *reinterpret_cast<float4*>(zrow + o) = make_float4(h1[o], h1[o + 1], h1[o + 2], h1[o + 3]);
    float* frow = s_f + tid * SF;
#pragma unroll
    for (int k = 0; k < kLevels; ++k) frow[k] = f[k];
    frow[7] = valid ? 1.f : 0.f;
    if (valid) {
#pragma unroll
      for (int k = 0; k < kLevels; ++k) a.dfeat[k][p] = df[k];
    }
    __syncthreads();
    if (worker) {
      if (unit < NUA) {   // rows c = 4 unit .. +3 of [dW_a | db_a]
        const int c0 = unit * 4;
        for (int q = grp; q < T; q += G) {
          const float4 dz = *reinterpret_cast<const float4*>(s_dz1 + q * SZ + c0);
          const float4 f0 = *reinterpret_cast<const float4*>(s_f + q * SF);
          const float4 f1 = *reinterpret_cast<const float4*>(s_f + q * SF + 4);
          const float dv[4] = {dz.x, dz.y, dz.z, dz.w};
          const float fv[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[r][k] = fmaf(dv[r], fv[k], acc[r][k]);
        }
      } else {            // cols 4 (unit - NUA) .. +3 of [dW_b | db_b]
        const int h0 = (unit - NUA) * 4;
        for (int q = grp; q < T; q += G) {
          const float4 dz = *reinterpret_cast<const float4*>(s_dz2 + q * SD);
          const float4 hv = *reinterpret_cast<const float4*>(s_h1 + q * SZ + h0);
          const float dv[4] = {dz.x, dz.y, dz.z, dz.w};
          const float hh[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[r][k] = fmaf(dv[r], hh[k], acc[r][k]);
        }
      }
    }
    __syncthreads();
  }
  // partial layout: W_a (C x 7), b_a (C), W_b (3 x C), b_b (3)
  float* red = sm;
  if (worker) {
    float* mine = red + grp * NP;
    if (unit < NUA) {
      const int c0 = unit * 4;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int k = 0; k < 7; ++k) mine[(c0 + r) * 7 + k] = acc[r][k];
        mine[7 * C + c0 + r] = acc[r][7];
      }
    } else {
      const int h0 = (unit - NUA) * 4;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int col = h0 + k;
          if (col < C) mine[8 * C + r * C + col] = acc[r][k];
          else if (col == C) mine[11 * C + r] = acc[r][k];
        }
    }
  }
  __syncthreads();
  for (int j = tid; j < NP; j += T) {
    float t = 0.f;
    for (int g = 0; g < G; ++g) t += red[g * NP + j];
    a.part[(long long)blockIdx.x * NP + j] = t;
  }
}

// ------------------------------------------------------------------ 3x3 residual layers

struct ConvArgs {
  const float* hin;    // [3][HW] layer input
  float* hout;         // [3][HW] layer output (forward)
  const float* dhout;  // [3][HW] gradient of the layer output (backward)
  float* dz;           // [3][HW] gradient of the pre-activation
  float* dhin;         // [3][HW] gradient of the layer input
  const float* x;      // [3][HW] image (last layer)
  float* part;         // per-CTA partials
  float dscale;        // 2 / (3 H W)
  int H, W;
};

__device__ __forceinline__ void gather3x3(float (&v)[27], const float* h, int y, int x, int H,
                                          int W) {
  const int HW = H * W;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    const int yy = clampi(y + dy, 0, H - 1);
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int xx = clampi(x + dx, 0, W - 1);
#pragma unroll
      for (int ci = 0; ci < 3; ++ci)
        v[ci * 9 + (dy + 1) * 3 + (dx + 1)] = __ldg(h + ci * HW + yy * W + xx);
    }
  }
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

template <int I, bool LAST>
__global__ void __launch_bounds__(256) k_conv_fwd(ConvArgs a) {
  const int HW = a.H * a.W;
  float dsum = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    const int y = p / a.W, x = p - y * a.W;
    float v[27];
    gather3x3(v, a.hin, y, x, a.H, a.W);
    float z[3];
    conv_z<I>(z, v);
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float out = v[o * 9 + 4] + (LAST ? z[o] : fmaxf(z[o], 0.f));
      a.hout[o * HW + p] = out;
      if (LAST) {
        const float d = out - __ldg(a.x + o * HW + p);
        dsum = fmaf(d, d, dsum);
        a.dz[o * HW + p] = d * a.dscale;   // dL/dx_hat, stored as the gradient buffer
      }
    }
  }
  if (LAST) {
    __shared__ float s_tmp[8];
    const float t = block_sum<256>(dsum, s_tmp);
    if (threadIdx.x == 0) a.part[blockIdx.x] = t;
  }
}

// dz = dL/dh_out * act'(z) and the layer's weight / bias gradient partials.
template <int I, bool LAST>
__global__ void __launch_bounds__(256) k_conv_dz(ConvArgs a) {
  const int HW = a.H * a.W;
  float acc[84];
#pragma unroll
  for (int k = 0; k < 84; ++k) acc[k] = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    const int y = p / a.W, x = p - y * a.W;
    float v[27];
    gather3x3(v, a.hin, y, x, a.H, a.W);
    float z[3];
    if (!LAST) conv_z<I>(z, v);
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float g = __ldg(a.dhout + o * HW + p);
      const float d = (LAST || z[o] > 0.f) ? g : 0.f;
      a.dz[o * HW + p] = d;
#pragma unroll
      for (int k = 0; k < 27; ++k) acc[o * 27 + k] = fmaf(d, v[k], acc[o * 27 + k]);
      acc[81 + o] += d;
    }
  }
  __shared__ float s_w[8][84];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 84; ++k) {
    float v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[wid][k] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 84; k += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += s_w[w][k];
    a.part[(long long)blockIdx.x * 84 + k] = t;
  }
}

// dL/dh_in = dL/dh_out + conv^T(dz): gathers, for each input pixel q, every (p, tap)
// whose replicate-clamped read landed on q.
template <int I>
__global__ void __launch_bounds__(256) k_conv_dx(ConvArgs a) {
  constexpr int Wo = I * k3x3;
  const int HW = a.H * a.W;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < HW; q += gridDim.x * blockDim.x) {
    const int qy = q / a.W, qx = q - qy * a.W;
    float acc[3];
#pragma unroll
    for (int ci = 0; ci < 3; ++ci) acc[ci] = __ldg(a.dhout + ci * HW + q);
    if (qy > 0 && qx > 0 && qy < a.H - 1 && qx < a.W - 1) {
      // interior: output p = q - (dy, dx) read q through tap (dy, dx), no clamping
      float d[27];
#pragma unroll
      for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx)
            d[o * 9 + (dy + 1) * 3 + (dx + 1)] = __ldg(a.dz + o * HW + q - dy * a.W - dx);
      // input channel outer: the nine taps of one (o, ci) pair are adjacent in the bank
#pragma unroll
      for (int ci = 0; ci < 3; ++ci)
#pragma unroll
        for (int o = 0; o < 3; ++o)
#pragma unroll
          for (int t = 0; t < 9; ++t)
            acc[ci] = fmaf(c_syn[Wo + o * 27 + ci * 9 + t], d[o * 9 + t], acc[ci]);
#pragma unroll
      for (int ci = 0; ci < 3; ++ci) a.dhin[ci * HW + q] = acc[ci];
      continue;
    }
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      for (int py = qy - dy - 1; py <= qy - dy + 1; ++py) {
        if (py < 0 || py >= a.H || clampi(py + dy, 0, a.H - 1) != qy) continue;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          for (int px = qx - dx - 1; px <= qx - dx + 1; ++px) {
            if (px < 0 || px >= a.W || clampi(px + dx, 0, a.W - 1) != qx) continue;
            const int pp = py * a.W + px;
#pragma unroll
            for (int o = 0; o < 3; ++o) {
              const float d = __ldg(a.dz + o * HW + pp);
#pragma unroll
              for (int ci = 0; ci < 3; ++ci)
                acc[ci] = fmaf(c_syn[Wo + o * 27 + ci * 9 + (dy + 1) * 3 + (dx + 1)], d, acc[ci]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int ci = 0; ci < 3; ++ci) a.dhin[ci * HW + q] = acc[ci];
  }
}

// ------------------------------------------------------------------ drivers

template <int C>
static cudaError_t syn1x1_fwd_t(const Syn1x1Args& a, int grid, cudaStream_t st) {
  k_syn1x1_fwd<C><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <int C>
static cudaError_t syn1x1_bwd_t(const Syn1x1Args& a, int grid, cudaStream_t st) {
  const size_t smem = (size_t)Syn1x1Shape<C>::smem_floats * sizeof(float);
  k_syn1x1_bwd<C><<<grid, kPixTile, smem, st>>>(a);
  return cudaGetLastError();
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

cudaError_t syn_forward(const Arch& ar, const Geo& g, const float* yhat, const UpPlan& up,
                        const float* x, float* hbuf, float* dxhat, float* part_d, int grid,
                        cudaStream_t st) {
  const int HW = g.H * g.W;
  Syn1x1Args s = make_1x1(g, yhat, up);
  s.h2 = hbuf;
  cudaError_t e;
  switch (ar.C) {
    case 8: e = syn1x1_fwd_t<8>(s, grid, st); break;
    case 16: e = syn1x1_fwd_t<16>(s, grid, st); break;
    case 40: e = syn1x1_fwd_t<40>(s, grid, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  for (int i = 0; i < ar.NR; ++i) {
    ConvArgs c{};
    c.hin = hbuf + (size_t)i * 3 * HW;
    c.hout = hbuf + (size_t)(i + 1) * 3 * HW;
    c.x = x; c.dz = dxhat; c.part = part_d;
    c.dscale = 2.0f / (3.0f * (float)HW);
    c.H = g.H; c.W = g.W;
    const bool last = i == ar.NR - 1;
    if (i == 0 && last) k_conv_fwd<0, true><<<grid, 256, 0, st>>>(c);
    else if (i == 0) k_conv_fwd<0, false><<<grid, 256, 0, st>>>(c);
    else k_conv_fwd<1, true><<<grid, 256, 0, st>>>(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// dhbuf holds NR + 1 gradient planes-of-3: dhbuf[NR] = dL/dx_hat (written by the forward).
cudaError_t syn_backward(const Arch& ar, const Geo& g, const float* yhat, const UpPlan& up,
                         float* hbuf, float* dhbuf, float* dz, float* gsyn, float* part_conv,
                         float* part_syn, int grid, cudaStream_t st) {
  const int HW = g.H * g.W;
  cudaError_t e;
  for (int i = ar.NR - 1; i >= 0; --i) {
    ConvArgs c{};
    c.hin = hbuf + (size_t)i * 3 * HW;
    c.dhout = dhbuf + (size_t)(i + 1) * 3 * HW;
    c.dz = dz;
    c.dhin = dhbuf + (size_t)i * 3 * HW;
    c.part = part_conv + (size_t)i * grid * 84;
    c.H = g.H; c.W = g.W;
    const bool last = i == ar.NR - 1;
    if (i == 0 && last) k_conv_dz<0, true><<<grid, 256, 0, st>>>(c);
    else if (i == 0) k_conv_dz<0, false><<<grid, 256, 0, st>>>(c);
    else k_conv_dz<1, true><<<grid, 256, 0, st>>>(c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (i == 0) k_conv_dx<0><<<grid, 256, 0, st>>>(c);
    else k_conv_dx<1><<<grid, 256, 0, st>>>(c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  Syn1x1Args s = make_1x1(g, yhat, up);
  s.dh2 = dhbuf;
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
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) out[p * 3 + c] = xh[c * HW + p];
  }
}

cudaError_t syn_decode(const Arch& a, const Geo& g, const float* hbuf_last, float* out_hwc,
                       cudaStream_t st) {
  (void)a;
  const int HW = g.H * g.W;
  k_planar_to_hwc<<<(HW + 255) / 256 < 2048 ? (HW + 255) / 256 : 2048, 256, 0, st>>>(
      hbuf_last, out_hwc, HW);
  return cudaGetLastError();
}

// Bank image from the flat parameters (synthesis section: W_a, b_a, W_b, b_b, then the 3x3
// layers; upsampling filters).
__global__ void k_syn_image(const float* __restrict__ syn, int C, int NR,
                            const float* __restrict__ filters, int n_filt, SynBank* img) {
  const int n3 = NR * k3x3;
  const float* p1 = syn;                   // W_a (C x 7), b_a, W_b (3 x C), b_b
  const float* p3 = syn + 11 * C + 3;      // 3x3 layers
  for (int i = threadIdx.x; i < kSynBank; i += blockDim.x) {
    float v = 0.f;
    if (i < n3) {
      v = p3[i];
    } else if (i >= kSyn1x1Base) {
      const int r = i - kSyn1x1Base;
      if (r < 8 * C) {
        v = p1[r];                          // W_a, b_a
      } else if (r < 12 * C) {
        const int o = (r - 8 * C) >> 2, j = (r - 8 * C) & 3;
        v = j < 3 ? p1[8 * C + j * C + o] : 0.f;   // W_b^T
      } else if (r < 12 * C + 3) {
        v = p1[11 * C + (r - 12 * C)];      // b_b
      }
    }
    img->syn[i] = v;
    img->synb[i] = v;
  }
  for (int i = threadIdx.x; i < (kLevels - 1) * 64; i += blockDim.x)
    img->up[i] = i < n_filt ? filters[i] : 0.f;
}

size_t syn_image_bytes() { return sizeof(SynBank); }

cudaError_t syn_upload(const float* d_params, const Layout& lay, const Arch& a, void* d_image,
                       cudaStream_t st) {
  k_syn_image<<<1, 256, 0, st>>>(d_params + lay.syn0, a.C, a.NR, d_params + lay.up0,
                                 lay.n_up * a.K * a.K, (SynBank*)d_image);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbolAsync(c_synbank, d_image, sizeof(SynBank), 0,
                                 cudaMemcpyDeviceToDevice, st);
}

}  // namespace cc
