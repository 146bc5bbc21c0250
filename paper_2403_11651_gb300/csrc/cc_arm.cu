// Auto-regressive probability model p_psi and the rate term of eq. (1).
//
// Sec. II "Decoding" item ii: the ARM is an MLP f_psi of the N causal neighbours of a
// latent in its own grid; Table 1 gives its layers (N-N-LinR x arm_layers, N-2-Lin).  Its
// two outputs are the mean mu and log-scale s of a Laplace law, and the rate of a latent
// is -log2 P(y_hat) with P the mass of [y_hat - 1/2, y_hat + 1/2] (eq. (1)).
//
// One thread owns one latent.  The weights live in a __constant__ bank refreshed before
// every pass, so every multiply-add of the forward and input-gradient passes takes its
// weight straight from the constant cache (all lanes read the same weight at once).  The
// weight gradients, sum over latents of dz (x) input, are contracted per tile of 128
// latents from shared memory: each thread owns an RB x RB block of one weight matrix
// for one interleaved quarter of the tile's latents and keeps it in registers for the
// whole persistent loop, so a CTA writes one partial sum per parameter at the end.
// Every sum has a fixed order, so results are bit-reproducible on a given device.
#include "cc_internal.cuh"
#include "cc_laplace.cuh"

namespace cc {

constexpr int kMaxN = 24;
constexpr int kMaxArmParams = 2 * (kMaxN * kMaxN + kMaxN) + 2 * kMaxN + 2;
// Constant bank of the ARM kernels, filled by one device-to-device copy of an image built
// on the device before every pass.  `wb` is a second copy of the weights read by the
// backward pass only: with a single copy the compiler keeps every weight used by both
// passes in a register between its two uses.
constexpr int kArmBankFloats = (kMaxArmParams + 3) & ~3;   // 16-byte aligned copies
struct __align__(16) ArmBank {
  float w[kArmBankFloats];
  float wb[kArmBankFloats];
  int2 off[kMaxN];  // (dy, dx) of each context slot, raster order
};
__constant__ ArmBank c_armbank;
#define c_arm c_armbank.w
#define c_armb c_armbank.wb
#define c_off c_armbank.off

struct ArmArgs {
  const float* yhat;   // zero-bordered copy (Geo::poff, Geo::pw)
  float* dctx;       // [N][n_pad]: d bits(p) / d context slot k of p
  float* gself;      // [n_pad]:    d bits(p) / d yhat(p)
  float* part_grad;  // [gridDim.x][n_arm]: per-CTA d bits / d psi
  float* part_bits;  // [gridDim.x]
  const int2* tiles; // (level, first latent of the tile within the level)
  int n_tiles;
  Geo g;
};

template <int N>
struct ArmBlocking {
  static constexpr int RB = (N % 6 == 0) ? 6 : 4;  // weight-gradient block edge
  static constexpr int NB = N / RB;                // blocks per matrix edge
};

template <int RB>
__device__ __forceinline__ void load_row(float (&v)[RB], const float* p) {
  if constexpr (RB % 4 == 0) {
#pragma unroll
    for (int k = 0; k < RB; k += 4) {
      const float4 t = *reinterpret_cast<const float4*>(p + k);
      v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < RB; k += 2) {
      const float2 t = *reinterpret_cast<const float2*>(p + k);
      v[k] = t.x; v[k + 1] = t.y;
    }
  }
}

template <int N>
__device__ __forceinline__ void store_row(float* p, const float (&v)[N]) {
#pragma unroll
  for (int k = 0; k < N; k += 4)
    *reinterpret_cast<float4*>(p + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
}

template <int N, int NL, int LPT>
struct ArmShape {
  static constexpr int S = N + 4;               // smem row stride (conflict-free float4 rows)
  static constexpr int LW = N * N + N;          // floats per LinR layer (W then b)
  static constexpr int OW = NL * LW;            // W_out
  static constexpr int OB = OW + 2 * N;         // b_out
  static constexpr int NP = OB + 2;             // ARM parameters
  static constexpr int T = kArmTile;            // latents per tile
  static constexpr int TT = kArmTile / LPT;     // threads per CTA
  // per-layer arrays are LS floats apart: T*S plus an 8-float skew, so that the same row
  // of two layers falls in different shared-memory banks
  static constexpr int LS = T * S + 8;
  static constexpr int tile_floats = 2 * NL * LS + T * S + 2 * T;
  static constexpr int NBLK = NL * ArmBlocking<N>::NB * ArmBlocking<N>::NB;
  static constexpr int G = TT / NBLK;           // interleaved latent groups
  static constexpr int NCH_B = NL * N / 4;      // bias chunks of 4
  static constexpr int NCH = NCH_B + N / 4;     // + W_out column chunks (b_out rides on #0)
  static constexpr int XPER = (NCH + NBLK - 1) / NBLK;
  static constexpr int red_floats = G * NP;
  static constexpr int smem_floats = tile_floats > red_floats ? tile_floats : red_floats;
  static_assert(TT % NBLK == 0 && G >= 1, "threads must split evenly into weight blocks");
};

// LPT latents per thread: thread t owns latents t, t + TT, ... of the tile, so each weight
// operand taken from the constant bank feeds LPT multiply-adds.
// CTAs per SM of the ARM kernels (one tile of kArmTile latents per CTA): one CTA of 12
// warps for the wider ARMs keeps every warp of an SM in the same phase of the tile, so
// they share the instruction stream of the fully unrolled layer code.
template <int N>
struct ArmOcc {
  static constexpr int blocks = N >= 16 ? 1 : 2;
};

template <int N, int NL, bool BWD, int LPT>
__global__ void __launch_bounds__(kArmTile / LPT, ArmOcc<N>::blocks) k_arm(ArmArgs a) {
  pdl_wait();
  pdl_trigger();
  using Sh = ArmShape<N, NL, LPT>;
  constexpr int S = Sh::S, LW = Sh::LW, OW = Sh::OW, OB = Sh::OB, NP = Sh::NP, T = Sh::T;
  constexpr int LS = Sh::LS, TT = Sh::TT;
  constexpr int RB = ArmBlocking<N>::RB, NB = ArmBlocking<N>::NB;
  constexpr int NBLK = Sh::NBLK, G = Sh::G, NCH_B = Sh::NCH_B, NCH = Sh::NCH;
  constexpr int XPER = Sh::XPER;

  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  float* s_in = sm;                    // [NL][T][S] input of LinR layer L (layer stride LS)
  float* s_dz = s_in + NL * LS;        // [NL][T][S] dz of LinR layer L (layer stride LS)
  float* s_ho = s_dz + NL * LS;        // [T][S]     input of the output layer
  float* s_do = s_ho + T * S;          // [T][2]     (d bits/d mu, d bits/d s)

  const int tid = threadIdx.x;
  const int unit = tid % NBLK, grp = tid / NBLK;
  const int uL = unit / (NB * NB), urb = (unit / NB) % NB, ucb = unit % NB;

  // weight-gradient block as packed pairs along its columns
  float2 acc[RB][RB / 2];
  float xacc[XPER][10];
  if constexpr (BWD) {
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < RB / 2; ++c) acc[r][c] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < XPER; ++q)
#pragma unroll
      for (int e = 0; e < 10; ++e) xacc[q][e] = 0.f;
  }
  float bits_acc = 0.f;

  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int2 td = a.tiles[tile];
    const int l = td.x;
    const int w = a.g.w[l];
    const int n_l = a.g.h[l] * w;
    const int pw = a.g.pw[l];
    // zero-bordered plane: every causal neighbour is inside the allocation, outside the
    // grid it reads the zero border
    bool valid[LPT];
    float h[LPT][N], yq[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
      const int i = td.y + tid + q * TT;
      valid[q] = i < n_l;
      int r = 0, c = 0;
      if (valid[q]) { r = i / w; c = i - r * w; }
      const float* ctr = a.yhat + a.g.poff[l] + (long long)(r + kCtxPad) * pw + c + kCtxPad;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int2 o = c_off[k];
        h[q][k] = valid[q] ? __ldg(ctr + o.x * pw + o.y) : 0.f;
      }
      yq[q] = valid[q] ? __ldg(ctr) : 0.f;
    }

    // forward: h <- h + relu(W h + b), NL times
    uint32_t mask[LPT][NL];
#pragma unroll
    for (int L = 0; L < NL; ++L) {
      if constexpr (BWD) {
#pragma unroll
        for (int q = 0; q < LPT; ++q) store_row<N>(s_in + L * LS + (tid + q * TT) * S, h[q]);
      }
      // packed FP32 pairs: (z[2m], z[2m+1]) += (W[2m][k], W[2m+1][k]) * (h[k], h[k]); the
      // forward bank stores every layer's weights in those pairs, input k innermost, so
      // consecutive multiply-adds use adjacent weights
      float2 zp[LPT][N / 2];
      {
        float2 hd[LPT][N];
#pragma unroll
        for (int q = 0; q < LPT; ++q)
#pragma unroll
          for (int k = 0; k < N; ++k) hd[q][k] = make_float2(h[q][k], h[q][k]);
        const float2* wp = reinterpret_cast<const float2*>(c_arm + L * LW);
#pragma unroll
        for (int m = 0; m < N / 2; ++m)
#pragma unroll
          for (int q = 0; q < LPT; ++q) zp[q][m] = wp[N * N / 2 + m];   // bias pair
#pragma unroll
        for (int m = 0; m < N / 2; ++m)
#pragma unroll
          for (int k = 0; k < N; ++k)
#pragma unroll
            for (int q = 0; q < LPT; ++q) zp[q][m] = __ffma2_rn(wp[m * N + k], hd[q][k], zp[q][m]);
      }
      float z[LPT][N];
#pragma unroll
      for (int q = 0; q < LPT; ++q)
#pragma unroll
        for (int m = 0; m < N / 2; ++m) { z[q][2 * m] = zp[q][m].x; z[q][2 * m + 1] = zp[q][m].y; }
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        uint32_t mk = 0;
#pragma unroll
        for (int o = 0; o < N; ++o) {
          mk |= (z[q][o] > 0.f ? 1u : 0u) << o;
          h[q][o] += fmaxf(z[q][o], 0.f);
        }
        mask[q][L] = mk;
      }
    }
    LapOut lo[LPT];
    {
      float mu[LPT], s[LPT];
      // (mu, s) as one packed pair; the forward bank stores W_out as (W_out[0][k], W_out[1][k])
      const float2* wo = reinterpret_cast<const float2*>(c_arm + OW);
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        if constexpr (BWD) store_row<N>(s_ho + (tid + q * TT) * S, h[q]);
        float2 ms = make_float2(c_arm[OB], c_arm[OB + 1]);
#pragma unroll
        for (int k = 0; k < N; ++k) ms = __ffma2_rn(wo[k], make_float2(h[q][k], h[q][k]), ms);
        mu[q] = ms.x;
        s[q] = ms.y;
      }
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        lo[q] = laplace_bits(yq[q], mu[q], s[q]);
        if (!valid[q]) lo[q].bits = lo[q].g_y = lo[q].g_mu = lo[q].g_s = 0.f;
        bits_acc += lo[q].bits;
      }
    }

    if constexpr (BWD) {
      // packed pairs over inputs: (dh[k], dh[k+1]) += (W[o][k], W[o][k+1]) * (dz[o], dz[o]),
      // read from the row-major copy of the weights (adjacent along k)
      float2 dhp[LPT][N / 2];
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        reinterpret_cast<float2*>(s_do)[tid + q * TT] = make_float2(lo[q].g_mu, lo[q].g_s);
        const float2* w0 = reinterpret_cast<const float2*>(c_armb + OW);
        const float2* w1 = reinterpret_cast<const float2*>(c_armb + OW + N);
        const float2 gm = make_float2(lo[q].g_mu, lo[q].g_mu), gs = make_float2(lo[q].g_s, lo[q].g_s);
#pragma unroll
        for (int j = 0; j < N / 2; ++j) dhp[q][j] = __ffma2_rn(w0[j], gm, __fmul2_rn(w1[j], gs));
      }
#pragma unroll
      for (int L = NL - 1; L >= 0; --L) {
        float2 dzd[LPT][N];
#pragma unroll
        for (int q = 0; q < LPT; ++q) {
          float dz[N];
#pragma unroll
          for (int o = 0; o < N; ++o) {
            const float dv = (o & 1) ? dhp[q][o >> 1].y : dhp[q][o >> 1].x;
            dz[o] = ((mask[q][L] >> o) & 1u) ? dv : 0.f;
            dzd[q][o] = make_float2(dz[o], dz[o]);
          }
          store_row<N>(s_dz + L * LS + (tid + q * TT) * S, dz);
        }
        const float2* wr = reinterpret_cast<const float2*>(c_armb + L * LW);
#pragma unroll
        for (int o = 0; o < N; ++o)
#pragma unroll
          for (int j = 0; j < N / 2; ++j)
#pragma unroll
            for (int q = 0; q < LPT; ++q)
              dhp[q][j] = __ffma2_rn(wr[o * (N / 2) + j], dzd[q][o], dhp[q][j]);
      }
      float dh[LPT][N];
#pragma unroll
      for (int q = 0; q < LPT; ++q)
#pragma unroll
        for (int j = 0; j < N / 2; ++j) { dh[q][2 * j] = dhp[q][j].x; dh[q][2 * j + 1] = dhp[q][j].y; }
#pragma unroll
      for (int q = 0; q < LPT; ++q) {
        if (valid[q]) {
          const long long qq = a.g.off[l] + td.y + tid + q * TT;
#pragma unroll
          for (int k = 0; k < N; ++k) a.dctx[k * a.g.n_pad + qq] = dh[q][k];
          a.gself[qq] = lo[q].g_y;
        }
      }
      __syncthreads();

      // weight gradients of the LinR layers: acc += sum_p dz_L[p][rows] (x) in_L[p][cols]
      {
        const float* A = s_dz + uL * LS + urb * RB;
        const float* B = s_in + uL * LS + ucb * RB;
#pragma unroll 2
        for (int p = grp; p < T; p += G) {
          float av[RB], bv[RB];
          load_row<RB>(av, A + p * S);
          load_row<RB>(bv, B + p * S);
#pragma unroll
          for (int rr = 0; rr < RB; ++rr) {
            const float2 ad = make_float2(av[rr], av[rr]);
#pragma unroll
            for (int cc = 0; cc < RB / 2; ++cc)
              acc[rr][cc] = __ffma2_rn(ad, make_float2(bv[2 * cc], bv[2 * cc + 1]), acc[rr][cc]);
          }
        }
      }
      // biases and the output layer, in chunks of four columns
#pragma unroll
      for (int qi = 0; qi < XPER; ++qi) {
        const int q = unit + qi * NBLK;
        if (q < NCH_B) {
          const int L = q / (N / 4), i0 = (q % (N / 4)) * 4;
          const float* A = s_dz + L * LS + i0;
          for (int p = grp; p < T; p += G) {
            const float4 t = *reinterpret_cast<const float4*>(A + p * S);
            xacc[qi][0] += t.x; xacc[qi][1] += t.y; xacc[qi][2] += t.z; xacc[qi][3] += t.w;
          }
        } else if (q < NCH) {
          const int j0 = (q - NCH_B) * 4;
          for (int p = grp; p < T; p += G) {
            const float4 t = *reinterpret_cast<const float4*>(s_ho + p * S + j0);
            const float2 d = reinterpret_cast<const float2*>(s_do)[p];
            xacc[qi][0] = fmaf(d.x, t.x, xacc[qi][0]); xacc[qi][1] = fmaf(d.x, t.y, xacc[qi][1]);
            xacc[qi][2] = fmaf(d.x, t.z, xacc[qi][2]); xacc[qi][3] = fmaf(d.x, t.w, xacc[qi][3]);
            xacc[qi][4] = fmaf(d.y, t.x, xacc[qi][4]); xacc[qi][5] = fmaf(d.y, t.y, xacc[qi][5]);
            xacc[qi][6] = fmaf(d.y, t.z, xacc[qi][6]); xacc[qi][7] = fmaf(d.y, t.w, xacc[qi][7]);
            xacc[qi][8] += d.x; xacc[qi][9] += d.y;
          }
        }
      }
      __syncthreads();
    }
  }

  // rate partial of this CTA
  {
    float v = bits_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ float s_bits[TT / 32];
    if ((tid & 31) == 0) s_bits[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < TT / 32; ++k) t += s_bits[k];
      a.part_bits[blockIdx.x] = t;
    }
  }

  if constexpr (BWD) {
    // every (group, parameter) slot is written exactly once, then summed over groups
    float* red = sm;
    float* mine = red + grp * NP;
#pragma unroll
    for (int rr = 0; rr < RB; ++rr)
#pragma unroll
      for (int cc = 0; cc < RB; ++cc)
        mine[uL * LW + (urb * RB + rr) * N + ucb * RB + cc] =
            (cc & 1) ? acc[rr][cc >> 1].y : acc[rr][cc >> 1].x;
#pragma unroll
    for (int qi = 0; qi < XPER; ++qi) {
      const int q = unit + qi * NBLK;
      if (q < NCH_B) {
        const int L = q / (N / 4), i0 = (q % (N / 4)) * 4;
#pragma unroll
        for (int e = 0; e < 4; ++e) mine[L * LW + N * N + i0 + e] = xacc[qi][e];
      } else if (q < NCH) {
        const int j0 = (q - NCH_B) * 4;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          mine[OW + j0 + e] = xacc[qi][e];
          mine[OW + N + j0 + e] = xacc[qi][4 + e];
        }
        if (j0 == 0) { mine[OB] = xacc[qi][8]; mine[OB + 1] = xacc[qi][9]; }
      }
    }
    __syncthreads();
    for (int j = tid; j < NP; j += TT) {
      float t = 0.f;
#pragma unroll
      for (int g = 0; g < G; ++g) t += red[g * NP + j];
      a.part_grad[(long long)blockIdx.x * NP + j] = t;
    }
  }
}

// latents per thread of the instantiated ARM kernels
template <int N, int NL>
struct ArmLpt {
  static constexpr int value = 1;
};

template <int N, int NL, bool BWD>
static cudaError_t launch_t(const ArmArgs& a, int grid, cudaStream_t st) {
  constexpr int LPT = ArmLpt<N, NL>::value;
  using Sh = ArmShape<N, NL, LPT>;
  const size_t smem = BWD ? (size_t)Sh::smem_floats * sizeof(float) : 0;
  k_arm<N, NL, BWD, LPT><<<grid, kArmTile / LPT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int N, int NL>
static cudaError_t prepare_t() {
  constexpr int LPT = ArmLpt<N, NL>::value;
  return cudaFuncSetAttribute(k_arm<N, NL, true, LPT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(ArmShape<N, NL, LPT>::smem_floats * sizeof(float)));
}

template <int N, int NL>
static size_t smem_t(bool bwd) {
  return bwd ? (size_t)ArmShape<N, NL, ArmLpt<N, NL>::value>::smem_floats * sizeof(float) : 0;
}

#define CC_ARM_DISPATCH(FN, ...)                                              \
  switch (a.N * 10 + a.NL) {                                                  \
    case 81: return FN<8, 1>(__VA_ARGS__);                                    \
    case 82: return FN<8, 2>(__VA_ARGS__);                                    \
    case 161: return FN<16, 1>(__VA_ARGS__);                                  \
    case 162: return FN<16, 2>(__VA_ARGS__);                                  \
    case 241: return FN<24, 1>(__VA_ARGS__);                                  \
    case 242: return FN<24, 2>(__VA_ARGS__);                                  \
    default: break;                                                           \
  }

template <int N, int NL>
static cudaError_t launch_nl(bool bwd, const ArmArgs& k, int grid, cudaStream_t st) {
  return bwd ? launch_t<N, NL, true>(k, grid, st) : launch_t<N, NL, false>(k, grid, st);
}

cudaError_t arm_launch(const Arch& a, bool backward, const float* yhat, const Geo& g,
                       const int2* tiles, int n_tiles, int grid, float* dctx, float* gself,
                       float* part_grad, float* part_bits, cudaStream_t st) {
  ArmArgs k;
  k.yhat = yhat; k.dctx = dctx; k.gself = gself; k.part_grad = part_grad;
  k.part_bits = part_bits; k.tiles = tiles; k.n_tiles = n_tiles; k.g = g;
  CC_ARM_DISPATCH(launch_nl, backward, k, grid, st);
  return cudaErrorInvalidValue;
}

cudaError_t arm_prepare(const Arch& a) {
  CC_ARM_DISPATCH(prepare_t);
  return cudaErrorInvalidValue;
}

size_t arm_smem_bytes(const Arch& a, bool backward) {
  CC_ARM_DISPATCH(smem_t, backward);
  return 0;
}

int arm_blocks_per_sm(const Arch& a, bool backward) {
  (void)backward;
  return a.N >= 16 ? ArmOcc<24>::blocks : ArmOcc<8>::blocks;
}

__global__ void k_arm_image(const float* __restrict__ params, int n_arm,
                            const int2* __restrict__ offs, int N, int NL, ArmBank* img) {
  pdl_wait();
  pdl_trigger();
  // wb: the flat row-major parameters; w: the same with each LinR layer's W stored as
  // pairs (W[2m][k], W[2m+1][k]) (m outer, k inner) and W_out as (W_out[0][k], W_out[1][k])
  const int LW = N * N + N, OW = NL * LW;
  for (int i = threadIdx.x; i < kArmBankFloats; i += blockDim.x) {
    const float v = i < n_arm ? params[i] : 0.f;
    img->wb[i] = v;
    float f = v;
    if (i < OW) {
      const int L = i / LW, r = i - L * LW;
      if (r < N * N) {
        const int pair = r >> 1, m = pair / N, k = pair - m * N;
        f = params[L * LW + (2 * m + (r & 1)) * N + k];
      }
    } else if (i < OW + 2 * N) {
      const int r = i - OW;
      f = params[OW + (r & 1) * N + (r >> 1)];
    }
    img->w[i] = f;
  }
  for (int k = threadIdx.x; k < kMaxN; k += blockDim.x)
    img->off[k] = k < N ? offs[k] : make_int2(0, 0);
}

size_t arm_image_bytes() { return sizeof(ArmBank); }

cudaError_t arm_upload(const float* d_params, int n_arm, const int2* d_offsets, int N,
                       void* d_image, cudaStream_t st) {
  const int NL = (n_arm - 2 * N - 2) / (N * N + N);
  k_arm_image<<<1, 256, 0, st>>>(d_params, n_arm, d_offsets, N, NL, (ArmBank*)d_image);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbolAsync(c_armbank, d_image, sizeof(ArmBank), 0,
                                 cudaMemcpyDeviceToDevice, st);
}

}  // namespace cc
