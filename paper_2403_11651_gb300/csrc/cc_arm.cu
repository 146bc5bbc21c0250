// Auto-regressive probability model p_psi and the rate term of eq. (1).
//
// Sec. II "Decoding" item ii: the ARM is an MLP f_psi of the N causal neighbours of a
// latent in its own grid; Table 1 gives its layers (N-N-LinR x arm_layers, N-2-Lin).  Its
// two outputs are the mean mu and log-scale s of a Laplace law, and the rate of a latent
// is -log2 P(y_hat) with P the mass of [y_hat - 1/2, y_hat + 1/2] (eq. (1)).
//
// One thread owns one latent; a tile is 128 latents of one level (kArmTile).  The weights
// live in a __constant__ bank refreshed before every pass.
//
// Forward and backward (the encoder iteration), k_arm_fb: one persistent loop over tiles of
// 4 x 32 latents, three CTAs of 128 threads per SM.  A tile's causal context (8 x 40
// floats of the zero-bordered y_hat plane) arrives by TMA, issued one tile ahead into a
// double buffer.  The N x N layers of the forward pass and of the input gradient run as
// packed FP32 pairs whose weight pairs come from the constant bank; the output layer, the
// Laplace rate, then the weight gradients (sums over latents of dz (x) input: RB x RB
// register blocks of packed pairs over the tile's rows staged in shared memory, kept in
// registers over the CTA's tiles).  Every sum has a fixed order, so results are
// bit-reproducible on a given device.
//
// Forward only (rate of a pass without gradients), k_arm_fwd: the same layers without the
// backward half.
#include "cc_internal.cuh"
#include "cc_laplace.cuh"
#include "cc_tc.cuh"

#include <cudaTypedefs.h>

#include <cstdlib>

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
  int* fault;        // set when a context-load wait gives up
  const int* stall;  // > 0: skip the first context load and wait this many cycles for it
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

// Latent (y, x) of thread tid in tile td = (level, y0 << 16 | x0): rows of kArmTileX.
__device__ __forceinline__ void tile_latent(int2 td, int tid, int& y, int& x) {
  y = (td.y >> 16) + tid / kArmTileX;
  x = (td.y & 0xFFFF) + tid % kArmTileX;
}

// The N causal neighbours of the thread's latent and the latent itself, read from the
// zero-bordered plane (every neighbour is inside the allocation; outside the grid it reads
// the zero border).  Returns whether the latent exists.
template <int N>
__device__ __forceinline__ bool gather_context(const ArmArgs& a, int2 td, int tid,
                                               float (&h)[N], float& yq) {
  const int l = td.x;
  int r, c;
  tile_latent(td, tid, r, c);
  const bool valid = r < a.g.h[l] && c < a.g.w[l];
  if (!valid) { r = 0; c = 0; }
  const int pw = a.g.pw[l];
  const float* ctr = a.yhat + a.g.poff[l] + (long long)(r + kCtxPad) * pw + c + kCtxPad;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int2 o = c_off[k];
    h[k] = valid ? __ldg(ctr + o.x * pw + o.y) : 0.f;
  }
  yq = valid ? __ldg(ctr) : 0.f;
  return valid;
}

// (mu, s) = W_out h + b_out as one packed pair; the forward bank stores W_out as
// (W_out[0][k], W_out[1][k])
template <int N, int NL>
__device__ __forceinline__ float2 output_layer(const float (&h)[N]) {
  constexpr int OW = NL * (N * N + N), OB = OW + 2 * N;
  const float2* wo = reinterpret_cast<const float2*>(c_arm + OW);
  float2 ms = make_float2(c_arm[OB], c_arm[OB + 1]);
#pragma unroll
  for (int k = 0; k < N; ++k) ms = __ffma2_rn(wo[k], make_float2(h[k], h[k]), ms);
  return ms;
}

// ------------------------------------------------------------ forward only (CUDA cores)

template <int N, int NL>
__global__ void __launch_bounds__(kArmTile) k_arm_fwd(ArmArgs a) {
  pdl_wait();
  pdl_trigger();
  constexpr int LW = N * N + N;
  const int tid = threadIdx.x;
  float bits_acc = 0.f;
  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int2 td = a.tiles[tile];
    float h[N], yq;
    const bool valid = gather_context<N>(a, td, tid, h, yq);
#pragma unroll
    for (int L = 0; L < NL; ++L) {
      // packed FP32 pairs: (z[2m], z[2m+1]) += (W[2m][k], W[2m+1][k]) * (h[k], h[k]); the
      // forward bank stores every layer's weights in those pairs, input k innermost
      float2 zp[N / 2];
      const float2* wp = reinterpret_cast<const float2*>(c_arm + L * LW);
#pragma unroll
      for (int m = 0; m < N / 2; ++m) zp[m] = wp[N * N / 2 + m];   // bias pair
#pragma unroll
      for (int m = 0; m < N / 2; ++m)
#pragma unroll
        for (int k = 0; k < N; ++k) zp[m] = __ffma2_rn(wp[m * N + k], make_float2(h[k], h[k]), zp[m]);
#pragma unroll
      for (int m = 0; m < N / 2; ++m) {
        h[2 * m] += fmaxf(zp[m].x, 0.f);
        h[2 * m + 1] += fmaxf(zp[m].y, 0.f);
      }
    }
    const float2 ms = output_layer<N, NL>(h);
    const LapOut lo = laplace_bits(yq, ms.x, ms.y);
    if (valid) bits_acc += lo.bits;
  }
  float v = bits_acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ float s_bits[kArmTile / 32];
  if ((tid & 31) == 0) s_bits[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < kArmTile / 32; ++k) t += s_bits[k];
    a.part_bits[blockIdx.x] = t;
  }
}

// wait budget of a context load (SM clocks, about half a second)
constexpr long long kTcWaitCycles = 1ll << 30;

// ------------------------------------------------------------ forward + backward (CUDA cores)
//
// Measured alone on all SMs at 512 x 768 with the 24-input ARM (GB300): 104 us.  Three
// alternatives were slower: the N x N layers on tcgen05 tensor cores (TF32 x 3, a chain of
// four MMA round trips per tile, two CTAs per SM): 121 us; scalar FMAs with constant-bank
// operands: 120 us (weights beyond what the immediate-constant cache holds are fetched
// one by one) and 146 us rolled over the inputs.

template <int N, int NL>
struct ArmFbShape {
  static constexpr int T = kArmTile;
  static constexpr int LW = N * N + N, OW = NL * LW, OB = OW + 2 * N, NP_ARM = OB + 2;
  static constexpr int S = N;                     // row stride of the staged rows
  static constexpr int LS = T * S + 8;            // per-layer arrays (8-float bank skew)
  static constexpr int F_FLOATS = 2 * NL * LS + T * S + 2 * T;
  static constexpr int NBLK = NL * ArmBlocking<N>::NB * ArmBlocking<N>::NB;
  static constexpr int G = T / NBLK;
  static constexpr int NCH_B = NL * N / 4;
  static constexpr int NCH = NCH_B + N / 4;
  static constexpr int XPER = (NCH + NBLK - 1) / NBLK;
  static constexpr int RED_FLOATS = G * NP_ARM;
  static constexpr int BYTES = (F_FLOATS > RED_FLOATS ? F_FLOATS : RED_FLOATS) * 4;
  static_assert(T % NBLK == 0 && G >= 1, "threads must split evenly into weight blocks");
};
constexpr int kArmFbBlocksPerSm = 3;

template <int N, int NL>
__global__ void __launch_bounds__(kArmTile, kArmFbBlocksPerSm)
k_arm_fb(ArmArgs a, const __grid_constant__ ArmMaps maps) {
  pdl_wait();
  pdl_trigger();
  using Sh = ArmFbShape<N, NL>;
  constexpr int T = Sh::T, LW = Sh::LW, OW = Sh::OW, OB = Sh::OB, NPA = Sh::NP_ARM;
  constexpr int S = Sh::S, LS = Sh::LS;
  constexpr int RB = ArmBlocking<N>::RB, NB = ArmBlocking<N>::NB;
  constexpr int NBLK = Sh::NBLK, G = Sh::G, NCH_B = Sh::NCH_B, NCH = Sh::NCH, XPER = Sh::XPER;

  extern __shared__ __align__(16) float sf[];
  float* s_in = sf;                  // [NL][T][S] input of LinR layer L (layer stride LS)
  float* s_dz = s_in + NL * LS;      // [NL][T][S] dz of LinR layer L
  float* s_ho = s_dz + NL * LS;      // [T][S]     input of the output layer
  float* s_do = s_ho + T * S;        // [T][2]     (d bits/d mu, d bits/d s)
  constexpr int HR = kArmTileY + kCtxPad, HC = kArmTileX + 2 * kCtxPad;
  constexpr uint32_t HALO_BYTES = HR * HC * 4;
  __shared__ __align__(128) float s_halo[2][HR * HC];
  __shared__ __align__(8) uint64_t s_tbar[2];

  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(smem_u32(&s_tbar[0]), 1);
    mbar_init(smem_u32(&s_tbar[1]), 1);
  }
  __syncthreads();

  float2 acc[RB][RB / 2];
  float xacc[XPER][10];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int c = 0; c < RB / 2; ++c) acc[r][c] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < XPER; ++q)
#pragma unroll
    for (int e = 0; e < 10; ++e) xacc[q][e] = 0.f;
  const int unit = tid % NBLK, grp = tid / NBLK;
  const int uL = unit / (NB * NB), urb = (unit / NB) % NB, ucb = unit % NB;
  float bits_acc = 0.f;
  bool ok = true;

  auto issue = [&](int t, int buf) {
    const int2 tq = a.tiles[t];
    fence_async_smem();
    const uint32_t bar = smem_u32(&s_tbar[buf]);
    mbar_expect_tx(bar, HALO_BYTES);
    tma_load_2d(smem_u32(&s_halo[buf][0]), &maps.m[tq.x], tq.y & 0xFFFF, tq.y >> 16, bar);
  };
  // fault injection (host-requested): the first load is not issued, so its wait runs out
  const int stall = *a.stall;
  const long long budget = stall > 0 ? (long long)stall : kTcWaitCycles;
  // bit b: a load issued into buffer b and not yet waited for
  unsigned inflight = 0u;
  if ((int)blockIdx.x < a.n_tiles && stall <= 0) {
    if (tid == 0) issue(blockIdx.x, 0);
    inflight |= 1u;
  }
  int it = 0;
  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
    const int buf = it & 1;
    if (tile + (int)gridDim.x < a.n_tiles) {
      if (tid == 0) issue(tile + gridDim.x, buf ^ 1);
      inflight |= 1u << (buf ^ 1);
    }
    const bool hok = mbar_wait(smem_u32(&s_tbar[buf]), (uint32_t)(it >> 1) & 1u, budget);
    if (__syncthreads_or(hok ? 0 : 1)) { ok = false; break; }
    inflight &= ~(1u << buf);
    const int2 td = a.tiles[tile];
    int ly, lx;
    tile_latent(td, tid, ly, lx);
    const bool valid = ly < a.g.h[td.x] && lx < a.g.w[td.x];
    const float* hb = &s_halo[buf][(tid / kArmTileX + kCtxPad) * HC + tid % kArmTileX + kCtxPad];
    float h[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int2 o = c_off[k];
      h[k] = valid ? hb[o.x * HC + o.y] : 0.f;
    }
    const float yq = valid ? hb[0] : 0.f;

    // forward: h <- h + relu(W h + b), NL times; every weight is the constant-bank operand
    // of a scalar FMA (packed pairs with a constant-bank pair operand measured 3x slower)
    uint32_t mask[NL];
#pragma unroll
    for (int L = 0; L < NL; ++L) {
      store_row<N>(s_in + L * LS + tid * S, h);
      // packed FP32 pairs over adjacent outputs, the weight pair (W[2m][k], W[2m+1][k])
      // read from the forward copy of the bank
      float z[N];
      {
        const float2* wp = reinterpret_cast<const float2*>(c_arm + L * LW);
        float2 zp[N / 2];
#pragma unroll
        for (int m = 0; m < N / 2; ++m) zp[m] = wp[N * N / 2 + m];   // bias pair
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const float2 hk = make_float2(h[k], h[k]);
#pragma unroll
          for (int m = 0; m < N / 2; ++m) zp[m] = __ffma2_rn(wp[m * N + k], hk, zp[m]);
        }
#pragma unroll
        for (int m = 0; m < N / 2; ++m) { z[2 * m] = zp[m].x; z[2 * m + 1] = zp[m].y; }
      }
      uint32_t mk = 0;
#pragma unroll
      for (int o = 0; o < N; ++o) {
        mk |= (z[o] > 0.f ? 1u : 0u) << o;
        h[o] += fmaxf(z[o], 0.f);
      }
      mask[L] = mk;
    }
    store_row<N>(s_ho + tid * S, h);
    // the forward reads the bank copy `w`, the backward the row-major copy `wb`: a weight
    // read by both from one copy is kept in a register between its two uses, and with
    // 1250 weights that pushes the rest out to separate loads
    float mu = c_arm[OB], sl = c_arm[OB + 1];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      mu = fmaf(c_arm[OW + 2 * k], h[k], mu);
      sl = fmaf(c_arm[OW + 2 * k + 1], h[k], sl);
    }
    LapOut lo = laplace_bits(yq, mu, sl);
    if (!valid) lo.bits = lo.g_y = lo.g_mu = lo.g_s = 0.f;
    bits_acc += lo.bits;

    // backward: dh = W_out^T (d mu, d s), then dh += W_L^T (mask_L * dh), L = NL-1 .. 0
    reinterpret_cast<float2*>(s_do)[tid] = make_float2(lo.g_mu, lo.g_s);
    float dh[N];
#pragma unroll
    for (int k = 0; k < N; ++k) dh[k] = fmaf(c_armb[OW + k], lo.g_mu, c_armb[OW + N + k] * lo.g_s);
#pragma unroll
    for (int L = NL - 1; L >= 0; --L) {
      float dz[N];
#pragma unroll
      for (int o = 0; o < N; ++o) dz[o] = ((mask[L] >> o) & 1u) ? dh[o] : 0.f;
      store_row<N>(s_dz + L * LS + tid * S, dz);
      // packed pairs over adjacent inputs, (W[o][2j], W[o][2j+1]) from the row-major copy
      const float2* wr = reinterpret_cast<const float2*>(c_armb + L * LW);
      float2 dhp[N / 2];
#pragma unroll
      for (int j = 0; j < N / 2; ++j) dhp[j] = make_float2(dh[2 * j], dh[2 * j + 1]);
#pragma unroll
      for (int o = 0; o < N; ++o) {
        const float2 d2 = make_float2(dz[o], dz[o]);
#pragma unroll
        for (int j = 0; j < N / 2; ++j) dhp[j] = __ffma2_rn(wr[o * (N / 2) + j], d2, dhp[j]);
      }
#pragma unroll
      for (int j = 0; j < N / 2; ++j) { dh[2 * j] = dhp[j].x; dh[2 * j + 1] = dhp[j].y; }
    }
    if (valid) {
      const long long qq = a.g.off[td.x] + (long long)ly * a.g.w[td.x] + lx;
#pragma unroll
      for (int k = 0; k < N; ++k) a.dctx[k * a.g.n_pad + qq] = dh[k];
      a.gself[qq] = lo.g_y;
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

  if (!ok) {
    // a context wait gave up at iteration it: report, give every load still in flight
    // another bounded wait (nothing may land in shared memory after the CTA has left) and
    // stop.  Buffer it & 1 has completed it >> 1 phases, the other (it + 1) >> 1.
    if (tid == 0) atomicExch(a.fault, 1);
    const int b = it & 1;
    if (inflight & (1u << b))
      mbar_wait(smem_u32(&s_tbar[b]), (uint32_t)(it >> 1) & 1u, kTcWaitCycles);
    if (inflight & (1u << (b ^ 1)))
      mbar_wait(smem_u32(&s_tbar[b ^ 1]), (uint32_t)((it + 1) >> 1) & 1u, kTcWaitCycles);
    __syncthreads();
    return;
  }

  // rate partial of this CTA
  {
    float v = bits_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ float s_bits[T / 32];
    if ((tid & 31) == 0) s_bits[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < T / 32; ++k) t += s_bits[k];
      a.part_bits[blockIdx.x] = t;
    }
  }
  // every (group, parameter) slot is written exactly once, then summed over groups
  float* red = sf;
  float* mine = red + grp * NPA;
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
  for (int j = tid; j < NPA; j += T) {
    float t = 0.f;
#pragma unroll
    for (int g = 0; g < G; ++g) t += red[g * NPA + j];
    a.part_grad[(long long)blockIdx.x * NPA + j] = t;
  }
}

template <int N, int NL>
static cudaError_t launch_t(bool bwd, const ArmArgs& a, const ArmMaps& maps, int grid,
                            cudaStream_t st) {
  if (bwd) {
    k_arm_fb<N, NL><<<grid, kArmTile, ArmFbShape<N, NL>::BYTES, st>>>(a, maps);
  } else {
    k_arm_fwd<N, NL><<<grid, kArmTile, 0, st>>>(a);
  }
  return cudaGetLastError();
}

template <int N, int NL>
static cudaError_t prepare_t() {
  return cudaFuncSetAttribute(k_arm_fb<N, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              ArmFbShape<N, NL>::BYTES);
}

template <int N, int NL>
static size_t smem_t(bool bwd) {
  return bwd ? (size_t)ArmFbShape<N, NL>::BYTES : 0;
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

cudaError_t arm_launch(const Arch& a, bool backward, const float* yhat, const Geo& g,
                       const ArmMaps& maps, const int2* tiles, int n_tiles, int grid,
                       float* dctx, float* gself, float* part_grad, float* part_bits,
                       int* fault, const int* stall, cudaStream_t st) {
  ArmArgs k;
  k.yhat = yhat; k.dctx = dctx; k.gself = gself; k.part_grad = part_grad;
  k.part_bits = part_bits; k.tiles = tiles; k.n_tiles = n_tiles; k.fault = fault;
  k.stall = stall; k.g = g;
  CC_ARM_DISPATCH(launch_t, backward, k, maps, grid, st);
  return cudaErrorInvalidValue;
}

cudaError_t arm_make_maps(const Geo& g, const float* yhat_bord, ArmMaps* out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  for (int l = 0; l < kLevels; ++l) {
    const cuuint64_t dims[2] = {(cuuint64_t)g.pw[l], (cuuint64_t)(g.h[l] + kCtxPad)};
    const cuuint64_t strides[1] = {(cuuint64_t)g.pw[l] * sizeof(float)};
    const cuuint32_t box[2] = {kArmTileX + 2 * kCtxPad, kArmTileY + kCtxPad};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(&out->m[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                              const_cast<float*>(yhat_bord + g.poff[l]), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t arm_prepare(const Arch& a) {
  CC_ARM_DISPATCH(prepare_t);
  return cudaErrorInvalidValue;
}

size_t arm_smem_bytes(const Arch& a, bool backward) {
  CC_ARM_DISPATCH(smem_t, backward);
  return 0;
}

// CTAs per SM of the backward kernel (its shared memory and registers allow three); the
// forward-only kernel runs on the same grid
int arm_blocks_per_sm(const Arch& a, bool backward) {
  (void)a;
  (void)backward;
  return kArmFbBlocksPerSm;
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

cudaError_t arm_build_image(const float* d_params, int n_arm, const int2* d_offsets, int N,
                            void* d_image, cudaStream_t st) {
  const int NL = (n_arm - 2 * N - 2) / (N * N + N);
  k_arm_image<<<1, 256, 0, st>>>(d_params, n_arm, d_offsets, N, NL, (ArmBank*)d_image);
  return cudaGetLastError();
}

cudaError_t arm_copy_bank(const void* d_image, cudaStream_t st) {
  return cudaMemcpyToSymbolAsync(c_armbank, d_image, sizeof(ArmBank), 0,
                                 cudaMemcpyDeviceToDevice, st);
}

cudaError_t arm_upload(const float* d_params, int n_arm, const int2* d_offsets, int N,
                       void* d_image, cudaStream_t st) {
  cudaError_t e = arm_build_image(d_params, n_arm, d_offsets, N, d_image, st);
  return e != cudaSuccess ? e : arm_copy_bank(d_image, st);
}

int arm_image_weight_floats() { return 2 * kArmBankFloats; }

}  // namespace cc
