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
// Forward and backward (the encoder iteration), k_arm_tc: the N x N layers of the forward
// pass (z = W h + b) and of the input gradient (dh += W^T dz) run on the tensor cores
// (tcgen05.mma kind::tf32 with operands split into TF32 high and low parts, FP32
// accumulation in tensor memory, cc_tc.cuh): M = the 128 latents of the tile, N = the
// layer width padded to a multiple of 16, K = N.  Each thread writes its latent's row of
// the A operand to shared memory and reads its row of the result back from its lane of
// the tensor memory.  The output layer (N -> 2), the Laplace rate and the weight gradients
// (sums over latents of dz (x) input: RB x RB register blocks of packed FP32 pairs over
// fp32 rows in shared memory, kept in registers over the CTA's tiles) run on the CUDA
// cores.  Every sum has a fixed order, so results are bit-reproducible on a given device.
//
// Forward only (rate of a pass without gradients), k_arm_fwd: every layer on the CUDA
// cores, weights as constant-bank operands in packed FP32 pairs.
#include "cc_internal.cuh"
#include "cc_laplace.cuh"
#include "cc_tc.cuh"

#include <cudaTypedefs.h>

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
  int* fault;        // set when a tensor-core wait gives up
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

// ------------------------------------------------------------ forward + backward (tensor cores)

template <int N, int NL>
struct ArmTcShape {
  static constexpr int T = kArmTile;            // latents per tile = threads per CTA
  static constexpr int NP = (N + 15) / 16 * 16; // MMA N: the layer width padded
  static constexpr int KS = N / 8;              // K steps of 8
  static constexpr int LW = N * N + N;          // floats per LinR layer (W then b)
  static constexpr int OW = NL * LW;            // W_out
  static constexpr int OB = OW + 2 * N;         // b_out
  static constexpr int NP_ARM = OB + 2;         // ARM parameters
  static constexpr int S = N;                   // fp32 row stride of the weight-gradient rows
  static constexpr int LS = T * S + 8;          // per-layer arrays (8-float bank skew)
  // bytes: A operand (hi, lo), then per layer W (hi, lo) and W^T (hi, lo), NP rows each
  static constexpr int A_BYTES = T * N * 4;
  static constexpr int W_BYTES = NP * N * 4;
  static constexpr int TC_BYTES = 2 * A_BYTES + NL * 4 * W_BYTES;
  // floats after the operands: s_in [NL][LS], s_dz [NL][LS], s_ho [T][S], s_do [T][2]
  static constexpr int F_FLOATS = 2 * NL * LS + T * S + 2 * T;
  static constexpr int NBLK = NL * ArmBlocking<N>::NB * ArmBlocking<N>::NB;
  static constexpr int G = T / NBLK;            // interleaved latent groups
  static constexpr int NCH_B = NL * N / 4;      // bias chunks of 4
  static constexpr int NCH = NCH_B + N / 4;     // + W_out column chunks (b_out rides on #0)
  static constexpr int XPER = (NCH + NBLK - 1) / NBLK;
  static constexpr int RED_FLOATS = G * NP_ARM;
  static constexpr int BYTES_MAIN = TC_BYTES + F_FLOATS * 4;
  static constexpr int BYTES = (BYTES_MAIN > RED_FLOATS * 4 ? BYTES_MAIN : RED_FLOATS * 4) + 16;
  static constexpr uint32_t TMEM_COLS = 32;
  static_assert(T % NBLK == 0 && G >= 1, "threads must split evenly into weight blocks");
  static_assert(N % 8 == 0 && NP <= 32, "tensor-core ARM widths: 8, 16, 24");
};

// wait budget of a tensor-core phase (SM clocks, about half a second)
constexpr long long kTcWaitCycles = 1ll << 30;

template <int N, int NL>
__global__ void __launch_bounds__(kArmTile, 2) k_arm_tc(ArmArgs a, const __grid_constant__ ArmMaps maps) {
  pdl_wait();
  pdl_trigger();
  using Sh = ArmTcShape<N, NL>;
  constexpr int T = Sh::T, NP = Sh::NP, KS = Sh::KS, LW = Sh::LW, OW = Sh::OW, OB = Sh::OB;
  constexpr int S = Sh::S, LS = Sh::LS, NPA = Sh::NP_ARM;
  constexpr int RB = ArmBlocking<N>::RB, NB = ArmBlocking<N>::NB;
  constexpr int NBLK = Sh::NBLK, G = Sh::G, NCH_B = Sh::NCH_B, NCH = Sh::NCH, XPER = Sh::XPER;
  constexpr uint32_t SBO_A = (N / 4) * 128;
  constexpr uint32_t IDESC = tc_idesc_tf32(T, NP);

  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA_hi = smem;
  unsigned char* sA_lo = sA_hi + Sh::A_BYTES;
  unsigned char* sW = sA_lo + Sh::A_BYTES;   // [L][W hi, W lo, W^T hi, W^T lo]
  float* sf = reinterpret_cast<float*>(smem + Sh::TC_BYTES);
  float* s_in = sf;                  // [NL][T][S] input of LinR layer L (layer stride LS)
  float* s_dz = s_in + NL * LS;      // [NL][T][S] dz of LinR layer L
  float* s_ho = s_dz + NL * LS;      // [T][S]     input of the output layer
  float* s_do = s_ho + T * S;        // [T][2]     (d bits/d mu, d bits/d s)
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  // causal context of a tile, loaded by TMA (double-buffered): rows y0 - kCtxPad .. y0 + 3,
  // columns x0 - kCtxPad .. x0 + 35 of the level (zeros outside it)
  constexpr int HR = kArmTileY + kCtxPad, HC = kArmTileX + 2 * kCtxPad;
  constexpr uint32_t HALO_BYTES = HR * HC * 4;
  __shared__ __align__(128) float s_halo[2][HR * HC];
  __shared__ __align__(8) uint64_t s_tbar[2];

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  // weights as B operands: W (K = input, rows = outputs) and W^T, split into TF32 parts;
  // rows N .. NP-1 are zero
  for (int i = tid; i < NL * NP * N; i += T) {
    const int L = i / (NP * N), rk = i - L * NP * N, row = rk / N, k = rk - row * N;
    const float wf = row < N ? c_armb[L * LW + row * N + k] : 0.f;   // W[row][k]
    const float wt = row < N ? c_armb[L * LW + k * N + row] : 0.f;   // W^T[row][k] = W[k][row]
    const float fh = tf32_hi(wf), th = tf32_hi(wt);
    unsigned char* base = sW + L * 4 * Sh::W_BYTES;
    const int off = tc_off(row, k, N);
    *reinterpret_cast<float*>(base + off) = fh;
    *reinterpret_cast<float*>(base + Sh::W_BYTES + off) = wf - fh;
    *reinterpret_cast<float*>(base + 2 * Sh::W_BYTES + off) = th;
    *reinterpret_cast<float*>(base + 3 * Sh::W_BYTES + off) = wt - th;
  }
  if (tid == 0) {
    mbar_init(smem_u32(&s_mbar), 1);
    mbar_init(smem_u32(&s_tbar[0]), 1);
    mbar_init(smem_u32(&s_tbar[1]), 1);
  }
  if (warp == 0) tc_alloc(smem_u32(&s_tmem), Sh::TMEM_COLS);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's lanes
  const uint32_t mbar = smem_u32(&s_mbar);
  uint32_t phase = 0;

  // Stage the A operand (this thread's row, split), run D = A B^T for B = layer L's W
  // (transpose = false) or W^T (true), and return this thread's row of D.  False when a
  // wait gave up (the CTA then stops).
  auto layer_mma = [&](const float (&x)[N], int L, bool transpose, float (&d)[NP]) -> bool {
#pragma unroll
    for (int k = 0; k < N; k += 4) {
      const float4 hi = make_float4(tf32_hi(x[k]), tf32_hi(x[k + 1]), tf32_hi(x[k + 2]),
                                    tf32_hi(x[k + 3]));
      const float4 lo = make_float4(x[k] - hi.x, x[k + 1] - hi.y, x[k + 2] - hi.z, x[k + 3] - hi.w);
      *reinterpret_cast<float4*>(sA_hi + tc_off(tid, k, N)) = hi;
      *reinterpret_cast<float4*>(sA_lo + tc_off(tid, k, N)) = lo;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = smem_u32(sA_hi), al = smem_u32(sA_lo);
      const uint32_t wb = smem_u32(sW + L * 4 * Sh::W_BYTES + (transpose ? 2 : 0) * Sh::W_BYTES);
      const uint32_t bh = wb, bl = wb + Sh::W_BYTES;
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        const uint32_t ko = (uint32_t)s * 256u;
        tc_mma_tf32(tmem, tc_desc(ah + ko, SBO_A), tc_desc(bh + ko, SBO_A), IDESC, s > 0 ? 1u : 0u);
        tc_mma_tf32(tmem, tc_desc(ah + ko, SBO_A), tc_desc(bl + ko, SBO_A), IDESC, 1u);
        tc_mma_tf32(tmem, tc_desc(al + ko, SBO_A), tc_desc(bh + ko, SBO_A), IDESC, 1u);
      }
      tc_commit(mbar);
    }
    const bool ok = mbar_wait(mbar, phase, kTcWaitCycles);
    phase ^= 1u;
    if (__syncthreads_or(ok ? 0 : 1)) return false;   // every thread takes the same branch
    tc_fence_after();
    tc_ld_row<NP>(t_row, d);
    return true;
  };

  float2 acc[RB][RB / 2];   // weight-gradient block as packed pairs along its columns
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

  // TMA of a tile's context into halo buffer `buf` (thread 0): the buffer's earlier
  // readers are ordered before the asynchronous write by a barrier and this fence
  auto issue = [&](int t, int buf) {
    const int2 tq = a.tiles[t];
    fence_async_smem();
    const uint32_t bar = smem_u32(&s_tbar[buf]);
    mbar_expect_tx(bar, HALO_BYTES);
    tma_load_2d(smem_u32(&s_halo[buf][0]), &maps.m[tq.x], tq.y & 0xFFFF, tq.y >> 16, bar);
  };
  if (tid == 0 && (int)blockIdx.x < a.n_tiles) issue(blockIdx.x, 0);
  int it = 0;
  bool pending = (int)blockIdx.x < a.n_tiles;   // a load in flight into buffer it & 1
  for (int tile = blockIdx.x; tile < a.n_tiles && ok; tile += gridDim.x, ++it) {
    const int buf = it & 1;
    // the next tile's context goes to the other buffer, read during the previous tile
    const bool more = tile + (int)gridDim.x < a.n_tiles;
    if (tid == 0 && more) issue(tile + gridDim.x, buf ^ 1);
    const bool hok = mbar_wait(smem_u32(&s_tbar[buf]), (uint32_t)(it >> 1) & 1u, kTcWaitCycles);
    if (__syncthreads_or(hok ? 0 : 1)) { ok = false; break; }
    pending = more;
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

    // forward: h <- h + relu(W h + b), NL times
    uint32_t mask[NL];
#pragma unroll
    for (int L = 0; L < NL; ++L) {
      store_row<N>(s_in + L * LS + tid * S, h);
      float z[NP];
      if (!layer_mma(h, L, false, z)) { ok = false; break; }
      uint32_t mk = 0;
#pragma unroll
      for (int o = 0; o < N; ++o) {
        const float zo = z[o] + c_armb[L * LW + N * N + o];
        mk |= (zo > 0.f ? 1u : 0u) << o;
        h[o] += fmaxf(zo, 0.f);
      }
      mask[L] = mk;
    }
    if (!ok) break;
    store_row<N>(s_ho + tid * S, h);
    const float2 ms = output_layer<N, NL>(h);
    LapOut lo = laplace_bits(yq, ms.x, ms.y);
    if (!valid) lo.bits = lo.g_y = lo.g_mu = lo.g_s = 0.f;
    bits_acc += lo.bits;

    // backward: dh = W_out^T (d mu, d s), then dh += W_L^T (mask_L * dh) for L = NL-1 .. 0
    reinterpret_cast<float2*>(s_do)[tid] = make_float2(lo.g_mu, lo.g_s);
    float dh[N];
#pragma unroll
    for (int k = 0; k < N; ++k)
      dh[k] = fmaf(c_armb[OW + k], lo.g_mu, c_armb[OW + N + k] * lo.g_s);
#pragma unroll
    for (int L = NL - 1; L >= 0; --L) {
      float dz[N];
#pragma unroll
      for (int o = 0; o < N; ++o) dz[o] = ((mask[L] >> o) & 1u) ? dh[o] : 0.f;
      store_row<N>(s_dz + L * LS + tid * S, dz);
      float t[NP];
      if (!layer_mma(dz, L, true, t)) { ok = false; break; }
#pragma unroll
      for (int k = 0; k < N; ++k) dh[k] += t[k];
    }
    if (!ok) break;
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
    // a tensor-core wait gave up: report, give the MMAs in flight another bounded wait,
    // free the tensor memory and stop
    if (tid == 0) atomicExch(a.fault, 1);
    mbar_wait(mbar, phase ^ 1u, kTcWaitCycles);
    if (pending)   // the context load still in flight
      mbar_wait(smem_u32(&s_tbar[(it + 1) & 1]), (uint32_t)((it + 1) >> 1) & 1u, kTcWaitCycles);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, Sh::TMEM_COLS);
    return;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, Sh::TMEM_COLS);

  // rate partial of this CTA
  {
    float v = bits_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ float s_bits[T / 32];
    if ((tid & 31) == 0) s_bits[warp] = v;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < T / 32; ++k) t += s_bits[k];
      a.part_bits[blockIdx.x] = t;
    }
  }
  // every (group, parameter) slot is written exactly once, then summed over groups
  float* red = reinterpret_cast<float*>(smem);
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
    k_arm_tc<N, NL><<<grid, kArmTile, ArmTcShape<N, NL>::BYTES, st>>>(a, maps);
  } else {
    k_arm_fwd<N, NL><<<grid, kArmTile, 0, st>>>(a);
  }
  return cudaGetLastError();
}

template <int N, int NL>
static cudaError_t prepare_t() {
  return cudaFuncSetAttribute(k_arm_tc<N, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              ArmTcShape<N, NL>::BYTES);
}

template <int N, int NL>
static size_t smem_t(bool bwd) {
  return bwd ? (size_t)ArmTcShape<N, NL>::BYTES : 0;
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
                       int* fault, cudaStream_t st) {
  ArmArgs k;
  k.yhat = yhat; k.dctx = dctx; k.gself = gself; k.part_grad = part_grad;
  k.part_bits = part_bits; k.tiles = tiles; k.n_tiles = n_tiles; k.fault = fault; k.g = g;
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

// two CTAs of the tensor-core kernel fit an SM (shared memory); the forward-only kernel
// runs on the same grid
int arm_blocks_per_sm(const Arch& a, bool backward) {
  (void)a;
  (void)backward;
  return 2;
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
