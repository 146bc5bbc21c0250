// Latent bitstream on the GPU: fixed-point ARM, Laplace frequency tables, per-row range
// coding and a wavefront decoder.
//
// Sec. II "Encoding": after the optimisation the latents are entropy coded with a range
// coder driven by the ARM's probability model p_psi.  Sec. II "Decoding" (Fig. 2): the
// decoder reads every latent grid with that model, each latent conditioned on its
// already-decoded causal neighbours.  The decoder re-runs the ARM on decoded values, so
// both sides must compute identical probabilities: the ARM runs here in integer
// arithmetic.
//
// Format (shared with the decoder, nothing float on the device):
//   ARM:    32-bit fixed point with 8 fractional bits (Q8): weights rounded half-to-even
//           and clamped to +-2^11 (|w| <= 8), biases to +-2^15; context = integer latents
//           clamped to [-128, 128] times 256; a layer computes
//           z = ((sum_j W[o, j] a[j]) + 128) >> 8 + b[o], saturated to +-2^15; a LinR
//           layer outputs a[o] + max(z, 0), saturated; the output layer gives (mu_q, s_q).
//           With N <= 24 every sum is below 24 * 2^26 < 2^31: exact in int32.
//   tables: s_q picks one of 93 log-scale bins of width 1/8 from -1179/256 (floor of
//           256 ln 0.01), clamped; mu_q = 256 m + 32 fi + rest; table (bin j, fi) is the
//           Laplace law of mean (fi + 1/2)/8 and scale exp(-1179/256 + (j + 1/2)/8) over
//           k = y_hat - m in [-64, 64] plus one escape symbol per tail.  Frequencies out
//           of 2^16: 1 + floor(p (2^16 - 131)), the remainder to the first largest.  The
//           tables are built on the host in IEEE double (C library exp, no contraction).
//   escape: |k| - 65 follows as an order-0 Exp-Golomb code of (|k| - 64) in equiprobable
//           binary decisions.
//   coder:  32-bit range, 33-bit low with carry propagation through held-back 0xFF
//           bytes; the always-zero first byte is not written; the final value is the one
//           of the last interval with the most trailing zero bits, and trailing zero
//           bytes are dropped (the decoder reads zeros past the end of a substream).
//   streams: one substream per latent row, so that rows decode as a wavefront.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cmath>
#include <mutex>
#include <vector>

#include "cc_internal.cuh"

namespace cc {

namespace {

constexpr int kQFrac = 8;
constexpr int kWLim = 1 << 11;
constexpr int kActLim = 1 << 15;
constexpr int kCtxLim = 128;
constexpr int kYLim = 1 << 20;
constexpr int kA = 64;
constexpr int kNsym = 2 * kA + 3;          // 131
constexpr int kNmu = 8;
constexpr int kNscale = 93;
constexpr int kLogbLoQ = -1179;
constexpr int kTabStride = 132;            // cum[0..130]; cum[131] = 2^16 is implicit
constexpr int kNtab = kNscale * kNmu;
constexpr uint32_t kTotal = 1u << 16;
constexpr int kMaxQArm = 2 * (24 * 24 + 24) + 2 * 24 + 2;
constexpr int kMaxEgBits = 40;             // Exp-Golomb prefix bound (latents < 2^21)

__constant__ int c_qarm[kMaxQArm];

__device__ __forceinline__ int sat(int v) { return min(max(v, -kActLim), kActLim); }

// (mu_q, s_q) of the fixed-point ARM for the integer context ctx; weights in c_qarm
template <int N, int NL>
__device__ __forceinline__ void arm_fixed(const int (&ctx)[N], int& mu, int& s) {
  int a[N];
#pragma unroll
  for (int j = 0; j < N; ++j) a[j] = min(max(ctx[j], -kCtxLim), kCtxLim) * (1 << kQFrac);
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const int* Wt = c_qarm + i * (N * N + N);   // the bank holds W transposed: Wt[j N + o]
    const int* b = Wt + N * N;
    int acc[N];                 // all N sums advance together: N independent chains
#pragma unroll
    for (int o = 0; o < N; ++o) acc[o] = 0;
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int o = 0; o < N; ++o) acc[o] += Wt[j * N + o] * a[j];
#pragma unroll
    for (int o = 0; o < N; ++o) a[o] = sat(a[o] + max(sat(((acc[o] + 128) >> kQFrac) + b[o]), 0));
  }
  const int* W = c_qarm + NL * (N * N + N);
  const int* b = W + 2 * N;
  int acc0 = 0, acc1 = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    acc0 += W[j] * a[j];
    acc1 += W[N + j] * a[j];
  }
  mu = sat(((acc0 + 128) >> kQFrac) + b[0]);
  s = sat(((acc1 + 128) >> kQFrac) + b[1]);
}

// table number and integer part of mu
__device__ __forceinline__ void table_of(int mu, int s, int& t, int& m) {
  const int j = min(max((s - kLogbLoQ) >> 5, 0), kNscale - 1);
  t = j * kNmu + ((mu & 255) >> 5);
  m = mu >> kQFrac;
}

__device__ __forceinline__ uint32_t cum_at(const uint16_t* row, int i) {
  return i == kNsym ? kTotal : (uint32_t)row[i];
}

struct RcEnc {
  unsigned long long low;
  uint32_t range, cache, pending;
  bool first, over;
  uint8_t* out;
  int n, cap;

  __device__ void init(uint8_t* o, int c) {
    low = 0; range = 0xFFFFFFFFu; cache = 0; pending = 1; first = true; over = false;
    out = o; n = 0; cap = c;
  }
  __device__ void put(uint32_t b) {
    if (n < cap) out[n] = (uint8_t)b; else over = true;
    ++n;
  }
  __device__ void shift_low() {
    if (low < 0xFF000000ull || low >= (1ull << 32)) {
      const uint32_t carry = (uint32_t)(low >> 32);
      if (first) first = false; else put(cache + carry);
      for (uint32_t i = 1; i < pending; ++i) put(0xFFu + carry);
      pending = 0;
      cache = (uint32_t)(low >> 24) & 0xFFu;
    }
    ++pending;
    low = (low & 0x00FFFFFFull) << 8;
  }
  __device__ void encode(uint32_t start, uint32_t freq) {
    const uint32_t r = range >> 16;
    low += (unsigned long long)r * start;
    range = r * freq;
    while (range < (1u << 24)) {
      range <<= 8;
      shift_low();
    }
  }
  __device__ void bit(uint32_t b) { encode(b << 15, 1u << 15); }
  __device__ void excess(uint32_t e) {   // order-0 Exp-Golomb of e + 1
    const uint32_t v = e + 1;
    const int nb = 31 - __clz(v);
    for (int i = 0; i < nb; ++i) bit(1);
    bit(0);
    for (int i = nb - 1; i >= 0; --i) bit((v >> i) & 1u);
  }
  __device__ void finish() {
    const unsigned long long top = low + range - 1;
    unsigned long long v = top;
    for (int k = 32; k >= 0; --k) {
      v = top & ~((1ull << k) - 1ull);
      if (v >= low) break;
    }
    low = v;
    for (int i = 0; i < 5; ++i) shift_low();
    if (!over)
      while (n > 0 && out[n - 1] == 0) --n;
  }
};

struct RcDec {
  uint32_t code, range, r;
  const uint8_t* p;
  int n, pos;

  __device__ uint32_t byte() {
    const uint32_t b = pos < n ? (uint32_t)p[pos] : 0u;
    ++pos;
    return b;
  }
  __device__ void init(const uint8_t* src, int len) {
    p = src; n = len; pos = 0; code = 0; range = 0xFFFFFFFFu; r = 0;
    for (int i = 0; i < 4; ++i) code = (code << 8) | byte();
  }
  __device__ uint32_t target() {
    r = range >> 16;
    const uint32_t q = code / r;
    return q < kTotal ? q : kTotal - 1;
  }
  __device__ void consume(uint32_t start, uint32_t freq) {
    code -= r * start;
    range = r * freq;
    while (range < (1u << 24)) {
      code = (code << 8) | byte();
      range <<= 8;
    }
  }
  __device__ uint32_t bit() {
    const uint32_t b = target() >= (1u << 15) ? 1u : 0u;
    consume(b << 15, 1u << 15);
    return b;
  }
  // order-0 Exp-Golomb; false for a prefix longer than any valid stream holds
  __device__ bool excess(uint32_t& e) {
    int nb = 0;
    while (bit()) {
      if (++nb > kMaxEgBits) return false;
    }
    unsigned long long v = 1;
    for (int i = 0; i < nb; ++i) v = (v << 1) | bit();
    e = (uint32_t)(v - 1);
    return nb <= 30;
  }
};

// symbol index of k = y_hat - m: 0 for the lower tail, kNsym - 1 for the upper one
__device__ __forceinline__ int sym_index(int k) {
  return k < -kA ? 0 : (k > kA ? kNsym - 1 : k + kA + 1);
}

// ---------------------------------------------------------------------------------------
// Encoder: fixed-point ARM of every latent (parallel), then one thread per row
// ---------------------------------------------------------------------------------------

template <int N, int NL>
__global__ void __launch_bounds__(256) k_codec_symbols(CodecGeo cg, Geo g,
                                                       const float* __restrict__ y,
                                                       const int2* __restrict__ offs,
                                                       int2* __restrict__ sym, int* flag) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cg.n_lat) return;
  int l = 0;
#pragma unroll
  for (int k = 1; k < kLevels; ++k) l = q >= cg.off[k] ? k : l;
  const int w = cg.w[l];
  const int i = (int)(q - cg.off[l]);
  const int r = i / w, x = i - r * w;
  const float* yl = y + g.off[l];
  int ctx[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const int2 o = offs[j];
    const int rr = r + o.x, xx = x + o.y;
    ctx[j] = (rr >= 0 && xx >= 0 && xx < w) ? (int)rintf(yl[(long long)rr * w + xx]) : 0;
  }
  const float yv = rintf(yl[(long long)r * w + x]);
  if (!(fabsf(yv) <= (float)kYLim)) {          // also catches NaN
    atomicOr(flag, 1);
    sym[q] = make_int2(0, 0);
    return;
  }
  int mu, s, t, m;
  arm_fixed<N, NL>(ctx, mu, s);
  table_of(mu, s, t, m);
  sym[q] = make_int2((int)yv - m, t);
}

__global__ void __launch_bounds__(128) k_codec_encode_rows(CodecGeo cg,
                                                           const int2* __restrict__ sym,
                                                           const uint16_t* __restrict__ tab,
                                                           uint8_t* rowbuf, int* row_len,
                                                           int* flag) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= cg.rows) return;
  int l = 0;
#pragma unroll
  for (int k = 1; k < kLevels; ++k) l = row >= cg.row0[k] ? k : l;
  const int r = row - cg.row0[l], w = cg.w[l];
  RcEnc enc;
  enc.init(rowbuf + cg.buf0[l] + (long long)r * cg.cap[l], cg.cap[l]);
  const int2* sr = sym + cg.off[l] + (long long)r * w;
  for (int x = 0; x < w; ++x) {
    const int2 sv = sr[x];
    const uint16_t* cr = tab + (long long)sv.y * kTabStride;
    const int idx = sym_index(sv.x);
    const uint32_t c0 = cum_at(cr, idx), c1 = cum_at(cr, idx + 1);
    enc.encode(c0, c1 - c0);
    if (idx == 0) enc.excess((uint32_t)(-kA - 1 - sv.x));
    else if (idx == kNsym - 1) enc.excess((uint32_t)(sv.x - kA - 1));
  }
  enc.finish();
  if (enc.over) atomicOr(flag, 2);
  row_len[row] = enc.over ? 0 : enc.n;
}

// one block per row: copy its bytes to their place in the packed stream
__global__ void __launch_bounds__(256) k_codec_pack(CodecGeo cg, const uint8_t* __restrict__ rowbuf,
                                                    const long long* __restrict__ dst_off,
                                                    const int* __restrict__ row_len,
                                                    uint8_t* __restrict__ out) {
  const int row = blockIdx.x;
  int l = 0;
#pragma unroll
  for (int k = 1; k < kLevels; ++k) l = row >= cg.row0[k] ? k : l;
  const uint8_t* src = rowbuf + cg.buf0[l] + (long long)(row - cg.row0[l]) * cg.cap[l];
  uint8_t* dst = out + dst_off[row];
  for (int i = threadIdx.x; i < row_len[row]; i += blockDim.x) dst[i] = src[i];
}

constexpr int kDecWarps = 4;                 // warps per block: one per scheduler
constexpr int kMaxPolls = 1 << 22;           // bounded wait on the predecessor band
constexpr int kRing = 64;                    // columns of the predecessor rows kept in smem

// The causal offsets (dy, dx) of N = 8, 16, 24 in raster order (the N nearest causal
// neighbours, ties by smaller |dy| then smaller dx) as compile-time tables: the decoder
// keeps recent values in registers and needs each offset's register index statically.
// The host checks them against the offsets the library builds at run time.
template <int N> __host__ __device__ constexpr int off_dy(int j);
template <int N> __host__ __device__ constexpr int off_dx(int j);
template <> __host__ __device__ constexpr int off_dy<8>(int j) {
  constexpr int t[8] = {-2, -1, -1, -1, -1, -1, 0, 0};
  return t[j];
}
template <> __host__ __device__ constexpr int off_dx<8>(int j) {
  constexpr int t[8] = {0, -2, -1, 0, 1, 2, -2, -1};
  return t[j];
}
template <> __host__ __device__ constexpr int off_dy<16>(int j) {
  constexpr int t[16] = {-3, -2, -2, -2, -2, -2, -1, -1, -1, -1, -1, -1, -1, 0, 0, 0};
  return t[j];
}
template <> __host__ __device__ constexpr int off_dx<16>(int j) {
  constexpr int t[16] = {0, -2, -1, 0, 1, 2, -3, -2, -1, 0, 1, 2, 3, -3, -2, -1};
  return t[j];
}
template <> __host__ __device__ constexpr int off_dy<24>(int j) {
  constexpr int t[24] = {-4, -3, -3, -3, -3, -3, -2, -2, -2, -2, -2, -2,
                         -2, -1, -1, -1, -1, -1, -1, -1, 0, 0, 0, 0};
  return t[j];
}
template <> __host__ __device__ constexpr int off_dx<24>(int j) {
  constexpr int t[24] = {0, -2, -1, 0, 1, 2, -3, -2, -1, 0, 1, 2,
                         3, -3, -2, -1, 0, 1, 2, 3, -4, -3, -2, -1};
  return t[j];
}
// wavefront lag: max over dy < 0 of ceil((dx + 1) / -dy)
template <int N> __host__ __device__ constexpr int lag_of() {
  int lag = 1;
  for (int j = 0; j < N; ++j)
    if (off_dy<N>(j) < 0) {
      const int d = -off_dy<N>(j), need = (off_dx<N>(j) + 1 + d - 1) / d;
      lag = need > lag ? need : lag;
    }
  return lag;
}
// rows above the current one that the context reaches
template <int N> __host__ __device__ constexpr int reach_of() {
  int r = 0;
  for (int j = 0; j < N; ++j) r = -off_dy<N>(j) > r ? -off_dy<N>(j) : r;
  return r;
}
// register index, in the window of the row the offset points to, of the value it reads:
// a lane's window entry k holds its row's value at (its position one step ago) - k
template <int N> __host__ __device__ constexpr int win_idx(int j) {
  return -lag_of<N>() * off_dy<N>(j) - 1 - off_dx<N>(j);
}
template <int N> __host__ __device__ constexpr int win_of() {
  int m = 0;
  for (int j = 0; j < N; ++j) m = win_idx<N>(j) > m ? win_idx<N>(j) : m;
  return m + 1;
}

// The fixed-point ARM with one row's LinR layers split over its P lanes: lane part p
// computes outputs [p N / P, (p + 1) N / P) from shared-memory weights (each LinR
// matrix transposed, as in the constant bank), the ReLU terms are exchanged by shuffles
// and every lane applies all of them, so that the activations stay replicated; the two
// outputs are computed whole by every lane.  Integer sums: the same bits as arm_fixed.
template <int N, int NL, int P>
__device__ __forceinline__ void arm_fixed_split(const int (&ctx)[N], const int* s_w, int p,
                                                int lane, int& mu, int& s) {
  constexpr int OPL = N / P;                 // outputs per lane, loaded as int2 pairs
  static_assert(N % (2 * P) == 0, "outputs per lane must be even");
  int a[N];
#pragma unroll
  for (int j = 0; j < N; ++j) a[j] = min(max(ctx[j], -kCtxLim), kCtxLim) * (1 << kQFrac);
  const int base = lane & ~(P - 1);
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const int* Wt = s_w + i * (N * N + N);
    const int* b = Wt + N * N;
    int acc[OPL];
#pragma unroll
    for (int k = 0; k < OPL; ++k) acc[k] = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int2* wr = reinterpret_cast<const int2*>(Wt + j * N + p * OPL);
#pragma unroll
      for (int k = 0; k < OPL / 2; ++k) {
        const int2 wv = wr[k];
        acc[2 * k] += wv.x * a[j];
        acc[2 * k + 1] += wv.y * a[j];
      }
    }
    int z[OPL];
#pragma unroll
    for (int k = 0; k < OPL; ++k) z[k] = max(sat(((acc[k] + 128) >> kQFrac) + b[p * OPL + k]), 0);
#pragma unroll
    for (int o = 0; o < N; ++o)
      a[o] = sat(a[o] + __shfl_sync(0xFFFFFFFFu, z[o % OPL], base | (o / OPL)));
  }
  const int* W = s_w + NL * (N * N + N);
  const int* b = W + 2 * N;
  int acc0 = 0, acc1 = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    acc0 += W[j] * a[j];
    acc1 += W[N + j] * a[j];
  }
  mu = sat(((acc0 + 128) >> kQFrac) + b[0]);
  s = sat(((acc1 + 128) >> kQFrac) + b[1]);
}

// ---------------------------------------------------------------------------------------
// Decoder.  The rows of a level form bands of 32 / P rows; a warp decodes one band at a
// time, the P lanes of row r0 + i together (they split the ARM, see
// arm_fixed_split, and all run the row's range decoder), row r0 + i decoding position x
// at the band's local step x + lag i: then every causal neighbour inside the band was
// decoded at an earlier step.  Each lane keeps its row's last win_of<N>() values in
// registers (0 before the row starts and after it ends); a neighbour in row
// r0 + i + dy comes from the registers of the same part of that row by a warp shuffle.
// Neighbours in the rows above the band come from a shared-memory ring of those rows,
// refilled every kFill steps (from L2) once the band above has completed enough steps;
// the band above publishes its completed step count every 4 steps (release) and the
// refill waits for it (acquire, bounded).  All levels run at once; warps take bands in
// increasing order, which keeps the waits acyclic, and the cooperative launch keeps every
// warp resident.
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr int kFill = 8;                     // steps between ring refills (16: slower)

template <int N, int NL, int P>
__global__ void __launch_bounds__(kDecWarps * 32) k_codec_decode(
    CodecGeo cg, const uint16_t* __restrict__ tab, const uint8_t* __restrict__ bytes,
    const long long* __restrict__ row_off, const int* __restrict__ row_len, int* planes,
    int* progress, int* flag, int max_polls, int stall_band) {
  constexpr int LAG = lag_of<N>(), R = reach_of<N>(), WIN = win_of<N>();
  constexpr int NW = NL * (N * N + N) + 2 * N + 2;
  constexpr int kBandRows = 32 / P;         // cg.band_rows, set by the host to match
  extern __shared__ __align__(16) uint16_t s_tab[];
  __shared__ int s_ring[kDecWarps][R][kRing];
  __shared__ __align__(16) int s_w[NW];
  for (int i = threadIdx.x; i < kNtab * kTabStride / 8; i += blockDim.x)
    reinterpret_cast<uint4*>(s_tab)[i] = reinterpret_cast<const uint4*>(tab)[i];
  for (int i = threadIdx.x; i < NW; i += blockDim.x) s_w[i] = c_qarm[i];
  __syncthreads();

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ri = lane / P, part = lane % P;
  int (*ring)[kRing] = s_ring[wid];
  const int tw = gridDim.x * kDecWarps;
  for (int gb = blockIdx.x * kDecWarps + wid; gb < cg.bands; gb += tw) {
    int l = 0;
#pragma unroll
    for (int k = 1; k < kLevels; ++k) l = gb >= cg.band0[k] ? k : l;
    const int b = gb - cg.band0[l];
    const int h = cg.h[l], w = cg.w[l];
    const int r0 = kBandRows * b;
    const int nr = min(kBandRows, h - r0);
    const int r = r0 + ri;
    int* plane = planes + cg.off[l];
    const int nsteps = w + LAG * (nr - 1);
    const int pred_steps = w + LAG * (kBandRows - 1);   // a predecessor band is full
    int win[WIN];
#pragma unroll
    for (int k = 0; k < WIN; ++k) win[k] = 0;
    RcDec dec;
    dec.init(bytes, 0);
    bool bad = false;
    for (int st = 0; st < nsteps; ++st) {
      if (st % kFill == 0) {                    // refill the ring of the rows above
        if (b > 0) {
          const int need = min(st + 2 * kFill + LAG * (kBandRows - 1), pred_steps);
          int v = 0;
          if (lane == 0) {
            for (int tries = 0; tries < max_polls; ++tries) {
              v = ld_acquire(progress + gb - 1);
              if (v >= need) break;
              __nanosleep(64);
            }
          }
          v = __shfl_sync(0xFFFFFFFFu, v, 0);
          if (v < need) {                       // the band above stalled: give up
            if (lane == 0) atomicOr(flag, 8);
            return;
          }
        }
        __syncwarp();
#pragma unroll
        for (int t = lane; t < 4 * kFill; t += 32) {
          const int m = t / kFill + 1, rr = r0 - m;
          if (m <= R) {
            const int c = st + kFill + (t % kFill);
            ring[m - 1][c % kRing] = (rr >= 0 && c < w) ? __ldcg(plane + (long long)rr * w + c) : 0;
            if (st == 0) {
              const int c0 = t % kFill;
              ring[m - 1][c0] = (rr >= 0 && c0 < w) ? __ldcg(plane + (long long)rr * w + c0) : 0;
            }
          }
        }
        __syncwarp();
      }
      const int x = st - LAG * ri;
      int ctx[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int dy = off_dy<N>(j), dx = off_dx<N>(j);
        int v;
        if (dy == 0) {
          v = win[-1 - dx];
        } else {
          v = __shfl_up_sync(0xFFFFFFFFu, win[win_idx<N>(j)], -dy * P);
          if (ri + dy < 0) v = ring[-(ri + dy) - 1][(x + dx) & (kRing - 1)];
        }
        ctx[j] = (r + dy >= 0 && x + dx >= 0 && x + dx < w) ? v : 0;
      }
      int mu, s;
      if constexpr (P == 1)
        arm_fixed<N, NL>(ctx, mu, s);                          // weights as bank operands
      else
        arm_fixed_split<N, NL, P>(ctx, s_w, part, lane, mu, s);   // shuffles inside
      int val = 0;
      if (ri < nr && x >= 0 && x < w) {
        if (x == 0) dec.init(bytes + row_off[cg.row0[l] + r], row_len[cg.row0[l] + r]);
        int t, m;
        table_of(mu, s, t, m);
        const uint16_t* cr = s_tab + t * kTabStride;
        const uint32_t q = dec.target();
        // largest idx with cum[idx] <= q: first the symbol k = 0 (the table's most
        // probable region), then a binary search on the side q falls
        int lo = kA + 1, hi = kA + 2;
        if ((uint32_t)cr[lo] > q) { hi = lo; lo = 0; }
        else if (q >= (uint32_t)cr[hi]) { lo = hi; hi = kNsym; }
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if ((uint32_t)cr[mid] <= q) lo = mid; else hi = mid;
        }
        const uint32_t c0 = cum_at(cr, lo), c1 = cum_at(cr, lo + 1);
        dec.consume(c0, c1 - c0);
        int k = lo - kA - 1;
        if (lo == 0 || lo == kNsym - 1) {
          uint32_t e = 0;
          if (!dec.excess(e)) bad = true;
          k = lo == 0 ? -kA - 1 - (int)e : kA + 1 + (int)e;
        }
        val = m + k;
        if (part == 0) plane[(long long)r * w + x] = val;
      }
#pragma unroll
      for (int k = WIN - 1; k > 0; --k) win[k] = win[k - 1];
      win[0] = val;
      if ((st & 3) == 3 || st == nsteps - 1) {
        __syncwarp();
        if (lane == 0 && gb != stall_band) st_release(progress + gb, st + 1);
      }
    }
    if (bad) atomicOr(flag, 4);
  }
}

template <int N>
cudaError_t symbols_t(const CodecGeo& cg, const Geo& g, const float* y, const int2* offs,
                      int NL, int2* sym, int* flag, cudaStream_t st) {
  const int blocks = (int)((cg.n_lat + 255) / 256);
  if (NL == 1) k_codec_symbols<N, 1><<<blocks, 256, 0, st>>>(cg, g, y, offs, sym, flag);
  else k_codec_symbols<N, 2><<<blocks, 256, 0, st>>>(cg, g, y, offs, sym, flag);
  return cudaGetLastError();
}

template <int N, int NL, int P>
cudaError_t decode_t(const CodecGeo& cg, const uint16_t* tab, const uint8_t* bytes,
                     const long long* row_off, const int* row_len, int* planes, int* progress,
                     int* flag, cudaStream_t st) {
  if (cg.band_rows != 32 / P) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kNtab * kTabStride * sizeof(uint16_t);
  auto kern = k_codec_decode<N, NL, P>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDecWarps * 32, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int want = (cg.bands + kDecWarps - 1) / kDecWarps;
  const int grid = want < sms * per_sm ? want : sms * per_sm;
  // failure injection for the bounded waits (tests): a band that never publishes its
  // progress, and a shorter wait bound
  int max_polls = kMaxPolls, stall_band = -1;
  if (const char* env = getenv("CC_DECODE_MAX_POLLS")) max_polls = std::max(1, atoi(env));
  if (const char* env = getenv("CC_DECODE_STALL_BAND")) stall_band = atoi(env);
  void* args[] = {(void*)&cg, (void*)&tab, (void*)&bytes, (void*)&row_off, (void*)&row_len,
                  (void*)&planes, (void*)&progress, (void*)&flag, (void*)&max_polls,
                  (void*)&stall_band};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kDecWarps * 32), args,
                                     smem, st);
}

std::vector<uint16_t> g_tables;
std::once_flag g_tables_once;

void build_tables() {
  g_tables.assign((size_t)kNtab * kTabStride, 0);
  for (int j = 0; j < kNscale; ++j) {
    for (int fi = 0; fi < kNmu; ++fi) {
      const double b = std::exp((double)kLogbLoQ / 256.0 + ((double)j + 0.5) / 8.0);
      const double f = ((double)fi + 0.5) / kNmu;
      auto F = [&](double x) {
        const double z = (x - f) / b;
        return z < 0.0 ? 0.5 * std::exp(z) : 1.0 - 0.5 * std::exp(-z);
      };
      double mass[kNsym];
      mass[0] = F(-kA - 0.5);
      for (int k = -kA; k <= kA; ++k) mass[k + kA + 1] = F(k + 0.5) - F(k - 0.5);
      mass[kNsym - 1] = 1.0 - F(kA + 0.5);
      long long freq[kNsym], sum = 0;
      for (int i = 0; i < kNsym; ++i) {
        freq[i] = 1 + (long long)std::floor(mass[i] * (double)(kTotal - kNsym));
        sum += freq[i];
      }
      int top = 0;
      for (int i = 1; i < kNsym; ++i) top = freq[i] > freq[top] ? i : top;
      freq[top] += (long long)kTotal - sum;
      uint16_t* row = g_tables.data() + (size_t)(j * kNmu + fi) * kTabStride;
      long long c = 0;
      row[0] = 0;
      for (int i = 0; i + 1 < kNsym; ++i) {
        c += freq[i];
        row[i + 1] = (uint16_t)c;
      }
    }
  }
}

}  // namespace

const std::vector<uint16_t>& codec_tables() {
  std::call_once(g_tables_once, build_tables);
  return g_tables;
}

size_t codec_table_bytes() { return (size_t)kNtab * kTabStride * sizeof(uint16_t); }

bool codec_quantize_arm(const float* params, int N, int NL, int32_t* q) {
  // Q8 rounding half to even; weights clamped to +-2^11, biases to +-2^15
  auto quant = [](float p, long long lim, int32_t& out) {
    const double d = std::nearbyint((double)p * 256.0);
    if (!std::isfinite(d)) return false;
    out = (int32_t)(d < (double)-lim ? -lim : (d > (double)lim ? lim : (long long)d));
    return true;
  };
  int k = 0;
  bool ok = true;
  for (int i = 0; i < NL; ++i)
    for (int j = 0; j < N * N + N; ++j, ++k) ok &= quant(params[k], j < N * N ? kWLim : kActLim, q[k]);
  for (int j = 0; j < 2 * N + 2; ++j, ++k) ok &= quant(params[k], j < 2 * N ? kWLim : kActLim, q[k]);
  return ok;
}

bool codec_offsets_match(const int2* offs, int N) {
  for (int j = 0; j < N; ++j) {
    int dy = 0, dx = 0;
    if (N == 8) { dy = off_dy<8>(j); dx = off_dx<8>(j); }
    else if (N == 16) { dy = off_dy<16>(j); dx = off_dx<16>(j); }
    else if (N == 24) { dy = off_dy<24>(j); dx = off_dx<24>(j); }
    else return false;
    if (offs[j].x != dy || offs[j].y != dx) return false;
  }
  return true;
}

bool codec_arm_in_range(const int32_t* q, int N, int NL) {
  int k = 0;
  for (int i = 0; i < NL; ++i)
    for (int j = 0; j < N * N + N; ++j, ++k)
      if (std::abs(q[k]) > (j < N * N ? kWLim : kActLim)) return false;
  for (int j = 0; j < 2 * N + 2; ++j, ++k)
    if (std::abs(q[k]) > (j < 2 * N ? kWLim : kActLim)) return false;
  return true;
}

int codec_row_capacity(int w) { return 8 * w + 16; }

cudaError_t codec_upload_arm(const int32_t* q, int N, int NL, cudaStream_t st) {
  // the constant bank holds each LinR weight matrix transposed (the device walks it along
  // the outputs); biases and the output layer as in the flat order
  static thread_local std::vector<int32_t> bank;
  const int n = NL * (N * N + N) + 2 * N + 2;
  bank.assign(q, q + n);
  for (int i = 0; i < NL; ++i) {
    const int32_t* W = q + i * (N * N + N);
    int32_t* Wt = bank.data() + i * (N * N + N);
    for (int o = 0; o < N; ++o)
      for (int j = 0; j < N; ++j) Wt[j * N + o] = W[o * N + j];
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_qarm, bank.data(), (size_t)n * sizeof(int32_t), 0,
                                          cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);   // the staging vector is reused by the next call
}

int codec_max_arm_ints() { return kMaxQArm; }

cudaError_t codec_symbols(const CodecGeo& cg, const Geo& g, const float* y, const int2* offs,
                          int N, int NL, int2* sym, int* flag, cudaStream_t st) {
  if (NL != 1 && NL != 2) return cudaErrorInvalidValue;
  switch (N) {
    case 8: return symbols_t<8>(cg, g, y, offs, NL, sym, flag, st);
    case 16: return symbols_t<16>(cg, g, y, offs, NL, sym, flag, st);
    case 24: return symbols_t<24>(cg, g, y, offs, NL, sym, flag, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t codec_encode_rows(const CodecGeo& cg, const int2* sym, const uint16_t* tab,
                              uint8_t* rowbuf, int* row_len, int* flag, cudaStream_t st) {
  k_codec_encode_rows<<<(cg.rows + 127) / 128, 128, 0, st>>>(cg, sym, tab, rowbuf, row_len, flag);
  return cudaGetLastError();
}

cudaError_t codec_pack(const CodecGeo& cg, const uint8_t* rowbuf, const long long* dst_off,
                       const int* row_len, uint8_t* out, cudaStream_t st) {
  k_codec_pack<<<cg.rows, 256, 0, st>>>(cg, rowbuf, dst_off, row_len, out);
  return cudaGetLastError();
}

cudaError_t codec_decode(const CodecGeo& cg, int N, int NL, const uint16_t* tab,
                         const uint8_t* bytes, const long long* row_off, const int* row_len,
                         int* planes, int* progress, int* flag, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(progress, 0, (size_t)cg.bands * sizeof(int), st);
  if (e != cudaSuccess) return e;
#define CC_DECODE_CASE(n, nl, p)                                                              \
  if (N == n && NL == nl && parts == p)                                                       \
    return decode_t<n, nl, p>(cg, tab, bytes, row_off, row_len, planes, progress, flag, st);
  const int parts = 32 / cg.band_rows;
  CC_DECODE_CASE(8, 1, 1) CC_DECODE_CASE(8, 2, 1) CC_DECODE_CASE(8, 1, 2) CC_DECODE_CASE(8, 2, 2)
  CC_DECODE_CASE(16, 1, 2) CC_DECODE_CASE(16, 2, 2)
  CC_DECODE_CASE(24, 1, 2) CC_DECODE_CASE(24, 2, 2) CC_DECODE_CASE(24, 1, 1) CC_DECODE_CASE(24, 2, 1)
#undef CC_DECODE_CASE
  return cudaErrorInvalidValue;
}

// integer latent planes (flat order) -> float latent buffer (padded layout)
__global__ void __launch_bounds__(256) k_codec_to_float(CodecGeo cg, Geo g, const int* __restrict__ planes,
                                                        float* __restrict__ y) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cg.n_lat) return;
  int l = 0;
#pragma unroll
  for (int k = 1; k < kLevels; ++k) l = q >= cg.off[k] ? k : l;
  y[g.off[l] + (q - cg.off[l])] = (float)planes[q];
}

cudaError_t codec_to_float(const CodecGeo& cg, const Geo& g, const int* planes, float* y,
                           cudaStream_t st) {
  k_codec_to_float<<<(int)((cg.n_lat + 255) / 256), 256, 0, st>>>(cg, g, planes, y);
  return cudaGetLastError();
}

// Lanes per row of the decoder, measured on GB300 at 2048 x 2048 (latent decode): the
// 8-input ARM is fastest with one lane per row and its weights as constant-bank operands
// (13.3 ms; 14.1 with two lanes), the 16- and 24-input ARMs with two lanes (24.9 ms for
// N = 24; 37.2 with one, 29.9 with four).  CC_DECODE_PARTS (1 or 2; 1 only for N = 8, 24)
// overrides it.
int codec_decode_parts(int N) {
  int p = N == 8 ? 1 : 2;
  if (const char* env = getenv("CC_DECODE_PARTS")) {
    const int v = atoi(env);
    if (v == 2 || (v == 1 && N != 16)) p = v;
  }
  return p;
}

CodecGeo codec_geo(const Geo& g, int band_rows) {
  CodecGeo cg;
  cg.band_rows = band_rows;
  long long off = 0, buf = 0;
  int rows = 0, bands = 0;
  for (int l = 0; l < kLevels; ++l) {
    cg.h[l] = g.h[l];
    cg.w[l] = g.w[l];
    cg.off[l] = off;
    cg.row0[l] = rows;
    cg.cap[l] = codec_row_capacity(g.w[l]);
    cg.buf0[l] = buf;
    cg.band0[l] = bands;
    bands += (g.h[l] + band_rows - 1) / band_rows;
    off += (long long)g.h[l] * g.w[l];
    rows += g.h[l];
    buf += (long long)g.h[l] * cg.cap[l];
  }
  cg.n_lat = off;
  cg.rows = rows;
  cg.bands = bands;
  cg.buf_bytes = buf;
  return cg;
}

}  // namespace cc
