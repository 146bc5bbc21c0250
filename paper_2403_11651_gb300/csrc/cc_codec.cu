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
//   ARM:    weights and biases rounded half-to-even to Q8 (8 fractional bits), weights
//           clamped to +-2^20, biases to +-2^28; inputs are integer latents times 256; a
//           layer computes z = ((sum_j W[o, j] a[j]) + 128) >> 8 + b[o] in 64-bit integers,
//           saturated to +-2^28; a LinR layer outputs a[o] + max(z, 0), saturated; the
//           output layer gives (mu_q, s_q) in Q8.
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
#include <cmath>
#include <mutex>
#include <vector>

#include "cc_internal.cuh"

namespace cc {

namespace {

constexpr int kQFrac = 8;
constexpr long long kWLim = 1ll << 20;
constexpr long long kActLim = 1ll << 28;
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

__device__ __forceinline__ long long sat(long long v) {
  return v < -kActLim ? -kActLim : (v > kActLim ? kActLim : v);
}

// (mu_q, s_q) of the fixed-point ARM for the integer context ctx
template <int N>
__device__ __forceinline__ void arm_fixed(const int (&ctx)[N], int NL, long long& mu,
                                          long long& s) {
  int a[N];
#pragma unroll
  for (int j = 0; j < N; ++j) a[j] = ctx[j] * (1 << kQFrac);
  for (int i = 0; i < NL; ++i) {
    const int* W = c_qarm + i * (N * N + N);
    const int* b = W + N * N;
    int z[N];
#pragma unroll
    for (int o = 0; o < N; ++o) {
      long long acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += (long long)W[o * N + j] * a[j];
      const long long v = sat(((acc + 128) >> kQFrac) + b[o]);
      z[o] = (int)(v > 0 ? v : 0);
    }
#pragma unroll
    for (int o = 0; o < N; ++o) a[o] = (int)sat((long long)a[o] + z[o]);
  }
  const int* W = c_qarm + NL * (N * N + N);
  const int* b = W + 2 * N;
  long long acc0 = 0, acc1 = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    acc0 += (long long)W[j] * a[j];
    acc1 += (long long)W[N + j] * a[j];
  }
  mu = sat(((acc0 + 128) >> kQFrac) + b[0]);
  s = sat(((acc1 + 128) >> kQFrac) + b[1]);
}

// table number and integer part of mu
__device__ __forceinline__ void table_of(long long mu, long long s, int& t, int& m) {
  long long j = (s - kLogbLoQ) >> 5;
  j = j < 0 ? 0 : (j > kNscale - 1 ? kNscale - 1 : j);
  t = (int)j * kNmu + (int)((mu & 255) >> 5);
  m = (int)(mu >> kQFrac);
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

template <int N>
__global__ void __launch_bounds__(256) k_codec_symbols(CodecGeo cg, Geo g,
                                                       const float* __restrict__ y,
                                                       const int2* __restrict__ offs, int NL,
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
  long long mu, s;
  arm_fixed<N>(ctx, NL, mu, s);
  int t, m;
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

// ---------------------------------------------------------------------------------------
// Decoder: one block per level; row r decodes position x at step x + lag r, so that every
// causal neighbour was decoded at an earlier step.  Rows are dealt to threads modulo the
// block size, which is at least the number of rows active at one step (ceil(w / lag)):
// a thread then holds one row's coder at a time.
// ---------------------------------------------------------------------------------------

template <int N>
__global__ void __launch_bounds__(1024) k_codec_decode(CodecGeo cg, const int2* __restrict__ offs,
                                                       int NL, int lag,
                                                       const uint16_t* __restrict__ tab,
                                                       const uint8_t* __restrict__ bytes,
                                                       const long long* __restrict__ row_off,
                                                       const int* __restrict__ row_len,
                                                       int* planes, int* flag) {
  extern __shared__ __align__(16) uint16_t s_tab[];
  __shared__ int2 s_offs[N];
  for (int i = threadIdx.x; i < kNtab * kTabStride / 8; i += blockDim.x)
    reinterpret_cast<uint4*>(s_tab)[i] = reinterpret_cast<const uint4*>(tab)[i];
  if (threadIdx.x < N) s_offs[threadIdx.x] = offs[threadIdx.x];
  __syncthreads();

  const int l = blockIdx.x;
  const int h = cg.h[l], w = cg.w[l];
  int* plane = planes + cg.off[l];
  const int T = blockDim.x, tid = threadIdx.x;
  const long long steps = (long long)w + (long long)lag * (h - 1);
  RcDec dec;
  dec.init(bytes, 0);
  bool bad = false;
  for (long long st = 0; st < steps; ++st) {
    const long long rmax_l = st / lag < h - 1 ? st / lag : h - 1;
    const int rmax = (int)rmax_l;
    if (tid <= rmax) {
      const int r = rmax - (rmax - tid) % T;
      const long long xl = st - (long long)lag * r;
      if (xl < w) {
        const int x = (int)xl;
        const int grow = cg.row0[l] + r;
        if (x == 0) dec.init(bytes + row_off[grow], row_len[grow]);
        int ctx[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int2 o = s_offs[j];
          const int rr = r + o.x, xx = x + o.y;
          ctx[j] = (rr >= 0 && xx >= 0 && xx < w) ? plane[(long long)rr * w + xx] : 0;
        }
        long long mu, s;
        arm_fixed<N>(ctx, NL, mu, s);
        int t, m;
        table_of(mu, s, t, m);
        const uint16_t* cr = s_tab + t * kTabStride;
        const uint32_t q = dec.target();
        int lo = 0, hi = kNsym;            // largest idx with cum[idx] <= q
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
        plane[(long long)r * w + x] = m + k;
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(flag, 4);
}

template <int N>
cudaError_t symbols_t(const CodecGeo& cg, const Geo& g, const float* y, const int2* offs,
                      int NL, int2* sym, int* flag, cudaStream_t st) {
  const int blocks = (int)((cg.n_lat + 255) / 256);
  k_codec_symbols<N><<<blocks, 256, 0, st>>>(cg, g, y, offs, NL, sym, flag);
  return cudaGetLastError();
}

template <int N>
cudaError_t decode_t(const CodecGeo& cg, const int2* offs, int NL, int lag, const uint16_t* tab,
                     const uint8_t* bytes, const long long* row_off, const int* row_len,
                     int* planes, int* flag, int threads, cudaStream_t st) {
  const size_t smem = (size_t)kNtab * kTabStride * sizeof(uint16_t);
  cudaError_t e = cudaFuncSetAttribute(k_codec_decode<N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_codec_decode<N><<<kLevels, threads, smem, st>>>(cg, offs, NL, lag, tab, bytes, row_off,
                                                    row_len, planes, flag);
  return cudaGetLastError();
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
  // Q8 rounding half to even; weights clamped to +-2^20, biases to +-2^28
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

int codec_lag(const int2* offs, int N) {
  int lag = 1;
  for (int j = 0; j < N; ++j) {
    const int dy = offs[j].x, dx = offs[j].y;
    if (dy < 0) {
      const int need = (dx + 1 + (-dy) - 1) / (-dy);   // ceil((dx + 1) / -dy), dx + 1 >= 0
      lag = need > lag ? need : lag;
    }
  }
  return lag;
}

int codec_row_capacity(int w) { return 8 * w + 16; }

cudaError_t codec_upload_arm(const int32_t* q, int n, cudaStream_t st) {
  return cudaMemcpyToSymbolAsync(c_qarm, q, (size_t)n * sizeof(int32_t), 0,
                                 cudaMemcpyHostToDevice, st);
}

int codec_max_arm_ints() { return kMaxQArm; }

cudaError_t codec_symbols(const CodecGeo& cg, const Geo& g, const float* y, const int2* offs,
                          int N, int NL, int2* sym, int* flag, cudaStream_t st) {
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

cudaError_t codec_decode(const CodecGeo& cg, const int2* offs, int N, int NL, int lag,
                         const uint16_t* tab, const uint8_t* bytes, const long long* row_off,
                         const int* row_len, int* planes, int* flag, int threads,
                         cudaStream_t st) {
  switch (N) {
    case 8: return decode_t<8>(cg, offs, NL, lag, tab, bytes, row_off, row_len, planes, flag, threads, st);
    case 16: return decode_t<16>(cg, offs, NL, lag, tab, bytes, row_off, row_len, planes, flag, threads, st);
    case 24: return decode_t<24>(cg, offs, NL, lag, tab, bytes, row_off, row_len, planes, flag, threads, st);
    default: return cudaErrorInvalidValue;
  }
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

CodecGeo codec_geo(const Geo& g) {
  CodecGeo cg;
  long long off = 0, buf = 0;
  int rows = 0;
  for (int l = 0; l < kLevels; ++l) {
    cg.h[l] = g.h[l];
    cg.w[l] = g.w[l];
    cg.off[l] = off;
    cg.row0[l] = rows;
    cg.cap[l] = codec_row_capacity(g.w[l]);
    cg.buf0[l] = buf;
    off += (long long)g.h[l] * g.w[l];
    rows += g.h[l];
    buf += (long long)g.h[l] * cg.cap[l];
  }
  cg.n_lat = off;
  cg.rows = rows;
  cg.buf_bytes = buf;
  return cg;
}

}  // namespace cc
