// cc_rate_bits_noalloc: the rate term of eq. (1) for a caller-supplied quantised latent
// pyramid, computed without allocating any device memory.
//
// Some callers of a coding library cannot allocate: for instance a decoder embedded in a
// process whose device memory is entirely owned by another allocator (a framework's
// caching allocator or a fixed pool carved up at start-up), or a real-time service that
// must never call cudaMalloc / cudaFree once it runs.  This entry point serves them: the
// caller passes its inputs and output, and the only scratch the kernels need -- one
// partial sum per tile of 128 latents and the final total -- lives in a file-scope
// __device__ array that every device loading the library holds until the process exits.
//
// It is a variant of the forward half of the ARM kernel in cc_arm.cu: the same context
// rule, MLP and Laplace bin mass, but gathering straight from the caller's flat latent
// array with bounds checks, one CTA per tile, and summing the tiles in a fixed order.
#include <cstdio>
#include <cstdlib>

#include "cc_internal.cuh"
#include "cc_laplace.cuh"
#include "../../include/coolchic.h"

namespace cc {
namespace {

constexpr int kNaThreads = 128;                       // latents per tile, one per thread
constexpr int kNaMaxTiles = CC_NOALLOC_MAX_TILES;
constexpr int kNaMaxDevices = 64;
constexpr int kNaMaxN = 24;

struct NoAllocScratch {
  float tile_bits[kNaMaxTiles];  // bits of each tile, every entry rewritten by each call
  double total;                  // sum of the tiles, written by each call
};

// The scratch.  In host code this name is only a stand-in for the device object: its
// device address comes from cudaGetSymbolAddress, once per device (see scratch_of).
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__constant__ float c_arm_na[2 * (kNaMaxN * kNaMaxN + kNaMaxN) + 2 * kNaMaxN + 2];
__constant__ int2 c_off_na[kNaMaxN];

struct NaGeo {
  int h[kLevels], w[kLevels];
  int tile0[kLevels + 1];      // first tile of each level; tile0[L] = number of tiles
  long long foff[kLevels];     // offset of each level in the flat latent array
};

template <int N, int NL>
__global__ void __launch_bounds__(kNaThreads) k_rate_noalloc(const float* __restrict__ yhat,
                                                             NaGeo g, float* tile_bits) {
  constexpr int LW = N * N + N, OW = NL * LW, OB = OW + 2 * N;
  const int tile = blockIdx.x;
  int l = 0;
  while (l < kLevels - 1 && tile >= g.tile0[l + 1]) ++l;
  const int w = g.w[l], n = g.h[l] * w;
  const int i = (tile - g.tile0[l]) * kNaThreads + threadIdx.x;
  const bool valid = i < n;
  const float* plane = yhat + g.foff[l];
  int r = 0, c = 0;
  if (valid) { r = i / w; c = i - r * w; }
  float h[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int2 o = c_off_na[k];
    const int rr = r + o.x, cc = c + o.y;
    h[k] = (valid && rr >= 0 && cc >= 0 && cc < w) ? __ldg(plane + rr * w + cc) : 0.f;
  }
  const float yq = valid ? __ldg(plane + i) : 0.f;
#pragma unroll
  for (int L = 0; L < NL; ++L) {
    float z[N];
#pragma unroll
    for (int o = 0; o < N; ++o) z[o] = c_arm_na[L * LW + N * N + o];
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int o = 0; o < N; ++o) z[o] = fmaf(c_arm_na[L * LW + o * N + k], h[k], z[o]);
#pragma unroll
    for (int o = 0; o < N; ++o) h[o] += fmaxf(z[o], 0.f);
  }
  float mu = c_arm_na[OB], s = c_arm_na[OB + 1];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    mu = fmaf(c_arm_na[OW + k], h[k], mu);
    s = fmaf(c_arm_na[OW + N + k], h[k], s);
  }
  float bits = valid ? laplace_bits(yq, mu, s).bits : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, o);
  __shared__ float s_w[kNaThreads / 32];
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = bits;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < kNaThreads / 32; ++k) t += s_w[k];
    tile_bits[tile] = t;
  }
}

// Sum of the n tile partials, in double, in a fixed order.
__global__ void __launch_bounds__(256) k_sum_tiles(const float* tile_bits, int n, double* total) {
  __shared__ double s[256];
  double a = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) a += (double)tile_bits[k];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s[0];
}

// Device address of the scratch on the current device, looked up once per device.
NoAllocScratch* g_scratch_ptr[kNaMaxDevices] = {};

cudaError_t scratch_of(int dev, NoAllocScratch** out) {
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// The n nearest causal neighbours, ties by smaller |dy| then smaller dx, in raster order
// (fixed-size arrays: nothing is allocated).
int causal_offsets_fixed(int n, int2* out) {
  int dy[84], dx[84], m = 0;
  for (int y = -6; y <= 0; ++y)
    for (int x = -6; x <= 6; ++x)
      if (y < 0 || x < 0) { dy[m] = y; dx[m] = x; ++m; }
  auto less_near = [&](int a, int b) {
    const int da = dy[a] * dy[a] + dx[a] * dx[a], db = dy[b] * dy[b] + dx[b] * dx[b];
    if (da != db) return da < db;
    if (abs(dy[a]) != abs(dy[b])) return abs(dy[a]) < abs(dy[b]);
    return dx[a] < dx[b];
  };
  int idx[84];
  for (int k = 0; k < m; ++k) idx[k] = k;
  for (int k = 1; k < m; ++k)
    for (int j = k; j > 0 && less_near(idx[j], idx[j - 1]); --j) {
      const int t = idx[j]; idx[j] = idx[j - 1]; idx[j - 1] = t;
    }
  for (int k = 1; k < n; ++k)  // raster order of the n chosen
    for (int j = k; j > 0 && (dy[idx[j]] < dy[idx[j - 1]] ||
                              (dy[idx[j]] == dy[idx[j - 1]] && dx[idx[j]] < dx[idx[j - 1]])); --j) {
      const int t = idx[j]; idx[j] = idx[j - 1]; idx[j - 1] = t;
    }
  for (int k = 0; k < n; ++k) out[k] = make_int2(dy[idx[k]], dx[idx[k]]);
  return n;
}

template <int N, int NL>
cudaError_t launch_na(const float* yhat, const NaGeo& g, float* tile_bits, cudaStream_t st) {
  k_rate_noalloc<N, NL><<<g.tile0[kLevels], kNaThreads, 0, st>>>(yhat, g, tile_bits);
  return cudaGetLastError();
}

}  // namespace
}  // namespace cc

extern "C" int cc_rate_bits_noalloc(const cc_config* cfg, const float* yhat_flat, int H, int W,
                                    const float* params, void* cuda_stream, double* bits_out) {
  using namespace cc;
  int n_params = 0;
  int e = cc_param_count(cfg, &n_params);  // validates the configuration
  if (e) return e;
  if (!yhat_flat || !params || !bits_out || H < 1 || W < 1 || H > 16384 || W > 16384)
    return CC_EINVAL;
  NaGeo g;
  long long fo = 0;
  int tiles = 0;
  for (int l = 0; l < kLevels; ++l) {
    g.h[l] = (H + (1 << l) - 1) >> l;
    g.w[l] = (W + (1 << l) - 1) >> l;
    g.foff[l] = fo;
    g.tile0[l] = tiles;
    const long long n = (long long)g.h[l] * g.w[l];
    fo += n;
    tiles += (int)((n + kNaThreads - 1) / kNaThreads);
  }
  g.tile0[kLevels] = tiles;
  if (tiles > kNaMaxTiles) {
    set_error_text("cc_rate_bits_noalloc: the latent pyramid needs more tiles of 128 latents "
                   "than its fixed scratch holds (CC_NOALLOC_MAX_TILES)");
    return CC_EINVAL;
  }
  const int N = cfg->arm_ctx, NL = cfg->arm_layers;
  const int n_arm = NL * (N * N + N) + 2 * N + 2;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  NoAllocScratch* scr = nullptr;
  if (ce == cudaSuccess) ce = scratch_of(dev, &scr);
  int2 offs[kNaMaxN];
  causal_offsets_fixed(N, offs);
  if (ce == cudaSuccess)
    ce = cudaMemcpyToSymbolAsync(c_arm_na, params, (size_t)n_arm * sizeof(float), 0,
                                 cudaMemcpyDeviceToDevice, st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyToSymbolAsync(c_off_na, offs, (size_t)N * sizeof(int2), 0,
                                 cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) {
    switch (N * 10 + NL) {
      case 81: ce = launch_na<8, 1>(yhat_flat, g, scr->tile_bits, st); break;
      case 82: ce = launch_na<8, 2>(yhat_flat, g, scr->tile_bits, st); break;
      case 161: ce = launch_na<16, 1>(yhat_flat, g, scr->tile_bits, st); break;
      case 162: ce = launch_na<16, 2>(yhat_flat, g, scr->tile_bits, st); break;
      case 241: ce = launch_na<24, 1>(yhat_flat, g, scr->tile_bits, st); break;
      case 242: ce = launch_na<24, 2>(yhat_flat, g, scr->tile_bits, st); break;
      default: return CC_EINVAL;
    }
  }
  if (ce == cudaSuccess) {
    k_sum_tiles<<<1, 256, 0, st>>>(scr->tile_bits, tiles, &scr->total);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(bits_out, &scr->total, sizeof(double), cudaMemcpyDefault, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "cc_rate_bits_noalloc: %s", cudaGetErrorString(ce));
    set_error_text(msg);
    return CC_ECUDA;
  }
  return CC_OK;
}
