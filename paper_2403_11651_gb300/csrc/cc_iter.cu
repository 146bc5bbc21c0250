// Quantisation proxy, gradient assembly and Adam (Sec. II "Encoding"; Adam of Kingma & Ba
// as used in Sec. IV-B), plus the deterministic reductions of the per-CTA partial sums.
#include "cc_internal.cuh"

#include <vector>

#include <cmath>
#include <cstdlib>

namespace cc {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3): ten rounds of
//   (x0, x1, x2, x3) <- (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0))
// with the key bumped by the Weyl constants after each round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint2 k) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, x.x), lo0 = M0 * x.x;
    const uint32_t hi1 = __umulhi(M1, x.z), lo1 = M1 * x.z;
    x = make_uint4(hi1 ^ x.y ^ k.x, lo1, hi0 ^ x.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return x;
}

// Modes: 0 follow the schedule, 1 rint, 2 y + given noise, 3 y + Philox noise,
//        4 write the Philox noise itself.
// Noise of latent i of level l at iteration t: word (i mod 4) of
// Philox4x32-10(counter (i div 4, l, t, 0), key (seed lo, seed hi)), u = (w >> 8) 2^-24 - 1/2.
// C3 soft rounding with temperature T (inv_t = 1/T, k = 1 / (2 tanh(1/(2T)))):
// s(x) = floor(x) + 1/2 + k tanh((x - floor(x) - 1/2) / T) and its derivative
// s'(x) = k (1 - tanh^2(...)) / T.
__device__ __forceinline__ float soft_round(float x, float inv_t, float k, float& ds) {
  const float f = floorf(x);
  const float th = tanhf((x - f - 0.5f) * inv_t);
  ds = k * (1.f - th * th) * inv_t;
  return f + 0.5f + k * th;
}

__global__ void __launch_bounds__(256) k_quantize(Geo g, const float* __restrict__ y,
                                                  float* __restrict__ yhat,
                                                  float* __restrict__ yhat_bord,
                                                  const float* __restrict__ noise, int mode,
                                                  const IterScalars* sc, int ste_start,
                                                  uint2 key, int iter_override, float soft_temp,
                                                  float* __restrict__ dq) {
  pdl_wait();
  pdl_trigger();
  const int l = blockIdx.y;
  const int n = g.h[l] * g.w[l];
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= n) return;
  const int t = iter_override >= 0 ? iter_override : sc->t;
  int m = mode;
  if (m == 0) m = t >= ste_start ? 1 : 3;
  const long long base = g.off[l];
  uint4 r = make_uint4(0, 0, 0, 0);
  if (m >= 3) r = philox4x32_10(make_uint4((uint32_t)(i0 >> 2), (uint32_t)l, (uint32_t)t, 0u), key);
  const uint32_t words[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int i = i0 + e;
    if (i >= n) break;
    const float yv = y[base + i];
    if (!isfinite(yv)) const_cast<IterScalars*>(sc)->nonfinite = 1;
    float out;
    if (m == 1) {
      out = rintf(yv);
    } else if (m == 4) {
      out = (float)(words[e] >> 8) * 5.9604644775390625e-08f - 0.5f;
    } else {
      const float u = m == 2 ? noise[base + i]
                             : (float)(words[e] >> 8) * 5.9604644775390625e-08f - 0.5f;
      if (soft_temp > 0.f) {
        // y_hat = s(s(y) + u), d y_hat / d y = s'(s(y) + u) s'(y)
        const float inv_t = 1.f / soft_temp, k = 0.5f / tanhf(0.5f * inv_t);
        float d1, d2;
        const float s1 = soft_round(yv, inv_t, k, d1);
        out = soft_round(s1 + u, inv_t, k, d2);
        dq[base + i] = d2 * d1;
      } else {
        out = yv + u;
      }
    }
    yhat[base + i] = out;
    if (yhat_bord) {
      const int r = i / g.w[l], c = i - r * g.w[l];
      yhat_bord[g.poff[l] + (long long)(r + kCtxPad) * g.pw[l] + c + kCtxPad] = out;
    }
  }
}

cudaError_t quantize_launch(const Geo& g, const float* y, float* yhat, float* yhat_bord,
                            const float* noise, int mode, const IterScalars* sc, int ste_start,
                            uint64_t seed, int iter_override, float soft_temp, float* dq,
                            cudaStream_t st) {
  int maxn = 0;
  for (int l = 0; l < kLevels; ++l) maxn = g.h[l] * g.w[l] > maxn ? g.h[l] * g.w[l] : maxn;
  const int groups = (maxn + 3) / 4;
  dim3 grid((groups + 255) / 256, kLevels);
  const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  k_quantize<<<grid, 256, 0, st>>>(g, y, yhat, yhat_bord, noise, mode, sc, ste_start, key,
                                   iter_override, dq ? soft_temp : 0.f, dq);
  return cudaGetLastError();
}

// part2[slice][col0 + j] = scale * sum over the slice's rows of part[row][j], rows summed
// in a fixed tree (8 interleaved sequential sums, then those 8 in order).  blockIdx.x runs
// over the (section, chunk of 32 columns) pairs of the table only; each thread issues all
// loads of its rows before adding them.
__global__ void __launch_bounds__(256) k_reduce_sections(SectionTable tab, float* part2,
                                                         int n_virtual) {
  pdl_wait();
  pdl_trigger();
  int sec = 0, chunk = blockIdx.x;
  while (sec + 1 < tab.n && chunk >= (tab.s[sec].cols + 31) / 32) {
    chunk -= (tab.s[sec].cols + 31) / 32;
    ++sec;
  }
  const Section s = tab.s[sec];
  const int j = chunk * 32 + threadIdx.x;
  const int slices = gridDim.y, slice = blockIdx.y;
  const int rps = (s.rows + slices - 1) / slices;
  const int r0 = slice * rps;
  const int r1 = min(s.rows, r0 + rps);
  float acc = 0.f;
  if (j < s.cols) {
    constexpr int B = 8;   // rows in flight per thread
    for (int rb = r0 + (int)threadIdx.y; rb < r1; rb += 8 * B) {
      float v[B];
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int r = rb + 8 * q;
        v[q] = r < r1 ? s.part[(long long)r * s.stride + j] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < B; ++q) acc += v[q];
    }
  }
  __shared__ float sm[8][33];
  sm[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && j < s.cols) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += sm[k][threadIdx.x];
    part2[(long long)slice * n_virtual + s.col0 + j] = t * s.scale;
  }
}

cudaError_t reduce_sections(const SectionTable& tab, float* part2, int n_virtual, int slices,
                            cudaStream_t st) {
  int chunks = 0;
  for (int i = 0; i < tab.n; ++i) chunks += (tab.s[i].cols + 31) / 32;
  dim3 grid(chunks, slices);
  k_reduce_sections<<<grid, dim3(32, 8), 0, st>>>(tab, part2, n_virtual);
  return cudaGetLastError();
}

struct AdamStep {
  float lr, inv_bc1, inv_sqrt_bc2;
};

__device__ __forceinline__ void adam_apply(float& p, float& m, float& v, float g,
                                           const AdamStep& a) {
  m = 0.9f * m + 0.1f * g;
  v = 0.999f * v + 0.001f * g * g;
  p -= a.lr * (m * a.inv_bc1) / (sqrtf(v) * a.inv_sqrt_bc2 + 1e-8f);
}

// Adam bias corrections of step s >= 1, (1 / (1 - beta1^s), 1 / sqrt(1 - beta2^s)), computed
// in FP64 on the host and rounded to float; from step kAdamBcSteps on both round to 1.0f
// (beta2^s < 2^-47).  The passes look them up instead of evaluating FP64 powers, divisions
// and square roots, which are slow on this GPU's FP64 units.
constexpr int kAdamBcSteps = 32768;
__device__ float2 g_adam_bc[kAdamBcSteps];

__device__ __forceinline__ float2 adam_bc(int s) {
  return s < kAdamBcSteps ? g_adam_bc[s] : make_float2(1.f, 1.f);
}

static float2 adam_bc_host(int s) {
  return make_float2((float)(1.0 / (1.0 - pow(0.9, (double)s))),
                     (float)(1.0 / sqrt(1.0 - pow(0.999, (double)s))));
}

cudaError_t adam_bc_upload(cudaStream_t st) {
  static const std::vector<float2> tab = [] {
    std::vector<float2> v(kAdamBcSteps, make_float2(1.f, 1.f));
    for (int s = 1; s < kAdamBcSteps; ++s) v[s] = adam_bc_host(s);
    return v;
  }();
  return cudaMemcpyToSymbolAsync(g_adam_bc, tab.data(), sizeof(float2) * kAdamBcSteps, 0,
                                 cudaMemcpyHostToDevice, st);
}

// D, R and the loss of the pass from the per-CTA partial sums, and the loss log entry of
// iteration t.  The partials are summed in float-float arithmetic over 256 virtual lanes
// (all loads of a lane issued together) and a tree, in a fixed order; run by one block of
// any power-of-two size up to 256.
constexpr int kLossLoads = 8;   // partials per virtual lane loaded at once
__device__ __forceinline__ float2 lane_sum(const float* part, int n, int v) {
  float2 a = make_float2(0.f, 0.f);
  for (int k0 = v; k0 < n; k0 += 256 * kLossLoads) {
    float x[kLossLoads];
#pragma unroll
    for (int j = 0; j < kLossLoads; ++j) x[j] = k0 + 256 * j < n ? part[k0 + 256 * j] : 0.f;
#pragma unroll
    for (int j = 0; j < kLossLoads; ++j) a = ff_add(a, make_float2(x[j], 0.f));
  }
  return a;
}

__device__ __forceinline__ void loss_block(const float* part_d, int nd, const float* part_bits,
                                           int nb, double d_scale, double r_scale, double lam,
                                           IterScalars* sc, double* log) {
  __shared__ float2 sd[256], sb[256];
  for (int v = threadIdx.x; v < 256; v += blockDim.x) {
    sd[v] = lane_sum(part_d, nd, v);
    sb[v] = lane_sum(part_bits, nb, v);
  }
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    for (int v = threadIdx.x; v < s; v += blockDim.x) {
      sd[v] = ff_add(sd[v], sd[v + s]);
      sb[v] = ff_add(sb[v], sb[v + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double D = ((double)sd[0].x + (double)sd[0].y) * d_scale;
    const double R = ((double)sb[0].x + (double)sb[0].y) * r_scale;
    sc->D = D;
    sc->R = R;
    sc->loss = D + lam * R;
    double* e = log + 3 * (long long)(sc->t % kLogCap);
    e[0] = D;
    e[1] = R;
    e[2] = D + lam * R;
  }
}

// The step to the next iteration: t and the Adam bias corrections of its update (one thread).
__device__ __forceinline__ void advance_step(IterScalars* sc) {
  const int t = sc->t;
  sc->t = t + 1;
  const float2 bc = adam_bc(t + 2);   // the update of iteration t + 1 is Adam step t + 2
  sc->inv_bc1 = bc.x;
  sc->inv_sqrt_bc2 = bc.y;
}

// The pass ends with the latent update and the parameter update, which may run on two
// streams at once; the last of their blocks to end (a ticket in IterScalars counting the
// blocks of both) takes the step to the next iteration, after every block has read the
// iteration's scalars.  The loss of the pass is computed beforehand (pass_loss).
struct FinishArgs {
  int advance;
  unsigned tickets;   // blocks that take a ticket: the latent update's, plus the parameter
                      // update's when it shares the finish
};

__device__ __forceinline__ void finish_if_last(IterScalars* sc, const FinishArgs& fa) {
  __shared__ bool s_last;
  // t and the next bias corrections are read before the ticket (no block changes them
  // before the last ticket), so that the last block only stores
  int t = 0;
  float2 bc = make_float2(1.f, 1.f);
  if (threadIdx.x == 0 && fa.advance) {
    t = sc->t;
    bc = adam_bc(t + 2);   // the update of iteration t + 1 is Adam step t + 2
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&sc->ticket, 1u) == fa.tickets - 1;
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    trace_point("finish_begin");
    if (fa.advance) {
      sc->t = t + 1;
      sc->inv_bc1 = bc.x;
      sc->inv_sqrt_bc2 = bc.y;
    }
    sc->ticket = 0u;
    trace_point("finish_end");
  }
}

struct VirtualMap {
  int n_arm, up0, syn0, n1x1, nconv, K2, n_up, per_level;
  int vsyn, vconv, vup, n_virtual;
};

__device__ __forceinline__ void param_update_one(const VirtualMap& vm, const float* part2,
                                                 int slices, float* params, float* m, float* v,
                                                 float* grad_out, int apply, float lr,
                                                 const IterScalars* sc, int j,
                                                 const ImageSlots& slots) {
  AdamStep st;
  st.lr = lr;
  st.inv_bc1 = sc->inv_bc1;
  st.inv_sqrt_bc2 = sc->inv_sqrt_bc2;
  int vs[kLevels - 1];
  int nv = 1;
  if (j < vm.n_arm) {
    vs[0] = j;
  } else if (j < vm.up0 + vm.n_up * vm.K2) {
    const int fi = (j - vm.up0) / vm.K2, u = (j - vm.up0) % vm.K2;
    if (vm.per_level) {
      vs[0] = vm.vup + fi * vm.K2 + u;
    } else {
      nv = kLevels - 1;
      for (int l = 0; l < kLevels - 1; ++l) vs[l] = vm.vup + l * vm.K2 + u;
    }
  } else if (j < vm.syn0 + vm.n1x1) {
    vs[0] = vm.vsyn + (j - vm.syn0);
  } else {
    vs[0] = vm.vconv + (j - vm.syn0 - vm.n1x1);
  }
  float g = 0.f;
  for (int k = 0; k < nv; ++k) {
    // the slices' loads issued together, then summed in slice order
    float v[kSlices];
#pragma unroll
    for (int s = 0; s < kSlices; ++s)
      v[s] = s < slices ? part2[(long long)s * vm.n_virtual + vs[k]] : 0.f;
    float t = 0.f;
#pragma unroll
    for (int s = 0; s < kSlices; ++s) t += v[s];
    g += t;
  }
  if (grad_out) grad_out[j] = g;
  if (apply) {
    float p = params[j];
    adam_apply(p, m[j], v[j], g, st);
    if (!isfinite(p) || !isfinite(v[j])) const_cast<IterScalars*>(sc)->nonfinite = 1;
    params[j] = p;
    const int4 d = slots.map[j];
    if (d.x >= 0) slots.arm_image[d.x] = p;
    if (d.y >= 0) slots.arm_image[d.y] = p;
    if (d.z >= 0) slots.syn_image[d.z] = p;
    if (d.w >= 0) slots.syn_image[d.w] = p;
  }
}

// Adam bias corrections of this iteration are read from IterScalars (set when t advanced).
__global__ void __launch_bounds__(128) k_param_update(VirtualMap vm, const float* part2,
                                                      int slices, float* params, float* m,
                                                      float* v, float* grad_out, int apply,
                                                      float lr, IterScalars* sc, int total,
                                                      ImageSlots slots, FinishArgs fa) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < total) param_update_one(vm, part2, slices, params, m, v, grad_out, apply, lr, sc, j,
                                  slots);
  if (threadIdx.x == 0) trace_point("param_block_done");
  if (fa.tickets) finish_if_last(sc, fa);
}

FinishArgs finish_args(bool advance, unsigned tickets) {
  FinishArgs fa;
  fa.advance = advance ? 1 : 0;
  fa.tickets = tickets;
  return fa;
}

unsigned param_update_blocks(const Layout& lay) { return (unsigned)((lay.total + 127) / 128); }
unsigned latent_update_blocks(const Geo& g) { return (unsigned)((g.n_pad + 255) / 256); }

cudaError_t param_update(const Layout& lay, const Arch& a, const float* part2, int slices,
                         float* params, float* m, float* v, float* grad_out, bool apply,
                         float lr, const IterScalars* sc, const ImageSlots& slots,
                         const PassFinish* pf, unsigned tickets, bool advance,
                         cudaStream_t st) {
  VirtualMap vm;
  vm.n_arm = lay.n_arm; vm.up0 = lay.up0; vm.syn0 = lay.syn0;
  vm.n1x1 = 11 * a.C + 3; vm.nconv = a.NR * 84; vm.K2 = a.K * a.K; vm.n_up = lay.n_up;
  vm.per_level = a.per_level;
  vm.vsyn = lay.n_arm; vm.vconv = vm.vsyn + vm.n1x1; vm.vup = vm.vconv + vm.nconv;
  vm.n_virtual = vm.vup + (kLevels - 1) * vm.K2;
  const FinishArgs fa = pf ? finish_args(advance, tickets) : FinishArgs{};
  return launch_k(k_param_update, dim3(param_update_blocks(lay)), dim3(128), 0, st, vm, part2,
                  slices, params, m, v, grad_out, apply ? 1 : 0, lr,
                  const_cast<IterScalars*>(sc), lay.total, slots, fa);
}

__global__ void __launch_bounds__(256) k_finish(const float* part_d, int nd,
                                                const float* part_bits, int nb, double d_scale,
                                                double r_scale, double lam, IterScalars* sc,
                                                double* log, int advance) {
  pdl_wait();
  pdl_trigger();
  loss_block(part_d, nd, part_bits, nb, d_scale, r_scale, lam, sc, log);
  if (advance && threadIdx.x == 0) advance_step(sc);
}

cudaError_t pass_loss(const PassFinish& pf, IterScalars* sc, cudaStream_t st) {
  k_finish<<<1, 256, 0, st>>>(pf.part_d, pf.nd, pf.part_bits, pf.nb, pf.d_scale, pf.r_scale,
                              pf.lam, sc, pf.log, 0);
  return cudaGetLastError();
}

// Gradient of a latent: the synthesis path, plus lambda/(HW) times the rate terms in
// which it appears, as the coded symbol (gself) and in the context of every latent p
// whose causal neighbourhood contains it (dctx of p at the matching slot).
__global__ void __launch_bounds__(256) k_latent_update(Geo g, const float* __restrict__ gsyn,
                                                       const float* __restrict__ grate,
                                                       float rate_scale, float* y, float* m,
                                                       float* v, float* grad_out, int apply,
                                                       float lr, IterScalars* sc, FinishArgs fa,
                                                       const float* __restrict__ dq, int soft,
                                                       int ste_start) {
  pdl_wait();
  pdl_trigger();
  // one thread per element of the latent-shaped buffers; alignment gaps between planes skip
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int l = 0;
#pragma unroll
  for (int k = 1; k < kLevels; ++k) l = q >= g.off[k] ? k : l;
  const long long i = q - g.off[l];
  if (q < g.n_pad && i < (long long)g.h[l] * g.w[l]) {
    float gt = __ldg(gsyn + q) + rate_scale * __ldg(grate + q);   // dL / d y_hat
    if (q == 0 && sc->t == sc->nan_at) gt = __int_as_float(0x7fc00000);   // injected fault
    // soft-rounding pass: dL/dy = dL/dy_hat * dy_hat/dy (1: always, 2: noise phase only)
    if (soft == 1 || (soft == 2 && sc->t < ste_start)) gt *= __ldg(dq + q);
    if (grad_out) {
      long long fo = 0;
      for (int k = 0; k < l; ++k) fo += (long long)g.h[k] * g.w[k];
      grad_out[fo + i] = gt;
    }
    if (apply) {
      AdamStep st;
      st.lr = lr;
      st.inv_bc1 = sc->inv_bc1;
      st.inv_sqrt_bc2 = sc->inv_sqrt_bc2;
      float yv = y[q], mv = m[q], vv = v[q];
      adam_apply(yv, mv, vv, gt, st);
      if (!isfinite(yv) || !isfinite(vv)) sc->nonfinite = 1;
      y[q] = yv; m[q] = mv; v[q] = vv;
    }
  }
  finish_if_last(sc, fa);
}

cudaError_t latent_update(const Geo& g, const float* gsyn, const float* grate, float rate_scale,
                          float* y, float* m, float* v, float* grad_out, bool apply, float lr,
                          IterScalars* sc, const PassFinish& pf, unsigned tickets, bool advance,
                          const float* dq, int soft, int ste_start, cudaStream_t st) {
  const FinishArgs fa = finish_args(advance, tickets);
  return launch_k(k_latent_update, dim3(latent_update_blocks(g)), dim3(256), 0, st, g, gsyn,
                  grate, rate_scale, y, m, v, grad_out, apply ? 1 : 0, lr, sc, fa, dq, soft,
                  ste_start);
}

cudaError_t finish_iteration(const float* part_d, int nd, const float* part_bits, int nb,
                             double d_scale, double r_scale, double lam, IterScalars* sc,
                             double* log, bool advance, cudaStream_t st, bool pdl) {
  if (pdl)
    return launch_k(k_finish, dim3(1), dim3(256), 0, st, part_d, nd, part_bits, nb, d_scale,
                    r_scale, lam, sc, log, advance ? 1 : 0);
  k_finish<<<1, 256, 0, st>>>(part_d, nd, part_bits, nb, d_scale, r_scale, lam, sc, log,
                              advance ? 1 : 0);
  return cudaGetLastError();
}

__global__ void k_image_to_planar(const uint8_t* __restrict__ rgb, float* __restrict__ x,
                                  int HW) {
  pdl_wait();
  pdl_trigger();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * HW + p] = (float)rgb[p * 3 + c] / 255.0f;
  }
}

cudaError_t image_to_planar(const uint8_t* rgb_hwc, float* x, int H, int W, cudaStream_t st) {
  const int HW = H * W;
  const int blocks = (HW + 255) / 256 < 4096 ? (HW + 255) / 256 : 4096;
  k_image_to_planar<<<blocks, 256, 0, st>>>(rgb_hwc, x, HW);
  return cudaGetLastError();
}

// One thread per latent of the whole pyramid (the latent-shaped buffer's padding skipped),
// so the grid holds only the blocks that have latents.
template <int N>
__global__ void __launch_bounds__(256) k_ctx_gather(Geo g, const int2* __restrict__ offs,
                                                    float* gself, const float* __restrict__ dctx) {
  pdl_wait();
  pdl_trigger();
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int l = 0;
#pragma unroll
  for (int k = 1; k < kLevels; ++k) l = q >= g.off[k] ? k : l;
  const int w = g.w[l], h = g.h[l];
  const long long i = q - g.off[l];
  if (q >= g.n_pad || i >= (long long)h * w) return;
  const int r = (int)(i / w), c = (int)(i - (long long)r * w);
  // the N context gradients are loaded together, then added in slot order
  float v[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int2 o = __ldg(offs + k);
    const int pr = r - o.x, pc = c - o.y;
    v[k] = (pr < h && pc >= 0 && pc < w) ? __ldg(dctx + (long long)k * g.n_pad + g.off[l] + pr * w + pc)
                                        : 0.f;
  }
  float gr = gself[q];
#pragma unroll
  for (int k = 0; k < N; ++k) gr += v[k];
  gself[q] = gr;
}

cudaError_t ctx_gather(const Geo& g, const int2* d_offsets, int N, float* gself,
                       const float* dctx, cudaStream_t st) {
  const dim3 grid((unsigned)((g.n_pad + 255) / 256));
  switch (N) {
    case 8: k_ctx_gather<8><<<grid, 256, 0, st>>>(g, d_offsets, gself, dctx); break;
    case 16: k_ctx_gather<16><<<grid, 256, 0, st>>>(g, d_offsets, gself, dctx); break;
    case 24: k_ctx_gather<24><<<grid, 256, 0, st>>>(g, d_offsets, gself, dctx); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

IterScalars iter_scalars_at(int t) {
  IterScalars s{};
  s.t = t;
  s.nan_at = -1;
  const float2 bc = adam_bc_host(t + 1);
  s.inv_bc1 = bc.x;
  s.inv_sqrt_bc2 = bc.y;
  return s;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("CC_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

}  // namespace cc

#ifdef CC_TRACE
// Traced build only: copies up to max_n records of the kernel-start trace to host memory
// (TraceRec layout) and resets it; returns the number of records written since the last
// reset.
extern "C" int cc_trace_dump(void* host, int max_n) {
  unsigned n = 0;
  if (cudaMemcpyFromSymbol(&n, cc::g_trace_n, sizeof(unsigned)) != cudaSuccess) return -1;
  int m = (int)(n < (unsigned)max_n ? n : (unsigned)max_n);
  if (m > cc::kTraceCap) m = cc::kTraceCap;
  if (m > 0 && cudaMemcpyFromSymbol(host, cc::g_trace, (size_t)m * sizeof(cc::TraceRec)) != cudaSuccess)
    return -1;
  const unsigned z = 0;
  if (cudaMemcpyToSymbol(cc::g_trace_n, &z, sizeof(unsigned)) != cudaSuccess) return -1;
  return (int)n;
}
#endif
