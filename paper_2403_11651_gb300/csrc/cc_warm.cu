// Warm-start predictor: image -> latent pyramid (levels 0 .. 4), trained on latents the
// encoder reached.  Four 3x3 stride-2 convolutions with 32 channels and ReLU (zero
// padding 1) give levels 1 .. 4 through 1x1 convolutions; a 3x3 stride-1 convolution of
// the image gives level 0; levels 5 and 6 start at 0.  Loss: the sum over the predicted
// levels of each level's mean squared error.  FP32 on the CUDA cores; every reduction in
// a fixed order.
//
// Convolution: out[co][y][x] = b[co] + sum_{ci, ky, kx} w[co][ci][ky][kx]
//                                        * in[ci][s y + ky - 1][s x + kx - 1]  (0 outside).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cc_internal.cuh"
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

// din[ci][iy][ix] = sum over co and taps (ky, kx) with s oy + ky - 1 = iy, s ox + kx - 1 = ix
// of w[co][ci][ky][kx] dout[co][oy][ox]; with accumulate, added to din
__global__ void __launch_bounds__(256) k_wconv_dgrad(const float* __restrict__ dout, int Co, int Ho,
                                                     int Wo, const float* __restrict__ w,
                                                     float* __restrict__ din, int Ci, int Hi, int Wi,
                                                     int s, int accumulate) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)Ci * Hi * Wi) return;
  const int ci = (int)(q / ((long long)Hi * Wi));
  const int r = (int)(q - (long long)ci * Hi * Wi), iy = r / Wi, ix = r - iy * Wi;
  float acc = 0.f;
  for (int co = 0; co < Co; ++co) {
    const float* wp = w + ((long long)co * Ci + ci) * 9;
    const float* dp = dout + (long long)co * Ho * Wo;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int ty = iy + 1 - ky;
      if (ty < 0 || ty % s) continue;
      const int oy = ty / s;
      if (oy >= Ho) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int tx = ix + 1 - kx;
        if (tx < 0 || tx % s) continue;
        const int ox = tx / s;
        if (ox < Wo) acc = fmaf(wp[ky * 3 + kx], dp[(long long)oy * Wo + ox], acc);
      }
    }
  }
  din[q] = accumulate ? din[q] + acc : acc;
}

// dw[co][ci][ky][kx] = sum over (oy, ox) of dout[co][oy][ox] in[ci][s oy + ky - 1][s ox + kx - 1];
// block (ci, co); the block with ci == 0 also sums db[co] = sum dout[co]
__global__ void __launch_bounds__(256) k_wconv_wgrad(const float* __restrict__ dout, int Co, int Ho,
                                                     int Wo, const float* __restrict__ in, int Ci,
                                                     int Hi, int Wi, int s, float* __restrict__ dw,
                                                     float* __restrict__ db) {
  const int ci = blockIdx.x, co = blockIdx.y;
  const float* dp = dout + (long long)co * Ho * Wo;
  const float* ip = in + (long long)ci * Hi * Wi;
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
  for (int p = threadIdx.x; p < Ho * Wo; p += blockDim.x) {
    const int oy = p / Wo, ox = p - oy * Wo;
    const float g = dp[p];
    acc[9] += g;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int iy = s * oy + ky - 1;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int ix = s * ox + kx - 1;
        if (iy >= 0 && iy < Hi && ix >= 0 && ix < Wi)
          acc[ky * 3 + kx] = fmaf(g, ip[(long long)iy * Wi + ix], acc[ky * 3 + kx]);
      }
    }
  }
  __shared__ float red[10][256];
#pragma unroll
  for (int k = 0; k < 10; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
#pragma unroll
      for (int k = 0; k < 10; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 9) dw[((long long)co * Ci + ci) * 9 + threadIdx.x] = red[threadIdx.x][0];
  if (threadIdx.x == 9 && ci == 0 && db) db[co] = red[9][0];
}

// 1x1 head: out[p] = b + sum_c w[c] a[c][p]
__global__ void __launch_bounds__(256) k_whead(const float* __restrict__ a, int C, int n,
                                               const float* __restrict__ w,
                                               const float* __restrict__ b, float* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float acc = b[0];
  for (int c = 0; c < C; ++c) acc = fmaf(w[c], a[(long long)c * n + p], acc);
  out[p] = acc;
}

// head backward into the activation gradient: da[c][p] (+)= w[c] dout[p]
__global__ void __launch_bounds__(256) k_whead_dgrad(const float* __restrict__ dout, int C, int n,
                                                     const float* __restrict__ w, float* da,
                                                     int accumulate) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)C * n) return;
  const int c = (int)(q / n), p = (int)(q - (long long)c * n);
  const float v = w[c] * dout[p];
  da[q] = accumulate ? da[q] + v : v;
}

__global__ void __launch_bounds__(256) k_wrelu_mask(const float* __restrict__ a, float* g, long long n) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n && !(a[q] > 0.f)) g[q] = 0.f;
}

// head weight gradient: block c < C: dw[c] = sum_p a[c][p] dout[p]; block C: db = sum dout
__global__ void __launch_bounds__(256) k_whead_wgrad(const float* __restrict__ a, int C, int n,
                                                     const float* __restrict__ dout,
                                                     float* __restrict__ dw, float* __restrict__ db) {
  const int c = blockIdx.x;
  float acc = 0.f;
  for (int p = threadIdx.x; p < n; p += blockDim.x)
    acc += (c < C ? a[(long long)c * n + p] : 1.f) * dout[p];
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (c < C) dw[c] = red[0]; else *db = red[0];
  }
}

// squared error of one level: per-block partial sums (fixed order) and d/dpred = 2 diff / n
__global__ void __launch_bounds__(256) k_wloss(const float* __restrict__ pred,
                                               const float* __restrict__ target, int n,
                                               float* __restrict__ dpred,
                                               double* __restrict__ part) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (p < n) {
    const float d = pred[p] - target[p];
    dpred[p] = 2.f * d / (float)n;
    e = (double)d * d / (double)n;
  }
  __shared__ double red[256];
  red[threadIdx.x] = e;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_wadam(float* p, float* m, float* v, const float* g, int n,
                                               float lr, float inv_bc1, float inv_sqrt_bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  m[i] = 0.9f * m[i] + 0.1f * gi;
  v[i] = 0.999f * v[i] + 0.001f * gi * gi;
  p[i] -= lr * (m[i] * inv_bc1) / (sqrtf(v[i]) * inv_sqrt_bc2 + 1e-8f);
}

int blocks(long long n) { return (int)((n + 255) / 256); }

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
  double* part;
  int n_part = 0;
  long long t = 0;
  double b1t = 1.0, b2t = 1.0;
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

// forward: image (already planar in x) -> act[1..4], pred (flat latent order; levels 5, 6 = 0)
int warm_forward(cc_warm* c) {
  const WarmLayout& L = c->L;
  float* P = c->params;
  const Geo& g = c->geo;
  WCK(cudaMemsetAsync(c->pred, 0, (size_t)g.n_lat * sizeof(float), c->st));
  long long fo[kLevels];
  long long o = 0;
  for (int l = 0; l < kLevels; ++l) { fo[l] = o; o += (long long)g.h[l] * g.w[l]; }
  // level 0: 3x3 stride 1 on the image
  k_wconv<<<blocks((long long)c->H * c->W), 256, 0, c->st>>>(c->x, 3, c->H, c->W, P + L.h_w[0],
                                                             P + L.h_b[0], c->pred + fo[0], 1,
                                                             c->H, c->W, 1, 0);
  for (int i = 1; i <= 4; ++i) {
    const float* in = i == 1 ? c->x : c->act[i - 1];
    const int Ci = i == 1 ? 3 : kWCh;
    const int Hi = i == 1 ? c->H : c->h[i - 1], Wi = i == 1 ? c->W : c->w[i - 1];
    k_wconv<<<blocks((long long)kWCh * c->h[i] * c->w[i]), 256, 0, c->st>>>(
        in, Ci, Hi, Wi, P + L.c_w[i], P + L.c_b[i], c->act[i], kWCh, c->h[i], c->w[i], 2, 1);
    const int n = c->h[i] * c->w[i];
    k_whead<<<blocks(n), 256, 0, c->st>>>(c->act[i], kWCh, n, P + L.h_w[i], P + L.h_b[i],
                                          c->pred + fo[i]);
  }
  WCK(cudaGetLastError());
  return CC_OK;
}

// loss and gradients into c->grads for targets (flat latent order, device)
int warm_backward(cc_warm* c, const float* target, double* loss) {
  const WarmLayout& L = c->L;
  const Geo& g = c->geo;
  float* P = c->params;
  float* G = c->grads;
  long long fo[kLevels];
  long long o = 0;
  for (int l = 0; l < kLevels; ++l) { fo[l] = o; o += (long long)g.h[l] * g.w[l]; }
  int nb = 0;
  for (int l = 0; l <= 4; ++l) {
    const int n = g.h[l] * g.w[l];
    k_wloss<<<blocks(n), 256, 0, c->st>>>(c->pred + fo[l], target + fo[l], n, c->dpred + fo[l],
                                          c->part + nb);
    nb += blocks(n);
  }
  // level 0 head (3x3 on the image): weight gradient only
  k_wconv_wgrad<<<dim3(3, 1), 256, 0, c->st>>>(c->dpred + fo[0], 1, c->H, c->W, c->x, 3, c->H,
                                                c->W, 1, G + L.h_w[0], G + L.h_b[0]);
  for (int i = 4; i >= 1; --i) {
    const int n = c->h[i] * c->w[i];
    k_whead_wgrad<<<kWCh + 1, 256, 0, c->st>>>(c->act[i], kWCh, n, c->dpred + fo[i],
                                               G + L.h_w[i], G + L.h_b[i]);
    // dact[i] holds conv i+1's input gradient (i < 4); add the head's
    k_whead_dgrad<<<blocks((long long)kWCh * n), 256, 0, c->st>>>(c->dpred + fo[i], kWCh, n,
                                                                  P + L.h_w[i], c->dact[i],
                                                                  i < 4 ? 1 : 0);
    k_wrelu_mask<<<blocks((long long)kWCh * n), 256, 0, c->st>>>(c->act[i], c->dact[i],
                                                                 (long long)kWCh * n);
    const float* in = i == 1 ? c->x : c->act[i - 1];
    const int Ci = i == 1 ? 3 : kWCh;
    const int Hi = i == 1 ? c->H : c->h[i - 1], Wi = i == 1 ? c->W : c->w[i - 1];
    k_wconv_wgrad<<<dim3(Ci, kWCh), 256, 0, c->st>>>(c->dact[i], kWCh, c->h[i], c->w[i], in, Ci,
                                                     Hi, Wi, 2, G + L.c_w[i], G + L.c_b[i]);
    if (i > 1)
      k_wconv_dgrad<<<blocks((long long)kWCh * Hi * Wi), 256, 0, c->st>>>(
          c->dact[i], kWCh, c->h[i], c->w[i], P + L.c_w[i], c->dact[i - 1], kWCh, Hi, Wi, 2, 0);
  }
  WCK(cudaGetLastError());
  std::vector<double> part((size_t)nb);
  WCK(cudaMemcpyAsync(part.data(), c->part, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      c->st));
  WCK(cudaStreamSynchronize(c->st));
  double sum = 0.0;
  for (double v : part) sum += v;
  if (loss) *loss = sum;
  return std::isfinite(sum) ? CC_OK : CC_ENONFINITE;
}

int warm_image(cc_warm* c, const uint8_t* rgb) {
  WCK(cudaMemcpyAsync(c->img, rgb, (size_t)3 * c->H * c->W, cudaMemcpyDefault, c->st));
  WCK(image_to_planar(c->img, c->x, c->H, c->W, c->st));
  return CC_OK;
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
  const size_t o_part = take((size_t)c->n_part * sizeof(double));
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
  c->img = (uint8_t*)(b + o_img); c->part = (double*)(b + o_part);
  if ((e = cudaMemsetAsync(c->mem, 0, off, c->st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->params, params, NP, cudaMemcpyDefault, c->st)) != cudaSuccess ||
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
  if (!e) e = warm_backward(c, c->target, loss);
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
  int e = cc_warm_loss_grad(c, rgb_hwc, target, loss, nullptr);
  if (e) return e;
  ++c->t;
  c->b1t *= 0.9;
  c->b2t *= 0.999;
  k_wadam<<<blocks(c->L.total), 256, 0, c->st>>>(c->params, c->m, c->v, c->grads, c->L.total, lr,
                                                  (float)(1.0 / (1.0 - c->b1t)),
                                                  (float)(1.0 / std::sqrt(1.0 - c->b2t)));
  WCK(cudaGetLastError());
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
  if (c->mem) cudaFree(c->mem);
  delete c;
}

}  // extern "C"
