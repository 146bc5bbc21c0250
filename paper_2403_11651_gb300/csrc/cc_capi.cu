// C ABI of the library (declared in include/coolchic.h): context set-up, device memory
// plan, the sequence of kernels of one iteration and its CUDA-graph capture.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "cc_internal.cuh"
#include "../../include/coolchic.h"

using namespace cc;

namespace {

thread_local char g_err[512] = "";
bool g_fail_next_alloc = false;   // cc_debug_inject(NULL, CC_FAULT_ALLOC, 0)

int fail_cuda(cudaError_t e, const char* what) {
  snprintf(g_err, sizeof(g_err), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  return CC_ECUDA;
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return fail_cuda(e_, #call);  \
  } while (0)

// The contexts of one device share this library's __constant__ weight banks.  Every
// operation that loads the banks and runs kernels on them takes a turn: under one
// process-wide lock its stream waits for the end of the previous turn on the device (an
// event), the work is enqueued, and the event is recorded after it.  Turns of one device
// thus run one after another on the GPU, whatever streams and host threads issue them.
std::mutex g_turn_mu;
std::vector<cudaEvent_t> g_turn_end;   // per device

class BankTurn {
 public:
  BankTurn(int dev, cudaStream_t s) : lock_(g_turn_mu), dev_(dev), s_(s) {
    if ((int)g_turn_end.size() <= dev) g_turn_end.resize(dev + 1, nullptr);
    if (g_turn_end[dev]) err_ = cudaStreamWaitEvent(s, g_turn_end[dev], 0);
  }
  // records the end of the turn after the work enqueued so far on the stream
  cudaError_t end() {
    if (err_ != cudaSuccess || ended_) return err_;
    ended_ = true;
    if (!g_turn_end[dev_])
      err_ = cudaEventCreateWithFlags(&g_turn_end[dev_], cudaEventDisableTiming);
    if (err_ == cudaSuccess) err_ = cudaEventRecord(g_turn_end[dev_], s_);
    return err_;
  }
  cudaError_t status() const { return err_; }
  ~BankTurn() { end(); }

 private:
  std::lock_guard<std::mutex> lock_;
  int dev_;
  cudaStream_t s_;
  cudaError_t err_ = cudaSuccess;
  bool ended_ = false;
};

#define CKE(call)                                        \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return e_;                    \
  } while (0)

constexpr uint32_t kStateMagic = 0x31534343u;  // "CCS1"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
  uint32_t magic, version;
  int32_t H, W, n_lat, n_params, iter, pad;
  uint64_t seed;
  int32_t arch[8];
};

long long align32(long long v) { return (v + 31) & ~31ll; }

// The N nearest causal neighbours (dy < 0, or dy = 0 and dx < 0), ties broken by smaller
// |dy| then smaller dx, listed in raster order.
std::vector<int2> causal_offsets(int n) {
  struct Cand { int dy, dx; };
  std::vector<Cand> c;
  for (int dy = -6; dy <= 0; ++dy)
    for (int dx = -6; dx <= 6; ++dx)
      if (dy < 0 || dx < 0) c.push_back({dy, dx});
  std::stable_sort(c.begin(), c.end(), [](const Cand& a, const Cand& b) {
    const int da = a.dy * a.dy + a.dx * a.dx, db = b.dy * b.dy + b.dx * b.dx;
    if (da != db) return da < db;
    if (std::abs(a.dy) != std::abs(b.dy)) return std::abs(a.dy) < std::abs(b.dy);
    return a.dx < b.dx;
  });
  c.resize(n);
  std::sort(c.begin(), c.end(), [](const Cand& a, const Cand& b) {
    return a.dy != b.dy ? a.dy < b.dy : a.dx < b.dx;
  });
  std::vector<int2> out;
  for (auto& v : c) out.push_back(make_int2(v.dy, v.dx));
  return out;
}

int validate(const cc_config* c) {
  if (!c) return CC_EINVAL;
  if (c->levels != kLevels) return CC_EINVAL;
  if (c->arm_ctx != 8 && c->arm_ctx != 16 && c->arm_ctx != 24) return CC_EINVAL;
  if (c->arm_layers != 1 && c->arm_layers != 2) return CC_EINVAL;
  if (c->up_kernel != 4 && c->up_kernel != 8) return CC_EINVAL;
  if (c->up_per_level != 0 && c->up_per_level != 1) return CC_EINVAL;
  if (c->syn_hidden != 8 && c->syn_hidden != 16 && c->syn_hidden != 40) return CC_EINVAL;
  if (c->syn_res3x3 != 1 && c->syn_res3x3 != 2) return CC_EINVAL;
  if (!(c->lam >= 0.f) || !(c->lr > 0.f) || c->total_iters < 0) return CC_EINVAL;
  if (!(c->ste_frac >= 0.f && c->ste_frac <= 1.f)) return CC_EINVAL;
  if (!(c->soft_temp >= 0.f && c->soft_temp < 1e30f)) return CC_EINVAL;
  return CC_OK;
}

Arch arch_of(const cc_config* c) {
  Arch a;
  a.N = c->arm_ctx; a.NL = c->arm_layers; a.K = c->up_kernel; a.per_level = c->up_per_level;
  a.C = c->syn_hidden; a.NR = c->syn_res3x3;
  return a;
}

Layout layout_of(const Arch& a) {
  Layout l;
  l.n_arm = a.NL * (a.N * a.N + a.N) + 2 * a.N + 2;
  l.up0 = l.n_arm;
  l.n_up = a.per_level ? kLevels - 1 : 1;
  l.syn0 = l.up0 + l.n_up * a.K * a.K;
  l.n_syn = 11 * a.C + 3 + a.NR * 84;
  l.total = l.syn0 + l.n_syn;
  return l;
}

Geo geo_of(int H, int W) {
  Geo g;
  g.H = H; g.W = W;
  long long off = 0;
  g.n_lat = 0;
  for (int l = 0; l < kLevels; ++l) {
    g.h[l] = (H + (1 << l) - 1) >> l;
    g.w[l] = (W + (1 << l) - 1) >> l;
    g.off[l] = off;
    off = align32(off + (long long)g.h[l] * g.w[l]);
    g.n_lat += g.h[l] * g.w[l];
  }
  g.n_pad = off;
  off = 0;
  for (int l = 0; l < kLevels; ++l) {
    g.pw[l] = (g.w[l] + 2 * kCtxPad + 3) & ~3;   // 16-byte rows (tensor-map stride)
    g.poff[l] = off;
    off = align32(off + (long long)(g.h[l] + kCtxPad) * g.pw[l]);
  }
  g.n_bord = off;
  return g;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

}  // namespace

void cc::set_error_text(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

struct cc_ctx {
  cc_config cfg;
  Arch arch;
  Layout lay;
  Geo geo;
  int HW = 0;
  int ste_start = 0;
  int dev = 0;
  cudaStream_t st = nullptr;
  cudaStream_t cap = nullptr;
  cudaStream_t side = nullptr;        // ARM branch of a pass, concurrent with the synthesis
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_chain = nullptr;   // upsampling adjoint done (main)
  cudaEvent_t ev_syn = nullptr;     // synthesis adjoint done (main)
  cudaEvent_t ev_red = nullptr;     // ARM, synthesis and 3x3 partials reduced (side)
  cudaStream_t up_st = nullptr;                         // image uploads
  cudaEvent_t ev_planar = nullptr, ev_uploaded = nullptr;
  cudaEvent_t ev_a0 = nullptr, ev_a1 = nullptr;   // timing of the ARM kernel in forked passes
  bool own_mem = false;
  void* mem = nullptr;
  size_t bytes = 0;
  float *x, *y, *my, *vy, *yhat, *yhat_bord, *gsyn, *gself, *dctx, *noise;
  float* dq;   // d y_hat / d y of the soft-rounding proxy
  float *params, *mp, *vp;
  float *hbuf, *dhbuf, *dz;
  float *part_arm, *part_bits, *part_d, *part_conv, *part_syn, *part_up, *part2;
  float* grad_scratch;
  uint8_t* img_u8;
  int2 *tiles, *offs;
  void *arm_image, *syn_image;   // constant-bank images built on the device
  int4* slot_map;                // parameter -> image slots (ImageSlots)
  IterScalars* sc;
  double* log;
  UpPlan up;
  std::vector<int2> h_tiles, h_offs;
  int n_tiles = 0, grid_arm = 0, grid_syn = 0, grid_tiles = 0, slices = kSlices, n_virtual = 0;
  SectionTable tab;                   // every section of the parameter gradient
  SectionTable tab_early, tab_late;   // the same split: ARM / 1x1 / 3x3, then upsampling
  ArmMaps maps;   // tensor maps of the zero-bordered y_hat planes (ARM context tiles)
  cudaGraphExec_t g1 = nullptr, g16 = nullptr;
  int iter = 0;
  int kernels_per_iter = 0;
  // device copy of the state taken before each chunk of cc_encode_iters_checked
  float *snap_y, *snap_my, *snap_vy, *snap_p, *snap_mp, *snap_vp;
  IterScalars* snap_sc;
};

namespace {

// Lay out every buffer in one allocation; with base == nullptr only the size is computed.
size_t plan(cc_ctx* c, char* base) {
  size_t off = 0;
  auto take = [&](size_t nbytes) -> char* {
    char* p = base ? base + off : nullptr;
    off = (off + nbytes + 255) & ~(size_t)255;
    return p;
  };
  const Geo& g = c->geo;
  const Arch& a = c->arch;
  const size_t HW = (size_t)c->HW;
  const size_t L = (size_t)g.n_pad * sizeof(float);
  c->x = (float*)take(3 * HW * sizeof(float));
  c->y = (float*)take(L);
  c->my = (float*)take(L);
  c->vy = (float*)take(L);
  c->yhat = (float*)take(L);
  c->yhat_bord = (float*)take((size_t)g.n_bord * sizeof(float));
  c->gsyn = (float*)take(L);
  c->gself = (float*)take(L);
  c->noise = (float*)take(L);
  c->dq = (float*)take(L);
  c->dctx = (float*)take((size_t)a.N * L);
  c->params = (float*)take((size_t)c->lay.total * sizeof(float));
  c->mp = (float*)take((size_t)c->lay.total * sizeof(float));
  c->vp = (float*)take((size_t)c->lay.total * sizeof(float));
  c->hbuf = (float*)take((size_t)(a.NR + 1) * 3 * HW * sizeof(float));
  c->dhbuf = (float*)take((size_t)(a.NR + 1) * 3 * HW * sizeof(float));
  c->dz = (float*)take(3 * HW * sizeof(float));
  c->part_arm = (float*)take((size_t)c->grid_arm * c->lay.n_arm * sizeof(float));
  c->part_bits = (float*)take((size_t)c->grid_arm * sizeof(float));
  c->part_d = (float*)take((size_t)c->grid_tiles * sizeof(float));
  c->part_conv = (float*)take((size_t)a.NR * c->grid_tiles * 84 * sizeof(float));
  c->part_syn = (float*)take((size_t)c->grid_tiles * (11 * a.C + 3) * sizeof(float));
  c->part_up = (float*)take((size_t)(kLevels - 1) * c->grid_syn * kLevels * a.K * a.K *
                            sizeof(float));
  c->part2 = (float*)take((size_t)c->slices * c->n_virtual * sizeof(float));
  c->grad_scratch = (float*)take((size_t)(g.n_lat + c->lay.total) * sizeof(float));
  c->img_u8 = (uint8_t*)take(3 * HW);
  c->tiles = (int2*)take((size_t)c->n_tiles * sizeof(int2));
  c->offs = (int2*)take(24 * sizeof(int2));
  c->slot_map = (int4*)take((size_t)c->lay.total * sizeof(int4));
  c->arm_image = take(arm_image_bytes());
  c->syn_image = take(syn_image_bytes());
  c->sc = (IterScalars*)take(sizeof(IterScalars));
  c->log = (double*)take((size_t)kLogCap * 3 * sizeof(double));
  c->snap_y = (float*)take(L);
  c->snap_my = (float*)take(L);
  c->snap_vy = (float*)take(L);
  c->snap_p = (float*)take((size_t)c->lay.total * sizeof(float));
  c->snap_mp = (float*)take((size_t)c->lay.total * sizeof(float));
  c->snap_vp = (float*)take((size_t)c->lay.total * sizeof(float));
  c->snap_sc = (IterScalars*)take(sizeof(IterScalars));
  for (int l = 1; l < kLevels; ++l)
    for (int j = 0; j < l; ++j) {
      const size_t n = (size_t)align32((long long)g.h[j] * g.w[j]) * sizeof(float);
      c->up.plane[l][j] = (float*)take(n);
      c->up.dplane[l][j] = (float*)take(n);
    }
  return off;
}

int setup(cc_ctx* c, const cc_config* cfg, int H, int W) {
  int e = validate(cfg);
  if (e) return e;
  if (H < 1 || W < 1 || H > 16384 || W > 16384) return CC_EINVAL;
  c->cfg = *cfg;
  c->arch = arch_of(cfg);
  c->lay = layout_of(c->arch);
  c->geo = geo_of(H, W);
  c->HW = H * W;
  // round half to even (the default rounding mode), the rule of rint for the latents too
  c->ste_start = (int)std::nearbyint((double)cfg->total_iters * (1.0 - (double)cfg->ste_frac));
  c->h_tiles.clear();
  // ARM tiles: blocks of kArmTileY x kArmTileX latents of one level, (level, y0 << 16 | x0)
  for (int l = 0; l < kLevels; ++l)
    for (int y0 = 0; y0 < c->geo.h[l]; y0 += kArmTileY)
      for (int x0 = 0; x0 < c->geo.w[l]; x0 += kArmTileX)
        c->h_tiles.push_back(make_int2(l, (y0 << 16) | x0));
  c->n_tiles = (int)c->h_tiles.size();
  const int sms = sm_count();
  if (sms <= 0) return fail_cuda(cudaErrorNoDevice, "cudaDeviceGetAttribute");
  // the ARM kernel runs beside the synthesis chain: it gets a share of the SMs
  // (CC_ARM_SM_SHARE, default 0.52: measured best against 0.48 and 0.5 at 512 x 768), the
  // rest stay free for the chain's kernels
  double share = 0.52;
  if (const char* env = getenv("CC_ARM_SM_SHARE")) share = atof(env);
  share = share < 0.05 ? 0.05 : (share > 1.0 ? 1.0 : share);
  const int arm_sms = std::max(1, (int)std::lround(share * sms));
  c->grid_arm = std::min(c->n_tiles, arm_sms * arm_blocks_per_sm(c->arch, true));
  c->grid_syn = std::max(1, std::min((c->HW + kPixTile - 1) / kPixTile, 2 * sms));
  // synthesis: CC_SYN_CTAS_PER_SM (default 4) CTAs per SM loop over the 8 x 32 tiles, so
  // that each sums its weight-gradient registers once for several tiles
  int syn_per_sm = 4;
  if (const char* env = getenv("CC_SYN_CTAS_PER_SM")) syn_per_sm = std::max(1, std::min(64, atoi(env)));
  c->grid_tiles = std::max(1, std::min(syn_tile_count(c->geo), syn_per_sm * sms));
  const int n1x1 = 11 * c->arch.C + 3;
  const int vconv = c->lay.n_arm + n1x1;
  const int vup = vconv + c->arch.NR * 84;
  const int K2 = c->arch.K * c->arch.K;
  c->n_virtual = vup + (kLevels - 1) * K2;
  c->h_offs = causal_offsets(c->arch.N);
  return CC_OK;
}

void build_sections(cc_ctx* c) {
  SectionTable& t = c->tab;
  const Arch& a = c->arch;
  const int n1x1 = 11 * a.C + 3;
  const int K2 = a.K * a.K;
  int n = 0;
  t.s[n++] = {c->part_arm, c->grid_arm, c->lay.n_arm, c->lay.n_arm, 0,
              (float)((double)c->cfg.lam / (double)c->HW)};
  t.s[n++] = {c->part_syn, c->grid_tiles, n1x1, n1x1, c->lay.n_arm, 1.f};
  for (int i = 0; i < a.NR; ++i)
    t.s[n++] = {c->part_conv + (size_t)i * c->grid_tiles * 84, c->grid_tiles, 84, 84,
                c->lay.n_arm + n1x1 + 84 * i, 1.f};
  const int vup = c->lay.n_arm + n1x1 + 84 * a.NR;
  for (int l = 1; l < kLevels; ++l)
    t.s[n++] = {c->part_up + (size_t)l * K2, l * c->grid_syn, K2, kLevels * K2,
                vup + (l - 1) * K2, 1.f};
  t.n = n;
  const int n_early = 2 + a.NR;
  c->tab_early.n = n_early;
  for (int i = 0; i < n_early; ++i) c->tab_early.s[i] = t.s[i];
  c->tab_late.n = n - n_early;
  for (int i = n_early; i < n; ++i) c->tab_late.s[i - n_early] = t.s[i];
}

// Whether a pass quantising with mode qmode used the soft-rounding proxy: 0 never (no
// temperature, or rint), 1 always (given or drawn noise), 2 in the noise phase of the
// schedule (decided on the device from the iteration index).
int soft_mode(const cc_ctx* c, int qmode) {
  if (!(c->cfg.soft_temp > 0.f) || qmode == 1) return 0;
  return qmode == 0 ? 2 : 1;
}

ImageSlots image_slots(cc_ctx* c) {
  ImageSlots sl;
  sl.map = c->slot_map;
  sl.arm_image = (float*)c->arm_image;
  sl.syn_image = (float*)c->syn_image;
  return sl;
}

// Rebuild both bank images from the parameters (after the host wrote them).
cudaError_t rebuild_images(cc_ctx* c, cudaStream_t st) {
  cudaError_t e = arm_build_image(c->params, c->lay.n_arm, c->offs, c->arch.N, c->arm_image, st);
  return e != cudaSuccess ? e : syn_build_image(c->params, c->lay, c->arch, c->syn_image, st);
}

// The parameter slots of the images: build both images from the index parameters
// p[j] = j + 1 (a scratch buffer) and read back where each index landed.  The image
// builders copy parameters without arithmetic, so every slot holds exactly one index.
int build_slot_map(cc_ctx* c) {
  const int total = c->lay.total;
  std::vector<float> idx(total);
  for (int j = 0; j < total; ++j) idx[j] = (float)(j + 1);
  float* scratch = c->grad_scratch;
  CK(cudaMemcpyAsync(scratch, idx.data(), (size_t)total * sizeof(float), cudaMemcpyHostToDevice,
                     c->st));
  CK(arm_build_image(scratch, c->lay.n_arm, c->offs, c->arch.N, c->arm_image, c->st));
  CK(syn_build_image(scratch, c->lay, c->arch, c->syn_image, c->st));
  const int na = arm_image_weight_floats(), ns = syn_image_weight_floats();
  std::vector<float> ia(na), is(ns);
  CK(cudaMemcpyAsync(ia.data(), c->arm_image, (size_t)na * sizeof(float), cudaMemcpyDeviceToHost,
                     c->st));
  CK(cudaMemcpyAsync(is.data(), c->syn_image, (size_t)ns * sizeof(float), cudaMemcpyDeviceToHost,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
  std::vector<int4> map(total, make_int4(-1, -1, -1, -1));
  auto add = [&](const std::vector<float>& img, bool arm) -> bool {
    for (size_t p = 0; p < img.size(); ++p) {
      const float v = img[p];
      if (!(v > 0.5f)) continue;
      const int j = (int)(v + 0.5f) - 1;
      if (j < 0 || j >= total) return false;
      int& a = arm ? map[j].x : map[j].z;
      int& b = arm ? map[j].y : map[j].w;
      if (a < 0) a = (int)p;
      else if (b < 0) b = (int)p;
      else return false;   // more than two slots: not a copy layout
    }
    return true;
  };
  if (!add(ia, true) || !add(is, false)) {
    set_error_text("bank image layout: a parameter has more than two slots");
    return CC_EINVAL;
  }
  CK(cudaMemcpyAsync(c->slot_map, map.data(), (size_t)total * sizeof(int4), cudaMemcpyHostToDevice,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
  return CC_OK;
}

// One pass of the hot path.  qmode: quantisation mode of k_quantize.  backward: run the
// backward kernels (and the update when apply).  grad_out: device buffer receiving dL/dy
// then dL/dparams, or nullptr.
// With ev (per-phase timing) every kernel runs in order on s; otherwise the ARM kernel
// runs on the side stream, concurrently with the upsampling and synthesis chain, and the
// reductions wait for both.
cudaError_t enqueue_pass(cc_ctx* c, cudaStream_t s, int qmode, bool backward, bool apply,
                         float* grad_out, bool advance, cudaEvent_t* ev = nullptr) {
  const Arch& a = c->arch;
  const size_t HW = (size_t)c->HW;
  auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
  const bool fork = ev == nullptr;
  cudaStream_t sa = fork ? c->side : s;
  CKE(mark(0));
  // the bank images track the parameters (image_slots); copy them into the banks
  CKE(arm_copy_bank(c->arm_image, s));
  CKE(syn_copy_bank(c->syn_image, s));
  CKE(quantize_launch(c->geo, c->y, c->yhat, c->yhat_bord, c->noise, qmode, c->sc, c->ste_start, c->cfg.seed,
                      -1, c->cfg.soft_temp, c->dq, s));
  CKE(mark(1));
  if (fork) {
    CKE(cudaEventRecord(c->ev_fork, s));
    CKE(cudaStreamWaitEvent(sa, c->ev_fork, 0));
  }
  // timing events around the ARM kernel: graph nodes when the pass is being captured
  auto record_on_side = [&](cudaEvent_t e) -> cudaError_t {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(sa, &cs);
    if (err != cudaSuccess) return err;
    return cs == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(e, sa, cudaEventRecordExternal)
               : cudaEventRecord(e, sa);
  };
  if (fork) CKE(record_on_side(c->ev_a0));
  CKE(arm_launch(a, backward, c->yhat_bord, c->geo, c->maps, c->tiles, c->n_tiles, c->grid_arm,
                 c->dctx, c->gself, c->part_arm, c->part_bits, &c->sc->fault,
                 &c->sc->arm_stall, sa));
  if (fork) CKE(record_on_side(c->ev_a1));
  // with gradients, the side stream continues once the synthesis adjoint is enqueued (below)
  if (fork && !backward) CKE(cudaEventRecord(c->ev_join, sa));
  CKE(mark(2));
  CKE(up_forward(a, c->geo, c->yhat, c->up, c->grid_syn, s));
  CKE(mark(3));
  // with gradients and two 3x3 layers, one kernel runs the 3x3 layers' forward and backward
  const bool pair = backward && a.NR == 2;
  CKE(syn_forward(a, c->geo, c->yhat, c->up, c->x, c->hbuf, c->dhbuf + (size_t)a.NR * 3 * HW,
                  c->part_d, c->part_conv, c->grid_tiles, s,
                  pair ? c->dhbuf + (size_t)3 * HW : nullptr, pair ? c->dz : nullptr));
  CKE(mark(4));
  if (backward) {
    PassFinish pf;
    pf.part_d = c->part_d; pf.nd = c->grid_tiles; pf.part_bits = c->part_bits;
    pf.nb = c->grid_arm; pf.d_scale = 1.0 / (3.0 * (double)HW); pf.r_scale = 1.0 / (double)HW;
    pf.lam = (double)c->cfg.lam; pf.log = c->log;
    CKE(syn_backward(a, c->geo, c->yhat, c->up, c->hbuf, c->dhbuf, c->dz, c->gsyn, c->part_conv,
                     c->part_syn, c->grid_tiles, s, pair));
    if (fork) {
      // after the ARM kernel and the synthesis adjoint, the side stream reduces the ARM,
      // 1x1 and 3x3 partials and those of D and R, then gathers the context gradients, while
      // the upsampling adjoint runs; only the upsampling partials are reduced at the end.
      // (Timed per phase, the gather runs after the upsampling adjoint instead, so that the
      // phase events stay in stream order.)  Measured against the gather first, or the
      // reductions on a third stream: 1-4 us shorter per iteration.
      CKE(cudaEventRecord(c->ev_syn, s));
      CKE(cudaStreamWaitEvent(sa, c->ev_syn, 0));
      CKE(reduce_sections(c->tab_early, c->part2, c->n_virtual, c->slices, sa));
      CKE(pass_loss(pf, c->sc, sa));
      CKE(cudaEventRecord(c->ev_red, sa));
      CKE(ctx_gather(c->geo, c->offs, a.N, c->gself, c->dctx, sa));
    }
    CKE(mark(5));
    CKE(up_backward(a, c->geo, c->yhat, c->up, c->gsyn, c->part_up, c->grid_syn, s));
    CKE(mark(6));
    // the parameter update (after the reduction of the partial sums) and the latent update
    // are independent; forked, they run at once and the last block of either finishes
    // the pass
    const unsigned tickets = latent_update_blocks(c->geo) + param_update_blocks(c->lay);
    const float rate_scale = (float)((double)c->cfg.lam / (double)c->HW);
    auto latents = [&](cudaStream_t q) {
      return latent_update(c->geo, c->gsyn, c->gself, rate_scale, c->y, c->my, c->vy, grad_out,
                           apply, c->cfg.lr, c->sc, pf, tickets, advance, c->dq,
                           soft_mode(c, qmode), c->ste_start, q);
    };
    if (fork) {
      CKE(cudaEventRecord(c->ev_chain, s));
      CKE(cudaStreamWaitEvent(sa, c->ev_chain, 0));
      CKE(latents(sa));
      CKE(cudaStreamWaitEvent(s, c->ev_red, 0));
      CKE(reduce_sections(c->tab_late, c->part2, c->n_virtual, c->slices, s));
    } else {
      CKE(ctx_gather(c->geo, c->offs, a.N, c->gself, c->dctx, s));
      CKE(reduce_sections(c->tab, c->part2, c->n_virtual, c->slices, s));
      CKE(pass_loss(pf, c->sc, s));
    }
    CKE(param_update(c->lay, a, c->part2, c->slices, c->params, c->mp, c->vp,
                     grad_out ? grad_out + c->geo.n_lat : nullptr, apply, c->cfg.lr, c->sc,
                     image_slots(c), &pf, tickets, advance, s));
    if (fork) {
      CKE(cudaEventRecord(c->ev_join, sa));
      CKE(cudaStreamWaitEvent(s, c->ev_join, 0));
    } else {
      CKE(latents(s));
    }
  } else {
    if (fork) CKE(cudaStreamWaitEvent(s, c->ev_join, 0));
    CKE(finish_iteration(c->part_d, c->grid_tiles, c->part_bits, c->grid_arm,
                         1.0 / (3.0 * (double)HW), 1.0 / (double)HW, (double)c->cfg.lam, c->sc,
                         c->log, advance, s, false));
  }
  return mark(7);
}

int build_graph(cc_ctx* c, int n, cudaGraphExec_t* out) {
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < n && err == cudaSuccess; ++k)
    err = enqueue_pass(c, c->cap, 0, true, true, nullptr, true);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
  if (err != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail_cuda(err, "iteration capture");
  }
  if (e2 != cudaSuccess) return fail_cuda(e2, "cudaStreamEndCapture");
  if (n == 1) {
    size_t nn = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess) {
      std::vector<cudaGraphNode_t> nodes(nn);
      cudaGraphGetNodes(graph, nodes.data(), &nn);
      int k = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
      }
      c->kernels_per_iter = k;
    }
  }
  cudaError_t e3 = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return fail_cuda(e3, "cudaGraphInstantiate");
  return CC_OK;
}

void default_params(const cc_ctx* c, std::vector<float>& p) {
  // splitmix64 (Steele, Lea & Flood, OOPSLA 2014) keyed by the seed
  uint64_t s = c->cfg.seed ^ 0x2545F4914F6CDD1Dull;
  auto next = [&]() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto uni = [&](int fan_in) {
    const double u = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
    return (float)((2.0 * u - 1.0) / std::sqrt((double)fan_in));
  };
  const Arch& a = c->arch;
  const Layout& L = c->lay;
  p.assign(L.total, 0.f);
  int k = 0;
  for (int i = 0; i < a.NL; ++i) {
    for (int j = 0; j < a.N * a.N; ++j) p[k++] = uni(a.N);
    k += a.N;
  }
  for (int j = 0; j < 2 * a.N; ++j) p[k++] = uni(a.N);
  k += 2;
  // upsampling: 2x resampling filter (Keys cubic, a = -0.75, for k = 8; linear for k = 4)
  auto keys = [](double x) {
    const double A = -0.75;
    x = std::fabs(x);
    if (x <= 1) return (A + 2) * x * x * x - (A + 3) * x * x + 1;
    if (x < 2) return A * x * x * x - 5 * A * x * x + 8 * A * x - 4 * A;
    return 0.0;
  };
  std::vector<double> f1;
  if (a.K == 8) {
    for (double d : {1.75, 1.25, 0.75, 0.25, 0.25, 0.75, 1.25, 1.75}) f1.push_back(keys(d));
  } else {
    f1 = {0.25, 0.75, 0.75, 0.25};
  }
  for (int f = 0; f < L.n_up; ++f)
    for (int u = 0; u < a.K; ++u)
      for (int v = 0; v < a.K; ++v) p[k++] = (float)(f1[u] * f1[v]);
  for (int j = 0; j < a.C * kLevels; ++j) p[k++] = uni(kLevels);
  k += a.C;
  for (int j = 0; j < 3 * a.C; ++j) p[k++] = uni(a.C);
  k += 3;
  for (int i = 0; i < a.NR; ++i) {
    for (int j = 0; j < 81; ++j) p[k++] = uni(27);
    k += 3;
  }
}

int init_common(const cc_config* cfg, const uint8_t* rgb_hwc, int H, int W,
                const float* init_params, void* stream, void* ws, size_t ws_bytes, cc_ctx** out) {
  if (!out || !rgb_hwc) return CC_EINVAL;
  *out = nullptr;
  cc_ctx* c = new cc_ctx();
  int e = setup(c, cfg, H, W);
  if (e) { delete c; return e; }
  cudaGetDevice(&c->dev);
  c->st = (cudaStream_t)stream;
  const size_t need = plan(c, nullptr);
  if (ws) {
    if (ws_bytes < need) { delete c; return CC_ENOMEM; }
    c->mem = ws;
    c->own_mem = false;
  } else {
    if (g_fail_next_alloc) {   // host-side fault injection (cc_debug_inject)
      g_fail_next_alloc = false;
      delete c;
      set_error_text("cc_init_image: injected allocation failure");
      return CC_ENOMEM;
    }
    cudaError_t ce = cudaMalloc(&c->mem, need);
    if (ce != cudaSuccess) { delete c; fail_cuda(ce, "cudaMalloc"); return CC_ENOMEM; }
    c->own_mem = true;
  }
  c->bytes = need;
  plan(c, (char*)c->mem);
  build_sections(c);
  if (cudaError_t me = arm_make_maps(c->geo, c->yhat_bord, &c->maps)) {
    cc_free(c);
    return fail_cuda(me, "cuTensorMapEncodeTiled");
  }
  auto bail = [&](int code) { cc_free(c); return code; };
  cudaError_t ce = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return bail(fail_cuda(ce, "cudaStreamCreate"));
  if ((ce = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(fail_cuda(ce, "cudaStreamCreate"));
  if ((ce = cudaStreamCreateWithFlags(&c->up_st, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(fail_cuda(ce, "cudaStreamCreate"));
  if ((ce = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&c->ev_chain, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&c->ev_syn, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&c->ev_red, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&c->ev_planar, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&c->ev_uploaded, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventCreate(&c->ev_a0)) != cudaSuccess ||
      (ce = cudaEventCreate(&c->ev_a1)) != cudaSuccess)
    return bail(fail_cuda(ce, "cudaEventCreate"));
  if ((ce = arm_prepare(c->arch)) != cudaSuccess) return bail(fail_cuda(ce, "arm_prepare"));
  if ((ce = syn_prepare(c->arch)) != cudaSuccess) return bail(fail_cuda(ce, "syn_prepare"));
  if ((ce = cudaMemsetAsync(c->mem, 0, need, c->st)) != cudaSuccess)
    return bail(fail_cuda(ce, "cudaMemsetAsync"));
  if ((ce = cudaMemcpyAsync(c->img_u8, rgb_hwc, (size_t)3 * c->HW, cudaMemcpyDefault, c->st)))
    return bail(fail_cuda(ce, "image copy"));
  if ((ce = image_to_planar(c->img_u8, c->x, H, W, c->st))) return bail(fail_cuda(ce, "image"));
  if ((ce = cudaEventRecord(c->ev_planar, c->st))) return bail(fail_cuda(ce, "event"));
  std::vector<float> hp;
  const float* src = init_params;
  if (!src) {
    default_params(c, hp);
    src = hp.data();
  }
  if ((ce = cudaMemcpyAsync(c->params, src, (size_t)c->lay.total * sizeof(float),
                            cudaMemcpyDefault, c->st)))
    return bail(fail_cuda(ce, "params copy"));
  const IterScalars sc0 = iter_scalars_at(0);
  if ((ce = cudaMemcpyAsync(c->sc, &sc0, sizeof(sc0), cudaMemcpyHostToDevice, c->st)))
    return bail(fail_cuda(ce, "scalars copy"));
  if ((ce = adam_bc_upload(c->st))) return bail(fail_cuda(ce, "Adam bias-correction table"));
  if ((ce = cudaMemcpyAsync(c->tiles, c->h_tiles.data(), c->h_tiles.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, c->st)))
    return bail(fail_cuda(ce, "tiles copy"));
  if ((ce = cudaMemcpyAsync(c->offs, c->h_offs.data(), c->h_offs.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, c->st)))
    return bail(fail_cuda(ce, "offsets copy"));
  if (int me = build_slot_map(c)) return bail(me);
  if ((ce = rebuild_images(c, c->st)) != cudaSuccess) return bail(fail_cuda(ce, "bank images"));
  if ((ce = cudaStreamSynchronize(c->st))) return bail(fail_cuda(ce, "init sync"));
  *out = c;
  return CC_OK;
}

int sync_copy_scalars(cc_ctx* c, IterScalars* h) {
  CK(cudaMemcpyAsync(h, c->sc, sizeof(IterScalars), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (h->fault) {
    set_error_text("a context-load wait of the ARM kernel gave up; results are invalid");
    return CC_ETIMEOUT;
  }
  return CC_OK;
}

// latent-shaped device buffer <-> flat latent order at `flat` (host or device)
int copy_latents(cc_ctx* c, float* dev, float* flat, bool to_flat) {
  long long fo = 0;
  for (int l = 0; l < kLevels; ++l) {
    const size_t n = (size_t)c->geo.h[l] * c->geo.w[l];
    if (to_flat)
      CK(cudaMemcpyAsync(flat + fo, dev + c->geo.off[l], n * sizeof(float), cudaMemcpyDefault, c->st));
    else
      CK(cudaMemcpyAsync(dev + c->geo.off[l], flat + fo, n * sizeof(float), cudaMemcpyDefault, c->st));
    fo += (long long)n;
  }
  return CC_OK;
}

cudaError_t copy_log(cc_ctx* c, int first, int count, double* out, cudaMemcpyKind kind);

// The host is writing new state: forget that an earlier pass saw non-finite values.
cudaError_t clear_nonfinite(cc_ctx* c) {
  static const int zero = 0;
  return cudaMemcpyAsync(&c->sc->nonfinite, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st);
}

// Device-to-device copies of the optimisation state (latents, parameters, Adam moments,
// iteration scalars) into (save) or out of (restore) the snapshot buffers.
cudaError_t snapshot_copy(cc_ctx* c, bool save) {
  const size_t L = (size_t)c->geo.n_pad * sizeof(float);
  const size_t P = (size_t)c->lay.total * sizeof(float);
  struct { float* live; float* snap; size_t n; } b[6] = {
      {c->y, c->snap_y, L}, {c->my, c->snap_my, L}, {c->vy, c->snap_vy, L},
      {c->params, c->snap_p, P}, {c->mp, c->snap_mp, P}, {c->vp, c->snap_vp, P}};
  for (auto& x : b)
    CKE(cudaMemcpyAsync(save ? x.snap : x.live, save ? x.live : x.snap, x.n,
                        cudaMemcpyDeviceToDevice, c->st));
  return cudaMemcpyAsync(save ? (void*)c->snap_sc : (void*)c->sc,
                         save ? (void*)c->sc : (void*)c->snap_sc, sizeof(IterScalars),
                         cudaMemcpyDeviceToDevice, c->st);
}

}  // namespace

extern "C" {

int cc_param_count(const cc_config* cfg, int* n_params) {
  if (!n_params) return CC_EINVAL;
  int e = validate(cfg);
  if (e) return e;
  *n_params = layout_of(arch_of(cfg)).total;
  return CC_OK;
}

int cc_latent_count(const cc_config* cfg, int H, int W, int* n_latents) {
  if (!n_latents || H < 1 || W < 1) return CC_EINVAL;
  int e = validate(cfg);
  if (e) return e;
  *n_latents = geo_of(H, W).n_lat;
  return CC_OK;
}

int cc_workspace_size(const cc_config* cfg, int H, int W, size_t* bytes) {
  if (!bytes) return CC_EINVAL;
  cc_ctx c;
  int e = setup(&c, cfg, H, W);
  if (e) return e;
  *bytes = plan(&c, nullptr);
  return CC_OK;
}

int cc_init_image(const cc_config* cfg, const uint8_t* rgb_hwc, int H, int W,
                  const float* init_params, void* cuda_stream, cc_ctx** out) {
  return init_common(cfg, rgb_hwc, H, W, init_params, cuda_stream, nullptr, 0, out);
}

int cc_init_image_ws(const cc_config* cfg, const uint8_t* rgb_hwc, int H, int W,
                     const float* init_params, void* cuda_stream, void* device_workspace,
                     size_t ws_bytes, cc_ctx** out) {
  if (!device_workspace) return CC_EINVAL;
  return init_common(cfg, rgb_hwc, H, W, init_params, cuda_stream, device_workspace, ws_bytes,
                     out);
}

int cc_set_image(cc_ctx* c, const uint8_t* rgb_hwc) {
  if (!c || !rgb_hwc) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  // the copy runs on its own stream as soon as the previous image has been converted, so
  // that it overlaps the iterations still running; only the conversion waits for them
  CK(cudaStreamWaitEvent(c->up_st, c->ev_planar, 0));
  CK(cudaMemcpyAsync(c->img_u8, rgb_hwc, (size_t)3 * c->HW, cudaMemcpyDefault, c->up_st));
  CK(cudaEventRecord(c->ev_uploaded, c->up_st));
  CK(cudaStreamWaitEvent(c->st, c->ev_uploaded, 0));
  CK(image_to_planar(c->img_u8, c->x, c->geo.H, c->geo.W, c->st));
  CK(cudaEventRecord(c->ev_planar, c->st));
  return CC_OK;
}

int cc_encode_iters(cc_ctx* c, int n_iters) {
  if (!c || n_iters < 0) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  if (!c->g1) {
    int e = build_graph(c, 1, &c->g1);
    if (e) return e;
  }
  if (n_iters >= 16 && !c->g16) {
    int e = build_graph(c, 16, &c->g16);
    if (e) return e;
  }
  BankTurn turn(c->dev, c->st);
  CK(turn.status());
  int left = n_iters;
  while (left >= 16) {
    CK(cudaGraphLaunch(c->g16, c->st));
    left -= 16;
  }
  while (left > 0) {
    CK(cudaGraphLaunch(c->g1, c->st));
    --left;
  }
  CK(turn.end());
  c->iter += n_iters;
  return CC_OK;
}

int cc_encode_iters_checked(cc_ctx* c, int n_iters, int check_every, int* iters_done) {
  if (!c || !iters_done || n_iters < 0 || check_every < 1 || check_every > kLogCap)
    return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  *iters_done = 0;
  std::vector<double> h;
  while (*iters_done < n_iters) {
    const int k = std::min(check_every, n_iters - *iters_done);
    CK(snapshot_copy(c, true));
    int e = cc_encode_iters(c, k);
    if (e) return e;
    h.resize(3 * (size_t)k);
    CK(copy_log(c, c->iter - k, k, h.data(), cudaMemcpyDeviceToHost));
    IterScalars sc;
    e = sync_copy_scalars(c, &sc);   // waits for the chunk; CC_ETIMEOUT on an ARM wait fault
    bool bad = e != CC_OK || sc.nonfinite;
    for (double v : h) bad = bad || !std::isfinite(v);
    if (bad) {
      // back to the state before the chunk; a one-shot injected fault does not return
      CK(snapshot_copy(c, false));
      const int never = -1, zero = 0;
      CK(cudaMemcpyAsync(&c->sc->nan_at, &never, sizeof(int), cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(&c->sc->fault, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(&c->sc->arm_stall, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
      CK(clear_nonfinite(c));
      CK(rebuild_images(c, c->st));
      CK(cudaStreamSynchronize(c->st));
      c->iter -= k;
      return e != CC_OK ? e : CC_ENONFINITE;
    }
    *iters_done += k;
  }
  return CC_OK;
}

int cc_debug_inject(cc_ctx* c, int fault, int at_iteration) {
  if (fault == CC_FAULT_ALLOC) {
    if (c) return CC_EINVAL;
    g_fail_next_alloc = true;
    return CC_OK;
  }
  if (fault == CC_FAULT_ARM_STALL) {
    if (!c) return CC_EINVAL;
    CK(cudaSetDevice(c->dev));
    const int cycles = 1 << 20;   // about half a millisecond
    CK(cudaMemcpyAsync(&c->sc->arm_stall, &cycles, sizeof(int), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    return CC_OK;
  }
  if (fault != CC_FAULT_NAN_GRAD || !c || at_iteration < c->iter) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  CK(cudaMemcpyAsync(&c->sc->nan_at, &at_iteration, sizeof(int), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return CC_OK;
}

int cc_rd_cost(cc_ctx* c, int hard_round, double* D, double* R_bpp, double* cost) {
  if (!c) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  {
    BankTurn turn(c->dev, c->st);
    CK(turn.status());
    CK(enqueue_pass(c, c->st, hard_round ? 1 : 3, false, false, nullptr, false));
    CK(turn.end());
  }
  IterScalars h;
  int e = sync_copy_scalars(c, &h);
  if (e) return e;
  if (D) *D = h.D;
  if (R_bpp) *R_bpp = h.R;
  if (cost) *cost = h.loss;
  return std::isfinite(h.loss) && !h.nonfinite ? CC_OK : CC_ENONFINITE;
}

int cc_decode(cc_ctx* c, float* rgb_out_hwc) {
  if (!c || !rgb_out_hwc) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  const Arch& a = c->arch;
  const size_t HW = (size_t)c->HW;
  {
    BankTurn turn(c->dev, c->st);
    CK(turn.status());
    CK(syn_upload(c->params, c->lay, a, c->syn_image, c->st));
    CK(quantize_launch(c->geo, c->y, c->yhat, c->yhat_bord, c->noise, 1, c->sc, c->ste_start,
                       c->cfg.seed, -1, 0.f, nullptr, c->st));
    CK(up_forward(a, c->geo, c->yhat, c->up, c->grid_syn, c->st));
    CK(syn_forward(a, c->geo, c->yhat, c->up, c->x, c->hbuf, c->dhbuf + (size_t)a.NR * 3 * HW,
                   c->part_d, c->part_conv, c->grid_tiles, c->st));
    CK(syn_decode(a, c->geo, c->hbuf + (size_t)a.NR * 3 * HW, c->dz, c->st));
    CK(turn.end());
  }
  CK(cudaMemcpyAsync(rgb_out_hwc, c->dz, 3 * HW * sizeof(float), cudaMemcpyDefault, c->st));
  CK(cudaStreamSynchronize(c->st));
  return CC_OK;
}

int cc_forward_backward(cc_ctx* c, const float* noise_override, int hard, float* grads_out,
                        double* D, double* R_bpp, double* loss) {
  if (!c || hard < -1 || hard > 1) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  int qmode = 0;
  if (hard == 1) {
    qmode = 1;
  } else if (noise_override) {
    int e = copy_latents(c, c->noise, const_cast<float*>(noise_override), false);
    if (e) return e;
    qmode = 2;
  } else if (hard == 0) {
    qmode = 3;
  }
  {
    BankTurn turn(c->dev, c->st);
    CK(turn.status());
    CK(enqueue_pass(c, c->st, qmode, true, false, c->grad_scratch, false));
    CK(turn.end());
  }
  if (grads_out)
    CK(cudaMemcpyAsync(grads_out, c->grad_scratch,
                       (size_t)(c->geo.n_lat + c->lay.total) * sizeof(float), cudaMemcpyDefault,
                       c->st));
  IterScalars h;
  int e = sync_copy_scalars(c, &h);
  if (e) return e;
  if (D) *D = h.D;
  if (R_bpp) *R_bpp = h.R;
  if (loss) *loss = h.loss;
  return std::isfinite(h.loss) && !h.nonfinite ? CC_OK : CC_ENONFINITE;
}

int cc_get_grads(cc_ctx* c, const float* noise_override, float* grads_out) {
  return cc_forward_backward(c, noise_override, -1, grads_out, nullptr, nullptr, nullptr);
}

}  // extern "C"

namespace {

// enqueue copies of log entries first .. first+count-1 (one or two contiguous runs of the
// ring) to out (3 doubles per entry)
cudaError_t copy_log(cc_ctx* c, int first, int count, double* out, cudaMemcpyKind kind) {
  int k = 0;
  while (k < count) {
    const int slot = (first + k) % kLogCap;
    const int run = std::min(count - k, kLogCap - slot);
    cudaError_t e = cudaMemcpyAsync(out + 3 * (size_t)k, c->log + 3 * (size_t)slot,
                                    3 * (size_t)run * sizeof(double), kind, c->st);
    if (e != cudaSuccess) return e;
    k += run;
  }
  return cudaSuccess;
}

bool log_range_ok(const cc_ctx* c, int first, int count) {
  return first >= 0 && count >= 0 && first + count <= c->iter && first >= c->iter - kLogCap;
}

}  // namespace

extern "C" {

int cc_get_losses(cc_ctx* c, int first, int count, double* out) {
  if (!c || !out || !log_range_ok(c, first, count)) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  std::vector<double> pick((size_t)count * 3);
  CK(copy_log(c, first, count, pick.data(), cudaMemcpyDeviceToHost));
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(out, pick.data(), pick.size() * sizeof(double), cudaMemcpyDefault));
  for (double v : pick)
    if (!std::isfinite(v)) return CC_ENONFINITE;
  return CC_OK;
}

int cc_get_losses_async(cc_ctx* c, int first, int count, double* out) {
  if (!c || !out || !log_range_ok(c, first, count)) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  CK(copy_log(c, first, count, out, cudaMemcpyDefault));
  return CC_OK;
}

int cc_set_latents(cc_ctx* c, const float* y_flat) {
  if (!c || !y_flat) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  CK(clear_nonfinite(c));
  return copy_latents(c, c->y, const_cast<float*>(y_flat), false);
}

int cc_get_latents(cc_ctx* c, float* y_flat) {
  if (!c || !y_flat) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  int e = copy_latents(c, c->y, y_flat, true);
  if (e) return e;
  CK(cudaStreamSynchronize(c->st));
  return CC_OK;
}

int cc_set_params(cc_ctx* c, const float* params) {
  if (!c || !params) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  CK(clear_nonfinite(c));
  CK(cudaMemcpyAsync(c->params, params, (size_t)c->lay.total * sizeof(float), cudaMemcpyDefault,
                     c->st));
  CK(rebuild_images(c, c->st));
  return CC_OK;
}

int cc_get_params(cc_ctx* c, float* params) {
  if (!c || !params) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  CK(cudaMemcpyAsync(params, c->params, (size_t)c->lay.total * sizeof(float), cudaMemcpyDefault,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
  return CC_OK;
}

int cc_profile_phases(cc_ctx* c, int reps, float* ms_out) {
  if (!c || !ms_out || reps < 1) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  cudaEvent_t ev[8];
  for (int k = 0; k < 8; ++k) CK(cudaEventCreate(&ev[k]));
  double acc[CC_N_PHASES] = {0};
  int rc = CC_OK;
  for (int r = 0; r < reps && rc == CC_OK; ++r) {
    cudaError_t e;
    {
      BankTurn turn(c->dev, c->st);
      e = turn.status();
      if (e == cudaSuccess) e = enqueue_pass(c, c->st, 0, true, true, nullptr, true, ev);
      if (e == cudaSuccess) e = turn.end();
    }
    if (e != cudaSuccess) { rc = fail_cuda(e, "profiled pass"); break; }
    if ((e = cudaEventSynchronize(ev[7])) != cudaSuccess) { rc = fail_cuda(e, "event sync"); break; }
    for (int k = 0; k < CC_N_PHASES; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      acc[k] += ms;
    }
    c->iter += 1;
  }
  for (int k = 0; k < 8; ++k) cudaEventDestroy(ev[k]);
  if (rc) return rc;
  for (int k = 0; k < CC_N_PHASES; ++k) ms_out[k] = (float)(acc[k] / reps);
  return CC_OK;
}

int cc_arm_kernel_ms(cc_ctx* c, float* ms) {
  if (!c || !ms) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  CK(cudaEventSynchronize(c->ev_a1));
  CK(cudaEventElapsedTime(ms, c->ev_a0, c->ev_a1));
  return CC_OK;
}

int cc_graph_kernel_count(cc_ctx* c, int* n_kernels) {
  if (!c || !n_kernels) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  if (!c->g1) {
    int e = build_graph(c, 1, &c->g1);
    if (e) return e;
  }
  *n_kernels = c->kernels_per_iter;
  return CC_OK;
}

int cc_iteration(cc_ctx* c, int* iter) {
  if (!c || !iter) return CC_EINVAL;
  *iter = c->iter;
  return CC_OK;
}

int cc_noise(cc_ctx* c, int iter, float* out) {
  if (!c || !out || iter < 0) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  CK(quantize_launch(c->geo, c->y, c->yhat, c->yhat_bord, c->noise, 4, c->sc, c->ste_start, c->cfg.seed, iter,
                     0.f, nullptr, c->st));
  int e = copy_latents(c, c->yhat, out, true);
  if (e) return e;
  CK(cudaStreamSynchronize(c->st));
  return CC_OK;
}

int cc_get_state(cc_ctx* c, void* buf, size_t* nbytes) {
  if (!c || !nbytes) return CC_EINVAL;
  const size_t nl = (size_t)c->geo.n_lat, np = (size_t)c->lay.total;
  const size_t need = sizeof(StateHeader) + (3 * nl + 3 * np) * sizeof(float);
  if (!buf) {
    *nbytes = need;
    return CC_OK;
  }
  if (*nbytes < need) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  StateHeader hd{};
  hd.magic = kStateMagic; hd.version = kStateVersion;
  hd.H = c->geo.H; hd.W = c->geo.W; hd.n_lat = (int)nl; hd.n_params = (int)np;
  hd.iter = c->iter; hd.seed = c->cfg.seed;
  const int ar[8] = {c->arch.N, c->arch.NL, c->arch.K, c->arch.per_level, c->arch.C, c->arch.NR,
                     kLevels, 0};
  memcpy(hd.arch, ar, sizeof(ar));
  char* p = (char*)buf;
  memcpy(p, &hd, sizeof(hd));
  float* f = (float*)(p + sizeof(hd));
  int e;
  if ((e = copy_latents(c, c->y, f, true))) return e;
  CK(cudaMemcpyAsync(f + nl, c->params, np * sizeof(float), cudaMemcpyDeviceToHost, c->st));
  if ((e = copy_latents(c, c->my, f + nl + np, true))) return e;
  if ((e = copy_latents(c, c->vy, f + 2 * nl + np, true))) return e;
  CK(cudaMemcpyAsync(f + 3 * nl + np, c->mp, np * sizeof(float), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(f + 3 * nl + 2 * np, c->vp, np * sizeof(float), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  *nbytes = need;
  return CC_OK;
}

int cc_set_state(cc_ctx* c, const void* buf, size_t nbytes) {
  if (!c || !buf || nbytes < sizeof(StateHeader)) return CC_EINVAL;
  StateHeader hd;
  memcpy(&hd, buf, sizeof(hd));
  const size_t nl = (size_t)c->geo.n_lat, np = (size_t)c->lay.total;
  const size_t need = sizeof(StateHeader) + (3 * nl + 3 * np) * sizeof(float);
  const int ar[8] = {c->arch.N, c->arch.NL, c->arch.K, c->arch.per_level, c->arch.C, c->arch.NR,
                     kLevels, 0};
  if (hd.magic != kStateMagic || hd.version != kStateVersion || nbytes != need ||
      hd.H != c->geo.H || hd.W != c->geo.W || hd.n_lat != (int)nl || hd.n_params != (int)np ||
      memcmp(hd.arch, ar, sizeof(ar)) != 0 || hd.iter < 0)
    return CC_ESTATE;
  CK(cudaSetDevice(c->dev));
  // the blob may be pageable host memory: stage through a host copy with a lifetime
  std::vector<float> f((3 * nl + 3 * np));
  memcpy(f.data(), (const char*)buf + sizeof(hd), f.size() * sizeof(float));
  int e;
  if ((e = copy_latents(c, c->y, f.data(), false))) return e;
  CK(cudaMemcpyAsync(c->params, f.data() + nl, np * sizeof(float), cudaMemcpyHostToDevice, c->st));
  CK(rebuild_images(c, c->st));
  if ((e = copy_latents(c, c->my, f.data() + nl + np, false))) return e;
  if ((e = copy_latents(c, c->vy, f.data() + 2 * nl + np, false))) return e;
  CK(cudaMemcpyAsync(c->mp, f.data() + 3 * nl + np, np * sizeof(float), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->vp, f.data() + 3 * nl + 2 * np, np * sizeof(float), cudaMemcpyHostToDevice,
                     c->st));
  const IterScalars sc = iter_scalars_at(hd.iter);
  CK(cudaMemcpyAsync(c->sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->iter = hd.iter;
  return CC_OK;
}

// ---- latent bitstream -------------------------------------------------------------------

}  // extern "C"

namespace {

constexpr uint8_t kBsMagic[4] = {'C', 'C', 'F', '1'};
constexpr int kBsFixed = 20;   // magic, H, W, 8 architecture bytes

// device buffer released on scope exit
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  cudaError_t alloc(size_t n) { return cudaMalloc(&p, n ? n : 1); }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

void put_u32(std::vector<uint8_t>& v, uint32_t x) {
  for (int i = 0; i < 4; ++i) v.push_back((uint8_t)(x >> (8 * i)));
}
uint32_t get_u32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
void put_leb128(std::vector<uint8_t>& v, uint32_t x) {
  do {
    const uint8_t b = x & 0x7F;
    x >>= 7;
    v.push_back(b | (x ? 0x80 : 0));
  } while (x);
}
bool get_leb128(const uint8_t* bs, size_t n, size_t& pos, uint32_t& x) {
  x = 0;
  for (int shift = 0; shift < 35; shift += 7) {
    if (pos >= n) return false;
    const uint8_t b = bs[pos++];
    x |= (uint32_t)(b & 0x7F) << shift;
    if (!(b & 0x80)) return true;
  }
  return false;
}

int set_msg(int code, const char* msg) {
  cc::set_error_text(msg);
  return code;
}

int parse_fixed(const uint8_t* bs, size_t n, cc_config* cfg, int* H, int* W) {
  if (!bs || n < (size_t)kBsFixed || std::memcmp(bs, kBsMagic, 4) != 0)
    return set_msg(CC_EINVAL, "not a latent bitstream (magic)");
  const uint32_t h = get_u32(bs + 4), w = get_u32(bs + 8);
  if (h < 1 || w < 1 || h > 16384 || w > 16384) return set_msg(CC_EINVAL, "bitstream image size");
  cc_config c;
  std::memset(&c, 0, sizeof(c));
  c.levels = bs[12]; c.arm_ctx = bs[13]; c.arm_layers = bs[14]; c.up_kernel = bs[15];
  c.up_per_level = bs[16]; c.syn_hidden = bs[17]; c.syn_res3x3 = bs[18];
  c.lam = 0.f; c.lr = 1.f; c.total_iters = 0; c.ste_frac = 0.f; c.seed = 0; c.soft_temp = 0.f;
  if (validate(&c) != CC_OK) return set_msg(CC_EINVAL, "bitstream architecture");
  *cfg = c;
  *H = (int)h;
  *W = (int)w;
  return CC_OK;
}

}  // namespace

extern "C" {

int cc_write_bitstream(cc_ctx* c, uint8_t* out, size_t capacity, size_t* nbytes) {
  if (!c || !nbytes) return CC_EINVAL;
  CK(cudaSetDevice(c->dev));
  const Arch& a = c->arch;
  cudaStream_t st = c->st;
  std::vector<float> p((size_t)c->lay.total);
  CK(cudaMemcpyAsync(p.data(), c->params, p.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<int32_t> q((size_t)c->lay.n_arm);
  if (!codec_quantize_arm(p.data(), a.N, a.NL, q.data()))
    return set_msg(CC_ENONFINITE, "non-finite ARM parameter");
  const CodecGeo cg = codec_geo(c->geo, 32);
  const std::vector<uint16_t>& tab = codec_tables();
  DevBuf d_tab, d_sym, d_rows, d_len, d_flag, d_off, d_out;
  CK(d_tab.alloc(codec_table_bytes()));
  CK(d_sym.alloc((size_t)cg.n_lat * sizeof(int2)));
  CK(d_rows.alloc((size_t)cg.buf_bytes));
  CK(d_len.alloc((size_t)cg.rows * sizeof(int)));
  CK(d_flag.alloc(sizeof(int)));
  CK(d_off.alloc((size_t)cg.rows * sizeof(long long)));
  CK(cudaMemcpyAsync(d_tab.p, tab.data(), codec_table_bytes(), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(d_flag.p, 0, sizeof(int), st));
  {
    BankTurn turn(c->dev, st);
    CK(turn.status());
    CK(codec_upload_arm(q.data(), a.N, a.NL, st));
    CK(codec_symbols(cg, c->geo, c->y, c->offs, a.N, a.NL, d_sym.as<int2>(), d_flag.as<int>(),
                     st));
    CK(turn.end());
  }
  CK(codec_encode_rows(cg, d_sym.as<int2>(), d_tab.as<uint16_t>(), d_rows.as<uint8_t>(),
                       d_len.as<int>(), d_flag.as<int>(), st));
  std::vector<int> len((size_t)cg.rows);
  int flag = 0;
  CK(cudaMemcpyAsync(len.data(), d_len.p, len.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&flag, d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag & 1) return set_msg(CC_EINVAL, "a quantised latent exceeds 2^20 in magnitude");
  if (flag & 2) return set_msg(CC_ECUDA, "substream overran its buffer");

  std::vector<uint8_t> hdr(kBsMagic, kBsMagic + 4);
  put_u32(hdr, (uint32_t)c->geo.H);
  put_u32(hdr, (uint32_t)c->geo.W);
  const uint8_t ab[8] = {(uint8_t)kLevels, (uint8_t)a.N, (uint8_t)a.NL, (uint8_t)a.K,
                         (uint8_t)a.per_level, (uint8_t)a.C, (uint8_t)a.NR, 0};
  hdr.insert(hdr.end(), ab, ab + 8);
  for (int32_t v : q) put_u32(hdr, (uint32_t)v);
  for (int k = c->lay.n_arm; k < c->lay.total; ++k) {
    uint32_t u;
    std::memcpy(&u, &p[(size_t)k], 4);
    put_u32(hdr, u);
  }
  std::vector<long long> off((size_t)cg.rows);
  long long body = 0;
  for (int r = 0; r < cg.rows; ++r) {
    put_leb128(hdr, (uint32_t)len[(size_t)r]);
    off[(size_t)r] = body;
    body += len[(size_t)r];
  }
  const size_t total = hdr.size() + (size_t)body;
  *nbytes = total;
  if (!out) return CC_OK;
  if (capacity < total) return set_msg(CC_ESIZE, "output buffer smaller than the bitstream");
  CK(d_out.alloc((size_t)body));
  CK(cudaMemcpyAsync(d_off.p, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
  CK(codec_pack(cg, d_rows.as<uint8_t>(), d_off.as<long long>(), d_len.as<int>(),
                d_out.as<uint8_t>(), st));
  CK(cudaMemcpyAsync(out, hdr.data(), hdr.size(), cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(out + hdr.size(), d_out.p, (size_t)body, cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  return CC_OK;
}

int cc_bitstream_info(const uint8_t* bs, size_t nbytes, cc_config* cfg, int* H, int* W) {
  if (!cfg || !H || !W) return CC_EINVAL;
  return parse_fixed(bs, nbytes, cfg, H, W);
}

int cc_decode_bitstream(const uint8_t* bs, size_t nbytes, void* cuda_stream, float* rgb_out_hwc,
                        int32_t* latents_out, float* latent_ms) {
  cc_config cfg;
  int H = 0, W = 0;
  int e = parse_fixed(bs, nbytes, &cfg, &H, &W);
  if (e) return e;
  const Arch a = arch_of(&cfg);
  const Layout lay = layout_of(a);
  size_t pos = kBsFixed;
  if (nbytes - pos < (size_t)lay.total * 4) return set_msg(CC_EINVAL, "truncated bitstream (parameters)");
  std::vector<int32_t> q((size_t)lay.n_arm);
  std::vector<float> params((size_t)lay.total);
  for (int k = 0; k < lay.total; ++k, pos += 4) {
    const uint32_t u = get_u32(bs + pos);
    if (k < lay.n_arm) {
      q[(size_t)k] = (int32_t)u;
      params[(size_t)k] = (float)((double)(int32_t)u / 256.0);
    } else {
      std::memcpy(&params[(size_t)k], &u, 4);
    }
  }
  const Geo g = geo_of(H, W);
  const CodecGeo cg = codec_geo(g, 32 / codec_decode_parts(a.N));
  std::vector<long long> row_off((size_t)cg.rows);
  std::vector<int> row_len((size_t)cg.rows);
  long long body = 0;
  for (int r = 0; r < cg.rows; ++r) {
    uint32_t n = 0;
    if (!get_leb128(bs, nbytes, pos, n)) return set_msg(CC_EINVAL, "truncated bitstream (lengths)");
    if (n > (uint32_t)INT32_MAX) return set_msg(CC_EINVAL, "substream length");
    row_off[(size_t)r] = body;
    row_len[(size_t)r] = (int)n;
    body += n;
  }
  if ((long long)(nbytes - pos) != body) return set_msg(CC_EINVAL, "bitstream length mismatch");
  if (!codec_arm_in_range(q.data(), a.N, a.NL))
    return set_msg(CC_EINVAL, "bitstream ARM parameters outside the fixed-point ranges");
  const std::vector<int2> offs = causal_offsets(a.N);
  if (!codec_offsets_match(offs.data(), a.N))
    return set_msg(CC_ECUDA, "decoder context tables disagree with the causal offsets");

  std::vector<uint8_t> zeros((size_t)3 * H * W, 0);
  cc_ctx* c = nullptr;
  if ((e = init_common(&cfg, zeros.data(), H, W, params.data(), cuda_stream, nullptr, 0, &c)))
    return e;
  struct Guard { cc_ctx* c; ~Guard() { cc_free(c); } } guard{c};
  cudaStream_t st = c->st;
  const std::vector<uint16_t>& tab = codec_tables();
  DevBuf d_tab, d_bytes, d_off, d_len, d_planes, d_flag, d_prog;
  CK(d_tab.alloc(codec_table_bytes()));
  CK(d_prog.alloc((size_t)cg.bands * sizeof(int)));
  CK(d_bytes.alloc((size_t)body));
  CK(d_off.alloc((size_t)cg.rows * sizeof(long long)));
  CK(d_len.alloc((size_t)cg.rows * sizeof(int)));
  CK(d_planes.alloc((size_t)cg.n_lat * sizeof(int)));
  CK(d_flag.alloc(sizeof(int)));
  CK(cudaMemcpyAsync(d_tab.p, tab.data(), codec_table_bytes(), cudaMemcpyHostToDevice, st));
  if (body) CK(cudaMemcpyAsync(d_bytes.p, bs + pos, (size_t)body, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_off.p, row_off.data(), row_off.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_len.p, row_len.data(), row_len.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(d_flag.p, 0, sizeof(int), st));
  {
    BankTurn turn(c->dev, st);
    CK(turn.status());
    CK(codec_upload_arm(q.data(), a.N, a.NL, st));
    CK(cudaEventRecord(c->ev_a0, st));
    CK(codec_decode(cg, a.N, a.NL, d_tab.as<uint16_t>(), d_bytes.as<uint8_t>(),
                    d_off.as<long long>(), d_len.as<int>(), d_planes.as<int>(),
                    d_prog.as<int>(), d_flag.as<int>(), st));
    CK(cudaEventRecord(c->ev_a1, st));
    CK(turn.end());
  }
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag & 8) return set_msg(CC_ETIMEOUT, "a decoding band waited too long on the band above");
  if (flag) return set_msg(CC_EINVAL, "corrupt substream (escape code too long)");
  if (latent_ms) CK(cudaEventElapsedTime(latent_ms, c->ev_a0, c->ev_a1));
  if (latents_out)
    CK(cudaMemcpyAsync(latents_out, d_planes.p, (size_t)cg.n_lat * sizeof(int), cudaMemcpyDefault, st));
  CK(codec_to_float(cg, c->geo, d_planes.as<int>(), c->y, st));
  if (rgb_out_hwc) {
    if ((e = cc_decode(c, rgb_out_hwc))) return e;
  }
  CK(cudaStreamSynchronize(st));
  return CC_OK;
}

void cc_free(cc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->g1) cudaGraphExecDestroy(c->g1);
  if (c->g16) cudaGraphExecDestroy(c->g16);
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->up_st) {
    cudaStreamSynchronize(c->up_st);
    cudaStreamDestroy(c->up_st);
  }
  if (c->ev_planar) cudaEventDestroy(c->ev_planar);
  if (c->ev_uploaded) cudaEventDestroy(c->ev_uploaded);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_chain) cudaEventDestroy(c->ev_chain);
  if (c->ev_syn) cudaEventDestroy(c->ev_syn);
  if (c->ev_red) cudaEventDestroy(c->ev_red);
  if (c->ev_a0) cudaEventDestroy(c->ev_a0);
  if (c->ev_a1) cudaEventDestroy(c->ev_a1);
  if (c->own_mem && c->mem) cudaFree(c->mem);
  delete c;
}

const char* cc_strerror(int code) {
  switch (code) {
    case CC_OK: return "ok";
    case CC_EINVAL: return "invalid argument or unsupported configuration";
    case CC_ENOMEM: return "out of device memory or workspace too small";
    case CC_ECUDA: return "CUDA runtime error";
    case CC_ETIMEOUT: return "bounded device wait timed out";
    case CC_ENONFINITE: return "non-finite loss";
    case CC_ESTATE: return "state blob does not match this context";
    case CC_ESIZE: return "output buffer too small (the size needed was returned)";
    default: return "unknown error";
  }
}

const char* cc_last_cuda_error(void) { return g_err; }

}  // extern "C"
