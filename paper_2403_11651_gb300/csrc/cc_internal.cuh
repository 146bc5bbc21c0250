// Internal declarations shared by the translation units of the Cool-chic library.
// Everything here is host/device plumbing; the arithmetic lives in the .cu files.
#pragma once

#include <cuda.h>   // CUtensorMap (types only; the encoder is reached through the runtime)
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <vector>

namespace cc {

constexpr int kLevels = 7;        // L of Sec. II "Decoding" item i (fixed by Table 1 "7-C")
constexpr int kArmTile = 128;     // latents per ARM tile (= threads per ARM block)
constexpr int kArmTileY = 4, kArmTileX = 32;   // an ARM tile: 4 rows x 32 latents of a level
constexpr int kPixTile = 256;     // pixels per synthesis block
constexpr int kLogCap = 4096;     // per-iteration loss log entries kept on the device
constexpr int kSlices = 16;       // slices of the first stage of the parameter-gradient sums

// Latent pyramid geometry.  Every latent-shaped buffer holds the L planes back to back,
// each plane row-major with row stride w_l, starting at a 32-float aligned offset.
struct Geo {
  int H, W;
  int h[kLevels], w[kLevels];
  long long off[kLevels];
  long long n_pad;   // floats in a latent-shaped buffer
  int n_lat;         // sum_l h_l w_l
  // zero-bordered copy of y_hat for the context gather: kCtxPad rows above and kCtxPad
  // columns on each side of every plane, row stride pw[l] = w[l] + 2 kCtxPad
  long long poff[kLevels];
  int pw[kLevels];
  long long n_bord;
};
constexpr int kCtxPad = 4;        // reach of the largest causal context (N = 24)

// Programmatic dependent launch.  Kernels of the upsampling / synthesis / update chain are
// launched (launch_k) with programmatic stream serialisation, so that the next kernel's
// blocks are placed while its predecessor drains.  Every kernel calls pdl_wait() before it
// touches memory: it returns once the kernels it depends on have completed and their
// writes are visible (at once for a kernel launched without the attribute).  pdl_trigger()
// lets the successor be placed; it is issued after the wait, so at most one kernel ahead
// holds blocks that wait.  CC_PDL=0 in the environment turns the attribute off.
#ifndef CC_TRACE
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void trace_point(const char*) {}
#else
// Traced build (all sources in one translation unit): block (0, 0, 0) of every kernel
// records, once its wait returns, the global timer, an FNV-1a hash of the kernel's name
// and its launch shape.
struct TraceRec {
  unsigned long long t;
  unsigned hash;
  int gx, gy, bx;
};
constexpr int kTraceCap = 8192;
__device__ TraceRec g_trace[kTraceCap];
__device__ unsigned g_trace_n;
__device__ __forceinline__ void pdl_wait_traced(const char* name) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (threadIdx.x == 0 && threadIdx.y == 0 && blockIdx.x == 0 && blockIdx.y == 0 &&
      blockIdx.z == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    unsigned h = 2166136261u;
    for (int i = 0; name[i] && i < 64; ++i) h = (h ^ (unsigned char)name[i]) * 16777619u;
    const unsigned k = atomicAdd(&g_trace_n, 1u) % kTraceCap;
    g_trace[k].t = t;
    g_trace[k].hash = h;
    g_trace[k].gx = gridDim.x;
    g_trace[k].gy = gridDim.y;
    g_trace[k].bx = blockDim.x * blockDim.y;
  }
}
#define pdl_wait() pdl_wait_traced(__func__)
// A point inside a kernel, recorded by the calling thread: the global timer, the tag's hash,
// the block index (gx) and gy = -1.
__device__ __forceinline__ void trace_point(const char* tag) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  unsigned h = 2166136261u;
  for (int i = 0; tag[i] && i < 64; ++i) h = (h ^ (unsigned char)tag[i]) * 16777619u;
  const unsigned k = atomicAdd(&g_trace_n, 1u) % kTraceCap;
  g_trace[k].t = t;
  g_trace[k].hash = h;
  g_trace[k].gx = blockIdx.x;
  g_trace[k].gy = -1;
  g_trace[k].bx = 0;
}
#endif
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
bool pdl_enabled();

template <typename... P, typename... A>
cudaError_t launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Architecture (Table 1 notation) as the kernels see it.
struct Arch {
  int N;        // ARM context size and width
  int NL;       // N-N-LinR layers
  int K;        // upsampling kernel
  int per_level;
  int C;        // synthesis hidden width
  int NR;       // 3x3 residual layers
};

// Offsets of the flat parameter vector (same order as include/coolchic.h).
struct Layout {
  int n_arm;          // [0, n_arm): ARM
  int up0, n_up;      // [up0, up0 + n_up * K*K): upsampling filters
  int syn0, n_syn;    // [syn0, syn0 + n_syn): synthesis
  int total;
};

// A block of per-CTA partial sums of some parameter gradients: rows x cols floats,
// row stride `stride`; column j adds into virtual gradient slot col0 + j, times scale.
struct Section {
  const float* part;
  int rows, cols, stride, col0;
  float scale;
};
constexpr int kMaxSections = 12;
struct SectionTable {
  Section s[kMaxSections];
  int n;
};

// a + b as the unevaluated pair (s, e) with s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b, v = s - a;
  return make_float2(s, (a - (s - v)) + (b - v));
}

// (a.x + a.y) + (b.x + b.y) in float-float arithmetic (Dekker): the exact sum of the high
// parts plus the low parts, renormalised.  For sums of non-negative terms the relative
// error is a few units of 2^-44.
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  const float e = s.y + (a.y + b.y);
  const float h = s.x + e;
  return make_float2(h, e - (h - s.x));
}

// Scalars of the current iteration, written on the device.
struct IterScalars {
  int t;              // index of the current iteration (0-based)
  float inv_bc1;      // Adam 1 / (1 - beta1^(t+1)) of the current update
  float inv_sqrt_bc2; // Adam 1 / sqrt(1 - beta2^(t+1))
  int fault;          // set when a bounded context-load wait of the ARM kernel gave up
  double D, R, loss;
  unsigned ticket;    // blocks of the latent update done (reset by the last one)
  int nan_at;         // fault injection: the latent update of this iteration makes the
                      // gradient of latent 0 NaN (-1: never; cc_debug_inject)
  int nonfinite;      // set when a pass read a non-finite latent or an update produced a
                      // non-finite latent or parameter; cleared when the host writes state
  int arm_stall;      // fault injection: > 0 makes the ARM kernel skip its first context
                      // load and wait that many cycles for it (cc_debug_inject)
};
// IterScalars of iteration t, computed on the host (context set-up, state restore).
IterScalars iter_scalars_at(int t);
// Fill the device's table of Adam bias corrections (before the first pass on a device).
cudaError_t adam_bc_upload(cudaStream_t st);

// ---- launchers (each returns the cudaError_t of its launch) ----
// ARM (cc_arm.cu)
// Build the ARM constant-bank image in d_image (arm_image_bytes()) and copy it to the bank.
// Bank images: built on the device from the flat parameters (build_image), copied into
// the __constant__ bank before a pass (copy_bank); upload = both.  Every float of the
// first *_image_weight_floats() of an image is a copy of one parameter (or zero padding).
cudaError_t arm_build_image(const float* d_params, int n_arm, const int2* d_offsets, int N,
                            void* d_image, cudaStream_t st);
cudaError_t arm_copy_bank(const void* d_image, cudaStream_t st);
int arm_image_weight_floats();
cudaError_t syn_build_image(const float* d_params, const Layout& lay, const Arch& a,
                            void* d_image, cudaStream_t st);
cudaError_t syn_copy_bank(const void* d_image, cudaStream_t st);
int syn_image_weight_floats();
cudaError_t arm_upload(const float* d_params, int n_arm, const int2* d_offsets, int N,
                       void* d_image, cudaStream_t st);
size_t arm_image_bytes();
// One tensor map per level over the zero-bordered y_hat plane (width pw, h + kCtxPad rows),
// box of (kArmTileY + kCtxPad) rows x (kArmTileX + 2 kCtxPad) floats: the causal context
// of one ARM tile; reads outside the plane return zeros.
struct ArmMaps {
  CUtensorMap m[kLevels];
};
cudaError_t arm_make_maps(const Geo& g, const float* yhat_bord, ArmMaps* out);
cudaError_t arm_launch(const Arch& a, bool backward, const float* yhat, const Geo& g,
                       const ArmMaps& maps, const int2* tiles, int n_tiles, int grid,
                       float* dctx, float* gself, float* part_grad, float* part_bits,
                       int* fault, const int* stall, cudaStream_t st);
int arm_blocks_per_sm(const Arch& a, bool backward);
cudaError_t arm_prepare(const Arch& a);   // kernel attributes; call once before capture
size_t arm_smem_bytes(const Arch& a, bool backward);

// synthesis + upsampling (cc_syn.cu)
struct UpPlan {
  // planes of level l at resolution j (j < l); j == l is the latent plane itself
  float* plane[kLevels][kLevels];
  float* dplane[kLevels][kLevels];
};
// Build the synthesis / upsampling bank image in d_image (syn_image_bytes()) and copy it.
cudaError_t syn_upload(const float* d_params, const Layout& lay, const Arch& a, void* d_image,
                       cudaStream_t st);
size_t syn_image_bytes();
cudaError_t up_forward(const Arch& a, const Geo& g, const float* yhat, const UpPlan& up,
                       int ctas, cudaStream_t st);
cudaError_t up_backward(const Arch& a, const Geo& g, const float* yhat, const UpPlan& up,
                        float* gsyn, float* part_up, int grid, cudaStream_t st);
// Synthesis kernels run on 8 x 32 pixel tiles; `grid` CTAs loop over syn_tile_count(g)
// tiles and write `grid` rows of partial sums (distortion; 84 per 3x3 layer; 11C + 3).
int syn_tile_count(const Geo& g);
// With dh and dz (two 3-layer with gradients), the forward's 3x3 kernel also computes the
// 3x3 part of the backward (layer 1's input gradient into dh, layer 0's pre-activation
// gradient into dz, both weight gradients); syn_backward is then called with convs_done.
cudaError_t syn_forward(const Arch& a, const Geo& g, const float* yhat, const UpPlan& up,
                        const float* x, float* hbuf, float* dxhat, float* part_d,
                        float* part_conv, int grid, cudaStream_t st, float* dh = nullptr,
                        float* dz = nullptr);
cudaError_t syn_backward(const Arch& a, const Geo& g, const float* yhat, const UpPlan& up,
                         float* hbuf, float* dhbuf, float* dz, float* gsyn,
                         float* part_conv, float* part_syn, int grid, cudaStream_t st,
                         bool convs_done = false);
cudaError_t syn_decode(const Arch& a, const Geo& g, const float* hbuf_last, float* out_hwc,
                       cudaStream_t st);
int syn1x1_partial_cols(const Arch& a);
cudaError_t syn_prepare(const Arch& a);   // kernel attributes; call once before capture

// iteration bookkeeping (cc_iter.cu)
cudaError_t quantize_launch(const Geo& g, const float* y, float* yhat, float* yhat_bord,
                            const float* noise, int mode, const IterScalars* sc, int ste_start,
                            uint64_t seed, int iter_override, float soft_temp, float* dq,
                            cudaStream_t st);
// Context gradient of the rate: gself[q] += sum over the N context positions k of
// dctx[k][q - offset_k] (the ARM's gradients with respect to its inputs), in place.
cudaError_t ctx_gather(const Geo& g, const int2* d_offsets, int N, float* gself,
                       const float* dctx, cudaStream_t st);
cudaError_t reduce_sections(const SectionTable& tab, float* part2, int n_virtual, int slices,
                            cudaStream_t st);
// Parameter slots of the bank images: per parameter up to two float indices into the ARM
// image and two into the synthesis image (-1: none).  param_update writes every updated
// value to its slots, so that the images stay current between passes.
struct ImageSlots {
  const int4* map;
  float* arm_image;
  float* syn_image;
};
// What finishing a pass reads: the per-CTA partial sums of D and of the bits, their
// scales, lambda and the loss log (finish_iteration).
struct PassFinish {
  const float* part_d;
  int nd;
  const float* part_bits;
  int nb;
  double d_scale, r_scale, lam;
  double* log;
};
// The step to the next iteration is taken by the last block to end among the latent
// update's blocks and, if it takes part (pf != nullptr), the parameter update's: tickets =
// the sum of their block counts (latent_update_blocks, param_update_blocks).
unsigned param_update_blocks(const Layout& lay);
unsigned latent_update_blocks(const Geo& g);
cudaError_t param_update(const Layout& lay, const Arch& a, const float* part2, int slices,
                         float* params, float* m, float* v, float* grad_out, bool apply,
                         float lr, const IterScalars* sc, const ImageSlots& slots,
                         const PassFinish* pf, unsigned tickets, bool advance, cudaStream_t st);
// Total latent gradient dD/dy_hat + lambda / (HW) * dR/dy_hat (grate: the rate gradient
// after ctx_gather) and Adam on the latents.
cudaError_t latent_update(const Geo& g, const float* gsyn, const float* grate, float rate_scale,
                          float* y, float* m, float* v, float* grad_out, bool apply, float lr,
                          IterScalars* sc, const PassFinish& pf, unsigned tickets, bool advance,
                          const float* dq, int soft, int ste_start, cudaStream_t st);
// D, R, the loss and the loss log entry of a pass with gradients (one block; the step to
// the next iteration is taken by the last update block).
cudaError_t pass_loss(const PassFinish& pf, IterScalars* sc, cudaStream_t st);
cudaError_t finish_iteration(const float* part_d, int nd, const float* part_bits, int nb,
                             double d_scale, double r_scale, double lam, IterScalars* sc,
                             double* log, bool advance, cudaStream_t st,
                             bool pdl);
cudaError_t image_to_planar(const uint8_t* rgb_hwc, float* x, int H, int W, cudaStream_t st);

// Stores a message for cc_last_cuda_error() (thread-local).
void set_error_text(const char* msg);


// ---- latent bitstream (cc_codec.cu) ------------------------------------------------------

// Flat geometry of the coded latents: levels in order, each row-major without padding;
// rows of all levels numbered level by level (one range-coder substream per row).
struct CodecGeo {
  int h[kLevels], w[kLevels];
  long long off[kLevels];     // first latent of each level
  int row0[kLevels];          // first row number of each level
  int cap[kLevels];           // bytes reserved for one row's substream while encoding
  long long buf0[kLevels];    // first byte of each level's row buffers
  int band0[kLevels];         // first decoding band (band_rows rows) of each level
  long long n_lat, buf_bytes;
  int rows, bands, band_rows;
};
// lanes per row of the decoder for context size N (band_rows = 32 / parts)
int codec_decode_parts(int N);
CodecGeo codec_geo(const Geo& g, int band_rows);
const std::vector<uint16_t>& codec_tables();
size_t codec_table_bytes();
bool codec_quantize_arm(const float* params, int N, int NL, int32_t* q);
int codec_max_arm_ints();
cudaError_t codec_upload_arm(const int32_t* q, int N, int NL, cudaStream_t st);
cudaError_t codec_symbols(const CodecGeo& cg, const Geo& g, const float* y, const int2* offs,
                          int N, int NL, int2* sym, int* flag, cudaStream_t st);
cudaError_t codec_encode_rows(const CodecGeo& cg, const int2* sym, const uint16_t* tab,
                              uint8_t* rowbuf, int* row_len, int* flag, cudaStream_t st);
cudaError_t codec_pack(const CodecGeo& cg, const uint8_t* rowbuf, const long long* dst_off,
                       const int* row_len, uint8_t* out, cudaStream_t st);
cudaError_t codec_decode(const CodecGeo& cg, int N, int NL, const uint16_t* tab,
                         const uint8_t* bytes, const long long* row_off, const int* row_len,
                         int* planes, int* progress, int* flag, cudaStream_t st);
bool codec_offsets_match(const int2* offs, int N);
bool codec_arm_in_range(const int32_t* q, int N, int NL);
cudaError_t codec_to_float(const CodecGeo& cg, const Geo& g, const int* planes, float* y,
                           cudaStream_t st);

}  // namespace cc
