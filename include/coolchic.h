/*
 * coolchic.h -- C ABI of the GB300 (sm_103a) Cool-chic overfitting library.
 *
 * One call of cc_encode_iters runs n iterations of the encoder optimisation of
 * Blard et al., "Overfitted image coding at reduced complexity", Sec. II, eq. (1):
 *
 *     min over (y, psi, upsilon, theta) of  D(x, f_theta(f_upsilon(Q(y)))) + lambda R(Q(y)),
 *     R = -log2 p_psi(Q(y)),
 *
 * where y is the L = 7 level latent pyramid (Sec. II "Decoding" item i), p_psi the
 * auto-regressive probability model (item ii), f_upsilon the learned 2x upsampling and
 * f_theta the synthesis (item iii), with the layer lists of Table 1.  One iteration is the
 * forward pass, its backward pass (Sec. IV-A, "Shorter training": weight and input
 * gradients of every layer) and one Adam update of every latent and parameter.
 *
 * Conventions for every entry point:
 *   - return 0 (CC_OK) on success, a negative CC_E* code otherwise; nothing throws;
 *   - pointers documented "host or device" may point to either (CUDA unified addressing);
 *   - input buffers stay owned by the caller and are copied in before the call returns
 *     (or, for asynchronous calls, before any later call on the same context);
 *   - the context owns its device memory (or borrows a caller workspace) until cc_free;
 *   - all GPU work of a context is issued on the stream given to cc_init_image;
 *   - the contexts of one device share its constant-memory weight banks (every pass loads
 *     its own weights first).  The library orders their passes itself: each call that
 *     runs passes makes its stream wait for the previous such call on the device, from
 *     any context, stream or host thread, so passes of two contexts never overlap on the
 *     GPU (they run one after another).  The banks belong to the loaded library: contexts
 *     created through separately loaded copies of it have their own and run concurrently;
 *   - the images are 8-bit RGB, row-major, channels last (H x W x 3); the library uses
 *     x = v / 255 in float32.
 *
 * Flat parameter order (cc_get_state, cc_get_grads, init_params):
 *   ARM:        for i < arm_layers: W_i (N x N, row-major out x in), b_i (N);
 *               W_out (2 x N), b_out (2)                 -- outputs (mu, log-scale)
 *   upsampling: one k x k filter per level l = 1..L-1 (up_per_level = 1) or one shared
 *               filter (up_per_level = 0), row-major
 *   synthesis:  W_a (C x L), b_a (C), W_b (3 x C), b_b (3),
 *               for each 3x3 layer: W (3 out x 3 in x 3 x 3), b (3)
 * Flat latent order: level 0 .. L-1, each level row-major, ceil(H/2^l) x ceil(W/2^l).
 *
 * Device memory per 512 x 768 image with the 2300-MAC decoder: about 120 MB.
 */
#ifndef COOLCHIC_H
#define COOLCHIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CC_OK = 0,
    CC_EINVAL = -1,       /* bad argument or unsupported configuration */
    CC_ENOMEM = -2,       /* device allocation failed or workspace too small */
    CC_ECUDA = -3,        /* a CUDA runtime call failed (see cc_last_cuda_error) */
    CC_ETIMEOUT = -4,     /* a bounded device wait gave up */
    CC_ENONFINITE = -5,   /* the loss became NaN or infinite */
    CC_ESTATE = -6,       /* state blob of the wrong size, version or shape */
    CC_ESIZE = -7         /* output buffer too small; the size needed was returned  */
};

typedef struct cc_ctx cc_ctx;

/* Architecture and training schedule.  Table 1 notation: N-N-LinR layers, N-2-Lin,
 * 1-1-TConv-k, 7-C-Conv-1, C-3-Conv-1, 3-3-ConvR-3. */
typedef struct {
    int levels;        /* L: number of latent grids; must be 7                          */
    int arm_ctx;       /* N: causal context size = ARM width; 8, 16 or 24               */
    int arm_layers;    /* number of N-N-LinR layers; 1 or 2                              */
    int up_kernel;     /* k of the stride-2 transposed conv; 4 or 8                      */
    int up_per_level;  /* 1: one filter per level; 0: one shared filter                 */
    int syn_hidden;    /* C of the 7-C-Conv-1 layer; 8, 16 or 40                         */
    int syn_res3x3;    /* number of 3-3-ConvR-3 layers; 1 or 2                           */
    float lam;         /* lambda of eq. (1)                                              */
    float lr;          /* Adam learning rate                                             */
    int total_iters;   /* schedule length; decides where straight-through rounding starts */
    float ste_frac;    /* last fraction of total_iters using rint + straight-through     */
    uint64_t seed;     /* key of the Philox4x32-10 quantisation noise                    */
    float soft_temp;   /* 0: noise phase y_hat = y + u.  T > 0: C3's soft-rounding proxy
                        * y_hat = s_T(s_T(y) + u), s_T(x) = floor(x) + 1/2 +
                        * tanh((x - floor(x) - 1/2)/T) / (2 tanh(1/(2T))), differentiated
                        * through both soft roundings (Sec. II "Encoding" refers to C3)    */
} cc_config;

/* Number of decoder parameters of a configuration (Table 1 "Param" column). */
int cc_param_count(const cc_config* cfg, int* n_params);

/* Number of latents sum_l ceil(H/2^l) ceil(W/2^l). */
int cc_latent_count(const cc_config* cfg, int H, int W, int* n_latents);

/* Bytes of device workspace cc_init_image_ws needs for this image size. */
int cc_workspace_size(const cc_config* cfg, int H, int W, size_t* bytes);

/* Create a context for one image: copies the image (host or device, H x W x 3 uint8),
 * sets y = 0, the parameters to init_params (host or device, cc_param_count floats;
 * NULL = the library's seeded default: uniform +-1/sqrt(fan_in) weights, zero biases,
 * resampling-filter upsampling), Adam moments to 0 and the iteration counter to 0.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).  The library
 * allocates its device memory with cudaMalloc.  Synchronises before returning. */
int cc_init_image(const cc_config* cfg, const uint8_t* rgb_hwc, int H, int W,
                  const float* init_params, void* cuda_stream, cc_ctx** out);

/* Same as cc_init_image, but all device memory is carved from a caller-owned device
 * workspace of ws_bytes >= cc_workspace_size bytes (e.g. a PyTorch allocation), which
 * must stay valid until cc_free.  Returns CC_ENOMEM if ws_bytes is too small. */
int cc_init_image_ws(const cc_config* cfg, const uint8_t* rgb_hwc, int H, int W,
                     const float* init_params, void* cuda_stream,
                     void* device_workspace, size_t ws_bytes, cc_ctx** out);

/* Replace the image of a context by another one of the same size (host or device).
 * Asynchronous: the copy is issued on a stream of the context's own, where it overlaps the
 * iterations already issued (it waits only for the previous image's conversion); the
 * conversion to the float planes the iterations read follows on the context stream.  The
 * caller keeps rgb_hwc unchanged until the context stream has passed this call; from
 * page-locked host memory the copy does not block the host. */
int cc_set_image(cc_ctx* ctx, const uint8_t* rgb_hwc);

/* Run n_iters overfitting iterations (forward, backward, Adam), asynchronously on the
 * context stream, replaying a CUDA graph of one iteration.  Iteration t (counted from 0
 * since cc_init_image) uses noise quantisation while t < round(total_iters (1 -
 * ste_frac)) (half-way cases to even) and rint + straight-through after.  Per-iteration D, R and loss are logged
 * on the device (see cc_get_losses). */
int cc_encode_iters(cc_ctx* ctx, int n_iters);

/* cc_encode_iters with a non-finite check and rollback (failure detection; the paper has
 * no counterpart).  Runs up to n_iters iterations in chunks of check_every (1 .. 4096):
 * before each chunk the optimisation state (latents, parameters, Adam moments, iteration
 * scalars) is copied on the device; after it the chunk's logged D, R and loss are read.
 * If any of them is NaN or infinite, or a pass of the chunk read a non-finite latent or
 * produced a non-finite latent or parameter, or an ARM tensor-core wait gave up, the
 * state is restored to the copy taken before the chunk, the iteration counter steps back,
 * and the call returns CC_ENONFINITE (or CC_ETIMEOUT); *iters_done (host) receives the
 * number of iterations kept.  (The kernels' ReLUs and clamps map a NaN input to a finite
 * value, so a NaN in the state need not show in the loss; every pass therefore also
 * checks the latents it reads and the values its updates write.)  Synchronises once per
 * chunk.  CC_OK: all n_iters ran. */
int cc_encode_iters_checked(cc_ctx* ctx, int n_iters, int check_every, int* iters_done);

/* Host-side fault injection for tests of the failure paths (no GPU fault is involved).
 *   CC_FAULT_NAN_GRAD (ctx given): the latent update of iteration at_iteration (>= the
 *     current iteration) replaces the gradient of latent 0 by NaN, once; a rollback of
 *     cc_encode_iters_checked clears it.
 *   CC_FAULT_ALLOC (ctx NULL, at_iteration ignored): the next cc_init_image of this
 *     process that would call cudaMalloc returns CC_ENOMEM instead, once.
 *   CC_FAULT_ARM_STALL (ctx given, at_iteration ignored): from the next pass on, every CTA
 *     of the ARM kernel leaves out its first context load and waits for it with a budget
 *     of about half a millisecond; the wait runs out, the kernel records the fault, waits
 *     for its loads in flight and returns, and the call that synchronises reports
 *     CC_ETIMEOUT.  A rollback of cc_encode_iters_checked clears it.
 * CC_EINVAL for any other combination. */
#define CC_FAULT_NAN_GRAD 1
#define CC_FAULT_ALLOC 2
#define CC_FAULT_ARM_STALL 3
int cc_debug_inject(cc_ctx* ctx, int fault, int at_iteration);

/* Rate-distortion cost of the current state, eq. (1): D = mean squared error over the
 * 3HW values, R_bpp = bits / (H W), cost = D + lambda R.  hard_round = 1: rint latents
 * (the decoded image); 0: the current iteration's noisy latents.  CC_ENONFINITE if the
 * cost is not finite or a latent is (values still written).  Synchronises. */
int cc_rd_cost(cc_ctx* ctx, int hard_round, double* D, double* R_bpp, double* cost);

/* Decoded image x_hat = f_theta(f_upsilon(rint(y))) as H x W x 3 float32 (host or
 * device, caller-owned), not clamped.  Synchronises. */
int cc_decode(cc_ctx* ctx, float* rgb_out_hwc);

/* One forward and backward pass at the current iteration without any update.
 * noise_override (host or device, n_latents floats in flat latent order) replaces the
 * quantisation noise, or NULL for the iteration's own noise / rounding.  grads_out
 * (host or device): n_latents + n_params floats, dL/dy then dL/dparams, flat orders.
 * Synchronises. */
int cc_get_grads(cc_ctx* ctx, const float* noise_override, float* grads_out);

/* cc_get_grads with the loss terms of that pass and an explicit mode:
 * hard = 1 forces rint latents (noise_override ignored), 0 forces noise, -1 follows the
 * schedule.  D, R_bpp and loss = D + lambda R_bpp (eq. (1)) are host doubles; each may be
 * NULL. */
int cc_forward_backward(cc_ctx* ctx, const float* noise_override, int hard,
                        float* grads_out, double* D, double* R_bpp, double* loss);

/* D, R_bpp and loss of iterations first .. first+count-1 (3 doubles each, host or
 * device).  Only the last 4096 iterations are kept.  Synchronises. */
int cc_get_losses(cc_ctx* ctx, int first, int count, double* out);

/* The same entries copied asynchronously: the copy is enqueued on the context stream
 * behind the iterations already issued and the call returns at once (no check for
 * non-finite values).  out: device or page-locked host memory (pageable host memory makes
 * the copy synchronous); valid to read once the stream has passed the copy (an event
 * recorded after this call, or a stream synchronisation).  Lets a training loop read each
 * step's loss without waiting for the step to finish. */
int cc_get_losses_async(cc_ctx* ctx, int first, int count, double* out);

/* Overwrite / read the latents y (n_latents floats, flat latent order) or the parameters
 * (cc_param_count floats, flat parameter order); host or device buffers.  The setters are
 * asynchronous on the context stream; the getters synchronise.  Adam moments and the
 * iteration counter are left unchanged. */
int cc_set_latents(cc_ctx* ctx, const float* y_flat);
int cc_get_latents(cc_ctx* ctx, float* y_flat);
int cc_set_params(cc_ctx* ctx, const float* params);
int cc_get_params(cc_ctx* ctx, float* params);

/* Number of iterations run so far. */
int cc_iteration(cc_ctx* ctx, int* iter);

/* The quantisation noise of iteration iter, n_latents floats in flat latent order
 * (host or device).  Synchronises. */
int cc_noise(cc_ctx* ctx, int iter, float* out);

/* Measurement support.  cc_profile_phases runs `reps` full iterations eagerly on the
 * context stream (forward, backward and update: the state advances by `reps` iterations),
 * recording CUDA events around each phase, and writes the mean milliseconds per phase to
 * ms_out[CC_N_PHASES] (host): 0 weight upload + quantisation, 1 ARM + rate forward and
 * backward, 2 upsampling forward, 3 synthesis forward + distortion, 4 synthesis backward,
 * 5 upsampling backward, 6 context-gradient gather, reductions, Adam and loss
 * bookkeeping.  Synchronises.
 * cc_graph_kernel_count gives the number of kernel launches in one captured iteration. */
#define CC_N_PHASES 7
int cc_profile_phases(cc_ctx* ctx, int reps, float* ms_out);
int cc_graph_kernel_count(cc_ctx* ctx, int* n_kernels);

/* Milliseconds of the ARM kernel (forward + backward, rate) in the most recent pass that
 * ran it beside the synthesis chain (a captured iteration replayed by cc_encode_iters, or
 * an eager pass), measured by two CUDA events recorded on the ARM's stream around its
 * launch.  Measurement support with no counterpart in the paper.  Waits for the second
 * event; CC_ECUDA (event not yet recorded) before the first such pass.  ms: host. */
int cc_arm_kernel_ms(cc_ctx* ctx, float* ms);

/* Checkpoint: a flat versioned blob with y, parameters, Adam moments, the iteration
 * counter and the seed.  With buf = NULL, *nbytes receives the size.  cc_set_state
 * restores a blob written for the same configuration and image size; resuming replays
 * the same noise, so a resumed run matches an uninterrupted one. */
int cc_get_state(cc_ctx* ctx, void* buf, size_t* nbytes);
int cc_set_state(cc_ctx* ctx, const void* buf, size_t nbytes);

/* Release the context and its device memory (not a caller workspace). */
void cc_free(cc_ctx* ctx);

/* Static description of an error code. */
const char* cc_strerror(int code);

/* Rate without allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- e.g. a decoder inside a process whose device
 * memory is all owned by another allocator (a framework's caching allocator, a fixed
 * pool), or a real-time service that must not allocate once running.
 *
 * Computes bits = sum over every latent of -log2 P(y_hat) under the ARM (the rate term of
 * eq. (1) before division by H W) for a caller-supplied quantised pyramid:
 *   yhat_flat: device, cc_latent_count floats in flat latent order (any real values);
 *   params:    device, cc_param_count floats in flat parameter order (ARM part read);
 *   bits_out:  host or device, one double;  cuda_stream: cudaStream_t or NULL.
 * Allocates nothing: its scratch -- one float per tile of 128 latents plus the double
 * total -- is a fixed file-scope __device__ array held by every device that loads the
 * library until the process exits.  The first call on a device (per loaded copy of the
 * library) is a warm-up: it looks up that array's device address (cudaGetSymbolAddress)
 * and caches it, and with CUDA's lazy module loading it is also the call that loads the
 * library's kernels onto the device, which may itself reserve device memory.  Make that
 * first call before the caller's no-allocation phase begins, and before any stream
 * capture; later calls allocate nothing.  cuda_stream must belong to the device that is
 * current when the call is made.  All calls share the scratch array and two
 * __constant__ banks holding the ARM weights and context offsets, which every call
 * overwrites before its kernels run: calls whose GPU work overlaps race on both, so issue
 * them on one stream or synchronise between them.  Every call rewrites all the scratch it
 * reads.  Pyramids needing more than CC_NOALLOC_MAX_TILES tiles (about 8.4 million
 * latents, e.g. 2048 x 3072 pixels) are rejected with CC_EINVAL and a message in
 * cc_last_cuda_error().  Synchronises before returning. */
#define CC_NOALLOC_MAX_TILES 65536
int cc_rate_bits_noalloc(const cc_config* cfg, const float* yhat_flat, int H, int W,
                         const float* params, void* cuda_stream, double* bits_out);

/* Latent bitstream.  Sec. II "Encoding": once the encoder has converged, the latents are
 * entropy coded with a range coder driven by the ARM's probability model p_psi; Sec. II
 * "Decoding" (Fig. 2): the decoder reads the latent grids with that model, each latent
 * conditioned on its already-decoded causal neighbours, then upsamples and synthesises.
 * The decoder re-evaluates the ARM, so both sides run it in integer arithmetic:
 *   - ARM weights and biases rounded (half to even) to multiples of 2^-8 (Q8; weights
 *     clamped to +-2^11 in Q8 units, i.e. |w| <= 8, biases to +-2^15); inputs = integer
 *     latents clamped to [-128, 128], times 256; a layer z = ((sum W a) + 128) >> 8 + b
 *     (round half up), every sum exact in 32-bit integers, saturated to +-2^15; LinR
 *     output a + max(z, 0), saturated; the output layer gives (mu, log-scale) in Q8;
 *   - probabilities from 744 Laplace frequency tables (93 log-scale bins of width 1/8 from
 *     ln 0.01, 8 bins of mu's fraction; symbols y - floor(mu) in [-64, 64] plus one escape
 *     per tail, the excess as an order-0 Exp-Golomb code), built on the host;
 *   - a 32-bit range coder with frequencies out of 2^16, one substream per latent row.
 * Layout: "CCF1", H, W (u32 little endian), 8 architecture bytes (levels, N, LinR layers,
 * k, per-level filters, C, 3x3 layers, 0), the Q8 ARM parameters (i32), the other
 * parameters (f32) in flat parameter order, the byte count of every row substream
 * (LEB128; levels 0..L-1, rows top to bottom), the substreams.
 *
 * cc_write_bitstream: codes rint(y) of the context's latents with its current
 *   parameters.  out (host or device) receives *nbytes bytes; with out == NULL only
 *   *nbytes is set; with capacity < *nbytes nothing is written and CC_ESIZE returned.
 *   A quantised latent above 2^20 in magnitude gives CC_EINVAL.  Synchronises.
 * cc_bitstream_info: configuration (architecture fields; lam, schedule and seed zero,
 *   lr 1) and image size of a bitstream in host memory.
 * cc_decode_bitstream: decodes a bitstream in host memory on the current device and
 *   the given stream (cudaStream_t or NULL): the latent rows as a wavefront (row r
 *   decodes position x at step x + lag r, lag 3 for N = 8 and 4 for N = 16 or 24), one
 *   warp per band of rows (32 rows of one lane each for N = 8, 16 rows of two lanes each
 *   for N = 16 or 24), every band waiting (bounded;
 *   CC_ETIMEOUT if it gives up) on the band above it, all levels at once in one
 *   cooperative launch; then the float32 upsampling and synthesis.  Optional outputs (host or device): rgb_out_hwc (H x W x 3 floats, not
 *   clamped, as cc_decode), latents_out (cc_latent_count int32, flat latent order),
 *   latent_ms (device time of the latent decoding).  It holds a temporary context (the
 *   memory of cc_init_image) for the call.  Synchronises. */
int cc_write_bitstream(cc_ctx* ctx, uint8_t* out, size_t capacity, size_t* nbytes);
int cc_bitstream_info(const uint8_t* bs, size_t nbytes, cc_config* cfg, int* H, int* W);
int cc_decode_bitstream(const uint8_t* bs, size_t nbytes, void* cuda_stream,
                        float* rgb_out_hwc, int32_t* latents_out, float* latent_ms);

/* Warm-start predictor.  The paper's encoder starts every image from zero latents; its
 * Sec. IV-B predicts the latents with an analysis network (the non-overfitted variant)
 * and Sec. V proposes fine-tuning such a prediction per image.  This small predictor
 * maps an image to latent levels 0 .. 4: four 3x3 stride-2 convolutions with 32
 * channels and ReLU (zero padding 1) whose outputs feed 1x1 convolutions giving levels
 * 1 .. 4, and a 3x3 stride-1 convolution of the image giving level 0; levels 5 and 6 are
 * 0.  It is trained on latents the encoder reached (loss: the sum over levels 0 .. 4 of
 * each level's mean squared error), with Adam (beta 0.9 / 0.999, eps 1e-8,
 * bias-corrected).  The three 32-to-32-channel convolutions run on the tensor cores with
 * BF16 operands (inputs, weights and output gradients rounded to nearest BF16, ties to
 * even) and FP32 accumulation, in the forward pass and both gradients; the rest is FP32.
 * Every cc_warm_* call runs on the stream given at creation; one predictor is not used
 * from two threads at once.
 * Flat parameter order: c1 (W 32 x 3 x 3 x 3, b 32), c2 .. c4 (W 32 x 32 x 3 x 3, b 32),
 * heads 1 .. 4 (W 32, b 1), head 0 (W 3 x 3 x 3, b 1).
 * cc_warm_create: predictor for H x W images (H, W >= 16); params (host or device,
 *   cc_warm_param_count floats) copied in; cuda_stream as cc_init_image.
 * cc_warm_predict: rgb_hwc (host or device, 8-bit H x W x 3) -> latents_out (host or
 *   device, cc_latent_count floats in flat latent order).  Synchronises.
 * cc_warm_loss_grad: loss against target latents (host or device, flat latent order;
 *   levels 5, 6 ignored) and, if grads_out is not NULL, its gradient (host or device,
 *   flat parameter order).  Synchronises.
 * cc_warm_train_step: the loss and its gradient, then one Adam step with learning rate
 *   lr, queued on the stream (the next call, or cc_warm_get_params, sees it).  With loss
 *   in host memory it synchronises, writes the loss and takes no step on a non-finite
 *   one; with loss in device memory the loss is copied there on the stream, and with loss
 *   NULL it is not written: neither synchronises nor checks.
 * Errors: CC_EINVAL (NULL pointer, H or W outside 16 .. 16384), CC_ENOMEM, CC_ECUDA,
 *   CC_ENONFINITE (loss not finite: *loss written, no gradient copied out, no Adam
 *   step taken), CC_ETIMEOUT (a bounded tensor-core wait gave up; results invalid). */
typedef struct cc_warm cc_warm;
int cc_warm_param_count(int* n_params);
int cc_warm_create(int H, int W, const float* params, void* cuda_stream, cc_warm** out);
int cc_warm_predict(cc_warm* w, const uint8_t* rgb_hwc, float* latents_out);
int cc_warm_loss_grad(cc_warm* w, const uint8_t* rgb_hwc, const float* target_latents,
                      double* loss, float* grads_out);
int cc_warm_train_step(cc_warm* w, const uint8_t* rgb_hwc, const float* target_latents,
                       float lr, double* loss);
int cc_warm_get_params(cc_warm* w, float* params);
int cc_warm_set_params(cc_warm* w, const float* params);
void cc_warm_free(cc_warm* w);

/* Text of the last error seen by the library in this thread ("" if none). */
const char* cc_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* COOLCHIC_H */
