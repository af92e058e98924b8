/*
 * hsc.h -- C ABI of libhsc, GB300 (sm_103a) kernels for deferred G-buffer
 * shading with Hadamard spectral codes ("Compact Hadamard Latent Codes for
 * Efficient Spectral Rendering", arXiv 2602.18741).
 *
 * The method (Sec. 4-6 of the paper): a non-negative linear encoder E (k x n)
 * and decoder D (n x k) map n-sample spectra to k-codes, k = 3B (Eq. 4);
 * scaling and addition stay exact in code space and the element-wise
 * (Hadamard) product of spectra is replaced by the blockwise product of codes
 * (Eq. 6).  Assets are encoded once, the k-code image is rendered as B RGB
 * passes and reassembled, then decoded once to spectra, XYZ or sRGB (Fig. 2b).
 *
 * Shading model (the paper path-traces in Mitsuba, Sec. 6.1; this library
 * shades a G-buffer instead): point lights l at p_l with intensity I_l, Lambert
 * BRDF rho/pi, inverse-square falloff, no visibility, plus an optional
 * indirect bounce through a secondary G-buffer point treated as a virtual
 * point light with clamp eps = 1e-2:
 *   g(x, n, l) = max(0, n.(p_l - x)) / |p_l - x|^3
 *   A(x, n)    = sum_l g(x, n, l) * (I_l / pi) * V_l          (V_l: SPD or code)
 *   h          = max(0, n1.d) max(0, -n2.d) / (|d|^2 max(|d|^2, eps)) / pi,  d = x2 - x1
 *   out        = R_m1 (.) (A(x1, n1) + h * (R_m2 (.) A(x2, n2)))
 * with (.) the element-wise product on n samples (spectral) or k channels
 * (latent, Eq. 6).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Pointers marked "device" must point to device memory of the context's
 *   GPU; the caller owns and frees all of them.  The library never frees or
 *   reallocates caller memory.  Float arrays need 4-byte alignment; the latent
 *   and output images of the vectorised kernels need 16-byte alignment where
 *   noted.
 * - Row-major layouts: a "P x c" array holds c consecutive values per pixel.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every call only enqueues work on that stream and returns; nothing
 *   synchronises unless stated.  Results are ready once the stream reaches
 *   that point.
 * - Errors are returned as hsc_status; hsc_last_error() gives a message for
 *   the calling thread.  Arguments are validated on the host before any
 *   launch (HSC_ERR_INVALID_ARG).  Problems found on the device (material
 *   index out of range) set a device error word; hsc_sync() reports it as
 *   HSC_ERR_DEVICE_CHECK and clears it.  No kernel traps or aborts.
 * - A context is not thread-safe: use one per host thread.  Calls on one
 *   context that share the context's scratch (noted below) must be ordered
 *   on one stream.
 */
#ifndef HSC_H_
#define HSC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HSC_API __attribute__((visibility("default")))
#else
#define HSC_API
#endif

#define HSC_VERSION 1
#define HSC_MAX_K 96      /* code length limit (multiple of 3)            */
#define HSC_MAX_N 128     /* spectral sample limit                        */
#define HSC_MAX_MAT (1 << 24)
#define HSC_NOALLOC_MAX_K 96  /* channel limit of hsc_quantize_fp8_noalloc   */
#define HSC_MAX_FRAMES_PER_CALL 512  /* frames per hsc_shade_frames call    */
#define HSC_QUEUE_SLOTS 256  /* streams per context with their own tile counter */
#define HSC_ASSETS_MAX_CODES 4096  /* n_mat x k limit of hsc_shade_latent_assets */
#define HSC_ASSETS_MAX_LIGHTS 256  /* light limit of hsc_shade_latent_assets       */
#define HSC_UPSAMPLE_HIDDEN 128      /* hidden width of the upsampling network */

typedef struct hsc_ctx hsc_ctx;

typedef enum {
  HSC_OK = 0,
  HSC_ERR_INVALID_ARG = 1,   /* bad size, null or misaligned pointer, bad enum   */
  HSC_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has details) */
  HSC_ERR_OOM = 3,           /* context scratch could not be allocated           */
  HSC_ERR_UNSUPPORTED = 4,   /* valid request the library does not implement     */
  HSC_ERR_TIMEOUT = 5,       /* a bounded device wait ran out                    */
  HSC_ERR_DEVICE_CHECK = 6   /* a kernel flagged bad input (see hsc_sync)        */
} hsc_status;

typedef enum { HSC_F32 = 0, HSC_BF16 = 1, HSC_F16 = 2, HSC_FP8_E4M3 = 3 } hsc_dtype;

/* PASSES: the k-code image is produced as k/3 three-channel passes and
 * reassembled (Fig. 2b).  FUSED: one launch shades all k channels, sharing
 * the geometry term; per channel it performs exactly the same FP32 operations
 * in the same order, so the two modes give bit-identical latent images.      */
typedef enum { HSC_PASSES = 0, HSC_FUSED = 1 } hsc_mode;

/* One G-buffer: per pixel a unit normal, a position and a material index.   */
typedef struct {
  const float* normal;   /* device, P x 3 float32                                 */
  const float* pos;      /* device, P x 3 float32                                 */
  const int32_t* mat;    /* device, P int32 in [0, n_mat); a pixel with an index
                          * outside it (in either G-buffer) is shaded black and
                          * sets the error word                                */
} hsc_gbuffer;

/* Point lights.                                                              */
typedef struct {
  const float* pos;        /* device, L x 3 float32                           */
  const float* intensity;  /* device, L float32 (scales the unit-peak SPD)    */
  int32_t count;           /* L >= 1                                          */
} hsc_lights;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (made current on the calling
 * thread).  Allocates a small fixed scratch block (error word, reduction
 * workspace); larger scratch for PASSES images and the fp8 path grows on
 * demand inside the calls that need it (see hsc_reserve).                  */
HSC_API hsc_status hsc_create(hsc_ctx** out, int device);
HSC_API void hsc_destroy(hsc_ctx* ctx);
/* Message for the last failing call on this thread ("" if none).  Valid
 * until the next call on this thread.                                       */
HSC_API const char* hsc_last_error(void);
/* Synchronise `stream`, surface asynchronous CUDA errors and the device error
 * word (HSC_ERR_DEVICE_CHECK, cleared on read).                              */
HSC_API hsc_status hsc_sync(hsc_ctx* ctx, void* stream);
/* Pre-allocate context scratch of at least `bytes` so later calls do not
 * allocate (required before capturing PASSES or fp8 calls in a CUDA graph).  */
HSC_API hsc_status hsc_reserve(hsc_ctx* ctx, size_t bytes);
/* Scratch bytes hsc_shade_latent needs for P pixels, code length k, `mode`
 * and `latent_dt`.                                                           */
HSC_API size_t hsc_shade_latent_scratch_bytes(int64_t pixels, int k, hsc_mode mode, hsc_dtype latent_dt);

/* Launch-configuration autotuning of the shading kernels.  The tile shape
 * (threads per CTA, pixels per thread, persistent or one-CTA-per-tile grid)
 * never changes what a channel computes, only how fast.  enable = 0 (the
 * default): fixed defaults.  enable = 1: the first call of each shape class
 * (kernel, channels, bounce on/off, light and pixel counts rounded up to
 * powers of two) times every candidate on its own inputs -- synchronising
 * the stream once -- and caches the fastest; calls made while a stream is
 * captured never tune.  A latency-bound caller (a serving loop) runs one
 * call of every shape class it will meet before its first deadline, or
 * loads a saved table with hsc_tune_load, so that no call tunes later.      */
HSC_API hsc_status hsc_set_autotune(hsc_ctx* ctx, int enable);
/* Text table of the tuned shape classes and candidate timings (valid until
 * the next tuning call on this context).                                   */
HSC_API const char* hsc_tune_report(hsc_ctx* ctx);
/* Save the tuned configurations as text (one line per shape class) into buf
 * (truncated to len - 1 bytes, NUL-terminated); returns the full length.
 * hsc_tune_load reads such text back, so a process can reuse the choices of
 * an earlier run without timing candidates again.                           */
HSC_API int hsc_tune_save(hsc_ctx* ctx, char* buf, size_t len);
HSC_API hsc_status hsc_tune_load(hsc_ctx* ctx, const char* text);
/* Force one launch configuration for every shading launch (testing and
 * benchmarking): ppt in {1, 2, 4} (spectral kernel: 1 or 2 shading points per
 * thread), block in {128, 256}, waves >= -1 (0 = one CTA per pixel tile,
 * -1 = one wave of persistent CTAs on an atomic tile queue; latent kernels),
 * vec = 1 (scalar FP32) or 2 (packed f32x2 pairs: pairs of shading points in
 * the latent kernels, pairs of wavelengths in the spectral kernel), chunk =
 * spectral channels per sweep (0 = default, 16, 28, 32, 44 or 84), or 1 for
 * the lane-group spectral kernel (8 lanes share 8 shading points, each lane
 * a register tile of 8 points x n/8 wavelengths, one geometry term per point
 * and light; ppt and vec ignored, waves 0 = one CTA per tile, > 0 =
 * persistent).
 * ppt <= 0 removes the override.                                            */
HSC_API hsc_status hsc_force_launch_config(hsc_ctx* ctx, int ppt, int block, int waves, int vec, int chunk);
/* FP32 issue-rate probe (measurement only; the shading kernels are FP32 issue
 * bound and compared with the ALU peak SMs x 128 lanes x SM clock).  One
 * launch of `ctas` CTAs of 256 threads (ctas <= 0: 8 per SM), each thread
 * running `iters` iterations of 32 register-only FFMAs (8 independent chains).
 *   sink: device, ctas x 256 float32, overwritten with meaningless values;
 *   lane_ops_out: host, may be null; receives the FMA lane-operations of the
 *   launch (ctas x 256 x iters x 32), which the caller divides by the time it
 *   measures on `stream`.  1 <= iters <= 2^24.                              */
HSC_API hsc_status hsc_fp32_peak_probe(hsc_ctx* ctx, int ctas, int iters, float* sink, int64_t* lane_ops_out,
                                       void* stream);
/* MUFU tanh rate probe (measurement only; the upsampling network's SiLU is
 * one hardware tanh per hidden value, so the MUFU rate bounds its epilogue).
 * One launch of `ctas` CTAs of 256 threads (ctas <= 0: 8 per SM), each thread
 * running `iters` iterations of 32 register-only tanh.approx operations (8
 * independent recurrences a <- tanh(a + 1/4)): packed = 0 in FP32
 * (tanh.approx.f32), packed = 1 on f16 pairs (tanh.approx.f16x2, the form the
 * upsampler uses; two results per operation).
 *   sink: device float32, at least ctas x 256 values (each thread's sum).
 *   tanh_ops_out: host, may be null; receives the tanh results of the launch,
 *   ctas x 256 x iters x 32 (x 2 when packed).  1 <= iters <= 2^24.        */
HSC_API hsc_status hsc_tanh_peak_probe(hsc_ctx* ctx, int ctas, int iters, int packed, float* sink,
                                       int64_t* tanh_ops_out, void* stream);

/* ----------------------------------------------------- colour projection */

/* Integration weights of the CIE 1931 2-degree observer on the grid
 * lambda_i = lambda0 + i*dlambda, i < n (paper: T_cmf in R^{3 x n}, colour
 * loss of Sec. 4.3).  The CMFs are the analytic multi-lobe Gaussian fit of
 * Wyman, Sloan and Shirley (JCGT 2013), evaluated in FP32;
 * T[c][i] = cmf_c(lambda_i) dlambda / sum_j ybar(lambda_j) dlambda with the
 * normalising sum accumulated in FP64, so the unit spectrum has Y = 1.
 *   T_out: device, 3 x n float32.                                           */
HSC_API hsc_status hsc_cmf_weights(hsc_ctx* ctx, int n, float lambda0, float dlambda,
                           float* T_out, void* stream);

/* Fold the colour projection into the decoder: M = T D (3 x k), so that
 * XYZ = T (D z) = M z (decode to XYZ, Fig. 2b).  FP32, sums over i in order.
 *   T: device 3 x n;  D: device n x k (decoder W_dec, Eq. 4);  M_out: device 3 x k. */
HSC_API hsc_status hsc_fold_xyz(hsc_ctx* ctx, const float* T, const float* D, int k, int n,
                        float* M_out, void* stream);

/* ------------------------------------------------------------------ encode */

/* Encode m spectra (Eq. 4, z = W_enc s); the paper encodes every spectral
 * asset a single time per scene (Fig. 2b): codes[j][c] = sum_i E[c][i] spectra[j][i], FP32
 * (per-lane partial sums, then a fixed butterfly), stored as `out_dt` (F32, BF16 or F16,
 * round-to-nearest-even).
 *   E: device k x n float32;  spectra: device m x n float32;
 *   codes_out: device m x k of out_dt.  1 <= n <= HSC_MAX_N, 1 <= k <= HSC_MAX_K. */
HSC_API hsc_status hsc_encode(hsc_ctx* ctx, const float* E, int k, int n, const float* spectra, int m,
                      void* codes_out, hsc_dtype out_dt, void* stream);

/* Encode a scene's material reflectances and light SPDs in one launch
 * (Eq. 4, Fig. 2b).  Every code value is summed exactly as hsc_encode sums
 * it, so the codes are the bits of hsc_encode on each set; one launch
 * instead of two is what a per-frame encode (a changing scene) saves.
 *   E: device k x n float32;  mat_spectra: device n_mat x n float32;
 *   light_spd: device n_lights x n float32;
 *   mat_codes_out: device n_mat x k and light_codes_out: device n_lights x k,
 *   both of out_dt (F32, BF16 or F16, round-to-nearest-even).
 *   n_mat, n_lights >= 0; a set with count 0 is skipped (its pointers may be NULL).
 *   1 <= n <= HSC_MAX_N, 1 <= k <= HSC_MAX_K.                                */
HSC_API hsc_status hsc_encode_assets(hsc_ctx* ctx, const float* E, int k, int n, const float* mat_spectra,
                             int n_mat, void* mat_codes_out, const float* light_spd, int n_lights,
                             void* light_codes_out, hsc_dtype out_dt, void* stream);

/* ----------------------------------------------------------- latent shade */

/* Shade one RGB pass: code channels 3b..3b+2 of every pixel (Fig. 2b: the
 * k-code is split into B three-channel blocks, each rendered on its own).
 *   g1: primary G-buffer (P pixels); g2: secondary G-buffer or NULL (direct only);
 *   mat_codes: device n_mat x k of code_dt;  light_codes: device L x k of code_dt;
 *   code_dt: F32, BF16 or F16 (converted to FP32 on load, FP32 accumulation);
 *   rgb_out: device P x 3 float32.                                           */
HSC_API hsc_status hsc_shade_pass(hsc_ctx* ctx, const hsc_gbuffer* g1, const hsc_gbuffer* g2, int64_t pixels,
                          const void* mat_codes, int n_mat, const hsc_lights* lights,
                          const void* light_codes, int k, hsc_dtype code_dt, int b,
                          float* rgb_out, void* stream);

/* Reassemble B pass images into the k-channel latent image (Fig. 2b): latent[p][3b + j] = pass_b[p][j].
 *   passes: host array of B device pointers, each P x 3 float32;
 *   latent_out: device P x 3B float32.                                       */
HSC_API hsc_status hsc_reassemble(hsc_ctx* ctx, const float* const* passes, int B, int64_t pixels,
                          float* latent_out, void* stream);

/* Latent shading of a whole frame (Sec. 4-6, Fig. 2b).
 *   mode: HSC_PASSES (B shade passes into context scratch + reassembly) or
 *         HSC_FUSED (one launch for k <= 15; larger k in chunks of 15).
 *   latent_out: device P x k, latent_dt F32 (16-byte aligned) or FP8_E4M3
 *         (then latent_scales, device k float32, receives the per-channel
 *         scales max_p z_c / 448 and the codes are RNE(z / scale), saturating).
 *   xyz_out: NULL, or device P x 3 float32 receiving XYZ = M_xyz z computed
 *         from the FP32 latent (fused for FUSED and k <= 15);
 *   srgb8_out: NULL, or device P x 3 bytes receiving the 8-bit sRGB of that
 *         XYZ, the same bytes hsc_decode_xyz gives for the FP32 latent (fused
 *         into the shading epilogue for FUSED and k <= 15);
 *   M_xyz: device 3 x k from hsc_fold_xyz (required when either is set).
 * Uses context scratch for PASSES images and for the fp8 path (such calls on
 * one context must be ordered on one stream).  A launch on the dynamic tile
 * queue (a tuned or forced waves = -1) takes its tiles from a counter of its
 * own stream, so F32 FUSED calls on different streams may overlap; after
 * HSC_QUEUE_SLOTS distinct streams a context launches on the static
 * persistent grid instead (same results).  Destroy a stream only once its
 * launches have finished: a new stream may reuse the handle, and its counter. */
HSC_API hsc_status hsc_shade_latent(hsc_ctx* ctx, const hsc_gbuffer* g1, const hsc_gbuffer* g2, int64_t pixels,
                            const void* mat_codes, int n_mat, const hsc_lights* lights,
                            const void* light_codes, int k, hsc_dtype code_dt, hsc_mode mode,
                            void* latent_out, hsc_dtype latent_dt, float* latent_scales,
                            float* xyz_out, uint8_t* srgb8_out, const float* M_xyz, void* stream);

/* A latent frame straight from spectral assets, in one launch (Eq. 4 and 6,
 * Fig. 2b).  The paper encodes materials and lights once per scene; for a
 * small frame the encode launches cost more than the encode, so here every
 * CTA of the fused shading launch first encodes the materials and lights into
 * shared memory, each code value summed exactly as hsc_encode sums it.  The
 * latent image, XYZ and sRGB8 are therefore the bits of hsc_encode (FP32
 * codes) followed by hsc_shade_latent (HSC_FUSED) with the same outputs.
 *   E: device k x n (W_enc);  mat_spectra: device n_mat x n;  light_spd:
 *   device L x n (unit-peak SPDs, scaled by the lights' intensities as in
 *   hsc_shade_latent);  latent_out: device P x k float32;  xyz_out, srgb8_out,
 *   M_xyz: as in hsc_shade_latent (nullable outputs).
 * Limits (HSC_ERR_INVALID_ARG beyond them): k in {3, 6, 9}, 1 <= n <=
 * HSC_MAX_N, n_mat x k <= HSC_ASSETS_MAX_CODES, L <= HSC_ASSETS_MAX_LIGHTS.
 * Every CTA repeats the encode (n_mat + L) x k dot products of length n, so
 * large frames or large asset sets are better served by hsc_encode once and
 * hsc_shade_latent per frame.  No scratch memory.                          */
HSC_API hsc_status hsc_shade_latent_assets(hsc_ctx* ctx, const hsc_gbuffer* g1, const hsc_gbuffer* g2,
                                           int64_t pixels, const float* E, int k, int n, const float* mat_spectra,
                                           int n_mat, const hsc_lights* lights, const float* light_spd,
                                           float* latent_out, float* xyz_out, uint8_t* srgb8_out,
                                           const float* M_xyz, void* stream);

/* Per-channel fp8 quantisation of an FP32 latent image: scale_c = max_p z_c / 448
 * (1 for an all-zero channel), code = RNE_e4m3(z * (1/scale_c)) saturating.
 *   latent: device P x k float32;  codes_out: device P x k bytes;  scales_out: device k.
 * Uses the context's reduction scratch.                                      */
HSC_API hsc_status hsc_quantize_fp8(hsc_ctx* ctx, const float* latent, int64_t pixels, int k,
                            uint8_t* codes_out, float* scales_out, void* stream);

/* Allocation-free fp8 quantiser.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory at all -- for
 * example a plugin inside a host renderer that owns the GPU's memory budget
 * through its own allocator, or a frame loop with a hard deadline that cannot
 * afford cudaMalloc's device-wide synchronisation.  Those callers cannot use
 * hsc_create (it allocates), so this call needs no context.
 * It computes exactly what hsc_quantize_fp8 computes.  Its only scratch, one
 * max word per channel, is a static device array of HSC_NOALLOC_MAX_K words
 * (384 bytes) that every GPU loading the library holds until process exit;
 * k > HSC_NOALLOC_MAX_K is rejected with HSC_ERR_INVALID_ARG.
 *   Runs on the calling thread's current device.  The first call on a device
 *   looks up the array's device address (cudaGetSymbolAddress) and caches it;
 *   make that first call before any stream capture.  Each call clears the
 *   words it uses, but all calls share the one array: calls whose work
 *   overlaps on the GPU (other streams, other threads) race on it and must be
 *   serialised by the caller.  Allocates nothing: no cudaMalloc, no cudaFree.
 *   latent: device P x k float32 (16-byte aligned);  codes_out: device P x k
 *   bytes (4-byte aligned);  scales_out: device k float32.                    */
HSC_API hsc_status hsc_quantize_fp8_noalloc(const float* latent, int64_t pixels, int k, uint8_t* codes_out,
                                            float* scales_out, void* stream);

/* ------------------------------------------------------------------ decode */

/* Decode a latent image to XYZ (and optionally 8-bit sRGB) with the folded
 * 3 x k matrix (the final decode of Fig. 2b):
 *   xyz = M_xyz z;  srgb = OETF(clamp(M_sRGB xyz, 0, 1)), u8 = floor(255 srgb + 0.5)
 * with M_sRGB the IEC 61966-2-1 matrix.
 *   latent: device P x k of dt (F32, BF16, F16 or FP8_E4M3 + scales);
 *   scales: device k float32 for FP8 (else ignored);
 *   xyz_out: device P x 3 float32, or NULL when only srgb8_out is wanted;
 *   srgb8_out: NULL or device P x 3 bytes (at least one output must be set). */
HSC_API hsc_status hsc_decode_xyz(hsc_ctx* ctx, const void* latent, hsc_dtype dt, const float* scales,
                          int64_t pixels, int k, const float* M_xyz, float* xyz_out,
                          uint8_t* srgb8_out, void* stream);

/* Decode a latent image to n-sample spectra, s_hat = W_dec z (Eq. 4).
 *   dt = F32, k <= 10: tensor cores with FP32 accuracy: z and D split into
 *        three bf16 parts each (hi + mid + lo), the six leading products
 *        laid side by side along K (K = 48 for k <= 8, 64 for k = 9, 10),
 *        FP32 accumulation.
 *   dt = F32, k > 10: FP32 FMAs on CUDA cores, sums over channels in order.
 *   dt = BF16 or FP8_E4M3 (+ scales): tensor-core contraction
 *        [P x 16 (k zero-padded)] x [16 x n] with BF16 operands (z exact in
 *        bf16 for fp8 codes; D * scale rounded to bf16) and FP32 accumulation.
 *   D: device n x k float32;  spectra_out: device P x n float32 (16-byte aligned). */
HSC_API hsc_status hsc_decode_spectra(hsc_ctx* ctx, const void* latent, hsc_dtype dt, const float* scales,
                              int64_t pixels, int k, const float* D, int n,
                              float* spectra_out, void* stream);

/* --------------------------------------------------------- spectral shade */

/* Naive n-sample spectral shading, the paper's ground truth whose cost is
 * linear in n (Sec. 1, Sec. 6): the shading model above on n samples, with
 * XYZ = T S fused.
 *   mat_spectra: device n_mat x n;  light_spd: device L x n (unit peak);
 *   T: device 3 x n from hsc_cmf_weights;  xyz_out: device P x 3;
 *   spectra_out: NULL or device P x n float32.                               */
HSC_API hsc_status hsc_shade_spectral(hsc_ctx* ctx, const hsc_gbuffer* g1, const hsc_gbuffer* g2, int64_t pixels,
                              const float* mat_spectra, int n_mat, const hsc_lights* lights,
                              const float* light_spd, int n, const float* T,
                              float* xyz_out, float* spectra_out, void* stream);

/* ------------------------------------------------------------ batched frames */

/* One frame of a batched launch: its own G-buffer(s), codes (from its own
 * codec), lights, code length and folded decode matrix.  Pointers are
 * device pointers, as in hsc_shade_latent.                                  */
typedef struct {
  hsc_gbuffer g1;
  hsc_gbuffer g2;          /* used when has_g2 != 0                          */
  int32_t has_g2;
  int64_t pixels;
  const void* mat_codes;   /* n_mat x k of code_dt                           */
  int32_t n_mat;
  hsc_lights lights;
  const void* light_codes; /* L x k of code_dt                               */
  int32_t k;               /* 6 or 9                                         */
  hsc_dtype code_dt;       /* F32, BF16 or F16                               */
  const float* M_xyz;      /* 3 x k                                          */
  float* xyz_out;          /* P x 3 float32                                  */
  float* latent_out;       /* P x k float32, or NULL                         */
} hsc_frame;

typedef struct hsc_batch hsc_batch;

/* Prepare a batch of frames of uneven size, light count, k and codec for
 * one persistent latent-shading launch with the XYZ decode fused (the
 * batched-serving extension; the paper renders one frame at a time).  Copies
 * the frame descriptors to the device, picks the tile shape (pixels per
 * thread, threads per CTA, scalar or f32x2) by timing every candidate on the
 * batch when autotuning is on (hsc_set_autotune), and records a CUDA graph of
 * the launch.  Synchronous; allocates the batch's own descriptors.  Every
 * frame's result is bit-identical to shading that frame alone with
 * hsc_shade_latent.  The frames' buffers must stay valid while the batch
 * exists.                                                                    */
HSC_API hsc_status hsc_batch_create(hsc_ctx* ctx, const hsc_frame* frames, int count, hsc_batch** out);
/* Replay the batch's graph on `stream` (queue reset + one kernel).          */
HSC_API hsc_status hsc_batch_shade(hsc_ctx* ctx, hsc_batch* batch, void* stream);
/* Synchronise the device and free the batch.                                */
HSC_API void hsc_batch_destroy(hsc_batch* batch);

/* One-shot batched launch for continuous batching: shades and decodes to XYZ
 * up to HSC_MAX_FRAMES_PER_CALL frames in one persistent launch on `stream`,
 * asynchronously (descriptors go through a ring of 8 pinned host buffers in
 * the context; a call takes a slot whose previous launch has finished and
 * blocks the host only when all 8 are still in flight).  Same results as hsc_batch_shade and as
 * shading each frame alone.  Tile shape: 2 pixels per thread, 128 threads,
 * unless hsc_force_launch_config overrides it.  The first call allocates the
 * ring (pinned host and device memory); count = 0 only does that, so a
 * server can prepare before its first request.                              */
HSC_API hsc_status hsc_shade_frames(hsc_ctx* ctx, const hsc_frame* frames, int count, void* stream);

/* ------------------------------------------------------ RGB-to-latent upsampling */

/* Latent upsampling from RGB (Sec. 5): per pixel a three-layer perceptron
 *     h1 = silu(W1 c + b1),  h2 = silu(W2 h1 + b2),  z = W3 h2 + b3,
 * silu(x) = x / (1 + exp(-x)), hidden width HSC_UPSAMPLE_HIDDEN (128).
 *   rgb: device P x 3 float32 linear RGB;  W1: device 128 x 3, b1: 128,
 *   W2: device 128 x 128 (row = output unit), b2: 128, W3: device k x 128,
 *   b3: k, all float32;  z_out: device P x k float32;  1 <= k <= 16.
 * Precision: the colour, the weights and both hidden activations are rounded
 * to f16 for the tensor cores and products accumulate in FP32; each bias b
 * enters its layer's product as the f16 pair hi = f16(b), lo = f16(b - hi)
 * (b to about 2^-22 relative); SiLU is FP32 through the hardware tanh
 * approximation (silu(x) = x/2 (1 + tanh(x/2))), its result rounded to f16.
 * Range: f16 holds magnitudes below 65504, so colours, weights, biases and
 * hidden activations must stay below that; beyond it they overflow to
 * infinity.
 * No scratch memory; asynchronous on `stream`.                              */
HSC_API hsc_status hsc_upsample_rgb(hsc_ctx* ctx, const float* rgb, int64_t pixels, const float* W1,
                                    const float* b1, const float* W2, const float* b2, const float* W3,
                                    const float* b3, int k, float* z_out, void* stream);

/* ------------------------------------------------------------- path tracing */

/* Path tracing with per-channel throughput (the renderer of Sec. 6): camera
 * rays through jittered pixel positions, Lambertian reflection sampled by the
 * cosine (each reflection multiplies the throughput by the reflectance), a
 * path ends on an emitting rectangle, on leaving the scene or after `depth`
 * reflections; pixel = mean over `spp` samples of emit (.) mat_{m_0} (.) ...
 * With spectra (channels = n, to_xyz = T) this is the naive spectral path
 * tracer; with codes (channels = k, to_xyz = M = T D) the latent one, the
 * per-channel product being the blockwise product of Eq. 6.  The paths do
 * not depend on the channels: both modes trace the same paths.
 *   quads: device n_quads x 8 float32 rows (axis 0/1/2, c, u0, u1, v0, v1,
 *     normal sign, material; material -1 = emitter): the rectangle
 *     x[axis] = c, u0 <= x[u] <= u1, v0 <= x[v] <= v1, (u, v) the other axes
 *     in increasing order;  spheres: device n_spheres x 5 (centre, radius,
 *     material; the normal is (hit - centre) / radius, so a negative radius
 *     makes the normals point inward: a closed room seen from inside);  camera: device 4 x 3 (origin, image-plane lower-left
 *     corner, horizontal and vertical spans; pixel index y * width + x with
 *     y up);  materials: device n_mat x channels;  emit: device channels;
 *   to_xyz: device 3 x channels;  xyz_out: device P x 3;  channels_out:
 *     device P x channels pixel means (nullable; channels <= 16).
 * Random numbers: Philox4x32-10 with counter (pixel, sample, vertex, 0) and
 * key (seed, 0).  Limits: 32 rectangles, 32 spheres, depth <= 16,
 * n_mat <= 255; out-of-range materials set the error word.               */
HSC_API hsc_status hsc_path_trace(hsc_ctx* ctx, const float* quads, int n_quads, const float* spheres,
                                  int n_spheres, const float* camera, int width, int height, int spp, int depth,
                                  uint32_t seed, const float* materials, int n_mat, const float* emit, int channels,
                                  const float* to_xyz, float* xyz_out, float* channels_out, void* stream);

/* ------------------------------------------------------- codec fitting sweep */

/* One Adam step of the paper's codec parameterisation (Sec. 4.1-4.5):
 * E = softplus(E~), D = softplus(D~) with beta `softplus_beta`, loss Eq. 8
 * (weights e2e, rec, code, col per variant) on one mini-batch shared by all
 * `variants`, for every variant at once (one CTA each).
 *   R_all, L_all: device rows of n float32 (training reflectances, lights);
 *   pair_r, pair_l: device `pairs` int32 row indices; pair_scale: device
 *   `pairs` float32 light scales (pair p is R_all[pair_r[p]],
 *   L_all[pair_l[p]] * pair_scale[p]);  T: device 3 x n (hsc_cmf_weights);
 *   weights: device variants x 4;  Et: device variants x k x n;  Dt: device
 *   variants x n x k;  mE, vE, mD, vD: Adam moments of the same shapes (zero
 *   before step 1); updated in place.  step: 1-based (bias correction).
 *   active: device `variants` int32 flags or NULL; a variant whose flag is
 *   0 is skipped (parameters, moments and outputs untouched).
 *   losses_out: device variants x 5 (total, e2e, rec, code, col) at the
 *   parameters before the step, or NULL;  grad_out: device variants x 2kn,
 *   dL/dE~ then dL/dD~, or NULL.
 * Limits: k a multiple of 3 up to 15, n <= 128, pairs <= 256.            */
HSC_API hsc_status hsc_codec_fit_step(hsc_ctx* ctx, int variants, int k, int n, const float* R_all,
                                      const float* L_all, const int32_t* pair_r, const int32_t* pair_l,
                                      const float* pair_scale, int pairs, const float* T, const float* weights,
                                      float* Et, float* Dt, float* mE, float* vE, float* mD, float* vD, int step,
                                      float lr, float beta1, float beta2, float eps, float softplus_beta,
                                      const int32_t* active, float* losses_out, float* grad_out, void* stream);

/* The Eq. 8 loss terms of every active variant at its current parameters on
 * one batch (the validation loss of the sweep, Sec. 4.5), without a step;
 * arguments as hsc_codec_fit_step.  E_out: device variants x k x n
 * softplus(E~), D_out: device variants x n x k softplus(D~) (each NULL or
 * written; the decoder and encoder the selection stage evaluates).  At least
 * one output must be given.                                                 */
HSC_API hsc_status hsc_codec_fit_eval(hsc_ctx* ctx, int variants, int k, int n, const float* R_all,
                                      const float* L_all, const int32_t* pair_r, const int32_t* pair_l,
                                      const float* pair_scale, int pairs, const float* T, const float* weights,
                                      const float* Et, const float* Dt, float softplus_beta, const int32_t* active,
                                      float* losses_out, float* E_out, float* D_out, void* stream);

/* Early stopping of the sweep (Sec. 4.5: training stops after `patience`
 * epochs without a lower validation loss).  Per variant v with active[v] != 0:
 * if val_loss[v * val_stride] < best_loss[v] the loss becomes best_loss[v],
 * wait[v] = 0 and Et[v], Dt[v] are copied to best_Et[v], best_Dt[v];
 * otherwise wait[v] += 1 and active[v] = 0 once wait[v] >= patience.  A NaN
 * loss is never an improvement.  Inactive variants are left as they are.
 *   Et, best_Et: device variants x k x n;  Dt, best_Dt: variants x n x k;
 *   best_loss: device variants float32 (+inf before the first epoch);  wait,
 *   active: device variants int32 (0 and 1 before the first epoch);
 *   epochs: device variants int32 or NULL, incremented for every variant
 *   active at the update (the number of epochs it trained);
 *   n_active_out: device int32 or NULL: the number of active variants after
 *   the update.  Uses one word of the context's scratch; launches that share a
 *   context must not overlap.                                               */
HSC_API hsc_status hsc_codec_fit_track(hsc_ctx* ctx, int variants, int k, int n, const float* val_loss,
                                       int val_stride, const float* Et, const float* Dt, float* best_Et,
                                       float* best_Dt, float* best_loss, int32_t* wait, int32_t* active,
                                       int32_t* epochs, int patience, int32_t* n_active_out, void* stream);

/* --------------------------------------------------------- multi-bounce chains */

/* Multi-bounce chains, the codec-selection proxy of Sec. 4.5: chain c starts
 * from light chain_light[c] and multiplies in reflectance chain_refl[c][b] at
 * bounce b (S(b) = R (.) S(b-1)); the latent chain runs the same recurrence on
 * codes with the blockwise product (Eq. 6).  At every depth both are taken to
 * XYZ (T S and M z with M = T D), scaled by 1 / max(T L) so the light's
 * largest tristimulus value is 1, converted to CIELAB with the equal-energy
 * white T @ 1, and compared by CIE94 (spectral chain as reference) and
 * CIEDE2000.
 *   refl: device n_refl x n;  lights: device n_lights x n;  E: k x n;  D: n x k;
 *   T: 3 x n (hsc_cmf_weights);  chain_light: device chains int32;
 *   chain_refl: device chains x depth int32 (depth <= 8);
 *   de94_out, de2000_out: device depth x chains float32 (depth-major);
 *   stats_out: device depth x 4 doubles {mean dE94, p95 dE94, mean dE2000, p95 dE2000}
 *   (p95 by nearest rank).  Out-of-range indices set the device error word.
 * Uses context scratch (codes) and the reduction scratch.                   */
HSC_API hsc_status hsc_chain_eval(hsc_ctx* ctx, const float* refl, int n_refl, const float* lights, int n_lights,
                                  const float* E, const float* D, int k, int n, const float* T,
                                  const int32_t* chain_light, const int32_t* chain_refl, int64_t chains, int depth,
                                  float* de94_out, float* de2000_out, double* stats_out, void* stream);

/* ----------------------------------------------------------------- metrics */

/* Colour difference of a test image against a reference image.  Both are
 * divided by Y_ref = max_p Y of the reference, converted to CIELAB with white
 * (T @ 1) (CIE 1976), and compared per pixel by CIEDE2000 (kL = kC = kH = 1),
 * CIE94 (graphic arts; the paper's codec-selection metric, Sec. 4.5) and
 * Delta E 76 (the paper's upsampler loss, Sec. 5.2).
 *   stats_out: device 8 doubles = {mean dE2000, p95 dE2000 (nearest rank),
 *              mean dE94, mean dE76, Y_ref, max dE2000, pixels, 0}.
 *   de_out: NULL or device P float32 per-pixel dE2000.
 * Uses the context's reduction scratch.                                      */
HSC_API hsc_status hsc_delta_e(hsc_ctx* ctx, const float* xyz_test, const float* xyz_ref, int64_t pixels,
                       const float* T, int n, float* de_out, double* stats_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HSC_H_ */
