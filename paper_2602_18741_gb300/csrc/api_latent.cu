// C-ABI entry points of latent shading: one RGB pass, reassembly, and the
// whole-frame call in PASSES or FUSED mode (Fig. 2b of the paper).
#include "common.cuh"
#include "shade_latent.cuh"
#include "tune.cuh"

namespace hsc {

hsc_status validate_gbuffer(const hsc_gbuffer* g, const char* name, int64_t pixels) {
  HSC_REQUIRE(g != nullptr, "%s is null", name);
  if (pixels == 0) return HSC_OK;  // empty images may carry null arrays
  HSC_REQUIRE(g->normal && g->pos && g->mat, "%s has a null array", name);
  HSC_REQUIRE(aligned(g->normal, 4) && aligned(g->pos, 4) && aligned(g->mat, 4), "%s arrays must be 4-byte aligned",
              name);
  return HSC_OK;
}

hsc_status validate_lights(const hsc_lights* l) {
  HSC_REQUIRE(l != nullptr, "lights is null");
  HSC_REQUIRE(l->count >= 1, "light count %d < 1", l->count);
  HSC_REQUIRE(l->pos && l->intensity, "light arrays are null");
  HSC_REQUIRE(aligned(l->pos, 4) && aligned(l->intensity, 4), "light arrays must be 4-byte aligned");
  return HSC_OK;
}

static hsc_status validate_common(const hsc_gbuffer* g1, const hsc_gbuffer* g2, int64_t P, const void* mat_codes,
                                  int n_mat, const hsc_lights* lights, const void* light_codes, int k,
                                  hsc_dtype code_dt) {
  HSC_REQUIRE(P >= 0, "pixel count %lld negative", (long long)P);
  HSC_REQUIRE(k >= 3 && k <= HSC_MAX_K && k % 3 == 0, "k=%d must be a multiple of 3 in [3, %d]", k, HSC_MAX_K);
  HSC_REQUIRE(code_dt == HSC_F32 || code_dt == HSC_BF16 || code_dt == HSC_F16, "code dtype must be F32, BF16 or F16");
  HSC_REQUIRE(n_mat >= 1 && n_mat <= HSC_MAX_MAT, "n_mat=%d out of range", n_mat);
  HSC_REQUIRE(mat_codes && light_codes, "code arrays are null");
  HSC_REQUIRE(aligned(mat_codes, code_dt == HSC_F32 ? 4 : 2) && aligned(light_codes, code_dt == HSC_F32 ? 4 : 2),
              "code arrays misaligned");
  HSC_TRY(validate_gbuffer(g1, "g1", P));
  if (g2) HSC_TRY(validate_gbuffer(g2, "g2", P));
  HSC_TRY(validate_lights(lights));
  return HSC_OK;
}

static ShadeArgs base_args(hsc_ctx* ctx, const hsc_gbuffer* g1, const hsc_gbuffer* g2, int64_t P,
                           const void* mat_codes, int n_mat, const hsc_lights* lights, const void* light_codes,
                           int k, hsc_dtype code_dt) {
  ShadeArgs a{};
  a.n1 = g1->normal;
  a.x1 = g1->pos;
  a.m1 = g1->mat;
  if (g2) {
    a.n2 = g2->normal;
    a.x2 = g2->pos;
    a.m2 = g2->mat;
  }
  a.P = P;
  a.mat_codes = mat_codes;
  a.n_mat = n_mat;
  a.lpos = lights->pos;
  a.linten = lights->intensity;
  a.L = lights->count;
  a.light_codes = light_codes;
  a.code_dt = (int)code_dt;
  a.k = k;
  a.err = ctx->d_err;
  return a;
}

// One shading launch of `kc` channels in the tuned (or default) configuration.
// A dynamically scheduled launch takes its tiles from the counter pair of its
// stream; with no pair left it runs as the persistent static grid instead
// (same bits: the schedule never changes what a pixel computes).
static hsc_status shade_launch(hsc_ctx* ctx, const ShadeArgs& a, int kc, bool sec, cudaStream_t s) {
  const TuneKey key = make_tune_key(a.srgb8 ? kTuneLatentSrgb : kTuneLatent, kc, sec, a.L, a.P, a.code_dt);
  unsigned int* queue = stream_queue(ctx, s);
  auto launch = [&](const LaunchCfg& c0) {
    LaunchCfg c = c0;
    c.queue = queue;
    if (c.waves < 0 && !queue) c.waves = 1;
    return launch_shade_codes(a, kc, sec, c, s);
  };
  LaunchCfg cfg;
  HSC_TRY(tuned_cfg(ctx, key, latent_candidates(ctx), launch, s, &cfg));
  return launch(cfg);
}

}  // namespace hsc

using hsc::ShadeArgs;

extern "C" {

size_t hsc_shade_latent_scratch_bytes(int64_t pixels, int k, hsc_mode mode, hsc_dtype latent_dt) {
  if (pixels <= 0 || k <= 0) return 0;
  size_t bytes = 0;
  const size_t img = (size_t)pixels * (size_t)k * sizeof(float);
  if (latent_dt != HSC_F32) bytes += img;   // FP32 latent before quantisation
  if (mode == HSC_PASSES) bytes += img;     // B pass images of P x 3
  return bytes;
}

hsc_status hsc_shade_pass(hsc_ctx* ctx, const hsc_gbuffer* g1, const hsc_gbuffer* g2, int64_t pixels,
                          const void* mat_codes, int n_mat, const hsc_lights* lights, const void* light_codes,
                          int k, hsc_dtype code_dt, int b, float* rgb_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_TRY(hsc::validate_common(g1, g2, pixels, mat_codes, n_mat, lights, light_codes, k, code_dt));
  HSC_REQUIRE(b >= 0 && 3 * b < k, "pass %d out of range for k=%d", b, k);
  HSC_REQUIRE(rgb_out && hsc::aligned(rgb_out, 4), "rgb_out null or misaligned");
  if (pixels == 0) return HSC_OK;
  HSC_GUARD(ctx);
  ShadeArgs a = hsc::base_args(ctx, g1, g2, pixels, mat_codes, n_mat, lights, light_codes, k, code_dt);
  a.c0 = 3 * b;
  a.out = rgb_out;
  a.out_stride = 3;
  a.out_c0 = 0;
  return hsc::shade_launch(ctx, a, 3, g2 != nullptr, hsc::as_stream(stream));
}

hsc_status hsc_reassemble(hsc_ctx* ctx, const float* const* passes, int B, int64_t pixels, float* latent_out,
                          void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(B >= 1 && 3 * B <= HSC_MAX_K, "B=%d out of range", B);
  HSC_REQUIRE(pixels >= 0, "negative pixel count");
  HSC_REQUIRE(passes != nullptr && latent_out != nullptr, "null pointer");
  for (int b = 0; b < B; ++b) HSC_REQUIRE(passes[b] != nullptr && hsc::aligned(passes[b], 4), "pass %d null", b);
  if (pixels == 0) return HSC_OK;
  HSC_GUARD(ctx);
  return hsc::launch_reassemble(passes, B, pixels, latent_out, ctx->sm_count, hsc::as_stream(stream));
}

hsc_status hsc_shade_latent(hsc_ctx* ctx, const hsc_gbuffer* g1, const hsc_gbuffer* g2, int64_t pixels,
                            const void* mat_codes, int n_mat, const hsc_lights* lights, const void* light_codes,
                            int k, hsc_dtype code_dt, hsc_mode mode, void* latent_out, hsc_dtype latent_dt,
                            float* latent_scales, float* xyz_out, uint8_t* srgb8_out, const float* M_xyz,
                            void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_TRY(hsc::validate_common(g1, g2, pixels, mat_codes, n_mat, lights, light_codes, k, code_dt));
  HSC_REQUIRE(mode == HSC_PASSES || mode == HSC_FUSED, "bad mode %d", (int)mode);
  HSC_REQUIRE(latent_dt == HSC_F32 || latent_dt == HSC_FP8_E4M3, "latent dtype must be F32 or FP8_E4M3");
  HSC_REQUIRE(latent_out != nullptr || pixels == 0, "latent_out is null");
  HSC_REQUIRE(latent_dt != HSC_F32 || hsc::aligned(latent_out, 16), "F32 latent_out must be 16-byte aligned");
  HSC_REQUIRE(latent_dt != HSC_FP8_E4M3 || hsc::aligned(latent_out, 4), "fp8 latent_out must be 4-byte aligned");
  HSC_REQUIRE(latent_dt != HSC_FP8_E4M3 || (latent_scales && hsc::aligned(latent_scales, 4)),
              "fp8 latent needs a latent_scales array");
  HSC_REQUIRE(!xyz_out || (M_xyz && hsc::aligned(xyz_out, 4) && hsc::aligned(M_xyz, 4)),
              "xyz_out needs M_xyz (both 4-byte aligned)");
  HSC_REQUIRE(!srgb8_out || (M_xyz && hsc::aligned(M_xyz, 4)), "srgb8_out needs M_xyz (4-byte aligned)");
  if (pixels == 0) return HSC_OK;
  HSC_GUARD(ctx);
  cudaStream_t s = hsc::as_stream(stream);
  const bool sec = g2 != nullptr;
  const int B = k / 3;
  const size_t img = (size_t)pixels * k * sizeof(float);
  HSC_TRY(hsc::ensure_big(ctx, hsc_shade_latent_scratch_bytes(pixels, k, mode, latent_dt), s));
  unsigned char* scratch = ctx->d_big;
  float* lat32 = (latent_dt == HSC_F32) ? reinterpret_cast<float*>(latent_out) : reinterpret_cast<float*>(scratch);
  if (latent_dt != HSC_F32) scratch += img;
  unsigned int* chan_max = reinterpret_cast<unsigned int*>(ctx->d_small + HSC_OFF_CHANMAX);
  ShadeArgs a = hsc::base_args(ctx, g1, g2, pixels, mat_codes, n_mat, lights, light_codes, k, code_dt);

  if (mode == HSC_PASSES) {
    const float* passes[HSC_MAX_K / 3];
    for (int b = 0; b < B; ++b) {
      float* img_b = reinterpret_cast<float*>(scratch) + (size_t)b * pixels * 3;
      passes[b] = img_b;
      ShadeArgs pa = a;
      pa.c0 = 3 * b;
      pa.out = img_b;
      pa.out_stride = 3;
      pa.out_c0 = 0;
      HSC_TRY(hsc::shade_launch(ctx, pa, 3, sec, s));
    }
    HSC_TRY(hsc::launch_reassemble(passes, B, pixels, lat32, ctx->sm_count, s));
    if (latent_dt == HSC_FP8_E4M3) {
      HSC_CUDA(cudaMemsetAsync(chan_max, 0, sizeof(unsigned int) * k, s));
      HSC_TRY(hsc::launch_channel_max(lat32, pixels, k, chan_max, ctx->sm_count, s));
    }
  } else {
    if (latent_dt == HSC_FP8_E4M3) HSC_CUDA(cudaMemsetAsync(chan_max, 0, sizeof(unsigned int) * k, s));
    for (int c0 = 0; c0 < k; c0 += 15) {
      const int kc = (k - c0) < 15 ? (k - c0) : 15;
      ShadeArgs fa = a;
      fa.c0 = c0;
      fa.out = lat32;
      fa.out_stride = k;
      fa.out_c0 = c0;
      fa.xyz = (k <= 15) ? xyz_out : nullptr;
      fa.srgb8 = (k <= 15) ? srgb8_out : nullptr;
      fa.M = M_xyz;
      fa.chan_max = (latent_dt == HSC_FP8_E4M3) ? chan_max : nullptr;
      HSC_TRY(hsc::shade_launch(ctx, fa, kc, sec, s));
    }
  }
  if (latent_dt == HSC_FP8_E4M3)
    HSC_TRY(hsc::launch_quantize(lat32, pixels, k, chan_max, reinterpret_cast<uint8_t*>(latent_out), latent_scales,
                                 ctx->sm_count, s));
  if ((xyz_out || srgb8_out) && (mode == HSC_PASSES || k > 15))
    HSC_TRY(hsc::launch_decode_xyz(lat32, HSC_F32, nullptr, pixels, k, M_xyz, xyz_out, srgb8_out, ctx->sm_count, s));
  return HSC_OK;
}

}  // extern "C"
