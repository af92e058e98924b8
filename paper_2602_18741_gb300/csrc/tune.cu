// Launch-configuration autotuner (see tune.cuh).
#include "tune.cuh"

#include <stdio.h>
#include <string.h>

namespace hsc {

static int ceil_log2(int64_t v) {
  int b = 0;
  while (((int64_t)1 << b) < v && b < 62) ++b;
  return b;
}

TuneKey make_tune_key(int kind, int channels, bool sec, int lights, int64_t pixels, int dtype) {
  TuneKey k;
  k.kind = kind;
  k.channels = channels;
  k.sec = sec ? 1 : 0;
  k.lbucket = ceil_log2(lights);
  k.pbucket = ceil_log2(pixels);
  k.dtype = dtype;
  return k;
}

std::vector<LaunchCfg> latent_candidates(const hsc_ctx* ctx) {
  std::vector<LaunchCfg> v;
  LaunchCfg d = default_cfg(ctx);
  v.push_back(d);
  for (int vec : {1, 2})
    for (int ppt : {1, 2, 4})
      for (int block : {128, 256})
        for (int waves : {1, 0, -1}) {
          LaunchCfg c = d;
          c.ppt = ppt;
          c.block = block;
          c.waves = waves;
          c.vec = vec;
          if (c.ppt == d.ppt && c.block == d.block && c.waves == d.waves && c.vec == d.vec) continue;
          v.push_back(c);
        }
  return v;
}

std::vector<LaunchCfg> spectral_candidates(const hsc_ctx* ctx) {
  std::vector<LaunchCfg> v;
  // default: the persistent lane-group kernel (one geometry term per point and
  // light, register tiles of 8 points)
  LaunchCfg d;
  d.sm_count = ctx->sm_count;
  d.block = 128;
  d.ppt = 1;
  d.waves = 1;
  d.vec = 1;
  d.chunk = 1;
  v.push_back(d);
  LaunchCfg one_cta_per_tile = d;
  one_cta_per_tile.waves = 0;
  v.push_back(one_cta_per_tile);
  // the chunked kernel (geometry term recomputed per chunk of the spectrum)
  for (int chunk : {0, 16, 28, 44})
    for (int vec : {1, 2})
      for (int ppt : {1, 2}) {
        LaunchCfg c = d;
        c.ppt = ppt;
        c.vec = vec;
        c.chunk = chunk;
        v.push_back(c);
      }
  return v;
}

hsc_status tuned_cfg(hsc_ctx* ctx, const TuneKey& key, const std::vector<LaunchCfg>& cands,
                     const std::function<hsc_status(const LaunchCfg&)>& launch, cudaStream_t s, LaunchCfg* out) {
  *out = cands[0];
  if (ctx->forced.ppt > 0) {
    *out = ctx->forced;
    out->sm_count = ctx->sm_count;
    return HSC_OK;
  }
  if (!ctx->autotune || cands.size() < 2) return HSC_OK;
  auto it = ctx->tuned.find(key);
  if (it != ctx->tuned.end()) {
    *out = it->second;
    out->sm_count = ctx->sm_count;
    return HSC_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return HSC_OK;
  cudaEvent_t e0, e1;
  HSC_CUDA(cudaEventCreate(&e0));
  HSC_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  LaunchCfg best_cfg = cands[0];
  char line[256];
  const char* kind = key.kind == kTuneLatent ? "latent" : (key.kind == kTuneLatentSrgb ? "latent+srgb8" : "spectral");
  snprintf(line, sizeof(line), "%s ch=%d sec=%d L<=2^%d P<=2^%d dt=%d:", kind, key.channels, key.sec, key.lbucket,
           key.pbucket, key.dtype);
  std::string rep = line;
  hsc_status st = HSC_OK;
  for (const LaunchCfg& c : cands) {
    if ((st = launch(c)) != HSC_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && st == HSC_OK; ++r) st = launch(c);
    if (st != HSC_OK) break;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = set_error(HSC_ERR_CUDA, "autotune event wait failed");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.0f;
    snprintf(line, sizeof(line), " [ppt=%d block=%d waves=%d vec=%d chunk=%d %.4f ms]", c.ppt, c.block, c.waves, c.vec,
             c.chunk, ms);
    rep += line;
    if (ms < best) {
      best = ms;
      best_cfg = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != HSC_OK) return st;
  snprintf(line, sizeof(line), " -> ppt=%d block=%d waves=%d vec=%d chunk=%d\n", best_cfg.ppt, best_cfg.block,
           best_cfg.waves, best_cfg.vec, best_cfg.chunk);
  rep += line;
  ctx->tune_report += rep;
  ctx->tuned[key] = best_cfg;
  *out = best_cfg;
  return HSC_OK;
}

}  // namespace hsc

extern "C" {

hsc_status hsc_set_autotune(hsc_ctx* ctx, int enable) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  ctx->autotune = enable ? 1 : 0;
  return HSC_OK;
}

const char* hsc_tune_report(hsc_ctx* ctx) { return ctx ? ctx->tune_report.c_str() : ""; }

int hsc_tune_save(hsc_ctx* ctx, char* buf, size_t len) {
  if (!ctx) return -1;
  std::string out;
  char line[160];
  for (const auto& kv : ctx->tuned) {
    const hsc::TuneKey& k = kv.first;
    const hsc::LaunchCfg& c = kv.second;
    snprintf(line, sizeof(line), "%d %d %d %d %d %d %d %d %d %d %d\n", k.kind, k.channels, k.sec, k.lbucket, k.pbucket,
             k.dtype, c.ppt, c.block, c.waves, c.vec, c.chunk);
    out += line;
  }
  if (buf && len > 0) {
    const size_t n = out.size() < len - 1 ? out.size() : len - 1;
    memcpy(buf, out.data(), n);
    buf[n] = '\0';
  }
  return (int)out.size();
}

hsc_status hsc_tune_load(hsc_ctx* ctx, const char* text) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(text != nullptr, "null text");
  const char* p = text;
  while (*p) {
    hsc::TuneKey k;
    hsc::LaunchCfg c;
    int used = 0;
    const int got = sscanf(p, "%d %d %d %d %d %d %d %d %d %d %d%n", &k.kind, &k.channels, &k.sec, &k.lbucket, &k.pbucket,
                           &k.dtype, &c.ppt, &c.block, &c.waves, &c.vec, &c.chunk, &used);
    if (got != 11) break;
    HSC_REQUIRE((c.ppt == 1 || c.ppt == 2 || c.ppt == 4) && (c.block == 128 || c.block == 256) && c.waves >= -1 &&
                    (c.vec == 1 || c.vec == 2) && c.chunk >= 0,
                "bad tuning entry");
    c.sm_count = ctx->sm_count;
    ctx->tuned[k] = c;
    p += used;
    while (*p == '\n' || *p == ' ' || *p == '\r') ++p;
  }
  return HSC_OK;
}

hsc_status hsc_force_launch_config(hsc_ctx* ctx, int ppt, int block, int waves, int vec, int chunk) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  if (ppt <= 0) {
    ctx->forced = hsc::LaunchCfg();
    ctx->forced.ppt = 0;
    return HSC_OK;
  }
  HSC_REQUIRE(ppt == 1 || ppt == 2 || ppt == 4, "ppt must be 1, 2 or 4");
  HSC_REQUIRE(block == 128 || block == 256, "block must be 128 or 256");
  HSC_REQUIRE(waves >= -1 && waves <= 64, "waves out of range");
  HSC_REQUIRE(vec == 1 || vec == 2, "vec must be 1 or 2");
  HSC_REQUIRE(chunk == 0 || chunk == 1 || chunk == 16 || chunk == 28 || chunk == 32 || chunk == 44 || chunk == 84,
              "chunk must be 0, 1, 16, 28, 32, 44 or 84");
  ctx->forced.vec = vec;
  ctx->forced.chunk = chunk;
  ctx->forced.ppt = ppt;
  ctx->forced.block = block;
  ctx->forced.waves = waves;
  return HSC_OK;
}

}  // extern "C"
