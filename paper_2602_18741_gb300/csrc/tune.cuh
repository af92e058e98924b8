// Launch-configuration autotuner of the shading kernels (tile shape: threads
// per CTA, pixels per thread, persistent or one-CTA-per-tile grid).
#pragma once

#include <functional>
#include <vector>

#include "common.cuh"
#include "shade_latent.cuh"

namespace hsc {

enum TuneKind { kTuneLatent = 1, kTuneSpectral = 2, kTuneLatentSrgb = 3 };  // sRGB epilogue: its own class

// Configurations are cached per shape class: kernel, channels per launch,
// secondary bounce on/off, and the light and pixel counts rounded up to
// powers of two.
TuneKey make_tune_key(int kind, int channels, bool sec, int lights, int64_t pixels, int dtype);

std::vector<LaunchCfg> latent_candidates(const hsc_ctx* ctx);
std::vector<LaunchCfg> spectral_candidates(const hsc_ctx* ctx);

// The configuration to launch with.  Tuning off: cands[0].  Tuning on: the
// cached choice for `key`, or -- on the first call of a shape class outside
// stream capture -- every candidate timed on the call's own inputs with CUDA
// events on `s` (one warm-up and three timed launches each), the fastest kept.
// The kernels only write their outputs, so the extra launches change nothing.
hsc_status tuned_cfg(hsc_ctx* ctx, const TuneKey& key, const std::vector<LaunchCfg>& cands,
                     const std::function<hsc_status(const LaunchCfg&)>& launch, cudaStream_t s, LaunchCfg* out);

}  // namespace hsc
