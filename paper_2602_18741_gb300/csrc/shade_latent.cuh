// Internal launch interface of the latent shading kernels.
#pragma once

#include "common.cuh"

namespace hsc {

constexpr int kLightTile = 256;   // lights staged per shared-memory tile

struct ShadeArgs {
  const float* n1;
  const float* x1;
  const int32_t* m1;
  const float* n2;  // secondary G-buffer (null when direct only)
  const float* x2;
  const int32_t* m2;
  int64_t P;
  const void* mat_codes;
  int n_mat;
  const float* lpos;
  const float* linten;
  int L;
  const void* light_codes;
  int code_dt;
  int k;           // code length: row stride of the code arrays and of M
  int c0;          // first code channel shaded by this launch
  float* out;      // P x out_stride float32
  int out_stride;
  int out_c0;      // channel offset of c0 inside an output row
  float* xyz;      // fused XYZ (only when this launch covers all k channels)
  uint8_t* srgb8;  // fused 8-bit sRGB of the same XYZ (same condition)
  const float* M;  // 3 x k
  unsigned int* chan_max;  // per-channel max bits for the fp8 scale (nullable)
  unsigned int* err;
  int64_t tiles;
  unsigned int* queue;  // dynamic tile queue (zeroed before the launch), or null for static striding
};

LaunchCfg default_cfg(const hsc_ctx* ctx);

// Defined in shade_latent_kernel.cuh, instantiated per KC in shade_latent_k*.cu.
template <int KC>
hsc_status launch_kc(const ShadeArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s);
extern template hsc_status launch_kc<3>(const ShadeArgs&, bool, const LaunchCfg&, cudaStream_t);
extern template hsc_status launch_kc<6>(const ShadeArgs&, bool, const LaunchCfg&, cudaStream_t);
extern template hsc_status launch_kc<9>(const ShadeArgs&, bool, const LaunchCfg&, cudaStream_t);
extern template hsc_status launch_kc<12>(const ShadeArgs&, bool, const LaunchCfg&, cudaStream_t);
extern template hsc_status launch_kc<15>(const ShadeArgs&, bool, const LaunchCfg&, cudaStream_t);
hsc_status launch_shade_codes(const ShadeArgs& a, int kc, bool sec, const LaunchCfg& cfg, cudaStream_t s);
hsc_status launch_reassemble(const float* const* passes, int B, int64_t P, float* out, int sm_count, cudaStream_t s);

// fp8 path (quant.cu)
hsc_status launch_channel_max(const float* latent, int64_t P, int k, unsigned int* chan_max, int sm_count,
                              cudaStream_t s);
hsc_status launch_quantize(const float* latent, int64_t P, int k, const unsigned int* chan_max, uint8_t* codes,
                           float* scales, int sm_count, cudaStream_t s);
// decode (decode.cu)
hsc_status launch_decode_xyz(const void* latent, int dt, const float* scales, int64_t P, int k, const float* M,
                             float* xyz, uint8_t* srgb8, int sm_count, cudaStream_t s);

}  // namespace hsc
