// Latent shading dispatch (channel chunk -> kernel instantiation) and the
// reassembly of k/3 RGB pass images into the k-channel latent image (Fig. 2b).
// The kernels themselves are in shade_latent_kernel.cuh.
#include "common.cuh"
#include "shade_latent.cuh"

namespace hsc {

hsc_status launch_shade_codes(const ShadeArgs& a, int kc, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  switch (kc) {
    case 3: return launch_kc<3>(a, sec, cfg, s);
    case 6: return launch_kc<6>(a, sec, cfg, s);
    case 9: return launch_kc<9>(a, sec, cfg, s);
    case 12: return launch_kc<12>(a, sec, cfg, s);
    case 15: return launch_kc<15>(a, sec, cfg, s);
    default: return set_error(HSC_ERR_UNSUPPORTED, "channel chunk %d not instantiated", kc);
  }
}

namespace {

struct PassPtrs {
  const float* p[HSC_MAX_K / 3];
};

__global__ void reassemble_kernel(PassPtrs pp, int B, int64_t P, float* __restrict__ out) {
  const int k = 3 * B;
  const int64_t total = P * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx / k;
    const int c = (int)(idx - p * k);
    const int b = c / 3;
    out[idx] = __ldg(pp.p[b] + 3 * p + (c - 3 * b));
  }
}

}  // namespace

hsc_status launch_reassemble(const float* const* passes, int B, int64_t P, float* out, int sm_count,
                             cudaStream_t s) {
  PassPtrs pp;
  for (int b = 0; b < B; ++b) pp.p[b] = passes[b];
  const int64_t total = P * 3 * B;
  int64_t grid = (total + 255) / 256;
  const int64_t cap = (int64_t)sm_count * 8;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  reassemble_kernel<<<(unsigned)grid, 256, 0, s>>>(pp, B, P, out);
  return check_launch("reassemble_kernel");
}

LaunchCfg default_cfg(const hsc_ctx* ctx) {
  LaunchCfg c;
  c.sm_count = ctx->sm_count;
  c.ppt = 2;
  c.waves = 1;
  return c;
}

}  // namespace hsc
