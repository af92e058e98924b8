// Instantiation of the latent shading kernels for 12 channels per launch.
#include "shade_latent_kernel.cuh"

namespace hsc {
template hsc_status launch_kc<12>(const ShadeArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s);
}  // namespace hsc
