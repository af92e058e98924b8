// Instantiation of the latent shading kernels for 9 channels per launch.
#include "shade_latent_kernel.cuh"

namespace hsc {
template hsc_status launch_kc<9>(const ShadeArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s);
}  // namespace hsc
