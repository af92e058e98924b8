// Tensor-core spectral decode (placeholder until the tcgen05 kernel lands).
#include "common.cuh"

namespace hsc {

hsc_status launch_decode_spectra_tc(hsc_ctx* ctx, const void* latent, int dt, const float* scales, int64_t P, int k,
                                    const float* D, int n, float* out, cudaStream_t s) {
  (void)ctx; (void)latent; (void)dt; (void)scales; (void)P; (void)k; (void)D; (void)n; (void)out; (void)s;
  return set_error(HSC_ERR_UNSUPPORTED, "tensor-core decode not built");
}

}  // namespace hsc
