// Asset encoding z = W_enc s (Eq. 4), done once per scene for every material
// reflectance and light SPD (Fig. 2b).  m*k outputs of n FMAs each: a few
// hundred thousand flops per scene, so one thread per code value is enough.
#include "common.cuh"

namespace {

__global__ void encode_kernel(const float* __restrict__ E, int k, int n, const float* __restrict__ S, int m,
                              void* __restrict__ out, int out_dt) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * k) return;
  const int j = (int)(idx / k), c = (int)(idx % k);
  const float* e = E + (int64_t)c * n;
  const float* s = S + (int64_t)j * n;
  float acc = 0.0f;
  for (int i = 0; i < n; ++i) acc = __fmaf_rn(__ldg(e + i), __ldg(s + i), acc);
  if (out_dt == HSC_F32)
    reinterpret_cast<float*>(out)[idx] = acc;
  else if (out_dt == HSC_BF16)
    reinterpret_cast<unsigned short*>(out)[idx] = hsc::float_to_bf16_bits(acc);
  else
    reinterpret_cast<unsigned short*>(out)[idx] = hsc::float_to_f16_bits(acc);
}

}  // namespace

extern "C" hsc_status hsc_encode(hsc_ctx* ctx, const float* E, int k, int n, const float* spectra, int m,
                                 void* codes_out, hsc_dtype out_dt, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(k >= 1 && k <= HSC_MAX_K, "k=%d out of range [1, %d]", k, HSC_MAX_K);
  HSC_REQUIRE(n >= 1 && n <= HSC_MAX_N, "n=%d out of range [1, %d]", n, HSC_MAX_N);
  HSC_REQUIRE(m >= 0, "m=%d negative", m);
  HSC_REQUIRE(out_dt == HSC_F32 || out_dt == HSC_BF16 || out_dt == HSC_F16, "codes dtype must be F32, BF16 or F16");
  if (m == 0) return HSC_OK;
  HSC_REQUIRE(E && spectra && codes_out, "null pointer");
  HSC_REQUIRE(hsc::aligned(E, 4) && hsc::aligned(spectra, 4) && hsc::aligned(codes_out, out_dt == HSC_F32 ? 4 : 2),
              "misaligned pointer");
  HSC_GUARD(ctx);
  const int64_t total = (int64_t)m * k;
  encode_kernel<<<hsc::ceil_div_i(total, 256), 256, 0, hsc::as_stream(stream)>>>(E, k, n, spectra, m, codes_out,
                                                                                  (int)out_dt);
  return hsc::check_launch("encode_kernel");
}
