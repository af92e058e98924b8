// Asset encoding z = W_enc s (Eq. 4), done once per scene for every material
// reflectance and light SPD (Fig. 2b).  m*k outputs of n FMAs each: a few
// hundred thousand flops per scene; latency bound, so each output gets a
// whole warp.
#include "common.cuh"

namespace {

// One warp per code value: lane i sums E[c][i'] s[j][i'] over i' = i, i+32,
// ..., then a butterfly reduction adds the 32 partial sums.
__global__ void __launch_bounds__(256) encode_kernel(const float* __restrict__ E, int k, int n,
                                                     const float* __restrict__ S, int m, void* __restrict__ out,
                                                     int out_dt) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)m * k) return;  // whole warps exit together
  const int j = (int)(w / k), c = (int)(w % k);
  const float* e = E + (int64_t)c * n;
  const float* s = S + (int64_t)j * n;
  float acc = 0.0f;
  for (int i = lane; i < n; i += 32) acc = __fmaf_rn(__ldg(e + i), __ldg(s + i), acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  if (lane == 0) {
    if (out_dt == HSC_F32)
      reinterpret_cast<float*>(out)[w] = acc;
    else if (out_dt == HSC_BF16)
      reinterpret_cast<unsigned short*>(out)[w] = hsc::float_to_bf16_bits(acc);
    else
      reinterpret_cast<unsigned short*>(out)[w] = hsc::float_to_f16_bits(acc);
  }
}

}  // namespace

namespace hsc {
hsc_status launch_encode(const float* E, int k, int n, const float* S, int m, void* out, int out_dt, cudaStream_t s) {
  if (m <= 0) return HSC_OK;
  const int64_t warps = (int64_t)m * k;
  encode_kernel<<<ceil_div_i(warps * 32, 256), 256, 0, s>>>(E, k, n, S, m, out, out_dt);
  return check_launch("encode_kernel");
}
}  // namespace hsc

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
  return hsc::launch_encode(E, k, n, spectra, m, codes_out, (int)out_dt, hsc::as_stream(stream));
}
