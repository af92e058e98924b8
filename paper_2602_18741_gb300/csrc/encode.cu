// Asset encoding z = W_enc s (Eq. 4), done once per scene for every material
// reflectance and light SPD (Fig. 2b).  m*k outputs of n FMAs each: a few
// hundred thousand flops per scene; latency bound, so each output gets a
// whole warp.  hsc_encode_assets encodes the materials and the lights in one
// launch: a per-frame encode (a changing scene) then pays one launch, not two.
#include "common.cuh"

namespace {

// Lane `lane`'s partial sum of E[c][i] s[i] over i = lane, lane + 32, ...:
// the loads of up to four products are issued before their FMAs, which
// then run in that same order of i.
__device__ __forceinline__ float lane_partial(const float* __restrict__ e, const float* __restrict__ s, int n,
                                              int lane) {
  float acc = 0.0f;
  for (int i0 = lane; i0 < n; i0 += 128) {
    float ev[4], sv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int i = min(i0 + 32 * t, n - 1);
      ev[t] = __ldg(e + i);
      sv[t] = __ldg(s + i);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (i0 + 32 * t < n) acc = __fmaf_rn(ev[t], sv[t], acc);
  }
  return acc;
}

// One set of spectra to encode: m rows of n samples into m x k codes.
struct EncodeSet {
  const float* S;
  int m;
  void* out;
};

// One warp per code value: lane partial sums, then a butterfly adds the 32
// partials.  The warps of set 0 come first, then those of set 1, so one
// launch encodes both.
__global__ void __launch_bounds__(256) encode_kernel(const float* __restrict__ E, int k, int n, EncodeSet s0,
                                                     EncodeSet s1, int out_dt) {
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  EncodeSet set = s0;
  if (w >= (int64_t)s0.m * k) {
    w -= (int64_t)s0.m * k;
    set = s1;
  }
  if (w >= (int64_t)set.m * k) return;  // whole warps exit together
  const int j = (int)(w / k), c = (int)(w % k);
  float acc = lane_partial(E + (int64_t)c * n, set.S + (int64_t)j * n, n, lane);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  if (lane == 0) {
    if (out_dt == HSC_F32)
      reinterpret_cast<float*>(set.out)[w] = acc;
    else if (out_dt == HSC_BF16)
      reinterpret_cast<unsigned short*>(set.out)[w] = hsc::float_to_bf16_bits(acc);
    else
      reinterpret_cast<unsigned short*>(set.out)[w] = hsc::float_to_f16_bits(acc);
  }
}

hsc_status launch_encode_sets(const float* E, int k, int n, EncodeSet s0, EncodeSet s1, int out_dt, cudaStream_t s) {
  const int64_t warps = ((int64_t)s0.m + s1.m) * k;
  if (warps <= 0) return HSC_OK;
  encode_kernel<<<hsc::ceil_div_i(warps * 32, 256), 256, 0, s>>>(E, k, n, s0, s1, out_dt);
  return hsc::check_launch("encode_kernel");
}

}  // namespace

namespace hsc {
hsc_status launch_encode(const float* E, int k, int n, const float* S, int m, void* out, int out_dt, cudaStream_t s) {
  if (m <= 0) return HSC_OK;
  return launch_encode_sets(E, k, n, EncodeSet{S, m, out}, EncodeSet{nullptr, 0, nullptr}, out_dt, s);
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

extern "C" hsc_status hsc_encode_assets(hsc_ctx* ctx, const float* E, int k, int n, const float* mat_spectra,
                                        int n_mat, void* mat_codes_out, const float* light_spd, int n_lights,
                                        void* light_codes_out, hsc_dtype out_dt, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(k >= 1 && k <= HSC_MAX_K, "k=%d out of range [1, %d]", k, HSC_MAX_K);
  HSC_REQUIRE(n >= 1 && n <= HSC_MAX_N, "n=%d out of range [1, %d]", n, HSC_MAX_N);
  HSC_REQUIRE(n_mat >= 0 && n_lights >= 0, "negative asset count (n_mat=%d, n_lights=%d)", n_mat, n_lights);
  HSC_REQUIRE(out_dt == HSC_F32 || out_dt == HSC_BF16 || out_dt == HSC_F16, "codes dtype must be F32, BF16 or F16");
  if (n_mat == 0 && n_lights == 0) return HSC_OK;
  const int oa = out_dt == HSC_F32 ? 4 : 2;
  HSC_REQUIRE(E && hsc::aligned(E, 4), "E null or misaligned");
  HSC_REQUIRE(n_mat == 0 || (mat_spectra && mat_codes_out && hsc::aligned(mat_spectra, 4) &&
                             hsc::aligned(mat_codes_out, oa)),
              "material spectra or codes null or misaligned");
  HSC_REQUIRE(n_lights == 0 || (light_spd && light_codes_out && hsc::aligned(light_spd, 4) &&
                                hsc::aligned(light_codes_out, oa)),
              "light spectra or codes null or misaligned");
  HSC_GUARD(ctx);
  return launch_encode_sets(E, k, n, EncodeSet{mat_spectra, n_mat, mat_codes_out},
                            EncodeSet{light_spd, n_lights, light_codes_out}, (int)out_dt, hsc::as_stream(stream));
}
