// FP32 issue-rate probe: the measured ceiling beside the nominal ALU peak
// (SMs x 128 FP32 lanes x SM clock) that the shading kernels are compared
// against.  Each thread runs kProbeChains independent FMA recurrences
// a <- a * m + s, so the loop is pure FFMA with enough independent work per
// warp to cover the pipe latency; the result is written so the loop is live.
#include "common.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 4;   // FMAs per chain per iteration

__global__ void __launch_bounds__(kProbeThreads) fp32_probe_kernel(int iters, float m, float s, float* sink) {
  float a[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) a[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) a[c] = fmaf(a[c], m, s);
    }
  }
  float t = 0.0f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) t += a[c];
  sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = t;
}

// MUFU tanh rate probe: the SiLU epilogue of the upsampling network is one
// hardware tanh per hidden value, so its throughput bound is the MUFU rate.
// Each thread runs kProbeChains independent recurrences a <- tanh(a + s), in
// FP32 (tanh.approx.f32) or on packed f16 pairs (tanh.approx.f16x2, two
// results per operation).
template <bool PACKED>
__global__ void __launch_bounds__(kProbeThreads) tanh_probe_kernel(int iters, float s, float* sink) {
  if constexpr (PACKED) {
    __half2 a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c)
      a[c] = __floats2half2_rn(threadIdx.x * 1e-3f + c * 0.1f, threadIdx.x * 1e-3f + c * 0.1f + 0.05f);
    const __half2 s2 = __float2half2_rn(s);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
          const __half2 x = __hadd2(a[c], s2);
          uint32_t y;
          asm("tanh.approx.f16x2 %0, %1;" : "=r"(y) : "r"(*reinterpret_cast<const uint32_t*>(&x)));
          a[c] = *reinterpret_cast<const __half2*>(&y);
        }
      }
    }
    float t = 0.0f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) t += __low2float(a[c]) + __high2float(a[c]);
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = t;
  } else {
    float a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = threadIdx.x * 1e-3f + c * 0.1f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
          float y;
          asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(a[c] + s));
          a[c] = y;
        }
      }
    }
    float t = 0.0f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) t += a[c];
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = t;
  }
}

}  // namespace

extern "C" {

hsc_status hsc_fp32_peak_probe(hsc_ctx* ctx, int ctas, int iters, float* sink, int64_t* lane_ops_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  if (ctas <= 0) ctas = 8 * ctx->sm_count;
  HSC_REQUIRE(ctas <= (1 << 20), "ctas=%d too large", ctas);
  HSC_REQUIRE(iters >= 1 && iters <= (1 << 24), "iters=%d out of range [1, 2^24]", iters);
  HSC_REQUIRE(sink && hsc::aligned(sink, 4), "sink is null or misaligned");
  HSC_GUARD(ctx);
  if (lane_ops_out)
    *lane_ops_out = (int64_t)ctas * kProbeThreads * iters * (kProbeChains * kProbeUnroll);
  fp32_probe_kernel<<<ctas, kProbeThreads, 0, hsc::as_stream(stream)>>>(iters, 0.999f, 1e-3f, sink);
  return hsc::check_launch("fp32_probe_kernel");
}

hsc_status hsc_tanh_peak_probe(hsc_ctx* ctx, int ctas, int iters, int packed, float* sink, int64_t* tanh_ops_out,
                               void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  if (ctas <= 0) ctas = 8 * ctx->sm_count;
  HSC_REQUIRE(ctas <= (1 << 20), "ctas=%d too large", ctas);
  HSC_REQUIRE(iters >= 1 && iters <= (1 << 24), "iters=%d out of range [1, 2^24]", iters);
  HSC_REQUIRE(sink && hsc::aligned(sink, 4), "sink is null or misaligned");
  HSC_GUARD(ctx);
  HSC_REQUIRE(packed == 0 || packed == 1, "packed=%d must be 0 (FP32) or 1 (f16x2)", packed);
  if (tanh_ops_out)
    *tanh_ops_out = (int64_t)ctas * kProbeThreads * iters * (kProbeChains * kProbeUnroll) * (packed ? 2 : 1);
  if (packed)
    tanh_probe_kernel<true><<<ctas, kProbeThreads, 0, hsc::as_stream(stream)>>>(iters, 0.25f, sink);
  else
    tanh_probe_kernel<false><<<ctas, kProbeThreads, 0, hsc::as_stream(stream)>>>(iters, 0.25f, sink);
  return hsc::check_launch("tanh_probe_kernel");
}

}  // extern "C"
