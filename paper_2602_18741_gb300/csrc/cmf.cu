// CMF integration weights and the decoder fold M = T D.
//
// The paper's colour projection T_cmf (3 x n) holds the CIE colour matching
// functions (colour loss, Sec. 4.3).  Here they are the analytic multi-lobe
// piecewise-Gaussian fit of the CIE 1931 2-degree observer published by
// Wyman, Sloan and Shirley (JCGT 2(2), 2013): each function is a sum of lobes
// a * exp(-((lambda - mu) / sigma)^2 / 2) with sigma taking one value below mu
// and another above.
#include "common.cuh"

namespace {

struct Lobe {
  float a, mu, s_lo, s_hi;
};

// Lobe coefficients of the Wyman-Sloan-Shirley multi-lobe fit.
__constant__ Lobe c_lobes[7] = {
    {1.056f, 599.8f, 37.9f, 31.0f}, {0.362f, 442.0f, 16.0f, 26.7f}, {-0.065f, 501.1f, 20.4f, 26.2f},  // x
    {0.821f, 568.8f, 46.9f, 40.5f}, {0.286f, 530.9f, 16.3f, 31.1f},                                   // y
    {1.217f, 437.0f, 11.8f, 36.0f}, {0.681f, 459.0f, 26.0f, 13.8f}};                                  // z

__device__ float cmf_eval(int c, float lam) {
  const int first = (c == 0) ? 0 : (c == 1 ? 3 : 5);
  const int count = (c == 0) ? 3 : 2;
  float s = 0.0f;
  for (int j = 0; j < count; ++j) {
    const Lobe L = c_lobes[first + j];
    const float sig = (lam < L.mu) ? L.s_lo : L.s_hi;
    const float t = (lam - L.mu) / sig;
    s += L.a * expf(-0.5f * t * t);
  }
  return s;
}

// One block: evaluate x, y, z at every sample (FP32), sum ybar * dlambda in
// FP64 (block reduction), then write T = cmf * dlambda / sum.
__global__ void __launch_bounds__(128) cmf_weights_kernel(int n, float lambda0, float dlambda, float* T) {
  __shared__ double s_part[128];
  const int t = threadIdx.x;
  double acc = 0.0;
  for (int i = t; i < n; i += blockDim.x) {
    const float lam = lambda0 + dlambda * (float)i;
    acc += (double)cmf_eval(1, lam) * (double)dlambda;
  }
  s_part[t] = acc;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (t < w) s_part[t] += s_part[t + w];
    __syncthreads();
  }
  const double ysum = s_part[0];
  for (int i = t; i < n; i += blockDim.x) {
    const float lam = lambda0 + dlambda * (float)i;
    for (int c = 0; c < 3; ++c) T[c * n + i] = (float)((double)cmf_eval(c, lam) * (double)dlambda / ysum);
  }
}

// M[c][j] = sum_i T[c][i] D[i][j], FP32 in order of i.
__global__ void fold_kernel(const float* __restrict__ T, const float* __restrict__ D, int k, int n,
                            float* __restrict__ M) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 3 * k) return;
  const int c = idx / k, j = idx % k;
  float s = 0.0f;
  for (int i = 0; i < n; ++i) s = __fmaf_rn(T[c * n + i], D[i * k + j], s);
  M[idx] = s;
}

}  // namespace

namespace hsc {
hsc_status launch_fold(const float* T, const float* D, int k, int n, float* M, cudaStream_t s) {
  fold_kernel<<<ceil_div_i(3 * k, 128), 128, 0, s>>>(T, D, k, n, M);
  return check_launch("fold_kernel");
}
}  // namespace hsc

extern "C" {

hsc_status hsc_cmf_weights(hsc_ctx* ctx, int n, float lambda0, float dlambda, float* T_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(n >= 1 && n <= HSC_MAX_N, "n=%d out of range [1, %d]", n, HSC_MAX_N);
  HSC_REQUIRE(dlambda > 0.0f && lambda0 > 0.0f, "grid must be positive (lambda0=%g, dlambda=%g)", lambda0, dlambda);
  HSC_REQUIRE(T_out && hsc::aligned(T_out, 4), "T_out is null or misaligned");
  HSC_GUARD(ctx);
  cmf_weights_kernel<<<1, 128, 0, hsc::as_stream(stream)>>>(n, lambda0, dlambda, T_out);
  return hsc::check_launch("cmf_weights_kernel");
}

hsc_status hsc_fold_xyz(hsc_ctx* ctx, const float* T, const float* D, int k, int n, float* M_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(n >= 1 && n <= HSC_MAX_N, "n=%d out of range", n);
  HSC_REQUIRE(k >= 1 && k <= HSC_MAX_K, "k=%d out of range", k);
  HSC_REQUIRE(T && D && M_out, "null pointer");
  HSC_GUARD(ctx);
  return hsc::launch_fold(T, D, k, n, M_out, hsc::as_stream(stream));
}

}  // extern "C"
