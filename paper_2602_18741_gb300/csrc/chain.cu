// Multi-bounce chains: the codec-selection proxy of Sec. 4.5.  A light L is
// multiplied by a fresh reflectance at every bounce, S(b) = R(b) (.) S(b-1),
// S(0) = L; the latent chain runs the same recurrence on codes with the
// blockwise product (Eq. 6), z(b) = E R(b) (.) z(b-1), z(0) = E L.  Per chain
// and depth both are projected to XYZ (T S(b) and M z(b), M = T D), scaled by
// 1 / max(T L) so that the light's largest tristimulus value is 1, converted
// to CIELAB with the equal-energy white T @ 1, and compared by CIE94
// (spectral chain as reference) and CIEDE2000.
//
// One thread per chain; the spectral chain walks the n samples once, carrying
// the running product and the XYZ sums of every depth, the latent chain walks
// the k channels the same way.  Per-depth mean and nearest-rank p95 follow
// from the generic reduction in metrics.cu.
#include "colour.cuh"
#include "common.cuh"

namespace hsc {

hsc_status launch_encode(const float* E, int k, int n, const float* S, int m, void* out, int out_dt, cudaStream_t s);
hsc_status launch_fold(const float* T, const float* D, int k, int n, float* M, cudaStream_t s);
hsc_status launch_mean_p95(hsc_ctx* ctx, const float* v, int64_t count, double* out, cudaStream_t s);

namespace {

constexpr int kMaxDepth = 8;

struct ChainArgs {
  const float* R;
  const float* L;
  const float* zR;
  const float* zL;
  const float* T;
  const float* M;
  int n, k, nR, nL;
  const int32_t* cl;
  const int32_t* cr;
  int64_t C;
  int depth;
  float* de94;
  float* de00;
  unsigned int* err;
};

__global__ void __launch_bounds__(128) chain_kernel(const ChainArgs a) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.C) return;
  int l = __ldg(a.cl + c);
  bool bad = l < 0 || l >= a.nL;
  int r[kMaxDepth];
#pragma unroll
  for (int b = 0; b < kMaxDepth; ++b) {
    r[b] = 0;
    if (b < a.depth) {
      r[b] = __ldg(a.cr + c * a.depth + b);
      if (r[b] < 0 || r[b] >= a.nR) {
        bad = true;
        r[b] = 0;
      }
    }
  }
  if (bad) {
    atomicOr(a.err, HSC_DEVERR_MATERIAL);
    l = 0;
  }
  // spectral chain; (wx, wy, wz) = T L, (ex, ey, ez) = T @ 1
  float wx = 0.0f, wy = 0.0f, wz = 0.0f, ex = 0.0f, ey = 0.0f, ez = 0.0f;
  float xs[kMaxDepth][3];
#pragma unroll
  for (int b = 0; b < kMaxDepth; ++b) xs[b][0] = xs[b][1] = xs[b][2] = 0.0f;
  for (int i = 0; i < a.n; ++i) {
    float s = __ldg(a.L + (int64_t)l * a.n + i);
    const float t0 = __ldg(a.T + i), t1 = __ldg(a.T + a.n + i), t2 = __ldg(a.T + 2 * a.n + i);
    wx = __fmaf_rn(t0, s, wx);
    wy = __fmaf_rn(t1, s, wy);
    wz = __fmaf_rn(t2, s, wz);
    ex = __fadd_rn(ex, t0);
    ey = __fadd_rn(ey, t1);
    ez = __fadd_rn(ez, t2);
#pragma unroll
    for (int b = 0; b < kMaxDepth; ++b) {
      if (b < a.depth) {
        s = __fmul_rn(__ldg(a.R + (int64_t)r[b] * a.n + i), s);
        xs[b][0] = __fmaf_rn(t0, s, xs[b][0]);
        xs[b][1] = __fmaf_rn(t1, s, xs[b][1]);
        xs[b][2] = __fmaf_rn(t2, s, xs[b][2]);
      }
    }
  }
  // latent chain
  float xl[kMaxDepth][3];
#pragma unroll
  for (int b = 0; b < kMaxDepth; ++b) xl[b][0] = xl[b][1] = xl[b][2] = 0.0f;
  for (int ch = 0; ch < a.k; ++ch) {
    float z = __ldg(a.zL + (int64_t)l * a.k + ch);
    const float m0 = __ldg(a.M + ch), m1 = __ldg(a.M + a.k + ch), m2 = __ldg(a.M + 2 * a.k + ch);
#pragma unroll
    for (int b = 0; b < kMaxDepth; ++b) {
      if (b < a.depth) {
        z = __fmul_rn(__ldg(a.zR + (int64_t)r[b] * a.k + ch), z);
        xl[b][0] = __fmaf_rn(m0, z, xl[b][0]);
        xl[b][1] = __fmaf_rn(m1, z, xl[b][1]);
        xl[b][2] = __fmaf_rn(m2, z, xl[b][2]);
      }
    }
  }
  const float wmax = fmaxf(wx, fmaxf(wy, wz));
  const bool dark = !(wmax > 0.0f);  // a light with no tristimulus response has no colour
  const float inv = dark ? 0.0f : 1.0f / wmax;
#pragma unroll
  for (int b = 0; b < kMaxDepth; ++b) {
    if (b < a.depth) {
      float L1, a1, b1, L2, a2, b2;
      to_lab_white(xs[b][0] * inv, xs[b][1] * inv, xs[b][2] * inv, ex, ey, ez, L1, a1, b1);
      to_lab_white(xl[b][0] * inv, xl[b][1] * inv, xl[b][2] * inv, ex, ey, ez, L2, a2, b2);
      a.de94[(int64_t)b * a.C + c] = (bad || dark) ? 0.0f : de94(L1, a1, b1, L2, a2, b2);
      a.de00[(int64_t)b * a.C + c] = (bad || dark) ? 0.0f : de2000(L1, a1, b1, L2, a2, b2);
    }
  }
}

}  // namespace

}  // namespace hsc

extern "C" hsc_status hsc_chain_eval(hsc_ctx* ctx, const float* refl, int n_refl, const float* lights, int n_lights,
                                     const float* E, const float* D, int k, int n, const float* T,
                                     const int32_t* chain_light, const int32_t* chain_refl, int64_t chains, int depth,
                                     float* de94_out, float* de2000_out, double* stats_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(k >= 1 && k <= HSC_MAX_K, "k=%d out of range", k);
  HSC_REQUIRE(n >= 1 && n <= HSC_MAX_N, "n=%d out of range", n);
  HSC_REQUIRE(n_refl >= 1 && n_lights >= 1, "empty spectral sets");
  HSC_REQUIRE(depth >= 1 && depth <= hsc::kMaxDepth, "depth must be in [1, %d]", hsc::kMaxDepth);
  HSC_REQUIRE(chains >= 1, "need at least one chain");
  HSC_REQUIRE(refl && lights && E && D && T && chain_light && chain_refl && de94_out && de2000_out && stats_out,
              "null pointer");
  HSC_REQUIRE(hsc::aligned(stats_out, 8), "stats_out must be 8-byte aligned");
  HSC_GUARD(ctx);
  cudaStream_t s = hsc::as_stream(stream);
  const size_t code_bytes = ((size_t)n_refl + n_lights) * k * sizeof(float);
  HSC_TRY(hsc::ensure_big(ctx, code_bytes + 3 * (size_t)k * sizeof(float) + 256, s));
  float* zR = reinterpret_cast<float*>(ctx->d_big);
  float* zL = zR + (size_t)n_refl * k;
  float* M = zL + (size_t)n_lights * k;
  HSC_TRY(hsc::launch_encode(E, k, n, refl, n_refl, zR, HSC_F32, s));
  HSC_TRY(hsc::launch_encode(E, k, n, lights, n_lights, zL, HSC_F32, s));
  HSC_TRY(hsc::launch_fold(T, D, k, n, M, s));
  hsc::ChainArgs a{refl, lights, zR, zL, T, M, n, k, n_refl, n_lights, chain_light, chain_refl,
                   chains, depth, de94_out, de2000_out, ctx->d_err};
  hsc::chain_kernel<<<hsc::ceil_div_i(chains, 128), 128, 0, s>>>(a);
  HSC_TRY(hsc::check_launch("chain_kernel"));
  for (int b = 0; b < depth; ++b) {
    HSC_TRY(hsc::launch_mean_p95(ctx, de94_out + (int64_t)b * chains, chains, stats_out + 4 * b, s));
    HSC_TRY(hsc::launch_mean_p95(ctx, de2000_out + (int64_t)b * chains, chains, stats_out + 4 * b + 2, s));
  }
  return HSC_OK;
}
