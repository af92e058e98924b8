// Colour-difference statistics of a test image against a reference image:
// mean / nearest-rank p95 of CIEDE2000, means of CIE94 and Delta E 76.
// The paper compares colours with CIE94 (codec selection, Sec. 4.5) and
// Delta E 76 after the CIELAB transform (upsampler loss, Sec. 5.2).
//
// Pipeline, all on the caller's stream, no host round trip:
//   1. max_p Y of the reference (unsigned max over float bits; Y >= 0).
//   2. per pixel: both XYZ / Y_ref -> CIELAB (white = T @ 1) -> dE00, dE94,
//      dE76; per-CTA FP64 partial sums written to scratch.
//   3. one CTA folds the partials into the stats.
//   4. p95 by exact radix select on the float bits of dE00 (non-negative):
//      three passes over 11 / 11 / 10-bit digits, each a histogram kernel and a
//      one-CTA scan that narrows the prefix and the rank.
#include "common.cuh"
#include "colour.cuh"

namespace hsc {

namespace {

constexpr int kMBlock = 256;

struct Scratch {
  unsigned int ymax_bits;
  unsigned int prefix;       // radix-select prefix (bits found so far)
  unsigned long long rank;   // rank still to find inside the current prefix
  float white[3];
  unsigned int pad;
  unsigned int hist[2048];
  double partial[1];         // [grid][4]
};

__global__ void ymax_kernel(const float* __restrict__ ref, int64_t P, const float* __restrict__ T, int n,
                            Scratch* sc) {
  __shared__ unsigned int s_m;
  if (threadIdx.x == 0) s_m = 0u;
  __syncthreads();
  unsigned int m = 0u;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fmaxf(__ldg(ref + 3 * p + 1), 0.0f)));
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(&s_m, m);
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&sc->ymax_bits, s_m);
  if (blockIdx.x == 0 && threadIdx.x < 3) {
    double w = 0.0;
    for (int i = 0; i < n; ++i) w += (double)T[threadIdx.x * n + i];
    sc->white[threadIdx.x] = (float)w;
  }
}

__global__ void __launch_bounds__(kMBlock) de_kernel(const float* __restrict__ test, const float* __restrict__ ref,
                                                     int64_t P, Scratch* sc, float* __restrict__ de_out) {
  __shared__ double s_red[kMBlock / 32][4];
  float yr = __uint_as_float(sc->ymax_bits);
  const float inv = (yr > 0.0f) ? 1.0f / yr : 1.0f;
  const float w[3] = {sc->white[0], sc->white[1], sc->white[2]};
  double s00 = 0.0, s94 = 0.0, s76 = 0.0, mx = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    float L1, a1, b1, L2, a2, b2;
    to_lab(__ldg(ref + 3 * p) * inv, __ldg(ref + 3 * p + 1) * inv, __ldg(ref + 3 * p + 2) * inv, w, L1, a1, b1);
    to_lab(__ldg(test + 3 * p) * inv, __ldg(test + 3 * p + 1) * inv, __ldg(test + 3 * p + 2) * inv, w, L2, a2, b2);
    const float d00 = de2000(L1, a1, b1, L2, a2, b2);
    const float d94 = de94(L1, a1, b1, L2, a2, b2);
    const float d76 = sqrtf((L1 - L2) * (L1 - L2) + (a1 - a2) * (a1 - a2) + (b1 - b2) * (b1 - b2));
    de_out[p] = d00;
    s00 += d00;
    s94 += d94;
    s76 += d76;
    mx = fmax(mx, (double)d00);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s00 += __shfl_xor_sync(0xffffffffu, s00, o);
    s94 += __shfl_xor_sync(0xffffffffu, s94, o);
    s76 += __shfl_xor_sync(0xffffffffu, s76, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_red[wid][0] = s00;
    s_red[wid][1] = s94;
    s_red[wid][2] = s76;
    s_red[wid][3] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int i = 0; i < kMBlock / 32; ++i) {
      t[0] += s_red[i][0];
      t[1] += s_red[i][1];
      t[2] += s_red[i][2];
      t[3] = fmax(t[3], s_red[i][3]);
    }
    for (int j = 0; j < 4; ++j) sc->partial[4 * blockIdx.x + j] = t[j];
  }
}

// One CTA of 256 threads: fold the per-CTA partials (thread t takes partials
// t, t+256, ..., then a fixed-shape tree), so the result is deterministic, and
// set up the radix select for rank ceil(0.95 P) - 1.
__global__ void __launch_bounds__(256) fold_kernel(Scratch* sc, int nblocks, int64_t P, double* stats) {
  __shared__ double s_r[4][256];
  const int t = threadIdx.x;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  for (int i = t; i < nblocks; i += 256) {
    a0 += sc->partial[4 * i];
    a1 += sc->partial[4 * i + 1];
    a2 += sc->partial[4 * i + 2];
    a3 = fmax(a3, sc->partial[4 * i + 3]);
  }
  s_r[0][t] = a0;
  s_r[1][t] = a1;
  s_r[2][t] = a2;
  s_r[3][t] = a3;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) {
      s_r[0][t] += s_r[0][t + w];
      s_r[1][t] += s_r[1][t + w];
      s_r[2][t] += s_r[2][t + w];
      s_r[3][t] = fmax(s_r[3][t], s_r[3][t + w]);
    }
    __syncthreads();
  }
  if (t == 0) {
    const double inv = P > 0 ? 1.0 / (double)P : 0.0;
    stats[0] = s_r[0][0] * inv;
    stats[2] = s_r[1][0] * inv;
    stats[3] = s_r[2][0] * inv;
    stats[4] = (double)__uint_as_float(sc->ymax_bits);
    stats[5] = s_r[3][0];
    stats[6] = (double)P;
    stats[7] = 0.0;
    long long r = (long long)ceil(0.95 * (double)P) - 1;
    sc->rank = (unsigned long long)(r < 0 ? 0 : r);
    sc->prefix = 0u;
  }
}

// Histogram of the digit (bits [shift, shift+width)) of every value whose
// higher bits equal the prefix found so far.
__global__ void __launch_bounds__(kMBlock) radix_hist_kernel(const float* __restrict__ v, int64_t P, Scratch* sc,
                                                             int shift, int width) {
  __shared__ unsigned int s_h[2048];
  const int bins = 1 << width;
  for (int i = threadIdx.x; i < bins; i += blockDim.x) s_h[i] = 0u;
  __syncthreads();
  const unsigned int prefix = sc->prefix;
  const int hi = shift + width;
  const unsigned int hmask = (hi >= 32) ? 0u : (0xffffffffu << hi);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned int u = __float_as_uint(fmaxf(__ldg(v + p), 0.0f));
    if ((u & hmask) == (prefix & hmask)) atomicAdd(&s_h[(u >> shift) & (bins - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < bins; i += blockDim.x)
    if (s_h[i]) atomicAdd(&sc->hist[i], s_h[i]);
}

// One CTA of 1024 threads: exclusive prefix sum over the (up to 2048) bins,
// the bin whose range holds the rank extends the prefix and reduces the rank;
// the histogram is cleared for the next pass.
__global__ void __launch_bounds__(1024) radix_select_kernel(Scratch* sc, int shift, int width, double* stats) {
  __shared__ unsigned long long s_warp[32];
  __shared__ int s_sel;
  __shared__ unsigned long long s_before;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int bins = 1 << width;
  const unsigned long long r = sc->rank;
  // thread t owns bins 2t and 2t+1
  const unsigned long long c0 = (2 * t < bins) ? sc->hist[2 * t] : 0ull;
  const unsigned long long c1 = (2 * t + 1 < bins) ? sc->hist[2 * t + 1] : 0ull;
  unsigned long long incl = c0 + c1;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[wid] = incl;
  if (t == 0) {
    s_sel = bins - 1;
    s_before = 0ull;
  }
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = s_warp[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const unsigned long long before = incl - (c0 + c1) + (wid > 0 ? s_warp[wid - 1] : 0ull);
  if (before <= r && r < before + c0) {
    s_sel = 2 * t;
    s_before = before;
  } else if (before + c0 <= r && r < before + c0 + c1) {
    s_sel = 2 * t + 1;
    s_before = before + c0;
  }
  __syncthreads();
  if (2 * t < bins) sc->hist[2 * t] = 0u;
  if (2 * t + 1 < bins) sc->hist[2 * t + 1] = 0u;
  if (t == 0) {
    sc->rank = r - s_before;
    sc->prefix |= ((unsigned int)s_sel) << shift;
    if (shift == 0) stats[1] = (double)__uint_as_float(sc->prefix);
  }
}

// Per-CTA FP64 sums of v[0..count) for the generic mean.
__global__ void __launch_bounds__(kMBlock) sum_kernel(const float* __restrict__ v, int64_t count, Scratch* sc) {
  __shared__ double s_red[kMBlock / 32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)__ldg(v + i);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kMBlock / 32; ++i) t += s_red[i];
    sc->partial[4 * blockIdx.x] = t;
  }
}

// Mean from the partial sums (fixed order) and the rank for the p95 select.
__global__ void __launch_bounds__(256) mean_fold_kernel(Scratch* sc, int nblocks, int64_t count, double* out) {
  __shared__ double s_r[256];
  const int t = threadIdx.x;
  double a0 = 0.0;
  for (int i = t; i < nblocks; i += 256) a0 += sc->partial[4 * i];
  s_r[t] = a0;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) s_r[t] += s_r[t + w];
    __syncthreads();
  }
  if (t == 0) {
    out[0] = count > 0 ? s_r[0] / (double)count : 0.0;
    long long r = (long long)ceil(0.95 * (double)count) - 1;
    sc->rank = (unsigned long long)(r < 0 ? 0 : r);
    sc->prefix = 0u;
  }
}

int stats_grid(const hsc_ctx* ctx, int64_t count) {
  int grid = ctx->sm_count * 4;
  const int64_t need = (count + kMBlock - 1) / kMBlock;
  if (grid > need) grid = (int)need;
  return grid < 1 ? 1 : grid;
}

hsc_status radix_p95(hsc_ctx* ctx, const float* v, int64_t count, Scratch* sc, int grid, double* stats,
                     cudaStream_t s) {
  const int shifts[3] = {21, 10, 0};
  const int widths[3] = {11, 11, 10};
  for (int i = 0; i < 3; ++i) {
    radix_hist_kernel<<<grid, kMBlock, 0, s>>>(v, count, sc, shifts[i], widths[i]);
    HSC_TRY(check_launch("radix_hist_kernel"));
    radix_select_kernel<<<1, 1024, 0, s>>>(sc, shifts[i], widths[i], stats);
    HSC_TRY(check_launch("radix_select_kernel"));
  }
  return HSC_OK;
}

}  // namespace

// Mean and nearest-rank p95 of count non-negative floats: out[0] = mean,
// out[1] = p95 (device doubles).  Uses the context's reduction scratch.
hsc_status launch_mean_p95(hsc_ctx* ctx, const float* v, int64_t count, double* out, cudaStream_t s) {
  auto* sc = reinterpret_cast<Scratch*>(ctx->d_small + HSC_OFF_REDUCE);
  const int grid = stats_grid(ctx, count);
  HSC_CUDA(cudaMemsetAsync(sc, 0, sizeof(Scratch), s));
  sum_kernel<<<grid, kMBlock, 0, s>>>(v, count, sc);
  HSC_TRY(check_launch("sum_kernel"));
  mean_fold_kernel<<<1, 256, 0, s>>>(sc, grid, count, out);
  HSC_TRY(check_launch("mean_fold_kernel"));
  return radix_p95(ctx, v, count, sc, grid, out, s);
}

}  // namespace hsc

extern "C" hsc_status hsc_delta_e(hsc_ctx* ctx, const float* xyz_test, const float* xyz_ref, int64_t pixels,
                                  const float* T, int n, float* de_out, double* stats_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(pixels >= 1, "need at least one pixel");
  HSC_REQUIRE(n >= 1 && n <= HSC_MAX_N, "n=%d out of range", n);
  HSC_REQUIRE(xyz_test && xyz_ref && T && stats_out, "null pointer");
  HSC_REQUIRE(hsc::aligned(xyz_test, 4) && hsc::aligned(xyz_ref, 4) && hsc::aligned(T, 4) &&
                  hsc::aligned(stats_out, 8) && (!de_out || hsc::aligned(de_out, 4)),
              "misaligned pointer");
  HSC_GUARD(ctx);
  cudaStream_t s = hsc::as_stream(stream);
  float* de = de_out;
  if (!de) {
    HSC_TRY(hsc::ensure_big(ctx, (size_t)pixels * sizeof(float), s));
    de = reinterpret_cast<float*>(ctx->d_big);
  }
  const int grid = hsc::stats_grid(ctx, pixels);
  auto* sc = reinterpret_cast<hsc::Scratch*>(ctx->d_small + HSC_OFF_REDUCE);
  HSC_CUDA(cudaMemsetAsync(sc, 0, sizeof(hsc::Scratch), s));
  hsc::ymax_kernel<<<grid, hsc::kMBlock, 0, s>>>(xyz_ref, pixels, T, n, sc);
  HSC_TRY(hsc::check_launch("ymax_kernel"));
  hsc::de_kernel<<<grid, hsc::kMBlock, 0, s>>>(xyz_test, xyz_ref, pixels, sc, de);
  HSC_TRY(hsc::check_launch("de_kernel"));
  hsc::fold_kernel<<<1, 256, 0, s>>>(sc, grid, pixels, stats_out);
  HSC_TRY(hsc::check_launch("fold_kernel"));
  return hsc::radix_p95(ctx, de, pixels, sc, grid, stats_out, s);
}
