// A latent frame straight from spectral assets in one launch: the encode of
// the materials and lights (Eq. 4, z = W_enc s) runs in the prologue of the
// fused shading kernel.  Fig. 2b encodes the assets once per scene; when a
// frame is small (a 256 x 256 G-buffer with a handful of lights shades in a
// few microseconds) the launches of a separate encode cost more than the
// encode itself, so each CTA encodes what it stages into shared memory.  Every
// code value is summed in exactly the order hsc_encode sums it (lane-strided
// partial sums, then a butterfly), so the codes -- and the latent image, XYZ
// and sRGB8 -- are the bits of hsc_encode (FP32 codes) followed by
// hsc_shade_latent (FUSED).
#include "common.cuh"
#include "shade_latent.cuh"
#include "shade_latent_kernel.cuh"

namespace hsc {

hsc_status validate_gbuffer(const hsc_gbuffer* g, const char* name, int64_t pixels);
hsc_status validate_lights(const hsc_lights* l);

namespace {

constexpr int kAssetBlock = 128;
constexpr int kAssetPPT = 2;
static_assert(HSC_ASSETS_MAX_CODES <= kMatStage, "the material table must fit the staged form of shade_tile");
static_assert(HSC_ASSETS_MAX_LIGHTS <= kLightTile, "the lights must fit one staged tile");

struct AssetArgs {
  ShadeArgs a;
  const float* E;     // k x n
  int n;
  const float* mats;  // n_mat x n
  const float* spd;   // L x n
};

// One code value z_c = sum_i E[c][i] s[i] by one thread, summed in the order
// of hsc_encode's warp: partial sum t (t < 32) accumulates the products
// i = t, t + 32, ... with FMAs, then the 32 partials are added as the
// xor-butterfly adds them for lane 0 (halves of 16, 8, 4, 2, 1; floating
// addition is commutative, so the operand order of each pair does not
// matter).  The loads of all products are independent, so a thread waits
// for memory once per code instead of once per shuffle step.
__device__ __forceinline__ float thread_code(const float* __restrict__ e, const float* __restrict__ s, int n) {
  float v[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) v[t] = 0.0f;
  for (int i0 = 0; i0 < n; i0 += 32) {
#pragma unroll
    for (int t = 0; t < 32; ++t)
      if (i0 + t < n) v[t] = __fmaf_rn(__ldg(e + i0 + t), __ldg(s + i0 + t), v[t]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int t = 0; t < o; ++t) v[t] = __fadd_rn(v[t], v[t + o]);
  return v[0];
}

// The same sum with E and the spectrum read from shared memory (the staged
// form): the same operations in the same order, so the same bits.
__device__ __forceinline__ float thread_code_smem(const float* e, const float* s, int n) {
  float v[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) v[t] = 0.0f;
  for (int i0 = 0; i0 < n; i0 += 32) {
#pragma unroll
    for (int t = 0; t < 32; ++t)
      if (i0 + t < n) v[t] = __fmaf_rn(e[i0 + t], s[i0 + t], v[t]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int t = 0; t < o; ++t) v[t] = __fadd_rn(v[t], v[t + o]);
  return v[0];
}

__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// STAGE: E, the light spectra and the material spectra are first copied into
// shared memory with coalesced loads (one pass over a few KB), and the codes
// are summed from there, instead of every code reading its 2 n operands
// from global memory.
template <int KC, bool SEC, bool RGB, bool STAGE>
__global__ void __launch_bounds__(kAssetBlock) shade_assets_kernel(const AssetArgs A) {
  constexpr int F4 = LightStage<KC, 1>::F4;
  // L x F4 staged lights, then n_mat x KC material codes, then (STAGE) E
  // (KC x n), the light spectra (L x n) and the material spectra (n_mat x n)
  extern __shared__ float4 s_light[];
  __shared__ float s_M[3 * KC];
  const ShadeArgs& a = A.a;
  float* sl = reinterpret_cast<float*>(s_light);
  float* s_mat = reinterpret_cast<float*>(s_light + a.L * F4);
  float* s_E = s_mat + a.n_mat * KC;
  float* s_spd = s_E + KC * A.n;
  float* s_mspec = s_spd + a.L * A.n;
  // the tile's G-buffer lines into L1 now, so that the shading's loads after
  // the encode find them there (the encode's own loads run meanwhile)
#pragma unroll
  for (int j = 0; j < kAssetPPT; ++j) {
    const int64_t p = (int64_t)blockIdx.x * (kAssetBlock * kAssetPPT) + (int64_t)j * kAssetBlock + threadIdx.x;
    if (p < a.P) {
      prefetch_l1(a.x1 + 3 * p);
      prefetch_l1(a.n1 + 3 * p);
      prefetch_l1(a.m1 + p);
      if (SEC) {
        prefetch_l1(a.x2 + 3 * p);
        prefetch_l1(a.n2 + 3 * p);
        prefetch_l1(a.m2 + p);
      }
    }
  }
  // light records in the scalar staging layout: position, codes x (I / pi), zeros
  for (int i = threadIdx.x; i < a.L * F4 * 4; i += kAssetBlock) {
    const int l = i / (F4 * 4), j = i - l * (F4 * 4);
    if (j < 3) sl[i] = __ldg(a.lpos + 3 * l + j);
    else if (j >= 3 + KC) sl[i] = 0.0f;
  }
  if constexpr (STAGE) {
    for (int i = threadIdx.x; i < KC * A.n; i += kAssetBlock) s_E[i] = __ldg(A.E + i);
    for (int i = threadIdx.x; i < a.L * A.n; i += kAssetBlock) s_spd[i] = __ldg(A.spd + i);
    for (int i = threadIdx.x; i < a.n_mat * A.n; i += kAssetBlock) s_mspec[i] = __ldg(A.mats + i);
    __syncthreads();
  }
  // one code value per thread: the light codes, then the material codes
  for (int w = threadIdx.x; w < (a.L + a.n_mat) * KC; w += kAssetBlock) {
    const int row = w / KC, c = w - row * KC;
    if (row < a.L) {
      const float z = STAGE ? thread_code_smem(s_E + c * A.n, s_spd + row * A.n, A.n)
                            : thread_code(A.E + (int64_t)c * A.n, A.spd + (int64_t)row * A.n, A.n);
      sl[row * F4 * 4 + 3 + c] = __fmul_rn(z, __fmul_rn(__ldg(a.linten + row), kInvPi));
    } else {
      const int m = row - a.L;
      s_mat[m * KC + c] = STAGE ? thread_code_smem(s_E + c * A.n, s_mspec + m * A.n, A.n)
                                : thread_code(A.E + (int64_t)c * A.n, A.mats + (int64_t)m * A.n, A.n);
    }
  }
  stage_decode_matrix<KC, kAssetBlock>(a, s_M);
  __syncthreads();
  shade_tile<KC, kAssetPPT, SEC, kAssetBlock, 1, RGB>(a, blockIdx.x, s_light, true, s_M, s_mat);
}

constexpr size_t kAssetStageBytes = 48 * 1024;  // shared memory up to which the assets are staged

template <int KC, bool SEC, bool RGB>
hsc_status launch_assets_t(const AssetArgs& A, cudaStream_t s) {
  constexpr int F4 = LightStage<KC, 1>::F4;
  const size_t smem = (size_t)A.a.L * F4 * sizeof(float4) + (size_t)A.a.n_mat * KC * sizeof(float);
  const size_t staged = smem + sizeof(float) * (size_t)A.n * (KC + A.a.L + A.a.n_mat);
  if (staged <= kAssetStageBytes)
    shade_assets_kernel<KC, SEC, RGB, true><<<(unsigned)A.a.tiles, kAssetBlock, staged, s>>>(A);
  else
    shade_assets_kernel<KC, SEC, RGB, false><<<(unsigned)A.a.tiles, kAssetBlock, smem, s>>>(A);
  return check_launch("shade_assets_kernel");
}

template <int KC>
hsc_status launch_assets_kc(const AssetArgs& A, bool sec, bool rgb, cudaStream_t s) {
  if (sec) return rgb ? launch_assets_t<KC, true, true>(A, s) : launch_assets_t<KC, true, false>(A, s);
  return rgb ? launch_assets_t<KC, false, true>(A, s) : launch_assets_t<KC, false, false>(A, s);
}

}  // namespace
}  // namespace hsc

extern "C" hsc_status hsc_shade_latent_assets(hsc_ctx* ctx, const hsc_gbuffer* g1, const hsc_gbuffer* g2,
                                              int64_t pixels, const float* E, int k, int n, const float* mat_spectra,
                                              int n_mat, const hsc_lights* lights, const float* light_spd,
                                              float* latent_out, float* xyz_out, uint8_t* srgb8_out,
                                              const float* M_xyz, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(pixels >= 0, "pixel count %lld negative", (long long)pixels);
  HSC_REQUIRE(k == 3 || k == 6 || k == 9, "k=%d: the one-launch asset path is built for k = 3, 6 and 9", k);
  HSC_REQUIRE(n >= 1 && n <= HSC_MAX_N, "n=%d out of range [1, %d]", n, HSC_MAX_N);
  HSC_REQUIRE(n_mat >= 1 && (int64_t)n_mat * k <= HSC_ASSETS_MAX_CODES,
              "n_mat x k = %lld exceeds the %d code values staged per CTA (encode with hsc_encode instead)",
              (long long)n_mat * k, HSC_ASSETS_MAX_CODES);
  HSC_TRY(hsc::validate_lights(lights));
  HSC_REQUIRE(lights->count <= HSC_ASSETS_MAX_LIGHTS, "%d lights exceed the %d staged per CTA", lights->count,
              HSC_ASSETS_MAX_LIGHTS);
  HSC_TRY(hsc::validate_gbuffer(g1, "g1", pixels));
  if (g2) HSC_TRY(hsc::validate_gbuffer(g2, "g2", pixels));
  HSC_REQUIRE(E && mat_spectra && light_spd, "null asset pointer");
  HSC_REQUIRE(hsc::aligned(E, 4) && hsc::aligned(mat_spectra, 4) && hsc::aligned(light_spd, 4),
              "asset arrays must be 4-byte aligned");
  HSC_REQUIRE(latent_out != nullptr || pixels == 0, "latent_out is null");
  HSC_REQUIRE(!latent_out || hsc::aligned(latent_out, 4), "latent_out must be 4-byte aligned");
  HSC_REQUIRE(!xyz_out || (M_xyz && hsc::aligned(xyz_out, 4) && hsc::aligned(M_xyz, 4)),
              "xyz_out needs M_xyz (both 4-byte aligned)");
  HSC_REQUIRE(!srgb8_out || (M_xyz && hsc::aligned(M_xyz, 4)), "srgb8_out needs M_xyz (4-byte aligned)");
  if (pixels == 0) return HSC_OK;
  HSC_GUARD(ctx);
  hsc::AssetArgs A{};
  hsc::ShadeArgs& a = A.a;
  a.n1 = g1->normal;
  a.x1 = g1->pos;
  a.m1 = g1->mat;
  if (g2) {
    a.n2 = g2->normal;
    a.x2 = g2->pos;
    a.m2 = g2->mat;
  }
  a.P = pixels;
  a.n_mat = n_mat;
  a.lpos = lights->pos;
  a.linten = lights->intensity;
  a.L = lights->count;
  a.code_dt = HSC_F32;
  a.k = k;
  a.c0 = 0;
  a.out = latent_out;
  a.out_stride = k;
  a.out_c0 = 0;
  a.xyz = xyz_out;
  a.srgb8 = srgb8_out;
  a.M = M_xyz;
  a.err = ctx->d_err;
  a.tiles = (pixels + hsc::kAssetBlock * hsc::kAssetPPT - 1) / (hsc::kAssetBlock * hsc::kAssetPPT);
  HSC_REQUIRE(a.tiles <= INT32_MAX, "%lld pixels exceed one launch of the asset path", (long long)pixels);
  A.E = E;
  A.n = n;
  A.mats = mat_spectra;
  A.spd = light_spd;
  cudaStream_t s = hsc::as_stream(stream);
  const bool sec = g2 != nullptr, rgb = srgb8_out != nullptr;
  switch (k) {
    case 3: return hsc::launch_assets_kc<3>(A, sec, rgb, s);
    case 6: return hsc::launch_assets_kc<6>(A, sec, rgb, s);
    default: return hsc::launch_assets_kc<9>(A, sec, rgb, s);
  }
}
