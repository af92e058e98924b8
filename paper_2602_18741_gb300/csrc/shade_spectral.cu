// Naive n-sample spectral shading: the paper's ground truth, whose cost grows
// in proportion to the number of wavelength samples (Sec. 1).  Same shading
// model and the same geometry_term instruction sequence as the latent
// kernels; per (pixel, light) it does the geometry term plus n FMAs instead
// of k.
//
// Mapping: one thread per pixel holds NCH >= n FP32 accumulators.  Lights and
// their (I/pi)-scaled SPDs are staged in shared memory and read as broadcast
// float4s.  With a secondary G-buffer the thread first sums the light at the
// secondary point, turns it into h * (R2 (.) A2), then adds the direct light
// of the primary point on top and multiplies by R1; XYZ = T S is fused.
#include "common.cuh"
#include "shade_latent.cuh"

namespace hsc {

namespace {

constexpr int kSpecBlock = 128;
constexpr int kSpecLightTile = 64;

struct SpecArgs {
  const float* n1;
  const float* x1;
  const int32_t* m1;
  const float* n2;
  const float* x2;
  const int32_t* m2;
  int64_t P;
  const float* mats;  // n_mat x n
  int n_mat;
  const float* lpos;
  const float* linten;
  const float* spd;  // L x n
  int L;
  int n;
  const float* T;  // 3 x n
  float* xyz;
  float* spectra;  // nullable, P x n
  unsigned int* err;
};

template <int NCH>
struct SpecLayout {
  static constexpr int V4 = (NCH + 3) / 4;  // float4s of spectrum per light
  static constexpr int F4 = 1 + V4;         // + one float4 for the position
};

template <int NCH>
__device__ __forceinline__ void stage_lights(const SpecArgs& a, float4* s_light, int l0, int nl) {
  constexpr int F4 = SpecLayout<NCH>::F4;
  float* s = reinterpret_cast<float*>(s_light);
  constexpr int per = F4 * 4;
  for (int idx = threadIdx.x; idx < nl * per; idx += blockDim.x) {
    const int l = idx / per, j = idx - l * per;
    const int lg = l0 + l;
    float v = 0.0f;
    if (j < 3) {
      v = __ldg(a.lpos + 3 * lg + j);
    } else if (j >= 4 && j - 4 < a.n) {
      const float sc = __fmul_rn(__ldg(a.linten + lg), kInvPi);
      v = __fmul_rn(__ldg(a.spd + (int64_t)lg * a.n + (j - 4)), sc);
    }
    s[idx] = v;
  }
}

template <int NCH>
__device__ __forceinline__ void sweep(const float4* s_light, int nl, float x, float y, float z, float nx, float ny,
                                      float nz, float (&acc)[NCH]) {
  constexpr int F4 = SpecLayout<NCH>::F4;
  constexpr int V4 = SpecLayout<NCH>::V4;
#pragma unroll 1
  for (int l = 0; l < nl; ++l) {
    const float4 pl = s_light[l * F4];
    const float g = geometry_term(x, y, z, nx, ny, nz, pl.x, pl.y, pl.z);
#pragma unroll
    for (int f = 0; f < V4; ++f) {
      const float4 v = s_light[l * F4 + 1 + f];
      if (4 * f + 0 < NCH) acc[4 * f + 0] = __fmaf_rn(g, v.x, acc[4 * f + 0]);
      if (4 * f + 1 < NCH) acc[4 * f + 1] = __fmaf_rn(g, v.y, acc[4 * f + 1]);
      if (4 * f + 2 < NCH) acc[4 * f + 2] = __fmaf_rn(g, v.z, acc[4 * f + 2]);
      if (4 * f + 3 < NCH) acc[4 * f + 3] = __fmaf_rn(g, v.w, acc[4 * f + 3]);
    }
  }
}

template <int NCH, bool SEC>
__global__ void __launch_bounds__(kSpecBlock) shade_spectral_kernel(const SpecArgs a) {
  extern __shared__ float4 s_light[];
  const bool multi_tile = a.L > kSpecLightTile;
  if (!multi_tile) {
    stage_lights<NCH>(a, s_light, 0, a.L);
    __syncthreads();
  }
  const int64_t tiles = (a.P + kSpecBlock - 1) / kSpecBlock;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t p = tile * kSpecBlock + threadIdx.x;
    const bool valid = p < a.P;
    const int64_t pc = valid ? p : a.P - 1;
    const float x1 = __ldg(a.x1 + 3 * pc), y1 = __ldg(a.x1 + 3 * pc + 1), z1 = __ldg(a.x1 + 3 * pc + 2);
    const float nx1 = __ldg(a.n1 + 3 * pc), ny1 = __ldg(a.n1 + 3 * pc + 1), nz1 = __ldg(a.n1 + 3 * pc + 2);
    const int m1 = __ldg(a.m1 + pc);
    bool bad = (m1 < 0 || m1 >= a.n_mat);
    float acc[NCH];
#pragma unroll
    for (int i = 0; i < NCH; ++i) acc[i] = 0.0f;

    if (SEC) {
      const float x2 = __ldg(a.x2 + 3 * pc), y2 = __ldg(a.x2 + 3 * pc + 1), z2 = __ldg(a.x2 + 3 * pc + 2);
      const float nx2 = __ldg(a.n2 + 3 * pc), ny2 = __ldg(a.n2 + 3 * pc + 1), nz2 = __ldg(a.n2 + 3 * pc + 2);
      const int m2 = __ldg(a.m2 + pc);
      const bool bad2 = (m2 < 0 || m2 >= a.n_mat);
      bad = bad || bad2;
      for (int l0 = 0; l0 < a.L; l0 += kSpecLightTile) {
        const int nl = min(kSpecLightTile, a.L - l0);
        if (multi_tile) {
          __syncthreads();
          stage_lights<NCH>(a, s_light, l0, nl);
          __syncthreads();
        }
        sweep<NCH>(s_light + 0, nl, x2, y2, z2, nx2, ny2, nz2, acc);
      }
      const float h = bounce_term(x1, y1, z1, nx1, ny1, nz1, x2, y2, z2, nx2, ny2, nz2);
      const float* r2 = a.mats + (int64_t)(bad2 ? 0 : m2) * a.n;
#pragma unroll
      for (int i = 0; i < NCH; ++i) {
        const float r = (i < a.n && !bad2) ? __ldg(r2 + i) : 0.0f;
        acc[i] = __fmul_rn(h, __fmul_rn(r, acc[i]));
      }
    }
    for (int l0 = 0; l0 < a.L; l0 += kSpecLightTile) {
      const int nl = min(kSpecLightTile, a.L - l0);
      if (multi_tile) {
        __syncthreads();
        stage_lights<NCH>(a, s_light, l0, nl);
        __syncthreads();
      }
      sweep<NCH>(s_light, nl, x1, y1, z1, nx1, ny1, nz1, acc);
    }
    const float* r1 = a.mats + (int64_t)(bad ? 0 : m1) * a.n;
    float X = 0.0f, Y = 0.0f, Z = 0.0f;
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
      if (i < a.n) {
        const float S = bad ? 0.0f : __fmul_rn(__ldg(r1 + i), acc[i]);
        X = __fmaf_rn(__ldg(a.T + i), S, X);
        Y = __fmaf_rn(__ldg(a.T + a.n + i), S, Y);
        Z = __fmaf_rn(__ldg(a.T + 2 * a.n + i), S, Z);
        if (a.spectra && valid) a.spectra[p * a.n + i] = S;
      }
    }
    if (valid) {
      a.xyz[3 * p] = X;
      a.xyz[3 * p + 1] = Y;
      a.xyz[3 * p + 2] = Z;
      if (bad) atomicOr(a.err, HSC_DEVERR_MATERIAL);
    }
  }
}

template <int NCH, bool SEC>
hsc_status launch_spec(const SpecArgs& a, int sm_count, cudaStream_t s) {
  constexpr int F4 = SpecLayout<NCH>::F4;
  auto kern = shade_spectral_kernel<NCH, SEC>;
  const size_t smem_max = (size_t)kSpecLightTile * F4 * sizeof(float4);
  const size_t smem = (size_t)min(a.L, kSpecLightTile) * F4 * sizeof(float4);
  static int occ = -1;
  if (occ < 0) {
    if (smem_max > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kSpecBlock, smem_max) != cudaSuccess) o = 1;
    occ = o > 0 ? o : 1;
  }
  const int64_t tiles = (a.P + kSpecBlock - 1) / kSpecBlock;
  int64_t grid = (int64_t)sm_count * occ;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kSpecBlock, smem, s>>>(a);
  return check_launch("shade_spectral_kernel");
}

template <int NCH>
hsc_status launch_spec_sec(const SpecArgs& a, bool sec, int sm_count, cudaStream_t s) {
  return sec ? launch_spec<NCH, true>(a, sm_count, s) : launch_spec<NCH, false>(a, sm_count, s);
}

}  // namespace

hsc_status validate_gbuffer(const hsc_gbuffer* g, const char* name, int64_t pixels);
hsc_status validate_lights(const hsc_lights* l);

}  // namespace hsc

extern "C" hsc_status hsc_shade_spectral(hsc_ctx* ctx, const hsc_gbuffer* g1, const hsc_gbuffer* g2, int64_t pixels,
                                         const float* mat_spectra, int n_mat, const hsc_lights* lights,
                                         const float* light_spd, int n, const float* T, float* xyz_out,
                                         float* spectra_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(pixels >= 0, "negative pixel count");
  HSC_REQUIRE(n >= 1 && n <= HSC_MAX_N, "n=%d out of range [1, %d]", n, HSC_MAX_N);
  HSC_REQUIRE(n_mat >= 1 && n_mat <= HSC_MAX_MAT, "n_mat=%d out of range", n_mat);
  HSC_REQUIRE(mat_spectra && light_spd && T && (xyz_out || pixels == 0), "null pointer");
  HSC_REQUIRE(hsc::aligned(mat_spectra, 4) && hsc::aligned(light_spd, 4) && hsc::aligned(T, 4) &&
                  hsc::aligned(xyz_out, 4) && (!spectra_out || hsc::aligned(spectra_out, 4)),
              "misaligned pointer");
  HSC_TRY(hsc::validate_gbuffer(g1, "g1", pixels));
  if (g2) HSC_TRY(hsc::validate_gbuffer(g2, "g2", pixels));
  HSC_TRY(hsc::validate_lights(lights));
  if (pixels == 0) return HSC_OK;
  HSC_GUARD(ctx);
  hsc::SpecArgs a{};
  a.n1 = g1->normal;
  a.x1 = g1->pos;
  a.m1 = g1->mat;
  if (g2) {
    a.n2 = g2->normal;
    a.x2 = g2->pos;
    a.m2 = g2->mat;
  }
  a.P = pixels;
  a.mats = mat_spectra;
  a.n_mat = n_mat;
  a.lpos = lights->pos;
  a.linten = lights->intensity;
  a.spd = light_spd;
  a.L = lights->count;
  a.n = n;
  a.T = T;
  a.xyz = xyz_out;
  a.spectra = spectra_out;
  a.err = ctx->d_err;
  const bool sec = g2 != nullptr;
  cudaStream_t s = hsc::as_stream(stream);
  const int sm = ctx->sm_count;
  if (n <= 8) return hsc::launch_spec_sec<8>(a, sec, sm, s);
  if (n <= 16) return hsc::launch_spec_sec<16>(a, sec, sm, s);
  if (n <= 32) return hsc::launch_spec_sec<32>(a, sec, sm, s);
  if (n <= 48) return hsc::launch_spec_sec<48>(a, sec, sm, s);
  if (n <= 64) return hsc::launch_spec_sec<64>(a, sec, sm, s);
  if (n <= 84) return hsc::launch_spec_sec<84>(a, sec, sm, s);
  if (n <= 96) return hsc::launch_spec_sec<96>(a, sec, sm, s);
  return hsc::launch_spec_sec<128>(a, sec, sm, s);
}
