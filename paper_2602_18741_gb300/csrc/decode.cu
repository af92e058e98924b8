// Decoding the latent image once per frame (Fig. 2b): to XYZ with the folded
// 3 x k matrix M = T D, to 8-bit sRGB, and to n-sample spectra s_hat = W_dec z
// (Eq. 4).  All three are HBM streams: per pixel a few dozen bytes in and 12
// (XYZ) or 4n (spectra) bytes out against a handful of FMAs per output.
#include "common.cuh"
#include "shade_latent.cuh"

namespace hsc {

namespace {

constexpr int kDBlock = 256;

template <int DT>
__device__ __forceinline__ float load_lat(const void* base, int64_t i, const float* s_scale, int c) {
  if (DT == HSC_F32) return __ldg(reinterpret_cast<const float*>(base) + i);
  if (DT == HSC_BF16)
    return __uint_as_float(((unsigned int)__ldg(reinterpret_cast<const unsigned short*>(base) + i)) << 16);
  if (DT == HSC_F16) return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(base) + i)));
  return __fmul_rn(fp8_e4m3_to_float(__ldg(reinterpret_cast<const unsigned char*>(base) + i)), s_scale[c]);
}

// One thread per pixel: XYZ = M z with the sums over c in order, then sRGB.
// KT > 0 fixes k at compile time (the loads of a pixel's codes then issue
// back to back); KT = 0 takes k at run time.
template <int DT, int KT>
__global__ void __launch_bounds__(kDBlock) decode_xyz_kernel(const void* __restrict__ latent,
                                                             const float* __restrict__ scales, int64_t P, int k_rt,
                                                             const float* __restrict__ M, float* __restrict__ xyz,
                                                             uint8_t* __restrict__ srgb8) {
  const int k = KT > 0 ? KT : k_rt;
  __shared__ float s_M[3 * HSC_MAX_K];
  __shared__ float s_scale[HSC_MAX_K];
  for (int i = threadIdx.x; i < 3 * k; i += blockDim.x) s_M[i] = M[i];
  if (DT == HSC_FP8_E4M3)
    for (int i = threadIdx.x; i < k; i += blockDim.x) s_scale[i] = scales[i];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if constexpr (KT > 0) {
    // four pixels per pass, all their codes loaded before any is used
    constexpr int U = 4;
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p0 < P; p0 += U * stride) {
      float z[U][KT];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t p = p0 + u * stride;
#pragma unroll
        for (int c = 0; c < KT; ++c) z[u][c] = p < P ? load_lat<DT>(latent, p * KT + c, s_scale, c) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t p = p0 + u * stride;
        if (p >= P) break;
        float X = 0.0f, Y = 0.0f, Z = 0.0f;
#pragma unroll
        for (int c = 0; c < KT; ++c) {
          X = __fmaf_rn(s_M[c], z[u][c], X);
          Y = __fmaf_rn(s_M[KT + c], z[u][c], Y);
          Z = __fmaf_rn(s_M[2 * KT + c], z[u][c], Z);
        }
        if (xyz) {
          xyz[3 * p + 0] = X;
          xyz[3 * p + 1] = Y;
          xyz[3 * p + 2] = Z;
        }
        if (srgb8) xyz_to_srgb8(X, Y, Z, srgb8 + 3 * p);
      }
    }
  } else {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
      float X = 0.0f, Y = 0.0f, Z = 0.0f;
      for (int c = 0; c < k; ++c) {
        const float z = load_lat<DT>(latent, p * k + c, s_scale, c);
        X = __fmaf_rn(s_M[c], z, X);
        Y = __fmaf_rn(s_M[k + c], z, Y);
        Z = __fmaf_rn(s_M[2 * k + c], z, Z);
      }
      if (xyz) {
        xyz[3 * p + 0] = X;
        xyz[3 * p + 1] = Y;
        xyz[3 * p + 2] = Z;
      }
      if (srgb8) xyz_to_srgb8(X, Y, Z, srgb8 + 3 * p);
    }
  }
}

// Spectral decode on CUDA cores (FP32 latent).  Thread (i, r) of an n x R
// CTA owns wavelength i -- its row of D stays in registers for the whole
// kernel -- and pixel rows r, r + R, ... of each tile.  A tile's latent rows
// are staged in shared memory (row stride padded to a multiple of 4 floats)
// and read as broadcast float4s; the 32 lanes of a warp then store 32
// consecutive floats of one output row, so every store is a full 128-byte
// line.  Sums over c run in order.
constexpr int kTP = 64;        // pixels per tile
constexpr int kDecThreads = 256;

template <int KP>  // k rounded up to a multiple of 4 (<= 16)
__global__ void __launch_bounds__(kDecThreads) decode_spectra_f32_kernel(const float* __restrict__ z, int64_t P,
                                                                         int k, const float* __restrict__ D, int n,
                                                                         int R, float* __restrict__ out) {
  __shared__ __align__(16) float s_z[kTP * KP];
  const int t = threadIdx.x;
  const int i = t % n, r = t / n;
  const bool active = r < R;
  float d[KP];
#pragma unroll
  for (int c = 0; c < KP; ++c) d[c] = (active && c < k) ? __ldg(D + i * k + c) : 0.0f;
  const int64_t tiles = (P + kTP - 1) / kTP;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t p0 = tile * kTP;
    const int tp = (int)min((int64_t)kTP, P - p0);
    __syncthreads();
    for (int e = t; e < kTP * KP; e += blockDim.x) {
      const int pl = e / KP, c = e - pl * KP;
      s_z[e] = (pl < tp && c < k) ? __ldg(z + (p0 + pl) * k + c) : 0.0f;
    }
    __syncthreads();
    if (!active) continue;
    for (int pl = r; pl < tp; pl += R) {
      const float4* zr = reinterpret_cast<const float4*>(s_z + pl * KP);
      float s = 0.0f;
#pragma unroll
      for (int q = 0; q < KP / 4; ++q) {
        const float4 v = zr[q];
        s = __fmaf_rn(d[4 * q + 0], v.x, s);
        s = __fmaf_rn(d[4 * q + 1], v.y, s);
        s = __fmaf_rn(d[4 * q + 2], v.z, s);
        s = __fmaf_rn(d[4 * q + 3], v.w, s);
      }
      out[(p0 + pl) * n + i] = s;
    }
  }
}

// Generic FP32 decode for k > 16: one thread per output, sums over c in order.
__global__ void __launch_bounds__(256) decode_spectra_f32_generic(const float* __restrict__ z, int64_t P, int k,
                                                                  const float* __restrict__ D, int n,
                                                                  float* __restrict__ out) {
  const int64_t total = P * n;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = f / n;
    const int i = (int)(f - p * n);
    float s = 0.0f;
    for (int c = 0; c < k; ++c) s = __fmaf_rn(__ldg(D + i * k + c), __ldg(z + p * k + c), s);
    out[f] = s;
  }
}

int64_t stream_grid(int64_t work, int block, int sm_count, int per_sm) {
  int64_t g = (work + block - 1) / block;
  const int64_t cap = (int64_t)sm_count * per_sm;
  if (g > cap) g = cap;
  return g < 1 ? 1 : g;
}

}  // namespace

hsc_status launch_decode_xyz(const void* latent, int dt, const float* scales, int64_t P, int k, const float* M,
                             float* xyz, uint8_t* srgb8, int sm_count, cudaStream_t s) {
  const int64_t grid = stream_grid(P, kDBlock, sm_count, 8);
  auto go = [&](auto kern) { kern<<<(unsigned)grid, kDBlock, 0, s>>>(latent, scales, P, k, M, xyz, srgb8); };
  switch (dt) {
    case HSC_F32:
      if (k == 6) go(decode_xyz_kernel<HSC_F32, 6>);
      else if (k == 9) go(decode_xyz_kernel<HSC_F32, 9>);
      else if (k == 3) go(decode_xyz_kernel<HSC_F32, 3>);
      else go(decode_xyz_kernel<HSC_F32, 0>);
      break;
    case HSC_BF16: go(decode_xyz_kernel<HSC_BF16, 0>); break;
    case HSC_F16: go(decode_xyz_kernel<HSC_F16, 0>); break;
    default:
      if (k == 6) go(decode_xyz_kernel<HSC_FP8_E4M3, 6>);
      else go(decode_xyz_kernel<HSC_FP8_E4M3, 0>);
      break;
  }
  return check_launch("decode_xyz_kernel");
}

hsc_status launch_decode_spectra_f32(const float* z, int64_t P, int k, const float* D, int n, float* out,
                                     int sm_count, cudaStream_t s) {
  if (k > 16) {
    const int64_t grid = stream_grid(P * n, 256, sm_count, 8);
    decode_spectra_f32_generic<<<(unsigned)grid, 256, 0, s>>>(z, P, k, D, n, out);
    return check_launch("decode_spectra_f32_generic");
  }
  const int R = kDecThreads / n > 0 ? kDecThreads / n : 1;   // pixel rows per CTA (n <= 128)
  const int64_t tiles = (P + kTP - 1) / kTP;
  int64_t grid = tiles < (int64_t)sm_count * 8 ? tiles : (int64_t)sm_count * 8;
  if (grid < 1) grid = 1;
  const int kp = (k + 3) / 4 * 4;
  switch (kp) {
    case 4: decode_spectra_f32_kernel<4><<<(unsigned)grid, kDecThreads, 0, s>>>(z, P, k, D, n, R, out); break;
    case 8: decode_spectra_f32_kernel<8><<<(unsigned)grid, kDecThreads, 0, s>>>(z, P, k, D, n, R, out); break;
    case 12: decode_spectra_f32_kernel<12><<<(unsigned)grid, kDecThreads, 0, s>>>(z, P, k, D, n, R, out); break;
    default: decode_spectra_f32_kernel<16><<<(unsigned)grid, kDecThreads, 0, s>>>(z, P, k, D, n, R, out); break;
  }
  return check_launch("decode_spectra_f32_kernel");
}

hsc_status launch_decode_spectra_tc(hsc_ctx* ctx, const void* latent, int dt, const float* scales, int64_t P, int k,
                                    const float* D, int n, float* out, cudaStream_t s);

}  // namespace hsc

extern "C" {

hsc_status hsc_decode_xyz(hsc_ctx* ctx, const void* latent, hsc_dtype dt, const float* scales, int64_t pixels, int k,
                          const float* M_xyz, float* xyz_out, uint8_t* srgb8_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(k >= 1 && k <= HSC_MAX_K, "k=%d out of range", k);
  HSC_REQUIRE(pixels >= 0, "negative pixel count");
  HSC_REQUIRE(dt == HSC_F32 || dt == HSC_BF16 || dt == HSC_F16 || dt == HSC_FP8_E4M3, "bad latent dtype");
  HSC_REQUIRE(pixels == 0 || (latent && M_xyz && (xyz_out || srgb8_out)), "null pointer");
  HSC_REQUIRE(dt != HSC_FP8_E4M3 || scales, "fp8 latent needs scales");
  HSC_REQUIRE(hsc::aligned(latent, dt == HSC_F32 ? 4 : (dt == HSC_FP8_E4M3 ? 1 : 2)) && hsc::aligned(xyz_out, 4) &&
                  hsc::aligned(M_xyz, 4),
              "misaligned pointer");
  if (pixels == 0) return HSC_OK;
  HSC_GUARD(ctx);
  return hsc::launch_decode_xyz(latent, (int)dt, scales, pixels, k, M_xyz, xyz_out, srgb8_out, ctx->sm_count,
                                hsc::as_stream(stream));
}

hsc_status hsc_decode_spectra(hsc_ctx* ctx, const void* latent, hsc_dtype dt, const float* scales, int64_t pixels,
                              int k, const float* D, int n, float* spectra_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(k >= 1 && k <= HSC_MAX_K, "k=%d out of range", k);
  HSC_REQUIRE(n >= 1 && n <= HSC_MAX_N, "n=%d out of range", n);
  HSC_REQUIRE(pixels >= 0, "negative pixel count");
  if (pixels == 0) return HSC_OK;
  HSC_REQUIRE(latent && D && spectra_out, "null pointer");
  HSC_REQUIRE(hsc::aligned(spectra_out, 16), "spectra_out must be 16-byte aligned");
  HSC_GUARD(ctx);
  cudaStream_t s = hsc::as_stream(stream);
  if (dt == HSC_F32) {
    HSC_REQUIRE(hsc::aligned(latent, 4), "misaligned latent");
    // k <= 10: tensor cores on the three-part bf16 split (FP32 accuracy);
    // otherwise CUDA cores
    if (k <= 10) return hsc::launch_decode_spectra_tc(ctx, latent, (int)dt, nullptr, pixels, k, D, n, spectra_out, s);
    return hsc::launch_decode_spectra_f32(reinterpret_cast<const float*>(latent), pixels, k, D, n, spectra_out,
                                          ctx->sm_count, s);
  }
  HSC_REQUIRE(dt == HSC_BF16 || dt == HSC_FP8_E4M3, "spectral decode takes F32, BF16 or FP8_E4M3 latents");
  HSC_REQUIRE(k <= 16, "tensor-core decode supports k <= 16 (got %d)", k);
  HSC_REQUIRE(dt != HSC_FP8_E4M3 || scales, "fp8 latent needs scales");
  return hsc::launch_decode_spectra_tc(ctx, latent, (int)dt, scales, pixels, k, D, n, spectra_out, s);
}

}  // extern "C"
