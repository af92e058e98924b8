// Shared host/device helpers of libhsc (GB300, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stdarg.h>
#include <stdio.h>

#include <map>
#include <string>
#include <tuple>

#include "../../include/hsc.h"

// ---------------------------------------------------------------- context

// Fixed scratch block, allocated once per context (bytes).
#define HSC_SMALL_SCRATCH (1u << 20)
// Offsets inside the fixed scratch block.
#define HSC_OFF_CHANMAX 0u          // HSC_MAX_K uint32 (fp8 per-channel max)
#define HSC_OFF_QUEUE (768u << 10)  // HSC_QUEUE_SLOTS pairs of uint32 tile counters, one pair per stream
#define HSC_OFF_FITTICKET 1024u     // one uint32 arrival ticket of hsc_codec_fit_track
#define HSC_OFF_REDUCE 4096u        // reduction workspace for hsc_delta_e

namespace hsc {
// Shape class of a tuned kernel launch (see tune.cuh).
struct TuneKey {
  int kind = 0, channels = 0, sec = 0, lbucket = 0, pbucket = 0, dtype = 0;
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, channels, sec, lbucket, pbucket, dtype) <
           std::tie(o.kind, o.channels, o.sec, o.lbucket, o.pbucket, o.dtype);
  }
};
struct LaunchCfg {
  int sm_count = 0;
  int ppt = 2;      // pixels (or shading points) per thread
  int block = 128;  // threads per CTA
  int waves = 1;    // persistent grid of waves x resident CTAs x SMs; 0 = one CTA per pixel tile;
                    // -1 = one wave of persistent CTAs taking tiles from an atomic queue
  int vec = 1;      // 1: scalar FP32; 2: shading points in f32x2 pairs
  int chunk = 0;    // spectral kernel: channels per sweep (0 = default)
  unsigned int* queue = nullptr;  // tile counter for waves = -1
};
}  // namespace hsc

struct hsc_ctx {
  int device = 0;
  int sm_count = 0;
  int max_smem_optin = 0;
  unsigned int* d_err = nullptr;   // device error word (bit flags)
  unsigned char* d_small = nullptr;
  unsigned char* d_big = nullptr;  // growable scratch (PASSES images, fp32 latent)
  size_t big_bytes = 0;
  int autotune = 0;                               // hsc_set_autotune
  std::map<hsc::TuneKey, hsc::LaunchCfg> tuned;   // chosen launch configurations
  std::string tune_report;                        // candidate timings, one line per shape class
  hsc::LaunchCfg forced{0, 0, 128, 1, 1, 0, nullptr};  // hsc_force_launch_config (ppt 0 = not forced)
  // hsc_shade_frames: ring of pinned host / device descriptor buffers
  static constexpr int kDescSlots = 8;
  struct DescSlot {
    void* h = nullptr;
    void* d = nullptr;
    cudaEvent_t ev = nullptr;
  } desc_ring[kDescSlots];
  int desc_next = 0;
  // dynamically scheduled shading launches: the tile-counter pair of each
  // stream seen so far (index into the HSC_OFF_QUEUE block), so launches on
  // different streams never share a counter
  std::map<void*, int> queue_slots;
};

// Device error flags.
#define HSC_DEVERR_MATERIAL 1u
#define HSC_DEVERR_TIMEOUT 2u

namespace hsc {

hsc_status set_error(hsc_status st, const char* fmt, ...);
hsc_status clear_error();
hsc_status check_launch(const char* what);
hsc_status ensure_big(hsc_ctx* ctx, size_t bytes, cudaStream_t stream);
// The tile-counter pair of `stream` for dynamically scheduled launches, or
// null once HSC_QUEUE_SLOTS streams have their own (launch statically then).
unsigned int* stream_queue(hsc_ctx* ctx, cudaStream_t stream);

// Makes ctx->device current for the scope of a call and restores the
// caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace hsc

#define HSC_CHECK_CTX(ctx)                                                        \
  do {                                                                            \
    if ((ctx) == nullptr) return hsc::set_error(HSC_ERR_INVALID_ARG, "null context"); \
  } while (0)

#define HSC_REQUIRE(cond, ...)                                                    \
  do {                                                                            \
    if (!(cond)) return hsc::set_error(HSC_ERR_INVALID_ARG, __VA_ARGS__);         \
  } while (0)

#define HSC_CUDA(call)                                                            \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return hsc::set_error(HSC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define HSC_TRY(expr)                                                             \
  do {                                                                            \
    hsc_status s_ = (expr);                                                       \
    if (s_ != HSC_OK) return s_;                                                  \
  } while (0)

#define HSC_GUARD(ctx)                                                            \
  hsc::DeviceGuard guard_((ctx)->device);                                         \
  if (!guard_.ok) return hsc::set_error(HSC_ERR_CUDA, "cannot select device %d", (ctx)->device)

// ---------------------------------------------------------------- device

namespace hsc {

// 1/pi rounded to float32.
constexpr float kInvPi = 0.318309886183790671538f;

// MUFU reciprocal square root (approximate, flush-to-zero), one instruction.
__device__ __forceinline__ float rsqrt_mufu(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// c * ri clamped to [0, 1] in one instruction (mul with saturation).
__device__ __forceinline__ float mul_sat(float a, float b) {
  float r;
  asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// Geometry term of one (shading point, light) pair:
//   g = max(0, n.(p - x)) / |p - x|^3 = sat(n.d / |d|) / |d|^2,  d = p - x.
// n.d / |d| is the cosine of the incidence angle, so clamping it to [0, 1]
// is max(0, .) (the upper clamp only absorbs rounding above 1).  Explicit
// round-to-nearest intrinsics fix the instruction sequence, so every kernel
// that calls this produces bit-identical g: 12 FP32 instructions + one MUFU.
__device__ __forceinline__ float geometry_term(float x, float y, float z, float nx, float ny, float nz,
                                               float px, float py, float pz) {
  const float dx = __fsub_rn(px, x);
  const float dy = __fsub_rn(py, y);
  const float dz = __fsub_rn(pz, z);
  const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
  const float c = __fmaf_rn(nz, dz, __fmaf_rn(ny, dy, __fmul_rn(nx, dx)));
  const float ri = rsqrt_mufu(r2);
  return __fmul_rn(mul_sat(c, ri), __fmul_rn(ri, ri));
}

// Packed FP32 pairs (sm_100+ f32x2 arithmetic): each half is rounded exactly
// like the scalar instruction, so a pair op equals two scalar ops bit for bit
// while taking one issue slot.
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// geometry_term for two shading points at once: the same operations in the
// same order per half, so each half equals geometry_term bit for bit.
__device__ __forceinline__ f2 geometry_term_x2(f2 x, f2 y, f2 z, f2 nx, f2 ny, f2 nz, f2 px, f2 py, f2 pz) {
  const f2 dx = f2_sub(px, x);
  const f2 dy = f2_sub(py, y);
  const f2 dz = f2_sub(pz, z);
  const f2 r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
  const f2 c = f2_fma(nz, dz, f2_fma(ny, dy, f2_mul(nx, dx)));
  float c0, c1, r0, r1;
  f2_unpack(c, c0, c1);
  f2_unpack(r2, r0, r1);
  const float ri0 = rsqrt_mufu(r0), ri1 = rsqrt_mufu(r1);
  const f2 ri = f2_pack(ri0, ri1);
  return f2_mul(f2_pack(mul_sat(c0, ri0), mul_sat(c1, ri1)), f2_mul(ri, ri));
}

// Virtual-point-light transfer from the secondary point to the primary,
// divided by pi (the secondary reflectance's Lambert 1/pi):
//   h = max(0, n1.d) max(0, -n2.d) / (|d|^2 max(|d|^2, 1e-2)) / pi,  d = x2 - x1
__device__ __forceinline__ float bounce_term(float x1, float y1, float z1, float nx1, float ny1, float nz1,
                                             float x2, float y2, float z2, float nx2, float ny2, float nz2) {
  const float dx = __fsub_rn(x2, x1);
  const float dy = __fsub_rn(y2, y1);
  const float dz = __fsub_rn(z2, z1);
  const float dd = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
  float c1 = __fmaf_rn(nz1, dz, __fmaf_rn(ny1, dy, __fmul_rn(nx1, dx)));
  float c2 = __fmaf_rn(nz2, dz, __fmaf_rn(ny2, dy, __fmul_rn(nx2, dx)));
  c1 = fmaxf(c1, 0.0f);
  c2 = fmaxf(-c2, 0.0f);
  const float den = __fmul_rn(dd, fmaxf(dd, 1e-2f));
  const float h = __fdiv_rn(__fmul_rn(c1, c2), den);
  return (den > 0.0f) ? __fmul_rn(h, kInvPi) : 0.0f;
}

// XYZ to 8-bit sRGB (IEC 61966-2-1): linear sRGB by the standard matrix with
// each sum in a fixed order, clamped to [0, 1], the transfer function (its
// power through the fast exp2/log2 intrinsics: the 8-bit output quantises
// it), u8 = floor(255 v + 0.5).  Shared by the decode kernels and the fused
// shading epilogue, so both give the same bytes for the same XYZ.
__device__ __forceinline__ float srgb_oetf(float v) {
  v = __saturatef(v);
  return (v <= 0.0031308f) ? __fmul_rn(12.92f, v) : __fmaf_rn(1.055f, __powf(v, 1.0f / 2.4f), -0.055f);
}

// u8 = floor(255 v + 0.5) for v in [0, 1].  x = 255 v + 0.5 lies in
// [0.5, 255.5]; adding 2^23 rounded toward minus infinity gives exactly
// 2^23 + floor(x) (the spacing of floats in [2^23, 2^24) is 1), whose low
// mantissa bits are floor(x): an FP32 add and a mask instead of a
// float-to-integer conversion.
__device__ __forceinline__ uint8_t srgb_u8(float v) {
  const float x = __fmaf_rn(v, 255.0f, 0.5f);
  return (uint8_t)(__float_as_uint(__fadd_rd(x, 8388608.0f)) & 0xFFu);
}

__device__ __forceinline__ void xyz_to_srgb8(float X, float Y, float Z, uint8_t* out) {
  const float r = __fmaf_rn(-0.4986f, Z, __fmaf_rn(-1.5372f, Y, __fmul_rn(3.2406f, X)));
  const float g = __fmaf_rn(0.0415f, Z, __fmaf_rn(1.8758f, Y, __fmul_rn(-0.9689f, X)));
  const float b = __fmaf_rn(1.0570f, Z, __fmaf_rn(-0.2040f, Y, __fmul_rn(0.0557f, X)));
  out[0] = srgb_u8(srgb_oetf(r));
  out[1] = srgb_u8(srgb_oetf(g));
  out[2] = srgb_u8(srgb_oetf(b));
}

// Load element i of a code array stored as F32 / BF16 / F16 as float.
__device__ __forceinline__ float load_code(const void* base, int dt, int64_t i) {
  if (dt == HSC_F32) return __ldg(reinterpret_cast<const float*>(base) + i);
  if (dt == HSC_BF16) {
    const unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(base) + i);
    return __uint_as_float(((unsigned int)u) << 16);
  }
  const unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(base) + i);
  return __half2float(__ushort_as_half(u));
}

// fp8 e4m3 (OCP FP8, bias 7, 3 mantissa bits, no infinities) -> float, exact:
// exponent field 0 is subnormal (mant * 2^-9); S.1111.111 is NaN.
__device__ __forceinline__ float fp8_e4m3_to_float(unsigned int b) {
  const unsigned int s = (b >> 7) & 1u, e = (b >> 3) & 15u, m = b & 7u;
  float v;
  if (e == 0u) {
    v = (float)m * 0.001953125f;  // 2^-9
  } else if (e == 15u && m == 7u) {
    v = __uint_as_float(0x7fc00000u);
  } else {
    v = __uint_as_float(((e + 120u) << 23) | (m << 20));
  }
  return s ? -v : v;
}

// float -> fp8 e4m3 byte, round to nearest even, saturating to +-448.  Both
// halves of the packed conversion get the same value, so the byte order of
// the packed result does not matter.
__device__ __forceinline__ unsigned int float_to_fp8_e4m3(float x) {
  unsigned short r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %1;" : "=h"(r) : "f"(x));
  return (unsigned int)(r & 0xFFu);
}

// float -> bf16 / f16 bits, round to nearest even.
__device__ __forceinline__ unsigned short float_to_bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ unsigned short float_to_f16_bits(float x) {
  return __half_as_ushort(__float2half_rn(x));
}

// Load element i of a latent image of dtype dt as float (fp8 dequantised with
// the channel's scale).
__device__ __forceinline__ float load_latent(const void* base, int dt, int64_t i, const float* scales, int c) {
  if (dt == HSC_FP8_E4M3) {
    const unsigned int b = __ldg(reinterpret_cast<const unsigned char*>(base) + i);
    return __fmul_rn(fp8_e4m3_to_float(b), __ldg(scales + c));
  }
  return load_code(base, dt, i);
}

}  // namespace hsc
