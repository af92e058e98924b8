// Latent (k-code) deferred shading: the k/3 RGB passes of Fig. 2b, their
// reassembly, and the fused single-launch k-channel form.
//
// Per pixel and per light the work is one geometry term g (13 FP32 ops + one
// MUFU rsqrt) and KC FMAs acc[c] += g * v_l[c], where v_l = (I_l / pi) * E(spd_l)
// is the light's scaled code.  After the light loop the blockwise Hadamard
// product with the material codes (Eq. 6, element-wise on R^k) and the
// indirect bounce give
//     z[c] = zR1[c] * (A1[c] + h * (zR2[c] * A2[c])).
// A pass (KC = 3) and the fused launch (KC = k) run the same template: each
// channel sees the same operations in the same order (same light order, same
// geometry_term instruction sequence, no reductions across channels), so the
// fused latent image is bit-identical to the reassembled passes.
//
// GB300 mapping: FP32 issue bound (~20 lane-ops per pixel-light for k = 6 vs
// 56 bytes of G-buffer per pixel amortised over 2L evaluations).  Lights and
// their pre-scaled codes are staged once per CTA in shared memory and read as
// broadcast float4s; each thread owns PPT pixels (x2 shading points with the
// secondary G-buffer) so one light load feeds 2*PPT geometry evaluations; the
// grid is either persistent (a multiple of the SM count striding over pixel
// tiles) or one CTA per tile.  The thread mapping never changes what a
// channel computes, so every configuration gives bit-identical results; the
// autotuner picks among them by timing.  VEC = 2 processes the shading
// points in pairs with the packed f32x2 instructions of sm_100+: half the
// FP32 issue slots for the same FP32 work.
#pragma once

#include "common.cuh"
#include "shade_latent.cuh"

namespace hsc {

namespace {

// Float4s per staged light.  VEC = 1: px py pz v0 .. v{KC-1} (padded);
// VEC = 2: every value duplicated (px px py py pz pz v0 v0 ...) so that a
// float4 load yields two ready-made f32x2 broadcast operands.
template <int KC, int VEC>
struct LightStage {
  static constexpr int F4 = VEC == 1 ? (3 + KC + 3) / 4 : (3 + KC + 1) / 2;
};

// Code element i as float for one storage format (the conversions of
// load_code, with the format fixed at compile time).
template <int DT>
__device__ __forceinline__ float code_at(const void* base, int64_t i) {
  if constexpr (DT == HSC_F32) {
    return __ldg(reinterpret_cast<const float*>(base) + i);
  } else {
    const unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(base) + i);
    if constexpr (DT == HSC_BF16)
      return __uint_as_float(((unsigned int)u) << 16);
    else
      return __half2float(__ushort_as_half(u));
  }
}

// Staging loads each thread issues before it writes any of them to shared
// memory: every CTA stages at its start, so the loads' latency is paid once
// per batch instead of once per element.
constexpr int kStageBatch = 8;

// Stages lights l0 .. l0+nl-1 of one launch: positions and the code channels
// c0 .. c0+KC-1 pre-multiplied by I/pi, laid out as LightStage describes.
// The prologue form: every load of a batch has an in-range address (the light
// index and the channel are clamped) and is selected afterwards, so a
// batch's loads issue back to back.
template <int KC, int VEC, int BLOCK, int DT>
__device__ __forceinline__ void stage_light_codes_dt(const ShadeArgs& a, float* s, int l0, int nl) {
  constexpr int per = LightStage<KC, VEC>::F4 * 4;
  const int n = nl * per;
  for (int base = threadIdx.x; base < n; base += kStageBatch * BLOCK) {
    float v[kStageBatch];
#pragma unroll
    for (int r = 0; r < kStageBatch; ++r) {
      const int idx = min(base + r * BLOCK, n - 1);
      const int l = idx / per, j0 = idx - l * per;
      const int j = VEC == 1 ? j0 : (j0 >> 1);
      const int lg = l0 + l;
      const float pos = __ldg(a.lpos + 3 * lg + min(j, 2));
      const float code = code_at<DT>(a.light_codes, (int64_t)lg * a.k + a.c0 + min(max(j - 3, 0), KC - 1));
      const float sc = __fmul_rn(__ldg(a.linten + lg), kInvPi);
      v[r] = j < 3 ? pos : (j < 3 + KC ? __fmul_rn(code, sc) : 0.0f);
    }
#pragma unroll
    for (int r = 0; r < kStageBatch; ++r)
      if (base + r * BLOCK < n) s[base + r * BLOCK] = v[r];
  }
}

// The same values one load at a time: the form used between light tiles
// inside the tile loop, where the batch's registers would add to the live
// accumulators.
template <int KC, int VEC, int BLOCK>
__device__ __forceinline__ void restage_light_codes(const ShadeArgs& a, float4* s_light, int l0, int nl) {
  constexpr int per = LightStage<KC, VEC>::F4 * 4;
  float* s = reinterpret_cast<float*>(s_light);
  for (int idx = threadIdx.x; idx < nl * per; idx += BLOCK) {
    const int l = idx / per, j0 = idx - l * per;
    const int j = VEC == 1 ? j0 : (j0 >> 1);
    const int lg = l0 + l;
    float v = 0.0f;
    if (j < 3) {
      v = __ldg(a.lpos + 3 * lg + j);
    } else if (j < 3 + KC) {
      const float sc = __fmul_rn(__ldg(a.linten + lg), kInvPi);
      v = __fmul_rn(load_code(a.light_codes, a.code_dt, (int64_t)lg * a.k + a.c0 + (j - 3)), sc);
    }
    s[idx] = v;
  }
}

template <int KC, int VEC, int BLOCK>
__device__ __forceinline__ void stage_light_codes(const ShadeArgs& a, float4* s_light, int l0, int nl) {
  float* s = reinterpret_cast<float*>(s_light);
  if (a.code_dt == HSC_F32)
    stage_light_codes_dt<KC, VEC, BLOCK, HSC_F32>(a, s, l0, nl);
  else if (a.code_dt == HSC_BF16)
    stage_light_codes_dt<KC, VEC, BLOCK, HSC_BF16>(a, s, l0, nl);
  else
    stage_light_codes_dt<KC, VEC, BLOCK, HSC_F16>(a, s, l0, nl);
}

// Material code tables of at most kMatStage values (n_mat x KC) are staged
// once per CTA in shared memory as FP32 (the same values the global path
// converts per row), so the epilogue's material reads are shared-memory
// loads; larger tables are read from global memory.
constexpr int kMatStage = 4096;

template <int KC>
__host__ __device__ __forceinline__ bool mat_staged(int n_mat) { return (int64_t)n_mat * KC <= kMatStage; }

template <int KC, int BLOCK, int DT>
__device__ __forceinline__ void stage_material_codes_dt(const ShadeArgs& a, float* s_mat) {
  const int n = a.n_mat * KC;
  for (int base = threadIdx.x; base < n; base += kStageBatch * BLOCK) {
    float v[kStageBatch];
#pragma unroll
    for (int r = 0; r < kStageBatch; ++r) {
      const int i = min(base + r * BLOCK, n - 1);
      const int row = i / KC, c = i - row * KC;
      v[r] = code_at<DT>(a.mat_codes, (int64_t)row * a.k + a.c0 + c);
    }
#pragma unroll
    for (int r = 0; r < kStageBatch; ++r)
      if (base + r * BLOCK < n) s_mat[base + r * BLOCK] = v[r];
  }
}

template <int KC, int BLOCK>
__device__ __forceinline__ void stage_material_codes(const ShadeArgs& a, float* s_mat) {
  if (a.code_dt == HSC_F32)
    stage_material_codes_dt<KC, BLOCK, HSC_F32>(a, s_mat);
  else if (a.code_dt == HSC_BF16)
    stage_material_codes_dt<KC, BLOCK, HSC_BF16>(a, s_mat);
  else
    stage_material_codes_dt<KC, BLOCK, HSC_F16>(a, s_mat);
}

// Resident CTAs per SM asked of the compiler: the 128-thread scalar form with
// at most two pixels per thread and six channels runs best at 7 CTAs per SM
// (72 registers); the others keep the compiler's choice.
template <int KC, int PPT, int BLOCK, int VEC>
constexpr int latent_min_blocks() { return (KC <= 6 && PPT <= 2 && BLOCK == 128 && VEC == 1) ? 7 : 1; }

// The KC code channels c0 .. c0+KC-1 of row `row` of a code table in its
// storage format; one format test per row instead of per channel.
template <int KC>
__device__ __forceinline__ void load_code_row(const ShadeArgs& a, int row, float (&z)[KC]) {
  const int64_t off = (int64_t)row * a.k + a.c0;
  if (a.code_dt == HSC_F32) {
    const float* q = reinterpret_cast<const float*>(a.mat_codes) + off;
#pragma unroll
    for (int c = 0; c < KC; ++c) z[c] = __ldg(q + c);
  } else {
    const unsigned short* q = reinterpret_cast<const unsigned short*>(a.mat_codes) + off;
    unsigned short u[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) u[c] = __ldg(q + c);
    if (a.code_dt == HSC_BF16) {
#pragma unroll
      for (int c = 0; c < KC; ++c) z[c] = __uint_as_float(((unsigned int)u[c]) << 16);
    } else {
#pragma unroll
      for (int c = 0; c < KC; ++c) z[c] = __half2float(__ushort_as_half(u[c]));
    }
  }
}

// Shades one tile of BLOCK * PPT pixels: loads the shading points, sums every
// light into KC accumulators per point, applies the blockwise product with the
// material codes and the bounce, writes the latent channels (and XYZ with the
// decode matrix staged at s_M, and the fp8 channel maxima when asked).  When the lights fit one shared-memory
// tile the caller has staged them already (`staged`); otherwise the light
// tiles are staged here.  Must be called by every thread of the CTA.
template <int KC, int PPT, bool SEC, int BLOCK, int VEC, bool RGB = false>
__device__ __forceinline__ void shade_tile(const ShadeArgs& a, int64_t tile, float4* s_light, bool staged,
                                           const float* s_M, const float* s_mat = nullptr,
                                           unsigned int* cmax = nullptr) {
  constexpr int F4 = LightStage<KC, VEC>::F4;
  constexpr int NPT = PPT * (SEC ? 2 : 1);
  static_assert(VEC == 1 || NPT % 2 == 0, "paired points need an even point count");
  const int tid = threadIdx.x;
  const bool multi_tile = !staged;
  auto stage = [&](int l0, int nl) { restage_light_codes<KC, VEC, BLOCK>(a, s_light, l0, nl); };
  {
    float px[NPT], py[NPT], pz[NPT], nx[NPT], ny[NPT], nz[NPT];
    float hb[PPT];          // bounce term of each pixel (SEC)
    int mi1[PPT], mi2[PPT];  // material indices
    int64_t pix[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int64_t p = tile * (BLOCK * PPT) + (int64_t)j * BLOCK + tid;
      pix[j] = p;
      const int64_t pc = p < a.P ? p : a.P - 1;
      mi1[j] = __ldg(a.m1 + pc);
      mi2[j] = SEC ? __ldg(a.m2 + pc) : 0;
      px[j] = __ldg(a.x1 + 3 * pc + 0);
      py[j] = __ldg(a.x1 + 3 * pc + 1);
      pz[j] = __ldg(a.x1 + 3 * pc + 2);
      nx[j] = __ldg(a.n1 + 3 * pc + 0);
      ny[j] = __ldg(a.n1 + 3 * pc + 1);
      nz[j] = __ldg(a.n1 + 3 * pc + 2);
      if (SEC) {
        px[PPT + j] = __ldg(a.x2 + 3 * pc + 0);
        py[PPT + j] = __ldg(a.x2 + 3 * pc + 1);
        pz[PPT + j] = __ldg(a.x2 + 3 * pc + 2);
        nx[PPT + j] = __ldg(a.n2 + 3 * pc + 0);
        ny[PPT + j] = __ldg(a.n2 + 3 * pc + 1);
        nz[PPT + j] = __ldg(a.n2 + 3 * pc + 2);
      }
    }
    // the bounce term needs only the G-buffer: computed here, its latency
    // overlaps the light loop instead of the epilogue
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      if constexpr (SEC)
        hb[j] = bounce_term(px[j], py[j], pz[j], nx[j], ny[j], nz[j], px[PPT + j], py[PPT + j], pz[PPT + j],
                            nx[PPT + j], ny[PPT + j], nz[PPT + j]);
      else
        hb[j] = 0.0f;
    }
    float acc[NPT][KC];
#pragma unroll
    for (int q = 0; q < NPT; ++q)
#pragma unroll
      for (int c = 0; c < KC; ++c) acc[q][c] = 0.0f;

    if constexpr (VEC == 1) {
      for (int l0 = 0; l0 < a.L; l0 += kLightTile) {
        const int nl = min(kLightTile, a.L - l0);
        if (multi_tile) {
          __syncthreads();
          stage(l0, nl);
          __syncthreads();
        }
        const float4* sp = s_light;
#pragma unroll 4
        for (int l = 0; l < nl; ++l, sp += F4) {
          float v[F4 * 4];
#pragma unroll
          for (int f = 0; f < F4; ++f) {
            const float4 t = sp[f];
            v[4 * f + 0] = t.x;
            v[4 * f + 1] = t.y;
            v[4 * f + 2] = t.z;
            v[4 * f + 3] = t.w;
          }
#pragma unroll
          for (int q = 0; q < NPT; ++q) {
            const float g = geometry_term(px[q], py[q], pz[q], nx[q], ny[q], nz[q], v[0], v[1], v[2]);
#pragma unroll
            for (int c = 0; c < KC; ++c) acc[q][c] = __fmaf_rn(g, v[3 + c], acc[q][c]);
          }
        }
      }
    } else {
      // Pairs of shading points in f32x2 registers: with the secondary
      // G-buffer pair j is (primary j, secondary j), otherwise (pixel 2m,
      // pixel 2m + 1).
      constexpr int NPR = NPT / 2 > 0 ? NPT / 2 : 1;
      f2 X[NPR], Y[NPR], Z[NPR], NX[NPR], NY[NPR], NZ[NPR], A[NPR][KC];
#pragma unroll
      for (int q = 0; q < NPR; ++q) {
        const int qa = SEC ? q : 2 * q, qb = SEC ? PPT + q : 2 * q + 1;
        X[q] = f2_pack(px[qa], px[qb]);
        Y[q] = f2_pack(py[qa], py[qb]);
        Z[q] = f2_pack(pz[qa], pz[qb]);
        NX[q] = f2_pack(nx[qa], nx[qb]);
        NY[q] = f2_pack(ny[qa], ny[qb]);
        NZ[q] = f2_pack(nz[qa], nz[qb]);
#pragma unroll
        for (int c = 0; c < KC; ++c) A[q][c] = 0ull;  // +0.0f in both halves
      }
      for (int l0 = 0; l0 < a.L; l0 += kLightTile) {
        const int nl = min(kLightTile, a.L - l0);
        if (multi_tile) {
          __syncthreads();
          stage(l0, nl);
          __syncthreads();
        }
        const ulonglong2* sl = reinterpret_cast<const ulonglong2*>(s_light);
        const ulonglong2* sp = sl;
#pragma unroll 4
        for (int l = 0; l < nl; ++l, sp += F4) {
          f2 v[F4 * 2];
#pragma unroll
          for (int f = 0; f < F4; ++f) {
            const ulonglong2 t = sp[f];
            v[2 * f + 0] = t.x;
            v[2 * f + 1] = t.y;
          }
#pragma unroll
          for (int q = 0; q < NPR; ++q) {
            const f2 g = geometry_term_x2(X[q], Y[q], Z[q], NX[q], NY[q], NZ[q], v[0], v[1], v[2]);
#pragma unroll
            for (int c = 0; c < KC; ++c) A[q][c] = f2_fma(g, v[3 + c], A[q][c]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NPR; ++q) {
        const int qa = SEC ? q : 2 * q, qb = SEC ? PPT + q : 2 * q + 1;
#pragma unroll
        for (int c = 0; c < KC; ++c) f2_unpack(A[q][c], acc[qa][c], acc[qb][c]);
      }
    }

    // Epilogue: blockwise Hadamard product with the material codes + bounce.
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int64_t p = pix[j];
      const bool valid = p < a.P;
      // an out-of-range material index (primary or secondary) gives the
      // pixel zero radiance and flags the error word
      const int m1 = mi1[j];
      bool bad = (unsigned)m1 >= (unsigned)a.n_mat;
      float zr1[KC], out[KC];
      auto code_row = [&](int row, float (&z)[KC]) {
        if (s_mat) {
#pragma unroll
          for (int c = 0; c < KC; ++c) z[c] = s_mat[row * KC + c];
        } else {
          load_code_row<KC>(a, row, z);
        }
      };
      code_row(bad ? 0 : m1, zr1);
      if (SEC) {
        const int m2 = mi2[j];
        const bool bad2 = (unsigned)m2 >= (unsigned)a.n_mat;
        bad = bad || bad2;
        float zr2[KC];
        code_row(bad2 ? 0 : m2, zr2);
        const float h = hb[j];
#pragma unroll
        for (int c = 0; c < KC; ++c)
          out[c] = __fmul_rn(zr1[c], __fmaf_rn(h, __fmul_rn(zr2[c], acc[PPT + j][c]), acc[j][c]));
      } else {
#pragma unroll
        for (int c = 0; c < KC; ++c) out[c] = __fmul_rn(zr1[c], acc[j][c]);
      }
#pragma unroll
      for (int c = 0; c < KC; ++c) out[c] = bad ? 0.0f : out[c];
      if (valid && bad) atomicOr(a.err, HSC_DEVERR_MATERIAL);
      if (valid) {
        if (a.out) {  // the batched launch may ask for XYZ only
          float* o = a.out + p * a.out_stride + a.out_c0;
#pragma unroll
          for (int c = 0; c < KC; ++c) o[c] = out[c];
        }
        if constexpr (RGB) {
          float t[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            float s = 0.0f;
#pragma unroll
            for (int c = 0; c < KC; ++c) s = __fmaf_rn(s_M[r * KC + c], out[c], s);
            t[r] = s;
          }
          if (a.xyz) {
#pragma unroll
            for (int r = 0; r < 3; ++r) a.xyz[3 * p + r] = t[r];
          }
          xyz_to_srgb8(t[0], t[1], t[2], a.srgb8 + 3 * p);
        } else if (a.xyz) {
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            float s = 0.0f;
#pragma unroll
            for (int c = 0; c < KC; ++c) s = __fmaf_rn(s_M[r * KC + c], out[c], s);
            a.xyz[3 * p + r] = s;
          }
        }
      }
      if (cmax) {
        // non-negative floats order like their bit patterns; one atomic per
        // warp and channel into the CTA's maxima (shared memory)
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          const unsigned int bits = valid ? __float_as_uint(fmaxf(out[c], 0.0f)) : 0u;
          const unsigned int mx = __reduce_max_sync(0xffffffffu, bits);
          if ((tid & 31) == 0 && mx) atomicMax(cmax + c, mx);
        }
      }
    }
  }
}

// Stages the 3 x KC decode matrix (channels c0 .. c0+KC-1 of M) for the
// fused XYZ epilogue.
template <int KC, int BLOCK>
__device__ __forceinline__ void stage_decode_matrix(const ShadeArgs& a, float* s_M) {
  if (a.xyz || a.srgb8)
    for (int i = threadIdx.x; i < 3 * KC; i += BLOCK) s_M[i] = __ldg(a.M + (i / KC) * a.k + a.c0 + (i % KC));
}

// Dynamic tile queue: queue[0] hands out tiles, queue[1] counts the CTAs that
// have left the tile loop; the last one puts both back to zero, so the next
// launch on the stream finds a fresh counter without a memset.
__device__ __forceinline__ void release_queue(unsigned int* queue) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
      atomicExch(queue, 0u);
      atomicExch(queue + 1, 0u);
    }
  }
}

// RGB: the epilogue also writes 8-bit sRGB (a separate instantiation, so the
// kernels without it keep their code).
template <int KC, int PPT, bool SEC, int BLOCK, int VEC, bool RGB>
__global__ void __launch_bounds__(BLOCK, (latent_min_blocks<KC, PPT, BLOCK, VEC>()))
    shade_codes_kernel(const ShadeArgs a) {
  // dynamic shared memory: the light tile, then the material table if it fits
  extern __shared__ float4 s_light[];
  __shared__ float s_M[3 * KC];
  __shared__ unsigned int s_cmax[KC];  // the CTA's channel maxima (fp8 path)
  const bool staged = a.L <= kLightTile;
  unsigned int* cmax = a.chan_max ? s_cmax : nullptr;
  if (threadIdx.x < KC) s_cmax[threadIdx.x] = 0u;
  // dynamic schedule: the first tile is claimed before the staging, so the
  // atomic's latency overlaps it
  __shared__ int64_t s_next;
  if (a.queue && threadIdx.x == 0) s_next = (int64_t)atomicAdd(a.queue, 1u);
  float* s_mat = mat_staged<KC>(a.n_mat)
                     ? reinterpret_cast<float*>(s_light + min(a.L, kLightTile) * LightStage<KC, VEC>::F4)
                     : nullptr;
  if (staged) stage_light_codes<KC, VEC, BLOCK>(a, s_light, 0, a.L);
  if (s_mat) stage_material_codes<KC, BLOCK>(a, s_mat);
  stage_decode_matrix<KC, BLOCK>(a, s_M);
  __syncthreads();
  if (a.queue) {
    // dynamic schedule: persistent CTAs take the next tile from a counter
    for (;;) {
      const int64_t tile = s_next;
      __syncthreads();  // every thread has read s_next before it is replaced
      if (tile >= a.tiles) break;
      shade_tile<KC, PPT, SEC, BLOCK, VEC, RGB>(a, tile, s_light, staged, s_M, s_mat, cmax);
      if (threadIdx.x == 0) s_next = (int64_t)atomicAdd(a.queue, 1u);
      __syncthreads();
    }
    release_queue(a.queue);
  } else {
    for (int64_t tile = blockIdx.x; tile < a.tiles; tile += gridDim.x)
      shade_tile<KC, PPT, SEC, BLOCK, VEC, RGB>(a, tile, s_light, staged, s_M, s_mat, cmax);
  }
  if (cmax) {
    // one global atomic per CTA and channel
    __syncthreads();
    if (threadIdx.x < KC && s_cmax[threadIdx.x]) atomicMax(a.chan_max + a.c0 + threadIdx.x, s_cmax[threadIdx.x]);
  }
}

template <int KC, int PPT, bool SEC, int BLOCK, int VEC, bool RGB>
hsc_status launch_one_rgb(const ShadeArgs& a0, const LaunchCfg& cfg, cudaStream_t stream) {
  constexpr int F4 = LightStage<KC, VEC>::F4;
  ShadeArgs a = a0;
  a.tiles = (a.P + (int64_t)BLOCK * PPT - 1) / ((int64_t)BLOCK * PPT);
  const size_t smem = (size_t)min(a.L, kLightTile) * F4 * sizeof(float4) +
                      (mat_staged<KC>(a.n_mat) ? (size_t)a.n_mat * KC * sizeof(float) : 0);
  auto kern = shade_codes_kernel<KC, PPT, SEC, BLOCK, VEC, RGB>;
  static int occ = -1;
  if (occ < 0) {
    // resident CTAs with the largest light tile and material table (which may
    // pass the 48 KB a launch gets without opting in)
    const int smem_max = (int)(kLightTile * F4 * sizeof(float4) + kMatStage * sizeof(float));
    if (smem_max > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess)
      return set_error(HSC_ERR_CUDA, "shared memory attribute of the latent shading kernel");
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, BLOCK,
                                                      kLightTile * F4 * sizeof(float4) + kMatStage * sizeof(float)) !=
        cudaSuccess)
      o = 1;
    occ = o > 0 ? o : 1;
  }
  // waves > 0: persistent grid of waves x (resident CTAs per SM) x SMs striding
  // over the pixel tiles; waves == 0: one CTA per tile; waves < 0: one wave of
  // persistent CTAs on a dynamic tile queue.
  a.queue = nullptr;
  if (cfg.waves < 0) {
    // the counter pair is zero at context creation and reset by the last CTA
    if (!cfg.queue) return set_error(HSC_ERR_INVALID_ARG, "dynamic schedule without a queue");
    a.queue = cfg.queue;
  }
  int64_t grid = cfg.waves > 0 ? (int64_t)cfg.sm_count * occ * cfg.waves
                               : (cfg.waves < 0 ? (int64_t)cfg.sm_count * occ : a.tiles);
  if (grid > a.tiles) grid = a.tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, BLOCK, smem, stream>>>(a);
  return check_launch("shade_codes_kernel");
}

template <int KC, int PPT, bool SEC, int BLOCK, int VEC>
hsc_status launch_one(const ShadeArgs& a, const LaunchCfg& cfg, cudaStream_t stream) {
  return a.srgb8 ? launch_one_rgb<KC, PPT, SEC, BLOCK, VEC, true>(a, cfg, stream)
                 : launch_one_rgb<KC, PPT, SEC, BLOCK, VEC, false>(a, cfg, stream);
}

template <int KC, int BLOCK>
hsc_status launch_kc_block(const ShadeArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  if (cfg.vec == 2) {
    // paired points: with the bounce every PPT pairs up; without it PPT must be even
    switch (cfg.ppt) {
      case 1: return sec ? launch_one<KC, 1, true, BLOCK, 2>(a, cfg, s) : launch_one<KC, 2, false, BLOCK, 2>(a, cfg, s);
      case 4: return sec ? launch_one<KC, 4, true, BLOCK, 2>(a, cfg, s) : launch_one<KC, 4, false, BLOCK, 2>(a, cfg, s);
      default: return sec ? launch_one<KC, 2, true, BLOCK, 2>(a, cfg, s) : launch_one<KC, 2, false, BLOCK, 2>(a, cfg, s);
    }
  }
  switch (cfg.ppt) {
    case 1: return sec ? launch_one<KC, 1, true, BLOCK, 1>(a, cfg, s) : launch_one<KC, 1, false, BLOCK, 1>(a, cfg, s);
    case 4: return sec ? launch_one<KC, 4, true, BLOCK, 1>(a, cfg, s) : launch_one<KC, 4, false, BLOCK, 1>(a, cfg, s);
    default: return sec ? launch_one<KC, 2, true, BLOCK, 1>(a, cfg, s) : launch_one<KC, 2, false, BLOCK, 1>(a, cfg, s);
  }
}

}  // namespace

// Launches the KC-channel shading kernel in the configuration `cfg`
// (pixels per thread 1/2/4, 128 or 256 threads, persistent or one CTA per
// tile, scalar or f32x2-paired points).
template <int KC>
hsc_status launch_kc(const ShadeArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  return cfg.block == 256 ? launch_kc_block<KC, 256>(a, sec, cfg, s) : launch_kc_block<KC, 128>(a, sec, cfg, s);
}

}  // namespace hsc
