// Latent (k-code) deferred shading: the k/3 RGB passes of Fig. 2b, their
// reassembly, and the fused single-launch k-channel form.
//
// Per pixel and per light the work is one geometry term g (13 FP32 ops + one
// MUFU rsqrt) and KC FMAs acc[c] += g * v_l[c], where v_l = (I_l / pi) * E(spd_l)
// is the light's scaled code.  After the light loop the blockwise Hadamard
// product with the material codes (Eq. 5, element-wise on R^k) and the
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
// grid is persistent (a multiple of the SM count) and strides over pixel tiles.
#include "common.cuh"
#include "shade_latent.cuh"

namespace hsc {

namespace {

template <int KC, int PPT, bool SEC, int BLOCK>
__global__ void __launch_bounds__(BLOCK) shade_codes_kernel(const ShadeArgs a) {
  constexpr int F4 = (3 + KC + 3) / 4;  // float4s per staged light: pos xyz + KC scaled code values
  constexpr int NPT = PPT * (SEC ? 2 : 1);
  extern __shared__ float4 s_light[];
  const int tid = threadIdx.x;
  const bool multi_tile = a.L > kLightTile;

  auto stage = [&](int l0, int nl) {
    float* s = reinterpret_cast<float*>(s_light);
    constexpr int per = F4 * 4;
    for (int idx = tid; idx < nl * per; idx += BLOCK) {
      const int l = idx / per, j = idx - l * per;
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
  };

  if (!multi_tile) {
    stage(0, a.L);
    __syncthreads();
  }

  for (int64_t tile = blockIdx.x; tile < a.tiles; tile += gridDim.x) {
    float px[NPT], py[NPT], pz[NPT], nx[NPT], ny[NPT], nz[NPT];
    int64_t pix[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int64_t p = tile * (BLOCK * PPT) + (int64_t)j * BLOCK + tid;
      pix[j] = p;
      const int64_t pc = p < a.P ? p : a.P - 1;
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
    float acc[NPT][KC];
#pragma unroll
    for (int q = 0; q < NPT; ++q)
#pragma unroll
      for (int c = 0; c < KC; ++c) acc[q][c] = 0.0f;

    for (int l0 = 0; l0 < a.L; l0 += kLightTile) {
      const int nl = min(kLightTile, a.L - l0);
      if (multi_tile) {
        __syncthreads();
        stage(l0, nl);
        __syncthreads();
      }
#pragma unroll 2
      for (int l = 0; l < nl; ++l) {
        float v[F4 * 4];
#pragma unroll
        for (int f = 0; f < F4; ++f) {
          const float4 t = s_light[l * F4 + f];
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

    // Epilogue: blockwise Hadamard product with the material codes + bounce.
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int64_t p = pix[j];
      const bool valid = p < a.P;
      const int64_t pc = valid ? p : a.P - 1;
      int m1 = __ldg(a.m1 + pc);
      bool bad = (m1 < 0 || m1 >= a.n_mat);
      float zr1[KC], out[KC];
#pragma unroll
      for (int c = 0; c < KC; ++c) zr1[c] = bad ? 0.0f : load_code(a.mat_codes, a.code_dt, (int64_t)m1 * a.k + a.c0 + c);
      if (SEC) {
        const int m2 = __ldg(a.m2 + pc);
        const bool bad2 = (m2 < 0 || m2 >= a.n_mat);
        bad = bad || bad2;
        const float h = bounce_term(px[j], py[j], pz[j], nx[j], ny[j], nz[j], px[PPT + j], py[PPT + j],
                                    pz[PPT + j], nx[PPT + j], ny[PPT + j], nz[PPT + j]);
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          const float zr2 = bad2 ? 0.0f : load_code(a.mat_codes, a.code_dt, (int64_t)m2 * a.k + a.c0 + c);
          out[c] = __fmul_rn(zr1[c], __fmaf_rn(h, __fmul_rn(zr2, acc[PPT + j][c]), acc[j][c]));
        }
      } else {
#pragma unroll
        for (int c = 0; c < KC; ++c) out[c] = __fmul_rn(zr1[c], acc[j][c]);
      }
      if (valid && bad) atomicOr(a.err, HSC_DEVERR_MATERIAL);
      if (valid) {
        float* o = a.out + p * a.out_stride + a.out_c0;
#pragma unroll
        for (int c = 0; c < KC; ++c) o[c] = out[c];
        if (a.xyz) {
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            float s = 0.0f;
#pragma unroll
            for (int c = 0; c < KC; ++c) s = __fmaf_rn(__ldg(a.M + r * a.k + c), out[c], s);
            a.xyz[3 * p + r] = s;
          }
        }
      }
      if (a.chan_max) {
        // non-negative floats order like their bit patterns
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          const unsigned int bits = valid ? __float_as_uint(fmaxf(out[c], 0.0f)) : 0u;
          const unsigned int mx = __reduce_max_sync(0xffffffffu, bits);
          if ((tid & 31) == 0 && mx) atomicMax(a.chan_max + a.c0 + c, mx);
        }
      }
    }
  }
}

template <int KC, int PPT, bool SEC>
hsc_status launch_one(const ShadeArgs& a0, const LaunchCfg& cfg, cudaStream_t stream) {
  constexpr int BLOCK = kShadeBlock;
  constexpr int F4 = (3 + KC + 3) / 4;
  ShadeArgs a = a0;
  a.tiles = (a.P + (int64_t)BLOCK * PPT - 1) / ((int64_t)BLOCK * PPT);
  const size_t smem = (size_t)min(a.L, kLightTile) * F4 * sizeof(float4);
  auto kern = shade_codes_kernel<KC, PPT, SEC, BLOCK>;
  static int occ = -1;
  if (occ < 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, BLOCK, kLightTile * F4 * sizeof(float4)) != cudaSuccess)
      o = 1;
    occ = o > 0 ? o : 1;
  }
  int64_t grid = (int64_t)cfg.sm_count * occ * (cfg.waves > 0 ? cfg.waves : 1);
  if (grid > a.tiles) grid = a.tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, BLOCK, smem, stream>>>(a);
  return check_launch("shade_codes_kernel");
}

template <int KC>
hsc_status launch_kc(const ShadeArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  switch (cfg.ppt) {
    case 1: return sec ? launch_one<KC, 1, true>(a, cfg, s) : launch_one<KC, 1, false>(a, cfg, s);
    case 4: return sec ? launch_one<KC, 4, true>(a, cfg, s) : launch_one<KC, 4, false>(a, cfg, s);
    default: return sec ? launch_one<KC, 2, true>(a, cfg, s) : launch_one<KC, 2, false>(a, cfg, s);
  }
}

}  // namespace

hsc_status launch_shade_codes(const ShadeArgs& a, int kc, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  switch (kc) {
    case 3: return launch_kc<3>(a, sec, cfg, s);
    case 6: return launch_kc<6>(a, sec, cfg, s);
    case 9: return launch_kc<9>(a, sec, cfg, s);
    case 12: return launch_kc<12>(a, sec, cfg, s);
    case 15: return launch_kc<15>(a, sec, cfg, s);
    default: return set_error(HSC_ERR_UNSUPPORTED, "channel chunk %d not instantiated", kc);
  }
}

namespace {

struct PassPtrs {
  const float* p[HSC_MAX_K / 3];
};

__global__ void reassemble_kernel(PassPtrs pp, int B, int64_t P, float* __restrict__ out) {
  const int k = 3 * B;
  const int64_t total = P * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx / k;
    const int c = (int)(idx - p * k);
    const int b = c / 3;
    out[idx] = __ldg(pp.p[b] + 3 * p + (c - 3 * b));
  }
}

}  // namespace

hsc_status launch_reassemble(const float* const* passes, int B, int64_t P, float* out, int sm_count,
                             cudaStream_t s) {
  PassPtrs pp;
  for (int b = 0; b < B; ++b) pp.p[b] = passes[b];
  const int64_t total = P * 3 * B;
  int64_t grid = (total + 255) / 256;
  const int64_t cap = (int64_t)sm_count * 8;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  reassemble_kernel<<<(unsigned)grid, 256, 0, s>>>(pp, B, P, out);
  return check_launch("reassemble_kernel");
}

LaunchCfg default_cfg(const hsc_ctx* ctx) {
  LaunchCfg c;
  c.sm_count = ctx->sm_count;
  c.ppt = 2;
  c.waves = 1;
  return c;
}

}  // namespace hsc
