// Path tracing with per-channel throughput: the renderer the paper uses for
// its latent images (Sec. 6), where every spectrum is replaced by its code and
// each surface interaction multiplies the path throughput by the material's
// code with the blockwise product (Eq. 6).  With C = n channels and spectra
// the same kernel is the naive spectral path tracer; with C = k and codes it
// is the latent one.  The paths do not depend on the channels, so both modes
// trace the same paths and differ only in the per-channel work, C multiplies
// per reflection and 3C FMAs to XYZ per path that meets the emitter.
//
// Scene: axis-aligned rectangles (one or more of them emitters) and spheres,
// Lambertian reflection with cosine-weighted sampling (the estimator weight
// of a reflection is the reflectance itself), no Russian roulette, at most
// `depth` reflections.  One thread per pixel loops over its samples.
//
// The geometry is IEEE float32 with every operation rounded to nearest in a
// fixed order (explicit __fadd_rn / __fmul_rn / __fdiv_rn / __fsqrt_rn, no
// contraction into FMAs), random numbers come from Philox4x32-10 (Salmon et
// al., SC'11) with counter (pixel, sample, vertex, 0) and key (seed, 0), the
// bounce direction from r = sqrt(u1), phi = 2 pi u2 with sin/cos of phi from
// Taylor polynomials on a quarter turn, and the tangent frame from the
// branchless construction of Duff et al. (JCGT 2017), so that the paths are
// reproducible bit for bit by any IEEE float32 implementation of the same
// steps.
#include "common.cuh"

namespace hsc {

namespace {

constexpr int kPTBlock = 128;
constexpr int kPTMaxQuads = 32;
constexpr int kPTMaxSpheres = 32;
constexpr int kPTMaxDepth = 16;

struct PTArgs {
  const float* quads;    // nq x 8: axis, c, u0, u1, v0, v1, normal sign, material (-1 = emitter)
  int nq;
  const float* spheres;  // ns x 5: cx, cy, cz, r, material
  int ns;
  const float* cam;      // 4 x 3: origin, lower-left, horizontal, vertical
  int width, height, spp, depth;
  uint32_t seed;
  const float* mats;     // n_mat x C reflectances (or their codes)
  int n_mat;
  const float* emit;     // C
  int C;
  const float* to_xyz;   // 3 x C
  float* xyz;            // P x 3
  float* chan;           // P x C pixel means of the channels (nullable, C <= 16)
  unsigned int* err;
};

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float bits(uint32_t u) { return __uint_as_float(u); }

// Philox4x32 with 10 rounds (multipliers 0xD2511F53 and 0xCD9E8D57, key
// increments 0x9E3779B9 and 0xBB67AE85).
__device__ __forceinline__ void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                       uint32_t (&out)[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// top 24 bits times 2^-24: exact, in [0, 1)
__device__ __forceinline__ float u01(uint32_t x) { return fmul(__uint2float_rn(x >> 8), bits(0x33800000u)); }

// sin and cos of 2 pi u: quadrant q = floor(4u), angle (4u - q) pi/2 on Taylor
// polynomials (coefficients 1/3!, 1/5!, ... and 1/2!, 1/4!, ... rounded to
// float32), rotated by q.
__device__ __forceinline__ void sincos_turn(float u, float& sn, float& cs) {
  const float x4 = fmul(u, 4.0f);
  const float qf = floorf(x4);
  const int q = (int)qf;
  const float th = fmul(fsub(x4, qf), bits(0x3FC90FDBu));
  const float t2 = fmul(th, th);
  float s = fsub(bits(0x3638EF1Du), fmul(t2, bits(0x32D7322Bu)));
  s = fsub(bits(0x39500D01u), fmul(t2, s));
  s = fsub(bits(0x3C088889u), fmul(t2, s));
  s = fsub(bits(0x3E2AAAABu), fmul(t2, s));
  s = fsub(1.0f, fmul(t2, s));
  s = fmul(th, s);
  float c = fsub(bits(0x3493F27Eu), fmul(t2, bits(0x310F76C7u)));
  c = fsub(bits(0x37D00D01u), fmul(t2, c));
  c = fsub(bits(0x3AB60B61u), fmul(t2, c));
  c = fsub(bits(0x3D2AAAABu), fmul(t2, c));
  c = fsub(0.5f, fmul(t2, c));
  c = fsub(1.0f, fmul(t2, c));
  sn = q == 0 ? s : (q == 1 ? c : (q == 2 ? -s : -c));
  cs = q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}

struct Hit {
  float t;
  int kind;  // 0 rectangle, 1 sphere, -1 none
  int idx;
};

// Nearest hit with t > 1e-4 over the rectangles, then the spheres, in order.
__device__ __forceinline__ Hit intersect(const float* sq, int nq, const float* ss, int ns, const float (&o)[3],
                                         const float (&d)[3]) {
  const float tmin = bits(0x38D1B717u);
  Hit h{__int_as_float(0x7F800000), -1, -1};
  for (int i = 0; i < nq; ++i) {
    const float* q = sq + 8 * i;
    const int ax = (int)q[0];
    const int ua = ax == 0 ? 1 : 0, va = ax == 2 ? 1 : 2;
    const float t = fdiv(fsub(q[1], o[ax]), d[ax]);
    const float pu = fadd(o[ua], fmul(t, d[ua]));
    const float pv = fadd(o[va], fmul(t, d[va]));
    if (t > tmin && t < h.t && pu >= q[2] && pu <= q[3] && pv >= q[4] && pv <= q[5]) {
      h.t = t;
      h.kind = 0;
      h.idx = i;
    }
  }
  for (int i = 0; i < ns; ++i) {
    const float* s = ss + 5 * i;
    const float ocx = fsub(o[0], s[0]), ocy = fsub(o[1], s[1]), ocz = fsub(o[2], s[2]);
    const float A = fadd(fadd(fmul(d[0], d[0]), fmul(d[1], d[1])), fmul(d[2], d[2]));
    const float B = fadd(fadd(fmul(ocx, d[0]), fmul(ocy, d[1])), fmul(ocz, d[2]));
    const float Cc = fsub(fadd(fadd(fmul(ocx, ocx), fmul(ocy, ocy)), fmul(ocz, ocz)), fmul(s[3], s[3]));
    const float disc = fsub(fmul(B, B), fmul(A, Cc));
    if (disc >= 0.0f) {
      const float sqd = __fsqrt_rn(disc);
      const float t0 = fdiv(fsub(-B, sqd), A);
      const float t1 = fdiv(fadd(-B, sqd), A);
      const float t = t0 > tmin ? t0 : t1;
      if (t > tmin && t < h.t) {
        h.t = t;
        h.kind = 1;
        h.idx = i;
      }
    }
  }
  return h;
}

__global__ void __launch_bounds__(kPTBlock) pathtrace_kernel(const PTArgs a) {
  extern __shared__ float sm[];
  float* sq = sm;                          // nq x 8
  float* ss = sq + 8 * a.nq;               // ns x 5
  float* sc = ss + 5 * a.ns;               // 12
  float* smat = sc + 12;                   // n_mat x C
  float* semit = smat + a.n_mat * a.C;     // C
  float* sx = semit + a.C;                 // 3 x C
  for (int i = threadIdx.x; i < 8 * a.nq; i += blockDim.x) sq[i] = a.quads[i];
  for (int i = threadIdx.x; i < 5 * a.ns; i += blockDim.x) ss[i] = a.spheres[i];
  for (int i = threadIdx.x; i < 12; i += blockDim.x) sc[i] = a.cam[i];
  for (int i = threadIdx.x; i < a.n_mat * a.C; i += blockDim.x) smat[i] = a.mats[i];
  for (int i = threadIdx.x; i < a.C; i += blockDim.x) semit[i] = a.emit[i];
  for (int i = threadIdx.x; i < 3 * a.C; i += blockDim.x) sx[i] = a.to_xyz[i];
  __syncthreads();

  const float offset = bits(0x3A83126Fu);
  const int64_t P = (int64_t)a.width * a.height;
  const float fw = (float)a.width, fh = (float)a.height;
  for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < P; pix += (int64_t)gridDim.x * blockDim.x) {
    const float px = (float)(pix % a.width), py = (float)(pix / a.width);
    float X = 0.0f, Y = 0.0f, Z = 0.0f;
    float ch[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) ch[c] = 0.0f;
    bool bad = false;
    for (int s = 0; s < a.spp; ++s) {
      uint32_t r[4];
      philox((uint32_t)pix, (uint32_t)s, 0u, 0u, a.seed, 0u, r);
      const float fx = fdiv(fadd(px, u01(r[0])), fw);
      const float fy = fdiv(fadd(py, u01(r[1])), fh);
      float o[3] = {sc[0], sc[1], sc[2]};
      float d[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) d[i] = fsub(fadd(fadd(sc[3 + i], fmul(fx, sc[6 + i])), fmul(fy, sc[9 + i])), sc[i]);
      int end = -1;
      uint32_t mpack[kPTMaxDepth / 4] = {0u, 0u, 0u, 0u};
      for (int v = 0; v <= a.depth; ++v) {
        const Hit h = intersect(sq, a.nq, ss, a.ns, o, d);
        if (h.kind < 0) break;
        if (h.kind == 0 && sq[8 * h.idx + 7] < 0.0f) {
          end = v;
          break;
        }
        if (v == a.depth) break;
        float hp[3], n[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) hp[i] = fadd(o[i], fmul(h.t, d[i]));
        int mat;
        if (h.kind == 0) {
          const float* q = sq + 8 * h.idx;
          const int ax = (int)q[0];
          n[0] = ax == 0 ? q[6] : 0.0f;
          n[1] = ax == 1 ? q[6] : 0.0f;
          n[2] = ax == 2 ? q[6] : 0.0f;
          mat = (int)q[7];
        } else {
          const float* sp = ss + 5 * h.idx;
#pragma unroll
          for (int i = 0; i < 3; ++i) n[i] = fdiv(fsub(hp[i], sp[i]), sp[3]);
          mat = (int)sp[4];
        }
        if (mat < 0 || mat >= a.n_mat) {
          bad = true;
          mat = 0;
        }
        mpack[v >> 2] |= (uint32_t)mat << (8 * (v & 3));
        philox((uint32_t)pix, (uint32_t)s, (uint32_t)(v + 1), 0u, a.seed, 0u, r);
        const float u1 = u01(r[2]), u2 = u01(r[3]);
        const float rad = __fsqrt_rn(u1);
        float sn, cs;
        sincos_turn(u2, sn, cs);
        const float lx = fmul(rad, cs), ly = fmul(rad, sn), lz = __fsqrt_rn(fsub(1.0f, u1));
        // tangent frame (Duff et al. 2017)
        const float sign = n[2] >= 0.0f ? 1.0f : -1.0f;
        const float aa = fdiv(-1.0f, fadd(sign, n[2]));
        const float bb = fmul(fmul(n[0], n[1]), aa);
        const float b1[3] = {fadd(1.0f, fmul(fmul(sign, fmul(n[0], n[0])), aa)), fmul(sign, bb), -fmul(sign, n[0])};
        const float b2[3] = {bb, fadd(sign, fmul(fmul(n[1], n[1]), aa)), -n[1]};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          d[i] = fadd(fadd(fmul(lx, b1[i]), fmul(ly, b2[i])), fmul(lz, n[i]));
          o[i] = fadd(hp[i], fmul(offset, n[i]));
        }
      }
      if (end < 0) continue;
      // per-channel throughput of the path, then its XYZ
      auto channel = [&](int c) {
        float t = semit[c];
        for (int j = 0; j < end; ++j) {
          const int m = (int)((mpack[j >> 2] >> (8 * (j & 3))) & 0xFFu);
          t = fmul(t, smat[m * a.C + c]);
        }
        X = __fmaf_rn(sx[c], t, X);
        Y = __fmaf_rn(sx[a.C + c], t, Y);
        Z = __fmaf_rn(sx[2 * a.C + c], t, Z);
        return t;
      };
      if (a.C <= 16) {  // codes: the channel sums stay in registers
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c < a.C) ch[c] = fadd(ch[c], channel(c));
      } else {
        for (int c = 0; c < a.C; ++c) channel(c);
      }
    }
    const float inv = fdiv(1.0f, (float)a.spp);
    a.xyz[3 * pix + 0] = fmul(X, inv);
    a.xyz[3 * pix + 1] = fmul(Y, inv);
    a.xyz[3 * pix + 2] = fmul(Z, inv);
    if (a.chan) {
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < a.C) a.chan[pix * a.C + c] = fmul(ch[c], inv);
    }
    if (bad) atomicOr(a.err, HSC_DEVERR_MATERIAL);
  }
}

}  // namespace

}  // namespace hsc

extern "C" hsc_status hsc_path_trace(hsc_ctx* ctx, const float* quads, int n_quads, const float* spheres,
                                     int n_spheres, const float* camera, int width, int height, int spp, int depth,
                                     uint32_t seed, const float* materials, int n_mat, const float* emit,
                                     int channels, const float* to_xyz, float* xyz_out, float* channels_out,
                                     void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(width >= 0 && height >= 0, "negative image size");
  HSC_REQUIRE(spp >= 1 && depth >= 0 && depth <= hsc::kPTMaxDepth, "spp >= 1 and 0 <= depth <= %d required",
              hsc::kPTMaxDepth);
  HSC_REQUIRE(n_quads >= 0 && n_quads <= hsc::kPTMaxQuads && n_spheres >= 0 && n_spheres <= hsc::kPTMaxSpheres,
              "at most %d rectangles and %d spheres", hsc::kPTMaxQuads, hsc::kPTMaxSpheres);
  HSC_REQUIRE(n_mat >= 1 && n_mat <= 255, "n_mat=%d out of range [1, 255]", n_mat);
  HSC_REQUIRE(channels >= 1 && channels <= HSC_MAX_N, "channels=%d out of range", channels);
  HSC_REQUIRE(!channels_out || channels <= 16, "per-pixel channel output needs channels <= 16");
  HSC_REQUIRE((n_quads == 0 || quads) && (n_spheres == 0 || spheres) && camera && materials && emit && to_xyz,
              "null pointer");
  const int64_t P = (int64_t)width * height;
  if (P == 0) return HSC_OK;
  HSC_REQUIRE(xyz_out, "null xyz_out");
  HSC_GUARD(ctx);
  hsc::PTArgs a{};
  a.quads = quads;
  a.nq = n_quads;
  a.spheres = spheres;
  a.ns = n_spheres;
  a.cam = camera;
  a.width = width;
  a.height = height;
  a.spp = spp;
  a.depth = depth;
  a.seed = seed;
  a.mats = materials;
  a.n_mat = n_mat;
  a.emit = emit;
  a.C = channels;
  a.to_xyz = to_xyz;
  a.xyz = xyz_out;
  a.chan = channels_out;
  a.err = ctx->d_err;
  const size_t smem = sizeof(float) * (8 * n_quads + 5 * n_spheres + 12 + (size_t)n_mat * channels + 4 * channels);
  HSC_REQUIRE(smem <= 48 * 1024, "scene tables of %zu bytes exceed 48 KB", smem);
  int64_t grid = (P + hsc::kPTBlock - 1) / hsc::kPTBlock;
  if (grid > (int64_t)ctx->sm_count * 16) grid = (int64_t)ctx->sm_count * 16;
  hsc::pathtrace_kernel<<<(unsigned)grid, hsc::kPTBlock, smem, hsc::as_stream(stream)>>>(a);
  return hsc::check_launch("pathtrace_kernel");
}
