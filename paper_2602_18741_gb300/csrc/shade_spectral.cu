// Naive n-sample spectral shading: the paper's ground truth, whose cost grows
// in proportion to the number of wavelength samples (Sec. 1).  Same shading
// model and the same geometry_term instruction sequence as the latent
// kernels; per (pixel, light) it does the geometry term plus n FMAs instead
// of k.
//
// Mapping: a thread owns PTS shading points (PTS = 2: the primary and the
// secondary point of one pixel, or two pixels when there is no secondary
// G-buffer) and sweeps the spectrum in chunks of CW samples with CW FP32
// accumulators per point.  Lights and their (I/pi)-scaled SPDs are staged in
// shared memory; every broadcast float4 load of a light's spectrum feeds
// 4 * PTS FMAs, which keeps the shared-memory pipe below the FP32 pipe (with
// one point per thread the loads, one per four FMAs, saturate it).  Smaller
// chunks cost one geometry term per chunk but free registers for more
// resident warps; VEC = 2 keeps the accumulators in f32x2 pairs along
// wavelength.  The autotuner picks PTS, CW and VEC.  With the secondary point
// the radiance is
//     S = R1 (.) (A1 + h (R2 (.) A2)),  XYZ = T S fused.
#include "common.cuh"
#include "shade_latent.cuh"
#include "tune.cuh"

namespace hsc {

namespace {

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
  int npad;  // n rounded up to a whole number of channel chunks
  const float* T;  // 3 x n
  float* xyz;
  float* spectra;  // nullable, P x n
  unsigned int* err;
};

// Staged light record: one float4 (position) + npad / 4 float4s of the
// (I/pi)-scaled spectrum, zero beyond n.
__device__ __forceinline__ int spec_f4(const SpecArgs& a) { return 1 + a.npad / 4; }

// Staging loads each thread issues before it writes any of them to shared
// memory (every load of a batch has an in-range address and its value is
// selected afterwards), so a CTA waits for memory once per batch instead of
// once per staged value.  The prologue stages this way; restaging between
// light tiles inside the tile loop (BATCH = 1) loads one value at a time, so
// that no batch registers add to the live accumulators there.
constexpr int kSpecStageBatch = 8;

template <int BATCH>
__device__ __forceinline__ void stage_lights(const SpecArgs& a, float4* s_light, int l0, int nl) {
  float* s = reinterpret_cast<float*>(s_light);
  const int per = spec_f4(a) * 4;
  if constexpr (BATCH == 1) {
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
    return;
  }
  const int total = nl * per;
  for (int base = threadIdx.x; base < total; base += BATCH * (int)blockDim.x) {
    float v[BATCH];
#pragma unroll
    for (int q = 0; q < BATCH; ++q) {
      const int idx = min(base + q * (int)blockDim.x, total - 1);
      const int l = idx / per, j = idx - l * per;
      const int lg = l0 + l;
      const float pos = __ldg(a.lpos + 3 * lg + min(j, 2));
      const float sc = __fmul_rn(__ldg(a.linten + lg), kInvPi);
      const float x = __ldg(a.spd + (int64_t)lg * a.n + min(max(j - 4, 0), a.n - 1));
      v[q] = j < 3 ? pos : ((j >= 4 && j - 4 < a.n) ? __fmul_rn(x, sc) : 0.0f);
    }
#pragma unroll
    for (int q = 0; q < BATCH; ++q)
      if (base + q * (int)blockDim.x < total) s[base + q * (int)blockDim.x] = v[q];
  }
}

struct Pt {
  float x, y, z, nx, ny, nz;
};

__device__ __forceinline__ Pt load_pt(const float* pos, const float* nrm, int64_t p) {
  Pt q;
  q.x = __ldg(pos + 3 * p);
  q.y = __ldg(pos + 3 * p + 1);
  q.z = __ldg(pos + 3 * p + 2);
  q.nx = __ldg(nrm + 3 * p);
  q.ny = __ldg(nrm + 3 * p + 1);
  q.nz = __ldg(nrm + 3 * p + 2);
  return q;
}

// acc[q][i] += g(q, l) * V_l[c0 + i], i < CW, for PTS points over nl staged lights.
template <int CW, int PTS>
__device__ __forceinline__ void sweep(const float4* s_light, int f4, int c0, int nl, const Pt (&pt)[PTS],
                                      float (&acc)[PTS][CW]) {
#pragma unroll 1
  for (int l = 0; l < nl; ++l) {
    const float4* rec = s_light + l * f4;
    const float4 pl = rec[0];
    float g[PTS];
#pragma unroll
    for (int q = 0; q < PTS; ++q)
      g[q] = geometry_term(pt[q].x, pt[q].y, pt[q].z, pt[q].nx, pt[q].ny, pt[q].nz, pl.x, pl.y, pl.z);
    const float4* vv = rec + 1 + c0 / 4;
#pragma unroll
    for (int f = 0; f < CW / 4; ++f) {
      const float4 v = vv[f];
#pragma unroll
      for (int q = 0; q < PTS; ++q) {
        acc[q][4 * f + 0] = __fmaf_rn(g[q], v.x, acc[q][4 * f + 0]);
        acc[q][4 * f + 1] = __fmaf_rn(g[q], v.y, acc[q][4 * f + 1]);
        acc[q][4 * f + 2] = __fmaf_rn(g[q], v.z, acc[q][4 * f + 2]);
        acc[q][4 * f + 3] = __fmaf_rn(g[q], v.w, acc[q][4 * f + 3]);
      }
    }
  }
}

// The same sweep with the accumulators in f32x2 pairs along wavelength (one
// packed FMA per two samples; each half is the scalar FMA, bit for bit).
template <int CW, int PTS>
__device__ __forceinline__ void sweep_x2(const float4* s_light, int f4, int c0, int nl, const Pt (&pt)[PTS],
                                         f2 (&acc)[PTS][CW / 2]) {
#pragma unroll 1
  for (int l = 0; l < nl; ++l) {
    const float4* rec = s_light + l * f4;
    const float4 pl = rec[0];
    f2 g[PTS];
#pragma unroll
    for (int q = 0; q < PTS; ++q) {
      const float gs = geometry_term(pt[q].x, pt[q].y, pt[q].z, pt[q].nx, pt[q].ny, pt[q].nz, pl.x, pl.y, pl.z);
      g[q] = f2_pack(gs, gs);
    }
    const ulonglong2* vv = reinterpret_cast<const ulonglong2*>(rec + 1 + c0 / 4);
#pragma unroll
    for (int f = 0; f < CW / 4; ++f) {
      const ulonglong2 v = vv[f];
#pragma unroll
      for (int q = 0; q < PTS; ++q) {
        acc[q][2 * f + 0] = f2_fma(g[q], v.x, acc[q][2 * f + 0]);
        acc[q][2 * f + 1] = f2_fma(g[q], v.y, acc[q][2 * f + 1]);
      }
    }
  }
}

// Sweeps the lights for channels c0 .. c0+CW-1, restaging light tiles when
// they do not fit shared memory at once.  Called by every thread of the CTA.
template <int CW, int PTS, int VEC>
__device__ __forceinline__ void sweep_all(const SpecArgs& a, float4* s_light, bool staged, int c0,
                                          const Pt (&pt)[PTS], float (&acc)[PTS][CW]) {
  const int f4 = spec_f4(a);
  if constexpr (VEC == 2) {
    f2 acc2[PTS][CW / 2];
#pragma unroll
    for (int q = 0; q < PTS; ++q)
#pragma unroll
      for (int i = 0; i < CW / 2; ++i) acc2[q][i] = f2_pack(acc[q][2 * i], acc[q][2 * i + 1]);
    for (int l0 = 0; l0 < a.L; l0 += kSpecLightTile) {
      const int nl = min(kSpecLightTile, a.L - l0);
      if (!staged) {
        __syncthreads();
        stage_lights<1>(a, s_light, l0, nl);
        __syncthreads();
      }
      sweep_x2<CW, PTS>(s_light, f4, c0, nl, pt, acc2);
    }
#pragma unroll
    for (int q = 0; q < PTS; ++q)
#pragma unroll
      for (int i = 0; i < CW / 2; ++i) f2_unpack(acc2[q][i], acc[q][2 * i], acc[q][2 * i + 1]);
  } else {
    for (int l0 = 0; l0 < a.L; l0 += kSpecLightTile) {
      const int nl = min(kSpecLightTile, a.L - l0);
      if (!staged) {
        __syncthreads();
        stage_lights<1>(a, s_light, l0, nl);
        __syncthreads();
      }
      sweep<CW, PTS>(s_light, f4, c0, nl, pt, acc);
    }
  }
}

// Spectral radiance of channels c0 .. c0+CW-1 of one pixel from acc[i] =
// A1 + h (R2 (.) A2): S = R1 (.) acc, XYZ partial sums, optional spectrum.
template <int CW>
__device__ __forceinline__ void finish_chunk(const SpecArgs& a, int64_t p, bool valid, int m1, bool bad, int c0,
                                             const float (&acc)[CW], float& X, float& Y, float& Z) {
  const float* r1 = a.mats + (int64_t)(bad ? 0 : m1) * a.n;
#pragma unroll
  for (int j = 0; j < CW; ++j) {
    const int i = c0 + j;
    if (i < a.n) {
      const float S = bad ? 0.0f : __fmul_rn(__ldg(r1 + i), acc[j]);
      X = __fmaf_rn(__ldg(a.T + i), S, X);
      Y = __fmaf_rn(__ldg(a.T + a.n + i), S, Y);
      Z = __fmaf_rn(__ldg(a.T + 2 * a.n + i), S, Z);
      if (a.spectra && valid) a.spectra[p * a.n + i] = S;
    }
  }
}

// A thread owns PTS shading points: PTS = 2 is the primary and secondary point
// of one pixel (both sum every staged light together) or two pixels without a
// secondary G-buffer; PTS = 1 is one point, the secondary sweep running first.
// Channels are processed in chunks of CW (fewer registers, more resident
// warps; each chunk recomputes the geometry term).
template <int CW, bool SEC, int PTS, int BLOCK, int VEC>
__global__ void __launch_bounds__(BLOCK) shade_spectral_kernel(const SpecArgs a) {
  extern __shared__ float4 s_light[];
  const bool staged = a.L <= kSpecLightTile;
  if (staged) {
    stage_lights<kSpecStageBatch>(a, s_light, 0, a.L);
    __syncthreads();
  }
  constexpr int PXT = (PTS == 2 && !SEC) ? 2 : 1;  // pixels per thread
  const int64_t tiles = (a.P + (int64_t)BLOCK * PXT - 1) / ((int64_t)BLOCK * PXT);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    int64_t pix[PXT];
    bool valid[PXT];
    int m1[PXT];
    bool bad[PXT];
    Pt pt[PTS];
#pragma unroll
    for (int j = 0; j < PXT; ++j) {
      pix[j] = tile * (BLOCK * PXT) + (int64_t)j * BLOCK + threadIdx.x;
      valid[j] = pix[j] < a.P;
      const int64_t pc = valid[j] ? pix[j] : a.P - 1;
      m1[j] = __ldg(a.m1 + pc);
      bad[j] = (m1[j] < 0 || m1[j] >= a.n_mat);
      pt[j] = load_pt(a.x1, a.n1, pc);
    }
    int m2 = 0;
    bool bad2 = false;
    float h = 0.0f;
    Pt s2{};
    if (SEC) {
      const int64_t pc = valid[0] ? pix[0] : a.P - 1;
      s2 = load_pt(a.x2, a.n2, pc);
      m2 = __ldg(a.m2 + pc);
      bad2 = (m2 < 0 || m2 >= a.n_mat);
      bad[0] = bad[0] || bad2;
      h = bounce_term(pt[0].x, pt[0].y, pt[0].z, pt[0].nx, pt[0].ny, pt[0].nz, s2.x, s2.y, s2.z, s2.nx, s2.ny,
                      s2.nz);
      if (PTS == 2) pt[PTS - 1] = s2;
    }
    const float* r2 = a.mats + (int64_t)(bad2 ? 0 : m2) * a.n;
    float X[PXT], Y[PXT], Z[PXT];
#pragma unroll
    for (int j = 0; j < PXT; ++j) X[j] = Y[j] = Z[j] = 0.0f;
    for (int c0 = 0; c0 < a.npad; c0 += CW) {
      float acc[PTS][CW];
#pragma unroll
      for (int q = 0; q < PTS; ++q)
#pragma unroll
        for (int i = 0; i < CW; ++i) acc[q][i] = 0.0f;
      if (SEC && PTS == 1) {
        // secondary sweep first, then acc = h (R2 (.) A2)
        Pt one[1] = {s2};
        float a2[1][CW];
#pragma unroll
        for (int i = 0; i < CW; ++i) a2[0][i] = 0.0f;
        sweep_all<CW, 1, VEC>(a, s_light, staged, c0, one, a2);
#pragma unroll
        for (int i = 0; i < CW; ++i) {
          const float r = (c0 + i < a.n && !bad2) ? __ldg(r2 + c0 + i) : 0.0f;
          acc[0][i] = __fmul_rn(h, __fmul_rn(r, a2[0][i]));
        }
      }
      sweep_all<CW, PTS, VEC>(a, s_light, staged, c0, pt, acc);
      if (SEC && PTS == 2) {
        // A1 + h (R2 (.) A2)
#pragma unroll
        for (int i = 0; i < CW; ++i) {
          const float r = (c0 + i < a.n && !bad2) ? __ldg(r2 + c0 + i) : 0.0f;
          acc[0][i] = __fmaf_rn(h, __fmul_rn(r, acc[PTS - 1][i]), acc[0][i]);
        }
      }
      finish_chunk<CW>(a, pix[0], valid[0], m1[0], bad[0], c0, acc[0], X[0], Y[0], Z[0]);
      if (PXT == 2)
        finish_chunk<CW>(a, pix[PXT - 1], valid[PXT - 1], m1[PXT - 1], bad[PXT - 1], c0, acc[PTS - 1], X[PXT - 1],
                         Y[PXT - 1], Z[PXT - 1]);
    }
#pragma unroll
    for (int j = 0; j < PXT; ++j) {
      if (valid[j]) {
        a.xyz[3 * pix[j]] = X[j];
        a.xyz[3 * pix[j] + 1] = Y[j];
        a.xyz[3 * pix[j] + 2] = Z[j];
        if (bad[j]) atomicOr(a.err, HSC_DEVERR_MATERIAL);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Lane-group form.  Eight consecutive lanes own a group of 8 shading points
// (4 pixels with their secondary points, or 8 pixels) and hold a register tile
// of 8 points x TL wavelengths each: lane g accumulates samples g TL .. g TL +
// TL - 1 of all 8 points, acc[q][i] += G(q, l) V_l[g TL + i].  The last
// R = n - 8 TL samples (R < 8) each lane takes for its own point only, so no
// lane does padded work.  Per light each lane computes the geometry term of
// its own point once (the geometry term is per (point, light), not per
// sample), and the group reads the 8 terms back from a per-warp exchange row
// of shared memory, kLB lights at a time.  Lights are staged once per CTA when
// they fit one stage, so the tile loop has no block barrier.  The XYZ partial
// sums of the 8 lanes are added by a butterfly whose every lane ends with the
// same bits.  For every (point, wavelength) the lights are summed in the same
// order with the same FMAs as in the chunked form, so the spectra are the
// same bits; only the XYZ sum is grouped differently.
constexpr int kLB = 4;   // lights per geometry exchange
constexpr int kLT = 64;  // lights per stage

template <int TL, int R>
struct LaneShape {
  static constexpr int VS = (TL + 3) / 4 * 4;               // floats per group row (16-byte aligned)
  static constexpr bool INPAD = R > 0 && R <= VS - TL;      // remainder in every row's padding
  static constexpr int RS = INPAD ? 0 : (R + 3) / 4 * 4;    // floats of a separate remainder row
  static constexpr int VROW = 8 * VS + RS;                  // floats per staged spectrum
  static constexpr int ROFF = INPAD ? TL : 8 * VS;          // remainder offset (from the group row / row)
};

// Sample held at offset r of a staged row, or -1 for padding.
template <int TL, int R>
__device__ __forceinline__ int lane_row_sample(int r, int n) {
  using SH = LaneShape<TL, R>;
  int lam = -1;
  if (r < 8 * SH::VS) {
    const int g = r / SH::VS, j = r - g * SH::VS;
    if (j < TL) lam = g * TL + j;
    else if (SH::INPAD && j - TL < R) lam = 8 * TL + (j - TL);
  } else if (r - 8 * SH::VS < R) {
    lam = 8 * TL + (r - 8 * SH::VS);
  }
  return lam < n ? lam : -1;
}

// Stages lights l0 .. l0+nl-1 (positions and (I/pi)-scaled spectra) and pads
// the stage to a whole number of kLB lights with far-away dark lights
// (spectrum 0: every FMA with them adds +0 to a non-negative sum, which
// leaves it unchanged bit for bit).
template <int TL, int R, int BLOCK, int BATCH>
__device__ __forceinline__ void stage_lane_lights(const SpecArgs& a, float* s_V, float4* s_pos, int l0, int nl) {
  constexpr int VROW = LaneShape<TL, R>::VROW;
  const int npad = (nl + kLB - 1) / kLB * kLB;
  const int total = npad * VROW;
  if constexpr (BATCH == 1) {
    for (int i = threadIdx.x; i < total; i += BLOCK) {
      const int l = i / VROW, r = i - l * VROW, lam = lane_row_sample<TL, R>(r, a.n);
      float v = 0.0f;
      if (lam >= 0 && l < nl) {
        const float sc = __fmul_rn(__ldg(a.linten + l0 + l), kInvPi);
        v = __fmul_rn(__ldg(a.spd + (int64_t)(l0 + l) * a.n + lam), sc);
      }
      s_V[i] = v;
    }
  }
  for (int base = threadIdx.x; BATCH > 1 && base < total; base += BATCH * BLOCK) {
    float v[BATCH];
#pragma unroll
    for (int q = 0; q < BATCH; ++q) {
      const int i = min(base + q * BLOCK, total - 1);
      const int l = i / VROW, r = i - l * VROW, lam = lane_row_sample<TL, R>(r, a.n);
      const int lc = min(l, nl - 1);
      const float sc = __fmul_rn(__ldg(a.linten + l0 + lc), kInvPi);
      const float x = __ldg(a.spd + (int64_t)(l0 + lc) * a.n + max(lam, 0));
      v[q] = (lam >= 0 && l < nl) ? __fmul_rn(x, sc) : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < BATCH; ++q)
      if (base + q * BLOCK < total) s_V[base + q * BLOCK] = v[q];
  }
  for (int l = threadIdx.x; l < npad; l += BLOCK)
    s_pos[l] = l < nl ? make_float4(__ldg(a.lpos + 3 * (l0 + l)), __ldg(a.lpos + 3 * (l0 + l) + 1),
                                    __ldg(a.lpos + 3 * (l0 + l) + 2), 0.0f)
                      : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
}

// EXACT: n = 8 TL + R (no sample index reaches n); WS: spectra are written;
// ONE: every light fits one stage (L <= kLT), so the tile loop has no block
// barrier and no restaging (a separate instantiation: the compiler allocates
// its registers better without the restaging path).
template <int TL, int R, bool SEC, bool EXACT, bool WS, bool ONE>
__global__ void __launch_bounds__(128, TL <= 12 ? 4 : 2) shade_spectral_lanes_kernel(const SpecArgs a) {
  using SH = LaneShape<TL, R>;
  constexpr int BLOCK = 128;
  constexpr int VS = SH::VS;
  constexpr int VROW = SH::VROW;
  constexpr int RN = R > 0 ? R : 1;
  constexpr int QP = SEC ? 4 : 8;              // pixels per lane group
  constexpr int PX = 16 * QP;                  // pixels per CTA tile (16 lane groups)
  extern __shared__ float4 smem4[];
  float* s_V = reinterpret_cast<float*>(smem4);                 // kLT x VROW
  float4* s_pos = reinterpret_cast<float4*>(s_V + kLT * VROW);  // kLT
  float* s_T = reinterpret_cast<float*>(s_pos + kLT);           // 3 x VROW
  float* s_gx = s_T + 3 * VROW;                                 // 4 warps x kLB x 32
  const int tid = threadIdx.x, lane = tid & 31, grp = lane & 7;
  const int pg = tid >> 3;                     // lane group within the CTA
  for (int i = tid; i < 3 * VROW; i += BLOCK) {
    const int c = i / VROW, r = i - c * VROW, lam = lane_row_sample<TL, R>(r, a.n);
    s_T[i] = lam >= 0 ? __ldg(a.T + c * a.n + lam) : 0.0f;
  }
  if (ONE) stage_lane_lights<TL, R, BLOCK, kSpecStageBatch>(a, s_V, s_pos, 0, a.L);
  __syncthreads();
  float* gx = s_gx + (tid >> 5) * (kLB * 32);
  const float* vr = s_V + grp * VS;            // this lane's group row of light 0
  const float* tw = s_T + grp * VS;
  const float* vrem = SH::INPAD ? vr + SH::ROFF : s_V + SH::ROFF;
  const float* trem = SH::INPAD ? tw + SH::ROFF : s_T + SH::ROFF;
  // pixel indices fit 32 bits: the host splits frames whose P x max(n, 3)
  // would not (each launch then covers a slice of the frame)
  const int P = (int)a.P;
  const int tiles = (P + PX - 1) / PX;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int pix0 = tile * PX + pg * QP;      // first pixel of this lane group
    // this lane's shading point; lanes grp < QP also hold pixel grp's record
    const bool second = SEC && grp >= 4;
    const int mypix = pix0 + (SEC ? (grp & 3) : grp);
    const int pc = mypix < P ? mypix : P - 1;
    const Pt pt = second ? load_pt(a.x2, a.n2, pc) : load_pt(a.x1, a.n1, pc);
    int m1 = __ldg(a.m1 + pc), m2 = 0;
    bool bad = m1 < 0 || m1 >= a.n_mat;
    if (SEC) {
      m2 = __ldg(a.m2 + pc);
      bad = bad || m2 < 0 || m2 >= a.n_mat;
    }
    float h = 0.0f;
    if (SEC) {
      // the secondary point of pixel grp & 3 lives on lane grp + 4 of the group
      const float sx = __shfl_down_sync(0xffffffffu, pt.x, 4, 8), sy = __shfl_down_sync(0xffffffffu, pt.y, 4, 8);
      const float sz = __shfl_down_sync(0xffffffffu, pt.z, 4, 8), snx = __shfl_down_sync(0xffffffffu, pt.nx, 4, 8);
      const float sny = __shfl_down_sync(0xffffffffu, pt.ny, 4, 8), snz = __shfl_down_sync(0xffffffffu, pt.nz, 4, 8);
      if (grp < 4) h = bounce_term(pt.x, pt.y, pt.z, pt.nx, pt.ny, pt.nz, sx, sy, sz, snx, sny, snz);
    }
    float acc[8][TL];
    float accr[RN];                            // this lane's point, the last R samples
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int i = 0; i < TL; ++i) acc[q][i] = 0.0f;
#pragma unroll
    for (int r = 0; r < RN; ++r) accr[r] = 0.0f;
    // lights lb .. lb + nl - 1 of the staged tile, kLB at a time
    auto sweep_stage = [&](int nl) {
      for (int lb = 0; lb < nl; lb += kLB) {
        float gown[kLB];
        __syncwarp();
#pragma unroll
        for (int b = 0; b < kLB; ++b) {
          const float4 pl = s_pos[lb + b];
          gown[b] = geometry_term(pt.x, pt.y, pt.z, pt.nx, pt.ny, pt.nz, pl.x, pl.y, pl.z);
          gx[b * 32 + lane] = gown[b];
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < kLB; ++b) {
          const float4 ga = *reinterpret_cast<const float4*>(gx + b * 32 + (lane & ~7));
          const float4 gb = *reinterpret_cast<const float4*>(gx + b * 32 + (lane & ~7) + 4);
          const float gq[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
          const int l = lb + b;
#pragma unroll
          for (int f = 0; f < VS / 4; ++f) {
            const float4 t = *reinterpret_cast<const float4*>(vr + l * VROW + 4 * f);
            const float v[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i = 4 * f + e;
              if (i < TL) {
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q][i] = __fmaf_rn(gq[q], v[e], acc[q][i]);
              } else if (SH::INPAD && i - TL < R) {
                accr[i - TL] = __fmaf_rn(gown[b], v[e], accr[i - TL]);
              }
            }
          }
          if constexpr (R > 0) {
            if constexpr (!SH::INPAD) {
#pragma unroll
              for (int f = 0; f < SH::RS / 4; ++f) {
                const float4 t = *reinterpret_cast<const float4*>(vrem + l * VROW + 4 * f);
                const float w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                  if (4 * f + e < R) accr[4 * f + e] = __fmaf_rn(gown[b], w[e], accr[4 * f + e]);
              }
            }
          }
        }
      }
    };
    if constexpr (ONE) {
      // every light is staged: one sweep, no block barrier in the tile loop
      sweep_stage(a.L);
    } else {
      for (int l0 = 0; l0 < a.L; l0 += kLT) {
        const int nl = min(kLT, a.L - l0);
        __syncthreads();
        stage_lane_lights<TL, R, BLOCK, 1>(a, s_V, s_pos, l0, nl);
        __syncthreads();
        sweep_stage(nl);
      }
    }
    // the last R samples of this lane's pixel (lanes grp < QP); added below to
    // the lane's own partial sums of that pixel
    float rX = 0.0f, rY = 0.0f, rZ = 0.0f;
    if constexpr (R > 0) {
      const float* r1o = a.mats + (int64_t)(bad ? 0 : m1) * a.n;
      const float* r2o = a.mats + (int64_t)(bad ? 0 : m2) * a.n;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int lam = 8 * TL + r;
        float A = accr[r];
        if (SEC) {
          const float A2 = __shfl_down_sync(0xffffffffu, accr[r], 4, 8);
          A = __fmaf_rn(h, __fmul_rn(__ldg(r2o + lam), A2), A);
        }
        const float S = bad ? 0.0f : __fmul_rn(__ldg(r1o + lam), A);
        rX = __fmaf_rn(trem[r], S, rX);
        rY = __fmaf_rn(trem[VROW + r], S, rY);
        rZ = __fmaf_rn(trem[2 * VROW + r], S, rZ);
        if (WS && grp < QP && mypix < P) a.spectra[mypix * a.n + lam] = S;
      }
    }
    // radiance of the group's pixels over this lane's wavelengths; XYZ by butterfly
#pragma unroll
    for (int j = 0; j < QP; ++j) {
      const int jm1 = __shfl_sync(0xffffffffu, bad ? -1 : m1, j, 8);
      const int jm2 = __shfl_sync(0xffffffffu, bad ? 0 : m2, j, 8);
      const float jh = __shfl_sync(0xffffffffu, h, j, 8);
      const int pix = pix0 + j;
      const bool jbad = jm1 < 0;
      if (jbad && grp == j && pix < P) atomicOr(a.err, HSC_DEVERR_MATERIAL);
      const float* r1 = a.mats + (int64_t)(jbad ? 0 : jm1) * a.n + grp * TL;
      const float* r2 = a.mats + (int64_t)jm2 * a.n + grp * TL;
      float X = 0.0f, Y = 0.0f, Z = 0.0f;
#pragma unroll
      for (int i = 0; i < TL; ++i) {
        if (EXACT || grp * TL + i < a.n) {
          float A = acc[j][i];
          if (SEC) A = __fmaf_rn(jh, __fmul_rn(__ldg(r2 + i), acc[QP + j][i]), A);
          const float S = jbad ? 0.0f : __fmul_rn(__ldg(r1 + i), A);
          X = __fmaf_rn(tw[i], S, X);
          Y = __fmaf_rn(tw[VROW + i], S, Y);
          Z = __fmaf_rn(tw[2 * VROW + i], S, Z);
          if (WS && pix < P) a.spectra[pix * a.n + grp * TL + i] = S;
        }
      }
      if (R > 0 && grp == j) {
        X = __fadd_rn(X, rX);
        Y = __fadd_rn(Y, rY);
        Z = __fadd_rn(Z, rZ);
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        X = __fadd_rn(X, __shfl_xor_sync(0xffffffffu, X, o, 8));
        Y = __fadd_rn(Y, __shfl_xor_sync(0xffffffffu, Y, o, 8));
        Z = __fadd_rn(Z, __shfl_xor_sync(0xffffffffu, Z, o, 8));
      }
      if (grp == j && pix < P) {
        a.xyz[3 * pix] = X;
        a.xyz[3 * pix + 1] = Y;
        a.xyz[3 * pix + 2] = Z;
      }
    }
  }
}

template <int TL, int R, bool SEC, bool EXACT, bool WS, bool ONE>
hsc_status launch_lanes_t(const SpecArgs& a, const LaunchCfg& cfg, cudaStream_t s) {
  auto kern = shade_spectral_lanes_kernel<TL, R, SEC, EXACT, WS, ONE>;
  constexpr int VROW = LaneShape<TL, R>::VROW;
  static_assert(kLT % kLB == 0, "light stages hold whole exchange batches");
  const size_t smem = sizeof(float) * ((size_t)kLT * VROW + 4 * kLT + 3 * VROW + 4 * kLB * 32);
  static int occ = -1;
  if (occ < 0) {
    if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return set_error(HSC_ERR_CUDA, "shared memory attribute of the lane-group spectral kernel");
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, 128, smem) != cudaSuccess) o = 1;
    occ = o > 0 ? o : 1;
  }
  constexpr int PX = 16 * (SEC ? 4 : 8);
  // the kernel indexes pixels, 3 x pixels and pixels x n in 32 bits: a frame
  // beyond that is shaded in slices (every pixel is independent)
  const int64_t width = a.n > 3 ? a.n : 3;
  const int64_t slice = (INT32_MAX / width) / PX * PX;
  for (int64_t p0 = 0; p0 < a.P; p0 += slice) {
    SpecArgs c = a;
    c.P = a.P - p0 < slice ? a.P - p0 : slice;
    c.n1 = a.n1 + 3 * p0;
    c.x1 = a.x1 + 3 * p0;
    c.m1 = a.m1 + p0;
    if (SEC) {
      c.n2 = a.n2 + 3 * p0;
      c.x2 = a.x2 + 3 * p0;
      c.m2 = a.m2 + p0;
    }
    c.xyz = a.xyz + 3 * p0;
    if (WS) c.spectra = a.spectra + p0 * a.n;
    const int64_t tiles = (c.P + PX - 1) / PX;
    int64_t grid = cfg.waves > 0 ? (int64_t)cfg.sm_count * occ * cfg.waves : tiles;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, 128, smem, s>>>(c);
    HSC_TRY(check_launch("shade_spectral_lanes_kernel"));
  }
  return HSC_OK;
}

template <int TL, int R, bool SEC, bool EXACT, bool WS>
hsc_status launch_lanes_one(const SpecArgs& a, const LaunchCfg& cfg, cudaStream_t s) {
  return a.L <= kLT ? launch_lanes_t<TL, R, SEC, EXACT, WS, true>(a, cfg, s)
                    : launch_lanes_t<TL, R, SEC, EXACT, WS, false>(a, cfg, s);
}

template <int TL, int R, bool EXACT>
hsc_status launch_lanes_n(const SpecArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  const bool ws = a.spectra != nullptr;
  if (sec)
    return ws ? launch_lanes_one<TL, R, true, EXACT, true>(a, cfg, s) : launch_lanes_one<TL, R, true, EXACT, false>(a, cfg, s);
  return ws ? launch_lanes_one<TL, R, false, EXACT, true>(a, cfg, s) : launch_lanes_one<TL, R, false, EXACT, false>(a, cfg, s);
}

// n = 81 and n = 31 split exactly (8 x 10 + 1, 8 x 3 + 7); other n round up
// to 8 groups of TL samples.
hsc_status launch_lanes(const SpecArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  if (a.n == 81) return launch_lanes_n<10, 1, true>(a, sec, cfg, s);
  if (a.n == 31) return launch_lanes_n<3, 7, true>(a, sec, cfg, s);
  if (a.n <= 32) return launch_lanes_n<4, 0, false>(a, sec, cfg, s);
  if (a.n <= 88) return launch_lanes_n<11, 0, false>(a, sec, cfg, s);
  return launch_lanes_n<16, 0, false>(a, sec, cfg, s);
}

template <int CW, bool SEC, int PTS, int BLOCK, int VEC>
hsc_status launch_spec(const SpecArgs& a0, const LaunchCfg& cfg, cudaStream_t s) {
  SpecArgs a = a0;
  a.npad = (a.n + CW - 1) / CW * CW;
  auto kern = shade_spectral_kernel<CW, SEC, PTS, BLOCK, VEC>;
  const int f4 = 1 + a.npad / 4;
  const size_t smem = (size_t)min(a.L, kSpecLightTile) * f4 * sizeof(float4);
  const size_t smem_max = (size_t)kSpecLightTile * (1 + (HSC_MAX_N + CW - 1) / CW * CW / 4) * sizeof(float4);
  static int occ = -1;
  if (occ < 0) {
    if (smem_max > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, BLOCK, smem) != cudaSuccess) o = 1;
    occ = o > 0 ? o : 1;
  }
  constexpr int PXT = (PTS == 2 && !SEC) ? 2 : 1;
  const int64_t tiles = (a.P + (int64_t)BLOCK * PXT - 1) / ((int64_t)BLOCK * PXT);
  int64_t grid = cfg.waves > 0 ? (int64_t)cfg.sm_count * occ * cfg.waves : tiles;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, BLOCK, smem, s>>>(a);
  return check_launch("shade_spectral_kernel");
}

template <int CW, int VEC>
hsc_status launch_spec_vec(const SpecArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  if (cfg.ppt == 2)
    return sec ? launch_spec<CW, true, 2, 128, VEC>(a, cfg, s) : launch_spec<CW, false, 2, 128, VEC>(a, cfg, s);
  return sec ? launch_spec<CW, true, 1, 128, VEC>(a, cfg, s) : launch_spec<CW, false, 1, 128, VEC>(a, cfg, s);
}

template <int CW>
hsc_status launch_spec_cw(const SpecArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  return cfg.vec == 2 ? launch_spec_vec<CW, 2>(a, sec, cfg, s) : launch_spec_vec<CW, 1>(a, sec, cfg, s);
}

// Channel chunk of a configuration: cfg.chunk, or by default the whole
// spectrum up to 84 samples (32 for n <= 32), else chunks of 44.
int spectral_chunk(const LaunchCfg& cfg, int n) {
  if (cfg.chunk > 0) return cfg.chunk;
  return n <= 32 ? 32 : (n <= 84 ? 84 : 44);
}

hsc_status launch_spectral(const SpecArgs& a, bool sec, const LaunchCfg& cfg, cudaStream_t s) {
  if (cfg.chunk == 1) return launch_lanes(a, sec, cfg, s);
  switch (spectral_chunk(cfg, a.n)) {
    case 16: return launch_spec_cw<16>(a, sec, cfg, s);
    case 28: return launch_spec_cw<28>(a, sec, cfg, s);
    case 32: return launch_spec_cw<32>(a, sec, cfg, s);
    case 44: return launch_spec_cw<44>(a, sec, cfg, s);
    default: return launch_spec_cw<84>(a, sec, cfg, s);
  }
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
  const hsc::TuneKey key = hsc::make_tune_key(hsc::kTuneSpectral, n, sec, lights->count, pixels, 0);
  auto launch = [&](const hsc::LaunchCfg& c) { return hsc::launch_spectral(a, sec, c, s); };
  hsc::LaunchCfg cfg;
  HSC_TRY(hsc::tuned_cfg(ctx, key, hsc::spectral_candidates(ctx), launch, s, &cfg));
  return launch(cfg);
}
