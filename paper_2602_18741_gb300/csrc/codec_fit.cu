// Batched codec fitting: one Adam step of the paper's parameterisation
// (E = softplus(E~), D = softplus(D~) with beta = 10, Sec. 4.1) on the Eq. 8
// loss, for many hyper-parameter variants at once (the selection sweep of
// Sec. 4.5).  One CTA per variant; all variants share the mini-batch.
//
// Per variant the loss needs, per pair p of the batch (R_p, L_p, Y_p = R_p (.)
// L_p): zR = E R_p, zL = E L_p, zRL = zR (.) zL (Eq. 6), S = D zRL, and for
// the reconstruction term D zR, D zL; the cosine in L_e2e and the batch MSE
// couple the pairs only through scalars.  So the kernel runs
//   A. E, D from the raw parameters; zR, zL, E Y for every pair (dot
//      products over the n samples), kept in shared memory;
//   B. per pair (a warp per pair, lanes over samples): the loss sums and the
//      per-pair scalars |S|, |Y|, cos, (S - Y) T^T; fixed-order reductions;
//   C. per pair again: dL/dS from the batch scalars, then the chain rule to
//      dL/dD, dL/dzRL, dL/dzR, dL/dzL and dL/dE, accumulated in per-warp
//      copies of the gradient that are summed in warp order (deterministic);
//   D. the softplus chain rule and the Adam update of every parameter.
// The loss terms written are those at the parameters before the step.  The
// same kernel in evaluation mode stops after B (validation losses, and E, D
// for the selection stage); variants whose `active` flag is 0 return at once.
// hsc_codec_fit_track keeps the early-stopping state of every variant
// (Sec. 4.5: best validation loss, epochs without improvement, the best
// parameters) and counts the variants still training.
#include "common.cuh"

namespace hsc {

namespace {

constexpr int kFitThreads = 256;
constexpr int kFitWarps = kFitThreads / 32;
constexpr int kFitMaxK = 15;
constexpr int kFitMaxN = 128;
constexpr int kFitMaxP = 256;

struct FitArgs {
  int V, k, n, P;
  const float* R_all;   // rows of reflectances (n each)
  const float* L_all;   // rows of lights
  const int* pair_r;    // P
  const int* pair_l;    // P
  const float* pair_scale;  // P
  const float* T;       // 3 x n
  const float* w;       // V x 4: e2e, rec, code, col
  float* Et;            // V x k x n
  float* Dt;            // V x n x k
  float* mE;
  float* vE;
  float* mD;
  float* vD;
  int t;                // 1-based step number (bias correction)
  float lr, b1, b2, eps, beta;
  float* losses;        // V x 5: total, e2e, rec, code, col (nullable)
  float* grad;          // V x (k n + n k): dL/dE~ then dL/dD~ (nullable)
  const int32_t* active;  // V flags (nullable): 0 = variant skipped
  int eval_only;        // 1: losses (and E, D) only, no update
  float* E_out;         // V x k x n softplus(E~) (evaluation mode, nullable)
  float* D_out;         // V x n x k softplus(D~) (evaluation mode, nullable)
};

__device__ __forceinline__ float softplus_f(float x, float beta) {
  const float bx = beta * x;
  return (fmaxf(bx, 0.0f) + log1pf(expf(-fabsf(bx)))) / beta;
}

__device__ __forceinline__ float sigmoid_f(float x) {
  const float e = expf(-fabsf(x));
  return x >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Row p of the batch: R_p and the scaled light L_p at sample i.
__device__ __forceinline__ float batch_r(const FitArgs& a, int p, int i) {
  return __ldg(a.R_all + (int64_t)__ldg(a.pair_r + p) * a.n + i);
}
__device__ __forceinline__ float batch_l(const FitArgs& a, int p, int i) {
  return __ldg(a.L_all + (int64_t)__ldg(a.pair_l + p) * a.n + i) * __ldg(a.pair_scale + p);
}

template <int K>
__global__ void __launch_bounds__(kFitThreads, K <= 6 ? 3 : (K <= 9 ? 2 : 1)) codec_fit_kernel(const FitArgs a) {
  extern __shared__ float sm[];
  constexpr int k = K;
  const int n = a.n, P = a.P, v = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (a.active && __ldg(a.active + v) == 0) return;  // uniform over the CTA
  float* sE = sm;                       // k x n
  float* sD = sE + k * n;               // n x k
  float* sT = sD + n * k;               // 3 x n
  float* zR = sT + 3 * n;               // P x k
  float* zL = zR + P * k;
  float* eY = zL + P * k;               // (E Y_p)
  float* rowS = eY + P * k;             // |S_p|
  float* rowY = rowS + P;               // |Y_p|
  float* rowC = rowY + P;               // cos(S_p, Y_p)
  float* rowX = rowC + P;               // P x 3: (S_p - Y_p) T^T
  float* wsum = rowX + 3 * P;           // kFitWarps x 8 loss partial sums
  float* gw = wsum + kFitWarps * 8;     // kFitWarps x (k n + n k) per-warp gradients
  const int G = k * n + n * k;
  const float* Et = a.Et + (int64_t)v * k * n;
  const float* Dt = a.Dt + (int64_t)v * n * k;
  const float we2e = __ldg(a.w + 4 * v), wrec = __ldg(a.w + 4 * v + 1), wcode = __ldg(a.w + 4 * v + 2),
              wcol = __ldg(a.w + 4 * v + 3);

  // A. parameters and the per-pair codes
  for (int i = t; i < k * n; i += kFitThreads) sE[i] = softplus_f(__ldg(Et + i), a.beta);
  for (int i = t; i < n * k; i += kFitThreads) sD[i] = softplus_f(__ldg(Dt + i), a.beta);
  for (int i = t; i < 3 * n; i += kFitThreads) sT[i] = __ldg(a.T + i);
  if (!a.eval_only)
    for (int i = t; i < kFitWarps * G; i += kFitThreads) gw[i] = 0.0f;
  __syncthreads();
  for (int idx = t; idx < P * k; idx += kFitThreads) {
    const int p = idx / k, c = idx - p * k;
    float r = 0.0f, l = 0.0f, y = 0.0f;
    for (int i = 0; i < n; ++i) {
      const float e = sE[c * n + i];
      const float ri = batch_r(a, p, i), li = batch_l(a, p, i);
      r = fmaf(e, ri, r);
      l = fmaf(e, li, l);
      y = fmaf(e, ri * li, y);
    }
    zR[idx] = r;
    zL[idx] = l;
    eY[idx] = y;
  }
  __syncthreads();

  // B. loss sums and per-pair scalars
  float acc_e2 = 0.0f, acc_cos = 0.0f, acc_rec = 0.0f, acc_code = 0.0f, acc_col = 0.0f;
  for (int p = warp; p < P; p += kFitWarps) {
    float zrl[K];
#pragma unroll
    for (int c = 0; c < K; ++c) zrl[c] = c < k ? zR[p * k + c] * zL[p * k + c] : 0.0f;
    float e2 = 0.0f, ss = 0.0f, yy = 0.0f, sy = 0.0f, rec = 0.0f, x0 = 0.0f, x1 = 0.0f, x2 = 0.0f;
    for (int i = lane; i < n; i += 32) {
      const float ri = batch_r(a, p, i), li = batch_l(a, p, i), yi = ri * li;
      float s = 0.0f, sr = 0.0f, sl = 0.0f;
#pragma unroll
      for (int c = 0; c < K; ++c) {
        if (c < k) {
          const float d = sD[i * k + c];
          s = fmaf(d, zrl[c], s);
          sr = fmaf(d, zR[p * k + c], sr);
          sl = fmaf(d, zL[p * k + c], sl);
        }
      }
      const float e = s - yi;
      e2 = fmaf(e, e, e2);
      ss = fmaf(s, s, ss);
      yy = fmaf(yi, yi, yy);
      sy = fmaf(s, yi, sy);
      rec = fmaf(sr - ri, sr - ri, rec);
      rec = fmaf(sl - li, sl - li, rec);
      x0 = fmaf(e, sT[i], x0);
      x1 = fmaf(e, sT[n + i], x1);
      x2 = fmaf(e, sT[2 * n + i], x2);
    }
    e2 = warp_sum(e2);
    ss = warp_sum(ss);
    yy = warp_sum(yy);
    sy = warp_sum(sy);
    rec = warp_sum(rec);
    x0 = warp_sum(x0);
    x1 = warp_sum(x1);
    x2 = warp_sum(x2);
    const float nS = sqrtf(ss), nY = sqrtf(yy), cs = sy / (nS * nY);
    if (lane == 0) {
      rowS[p] = nS;
      rowY[p] = nY;
      rowC[p] = cs;
      rowX[3 * p] = x0;
      rowX[3 * p + 1] = x1;
      rowX[3 * p + 2] = x2;
    }
    float code = 0.0f;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      if (c < k) {
        const float r = zrl[c] - eY[p * k + c];
        code = fmaf(r, r, code);
      }
    }
    acc_e2 += e2;
    acc_cos += cs;
    acc_rec += rec;
    acc_code += code;
    acc_col += x0 * x0 + x1 * x1 + x2 * x2;
  }
  if (lane == 0) {
    wsum[warp * 8 + 0] = acc_e2;
    wsum[warp * 8 + 1] = acc_cos;
    wsum[warp * 8 + 2] = acc_rec;
    wsum[warp * 8 + 3] = acc_code;
    wsum[warp * 8 + 4] = acc_col;
  }
  __syncthreads();
  float tot[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int q = 0; q < kFitWarps; ++q)
#pragma unroll
    for (int j = 0; j < 5; ++j) tot[j] += wsum[q * 8 + j];
  const float N = (float)P * (float)n;
  const float m = tot[0] / N;                  // MSE(S, Y)
  const float cbar = tot[1] / (float)P;        // mean cosine
  const float L_e2e = m * (2.0f - cbar);
  const float L_rec = tot[2] / N;              // MSE(D zR, R) + MSE(D zL, L)
  const float L_code = tot[3] / ((float)P * (float)k);
  const float L_col = tot[4] / (3.0f * (float)P);
  if (t == 0 && a.losses) {
    float* lo = a.losses + 5 * v;
    lo[0] = we2e * L_e2e + wrec * L_rec + wcode * L_code + wcol * L_col;
    lo[1] = L_e2e;
    lo[2] = L_rec;
    lo[3] = L_code;
    lo[4] = L_col;
  }
  if (a.eval_only) {
    if (a.E_out)
      for (int i = t; i < k * n; i += kFitThreads) a.E_out[(int64_t)v * k * n + i] = sE[i];
    if (a.D_out)
      for (int i = t; i < n * k; i += kFitThreads) a.D_out[(int64_t)v * n * k + i] = sD[i];
    return;
  }

  // C. gradients, per pair, into this warp's copy
  float* gE = gw + warp * G;  // k x n
  float* gD = gE + k * n;     // n x k
  for (int p = warp; p < P; p += kFitWarps) {
    float zr[K], zl[K], zrl[K], grc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      zr[c] = c < k ? zR[p * k + c] : 0.0f;
      zl[c] = c < k ? zL[p * k + c] : 0.0f;
      zrl[c] = zr[c] * zl[c];
      grc[c] = c < k ? wcode * 2.0f * (zrl[c] - eY[p * k + c]) / ((float)P * (float)k) : 0.0f;
    }
    const float nS = rowS[p], nY = rowY[p], cs = rowC[p];
    const float cx0 = rowX[3 * p], cx1 = rowX[3 * p + 1], cx2 = rowX[3 * p + 2];
    const float colk = wcol * 2.0f / (3.0f * (float)P);
    float gzrl[K], gzr[K], gzl[K];
#pragma unroll
    for (int c = 0; c < K; ++c) gzrl[c] = gzr[c] = gzl[c] = 0.0f;
    constexpr int kLanesI = (kFitMaxN + 31) / 32;
    float gs_i[kLanesI], grr_i[kLanesI], grl_i[kLanesI], r_i[kLanesI], l_i[kLanesI];
#pragma unroll
    for (int j = 0; j < kLanesI; ++j) {
      const int i = lane + 32 * j;
      gs_i[j] = grr_i[j] = grl_i[j] = r_i[j] = l_i[j] = 0.0f;
      if (i < n) {
        const float ri = batch_r(a, p, i), li = batch_l(a, p, i), yi = ri * li;
        float s = 0.0f, sr = 0.0f, sl = 0.0f;
#pragma unroll
        for (int c = 0; c < K; ++c) {
          if (c < k) {
            const float d = sD[i * k + c];
            s = fmaf(d, zrl[c], s);
            sr = fmaf(d, zr[c], sr);
            sl = fmaf(d, zl[c], sl);
          }
        }
        // dL/dS_i: e2e (MSE and cosine parts) and colour
        const float dm = 2.0f * (s - yi) / N;
        const float dc = (yi / (nS * nY) - cs * s / (nS * nS)) / (float)P;
        float g = we2e * ((2.0f - cbar) * dm - m * dc);
        g = fmaf(colk, cx0 * sT[i] + cx1 * sT[n + i] + cx2 * sT[2 * n + i], g);
        gs_i[j] = g;
        grr_i[j] = wrec * 2.0f * (sr - ri) / N;
        grl_i[j] = wrec * 2.0f * (sl - li) / N;
        r_i[j] = ri;
        l_i[j] = li;
#pragma unroll
        for (int c = 0; c < K; ++c) {
          if (c < k) {
            const float d = sD[i * k + c];
            gzrl[c] = fmaf(g, d, gzrl[c]);
            gzr[c] = fmaf(grr_i[j], d, gzr[c]);
            gzl[c] = fmaf(grl_i[j], d, gzl[c]);
            // dL/dD_{i,c}
            gD[i * k + c] += g * zrl[c] + grr_i[j] * zr[c] + grl_i[j] * zl[c];
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
      if (c < k) {
        const float gr = warp_sum(gzrl[c]) + grc[c];  // dL/dzRL_c
        gzr[c] = warp_sum(gzr[c]) + gr * zl[c];        // dL/dzR_c
        gzl[c] = warp_sum(gzl[c]) + gr * zr[c];        // dL/dzL_c
      }
    }
    // dL/dE_{c,i} = dzR_c R_i + dzL_c L_i - g_rc_c Y_i
#pragma unroll
    for (int j = 0; j < kLanesI; ++j) {
      const int i = lane + 32 * j;
      if (i < n) {
#pragma unroll
        for (int c = 0; c < K; ++c)
          if (c < k) gE[c * n + i] += gzr[c] * r_i[j] + gzl[c] * l_i[j] - grc[c] * (r_i[j] * l_i[j]);
      }
    }
  }
  __syncthreads();

  // D. sum the warp copies in order, softplus chain rule, Adam
  const float bc1 = 1.0f - powf(a.b1, (float)a.t), bc2 = 1.0f - powf(a.b2, (float)a.t);
  for (int e = t; e < G; e += kFitThreads) {
    float g = 0.0f;
#pragma unroll
    for (int q = 0; q < kFitWarps; ++q) g += gw[q * G + e];
    const bool isE = e < k * n;
    const int64_t off = isE ? (int64_t)v * k * n + e : (int64_t)v * n * k + (e - k * n);
    float* X = isE ? a.Et : a.Dt;
    float* M = isE ? a.mE : a.mD;
    float* Vv = isE ? a.vE : a.vD;
    const float x = X[off];
    g *= sigmoid_f(a.beta * x);
    if (a.grad) a.grad[(int64_t)v * G + e] = g;
    const float mn = a.b1 * M[off] + (1.0f - a.b1) * g;
    const float vn = a.b2 * Vv[off] + (1.0f - a.b2) * g * g;
    M[off] = mn;
    Vv[off] = vn;
    X[off] = x - a.lr * (mn / bc1) / (sqrtf(vn / bc2) + a.eps);
  }
}

struct TrackArgs {
  int V, GE, GD;            // variants, k n, n k
  const float* val;         // validation loss of variant v at val[v * val_stride]
  int val_stride;
  const float* Et;
  const float* Dt;
  float* best_Et;
  float* best_Dt;
  float* best_loss;         // V
  int32_t* wait;            // V epochs without improvement
  int32_t* active;          // V
  int32_t* epochs;          // V updates seen while active (nullable)
  int patience;
  int32_t* n_active;        // nullable: variants still active after this update
  unsigned int* ticket;     // arrival counter, zero between launches
};

constexpr int kTrackThreads = 256;

// One CTA per variant: an active variant whose validation loss is below its
// best so far takes it as the new best and copies its parameters; otherwise
// its count of epochs without improvement grows and reaching `patience`
// deactivates it.  The last CTA to arrive counts the active flags and resets
// the ticket.
__global__ void __launch_bounds__(kTrackThreads) codec_track_kernel(const TrackArgs a) {
  __shared__ int s_improved, s_last;
  __shared__ int s_part[kTrackThreads / 32];
  const int v = blockIdx.x, t = threadIdx.x;
  if (t == 0) {
    int imp = 0;
    if (a.active[v]) {
      if (a.epochs) a.epochs[v] += 1;
      const float val = a.val[(int64_t)v * a.val_stride];
      if (val < a.best_loss[v]) {
        a.best_loss[v] = val;
        a.wait[v] = 0;
        imp = 1;
      } else {
        const int w = a.wait[v] + 1;
        a.wait[v] = w;
        if (w >= a.patience) a.active[v] = 0;
      }
    }
    s_improved = imp;
  }
  __syncthreads();
  if (s_improved) {
    for (int i = t; i < a.GE; i += kTrackThreads) a.best_Et[(int64_t)v * a.GE + i] = a.Et[(int64_t)v * a.GE + i];
    for (int i = t; i < a.GD; i += kTrackThreads) a.best_Dt[(int64_t)v * a.GD + i] = a.Dt[(int64_t)v * a.GD + i];
  }
  if (t == 0) {
    __threadfence();
    s_last = atomicAdd(a.ticket, 1u) == (unsigned)(a.V - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  int cnt = 0;
  const volatile int32_t* act = a.active;
  for (int i = t; i < a.V; i += kTrackThreads) cnt += act[i] != 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((t & 31) == 0) s_part[t >> 5] = cnt;
  __syncthreads();
  if (t == 0) {
    int total = 0;
    for (int q = 0; q < kTrackThreads / 32; ++q) total += s_part[q];
    if (a.n_active) *a.n_active = total;
    atomicExch(a.ticket, 0u);
  }
}

// Launches codec_fit_kernel for the arguments in `a` (validated by the caller).
hsc_status launch_fit(const FitArgs& a, cudaStream_t stream) {
  const int k = a.k, n = a.n, P = a.P;
  const int G = 2 * k * n;
  const size_t grad_floats = a.eval_only ? 0 : (size_t)kFitWarps * G;
  const size_t smem = sizeof(float) * ((size_t)2 * k * n + 3 * n + 3 * (size_t)P * k + 6 * (size_t)P +
                                       kFitWarps * 8 + grad_floats);
  auto kern = k == 3 ? codec_fit_kernel<3>
              : k == 6 ? codec_fit_kernel<6>
              : k == 9 ? codec_fit_kernel<9>
              : k == 12 ? codec_fit_kernel<12>
                        : codec_fit_kernel<15>;
  HSC_REQUIRE(smem <= 227 * 1024, "shared memory plan of %zu bytes too large", smem);
  if (smem > 48 * 1024) HSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)a.V, kFitThreads, smem, stream>>>(a);
  return check_launch("codec_fit_kernel");
}

}  // namespace

}  // namespace hsc

namespace {

hsc_status check_fit_shape(int variants, int k, int n, int pairs) {
  HSC_REQUIRE(variants >= 0, "negative variant count");
  HSC_REQUIRE(k >= 3 && k <= hsc::kFitMaxK && k % 3 == 0, "k=%d must be a multiple of 3 in [3, %d]", k,
              hsc::kFitMaxK);
  HSC_REQUIRE(n >= 1 && n <= hsc::kFitMaxN, "n=%d out of range [1, %d]", n, hsc::kFitMaxN);
  HSC_REQUIRE(pairs >= 1 && pairs <= hsc::kFitMaxP, "pairs=%d out of range [1, %d]", pairs, hsc::kFitMaxP);
  return HSC_OK;
}

hsc::FitArgs fit_args(int variants, int k, int n, const float* R_all, const float* L_all, const int32_t* pair_r,
                      const int32_t* pair_l, const float* pair_scale, int pairs, const float* T,
                      const float* weights, const float* Et, const float* Dt, float softplus_beta,
                      const int32_t* active) {
  hsc::FitArgs a{};
  a.V = variants;
  a.k = k;
  a.n = n;
  a.P = pairs;
  a.R_all = R_all;
  a.L_all = L_all;
  a.pair_r = pair_r;
  a.pair_l = pair_l;
  a.pair_scale = pair_scale;
  a.T = T;
  a.w = weights;
  a.Et = const_cast<float*>(Et);
  a.Dt = const_cast<float*>(Dt);
  a.beta = softplus_beta;
  a.active = active;
  return a;
}

}  // namespace

extern "C" hsc_status hsc_codec_fit_step(hsc_ctx* ctx, int variants, int k, int n, const float* R_all,
                                         const float* L_all, const int32_t* pair_r, const int32_t* pair_l,
                                         const float* pair_scale, int pairs, const float* T, const float* weights,
                                         float* Et, float* Dt, float* mE, float* vE, float* mD, float* vD, int step,
                                         float lr, float beta1, float beta2, float eps, float softplus_beta,
                                         const int32_t* active, float* losses_out, float* grad_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_TRY(check_fit_shape(variants, k, n, pairs));
  HSC_REQUIRE(step >= 1, "step numbers start at 1");
  HSC_REQUIRE(lr > 0.0f && beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps >= 0.0f &&
                  softplus_beta > 0.0f,
              "invalid optimiser settings");
  if (variants == 0) return HSC_OK;
  HSC_REQUIRE(R_all && L_all && pair_r && pair_l && pair_scale && T && weights && Et && Dt && mE && vE && mD && vD,
              "null pointer");
  HSC_GUARD(ctx);
  hsc::FitArgs a = fit_args(variants, k, n, R_all, L_all, pair_r, pair_l, pair_scale, pairs, T, weights, Et, Dt,
                            softplus_beta, active);
  a.mE = mE;
  a.vE = vE;
  a.mD = mD;
  a.vD = vD;
  a.t = step;
  a.lr = lr;
  a.b1 = beta1;
  a.b2 = beta2;
  a.eps = eps;
  a.losses = losses_out;
  a.grad = grad_out;
  return hsc::launch_fit(a, hsc::as_stream(stream));
}

extern "C" hsc_status hsc_codec_fit_eval(hsc_ctx* ctx, int variants, int k, int n, const float* R_all,
                                         const float* L_all, const int32_t* pair_r, const int32_t* pair_l,
                                         const float* pair_scale, int pairs, const float* T, const float* weights,
                                         const float* Et, const float* Dt, float softplus_beta,
                                         const int32_t* active, float* losses_out, float* E_out, float* D_out,
                                         void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_TRY(check_fit_shape(variants, k, n, pairs));
  HSC_REQUIRE(softplus_beta > 0.0f, "softplus beta must be positive");
  if (variants == 0) return HSC_OK;
  HSC_REQUIRE(R_all && L_all && pair_r && pair_l && pair_scale && T && weights && Et && Dt, "null pointer");
  HSC_REQUIRE(losses_out || E_out || D_out, "nothing to write");
  HSC_GUARD(ctx);
  hsc::FitArgs a = fit_args(variants, k, n, R_all, L_all, pair_r, pair_l, pair_scale, pairs, T, weights, Et, Dt,
                            softplus_beta, active);
  a.eval_only = 1;
  a.losses = losses_out;
  a.E_out = E_out;
  a.D_out = D_out;
  return hsc::launch_fit(a, hsc::as_stream(stream));
}

extern "C" hsc_status hsc_codec_fit_track(hsc_ctx* ctx, int variants, int k, int n, const float* val_loss,
                                          int val_stride, const float* Et, const float* Dt, float* best_Et,
                                          float* best_Dt, float* best_loss, int32_t* wait, int32_t* active,
                                          int32_t* epochs, int patience, int32_t* n_active_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(variants >= 0, "negative variant count");
  HSC_REQUIRE(k >= 1 && n >= 1 && (int64_t)k * n <= (1 << 24), "bad parameter shape k=%d n=%d", k, n);
  HSC_REQUIRE(val_stride >= 1, "val_stride must be >= 1");
  HSC_REQUIRE(patience >= 1, "patience must be >= 1");
  if (variants == 0) return HSC_OK;
  HSC_REQUIRE(val_loss && Et && Dt && best_Et && best_Dt && best_loss && wait && active, "null pointer");
  HSC_GUARD(ctx);
  hsc::TrackArgs a{};
  a.V = variants;
  a.GE = k * n;
  a.GD = n * k;
  a.val = val_loss;
  a.val_stride = val_stride;
  a.Et = Et;
  a.Dt = Dt;
  a.best_Et = best_Et;
  a.best_Dt = best_Dt;
  a.best_loss = best_loss;
  a.wait = wait;
  a.active = active;
  a.epochs = epochs;
  a.patience = patience;
  a.n_active = n_active_out;
  a.ticket = reinterpret_cast<unsigned int*>(ctx->d_small + HSC_OFF_FITTICKET);
  hsc::codec_track_kernel<<<(unsigned)variants, hsc::kTrackThreads, 0, hsc::as_stream(stream)>>>(a);
  return hsc::check_launch("codec_track_kernel");
}
