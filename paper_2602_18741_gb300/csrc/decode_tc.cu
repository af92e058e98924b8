// Spectral decode s_hat = W_dec z (Eq. 4) on the 5th-generation tensor cores.
//
// Per tile of 128 pixels the decode is one [128 x 16] x [16 x N] BF16 MMA with
// FP32 accumulation (k <= 16 code channels zero-padded to K = 16, n samples
// padded to N = 16 * ceil(n / 16)).  The work is HBM-store bound (4n bytes
// out per pixel against 2*16*N flops), so the kernel is shaped around the
// output stream:
//   * persistent CTAs (up to 4 per SM: 4 x 128 TMEM columns), 128 threads;
//     thread t owns pixel row t and loads its next tile's latent row while the
//     current tile's MMA and epilogue run;
//   * the A tile (latent rows, fp8 codes converted exactly to bf16) is written
//     to shared memory in the no-swizzle K-major canonical layout (8-row x
//     16-byte core matrices); B = bf16(D * diag(scale)) is staged once;
//   * one elected thread issues tcgen05.mma into a 128-lane x N-column TMEM
//     accumulator and commits to an mbarrier;
//   * each warp reads its 32 TMEM lanes (all columns, one wait) with
//     tcgen05.ld, writes its rows to its quarter of a [128 x n] FP32 staging
//     tile, and its lane 0 streams those 32 rows (32 * n * 4 contiguous bytes)
//     to global memory with a bulk async copy (cp.async.bulk), which overlaps
//     the next tile's MMA; no block barrier stands between a warp's epilogue
//     and its store.
// FP32 latents (k <= 10) take the same path with each FP32 value split into
// three bf16 parts, z = hi + mid + lo (each remainder is exact in FP32), and
// the six products hi.hi, hi.mid, mid.hi, hi.lo, mid.mid, lo.hi laid side by
// side along K in segments of 8 columns for k <= 8 (K = 48: three K = 16 MMAs
// into one accumulator) or 10 columns for k = 9, 10 (K = 60 padded to 64:
// four MMAs); every
// product is exact in FP32 and the dropped ones are below 2^-24 relative, so
// the result has FP32 accuracy.
// Every mbarrier wait is bounded; on expiry the kernel sets an error bit,
// waits (bounded) for the MMA it issued and for its bulk copies, frees its
// TMEM and returns.
#include "common.cuh"
#include "tcgen05.cuh"

namespace hsc {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;          // MMA M
constexpr unsigned kTmemCols = 128;   // power of two >= N (N <= 128)

using namespace tc;

struct TcArgs {
  const void* latent;
  int dt;  // HSC_BF16, HSC_FP8_E4M3 or HSC_F32 (split into three bf16 parts)
  const float* scales;
  int64_t P;
  int k;
  const float* D;  // n x k
  int n;
  int npad;  // N of the MMA
  float* out;
  unsigned int* err;
};

__device__ __forceinline__ float to_bf16_value(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// z = hi + mid + lo with each part a bf16 value; the two remainders are exact
// in FP32, lo is rounded.
__device__ __forceinline__ void split3(float z, float (&part)[3]) {
  part[0] = to_bf16_value(z);
  const float r1 = __fsub_rn(z, part[0]);
  part[1] = to_bf16_value(r1);
  part[2] = to_bf16_value(__fsub_rn(r1, part[1]));
}

// K segments of the split FP32 form: columns SW s .. SW s + SW - 1 (segment
// width SW = 8 for KB = 3, 10 for KB = 4) hold, for every code c < k, parts
// (hi, hi, mid, hi, mid, lo)[s] of z_c in A and parts
// kSegB[s] = (hi, mid, hi, lo, mid, hi)[s] of D_{i,c} in B.
__constant__ int kSegB[6] = {0, 1, 0, 2, 1, 0};
template <int KB>
constexpr int seg_width() { return KB == 4 ? 10 : 8; }

// Latent row p in two steps, so that the loads of the next tile are in
// flight while the current tile's MMA and epilogue run: load_a_raw issues the
// loads (raw element bits, zero beyond k and beyond P), pack_a_row turns them
// into 8 * KB packed bf16 pairs (K = 16 * KB): the values themselves (KB = 1)
// or the six segments of the three-part split (KB = 3, 4).
template <int KB>
struct RawRow {
  // KB = 1: elements as 16-bit units, two per word (bf16 bits, or an fp8 byte);
  // KB = 3, 4: the FP32 values of codes 0 .. SW - 1
  uint32_t v[KB == 1 ? 8 : seg_width<KB>()];
};

template <int KB>
__device__ __forceinline__ void load_a_raw(const TcArgs& a, int64_t p, bool valid, RawRow<KB>& r) {
#pragma unroll
  for (int j = 0; j < (KB == 1 ? 8 : seg_width<KB>()); ++j) r.v[j] = 0u;
  if constexpr (KB != 1) {
#pragma unroll
    for (int e = 0; e < seg_width<KB>(); ++e)
      if (valid && e < a.k) r.v[e] = __float_as_uint(__ldg(reinterpret_cast<const float*>(a.latent) + p * a.k + e));
  } else {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      if (valid && e < a.k) {
        const uint32_t bits = a.dt == HSC_FP8_E4M3
                                  ? (uint32_t)__ldg(reinterpret_cast<const unsigned char*>(a.latent) + p * a.k + e)
                                  : (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(a.latent) + p * a.k + e);
        r.v[e >> 1] |= bits << ((e & 1) * 16);
      }
    }
  }
}

template <int KB>
__device__ __forceinline__ void pack_a_row(const TcArgs& a, const RawRow<KB>& r, uint32_t (&w)[8 * KB]) {
#pragma unroll
  for (int j = 0; j < 8 * KB; ++j) w[j] = 0u;
  auto put = [&](int e, float v) {
    const uint32_t bits = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
    w[e >> 1] |= bits << ((e & 1) * 16);
  };
  if constexpr (KB == 1) {
    if (a.dt == HSC_FP8_E4M3) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        if (e >= a.k) break;
        put(e, fp8_e4m3_to_float((unsigned char)(r.v[e >> 1] >> ((e & 1) * 16))));
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = r.v[j];   // already bf16 pairs
    }
  } else {
    constexpr int SW = seg_width<KB>();
#pragma unroll
    for (int c = 0; c < SW; ++c) {
      float part[3];
      split3(__uint_as_float(r.v[c]), part);
      // segments of SW columns: hi, hi, mid, hi, mid, lo
      put(0 * SW + c, part[0]);
      put(1 * SW + c, part[0]);
      put(2 * SW + c, part[1]);
      put(3 * SW + c, part[0]);
      put(4 * SW + c, part[1]);
      put(5 * SW + c, part[2]);
    }
  }
}

template <int NPAD, int KB>
__global__ void __launch_bounds__(kTcThreads) decode_spectra_tc_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = base;                                           // KB x [128 x 16] bf16 (4096 B each)
  unsigned char* sB = base + KB * 4096;                               // KB x [NPAD x 16] bf16
  float* sOut = reinterpret_cast<float*>(base + KB * (4096 + NPAD * 32));  // [128 x n] staging tile
  uint64_t* sBar = reinterpret_cast<uint64_t*>(sOut + kTcRows * a.n + 4);  // [0] MMA done, [1] drain
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(sBar + 2);
  int* sOk = reinterpret_cast<int*>(sTmem + 1);

  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int n = a.n;

  // TMEM allocation (one warp), mbarrier init, B staging.
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sBar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sBar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sOk = 1;
  }
  for (int idx = t; idx < NPAD * 16 * KB; idx += kTcThreads) {
    const int r = idx / (16 * KB), e = idx - r * (16 * KB);
    float v = 0.0f;
    if (KB == 1) {
      if (r < n && e < a.k) {
        v = __ldg(a.D + r * a.k + e);
        if (a.dt == HSC_FP8_E4M3) v = __fmul_rn(v, __ldg(a.scales + e));
      }
    } else if (r < n && e < 6 * seg_width<KB>() && e % seg_width<KB>() < a.k) {
      const int seg = e / seg_width<KB>(), c = e % seg_width<KB>();
      float part[3];
      split3(__ldg(a.D + r * a.k + c), part);
      v = part[kSegB[seg]];
    }
    *reinterpret_cast<__nv_bfloat16*>(sB + (e >> 4) * (NPAD * 32) + kmajor_off(r, e & 15)) = __float2bfloat16_rn(v);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *sTmem;
  const uint32_t bar = smem_u32(sBar);

  constexpr uint32_t idesc = instr_desc_bf16(kTcRows, NPAD);

  const int64_t tiles = (a.P + kTcRows - 1) / kTcRows;
  uint32_t phase = 0;
  // this thread's latent row of the first tile
  uint32_t wA[8 * KB];
  RawRow<KB> raw;
  {
    const int64_t p = (int64_t)blockIdx.x * kTcRows + t;
    load_a_raw<KB>(a, p, blockIdx.x < tiles && p < a.P, raw);
    pack_a_row<KB>(a, raw, wA);
  }
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t p0 = tile * kTcRows;
    const int rows = (int)min((int64_t)kTcRows, a.P - p0);
    // A tile: row t in the canonical K-major layout, one [128 x 16] block per K step
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) {
      *reinterpret_cast<uint4*>(sA + kb * 4096 + kmajor_off(t, 0)) =
          make_uint4(wA[8 * kb + 0], wA[8 * kb + 1], wA[8 * kb + 2], wA[8 * kb + 3]);
      *reinterpret_cast<uint4*>(sA + kb * 4096 + kmajor_off(t, 8)) =
          make_uint4(wA[8 * kb + 4], wA[8 * kb + 5], wA[8 * kb + 6], wA[8 * kb + 7]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0) {
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) {
        const uint64_t adesc = smem_desc(smem_u32(sA + kb * 4096), 128, 256);
        const uint64_t bdesc = smem_desc(smem_u32(sB + kb * NPAD * 32), 128, 256);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(kb)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
    }
    // next tile's row: the loads stay in flight through the MMA and this
    // tile's epilogue and are packed at the end of the iteration
    {
      const int64_t nt = tile + gridDim.x;
      const int64_t p = nt * kTcRows + t;
      load_a_raw<KB>(a, p, nt < tiles && p < a.P, raw);
    }
    if (t == 0) {
      if (!mbar_wait(bar, phase)) {
        *sOk = 0;
        atomicOr(a.err, HSC_DEVERR_TIMEOUT);
      }
    }
    __syncthreads();
    if (!*sOk) break;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // all accumulator columns of this warp's 32 lanes, one wait
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t v[NPAD];
#pragma unroll
    for (int c0 = 0; c0 < NPAD; c0 += 16) TC_LD16(trow + (uint32_t)c0, (v + c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const bool full = rows == kTcRows;
    // this warp's staging rows are free once its previous store has read them
    if ((t & 31) == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncwarp();
#pragma unroll
    for (int c = 0; c < NPAD; ++c) {
      if (c < n) {
        const float x = __uint_as_float(v[c]);
        if (full)
          sOut[t * n + c] = x;
        else if (t < rows)
          a.out[(p0 + t) * n + c] = x;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (full) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if ((t & 31) == 0) {
        const int r0 = warp * 32;
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(a.out + (p0 + r0) * n),
                     "r"(smem_u32(sOut + r0 * n)), "r"((uint32_t)(32 * n * 4))
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    pack_a_row<KB>(a, raw, wA);
  }
  // after an expired wait the MMA may still be running: drain it (bounded)
  // before TMEM is freed; every warp's bulk stores finish before the exit
  if (t == 0 && !*sOk) drain_mma(smem_u32(sBar + 1));
  if ((t & 31) == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

template <int NPAD, int KB>
hsc_status launch_tc(const TcArgs& a, int sm_count, cudaStream_t s) {
  const size_t smem = 1024 + KB * (4096 + NPAD * 32) + (size_t)kTcRows * a.n * 4 + 64;
  auto kern = decode_spectra_tc_kernel<NPAD, KB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return set_error(HSC_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(e));
  const int64_t tiles = (a.P + kTcRows - 1) / kTcRows;
  // resident CTAs per SM: shared memory allows floor(227 KB / smem); TMEM
  // allows 512 / 128 = 4
  int per_sm = (int)((227 * 1024) / (smem + 1024));
  if (per_sm > 4) per_sm = 4;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sm_count * per_sm;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kTcThreads, smem, s>>>(a);
  return check_launch("decode_spectra_tc_kernel");
}

template <int KB>
hsc_status launch_tc_n(const TcArgs& a, int sm_count, cudaStream_t s) {
  switch (a.npad) {
    case 16: return launch_tc<16, KB>(a, sm_count, s);
    case 32: return launch_tc<32, KB>(a, sm_count, s);
    case 48: return launch_tc<48, KB>(a, sm_count, s);
    case 64: return launch_tc<64, KB>(a, sm_count, s);
    case 80: return launch_tc<80, KB>(a, sm_count, s);
    case 96: return launch_tc<96, KB>(a, sm_count, s);
    case 112: return launch_tc<112, KB>(a, sm_count, s);
    default: return launch_tc<128, KB>(a, sm_count, s);
  }
}

}  // namespace

hsc_status launch_decode_spectra_tc(hsc_ctx* ctx, const void* latent, int dt, const float* scales, int64_t P, int k,
                                    const float* D, int n, float* out, cudaStream_t s) {
  TcArgs a{};
  a.latent = latent;
  a.dt = dt;
  a.scales = scales;
  a.P = P;
  a.k = k;
  a.D = D;
  a.n = n;
  a.npad = (n + 15) / 16 * 16;
  a.out = out;
  a.err = ctx->d_err;
  if (dt == HSC_F32) return k <= 8 ? launch_tc_n<3>(a, ctx->sm_count, s) : launch_tc_n<4>(a, ctx->sm_count, s);
  return launch_tc_n<1>(a, ctx->sm_count, s);
}

}  // namespace hsc
