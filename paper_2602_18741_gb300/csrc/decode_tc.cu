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
//     tcgen05.ld, writes its rows to a [128 x n] FP32 staging tile, and one
//     thread streams the whole tile (128 * n * 4 contiguous bytes) to global
//     memory with a bulk async copy (cp.async.bulk), which overlaps the next
//     tile's MMA.
// Every mbarrier wait is bounded; on expiry the kernel sets an error bit,
// drains its bulk copies, frees its TMEM and returns.
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
  int dt;  // HSC_BF16 or HSC_FP8_E4M3
  const float* scales;
  int64_t P;
  int k;
  const float* D;  // n x k
  int n;
  int npad;  // N of the MMA
  float* out;
  unsigned int* err;
};

// Latent row p (k codes) as 8 packed bf16 pairs, zero beyond k (and beyond P).
__device__ __forceinline__ void load_a_row(const TcArgs& a, int64_t p, bool valid, uint32_t (&w)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) w[j] = 0u;
  if (!valid) return;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    if (e >= a.k) break;
    float v;
    if (a.dt == HSC_FP8_E4M3)
      v = fp8_e4m3_to_float(__ldg(reinterpret_cast<const unsigned char*>(a.latent) + p * a.k + e));
    else
      v = __uint_as_float(((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(a.latent) + p * a.k + e)) << 16);
    const uint32_t bits = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
    w[e >> 1] |= bits << ((e & 1) * 16);
  }
}

template <int NPAD>
__global__ void __launch_bounds__(kTcThreads) decode_spectra_tc_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = base;                                           // 128 x 16 bf16 = 4096 B
  unsigned char* sB = base + 4096;                                    // NPAD x 16 bf16
  float* sOut = reinterpret_cast<float*>(base + 4096 + NPAD * 32);    // [128 x n] staging tile
  uint64_t* sBar = reinterpret_cast<uint64_t*>(sOut + kTcRows * a.n + 4);
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(sBar + 1);
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
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sOk = 1;
  }
  for (int idx = t; idx < NPAD * 16; idx += kTcThreads) {
    const int r = idx >> 4, e = idx & 15;
    float v = 0.0f;
    if (r < n && e < a.k) {
      v = __ldg(a.D + r * a.k + e);
      if (a.dt == HSC_FP8_E4M3) v = __fmul_rn(v, __ldg(a.scales + e));
    }
    *reinterpret_cast<__nv_bfloat16*>(sB + kmajor_off(r, e)) = __float2bfloat16_rn(v);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *sTmem;
  const uint32_t bar = smem_u32(sBar);
  const uint64_t adesc = smem_desc(smem_u32(sA), 128, 256);
  const uint64_t bdesc = smem_desc(smem_u32(sB), 128, 256);
  constexpr uint32_t idesc = instr_desc_bf16(kTcRows, NPAD);

  const int64_t tiles = (a.P + kTcRows - 1) / kTcRows;
  uint32_t phase = 0;
  // this thread's latent row of the first tile, loaded ahead
  uint32_t wA[8];
  {
    const int64_t p = (int64_t)blockIdx.x * kTcRows + t;
    load_a_row(a, p, blockIdx.x < tiles && p < a.P, wA);
  }
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t p0 = tile * kTcRows;
    const int rows = (int)min((int64_t)kTcRows, a.P - p0);
    // A tile: row t in the canonical K-major layout
    *reinterpret_cast<uint4*>(sA + kmajor_off(t, 0)) = make_uint4(wA[0], wA[1], wA[2], wA[3]);
    *reinterpret_cast<uint4*>(sA + kmajor_off(t, 8)) = make_uint4(wA[4], wA[5], wA[6], wA[7]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0) {
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(adesc), "l"(bdesc), "r"(idesc), "r"(0)
          : "memory");
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
    }
    // next tile's row, in flight while the MMA and this tile's epilogue run
    {
      const int64_t nt = tile + gridDim.x;
      const int64_t p = nt * kTcRows + t;
      load_a_row(a, p, nt < tiles && p < a.P, wA);
    }
    if (t == 0) {
      if (!mbar_wait(bar, phase)) {
        *sOk = 0;
        atomicOr(a.err, HSC_DEVERR_TIMEOUT);
      }
      // the staging tile is free once the previous bulk store has read it
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
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
      __syncthreads();
      if (t == 0) {
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(a.out + p0 * n),
                     "r"(smem_u32(sOut)), "r"((uint32_t)(kTcRows * n * 4))
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
  }
  if (t == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

template <int NPAD>
hsc_status launch_tc(const TcArgs& a, int sm_count, cudaStream_t s) {
  const size_t smem = 1024 + 4096 + NPAD * 32 + (size_t)kTcRows * a.n * 4 + 64;
  auto kern = decode_spectra_tc_kernel<NPAD>;
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
  switch (a.npad) {
    case 16: return launch_tc<16>(a, ctx->sm_count, s);
    case 32: return launch_tc<32>(a, ctx->sm_count, s);
    case 48: return launch_tc<48>(a, ctx->sm_count, s);
    case 64: return launch_tc<64>(a, ctx->sm_count, s);
    case 80: return launch_tc<80>(a, ctx->sm_count, s);
    case 96: return launch_tc<96>(a, ctx->sm_count, s);
    case 112: return launch_tc<112>(a, ctx->sm_count, s);
    default: return launch_tc<128>(a, ctx->sm_count, s);
  }
}

}  // namespace hsc
