// Spectral decode s_hat = W_dec z (Eq. 4) on the 5th-generation tensor cores.
//
// Per tile of 128 pixels the decode is one [128 x 16] x [16 x N] BF16 MMA with
// FP32 accumulation (k <= 16 code channels zero-padded to K = 16, n samples
// padded to N = 16 * ceil(n / 16)).  The work is HBM-store bound (4n bytes
// out per pixel against 2*16*N flops), so the kernel is shaped around the
// output stream, with warps specialised by role (192 threads per CTA, two
// CTAs per SM: 2 x 256 TMEM columns):
//   * a producer warp loads each tile's latent rows (four rows per lane, the
//     next tile's loads in flight while it packs the current one; BF16 rows
//     as whole 32-bit pairs, FP8 rows as byte pairs converted in one step
//     each) and writes the A tile in the no-swizzle K-major canonical layout
//     (8-row x 16-byte core matrices) into one of two A stages;
//     B = bf16(D * diag(scale)) is staged once;
//   * one lane of an MMA warp issues tcgen05.mma into one of two 128-lane x
//     N-column TMEM accumulators and commits to mbarriers that free the A
//     stage and fill the accumulator;
//   * four epilogue warps (warp w owns TMEM lanes, i.e. pixel rows, 32 w ..
//     32 w + 31) read their rows with tcgen05.ld, hand the accumulator back,
//     write the rows into their part of a [128 x n] FP32 staging tile, and
//     lane 0 streams those 32 rows (32 * n * 4 contiguous bytes) to global
//     memory with one bulk async copy (cp.async.bulk).
// FP32 latents (k <= 10) take the same path with each FP32 value split into
// three bf16 parts, z = hi + mid + lo (each remainder is exact in FP32), and
// the six products hi.hi, hi.mid, mid.hi, hi.lo, mid.mid, lo.hi laid side by
// side along K in segments of 8 columns for k <= 8 (K = 48: three K = 16 MMAs
// into one accumulator) or 10 columns for k = 9, 10 (K = 60 padded to 64:
// four MMAs); every
// product is exact in FP32 and the dropped ones are below 2^-24 relative, so
// the result has FP32 accuracy.
// Every mbarrier wait is bounded; on expiry the kernel sets an error bit,
// every role leaves its loop at its next wait, the MMA lane waits (bounded)
// for the MMAs it issued, the epilogue warps for their bulk copies, and TMEM
// is freed after a final block barrier.
#include "common.cuh"
#include "tcgen05.cuh"

namespace hsc {

namespace {

constexpr int kTcRows = 128;          // MMA M

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
  bool pairs;  // BF16 / FP8 with k even and the latent aligned to 4 (BF16) or 2 (FP8) bytes: whole-pair loads
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
  // KB = 1: two elements per word (bf16 bits as 16-bit halves; fp8 codes as
  // the two low bytes);
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
    // every element's load goes out before any is combined, so a thread
    // waits for memory once per row, not once per element
    if (a.pairs) {
      // k even, rows aligned to whole pairs: a bf16 row is k / 2 words that
      // are the packed pairs themselves; an fp8 row is k / 2 byte pairs
      const int np = a.k >> 1;
      if (a.dt == HSC_FP8_E4M3) {
        const unsigned short* src = reinterpret_cast<const unsigned short*>(a.latent) + p * np;
        uint32_t h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = (valid && j < np) ? (uint32_t)__ldg(src + j) : 0u;
        // kept as byte pairs; pack_a_row converts each pair in one step
#pragma unroll
        for (int j = 0; j < 8; ++j) r.v[j] = h[j];
      } else {
        const unsigned int* src = reinterpret_cast<const unsigned int*>(a.latent) + p * np;
#pragma unroll
        for (int j = 0; j < 8; ++j) r.v[j] = (valid && j < np) ? __ldg(src + j) : 0u;
      }
      return;
    }
    uint32_t b[16];
    if (a.dt == HSC_FP8_E4M3) {
      const unsigned char* src = reinterpret_cast<const unsigned char*>(a.latent) + p * a.k;
#pragma unroll
      for (int e = 0; e < 16; ++e) b[e] = (valid && e < a.k) ? (uint32_t)__ldg(src + e) : 0u;
      // byte pairs, as the whole-pair path loads them
#pragma unroll
      for (int j = 0; j < 8; ++j) r.v[j] = b[2 * j] | (b[2 * j + 1] << 8);
      return;
    } else {
      const unsigned short* src = reinterpret_cast<const unsigned short*>(a.latent) + p * a.k;
#pragma unroll
      for (int e = 0; e < 16; ++e) b[e] = (valid && e < a.k) ? (uint32_t)__ldg(src + e) : 0u;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) r.v[j] = b[2 * j] | (b[2 * j + 1] << 16);
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
      // each word holds two e4m3 codes (byte pairs): to f16x2 in one
      // conversion, then to bf16x2; every step is exact for e4m3 values
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t hh;
        asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(hh) : "h"((unsigned short)r.v[j]));
        const __half2 h2 = *reinterpret_cast<const __half2*>(&hh);
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(__low2float(h2), __high2float(h2));
        w[j] = *reinterpret_cast<const uint32_t*>(&b2);
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

// ---------------------------------------------------------------------------
// The kernel.  Roles: one warp stages the latent tiles (two A stages), one
// lane issues the MMAs into two TMEM accumulators, and four epilogue warps
// drain the accumulators into their staging rows (two buffers per warp when
// two CTAs fit) and bulk-store them, so each role runs ahead of the next as
// far as its buffers allow and the output stream does not stop for the MMA.
// Hand-offs are mbarriers: A full (32 producer arrivals) / A empty (MMA
// commit), and accumulator full (MMA commit) / accumulator empty (one
// arrival per epilogue warp).  A wait on an "empty" barrier starts at parity
// 1, which a fresh barrier reports complete.
constexpr int kWsThreads = 192;       // warps 0-3 epilogue, 4 producer, 5 MMA
constexpr unsigned kWsTmemCols = 256;  // two 128-column accumulators

template <int NPAD, int KB, bool DS>
__global__ void __launch_bounds__(kWsThreads) decode_spectra_ws_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kStageA = KB * 4096;                                  // one A stage: KB x [128 x 16] bf16
  unsigned char* sA = base;                                           // 2 stages
  unsigned char* sB = base + 2 * kStageA;                             // KB x [NPAD x 16] bf16
  float* sOut = reinterpret_cast<float*>(sB + KB * NPAD * 32);        // (DS ? 2 : 1) x [128 x n]
  const int n = a.n;
  uint64_t* sBar = reinterpret_cast<uint64_t*>(sOut + (DS ? 2 : 1) * kTcRows * n + 4);
  // [0,1] A full, [2,3] A empty, [4,5] accumulator full, [6,7] accumulator empty, [8] drain
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(sBar + 9);
  volatile int* sOk = reinterpret_cast<volatile int*>(sTmem + 1);

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                 "r"(kWsTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" ::"r"(smem_u32(sBar + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sBar + 2 + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sBar + 4 + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(sBar + 6 + i)) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sBar + 8)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sOk = 1;
  }
  for (int idx = t; idx < NPAD * 16 * KB; idx += kWsThreads) {
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
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *sTmem;
  const int64_t tiles = (a.P + kTcRows - 1) / kTcRows;

  // bounded wait; an expiry records the timeout, and every role leaves its
  // loop at its next wait once the status word is cleared
  auto wait = [&](int b, uint32_t parity) {
    if (*sOk == 0) return false;
    if (mbar_wait(smem_u32(sBar + b), parity)) return true;
    *sOk = 0;
    atomicOr(a.err, HSC_DEVERR_TIMEOUT);
    return false;
  };

  if (warp == 4) {
    // producer: rows lane, lane + 32, lane + 64, lane + 96 of each tile; the
    // next tile's loads are issued before this tile is packed, so they are in
    // flight while the producer packs, hands over and waits for a free stage
    RawRow<KB> raw[4], nxt[4];
    auto load_tile = [&](int64_t tile, RawRow<KB>(&r)[4]) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t p = tile * kTcRows + lane + 32 * q;
        load_a_raw<KB>(a, p, tile < tiles && p < a.P, r[q]);
      }
    };
    load_tile(blockIdx.x, nxt);
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
      const int s = it & 1;
#pragma unroll
      for (int q = 0; q < 4; ++q) raw[q] = nxt[q];
      load_tile(tile + gridDim.x, nxt);
      if (!wait(2 + s, ((it >> 1) & 1) ^ 1)) break;
      unsigned char* sAs = sA + s * kStageA;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t w[8 * KB];
        pack_a_row<KB>(a, raw[q], w);
        const int row = lane + 32 * q;
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          *reinterpret_cast<uint4*>(sAs + kb * 4096 + kmajor_off(row, 0)) =
              make_uint4(w[8 * kb + 0], w[8 * kb + 1], w[8 * kb + 2], w[8 * kb + 3]);
          *reinterpret_cast<uint4*>(sAs + kb * 4096 + kmajor_off(row, 8)) =
              make_uint4(w[8 * kb + 4], w[8 * kb + 5], w[8 * kb + 6], w[8 * kb + 7]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(sBar + s)) : "memory");
    }
  } else if (warp == 5) {
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc_bf16(kTcRows, NPAD);
      bool ok = true;
      int it = 0;
      for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
        const int s = it & 1;
        if (!wait(s, (it >> 1) & 1) || !wait(6 + s, ((it >> 1) & 1) ^ 1)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(128 * s);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          const uint64_t adesc = smem_desc(smem_u32(sA + s * kStageA + kb * 4096), 128, 256);
          const uint64_t bdesc = smem_desc(smem_u32(sB + kb * NPAD * 32), 128, 256);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                  d),
              "l"(adesc), "l"(bdesc), "r"(idesc), "r"(kb)
              : "memory");
        }
        // the A stage is free and the accumulator full once these MMAs finish
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(sBar + 2 + s))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(sBar + 4 + s))
                     : "memory");
      }
      // after an expired wait MMAs may still be running: drain them (bounded)
      if (!ok) drain_mma(smem_u32(sBar + 8));
    }
  } else {
    // epilogue: warp w owns TMEM lanes (pixel rows) 32 w .. 32 w + 31
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
      const int s = it & 1;
      if (!wait(4 + s, (it >> 1) & 1)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t trow = tmem + (uint32_t)(128 * s) + ((uint32_t)(warp * 32) << 16);
      uint32_t v[NPAD];
#pragma unroll
      for (int c0 = 0; c0 < NPAD; c0 += 16) TC_LD16(trow + (uint32_t)c0, (v + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(sBar + 6 + s)) : "memory");
      const int64_t p0 = tile * kTcRows;
      const int rows = (int)min((int64_t)kTcRows, a.P - p0);
      const int r = warp * 32 + lane;
      if (rows == kTcRows) {
        float* so = sOut + (DS ? s : 0) * kTcRows * n;
        // this warp's rows of the buffer are free once the store that last
        // read them has read them
        if (lane == 0) {
          if (DS) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          else asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < NPAD; ++c)
          if (c < n) so[r * n + c] = __uint_as_float(v[c]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(a.out + (p0 + warp * 32) * n),
                       "r"(smem_u32(so + warp * 32 * n)), "r"((uint32_t)(32 * n * 4))
                       : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      } else if (r < rows) {
#pragma unroll
        for (int c = 0; c < NPAD; ++c)
          if (c < n) a.out[(p0 + r) * n + c] = __uint_as_float(v[c]);
      }
    }
    // every bulk store of this warp has finished before TMEM is freed and
    // the kernel exits
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWsTmemCols) : "memory");
  }
}

template <int NPAD, int KB, bool DS>
size_t ws_smem(int n) {
  return 1024 + 2 * KB * 4096 + (size_t)KB * NPAD * 32 + (size_t)(DS ? 2 : 1) * kTcRows * n * 4 + 16 + 9 * 8 + 16;
}

template <int NPAD, int KB, bool DS>
hsc_status launch_ws(const TcArgs& a, int sm_count, int per_sm, cudaStream_t s) {
  // at least a third of the SM's shared memory per CTA, so that no more than
  // two CTAs (all the TMEM holds) are resident on an SM
  size_t smem = ws_smem<NPAD, KB, DS>(a.n);
  if (smem < 77 * 1024) smem = 77 * 1024;
  auto kern = decode_spectra_ws_kernel<NPAD, KB, DS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return set_error(HSC_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(e));
  const int64_t tiles = (a.P + kTcRows - 1) / kTcRows;
  int64_t grid = (int64_t)sm_count * per_sm;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kWsThreads, smem, s>>>(a);
  return check_launch("decode_spectra_ws_kernel");
}

// Two CTAs per SM (the TMEM holds two of 256 columns) when their shared
// memory fits, with two staging buffers per warp if those fit as well.
template <int NPAD, int KB>
hsc_status launch_ws_n(const TcArgs& a, int sm_count, cudaStream_t s) {
  constexpr size_t kSm = 227 * 1024;
  if (2 * (ws_smem<NPAD, KB, true>(a.n) + 1024) <= kSm) return launch_ws<NPAD, KB, true>(a, sm_count, 2, s);
  if (2 * (ws_smem<NPAD, KB, false>(a.n) + 1024) <= kSm) return launch_ws<NPAD, KB, false>(a, sm_count, 2, s);
  return launch_ws<NPAD, KB, false>(a, sm_count, 1, s);
}

template <int KB>
hsc_status launch_tc_n(const TcArgs& a, int sm_count, cudaStream_t s) {
  switch (a.npad) {
    case 16: return launch_ws_n<16, KB>(a, sm_count, s);
    case 32: return launch_ws_n<32, KB>(a, sm_count, s);
    case 48: return launch_ws_n<48, KB>(a, sm_count, s);
    case 64: return launch_ws_n<64, KB>(a, sm_count, s);
    case 80: return launch_ws_n<80, KB>(a, sm_count, s);
    case 96: return launch_ws_n<96, KB>(a, sm_count, s);
    case 112: return launch_ws_n<112, KB>(a, sm_count, s);
    default: return launch_ws_n<128, KB>(a, sm_count, s);
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
  a.pairs = dt != HSC_F32 && k % 2 == 0 && aligned(latent, dt == HSC_BF16 ? 4 : 2);
  a.out = out;
  a.err = ctx->d_err;
  if (dt == HSC_F32) return k <= 8 ? launch_tc_n<3>(a, ctx->sm_count, s) : launch_tc_n<4>(a, ctx->sm_count, s);
  return launch_tc_n<1>(a, ctx->sm_count, s);
}

}  // namespace hsc
