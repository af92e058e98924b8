// RGB-to-latent upsampling (Sec. 5): per pixel a three-layer perceptron,
//     h1 = silu(W1 c + b1),  h2 = silu(W2 h1 + b2),  z = W3 h2 + b3,
// hidden width 128, on the 5th-generation tensor cores.
//
// A CTA takes tiles of 128 pixels; 16 epilogue warps and one MMA warp.  Per
// tile three BF16 MMAs with FP32 accumulation run in sequence, each issued by
// the MMA warp's first lane and committed to the slot's "done" mbarrier:
//   layer 1: [128 x 16] x [16 x 128]   (the colour in K columns 0..2),
//   layer 2: [128 x 128] x [128 x 128] (eight K = 16 steps),
//   layer 3: [128 x 128] x [128 x 16]  (k <= 16 outputs, zero-padded).
// Between them the epilogue runs on the 16 epilogue warps: pixel row r is
// TMEM lane r, read by the four warps of lane quadrant r / 32, each for 32 of
// the 128 hidden columns (tcgen05.ld); a thread adds the bias, applies SiLU
// and rounds to bf16, writing its 32 values into the next layer's A operand
// in shared memory (no-swizzle K-major layout).  The weights and biases of
// the hidden layers are staged at half scale (exact in bf16 and FP32), so the
// accumulator plus bias is already x/2 and SiLU(x) = x/2 (1 + tanh(x/2)) is
// one FMA around the hardware tanh.  One CTA per SM works on four tiles at
// once (four A buffers, four 128-column TMEM regions; layer 3 reuses the
// first 16 columns of its tile's region once layer 2 has been read); the
// hand-offs are
// mbarriers, not block barriers: every epilogue thread arrives on the slot's
// "operand ready" barrier once its shared-memory writes and TMEM reads are
// done and goes on with the next slot, and the MMA lane waits for all 512
// arrivals before it issues; per layer the slots are taken in turn,
//   MMA1(a..d) | epi1(a) MMA2(a) | epi1(b) MMA2(b) | ... | epi2(d) MMA3(d) |
//   out(a..d),
// so each tile's tensor-core work runs while the epilogue works on the other
// three.
// Every mbarrier wait is bounded; on expiry the kernel sets the timeout bit,
// the MMA lane drains its MMAs (bounded), and TMEM is freed after a final
// block barrier.
#include "common.cuh"
#include "tcgen05.cuh"

namespace hsc {

namespace {

using namespace tc;

constexpr int kUpThreads = 512;             // epilogue threads (16 warps)
constexpr int kUpBlock = kUpThreads + 32;    // + the MMA warp
constexpr int kUpRows = 128;            // MMA M, pixels per tile
constexpr int kHidden = HSC_UPSAMPLE_HIDDEN;
constexpr int kKBlocks = kHidden / 16;  // K = 16 steps of the hidden layers
constexpr int kSlots = 4;              // tiles in flight per CTA
constexpr unsigned kUpTmemCols = 512;   // slot s: columns [128 s, +128) for every layer (layer 3 in the first 16)
constexpr int kBlockBytes = kUpRows * 16 * 2;  // one [128 x 16] bf16 K-block

struct UpArgs {
  const float* rgb;  // P x 3
  int64_t P;
  const float* W1;   // 128 x 3
  const float* b1;
  const float* W2;   // 128 x 128
  const float* b2;
  const float* W3;   // k x 128
  const float* b3;
  int k;
  float* z;          // P x k
  unsigned int* err;
};

// Shared-memory plan (offsets from a 1024-byte aligned base).
constexpr int kOffW1 = 0;                                  // [128 x 16] bf16
constexpr int kOffW2 = kOffW1 + kBlockBytes;               // 8 x [128 x 16]
constexpr int kOffW3 = kOffW2 + kKBlocks * kBlockBytes;    // 8 x [16 x 16]
constexpr int kOffA1 = kOffW3 + kKBlocks * 512;            // kSlots x [128 x 16]
constexpr int kOffH = kOffA1 + kSlots * kBlockBytes;       // kSlots x 8 x [128 x 16]
constexpr int kSlotH = kKBlocks * kBlockBytes;
constexpr int kOffBias = kOffH + kSlots * kSlotH;          // b1, b2 (128 each), b3 (16)
constexpr int kOffBar = kOffBias + (2 * kHidden + 16) * 4; // 2 kSlots + 1 mbarriers, TMEM address, status
constexpr int kUpSmem = kOffBar + 128 + 1024;              // + alignment slack
static_assert(kSlots * kUpRows == kUpThreads, "every epilogue thread feeds one colour row");
static_assert(kSlots * 128 <= 512, "the slots' accumulators fit the TMEM");

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// SiLU of x given h = x / 2: x/2 (1 + tanh(x/2)) = h + h tanh(h).
__device__ __forceinline__ float silu_half(float h) { return __fmaf_rn(h, tanh_approx(h), h); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half)
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void issue_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Hand the shared-memory writes of every thread to the tensor core and order
// them before the MMA issued after the barrier (set-up only).
__device__ __forceinline__ void smem_to_mma_barrier() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// An epilogue thread's shared-memory writes (the next A operand) and its
// finished TMEM reads are handed to the MMA warp: proxy and tcgen05 fences,
// then one arrival on the slot's "operand ready" barrier (512 per phase).
__device__ __forceinline__ void operand_ready(uint32_t bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for a phase of an mbarrier; on expiry the status word and the
// device error word record it.  False also when another thread has already
// recorded an expiry, so every thread leaves the tile loop.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t& phase, volatile int* sOk, unsigned int* err) {
  const bool ok = mbar_wait(bar, phase);
  phase ^= 1u;
  if (!ok) {
    *sOk = 0;
    atomicOr(err, HSC_DEVERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return ok && *sOk != 0;
}

// Reads accumulator columns c0 .. c0+31 of this thread's TMEM lane, applies
// bias + SiLU, and writes them as bf16 into row `row` of the A operand `sH`
// (eight K = 16 blocks).
__device__ __forceinline__ void hidden_epilogue(uint32_t trow, int c0, const float* bias, unsigned char* sH,
                                                int row) {
  uint32_t v[32];
  TC_LD16(trow + (uint32_t)c0, v);
  TC_LD16(trow + (uint32_t)(c0 + 16), (v + 16));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int h = 0; h < 4; ++h) {  // 8 columns = 16 bytes of one core-matrix row
    const float4 bl = *reinterpret_cast<const float4*>(bias + c0 + 8 * h);
    const float4 bh = *reinterpret_cast<const float4*>(bias + c0 + 8 * h + 4);
    const float bb[8] = {bl.x, bl.y, bl.z, bl.w, bh.x, bh.y, bh.z, bh.w};
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x0 = silu_half(__fadd_rn(__uint_as_float(v[8 * h + 2 * q]), bb[2 * q]));
      const float x1 = silu_half(__fadd_rn(__uint_as_float(v[8 * h + 2 * q + 1]), bb[2 * q + 1]));
      w[q] = pack_bf16x2(x0, x1);
    }
    const int col = c0 + 8 * h;
    *reinterpret_cast<uint4*>(sH + (col >> 4) * kBlockBytes + kmajor_off(row, col & 15)) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__global__ void __launch_bounds__(kUpBlock, 1) upsample_tc_kernel(const UpArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sW1 = base + kOffW1;
  unsigned char* sW2 = base + kOffW2;
  unsigned char* sW3 = base + kOffW3;
  unsigned char* sA1 = base + kOffA1;
  unsigned char* sH = base + kOffH;
  float* sB1 = reinterpret_cast<float*>(base + kOffBias);
  float* sB2 = sB1 + kHidden;
  float* sB3 = sB2 + kHidden;
  // mbarriers: [s] MMA done of slot s (1 arrival: the commit), [kSlots + s]
  // operand ready of slot s (512 arrivals), [2 kSlots] drain
  uint64_t* sBar = reinterpret_cast<uint64_t*>(base + kOffBar);
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(sBar + 2 * kSlots + 1);
  volatile int* sOk = reinterpret_cast<volatile int*>(sTmem + 1);

  const int t = threadIdx.x;
  const int warp = t >> 5;
  const bool mma_warp = warp == kUpThreads / 32;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                 "r"(kUpTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int i = 0; i < kSlots; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sBar + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(sBar + kSlots + i)), "r"(kUpThreads)
                   : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sBar + 2 * kSlots)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sOk = 1;
  }
  // weights as bf16 B operands ([N x K], K-major), biases as FP32; the hidden
  // layers' weights and biases at half scale (exact), so that accumulator +
  // bias is x / 2 for the SiLU
  for (int idx = t; idx < kHidden * 16; idx += kUpBlock) {
    const int r = idx >> 4, e = idx & 15;
    const float v = e < 3 ? __ldg(a.W1 + r * 3 + e) : 0.0f;
    *reinterpret_cast<__nv_bfloat16*>(sW1 + kmajor_off(r, e)) = __float2bfloat16_rn(__fmul_rn(0.5f, v));
  }
  for (int idx = t; idx < kHidden * kHidden; idx += kUpBlock) {
    const int r = idx / kHidden, i = idx - r * kHidden;
    *reinterpret_cast<__nv_bfloat16*>(sW2 + (i >> 4) * kBlockBytes + kmajor_off(r, i & 15)) =
        __float2bfloat16_rn(__fmul_rn(0.5f, __ldg(a.W2 + idx)));
  }
  for (int idx = t; idx < 16 * kHidden; idx += kUpBlock) {
    const int r = idx / kHidden, i = idx - r * kHidden;
    const float v = r < a.k ? __ldg(a.W3 + r * kHidden + i) : 0.0f;
    *reinterpret_cast<__nv_bfloat16*>(sW3 + (i >> 4) * 512 + kmajor_off(r, i & 15)) = __float2bfloat16_rn(v);
  }
  for (int idx = t; idx < kHidden; idx += kUpBlock) {
    sB1[idx] = __fmul_rn(0.5f, __ldg(a.b1 + idx));
    sB2[idx] = __fmul_rn(0.5f, __ldg(a.b2 + idx));
  }
  if (t < 16) sB3[t] = t < a.k ? __ldg(a.b3 + t) : 0.0f;

  const int quad = warp & 3;                 // TMEM lane quadrant of this warp
  const int row = quad * 32 + (t & 31);      // pixel row = TMEM lane
  const int c0 = (warp >> 2) * 32;           // this thread's 32 hidden columns
  const int64_t tiles = (a.P + kUpRows - 1) / kUpRows;
  const int64_t groups = (tiles + kSlots - 1) / kSlots;   // kSlots tiles per group

  // Epilogue thread t feeds the colour of row t & 127 of slot t >> 7.
  const int feed_slot = t >> 7, feed_row = t & 127;
  float cr = 0.0f, cg = 0.0f, cb = 0.0f;
  auto load_colour = [&](int64_t group) {
    const int64_t p = (kSlots * group + feed_slot) * kUpRows + feed_row;
    const bool ok = t < kUpThreads && group < groups && p < a.P;
    cr = ok ? __ldg(a.rgb + 3 * p) : 0.0f;
    cg = ok ? __ldg(a.rgb + 3 * p + 1) : 0.0f;
    cb = ok ? __ldg(a.rgb + 3 * p + 2) : 0.0f;
  };
  load_colour(blockIdx.x);
  if (t < kUpThreads)  // the A1 rows' K columns 8..15 stay zero
    *reinterpret_cast<uint4*>(sA1 + feed_slot * kBlockBytes + kmajor_off(feed_row, 8)) = make_uint4(0u, 0u, 0u, 0u);
  smem_to_mma_barrier();
  const uint32_t tm = *sTmem;  // TMEM base address, published by the barrier above

  if (mma_warp) {
    if ((t & 31) == 0) {
      const uint32_t id_hidden = instr_desc_bf16(kUpRows, kHidden);
      const uint32_t id_out = instr_desc_bf16(kUpRows, 16);
      uint32_t rphase[kSlots] = {};
      bool ok = true;
      for (int64_t group = blockIdx.x; ok && group < groups; group += gridDim.x) {
        for (int layer = 1; ok && layer <= 3; ++layer) {
          for (int slot = 0; slot < kSlots; ++slot) {
            if (!wait_phase(smem_u32(sBar + kSlots + slot), rphase[slot], sOk, a.err)) {
              ok = false;
              break;
            }
            const uint32_t d = tm + (uint32_t)(128 * slot);
            if (layer == 1) {
              issue_mma(d, smem_desc(smem_u32(sA1 + slot * kBlockBytes), 128, 256), smem_desc(smem_u32(sW1), 128, 256),
                        id_hidden, 0);
            } else {
              const unsigned char* B = layer == 2 ? sW2 : sW3;
              const uint32_t bstride = layer == 2 ? (uint32_t)kBlockBytes : 512u;
#pragma unroll 1
              for (int kb = 0; kb < kKBlocks; ++kb)
                issue_mma(d, smem_desc(smem_u32(sH + slot * kSlotH + kb * kBlockBytes), 128, 256),
                          smem_desc(smem_u32(B + kb * bstride), 128, 256), layer == 2 ? id_hidden : id_out, kb > 0);
            }
            commit(smem_u32(sBar + slot));
          }
        }
      }
      // after an expired wait MMAs may still be running: drain them (bounded)
      // before TMEM is freed
      if (!ok) drain_mma(smem_u32(sBar + 2 * kSlots));
    }
  } else {
    auto trow = [&](int slot) { return tm + (uint32_t)(128 * slot) + ((uint32_t)(quad * 32) << 16); };
    auto ready = [&](int slot) { operand_ready(smem_u32(sBar + kSlots + slot)); };
    uint32_t dphase[kSlots] = {};
    auto done = [&](int slot) { return wait_phase(smem_u32(sBar + slot), dphase[slot], sOk, a.err); };
    auto out = [&](int slot, int64_t group) {
      if (warp < 4) {  // the layer-3 columns, one warp per lane quadrant
        uint32_t v[16];
        TC_LD16(trow(slot), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int64_t p = (kSlots * group + slot) * kUpRows + row;
        if (p < a.P) {
          float* zo = a.z + p * a.k;
#pragma unroll
          for (int o = 0; o < 16; ++o)
            if (o < a.k) zo[o] = __fadd_rn(__uint_as_float(v[o]), sB3[o]);
        }
      }
    };
    bool ok = true;
    for (int64_t group = blockIdx.x; ok && group < groups; group += gridDim.x) {
      // layer 1 A rows of every slot: the colours in bf16, K columns 0..2
      *reinterpret_cast<uint4*>(sA1 + feed_slot * kBlockBytes + kmajor_off(feed_row, 0)) =
          make_uint4(pack_bf16x2(cr, cg), pack_bf16x2(cb, 0.0f), 0u, 0u);
#pragma unroll 1
      for (int slot = 0; slot < kSlots; ++slot) ready(slot);
      load_colour(group + gridDim.x);  // the next group's colours, in flight from here on
      // the two hidden layers: while the tensor core runs one slot's MMA, the
      // epilogue works on the other slots
#pragma unroll 1
      for (int layer = 0; ok && layer < 2; ++layer) {
        const float* bias = layer == 0 ? sB1 : sB2;
#pragma unroll 1
        for (int slot = 0; slot < kSlots; ++slot) {
          if (!done(slot)) {
            ok = false;
            break;
          }
          // h2 replaces h1 in the slot's buffer: layer 2 has finished reading it
          hidden_epilogue(trow(slot), c0, bias, sH + slot * kSlotH, row);
          ready(slot);
        }
      }
#pragma unroll 1
      for (int slot = 0; ok && slot < kSlots; ++slot) {
        if (!done(slot)) {
          ok = false;
          break;
        }
        out(slot, group);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kUpTmemCols) : "memory");
  }
}

}  // namespace

}  // namespace hsc

extern "C" hsc_status hsc_upsample_rgb(hsc_ctx* ctx, const float* rgb, int64_t pixels, const float* W1,
                                       const float* b1, const float* W2, const float* b2, const float* W3,
                                       const float* b3, int k, float* z_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(pixels >= 0, "negative pixel count");
  HSC_REQUIRE(k >= 1 && k <= 16, "k=%d out of range [1, 16]", k);
  HSC_REQUIRE(W1 && b1 && W2 && b2 && W3 && b3, "null weight pointer");
  if (pixels == 0) return HSC_OK;
  HSC_REQUIRE(rgb && z_out, "null pointer");
  HSC_REQUIRE(hsc::aligned(rgb, 4) && hsc::aligned(z_out, 4) && hsc::aligned(W1, 4) && hsc::aligned(W2, 4) &&
                  hsc::aligned(W3, 4),
              "misaligned pointer");
  HSC_GUARD(ctx);
  hsc::UpArgs a{};
  a.rgb = rgb;
  a.P = pixels;
  a.W1 = W1;
  a.b1 = b1;
  a.W2 = W2;
  a.b2 = b2;
  a.W3 = W3;
  a.b3 = b3;
  a.k = k;
  a.z = z_out;
  a.err = ctx->d_err;
  cudaStream_t s = hsc::as_stream(stream);
  auto kern = hsc::upsample_tc_kernel;
  HSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, hsc::kUpSmem));
  const int64_t tiles = (pixels + hsc::kUpRows - 1) / hsc::kUpRows;
  const int64_t groups = (tiles + hsc::kSlots - 1) / hsc::kSlots;
  int64_t grid = ctx->sm_count;  // one CTA per SM (all 512 TMEM columns)
  if (grid > groups) grid = groups;
  kern<<<(unsigned)grid, hsc::kUpBlock, hsc::kUpSmem, s>>>(a);
  return hsc::check_launch("upsample_tc_kernel");
}
