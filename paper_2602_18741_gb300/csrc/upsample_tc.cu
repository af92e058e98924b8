// RGB-to-latent upsampling (Sec. 5): per pixel a three-layer perceptron,
//     h1 = silu(W1 c + b1),  h2 = silu(W2 h1 + b2),  z = W3 h2 + b3,
// hidden width 128, on the 5th-generation tensor cores.
//
// A CTA takes tiles of 128 pixels; 16 epilogue warps and two MMA warps.  Per
// tile three FP16 MMAs with FP32 accumulation run in sequence, each issued by
// the first lane of an MMA warp and committed to the slot's "done" mbarrier:
//   layer 1: [128 x 16] x [16 x 128]   (colour in K columns 0..2, ones in 3..4),
//   layer 2: [128 x 144] x [144 x 128] (nine K = 16 steps),
//   layer 3: [128 x 144] x [144 x 16]  (k <= 16 outputs, zero-padded).
// The biases ride in the products: a bias b is the f16 pair hi = f16(b),
// lo = f16(b - hi) in two K columns of B, against two columns of ones in A
// (for layers 2 and 3 a ninth K step whose A block, ones in columns 0 and 1,
// is shared by every tile); 1 x hi and 1 x lo are exact, so the accumulator
// holds W x + b with b to about 2^-22 relative.
// The hidden layers' weights and biases are staged at half scale (exact), so
// an accumulator is h = x / 2 and SiLU(x) = x/2 (1 + tanh(x/2)) = h + h tanh(h):
// one hardware tanh and one FMA per value, the result rounded to f16 into the
// next layer's A operand in shared memory (no-swizzle K-major layout).  The
// MUFU tanh rate bounds the kernel.
// One CTA per SM works on four tiles at once (four A buffers, four
// 128-column TMEM regions; layer 3 reuses the first 16 columns of its tile's
// region once layer 2 has been read).  The epilogue warps form two teams of
// eight, team 0 for slots 0 and 2 and team 1 for slots 1 and 3; pixel row r
// is TMEM lane r, read by the two warps of the team in lane quadrant r / 32,
// each for 64 of the 128 hidden columns (tcgen05.ld in chunks of 16, the next
// chunk's load in flight during the SiLU of the current one).  A team works
// on one slot while the tensor core runs its other slot's MMA, and the two
// teams run independently, so the waits and hand-offs of one overlap the
// other's SiLU work on the shared MUFU units.  The hand-offs are mbarriers:
// every thread of a team arrives on the slot's "operand ready" barrier once
// its shared-memory writes and TMEM reads are done, and each team has its
// own MMA warp, which waits for its team's slots in the team's order (one
// lane serving all four slots in a fixed order would couple the teams, and
// one polling all four barriers issued too late).
// Every mbarrier wait is bounded (polls that may suspend the thread for a
// bounded time); on expiry the kernel sets the timeout bit, the MMA lane
// drains its MMAs (bounded), and TMEM is freed after a final block barrier.
#include "common.cuh"
#include "tcgen05.cuh"

namespace hsc {

namespace {

using namespace tc;

constexpr int kUpThreads = 512;             // epilogue threads (16 warps, two teams)
constexpr int kTeamThreads = kUpThreads / 2; // a team: 8 warps, 2 per TMEM lane quadrant
constexpr int kUpBlock = kUpThreads + 64;    // + one MMA warp per team
constexpr int kUpRows = 128;            // MMA M, pixels per tile
constexpr int kHidden = HSC_UPSAMPLE_HIDDEN;
constexpr int kKBlocks = kHidden / 16;  // K = 16 steps over the hidden units
constexpr int kKB = kKBlocks + 1;       // + the bias step
constexpr int kSlots = 4;              // tiles in flight per CTA
constexpr unsigned kUpTmemCols = 512;   // slot s: columns [128 s, +128) for every layer (layer 3 in the first 16)
constexpr int kBlockBytes = kUpRows * 16 * 2;  // one [128 x 16] f16 K-block

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
  bool z_pairs;      // k even and z 8-byte aligned
  unsigned int* err;
};

// Shared-memory plan (offsets from a 1024-byte aligned base).
constexpr int kOffW1 = 0;                                  // [128 x 16] f16
constexpr int kOffW2 = kOffW1 + kBlockBytes;               // 9 x [128 x 16]
constexpr int kOffW3 = kOffW2 + kKB * kBlockBytes;         // 9 x [16 x 16]
constexpr int kOffOnes = kOffW3 + kKB * 512;               // [128 x 16], ones in K columns 0 and 1
constexpr int kOffA1 = kOffOnes + kBlockBytes;             // kSlots x [128 x 16]
constexpr int kOffH = kOffA1 + kSlots * kBlockBytes;       // kSlots x 8 x [128 x 16]
constexpr int kSlotH = kKBlocks * kBlockBytes;
constexpr int kOffBar = kOffH + kSlots * kSlotH;           // 2 kSlots + 3 mbarriers, TMEM address, status
constexpr int kUpSmem = kOffBar + 128 + 1024;              // + alignment slack
static_assert(kUpSmem <= 227 * 1024, "shared-memory plan exceeds a CTA's 227 KB");
static_assert(kSlots * kUpRows == kUpThreads, "every epilogue thread feeds one colour row");
static_assert(kSlots == 4 && kTeamThreads == 2 * kUpRows, "two teams of two slots each");
static_assert(kSlots * 128 <= 512, "the slots' accumulators fit the TMEM");

__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
  const __half2 v = __floats2half2_rn(lo, hi);  // .x = lo (low half)
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// SiLU of x given h = x / 2: x/2 (1 + tanh(x/2)) = h + h tanh(h).  (The
// packed tanh.approx.f16x2 form runs at the same MUFU rate per result, so
// the FP32 form is used and only the result is rounded to f16.)
__device__ __forceinline__ float silu_half(float h) { return __fmaf_rn(h, tanh_approx(h), h); }

// A bias as two f16 values whose sum is b to about 2^-22 relative.
__device__ __forceinline__ __half bias_part(float b, bool low) {
  const __half hi = __float2half_rn(b);
  return low ? __float2half_rn(__fsub_rn(b, __half2float(hi))) : hi;
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
// then one arrival on the slot's "operand ready" barrier (kTeamThreads per
// phase).
__device__ __forceinline__ void operand_ready(uint32_t bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for a phase of an mbarrier (bit `bit` of `phases` holds the
// parity to wait for, flipped afterwards): one non-blocking test first (in
// the steady state the phase has long completed), then polls that may
// suspend the thread until the phase completes, for at most kSleepHintNs
// each.  On expiry the status word and the device error word record it and
// the thread leaves its loop; the others leave theirs at their own next wait,
// which can no longer complete (the status word is not read on success: each
// read would queue behind the SiLU's MUFU work).
constexpr uint32_t kSleepHintNs = 20000;     // per poll
constexpr unsigned kSleepPolls = 1u << 16;   // polls before a wait gives up (~1.3 s at most)

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  for (unsigned it = 0; it < kSleepPolls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(kSleepHintNs)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void record_timeout(volatile int* sOk, unsigned int* err) {
  *sOk = 0;
  atomicOr(err, HSC_DEVERR_TIMEOUT);
}

__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t& phases, int bit, volatile int* sOk,
                                           unsigned int* err) {
  const bool ok = mbar_wait_sleep(bar, (phases >> bit) & 1u);
  phases ^= 1u << bit;
  if (!ok) record_timeout(sOk, err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return ok;
}

// The registers a tcgen05.ld wrote are defined only after tcgen05.wait::ld;
// an empty asm that "modifies" each of them after the wait keeps the
// compiler from moving their first use above it.
template <int N>
__device__ __forceinline__ void tmem_regs_after_wait(uint32_t* v) {
#pragma unroll
  for (int i = 0; i < N; ++i) asm volatile("" : "+r"(v[i]));
}

// SiLU of 16 accumulators (each h = x / 2 with the bias already in) written
// as f16 into row `row`, columns c0 .. c0+15, of the A operand `sH` (eight
// K = 16 blocks).
__device__ __forceinline__ void silu_store16(const uint32_t* v, int c0, unsigned char* sH, int row) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // 8 columns = 16 bytes of one core-matrix row
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      w[q] = pack_f16x2(silu_half(__uint_as_float(v[8 * h + 2 * q])), silu_half(__uint_as_float(v[8 * h + 2 * q + 1])));
    const int col = c0 + 8 * h;
    *reinterpret_cast<uint4*>(sH + (col >> 4) * kBlockBytes + kmajor_off(row, col & 15)) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// A thread's 64 hidden columns c0 .. c0+63 of its TMEM lane in four chunks of
// 16: each chunk's TMEM load is in flight while the previous chunk's SiLU
// runs.
__device__ __forceinline__ void hidden_epilogue(uint32_t trow, int c0, unsigned char* sH, int row) {
  uint32_t va[16], vb[16];
  TC_LD16(trow + (uint32_t)c0, va);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  tmem_regs_after_wait<16>(va);
#pragma unroll
  for (int ch = 0; ch < 4; ch += 2) {
    TC_LD16(trow + (uint32_t)(c0 + 16 * ch + 16), vb);
    silu_store16(va, c0 + 16 * ch, sH, row);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    tmem_regs_after_wait<16>(vb);
    if (ch + 2 < 4) TC_LD16(trow + (uint32_t)(c0 + 16 * ch + 32), va);
    silu_store16(vb, c0 + 16 * ch + 16, sH, row);
    if (ch + 2 < 4) {
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      tmem_regs_after_wait<16>(va);
    }
  }
}

__global__ void __launch_bounds__(kUpBlock, 1) upsample_tc_kernel(const UpArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // pointer arithmetic on the shared array itself (not through an integer),
  // so the compiler keeps every access below in the shared address space
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sW1 = base + kOffW1;
  unsigned char* sW2 = base + kOffW2;
  unsigned char* sW3 = base + kOffW3;
  unsigned char* sOnes = base + kOffOnes;
  unsigned char* sA1 = base + kOffA1;
  unsigned char* sH = base + kOffH;
  // mbarriers: [s] MMA done of slot s (1 arrival: the commit), [kSlots + s]
  // operand ready of slot s (kTeamThreads arrivals), [2 kSlots + m] drain of
  // MMA warp m, [2 kSlots + 2] team 1's start (1 arrival)
  uint64_t* sBar = reinterpret_cast<uint64_t*>(base + kOffBar);
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(sBar + 2 * kSlots + 3);
  volatile int* sOk = reinterpret_cast<volatile int*>(sTmem + 1);

  const int t = threadIdx.x;
  const int warp = t >> 5;
  const bool mma_warp = warp >= kUpThreads / 32;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                 "r"(kUpTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int i = 0; i < kSlots; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sBar + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(sBar + kSlots + i)), "r"(kTeamThreads)
                   : "memory");
    }
    for (int i = 0; i < 3; ++i)  // the two drains and team 1's start
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sBar + 2 * kSlots + i)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sOk = 1;
  }
  // weights as f16 B operands ([N x K], K-major), each bias as an (hi, lo)
  // pair in the K columns that meet the ones of A; the hidden layers' weights
  // and biases at half scale (exact), so that the accumulator is x / 2 for
  // the SiLU
  for (int idx = t; idx < kHidden * 16; idx += kUpBlock) {
    const int r = idx >> 4, e = idx & 15;
    __half v = __float2half_rn(0.0f);
    if (e < 3) v = __float2half_rn(__fmul_rn(0.5f, __ldg(a.W1 + r * 3 + e)));
    else if (e < 5) v = bias_part(__fmul_rn(0.5f, __ldg(a.b1 + r)), e == 4);
    *reinterpret_cast<__half*>(sW1 + kmajor_off(r, e)) = v;
  }
  for (int idx = t; idx < kHidden * kKB * 16; idx += kUpBlock) {
    const int r = idx / (kKB * 16), i = idx - r * (kKB * 16);
    __half v = __float2half_rn(0.0f);
    if (i < kHidden) v = __float2half_rn(__fmul_rn(0.5f, __ldg(a.W2 + r * kHidden + i)));
    else if (i < kHidden + 2) v = bias_part(__fmul_rn(0.5f, __ldg(a.b2 + r)), i == kHidden + 1);
    *reinterpret_cast<__half*>(sW2 + (i >> 4) * kBlockBytes + kmajor_off(r, i & 15)) = v;
  }
  for (int idx = t; idx < 16 * kKB * 16; idx += kUpBlock) {
    const int r = idx / (kKB * 16), i = idx - r * (kKB * 16);
    __half v = __float2half_rn(0.0f);
    if (r < a.k) {
      if (i < kHidden) v = __float2half_rn(__ldg(a.W3 + r * kHidden + i));
      else if (i < kHidden + 2) v = bias_part(__ldg(a.b3 + r), i == kHidden + 1);
    }
    *reinterpret_cast<__half*>(sW3 + (i >> 4) * 512 + kmajor_off(r, i & 15)) = v;
  }
  for (int idx = t; idx < kUpRows * 16; idx += kUpBlock) {
    const int r = idx >> 4, e = idx & 15;
    *reinterpret_cast<__half*>(sOnes + kmajor_off(r, e)) = __float2half_rn(e < 2 ? 1.0f : 0.0f);
  }

  const int quad = warp & 3;                 // TMEM lane quadrant of this warp
  const int row = quad * 32 + (t & 31);      // pixel row = TMEM lane
  const int cg = warp >> 2;                  // column group 0..3
  const int team = cg >> 1;                  // team 0: slots 0, 2; team 1: slots 1, 3
  const int c0 = (cg & 1) * 64;              // this thread's 64 hidden columns
  const int64_t tiles = (a.P + kUpRows - 1) / kUpRows;
  const int64_t groups = (tiles + kSlots - 1) / kSlots;   // kSlots tiles per group

  // Team thread tt = t & 255 feeds the colour of row tt & 127 of the team's
  // slot team + 2 (tt >> 7).
  const int feed_slot = team + 2 * ((t & 255) >> 7), feed_row = t & 127;
  float cr = 0.0f, cg_ = 0.0f, cb = 0.0f;
  auto load_colour = [&](int64_t group) {
    const int64_t p = (kSlots * group + feed_slot) * kUpRows + feed_row;
    const bool ok = t < kUpThreads && group < groups && p < a.P;
    cr = ok ? __ldg(a.rgb + 3 * p) : 0.0f;
    cg_ = ok ? __ldg(a.rgb + 3 * p + 1) : 0.0f;
    cb = ok ? __ldg(a.rgb + 3 * p + 2) : 0.0f;
  };
  load_colour(blockIdx.x);
  if (t < kUpThreads)  // the A1 rows' K columns 8..15 stay zero
    *reinterpret_cast<uint4*>(sA1 + feed_slot * kBlockBytes + kmajor_off(feed_row, 8)) = make_uint4(0u, 0u, 0u, 0u);
  smem_to_mma_barrier();
  const uint32_t tm = *sTmem;  // TMEM base address, published by the barrier above

  if (mma_warp) {
    if ((t & 31) == 0) {
      // This warp's lane 0 issues every MMA of its team's two slots, in the
      // order the team hands them over: per group layer 1, 2, 3, each for
      // slot mteam then slot mteam + 2.
      const int mteam = warp - kUpThreads / 32;
      const uint32_t id_hidden = instr_desc_f16(kUpRows, kHidden);
      const uint32_t id_out = instr_desc_f16(kUpRows, 16);
      uint32_t rphase = 0u;  // parity bit per team slot
      bool ok = true;
      for (int64_t group = blockIdx.x; ok && group < groups; group += gridDim.x) {
        for (int layer = 1; ok && layer <= 3; ++layer) {
          for (int j = 0; j < 2; ++j) {
            const int slot = mteam + 2 * j;
            if (!wait_phase(smem_u32(sBar + kSlots + slot), rphase, j, sOk, a.err)) {
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
              for (int kb = 0; kb < kKB; ++kb) {  // the last step: ones x bias
                const unsigned char* A = kb < kKBlocks ? sH + slot * kSlotH + kb * kBlockBytes : sOnes;
                issue_mma(d, smem_desc(smem_u32(A), 128, 256), smem_desc(smem_u32(B + kb * bstride), 128, 256),
                          layer == 2 ? id_hidden : id_out, kb > 0);
              }
            }
            commit(smem_u32(sBar + slot));
          }
        }
      }
      // after an expired wait MMAs may still be running: drain them (bounded)
      // before TMEM is freed
      if (!ok) drain_mma(smem_u32(sBar + 2 * kSlots + mteam));
    }
  } else {
    auto trow = [&](int slot) { return tm + (uint32_t)(128 * slot) + ((uint32_t)(quad * 32) << 16); };
    auto ready = [&](int slot) { operand_ready(smem_u32(sBar + kSlots + slot)); };
    uint32_t dphase = 0u;  // parity bit per team slot (bit j: slot team + 2 j)
    auto done = [&](int j) { return wait_phase(smem_u32(sBar + team + 2 * j), dphase, j, sOk, a.err); };
    auto out = [&](int slot, int64_t group) {
      if ((cg & 1) == 0) {  // the layer-3 columns, one warp per lane quadrant
        uint32_t v[16];
        TC_LD16(trow(slot), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tmem_regs_after_wait<16>(v);
        const int64_t p = (kSlots * group + slot) * kUpRows + row;
        if (p < a.P) {
          float* zo = a.z + p * a.k;
          if (a.z_pairs) {  // k even and z 8-byte aligned: float2 stores
#pragma unroll
            for (int o = 0; o < 16; o += 2)
              if (o < a.k)
                *reinterpret_cast<float2*>(zo + o) = make_float2(__uint_as_float(v[o]), __uint_as_float(v[o + 1]));
          } else {
#pragma unroll
            for (int o = 0; o < 16; ++o)
              if (o < a.k) zo[o] = __uint_as_float(v[o]);
          }
        }
      }
    };
    bool ok = true;
    // Team 1 starts half a group after team 0 (once team 0 has run its first
    // layer-1 epilogues), so that the exposed waits of one team (the MMA
    // that a step has just handed over) fall in the other's SiLU work.
    const uint32_t start_bar = smem_u32(sBar + 2 * kSlots + 2);
    if (team == 1) {
      uint32_t sphase = 0u;
      ok = wait_phase(start_bar, sphase, 0, sOk, a.err);
    }
    bool started = team == 1;
    for (int64_t group = blockIdx.x; ok && group < groups; group += gridDim.x) {
      // layer 1 A rows of the team's slots: the colour in f16 (K columns
      // 0..2) and the ones that meet the bias pair (columns 3, 4)
      *reinterpret_cast<uint4*>(sA1 + feed_slot * kBlockBytes + kmajor_off(feed_row, 0)) =
          make_uint4(pack_f16x2(cr, cg_), pack_f16x2(cb, 1.0f), pack_f16x2(1.0f, 0.0f), 0u);
      ready(team);
      ready(team + 2);
      load_colour(group + gridDim.x);  // the next group's colours, in flight from here on
      // the two hidden layers: while the tensor core runs one slot's MMA, the
      // team works on its other slot (and the other team on its own two)
#pragma unroll 1
      for (int layer = 0; ok && layer < 2; ++layer) {
#pragma unroll 1
        for (int j = 0; j < 2; ++j) {
          if (!done(j)) {
            ok = false;
            break;
          }
          // h2 replaces h1 in the slot's buffer: layer 2 has finished reading it
          const int slot = team + 2 * j;
          hidden_epilogue(trow(slot), c0, sH + slot * kSlotH, row);
          ready(slot);
        }
        if (!started && ok) {
          started = true;
          if (t == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(start_bar) : "memory");
        }
      }
#pragma unroll 1
      for (int j = 0; ok && j < 2; ++j) {
        if (!done(j)) {
          ok = false;
          break;
        }
        out(team + 2 * j, group);
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
  HSC_REQUIRE(pixels <= (int64_t(1) << 38), "%lld pixels exceed one launch of the upsampler (2^38)",
              (long long)pixels);
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
  a.z_pairs = k % 2 == 0 && hsc::aligned(z_out, 8);
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
