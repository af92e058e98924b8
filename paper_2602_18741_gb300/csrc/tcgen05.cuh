// Building blocks for the tcgen05 (5th-generation tensor core) kernels:
// shared-memory and instruction descriptors for the no-swizzle K-major
// layout, bounded mbarrier waits, and the 32x32b TMEM load.
#pragma once

#include "common.cuh"

namespace hsc {
namespace tc {

constexpr unsigned kWaitLimit = 1u << 26;  // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05 format): start address >> 4 in
// bits 0-13, leading-dimension byte offset >> 4 in 16-29, stride-dimension
// byte offset >> 4 in 32-45, the fixed value 0b001 in 46-48, base offset 0,
// swizzle mode 0 (none) in 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in 24-28.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with A = B = F16 (format code 0 in bits 7-9 and 10-12).
__host__ __device__ constexpr uint32_t instr_desc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row r, k-element e) in the no-swizzle K-major
// canonical layout with K = 16 bf16: core matrices of 8 rows x 16 bytes,
// the two K-halves 128 bytes apart (LBO), 8-row groups 256 bytes apart (SBO).
__device__ __forceinline__ uint32_t kmajor_off(int r, int e) {
  return (uint32_t)((r >> 3) * 256 + (e >> 3) * 128 + (r & 7) * 16 + (e & 7) * 2);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Expiry path of the kernels whose thread 0 issues every tcgen05.mma: one
// more commit, to `drain_bar` (an mbarrier initialised for one arrival and
// not used otherwise), makes that barrier track the completion of every
// asynchronous tcgen05 operation the thread issued before; thread 0 then
// waits for it, bounded, so that TMEM is freed only after the MMAs that may
// still write it have finished.  False if this wait expires as well.
__device__ __forceinline__ bool drain_mma(uint32_t drain_bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(drain_bar)
               : "memory");
  return mbar_wait(drain_bar, 0);
}

#define TC_LD16(taddr, v)                                                                                      \
  asm volatile(                                                                                                \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),        \
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])    \
      : "r"(taddr))

}  // namespace tc
}  // namespace hsc
