// tcgen05 building blocks shared by the tensor-core kernels (mor_tc.cu, mor_sparse.cu):
// shared-memory matrix descriptors for K-major operands without swizzle, the instruction
// descriptor of a kind::f16 MMA with bf16 operands and an FP32 accumulator, the byte
// offset of an element in the K-major core-matrix layout, and a bounded mbarrier wait.
#pragma once
#include <stdint.h>

namespace mor {
namespace tc {

constexpr int kKB = 32;  // K rows per operand block (two K = 16 MMA steps)

// start address, leading byte offset (between core matrices along K) and stride byte
// offset (between 8-row groups along M / N), each in 16-byte units; version 1 at bit 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; base offset 0, no swizzle
  return d;
}
__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  return (1u << 4)                       // accumulator FP32
         | (1u << 7) | (1u << 10)        // A, B bf16
         | ((uint32_t)(N >> 3) << 17)    // N / 8 (A, B K-major: bits 15, 16 zero)
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}
// byte offset of element (row r, k) of a K-major operand block of kKB columns: 8 x 8 core
// matrices of 128 bytes, 128 bytes apart along K and (kKB / 8) * 128 bytes apart along r
__device__ __forceinline__ uint32_t kmajor(int r, int k) {
  return (uint32_t)((r >> 3) * ((kKB / 8) * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// wait for phase `parity` of the mbarrier at shared address mb, for at most `budget`
// clock cycles; false when the budget ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mb), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}

}  // namespace tc
}  // namespace mor
