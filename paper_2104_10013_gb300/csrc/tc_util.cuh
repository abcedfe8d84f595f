// Shared pieces of the tensor-core kernels (eval_tc.cu, step_tc.cu):
// tcgen05 instruction and shared-memory descriptors, the MMA issue, the
// TF32 hi/lo split and tensor-memory loads.
//
// Operands are K-major in the no-swizzle canonical layout: a core matrix is
// 8 rows (of M or N) x 16 bytes (4 tf32 values along K), stored contiguously
// (128 bytes); the descriptor gives the byte distance between core matrices
// adjacent in K (lbo) and between 8-row groups (sbo).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace xp {

constexpr int TC_ROWS = 128;
constexpr int TC_A_LBO = TC_ROWS * 16;   // bytes between K-adjacent core matrices of A

// kind::tf32, D f32, A and B tf32, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t tc_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);
}

// no-swizzle K-major shared-memory descriptor: lbo = bytes between core
// matrices adjacent in K, sbo = bytes between 8-row groups
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// x rounded to the nearest tf32 value (10 explicit mantissa bits; halfway
// cases away from zero) by integer arithmetic on the fp32 bit pattern; the
// tensor cores then read it exactly.
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// hi/lo split: x = hi + lo + e with hi = rna(x), lo = rna(x - hi) and
// |e| <= 2^-22 |x| (x - hi is exact in fp32 and |x - hi| <= 2^-11 |x|)
__device__ __forceinline__ float2 tf32_split(float x) {
  const float hi = tf32_rna(x);
  return make_float2(hi, tf32_rna(x - hi));
}

// A element (row r, column j): 8-row groups 128 bytes apart, K-adjacent core
// matrices TC_A_LBO bytes apart, so the 16-byte chunks of a column group sit
// row after row (conflict-free across a warp).
__device__ __forceinline__ int a_off(int r, int j) { return (j >> 2) * (TC_A_LBO / 4) + r * 4 + (j & 3); }

// Loads 16 columns of this thread's tensor-memory lane (no wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

// Ties registers loaded from tensor memory to the wait before it: no use of
// them moves above the wait.
__device__ __forceinline__ void tmem_fence_regs8(uint32_t* v) {
  asm volatile("" : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]));
}

}  // namespace xp
