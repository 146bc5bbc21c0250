// tcgen05 with BF16 operands (kind::f16, FP32 accumulator in tensor memory): helpers in
// inline PTX for sm_103a, used with those of cc_tc.cuh (allocation, commit, waits, loads).
//
// Operands in shared memory without swizzle, as core matrices of 8 rows x 16 bytes.
// K-major: a core matrix holds 8 rows (M or N) x 8 consecutive BF16 values of K.
// MN-major: it holds 8 consecutive K indices (its rows) x 8 consecutive values of M or N.
// In both, the descriptor's leading byte offset is the step between core matrices adjacent
// along K, the stride byte offset the step between those adjacent along M or N.  One MMA
// consumes K = 16: two core matrices along K.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "cc_tc.cuh"

namespace cc {

// shared-memory matrix descriptor: start address, lbo (along K), sbo (along M or N),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc16_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B; a_mn / b_mn select
// the MN-major reading of A / B; N >> 3 and M >> 4 in their fields
__host__ __device__ constexpr uint32_t tc16_idesc(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) |
         ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) = A B^T (+ D when accumulate), issued by one thread
__device__ __forceinline__ void tc16_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :: "r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// eight FP32 values rounded to BF16 (to nearest, ties to even), packed into 16 bytes
__device__ __forceinline__ uint4 pack_bf16x8(const float (&v)[8]) {
  uint4 r;
  __nv_bfloat162 t;
  t = __floats2bfloat162_rn(v[0], v[1]); r.x = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[2], v[3]); r.y = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[4], v[5]); r.z = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[6], v[7]); r.w = *reinterpret_cast<uint32_t*>(&t);
  return r;
}

}  // namespace cc
