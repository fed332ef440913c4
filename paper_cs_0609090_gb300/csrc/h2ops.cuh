// h2ops.cuh -- packed binary16 helpers for exact small-integer arithmetic.
//
// Every value handled with these helpers is an integer of magnitude < 2048, which
// binary16 represents exactly; add, sub, fma and min/max of such values (with
// results in range) are therefore exact, two frames per instruction.
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

namespace ldpc {

// binary16 bit pattern of a small non-negative integer (compile time).
__host__ __device__ constexpr uint32_t hbits(int v) {
  int e = 0;
  while ((2 << e) <= v) ++e;
  return v == 0 ? 0u
                : (uint32_t)(((e + 15) << 10) |
                             (e <= 10 ? ((v - (1 << e)) << (10 - e)) : ((v - (1 << e)) >> (e - 10))));
}
__host__ __device__ constexpr uint32_t h2c(int v) { return hbits(v) * 0x10001u; }
// Pair of v 2^-11 for 0 <= v < 2048 (the exponent of v's pattern lowered by 11;
// every such value is a normal binary16 number).
__host__ __device__ constexpr uint32_t h2c_q11(int v) { return v == 0 ? 0u : (hbits(v) - (11u << 10)) * 0x10001u; }

__device__ __forceinline__ uint32_t hadd(uint32_t a, uint32_t b) {
  uint32_t d; asm("add.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d;
}
__device__ __forceinline__ uint32_t hsub(uint32_t a, uint32_t b) {
  uint32_t d; asm("sub.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d;
}
__device__ __forceinline__ uint32_t hfma(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d; asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); return d;
}
__device__ __forceinline__ uint32_t hfma_relu(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d; asm("fma.rn.relu.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); return d;
}
// a b + c clamped to [0, 1].
__device__ __forceinline__ uint32_t hfma_sat(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d; asm("fma.rn.sat.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); return d;
}
__device__ __forceinline__ uint32_t hmin(uint32_t a, uint32_t b) {
  uint32_t d; asm("min.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d;
}
__device__ __forceinline__ uint32_t hmax(uint32_t a, uint32_t b) {
  uint32_t d; asm("max.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d;
}
__device__ __forceinline__ uint32_t habs(uint32_t a) { return a & 0x7fff7fffu; }
__device__ __forceinline__ uint32_t heq_mask(uint32_t a, uint32_t b) {
  uint32_t d; asm("set.eq.u32.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d;
}
// 1.0 where the halves are equal, 0.0 elsewhere (binary16 pair).
__device__ __forceinline__ uint32_t heq_one(uint32_t a, uint32_t b) {
  uint32_t d; asm("set.eq.f16x2.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d;
}

// Exact conversions between int pairs (|v| < 2^22) and half2 (|v| <= 2048).
__device__ __forceinline__ uint32_t ints_to_h2(int32_t lo, int32_t hi) {
  const float flo = __int_as_float(0x4B400000 + lo) - 12582912.0f;
  const float fhi = __int_as_float(0x4B400000 + hi) - 12582912.0f;
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(fhi), "f"(flo));
  return d;
}
__device__ __forceinline__ int32_t h_lo_int(uint32_t h) { return __half2int_rz(__ushort_as_half((unsigned short)(h & 0xffffu))); }
__device__ __forceinline__ int32_t h_hi_int(uint32_t h) { return __half2int_rz(__ushort_as_half((unsigned short)(h >> 16))); }
// Small non-negative ints (< 1024) to half2: bit pattern 0x6400 + v is 1024 + v.
__device__ __forceinline__ uint32_t small_to_h2(int32_t lo, int32_t hi) {
  return hsub(0x64006400u + (uint32_t)lo + ((uint32_t)hi << 16), h2c(1024));
}

// prmt with sign replication: each output byte copies the sign of the selected byte
// when bit 3 of its selector nibble is set.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d; asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel)); return d;
}

// Decision x = 1 iff Z <= 0, as the sign bit of Z - 0.5 (Z is an integer).
__device__ __forceinline__ uint32_t dec_bits(uint32_t z) { return hsub(z, 0x38003800u); }


}  // namespace ldpc
