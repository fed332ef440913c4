// common.cuh -- device-side types shared by the decoder kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ldpc {

// Check->variable adjacency N(m) of H (Section II), resident in device memory.
struct DevCode {
  int32_t N, M, E;
  const int32_t* __restrict__ rp;  // [M+1]
  const int32_t* __restrict__ ci;  // [E]
  const int32_t* __restrict__ cdeg;  // [N] number of checks of each variable, |M(n)|
  // The same adjacency transposed to edge-slot-major order for coalesced loads,
  // with the checks in an internal order sorted by degree: variable of position j
  // of internal check i at ell[j * M + i] (j < ell_w, padded with the check's last
  // variable); uint16 when N <= 65535, else int32.
  const uint16_t* __restrict__ ell16;
  const int32_t* __restrict__ ell32;
  const uint8_t* __restrict__ rdeg;  // [M] degrees |N(m)| in the internal check order
  int32_t ell_w;
  // Variable->check adjacency M(n) for the two-scan comparator only: the edge
  // slots (j * M + m) of variable n are cslot[cptr[n] .. cptr[n+1]-1].
  const int32_t* __restrict__ cptr;   // [N+1]
  const int32_t* __restrict__ cslot;  // [E]
  // The same edges as (internal check index) | (position j << 24) (the
  // compressed two-scan's vertical scan); null when M >= 2^24.
  const uint32_t* __restrict__ ccj;   // [E]
  // The internal order sorted by degree as runs: checks [dc_end[i-1], dc_end[i])
  // have degree dc_deg[i] (n_dc <= 4 runs; otherwise n_dc = 0 and rdeg serves).
  int32_t n_dc;
  int32_t dc_end[4];
  int32_t dc_deg[4];
  __device__ __forceinline__ int col(int j, int m) const {
    return ell16 != nullptr ? (int)__ldg(ell16 + (size_t)j * M + m) : __ldg(ell32 + (size_t)j * M + m);
  }
  __device__ __forceinline__ int deg(int m) const {
    if (n_dc == 0) return (int)__ldg(rdeg + m);
    int d = dc_deg[0];
#pragma unroll
    for (int i = 1; i < 4; ++i)
      if (i < n_dc && m >= dc_end[i - 1]) d = dc_deg[i];
    return d;
  }
};

// Magnitude modification of Section III applied to integer magnitudes:
// plain; offset |L| <- max(|L| - beta, 0); normalized |L| <- floor(num |L| / 2^shift).
struct IntRule {
  int32_t rule;   // 0 plain, 1 offset, 2 normalized
  int32_t beta;
  int32_t num;
  int32_t shift;
  int32_t qm;     // message saturation Qm
  int32_t psat;   // > 0: the stored posterior is clamped to [-psat, psat] (8-bit posterior); 0: exact
  __device__ __forceinline__ int32_t g(int32_t mag) const {
    if (rule == 1) return max(mag - beta, 0);
    if (rule == 2) return (mag * num) >> shift;
    return mag;
  }
};

struct F32Rule {
  int32_t rule;
  float beta;
  float lambda;
  __device__ __forceinline__ float g(float mag) const {
    if (rule == 1) return fmaxf(mag - beta, 0.0f);
    if (rule == 2) return lambda * mag;
    return mag;
  }
};

// Two int16 posteriors of a frame pair packed in one 32-bit word as independent
// halves (low half = even frame).
__device__ __forceinline__ int32_t lo16(uint32_t w) { return (int32_t)(int16_t)(w & 0xffffu); }
__device__ __forceinline__ int32_t hi16(uint32_t w) { return ((int32_t)w) >> 16; }
__device__ __forceinline__ uint32_t pack16(int32_t lo, int32_t hi) {
  return ((uint32_t)lo & 0xffffu) | ((uint32_t)hi << 16);
}

// Accumulator form of a frame pair: the integer lo + 65536 hi.  Integer addition
// is associative, so atomically adding (l_lo + 65536 l_hi) from any number of
// checks in any order gives exactly (sum_lo + 65536 sum_hi); as long as both
// final sums lie in [-32768, 32767] they are recovered exactly by acc_to_pair.
__device__ __forceinline__ int32_t acc_pack(int32_t lo, int32_t hi) {
  return (int32_t)((uint32_t)lo + ((uint32_t)hi << 16));
}
// Convert accumulator form to independent halves: the high half of the integer
// lo + 65536 hi is hi - 1 exactly when lo < 0 (bit 15 of the low half set).
__device__ __forceinline__ uint32_t acc_to_pair(int32_t a) {
  const uint32_t w = (uint32_t)a;
  return w + ((w & 0x8000u) << 1);
}

}  // namespace ldpc
