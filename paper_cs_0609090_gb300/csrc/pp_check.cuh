// pp_check.cuh -- one check of the single scan (Section IV Eq. (3)) with the
// Section V state, on a frame pair in exact binary16 arithmetic: the pieces that
// the ping-pong decoders (pingpong.cu, persist.cu) share.  Every value is an
// integer of magnitude < 2048, so each f16x2 operation below is exact.
#pragma once
#include "h2_body.cuh"

namespace ldpc {

// Section V state of one check and frame pair as binary16 pairs: A, B, n~, and
// the sign word (sign of position j of the even frame at bit 15 - j, of the odd
// frame at bit 31 - j).
struct SV {
  uint32_t A, B, I, S;
};
template <bool C8>
struct SVUnit;
// 8 bytes: {A_even, A_odd, B_even, B_odd} and n~_even | signs_even << 8 |
// n~_odd << 16 | signs_odd << 24 (the signs where the 16-byte form has them)
template <>
struct SVUnit<true> {
  using T = uint2;
  __device__ __forceinline__ static SV unpack(uint2 s) {
    SV v;
    v.A = hsub(__byte_perm(s.x, 0x64u, 0x4140), 0x64006400u);
    v.B = hsub(__byte_perm(s.x, 0x64u, 0x4342), 0x64006400u);
    v.I = hsub(__byte_perm(s.y, 0x64u, 0x4240), 0x64006400u);
    v.S = s.y;
    return v;
  }
};
template <>
struct SVUnit<false> {
  using T = uint4;
  __device__ __forceinline__ static SV unpack(uint4 s) { return SV{s.x, s.y, s.z, s.w}; }
};

// Minima, first argmin and signs of one check (pass 1 of Eq. (3)): u_j = Z_j -
// L^(k-1)_j, keys (16 min(|u_j|, Qm) + j) 2^-11 from one saturating multiply-add
// (minima started at the saturated key), sign bits of u gathered at 15 - j /
// 31 - j.  Then the magnitudes g(min1), g(min2) of Section III's rule.
struct NewState {
  uint32_t An, Bn, In, Sn;  // binary16 pairs / sign word
  int32_t al, ah, bl, bh, il, ih;
};
__device__ __forceinline__ NewState finish_state(uint32_t K1, uint32_t K2, uint32_t NEG, int dd, const H2Rule& rule) {
  NewState n;
  const uint32_t dlane = ((1u << dd) - 1u) << (16 - dd);  // bits 16-d .. 15
  const uint32_t pm = ((__popc(NEG & 0xffffu) & 1) ? 0x0000ffffu : 0u) | ((__popc(NEG >> 16) & 1) ? 0xffff0000u : 0u);
  n.Sn = (NEG ^ pm) & (dlane | (dlane << 16));
  const uint32_t k1 = hfma(K1, h2c(2048), 0u), k2 = hfma(K2, h2c(2048), 0u);
  const int32_t k1l = h_lo_int(k1), k1h = h_hi_int(k1);
  const int32_t k2l = h_lo_int(k2), k2h = h_hi_int(k2);
  n.al = rule.g(k1l >> 4);
  n.ah = rule.g(k1h >> 4);
  n.bl = rule.g(k2l >> 4);
  n.bh = rule.g(k2h >> 4);
  n.il = k1l & 15;
  n.ih = k1h & 15;
  n.An = small_to_h2(n.al, n.ah);
  n.Bn = small_to_h2(n.bl, n.bh);
  n.In = small_to_h2(n.il, n.ih);
  return n;
}

// Position j of a check; K1 = K2 = the saturated key before position 0.  At
// j = 0 the second minimum stays the saturated key (every key is at most 1 and
// min(ksat, max(ksat, key)) = ksat), so only the first is updated.
__device__ __forceinline__ void key_step(uint32_t u, int j, uint32_t& K1, uint32_t& K2, uint32_t& NEG) {
  if (j == 0) NEG = u & 0x80008000u;
  else NEG = umad_hi(u & 0x80008000u, 1u << (32 - j), NEG);
  const uint32_t key = hfma_sat(hab(u), h2c_q11(16), h2c_q11(j));
  if (j != 0) K2 = hmin(K2, hmax(K1, key));
  K1 = hmin(K1, key);
}

// Pass 1 of one check, Section V form: w[j] = Z^(k-1) of position j, o1 the
// state of iteration k-1; returns the minima, the first argmin and the signs
// (as new state) and, in par, the decision parity of x^(k-1) (bit 0 even frame,
// bit 1 odd frame).
// `two` doubles the running sign word (x * two, two = 2): a constant lets the
// compiler shift or add; a value it cannot see (a kernel argument) makes it an
// integer multiply, which runs on the FMA pipe instead of the ALU pipe.
template <int D, int DMAX, bool ES>
__device__ __forceinline__ NewState sv_pass1(const uint32_t* w, int d, const SV& o1, const H2Rule& rule,
                                             uint32_t ksat, uint32_t& par, uint32_t two = 2u) {
  constexpr int NJ = D > 0 ? D : DMAX;
  uint32_t K1 = ksat, K2 = ksat, NEG = 0, Y = 0, SR = o1.S;
  const uint32_t D1 = hsub(o1.B, o1.A);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      // f(A, B, n, n~) = A + (B - A) [j = n~], the sign s_mn on the binary16 sign bit
      const uint32_t L = hfma(D1, heq_one(o1.I, h2c(j)), o1.A) ^ (SR & 0x80008000u);
      SR *= two;
      const uint32_t u = hsub(w[j], L);
      if (ES) Y ^= dec_bits(w[j]);
      key_step(u, j, K1, K2, NEG);
    }
  }
  if (ES) par = ((Y >> 15) & 1u) | ((Y >> 30) & 2u);
  return finish_state(K1, K2, NEG, D > 0 ? D : d, rule);
}

// byte pair L + 128 (u16) -> binary16 pair L: 128 + (L + 128)/8 -> 8 h - 1152
__device__ __forceinline__ uint32_t pe_to_h2(uint32_t b) {
  return hfma(__byte_perm(b, 0x58u, 0x4140), h2c(8), 0xE480E480u);
}
// binary16 pair L -> byte pair L + 128
__device__ __forceinline__ uint32_t h2_to_pe(uint32_t L) {
  return __byte_perm(hfma(L, 0x30003000u /* 0.125 */, h2c(144)), 0u, 0x4420) & 0xffffu;
}

}  // namespace ldpc
