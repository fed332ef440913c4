// h2_body.cuh -- one check of single-scan min-sum on packed binary16 frame pairs,
// shared by the frame-resident kernels (onchip_h2.cu: one CTA per frame group;
// multi_h2.cu: CTA sub-teams and thread-block clusters).
//
// Eq. (3) of Section IV with the Section V state (FORM 1: A, B, n~ and the signs
// per check) or per-edge messages (FORM 0).  Every quantity is an integer of
// magnitude < 2048, so binary16 holds it exactly and every f16x2 add, fma, min and
// max below is exact: the results are bit-identical to integer arithmetic.
//
// Where the posterior of a variable lives is a policy (Addr):
//   Addr::H                    handle of variable j of check m (index or pointer)
//   at(tab, Zs, j, m) -> H     look the handle up in the column table
//   load(Zs, h, w[P])          posterior pairs Z^(k-1) of the variable
//   add(Acc, h, p, v)          atomically add the message pattern v of pair p
//   st(m), lm(j, m)            element index of check m's state / of the
//                              message slot of its position j (pair 0)
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"
#include "h2ops.cuh"

namespace ldpc {

template <int G>
__device__ __forceinline__ void ld_pairs(const uint32_t* __restrict__ Zs, int n, uint32_t (&w)[G / 2]) {
  if constexpr (G == 2) {
    w[0] = Zs[n];
  } else {
    const uint2 v = reinterpret_cast<const uint2*>(Zs)[n];
    w[0] = v.x;
    w[1] = v.y;
  }
}
template <int G>
__device__ __forceinline__ void st_pairs(uint32_t* __restrict__ Zs, int n, const uint32_t (&w)[G / 2]) {
  if constexpr (G == 2) Zs[n] = w[0];
  else reinterpret_cast<uint2*>(Zs)[n] = make_uint2(w[0], w[1]);
}

// The policies hold only scalars: the table and posterior pointers are passed to
// check_body as __restrict__ parameters, so that loads of the table and of Zs
// may move past the accumulator atomics.
//
// Posteriors of this CTA's shared memory: Zs [N][P] half2, Acc [N][P] i32, with
// the edge-slot-major column table in shared memory (SIDX) or global memory.
template <int G, bool SIDX>
struct LocalAddr {
  static constexpr int P = G / 2;
  using H = int;
  int M;
  __device__ __forceinline__ H at(const uint16_t* __restrict__ tab, const uint32_t*, int j, int m) const {
    if constexpr (SIDX) return (int)tab[j * M + m];
    else return (int)__ldg(tab + j * M + m);
  }
  __device__ __forceinline__ void load(const uint32_t* __restrict__ Zs, H n, uint32_t (&w)[P]) const {
    ld_pairs<G>(Zs, n, w);
  }
  __device__ __forceinline__ void add(int32_t* __restrict__ Acc, H n, int p, int32_t v) const {
    atomicAdd(Acc + n * P + p, v);
  }
  __device__ __forceinline__ int st(int m) const { return m * P; }
  __device__ __forceinline__ int lm(int j, int m) const { return j * M + m; }
};

// (a b) >> 32 + c on 32-bit unsigned operands.
__device__ __forceinline__ uint32_t umad_hi(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d; asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); return d;
}

// |x| of both halves (an operand modifier of the instruction that consumes it).
__device__ __forceinline__ uint32_t hab(uint32_t a) {
  uint32_t d; asm("abs.f16x2 %0, %1;" : "=r"(d) : "r"(a)); return d;
}

// Section III's magnitude rule without branches: g(x) = max((x - beta) num, 0)
// >> shift (plain: beta 0, num 1, shift 0; offset: beta, 1, 0; normalized: 0,
// num, shift), which floors the normalized magnitude like the integer rule.
struct H2Rule {
  int32_t beta, num, shift;
  uint32_t cb;  // binary16 pair of 1025 - beta
  uint32_t c2;  // -0x64016401 num (mod 2^32)
  __device__ __forceinline__ int32_t g(int32_t x) const { return max((x - beta) * num, 0) >> shift; }
  // The same rule on a minimum's key K = (16 m + j - 7) 2^-11 (0 <= j <= 14),
  // without leaving binary16 for the offset: 1025 - beta + 128 K rounds to the
  // integer 1025 + m - beta (|j - 7| / 16 < 1/2; every value from 1024.5 on
  // has an exact integer grid), and the max with 1025 is 1025 + max(m - beta,
  // 0).  The scaling then acts on the integer halves of that pattern (0x6401 +
  // the value): pattern num - 0x64016401 num = value num per half (< 2^16, so
  // no carry crosses), shifted; bytes 0 and 2 hold g < 256.  Returns the
  // binary16 pair 1024 + g(m).
  __device__ __forceinline__ uint32_t pat(uint32_t K) const {
    const uint32_t a = hmax(hfma(K, h2c(128), cb), h2c(1025));
    return __byte_perm((a * (uint32_t)num + c2) >> shift, 0x64u, 0x4240);
  }
};
// beta, num, shift as H2Rule::g takes them (plain: 0, 1, 0; offset: beta, 1,
// 0; normalized: 0, num, shift), with beta <= 127.
__host__ __device__ inline H2Rule h2rule(int32_t beta, int32_t num, int32_t shift) {
  H2Rule h;
  h.beta = beta;
  h.num = num;
  h.shift = shift;
  h.cb = hbits(1025 - beta) * 0x10001u;
  h.c2 = 0u - 0x64016401u * (uint32_t)num;
  return h;
}
__host__ __device__ inline H2Rule make_h2rule(const IntRule& r) {
  return h2rule(r.rule == 1 ? r.beta : 0, r.rule == 2 ? r.num : 1, r.rule == 2 ? r.shift : 0);
}

// (j - 7) 2^-11 as a binary16 pair: the position term of the keys of checks of
// degree <= 15.
__host__ __device__ constexpr uint32_t key_pos15(int j) {
  return j >= 7 ? h2c_q11(j - 7) : (h2c_q11(7 - j) | 0x80008000u);
}

// Decision parity of check m for the G frames (bit g set: unsatisfied).
template <int G, int D, int DMAX, class Addr>
__device__ __forceinline__ uint32_t row_parity_body(const Addr& ad, const uint16_t* __restrict__ tab,
                                                    const uint32_t* __restrict__ Zs, int m, int d) {
  constexpr int P = G / 2;
  constexpr int NJ = D > 0 ? D : DMAX;
  uint32_t y[P];
#pragma unroll
  for (int p = 0; p < P; ++p) y[p] = 0;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      uint32_t w[P];
      ad.load(Zs, ad.at(tab, Zs, j, m), w);
#pragma unroll
      for (int p = 0; p < P; ++p) y[p] ^= dec_bits(w[p]);
    }
  }
  uint32_t par = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) par |= ((y[p] >> 15) & 1u) << (2 * p) | ((y[p] >> 31) & 1u) << (2 * p + 1);
  return par;
}

// One check m for all G frames: Eq. (3) with the Section V state (FORM 1) or
// per-edge messages (FORM 0).  D > 0: the check has exactly D positions (fully
// unrolled); D == 0: d <= DMAX positions, guarded.  Returns the decision parity
// bits of x^(k-1) when ES.
//   St  (FORM 1) [rows][P] {A, B, n~ as half2; signs, bit-reversed: the sign of
//       position j of the even frame at bit 15 - j, of the odd frame at bit
//       31 - j, so that shifting the word left by j (a running S + S) brings both
//       to the binary16 sign bits}
//       C8 (checks of degree <= 8, magnitudes <= 255): 8 bytes per frame pair,
//       the size of Section V's state, [rows][P] uint2 (St then addresses uint2
//       entries) {A_even, A_odd, B_even, B_odd as bytes; n~_even | signs_even
//       << 8 | n~_odd << 16 | signs_odd << 24}: the sign bytes sit where the
//       16-byte form keeps them, and the bytes below them are never shifted up
//       to a sign bit within 8 positions
//   Lm  (FORM 0) [ell_w][rows][P] u16: L + 128 per frame (one byte each)
//   ACC: how the new messages reach the posteriors.  0: add L^(k) into the
//       accumulator; 1: add L^(k) - L^(k-1) (an accumulator that holds Z^(k-1)
//       and is never reset; the streaming kernels); 2: update the posterior in
//       place, Z_n <- Z_n + L^(k) - L^(k-1), through Addr::update (the layered
//       schedule, where the checks running together share no variable)
template <int G, int FORM, int D, int DMAX, bool ES, class Addr, int ACC = 0, bool C8 = false>
__device__ __forceinline__ uint32_t check_body(const Addr& ad, const uint16_t* __restrict__ tab,
                                               const uint32_t* __restrict__ Zs, int32_t* __restrict__ Acc,
                                               const H2Rule& rule, uint32_t qm2, int m, int d,
                                               uint4* __restrict__ St, uint16_t* __restrict__ Lm) {
  constexpr int P = G / 2;
  constexpr int NJ = D > 0 ? D : DMAX;
  // Checks of degree <= 8 (KH): keys (16 |u| + j - 7) 2^-11 and the minima
  // decoded in binary16 (H2Rule::pat); wider checks: keys (16 |u| + j) 2^-11
  // clamped to 1, decoded through integers.  The minima start at the key of a
  // magnitude saturated to Qm at the last position the key form holds:
  // (16 Qm + 7) 2^-11 or (16 Qm + 15) 2^-11.  (The binary16 decode holds up
  // to degree 15, but on the N=7493 code's checks of degree 14 and 15 the
  // frame-resident kernel ran 3 % slower with it: 2.89 against 2.80 ms.)
  constexpr bool KH = NJ <= 8;
  const uint32_t ksat = hfma(qm2, h2c_q11(16), h2c_q11(KH ? 7 : 15));
  // position constants of the stored n~: the pattern 1024 + n~ (8-byte state
  // under KH) or the value n~
  constexpr int IB = (KH && C8) ? 1024 : 0;
  // one frame pair: the pass-1 handles stay in registers for pass 2; two pairs
  // need those registers for state and reload them
  constexpr bool KEEP = (P == 1 && FORM == 1 && !ES && ACC != 2);
  using H = typename Addr::H;
  static_assert(!C8 || (FORM == 1 && DMAX <= 8 && D <= 8), "the 8-byte state holds checks of degree <= 8");
  uint32_t A2[P], B2[P], I2[P], S[P];
  if constexpr (FORM == 1) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      if constexpr (C8) {
        // byte b -> binary16 pattern 0x6400 + b = 1024 + b, minus 1024: exact
        const uint2 s = reinterpret_cast<const uint2*>(St)[ad.st(m) + p];
        A2[p] = hsub(__byte_perm(s.x, 0x64u, 0x4140), 0x64006400u);
        B2[p] = hsub(__byte_perm(s.x, 0x64u, 0x4342), 0x64006400u);
        I2[p] = __byte_perm(s.y, 0x64u, 0x4240);
        if constexpr (IB == 0) I2[p] = hsub(I2[p], 0x64006400u);
        S[p] = s.y;
      } else {
        const uint4 s = St[ad.st(m) + p];
        A2[p] = s.x;
        B2[p] = s.y;
        I2[p] = s.z;
        S[p] = s.w;
      }
    }
  }
  uint32_t K1[P], K2[P], NEG[P], Y[P], SR[P], D2[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    K1[p] = ksat;  // the minima start at the saturated key, so they never exceed it
    K2[p] = ksat;
    NEG[p] = 0;
    Y[p] = 0;
    if constexpr (FORM == 1) {
      SR[p] = S[p];
      D2[p] = hsub(B2[p], A2[p]);
    }
  }
  H col[KEEP ? NJ : 1];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      const H n = ad.at(tab, Zs, j, m);
      if constexpr (KEEP) col[j] = n;
      uint32_t w[P];
      ad.load(Zs, n, w);
      uint32_t lv = 0;
      if constexpr (FORM == 0) {
        if constexpr (P == 1) lv = Lm[ad.lm(j, m)];
        else lv = reinterpret_cast<const uint32_t*>(Lm)[ad.lm(j, m)];
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        uint32_t L;
        if constexpr (FORM == 1) {
          // f(A, B, n, n~) = A + (B - A) [j = n~] (exact: small integers), and the
          // stored sign s_mn on the binary16 sign bit
          L = hfma(D2[p], heq_one(I2[p], h2c(IB + j)), A2[p]) ^ (SR[p] & 0x80008000u);
          SR[p] += SR[p];
        } else {
          // byte L + 128 -> binary16 128 + (L + 128)/8 -> 8 h - 1152 = L
          const uint32_t b = (P == 1) ? lv : (lv >> (16 * p));
          L = hfma(__byte_perm(b, 0x58u, 0x4140), h2c(8), 0xE480E480u /* -1152 */);
        }
        const uint32_t u = hsub(w[p], L);
        if constexpr (ES) Y[p] ^= dec_bits(w[p]);
        // sign of u_j at bit 15 - j / 31 - j: the high word of (u & signs) 2^(32-j)
        // added to NEG (the bits are disjoint), one multiply-add on the FMA pipe
        if (j == 0) NEG[p] = u & 0x80008000u;
        else NEG[p] = umad_hi(u & 0x80008000u, 1u << (32 - j), NEG[p]);
        // key (16 |u| + j) 2^-11 clamped to 1 by one saturating multiply-add:
        // exact for |u| <= 127 (16 |u| + j < 2048 fits 11 significand bits).
        // Keys of |u| > Qm (Qm <= 127) exceed the minima's start (16 Qm + 15)
        // 2^-11, so the minima come out as 16 min(|u|, Qm) + j; where both
        // are saturated A = B and the position of the first does not matter.
        // KH: (16 |u| + j - 7) 2^-11, exact for |u| <= 127 and above the
        // start (16 Qm + 7) 2^-11 for every |u| > Qm (no clamp needed)
        const uint32_t key = KH ? hfma(hab(u), h2c_q11(16), key_pos15(j)) : hfma_sat(hab(u), h2c_q11(16), h2c_q11(j));
        // at j = 0 the second minimum stays the start value: every key is at
        // most 1, so min(ksat, max(ksat, key)) = ksat
        if (j != 0) K2[p] = hmin(K2[p], hmax(K1[p], key));
        K1[p] = hmin(K1[p], key);
      }
    }
  }

  const int dd = D > 0 ? D : d;
  const uint32_t dlane = ((1u << dd) - 1u) << (16 - dd);  // bits 16-d .. 15
  uint32_t An[P], Bn[P], In[P], Sn[P];
  uint32_t W0[C8 ? P : 1], W1[C8 ? P : 1];
  uint32_t par = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    // sign of L^(k)_mj = parity of all input signs xor own sign
    const uint32_t pm = ((__popc(NEG[p] & 0xffffu) & 1) ? 0x0000ffffu : 0u) |
                        ((__popc(NEG[p] >> 16) & 1) ? 0xffff0000u : 0u);
    Sn[p] = (NEG[p] ^ pm) & (dlane | (dlane << 16));
    if constexpr (KH) {
      // 1025 + m1 (the rounding of H2Rule::pat with beta = 0), then
      // 2048 K1 + (17424 - 16 (1025 + m1)) = 16 m1 + n~ - 7 + 1024 - 16 m1:
      // In holds the pattern 1017 + n~ (exact: the integers from 512 on)
      const uint32_t M1 = hfma(K1[p], h2c(128), h2c(1025));
      In[p] = hfma(K1[p], h2c(2048), hfma(M1, h2c(16) | 0x80008000u, h2c(17424)));
      const uint32_t Ap = rule.pat(K1[p]), Bp = rule.pat(K2[p]);  // 1024 + g(m)
      An[p] = hsub(Ap, 0x64006400u);
      Bn[p] = hsub(Bp, 0x64006400u);
      if constexpr (C8) {
        W0[p] = __byte_perm(Ap, Bp, 0x6420);
        W1[p] = (hadd(In[p], h2c(7)) & 0x00ff00ffu) | (Sn[p] & 0xff00ff00u);
      }
    } else {
      // keys back to 16 min(|u|, Qm) + j (exact: a power of two)
      const uint32_t k1 = hfma(K1[p], h2c(2048), 0u), k2 = hfma(K2[p], h2c(2048), 0u);
      const int32_t k1l = h_lo_int(k1), k1h = h_hi_int(k1);
      const int32_t k2l = h_lo_int(k2), k2h = h_hi_int(k2);
      const int32_t al = rule.g(k1l >> 4), ah = rule.g(k1h >> 4);
      const int32_t bl = rule.g(k2l >> 4), bh = rule.g(k2h >> 4);
      An[p] = small_to_h2(al, ah);
      Bn[p] = small_to_h2(bl, bh);
      In[p] = small_to_h2(k1l & 15, k1h & 15);
      if constexpr (C8) {
        W0[p] = (uint32_t)al | ((uint32_t)ah << 8) | ((uint32_t)bl << 16) | ((uint32_t)bh << 24);
        W1[p] = (uint32_t)(k1l & 15) | ((uint32_t)(k1h & 15) << 16) | (Sn[p] & 0xff00ff00u);
      }
    }
    if constexpr (ES) par |= ((Y[p] >> 15) & 1u) << (2 * p) | ((Y[p] >> 31) & 1u) << (2 * p + 1);
  }

  uint32_t SN[P], SO[P], Dn[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    SN[p] = Sn[p];
    Dn[p] = hsub(Bn[p], An[p]);
    if constexpr (ACC != 0 && FORM == 1) SO[p] = S[p];
  }
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      H n;
      if constexpr (KEEP) n = col[j];
      else n = ad.at(tab, Zs, j, m);
      uint32_t sv = 0;
      uint32_t lold = 0;
      if constexpr (ACC != 0 && FORM == 0) {
        if constexpr (P == 1) lold = Lm[ad.lm(j, m)];
        else lold = reinterpret_cast<const uint32_t*>(Lm)[ad.lm(j, m)];
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const uint32_t L = hfma(Dn[p], heq_one(In[p], h2c(KH ? 1017 + j : j)), An[p]) ^ (SN[p] & 0x80008000u);
        SN[p] += SN[p];
        int32_t v = (int32_t)hadd(L, h2c(1536));
        uint32_t Lo = 0;
        if constexpr (ACC != 0) {
          // the previous message of this position, as in pass 1
          if constexpr (FORM == 1) {
            Lo = hfma(D2[p], heq_one(I2[p], h2c(IB + j)), A2[p]) ^ (SO[p] & 0x80008000u);
            SO[p] += SO[p];
          } else {
            const uint32_t b = (P == 1) ? lold : (lold >> (16 * p));
            Lo = hfma(__byte_perm(b, 0x58u, 0x4140), h2c(8), 0xE480E480u);
          }
          // lane patterns 0x6600 + L: the 32-bit difference is the exact integer
          // (L - Lo)_lo + 65536 (L - Lo)_hi
          v -= (int32_t)hadd(Lo, h2c(1536));
        }
        if constexpr (ACC == 2) ad.update(n, p, L, Lo);
        else ad.add(Acc, n, p, v);
        if constexpr (FORM == 0) {
          const uint32_t hb = hfma(L, 0x30003000u /* 0.125 */, h2c(144));
          sv |= (uint32_t)__byte_perm(hb, 0u, 0x4420) << (16 * p);
        }
      }
      if constexpr (FORM == 0) {
        if constexpr (P == 1) Lm[ad.lm(j, m)] = (uint16_t)sv;
        else reinterpret_cast<uint32_t*>(Lm)[ad.lm(j, m)] = sv;
      }
    }
  }
  if constexpr (FORM == 1) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      if constexpr (C8) reinterpret_cast<uint2*>(St)[ad.st(m) + p] = make_uint2(W0[p], W1[p]);
      else St[ad.st(m) + p] = make_uint4(An[p], Bn[p], KH ? hsub(In[p], h2c(1017)) : In[p], Sn[p]);
    }
  }
  return par;
}

}  // namespace ldpc
