// pingpong.cu -- single-scan min-sum (Section IV Eq. (3); Section V) with the
// frame state in device memory, one kernel launch per iteration and no column
// pass, for codes whose checks all have degree <= 8.
//
// Workspace (lane unit = frame pair, FP pairs, a multiple of 64; a warp lane
// takes two neighbouring pairs, so a warp covers 64 pairs = 128 frames):
//   zb [2][N][FP] half2  two posterior buffers.  Iteration k reads Z^(k-1) from
//                        zb[(k-1)&1] and adds L^(k) - L^(k-2) into zb[k&1], which
//                        holds Z^(k-2): afterwards zb[k&1] holds Z^(k).  Both
//                        buffers start at Z^(0) = q0, with L^(0) = L^(-1) = 0.  The
//                        adds are f16x2 atomics (two pairs per 8-byte add).  Every
//                        partial sum is q0_n plus one message of each check of n
//                        (of iteration k or k-2), an integer of magnitude <= 128 +
//                        d_v Qm < 2048, which binary16 holds exactly: the sums are
//                        exact and do not depend on the order of the atomics.
//   st [2][rows][FP]     Section V state of iterations k-1 and k-2 in 8 bytes per
//                        pair (A, B, n~, signs; rows = M), or per-edge bytes L +
//                        128 (u16 per pair, rows = ell_w M edge slots);
//                        iteration k reads both and overwrites the older.
//   act/fail [3][FP]     bit masks per pair: frames running at iteration j, and
//                        frames whose decisions x^(j-1) fail a check (found by
//                        iteration j), at index j mod 3.
//   iters [2 FP], okw [FP].
//
// Kernels per decode: init (channel values to both buffers, flags), one row
// kernel per iteration, the final syndrome, the output.  The row kernel of
// iteration k finds the parity of x^(k-1); that of k+1 stops the frames whose
// x^(k-1) satisfied H (Section III's stop rule, also checked before the first
// iteration): their result Z^(k-1) is in zb[(k-1)&1], and they are masked out
// of every later atomic.
#include <algorithm>

#include "async_copy.cuh"
#include "h2_body.cuh"
#include "kernels.h"
#include "pp_check.cuh"

namespace ldpc {
namespace {

// Section V rows of uniform degree stage the next check's inputs in shared
// memory (rows_staged); 0 reads them straight from global memory.
#ifndef LDPC_PP2_STAGED
#define LDPC_PP2_STAGED 1
#endif

constexpr uint32_t kFull = 0xffffffffu;
// CTAs per SM of the per-edge row kernel (registers 65536 / (256 x this)): its
// staged body needs 80 registers; at 64 it spills 580 bytes (N=64800 per-edge
// decode: 11.05 ms staged at 3, 14.10 ms staged at 4, 11.36 ms unstaged at 4)
#ifndef LDPC_PP2_MINB0
#define LDPC_PP2_MINB0 3
#endif
#ifndef LDPC_PP2_STAGED_PE
#define LDPC_PP2_STAGED_PE 1
#endif
#ifndef LDPC_PP2_STAGES
#define LDPC_PP2_STAGES 2
#endif
#ifndef LDPC_PP2_GROUPS
#define LDPC_PP2_GROUPS 1
#endif
#ifndef LDPC_PP2_MINB1
#define LDPC_PP2_MINB1 4
#endif
#ifndef LDPC_PP2_SHIFT_FMA
#define LDPC_PP2_SHIFT_FMA 1
#endif
#ifndef LDPC_PP2_EQ_FMA
#define LDPC_PP2_EQ_FMA 0
#endif
#ifndef LDPC_PP2_UNROLL
#define LDPC_PP2_UNROLL 4
#endif
#ifndef LDPC_PP2_ALT_ORDER
#define LDPC_PP2_ALT_ORDER 1
#endif

constexpr int kWarps = 8;   // per block of pp2_final (the row kernel takes its block size from the caller)
constexpr int kRowWarpsMax = 16;  // the row kernel takes 4, 8 or 16 warps per block
// registers per thread of the row kernel: those of MINB CTAs of 256 threads per
// SM, rounded down to the allocation unit of 8
constexpr int kRegs1 = (65536 / (LDPC_PP2_MINB1 * 256)) & ~7;
constexpr int kRegs0 = (65536 / (LDPC_PP2_MINB0 * 256)) & ~7;
constexpr int kRows = 4;    // checks per handle group (kRows x degree <= 32 lanes)
constexpr int kTile = kWarps * kRows;
constexpr int kStages = LDPC_PP2_STAGES;  // staged checks in flight + 1
constexpr int kGroups = LDPC_PP2_GROUPS;  // handle groups per warp in the row kernel
constexpr int kUnroll = LDPC_PP2_UNROLL;   // unrolling of the staged check loop
// sign-word doubling as a multiply (N=64800, same GB300: 7.617 against 7.653 ms)
constexpr bool kShiftFma = LDPC_PP2_SHIFT_FMA != 0;
// position indicators of the delta on the FMA pipe: more instructions for a
// lighter ALU pipe, which lost (N=64800: 8.00 against 7.59 ms)
constexpr bool kEqFma = LDPC_PP2_EQ_FMA != 0;

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Chunk (64 pairs) of a row or syndrome launch for iteration k.  Blocks start in
// chunk-major order (blockIdx.y is the slow index), and successive iterations
// take the chunks in opposite orders, so that each iteration starts on the
// chunks whose posterior lines and states the previous one touched last and
// left in L2.
__device__ __forceinline__ int chunk_of(int k) {
  return (LDPC_PP2_ALT_ORDER && (k & 1)) ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
}

struct PP2 {
  uint32_t* zb;    // [2][N][FP]
  char* st;        // [2][rows][FP] units of ub bytes
  uint32_t* act;   // [3][FP]
  uint32_t* fail;  // [3][FP]
  int32_t* iters;  // [2 FP]
  uint32_t* okw;   // [FP]
  int32_t F, FP, rows, ub;
  uint32_t two;    // 2 (a value the compiler cannot fold; see sv_pass1)
};

__device__ __forceinline__ uint32_t half_mask(uint32_t b) {
  return ((b & 1u) ? 0x0000ffffu : 0u) | ((b & 2u) ? 0xffff0000u : 0u);
}
__device__ __forceinline__ uint32_t valid_bits(int p, int F) {
  return (2 * p < F ? 1u : 0u) | (2 * p + 1 < F ? 2u : 0u);
}

// 8-byte f16x2 atomic add of two frame pairs (no result).  No "memory" clobber:
// within a row kernel only these atomics touch the buffer they add to, so the
// compiler may move the next check's loads (other buffers) ahead of them.
__device__ __forceinline__ void red_add_h2x2(uint32_t* p, uint32_t a, uint32_t b) {
  asm volatile("red.global.add.noftz.v2.f16x2 [%0], {%1, %2};" ::"l"(p), "r"(a), "r"(b));
}

// Section V state of one check and frame pair as the row pass reads it: A and
// B - A as binary16 values, n~ as the pattern of 1024 + n~ (compared with
// 1024 + j), and the sign word.  The stored bytes become patterns 1024 + v with
// one byte permute each.
struct SVD {
  uint32_t A, D, Ip, S;
};
__device__ __forceinline__ SVD unpack_d(uint32_t x, uint32_t y) {
  const uint32_t Ap = __byte_perm(x, 0x64u, 0x4140), Bp = __byte_perm(x, 0x64u, 0x4342);
  return SVD{hsub(Ap, h2c(1024)), hsub(Bp, Ap), __byte_perm(y, 0x64u, 0x4240), y};
}

// [j = n~] as 1.0 / 0.0 from the pattern of 1024 + n~: a set instruction (ALU
// pipe), or sat(1 - |n~ - j|) with two FMA-pipe instructions (kEqFma)
__device__ __forceinline__ uint32_t pos_ind(uint32_t Ip, int j) {
  if constexpr (kEqFma) return hfma_sat(hab(hsub(Ip, h2c(1024 + j))), 0xBC00BC00u, 0x3C003C00u);
  else return heq_one(Ip, h2c(1024 + j));
}

// The new state of one check and frame pair from the keys K1, K2 = (16 m + j)
// 2^-11 of the two minima (j <= 7) and the sign bits NEG, all in binary16
// pairs.  1024 + 128 K rounds to the integer 1024 + m (j / 16 < 1/2), and
// 2048 K + (1024 - 16 m) = 1024 + j gives n~.  The rule g (Section III) acts
// on these patterns: the offset as max(1024 - beta + 128 K, 1024), again
// rounding away j / 16; the normalized scaling floor(m num / 2^shift) on the
// integer halves of the pattern, whose low 10 bits hold m.  A pattern 1024 + v
// (v < 256) keeps v in its low byte, so the stored bytes are byte permutes.
struct NewD {
  uint32_t An, Dn, Ip, Sn;  // A, B - A (values), 1024 + n~ (pattern), signs
  uint2 st;                 // the 8-byte stored state (pack layout of SVUnit<true>)
};
struct FinArgs {
  uint32_t cb;         // pair of 1024 - beta (offset rule)
  uint32_t num, shift; // normalized rule
};
template <bool NORM>
__device__ __forceinline__ NewD finish_d(uint32_t K1, uint32_t K2, uint32_t NEG, int dd, const FinArgs& f) {
  NewD n;
  const uint32_t dlane = ((1u << dd) - 1u) << (16 - dd);  // bits 16-d .. 15
  const uint32_t pm = ((__popc(NEG & 0xffffu) & 1) ? 0x0000ffffu : 0u) | ((__popc(NEG >> 16) & 1) ? 0xffff0000u : 0u);
  n.Sn = (NEG ^ pm) & (dlane | (dlane << 16));
  const uint32_t M1 = hfma(K1, h2c(128), h2c(1024));                               // 1024 + m1
  n.Ip = hfma(K1, h2c(2048), hfma(M1, h2c(16) | 0x80008000u, h2c(17408)));         // 1024 + n~
  uint32_t Ap, Bp;
  if constexpr (NORM) {
    const uint32_t M2 = hfma(K2, h2c(128), h2c(1024));
    Ap = __byte_perm(((M1 & 0x03ff03ffu) * f.num) >> f.shift, 0x64u, 0x4240);
    Bp = __byte_perm(((M2 & 0x03ff03ffu) * f.num) >> f.shift, 0x64u, 0x4240);
  } else {
    Ap = hmax(hfma(K1, h2c(128), f.cb), h2c(1024));
    Bp = hmax(hfma(K2, h2c(128), f.cb), h2c(1024));
  }
  n.An = hsub(Ap, h2c(1024));
  n.Dn = hsub(Bp, Ap);
  n.st = make_uint2(__byte_perm(Ap, Bp, 0x6420), (n.Ip & 0x00ff00ffu) | (n.Sn & 0xff00ff00u));
  return n;
}

// Pass 1 of one check (Section IV Eq. (3)) on the state of iteration k-1:
// u_j = Z_j - L^(k-1)_j with L rebuilt as A + (B - A) [j = n~] under the sign
// bit, minima keys and sign bits (key_step), and the decision parity of
// x^(k-1) (bit 0 even frame, bit 1 odd frame) when ES.
template <int D, bool ES>
__device__ __forceinline__ void pass1_d(const uint32_t* w, int d, const SVD& o, uint32_t ksat, uint32_t two,
                                        uint32_t& K1, uint32_t& K2, uint32_t& NEG, uint32_t& par) {
  constexpr int NJ = D > 0 ? D : 8;
  K1 = ksat;
  K2 = ksat;
  NEG = 0;
  uint32_t Y = 0, SR = o.S;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      const uint32_t L = hfma(o.D, pos_ind(o.Ip, j), o.A) ^ (SR & 0x80008000u);
      SR *= two;
      const uint32_t u = hsub(w[j], L);
      if (ES) Y ^= dec_bits(w[j]);
      key_step(u, j, K1, K2, NEG);
    }
  }
  if (ES) par = ((Y >> 15) & 1u) | ((Y >> 30) & 2u);
}

// L^(k)_j - L^(k-2)_j for successive positions j of one check and frame pair.
struct Delta {
  uint32_t An, Dn, In, SN;  // iteration k: A, B - A, 1024 + n~, signs (shifted as j advances)
  uint32_t Ao, Do, Io, SO;  // iteration k-2
  __device__ __forceinline__ Delta(const NewD& n, const SVD& o)
      : An(n.An), Dn(n.Dn), In(n.Ip), SN(n.Sn), Ao(o.A), Do(o.D), Io(o.Ip), SO(o.S) {}
  __device__ __forceinline__ uint32_t next(int j, uint32_t two) {
    const uint32_t Ln = hfma(Dn, pos_ind(In, j), An) ^ (SN & 0x80008000u);
    const uint32_t Lo = hfma(Do, pos_ind(Io, j), Ao) ^ (SO & 0x80008000u);
    SN *= two;
    SO *= two;
    return hsub(Ln, Lo);
  }
};

struct RowArgs {
  const uint32_t* Zr;  // Z^(k-1) at the lane's first pair
  uint32_t* Za;        // Z^(k-2) -> Z^(k), at the lane's first pair
  const char* S1;      // state of k-1 at the lane's first pair (bytes)
  char* S2;            // state of k-2, overwritten with k
  uint32_t FP, M;
  uint32_t amA, amB;   // running halves of the lane's two pairs
  uint32_t ksat;       // (16 Qm + 7) 2^-11: the largest key of a magnitude saturated to Qm
  uint32_t two;        // 2, doubling the running sign words (see sv_pass1)
  FinArgs fin;
};

// The Section V check from its inputs: posteriors wa / wb of the lane's two
// pairs at the check's positions, the 16-byte state words of iterations k-1
// (s1) and k-2 (s2).  Adds L^(k) - L^(k-2) at the handles h[j] and overwrites
// the k-2 state with the new one.  Returns the decision parities as check2.
template <bool ES, bool NORM, int D>
__device__ __forceinline__ uint32_t check2_sv(const RowArgs& x, int m, int d, const uint32_t* h, const uint32_t* wa,
                                              const uint32_t* wb, uint4 s1, uint4 s2) {
  constexpr int NJ = D > 0 ? D : 8;
  uint32_t pa = 0, pb = 0;
  const uint32_t two = kShiftFma ? x.two : 2u;
  uint32_t K1a, K2a, NEGa, K1b, K2b, NEGb;
  pass1_d<D, ES>(wa, d, unpack_d(s1.x, s1.y), x.ksat, two, K1a, K2a, NEGa, pa);
  pass1_d<D, ES>(wb, d, unpack_d(s1.z, s1.w), x.ksat, two, K1b, K2b, NEGb, pb);
  const int dd = D > 0 ? D : d;
  const NewD na = finish_d<NORM>(K1a, K2a, NEGa, dd, x.fin), nb = finish_d<NORM>(K1b, K2b, NEGb, dd, x.fin);
  Delta ga(na, unpack_d(s2.x, s2.y));
  Delta gb(nb, unpack_d(s2.z, s2.w));
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      // without early stop no frame is ever masked: the lanes past the batch
      // decode all-zero channel values (exact zeros throughout) that no output reads
      const uint32_t da = ES ? ga.next(j, two) & x.amA : ga.next(j, two);
      const uint32_t db = ES ? gb.next(j, two) & x.amB : gb.next(j, two);
      if (!ES || (x.amA | x.amB) != 0u) red_add_h2x2(x.Za + h[j], da, db);
    }
  }
  __stcg(reinterpret_cast<uint4*>(x.S2 + (size_t)m * x.FP * 8), make_uint4(na.st.x, na.st.y, nb.st.x, nb.st.y));
  return pa | (pb << 2);
}

// The per-edge check from its inputs: posteriors wa / wb of the lane's two
// pairs, the per-edge byte pairs of iterations k-1 (l1) and k-2 (l2) at each
// position.  Adds L^(k) - L^(k-2) at the handles h[j] and overwrites the k-2
// slots with L^(k).  Returns the decision parities as check2.
template <bool ES, bool NORM, int D>
__device__ __forceinline__ uint32_t check2_pe(const RowArgs& x, int m, int d, const uint32_t* h, const uint32_t* wa,
                                              const uint32_t* wb, const uint32_t* l1, const uint32_t* l2) {
  constexpr int NJ = D > 0 ? D : 8;
  uint32_t pa = 0, pb = 0;
  uint32_t K1a = x.ksat, K2a = x.ksat, NEGa = 0, Ya = 0, K1b = x.ksat, K2b = x.ksat, NEGb = 0, Yb = 0;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      key_step(hsub(wa[j], pe_to_h2(l1[j] & 0xffffu)), j, K1a, K2a, NEGa);
      key_step(hsub(wb[j], pe_to_h2(l1[j] >> 16)), j, K1b, K2b, NEGb);
      if (ES) {
        Ya ^= dec_bits(wa[j]);
        Yb ^= dec_bits(wb[j]);
      }
    }
  }
  const int dd = D > 0 ? D : d;
  const NewD na = finish_d<NORM>(K1a, K2a, NEGa, dd, x.fin), nb = finish_d<NORM>(K1b, K2b, NEGb, dd, x.fin);
  uint32_t SNa = na.Sn, SNb = nb.Sn;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      const uint32_t La = hfma(na.Dn, pos_ind(na.Ip, j), na.An) ^ (SNa & 0x80008000u);
      const uint32_t Lb = hfma(nb.Dn, pos_ind(nb.Ip, j), nb.An) ^ (SNb & 0x80008000u);
      SNa += SNa;
      SNb += SNb;
      const uint32_t da = ES ? hsub(La, pe_to_h2(l2[j] & 0xffffu)) & x.amA : hsub(La, pe_to_h2(l2[j] & 0xffffu));
      const uint32_t db = ES ? hsub(Lb, pe_to_h2(l2[j] >> 16)) & x.amB : hsub(Lb, pe_to_h2(l2[j] >> 16));
      if (!ES || (x.amA | x.amB) != 0u) red_add_h2x2(x.Za + h[j], da, db);
      __stcg(reinterpret_cast<uint32_t*>(x.S2 + (size_t)(j * x.M + m) * x.FP * 2), h2_to_pe(La) | (h2_to_pe(Lb) << 16));
    }
  }
  if (ES) {
    pa = ((Ya >> 15) & 1u) | ((Ya >> 30) & 2u);
    pb = ((Yb >> 15) & 1u) | ((Yb >> 30) & 2u);
  }
  return pa | (pb << 2);
}

// One check m of degree d (D > 0: exactly D) for the lane's two pairs, handles
// h[j] (variable x FP).  Returns the decision parities of x^(k-1) of both pairs
// (bits 0-1 first pair, 2-3 second).
template <int FORM, bool ES, bool NORM, int D>
__device__ __forceinline__ uint32_t check2(const RowArgs& x, int m, int d, const uint32_t* h) {
  constexpr int NJ = D > 0 ? D : 8;
  uint32_t wa[NJ], wb[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      const uint2 v = __ldcg(reinterpret_cast<const uint2*>(x.Zr + h[j]));
      wa[j] = v.x;
      wb[j] = v.y;
    }
  }
  if constexpr (FORM == 1) {
    const size_t so = (size_t)m * x.FP * 8;
    const uint4 s1 = __ldcg(reinterpret_cast<const uint4*>(x.S1 + so));
    const uint4 s2 = __ldcg(reinterpret_cast<const uint4*>(x.S2 + so));
    return check2_sv<ES, NORM, D>(x, m, d, h, wa, wb, s1, s2);
  } else {
    // per-edge: slot j M + m holds the byte pairs of both pairs in one word
    uint32_t l1[NJ], l2[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      if (D > 0 || j < d) {
        const size_t so = (size_t)(j * x.M + m) * x.FP * 2;
        l1[j] = __ldcg(reinterpret_cast<const uint32_t*>(x.S1 + so));
        l2[j] = __ldcg(reinterpret_cast<const uint32_t*>(x.S2 + so));
      }
    }
    return check2_pe<ES, NORM, D>(x, m, d, h, wa, wb, l1, l2);
  }
}

// Per-warp staging of the Section V checks of uniform degree D <= 7: the
// inputs of the checks kStages - 1 ahead (D posterior pairs and both state
// words per lane) are copied into shared memory while the current check
// computes, so that the gathers' latency overlaps the arithmetic instead of
// stalling it.  A warp takes kGroups groups of kRows checks (one lane-held
// handle word per group).  Measured on the N=64800 code (1024 frames, 50
// iterations, same GB300), two stages, one group: 8.13 ms against 8.73 ms with
// the inputs read straight from global memory; three stages 8.87 ms, two
// groups 8.35 ms, four groups 13.1 ms; the loop unrolled 1 or 2 times instead
// of 4: +1.6 % / +1.3 %.
template <int FORM>
struct Stage;
template <>
struct Stage<1> {  // posterior pairs and both 16-byte state words per lane
  uint2 z[kStages][7][32];
  uint4 s[kStages][2][32];
};
template <>
struct Stage<0> {  // posterior pairs and the k-1 / k-2 message words of each position
  uint2 z[kStages][7][32];
  uint32_t l1[kStages][7][32];
  uint32_t l2[kStages][7][32];
};
// per-edge staging: 57,344 bytes per 8-warp CTA, so that 4 CTAs with their
// 1 KB reservations fill the SM's 233,472 bytes exactly

template <int FORM, bool ES, bool NORM, int D>
__device__ __forceinline__ uint32_t rows_staged(const RowArgs& x, int m0, const uint32_t* hl, int lane,
                                                Stage<FORM>& sg) {
  constexpr int T = kRows * kGroups;
  const auto issue = [&](int t) {
    const int b = t % kStages, g = t / kRows, r = t - g * kRows;
#pragma unroll
    for (int j = 0; j < D; ++j) cp_async8(&sg.z[b][j][lane], x.Zr + __shfl_sync(kFull, hl[g], r * D + j));
    if constexpr (FORM == 1) {
      const size_t so = (size_t)(m0 + t) * x.FP * 8;
      cp_async16(&sg.s[b][0][lane], x.S1 + so);
      cp_async16(&sg.s[b][1][lane], x.S2 + so);
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const size_t so = (size_t)(j * x.M + m0 + t) * x.FP * 2;
        cp_async4(&sg.l1[b][j][lane], x.S1 + so);
        cp_async4(&sg.l2[b][j][lane], x.S2 + so);
      }
    }
  };
  uint32_t fail = 0;
#pragma unroll
  for (int t = 0; t < kStages - 1; ++t) {
    if (t < T) issue(t);
    cp_async_commit();
  }
#pragma unroll kUnroll
  for (int t = 0; t < T; ++t) {
    // one group is committed per check (empty past the end), so waiting for
    // all but the newest kStages - 1 groups completes check t's copies
    if (t + kStages - 1 < T) issue(t + kStages - 1);
    cp_async_commit();
    cp_async_wait<kStages - 1>();
    const int b = t % kStages, g = t / kRows, r = t - g * kRows;
    uint32_t h[D], wa[D], wb[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      h[j] = __shfl_sync(kFull, hl[g], r * D + j);
      const uint2 v = sg.z[b][j][lane];
      wa[j] = v.x;
      wb[j] = v.y;
    }
    if constexpr (FORM == 1) {
      fail |= check2_sv<ES, NORM, D>(x, m0 + t, D, h, wa, wb, sg.s[b][0][lane], sg.s[b][1][lane]);
    } else {
      uint32_t l1[D], l2[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        l1[j] = sg.l1[b][j][lane];
        l2[j] = sg.l2[b][j][lane];
      }
      fail |= check2_pe<ES, NORM, D>(x, m0 + t, D, h, wa, wb, l1, l2);
    }
  }
  return fail;
}

// Row kernel of iteration k: block (bx, chunk) of nw warps takes nw kRows
// kGroups checks of the degree-sorted order for the chunk's 64 pairs (warp w:
// checks (bx nw + w) kRows kGroups ..., lane l: pairs chunk 64 + 2 l, + 1).
template <int FORM, bool ES, bool NORM>
// CTAs per SM (registers 65536 / (256 x LDPC_PP2_MINB1 or _MINB0)), measured on
// the N=64800 code: Section V with staged inputs 4 (7.83 ms, 52 bytes of spills,
// against 8.16 ms at 3 without spills; 5 spills 436 bytes); per edge 3.
// Blocks of 4, 8 or 16 warps (blockDim.x / 32 = nw); the bound keeps the
// registers of 256 threads x MINB1 CTAs for every block size.
__global__ void __launch_bounds__(kRowWarpsMax * 32) __maxnreg__(FORM == 1 ? kRegs1 : kRegs0)
pp2_rows(const DevCode c, const IntRule ir, PP2 s, int k) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = chunk_of(k) * 64 + 2 * lane;
  const int FP = s.FP;
  uint32_t aA = valid_bits(p, s.F), aB = valid_bits(p + 1, s.F);
  if (ES) {
    const int pb = (k - 1) % 3;
    const uint2 a = *reinterpret_cast<const uint2*>(s.act + pb * FP + p);
    const uint2 f = *reinterpret_cast<const uint2*>(s.fail + pb * FP + p);
    aA = a.x & f.x;
    aB = a.y & f.y;
    if (blockIdx.x == 0 && warp == 0) {
      // frames whose x^(k-2) satisfied H stop with k - 2 iterations
      const uint32_t st[2] = {a.x & ~f.x, a.y & ~f.y};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (st[q] & 1u) s.iters[2 * (p + q)] = k - 2;
        if (st[q] & 2u) s.iters[2 * (p + q) + 1] = k - 2;
        if (st[q]) s.okw[p + q] |= st[q];
      }
      *reinterpret_cast<uint2*>(s.act + (k % 3) * FP + p) = make_uint2(aA, aB);
      *reinterpret_cast<uint2*>(s.fail + ((k + 1) % 3) * FP + p) = make_uint2(0u, 0u);
    }
  }
  if (__all_sync(kFull, (aA | aB) == 0u)) return;
  RowArgs x;
  const size_t nfp = (size_t)c.N * FP, sfp = (size_t)s.rows * FP * s.ub;
  x.Zr = s.zb + (size_t)((k - 1) & 1) * nfp + p;
  x.Za = s.zb + (size_t)(k & 1) * nfp + p;
  x.S1 = s.st + (size_t)((k - 1) & 1) * sfp + (size_t)p * s.ub;
  x.S2 = s.st + (size_t)(k & 1) * sfp + (size_t)p * s.ub;
  x.FP = (uint32_t)FP;
  x.M = (uint32_t)c.M;
  x.amA = half_mask(aA);
  x.amB = half_mask(aB);
  // offset rule (beta <= 127): 1024 - beta; normalized: num / 2^shift; plain: neither
  const int beta = ir.rule == 1 ? ir.beta : 0;
  x.fin.cb = ints_to_h2(1024 - beta, 1024 - beta);
  x.fin.num = (uint32_t)ir.num;
  x.fin.shift = (uint32_t)ir.shift;
  // (16 Qm + 7) 2^-11: the key of a magnitude saturated to Qm at position 7
  // (every position of these checks is <= 7, so the minima decode above holds)
  x.ksat = hfma(ints_to_h2(ir.qm, ir.qm), h2c_q11(16), h2c_q11(7));
  x.two = s.two;
  const int nw = blockDim.x >> 5;
  const int m0 = (blockIdx.x * nw + warp) * kRows * kGroups;
  const int nr = min(kRows * kGroups, c.M - m0);
  if (nr <= 0) return;
  uint32_t fail = 0;
  const int d0 = c.deg(m0);
  if (nr == kRows * kGroups && d0 == c.deg(m0 + nr - 1) && (d0 == 6 || d0 == 7)) {
    // lane l < kRows d0 of group g holds the handle of (check m0 + g kRows +
    // l / d0, position l % d0)
    uint32_t hl[kGroups];
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
      hl[g] = 0;
      if (lane < kRows * d0) {
        const int r = lane / d0, j = lane - r * d0;
        hl[g] = (uint32_t)c.col(j, m0 + g * kRows + r) * x.FP;
      }
    }
#if LDPC_PP2_STAGED
    if constexpr (FORM == 1 || LDPC_PP2_STAGED_PE) {
      extern __shared__ __align__(16) unsigned char pp2_smem[];
      Stage<FORM>& sg = reinterpret_cast<Stage<FORM>*>(pp2_smem)[warp];
      fail = d0 == 6 ? rows_staged<FORM, ES, NORM, 6>(x, m0, hl, lane, sg)
                     : rows_staged<FORM, ES, NORM, 7>(x, m0, hl, lane, sg);
    } else
#endif
#pragma unroll
    for (int t = 0; t < kRows * kGroups; ++t) {
      const int g = t / kRows, r = t - g * kRows;
      uint32_t h[8];
      if (d0 == 6) {
#pragma unroll
        for (int j = 0; j < 6; ++j) h[j] = __shfl_sync(kFull, hl[g], r * 6 + j);
        fail |= check2<FORM, ES, NORM, 6>(x, m0 + t, 6, h);
      } else {
#pragma unroll
        for (int j = 0; j < 7; ++j) h[j] = __shfl_sync(kFull, hl[g], r * 7 + j);
        fail |= check2<FORM, ES, NORM, 7>(x, m0 + t, 7, h);
      }
    }
  } else {
    for (int r = 0; r < nr; ++r) {
      const int m = m0 + r, d = c.deg(m);
      uint32_t h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j < d) h[j] = (uint32_t)c.col(j, m) * x.FP;
      fail |= check2<FORM, ES, NORM, 0>(x, m, d, h);
    }
  }
  if (ES) {
    const uint32_t fa = fail & 3u & aA, fb = (fail >> 2) & aB;
    if (fa) atomicOr(s.fail + (k % 3) * FP + p, fa);
    if (fb) atomicOr(s.fail + (k % 3) * FP + p + 1, fb);
  }
}

// Channel values (frame-major int8) into both posterior buffers as binary16
// pairs; flags.  Tile: 64 variables x 32 pairs.
template <bool ES>
__global__ void __launch_bounds__(256) pp2_init(const DevCode c, const int8_t* __restrict__ llr, PP2 s, int K) {
  __shared__ int8_t tile[64][65];  // [frame][variable]
  const int n0 = blockIdx.x * 64, p0 = blockIdx.y * 32;
  const int N = c.N, F = s.F, FP = s.FP;
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    const int fl = i >> 6, nl = i & 63;
    const int f = 2 * p0 + fl, n = n0 + nl;
    tile[fl][nl] = (f < F && n < N) ? llr[(size_t)f * N + n] : (int8_t)0;
  }
  __syncthreads();
  const size_t nfp = (size_t)N * FP;
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
    const int nl = i >> 5, pl = i & 31;
    const int n = n0 + nl, p = p0 + pl;
    if (n >= N) continue;
    const uint32_t hz = ints_to_h2(tile[2 * pl][nl], tile[2 * pl + 1][nl]);
    const size_t o = (size_t)n * FP + p;
    s.zb[o] = hz;
    s.zb[nfp + o] = hz;
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    const int p = p0 + threadIdx.x;
    s.act[p] = valid_bits(p, F);
    s.fail[p] = ES ? kFull : 0u;  // "x^(-1) failed": every valid frame runs iteration 1
    s.fail[FP + p] = 0u;
    s.fail[2 * FP + p] = 0u;
    s.iters[2 * p] = K;
    s.iters[2 * p + 1] = K;
    s.okw[p] = 0u;
  }
}

// Syndrome of x^(K) for the frames still running; frames whose x^(K-1) satisfied
// H stop with K - 1 iterations.
template <bool ES>
__global__ void __launch_bounds__(kWarps * 32) pp2_final(const DevCode c, PP2 s, int K) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = chunk_of(K + 1) * 64 + 2 * lane;
  const int FP = s.FP;
  uint32_t aA = valid_bits(p, s.F), aB = valid_bits(p + 1, s.F);
  if (ES) {
    const int pb = K % 3;
    const uint2 a = *reinterpret_cast<const uint2*>(s.act + pb * FP + p);
    const uint2 f = *reinterpret_cast<const uint2*>(s.fail + pb * FP + p);
    aA = a.x & f.x;
    aB = a.y & f.y;
    if (blockIdx.x == 0 && warp == 0) {
      const uint32_t st[2] = {a.x & ~f.x, a.y & ~f.y};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (st[q] & 1u) s.iters[2 * (p + q)] = K - 1;
        if (st[q] & 2u) s.iters[2 * (p + q) + 1] = K - 1;
        if (st[q]) s.okw[p + q] |= st[q];
      }
    }
  }
  if (blockIdx.x == 0 && warp == 0) *reinterpret_cast<uint2*>(s.act + ((K + 1) % 3) * FP + p) = make_uint2(aA, aB);
  if (__all_sync(kFull, (aA | aB) == 0u)) return;
  const uint32_t* Zk = s.zb + (size_t)(K & 1) * c.N * FP + p;
  const int m0 = blockIdx.x * kTile + warp * kRows;
  const int nr = min(kRows, c.M - m0);
  uint32_t fa = 0, fb = 0;
  if (nr <= 0) return;
  const int d0 = c.deg(m0);
  if (nr == kRows && d0 == c.deg(m0 + nr - 1)) {
    // every gather of the warp's checks goes out before the first is used; lane
    // l < kRows d0 holds the handle of (check m0 + l / d0, position l % d0)
    uint32_t hl = 0;
    if (lane < kRows * d0) {
      const int r = lane / d0, j = lane - r * d0;
      hl = (uint32_t)c.col(j, m0 + r) * FP;
    }
    uint2 v[kRows][8];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j < d0) v[r][j] = *reinterpret_cast<const uint2*>(Zk + __shfl_sync(kFull, hl, r * d0 + j));
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      uint32_t ya = 0, yb = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (j < d0) {
          ya ^= dec_bits(v[r][j].x);
          yb ^= dec_bits(v[r][j].y);
        }
      }
      fa |= ((ya >> 15) & 1u) | ((ya >> 30) & 2u);
      fb |= ((yb >> 15) & 1u) | ((yb >> 30) & 2u);
    }
  } else {
    for (int m = m0; m < m0 + nr; ++m) {
      const int d = c.deg(m);
      uint32_t ya = 0, yb = 0;
      for (int j = 0; j < d; ++j) {
        const uint2 v = *reinterpret_cast<const uint2*>(Zk + (size_t)c.col(j, m) * FP);
        ya ^= dec_bits(v.x);
        yb ^= dec_bits(v.y);
      }
      fa |= ((ya >> 15) & 1u) | ((ya >> 30) & 2u);
      fb |= ((yb >> 15) & 1u) | ((yb >> 30) & 2u);
    }
  }
  fa &= aA;
  fb &= aB;
  if (fa) atomicOr(s.fail + ((K + 1) % 3) * FP + p, fa);
  if (fb) atomicOr(s.fail + ((K + 1) % 3) * FP + p + 1, fb);
}

// Frame-major outputs through a 64-variable x 32-pair tile; each frame's result
// is the buffer of its iteration count.
__global__ void __launch_bounds__(256) pp2_output(const DevCode c, PP2 s, int K, uint8_t* bits, int32_t* iters,
                                                  uint8_t* okf, int16_t* zout) {
  __shared__ uint32_t tile[64][33];  // [variable][pair]
  const int n0 = blockIdx.x * 64, p0 = blockIdx.y * 32;
  const int N = c.N, N8 = (N + 7) >> 3, FP = s.FP, F = s.F;
  const size_t nfp = (size_t)N * FP;
  const int pl = threadIdx.x & 31, p = p0 + pl;
  const uint32_t* zl = s.zb + (size_t)(s.iters[2 * p] & 1) * nfp + p;
  const uint32_t* zh = s.zb + (size_t)(s.iters[2 * p + 1] & 1) * nfp + p;
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
    const int nl = i >> 5;
    const int n = n0 + nl;
    uint32_t v = 0;
    if (n < N) {
      const uint32_t a = zl[(size_t)n * FP];
      v = (zl == zh) ? a : ((a & 0xffffu) | (zh[(size_t)n * FP] & 0xffff0000u));
    }
    tile[nl][pl] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 64 * 8; i += blockDim.x) {
    const int fl = i >> 3, bl = i & 7;
    const int f = 2 * p0 + fl, b = (n0 >> 3) + bl;
    if (f >= F || b >= N8) continue;
    uint32_t byte = 0;
    for (int t = 0; t < 8; ++t) {
      const int nl = bl * 8 + t;
      if (n0 + nl < N) byte |= ((dec_bits(tile[nl][fl >> 1] >> (16 * (fl & 1))) >> 15) & 1u) << t;
    }
    bits[(size_t)f * N8 + b] = (uint8_t)byte;
  }
  if (zout != nullptr) {
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
      const int fl = i >> 6, nl = i & 63;
      const int f = 2 * p0 + fl, n = n0 + nl;
      if (f >= F || n >= N) continue;
      const uint32_t hz = tile[nl][fl >> 1];
      zout[(size_t)f * N + n] = (int16_t)((fl & 1) ? h_hi_int(hz) : h_lo_int(hz));
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 64) {
    const int f = 2 * p0 + threadIdx.x;
    if (f < F) {
      const int pp = f >> 1, b = f & 1, kb = (K + 1) % 3;
      const uint32_t a = s.act[kb * FP + pp], fl = s.fail[kb * FP + pp];
      iters[f] = s.iters[f];
      okf[f] = ((a >> b) & 1u) ? (uint8_t)(((fl >> b) & 1u) ^ 1u) : (uint8_t)((s.okw[pp] >> b) & 1u);
    }
  }
}

template <int FORM, bool ES>
cudaError_t pp2_run(const DevCode& c, const IntRule& r, const PP2& s, int warps, const int8_t* llr, int K, uint8_t* bits,
                    int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st) {
  const dim3 tgrid((unsigned)((c.N + 63) / 64), (unsigned)(s.FP / 32));
  const dim3 rgrid((unsigned)((c.M + kTile - 1) / kTile), (unsigned)(s.FP / 64));
  const int row_tile = warps * kRows * kGroups;
  const dim3 rgrid_rows((unsigned)((c.M + row_tile - 1) / row_tile), (unsigned)(s.FP / 64));
  pp2_init<ES><<<tgrid, 256, 0, st>>>(c, llr, s, K);
  const size_t smem = LDPC_PP2_STAGED && (FORM == 1 || LDPC_PP2_STAGED_PE) ? sizeof(Stage<FORM>) * warps : 0;
  // the normalized rule scales integer halves, the offset and plain rules take max(., 1024)
  const auto rows = r.rule == 2 ? pp2_rows<FORM, ES, true> : pp2_rows<FORM, ES, false>;
  for (int k = 1; k <= K; ++k) rows<<<rgrid_rows, warps * 32, smem, st>>>(c, r, s, k);
  pp2_final<ES><<<rgrid, kWarps * 32, 0, st>>>(c, s, K);
  pp2_output<<<tgrid, 256, 0, st>>>(c, s, K, bits, iters, ok, zout);
  return cudaGetLastError();
}

}  // namespace

cudaError_t pingpong_prepare() {
  // the staged row kernels take up to kRowWarpsMax Stage<FORM> of dynamic shared memory;
  // set on the current device outside any stream capture (code creation)
  for (auto f : {pp2_rows<1, false, false>, pp2_rows<1, true, false>, pp2_rows<1, false, true>, pp2_rows<1, true, true>}) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(Stage<1>) * kRowWarpsMax));
    if (e != cudaSuccess) return e;
  }
  for (auto f : {pp2_rows<0, false, false>, pp2_rows<0, true, false>, pp2_rows<0, false, true>, pp2_rows<0, true, true>}) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(Stage<0>) * kRowWarpsMax));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

PingpongLayout pingpong_layout(int form, int N, int M, int ell_w, int F) {
  PingpongLayout L;
  L.lanes = (((F + 1) / 2) + 63) / 64 * 64;
  L.ub = form == 1 ? 8 : 2;
  L.rows = form == 1 ? M : ell_w * M;
  const size_t lanes = (size_t)L.lanes;
  size_t off = 0;
  L.zb = off;    off = al256(off + 2 * (size_t)N * lanes * 4);
  L.st = off;    off = al256(off + 2 * (size_t)L.rows * lanes * L.ub);
  L.act = off;   off = al256(off + 3 * lanes * 4);
  L.fail = off;  off = al256(off + 3 * lanes * 4);
  L.iters = off; off = al256(off + 2 * lanes * 4);
  L.ok = off;    off = al256(off + lanes * 4);
  L.total = off;
  return L;
}

bool pingpong_int8_eligible(int N, int M, int ell_w, int max_row_deg, int max_col_deg, int qm, int form, int F) {
  if (max_row_deg > 8 || 128 + (int64_t)(max_col_deg + 1) * qm > 2048) return false;
  const PingpongLayout L = pingpong_layout(form, N, M, ell_w, F);
  // element offsets within one buffer fit 32 bits
  return (uint64_t)N * L.lanes < (1ull << 32) && (uint64_t)L.rows * L.lanes < (1ull << 32);
}

cudaError_t pingpong_int8_decode(const DevCode& c, const IntRule& r, int form, const PingpongLayout& L, void* ws,
                                 const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop, uint8_t* bits,
                                 int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st, int warps) {
  if (warps != 4 && warps != 8 && warps != 16) return cudaErrorInvalidValue;
  char* b = static_cast<char*>(ws);
  PP2 s;
  s.zb = reinterpret_cast<uint32_t*>(b + L.zb);
  s.st = b + L.st;
  s.act = reinterpret_cast<uint32_t*>(b + L.act);
  s.fail = reinterpret_cast<uint32_t*>(b + L.fail);
  s.iters = reinterpret_cast<int32_t*>(b + L.iters);
  s.okw = reinterpret_cast<uint32_t*>(b + L.ok);
  s.F = F;
  s.FP = L.lanes;
  s.rows = L.rows;
  s.ub = L.ub;
  s.two = 2u;
  // L^(0) = L^(-1) = 0: Section V state all zero, per-edge bytes L + 128 = 0x80
  cudaError_t e = cudaMemsetAsync(b + L.st, form == 1 ? 0 : 0x80, L.act - L.st, st);
  if (e != cudaSuccess) return e;
  if (form == 1) return early_stop ? pp2_run<1, true>(c, r, s, warps, llr, max_iter, bits, iters, ok, zout, st)
                                   : pp2_run<1, false>(c, r, s, warps, llr, max_iter, bits, iters, ok, zout, st);
  return early_stop ? pp2_run<0, true>(c, r, s, warps, llr, max_iter, bits, iters, ok, zout, st)
                    : pp2_run<0, false>(c, r, s, warps, llr, max_iter, bits, iters, ok, zout, st);
}

}  // namespace ldpc
