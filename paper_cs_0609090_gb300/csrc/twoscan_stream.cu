// twoscan_stream.cu -- the two-scan min-sum of Section III (Eq. (1) horizontal
// scan, Eq. (2) vertical scan) with the frame state in device memory, for any
// code size: the comparator of the single scan.  Two storages of the check
// messages:
//   literal (LDPC_FORM_TWO_SCAN): one message L_mn per edge;
//   compressed (LDPC_FORM_TWO_SCAN_1BIT): the check's Section V state (A, B, n~
//     and one sign per edge), from which the vertical scan rebuilds L_mn --
//     Section V notes that this storage applies to the original algorithm too.
// Both compute exactly the integers of the literal two-scan definition.
//
// Workspace (lane unit = frame pair, FP pairs, a multiple of 64; a warp lane
// takes two neighbouring pairs):
//   zmn [ell_w M][FP] u16   Z_mn of every edge slot (j M + m of the degree-sorted
//                           table) as two biased bytes, saturated to [-128, 127]
//                           (the check saturates |Z_mn| to Qm <= 127 anyway)
//   lmn [ell_w M][FP] u16   literal: L_mn + 128 per frame
//   st [M][FP]              compressed: 8 bytes per pair (degree <= 8) or 16
//   q0 [N][FP] u16          channel values
//   zp [N][FP] half2        posterior Z_n (written by the last vertical scan, and
//                           by every one when frames stop early)
//   act/fail [3][FP], iters [2 FP], okw [FP]
// Per iteration k: horizontal kernel (checks: Z_mn in, L_mn or state out; with
// early stop also the parity of x^(k-1) from zp), then vertical kernel
// (variables: Z_n = q0 + sum_m L_mn, Z_mn = Z_n - L_mn).  The decode starts with
// a vertical scan over L = 0 (Z_mn = q0) and ends with the syndrome of x^(K).
#include <algorithm>
#include <type_traits>

#include "async_copy.cuh"
#include "h2_body.cuh"
#include "kernels.h"
#include "pp_check.cuh"

namespace ldpc {
namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kWarps = 8;
constexpr int kRows = 4;   // checks per warp (horizontal)
constexpr int kCols = 4;   // variables per warp (vertical)
constexpr int kDvMax = 16; // column degrees the vertical kernel keeps in registers

// The literal form's vertical scan stages the next variable's inputs (below).
#ifndef LDPC_TS_VSTAGED
#define LDPC_TS_VSTAGED 1
#endif
constexpr bool kVStaged = LDPC_TS_VSTAGED != 0;
// ... and the horizontal scan the next check's Z_mn words (without early stop)
#ifndef LDPC_TS_HSTAGED
#define LDPC_TS_HSTAGED 1
#endif
constexpr bool kHStaged = LDPC_TS_HSTAGED != 0;

// Per-warp staging of the vertical scan, two buffers: the channel word of one
// variable per lane and, per edge, the message word (literal form) or the
// 16-byte state word of the edge's check (Section V messages, 8-byte state).
template <int FORM2, int DVM>
struct VStage {
  uint32_t q[2][32];
  typename std::conditional<FORM2 == 0, uint32_t, uint4>::type l[2][DVM][32];
};
// the vertical kernels that stage (the others take no dynamic shared memory)
template <int FORM2, bool C8, int DVM>
__host__ __device__ constexpr bool vstaged() { return kVStaged && (FORM2 == 0 || (C8 && DVM == 8)); }

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct TS {
  uint16_t* zmn;   // [slots][FP]
  uint16_t* lmn;   // [slots][FP] (literal)
  char* st;        // [M][FP] units of ub bytes (compressed)
  uint16_t* q0;    // [N][FP]
  uint32_t* zp;    // [N][FP]
  uint32_t* act;   // [3][FP]
  uint32_t* fail;  // [3][FP]
  int32_t* iters;  // [2 FP]
  uint32_t* okw;   // [FP]
  int32_t F, FP, ub;
};

__device__ __forceinline__ uint32_t half_mask(uint32_t b) {
  return ((b & 1u) ? 0x0000ffffu : 0u) | ((b & 2u) ? 0xffff0000u : 0u);
}
__device__ __forceinline__ uint32_t valid_bits(int p, int F) {
  return (2 * p < F ? 1u : 0u) | (2 * p + 1 < F ? 2u : 0u);
}
// Two biased bytes (one pair) to a binary16 pair, and back (saturating to
// [-128, 127] first).
__device__ __forceinline__ uint32_t by_to_h2(uint32_t b) { return pe_to_h2(b & 0xffffu); }
__device__ __forceinline__ uint32_t h2_to_by_sat(uint32_t z) {
  return h2_to_pe(hmax(hmin(z, h2c(127) ), 0xD800D800u /* -128 */));
}

// Frames running at iteration k (k >= 1) of pair p.
template <bool ES>
__device__ __forceinline__ uint32_t running(const TS& s, int k, int p) {
  if (!ES) return valid_bits(p, s.F);
  return s.act[(k % 3) * s.FP + p];
}

// ------------------------------------------------------------ horizontal scan

// One check m of degree d (D > 0: exactly D), both pairs of the lane: Eq. (1)
// on the stored Z_mn, then the rule; writes L_mn (literal) or the state
// (compressed).  With early stop also returns the parities of x^(k-1) (bits 0-1
// first pair, 2-3 second) from the posteriors at the handles h[j].
template <int FORM2, bool C8, bool ES, int D, int DMAX>
__device__ __forceinline__ uint32_t ts_check(const TS& s, int m, int d, int M, int p, const uint32_t* h,
                                             const H2Rule& rule, uint32_t ksat, const uint32_t* zin = nullptr) {
  constexpr int NJ = D > 0 ? D : DMAX;
  const int FP = s.FP;
  uint32_t K1a = ksat, K2a = ksat, NEGa = 0, K1b = ksat, K2b = ksat, NEGb = 0, Ya = 0, Yb = 0;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      // the check's Z_mn words: staged by the caller (zin), else read here
      const uint32_t z = zin ? zin[j] : __ldcg(reinterpret_cast<const uint32_t*>(s.zmn + (size_t)(j * M + m) * FP + p));
      key_step(by_to_h2(z), j, K1a, K2a, NEGa);
      key_step(by_to_h2(z >> 16), j, K1b, K2b, NEGb);
      if (ES) {
        const uint2 zz = __ldcg(reinterpret_cast<const uint2*>(s.zp + h[j]));
        Ya ^= dec_bits(zz.x);
        Yb ^= dec_bits(zz.y);
      }
    }
  }
  const int dd = D > 0 ? D : d;
  const NewState na = finish_state(K1a, K2a, NEGa, dd, rule), nb = finish_state(K1b, K2b, NEGb, dd, rule);
  if constexpr (FORM2 == 0) {
    const uint32_t Dna = hsub(na.Bn, na.An), Dnb = hsub(nb.Bn, nb.An);
    uint32_t SNa = na.Sn, SNb = nb.Sn;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      if (D > 0 || j < d) {
        const uint32_t La = hfma(Dna, heq_one(na.In, h2c(j)), na.An) ^ (SNa & 0x80008000u);
        const uint32_t Lb = hfma(Dnb, heq_one(nb.In, h2c(j)), nb.An) ^ (SNb & 0x80008000u);
        SNa += SNa;
        SNb += SNb;
        __stcg(reinterpret_cast<uint32_t*>(s.lmn + (size_t)(j * M + m) * FP + p), h2_to_pe(La) | (h2_to_pe(Lb) << 16));
      }
    }
  } else if constexpr (C8) {
    auto pk = [](const NewState& n) {
      return make_uint2((uint32_t)n.al | ((uint32_t)n.ah << 8) | ((uint32_t)n.bl << 16) | ((uint32_t)n.bh << 24),
                        (uint32_t)n.il | ((uint32_t)n.ih << 16) | (n.Sn & 0xff00ff00u));
    };
    const uint2 ua = pk(na), ub = pk(nb);
    __stcg(reinterpret_cast<uint4*>(s.st + ((size_t)m * FP + p) * 8), make_uint4(ua.x, ua.y, ub.x, ub.y));
  } else {
    uint4* S = reinterpret_cast<uint4*>(s.st + ((size_t)m * FP + p) * 16);
    __stcg(S, make_uint4(na.An, na.Bn, na.In, na.Sn));
    __stcg(S + 1, make_uint4(nb.An, nb.Bn, nb.In, nb.Sn));
  }
  return ES ? (((Ya >> 15) & 1u) | ((Ya >> 30) & 2u) | (((Yb >> 15) & 1u) << 2) | (((Yb >> 30) & 2u) << 2)) : 0u;
}

template <int FORM2, bool C8, bool ES>
__global__ void __launch_bounds__(kWarps * 32) ts_horizontal(const DevCode c, const IntRule ir, TS s, int k) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.y * 64 + 2 * lane;
  const uint32_t aA = running<ES>(s, k, p), aB = running<ES>(s, k, p + 1);
  if (__all_sync(kFull, (aA | aB) == 0u)) return;
  const H2Rule rule = make_h2rule(ir);
  const uint32_t ksat = hfma(ints_to_h2(ir.qm, ir.qm), h2c_q11(16), h2c_q11(15));
  const int m0 = (blockIdx.x * kWarps + warp) * kRows;
  const int m1 = min(m0 + kRows, c.M);
  const int DM = (FORM2 == 1 && C8) ? 8 : 16;
  uint32_t fail = 0;
  if (kHStaged && !ES && m1 - m0 == kRows && c.deg(m0) == c.deg(m1 - 1) && (c.deg(m0) == 6 || c.deg(m0) == 7)) {
    // checks of one degree (6 or 7) without early stop: the Z_mn words of check
    // r + 1 are copied into shared memory while check r computes
    __shared__ uint32_t hz[kWarps][2][7][32];
    const int d = c.deg(m0);
    const auto issue = [&](int r) {
      for (int j = 0; j < d; ++j)
        cp_async4(&hz[warp][r & 1][j][lane], s.zmn + (size_t)(j * c.M + m0 + r) * s.FP + p);
    };
    issue(0);
    cp_async_commit();
#pragma unroll 1
    for (int r = 0; r < kRows; ++r) {
      if (r + 1 < kRows) issue(r + 1);
      cp_async_commit();
      cp_async_wait<1>();
      uint32_t z[7];
#pragma unroll
      for (int j = 0; j < 7; ++j) z[j] = hz[warp][r & 1][j][lane];
      uint32_t h[16];
      if (d == 6) ts_check<FORM2, C8, ES, 6, 6>(s, m0 + r, d, c.M, p, h, rule, ksat, z);
      else ts_check<FORM2, C8, ES, 7, 7>(s, m0 + r, d, c.M, p, h, rule, ksat, z);
    }
    return;
  }
  for (int m = m0; m < m1; ++m) {
    const int d = c.deg(m);
    uint32_t h[16];
    if (ES) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < d) h[j] = (uint32_t)c.col(j, m) * s.FP + p;
    }
    if (d == 6) fail |= ts_check<FORM2, C8, ES, 6, 6>(s, m, d, c.M, p, h, rule, ksat);
    else if (d == 7) fail |= ts_check<FORM2, C8, ES, 7, 7>(s, m, d, c.M, p, h, rule, ksat);
    else if (DM == 8) fail |= ts_check<FORM2, C8, ES, 0, 8>(s, m, d, c.M, p, h, rule, ksat);
    else fail |= ts_check<FORM2, C8, ES, 0, 16>(s, m, d, c.M, p, h, rule, ksat);
  }
  if (ES) {
    const uint32_t fa = fail & 3u & aA, fb = (fail >> 2) & aB;
    if (fa) atomicOr(s.fail + (k % 3) * s.FP + p, fa);
    if (fb) atomicOr(s.fail + (k % 3) * s.FP + p + 1, fb);
  }
}

// ------------------------------------------------------------ vertical scan

// Eq. (2) for kCols variables per warp: Z_n = q0_n + sum over M(n) of L_mn, then
// Z_mn = Z_n - L_mn for every edge.  k = 0 is the start (L = 0).  Writes the
// posterior when `post` (the last iteration, or every one with early stop) for
// the frames that continue; with early stop the first block of a chunk stops
// the frames whose x^(k-1) satisfied H.
template <int FORM2, bool C8, bool ES, int DVM>
__global__ void __launch_bounds__(kWarps * 32) ts_vertical(const DevCode c, TS s, int k, int post) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.y * 64 + 2 * lane;
  const int FP = s.FP;
  uint32_t aA = valid_bits(p, s.F), aB = valid_bits(p + 1, s.F);
  if (ES && k >= 1) {
    const int kb = k % 3;
    const uint2 a = *reinterpret_cast<const uint2*>(s.act + kb * FP + p);
    const uint2 f = *reinterpret_cast<const uint2*>(s.fail + kb * FP + p);
    aA = a.x & f.x;
    aB = a.y & f.y;
    if (blockIdx.x == 0 && warp == 0) {
      const uint32_t st[2] = {a.x & ~f.x, a.y & ~f.y};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (st[q] & 1u) s.iters[2 * (p + q)] = k - 1;
        if (st[q] & 2u) s.iters[2 * (p + q) + 1] = k - 1;
        if (st[q]) s.okw[p + q] |= st[q];
      }
      *reinterpret_cast<uint2*>(s.act + ((k + 1) % 3) * FP + p) = make_uint2(aA, aB);
      *reinterpret_cast<uint2*>(s.fail + ((k + 1) % 3) * FP + p) = make_uint2(0u, 0u);
    }
  } else if (ES && blockIdx.x == 0 && warp == 0) {
    *reinterpret_cast<uint2*>(s.act + 1 * FP + p) = make_uint2(aA, aB);
    *reinterpret_cast<uint2*>(s.fail + 1 * FP + p) = make_uint2(0u, 0u);
  }
  if (__all_sync(kFull, (aA | aB) == 0u)) return;
  const uint32_t selA = half_mask(aA), selB = half_mask(aB);
  const int n0 = (blockIdx.x * kWarps + warp) * kCols;
  const int n1 = min(n0 + kCols, c.N);
  if (n0 >= n1) return;
  // the edge slots (and, compressed, the check / position words) of the warp's
  // variables, one per lane, loaded together: at most kCols DVM <= 64 edges, so
  // two words per lane; each variable then reads them with shuffles instead of
  // a dependent load ahead of its message gathers
  constexpr int kEdgeWords = (kCols * DVM + 31) / 32;
  const int ew0 = __ldg(c.cptr + n0), ewn = __ldg(c.cptr + n1) - ew0;
  uint32_t slw[kEdgeWords], cjw[kEdgeWords];
#pragma unroll
  for (int q = 0; q < kEdgeWords; ++q) {
    const int e = q * 32 + lane;
    slw[q] = e < ewn ? (uint32_t)__ldg(c.cslot + ew0 + e) : 0u;
    cjw[q] = 0u;
    if constexpr (FORM2 == 1) cjw[q] = e < ewn ? __ldg(c.ccj + ew0 + e) : 0u;
  }
  const auto pick = [&](const uint32_t* w, int e) {
    uint32_t v = __shfl_sync(kFull, w[0], e & 31);
#pragma unroll
    for (int q = 1; q < kEdgeWords; ++q) {
      const uint32_t u = __shfl_sync(kFull, w[q], e & 31);
      if ((e >> 5) == q) v = u;
    }
    return v;
  };
  if constexpr (vstaged<FORM2, C8, DVM>()) {
    // the channel word and the message (or check state) words of variable t + 1
    // are copied into shared memory while variable t computes
    extern __shared__ __align__(16) unsigned char ts_smem[];
    VStage<FORM2, DVM>& vs = reinterpret_cast<VStage<FORM2, DVM>*>(ts_smem)[warp];
    const int nv = n1 - n0;
    const auto issue = [&](int t) {
      const int n = n0 + t, b = t & 1;
      const int e0 = __ldg(c.cptr + n), dv = __ldg(c.cptr + n + 1) - e0;
      cp_async4(&vs.q[b][lane], s.q0 + (size_t)n * FP + p);
#pragma unroll
      for (int a = 0; a < DVM; ++a) {
        if (a < dv && k > 0) {  // warp-uniform: every lane takes part in the shuffles
          if constexpr (FORM2 == 0) {
            const uint32_t sl = pick(slw, e0 - ew0 + a);
            cp_async4(&vs.l[b][a][lane], s.lmn + (size_t)sl * FP + p);
          } else {
            const uint32_t m = pick(cjw, e0 - ew0 + a) & 0xffffffu;
            cp_async16(&vs.l[b][a][lane], s.st + ((size_t)m * FP + p) * 8);
          }
        }
      }
    };
    issue(0);
    cp_async_commit();
    for (int t = 0; t < nv; ++t) {
      if (t + 1 < nv) issue(t + 1);
      cp_async_commit();
      cp_async_wait<1>();
      const int n = n0 + t, b = t & 1;
      const int e0 = __ldg(c.cptr + n), dv = __ldg(c.cptr + n + 1) - e0;
      const uint32_t q = vs.q[b][lane];
      uint32_t za = by_to_h2(q), zb = by_to_h2(q >> 16);
      uint32_t La[DVM], Lb[DVM];
#pragma unroll
      for (int a = 0; a < DVM; ++a) {
        if (a < dv) {
          if (k == 0) {
            La[a] = 0u;
            Lb[a] = 0u;
          } else if constexpr (FORM2 == 0) {
            const uint32_t l = vs.l[b][a][lane];
            La[a] = by_to_h2(l);
            Lb[a] = by_to_h2(l >> 16);
          } else {
            const uint32_t j = pick(cjw, e0 - ew0 + a) >> 24;
            const uint4 u = vs.l[b][a][lane];
            const SV oa = SVUnit<true>::unpack(make_uint2(u.x, u.y)), ob = SVUnit<true>::unpack(make_uint2(u.z, u.w));
            const uint32_t jh = small_to_h2((int32_t)j, (int32_t)j);
            La[a] = hfma(hsub(oa.B, oa.A), heq_one(oa.I, jh), oa.A) ^ ((oa.S << j) & 0x80008000u);
            Lb[a] = hfma(hsub(ob.B, ob.A), heq_one(ob.I, jh), ob.A) ^ ((ob.S << j) & 0x80008000u);
          }
          za = hadd(za, La[a]);
          zb = hadd(zb, Lb[a]);
        }
      }
      if (post) {
        uint2* Z = reinterpret_cast<uint2*>(s.zp + (size_t)n * FP + p);
        uint2 v = make_uint2(za, zb);
        if ((selA & selB) != kFull) {
          const uint2 o = __ldcg(Z);
          v = make_uint2((za & selA) | (o.x & ~selA), (zb & selB) | (o.y & ~selB));
        }
        __stcg(Z, v);
      }
#pragma unroll
      for (int a = 0; a < DVM; ++a) {
        if (a < dv) {
          const uint32_t sl = pick(slw, e0 - ew0 + a);
          const uint32_t ba = h2_to_by_sat(hsub(za, La[a])), bb = h2_to_by_sat(hsub(zb, Lb[a]));
          __stcg(reinterpret_cast<uint32_t*>(s.zmn + (size_t)sl * FP + p), ba | (bb << 16));
        }
      }
    }
    return;
  }
  for (int n = n0; n < n1; ++n) {
    const int e0 = __ldg(c.cptr + n), dv = __ldg(c.cptr + n + 1) - e0;
    const uint32_t q = __ldcg(reinterpret_cast<const uint32_t*>(s.q0 + (size_t)n * FP + p));
    uint32_t za = by_to_h2(q), zb = by_to_h2(q >> 16);
    uint32_t La[DVM], Lb[DVM];
    uint32_t sl[DVM];
#pragma unroll
    for (int a = 0; a < DVM; ++a) {
      // warp-uniform bound: every lane takes part in the shuffles
      if (a < dv) {
        sl[a] = pick(slw, e0 - ew0 + a);
        if (k == 0) {
          La[a] = 0u;
          Lb[a] = 0u;
        } else if constexpr (FORM2 == 0) {
          const uint32_t l = __ldcg(reinterpret_cast<const uint32_t*>(s.lmn + (size_t)sl[a] * FP + p));
          La[a] = by_to_h2(l);
          Lb[a] = by_to_h2(l >> 16);
        } else {
          const uint32_t cj = pick(cjw, e0 - ew0 + a);  // internal check | position << 24
          const uint32_t m = cj & 0xffffffu, j = cj >> 24;
          SV oa, ob;
          if constexpr (C8) {
            const uint4 u = __ldcg(reinterpret_cast<const uint4*>(s.st + ((size_t)m * FP + p) * 8));
            oa = SVUnit<true>::unpack(make_uint2(u.x, u.y));
            ob = SVUnit<true>::unpack(make_uint2(u.z, u.w));
          } else {
            const uint4* S = reinterpret_cast<const uint4*>(s.st + ((size_t)m * FP + p) * 16);
            const uint4 u0 = __ldcg(S), u1 = __ldcg(S + 1);
            oa = SV{u0.x, u0.y, u0.z, u0.w};
            ob = SV{u1.x, u1.y, u1.z, u1.w};
          }
          // f(A, B, n, n~) with the sign of position j (bits 15 - j / 31 - j of the sign word)
          const uint32_t jh = small_to_h2((int32_t)j, (int32_t)j);
          La[a] = hfma(hsub(oa.B, oa.A), heq_one(oa.I, jh), oa.A) ^ ((oa.S << j) & 0x80008000u);
          Lb[a] = hfma(hsub(ob.B, ob.A), heq_one(ob.I, jh), ob.A) ^ ((ob.S << j) & 0x80008000u);
        }
        za = hadd(za, La[a]);
        zb = hadd(zb, Lb[a]);
      }
    }
    if (post) {
      uint2* Z = reinterpret_cast<uint2*>(s.zp + (size_t)n * FP + p);
      uint2 v = make_uint2(za, zb);
      if ((selA & selB) != kFull) {
        const uint2 o = __ldcg(Z);
        v = make_uint2((za & selA) | (o.x & ~selA), (zb & selB) | (o.y & ~selB));
      }
      __stcg(Z, v);
    }
#pragma unroll
    for (int a = 0; a < DVM; ++a) {
      if (a < dv) {
        const uint32_t ba = h2_to_by_sat(hsub(za, La[a])), bb = h2_to_by_sat(hsub(zb, Lb[a]));
        __stcg(reinterpret_cast<uint32_t*>(s.zmn + (size_t)sl[a] * FP + p), ba | (bb << 16));
      }
    }
  }
}

// ------------------------------------------------------------ in and out

// Channel values into q0 (two int8 per pair) and flags; tile 64 variables x 32 pairs.
template <bool ES>
__global__ void __launch_bounds__(256) ts_init(const DevCode c, const int8_t* __restrict__ llr, TS s, int K) {
  __shared__ int8_t tile[64][65];  // [frame][variable]
  const int n0 = blockIdx.x * 64, p0 = blockIdx.y * 32;
  const int N = c.N, F = s.F, FP = s.FP;
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    const int fl = i >> 6, nl = i & 63;
    const int f = 2 * p0 + fl, n = n0 + nl;
    tile[fl][nl] = (f < F && n < N) ? llr[(size_t)f * N + n] : (int8_t)0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
    const int nl = i >> 5, pl = i & 31;
    const int n = n0 + nl, p = p0 + pl;
    if (n >= N) continue;
    // biased bytes v + 128
    s.q0[(size_t)n * FP + p] =
        (uint16_t)(((uint32_t)(tile[2 * pl][nl] + 128) & 0xffu) | (((uint32_t)(tile[2 * pl + 1][nl] + 128) & 0xffu) << 8));
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    const int p = p0 + threadIdx.x;
    s.iters[2 * p] = K;
    s.iters[2 * p + 1] = K;
    s.okw[p] = 0u;
    s.act[p] = valid_bits(p, F);
    s.fail[p] = 0u;
    s.act[FP + p] = valid_bits(p, F);
    s.fail[FP + p] = 0u;
    s.fail[2 * FP + p] = 0u;
  }
}

// Syndrome of x^(K) for the frames still running.
template <bool ES>
__global__ void __launch_bounds__(kWarps * 32) ts_final(const DevCode c, TS s, int K) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.y * 64 + 2 * lane;
  const int FP = s.FP;
  const int kb = (K + 1) % 3;
  uint32_t aA = valid_bits(p, s.F), aB = valid_bits(p + 1, s.F);
  if (ES) {
    aA = s.act[kb * FP + p];
    aB = s.act[kb * FP + p + 1];
  } else if (blockIdx.x == 0 && warp == 0) {
    *reinterpret_cast<uint2*>(s.act + kb * FP + p) = make_uint2(aA, aB);
  }
  if (__all_sync(kFull, (aA | aB) == 0u)) return;
  const int m0 = (blockIdx.x * kWarps + warp) * kRows;
  const int m1 = min(m0 + kRows, c.M);
  uint32_t fa = 0, fb = 0;
  for (int m = m0; m < m1; ++m) {
    const int d = c.deg(m);
    uint32_t ya = 0, yb = 0;
    for (int j = 0; j < d; ++j) {
      const uint2 v = *reinterpret_cast<const uint2*>(s.zp + (size_t)c.col(j, m) * FP + p);
      ya ^= dec_bits(v.x);
      yb ^= dec_bits(v.y);
    }
    fa |= ((ya >> 15) & 1u) | ((ya >> 30) & 2u);
    fb |= ((yb >> 15) & 1u) | ((yb >> 30) & 2u);
  }
  fa &= aA;
  fb &= aB;
  if (fa) atomicOr(s.fail + kb * FP + p, fa);
  if (fb) atomicOr(s.fail + kb * FP + p + 1, fb);
}

__global__ void __launch_bounds__(256) ts_output(const DevCode c, TS s, int K, uint8_t* bits, int32_t* iters,
                                                 uint8_t* okf, int16_t* zout) {
  __shared__ uint32_t tile[64][33];  // [variable][pair]
  const int n0 = blockIdx.x * 64, p0 = blockIdx.y * 32;
  const int N = c.N, N8 = (N + 7) >> 3, FP = s.FP, F = s.F;
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
    const int nl = i >> 5, pl = i & 31;
    const int n = n0 + nl;
    tile[nl][pl] = n < N ? s.zp[(size_t)n * FP + p0 + pl] : 0u;
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

template <int FORM2, bool C8, bool ES, int DVM>
cudaError_t ts_run(const DevCode& c, const IntRule& r, const TS& s, const int8_t* llr, int K, uint8_t* bits,
                   int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st) {
  const dim3 tgrid((unsigned)((c.N + 63) / 64), (unsigned)(s.FP / 32));
  const dim3 hgrid((unsigned)((c.M + kWarps * kRows - 1) / (kWarps * kRows)), (unsigned)(s.FP / 64));
  const dim3 vgrid((unsigned)((c.N + kWarps * kCols - 1) / (kWarps * kCols)), (unsigned)(s.FP / 64));
  ts_init<ES><<<tgrid, 256, 0, st>>>(c, llr, s, K);
  const size_t vsm = vstaged<FORM2, C8, DVM>() ? sizeof(VStage<FORM2, DVM>) * kWarps : 0;
  ts_vertical<FORM2, C8, ES, DVM><<<vgrid, kWarps * 32, vsm, st>>>(c, s, 0, (ES || K == 0) ? 1 : 0);
  for (int k = 1; k <= K; ++k) {
    ts_horizontal<FORM2, C8, ES><<<hgrid, kWarps * 32, 0, st>>>(c, r, s, k);
    ts_vertical<FORM2, C8, ES, DVM><<<vgrid, kWarps * 32, vsm, st>>>(c, s, k, (ES || k == K) ? 1 : 0);
  }
  ts_final<ES><<<hgrid, kWarps * 32, 0, st>>>(c, s, K);
  ts_output<<<tgrid, 256, 0, st>>>(c, s, K, bits, iters, ok, zout);
  return cudaGetLastError();
}

}  // namespace

cudaError_t twoscan_prepare() {
  // the staged vertical kernels of the Section V-message form take more than
  // the default 48 KB of dynamic shared memory; set on the current device
  // outside any stream capture (code creation)
  for (auto f : {ts_vertical<1, true, false, 8>, ts_vertical<1, true, true, 8>}) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(VStage<1, 8>) * kWarps));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

TwoScanLayout twoscan_layout(int form2, int N, int M, int ell_w, int F) {
  TwoScanLayout L;
  L.lanes = (((F + 1) / 2) + 63) / 64 * 64;
  L.c8 = ell_w <= 8;
  L.ub = L.c8 ? 8 : 32;  // compressed state: 8 bytes per pair, or 16 per pair stored per lane as 32
  const size_t lanes = (size_t)L.lanes, slots = (size_t)ell_w * M;
  size_t off = 0;
  L.zmn = off;   off = al256(off + slots * lanes * 2);
  L.lmn = off;   if (form2 == 0) off = al256(off + slots * lanes * 2);
  L.st = off;    if (form2 == 1) off = al256(off + (size_t)M * lanes * (L.c8 ? 8 : 16));
  L.q0 = off;    off = al256(off + (size_t)N * lanes * 2);
  L.zp = off;    off = al256(off + (size_t)N * lanes * 4);
  L.act = off;   off = al256(off + 3 * lanes * 4);
  L.fail = off;  off = al256(off + 3 * lanes * 4);
  L.iters = off; off = al256(off + 2 * lanes * 4);
  L.ok = off;    off = al256(off + lanes * 4);
  L.total = off;
  return L;
}

bool twoscan_stream_eligible(int N, int M, int ell_w, int max_row_deg, int max_col_deg, int qm, int form2, int F) {
  if (max_row_deg > 16 || max_col_deg > kDvMax || 128 + (int64_t)(max_col_deg + 1) * qm > 2048) return false;
  if (form2 == 1 && M >= (1 << 24)) return false;
  const TwoScanLayout L = twoscan_layout(form2, N, M, ell_w, F);
  return (uint64_t)ell_w * M * L.lanes < (1ull << 32) && (uint64_t)N * L.lanes < (1ull << 32);
}

cudaError_t twoscan_stream_decode(const DevCode& c, const IntRule& r, int form2, const TwoScanLayout& L, void* ws,
                                  const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop, uint8_t* bits,
                                  int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st) {
  char* b = static_cast<char*>(ws);
  TS s;
  s.zmn = reinterpret_cast<uint16_t*>(b + L.zmn);
  s.lmn = reinterpret_cast<uint16_t*>(b + L.lmn);
  s.st = b + L.st;
  s.q0 = reinterpret_cast<uint16_t*>(b + L.q0);
  s.zp = reinterpret_cast<uint32_t*>(b + L.zp);
  s.act = reinterpret_cast<uint32_t*>(b + L.act);
  s.fail = reinterpret_cast<uint32_t*>(b + L.fail);
  s.iters = reinterpret_cast<int32_t*>(b + L.iters);
  s.okw = reinterpret_cast<uint32_t*>(b + L.ok);
  s.F = F;
  s.FP = L.lanes;
  s.ub = L.ub;
  const bool es = early_stop != 0;
  // the vertical kernel keeps a column's messages in arrays of 8 entries when
  // every column has degree <= 8 (fewer registers, more warps), else 16
  const auto run = [&](auto dvm) {
    constexpr int DVM = decltype(dvm)::value;
    if (form2 == 0) return es ? ts_run<0, true, true, DVM>(c, r, s, llr, max_iter, bits, iters, ok, zout, st)
                              : ts_run<0, true, false, DVM>(c, r, s, llr, max_iter, bits, iters, ok, zout, st);
    if (L.c8) return es ? ts_run<1, true, true, DVM>(c, r, s, llr, max_iter, bits, iters, ok, zout, st)
                        : ts_run<1, true, false, DVM>(c, r, s, llr, max_iter, bits, iters, ok, zout, st);
    return es ? ts_run<1, false, true, DVM>(c, r, s, llr, max_iter, bits, iters, ok, zout, st)
              : ts_run<1, false, false, DVM>(c, r, s, llr, max_iter, bits, iters, ok, zout, st);
  };
  return L.dvmax <= 8 ? run(std::integral_constant<int, 8>{}) : run(std::integral_constant<int, kDvMax>{});
}

}  // namespace ldpc
