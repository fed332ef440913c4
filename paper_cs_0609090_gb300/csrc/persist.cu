// persist.cu -- single-scan min-sum (Section IV Eq. (3); Section V) for codes
// whose frame state does not fit one SM, run as ONE persistent kernel launch per
// decode that keeps a group of frames resident in L2 for all its iterations.
//
// Frame state in the workspace (lane = frame pair; FP lanes, 32 per chunk):
//   zb [2][N][FP] half2  two posterior buffers.  Iteration k reads Z^(k-1) from
//                        zb[(k-1)&1] and adds L^(k) - L^(k-2) into zb[k&1], which
//                        holds Z^(k-2); afterwards zb[k&1] holds Z^(k).  Both
//                        buffers start at Z^(0) = q0 (L^(0) = L^(-1) = 0).  The
//                        adds are f16x2 atomics.  Every partial sum is q0_n plus
//                        one message of each check of n (either L^(k) or
//                        L^(k-2)), an integer of magnitude <= 127 + d_v Qm < 2048,
//                        which binary16 holds exactly: the sums are exact and do
//                        not depend on the order of the atomics.  There is no
//                        column pass and no accumulator reset.
//   st [2][rows][FP]     Section V state (A, B, n~, signs) of iterations k-1 and
//                        k-2: 8 bytes per pair when every check has degree <= 8,
//                        else 16 (rows = M); or per-edge bytes L + 128 (u16 per
//                        pair, rows = ell_w M edge slots).  Iteration k reads
//                        both and overwrites the older.
//   act/fail [3][FP]     per-pair bit masks: frames running at iteration j, and
//                        frames whose decisions x^(j-1) fail a check (found by
//                        iteration j), at index j mod 3.
//   iters [2 FP], okw [FP], and the control block of the work queue.
//
// Work items (persist.cuh), per group of W chunks, in this order:
//   INIT    (chunk, 64-variable tile): channel values to both posterior buffers,
//           a slice of the state cleared, the chunk's flags set;
//   ROW k   (k = 1 .. max_iter; chunk, tile of kPPTile checks of the
//           degree-sorted order): Eq. (3) with the stored state, waits for ROW
//           k-1 of its chunk;
//   FINAL   (chunk, tile of checks): syndrome of x^(max_iter);
//   OUTPUT  (chunk, 64-variable tile): decisions, posteriors, iterations, flags
//           back to frame-major order.
// A group's state (about 33 MB per chunk on the N = 64800 code) stays in L2
// from its first iteration to its last.
//
// Stop rule (Section III, checked before the first iteration too): ROW k finds
// the parity of x^(k-1); ROW k+1 stops the frames whose x^(k-1) satisfied H
// (their result is Z^(k-1), in zb[(k-1)&1], which no later item of that frame
// changes) and masks them out of its atomics.
#include <algorithm>
#include <mutex>

#include "h2_body.cuh"
#include "kernels.h"
#include "persist.cuh"
#include "pp_check.cuh"

namespace ldpc {
namespace {

constexpr int kPPWarps = 8;
constexpr int kPPThreads = kPPWarps * 32;
constexpr uint32_t kFull = 0xffffffffu;
// CTAs per SM the Section V kernel is compiled for (registers: 65536 / (256 x this))
#ifndef LDPC_PP_MINB
#define LDPC_PP_MINB 4
#endif

enum : uint32_t { IT_DONE = 0, IT_INIT = 1, IT_ROW = 2, IT_FINAL = 3, IT_OUTPUT = 4, IT_ABORT = 5 };

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct PPView {
  uint32_t* zb;    // [2][N][FP]
  char* st;        // [2][rows][FP] units of ub bytes
  uint32_t* act;   // [3][FP]
  uint32_t* fail;  // [3][FP]
  int32_t* iters;  // [2 FP]
  uint32_t* okw;   // [FP]
  PQueue q;
  const int8_t* llr;
  uint8_t* bits;
  int32_t* iters_out;
  uint8_t* ok_out;
  int16_t* zout;
  int32_t F, FP, K;
  int32_t chunks, W, groups, nvt, T;
  int32_t rows, ub;
  uint32_t max_spins;
};

__device__ __forceinline__ uint32_t half_mask(uint32_t b) {
  return ((b & 1u) ? 0x0000ffffu : 0u) | ((b & 2u) ? 0xffff0000u : 0u);
}
__device__ __forceinline__ uint32_t valid_bits(int p, int F) {
  return (2 * p < F ? 1u : 0u) | (2 * p + 1 < F ? 2u : 0u);
}

// ------------------------------------------------------------ check updates

// Pass 2: adds L^(k) - L^(k-2) (masked to the running frames) at the handles h[j]
// of Za, o2 being the state of iteration k-2; returns the new state unit.
template <int D, int DMAX, bool C8>
__device__ __forceinline__ typename SVUnit<C8>::T sv_pass2(const NewState& n, const SV& o2, const uint32_t* h, int d,
                                                           uint32_t* __restrict__ Za, uint32_t amask) {
  constexpr int NJ = D > 0 ? D : DMAX;
  const uint32_t Dn = hsub(n.Bn, n.An), D2 = hsub(o2.B, o2.A);
  uint32_t SN = n.Sn, SO = o2.S;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      const uint32_t Ln = hfma(Dn, heq_one(n.In, h2c(j)), n.An) ^ (SN & 0x80008000u);
      const uint32_t Lo = hfma(D2, heq_one(o2.I, h2c(j)), o2.A) ^ (SO & 0x80008000u);
      SN += SN;
      SO += SO;
      if (amask != 0u) red_add_h2(Za + h[j], hsub(Ln, Lo) & amask);
    }
  }
  if constexpr (C8) {
    return make_uint2((uint32_t)n.al | ((uint32_t)n.ah << 8) | ((uint32_t)n.bl << 16) | ((uint32_t)n.bh << 24),
                      (uint32_t)n.il | ((uint32_t)n.ih << 16) | (n.Sn & 0xff00ff00u));
  } else {
    return make_uint4(n.An, n.Bn, n.In, n.Sn);
  }
}

// One check, per-edge form: l1[j] / l2[j] the stored messages of iterations k-1 /
// k-2 (byte pairs); returns the new ones in l2.
template <int D, int DMAX, bool ES>
__device__ __forceinline__ void pe_check(const uint32_t* w, const uint32_t* h, int d, const uint32_t* l1, uint32_t* l2,
                                         const H2Rule& rule, uint32_t ksat, uint32_t* __restrict__ Za, uint32_t amask,
                                         uint32_t& par) {
  constexpr int NJ = D > 0 ? D : DMAX;
  uint32_t K1 = ksat, K2 = ksat, NEG = 0, Y = 0;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      const uint32_t u = hsub(w[j], pe_to_h2(l1[j]));
      if (ES) Y ^= dec_bits(w[j]);
      key_step(u, j, K1, K2, NEG);
    }
  }
  const NewState n = finish_state(K1, K2, NEG, D > 0 ? D : d, rule);
  const uint32_t Dn = hsub(n.Bn, n.An);
  uint32_t SN = n.Sn;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      const uint32_t Ln = hfma(Dn, heq_one(n.In, h2c(j)), n.An) ^ (SN & 0x80008000u);
      SN += SN;
      if (amask != 0u) red_add_h2(Za + h[j], hsub(Ln, pe_to_h2(l2[j])) & amask);
      l2[j] = h2_to_pe(Ln);
    }
  }
  if (ES) par = ((Y >> 15) & 1u) | ((Y >> 30) & 2u);
}

// ------------------------------------------------------------ warp items

#ifndef LDPC_PP_ROWS
#define LDPC_PP_ROWS 8
#endif
#ifndef LDPC_PP_STAGES
#define LDPC_PP_STAGES 4
#endif
constexpr int kPPRows = LDPC_PP_ROWS;  // checks per ROW or FINAL item (one warp)
constexpr int kPPVars = 32;   // variables per INIT or OUTPUT item (one warp)
constexpr int kStages = LDPC_PP_STAGES;  // cp.async ring: checks whose loads a warp keeps in flight
constexpr int kHandles = (kPPRows * 8 + 31) / 32 * 32;

// Per-warp shared memory.  ROW items: the item's handles (variable x FP) and a
// ring of kStages stages, each holding one check's inputs as copied from L2:
//   Section V (8-byte state): 8 posterior lines [8][128 B] | S1 [32][8 B] | S2 [32][8 B]
//   per edge: 8 posterior lines [8][128 B] | L1 [8][64 B] | L2 [8][64 B]
// INIT items: int8 [64 frames][kInStride]; OUTPUT items: u32 [32 variables][33].
template <int FORM>
struct Stage {
  static constexpr int kBytes = FORM == 1 ? 1536 : 2048;
};
constexpr int kInStride = 36;
template <int FORM>
constexpr int warp_smem_bytes() {
  return std::max(kHandles * 4 + kStages * Stage<FORM>::kBytes, std::max(64 * kInStride, 32 * 33 * 4));
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct RowCtx {
  const uint32_t* Zc;  // Z^(k-1) at the chunk's first pair
  const uint32_t* Zr;  // Z^(k-1) at the lane's pair
  uint32_t* Za;        // Z^(k-2) -> Z^(k), at the lane's pair
  const char* S1c;     // state of k-1 at the chunk's first pair (bytes)
  const char* S2c;     // state of k-2 at the chunk's first pair
  const char* S1;      // the same at the lane's pair
  char* S2;
  uint32_t FP, M, ub;
  uint32_t amask, ksat;
  H2Rule rule;
};

// Copies the inputs of check m (position handles hs[0 .. D-1]) into a stage at
// shared address sb: 16 bytes per lane and copy, L2 only (cp.async.cg).
template <int FORM, int D>
__device__ __forceinline__ void stage_check(const RowCtx& x, const uint32_t* hs, int m, uint32_t sb, int lane) {
  if constexpr (FORM == 1) {
    constexpr int NQ = 8 * D + 32;
    const size_t so = (size_t)m * x.FP * 8;
#pragma unroll
    for (int q0 = 0; q0 < NQ; q0 += 32) {
      const int q = q0 + lane;
      if (q < 8 * D) {
        const int j = q >> 3, part = q & 7;
        cp16(sb + j * 128 + part * 16, x.Zc + hs[j] + part * 4);
      } else if (q < 8 * D + 16) {
        const int part = q - 8 * D;
        cp16(sb + 1024 + part * 16, x.S1c + so + part * 16);
      } else if (q < NQ) {
        const int part = q - 8 * D - 16;
        cp16(sb + 1280 + part * 16, x.S2c + so + part * 16);
      }
    }
  } else {
    constexpr int NQ = 16 * D;
#pragma unroll
    for (int q0 = 0; q0 < NQ; q0 += 32) {
      const int q = q0 + lane;
      if (q < 8 * D) {
        const int j = q >> 3, part = q & 7;
        cp16(sb + j * 128 + part * 16, x.Zc + hs[j] + part * 4);
      } else if (q < 12 * D) {
        const int j = (q - 8 * D) >> 2, part = (q - 8 * D) & 3;
        cp16(sb + 1024 + j * 64 + part * 16, x.S1c + (size_t)(j * x.M + m) * x.FP * 2 + part * 16);
      } else if (q < NQ) {
        const int j = (q - 12 * D) >> 2, part = (q - 12 * D) & 3;
        cp16(sb + 1536 + j * 64 + part * 16, x.S2c + (size_t)(j * x.M + m) * x.FP * 2 + part * 16);
      }
    }
  }
}

// kPPRows checks of degree D from m0 (Section V state in 8 bytes, or per edge):
// the inputs of the next kStages - 1 checks are in flight while one is computed.
template <int FORM, bool ES, int D>
__device__ __forceinline__ uint32_t row_staged(const DevCode& c, const RowCtx& x, int m0, int lane, uint32_t* hs,
                                            const char* stages, uint32_t sstages) {
  constexpr int SB = Stage<FORM>::kBytes;
  for (int e = lane; e < kPPRows * D; e += 32) {
    const int r = e / D, j = e - r * D;
    hs[e] = (uint32_t)c.col(j, m0 + r) * x.FP;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < kStages - 1; ++r) {
    stage_check<FORM, D>(x, hs + r * D, m0 + r, sstages + r * SB, lane);
    cp_commit();
  }
  uint32_t fail = 0;
#pragma unroll 1
  for (int r = 0; r < kPPRows; ++r) {
    const int rn = r + kStages - 1;
    __syncwarp();  // every lane has read the stage that check rn reuses
    if (rn < kPPRows) stage_check<FORM, D>(x, hs + rn * D, m0 + rn, sstages + (rn % kStages) * SB, lane);
    cp_commit();
    cp_wait<kStages - 1>();
    __syncwarp();
    const char* sp = stages + (r % kStages) * SB;
    const int m = m0 + r;
    uint32_t w[D];
#pragma unroll
    for (int j = 0; j < D; ++j) w[j] = reinterpret_cast<const uint32_t*>(sp + j * 128)[lane];
    uint32_t par = 0;
    if constexpr (FORM == 1) {
      const uint2 s1 = reinterpret_cast<const uint2*>(sp + 1024)[lane];
      const uint2 s2 = reinterpret_cast<const uint2*>(sp + 1280)[lane];
      const NewState n = sv_pass1<D, D, ES>(w, D, SVUnit<true>::unpack(s1), x.rule, x.ksat, par);
      __stcg(reinterpret_cast<uint2*>(x.S2) + (size_t)m * x.FP,
             sv_pass2<D, D, true>(n, SVUnit<true>::unpack(s2), hs + r * D, D, x.Za, x.amask));
    } else {
      uint32_t l1[D], l2[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        l1[j] = reinterpret_cast<const uint16_t*>(sp + 1024 + j * 64)[lane];
        l2[j] = reinterpret_cast<const uint16_t*>(sp + 1536 + j * 64)[lane];
      }
      pe_check<D, D, ES>(w, hs + r * D, D, l1, l2, x.rule, x.ksat, x.Za, x.amask, par);
#pragma unroll
      for (int j = 0; j < D; ++j)
        __stcg(reinterpret_cast<uint16_t*>(x.S2) + (size_t)(j * x.M + m) * x.FP, (uint16_t)l2[j]);
    }
    fail |= par;
  }
  return fail;
}

// Any item: checks one at a time from registers, degrees up to DMAX.
template <int FORM, bool C8, bool ES>
__device__ __forceinline__ uint32_t row_generic(const DevCode& c, const RowCtx& x, int m0, int nr) {
  constexpr int DMAX = (FORM == 1 && C8) ? 8 : 16;
  using U = typename SVUnit<C8>::T;
  uint32_t fail = 0;
  for (int r = 0; r < nr; ++r) {
    const int m = m0 + r;
    const int d = c.deg(m);
    uint32_t h[DMAX], w[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
      if (j < d) {
        h[j] = (uint32_t)c.col(j, m) * x.FP;
        w[j] = __ldcg(x.Zr + h[j]);
      }
    }
    uint32_t par = 0;
    if constexpr (FORM == 1) {
      const U s1 = __ldcg(reinterpret_cast<const U*>(x.S1) + (size_t)m * x.FP);
      const U s2 = __ldcg(reinterpret_cast<const U*>(x.S2) + (size_t)m * x.FP);
      const NewState n = sv_pass1<0, DMAX, ES>(w, d, SVUnit<C8>::unpack(s1), x.rule, x.ksat, par);
      __stcg(reinterpret_cast<U*>(x.S2) + (size_t)m * x.FP,
             sv_pass2<0, DMAX, C8>(n, SVUnit<C8>::unpack(s2), h, d, x.Za, x.amask));
    } else {
      const uint16_t* L1 = reinterpret_cast<const uint16_t*>(x.S1);
      uint16_t* L2 = reinterpret_cast<uint16_t*>(x.S2);
      uint32_t l1[DMAX], l2[DMAX];
#pragma unroll
      for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
          const size_t sl = (size_t)(j * x.M + m) * x.FP;
          l1[j] = __ldcg(L1 + sl);
          l2[j] = __ldcg(L2 + sl);
        }
      }
      pe_check<0, DMAX, ES>(w, h, d, l1, l2, x.rule, x.ksat, x.Za, x.amask, par);
#pragma unroll
      for (int j = 0; j < DMAX; ++j)
        if (j < d) __stcg(L2 + (size_t)(j * x.M + m) * x.FP, (uint16_t)l2[j]);
    }
    fail |= par;
  }
  return fail;
}

template <int FORM, bool C8, bool ES>
__device__ __forceinline__ void pp_row(const DevCode& c, const IntRule& ir, const PPView& s, int k, int ch, int t,
                                       int lane, char* wsm, uint32_t wsm_s) {
  const int p = ch * 32 + lane;
  const int FP = s.FP;
  uint32_t actk = valid_bits(p, s.F);
  if (ES) {
    const int pb = (k - 1) % 3;
    const uint32_t a = __ldcg(s.act + pb * FP + p), f = __ldcg(s.fail + pb * FP + p);
    actk = a & f;
    if (t == 0) {
      // frames whose x^(k-2) satisfied H stop with k - 2 iterations
      const uint32_t stop = a & ~f;
      if (stop & 1u) __stcg(s.iters + 2 * p, k - 2);
      if (stop & 2u) __stcg(s.iters + 2 * p + 1, k - 2);
      if (stop) __stcg(s.okw + p, __ldcg(s.okw + p) | stop);
      __stcg(s.act + (k % 3) * FP + p, actk);
      __stcg(s.fail + ((k + 1) % 3) * FP + p, 0u);
    }
  }
  if (__all_sync(kFull, actk == 0u)) return;
  RowCtx x;
  const size_t nfp = (size_t)c.N * FP, sfp = (size_t)s.rows * FP * s.ub;
  const int rb = (k - 1) & 1, wb = k & 1;
  x.Zc = s.zb + (size_t)rb * nfp + ch * 32;
  x.Zr = x.Zc + lane;
  x.Za = s.zb + (size_t)wb * nfp + p;
  x.S1c = s.st + (size_t)rb * sfp + (size_t)ch * 32 * s.ub;
  x.S2c = s.st + (size_t)wb * sfp + (size_t)ch * 32 * s.ub;
  x.S1 = x.S1c + (size_t)lane * s.ub;
  x.S2 = const_cast<char*>(x.S2c) + (size_t)lane * s.ub;
  x.FP = (uint32_t)FP;
  x.M = (uint32_t)c.M;
  x.ub = (uint32_t)s.ub;
  x.amask = half_mask(actk);
  x.rule = make_h2rule(ir);
  // (16 Qm + 15) 2^-11: the largest key of a magnitude saturated to Qm
  x.ksat = hfma(ints_to_h2(ir.qm, ir.qm), h2c_q11(16), h2c_q11(15));
  const int m0 = t * kPPRows;
  const int nr = min(kPPRows, c.M - m0);
  if (nr <= 0) return;
  uint32_t fail;
  const int d0 = c.deg(m0);
  uint32_t* hs = reinterpret_cast<uint32_t*>(wsm);
  const char* stages = wsm + kHandles * 4;
  const uint32_t sst = wsm_s + kHandles * 4;
  if ((FORM == 0 || C8) && nr == kPPRows && d0 == c.deg(m0 + nr - 1) && (d0 == 6 || d0 == 7)) {
    fail = d0 == 6 ? row_staged<FORM, ES, 6>(c, x, m0, lane, hs, stages, sst)
                   : row_staged<FORM, ES, 7>(c, x, m0, lane, hs, stages, sst);
  } else {
    fail = row_generic<FORM, C8, ES>(c, x, m0, nr);
  }
  if (ES && (fail & actk)) atomicOr(s.fail + (k % 3) * FP + p, fail & actk);
}

template <bool ES>
__device__ __forceinline__ void pp_final(const DevCode& c, const PPView& s, int ch, int t, int lane) {
  const int p = ch * 32 + lane, FP = s.FP, K = s.K;
  uint32_t act1 = valid_bits(p, s.F);
  if (ES) {
    const int pb = K % 3;
    const uint32_t a = __ldcg(s.act + pb * FP + p), f = __ldcg(s.fail + pb * FP + p);
    act1 = a & f;
    if (t == 0) {
      const uint32_t stop = a & ~f;
      if (stop & 1u) __stcg(s.iters + 2 * p, K - 1);
      if (stop & 2u) __stcg(s.iters + 2 * p + 1, K - 1);
      if (stop) __stcg(s.okw + p, __ldcg(s.okw + p) | stop);
    }
  }
  if (t == 0) __stcg(s.act + ((K + 1) % 3) * FP + p, act1);
  if (__all_sync(kFull, act1 == 0u)) return;
  const uint32_t* Zk = s.zb + (size_t)(K & 1) * c.N * FP + p;
  const int m0 = t * kPPRows;
  const int m1 = min(m0 + kPPRows, c.M);
  uint32_t fail = 0;
  for (int m = m0; m < m1; ++m) {
    const int d = c.deg(m);
    uint32_t y = 0;
    for (int j = 0; j < d; ++j) y ^= dec_bits(__ldcg(Zk + (size_t)c.col(j, m) * FP));
    fail |= ((y >> 15) & 1u) | ((y >> 30) & 2u);
  }
  if (fail & act1) atomicOr(s.fail + ((K + 1) % 3) * FP + p, fail & act1);
}

// Channel values of 32 variables and the chunk's 64 frames into both posterior
// buffers; a slice of the state cleared; the chunk's flags (first item).
template <int FORM, bool ES>
__device__ __forceinline__ void pp_init(const DevCode& c, const PPView& s, int ch, int i, int lane, char* wsm) {
  const int N = c.N, FP = s.FP, F = s.F;
  const int n0 = i * kPPVars, p0 = ch * 32;
  int8_t* tile = reinterpret_cast<int8_t*>(wsm);  // [64 frames][kInStride]
  const bool nin = n0 + lane < N;
#pragma unroll 4
  for (int fl = 0; fl < 64; ++fl) {
    const int f = 2 * p0 + fl;
    tile[fl * kInStride + lane] = (f < F && nin) ? __ldg(s.llr + (size_t)f * N + n0 + lane) : (int8_t)0;
  }
  __syncwarp();
  uint32_t* z0 = s.zb + p0 + lane;
  uint32_t* z1 = s.zb + (size_t)N * FP + p0 + lane;
  const int nl1 = min(kPPVars, N - n0);
  for (int nl = 0; nl < nl1; ++nl) {
    const uint32_t hz = ints_to_h2(tile[(2 * lane) * kInStride + nl], tile[(2 * lane + 1) * kInStride + nl]);
    const size_t o = (size_t)(n0 + nl) * FP;
    __stcg(z0 + o, hz);
    __stcg(z1 + o, hz);
  }
  // L^(0) = L^(-1) = 0: this item's slice of the state, both buffers (Section V:
  // all zero; per edge: bytes 0x80)
  const int per = (s.rows + s.nvt - 1) / s.nvt;
  const int r0 = i * per, r1 = min(s.rows, r0 + per);
  const int q = 32 * s.ub / 16;  // 16-byte words per row of the chunk
  const uint32_t fv = FORM == 1 ? 0u : 0x80808080u;
  const uint4 fill = make_uint4(fv, fv, fv, fv);
  for (int b = 0; b < 2; ++b) {
    char* base = s.st + (size_t)b * s.rows * FP * s.ub + (size_t)p0 * s.ub;
    for (int e = lane; e < (r1 - r0) * q; e += 32) {
      const int r = r0 + e / q, part = e - (e / q) * q;
      __stcg(reinterpret_cast<uint4*>(base + (size_t)r * FP * s.ub) + part, fill);
    }
  }
  if (i == 0) {
    const int p = p0 + lane;
    __stcg(s.act + p, valid_bits(p, F));
    __stcg(s.fail + p, ES ? kFull : 0u);  // "x^(-1) failed": every valid frame runs iteration 1
    __stcg(s.fail + FP + p, 0u);
    __stcg(s.fail + 2 * FP + p, 0u);
    __stcg(s.iters + 2 * p, s.K);
    __stcg(s.iters + 2 * p + 1, s.K);
    __stcg(s.okw + p, 0u);
  }
  __syncwarp();
}

// Decisions (and posteriors) of 32 variables of the chunk's frames back to
// frame-major order; iterations and flags (first item).
__device__ __forceinline__ void pp_output(const DevCode& c, const PPView& s, int ch, int i, int lane, char* wsm) {
  const int N = c.N, FP = s.FP, F = s.F, N8 = (N + 7) >> 3;
  const int n0 = i * kPPVars, p0 = ch * 32, p = p0 + lane;
  uint32_t* tile = reinterpret_cast<uint32_t*>(wsm);  // [32 variables][33]
  // each frame's result is the buffer of its iteration count
  const int32_t itl = __ldcg(s.iters + 2 * p), ith = __ldcg(s.iters + 2 * p + 1);
  const size_t nfp = (size_t)N * FP;
  const uint32_t* zl = s.zb + (size_t)(itl & 1) * nfp + p;
  const uint32_t* zh = s.zb + (size_t)(ith & 1) * nfp + p;
  const int nl1 = min(kPPVars, N - n0);
  for (int nl = 0; nl < nl1; ++nl) {
    const size_t o = (size_t)(n0 + nl) * FP;
    const uint32_t a = __ldcg(zl + o);
    tile[nl * 33 + lane] = (zl == zh) ? a : ((a & 0xffffu) | (__ldcg(zh + o) & 0xffff0000u));
  }
  __syncwarp();
  // 4 bytes of decisions per frame; this lane: frames 2 lane, 2 lane + 1
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int f = 2 * p0 + 2 * lane + h;
    if (f >= F) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int nb = (n0 >> 3) + b;
      if (nb >= N8) continue;
      uint32_t byte = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int nl = 8 * b + u;
        if (nl < nl1) byte |= ((dec_bits(tile[nl * 33 + lane] >> (16 * h)) >> 15) & 1u) << u;
      }
      s.bits[(size_t)f * N8 + nb] = (uint8_t)byte;
    }
  }
  if (s.zout != nullptr && lane < nl1) {
    for (int fl = 0; fl < 64; ++fl) {
      const int f = 2 * p0 + fl;
      if (f >= F) break;
      const uint32_t hz = tile[lane * 33 + (fl >> 1)];
      s.zout[(size_t)f * N + n0 + lane] = (int16_t)((fl & 1) ? h_hi_int(hz) : h_lo_int(hz));
    }
  }
  if (i == 0) {
    const int kb = (s.K + 1) % 3;
    const uint32_t a = __ldcg(s.act + kb * FP + p), fl = __ldcg(s.fail + kb * FP + p);
    const uint32_t okw = __ldcg(s.okw + p);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int f = 2 * p + h;
      if (f >= F) continue;
      s.iters_out[f] = h ? ith : itl;
      s.ok_out[f] = ((a >> h) & 1u) ? (uint8_t)(((fl >> h) & 1u) ^ 1u) : (uint8_t)((okw >> h) & 1u);
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------ the kernel

// Item it (every lane computes it): kind, chunk, index within the chunk's
// phase, iteration, and the chunk counter value it waits for.
__device__ __forceinline__ void pp_item(const PPView& s, uint32_t tk, uint32_t& kind, uint32_t& ch, uint32_t& idx,
                                        uint32_t& k, uint32_t& target) {
  const uint32_t nvt = (uint32_t)s.nvt, T = (uint32_t)s.T, K = (uint32_t)s.K;
  const uint32_t per_chunk = 2 * nvt + (K + 1) * T;
  const uint32_t Ig = (uint32_t)s.W * per_chunk;
  const uint32_t g = tk / Ig;
  uint32_t o = tk - g * Ig;
  kind = IT_DONE;
  ch = idx = k = target = 0;
  if (g >= (uint32_t)s.groups) return;
  const uint32_t w = min((uint32_t)s.W, (uint32_t)s.chunks - g * (uint32_t)s.W);
  if (o >= w * per_chunk) return;
  const uint32_t c0 = g * (uint32_t)s.W;
  if (o < w * nvt) {
    kind = IT_INIT;
    ch = c0 + o / nvt;
    idx = o % nvt;
    return;
  }
  o -= w * nvt;
  if (o < K * w * T) {
    kind = IT_ROW;
    k = o / (w * T) + 1;
    const uint32_t r = o - (k - 1) * w * T;
    ch = c0 + r / T;
    idx = r % T;
    target = nvt + (k - 1) * T;
    return;
  }
  o -= K * w * T;
  if (o < w * T) {
    kind = IT_FINAL;
    ch = c0 + o / T;
    idx = o % T;
    target = nvt + K * T;
    return;
  }
  o -= w * T;
  kind = IT_OUTPUT;
  ch = c0 + o / nvt;
  idx = o % nvt;
  target = nvt + (K + 1) * T;
}

// All lanes: waits until every lane's acquire load of *cnt reads >= target.
// false when it gave up (setting the error word) or another warp had set it.
__device__ __forceinline__ bool pq_wait_warp(const PQueue& q, const uint32_t* cnt, uint32_t target,
                                             uint32_t max_spins) {
  if (__all_sync(kFull, ld_acquire_gpu(cnt) >= target)) return true;
  for (uint32_t i = 0; i < max_spins; ++i) {
    __nanosleep(128);
    if (__all_sync(kFull, ld_acquire_gpu(cnt) >= target)) return true;
    if ((i & 63u) == 63u && __any_sync(kFull, ld_relaxed_gpu(q.err()) != 0u)) return false;
  }
  if ((threadIdx.x & 31) == 0) atomicOr(q.err(), 1u);
  return false;
}

// Warp-granular items handed out round-robin: warp g of the grid (G warps) takes
// items g, g + G, g + 2G, ...  An item depends only on lower-numbered items of
// its chunk, each held by a warp that is running (the launch is cooperative, so
// every warp of the grid is resident) and that takes its items in order; so the
// lowest unfinished item can always proceed.
template <int FORM, bool C8, bool ES>
__global__ void __launch_bounds__(kPPThreads, FORM == 1 ? LDPC_PP_MINB : 3) pp_kernel(const DevCode c, const IntRule ir,
                                                                                      const PPView s) {
  extern __shared__ __align__(16) char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int WB = warp_smem_bytes<FORM>();
  char* wsm = smem + warp * WB;
  const uint32_t wsm_s = (uint32_t)__cvta_generic_to_shared(wsm);
  const uint32_t G = gridDim.x * kPPWarps;
  uint32_t last_ch = ~0u, last_target = 0;
  for (uint32_t it = blockIdx.x * kPPWarps + warp;; it += G) {
    uint32_t kind, ch, idx, k, target;
    pp_item(s, it, kind, ch, idx, k, target);
    if (kind == IT_DONE) break;
    if (kind != IT_INIT && !(ch == last_ch && target <= last_target)) {
      if (!pq_wait_warp(s.q, s.q.cnt((int)ch), target, s.max_spins)) break;
      last_ch = ch;
      last_target = target;
    }
    if (kind == IT_ROW) pp_row<FORM, C8, ES>(c, ir, s, (int)k, (int)ch, (int)idx, lane, wsm, wsm_s);
    else if (kind == IT_INIT) pp_init<FORM, ES>(c, s, (int)ch, (int)idx, lane, wsm);
    else if (kind == IT_FINAL) pp_final<ES>(c, s, (int)ch, (int)idx, lane);
    else pp_output(c, s, (int)ch, (int)idx, lane, wsm);
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(s.q.cnt((int)ch), 1u);
  }
}

// After the decode: if a wait gave up, every frame reports iters = -1, ok = 0.
__global__ void pp_epilogue(const uint32_t* err, int32_t F, int32_t* iters, uint8_t* ok) {
  if (ld_relaxed_gpu(err) == 0u) return;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x) {
    iters[f] = -1;
    ok[f] = 0;
  }
}

// A CTA that waits on a counter nothing increments, with the given bound.
__global__ void pp_wait_probe(PQueue q, uint32_t max_spins) {
  if (threadIdx.x < 32) pq_wait_warp(q, q.cnt(0), 1u, max_spins);
}

template <int FORM, bool C8, bool ES>
cudaError_t pp_launch(const DevCode& c, const IntRule& r, const PPView& v, int sm_count, cudaStream_t st) {
  constexpr int smem = kPPWarps * warp_smem_bytes<FORM>();
  static std::mutex mu;
  static int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (per_sm == 0) {
      cudaError_t e = cudaFuncSetAttribute(pp_kernel<FORM, C8, ES>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pp_kernel<FORM, C8, ES>, kPPThreads, smem);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(per_sm * sm_count));
  cfg.blockDim = dim3(kPPThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, pp_kernel<FORM, C8, ES>, c, r, v);
}

}  // namespace

PersistLayout persist_layout(int form, int N, int M, int ell_w, int F, int group_chunks) {
  PersistLayout L;
  L.lanes = (((F + 1) / 2) + 31) / 32 * 32;
  L.chunks = L.lanes / 32;
  L.W = std::max(1, std::min(group_chunks, L.chunks));
  L.c8 = form == 1 && ell_w <= 8;
  L.ub = form == 1 ? (L.c8 ? 8 : 16) : 2;
  L.rows = form == 1 ? M : ell_w * M;
  const size_t lanes = (size_t)L.lanes;
  size_t off = 0;
  L.zb = off;    off = al256(off + 2 * (size_t)N * lanes * 4);
  L.st = off;    off = al256(off + 2 * (size_t)L.rows * lanes * L.ub);
  L.act = off;   off = al256(off + 3 * lanes * 4);
  L.fail = off;  off = al256(off + 3 * lanes * 4);
  L.iters = off; off = al256(off + 2 * lanes * 4);
  L.ok = off;    off = al256(off + lanes * 4);
  L.ctl = off;   off = al256(off + pq_ctl_bytes(L.chunks));
  L.total = off;
  return L;
}

bool persist_int8_eligible(int N, int M, int ell_w, int max_row_deg, int max_col_deg, int qm, int form, int F) {
  if (max_row_deg > 16 || 128 + (int64_t)(max_col_deg + 1) * qm > 2048) return false;
  const PersistLayout L = persist_layout(form, N, M, ell_w, F, 1);
  // 32-bit element offsets within one buffer
  return (uint64_t)N * L.lanes < (1ull << 32) && (uint64_t)L.rows * L.lanes < (1ull << 32);
}

cudaError_t persist_int8_decode(const DevCode& c, const IntRule& r, int form, const PersistLayout& L, void* ws,
                                int sm_count, const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop,
                                uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st) {
  char* b = static_cast<char*>(ws);
  PPView v;
  v.zb = reinterpret_cast<uint32_t*>(b + L.zb);
  v.st = b + L.st;
  v.act = reinterpret_cast<uint32_t*>(b + L.act);
  v.fail = reinterpret_cast<uint32_t*>(b + L.fail);
  v.iters = reinterpret_cast<int32_t*>(b + L.iters);
  v.okw = reinterpret_cast<uint32_t*>(b + L.ok);
  v.q.ctl = reinterpret_cast<uint32_t*>(b + L.ctl);
  v.llr = llr;
  v.bits = bits;
  v.iters_out = iters;
  v.ok_out = ok;
  v.zout = zout;
  v.F = F;
  v.FP = L.lanes;
  v.K = max_iter;
  v.chunks = L.chunks;
  v.W = L.W;
  v.groups = (L.chunks + L.W - 1) / L.W;
  v.nvt = (c.N + kPPVars - 1) / kPPVars;
  v.T = (c.M + kPPRows - 1) / kPPRows;
  v.rows = L.rows;
  v.ub = L.ub;
  v.max_spins = kWaitSpins;
  cudaError_t e = cudaMemsetAsync(b + L.ctl, 0, pq_ctl_bytes(L.chunks), st);
  if (e != cudaSuccess) return e;
  const bool es = early_stop != 0;
  if (form == 1 && L.c8) e = es ? pp_launch<1, true, true>(c, r, v, sm_count, st) : pp_launch<1, true, false>(c, r, v, sm_count, st);
  else if (form == 1) e = es ? pp_launch<1, false, true>(c, r, v, sm_count, st) : pp_launch<1, false, false>(c, r, v, sm_count, st);
  else e = es ? pp_launch<0, false, true>(c, r, v, sm_count, st) : pp_launch<0, false, false>(c, r, v, sm_count, st);
  if (e != cudaSuccess) return e;
  pp_epilogue<<<std::max(1, std::min(64, (F + 255) / 256)), 256, 0, st>>>(v.q.err(), F, iters, ok);
  return cudaGetLastError();
}

cudaError_t persist_wait_selftest(uint32_t max_spins, bool* gave_up) {
  uint32_t* ctl = nullptr;
  cudaError_t e = cudaMalloc(&ctl, pq_ctl_bytes(1));
  if (e != cudaSuccess) return e;
  uint32_t err = 0;
  if ((e = cudaMemset(ctl, 0, pq_ctl_bytes(1))) == cudaSuccess) {
    pp_wait_probe<<<1, 32>>>(PQueue{ctl}, max_spins);
    if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaDeviceSynchronize()) == cudaSuccess)
      e = cudaMemcpy(&err, ctl + kCtlLine, sizeof err, cudaMemcpyDeviceToHost);
  }
  cudaFree(ctl);
  *gave_up = err != 0u;
  return e;
}

}  // namespace ldpc
