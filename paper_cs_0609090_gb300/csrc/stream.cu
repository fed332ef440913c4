// stream.cu -- single-scan min-sum with frame state in device memory, for codes
// whose per-frame state does not fit one SM (Section IV Eq. (3), Section V).
//
// Workspace layout (frame-pair or frame index innermost, so that the lanes of a
// warp -- consecutive frames -- read and atomically update consecutive words):
//   int8 path, lane = frame pair, exact binary16 arithmetic (see h2ops.cuh):
//     Zs [N][FP] half2, Acc [N][FP] i32 (lo + 65536 hi, biased like onchip_h2),
//     state [M][FP] (Section V: uint4, or uint2 when every check has degree
//     <= 8) or [ell_w M][FP] u16 (per-edge bytes L + 128 per edge slot j M + m
//     of the degree-sorted table; by CSR edge in the fallback kernel),
//     q0 [N][FP] u16 (int8 pair), act/fail [2][FP] u32 bit masks, iters [2 FP]
//   float path (stream_f32.cu), lane = frame:
//     Z [2][N][FL] f32 (two posterior buffers), state [M][FL] (Section V:
//     uint4, or 10 bytes when every check has degree <= 8) or per-edge f32,
//     q0 [N][FL] f32, act/fail [2][FL] u32, iters [FL]
// Per iteration: a row kernel (one warp = kRowsPerWarp checks of the
// degree-sorted order for 32 lanes; the checks' column indices are
// warp-uniform loads; warp order per stream_grid.h) then a column kernel that
// applies the stop rule, four lanes per thread.  int8: the row kernel adds
// L^(k) - L^(k-1) to an accumulator that always holds the current posterior
// (exact integer sums), so the column kernel only converts it for the frames
// that continue; the CSR fallback adds L^(k) and its column kernel resets the
// accumulator to Z0.  The syndrome of x^(k-1) is computed by the row kernel of
// iteration k.
#include <algorithm>

#include "h2_body.cuh"
#include "kernels.h"
#include "stream_grid.h"

namespace ldpc {
namespace {

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// E = message slots of the per-edge form: the degree-sorted table's ell_w * M;
// float32 is given max(E, ell_w * M), the sum-product rule addressing the E
// edges of H.  For float32, z and acc are the two posterior buffers.
StreamLayout stream_layout(int dtype, int form, int N, int M, int E, int F) {
  StreamLayout L;
  const bool f32 = dtype == 1;
  const size_t lanes = f32 ? (size_t)((F + 31) / 32) * 32 : (size_t)(((F + 1) / 2 + 31) / 32) * 32;
  L.lanes = (int)lanes;
  size_t off = 0;
  L.z = off;     off = al256(off + (size_t)N * lanes * 4);
  L.acc = off;   off = al256(off + (size_t)N * lanes * 4);
  L.st = off;
  if (form == 1) off = al256(off + (size_t)M * lanes * 16);
  else off = al256(off + (size_t)E * lanes * (f32 ? 4 : 2));
  L.q0 = off;    off = al256(off + (size_t)N * lanes * (f32 ? 4 : 2));
  L.act = off;   off = al256(off + 2 * lanes * 4);
  L.fail = off;  off = al256(off + 2 * lanes * 4);
  L.iters = off; off = al256(off + 2 * lanes * 4);
  L.ok = off;    off = al256(off + 2 * lanes * 4);
  L.total = off;
  return L;
}

bool stream_int8_eligible(int max_row_deg, int max_col_deg, int qm) {
  return max_row_deg <= 16 && 128 + (int64_t)max_col_deg * qm + qm <= 2048;
}

namespace {

// ------------------------------------------------------------------ int8, packed

struct H2S {
  uint32_t* z;
  int32_t* acc;
  uint4* st;
  uint16_t* lm;
  uint16_t* q0;
  uint32_t* act;   // [2][FP]
  uint32_t* fail;  // [2][FP]
  int32_t* iters;  // [2 FP]: frame 2p + b
  uint32_t* ok;    // [FP]
  int FP;
  int psat;        // > 0: the stored posterior Zs is clamped to [-psat, psat]; 0: exact
};

H2S h2s_view(void* ws, const StreamLayout& L) {
  char* b = static_cast<char*>(ws);
  H2S s;
  s.z = reinterpret_cast<uint32_t*>(b + L.z);
  s.acc = reinterpret_cast<int32_t*>(b + L.acc);
  s.st = reinterpret_cast<uint4*>(b + L.st);
  s.lm = reinterpret_cast<uint16_t*>(b + L.st);
  s.q0 = reinterpret_cast<uint16_t*>(b + L.q0);
  s.act = reinterpret_cast<uint32_t*>(b + L.act);
  s.fail = reinterpret_cast<uint32_t*>(b + L.fail);
  s.iters = reinterpret_cast<int32_t*>(b + L.iters);
  s.ok = reinterpret_cast<uint32_t*>(b + L.ok);
  s.FP = L.lanes;
  s.psat = 0;
  return s;
}

// Transposes the frame-major int8 LLRs into pair-interleaved order and sets
// Z^(0), the biased accumulator and the per-pair flags.  Tile: 64 variables x
// 32 pairs (64 frames).
__global__ void __launch_bounds__(256) h2s_init(const DevCode c, const int8_t* __restrict__ llr, int32_t F,
                                                int32_t max_iter, H2S s, int32_t delta) {
  __shared__ int8_t tile[64][65];  // [frame][variable]
  const int n0 = blockIdx.x * 64, p0 = blockIdx.y * 32;
  const int N = c.N;
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
    const int32_t lo = tile[2 * pl][nl], hi = tile[2 * pl + 1][nl];
    const size_t o = (size_t)n * s.FP + p;
    s.q0[o] = (uint16_t)(((uint32_t)lo & 0xffu) | (((uint32_t)hi & 0xffu) << 8));
    s.z[o] = ints_to_h2(lo, hi);
    // delta accumulation holds Z^(k-1) itself; the reset form holds Z0 minus the
    // pattern bias of the col_degree(n) messages that will be added
    s.acc[o] = (int32_t)((uint32_t)acc_pack(lo, hi) - (delta ? 0u : (uint32_t)__ldg(c.cdeg + n) * 0x66006600u));
  }
  if (blockIdx.x == 0) {
    for (int pl = threadIdx.x; pl < 32; pl += blockDim.x) {
      const int p = p0 + pl;
      const uint32_t valid = (2 * p < F ? 1u : 0u) | (2 * p + 1 < F ? 2u : 0u);
      s.act[s.FP + p] = valid;  // read at k = 1 (odd)
      s.act[p] = 0u;
      s.fail[p] = 0u;
      s.fail[s.FP + p] = 0u;
      s.iters[2 * p] = max_iter;
      s.iters[2 * p + 1] = max_iter;
      s.ok[p] = 0u;
    }
  }
}

// One check for the frame pair of this lane (Eq. (3); Section V state or
// per-edge bytes).  Returns the decision parity of x^(k-1) (bit 0 lo, bit 1 hi).
template <int FORM, bool ES>
__device__ __forceinline__ uint32_t h2s_check(const DevCode& c, const IntRule& r, uint32_t qm2, int m, int p,
                                              const H2S& s) {
  const size_t FP = (size_t)s.FP;
  const int e0 = __ldg(c.rp + m);
  const int d = __ldg(c.rp + m + 1) - e0;
  uint32_t A2 = 0, B2 = 0, I2 = 0, S = 0;
  if constexpr (FORM == 1) {
    const uint4 st = s.st[(size_t)m * FP + p];
    A2 = st.x;
    B2 = st.y;
    I2 = st.z;
    S = st.w;
  }
  uint32_t K1 = h2c(2048), K2 = h2c(2048), X = 0, NEG = 0, Y = 0;
  uint32_t jj = 0;  // position j as half2
  for (int j = 0; j < d; ++j, jj = hadd(jj, h2c(1))) {
    const int n = __ldg(c.ci + e0 + j);
    const uint32_t w = s.z[(size_t)n * FP + p];
    uint32_t L;
    if constexpr (FORM == 1) {
      // f(A, B, n, n~) with the sign s_mn applied to the binary16 sign bit
      const uint32_t msk = heq_mask(I2, jj);
      L = ((B2 & msk) | (A2 & ~msk)) ^ ((S << (15 - j)) & 0x80008000u);
    } else {
      const uint32_t b = s.lm[(size_t)(e0 + j) * FP + p];
      L = hfma(__byte_perm(b, 0x58u, 0x4140), h2c(8), 0xE480E480u);
    }
    const uint32_t u = hsub(w, L);
    X ^= u;
    if constexpr (ES) Y ^= dec_bits(w);
    NEG |= (u & 0x80008000u) >> (15 - j);
    const uint32_t key = hfma(hmin(habs(u), qm2), h2c(16), jj);
    K2 = hmin(K2, hmax(K1, key));
    K1 = hmin(K1, key);
  }
  const uint32_t dm = (d >= 16) ? 0xffffu : ((1u << d) - 1u);
  const uint32_t Sn = (NEG ^ prmt(X, 0u, 0xBB99u)) & (dm | (dm << 16));
  const int32_t k1l = h_lo_int(K1), k1h = h_hi_int(K1), k2l = h_lo_int(K2), k2h = h_hi_int(K2);
  const uint32_t An = small_to_h2(r.g(k1l >> 4), r.g(k1h >> 4));
  const uint32_t Bn = small_to_h2(r.g(k2l >> 4), r.g(k2h >> 4));
  const uint32_t In = small_to_h2(k1l & 15, k1h & 15);
  jj = 0;
  for (int j = 0; j < d; ++j, jj = hadd(jj, h2c(1))) {
    const int n = __ldg(c.ci + e0 + j);
    const uint32_t msk = heq_mask(In, jj);
    const uint32_t mag = (Bn & msk) | (An & ~msk);
    const uint32_t L = mag ^ ((Sn << (15 - j)) & 0x80008000u);
    atomicAdd(s.acc + (size_t)n * FP + p, (int32_t)hadd(L, h2c(1536)));
    if constexpr (FORM == 0) {
      const uint32_t hb = hfma(L, 0x30003000u, h2c(144));
      s.lm[(size_t)(e0 + j) * FP + p] = (uint16_t)__byte_perm(hb, 0u, 0x4420);
    }
  }
  if constexpr (FORM == 1) s.st[(size_t)m * FP + p] = make_uint4(An, Bn, In, Sn);
  return ES ? (((Y >> 15) & 1u) | ((Y >> 30) & 2u)) : 0u;
}

template <int FORM, bool ES>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) h2s_rows(const DevCode c, const IntRule r, H2S s, int k) {
  const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  int chunk, m0;
  if (!row_map_all(warp, c.M, s.FP, chunk, m0)) return;
  const int p = chunk * 32 + lane;
  const int cur = k & 1;
  if (__all_sync(0xffffffffu, s.act[cur * s.FP + p] == 0u)) return;
  const uint32_t qm2 = ints_to_h2(r.qm, r.qm);
  uint32_t fail = 0;
  const int m1 = min(m0 + kRowsPerWarp, c.M);
  for (int m = m0; m < m1; ++m) fail |= h2s_check<FORM, ES>(c, r, qm2, m, p, s);
  if (ES && fail) atomicOr(s.fail + cur * s.FP + p, fail);
}

// The frame-pair streaming layout as an addressing policy of the shared check
// body (h2_body.cuh): handles are 32-bit element offsets n FP, the lane's own
// pair p is folded into the base pointers, and the column index of a position
// (the same for the whole warp) comes from the degree-sorted edge-slot table.
template <bool WIDE>
struct StreamAddr {
  using H = uint32_t;
  int M;
  uint32_t FP;
  const uint16_t* __restrict__ t16;
  const int32_t* __restrict__ t32;
  __device__ __forceinline__ H at(const uint16_t*, const uint32_t*, int j, int m) const {
    const int n = WIDE ? __ldg(t32 + j * M + m) : (int)__ldg(t16 + j * M + m);
    return (uint32_t)n * FP;
  }
  __device__ __forceinline__ void load(const uint32_t* __restrict__ Zs, H h, uint32_t (&w)[1]) const { w[0] = Zs[h]; }
  __device__ __forceinline__ void add(int32_t* __restrict__ Acc, H h, int, int32_t v) const { atomicAdd(Acc + h, v); }
  __device__ __forceinline__ uint32_t st(int m) const { return (uint32_t)m * FP; }
  __device__ __forceinline__ uint32_t lm(int j, int m) const { return (uint32_t)(j * M + m) * FP; }
};

// Row pass with the exact-degree bodies: one warp = kRowsPerWarp consecutive
// checks of the degree-sorted order for 32 frame pairs.  Per-edge messages are
// kept per edge slot (j * M + internal check).  Offsets are 32-bit (the host
// checks N FP and ell_w M FP < 2^32).  C8: the Section V state in 8 bytes per
// frame pair (codes whose checks all have degree <= 8).
template <int FORM, bool ES, bool WIDE, int MINB, bool DELTA, bool C8 = false>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, MINB) h2s_rows_ell(const DevCode c, const IntRule r, H2S s, int k) {
  const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  int chunk, m0;
  if constexpr (FORM == 1) {
    if (!row_map<kChunksSV>(blockIdx.x, blockIdx.y, threadIdx.x >> 5, c.M, s.FP, chunk, m0)) return;
  } else {
    if (!row_map_all(warp, c.M, s.FP, chunk, m0)) return;
  }
  const int p = chunk * 32 + lane;
  const int cur = k & 1;
  if (__all_sync(0xffffffffu, s.act[cur * s.FP + p] == 0u)) return;
  const uint32_t qm2 = ints_to_h2(r.qm, r.qm);
  const H2Rule hr = make_h2rule(r);
  const StreamAddr<WIDE> ad{c.M, (uint32_t)s.FP, c.ell16, c.ell32};
  const uint32_t* Zs = s.z + p;
  int32_t* Acc = s.acc + p;
  uint4* St = C8 ? reinterpret_cast<uint4*>(reinterpret_cast<uint2*>(s.st) + p) : s.st + p;
  uint16_t* Lm = s.lm + p;
  uint32_t fail = 0;
  const int m1 = min(m0 + kRowsPerWarp, c.M);
  for (int m = m0; m < m1; ++m) {
    const int d = c.deg(m);
    if (FORM == 1 && m + 1 < m1) {
      // pull the next check's posterior lines and state into L1 while this
      // check waits on its own (the row pass is bound by memory latency;
      // measured -3.5 % on the N=64800 code; the per-edge form spills with it)
      const int dn = c.deg(m + 1);
      for (int j = 0; j < dn; ++j) {
        const uint32_t h = ad.at(nullptr, nullptr, j, m + 1);
        asm volatile("prefetch.global.L1 [%0];" ::"l"(Zs + h));
      }
      const void* sn = C8 ? static_cast<const void*>(reinterpret_cast<const uint2*>(St) + ad.st(m + 1))
                          : static_cast<const void*>(St + ad.st(m + 1));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(sn));
    }
    using A = StreamAddr<WIDE>;
    if constexpr (C8) {
      switch (d) {
        case 6: fail |= check_body<2, 1, 6, 8, ES, A, DELTA ? 1 : 0, true>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm); break;
        case 7: fail |= check_body<2, 1, 7, 8, ES, A, DELTA ? 1 : 0, true>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm); break;
        default: fail |= check_body<2, 1, 0, 8, ES, A, DELTA ? 1 : 0, true>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm); break;
      }
    } else if constexpr (FORM == 1) {
      switch (d) {
        case 6: fail |= check_body<2, FORM, 6, 16, ES, A, DELTA ? 1 : 0>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm); break;
        case 7: fail |= check_body<2, FORM, 7, 16, ES, A, DELTA ? 1 : 0>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm); break;
        case 14: fail |= check_body<2, FORM, 14, 16, ES, A, DELTA ? 1 : 0>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm); break;
        case 15: fail |= check_body<2, FORM, 15, 16, ES, A, DELTA ? 1 : 0>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm); break;
        default: fail |= check_body<2, FORM, 0, 16, ES, A, DELTA ? 1 : 0>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm); break;
      }
    } else {
      // (per-edge: more exact-degree bodies here cost the kernel spills)
      if (d == 6) fail |= check_body<2, FORM, 6, 16, ES, A, DELTA ? 1 : 0>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm);
      else if (d == 7) fail |= check_body<2, FORM, 7, 16, ES, A, DELTA ? 1 : 0>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm);
      else fail |= check_body<2, FORM, 0, 16, ES, A, DELTA ? 1 : 0>(ad, nullptr, Zs, Acc, hr, qm2, m, d, St, Lm);
    }
  }
  if (ES && fail) atomicOr(s.fail + cur * s.FP + p, fail);
}

// The column pass of the delta form with four frame pairs per thread: 16-byte
// accesses (a warp moves 512 bytes per variable), so that the pass streams at
// copy speed; the frames that continue take Z^(k), the others keep theirs.
// Pair-level flags are advanced by the threads of the first variable slice.
// The frame-pair count is a multiple of 32, so groups of 4 pairs never
// straddle it.
template <bool ES>
__global__ void __launch_bounds__(256) h2s_cols4(const DevCode c, H2S s, int k) {
  const int p0 = (blockIdx.y * 32 + (threadIdx.x & 31)) * 4;
  if (p0 >= s.FP) return;
  const int cur = k & 1, nxt = cur ^ 1;
  const uint4 act = *reinterpret_cast<const uint4*>(s.act + cur * s.FP + p0);
  uint4 fail = make_uint4(0u, 0u, 0u, 0u);
  if (ES) fail = *reinterpret_cast<const uint4*>(s.fail + cur * s.FP + p0);
  const uint4 stop = ES ? make_uint4(act.x & ~fail.x, act.y & ~fail.y, act.z & ~fail.z, act.w & ~fail.w)
                        : make_uint4(0u, 0u, 0u, 0u);
  const uint4 cont = make_uint4(act.x & ~stop.x, act.y & ~stop.y, act.z & ~stop.z, act.w & ~stop.w);
  auto selm = [](uint32_t cn) { return ((cn & 1u) ? 0x0000ffffu : 0u) | ((cn & 2u) ? 0xffff0000u : 0u); };
  const uint4 sel = make_uint4(selm(cont.x), selm(cont.y), selm(cont.z), selm(cont.w));
  const bool all = (sel.x & sel.y & sel.z & sel.w) == 0xffffffffu;
  const bool any = (cont.x | cont.y | cont.z | cont.w) != 0u;
  // the 8-bit posterior stores Z^(k) clamped (the accumulator stays exact)
  const uint32_t sat2 = ints_to_h2(s.psat, s.psat), nsat2 = ints_to_h2(-s.psat, -s.psat);
  const bool sat = s.psat > 0;
  auto conv = [sat, sat2, nsat2](uint32_t a) {
    const uint32_t zz = acc_to_pair((int32_t)a);
    const uint32_t h = ints_to_h2(lo16(zz), hi16(zz));
    return sat ? hmin(hmax(h, nsat2), sat2) : h;
  };
  if (any) {
#pragma unroll 4
    for (int n = blockIdx.x * 8 + (threadIdx.x >> 5); n < c.N; n += gridDim.x * 8) {
      const size_t o = (size_t)n * s.FP + p0;
      const uint4 a = *reinterpret_cast<const uint4*>(s.acc + o);
      uint4 h = make_uint4(conv(a.x), conv(a.y), conv(a.z), conv(a.w));
      if (!all) {
        const uint4 z = *reinterpret_cast<const uint4*>(s.z + o);
        h = make_uint4((h.x & sel.x) | (z.x & ~sel.x), (h.y & sel.y) | (z.y & ~sel.y),
                       (h.z & sel.z) | (z.z & ~sel.z), (h.w & sel.w) | (z.w & ~sel.w));
      }
      *reinterpret_cast<uint4*>(s.z + o) = h;
    }
  }
  if (blockIdx.x == 0) {
    *reinterpret_cast<uint4*>(s.act + nxt * s.FP + p0) = cont;
    *reinterpret_cast<uint4*>(s.fail + nxt * s.FP + p0) = make_uint4(0u, 0u, 0u, 0u);
    if (ES) {
      const uint32_t st[4] = {stop.x, stop.y, stop.z, stop.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (st[q] & 1u) s.iters[2 * (p0 + q)] = k - 1;
        if (st[q] & 2u) s.iters[2 * (p0 + q) + 1] = k - 1;
        s.ok[p0 + q] |= st[q];
      }
    }
  }
}

// The column pass of the CSR kernel's resetting form: stop rule, Z^(k) for the
// frames that continue, accumulator reset to Z0 for every (variable, pair);
// pair-level flags are advanced by the threads of variable 0.
template <bool ES>
__global__ void __launch_bounds__(256) h2s_cols(const DevCode c, H2S s, int k) {
  const int p = blockIdx.y * 32 + (threadIdx.x & 31);
  const int cur = k & 1, nxt = cur ^ 1;
  const uint32_t act = s.act[cur * s.FP + p];
  const uint32_t stop = ES ? (act & ~s.fail[cur * s.FP + p]) : 0u;
  const uint32_t cont = act & ~stop;
  const uint32_t sel = ((cont & 1u) ? 0x0000ffffu : 0u) | ((cont & 2u) ? 0xffff0000u : 0u);
  const uint32_t sat2 = ints_to_h2(s.psat, s.psat), nsat2 = ints_to_h2(-s.psat, -s.psat);
  for (int n = blockIdx.x * 8 + (threadIdx.x >> 5); n < c.N; n += gridDim.x * 8) {
    const size_t o = (size_t)n * s.FP + p;
    const uint32_t zz = acc_to_pair(s.acc[o]);
    uint32_t h = ints_to_h2(lo16(zz), hi16(zz));
    if (s.psat > 0) h = hmin(hmax(h, nsat2), sat2);  // the 8-bit posterior
    s.z[o] = (h & sel) | (s.z[o] & ~sel);
    const uint32_t q = s.q0[o];
    s.acc[o] = (int32_t)((uint32_t)acc_pack((int32_t)(int8_t)(q & 0xffu), (int32_t)(int8_t)(q >> 8)) -
                         (uint32_t)__ldg(c.cdeg + n) * 0x66006600u);
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    s.act[nxt * s.FP + p] = cont;
    s.fail[nxt * s.FP + p] = 0u;
    if (ES) {
      if (stop & 1u) s.iters[2 * p] = k - 1;
      if (stop & 2u) s.iters[2 * p + 1] = k - 1;
      s.ok[p] |= stop;
    }
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32) h2s_final_syndrome(const DevCode c, H2S s, int kf) {
  const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  int chunk, m0;
  if (!row_map_all(warp, c.M, s.FP, chunk, m0)) return;
  const int p = chunk * 32 + lane;
  const int cur = kf & 1;
  if (__all_sync(0xffffffffu, s.act[cur * s.FP + p] == 0u)) return;
  uint32_t fail = 0;
  const int m1 = min(m0 + kRowsPerWarp, c.M);
  for (int m = m0; m < m1; ++m) {
    uint32_t y = 0;
    for (int e = __ldg(c.rp + m); e < __ldg(c.rp + m + 1); ++e)
      y ^= dec_bits(s.z[(size_t)__ldg(c.ci + e) * s.FP + p]);
    fail |= ((y >> 15) & 1u) | ((y >> 30) & 2u);
  }
  if (fail) atomicOr(s.fail + cur * s.FP + p, fail);
}

// Frame-major outputs through a 64-variable x 32-pair tile.
__global__ void __launch_bounds__(256) h2s_output(const DevCode c, H2S s, int kf, int32_t F, uint8_t* bits,
                                                  int32_t* iters, uint8_t* okf, int16_t* zout) {
  __shared__ uint32_t tile[64][33];  // [variable][pair]
  const int n0 = blockIdx.x * 64, p0 = blockIdx.y * 32;
  const int N = c.N, N8 = (N + 7) >> 3;
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
    const int nl = i >> 5, pl = i & 31;
    const int n = n0 + nl;
    tile[nl][pl] = n < N ? s.z[(size_t)n * s.FP + p0 + pl] : 0u;
  }
  __syncthreads();
  // decisions: 8 bytes (64 variables) per frame
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
      const uint32_t h = tile[nl][fl >> 1];
      zout[(size_t)f * N + n] = (int16_t)((fl & 1) ? h_hi_int(h) : h_lo_int(h));
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 64) {
    const int f = 2 * p0 + threadIdx.x;
    if (f < F) {
      const int p = f >> 1, b = f & 1;
      const int cur = kf & 1;
      const uint32_t act = s.act[cur * s.FP + p];
      const uint32_t fail = s.fail[cur * s.FP + p];
      const bool running = (act >> b) & 1u;
      iters[f] = s.iters[f];
      okf[f] = running ? (uint8_t)(((fail >> b) & 1u) ^ 1u) : (uint8_t)((s.ok[p] >> b) & 1u);
    }
  }
}


// Per iteration: the degree-sorted row kernel with delta accumulation and the
// converting column kernel (delta == true), or the CSR row kernel with the
// resetting column kernel when 32-bit element offsets do not reach.  Measured
// on the N=64800 staircase code (1024 frames, 50 iterations), when delta
// accumulation came in: 17.4 / 20.9 ms (Section V / per-edge) against 20.2 /
// 22.3 ms for the best resetting kernels; 4 CTAs per SM beat 3 (19.1 / 21.3 ms)
// and 2.  With the 8-byte state, chunk-major rows and the four-pair column
// pass since: 14.4 / 18.7 ms.
template <int FORM, bool ES>
cudaError_t h2s_run(const DevCode& c, const IntRule& r, const StreamLayout& L, H2S s, int sm_count,
                    int32_t max_iter, bool delta, cudaStream_t st) {
  const int rgrid = rows_grid(c.M, L.lanes);
  // the degree-sorted kernel: Section V form on a 2-D grid (chunk groups),
  // per-edge form on the 1-D check-major grid
  const RowGrid g2 = rows_grid_g(c.M, L.lanes, kChunksSV);
  const dim3 egrid = FORM == 1 ? dim3((unsigned)g2.x, (unsigned)g2.y) : dim3((unsigned)rgrid);
  const dim3 cgrid((unsigned)std::max(1, std::min((c.N + 7) / 8, 4 * sm_count * 32 / std::max(1, L.lanes / 32))),
                   L.lanes / 32);
  const int gy4 = (L.lanes / 4 + 31) / 32;  // groups of 32 threads x 4 pairs
  const dim3 cgrid4((unsigned)std::max(1, std::min((c.N + 7) / 8, 4 * sm_count * 32 / gy4)), (unsigned)gy4);
  const bool wide = c.ell16 == nullptr;
  const bool c8 = c.ell_w <= 8;  // every check of degree <= 8: the 8-byte Section V state
  for (int k = 1; k <= max_iter; ++k) {
    if (delta) {
      if (FORM == 1 && c8) {
        if (wide) h2s_rows_ell<1, ES, true, 4, true, true><<<egrid, kWarpsPerBlock * 32, 0, st>>>(c, r, s, k);
        else h2s_rows_ell<1, ES, false, 4, true, true><<<egrid, kWarpsPerBlock * 32, 0, st>>>(c, r, s, k);
      } else if (wide) h2s_rows_ell<FORM, ES, true, 4, true><<<egrid, kWarpsPerBlock * 32, 0, st>>>(c, r, s, k);
      else h2s_rows_ell<FORM, ES, false, 4, true><<<egrid, kWarpsPerBlock * 32, 0, st>>>(c, r, s, k);
      h2s_cols4<ES><<<cgrid4, 256, 0, st>>>(c, s, k);
    } else {
      h2s_rows<FORM, ES><<<rgrid, kWarpsPerBlock * 32, 0, st>>>(c, r, s, k);
      h2s_cols<ES><<<cgrid, 256, 0, st>>>(c, s, k);
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t stream_int8_decode(const DevCode& c, const IntRule& r, int form, const StreamLayout& L, void* ws,
                               int sm_count, const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop,
                               uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st) {
  H2S s = h2s_view(ws, L);
  s.psat = r.psat;
  const dim3 tgrid((c.N + 63) / 64, L.lanes / 32);
  // L^(0) = 0: Section V state all zero, per-edge bytes L + 128 = 0x80
  cudaError_t e0 = cudaMemsetAsync(static_cast<char*>(ws) + L.st, form == 1 ? 0 : 0x80, L.q0 - L.st, st);
  if (e0 != cudaSuccess) return e0;
  // the degree-sorted kernels address the state with 32-bit element offsets
  const uint64_t span = std::max((uint64_t)c.N, (uint64_t)c.ell_w * (uint64_t)c.M) * (uint64_t)L.lanes;
  const bool delta = span < (1ull << 32);
  h2s_init<<<tgrid, 256, 0, st>>>(c, llr, F, max_iter, s, delta ? 1 : 0);
  cudaError_t e;
  const bool es = early_stop != 0;
  if (form == 1) e = es ? h2s_run<1, true>(c, r, L, s, sm_count, max_iter, delta, st)
                        : h2s_run<1, false>(c, r, L, s, sm_count, max_iter, delta, st);
  else e = es ? h2s_run<0, true>(c, r, L, s, sm_count, max_iter, delta, st)
              : h2s_run<0, false>(c, r, L, s, sm_count, max_iter, delta, st);
  if (e != cudaSuccess) return e;
  const int kf = max_iter + 1;
  h2s_final_syndrome<<<rows_grid(c.M, L.lanes), kWarpsPerBlock * 32, 0, st>>>(c, s, kf);
  h2s_output<<<tgrid, 256, 0, st>>>(c, s, kf, F, bits, iters, ok, zout);
  return cudaGetLastError();
}

}  // namespace ldpc
