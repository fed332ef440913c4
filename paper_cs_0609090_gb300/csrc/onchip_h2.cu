// onchip_h2.cu -- frame-resident single-scan min-sum, int8 path, two frames per
// instruction.
//
// Same algorithm and results as onchip_int8.cu (Section IV Eq. (3) and the
// Section V state), restricted to codes where every quantity is an integer of
// magnitude < 2048: then IEEE binary16 represents all of them exactly and every
// f16x2 add, multiply-add, min and max below is exact, so the results are
// bit-identical to integer arithmetic.  Conditions (checked by the host):
//   128 + max_col_degree * Qm + Qm <= 2048   (|Z - L| bound)
//   max row degree <= 16                     (key = min(|u|, Qm) * 16 + j <= 2047)
//   N <= 65535                               (16-bit column indices)
//
// Shared memory per CTA (P = G/2 frame pairs):
//   Zs   [N][P]  half2  posterior Z^(k-1)
//   Acc  [N][P]  i32    Z^(k) as the integer lo + 65536 hi; every message adds the
//                       bit pattern of (L + 1536) per lane, i.e. 0x6600 + L, and
//                       the resets subtract col_degree(n) * 0x66006600
//   form 1 (Section V): [M][P] {A, B, n~ as half2; signs, bit-reversed: the
//                       sign of position j of the even frame at bit 15 - j, of
//                       the odd frame at bit 31 - j, so that shifting the word
//                       left by j (a running S + S) brings both to the binary16
//                       sign bits}
//   form 0 (Section IV): [E][P] u16: L + 128 per frame (one byte each)
#include <cuda_fp16.h>

#include <type_traits>

#include "h2_body.cuh"
#include "kernels.h"
#include "launch_util.h"

namespace ldpc {
namespace {

constexpr int kThreadsMax = 1024;

__host__ __device__ constexpr size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

struct H2Layout {
  size_t zs, acc, st, idx, rs, total;
};
// E here is the number of edge slots, ell_w * M.  With sidx the edge-slot-major
// column table (uint16) is copied into shared memory once per CTA; with rset
// the accumulator's reset value (Z0 minus the message bias) is kept per
// variable and frame pair for the frame group.
__host__ __device__ inline H2Layout h2_layout(int N, int M, int E, int G, int form, bool sidx, bool rset = false) {
  const size_t P = (size_t)G / 2;
  H2Layout L;
  L.zs = 0;
  L.acc = a16((size_t)N * P * 4);
  L.st = L.acc + a16((size_t)N * P * 4);
  L.idx = L.st + a16(form == 1 ? (size_t)M * P * 16 : (size_t)E * P * 2);
  L.rs = L.idx + (sidx ? a16((size_t)E * 2) : 0);
  L.total = L.rs + (rset ? a16((size_t)N * P * 4) : 0);
  return L;
}

// Degrees with a fully unrolled body; other degrees take the guarded loop.
template <int DMAX>
struct Fast {
  static constexpr int a = DMAX <= 8 ? 6 : 14;
  static constexpr int b = DMAX <= 8 ? 7 : 15;
};

template <int G, int FORM, int DMAX, bool ES, class Addr>
__device__ __forceinline__ uint32_t check_update_h2(const Addr& ad, const uint16_t* __restrict__ tab,
                                                    const uint32_t* __restrict__ Zs, int32_t* __restrict__ Acc,
                                                    const uint8_t* __restrict__ rdeg, const H2Rule& r,
                                                    uint32_t qm2, int m, uint4* __restrict__ St,
                                                    uint16_t* __restrict__ Lm) {
  // (a load of the degree byte measured faster here than deriving it from the
  // degree runs, which the streaming kernels use)
  const int d = (int)__ldg(rdeg + m);
  if (d == Fast<DMAX>::a)
    return check_body<G, FORM, Fast<DMAX>::a, DMAX, ES>(ad, tab, Zs, Acc, r, qm2, m, d, St, Lm);
  if (d == Fast<DMAX>::b)
    return check_body<G, FORM, Fast<DMAX>::b, DMAX, ES>(ad, tab, Zs, Acc, r, qm2, m, d, St, Lm);
  return check_body<G, FORM, 0, DMAX, ES>(ad, tab, Zs, Acc, r, qm2, m, d, St, Lm);
}

__device__ __forceinline__ int32_t q0v(const int8_t* __restrict__ llr, int32_t N, int32_t f, int32_t F, int n) {
  return f < F ? (int32_t)__ldg(llr + (size_t)f * N + n) : 0;
}

template <int G, int FORM, int DMAX, bool ES, bool SIDX, bool RSET>
__global__ void __launch_bounds__(kThreadsMax, 1)
onchip_h2_kernel(const DevCode c, const IntRule r, const int8_t* __restrict__ llr, int32_t F, int32_t max_iter,
                 uint8_t* __restrict__ bits, int32_t* __restrict__ iters, uint8_t* __restrict__ okf,
                 int16_t* __restrict__ zout, int32_t n_groups) {
  constexpr int P = G / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = c.N, M = c.M;
  const H2Layout Ly = h2_layout(N, M, c.ell_w * M, G, FORM, SIDX, RSET);
  int32_t* Rs = reinterpret_cast<int32_t*>(smem + Ly.rs);
  uint32_t* Zs = reinterpret_cast<uint32_t*>(smem + Ly.zs);
  int32_t* Acc = reinterpret_cast<int32_t*>(smem + Ly.acc);
  uint4* St = reinterpret_cast<uint4*>(smem + Ly.st);
  uint16_t* Lm = reinterpret_cast<uint16_t*>(smem + Ly.st);
  uint16_t* sidx = reinterpret_cast<uint16_t*>(smem + Ly.idx);
  __shared__ uint32_t s_fail[3];
  __shared__ int32_t s_iters[G];
  __shared__ uint32_t s_ok;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int N8 = (N + 7) >> 3;
  const uint32_t qm2 = ints_to_h2(r.qm, r.qm);
  const H2Rule hr = make_h2rule(r);
  const LocalAddr<G, SIDX> ad{c.M};
  if constexpr (SIDX) {
    // the column table is the same for every frame group: copy it once
    const int words = (c.ell_w * M) >> 1;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(c.ell16);
    for (int i = tid; i < words; i += nt) reinterpret_cast<uint32_t*>(sidx)[i] = __ldg(src + i);
    if ((c.ell_w * M) & 1) {
      if (tid == 0) sidx[c.ell_w * M - 1] = __ldg(c.ell16 + c.ell_w * M - 1);
    }
  }

  for (int grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const int f0 = grp * G;
    const int nvalid = min(G, F - f0);
    uint32_t act = (1u << nvalid) - 1u;

    for (int n = tid; n < N; n += nt) {
      const uint32_t bias = (uint32_t)__ldg(c.cdeg + n) * 0x66006600u;
      uint32_t w[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int32_t lo = q0v(llr, N, f0 + 2 * p, F, n), hi = q0v(llr, N, f0 + 2 * p + 1, F, n);
        w[p] = ints_to_h2(lo, hi);
        const int32_t reset = (int32_t)((uint32_t)acc_pack(lo, hi) - bias);
        Acc[(size_t)n * P + p] = reset;
        if constexpr (RSET) Rs[(size_t)n * P + p] = reset;
      }
      st_pairs<G>(Zs, n, w);
    }
    if constexpr (FORM == 1) {
      for (int i = tid; i < M * P; i += nt) St[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
      // L^(0) = 0 is the byte 128 in every frame
      for (int i = tid; i < c.ell_w * M * P; i += nt) Lm[i] = 0x8080u;
    }
    if (tid < 3) s_fail[tid] = 0;
    if (tid < G) s_iters[tid] = max_iter;
    if (tid == 0) s_ok = 0;
    __syncthreads();

    for (int k = 1; k <= max_iter && act != 0u; ++k) {
      const int kp = k & 1;
      uint32_t fail = 0;
      for (int m = tid; m < M; m += nt)
        fail |= check_update_h2<G, FORM, DMAX, ES>(ad, SIDX ? sidx : c.ell16, Zs, Acc, c.rdeg, hr, qm2, m, St, Lm);
      if constexpr (ES) {
        fail = __reduce_or_sync(0xffffffffu, fail);
        if ((tid & 31) == 0 && (fail & act)) atomicOr(&s_fail[kp], fail & act);
      }
      __syncthreads();
      const uint32_t stop = ES ? (act & ~s_fail[kp]) : 0u;
      const uint32_t cont = act & ~stop;
      // without early stop every valid frame continues; the lanes of a missing
      // frame (an odd batch) hold values nobody reads
      const bool all = !ES || cont == (1u << G) - 1u;
      // the 8-bit posterior (r.psat > 0) stores Z^(k) clamped; the choice is
      // made once per pass, so the exact decode runs the pass without it
      const auto col_pass = [&](auto clamp) {
        for (int n = tid; n < N; n += nt) {
          uint32_t w[P];
          if (!all) ld_pairs<G>(Zs, n, w);
#pragma unroll
          for (int p = 0; p < P; ++p) {
            const uint32_t zz = acc_to_pair(Acc[(size_t)n * P + p]);
            uint32_t h = ints_to_h2(lo16(zz), hi16(zz));
            if constexpr (decltype(clamp)::value)
              h = hmin(hmax(h, ints_to_h2(-r.psat, -r.psat)), ints_to_h2(r.psat, r.psat));
            if (all) {
              w[p] = h;
            } else {
              const uint32_t sel = (((cont >> (2 * p)) & 1u) ? 0x0000ffffu : 0u) |
                                   (((cont >> (2 * p + 1)) & 1u) ? 0xffff0000u : 0u);
              w[p] = (h & sel) | (w[p] & ~sel);
            }
            if constexpr (RSET) {
              Acc[(size_t)n * P + p] = Rs[(size_t)n * P + p];
            } else {
              const uint32_t bias = (uint32_t)__ldg(c.cdeg + n) * 0x66006600u;
              const int32_t lo = q0v(llr, N, f0 + 2 * p, F, n), hi = q0v(llr, N, f0 + 2 * p + 1, F, n);
              Acc[(size_t)n * P + p] = (int32_t)((uint32_t)acc_pack(lo, hi) - bias);
            }
          }
          st_pairs<G>(Zs, n, w);
        }
      };
      if (r.psat > 0) col_pass(std::true_type{});
      else col_pass(std::false_type{});
      if (ES) {
        if (tid < G && ((stop >> tid) & 1u)) s_iters[tid] = k - 1;
        if (tid == 0) s_ok |= stop;
      }
      __syncthreads();
      if (tid == 0) s_fail[kp] = 0;
      act = cont;
    }

    if (act != 0u) {
      uint32_t fail = 0;
      for (int m = tid; m < M; m += nt) fail |= row_parity_body<G, 0, DMAX>(ad, SIDX ? sidx : c.ell16, Zs, m, (int)__ldg(c.rdeg + m));
      fail = __reduce_or_sync(0xffffffffu, fail);
      if ((tid & 31) == 0 && (fail & act)) atomicOr(&s_fail[2], fail & act);
      __syncthreads();
      if (tid == 0) s_ok |= act & ~s_fail[2];
    }
    __syncthreads();

    for (int i = tid; i < nvalid * N8; i += nt) {
      const int g = i / N8, b = i - g * N8;
      uint32_t byte = 0;
      for (int t = 0; t < 8; ++t) {
        const int n = b * 8 + t;
        if (n < N) {
          const uint32_t h = Zs[(size_t)n * P + g / 2] >> (16 * (g & 1));
          byte |= ((dec_bits(h) >> 15) & 1u) << t;
        }
      }
      bits[(size_t)(f0 + g) * N8 + b] = (uint8_t)byte;
    }
    if (zout != nullptr) {
      for (int i = tid; i < nvalid * N; i += nt) {
        const int g = i / N, n = i - g * N;
        const uint32_t h = Zs[(size_t)n * P + g / 2];
        zout[(size_t)(f0 + g) * N + n] = (int16_t)((g & 1) ? h_hi_int(h) : h_lo_int(h));
      }
    }
    if (tid < nvalid) {
      iters[f0 + tid] = s_iters[tid];
      okf[f0 + tid] = (uint8_t)((s_ok >> tid) & 1u);
    }
    __syncthreads();
  }
}

template <int G, int FORM, int DMAX, bool ES, bool SIDX, bool RSET>
cudaError_t h2_launch_t(const DevCode& c, const IntRule& r, OnchipPlan& plan, int sm_count, const int8_t* llr,
                        int32_t F, int32_t max_iter, uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout,
                        cudaStream_t stream, bool occupancy_only) {
  auto kern = onchip_h2_kernel<G, FORM, DMAX, ES, SIDX, RSET>;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(kern), plan.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, plan.threads, plan.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t cap = (int64_t)sm_count * per_sm;
  plan.grid = (int)((int64_t)plan.n_groups < cap ? plan.n_groups : cap);
  if (occupancy_only) return cudaSuccess;
  kern<<<plan.grid, plan.threads, plan.smem, stream>>>(c, r, llr, F, max_iter, bits, iters, ok, zout, plan.n_groups);
  return cudaGetLastError();
}

template <int G, int FORM, int DMAX>
cudaError_t h2_dispatch_es(bool es, const DevCode& c, const IntRule& r, OnchipPlan& plan, int sm_count,
                           const int8_t* llr, int32_t F, int32_t max_iter, uint8_t* bits, int32_t* iters,
                           uint8_t* ok, int16_t* zout, cudaStream_t stream, bool occ) {
  if (plan.sidx && plan.rset)
    return es ? h2_launch_t<G, FORM, DMAX, true, true, true>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ)
              : h2_launch_t<G, FORM, DMAX, false, true, true>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ);
  if (plan.sidx)
    return es ? h2_launch_t<G, FORM, DMAX, true, true, false>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ)
              : h2_launch_t<G, FORM, DMAX, false, true, false>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ);
  if (plan.rset)
    return es ? h2_launch_t<G, FORM, DMAX, true, false, true>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ)
              : h2_launch_t<G, FORM, DMAX, false, false, true>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ);
  return es ? h2_launch_t<G, FORM, DMAX, true, false, false>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ)
            : h2_launch_t<G, FORM, DMAX, false, false, false>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ);
}

}  // namespace

bool onchip_h2_eligible(int n_vars, int max_row_deg, int max_col_deg, int qm, int rule, int num) {
  (void)rule;
  (void)num;
  return n_vars <= 65535 && max_row_deg <= 16 && 128 + (int64_t)max_col_deg * qm + qm <= 2048;
}

bool onchip_h2_plan(const DevCode& c, int form, int32_t n_frames, int sm_count, size_t smem_optin,
                    int max_row_deg, OnchipPlan* plan) {
  const size_t static_smem = 64;
  auto fits = [&](int g, bool si) {
    return h2_layout(c.N, c.M, c.ell_w * c.M, g, form, si).total + static_smem <= smem_optin;
  };
  // The column table in shared memory removes the L2 round trips of the index
  // loads; it is preferred over a larger frame group.
  // Two frame pairs per thread only for checks of degree <= 8 (registers).
  const int gmax = max_row_deg <= 8 ? 4 : 2;
  int G = 0;
  bool sidx = false;
  for (int g = gmax; g >= 2; g /= 2)
    if (fits(g, true)) { G = g; sidx = true; break; }
  if (G == 0)
    for (int g = gmax; g >= 2; g /= 2)
      if (fits(g, false)) { G = g; break; }
  if (G == 0) return false;
  while (G > 2 && (int64_t)n_frames < (int64_t)sm_count * G) G /= 2;
  // the accumulator reset values in shared memory too, when they fit
  const bool rset = h2_layout(c.N, c.M, c.ell_w * c.M, G, form, sidx, true).total + static_smem <= smem_optin;
  plan->G = G;
  plan->sidx = sidx;
  plan->rset = rset;
  plan->dmax = max_row_deg <= 8 ? 8 : 16;
  plan->smem = h2_layout(c.N, c.M, c.ell_w * c.M, G, form, sidx, rset).total;
  int threads = ((c.M + 31) / 32) * 32;
  threads = threads > kThreadsMax ? kThreadsMax : (threads < 128 ? 128 : threads);
  plan->threads = threads;
  plan->n_groups = (n_frames + G - 1) / G;
  plan->grid = 0;
  return true;
}

cudaError_t onchip_h2_launch(const DevCode& c, const IntRule& r, int form, OnchipPlan& plan, int sm_count,
                             const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop, uint8_t* bits,
                             int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t stream, bool occupancy_only) {
  const bool es = early_stop != 0;
#define LDPC_H2_CASE(GG, FF, DD)                                                                             \
  if (plan.G == GG && form == FF && plan.dmax == DD)                                                        \
    return h2_dispatch_es<GG, FF, DD>(es, c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, \
                                      occupancy_only);
  LDPC_H2_CASE(2, 1, 16)
  LDPC_H2_CASE(4, 1, 8)
  LDPC_H2_CASE(2, 1, 8)
  LDPC_H2_CASE(2, 0, 16)
  LDPC_H2_CASE(4, 0, 8)
  LDPC_H2_CASE(2, 0, 8)
#undef LDPC_H2_CASE
  return cudaErrorInvalidValue;
}

}  // namespace ldpc
