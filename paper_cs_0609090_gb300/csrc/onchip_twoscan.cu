// onchip_twoscan.cu -- the original two-scan min-sum (Section III, Eqs. (1) and
// (2)) as a frame-resident comparator for the single-scan kernels.
//
// Same conventions as onchip_h2.cu (exact binary16 pairs, two frames per
// instruction, G frames per CTA, all iterations on chip).  Per edge there is one
// shared-memory cell that holds Z_mn before the horizontal scan and L_mn after
// it, as Section V describes for the original algorithm ("one memory cell to
// store both").  Unlike the single scan, the vertical scan needs the
// variable->check addressing M(n): for each variable the list of its edge cells.
//
// Shared memory per CTA (P = G/2 pairs):
//   Cell [ell_w * M][P] half2   edge cells, edge-slot-major (slot j * M + m)
//   Zp   [N][P]         half2   posterior Z_n (decisions, syndrome, outputs)
//
// Iteration k:
//   horizontal scan (thread per check): Eq. (1) on the cells' Z_mn (|Z_mn|
//     saturated to Qm), offset/normalization, L_mn written back into the cells;
//     with early stop, also the decision parity of x^(k-1) from Zp
//   vertical scan (thread per variable): S = Z0_n + sum over M(n) of L_mn; the
//     posterior Z_n = S (Section III decoding step); then each cell becomes
//     Z_mn = S - L_mn, which is Eq. (2)'s Z0_n + sum over M(n)\m of L_m'n.
#include <algorithm>

#include "h2ops.cuh"
#include "kernels.h"
#include "launch_util.h"
#include "pp_check.cuh"

namespace ldpc {
namespace {

constexpr int kTsThreads = 1024;

__host__ __device__ constexpr size_t ts_a16(size_t x) { return (x + 15) & ~size_t(15); }

struct TsLayout {
  size_t cell, zp, total;
};
__host__ __device__ inline TsLayout ts_layout(int N, int slots, int G) {
  const size_t P = (size_t)G / 2;
  TsLayout L;
  L.cell = 0;
  L.zp = ts_a16((size_t)slots * P * 4);
  L.total = L.zp + ts_a16((size_t)N * P * 4);
  return L;
}

template <int G>
__device__ __forceinline__ void ts_ld(const uint32_t* __restrict__ a, size_t i, uint32_t (&w)[G / 2]) {
  if constexpr (G == 2) {
    w[0] = a[i];
  } else {
    const uint2 v = reinterpret_cast<const uint2*>(a)[i];
    w[0] = v.x;
    w[1] = v.y;
  }
}
template <int G>
__device__ __forceinline__ void ts_st(uint32_t* __restrict__ a, size_t i, const uint32_t (&w)[G / 2]) {
  if constexpr (G == 2) a[i] = w[0];
  else reinterpret_cast<uint2*>(a)[i] = make_uint2(w[0], w[1]);
}

__device__ __forceinline__ int32_t ts_q0(const int8_t* __restrict__ llr, int32_t N, int32_t f, int32_t F, int n) {
  return f < F ? (int32_t)__ldg(llr + (size_t)f * N + n) : 0;
}

// Horizontal scan of check m, Eq. (1), for the G frames: the min-search key
// (16 |Z_mn| + j) 2^-11 of one saturating multiply-add per position, with the
// minima started at the key of Qm (so that they decode to 16 min(|Z_mn|, Qm) +
// j), the rule and the signs as in the single-scan kernels (key_step,
// finish_state), L_mn written back into the cells.  Returns the decision
// parity bits of x^(k-1) (from Zp) when ES.
template <int G, int DMAX, bool ES>
__device__ __forceinline__ uint32_t ts_horizontal(const DevCode& c, const H2Rule& rule, uint32_t ksat, int m,
                                                  uint32_t* __restrict__ Cell, const uint32_t* __restrict__ Zp) {
  constexpr int P = G / 2;
  const int M = c.M;
  const int d = c.deg(m);
  uint32_t K1[P], K2[P], NEG[P], Y[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    K1[p] = ksat;
    K2[p] = ksat;
    NEG[p] = 0;
    Y[p] = 0;
  }
#pragma unroll
  for (int j = 0; j < DMAX; ++j) {
    if (j < d) {
      uint32_t z[P];
      ts_ld<G>(Cell, (size_t)j * M + m, z);
      if constexpr (ES) {
        uint32_t w[P];
        ts_ld<G>(Zp, (size_t)__ldg(c.ell16 + (size_t)j * M + m), w);
#pragma unroll
        for (int p = 0; p < P; ++p) Y[p] ^= dec_bits(w[p]);
      }
#pragma unroll
      for (int p = 0; p < P; ++p) key_step(z[p], j, K1[p], K2[p], NEG[p]);
    }
  }
  uint32_t par = 0;
  uint32_t An[P], Dn[P], In[P], SN[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const NewState n = finish_state(K1[p], K2[p], NEG[p], d, rule);
    An[p] = n.An;
    Dn[p] = hsub(n.Bn, n.An);
    In[p] = n.In;
    SN[p] = n.Sn;
    if constexpr (ES) par |= ((Y[p] >> 15) & 1u) << (2 * p) | ((Y[p] >> 31) & 1u) << (2 * p + 1);
  }
#pragma unroll
  for (int j = 0; j < DMAX; ++j) {
    if (j < d) {
      uint32_t l[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        // f(A, B, n, n~) = A + (B - A) [j = n~], the sign on the binary16 sign bit
        l[p] = hfma(Dn[p], heq_one(In[p], h2c(j)), An[p]) ^ (SN[p] & 0x80008000u);
        SN[p] += SN[p];
      }
      ts_st<G>(Cell, (size_t)j * M + m, l);
    }
  }
  return par;
}

template <int G, int DMAX>
__device__ __forceinline__ uint32_t ts_row_parity(const DevCode& c, const uint32_t* __restrict__ Zp, int m) {
  constexpr int P = G / 2;
  const int d = c.deg(m);
  uint32_t y[P];
#pragma unroll
  for (int p = 0; p < P; ++p) y[p] = 0;
#pragma unroll
  for (int j = 0; j < DMAX; ++j) {
    if (j < d) {
      uint32_t w[P];
      ts_ld<G>(Zp, (size_t)__ldg(c.ell16 + (size_t)j * c.M + m), w);
#pragma unroll
      for (int p = 0; p < P; ++p) y[p] ^= dec_bits(w[p]);
    }
  }
  uint32_t par = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) par |= ((y[p] >> 15) & 1u) << (2 * p) | ((y[p] >> 31) & 1u) << (2 * p + 1);
  return par;
}

template <int G, int DMAX, bool ES>
__global__ void __launch_bounds__(kTsThreads, 1)
onchip_twoscan_kernel(const DevCode c, const IntRule r, const int8_t* __restrict__ llr, int32_t F, int32_t max_iter,
                      uint8_t* __restrict__ bits, int32_t* __restrict__ iters, uint8_t* __restrict__ okf,
                      int16_t* __restrict__ zout, int32_t n_groups) {
  constexpr int P = G / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = c.N, M = c.M;
  const int slots = c.ell_w * M;
  const TsLayout Ly = ts_layout(N, slots, G);
  uint32_t* Cell = reinterpret_cast<uint32_t*>(smem + Ly.cell);
  uint32_t* Zp = reinterpret_cast<uint32_t*>(smem + Ly.zp);
  __shared__ uint32_t s_fail[3];
  __shared__ int32_t s_iters[G];
  __shared__ uint32_t s_ok;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int N8 = (N + 7) >> 3;
  const uint32_t qm2 = ints_to_h2(r.qm, r.qm);
  const H2Rule hr = make_h2rule(r);
  // (16 Qm + 15) 2^-11: the largest key of a magnitude saturated to Qm
  const uint32_t ksat = hfma(qm2, h2c_q11(16), h2c_q11(15));

  for (int grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const int f0 = grp * G;
    const int nvalid = min(G, F - f0);
    uint32_t act = (1u << nvalid) - 1u;

    // Section III initialization: Z^(0)_mn = Z^(0)_n in every cell, Z_n = Z0_n
    for (int n = tid; n < N; n += nt) {
      uint32_t w[P];
#pragma unroll
      for (int p = 0; p < P; ++p)
        w[p] = ints_to_h2(ts_q0(llr, N, f0 + 2 * p, F, n), ts_q0(llr, N, f0 + 2 * p + 1, F, n));
      ts_st<G>(Zp, n, w);
    }
    if (tid < 3) s_fail[tid] = 0;
    if (tid < G) s_iters[tid] = max_iter;
    if (tid == 0) s_ok = 0;
    __syncthreads();
    for (int i = tid; i < slots; i += nt) {
      uint32_t w[P];
      ts_ld<G>(Zp, (size_t)__ldg(c.ell16 + i), w);
      ts_st<G>(Cell, i, w);
    }
    __syncthreads();

    for (int k = 1; k <= max_iter && act != 0u; ++k) {
      const int kp = k & 1;
      uint32_t fail = 0;
      for (int m = tid; m < M; m += nt) fail |= ts_horizontal<G, DMAX, ES>(c, hr, ksat, m, Cell, Zp);
      if constexpr (ES) {
        fail = __reduce_or_sync(0xffffffffu, fail);
        if ((tid & 31) == 0 && (fail & act)) atomicOr(&s_fail[kp], fail & act);
      }
      __syncthreads();
      const uint32_t stop = ES ? (act & ~s_fail[kp]) : 0u;
      const uint32_t cont = act & ~stop;
      constexpr int kTsDv = G == 2 ? 16 : 8;  // column degrees the vertical scan unrolls
      for (int n = tid; n < N; n += nt) {
        const int a0 = __ldg(c.cptr + n), a1 = __ldg(c.cptr + n + 1);
        uint32_t S[P];
#pragma unroll
        for (int p = 0; p < P; ++p)
          S[p] = ints_to_h2(ts_q0(llr, N, f0 + 2 * p, F, n), ts_q0(llr, N, f0 + 2 * p + 1, F, n));
        if (a1 - a0 <= kTsDv) {
          // unrolled over the column degree: the slot indices of all the
          // variable's edges are loaded together, then their cells, instead of
          // one index -> cell chain per edge
          const int dv = a1 - a0;
          uint32_t sl[kTsDv], lv[kTsDv][P];
#pragma unroll
          for (int a = 0; a < kTsDv; ++a)
            if (a < dv) sl[a] = (uint32_t)__ldg(c.cslot + a0 + a);
#pragma unroll
          for (int a = 0; a < kTsDv; ++a) {
            if (a < dv) {
              ts_ld<G>(Cell, sl[a], lv[a]);
#pragma unroll
              for (int p = 0; p < P; ++p) S[p] = hadd(S[p], lv[a][p]);
            }
          }
#pragma unroll
          for (int a = 0; a < kTsDv; ++a) {
            if (a < dv) {
              uint32_t l[P];
#pragma unroll
              for (int p = 0; p < P; ++p) l[p] = hsub(S[p], lv[a][p]);
              ts_st<G>(Cell, sl[a], l);
            }
          }
        } else {
          for (int a = a0; a < a1; ++a) {
            uint32_t l[P];
            ts_ld<G>(Cell, (size_t)__ldg(c.cslot + a), l);
#pragma unroll
            for (int p = 0; p < P; ++p) S[p] = hadd(S[p], l[p]);
          }
          for (int a = a0; a < a1; ++a) {
            const size_t sl = (size_t)__ldg(c.cslot + a);
            uint32_t l[P];
            ts_ld<G>(Cell, sl, l);
#pragma unroll
            for (int p = 0; p < P; ++p) l[p] = hsub(S[p], l[p]);
            ts_st<G>(Cell, sl, l);
          }
        }
        uint32_t w[P];
        ts_ld<G>(Zp, n, w);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const uint32_t sel = (((cont >> (2 * p)) & 1u) ? 0x0000ffffu : 0u) |
                               (((cont >> (2 * p + 1)) & 1u) ? 0xffff0000u : 0u);
          w[p] = (S[p] & sel) | (w[p] & ~sel);
        }
        ts_st<G>(Zp, n, w);
      }
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
      for (int m = tid; m < M; m += nt) fail |= ts_row_parity<G, DMAX>(c, Zp, m);
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
        if (n < N) byte |= ((dec_bits(Zp[(size_t)n * P + g / 2] >> (16 * (g & 1))) >> 15) & 1u) << t;
      }
      bits[(size_t)(f0 + g) * N8 + b] = (uint8_t)byte;
    }
    if (zout != nullptr) {
      for (int i = tid; i < nvalid * N; i += nt) {
        const int g = i / N, n = i - g * N;
        const uint32_t h = Zp[(size_t)n * P + g / 2];
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

template <int G, int DMAX, bool ES>
cudaError_t ts_launch_t(const DevCode& c, const IntRule& r, OnchipPlan& plan, int sm_count, const int8_t* llr,
                        int32_t F, int32_t max_iter, uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout,
                        cudaStream_t stream) {
  auto kern = onchip_twoscan_kernel<G, DMAX, ES>;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(kern), plan.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, plan.threads, plan.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t cap = (int64_t)sm_count * per_sm;
  plan.grid = (int)((int64_t)plan.n_groups < cap ? plan.n_groups : cap);
  kern<<<plan.grid, plan.threads, plan.smem, stream>>>(c, r, llr, F, max_iter, bits, iters, ok, zout, plan.n_groups);
  return cudaGetLastError();
}

}  // namespace

bool onchip_twoscan_plan(const DevCode& c, int32_t n_frames, int sm_count, size_t smem_optin, int max_row_deg,
                         OnchipPlan* plan) {
  const size_t static_smem = 64;
  int G = 0;
  for (int g : {4, 2})
    if (ts_layout(c.N, c.ell_w * c.M, g).total + static_smem <= smem_optin) { G = g; break; }
  if (G == 0) return false;
  while (G > 2 && (int64_t)n_frames < (int64_t)sm_count * G) G /= 2;
  plan->G = G;
  plan->dmax = max_row_deg <= 8 ? 8 : 16;
  plan->smem = ts_layout(c.N, c.ell_w * c.M, G).total;
  int threads = ((std::max(c.M, c.N) + 31) / 32) * 32;
  plan->threads = threads > kTsThreads ? kTsThreads : (threads < 128 ? 128 : threads);
  plan->n_groups = (n_frames + G - 1) / G;
  plan->grid = 0;
  return true;
}

cudaError_t onchip_twoscan_launch(const DevCode& c, const IntRule& r, OnchipPlan& plan, int sm_count,
                                  const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop, uint8_t* bits,
                                  int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t stream) {
  const bool es = early_stop != 0;
#define LDPC_TS_CASE(GG, DD)                                                                                   \
  if (plan.G == GG && plan.dmax == DD)                                                                        \
    return es ? ts_launch_t<GG, DD, true>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream) \
              : ts_launch_t<GG, DD, false>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream);
  LDPC_TS_CASE(4, 16)
  LDPC_TS_CASE(2, 16)
  LDPC_TS_CASE(4, 8)
  LDPC_TS_CASE(2, 8)
#undef LDPC_TS_CASE
  return cudaErrorInvalidValue;
}

}  // namespace ldpc
