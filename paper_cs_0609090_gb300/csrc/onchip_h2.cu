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

#include "h2ops.cuh"
#include "kernels.h"

namespace ldpc {
namespace {

constexpr int kThreadsMax = 1024;

__host__ __device__ constexpr size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

struct H2Layout {
  size_t zs, acc, st, idx, total;
};
// E here is the number of edge slots, ell_w * M.  With sidx the edge-slot-major
// column table (uint16) is copied into shared memory once per CTA.
__host__ __device__ inline H2Layout h2_layout(int N, int M, int E, int G, int form, bool sidx) {
  const size_t P = (size_t)G / 2;
  H2Layout L;
  L.zs = 0;
  L.acc = a16((size_t)N * P * 4);
  L.st = L.acc + a16((size_t)N * P * 4);
  L.idx = L.st + a16(form == 1 ? (size_t)M * P * 16 : (size_t)E * P * 2);
  L.total = L.idx + (sidx ? a16((size_t)E * 2) : 0);
  return L;
}

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

// Column of position j of check m: from the shared-memory copy or from global.
// Column of position j of internal check m: shared-memory copy or global table.
template <bool SIDX>
__device__ __forceinline__ int colj(const DevCode& c, const uint16_t* __restrict__ sidx, int j, int m) {
  if constexpr (SIDX) return (int)sidx[j * c.M + m];
  else return (int)__ldg(c.ell16 + j * c.M + m);
}

// |x| of both halves (an operand modifier of the instruction that consumes it).
__device__ __forceinline__ uint32_t hab(uint32_t a) {
  uint32_t d; asm("abs.f16x2 %0, %1;" : "=r"(d) : "r"(a)); return d;
}

// Decision parity of check m for the G frames (bit g set: unsatisfied).
template <int G, int D, int DMAX, bool SIDX>
__device__ __forceinline__ uint32_t row_parity_body(const DevCode& c, const uint16_t* __restrict__ sidx,
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
      ld_pairs<G>(Zs, colj<SIDX>(c, sidx, j, m), w);
#pragma unroll
      for (int p = 0; p < P; ++p) y[p] ^= dec_bits(w[p]);
    }
  }
  uint32_t par = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) par |= ((y[p] >> 15) & 1u) << (2 * p) | ((y[p] >> 31) & 1u) << (2 * p + 1);
  return par;
}

// Section III's magnitude rule without branches: g(x) = max((x - beta) num, 0)
// >> shift (plain: beta 0, num 1, shift 0; offset: beta, 1, 0; normalized: 0,
// num, shift), which floors the normalized magnitude like the integer rule.
struct H2Rule {
  int32_t beta, num, shift;
  __device__ __forceinline__ int32_t g(int32_t x) const { return max((x - beta) * num, 0) >> shift; }
};
__device__ inline H2Rule make_h2rule(const IntRule& r) {
  H2Rule h;
  h.beta = r.rule == 1 ? r.beta : 0;
  h.num = r.rule == 2 ? r.num : 1;
  h.shift = r.rule == 2 ? r.shift : 0;
  return h;
}

// One check m for all G frames: Eq. (3) with the Section V state (FORM 1) or
// per-edge messages (FORM 0).  D > 0: the check has exactly D positions (fully
// unrolled); D == 0: d <= DMAX positions, guarded.  Returns the decision parity
// bits of x^(k-1) when ES.
template <int G, int FORM, int D, int DMAX, bool ES, bool SIDX>
__device__ __forceinline__ uint32_t check_body(const DevCode& c, const H2Rule& rule, uint32_t qm2, int m, int d,
                                               const uint32_t* __restrict__ Zs, int32_t* __restrict__ Acc,
                                               uint4* __restrict__ St, uint16_t* __restrict__ Lm,
                                               const uint16_t* __restrict__ sidx) {
  constexpr int P = G / 2;
  constexpr int NJ = D > 0 ? D : DMAX;
  // one frame pair: the pass-1 column indices stay in registers for pass 2;
  // two pairs need those registers for state and reload them
  constexpr bool KEEP = (P == 1 && FORM == 1 && !ES);
  const int M = c.M;
  uint32_t A2[P], B2[P], I2[P], S[P];
  if constexpr (FORM == 1) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const uint4 s = St[m * P + p];
      A2[p] = s.x;
      B2[p] = s.y;
      I2[p] = s.z;
      S[p] = s.w;
    }
  }
  uint32_t K1[P], K2[P], NEG[P], Y[P], SR[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    K1[p] = h2c(2048);
    K2[p] = h2c(2048);
    NEG[p] = 0;
    Y[p] = 0;
    if constexpr (FORM == 1) SR[p] = S[p];
  }
  int col[KEEP ? NJ : 1];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      const int n = colj<SIDX>(c, sidx, j, m);
      if constexpr (KEEP) col[j] = n;
      uint32_t w[P];
      ld_pairs<G>(Zs, n, w);
      uint32_t lv = 0;
      if constexpr (FORM == 0) {
        if constexpr (P == 1) lv = Lm[j * M + m];
        else lv = reinterpret_cast<const uint32_t*>(Lm)[j * M + m];
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        uint32_t L;
        if constexpr (FORM == 1) {
          // f(A, B, n, n~) and the stored sign s_mn on the binary16 sign bit
          const uint32_t msk = heq_mask(I2[p], h2c(j));
          L = ((B2[p] & msk) | (A2[p] & ~msk)) ^ (SR[p] & 0x80008000u);
          SR[p] += SR[p];
        } else {
          // byte L + 128 -> binary16 128 + (L + 128)/8 -> 8 h - 1152 = L
          const uint32_t b = (P == 1) ? lv : (lv >> (16 * p));
          L = hfma(__byte_perm(b, 0x58u, 0x4140), h2c(8), 0xE480E480u /* -1152 */);
        }
        const uint32_t u = hsub(w[p], L);
        if constexpr (ES) Y[p] ^= dec_bits(w[p]);
        NEG[p] |= (u >> j) & (0x80008000u >> j);  // sign of u_j at bit 15 - j / 31 - j
        const uint32_t key = hfma(hmin(hab(u), qm2), h2c(16), h2c(j));
        K2[p] = hmin(K2[p], hmax(K1[p], key));
        K1[p] = hmin(K1[p], key);
      }
    }
  }

  const int dd = D > 0 ? D : d;
  const uint32_t dlane = ((1u << dd) - 1u) << (16 - dd);  // bits 16-d .. 15
  uint32_t An[P], Bn[P], In[P], Sn[P];
  uint32_t par = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    // sign of L^(k)_mj = parity of all input signs xor own sign
    const uint32_t pm = ((__popc(NEG[p] & 0xffffu) & 1) ? 0x0000ffffu : 0u) |
                        ((__popc(NEG[p] >> 16) & 1) ? 0xffff0000u : 0u);
    Sn[p] = (NEG[p] ^ pm) & (dlane | (dlane << 16));
    const int32_t k1l = h_lo_int(K1[p]), k1h = h_hi_int(K1[p]);
    const int32_t k2l = h_lo_int(K2[p]), k2h = h_hi_int(K2[p]);
    An[p] = small_to_h2(rule.g(k1l >> 4), rule.g(k1h >> 4));
    Bn[p] = small_to_h2(rule.g(k2l >> 4), rule.g(k2h >> 4));
    In[p] = small_to_h2(k1l & 15, k1h & 15);
    if constexpr (ES) par |= ((Y[p] >> 15) & 1u) << (2 * p) | ((Y[p] >> 31) & 1u) << (2 * p + 1);
  }

  uint32_t SN[P];
#pragma unroll
  for (int p = 0; p < P; ++p) SN[p] = Sn[p];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    if (D > 0 || j < d) {
      int n;
      if constexpr (KEEP) n = col[j];
      else n = colj<SIDX>(c, sidx, j, m);
      uint32_t sv = 0;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const uint32_t msk = heq_mask(In[p], h2c(j));
        const uint32_t L = ((Bn[p] & msk) | (An[p] & ~msk)) ^ (SN[p] & 0x80008000u);
        SN[p] += SN[p];
        atomicAdd(Acc + n * P + p, (int32_t)hadd(L, h2c(1536)));
        if constexpr (FORM == 0) {
          const uint32_t hb = hfma(L, 0x30003000u /* 0.125 */, h2c(144));
          sv |= (uint32_t)__byte_perm(hb, 0u, 0x4420) << (16 * p);
        }
      }
      if constexpr (FORM == 0) {
        if constexpr (P == 1) Lm[j * M + m] = (uint16_t)sv;
        else reinterpret_cast<uint32_t*>(Lm)[j * M + m] = sv;
      }
    }
  }
  if constexpr (FORM == 1) {
#pragma unroll
    for (int p = 0; p < P; ++p) St[m * P + p] = make_uint4(An[p], Bn[p], In[p], Sn[p]);
  }
  return par;
}

// Degrees with a fully unrolled body; other degrees take the guarded loop.
template <int DMAX>
struct Fast {
  static constexpr int a = DMAX <= 8 ? 6 : 14;
  static constexpr int b = DMAX <= 8 ? 7 : 15;
};

template <int G, int FORM, int DMAX, bool ES, bool SIDX>
__device__ __forceinline__ uint32_t check_update_h2(const DevCode& c, const H2Rule& r, uint32_t qm2, int m,
                                                    const uint32_t* __restrict__ Zs, int32_t* __restrict__ Acc,
                                                    uint4* __restrict__ St, uint16_t* __restrict__ Lm,
                                                    const uint16_t* __restrict__ sidx) {
  const int d = c.deg(m);
  if (d == Fast<DMAX>::a)
    return check_body<G, FORM, Fast<DMAX>::a, DMAX, ES, SIDX>(c, r, qm2, m, d, Zs, Acc, St, Lm, sidx);
  if (d == Fast<DMAX>::b)
    return check_body<G, FORM, Fast<DMAX>::b, DMAX, ES, SIDX>(c, r, qm2, m, d, Zs, Acc, St, Lm, sidx);
  return check_body<G, FORM, 0, DMAX, ES, SIDX>(c, r, qm2, m, d, Zs, Acc, St, Lm, sidx);
}

template <int G, int DMAX, bool SIDX>
__device__ __forceinline__ uint32_t row_parity_h2(const DevCode& c, const uint16_t* __restrict__ sidx,
                                                  const uint32_t* __restrict__ Zs, int m) {
  return row_parity_body<G, 0, DMAX, SIDX>(c, sidx, Zs, m, c.deg(m));
}

__device__ __forceinline__ int32_t q0v(const int8_t* __restrict__ llr, int32_t N, int32_t f, int32_t F, int n) {
  return f < F ? (int32_t)__ldg(llr + (size_t)f * N + n) : 0;
}

template <int G, int FORM, int DMAX, bool ES, bool SIDX>
__global__ void __launch_bounds__(kThreadsMax, 1)
onchip_h2_kernel(const DevCode c, const IntRule r, const int8_t* __restrict__ llr, int32_t F, int32_t max_iter,
                 uint8_t* __restrict__ bits, int32_t* __restrict__ iters, uint8_t* __restrict__ okf,
                 int16_t* __restrict__ zout, int32_t n_groups) {
  constexpr int P = G / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = c.N, M = c.M;
  const H2Layout Ly = h2_layout(N, M, c.ell_w * M, G, FORM, SIDX);
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
        Acc[(size_t)n * P + p] = (int32_t)((uint32_t)acc_pack(lo, hi) - bias);
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
        fail |= check_update_h2<G, FORM, DMAX, ES, SIDX>(c, hr, qm2, m, Zs, Acc, St, Lm, sidx);
      if constexpr (ES) {
        fail = __reduce_or_sync(0xffffffffu, fail);
        if ((tid & 31) == 0 && (fail & act)) atomicOr(&s_fail[kp], fail & act);
      }
      __syncthreads();
      const uint32_t stop = ES ? (act & ~s_fail[kp]) : 0u;
      const uint32_t cont = act & ~stop;
      for (int n = tid; n < N; n += nt) {
        const uint32_t bias = (uint32_t)__ldg(c.cdeg + n) * 0x66006600u;
        uint32_t w[P];
        ld_pairs<G>(Zs, n, w);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const uint32_t zz = acc_to_pair(Acc[(size_t)n * P + p]);
          const uint32_t h = ints_to_h2(lo16(zz), hi16(zz));
          const uint32_t sel = (((cont >> (2 * p)) & 1u) ? 0x0000ffffu : 0u) |
                               (((cont >> (2 * p + 1)) & 1u) ? 0xffff0000u : 0u);
          w[p] = (h & sel) | (w[p] & ~sel);
          const int32_t lo = q0v(llr, N, f0 + 2 * p, F, n), hi = q0v(llr, N, f0 + 2 * p + 1, F, n);
          Acc[(size_t)n * P + p] = (int32_t)((uint32_t)acc_pack(lo, hi) - bias);
        }
        st_pairs<G>(Zs, n, w);
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
      for (int m = tid; m < M; m += nt) fail |= row_parity_h2<G, DMAX, SIDX>(c, sidx, Zs, m);
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

template <int G, int FORM, int DMAX, bool ES, bool SIDX>
cudaError_t h2_launch_t(const DevCode& c, const IntRule& r, OnchipPlan& plan, int sm_count, const int8_t* llr,
                        int32_t F, int32_t max_iter, uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout,
                        cudaStream_t stream, bool occupancy_only) {
  auto kern = onchip_h2_kernel<G, FORM, DMAX, ES, SIDX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
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
  if (plan.sidx)
    return es ? h2_launch_t<G, FORM, DMAX, true, true>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ)
              : h2_launch_t<G, FORM, DMAX, false, true>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ);
  return es ? h2_launch_t<G, FORM, DMAX, true, false>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ)
            : h2_launch_t<G, FORM, DMAX, false, false>(c, r, plan, sm_count, llr, F, max_iter, bits, iters, ok, zout, stream, occ);
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
  plan->G = G;
  plan->sidx = sidx;
  plan->dmax = max_row_deg <= 8 ? 8 : 16;
  plan->smem = h2_layout(c.N, c.M, c.ell_w * c.M, G, form, sidx).total;
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
