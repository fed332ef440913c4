// onchip_int8.cu -- frame-resident single-scan min-sum decoder, int8 path.
//
// One CTA owns G frames at a time and runs every iteration of Section IV's
// single scan (Eq. (3)) for them without leaving the SM:
//
//   Zs   [N][G/2]  u32   posterior Z^(k-1) of frame pairs, int16 halves
//   Acc  [N][G/2]  i32   Z^(k) being accumulated, as the integer lo + 65536 hi
//   state           form 1 (Section V): per check and frame (A, B, n~) and a
//                   sign word, 8 bytes;  form 0 (Section IV): L_mn, int8 per
//                   edge and frame.
//
// Iteration k:
//   row pass    each thread takes whole checks m; for each frame it rebuilds
//               L^(k-1)_mn' (Section V f(A, B, n, n~) or the stored byte), forms
//               u = Z^(k-1)_n' - L^(k-1)_mn', saturates |u| to Qm, tracks
//               min1/min2/first argmin in one packed key and the sign parity,
//               applies the offset/normalization (Eqs. (4)-(5) as modified in
//               Section V), then adds L^(k)_mn into Acc with one 32-bit shared
//               atomic per frame pair (order-independent, exact), and stores
//               the new state.  The same gathers give the parity of the
//               decisions x^(k-1) (Section III stop rule), fused into the pass.
//   column pass frames whose x^(k-1) satisfied H stop with Z^(k-1); the others
//               take Z^(k) = Acc, and Acc is reset to Z^(0) (Eq. (3) first line).
// After the cap a final syndrome pass gives the flags of frames still running.
#include "kernels.h"
#include "launch_util.h"

namespace ldpc {
namespace {

constexpr int kMaxThreads = 1024;

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct SmemLayout {
  size_t zs, acc, st, total;
};

__host__ __device__ inline SmemLayout layout(int N, int M, int E, int G, int form) {
  SmemLayout L;
  const size_t P = (size_t)G / 2;
  L.zs = 0;
  L.acc = align16((size_t)N * P * 4);
  L.st = L.acc + align16((size_t)N * P * 4);
  const size_t st_bytes = form == 1 ? (size_t)M * G * 8 : (size_t)E * G;
  L.total = L.st + align16(st_bytes);
  return L;
}

template <int G>
__device__ __forceinline__ void load_pairs(const uint32_t* __restrict__ Zs, int n, uint32_t (&w)[G / 2]) {
  if constexpr (G == 2) {
    w[0] = Zs[n];
  } else {
    const uint2 v = reinterpret_cast<const uint2*>(Zs)[n];
    w[0] = v.x;
    w[1] = v.y;
  }
}

template <int G>
__device__ __forceinline__ void store_pairs(uint32_t* __restrict__ Zs, int n, const uint32_t (&w)[G / 2]) {
  if constexpr (G == 2) {
    Zs[n] = w[0];
  } else {
    reinterpret_cast<uint2*>(Zs)[n] = make_uint2(w[0], w[1]);
  }
}

// Per-edge messages of G frames (form 0), one byte each.
template <int G>
__device__ __forceinline__ uint32_t load_edge(const int8_t* __restrict__ Lm, int e) {
  if constexpr (G == 2) return (uint32_t) reinterpret_cast<const uint16_t*>(Lm)[e];
  else return reinterpret_cast<const uint32_t*>(Lm)[e];
}
template <int G>
__device__ __forceinline__ void store_edge(int8_t* __restrict__ Lm, int e, uint32_t v) {
  if constexpr (G == 2) reinterpret_cast<uint16_t*>(Lm)[e] = (uint16_t)v;
  else reinterpret_cast<uint32_t*>(Lm)[e] = v;
}
__device__ __forceinline__ int32_t sbyte(uint32_t v, int g) { return (int32_t)(int8_t)(v >> (8 * g)); }

// Syndrome of the decisions x = (Z <= 0) held in Zs, for the frames of one
// check: bit g of the result is set when check m is unsatisfied for frame g.
template <int G>
__device__ __forceinline__ uint32_t row_parity(const DevCode& c, const uint32_t* __restrict__ Zs, int m) {
  const int d = c.deg(m);
  uint32_t par = 0;
  for (int j = 0; j < d; ++j) {
    const int n = c.col(j, m);
    uint32_t w[G / 2];
    load_pairs<G>(Zs, n, w);
#pragma unroll
    for (int p = 0; p < G / 2; ++p) {
      par ^= (uint32_t)(lo16(w[p]) <= 0) << (2 * p);
      par ^= (uint32_t)(hi16(w[p]) <= 0) << (2 * p + 1);
    }
  }
  return par;
}

// One check m, all G frames: Eq. (3) with the Section V state (FORM 1) or the
// per-edge messages (FORM 0).  Returns the decision-parity bits of x^(k-1).
template <int G, int FORM>
__device__ __forceinline__ uint32_t check_update(const DevCode& c, const IntRule& r, int m,
                                                 const uint32_t* __restrict__ Zs, int32_t* __restrict__ Acc,
                                                 uint2* __restrict__ St, int8_t* __restrict__ Lm) {
  constexpr int P = G / 2;
  const int d = c.deg(m);
  const int M = c.M;

  // previous state: A, B, n~ packed in .x (8/8/8 bits), signs in .y
  uint32_t sa[G], ss[G];
  if constexpr (FORM == 1) {
#pragma unroll
    for (int g = 0; g < G; g += 2) {
      const uint4 v = reinterpret_cast<const uint4*>(St + (size_t)m * G)[g / 2];
      sa[g] = v.x; ss[g] = v.y; sa[g + 1] = v.z; ss[g + 1] = v.w;
    }
  }
  int32_t k1[G], k2[G];
  uint32_t neg[G];
  uint32_t par = 0;
#pragma unroll
  for (int g = 0; g < G; ++g) { k1[g] = 0x7fffffff; k2[g] = 0x7fffffff; neg[g] = 0; }

  for (int j = 0; j < d; ++j) {
    const int n = c.col(j, m);
    uint32_t w[P];
    load_pairs<G>(Zs, n, w);
    uint32_t lv = 0;
    if constexpr (FORM == 0) lv = load_edge<G>(Lm, j * M + m);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int32_t z = (g & 1) ? hi16(w[g / 2]) : lo16(w[g / 2]);
      par ^= (uint32_t)(z <= 0) << g;
      int32_t lold;
      if constexpr (FORM == 1) {
        const int32_t mag = (j == (int)((sa[g] >> 16) & 0xff)) ? (int32_t)((sa[g] >> 8) & 0xff)
                                                               : (int32_t)(sa[g] & 0xff);
        lold = ((ss[g] >> j) & 1u) ? -mag : mag;
      } else {
        lold = sbyte(lv, g);
      }
      const int32_t u = z - lold;
      neg[g] |= (uint32_t)(u < 0) << j;
      const int32_t a = min(abs(u), r.qm);
      const int32_t key = (a << 5) | j;
      k2[g] = min(k2[g], max(k1[g], key));
      k1[g] = min(k1[g], key);
    }
  }

  const uint32_t dmask = d >= 32 ? 0xffffffffu : ((1u << d) - 1u);
  int32_t An[G], Bn[G], In[G];
  uint32_t Sn[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    An[g] = r.g(k1[g] >> 5);
    Bn[g] = r.g(k2[g] >> 5);
    In[g] = k1[g] & 31;
    Sn[g] = ((__popc(neg[g]) & 1) ? ~neg[g] : neg[g]) & dmask;  // sign of L^(k)_mj: parity xor own
  }

  for (int j = 0; j < d; ++j) {
    const int n = c.col(j, m);
    int32_t l[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int32_t mag = (j == In[g]) ? Bn[g] : An[g];
      l[g] = ((Sn[g] >> j) & 1u) ? -mag : mag;
    }
#pragma unroll
    for (int p = 0; p < P; ++p) atomicAdd(Acc + (size_t)n * P + p, acc_pack(l[2 * p], l[2 * p + 1]));
    if constexpr (FORM == 0) {
      uint32_t v = 0;
#pragma unroll
      for (int g = 0; g < G; ++g) v |= ((uint32_t)l[g] & 0xffu) << (8 * g);
      store_edge<G>(Lm, j * M + m, v);
    }
  }
  if constexpr (FORM == 1) {
#pragma unroll
    for (int g = 0; g < G; g += 2) {
      const uint32_t a0 = (uint32_t)An[g] | ((uint32_t)Bn[g] << 8) | ((uint32_t)In[g] << 16);
      const uint32_t a1 = (uint32_t)An[g + 1] | ((uint32_t)Bn[g + 1] << 8) | ((uint32_t)In[g + 1] << 16);
      reinterpret_cast<uint4*>(St + (size_t)m * G)[g / 2] = make_uint4(a0, Sn[g], a1, Sn[g + 1]);
    }
  }
  return par;
}

__device__ __forceinline__ int32_t q0_at(const int8_t* __restrict__ llr, int32_t N, int32_t f, int32_t F, int n) {
  return f < F ? (int32_t)__ldg(llr + (size_t)f * N + n) : 0;
}

template <int G, int FORM>
__global__ void __launch_bounds__(kMaxThreads, 1)
onchip_int8_kernel(const DevCode c, const IntRule r, const int8_t* __restrict__ llr, int32_t F,
                   int32_t max_iter, int32_t early_stop, uint8_t* __restrict__ bits,
                   int32_t* __restrict__ iters, uint8_t* __restrict__ okf, int16_t* __restrict__ zout,
                   int32_t n_groups) {
  constexpr int P = G / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = c.N, M = c.M;
  const SmemLayout L = layout(N, M, c.ell_w * M, G, FORM);
  uint32_t* Zs = reinterpret_cast<uint32_t*>(smem + L.zs);
  int32_t* Acc = reinterpret_cast<int32_t*>(smem + L.acc);
  uint2* St = reinterpret_cast<uint2*>(smem + L.st);
  int8_t* Lm = reinterpret_cast<int8_t*>(smem + L.st);
  __shared__ uint32_t s_fail[3];
  __shared__ int32_t s_iters[G];
  __shared__ uint32_t s_ok;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int N8 = (N + 7) >> 3;

  for (int grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const int f0 = grp * G;
    const int nvalid = min(G, F - f0);
    uint32_t act = (1u << nvalid) - 1u;

    // k = 0: Z^(0) = q0 and L^(0) = 0.
    for (int n = tid; n < N; n += nt) {
      uint32_t w[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int32_t lo = q0_at(llr, N, f0 + 2 * p, F, n), hi = q0_at(llr, N, f0 + 2 * p + 1, F, n);
        w[p] = pack16(lo, hi);
        Acc[(size_t)n * P + p] = acc_pack(lo, hi);
      }
      store_pairs<G>(Zs, n, w);
    }
    if constexpr (FORM == 1) {
      for (int i = tid; i < M * G; i += nt) St[i] = make_uint2(0u, 0u);
    } else {
      for (int i = tid; i < c.ell_w * M; i += nt) store_edge<G>(Lm, i, 0u);
    }
    if (tid < 3) s_fail[tid] = 0;
    if (tid < G) s_iters[tid] = max_iter;
    if (tid == 0) s_ok = 0;
    __syncthreads();

    for (int k = 1; k <= max_iter && act != 0u; ++k) {
      const int kp = k & 1;
      uint32_t fail = 0;
      for (int m = tid; m < M; m += nt) fail |= check_update<G, FORM>(c, r, m, Zs, Acc, St, Lm);
      fail = __reduce_or_sync(0xffffffffu, fail);
      if ((tid & 31) == 0 && (fail & act)) atomicOr(&s_fail[kp], fail & act);
      __syncthreads();
      const uint32_t stop = early_stop ? (act & ~s_fail[kp]) : 0u;
      const uint32_t cont = act & ~stop;
      for (int n = tid; n < N; n += nt) {
        uint32_t w[P];
        load_pairs<G>(Zs, n, w);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const uint32_t z = acc_to_pair(Acc[(size_t)n * P + p]);
          const uint32_t sel = (((cont >> (2 * p)) & 1u) ? 0x0000ffffu : 0u) |
                               (((cont >> (2 * p + 1)) & 1u) ? 0xffff0000u : 0u);
          w[p] = (z & sel) | (w[p] & ~sel);
          Acc[(size_t)n * P + p] =
              acc_pack(q0_at(llr, N, f0 + 2 * p, F, n), q0_at(llr, N, f0 + 2 * p + 1, F, n));
        }
        store_pairs<G>(Zs, n, w);
      }
      if (tid < G && ((stop >> tid) & 1u)) s_iters[tid] = k - 1;
      if (tid == 0) s_ok |= stop;
      __syncthreads();
      if (tid == 0) s_fail[kp] = 0;  // next written at iteration k + 2
      act = cont;
    }

    // Frames that ran to the cap: syndrome of their final decisions.
    if (act != 0u) {
      uint32_t fail = 0;
      for (int m = tid; m < M; m += nt) fail |= row_parity<G>(c, Zs, m);
      fail = __reduce_or_sync(0xffffffffu, fail);
      if ((tid & 31) == 0 && (fail & act)) atomicOr(&s_fail[2], fail & act);
      __syncthreads();
      if (tid == 0) s_ok |= act & ~s_fail[2];
    }
    __syncthreads();

    // Outputs: packed decisions, iterations, flags, optional posterior.
    for (int i = tid; i < nvalid * N8; i += nt) {
      const int g = i / N8, b = i - g * N8;
      uint32_t byte = 0;
      for (int t = 0; t < 8; ++t) {
        const int n = b * 8 + t;
        if (n < N) {
          const uint32_t w = Zs[(size_t)n * P + g / 2];
          const int32_t z = (g & 1) ? hi16(w) : lo16(w);
          byte |= (uint32_t)(z <= 0) << t;
        }
      }
      bits[(size_t)(f0 + g) * N8 + b] = (uint8_t)byte;
    }
    if (zout != nullptr) {
      for (int i = tid; i < nvalid * N; i += nt) {
        const int g = i / N, n = i - g * N;
        const uint32_t w = Zs[(size_t)n * P + g / 2];
        zout[(size_t)(f0 + g) * N + n] = (int16_t)((g & 1) ? hi16(w) : lo16(w));
      }
    }
    if (tid < nvalid) {
      iters[f0 + tid] = s_iters[tid];
      okf[f0 + tid] = (uint8_t)((s_ok >> tid) & 1u);
    }
    __syncthreads();
  }
}

template <int G, int FORM>
cudaError_t launch_t(const DevCode& c, const IntRule& r, const OnchipPlan& plan, const int8_t* llr,
                     int32_t F, int32_t max_iter, int32_t early_stop, uint8_t* bits, int32_t* iters,
                     uint8_t* ok, int16_t* zout, cudaStream_t stream) {
  auto kern = onchip_int8_kernel<G, FORM>;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(kern), plan.smem);
  if (e != cudaSuccess) return e;
  kern<<<plan.grid, plan.threads, plan.smem, stream>>>(c, r, llr, F, max_iter, early_stop, bits, iters,
                                                      ok, zout, plan.n_groups);
  return cudaGetLastError();
}

template <int G, int FORM>
cudaError_t occupancy_t(OnchipPlan* plan, int sm_count) {
  auto kern = onchip_int8_kernel<G, FORM>;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(kern), plan->smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, plan->threads, plan->smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t cap = (int64_t)sm_count * per_sm;
  plan->grid = (int)((int64_t)plan->n_groups < cap ? plan->n_groups : cap);
  return cudaSuccess;
}

}  // namespace

cudaError_t onchip_int8_occupancy(int form, int sm_count, OnchipPlan* plan) {
  if (plan->G == 4 && form == 1) return occupancy_t<4, 1>(plan, sm_count);
  if (plan->G == 2 && form == 1) return occupancy_t<2, 1>(plan, sm_count);
  if (plan->G == 4 && form == 0) return occupancy_t<4, 0>(plan, sm_count);
  if (plan->G == 2 && form == 0) return occupancy_t<2, 0>(plan, sm_count);
  return cudaErrorInvalidValue;
}

bool onchip_int8_plan(const DevCode& c, int form, int32_t n_frames, int sm_count, size_t smem_optin,
                      int max_row_deg, OnchipPlan* plan) {
  (void)max_row_deg;
  const size_t static_smem = 64;  // s_fail, s_iters, s_ok
  int G = 0;
  for (int g : {4, 2}) {
    if (layout(c.N, c.M, c.ell_w * c.M, g, form).total + static_smem <= smem_optin) { G = g; break; }
  }
  if (G == 0) return false;
  // Fewer frames per CTA when that is what it takes to give every SM work.
  while (G > 2 && (int64_t)n_frames < (int64_t)sm_count * G) G /= 2;
  plan->G = G;
  plan->smem = layout(c.N, c.M, c.ell_w * c.M, G, form).total;
  int threads = ((c.M + 31) / 32) * 32;
  if (threads > kMaxThreads) threads = kMaxThreads;
  if (threads < 128) threads = 128;
  plan->threads = threads;
  plan->n_groups = (n_frames + G - 1) / G;
  plan->grid = 0;  // set by onchip_int8_occupancy
  return true;
}

cudaError_t onchip_int8_launch(const DevCode& c, const IntRule& r, int form, const OnchipPlan& plan,
                               const int8_t* llr, int32_t n_frames, int32_t max_iter, int32_t early_stop,
                               uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout,
                               cudaStream_t stream) {
  if (plan.G == 4 && form == 1)
    return launch_t<4, 1>(c, r, plan, llr, n_frames, max_iter, early_stop, bits, iters, ok, zout, stream);
  if (plan.G == 2 && form == 1)
    return launch_t<2, 1>(c, r, plan, llr, n_frames, max_iter, early_stop, bits, iters, ok, zout, stream);
  if (plan.G == 4 && form == 0)
    return launch_t<4, 0>(c, r, plan, llr, n_frames, max_iter, early_stop, bits, iters, ok, zout, stream);
  if (plan.G == 2 && form == 0)
    return launch_t<2, 0>(c, r, plan, llr, n_frames, max_iter, early_stop, bits, iters, ok, zout, stream);
  return cudaErrorInvalidValue;
}

}  // namespace ldpc
