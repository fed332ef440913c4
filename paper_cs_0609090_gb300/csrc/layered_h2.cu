// layered_h2.cu -- the single scan of Eq. (3) in a layered schedule, int8 path,
// exact packed binary16 frame pairs (the arithmetic of onchip_h2.cu).
//
// The checks are grouped into layers whose checks share no variable.  Within
// an iteration the layers run in order; every check of a layer reads the
// posteriors as the previous layers left them and updates them in place,
// Z_n <- Z_n + L^(k)_mn - L^(k-1)_mn, which equals (Z_n - L^(k-1)_mn) + L^(k)_mn
// exactly (integers below 2048 in binary16).  Checks of one layer touch
// disjoint variables, so they run in parallel with plain stores, no atomics
// and no column pass.  (Section I cites layered decoding; the paper's own
// schedule is flooding.)  The stop rule checks the decisions after each whole
// iteration (and before the first) with a parity pass over all checks.
//
// Frames are split into chunks of PW frame pairs; one CTA owns a chunk for the
// whole decode, so only its own barrier separates the layers.  Chunk state,
// chunk-major with the pair innermost:
//   Z  [N][PW] half2      posterior pairs: in shared memory when they fit next
//                         to the column table (ZSM, PW = 4), else in the
//                         workspace (PW = 8)
//   St [M][PW] uint4 (Section V state)  or  Lm [ell_w M][PW] u16 (per edge), in
//                         the workspace
// A thread owns one check of the current layer for one pair (kThreads / PW
// checks per step).  512 threads: the in-place body needs about 128 registers
// (measured on the N=7493 code, 30 iterations, Z in the workspace: 5.38 ms
// against 5.80 ms with 1024 threads limited to 64 registers and spilling).
#include <cuda_fp16.h>

#include <algorithm>

#include "h2_body.cuh"
#include "kernels.h"
#include "launch_util.h"

namespace ldpc {
namespace {

constexpr int kThreads = 512;

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// One pair lane of a chunk: handles are element offsets n kPW from the lane's
// base; the column index comes from the degree-sorted edge-slot table (shared
// memory copy when SIDX).  sel: the halves this lane may change (frames still
// running).
template <bool WIDE, bool SIDX, int kPW>
struct LayAddr {
  using H = uint32_t;
  int M;
  const uint16_t* __restrict__ t16;
  const int32_t* __restrict__ t32;
  uint32_t* Z;
  uint32_t sel;
  __device__ __forceinline__ H at(const uint16_t*, const uint32_t*, int j, int m) const {
    int n;
    if constexpr (SIDX) n = (int)t16[j * M + m];
    else if constexpr (WIDE) n = __ldg(t32 + j * M + m);
    else n = (int)__ldg(t16 + j * M + m);
    return (uint32_t)n * kPW;
  }
  __device__ __forceinline__ void load(const uint32_t*, H h, uint32_t (&w)[1]) const { w[0] = Z[h]; }
  __device__ __forceinline__ void update(H h, int, uint32_t Ln, uint32_t Lo) const {
    const uint32_t w = Z[h];
    const uint32_t z = hadd(w, hsub(Ln, Lo));
    Z[h] = (z & sel) | (w & ~sel);
  }
  __device__ __forceinline__ void add(int32_t*, H, int, int32_t) const {}
  __device__ __forceinline__ uint32_t st(int m) const { return (uint32_t)m * kPW; }
  __device__ __forceinline__ uint32_t lm(int j, int m) const { return (uint32_t)(j * M + m) * kPW; }
};

template <int FORM, class A>
__device__ __forceinline__ void lay_check(const A& ad, const H2Rule& r, uint32_t qm2, int m, int d, uint4* St,
                                          uint16_t* Lm) {
  switch (d) {
    case 6: check_body<2, FORM, 6, 16, false, A, 2>(ad, nullptr, nullptr, nullptr, r, qm2, m, d, St, Lm); break;
    case 7: check_body<2, FORM, 7, 16, false, A, 2>(ad, nullptr, nullptr, nullptr, r, qm2, m, d, St, Lm); break;
    case 14: check_body<2, FORM, 14, 16, false, A, 2>(ad, nullptr, nullptr, nullptr, r, qm2, m, d, St, Lm); break;
    case 15: check_body<2, FORM, 15, 16, false, A, 2>(ad, nullptr, nullptr, nullptr, r, qm2, m, d, St, Lm); break;
    default: check_body<2, FORM, 0, 16, false, A, 2>(ad, nullptr, nullptr, nullptr, r, qm2, m, d, St, Lm); break;
  }
}

__device__ __forceinline__ int32_t q0v(const int8_t* __restrict__ llr, int32_t N, int32_t f, int32_t F, int n) {
  return f < F ? (int32_t)__ldg(llr + (size_t)f * N + n) : 0;
}

template <int FORM, bool ES, bool WIDE, bool SIDX, int kPW, bool ZSM>
__global__ void __launch_bounds__(kThreads, 1)
layered_kernel(const DevCode c, const IntRule r, const int32_t* __restrict__ lay_ptr,
               const int32_t* __restrict__ lay_rows, int32_t n_layers, const int8_t* __restrict__ llr, int32_t F,
               int32_t max_iter, uint8_t* __restrict__ bits, int32_t* __restrict__ iters,
               uint8_t* __restrict__ okf, int16_t* __restrict__ zout, void* ws, size_t chunk_bytes,
               size_t st_off, int32_t n_chunks, uint32_t zsm_off, int32_t* __restrict__ queue) {
  constexpr int kSlots = kThreads / kPW;  // checks of a layer per step
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_act[kPW], s_fail[kPW], s_ok[kPW];
  __shared__ int32_t s_iters[2 * kPW];
  __shared__ int s_any, s_chunk;
  const int tid = threadIdx.x;
  const int N = c.N, M = c.M;
  const int slot = tid / kPW, p = tid % kPW;
  uint16_t* stab = reinterpret_cast<uint16_t*>(smem);
  if constexpr (SIDX) {
    const int cnt = c.ell_w * M;
    for (int i = tid; i < cnt; i += kThreads) stab[i] = __ldg(c.ell16 + i);
  }
  const uint32_t qm2 = ints_to_h2(r.qm, r.qm);
  const H2Rule hr = make_h2rule(r);
  const int N8 = (N + 7) >> 3;

  // chunks from a queue in the workspace (frames that run to the cap make some
  // chunks much longer than others under early stop)
  for (;;) {
    if (tid == 0) s_chunk = atomicAdd(queue, 1);
    __syncthreads();
    const int ch = s_chunk;
    if (ch >= n_chunks) break;
    unsigned char* base = static_cast<unsigned char*>(ws) + (size_t)ch * chunk_bytes;
    uint32_t* Z = ZSM ? reinterpret_cast<uint32_t*>(smem + zsm_off) : reinterpret_cast<uint32_t*>(base);
    uint4* St = reinterpret_cast<uint4*>(base + st_off);
    uint16_t* Lm = reinterpret_cast<uint16_t*>(base + st_off);
    const int pair0 = ch * kPW;
    // Z^(0) = q0, L^(0) = 0
    for (int i = tid; i < N * kPW; i += kThreads) {
      const int n = i / kPW, q = i - n * kPW;
      const int f = 2 * (pair0 + q);
      Z[i] = ints_to_h2(q0v(llr, N, f, F, n), q0v(llr, N, f + 1, F, n));
    }
    if constexpr (FORM == 1) {
      for (int i = tid; i < M * kPW; i += kThreads) St[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
      for (int i = tid; i < c.ell_w * M * kPW; i += kThreads) Lm[i] = 0x8080u;
    }
    if (tid < kPW) {
      const int f = 2 * (pair0 + tid);
      s_act[tid] = (f < F ? 1u : 0u) | (f + 1 < F ? 2u : 0u);
      s_fail[tid] = 0;
      s_ok[tid] = 0;
      s_iters[2 * tid] = max_iter;
      s_iters[2 * tid + 1] = max_iter;
    }
    __syncthreads();
    LayAddr<WIDE, SIDX, kPW> ad{M, SIDX ? stab : c.ell16, c.ell32, Z + p, 0u};

    // parity of the decisions of every check, ORed per pair lane into s_fail
    auto syndrome = [&]() {
      for (int m = slot; m < M; m += kSlots) {
        const uint32_t par = row_parity_body<2, 0, 16>(ad, nullptr, nullptr, m, (int)__ldg(c.rdeg + m));
        if (par) atomicOr(&s_fail[p], par);
      }
      __syncthreads();
    };
    if (ES) {
      syndrome();
      if (tid < kPW) {
        const uint32_t stop = s_act[tid] & ~s_fail[tid];
        if (stop & 1u) s_iters[2 * tid] = 0;
        if (stop & 2u) s_iters[2 * tid + 1] = 0;
        s_ok[tid] |= stop;
        s_act[tid] &= s_fail[tid];
        s_fail[tid] = 0;
      }
      __syncthreads();
    }
    for (int k = 1; k <= max_iter; ++k) {
      if (tid == 0) {
        uint32_t any = 0;
        for (int q = 0; q < kPW; ++q) any |= s_act[q];
        s_any = any != 0u;
      }
      __syncthreads();
      if (!s_any) break;
      const uint32_t act = s_act[p];
      ad.sel = ((act & 1u) ? 0x0000ffffu : 0u) | ((act & 2u) ? 0xffff0000u : 0u);
      for (int l = 0; l < n_layers; ++l) {
        const int r0 = __ldg(lay_ptr + l), r1 = __ldg(lay_ptr + l + 1);
        for (int i = r0 + slot; i < r1; i += kSlots) {
          const int m = __ldg(lay_rows + i);
          lay_check<FORM>(ad, hr, qm2, m, (int)__ldg(c.rdeg + m), St + p, Lm + p);
        }
        __syncthreads();
      }
      if (ES) {
        syndrome();
        if (tid < kPW) {
          const uint32_t stop = s_act[tid] & ~s_fail[tid];
          if (stop & 1u) s_iters[2 * tid] = k;
          if (stop & 2u) s_iters[2 * tid + 1] = k;
          s_ok[tid] |= stop;
          s_act[tid] &= s_fail[tid];
          s_fail[tid] = 0;
        }
        __syncthreads();
      }
    }
    // frames still running after the cap: the syndrome of their final decisions
    if (tid < kPW) s_fail[tid] = 0;
    __syncthreads();
    syndrome();
    if (tid < kPW) s_ok[tid] |= s_act[tid] & ~s_fail[tid];
    __syncthreads();

    for (int i = tid; i < 2 * kPW * N8; i += kThreads) {
      const int fl = i / N8, b = i - fl * N8;
      const int f = 2 * pair0 + fl;
      if (f >= F) continue;
      uint32_t byte = 0;
      for (int t = 0; t < 8; ++t) {
        const int n = b * 8 + t;
        if (n < N) byte |= ((dec_bits(Z[n * kPW + (fl >> 1)] >> (16 * (fl & 1))) >> 15) & 1u) << t;
      }
      bits[(size_t)f * N8 + b] = (uint8_t)byte;
    }
    if (zout != nullptr) {
      for (int i = tid; i < 2 * kPW * N; i += kThreads) {
        const int fl = i / N, n = i - fl * N;
        const int f = 2 * pair0 + fl;
        if (f >= F) continue;
        const uint32_t h = Z[n * kPW + (fl >> 1)];
        zout[(size_t)f * N + n] = (int16_t)((fl & 1) ? h_hi_int(h) : h_lo_int(h));
      }
    }
    if (tid < 2 * kPW) {
      const int f = 2 * pair0 + tid;
      if (f < F) {
        iters[f] = s_iters[tid];
        okf[f] = (uint8_t)((s_ok[tid >> 1] >> (tid & 1)) & 1u);
      }
    }
    __syncthreads();
  }
}

template <int FORM, bool ES, bool WIDE, bool SIDX, int PW, bool ZSM>
cudaError_t lay_launch_t(const DevCode& c, const IntRule& r, const int32_t* lay_ptr, const int32_t* lay_rows,
                         int n_layers, const int8_t* llr, int32_t F, int32_t max_iter, uint8_t* bits, int32_t* iters,
                         uint8_t* ok, int16_t* zout, void* ws, const LayeredLayout& L, int sm_count,
                         cudaStream_t st) {
  auto kern = layered_kernel<FORM, ES, WIDE, SIDX, PW, ZSM>;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(kern), L.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(L.chunks, per_sm * sm_count);
  char* w = static_cast<char*>(ws);
  e = cudaMemsetAsync(w, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, L.smem, st>>>(c, r, lay_ptr, lay_rows, n_layers, llr, F, max_iter, bits, iters, ok, zout,
                                       w + L.hdr, L.chunk_bytes, L.st_off, L.chunks, (uint32_t)L.zsm_off,
                                       reinterpret_cast<int32_t*>(w));
  return cudaGetLastError();
}

}  // namespace

LayeredLayout layered_layout(int form, int N, int M, int ell_w, int F, bool narrow, size_t smem_optin) {
  LayeredLayout L;
  const size_t reserve = 1024;  // static shared memory, rounded up
  const size_t tab = ((size_t)ell_w * M * 2 + 15) & ~size_t(15);
  L.sidx = narrow && tab + reserve <= smem_optin;
  // posteriors of a 4-pair chunk in shared memory next to the table
  L.zsm = L.sidx && tab + (size_t)N * 4 * 4 + reserve <= smem_optin;
  L.pw = L.zsm ? 4 : 8;
  L.zsm_off = tab;
  L.smem = (L.sidx ? tab : 0) + (L.zsm ? (size_t)N * L.pw * 4 : 0);
  L.chunks = ((F + 1) / 2 + L.pw - 1) / L.pw;
  L.st_off = L.zsm ? 0 : al256((size_t)N * L.pw * 4);
  L.chunk_bytes = al256(L.st_off + (form == 1 ? (size_t)M * L.pw * 16 : (size_t)ell_w * M * L.pw * 2));
  L.hdr = 256;  // the chunk queue counter
  L.total = L.hdr + (size_t)L.chunks * L.chunk_bytes;
  return L;
}

cudaError_t layered_decode(const DevCode& c, const IntRule& r, int form, const int32_t* lay_ptr,
                           const int32_t* lay_rows, int n_layers, const int8_t* llr, int32_t F, int32_t max_iter,
                           int32_t early_stop, uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout, void* ws,
                           const LayeredLayout& L, int sm_count, cudaStream_t st) {
  const bool es = early_stop != 0;
  const bool wide = c.ell16 == nullptr;
#define LDPC_LAY(FF, EE, WW, SS, PP, ZZ)                                                                          \
  if (form == FF && es == EE && wide == WW && L.sidx == SS && L.pw == PP && L.zsm == ZZ)                         \
    return lay_launch_t<FF, EE, WW, SS, PP, ZZ>(c, r, lay_ptr, lay_rows, n_layers, llr, F, max_iter, bits, iters, \
                                                ok, zout, ws, L, sm_count, st);
  LDPC_LAY(1, true, false, true, 4, true)
  LDPC_LAY(1, false, false, true, 4, true)
  LDPC_LAY(0, true, false, true, 4, true)
  LDPC_LAY(0, false, false, true, 4, true)
  LDPC_LAY(1, true, false, true, 8, false)
  LDPC_LAY(1, false, false, true, 8, false)
  LDPC_LAY(0, true, false, true, 8, false)
  LDPC_LAY(0, false, false, true, 8, false)
  LDPC_LAY(1, true, false, false, 8, false)
  LDPC_LAY(1, false, false, false, 8, false)
  LDPC_LAY(0, true, false, false, 8, false)
  LDPC_LAY(0, false, false, false, 8, false)
  LDPC_LAY(1, true, true, false, 8, false)
  LDPC_LAY(1, false, true, false, 8, false)
  LDPC_LAY(0, true, true, false, 8, false)
  LDPC_LAY(0, false, true, false, 8, false)
#undef LDPC_LAY
  return cudaErrorInvalidValue;
}

}  // namespace ldpc
