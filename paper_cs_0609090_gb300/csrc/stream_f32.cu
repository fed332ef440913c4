// stream_f32.cu -- the float32 streaming decoder: single-scan min-sum (Eq. (3),
// offset / normalized rules of Section III) and the sum-product check rule on
// float32 frames whose state lives in device memory, one frame per lane.
//
// Workspace (StreamLayout, frame index innermost): two posterior buffers
// [N][FL] f32 each, the message state [M][FL] uint4 {A, B, n~, signs}
// (Section V; 10 bytes per frame when every check has degree <= 8) or per-edge
// f32 [slot][FL] (slot j M + m of the degree-sorted table for min-sum, the CSR
// edge for sum-product), q0 [N][FL] f32, act/fail [2][FL] u32, iters [FL],
// ok [FL].  The row passes run chunk-major (stream_grid.h), the column pass
// takes four frames per thread.  The posterior accumulation uses
// floating-point atomics, so its rounding depends on the order of the additions.
#include <algorithm>

#include "kernels.h"
#include "stream_grid.h"

namespace ldpc {
namespace {

// ------------------------------------------------------------------ float32

// One frame per lane.  The posterior is double-buffered: Z^(k) lives in
// zb[k & 1].  The row pass of iteration k reads Z^(k-1) from one buffer and
// adds its messages into the other, which holds Z0 on entry, so that it holds
// Z0 + sum_m L^(k)_mn = Z^(k) (Eq. (3)) when the pass ends.  The column pass
// then only decides the stops and resets the buffer just read to Z0 for the
// frames that go on.  A stopped frame's buffers are never written again, and
// its result is the buffer of its iteration count.
struct F32S {
  float* zb0;
  float* zb1;
  uint4* st;
  float* lm;
  float* q0;
  uint32_t* act;
  uint32_t* fail;
  int32_t* iters;
  uint32_t* ok;
  int FL;
  __device__ __forceinline__ float* zb(int k) const { return (k & 1) ? zb1 : zb0; }
};

F32S f32s_view(void* ws, const StreamLayout& L) {
  char* b = static_cast<char*>(ws);
  F32S s;
  s.zb0 = reinterpret_cast<float*>(b + L.z);
  s.zb1 = reinterpret_cast<float*>(b + L.acc);
  s.st = reinterpret_cast<uint4*>(b + L.st);
  s.lm = reinterpret_cast<float*>(b + L.st);
  s.q0 = reinterpret_cast<float*>(b + L.q0);
  s.act = reinterpret_cast<uint32_t*>(b + L.act);
  s.fail = reinterpret_cast<uint32_t*>(b + L.fail);
  s.iters = reinterpret_cast<int32_t*>(b + L.iters);
  s.ok = reinterpret_cast<uint32_t*>(b + L.ok);
  s.FL = L.lanes;
  return s;
}

__global__ void __launch_bounds__(256) f32s_init(const DevCode c, const float* __restrict__ llr, int32_t F,
                                                 int32_t max_iter, F32S s) {
  __shared__ float tile[32][65];  // [frame][variable]
  const int n0 = blockIdx.x * 64, f0 = blockIdx.y * 32;
  const int N = c.N;
  for (int i = threadIdx.x; i < 32 * 64; i += blockDim.x) {
    const int fl = i >> 6, nl = i & 63;
    const int f = f0 + fl, n = n0 + nl;
    tile[fl][nl] = (f < F && n < N) ? llr[(size_t)f * N + n] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
    const int nl = i >> 5, fl = i & 31;
    const int n = n0 + nl;
    if (n >= N) continue;
    const size_t o = (size_t)n * s.FL + f0 + fl;
    const float q = tile[fl][nl];
    s.q0[o] = q;
    s.zb0[o] = q;  // Z^(0)
    s.zb1[o] = q;  // accumulates Z^(1)
  }
  if (blockIdx.x == 0) {
    for (int fl = threadIdx.x; fl < 32; fl += blockDim.x) {
      const int f = f0 + fl;
      s.act[s.FL + f] = f < F ? 1u : 0u;
      s.act[f] = 0u;
      s.fail[f] = 0u;
      s.fail[s.FL + f] = 0u;
      s.iters[f] = max_iter;
      s.ok[f] = 0u;
    }
  }
}

// One check of Eq. (3) for one frame, its variables read from the
// degree-sorted table (position j of internal check m at ell[j * M + m]):
// rebuild L^(k-1)_mn (from the Section V state (A, B, n~, signs) or the stored
// per-edge message), form u = Z^(k-1)_n - L^(k-1)_mn, take min1, min2, the
// first position of min1 and the sign parity, and add L^(k)_mn into Zn.  With
// D > 0 the degree is D and the loops are unrolled, so that the check's table
// and posterior loads are all in flight together; D = 0 takes the degree d.
// C8 (checks of degree <= 8): the state in 10 bytes per frame, the size of
// Section V's float form: {A, B} in St (uint2 entries) and n~ | signs << 8 in Sx.
template <int FORM, bool ES, int D, bool WIDE, bool C8 = false>
__device__ __forceinline__ uint32_t f32s_check_ell(const DevCode& c, const F32Rule& r, int m, int d, size_t FL,
                                                   const float* __restrict__ Zp, float* __restrict__ Zn,
                                                   uint4* __restrict__ St, uint16_t* __restrict__ Sx,
                                                   float* __restrict__ Lm) {
  static_assert(!C8 || (FORM == 1 && D <= 8), "the 10-byte state holds checks of degree <= 8");
  const int M = c.M;
  auto col = [&](int j) -> int {
    return WIDE ? __ldg(c.ell32 + (size_t)j * M + m) : (int)__ldg(c.ell16 + (size_t)j * M + m);
  };
  float A = 0.f, B = 0.f;
  int I = 0;
  uint32_t S = 0;
  if constexpr (FORM == 1 && C8) {
    const uint2 ab = reinterpret_cast<const uint2*>(St)[(size_t)m * FL];
    const uint32_t is = Sx[(size_t)m * FL];
    A = __uint_as_float(ab.x);
    B = __uint_as_float(ab.y);
    I = (int)(is & 0xffu);
    S = is >> 8;
  } else if constexpr (FORM == 1) {
    const uint4 st = St[(size_t)m * FL];
    A = __uint_as_float(st.x);
    B = __uint_as_float(st.y);
    I = (int)st.z;
    S = st.w;
  }
  float mn1 = __int_as_float(0x7f800000), mn2 = __int_as_float(0x7f800000);
  int idx = 0;
  uint32_t neg = 0, par = 0;
  auto take = [&](int j, int n) {
    const float z = Zp[(size_t)n * FL];
    float lold;
    if constexpr (FORM == 1) {
      const float mag = (j == I) ? B : A;
      lold = ((S >> j) & 1u) ? -mag : mag;
    } else {
      lold = Lm[((size_t)j * M + m) * FL];
    }
    if (ES) par ^= (z <= 0.0f) ? 1u : 0u;
    const float u = z - lold;
    neg |= (u < 0.0f ? 1u : 0u) << j;
    const float a = fabsf(u);
    if (a < mn1) { mn2 = mn1; mn1 = a; idx = j; }
    else if (a < mn2) { mn2 = a; }
  };
  constexpr int R = D > 0 ? D : 1;
  int nn[R];
  if constexpr (D > 0) {
#pragma unroll
    for (int j = 0; j < D; ++j) nn[j] = col(j);
#pragma unroll
    for (int j = 0; j < D; ++j) take(j, nn[j]);
  } else {
    for (int j = 0; j < d; ++j) take(j, col(j));
  }
  const int dd = D > 0 ? D : d;
  const uint32_t dm = dd >= 32 ? 0xffffffffu : ((1u << dd) - 1u);
  const uint32_t Sn = ((__popc(neg) & 1) ? ~neg : neg) & dm;
  const float An = r.g(mn1), Bn = r.g(mn2);
  auto emit = [&](int j, int n) {
    const float mag = (j == idx) ? Bn : An;
    const float l = ((Sn >> j) & 1u) ? -mag : mag;
    atomicAdd(Zn + (size_t)n * FL, l);
    if constexpr (FORM == 0) Lm[((size_t)j * M + m) * FL] = l;
  };
  if constexpr (D > 0) {
#pragma unroll
    for (int j = 0; j < D; ++j) emit(j, nn[j]);
  } else {
    for (int j = 0; j < d; ++j) emit(j, col(j));
  }
  if constexpr (FORM == 1 && C8) {
    reinterpret_cast<uint2*>(St)[(size_t)m * FL] = make_uint2(__float_as_uint(An), __float_as_uint(Bn));
    Sx[(size_t)m * FL] = (uint16_t)((uint32_t)idx | (Sn << 8));
  } else if constexpr (FORM == 1) {
    St[(size_t)m * FL] = make_uint4(__float_as_uint(An), __float_as_uint(Bn), (uint32_t)idx, Sn);
  }
  return par;
}

// Row pass of iteration k: one warp = kRowsPerWarp consecutive internal checks
// for 32 frames.  C8: the 10-byte state, {A, B} as [M][FL] uint2 followed by
// [M][FL] u16 {n~, signs} in the state region.
template <int FORM, bool ES, bool WIDE, bool C8 = false>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4) f32s_rows_ell(const DevCode c, const F32Rule r, F32S s,
                                                                         int k) {
  const int lane = threadIdx.x & 31;
  int chunk, m0;
  if (!row_map<FORM == 1 ? kChunksSV : kChunksF32PE>(blockIdx.x, blockIdx.y, threadIdx.x >> 5, c.M, s.FL, chunk, m0))
    return;
  const int f = chunk * 32 + lane;
  const int cur = k & 1;
  const bool active = s.act[cur * s.FL + f] != 0u;
  if (__all_sync(0xffffffffu, !active)) return;
  if (!active) return;  // a stopped frame's buffers stay as they are
  const size_t FL = (size_t)s.FL;
  const float* Zp = s.zb(k - 1) + f;
  float* Zn = s.zb(k) + f;
  uint4* St = C8 ? reinterpret_cast<uint4*>(reinterpret_cast<uint2*>(s.st) + f) : s.st + f;
  uint16_t* Sx = reinterpret_cast<uint16_t*>(reinterpret_cast<uint2*>(s.st) + (size_t)c.M * FL) + f;
  float* Lm = s.lm + f;
  uint32_t fail = 0;
  const int m1 = min(m0 + kRowsPerWarp, c.M);
  for (int m = m0; m < m1; ++m) {
    const int d = c.deg(m);
    if constexpr (C8) {
      switch (d) {
        case 6: fail |= f32s_check_ell<1, ES, 6, WIDE, true>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm); break;
        case 7: fail |= f32s_check_ell<1, ES, 7, WIDE, true>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm); break;
        default: fail |= f32s_check_ell<1, ES, 0, WIDE, true>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm); break;
      }
    } else if constexpr (FORM == 1) {
      switch (d) {
        case 6: fail |= f32s_check_ell<1, ES, 6, WIDE>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm); break;
        case 7: fail |= f32s_check_ell<1, ES, 7, WIDE>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm); break;
        case 14: fail |= f32s_check_ell<1, ES, 14, WIDE>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm); break;
        case 15: fail |= f32s_check_ell<1, ES, 15, WIDE>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm); break;
        default: fail |= f32s_check_ell<1, ES, 0, WIDE>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm); break;
      }
    } else {
      if (d == 6) fail |= f32s_check_ell<0, ES, 6, WIDE>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm);
      else if (d == 7) fail |= f32s_check_ell<0, ES, 7, WIDE>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm);
      else fail |= f32s_check_ell<0, ES, 0, WIDE>(c, r, m, d, FL, Zp, Zn, St, Sx, Lm);
    }
  }
  if (ES && fail) atomicOr(s.fail + cur * s.FL + f, 1u);
}

// The sum-product check rule on per-edge messages: for every position the
// product of the other inputs' signs times phi(sum over the other positions of
// phi(min(|u|, 30))), phi(x) = ln(1 + 2 / (e^x - 1)) = -ln tanh(x/2) (phi(0) =
// inf, phi(inf) = 0 fall out of the formula).  The sum over the other positions
// is the total minus the position's own term, except for the position with the
// largest term, whose sum of the others is accumulated separately (the
// subtraction would cancel there).
__device__ __forceinline__ float spa_phi(float x) { return log1pf(2.0f / expm1f(x)); }

template <bool ES>
__device__ __forceinline__ uint32_t f32s_check_spa(const DevCode& c, int m, size_t FL, const float* __restrict__ Zp,
                                                   float* __restrict__ Zn, float* __restrict__ Lm) {
  const int e0 = __ldg(c.rp + m);
  const int d = __ldg(c.rp + m + 1) - e0;
  float total = 0.0f, top = -1.0f, rest = 0.0f;
  int jtop = 0;
  uint32_t neg = 0, zero = 0, par = 0;
  for (int j = 0; j < d; ++j) {
    const int n = __ldg(c.ci + e0 + j);
    const float z = Zp[(size_t)n * FL];
    const float u = z - Lm[(size_t)(e0 + j) * FL];
    if (ES) par ^= (z <= 0.0f) ? 1u : 0u;
    neg |= (u < 0.0f ? 1u : 0u) << j;
    zero += (u == 0.0f) ? 1u : 0u;
    const float ph = spa_phi(fminf(fabsf(u), 30.0f));
    total += ph;
    if (ph > top) {
      if (top >= 0.0f) rest += top;
      top = ph;
      jtop = j;
    } else {
      rest += ph;
    }
  }
  const uint32_t par_neg = __popc(neg) & 1u;
  for (int j = 0; j < d; ++j) {
    const int n = __ldg(c.ci + e0 + j);
    float l;
    const float u = Zp[(size_t)n * FL] - Lm[(size_t)(e0 + j) * FL];
    // a zero input among the others makes the message zero
    if (zero > (u == 0.0f ? 1u : 0u)) {
      l = 0.0f;
    } else {
      const float others = (j == jtop) ? rest : total - spa_phi(fminf(fabsf(u), 30.0f));
      const float mag = spa_phi(others);
      l = ((par_neg ^ ((neg >> j) & 1u)) != 0u) ? -mag : mag;
    }
    atomicAdd(Zn + (size_t)n * FL, l);
    Lm[(size_t)(e0 + j) * FL] = l;
  }
  return par;
}

template <bool ES>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) f32s_rows_spa(const DevCode c, F32S s, int k) {
  const int lane = threadIdx.x & 31;
  int chunk, m0;
  if (!row_map<kChunksF32PE>(blockIdx.x, blockIdx.y, threadIdx.x >> 5, c.M, s.FL, chunk, m0)) return;
  const int f = chunk * 32 + lane;
  const int cur = k & 1;
  const bool active = s.act[cur * s.FL + f] != 0u;
  if (__all_sync(0xffffffffu, !active)) return;
  if (!active) return;
  const size_t FL = (size_t)s.FL;
  const float* Zp = s.zb(k - 1) + f;
  float* Zn = s.zb(k) + f;
  float* Lm = s.lm + f;
  uint32_t fail = 0;
  const int m1 = min(m0 + kRowsPerWarp, c.M);
  for (int m = m0; m < m1; ++m) fail |= f32s_check_spa<ES>(c, m, FL, Zp, Zn, Lm);
  if (ES && fail) atomicOr(s.fail + cur * s.FL + f, 1u);
}

// Column pass of iteration k: a frame whose Z^(k-1) satisfied every check
// (seen by the row pass) stops at k - 1 with its result in zb(k - 1); a frame
// that goes on has Z^(k) in zb(k), and zb(k - 1) is reset to Z0 to accumulate
// Z^(k+1) (skipped after the last iteration).  Four frames per thread: 16-byte
// accesses (a warp moves 512 bytes per variable); the frame count is a
// multiple of 32, so groups of 4 never straddle it.  Frame flags are advanced
// by the threads of the first variable slice.
template <bool ES>
__global__ void __launch_bounds__(256) f32s_cols(const DevCode c, F32S s, int k, int reset) {
  const int f0 = (blockIdx.y * 32 + (threadIdx.x & 31)) * 4;
  if (f0 >= s.FL) return;
  const int cur = k & 1, nxt = cur ^ 1;
  const uint4 act = *reinterpret_cast<const uint4*>(s.act + cur * s.FL + f0);
  uint4 fail = make_uint4(0u, 0u, 0u, 0u);
  if (ES) fail = *reinterpret_cast<const uint4*>(s.fail + cur * s.FL + f0);
  const uint4 stop = ES ? make_uint4(act.x & (fail.x ^ 1u), act.y & (fail.y ^ 1u), act.z & (fail.z ^ 1u),
                                     act.w & (fail.w ^ 1u))
                        : make_uint4(0u, 0u, 0u, 0u);
  const uint4 cont = make_uint4(act.x & ~stop.x, act.y & ~stop.y, act.z & ~stop.z, act.w & ~stop.w);
  const bool all = (cont.x & cont.y & cont.z & cont.w) != 0u;
  const bool any = (cont.x | cont.y | cont.z | cont.w) != 0u;
  if (reset && any) {
    float* Zo = s.zb(k - 1);
#pragma unroll 4
    for (int n = blockIdx.x * 8 + (threadIdx.x >> 5); n < c.N; n += gridDim.x * 8) {
      const size_t o = (size_t)n * s.FL + f0;
      const float4 q = *reinterpret_cast<const float4*>(s.q0 + o);
      if (all) {
        *reinterpret_cast<float4*>(Zo + o) = q;
      } else {
        if (cont.x) Zo[o] = q.x;
        if (cont.y) Zo[o + 1] = q.y;
        if (cont.z) Zo[o + 2] = q.z;
        if (cont.w) Zo[o + 3] = q.w;
      }
    }
  }
  if (blockIdx.x == 0) {
    *reinterpret_cast<uint4*>(s.act + nxt * s.FL + f0) = cont;
    *reinterpret_cast<uint4*>(s.fail + nxt * s.FL + f0) = make_uint4(0u, 0u, 0u, 0u);
    if (ES) {
      const uint32_t st[4] = {stop.x, stop.y, stop.z, stop.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (st[q]) {
          s.iters[f0 + q] = k - 1;
          s.ok[f0 + q] = 1u;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32) f32s_final_syndrome(const DevCode c, F32S s, int kf) {
  const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  int chunk, m0;
  if (!row_map_all(warp, c.M, s.FL, chunk, m0)) return;
  const int f = chunk * 32 + lane;
  const int cur = kf & 1;
  const bool active = s.act[cur * s.FL + f] != 0u;
  if (__all_sync(0xffffffffu, !active)) return;
  if (!active) return;
  const float* Z = s.zb(kf - 1) + f;  // Z^(max_iter) of every frame still running
  uint32_t fail = 0;
  const int m1 = min(m0 + kRowsPerWarp, c.M);
  for (int m = m0; m < m1; ++m) {
    uint32_t y = 0;
    for (int e = __ldg(c.rp + m); e < __ldg(c.rp + m + 1); ++e)
      y ^= (Z[(size_t)__ldg(c.ci + e) * s.FL] <= 0.0f) ? 1u : 0u;
    fail |= y;
  }
  if (fail) atomicOr(s.fail + cur * s.FL + f, 1u);
}

__global__ void __launch_bounds__(256) f32s_output(const DevCode c, F32S s, int kf, int32_t F, uint8_t* bits,
                                                   int32_t* iters, uint8_t* okf, float* zout) {
  __shared__ float tile[64][33];  // [variable][frame]
  const int n0 = blockIdx.x * 64, f0 = blockIdx.y * 32;
  const int N = c.N, N8 = (N + 7) >> 3;
  {
    // every thread handles one frame (threadIdx.x & 31) of the tile: the frame's
    // result is the buffer of its iteration count
    const int fl = threadIdx.x & 31;
    const float* Z = s.zb(s.iters[f0 + fl]) + f0 + fl;
    for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
      const int nl = i >> 5;
      const int n = n0 + nl;
      tile[nl][fl] = n < N ? Z[(size_t)n * s.FL] : 0.0f;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * 8; i += blockDim.x) {
    const int fl = i >> 3, bl = i & 7;
    const int f = f0 + fl, b = (n0 >> 3) + bl;
    if (f >= F || b >= N8) continue;
    uint32_t byte = 0;
    for (int t = 0; t < 8; ++t) {
      const int nl = bl * 8 + t;
      if (n0 + nl < N) byte |= (tile[nl][fl] <= 0.0f ? 1u : 0u) << t;
    }
    bits[(size_t)f * N8 + b] = (uint8_t)byte;
  }
  if (zout != nullptr) {
    for (int i = threadIdx.x; i < 32 * 64; i += blockDim.x) {
      const int fl = i >> 6, nl = i & 63;
      const int f = f0 + fl, n = n0 + nl;
      if (f < F && n < N) zout[(size_t)f * N + n] = tile[nl][fl];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    const int f = f0 + threadIdx.x;
    if (f < F) {
      const int cur = kf & 1;
      const bool running = s.act[cur * s.FL + f] != 0u;
      iters[f] = s.iters[f];
      okf[f] = running ? (uint8_t)(s.fail[cur * s.FL + f] ^ 1u) : (uint8_t)s.ok[f];
    }
  }
}

template <int FORM, bool ES>
cudaError_t f32s_run(const DevCode& c, const F32Rule& r, const StreamLayout& L, F32S s, int sm_count,
                     int32_t max_iter, cudaStream_t st) {
  // row passes on 2-D grids of chunk groups (Section V form and per-edge form
  // group sizes differ)
  const RowGrid g2 = rows_grid_g(c.M, L.lanes, FORM == 1 ? kChunksSV : kChunksF32PE);
  const dim3 rgrid((unsigned)g2.x, (unsigned)g2.y);
  const int gy4 = (L.lanes / 4 + 31) / 32;  // groups of 32 threads x 4 frames
  const dim3 cgrid((unsigned)std::max(1, std::min((c.N + 7) / 8, 4 * sm_count * 32 / gy4)), (unsigned)gy4);
  const bool wide = c.ell16 == nullptr;
  const bool c8 = c.ell_w <= 8;  // every check of degree <= 8: the 10-byte Section V state
  for (int k = 1; k <= max_iter; ++k) {
    if (FORM == 0 && r.rule == 3) f32s_rows_spa<ES><<<rgrid, kWarpsPerBlock * 32, 0, st>>>(c, s, k);
    else if (FORM == 1 && c8 && wide) f32s_rows_ell<1, ES, true, true><<<rgrid, kWarpsPerBlock * 32, 0, st>>>(c, r, s, k);
    else if (FORM == 1 && c8) f32s_rows_ell<1, ES, false, true><<<rgrid, kWarpsPerBlock * 32, 0, st>>>(c, r, s, k);
    else if (wide) f32s_rows_ell<FORM, ES, true><<<rgrid, kWarpsPerBlock * 32, 0, st>>>(c, r, s, k);
    else f32s_rows_ell<FORM, ES, false><<<rgrid, kWarpsPerBlock * 32, 0, st>>>(c, r, s, k);
    f32s_cols<ES><<<cgrid, 256, 0, st>>>(c, s, k, k < max_iter ? 1 : 0);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t stream_f32_decode(const DevCode& c, const F32Rule& r, int form, const StreamLayout& L, void* ws,
                              int sm_count, const float* llr, int32_t F, int32_t max_iter, int32_t early_stop,
                              uint8_t* bits, int32_t* iters, uint8_t* ok, float* zout, cudaStream_t st) {
  F32S s = f32s_view(ws, L);
  const dim3 tgrid((c.N + 63) / 64, L.lanes / 32);
  cudaError_t e0 = cudaMemsetAsync(static_cast<char*>(ws) + L.st, 0, L.q0 - L.st, st);  // L^(0) = 0
  if (e0 != cudaSuccess) return e0;
  f32s_init<<<tgrid, 256, 0, st>>>(c, llr, F, max_iter, s);
  cudaError_t e;
  const bool es = early_stop != 0;
  if (form == 1) e = es ? f32s_run<1, true>(c, r, L, s, sm_count, max_iter, st)
                        : f32s_run<1, false>(c, r, L, s, sm_count, max_iter, st);
  else e = es ? f32s_run<0, true>(c, r, L, s, sm_count, max_iter, st)
              : f32s_run<0, false>(c, r, L, s, sm_count, max_iter, st);
  if (e != cudaSuccess) return e;
  const int kf = max_iter + 1;
  f32s_final_syndrome<<<rows_grid(c.M, L.lanes), kWarpsPerBlock * 32, 0, st>>>(c, s, kf);
  f32s_output<<<tgrid, 256, 0, st>>>(c, s, kf, F, bits, iters, ok, zout);
  return cudaGetLastError();
}

}  // namespace ldpc
