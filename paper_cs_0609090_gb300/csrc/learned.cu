// learned.cu -- offset min-sum with learned per-iteration, per-check-degree
// offsets: float32 forward with checkpoints, hand-written adjoint (backward),
// BCE loss, Adam, and the device AWGN generator used to train it.
//
// The decoder is the Section V single scan with the offset rule of Section III
// (|L| <- max(|L| - beta, 0)), where beta depends on the iteration k and on the
// degree class of the check: beta[k][class(m)].
//
// Workspace (lane = frame, FL = frames padded to 32, index [.][FL] innermost):
//   zck  (K+1) x [N][FL] f32   Z^(0) .. Z^(K) posteriors (checkpoints)
//   sck   K    x [M][FL] uint4 Section V state after iteration k: {A, B, n~, signs}
//                              (checks in the degree-sorted internal order, as
//                              in du; their variables from the sorted table)
//   (no accumulator: the forward's row pass of iteration k adds its messages
//    into zck[k], which holds Z^(0) beforehand, so that it ends as Z^(k))
//   dz    2 x [N][FL] f32      gradient w.r.t. Z^(k) (ping-pong)
//   du    2 x [M][FL] uint4    per check: {n~, second-min position, dU at n~,
//                              dU at second} -- the only nonzero entries of
//                              dLoss/du for the check (ping-pong)
//   part  [tasks][C] f32       per-task partial sums of dLoss/dbeta (summed in a
//                              fixed order: the gradient is deterministic)
//   lpart [blocks] f32         per-block partial sums of the loss; also the
//                              staged class sums of the offset gradient
//
// Backward through iteration k (the forward quantities are recomputed from the
// checkpoints Z^(k-1), S^(k-1) rather than stored):
//   u_j = Z^(k-1)_{n_j} - L^(k-1)_{mj};  min1 = |u_a|, min2 = |u_b| (a: first
//   argmin, b: position of the second smallest (|u|, j));  A = relu(min1 - beta),
//   B = relu(min2 - beta);  L^(k)_j = s_j (j == a ? B : A).
//   G_j = dLoss/dL^(k)_j = dZ^(k)_{n_j} - dU^(k+1)_j  (Z^(k) = Z0 + sum L^(k) and
//   u^(k+1) = Z^(k) - L^(k)).  dA = sum_{j != a} G_j s_j, dB = G_a s_a;
//   gA = dA [min1 > beta], gB = dB [min2 > beta];  dLoss/dbeta -= gA + gB;
//   dU_a = gA sgn(u_a), dU_b = gB sgn(u_b) (sgn(0) = +1; subgradient with the
//   lowest-position tie-break);  dZ^(k-1)_{n_a} += dU_a, dZ^(k-1)_{n_b} += dU_b.
#include <algorithm>
#include <cmath>

#include "kernels.h"
#include "stream_grid.h"

namespace ldpc {
namespace {

constexpr int kLRows = kRowsPerWarp;    // checks per warp task
constexpr int kLWarps = kWarpsPerBlock;  // warps per block

inline size_t lal(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

LearnedLayout learned_layout(int N, int M, int K, int C, int F) {
  LearnedLayout L;
  const size_t FL = (size_t)((F + 31) / 32) * 32;
  L.FL = (int)FL;
  L.tasks = (int)(((size_t)(M + kLRows - 1) / kLRows) * (FL / 32));
  size_t off = 0;
  L.zck = off;   off = lal(off + (size_t)(K + 1) * N * FL * 4);
  L.sck = off;   off = lal(off + (size_t)std::max(K, 1) * M * FL * 16);
  L.dz = off;    off = lal(off + 2 * (size_t)N * FL * 4);
  L.du = off;    off = lal(off + 2 * (size_t)M * FL * 16);
  L.part = off;  off = lal(off + (size_t)L.tasks * C * 4);
  L.lpart = off; off = lal(off + (size_t)4096 * 4);
  L.total = off;
  return L;
}

namespace {

struct LView {
  int N, M, K, C, FL;
  float* zck;
  uint4* sck;
  float* dz;
  uint4* du;
  float* part;
  float* lpart;
  __host__ __device__ __forceinline__ float* z(int k) const { return zck + (size_t)k * N * FL; }
  __host__ __device__ __forceinline__ uint4* s(int k) const { return sck + (size_t)(k - 1) * M * FL; }  // k >= 1
  __host__ __device__ __forceinline__ float* dzb(int i) const { return dz + (size_t)i * N * FL; }
  __host__ __device__ __forceinline__ uint4* dub(int i) const { return du + (size_t)i * M * FL; }
};

LView lview(void* ws, const LearnedLayout& L, int N, int M, int K, int C) {
  char* b = static_cast<char*>(ws);
  LView v;
  v.N = N; v.M = M; v.K = K; v.C = C; v.FL = L.FL;
  v.zck = reinterpret_cast<float*>(b + L.zck);
  v.sck = reinterpret_cast<uint4*>(b + L.sck);
  v.dz = reinterpret_cast<float*>(b + L.dz);
  v.du = reinterpret_cast<uint4*>(b + L.du);
  v.part = reinterpret_cast<float*>(b + L.part);
  v.lpart = reinterpret_cast<float*>(b + L.lpart);
  return v;
}

// frame-major [F][N] <-> lane-interleaved [N][FL] through 32 x 64 tiles
__global__ void __launch_bounds__(256) to_lanes(const float* __restrict__ src, int F, int N, int FL,
                                                float* __restrict__ dst0, float* __restrict__ dst1) {
  __shared__ float tile[32][65];
  const int n0 = blockIdx.x * 64, f0 = blockIdx.y * 32;
  for (int i = threadIdx.x; i < 32 * 64; i += blockDim.x) {
    const int fl = i >> 6, nl = i & 63;
    const int f = f0 + fl, n = n0 + nl;
    tile[fl][nl] = (f < F && n < N) ? src[(size_t)f * N + n] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
    const int nl = i >> 5, fl = i & 31;
    const int n = n0 + nl;
    if (n >= N) continue;
    const size_t o = (size_t)n * FL + f0 + fl;
    dst0[o] = tile[fl][nl];
    if (dst1 != nullptr) dst1[o] = tile[fl][nl];
  }
}

__global__ void __launch_bounds__(256) from_lanes(const float* __restrict__ src, int F, int N, int FL,
                                                  float* __restrict__ dst) {
  __shared__ float tile[64][33];
  const int n0 = blockIdx.x * 64, f0 = blockIdx.y * 32;
  for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
    const int nl = i >> 5, fl = i & 31;
    const int n = n0 + nl;
    tile[nl][fl] = n < N ? src[(size_t)n * FL + f0 + fl] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * 64; i += blockDim.x) {
    const int fl = i >> 6, nl = i & 63;
    const int f = f0 + fl, n = n0 + nl;
    if (f < F && n < N) dst[(size_t)f * N + n] = tile[nl][fl];
  }
}

// Forward iteration k: Eq. (3) with the Section V state and beta[k][class].
// Degree class of internal check i: the checks are sorted by degree and the
// classes are the distinct degrees in ascending order, so the class is the
// index of the degree run the check falls in (at most 4 classes).
__device__ __forceinline__ int check_class(const DevCode& c, int i) {
  int r = 0;
#pragma unroll
  for (int q = 1; q < 4; ++q)
    if (q < c.n_dc && i >= c.dc_end[q - 1]) r = q;
  return r;
}

// Forward of internal check i for one frame (lane-offset pointers): Eq. (3)
// with the Section V state and the offset bt, its variables from the
// degree-sorted table (positions in row order).  D > 0: exactly D positions,
// unrolled so that the check's loads are in flight together; D = 0: d.
template <int D, bool WIDE>
__device__ __forceinline__ void lf_check(const DevCode& c, int i, int d, float bt, size_t FL,
                                         const float* __restrict__ zp, float* __restrict__ acc,
                                         const uint4* __restrict__ sp, uint4* __restrict__ sn) {
  const int M = c.M;
  auto col = [&](int j) -> int {
    return WIDE ? __ldg(c.ell32 + (size_t)j * M + i) : (int)__ldg(c.ell16 + (size_t)j * M + i);
  };
  float A = 0.f, B = 0.f;
  int I = 0;
  uint32_t S = 0;
  if (sp != nullptr) {
    const uint4 st = sp[(size_t)i * FL];
    A = __uint_as_float(st.x); B = __uint_as_float(st.y); I = (int)st.z; S = st.w;
  }
  float mn1 = INFINITY, mn2 = INFINITY;
  int idx = 0;
  uint32_t neg = 0;
  auto take = [&](int j, int n) {
    const float z = zp[(size_t)n * FL];
    const float mag = (j == I) ? B : A;
    const float u = z - (((S >> j) & 1u) ? -mag : mag);
    neg |= (u < 0.0f ? 1u : 0u) << j;
    const float x = fabsf(u);
    if (x < mn1) { mn2 = mn1; mn1 = x; idx = j; }
    else if (x < mn2) { mn2 = x; }
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
  const float An = fmaxf(mn1 - bt, 0.0f), Bn = fmaxf(mn2 - bt, 0.0f);
  auto emit = [&](int j, int n) {
    const float mag = (j == idx) ? Bn : An;
    atomicAdd(acc + (size_t)n * FL, ((Sn >> j) & 1u) ? -mag : mag);
  };
  if constexpr (D > 0) {
#pragma unroll
    for (int j = 0; j < D; ++j) emit(j, nn[j]);
  } else {
    for (int j = 0; j < d; ++j) emit(j, col(j));
  }
  sn[(size_t)i * FL] = make_uint4(__float_as_uint(An), __float_as_uint(Bn), (uint32_t)idx, Sn);
}

// Forward iteration k: Eq. (3) with the Section V state and beta[k][class].
// One warp = kLRows internal checks for one chunk of 32 frames, chunk-major (a
// 2-D grid, blockIdx.y = chunk): the checkpoint lines the warps in flight
// gather stay in L2.
template <bool WIDE>
__global__ void __launch_bounds__(kLWarps * 32, 4) lf_rows(const DevCode c, const float* __restrict__ beta, LView v,
                                                           int k) {
  const int lane = threadIdx.x & 31;
  int chunk, m0;
  if (!row_map<1>(blockIdx.x, blockIdx.y, threadIdx.x >> 5, c.M, v.FL, chunk, m0)) return;
  const int f = chunk * 32 + lane;
  const size_t FL = (size_t)v.FL;
  const float* zp = v.z(k - 1) + f;
  float* acc = v.z(k) + f;  // holds Z^(0); Z^(k) after the pass
  const uint4* sp = k > 1 ? v.s(k - 1) + f : nullptr;
  uint4* sn = v.s(k) + f;
  const int m1 = min(m0 + kLRows, c.M);
  for (int i = m0; i < m1; ++i) {
    const int d = c.deg(i);
    const float bt = __ldg(beta + (size_t)(k - 1) * v.C + check_class(c, i));
    switch (d) {
      case 6: lf_check<6, WIDE>(c, i, d, bt, FL, zp, acc, sp, sn); break;
      case 7: lf_check<7, WIDE>(c, i, d, bt, FL, zp, acc, sp, sn); break;
      case 14: lf_check<14, WIDE>(c, i, d, bt, FL, zp, acc, sp, sn); break;
      case 15: lf_check<15, WIDE>(c, i, d, bt, FL, zp, acc, sp, sn); break;
      default: lf_check<0, WIDE>(c, i, d, bt, FL, zp, acc, sp, sn); break;
    }
  }
}

// Z^(0) into checkpoint k, where the row pass of iteration k accumulates Z^(k).
__global__ void __launch_bounds__(256) lf_init(LView v, int k) {
  const size_t total = (size_t)v.N * v.FL;
  float4* zk = reinterpret_cast<float4*>(v.z(k));
  const float4* z0 = reinterpret_cast<const float4*>(v.z(0));
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total / 4; i += (size_t)gridDim.x * blockDim.x)
    zk[i] = z0[i];
}

__device__ __forceinline__ float warp_sum(float x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Backward of internal check i through iteration k for one frame (see the
// file comment; lane-offset pointers).  Returns the check's dLoss/dbeta.
template <int D, bool WIDE>
__device__ __forceinline__ float lb_check(const DevCode& c, int i, int d, float bt, bool live, size_t FL,
                                          const float* __restrict__ zp, const uint4* __restrict__ sp,
                                          const float* __restrict__ dzk, const uint4* __restrict__ dun,
                                          uint4* __restrict__ duc, float* __restrict__ dzp) {
  const int M = c.M;
  auto col = [&](int j) -> int {
    return WIDE ? __ldg(c.ell32 + (size_t)j * M + i) : (int)__ldg(c.ell16 + (size_t)j * M + i);
  };
  float A = 0.f, B = 0.f;
  int I = 0;
  uint32_t S = 0;
  if (sp != nullptr) {
    const uint4 st = sp[(size_t)i * FL];
    A = __uint_as_float(st.x); B = __uint_as_float(st.y); I = (int)st.z; S = st.w;
  }
  // recompute the forward row reduction
  float mn1 = INFINITY, mn2 = INFINITY, u1 = 0.f, u2 = 0.f;
  int a = 0, b = 1;
  uint32_t neg = 0;
  auto take = [&](int j, int n) {
    const float z = zp[(size_t)n * FL];
    const float mag = (j == I) ? B : A;
    const float u = z - (((S >> j) & 1u) ? -mag : mag);
    neg |= (u < 0.0f ? 1u : 0u) << j;
    const float x = fabsf(u);
    if (x < mn1) { mn2 = mn1; u2 = u1; b = a; mn1 = x; u1 = u; a = j; }
    else if (x < mn2) { mn2 = x; u2 = u; b = j; }
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
  const uint32_t sgnw = ((__popc(neg) & 1) ? ~neg : neg);  // bit j set: L^(k)_j negative
  // sparse dLoss/du^(k+1) of this check
  uint32_t na = 0xffffffffu, nb = 0xffffffffu;
  float da = 0.f, db = 0.f;
  if (dun != nullptr) {
    const uint4 t = dun[(size_t)i * FL];
    na = t.x; nb = t.y; da = __uint_as_float(t.z); db = __uint_as_float(t.w);
  }
  float dA = 0.f, dB = 0.f;
  auto grad = [&](int j, int n) {
    float G = dzk[(size_t)n * FL];
    if ((uint32_t)j == na) G -= da;
    if ((uint32_t)j == nb) G -= db;
    const float sG = ((sgnw >> j) & 1u) ? -G : G;
    if (j == a) dB += sG; else dA += sG;
  };
  // (the columns are loaded again rather than kept: keeping them spills at 4 CTAs
  // per SM, and 3 CTAs per SM measured slower)
#pragma unroll
  for (int j = 0; j < (D > 0 ? D : d); ++j) grad(j, col(j));
  const float gA = (mn1 > bt) ? dA : 0.0f;
  const float gB = (mn2 > bt) ? dB : 0.0f;
  const float dua = live ? gA * (u1 < 0.0f ? -1.0f : 1.0f) : 0.0f;
  const float dub = live ? gB * (u2 < 0.0f ? -1.0f : 1.0f) : 0.0f;
  duc[(size_t)i * FL] = make_uint4((uint32_t)a, (uint32_t)b, __float_as_uint(dua), __float_as_uint(dub));
  if (dua != 0.0f) atomicAdd(dzp + (size_t)col(a) * FL, dua);
  if (dub != 0.0f) atomicAdd(dzp + (size_t)col(b) * FL, dub);
  return live ? -(gA + gB) : 0.0f;
}

// Backward through iteration k (see the file comment).  dzk: dLoss/dZ^(k);
// dun: sparse dLoss/du^(k+1) of every check (nullptr when k == K); writes duc
// (dLoss/du^(k)), adds into dzp (dLoss/dZ^(k-1)) and one partial dLoss/dbeta per
// (task, class).  Same warp order and check bodies as the forward.
template <bool WIDE>
__global__ void __launch_bounds__(kLWarps * 32, 4) lb_rows(const DevCode c, const float* __restrict__ beta, LView v,
                                                           int k, const float* __restrict__ dzk,
                                                           const uint4* __restrict__ dun, uint4* __restrict__ duc,
                                                           float* __restrict__ dzp, int F) {
  const int lane = threadIdx.x & 31;
  int chunk, m0;
  if (!row_map<1>(blockIdx.x, blockIdx.y, threadIdx.x >> 5, c.M, v.FL, chunk, m0)) return;
  const int f = chunk * 32 + lane;
  // task = (chunk, check group): one row of partial offset gradients each
  const size_t task = (size_t)chunk * ((c.M + kLRows - 1) / kLRows) + m0 / kLRows;
  const bool live = f < F;
  const size_t FL = (size_t)v.FL;
  const float* zp = v.z(k - 1) + f;
  const uint4* sp = k > 1 ? v.s(k - 1) + f : nullptr;
  dzk += f;
  if (dun != nullptr) dun += f;
  duc += f;
  dzp += f;
  float gpart[4] = {0.f, 0.f, 0.f, 0.f};  // per class, up to 4 classes in registers
  const int m1 = min(m0 + kLRows, c.M);
  for (int i = m0; i < m1; ++i) {
    const int d = c.deg(i);
    const int cls = check_class(c, i);
    const float bt = __ldg(beta + (size_t)(k - 1) * v.C + cls);
    float g;
    switch (d) {
      case 6: g = lb_check<6, WIDE>(c, i, d, bt, live, FL, zp, sp, dzk, dun, duc, dzp); break;
      case 7: g = lb_check<7, WIDE>(c, i, d, bt, live, FL, zp, sp, dzk, dun, duc, dzp); break;
      case 14: g = lb_check<14, WIDE>(c, i, d, bt, live, FL, zp, sp, dzk, dun, duc, dzp); break;
      case 15: g = lb_check<15, WIDE>(c, i, d, bt, live, FL, zp, sp, dzk, dun, duc, dzp); break;
      default: g = lb_check<0, WIDE>(c, i, d, bt, live, FL, zp, sp, dzk, dun, duc, dzp); break;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) gpart[q] += (cls == q) ? g : 0.0f;
  }
  float* prow = v.part + task * v.C;
  for (int q = 0; q < v.C && q < 4; ++q) {
    const float s = warp_sum(gpart[q]);
    if (lane == 0) prow[q] = s;
  }
}

// dbeta[k-1][c] = sum over tasks of part[task][c], in a fixed order: block b
// sums the tasks [b T / nb, (b+1) T / nb) of every class into stage[b][c]
// (lb_reduce1), then one block sums stage[0..nb) (lb_reduce2).  The partition
// and both in-block trees are fixed, so the result does not depend on timing.
constexpr int kReduceBlocks = 256;

__device__ __forceinline__ float block_sum(float s, float* sm) {
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  const float r = sm[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) lb_reduce1(const float* __restrict__ part, int tasks, int C,
                                                  float* __restrict__ stage) {
  __shared__ float sm[256];
  const int t0 = (int)((int64_t)tasks * blockIdx.x / gridDim.x);
  const int t1 = (int)((int64_t)tasks * (blockIdx.x + 1) / gridDim.x);
  for (int cls = 0; cls < C; ++cls) {
    float s = 0.f;
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) s += part[(size_t)t * C + cls];
    s = block_sum(s, sm);
    if (threadIdx.x == 0) stage[blockIdx.x * C + cls] = s;
  }
}

__global__ void __launch_bounds__(256) lb_reduce2(const float* __restrict__ stage, int nb, int C,
                                                  float* __restrict__ out) {
  __shared__ float sm[256];
  for (int cls = 0; cls < C; ++cls) {
    float s = 0.f;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += stage[b * C + cls];
    s = block_sum(s, sm);
    if (threadIdx.x == 0) out[cls] = s;
  }
}

__global__ void __launch_bounds__(256) zero_f(float* __restrict__ p, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = 0.0f;
}

// Mean binary cross-entropy of the soft decisions sigma(-Z^(K)) (probability of
// bit 1) against the transmitted bits, and its gradient w.r.t. Z^(K):
//   loss = softplus(-Z) for bit 0, softplus(Z) for bit 1;  d/dZ = sigma(Z) - 1
//   for bit 0, sigma(Z) for bit 1; both divided by F N.
__global__ void __launch_bounds__(256) bce_kernel(LView v, int F, const uint8_t* __restrict__ tbits,
                                                  float* __restrict__ lpart, float* __restrict__ dzk) {
  __shared__ float sm[256];
  const int N = v.N, N8 = (N + 7) >> 3;
  const float scale = 1.0f / ((float)F * (float)N);
  const float* zk = v.z(v.K);
  float acc = 0.f;
  const size_t total = (size_t)N * v.FL;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(i / v.FL), f = (int)(i % v.FL);
    float g = 0.f;
    if (f < F) {
      const float z = zk[i];
      const int t = tbits != nullptr ? (tbits[(size_t)f * N8 + (n >> 3)] >> (n & 7)) & 1 : 0;
      const float x = t ? z : -z;  // loss = softplus(x)
      acc += fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x)));
      const float sz = 1.0f / (1.0f + expf(-z));
      g = (t ? sz : sz - 1.0f) * scale;
    }
    if (dzk != nullptr) dzk[i] = g;
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(256) bce_reduce(const float* __restrict__ lpart, int nb, float scale,
                                                  float* __restrict__ out) {
  __shared__ float sm[256];
  float s = 0.f;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) s += lpart[t];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0] * scale;
}

// Adam (Kingma & Ba, 2015) with bias-corrected moments.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------- AWGN frames

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC 2011): 10 rounds of two 32x32->64 multiplies on a 4-word
// counter with a 2-word key bumped by the Weyl constants after each round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, ctr.x), lo0 = 0xD2511F53u * ctr.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, ctr.z), lo1 = 0xCD9E8D57u * ctr.z;
    ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    key.x += 0x9E3779B9u;
    key.y += 0xBB67AE85u;
  }
  return ctr;
}

// uniform in (0, 1]: the top 24 bits plus one, times 2^-24 (exact in float)
__device__ __forceinline__ float u01(uint32_t w) { return ((float)(w >> 8) + 1.0f) * (1.0f / 16777216.0f); }

// Frame f, variables 4c..4c+3 use counter (4c/4 = c, f_lo, f_hi, 0); the frame's
// Eb/N0 uses counter (0xffffffff, f_lo, f_hi, 1).  Two Box-Muller pairs per
// counter.  y = (1 - 2x) + sigma xi, LLR = 2 y / sigma^2,
// sigma^2 = 1 / (2 R 10^(EbN0/10)).
__global__ void __launch_bounds__(256) awgn_kernel(int N, uint64_t seed, uint64_t first_frame, int F, float lo,
                                                   float hi, float rate, const uint8_t* __restrict__ cw,
                                                   float* __restrict__ llr, float* __restrict__ ebn0_out) {
  for (int f = blockIdx.y; f < F; f += gridDim.y) {
  const uint64_t fr = first_frame + (uint64_t)f;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 ue = philox4x32_10(make_uint4(0xffffffffu, (uint32_t)fr, (uint32_t)(fr >> 32), 1u), key);
  const float eb = lo + (hi - lo) * (u01(ue.x) - 1.0f / 16777216.0f);
  if (ebn0_out != nullptr && blockIdx.x == 0 && threadIdx.x == 0) ebn0_out[f] = eb;
  const float s2 = 1.0f / (2.0f * rate * exp10f(eb / 10.0f));
  const float sg = sqrtf(s2);
  const int N8 = (N + 7) >> 3;
  const int groups = (N + 3) / 4;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)fr, (uint32_t)(fr >> 32), 0u), key);
    const float r0 = sqrtf(-2.0f * logf(u01(w.x))), r1 = sqrtf(-2.0f * logf(u01(w.z)));
    float s0, c0, s1, c1;
    sincosf(6.28318530717958647692f * u01(w.y), &s0, &c0);
    sincosf(6.28318530717958647692f * u01(w.w), &s1, &c1);
    const float xi[4] = {r0 * c0, r0 * s0, r1 * c1, r1 * s1};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int n = 4 * g + t;
      if (n >= N) break;
      const int bit = cw != nullptr ? (cw[(size_t)f * N8 + (n >> 3)] >> (n & 7)) & 1 : 0;
      const float y = (bit ? -1.0f : 1.0f) + sg * xi[t];
      llr[(size_t)f * N + n] = 2.0f * y / s2;
    }
  }
  }
}

// q = clamp(round_half_away(llr / delta), -qc, qc)
__global__ void __launch_bounds__(256) quantize_kernel(const float* __restrict__ llr, size_t n, float delta, int qc,
                                                       int8_t* __restrict__ q) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float x = llr[i] / delta;
    float r = truncf(fabsf(x) + 0.5f);
    r = fminf(r, (float)qc);
    q[i] = (int8_t)(x < 0.0f ? -r : r);
  }
}

dim3 rows_blocks(int M, int FL) {
  const RowGrid g = rows_grid_g(M, FL, 1);
  return dim3((unsigned)g.x, (unsigned)g.y);
}

}  // namespace

cudaError_t learned_forward(const DevCode& c, int C, int K, const float* beta, const LearnedLayout& L, void* ws,
                            const float* llr, int F, float* zout, cudaStream_t st) {
  LView v = lview(ws, L, c.N, c.M, K, C);
  const dim3 tg((c.N + 63) / 64, L.FL / 32);
  to_lanes<<<tg, 256, 0, st>>>(llr, F, c.N, L.FL, v.z(0), K >= 1 ? v.z(1) : nullptr);
  const dim3 rb = rows_blocks(c.M, L.FL);
  const int cb = (int)std::min<size_t>(((size_t)c.N * L.FL + 255) / 256, 8192);
  const bool wide = c.ell16 == nullptr;
  for (int k = 1; k <= K; ++k) {
    if (wide) lf_rows<true><<<rb, kLWarps * 32, 0, st>>>(c, beta, v, k);
    else lf_rows<false><<<rb, kLWarps * 32, 0, st>>>(c, beta, v, k);
    if (k < K) lf_init<<<cb, 256, 0, st>>>(v, k + 1);
  }
  if (zout != nullptr) from_lanes<<<tg, 256, 0, st>>>(v.z(K), F, c.N, L.FL, zout);
  return cudaGetLastError();
}

cudaError_t learned_bce(const DevCode& c, int C, int K, const LearnedLayout& L, void* ws, int F,
                        const uint8_t* tbits, float* loss, bool want_grad, cudaStream_t st) {
  LView v = lview(ws, L, c.N, c.M, K, C);
  const int nb = 1024;
  bce_kernel<<<nb, 256, 0, st>>>(v, F, tbits, v.lpart, want_grad ? v.dzb(K & 1) : nullptr);
  bce_reduce<<<1, 256, 0, st>>>(v.lpart, nb, 1.0f / ((float)F * (float)c.N), loss);
  return cudaGetLastError();
}

cudaError_t learned_backward(const DevCode& c, int C, int K, const float* beta, const LearnedLayout& L, void* ws,
                             const float* dz_in, int F, float* dbeta, cudaStream_t st) {
  LView v = lview(ws, L, c.N, c.M, K, C);
  const size_t nfl = (size_t)c.N * L.FL;
  if (dz_in != nullptr) {
    const dim3 tg((c.N + 63) / 64, L.FL / 32);
    to_lanes<<<tg, 256, 0, st>>>(dz_in, F, c.N, L.FL, v.dzb(K & 1), nullptr);
  }
  const dim3 rb = rows_blocks(c.M, L.FL);
  const int zb = (int)std::min<size_t>((nfl + 255) / 256, 8192);
  for (int k = K; k >= 1; --k) {
    float* dzk = v.dzb(k & 1);
    float* dzp = v.dzb((k - 1) & 1);
    zero_f<<<zb, 256, 0, st>>>(dzp, nfl);
    const uint4* dun = (k == K) ? nullptr : v.dub((k + 1) & 1);
    uint4* duc = v.dub(k & 1);
    if (c.ell16 == nullptr) lb_rows<true><<<rb, kLWarps * 32, 0, st>>>(c, beta, v, k, dzk, dun, duc, dzp, F);
    else lb_rows<false><<<rb, kLWarps * 32, 0, st>>>(c, beta, v, k, dzk, dun, duc, dzp, F);
    // stage partials in the loss-partials buffer (4096 floats >= kReduceBlocks * C)
    lb_reduce1<<<kReduceBlocks, 256, 0, st>>>(v.part, L.tasks, C, v.lpart);
    lb_reduce2<<<1, 256, 0, st>>>(v.lpart, kReduceBlocks, C, dbeta + (size_t)(k - 1) * C);
  }
  return cudaGetLastError();
}

cudaError_t adam_step(float* p, const float* g, float* m, float* v, int n, int step, float lr, float b1, float b2,
                      float eps, cudaStream_t st) {
  const float c1 = 1.0f - std::pow(b1, (float)step), c2 = 1.0f - std::pow(b2, (float)step);
  adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t awgn_llr(int N, uint64_t seed, uint64_t first_frame, int F, float lo, float hi, float rate,
                     const uint8_t* cw, float* llr, float* ebn0_out, cudaStream_t st) {
  const int groups = (N + 3) / 4;
  const dim3 grid((unsigned)std::min(64, (groups + 255) / 256), (unsigned)std::min(F, 32768));
  awgn_kernel<<<grid, 256, 0, st>>>(N, seed, first_frame, F, lo, hi, rate, cw, llr, ebn0_out);
  return cudaGetLastError();
}

cudaError_t quantize_llr(const float* llr, size_t n, float delta, int qc, int8_t* q, cudaStream_t st) {
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 16384);
  quantize_kernel<<<blocks, 256, 0, st>>>(llr, n, delta, qc, q);
  return cudaGetLastError();
}

}  // namespace ldpc
