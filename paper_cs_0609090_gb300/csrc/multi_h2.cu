// multi_h2.cu -- one persistent launch that decodes the frames of several codes
// (single-scan min-sum of Section IV, Eq. (3), with the Section V state or
// per-edge messages; exact packed binary16 frame pairs as in onchip_h2.cu).
//
// Work items are frame pairs.  A code whose pair state fits one CTA ("local")
// is decoded by CTA sub-teams: a CTA holds `sub` pairs of that code at once, each
// on T / sub threads with its own named barrier.  A code too large for one SM
// ("cluster") is split over the `cs` CTAs of a thread-block cluster: CTA rank r
// keeps the posteriors of variables [r ns, (r+1) ns) and the state of its own
// checks; a check reads the posteriors of its variables and adds its messages to
// their accumulators through distributed shared memory, and the cluster
// barrier separates the check pass from the variable pass.  Everything of a
// pair (posteriors, accumulators, check state and the column table) stays in
// shared memory for all iterations.
//
// Items are handed out longest first (cluster items, then local bundles) from
// two counters in device memory, or round-robin when no counter is given.  The
// launch takes all of its data in the kernel parameters, so it needs no upload
// and can be captured in a CUDA graph.
//
// Shared memory of one CTA:
//   [column table: local ell_w x M, cluster this rank's ell_w x mr; u16]
//   per pair slot: Zs [nv] half2 | Acc [nv] i32 | St [rows] uint4 or Lm [ell_w][rows] u16
#include <cuda_fp16.h>

#include <atomic>

#include "h2_body.cuh"
#include "kernels.h"

namespace ldpc {
namespace {

constexpr int kMultiThreadsMax = 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_or(uint32_t a, uint32_t v) {
  asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_st(uint32_t a, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync() {
  __cluster_barrier_arrive();
  __cluster_barrier_wait();
}
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Posteriors spread over the cluster: table entry (rank << lb) | local index;
// Zs[local] of CTA rank through 32-bit shared::cluster addresses.  Loads and
// reductions are volatile so that they stay between the cluster barriers.
struct ClusterAddr {
  using H = uint32_t;
  int M;
  uint32_t lmask;
  int lb;
  uint32_t zs;      // shared address of this CTA's Zs
  uint32_t accoff;  // bytes from Zs to Acc
  __device__ __forceinline__ H at(const uint16_t* __restrict__ tab, const uint32_t*, int j, int m) const {
    const uint32_t a = tab[j * M + m];
    return cl_map(zs + ((a & lmask) << 2), a >> lb);
  }
  __device__ __forceinline__ void load(const uint32_t*, H h, uint32_t (&w)[1]) const {
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(w[0]) : "r"(h));
  }
  __device__ __forceinline__ void add(int32_t*, H h, int, int32_t v) const {
    asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(h + accoff), "r"(v));
  }
  __device__ __forceinline__ int st(int m) const { return m; }
  __device__ __forceinline__ int lm(int j, int m) const { return j * M + m; }
};

// Exact-degree bodies for the check degrees of the supported families (6/7:
// regular (3,6) and staircase codes; 14/15: the quasi-cyclic base), the guarded
// loop for any other degree <= 16.
template <int FORM, bool ES, class Addr>
__device__ __forceinline__ uint32_t check_any(const Addr& ad, const uint16_t* __restrict__ tab,
                                              const uint32_t* __restrict__ Zs, int32_t* __restrict__ Acc,
                                              const H2Rule& r, uint32_t qm2, int m, int d, uint4* __restrict__ St,
                                              uint16_t* __restrict__ Lm) {
  switch (d) {
    case 6: return check_body<2, FORM, 6, 16, ES>(ad, tab, Zs, Acc, r, qm2, m, d, St, Lm);
    case 7: return check_body<2, FORM, 7, 16, ES>(ad, tab, Zs, Acc, r, qm2, m, d, St, Lm);
    case 14: return check_body<2, FORM, 14, 16, ES>(ad, tab, Zs, Acc, r, qm2, m, d, St, Lm);
    case 15: return check_body<2, FORM, 15, 16, ES>(ad, tab, Zs, Acc, r, qm2, m, d, St, Lm);
    default: return check_body<2, FORM, 0, 16, ES>(ad, tab, Zs, Acc, r, qm2, m, d, St, Lm);
  }
}

struct MultiShared {
  uint32_t fail[kMultiMaxSub][3];
  int32_t iters[kMultiMaxSub][2];
  uint32_t ok[kMultiMaxSub];
  int32_t item;
};

__device__ __forceinline__ int32_t q0v(const int8_t* __restrict__ llr, int32_t N, int32_t f, int32_t F, int n) {
  return f < F ? (int32_t)__ldg(llr + (size_t)f * N + n) : 0;
}

// Decodes frame pair `pair` of job jb.  CL: this CTA is rank `rank` of the
// cluster that owns the pair (tid/nt: the whole CTA); otherwise sub-team s of
// this CTA (tid/nt: its threads) owns it alone.
template <int FORM, bool ES, bool CL>
__device__ void decode_pair(const MultiJob& jb, int pair, unsigned char* smem, MultiShared& sh, int s, int tid, int nt,
                            uint32_t rank, uint32_t cs) {
  const int N = jb.N;
  const int F = jb.F;
  const uint16_t* tab = reinterpret_cast<const uint16_t*>(smem);
  unsigned char* base = smem + jb.tab_bytes + (size_t)s * jb.slot_bytes;
  uint32_t* Zs = reinterpret_cast<uint32_t*>(base);
  int32_t* Acc = reinterpret_cast<int32_t*>(base + jb.acc_off);
  uint4* St = reinterpret_cast<uint4*>(base + jb.st_off);
  uint16_t* Lm = reinterpret_cast<uint16_t*>(base + jb.st_off);
  int32_t* Rs = reinterpret_cast<int32_t*>(base + jb.rs_off);
  const bool rset = !CL && jb.rs_off != 0u;
  const int v0 = CL ? (int)rank * jb.ns : 0;
  const int nv = CL ? max(0, min(N - v0, jb.ns)) : N;
  const int rows = CL ? __ldg(jb.rows + rank) : jb.M;
  const uint8_t* __restrict__ rdeg = jb.rdeg + (CL ? (size_t)rank * jb.mr : 0);
  const H2Rule hr = h2rule(jb.beta, jb.num, jb.shift);
  const uint32_t qm2 = ints_to_h2(jb.qm, jb.qm);
  const int slot = CL ? 0 : s;
  const bool es = ES && jb.early_stop != 0;
  const int f0 = 2 * pair;
  const int nvalid = min(2, F - f0);
  uint32_t act = (1u << nvalid) - 1u;
  auto tsync = [&]() {
    if constexpr (CL) cluster_sync();
    else named_sync(1 + s, nt);
  };
  auto publish = [&](int idx, uint32_t bits) {
    bits = __reduce_or_sync(0xffffffffu, bits) & act;
    if (bits != 0u) {
      const int lane = tid & 31;
      if constexpr (CL) {
        if (lane < (int)cs) cl_or(cl_map(smem_u32(&sh.fail[0][idx]), (uint32_t)lane), bits);
      } else {
        if (lane == 0) atomicOr(&sh.fail[s][idx], bits);
      }
    }
  };

  for (int i = tid; i < nv; i += nt) {
    const int n = v0 + i;
    const uint32_t bias = (uint32_t)__ldg(jb.cdeg + n) * 0x66006600u;
    const int32_t lo = q0v(jb.llr, N, f0, F, n), hi = q0v(jb.llr, N, f0 + 1, F, n);
    Zs[i] = ints_to_h2(lo, hi);
    const int32_t reset = (int32_t)((uint32_t)acc_pack(lo, hi) - bias);
    Acc[i] = reset;
    if (rset) Rs[i] = reset;
  }
  if constexpr (FORM == 1) {
    for (int i = tid; i < rows; i += nt) St[i] = make_uint4(0u, 0u, 0u, 0u);
  } else {
    // L^(0) = 0 is the byte 128 in both frames
    for (int i = tid; i < jb.ell_w * jb.mr; i += nt) Lm[i] = 0x8080u;
  }
  if (tid < 3) sh.fail[slot][tid] = 0;
  if (tid < 2) sh.iters[slot][tid] = jb.max_iter;
  if (tid == 0) sh.ok[slot] = 0;
  tsync();

  for (int k = 1; k <= jb.max_iter && act != 0u; ++k) {
    const int kp = k & 1;
    uint32_t fail = 0;
    if constexpr (CL) {
      const ClusterAddr ad{jb.mr, (1u << jb.lb) - 1u, jb.lb, smem_u32(Zs), (uint32_t)jb.acc_off};
      for (int m = tid; m < rows; m += nt)
        fail |= check_any<FORM, ES>(ad, tab, Zs, Acc, hr, qm2, m, (int)__ldg(rdeg + m), St, Lm);
    } else {
      const LocalAddr<2, true> ad{jb.M};
      for (int m = tid; m < rows; m += nt)
        fail |= check_any<FORM, ES>(ad, tab, Zs, Acc, hr, qm2, m, (int)__ldg(rdeg + m), St, Lm);
    }
    if constexpr (ES) publish(kp, fail);
    tsync();
    const uint32_t stop = es ? (act & ~sh.fail[slot][kp]) : 0u;
    const uint32_t cont = act & ~stop;
    const uint32_t sel = ((cont & 1u) ? 0x0000ffffu : 0u) | ((cont & 2u) ? 0xffff0000u : 0u);
    for (int i = tid; i < nv; i += nt) {
      const uint32_t zz = acc_to_pair(Acc[i]);
      const uint32_t h = ints_to_h2(lo16(zz), hi16(zz));
      Zs[i] = (h & sel) | (Zs[i] & ~sel);
      if (rset) {
        Acc[i] = Rs[i];
      } else {
        const int n = v0 + i;
        const uint32_t bias = (uint32_t)__ldg(jb.cdeg + n) * 0x66006600u;
        const int32_t lo = q0v(jb.llr, N, f0, F, n), hi = q0v(jb.llr, N, f0 + 1, F, n);
        Acc[i] = (int32_t)((uint32_t)acc_pack(lo, hi) - bias);
      }
    }
    if (es) {
      if (tid < 2 && ((stop >> tid) & 1u)) sh.iters[slot][tid] = k - 1;
      if (tid == 0) sh.ok[slot] |= stop;
    }
    tsync();
    if (tid == 0) sh.fail[slot][kp] = 0;
    act = cont;
  }

  if (act != 0u) {
    // syndrome of the final decision
    uint32_t fail = 0;
    if constexpr (CL) {
      const ClusterAddr ad{jb.mr, (1u << jb.lb) - 1u, jb.lb, smem_u32(Zs), (uint32_t)jb.acc_off};
      for (int m = tid; m < rows; m += nt) fail |= row_parity_body<2, 0, 16>(ad, tab, Zs, m, (int)__ldg(rdeg + m));
    } else {
      const LocalAddr<2, true> ad{jb.M};
      for (int m = tid; m < rows; m += nt) fail |= row_parity_body<2, 0, 16>(ad, tab, Zs, m, (int)__ldg(rdeg + m));
    }
    publish(2, fail);
    tsync();
    if (tid == 0) sh.ok[slot] |= act & ~sh.fail[slot][2];
  }
  if constexpr (CL) __syncthreads();
  else named_sync(1 + s, nt);

  const int N8 = (N + 7) >> 3;
  const int nb = (nv + 7) >> 3;
  const int b0 = v0 >> 3;
  for (int i = tid; i < nvalid * nb; i += nt) {
    const int g = i / nb, b = i - g * nb;
    uint32_t byte = 0;
    for (int t = 0; t < 8; ++t) {
      const int li = b * 8 + t;
      if (li < nv) byte |= ((dec_bits(Zs[li] >> (16 * g)) >> 15) & 1u) << t;
    }
    jb.bits[(size_t)(f0 + g) * N8 + b0 + b] = (uint8_t)byte;
  }
  if (jb.zout != nullptr) {
    for (int i = tid; i < nvalid * nv; i += nt) {
      const int g = i / nv, li = i - g * nv;
      const uint32_t h = Zs[li];
      jb.zout[(size_t)(f0 + g) * N + v0 + li] = (int16_t)(g ? h_hi_int(h) : h_lo_int(h));
    }
  }
  if ((!CL || rank == 0) && tid < nvalid) {
    jb.iters[f0 + tid] = sh.iters[slot][tid];
    jb.ok[f0 + tid] = (uint8_t)((sh.ok[slot] >> tid) & 1u);
  }
}

// Copies the column table of job j (this rank's part for a cluster job) into
// the start of shared memory.
__device__ void load_table(const MultiJob& jb, unsigned char* smem, uint32_t rank, bool cl) {
  const int cnt = jb.ell_w * jb.mr;
  const uint16_t* src = jb.tab + (cl ? (size_t)rank * cnt : 0);
  uint16_t* dst = reinterpret_cast<uint16_t*>(smem);
  // (a cluster table has an even number of entries per rank: 4-byte aligned)
  const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d32 = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < cnt / 2; i += blockDim.x) d32[i] = __ldg(s32 + i);
  if ((cnt & 1) && threadIdx.x == 0) dst[cnt - 1] = __ldg(src + cnt - 1);
}

__device__ __forceinline__ int find_job(const MultiParams& mp, int lo, int hi, int item) {
  int j = lo;
  while (j + 1 < hi && item >= mp.job[j + 1].item0) ++j;
  return j;
}

template <int FORM, bool ES>
__global__ void __launch_bounds__(kMultiThreadsMax, 1) multi_h2_kernel(const __grid_constant__ MultiParams mp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ MultiShared sh;
  const int tid = threadIdx.x, T = blockDim.x;
  int cur = -1;  // job whose table is in shared memory

  if (mp.n_citems > 0) {
    const uint32_t cs = mp.cs;
    const uint32_t rank = __clusterRelativeBlockRank();
    const int cid = (int)__clusterIdx().x, ncl = (int)__clusterGridDimInClusters().x;
    // every CTA of the cluster has started before any distributed shared memory access
    cluster_sync();
    for (int t = 0;; ++t) {
      int it;
      if (mp.counters != nullptr) {
        if (rank == 0 && tid == 0) {
          const int v = atomicAdd(mp.counters, 1);
          for (uint32_t r = 0; r < cs; ++r) cl_st(cl_map(smem_u32(&sh.item), r), (uint32_t)v);
        }
        cluster_sync();
        it = sh.item;
      } else {
        it = cid + t * ncl;
      }
      if (it >= mp.n_citems) break;
      const int j = find_job(mp, 0, mp.n_cjobs, it);
      const MultiJob& jb = mp.job[j];
      if (j != cur) {
        load_table(jb, smem, rank, true);
        cur = j;
        __syncthreads();
      }
      decode_pair<FORM, ES, true>(jb, it - jb.item0, smem, sh, 0, tid, T, rank, cs);
    }
    cur = -1;
    __syncthreads();
  }

  if (mp.n_litems > 0) {
    for (int t = 0;; ++t) {
      int it;
      if (mp.counters != nullptr) {
        if (tid == 0) sh.item = atomicAdd(mp.counters + 1, 1);
        __syncthreads();
        it = sh.item;
      } else {
        it = (int)blockIdx.x + t * (int)gridDim.x;
      }
      if (it >= mp.n_litems) break;
      const int j = find_job(mp, mp.n_cjobs, mp.n_jobs, it);
      const MultiJob& jb = mp.job[j];
      if (j != cur) {
        load_table(jb, smem, 0, false);
        cur = j;
      }
      __syncthreads();
      const int nts = T / jb.sub;
      const int s = tid / nts;
      const int pair = (it - jb.item0) * jb.sub + s;
      if (pair < jb.n_pairs) decode_pair<FORM, ES, false>(jb, pair, smem, sh, s, tid - s * nts, nts, 0, 1);
      __syncthreads();
    }
  }
}

// Function attributes already set on a device, so that a launch inside a CUDA
// graph capture makes no attribute call (the first launch comes before).
constexpr int kMaxDevices = 64;
struct AttrCache {
  std::atomic<int> smem[kMaxDevices];
  std::atomic<int> nonportable[kMaxDevices];
};

template <int FORM, bool ES>
cudaError_t multi_launch_t(const MultiParams& mp, int threads, size_t smem, int grid, cudaStream_t st,
                           int* max_grid) {
  static AttrCache cache;
  auto kern = multi_h2_kernel<FORM, ES>;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (cache.smem[dev].load() < (int)smem) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cache.smem[dev].store((int)smem);
  }
  if (mp.cs > 8 && cache.nonportable[dev].load() == 0) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cache.nonportable[dev].store(1);
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  const int cs = mp.n_citems > 0 ? mp.cs : 1;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cs > 1 ? 1 : 0;
  if (max_grid != nullptr) {
    // persistent grid: every cluster (or CTA) that can be resident at once
    cfg.gridDim = dim3((unsigned)cs, 1, 1);
    int n = 0;
    if (cs > 1) {
      e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
      if (e != cudaSuccess) return e;
      *max_grid = n * cs;
    } else {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem);
      if (e != cudaSuccess) return e;
      int sms = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      *max_grid = n * sms;
    }
    return cudaSuccess;
  }
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, mp);
}

}  // namespace

size_t multi_local_slot_bytes(int N, int M, int ell_w, int form, size_t* acc_off, size_t* st_off, bool rset,
                              size_t* rs_off) {
  const size_t zs = ((size_t)N * 4 + 15) & ~size_t(15);
  const size_t st = form == 1 ? (size_t)M * 16 : (((size_t)ell_w * M * 2 + 15) & ~size_t(15));
  if (acc_off) *acc_off = zs;
  if (st_off) *st_off = 2 * zs;
  if (rs_off) *rs_off = rset ? 2 * zs + st : 0;
  return 2 * zs + st + (rset ? zs : 0);
}

cudaError_t multi_launch(int form, bool es, const MultiParams& mp, int threads, size_t smem, int grid,
                         cudaStream_t st, int* max_grid) {
  if (form == 1) return es ? multi_launch_t<1, true>(mp, threads, smem, grid, st, max_grid)
                           : multi_launch_t<1, false>(mp, threads, smem, grid, st, max_grid);
  return es ? multi_launch_t<0, true>(mp, threads, smem, grid, st, max_grid)
            : multi_launch_t<0, false>(mp, threads, smem, grid, st, max_grid);
}

}  // namespace ldpc
