// persist.cuh -- the work queue of the persistent streaming decoders (persist.cu).
//
// One kernel launch runs a whole decode.  Its work is a numbered sequence of
// items (transpose a tile of channel values in, update a tile of checks for one
// iteration, ..., transpose a tile of results out).  A CTA takes the next number
// from a ticket counter, waits until the items it depends on are complete, does
// the work and counts it as complete.  Every item depends only on items with
// smaller numbers, and those were taken by CTAs that were running when they took
// them.  So the decode always makes progress, whether or not every CTA of the
// grid is resident at once.  The dependencies are per chunk of 32 frame-pair
// lanes: each chunk has a monotone counter of completed items on its own
// 128-byte line.
//
// Every wait is bounded.  After max_spins polls (about half a second at the
// default) the CTA sets the error word and leaves, and every other CTA leaves at
// its next item or poll.  A decode whose dependencies cannot be met therefore
// ends in bounded time with the error word set, and the host reads the error.
//
// Data that items of one launch write and other items read (posteriors, state,
// flags) are read with ld.global.cg and written with st.global.cg or L2 atomics:
// L1 is not coherent across SMs, and a persistent kernel gets no L1 flush
// between its iterations.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ldpc {

constexpr uint32_t kWaitSpins = 1u << 22;  // polls of a bounded wait, 128 ns apart
constexpr int kCtlLine = 32;               // 32-bit words per 128-byte line

// Control block of a persistent launch (zeroed before it): the ticket at word 0,
// the error word at word kCtlLine, the counter of chunk c at word (2 + c) kCtlLine.
struct PQueue {
  uint32_t* ctl;
  __host__ __device__ __forceinline__ uint32_t* ticket() const { return ctl; }
  __host__ __device__ __forceinline__ uint32_t* err() const { return ctl + kCtlLine; }
  __host__ __device__ __forceinline__ uint32_t* cnt(int c) const { return ctl + (size_t)(2 + c) * kCtlLine; }
};
inline size_t pq_ctl_bytes(int chunks) { return (size_t)(2 + chunks) * kCtlLine * 4; }

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0: waits until *cnt >= target.  Returns false when it gave up (and set
// the error word) or when another CTA had set it.
__device__ __forceinline__ bool pq_wait(const PQueue& q, const uint32_t* cnt, uint32_t target,
                                        uint32_t max_spins) {
  if (ld_acquire_gpu(cnt) >= target) return true;
  for (uint32_t i = 0; i < max_spins; ++i) {
    __nanosleep(128);
    if (ld_acquire_gpu(cnt) >= target) return true;
    if ((i & 63u) == 63u && ld_relaxed_gpu(q.err()) != 0u) return false;
  }
  atomicOr(q.err(), 1u);
  return false;
}

// Thread 0, after a __syncthreads() that follows the item's last memory
// operation: makes the CTA's writes visible at GPU scope, then counts the item.
__device__ __forceinline__ void pq_done(const PQueue& q, int c) {
  __threadfence();
  atomicAdd(q.cnt(c), 1u);
}

// f16x2 atomic add in L2 (no result).
__device__ __forceinline__ void red_add_h2(uint32_t* p, uint32_t v) {
  asm volatile("red.global.add.noftz.f16x2 [%0], %1;" ::"l"(p), "r"(v));
}

}  // namespace ldpc
