// stream_grid.h -- launch geometry shared by the streaming row kernels: one
// warp takes kRowsPerWarp consecutive checks for 32 lanes (frames or frame
// pairs); a block holds kWarpsPerBlock warps.
#pragma once
#include <cstdint>
#ifdef __CUDACC__
#include <cuda_runtime.h>
#else  // host compilers (the CPU check of the warp mapping)
#define __device__
#define __forceinline__ inline
#endif

namespace ldpc {

constexpr int kRowsPerWarp = 4;
constexpr int kWarpsPerBlock = 8;

// Warp -> (chunk of 32 lanes, first check), all chunks of a check together
// (check-major, a 1-D grid of rows_grid blocks): each variable's lines of all
// chunks are read as one contiguous run.
__device__ __forceinline__ bool row_map_all(int warp, int M, int lanes, int& chunk, int& m0) {
  const int n_chunks = lanes / 32;
  const int q = warp / n_chunks;
  chunk = warp - q * n_chunks;
  m0 = q * kRowsPerWarp;
  return m0 < M;
}

inline int rows_grid(int M, int lanes) {
  const int64_t warps = (int64_t)((M + kRowsPerWarp - 1) / kRowsPerWarp) * (lanes / 32);
  return (int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
}

// Warp w of block (bx, by) -> (chunk, first check) with G chunks interleaved
// (a 2-D grid of rows_grid_g blocks, by = chunk group): the warps of G
// neighbouring chunks take the same checks one after another, and the chunk
// groups follow each other, so the warps in flight at one time cover few chunks
// and the posterior lines their checks gather and update stay in L2 between
// the checks that share a variable.  G is a compile-time constant: the row
// warps are short-lived and a runtime division before their first load cost
// the int8 per-edge pass 9 %.
template <int G>
__device__ __forceinline__ bool row_map(int bx, int by, int w, int M, int lanes, int& chunk, int& m0) {
  const int rem = bx * kWarpsPerBlock + w;
  const int q = rem / G;
  chunk = by * G + (rem - q * G);
  m0 = q * kRowsPerWarp;
  return m0 < M && chunk < lanes / 32;
}

struct RowGrid {
  int x, y;
};
inline RowGrid rows_grid_g(int M, int lanes, int G) {
  const int64_t warps = (int64_t)((M + kRowsPerWarp - 1) / kRowsPerWarp) * G;
  return RowGrid{(int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock), (lanes / 32 + G - 1) / G};
}

// Chunks per group of the row passes, measured on the N=64800 code (1024
// frames, 50 iterations): the Section V forms take 1 (int8 16.96 -> 16.13 ms,
// DRAM bytes of a row pass 1.29 -> 0.61 GB with the 8-byte state; float32
// 32.9 -> 27.4 ms), the float32 per-edge form 2 (41.9 -> 37.4 ms); the int8
// per-edge form keeps all chunks of a check together (2 or 4 cost it 3 %).
constexpr int kChunksSV = 1;
constexpr int kChunksF32PE = 2;

}  // namespace ldpc
