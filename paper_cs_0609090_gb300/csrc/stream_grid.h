// stream_grid.h -- launch geometry shared by the streaming row kernels: one
// warp takes kRowsPerWarp consecutive checks for 32 lanes (frames or frame
// pairs); a block holds kWarpsPerBlock warps.
#pragma once
#include <cstdint>

namespace ldpc {

constexpr int kRowsPerWarp = 4;
constexpr int kWarpsPerBlock = 8;

inline int rows_grid(int M, int lanes) {
  const int64_t warps = (int64_t)((M + kRowsPerWarp - 1) / kRowsPerWarp) * (lanes / 32);
  return (int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
}

}  // namespace ldpc
