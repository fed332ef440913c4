// Host check of the streaming row kernels' warp mappings
// (paper_cs_0609090_gb300/csrc/stream_grid.h): over the grid that the launch
// uses, every (chunk of 32 lanes, group of kRowsPerWarp checks) is taken by
// exactly one warp -- row_map_all on the 1-D rows_grid, row_map<G> on the 2-D
// rows_grid_g for every chunk interleave G, including chunk counts that G does
// not divide.  Prints the number of failing cases and exits non-zero if there
// is one.
#include <cstdio>
#include <vector>

#include "stream_grid.h"

namespace {

int g_bad = 0, g_cases = 0;

template <class F>
void check(const char* what, int M, int nch, int G, long warps, F map) {
  ++g_cases;
  const int groups = (M + ldpc::kRowsPerWarp - 1) / ldpc::kRowsPerWarp;
  std::vector<int> seen((size_t)groups * nch, 0);
  bool ok = true;
  for (long w = 0; w < warps && ok; ++w) {
    int chunk = -1, m0 = -1;
    if (!map(w, chunk, m0)) continue;
    if (chunk < 0 || chunk >= nch || m0 < 0 || m0 >= M || m0 % ldpc::kRowsPerWarp != 0) ok = false;
    else ++seen[(size_t)chunk * groups + m0 / ldpc::kRowsPerWarp];
  }
  for (int v : seen) ok = ok && v == 1;
  if (!ok) {
    ++g_bad;
    std::printf("%s M=%d chunks=%d G=%d: not a one-to-one cover\n", what, M, nch, G);
  }
}

template <int G>
void check_g(int M, int nch) {
  const int lanes = 32 * nch;
  const ldpc::RowGrid g = ldpc::rows_grid_g(M, lanes, G);
  const long per_block = ldpc::kWarpsPerBlock;
  check("row_map", M, nch, G, (long)g.x * g.y * per_block, [&](long w, int& chunk, int& m0) {
    const int blk = (int)(w / per_block), wi = (int)(w % per_block);
    return ldpc::row_map<G>(blk % g.x, blk / g.x, wi, M, lanes, chunk, m0);
  });
}

}  // namespace

int main() {
  const int Ms[] = {1, 2, 3, 4, 5, 7, 8, 9, 33, 504, 3048, 32400};
  for (int M : Ms) {
    for (int nch = 1; nch <= 19; ++nch) {
      const int lanes = 32 * nch;
      check("row_map_all", M, nch, nch, (long)ldpc::rows_grid(M, lanes) * ldpc::kWarpsPerBlock,
            [&](long w, int& chunk, int& m0) { return ldpc::row_map_all((int)w, M, lanes, chunk, m0); });
      check_g<1>(M, nch);
      check_g<2>(M, nch);
      check_g<3>(M, nch);
      check_g<4>(M, nch);
      check_g<8>(M, nch);
    }
  }
  std::printf("%d of %d cases fail\n", g_bad, g_cases);
  return g_bad == 0 ? 0 : 1;
}
