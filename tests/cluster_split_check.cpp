// Host harness for the cluster split (paper_cs_0609090_gb300/csrc/cluster_split.h):
// reads a code (int32 N, M, W, cs, then rp[M+1], ci[E]) from argv[1] and writes
// int32 ok, ns, lb, mr, rows[cs], then rdeg[cs*mr] (u8) and tab[cs*W*mr] (u16)
// to argv[2].
#include <cstdio>
#include <vector>

#include "cluster_split.h"

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 3;
  int32_t hdr[4];
  if (std::fread(hdr, 4, 4, f) != 4) return 4;
  const int N = hdr[0], M = hdr[1], W = hdr[2], cs = hdr[3];
  std::vector<int32_t> rp((size_t)M + 1);
  if (std::fread(rp.data(), 4, rp.size(), f) != rp.size()) return 5;
  std::vector<int32_t> ci((size_t)rp[(size_t)M]);
  if (std::fread(ci.data(), 4, ci.size(), f) != ci.size()) return 6;
  std::fclose(f);
  const ldpc::ClusterSplit t = ldpc::split_for_cluster(N, M, rp.data(), ci.data(), W, cs);
  FILE* o = std::fopen(argv[2], "wb");
  if (!o) return 7;
  const int32_t out[4] = {t.ok ? 1 : 0, t.ns, t.lb, t.mr};
  std::fwrite(out, 4, 4, o);
  if (t.ok) {
    std::fwrite(t.rows.data(), 4, t.rows.size(), o);
    std::fwrite(t.rdeg.data(), 1, t.rdeg.size(), o);
    std::fwrite(t.tab.data(), 2, t.tab.size(), o);
  }
  std::fclose(o);
  return 0;
}
