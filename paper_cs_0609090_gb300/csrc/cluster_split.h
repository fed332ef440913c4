// cluster_split.h -- host-only split of a code over the cs CTAs of a
// thread-block cluster (no CUDA; also compiled by a CPU test).
//
// Variables go to ranks in contiguous slices of ns (a multiple of 8, so that no
// byte of packed decisions spans two ranks).  A check goes to the rank that
// holds most of its variables (lowest rank on ties); ranks over the cap
// ceil(M / cs) then hand the checks with the fewest local variables to the
// ranks with room (to the one holding most of the check's variables).  Within
// a rank the checks are sorted by degree.  The order of checks does not change
// any result: every check's messages depend only on the previous iteration and
// the posteriors are exact integer sums.
//
// Entry (r, j, i) of tab ([cs][W][mr]) is (rank << lb) | (n - rank ns) for the
// variable n at position j of rank r's i-th check; positions past the check's
// degree repeat its last variable; rows past rows[r] are zero padding.  mr is
// even, so every rank's part of tab is 4-byte aligned.
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>

namespace ldpc {

struct ClusterSplit {
  int cs = 0, ns = 0, lb = 0, mr = 0;
  bool ok = false;  // false: rank and local index do not fit 16 bits
  std::vector<uint16_t> tab;
  std::vector<uint8_t> rdeg;
  std::vector<int32_t> rows;
};

inline ClusterSplit split_for_cluster(int N, int M, const int32_t* rp, const int32_t* ci, int W, int cs) {
  ClusterSplit t;
  t.cs = cs;
  t.ns = ((N + cs - 1) / cs + 7) & ~7;
  int lb = 1;
  while ((1 << lb) < t.ns) ++lb;
  int rb = 0;
  while ((1 << rb) < cs) ++rb;
  t.lb = lb;
  if (lb + rb > 16) return t;
  const int ns = t.ns;
  auto local_count = [&](int m, int r) {
    int k = 0;
    for (int e = rp[m]; e < rp[m + 1]; ++e) k += (ci[e] / ns == r);
    return k;
  };
  std::vector<int> cnt((size_t)cs);
  std::vector<std::vector<int>> bucket((size_t)cs);
  for (int m = 0; m < M; ++m) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int e = rp[m]; e < rp[m + 1]; ++e) cnt[(size_t)(ci[e] / ns)]++;
    bucket[(size_t)(std::max_element(cnt.begin(), cnt.end()) - cnt.begin())].push_back(m);
  }
  const int cap = (M + cs - 1) / cs;
  std::vector<int> pool;
  for (int r = 0; r < cs; ++r) {
    std::vector<int>& bk = bucket[(size_t)r];
    if ((int)bk.size() <= cap) continue;
    std::stable_sort(bk.begin(), bk.end(), [&](int a, int b) { return local_count(a, r) > local_count(b, r); });
    pool.insert(pool.end(), bk.begin() + cap, bk.end());
    bk.resize((size_t)cap);
  }
  for (int m : pool) {
    int best = -1, best_k = -1;
    for (int r = 0; r < cs; ++r) {
      if ((int)bucket[(size_t)r].size() >= cap) continue;
      const int k = local_count(m, r);
      if (k > best_k) best = r, best_k = k;
    }
    bucket[(size_t)best].push_back(m);
  }
  t.mr = (cap + 1) & ~1;
  t.tab.assign((size_t)cs * W * t.mr, 0);
  t.rdeg.assign((size_t)cs * t.mr, 0);
  t.rows.assign((size_t)cs, 0);
  for (int r = 0; r < cs; ++r) {
    std::vector<int>& bk = bucket[(size_t)r];
    std::stable_sort(bk.begin(), bk.end(), [&](int a, int b) { return rp[a + 1] - rp[a] < rp[b + 1] - rp[b]; });
    t.rows[(size_t)r] = (int32_t)bk.size();
    for (size_t i = 0; i < bk.size(); ++i) {
      const int m = bk[i], d = rp[m + 1] - rp[m];
      t.rdeg[(size_t)r * t.mr + i] = (uint8_t)d;
      for (int j = 0; j < W; ++j) {
        const int n = ci[rp[m] + (j < d ? j : d - 1)];
        t.tab[((size_t)r * W + j) * t.mr + i] = (uint16_t)(((n / ns) << lb) | (n % ns));
      }
    }
  }
  t.ok = true;
  return t;
}

}  // namespace ldpc
