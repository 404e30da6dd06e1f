// Host-only check of the persistent kernels' work lists (tc_single_items for
// the one-SM kernel, tc_pair_items for the two-SM kernel), built by
// tests/test_work_lists.py with nvcc and run on the CPU: no device call.
// For every shape and cluster/SM count it checks that
//   - every upper-triangle tile (I <= J) is covered exactly once over the
//     whole chunk range [0, nc), by contiguous K pieces;
//   - a tile covered by several pieces is in the split-tile list (its counts
//     are accumulated and finalised), and every listed tile is split;
//   - no item spans more than 2^21 markers (exact FP32 accumulation);
//   - pair items hold I0 <= J, I1 <= J or -1, I0 != I1.
// Prints one line per failure and "checked N lists, F failures".
#include "../paper_1410_4803_gb300/csrc/ibs_tc.cu"

#include <map>
#include <set>
#include <utility>

namespace {

int failures = 0;
void fail(const char* what, int64_t n, int64_t m, int c) {
  ++failures;
  printf("FAIL %s: n=%lld m=%lld units=%d\n", what, (long long)n, (long long)m, c);
}

using Cover = std::map<std::pair<int, int>, std::vector<std::pair<int, int>>>;

void check_cover(const Cover& cov, const std::set<std::pair<int, int>>& split, int64_t T, int64_t nc, int64_t n,
                 int64_t m, int c) {
  if ((int64_t)cov.size() != T * (T + 1) / 2) fail("tile count", n, m, c);
  for (const auto& kv : cov) {
    auto v = kv.second;
    std::sort(v.begin(), v.end());
    int64_t e = 0;
    for (const auto& r : v) {
      if (r.first != e || r.second <= r.first) fail("K ranges not contiguous", n, m, c);
      if ((int64_t)(r.second - r.first) * 64 > ((int64_t)1 << 21)) fail("item beyond 2^21 markers", n, m, c);
      e = r.second;
    }
    if (e != nc) fail("K ranges do not end at nc", n, m, c);
    if ((v.size() > 1) != (split.count(kv.first) > 0)) fail("split list", n, m, c);
  }
}

}  // namespace

int main() {
  int lists = 0;
  const int64_t ns[] = {1, 127, 128, 129, 256, 300, 1000, 4096, 5000, 20000};
  const int64_t ms[] = {1, 64, 65, 1000, 100000, 262144, 500000, 2200000};
  for (int64_t n : ns)
    for (int64_t m : ms) {
      const int64_t T = (n + 127) / 128, nc = (m + 63) / 64;
      if (T * (T + 1) / 2 * (nc / 4096 + 1) > 2000000) continue;  // keep the run short
      for (int c : {1, 5, 74, 76, 152}) {
        {
          std::vector<ibs::WorkItem> items;
          std::vector<int2> sp;
          ibs::tc_single_items(n, m, ibs::kTcFp4, c, 16, items, sp);
          Cover cov;
          std::set<std::pair<int, int>> split;
          for (const auto& s : sp) split.insert({s.x, s.y});
          for (const auto& w : items) {
            if (w.I > w.J || w.I < 0 || w.J >= T) fail("single tile outside the triangle", n, m, c);
            if ((w.split != 0) != (split.count({w.I, w.J}) > 0)) fail("single split flag", n, m, c);
            cov[{w.I, w.J}].push_back({w.c0, w.c1});
          }
          check_cover(cov, split, T, nc, n, m, c);
          ++lists;
        }
        if (T >= 2) {
          std::vector<ibs::PairItem> items;
          std::vector<int2> sp;
          ibs::tc_pair_items(n, m, ibs::kTcFp4, c, 16, items, sp);
          Cover cov;
          std::set<std::pair<int, int>> split;
          for (const auto& s : sp) split.insert({s.x, s.y});
          for (const auto& w : items) {
            if (w.I0 < 0 || w.I0 > w.J || w.J >= T || w.I1 > w.J || w.I1 == w.I0 || w.I1 < -1)
              fail("pair item outside the triangle", n, m, c);
            if ((w.split != 0) != (split.count({w.I0, w.J}) > 0)) fail("pair split flag", n, m, c);
            cov[{w.I0, w.J}].push_back({w.c0, w.c1});
            if (w.I1 >= 0) cov[{w.I1, w.J}].push_back({w.c0, w.c1});
          }
          check_cover(cov, split, T, nc, n, m, c);
          ++lists;
        }
      }
    }
  printf("checked %d lists, %d failures\n", lists, failures);
  return failures == 0 ? 0 : 1;
}
