// Host check of the trailing update's unit enumeration (tc::window_units,
// tc::window_unit): for every window of m tile columns over n tile rows, in
// single tiles and in tile pairs, the units cover each tile of the window's
// lower part (rows >= columns in its m x m triangle, all m columns below)
// exactly once, a pair's second tile lies in the same tile row next to the
// first, and the unit count equals the closed form the set-up uses.  Also
// the split of a backward block's ancestor-row product (bwd_parts,
// bwd_part_rows): at most BWD_PARTS_MAX parts of 128-row multiples, none
// empty, together covering every ancestor row.
#include <cstdio>
#include <vector>

#include "../paper_2107_03285_gb300/csrc/common.cuh"
#include "../paper_2107_03285_gb300/csrc/tc_update.cuh"

int main() {
  using namespace sgn::tc;
  int bad = 0;
  for (int pair = 0; pair < 2; ++pair)
    for (int m = 1; m <= 48; ++m)
      for (int n = m; n <= m + 40; ++n) {
        TileJob job{};
        job.win0 = 3;  // any window start: coordinates are absolute
        job.m = m;
        job.pair = pair;
        std::vector<int> hits((size_t)n * m, 0);
        const int units = window_units(m, n, pair != 0);
        for (int t = 0; t < units; ++t) {
          int bi, bj;
          bool two;
          window_unit(job, t, bi, bj, two);
          const int r = bi - job.win0, c = bj - job.win0;
          for (int e = 0; e < (two ? 2 : 1); ++e) {
            const int cc = c + e;
            if (r < 0 || r >= n || cc < 0 || cc >= m || cc > r) {
              ++bad;
              continue;
            }
            ++hits[(size_t)r * m + cc];
          }
          if (two && !pair) ++bad;
        }
        for (int r = 0; r < n; ++r)
          for (int c = 0; c < m; ++c)
            if (hits[(size_t)r * m + c] != (c <= r ? 1 : 0)) ++bad;
      }
  for (int64_t rows = 0; rows <= 200000; rows += rows < 20000 ? 1 : 97) {
    const int h = sgn::bwd_parts(rows);
    if (rows <= sgn::BWD_PART_MIN_ROWS) {
      if (h != 0) ++bad;
      continue;
    }
    const int64_t rp = sgn::bwd_part_rows(rows);
    if (h < 1 || h > sgn::BWD_PARTS_MAX || rp % 128 != 0 || (int64_t)(h - 1) * rp >= rows || (int64_t)h * rp < rows)
      ++bad;
  }
  std::printf("%s %d\n", bad ? "FAIL" : "ok", bad);
  return bad ? 1 : 0;
}
