// Host check of the raster ordering (paper_1902_08410_gb300/csrc/snn_raster.h):
// rasters built like the library builds them (entries grouped by step in
// increasing order, the ids of a step shuffled), with and without an already
// ordered head, and rasters that are not grouped by step (the fallback), must
// come out exactly as std::sort orders them; the split into step and id arrays
// must reproduce every entry.  Exit status 0 on success.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "snn_raster.h"

int main() {
  std::mt19937_64 rng(5);
  int fails = 0;
  for (int trial = 0; trial < 60; ++trial) {
    std::vector<unsigned long long> r;
    const size_t head = trial % 3 == 0 ? 1000 : 0;
    for (size_t i = 0; i < head; ++i) r.push_back(i);   // step 0, already ordered
    const int steps = 20 + (int)(rng() % 3000);
    for (int t = 1; t <= steps; ++t) {
      const int k = (int)(rng() % (trial % 4 == 1 ? 5000u : 900u));
      std::vector<uint32_t> ids;
      for (int i = 0; i < k; ++i) ids.push_back((uint32_t)(rng() % (1u << 24)));
      std::sort(ids.begin(), ids.end());
      ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
      std::shuffle(ids.begin(), ids.end(), rng);
      for (uint32_t id : ids) r.push_back(((unsigned long long)t << 32) | id);
    }
    if (trial % 5 == 4 && r.size() > head + 10) std::swap(r[head + 3], r[r.size() - 2]);   // not grouped
    std::vector<unsigned long long> ref = r;
    std::sort(ref.begin() + (std::ptrdiff_t)head, ref.end());
    snn::order_raster(r, head);
    if (r != ref) {
      ++fails;
      std::printf("trial %d: order differs (%zu entries)\n", trial, r.size());
    }
  }
  // split into step and id arrays: below and above the parallel threshold
  for (size_t n : {(size_t)0, (size_t)1, (size_t)1000, (size_t)5000003}) {
    std::vector<unsigned long long> r(n);
    for (size_t i = 0; i < n; ++i) r[i] = ((unsigned long long)(i / 7) << 32) | (uint32_t)(rng() % (1u << 24));
    std::vector<uint32_t> st(n + 1, 0xDEADBEEFu), id(n + 1, 0xDEADBEEFu);
    snn::split_raster(r.data(), n, st.data(), id.data());
    bool ok = st[n] == 0xDEADBEEFu && id[n] == 0xDEADBEEFu;
    for (size_t i = 0; i < n && ok; ++i) ok = st[i] == (uint32_t)(r[i] >> 32) && id[i] == (uint32_t)r[i];
    if (!ok) {
      ++fails;
      std::printf("split of %zu entries differs\n", n);
    }
  }
  std::printf("%s\n", fails ? "FAIL" : "ok");
  return fails ? 1 : 0;
}
