// snn_raster.h -- ordering of the host raster (header-only so that the host
// logic can be checked without a GPU).
//
// Raster entries are (step << 32 | neuron id), ids below 2^24.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <thread>
#include <utility>
#include <vector>

namespace snn {

// Order raster[from, end) by (step, id).  Entries arrive grouped by step in
// increasing order (each step's kernels append before the next step's run),
// with the ids of a step in warp order, so each step's run is sorted on its
// own (ids are below 2^24: a 3-pass LSD radix sort), in parallel over ranges
// of steps; anything else falls back to one sort.
inline void sort_run_by_id(unsigned long long *a, size_t n, std::vector<unsigned long long> &tmp) {
  if (n < 64) {
    std::sort(a, a + n);
    return;
  }
  tmp.resize(n);
  unsigned long long *src = a, *dst = tmp.data();
  for (int sh = 0; sh < 24; sh += 8) {
    size_t cnt[257] = {0};
    for (size_t i = 0; i < n; ++i) ++cnt[((src[i] >> sh) & 0xFFu) + 1];
    for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
    for (size_t i = 0; i < n; ++i) dst[cnt[(src[i] >> sh) & 0xFFu]++] = src[i];
    std::swap(src, dst);
  }
  if (src != a) std::copy(src, src + n, a);   // three passes end in tmp
}

inline void order_raster(std::vector<unsigned long long> &r, size_t from) {
  const size_t n = r.size() - from;
  if (n == 0) return;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t parts = std::min<size_t>(std::min<size_t>(hw, 16), std::max<size_t>(1, n / (1u << 16)));
  // cut points on step boundaries (the first entry of a step)
  std::vector<size_t> cut(parts + 1, r.size());
  cut[0] = from;
  for (size_t p = 1; p < parts; ++p) {
    size_t c = std::max(cut[p - 1], from + n * p / parts);
    while (c < r.size() && c > from && (r[c] >> 32) == (r[c - 1] >> 32)) ++c;
    cut[p] = c;
  }
  std::vector<char> grouped(parts, 1);
  auto work = [&r, &cut, &grouped](size_t p) {
    const size_t a = cut[p], b = cut[p + 1];
    for (size_t i = a + 1; i < b; ++i)
      if ((r[i] >> 32) < (r[i - 1] >> 32)) {
        grouped[p] = 0;
        return;
      }
    std::vector<unsigned long long> tmp;
    size_t s = a;
    while (s < b) {
      size_t e = s + 1;
      while (e < b && (r[e] >> 32) == (r[s] >> 32)) ++e;
      sort_run_by_id(r.data() + s, e - s, tmp);
      s = e;
    }
  };
  if (parts <= 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    for (size_t p = 0; p < parts; ++p)
      if (cut[p] < cut[p + 1]) th.emplace_back(work, p);
    for (auto &t : th) t.join();
  }
  bool ok = true;
  for (size_t p = 0; p < parts; ++p) ok &= grouped[p] != 0;
  for (size_t p = 1; p < parts && ok; ++p)   // ranges in order at their boundaries
    if (cut[p] > from && cut[p] < r.size()) ok &= (r[cut[p]] >> 32) > (r[cut[p] - 1] >> 32);
  if (!ok) std::sort(r.begin() + (ptrdiff_t)from, r.end());
}

// Split entries a[0, n) into step and id arrays, in parallel over ranges for
// large reads.
inline void split_raster(const unsigned long long *a, size_t n, uint32_t *step_out, uint32_t *id_out) {
  auto work = [=](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; ++i) {
      step_out[i] = (uint32_t)(a[i] >> 32);
      id_out[i] = (uint32_t)(a[i] & 0xFFFFFFFFull);
    }
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t parts = std::min<size_t>(std::min<size_t>(hw, 16), std::max<size_t>(1, n / (1u << 20)));
  if (parts <= 1) {
    work(0, n);
    return;
  }
  std::vector<std::thread> th;
  for (size_t p = 0; p < parts; ++p) th.emplace_back(work, n * p / parts, n * (p + 1) / parts);
  for (auto &t : th) t.join();
}

}  // namespace snn
