// Host side of the sliced-ELL layout of K and K' (see SellMat in
// pdlp_internal.cuh): the internal row order, where every row's entries go,
// and the work items in schedule order.  Only row lengths are needed here;
// the device copies the entries (pdlp_setup.cu, setup_sell_fill).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "pdlp_internal.cuh"

namespace pdlp {

struct SellLayout {
  std::vector<int32_t> perm;    // internal row -> original row
  std::vector<int32_t> base;    // internal row -> position of its entry 0
  std::vector<uint8_t> lane;    // internal row -> 1: entries 32 apart (slice), 0: contiguous (long row)
  std::vector<int4> items;      // schedule order
  int64_t total = 0;            // stored entries, padding included
  int32_t nlong = 0, nslices = 0;
};

// Rows [0, split) and [split, rows) of the original order form two groups
// that keep their order relative to each other (the equality rows of K come
// first, so the dual projection still tests "internal row >= n_eq"); inside a
// group rows are sorted by length, longest first (stable).  Rows longer than
// SELL_LONG become long-row items, the others fill slices of 32 consecutive
// internal rows that never cross a group.  Items are then ordered by
// estimated cost, longest first, which the kernels walk in a snake order
// over the warps of the grid (balanced within a fraction of one item).
inline SellLayout sell_layout(const int32_t *ptr, int32_t rows, int32_t split) {
  SellLayout S;
  S.perm.resize(rows);
  S.base.resize(rows);
  S.lane.resize(rows);
  int32_t maxlen = 0;
  for (int32_t i = 0; i < rows; ++i) maxlen = std::max(maxlen, ptr[i + 1] - ptr[i]);
  std::vector<int32_t> cnt((size_t)maxlen + 2);
  int32_t at = 0;  // next internal row
  int64_t off = 0;
  struct Cost {
    int64_t cost;
    int32_t k;
  };
  std::vector<Cost> order;
  const int32_t bounds[3] = {0, split, rows};
  for (int g = 0; g < 2; ++g) {
    const int32_t r0 = bounds[g], r1 = bounds[g + 1];
    if (r1 <= r0) continue;
    // stable counting sort of the group's rows by length, descending
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int32_t i = r0; i < r1; ++i) cnt[maxlen - (ptr[i + 1] - ptr[i])]++;
    int32_t acc = at;
    for (int32_t k = 0; k <= maxlen; ++k) {
      const int32_t c = cnt[k];
      cnt[k] = acc;
      acc += c;
    }
    for (int32_t i = r0; i < r1; ++i) S.perm[cnt[maxlen - (ptr[i + 1] - ptr[i])]++] = i;
    int32_t r = at;
    const int32_t end = at + (r1 - r0);
    for (; r < end; ++r) {  // long rows lead the group
      const int32_t len = ptr[S.perm[r] + 1] - ptr[S.perm[r]];
      if (len <= SELL_LONG) break;
      S.base[r] = (int32_t)off;
      S.lane[r] = 0;
      S.items.push_back(make_int4(r, -1, len, (int32_t)off));
      order.push_back({(int64_t)(len + 31) / 32 + 2, (int32_t)S.items.size() - 1});
      off += (int64_t)(len + 31) / 32 * 32;
      S.nlong++;
    }
    for (; r < end; r += 32) {  // slices
      const int32_t nr = std::min<int32_t>(32, end - r);
      const int32_t L = ptr[S.perm[r] + 1] - ptr[S.perm[r]];
      for (int32_t l = 0; l < nr; ++l) {
        S.base[r + l] = (int32_t)(off + l);
        S.lane[r + l] = 1;
      }
      S.items.push_back(make_int4(r, nr, L, (int32_t)off));
      order.push_back({(int64_t)L + 2, (int32_t)S.items.size() - 1});
      off += (int64_t)32 * L;
      S.nslices++;
    }
    at = end;
  }
  S.total = off;
  std::stable_sort(order.begin(), order.end(), [](const Cost &a, const Cost &b) { return a.cost > b.cost; });
  std::vector<int4> sorted(S.items.size());
  for (size_t k = 0; k < order.size(); ++k) sorted[k] = S.items[order[k].k];
  S.items.swap(sorted);
  return S;
}

}  // namespace pdlp
