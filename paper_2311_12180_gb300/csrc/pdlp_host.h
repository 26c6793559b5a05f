// Host-side helpers of the create paths: a small thread pool loop and the
// stable CSR transpose that builds K' from K on the host (the batched
// solver's LPs, and a single LP with a column longer than the device
// transpose's per-column sort takes).
#pragma once

#include <stdint.h>

#include <algorithm>
#include <thread>
#include <vector>

namespace pdlp {

// Threads for host work of `work` elements: at most 16, one per 2^16 elements.
inline int host_threads(int64_t work) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int64_t by_work = work / 65536 + 1;
  return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)hw, (int64_t)16, by_work}));
}

// Runs f(t) for t in [0, T) on T threads (t = 0 on the calling thread).
template <class F>
void parallel_for(int T, F f) {
  if (T <= 1) {
    f(0);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(T - 1);
  for (int t = 1; t < T; ++t) pool.emplace_back(f, t);
  f(0);
  for (auto &th : pool) th.join();
}

// K' (n rows) of K (m x n, CSR) by a counting sort that keeps, within each
// column of K, the row order: tp (n + 1), ti and tv (nnz) are exactly what
// the one-thread sort produces.  The rows of K are split into T contiguous
// ranges of about equal nonzeros; each thread counts its range's entries per
// column, the per-column counts are turned into per-thread offsets in thread
// order, and each thread then places its entries.
inline void csr_transpose(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci, const double *v, int32_t *tp,
                          int32_t *ti, double *tv) {
  const int64_t nnz = rp[m];
  const int T = std::max(1, std::min(host_threads(nnz), std::max(1, m)));
  std::vector<int32_t> rb(T + 1);
  for (int t = 0; t <= T; ++t) {
    const int64_t target = nnz * t / T;
    rb[t] = (int32_t)(std::lower_bound(rp, rp + m + 1, target) - rp);
    if (rb[t] > m) rb[t] = m;
  }
  rb[0] = 0;
  rb[T] = m;
  std::vector<int32_t> cnt((size_t)T * n, 0);
  parallel_for(T, [&](int t) {
    int32_t *c = cnt.data() + (size_t)t * n;
    for (int64_t e = rp[rb[t]]; e < rp[rb[t + 1]]; ++e) ++c[ci[e]];
  });
  // per-column totals and per-thread offsets (in thread order), column ranges in parallel
  std::vector<int32_t> tot(n);
  const int TC = host_threads(n);
  parallel_for(TC, [&](int w) {
    const int32_t c0 = (int32_t)((int64_t)n * w / TC), c1 = (int32_t)((int64_t)n * (w + 1) / TC);
    for (int32_t c = c0; c < c1; ++c) tot[c] = 0;
    for (int t = 0; t < T; ++t) {
      int32_t *row = cnt.data() + (size_t)t * n;
      for (int32_t c = c0; c < c1; ++c) {
        const int32_t k = row[c];
        row[c] = tot[c];
        tot[c] += k;
      }
    }
  });
  tp[0] = 0;
  for (int32_t c = 0; c < n; ++c) tp[c + 1] = tp[c] + tot[c];
  parallel_for(T, [&](int t) {
    int32_t *off = cnt.data() + (size_t)t * n;
    for (int32_t i = rb[t]; i < rb[t + 1]; ++i)
      for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
        const int32_t c = ci[e];
        const int32_t pos = tp[c] + off[c]++;
        ti[pos] = i;
        tv[pos] = v[e];
      }
  });
}

}  // namespace pdlp
