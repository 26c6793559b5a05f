// Host driver for the threaded stable CSR transpose (csr_transpose in
// paper_2311_12180_gb300/csrc/pdlp_host.h), used by
// tests/test_sell_layout_host.py: reads "m n nnz", the m + 1 row starts, the
// column indices and the values (as hexadecimal IEEE bits) from stdin, and
// prints the n + 1 row starts of K', its column indices and its values' bits.
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <vector>

#include "pdlp_host.h"

int main() {
  int m = 0, n = 0;
  long long nnz = 0;
  if (std::scanf("%d %d %lld", &m, &n, &nnz) != 3 || m < 0 || n < 0 || nnz < 0) return 2;
  std::vector<int32_t> rp((size_t)m + 1), ci((size_t)nnz + 1), tp((size_t)n + 1), ti((size_t)nnz + 1);
  std::vector<double> v((size_t)nnz + 1), tv((size_t)nnz + 1);
  for (int i = 0; i <= m; ++i)
    if (std::scanf("%d", &rp[i]) != 1) return 2;
  for (long long e = 0; e < nnz; ++e)
    if (std::scanf("%d", &ci[e]) != 1) return 2;
  for (long long e = 0; e < nnz; ++e) {
    uint64_t bits = 0;
    if (std::scanf("%" SCNx64, &bits) != 1) return 2;
    std::memcpy(&v[e], &bits, 8);
  }
  pdlp::csr_transpose(m, n, rp.data(), ci.data(), v.data(), tp.data(), ti.data(), tv.data());
  for (int c = 0; c <= n; ++c) std::printf("%d ", tp[c]);
  std::printf("\n");
  for (long long e = 0; e < nnz; ++e) std::printf("%d ", ti[e]);
  std::printf("\n");
  for (long long e = 0; e < nnz; ++e) {
    uint64_t bits;
    std::memcpy(&bits, &tv[e], 8);
    std::printf("%" PRIx64 " ", bits);
  }
  std::printf("\n");
  return 0;
}
