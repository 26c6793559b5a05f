// Host driver for the sliced-ELL layout (paper_2311_12180_gb300/csrc/pdlp_sell.h),
// used by tests/test_sell_layout_host.py: reads "rows split" and the rows + 1
// CSR row starts from stdin, runs sell_layout, and prints the layout as text:
// "total nlong nslices nitems", then perm, base, lane (one line each), then
// one line per work item (first row, rows or -1, length, offset).
#include <cstdio>
#include <vector>

#include "pdlp_sell.h"

int main() {
  int rows = 0, split = 0;
  if (std::scanf("%d %d", &rows, &split) != 2 || rows < 0 || split < 0 || split > rows) return 2;
  std::vector<int32_t> ptr((size_t)rows + 1);
  for (int i = 0; i <= rows; ++i)
    if (std::scanf("%d", &ptr[i]) != 1) return 2;
  const pdlp::SellLayout S = pdlp::sell_layout(ptr.data(), rows, split);
  std::printf("%lld %d %d %zu\n", (long long)S.total, S.nlong, S.nslices, S.items.size());
  for (int i = 0; i < rows; ++i) std::printf("%d ", S.perm[i]);
  std::printf("\n");
  for (int i = 0; i < rows; ++i) std::printf("%d ", S.base[i]);
  std::printf("\n");
  for (int i = 0; i < rows; ++i) std::printf("%d ", (int)S.lane[i]);
  std::printf("\n");
  for (const int4 &it : S.items) std::printf("%d %d %d %d\n", it.x, it.y, it.z, it.w);
  return 0;
}
