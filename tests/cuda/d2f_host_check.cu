// Test harness (not part of the library): the integer double -> float conversion
// of the doubles outside the normal float range (d2f_edge_bits in
// csrc/adg_math.cuh), compiled for the host, against the host's own conversion
// (IEEE round to nearest even, subnormals kept), bit for bit; NaN only as NaN.
// Prints one JSON line.
#include <cstdio>
#include <cstring>

#include "../../paper_2501_01747_gb300/csrc/adg_math.cuh"
#include "d2f_edge_values.h"

int main() {
  srand(2501);
  const std::vector<double> v = d2f_edge_values(1 << 20);
  long long checked = 0, mismatch = 0, nan_bad = 0;
  for (double x : v) {
    unsigned long long b;
    std::memcpy(&b, &x, 8);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int ef = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (!(ef <= 0 || ef >= 255)) continue;  // the fast conversion's domain
    ++checked;
    const unsigned got = adg::d2f_edge_bits(hi, lo);
    const float ref = (float)x;
    unsigned rb;
    std::memcpy(&rb, &ref, 4);
    if (std::isnan(x)) {
      float g;
      std::memcpy(&g, &got, 4);
      if (!std::isnan(g)) ++nan_bad;
    } else if (got != rb) {
      if (mismatch < 5) printf("# x=%a got=%08x ref=%08x\n", x, got, rb);
      ++mismatch;
    }
  }
  printf("{\"checked\": %lld, \"mismatch\": %lld, \"nan_bad\": %lld}\n", checked, mismatch,
         nan_bad);
  return 0;
}
