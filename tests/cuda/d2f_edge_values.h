// Test inputs (not part of the library): doubles at and beyond the edges of the
// float range, for the integer-pipe double -> float conversion. Signed zeros,
// subnormal doubles, values whose float is subnormal (random significands, exact
// ties between neighbouring subnormals, half the smallest subnormal and just
// around it), the boundary to the normal range, the largest float and the ties
// and values around it, values beyond the float range, infinities and NaN.
#pragma once
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <vector>

inline std::vector<double> d2f_edge_values(int n_random) {
  std::vector<double> v = {0.0, -0.0, 4.9406564584124654e-324, -2.2250738585072009e-308,
                           ldexp(1.0, -150), ldexp(1.0, -151), ldexp(1.0, -149),
                           ldexp(3.0, -151), ldexp(1.0, -126), ldexp(1.0 - ldexp(1.0, -24), -126),
                           ldexp(1.0 - ldexp(1.0, -25), -126), (double)FLT_MAX,
                           (double)FLT_MAX + ldexp(1.0, 103), (double)FLT_MAX + ldexp(1.0, 102),
                           (double)FLT_MAX + ldexp(1.0, 103) - ldexp(1.0, 75), ldexp(1.0, 128),
                           1e39, DBL_MAX, INFINITY, -INFINITY, NAN, -NAN};
  for (int k = -160; k <= -120; ++k)
    for (int j = 0; j < 16; ++j) v.push_back(ldexp(1.0 + j / 16.0, k));
  for (int i = 0; i < n_random; ++i) {
    const double u = (double)rand() / RAND_MAX;
    const int q = rand() & 0x7fffff;
    switch (i % 5) {
      case 0: v.push_back(ldexp(1.0 + u, -127 - (i / 5) % 30)); break;  // subnormal floats
      case 1: v.push_back(ldexp(q + 0.5, -149)); break;                  // exact ties
      case 2: v.push_back(ldexp(q + 0.5 + ldexp(1.0, -20), -149)); break;  // just above
      case 3: v.push_back(ldexp(1.0 + u, 128 + (i / 5) % 500)); break;   // beyond the range
      default: v.push_back(ldexp(1.0 + u, -1022 - (i / 5) % 40)); break;  // tiny doubles
    }
    if (i & 1) v.back() = -v.back();
  }
  return v;
}
