// Test harness (not part of the library): the library's integer-pipeline exp
// (csrc/adg_math.cuh), compiled for the host, against expl in extended precision
// over the argument ranges the chemistry uses. Prints the largest error in units
// in the last place of the correctly rounded result as one JSON line.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "../../paper_2501_01747_gb300/csrc/adg_math.cuh"

int main() {
  const adg::IExpTable tab = {ADG_IEXP_TABLE, ADG_IEXP_TABLE32};
  const int n = 1 << 22;
  srand(2501);
  double max_ulp = 0.0, worst = 0.0, max_ulp_f = 0.0;
  long long exact = 0, exact_f = 0;
  for (int i = 0; i < n; ++i) {
    double u = (double)rand() / RAND_MAX;
    double x;
    if (i % 5 == 0) x = -700.0 + 1400.0 * u;     // whole range
    else if (i % 5 == 1) x = -80.0 + 120.0 * u;  // Arrhenius arguments
    else if (i % 5 == 2) x = (u - 0.5) * 1e-3;   // near zero
    else if (i % 5 == 3) x = ldexp(u - 0.5, -(i % 60));  // tiny arguments
    else x = (double)((i / 5) % 2000 - 1000) * (0.6931471805599453 / 32.0);  // table nodes
    double got = adg::iexp(x, tab);
    long double ref = expl((long double)x);
    double rd = (double)ref;
    double ulp = std::nextafter(rd, INFINITY) - rd;
    double e = (double)fabsl((long double)got - ref) / ulp;
    if (got == rd) ++exact;
    if (e > max_ulp) {
      max_ulp = e;
      worst = x;
    }
    // the float variant, where the result is a normal float
    if (ref > 1.2e-38L && ref < 3.4e38L) {
      float gf = adg::iexpf(x, tab), rf = (float)ref;
      float ulpf = std::nextafter(rf, INFINITY) - rf;
      double ef = (double)(fabsl((long double)gf - ref) / ulpf);
      if (gf == rf) ++exact_f;
      if (ef > max_ulp_f) max_ulp_f = ef;
    }
  }
  printf("{\"n\": %d, \"max_ulp\": %.4f, \"worst_x\": %.17g, \"correctly_rounded\": %.6f, "
         "\"float_max_ulp\": %.4f}\n", n, max_ulp, worst, (double)exact / n, max_ulp_f);
  return 0;
}
