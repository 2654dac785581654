// Test harness (not part of the library): the library's integer-pipeline exp
// and its table-driven logarithm (csrc/adg_math.cuh), compiled for the host,
// against expl and logl in extended precision over the argument ranges the
// chemistry uses. Prints the largest error in units
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
  // the FP32-pipe exp of a df32 argument (the mixed chemistry), over the
  // argument range whose result is a normal float
  float tf[64];
  for (int j = 0; j < 32; ++j) adg::iexp_table_df(tab.t32[j], tf + 2 * j, tf + 2 * j + 1);
  double max_ulp_df = 0.0, worst_df = 0.0;
  long long exact_df = 0, n_df = 0;
  for (int i = 0; i < n; ++i) {
    double u = (double)rand() / RAND_MAX;
    double x = (i % 3 == 0) ? -87.0 + 175.0 * u : (i % 3 == 1 ? -40.0 + 60.0 * u : (u - 0.5) * 1e-2);
    const adg::DF d = adg::df_split(x);
    long double ref = expl((long double)d.hi + (long double)d.lo);
    if (!(ref > 1.2e-38L && ref < 3.4e38L)) continue;
    float g = adg::exp_df(d, tf), rf = (float)ref;
    float ulpf = std::nextafter(rf, INFINITY) - rf;
    double e = (double)(fabsl((long double)g - ref) / ulpf);
    ++n_df;
    if (g == rf) ++exact_df;
    if (e > max_ulp_df) {
      max_ulp_df = e;
      worst_df = x;
    }
  }
  // the table-driven logarithm of the mixed variant's ln T: temperatures, the
  // table nodes and their neighbours, and the whole normal range
  const adg::LogTable ltab = {ADG_LOG_TABLE_LN, ADG_LOG_TABLE_INV};
  double max_ulp_ln = 0.0, worst_ln = 0.0, max_abs_t = 0.0;
  for (int i = 0; i < n; ++i) {
    double u = (double)rand() / RAND_MAX;
    double x;
    if (i % 4 == 0) x = 50.0 + 9950.0 * u;                                  // temperatures
    else if (i % 4 == 1) x = ldexp(1.0 + ((i / 4) % 128) / 128.0, (i / 512) % 40 - 20);  // nodes
    else if (i % 4 == 2) x = std::nextafter(ldexp(1.0 + ((i / 4) % 128) / 128.0, (i / 512) % 40 - 20), 0.0);
    else x = ldexp(0.5 + 0.5 * u, (i / 4) % 2040 - 1020);                    // whole range
    const double got = adg::log_tab(x, ltab);
    const long double ref = logl((long double)x);
    const double rd = (double)ref;
    if (rd == 0.0) {
      if (got != 0.0) max_ulp_ln = 1e30;
      continue;
    }
    const double ulp = std::nextafter(fabs(rd), INFINITY) - fabs(rd);
    const double e = (double)(fabsl((long double)got - ref) / ulp);
    if (e > max_ulp_ln) {
      max_ulp_ln = e;
      worst_ln = x;
    }
    if (i % 4 == 0) max_abs_t = fmax(max_abs_t, (double)fabsl((long double)got - ref));
  }
  // both sides of x = 1 (the library's logarithm) and the edges of [1/2, 2)
  for (int i = 0; i < n / 8; ++i) {
    const double x = (i % 3 == 0) ? 1.0 + ldexp((double)rand() / RAND_MAX - 0.5, -(i % 50) - 1)
                     : ldexp(1.0, (i % 3 == 1) ? -1 : 1) *
                           (1.0 + ldexp((double)rand() / RAND_MAX - 0.5, -(i % 50) - 2));
    const double got = adg::log_tab(x, ltab);
    const long double ref = logl((long double)x);
    const double rd = (double)ref;
    if (rd == 0.0) continue;
    const double ulp = std::nextafter(fabs(rd), INFINITY) - fabs(rd);
    const double e = (double)(fabsl((long double)got - ref) / ulp);
    if (e > max_ulp_ln) {
      max_ulp_ln = e;
      worst_ln = x;
    }
  }
  printf("{\"n\": %d, \"max_ulp\": %.4f, \"worst_x\": %.17g, \"correctly_rounded\": %.6f, "
         "\"float_max_ulp\": %.4f, \"df_max_ulp\": %.4f, \"df_worst_x\": %.9g, "
         "\"df_correctly_rounded\": %.4f, \"log_max_ulp\": %.4f, \"log_worst_x\": %.17g, "
         "\"log_max_abs_T\": %.3g}\n", n, max_ulp, worst, (double)exact / n, max_ulp_f,
         max_ulp_df, worst_df, (double)exact_df / (n_df ? n_df : 1), max_ulp_ln, worst_ln,
         max_abs_t);
  return 0;
}
