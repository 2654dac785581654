// FP64 exponential for the Arrhenius and equilibrium factors of the chemistry.
//
// Method: the table-driven reduction of P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic",
// ACM TOMS 15(2), 1989: x = (32 m + j) ln2/32 + r with |r| <= ln2/64, so
// exp(x) = 2^m * 2^(j/32) * exp(r). Here 2^(j/32) comes from a 32-entry table
// of doubles, exp(r) from its Taylor polynomial of degree 6 (truncation below
// 4e-18 relative for |r| <= ln2/64), the rounding of x*32/ln2 to an integer from
// the usual add-and-subtract of 1.5*2^52, and ln2/32 is split in two parts so
// that N * hi is exact for |N| < 2^21. The scaling by 2^m adds m to the exponent
// field. About 11 FP64 operations instead of the ~20 of a general exp; accuracy
// within a few ulp (checked against CUDA's exp by the tests).
#pragma once
#include <cstdint>

namespace adg {

constexpr double EXP_SHIFTER = 6755399441055744.0;        // 1.5 * 2^52
constexpr double EXP_INV_L = 46.16624130844682836;        // 32 / ln 2
constexpr double EXP_MAX_ARG = 700.0;

// Table and the hi/lo split of ln2/32 (hi with 32 significant bits), computed on
// the host in extended precision.
struct ExpTable {
  double t[32];     // 2^(j/32), rounded to double
  double l_hi, l_lo;
};

// exp(x) with the table in shared memory (tab). Falls back to the library exp
// outside |x| <= 700, where the exponent-field scaling could leave the range.
__device__ __forceinline__ double fexp(double x, const ExpTable &tab) {
  // |x| <= 700 tested on the high word (0x4085E000 is that of 700.0), off the FP64 pipe;
  // NaN and infinities take the library path too
  if ((__double2hiint(x) & 0x7fffffff) > 0x4085E000) return exp(x);
  double t = fma(x, EXP_INV_L, EXP_SHIFTER);
  double nd = t - EXP_SHIFTER;
  int n = (int)(__double2loint(t));          // the low mantissa bits hold N
  double r = fma(-nd, tab.l_hi, x);
  r = fma(-nd, tab.l_lo, r);
  double p = 1.0 / 720.0;
  p = fma(p, r, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  int j = n & 31;
  int m = n >> 5;                             // arithmetic shift: floor division
  double v = tab.t[j] * p;
  long long bits = __double_as_longlong(v) + ((long long)m << 52);
  return __longlong_as_double(bits);
}

}  // namespace adg
