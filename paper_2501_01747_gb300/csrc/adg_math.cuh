// FP64 exponential for the Arrhenius and equilibrium factors of the chemistry,
// evaluated on the integer pipeline.
//
// Method: the table-driven reduction of P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic",
// ACM TOMS 15(2), 1989: x = (32 m + j) ln2/32 + r with |r| <= ln2/64, so
// exp(x) = 2^m * 2^(j/32) * exp(r). Every step is carried out in 64-bit fixed
// point instead of double arithmetic, because on this GPU a double instruction
// occupies the FP64 unit for 16 cycles while integer multiply-adds issue at the
// rate of single-precision ones:
//   n = round(|x| 32/ln2) from the high half of |x| 2^53 * round(2^56 32/ln2),
//   r 2^69 = |x| 2^69 - n (2^69 ln2/32), with |x| 2^69 the significand shifted
//   left (modulo 2^64: the true value is below 2^62.5 in magnitude, so the low
//   64 bits are exact) and 2^69 ln2/32 as a 64-bit integer plus a 32-bit
//   fraction; exact for |x| >= 2^-17 and to 2^-70 below,
//   exp(r) = 1 + r(1 + r(1/2 + r(1/6 + r(1/24 + r(1/120 + r/720))))) by Horner with
//   64-bit high multiplies (coefficients and partial sums scaled by 2^62, r by
//   2^64; the truncated Taylor term is below 2^-58 for |r| <= ln2/64),
//   2^(j/32) exp(r) from the high half of the product with the table entry
//   (scaled by 2^62), then rounded to a 53-bit significand with m added to the
//   exponent. Negative x use n -> -n, r -> -r.
// The error is about half a unit in the last place; the tests compare it with
// the host's and with CUDA's exp.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

namespace adg {

// 2^(j/32) * 2^62 and the constants below, rounded to the nearest integer from
// 60-digit decimal evaluations of their definitions.
#define ADG_IEXP_TABLE                                                              \
  {0x4000000000000000ull, 0x4166c34c5615d0ecull, 0x42d561b3e6243d8aull,            \
   0x444c0740496d4294ull, 0x45cae0f1f545eb73ull, 0x47521cc5a2e6a9e0ull,            \
   0x48e1e9b9d588e19bull, 0x4a7a77d47f7b84b1ull, 0x4c1bf828c6dc54b8ull,            \
   0x4dc69cdceaa72a9cull, 0x4f7a993048d088d7ull, 0x513821818624b40cull,            \
   0x52ff6b54d8a89c75ull, 0x54d0ad5a753e077cull, 0x56ac1f752150a563ull,            \
   0x5891fac0e95612c8ull, 0x5a827999fcef3242ull, 0x5c7dd7a3b17dcf75ull,            \
   0x5e8451cfac061b5full, 0x6096266533384a2bull, 0x62b39508aa836d6full,            \
   0x64dcdec3371793d1ull, 0x6712460a8fc24072ull, 0x69540ec8f895722dull,            \
   0x6ba27e656b4eb57aull, 0x6dfddbcbed791babull, 0x70666f76154a7089ull,            \
   0x72dc8373be41a454ull, 0x75606373ee921c97ull, 0x77f25ccdee6d7ae6ull,            \
   0x7a92be8a92436616ull, 0x7d41d96db915019dull}

// 2^(j/32) * 2^31, rounded to the nearest integer (the float-result variant).
#define ADG_IEXP_TABLE32                                                            \
  {0x80000000u, 0x82cd8699u, 0x85aac368u, 0x88980e81u, 0x8b95c1e4u, 0x8ea4398bu,   \
   0x91c3d374u, 0x94f4efa9u, 0x9837f052u, 0x9b8d39bau, 0x9ef53261u, 0xa2704303u,   \
   0xa5fed6aau, 0xa9a15ab5u, 0xad583eeau, 0xb123f582u, 0xb504f334u, 0xb8fbaf47u,   \
   0xbd08a39fu, 0xc12c4ccau, 0xc5672a11u, 0xc9b9bd86u, 0xce248c15u, 0xd2a81d92u,   \
   0xd744fccbu, 0xdbfbb798u, 0xe0ccdeecu, 0xe5b906e7u, 0xeac0c6e8u, 0xefe4b99cu,   \
   0xf5257d15u, 0xfa83b2dbu}

struct IExpTable {
  unsigned long long t[32];
  unsigned int t32[32];
  float tf[64];  // 2^(j/32) as float pairs (iexp_table_df), filled where used
};

constexpr unsigned long long IEXP_K = 3326628274461080623ull;   // 2^56 * 32/ln2
constexpr unsigned long long IEXP_L = 12786308645202655660ull;  // 2^69 * ln2/32
constexpr long long IEXP_LC = -907824232ll;  // (2^69 ln2/32 - IEXP_L) * 2^32
constexpr long long IEXP_C0 = 4611686018427387904ll;            // 2^62 / k!
constexpr long long IEXP_C2 = 2305843009213693952ll;
constexpr long long IEXP_C3 = 768614336404564651ll;
constexpr long long IEXP_C4 = 192153584101141163ll;
constexpr long long IEXP_C5 = 38430716820228233ll;
constexpr long long IEXP_C6 = 6405119470038039ll;
constexpr int IEXPF_C0 = 1073741824;  // 2^30 / k!
constexpr int IEXPF_C2 = 536870912;
constexpr int IEXPF_C3 = 178956971;
constexpr int IEXPF_C4 = 44739243;

__host__ __device__ __forceinline__ unsigned long long iexp_umulhi(unsigned long long a,
                                                                   unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ long long iexp_smulhi(long long a, long long b) {
#ifdef __CUDA_ARCH__
  return __mul64hi(a, b);
#else
  return (long long)(((__int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ long long iexp_bits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}

__host__ __device__ __forceinline__ double iexp_double(long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}

__host__ __device__ __forceinline__ int iexp_clz(unsigned long long v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

__host__ __device__ __forceinline__ int iexp_mulhi32(int a, int b) {
#ifdef __CUDA_ARCH__
  return __mulhi(a, b);
#else
  return (int)(((long long)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ unsigned int iexp_umulhi32(unsigned int a, unsigned int b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (unsigned int)(((unsigned long long)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ int iexp_clz32(unsigned int v) {
#ifdef __CUDA_ARCH__
  return __clz((int)v);
#else
  return __builtin_clz(v);
#endif
}

// Argument reduction, exact in 64-bit fixed point: for |x| <= 700,
// x = n ln2/32 + r with r 2^69 = R, |r| <= ln2/64.
struct IExpRed {
  long long R, n;
};

__host__ __device__ __forceinline__ IExpRed iexp_reduce(long long bits) {
  const int E = (int)((bits >> 52) & 0x7ff);
  const unsigned long long mant = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - 1022;  // |x| 2^53 = mant 2^sh, sh <= 10
  const unsigned long long X = sh >= 0 ? mant << sh : (sh > -60 ? mant >> -sh : 0ull);
  const long long n = (long long)((iexp_umulhi(X, IEXP_K) + (1ull << 44)) >> 45);
  const int t = E - 1006;  // |x| 2^69 = mant 2^t, t <= 26
  const unsigned long long X69 =
      t >= 0 ? mant << t : (t > -60 ? ((mant >> (-t - 1)) + 1) >> 1 : 0ull);
  IExpRed o;
  o.R = (long long)(X69 - (unsigned long long)n * IEXP_L) - ((n * IEXP_LC) >> 32);
  o.n = n;
  if (bits < 0) {
    o.R = -o.R;
    o.n = -o.n;
  }
  return o;
}

// Fixed-point core: for |x| <= 700, exp(x) = V 2^(m-60) with 2^59.9 < V < 2^61.1.
struct IExpParts {
  unsigned long long V;
  int m;
};

__host__ __device__ __forceinline__ IExpParts iexp_parts(long long bits, const IExpTable &tab) {
  const IExpRed red = iexp_reduce(bits);
  const long long r = red.R >> 5;  // r 2^64
  long long A = IEXP_C6;
  A = IEXP_C5 + iexp_smulhi(r, A);
  A = IEXP_C4 + iexp_smulhi(r, A);
  A = IEXP_C3 + iexp_smulhi(r, A);
  A = IEXP_C2 + iexp_smulhi(r, A);
  A = IEXP_C0 + iexp_smulhi(r, A);
  A = IEXP_C0 + iexp_smulhi(r, A);  // exp(r) 2^62
  IExpParts o;
  o.V = iexp_umulhi(tab.t[(int)(red.n & 31)], (unsigned long long)A);  // 2^(j/32) exp(r) 2^60
  o.m = (int)(red.n >> 5);  // arithmetic shift: floor division
  return o;
}

// exp(x) with the table in shared (or host) memory. Outside |x| <= 700 (and for
// NaN and infinities) the library exp is returned.
__host__ __device__ __forceinline__ double iexp(double x, const IExpTable &tab) {
  const long long bits = iexp_bits(x);
  // 0x4085E000 is the high word of 700.0
  if ((int)((bits >> 32) & 0x7fffffff) > 0x4085E000) return exp(x);
  const IExpParts p = iexp_parts(bits, tab);
  const int s = 11 - iexp_clz(p.V);  // leading bit 59..61 -> s = 7..9
  const unsigned long long mt = (p.V + (1ull << (s - 1))) >> s;  // 2^52 <= mt <= 2^53
  const long long eb = (long long)(s - 8 + p.m + 1023) << 52;
  return iexp_double(eb + (long long)(mt - (1ull << 52)));
}

__host__ __device__ __forceinline__ float iexp_float(int b) {
#ifdef __CUDA_ARCH__
  return __int_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, 4);
  return x;
#endif
}

// The exponential of a double argument rounded once to float (results below the
// smallest normal float flush to zero, above the largest give +inf). The
// reduction is the exact 64-bit one above; a float needs only 24 bits of exp(r)
// and 2^(j/32), so those run in 32-bit fixed point: degree-4 Taylor Horner with
// r scaled by 2^32 and the partial sums by 2^30 (truncation r^5/120 < 2^-39),
// the table scaled by 2^31. The value before the rounding is good to ~2^-29.
__host__ __device__ __forceinline__ float iexpf(double x, const IExpTable &tab) {
  const long long bits = iexp_bits(x);
  if ((int)((bits >> 32) & 0x7fffffff) > 0x4085E000) return (float)exp(x);
  const IExpRed red = iexp_reduce(bits);
  const int r = (int)(red.R >> 37);  // r 2^32, |r| < 2^26
  int A = IEXPF_C4;
  A = IEXPF_C3 + iexp_mulhi32(r, A);
  A = IEXPF_C2 + iexp_mulhi32(r, A);
  A = IEXPF_C0 + iexp_mulhi32(r, A);
  A = IEXPF_C0 + iexp_mulhi32(r, A);  // exp(r) 2^30
  const unsigned int V = iexp_umulhi32(tab.t32[(int)(red.n & 31)], (unsigned int)A);  // 2^29 scale
  const int m = (int)(red.n >> 5);
  const int s = 8 - iexp_clz32(V);  // leading bit 28..30 -> s = 5..7
  const unsigned int mt = (V + (1u << (s - 1))) >> s;  // 2^23 <= mt <= 2^24
  const int e = s - 6 + m + 127;  // biased exponent of mt 2^(s-29+m-23)
  if (e <= 0) return 0.0f;
  if (e >= 255) return iexp_float(0x7f800000);
  return iexp_float((e << 23) + (int)(mt - (1u << 23)));
}

// ---------------------------------------------------------------------------
// Float-float ("df32") arithmetic for the mixed-precision chemistry: a value is
// hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits, on the FP32 pipe
// (on this GPU FP64 instructions and double<->float conversions both occupy the
// scarce FP64 unit). Error-free transforms: Dekker's product by a fused
// multiply-add and Knuth's two-sum (Dekker, Numer. Math. 18, 1971; Knuth, TAOCP
// vol. 2). The _rn intrinsics keep the compiler from contracting the sums.
struct DF {
  float hi, lo;
};

#ifdef __CUDA_ARCH__
#define ADG_FADD(a, b) __fadd_rn(a, b)
#define ADG_FSUB(a, b) __fsub_rn(a, b)
#define ADG_FMUL(a, b) __fmul_rn(a, b)
#else
#define ADG_FADD(a, b) ((a) + (b))
#define ADG_FSUB(a, b) ((a) - (b))
#define ADG_FMUL(a, b) ((a) * (b))
#endif

// The df32 value nearest to x (hi the rounded float, lo the rounded remainder).
__host__ __device__ __forceinline__ DF df_split(double x) {
  const float h = (float)x;
  return DF{h, (float)(x - (double)h)};
}

// a b + c, all df32 (relative error about 2^-46).
__host__ __device__ __forceinline__ DF df_fma(DF a, DF b, DF c) {
  const float p = ADG_FMUL(a.hi, b.hi);
  float pe = fmaf(a.hi, b.hi, -p);  // the rounding error of p, exactly
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  const float s = ADG_FADD(p, c.hi);  // two-sum of p and c.hi
  const float bb = ADG_FSUB(s, p);
  float e = ADG_FADD(ADG_FSUB(p, ADG_FSUB(s, bb)), ADG_FSUB(c.hi, bb));
  e = ADG_FADD(e, ADG_FADD(pe, c.lo));
  const float h = ADG_FADD(s, e);  // renormalise
  return DF{h, ADG_FSUB(e, ADG_FSUB(h, s))};
}

// 2^(j/32) as a float pair tf[2j] + tf[2j+1] (the rounded float and the
// remainder), from the 32-bit table entry (scaled by 2^31): good to about 2^-32.
__host__ __device__ __forceinline__ void iexp_table_df(unsigned int t32, float *hi, float *lo) {
  const float h = (float)t32;                                 // 24 leading bits
  const float l = (float)((long long)t32 - (long long)h);     // the rest, exactly
  *hi = ADG_FMUL(h, 4.656612873077393e-10f);                  // 2^-31, exact
  *lo = ADG_FMUL(l, 4.656612873077393e-10f);
}

// exp(x) for a df32 argument, float result, on the FP32 pipe: Tang's table
// reduction (ACM TOMS 15(2), 1989) in float-float, t = x 32/ln2, n = rint(t),
// r = (t - n) ln2/32 with |r| <= ln2/64, exp(x) = 2^(n >> 5) 2^((n & 31)/32) e^r
// with e^r - 1 by the degree-4 Taylor polynomial (truncation below r^5/120 <
// 2^-38) and the table entry as a float pair, combined as
// t_hi + (t_hi (e^r - 1) + t_lo) so that one final rounding dominates: about half
// a unit in the last place. Results below the normal range are flushed to zero;
// above it the result is infinity.
__host__ __device__ __forceinline__ float exp_df(DF x, const float *tf) {
  const DF K = {46.16624069f, 6.1630817e-07f};  // 32/ln2 as df32
  if (!(x.hi < 88.8f)) return (x.hi != x.hi) ? x.hi : iexp_float(0x7f800000);
  if (!(x.hi > -103.0f)) return 0.0f;
  const DF t = df_fma(x, K, DF{0.0f, 0.0f});
  const float nf = rintf(t.hi);
  const int n = (int)nf;
  const float r = ADG_FMUL(ADG_FADD(ADG_FSUB(t.hi, nf), t.lo), 0.021660849f);  // ln2/32
  float q = fmaf(r, 0.041666668f, 0.16666667f);
  q = fmaf(r, q, 0.5f);
  q = fmaf(r, q, 1.0f);
  q = ADG_FMUL(r, q);  // e^r - 1
  const float th = tf[2 * (n & 31)], tl = tf[2 * (n & 31) + 1];
  const float v = ADG_FADD(th, fmaf(th, q, tl));  // in [0.98, 2.03)
  int vb;
  std::memcpy(&vb, &v, 4);
  const int e = ((vb >> 23) & 0xff) + (n >> 5);
  if (e <= 0) return 0.0f;
  if (e >= 255) return iexp_float(0x7f800000);
  vb += (n >> 5) << 23;
  float o;
  std::memcpy(&o, &vb, 4);
  return o;
}

}  // namespace adg
