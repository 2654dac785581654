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

// The library exp for the rare arguments iexp leaves to it, out of line: inline,
// its FP64 instructions may be issued, predicated off, on every call.
static __host__ __device__ __noinline__ double iexp_slow(double x) { return exp(x); }

// exp(x) with the table in shared (or host) memory. Outside |x| <= 700 (and for
// NaN and infinities) the library exp is returned.
__host__ __device__ __forceinline__ double iexp(double x, const IExpTable &tab) {
  const long long bits = iexp_bits(x);
  // 0x4085E000 is the high word of 700.0
  if ((int)((bits >> 32) & 0x7fffffff) > 0x4085E000) return iexp_slow(x);
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
struct alignas(8) DF {
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

// a + b, a - b and a b, all df32 (relative error about 2^-46; the sum by
// Knuth's two-sum of the high parts, the product by Dekker's with an FMA).
__host__ __device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = ADG_FADD(a.hi, b.hi);
  const float bb = ADG_FSUB(s, a.hi);
  float e = ADG_FADD(ADG_FSUB(a.hi, ADG_FSUB(s, bb)), ADG_FSUB(b.hi, bb));
  e = ADG_FADD(e, ADG_FADD(a.lo, b.lo));
  const float h = ADG_FADD(s, e);
  return DF{h, ADG_FSUB(e, ADG_FSUB(h, s))};
}
__host__ __device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
__host__ __device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = ADG_FMUL(a.hi, b.hi);
  float pe = fmaf(a.hi, b.hi, -p);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  const float h = ADG_FADD(p, pe);
  return DF{h, ADG_FSUB(pe, ADG_FSUB(h, p))};
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

// Natural logarithm for the mixed variant's ln T (its float-float Arrhenius
// arguments need about 1e-12): the table-driven method of P. T. P. Tang,
// "Table-driven implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16(4), 1990. x = 2^k m with m in [1, 2); the node
// c = 1 + j/128 at or below m (j the top 7 bits of m's fraction) makes m - c
// exact and u = (m - c)/c, taken as (m - c) times the table's 1/c, lie in
// [0, 1/128); ln x = k ln2 + ln c + ln(1 + u), with ln(1 + u) by its Taylor
// series to u^7 (the first omitted term is below 2^-59) and ln2 split so that
// k L_hi is exact. For x >= 2 the three terms are positive, and for x < 1/2
// they cancel by at most a factor 2, so the error stays near one unit in the
// last place, in 13 double operations where a full-precision library logarithm
// takes several times that. x in [1/2, 2), where k ln2 and ln c would cancel,
// and x that is not a positive normal number take the library logarithm.
// ln(1 + j/128) and 128/(128 + j), rounded to nearest from 60-digit evaluations.
#define ADG_LOG_TABLE_LN \
  {0x0.0p+0, 0x1.fe02a6b106789p-8, 0x1.fc0a8b0fc03e4p-7, 0x1.7b91b07d5b11bp-6, \
   0x1.f829b0e783300p-6, 0x1.39e87b9febd60p-5, 0x1.77458f632dcfcp-5, 0x1.b42dd711971bfp-5, \
   0x1.f0a30c01162a6p-5, 0x1.16536eea37ae1p-4, 0x1.341d7961bd1d1p-4, 0x1.51b073f06183fp-4, \
   0x1.6f0d28ae56b4cp-4, 0x1.8c345d6319b21p-4, 0x1.a926d3a4ad563p-4, 0x1.c5e548f5bc743p-4, \
   0x1.e27076e2af2e6p-4, 0x1.fec9131dbeabbp-4, 0x1.0d77e7cd08e59p-3, 0x1.1b72ad52f67a0p-3, \
   0x1.29552f81ff523p-3, 0x1.371fc201e8f74p-3, 0x1.44d2b6ccb7d1ep-3, 0x1.526e5e3a1b438p-3, \
   0x1.5ff3070a793d4p-3, 0x1.6d60fe719d21dp-3, 0x1.7ab890210d909p-3, 0x1.87fa06520c911p-3, \
   0x1.9525a9cf456b4p-3, 0x1.a23bc1fe2b563p-3, 0x1.af3c94e80bff3p-3, 0x1.bc286742d8cd6p-3, \
   0x1.c8ff7c79a9a22p-3, 0x1.d5c216b4fbb91p-3, 0x1.e27076e2af2e6p-3, 0x1.ef0adcbdc5936p-3, \
   0x1.fb9186d5e3e2bp-3, 0x1.0402594b4d041p-2, 0x1.0a324e27390e3p-2, 0x1.1058bf9ae4ad5p-2, \
   0x1.1675cababa60ep-2, 0x1.1c898c16999fbp-2, 0x1.22941fbcf7966p-2, 0x1.2895a13de86a3p-2, \
   0x1.2e8e2bae11d31p-2, 0x1.347dd9a987d55p-2, 0x1.3a64c556945eap-2, 0x1.404308686a7e4p-2, \
   0x1.4618bc21c5ec2p-2, 0x1.4be5f957778a1p-2, 0x1.51aad872df82dp-2, 0x1.5767717455a6cp-2, \
   0x1.5d1bdbf5809cap-2, 0x1.62c82f2b9c795p-2, 0x1.686c81e9b14afp-2, 0x1.6e08eaa2ba1e4p-2, \
   0x1.739d7f6bbd007p-2, 0x1.792a55fdd47a2p-2, 0x1.7eaf83b82afc3p-2, 0x1.842d1da1e8b17p-2, \
   0x1.89a3386c1425bp-2, 0x1.8f11e873662c7p-2, 0x1.947941c2116fbp-2, 0x1.99d958117e08bp-2, \
   0x1.9f323ecbf984cp-2, 0x1.a484090e5bb0ap-2, 0x1.a9cec9a9a084ap-2, 0x1.af1293247786bp-2, \
   0x1.b44f77bcc8f63p-2, 0x1.b9858969310fbp-2, 0x1.beb4d9da71b7cp-2, 0x1.c3dd7a7cdad4dp-2, \
   0x1.c8ff7c79a9a22p-2, 0x1.ce1af0b85f3ebp-2, 0x1.d32fe7e00ebd5p-2, 0x1.d83e7258a2f3ep-2, \
   0x1.dd46a04c1c4a1p-2, 0x1.e24881a7c6c26p-2, 0x1.e744261d68788p-2, 0x1.ec399d2468cc0p-2, \
   0x1.f128f5faf06edp-2, 0x1.f6123fa7028acp-2, 0x1.faf588f78f31fp-2, 0x1.ffd2e0857f498p-2, \
   0x1.02552a5a5d0ffp-1, 0x1.04bdf9da926d2p-1, 0x1.0723e5c1cdf40p-1, 0x1.0986f4f573521p-1, \
   0x1.0be72e4252a83p-1, 0x1.0e44985d1cc8cp-1, 0x1.109f39e2d4c97p-1, 0x1.12f719593efbcp-1, \
   0x1.154c3d2f4d5eap-1, 0x1.179eabbd899a1p-1, 0x1.19ee6b467c96fp-1, 0x1.1c3b81f713c25p-1, \
   0x1.1e85f5e7040d0p-1, 0x1.20cdcd192ab6ep-1, 0x1.23130d7bebf43p-1, 0x1.2555bce98f7cbp-1, \
   0x1.2795e1289b11bp-1, 0x1.29d37fec2b08bp-1, 0x1.2c0e9ed448e8cp-1, 0x1.2e47436e40268p-1, \
   0x1.307d7334f10bep-1, 0x1.32b1339121d71p-1, 0x1.34e289d9ce1d3p-1, 0x1.37117b54747b6p-1, \
   0x1.393e0d3562a1ap-1, 0x1.3b68449fffc23p-1, 0x1.3d9026a7156fbp-1, 0x1.3fb5b84d16f42p-1, \
   0x1.41d8fe84672aep-1, 0x1.43f9fe2f9ce67p-1, 0x1.4618bc21c5ec2p-1, 0x1.48353d1ea88dfp-1, \
   0x1.4a4f85db03ebbp-1, 0x1.4c679afccee3ap-1, 0x1.4e7d811b75bb1p-1, 0x1.50913cc01686bp-1, \
   0x1.52a2d265bc5abp-1, 0x1.54b2467999498p-1, 0x1.56bf9d5b3f399p-1, 0x1.58cadb5cd7989p-1, \
   0x1.5ad404c359f2dp-1, 0x1.5cdb1dc6c1765p-1, 0x1.5ee02a9241675p-1, 0x1.60e32f44788d9p-1}
#define ADG_LOG_TABLE_INV \
  {0x1.0000000000000p+0, 0x1.fc07f01fc07f0p-1, 0x1.f81f81f81f820p-1, 0x1.f44659e4a4271p-1, \
   0x1.f07c1f07c1f08p-1, 0x1.ecc07b301ecc0p-1, 0x1.e9131abf0b767p-1, 0x1.e573ac901e574p-1, \
   0x1.e1e1e1e1e1e1ep-1, 0x1.de5d6e3f8868ap-1, 0x1.dae6076b981dbp-1, 0x1.d77b654b82c34p-1, \
   0x1.d41d41d41d41dp-1, 0x1.d0cb58f6ec074p-1, 0x1.cd85689039b0bp-1, 0x1.ca4b3055ee191p-1, \
   0x1.c71c71c71c71cp-1, 0x1.c3f8f01c3f8f0p-1, 0x1.c0e070381c0e0p-1, 0x1.bdd2b899406f7p-1, \
   0x1.bacf914c1bad0p-1, 0x1.b7d6c3dda338bp-1, 0x1.b4e81b4e81b4fp-1, 0x1.b2036406c80d9p-1, \
   0x1.af286bca1af28p-1, 0x1.ac5701ac5701bp-1, 0x1.a98ef606a63bep-1, 0x1.a6d01a6d01a6dp-1, \
   0x1.a41a41a41a41ap-1, 0x1.a16d3f97a4b02p-1, 0x1.9ec8e951033d9p-1, 0x1.9c2d14ee4a102p-1, \
   0x1.999999999999ap-1, 0x1.970e4f80cb872p-1, 0x1.948b0fcd6e9e0p-1, 0x1.920fb49d0e229p-1, \
   0x1.8f9c18f9c18fap-1, 0x1.8d3018d3018d3p-1, 0x1.8acb90f6bf3aap-1, 0x1.886e5f0abb04ap-1, \
   0x1.8618618618618p-1, 0x1.83c977ab2beddp-1, 0x1.8181818181818p-1, 0x1.7f405fd017f40p-1, \
   0x1.7d05f417d05f4p-1, 0x1.7ad2208e0ecc3p-1, 0x1.78a4c8178a4c8p-1, 0x1.767dce434a9b1p-1, \
   0x1.745d1745d1746p-1, 0x1.724287f46debcp-1, 0x1.702e05c0b8170p-1, 0x1.6e1f76b4337c7p-1, \
   0x1.6c16c16c16c17p-1, 0x1.6a13cd1537290p-1, 0x1.6816816816817p-1, 0x1.661ec6a5122f9p-1, \
   0x1.642c8590b2164p-1, 0x1.623fa77016240p-1, 0x1.6058160581606p-1, 0x1.5e75bb8d015e7p-1, \
   0x1.5c9882b931057p-1, 0x1.5ac056b015ac0p-1, 0x1.58ed2308158edp-1, 0x1.571ed3c506b3ap-1, \
   0x1.5555555555555p-1, 0x1.5390948f40febp-1, 0x1.51d07eae2f815p-1, 0x1.5015015015015p-1, \
   0x1.4e5e0a72f0539p-1, 0x1.4cab88725af6ep-1, 0x1.4afd6a052bf5bp-1, 0x1.49539e3b2d067p-1, \
   0x1.47ae147ae147bp-1, 0x1.460cbc7f5cf9ap-1, 0x1.446f86562d9fbp-1, 0x1.42d6625d51f87p-1, \
   0x1.4141414141414p-1, 0x1.3fb013fb013fbp-1, 0x1.3e22cbce4a902p-1, 0x1.3c995a47babe7p-1, \
   0x1.3b13b13b13b14p-1, 0x1.3991c2c187f63p-1, 0x1.3813813813814p-1, 0x1.3698df3de0748p-1, \
   0x1.3521cfb2b78c1p-1, 0x1.33ae45b57bcb2p-1, 0x1.323e34a2b10bfp-1, 0x1.30d190130d190p-1, \
   0x1.2f684bda12f68p-1, 0x1.2e025c04b8097p-1, 0x1.2c9fb4d812ca0p-1, 0x1.2b404ad012b40p-1, \
   0x1.29e4129e4129ep-1, 0x1.288b01288b013p-1, 0x1.27350b8812735p-1, 0x1.25e22708092f1p-1, \
   0x1.2492492492492p-1, 0x1.23456789abcdfp-1, 0x1.21fb78121fb78p-1, 0x1.20b470c67c0d9p-1, \
   0x1.1f7047dc11f70p-1, 0x1.1e2ef3b3fb874p-1, 0x1.1cf06ada2811dp-1, 0x1.1bb4a4046ed29p-1, \
   0x1.1a7b9611a7b96p-1, 0x1.19453808ca29cp-1, 0x1.1811811811812p-1, 0x1.16e0689427379p-1, \
   0x1.15b1e5f75270dp-1, 0x1.1485f0e0acd3bp-1, 0x1.135c81135c811p-1, 0x1.12358e75d3033p-1, \
   0x1.1111111111111p-1, 0x1.0fef010fef011p-1, 0x1.0ecf56be69c90p-1, 0x1.0db20a88f4696p-1, \
   0x1.0c9714fbcda3bp-1, 0x1.0b7e6ec259dc8p-1, 0x1.0a6810a6810a7p-1, 0x1.0953f39010954p-1, \
   0x1.0842108421084p-1, 0x1.073260a47f7c6p-1, 0x1.0624dd2f1a9fcp-1, 0x1.05197f7d73404p-1, \
   0x1.0410410410410p-1, 0x1.03091b51f5e1ap-1, 0x1.0204081020408p-1, 0x1.0101010101010p-1}

struct LogTable {
  double ln[128];
  double inv[128];
};

// The library log for the arguments log_tab leaves to it, out of line (as
// iexp_slow).
static __host__ __device__ __noinline__ double log_slow(double x) { return log(x); }

__host__ __device__ __forceinline__ double log_tab(double x, const LogTable &tb) {
  unsigned long long b;
  std::memcpy(&b, &x, 8);
  const unsigned ex = (unsigned)(b >> 52);  // sign and biased exponent
  if (ex == 0u || ex >= 2047u || ex == 1022u || ex == 1023u) return log_slow(x);
  const int k = (int)ex - 1023;
  const int j = (int)((b >> 45) & 127u);
  const unsigned long long mb = (b & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
  const unsigned long long cb = 0x3ff0000000000000ull | ((unsigned long long)j << 45);
  double m, c;
  std::memcpy(&m, &mb, 8);
  std::memcpy(&c, &cb, 8);
  const double u = (m - c) * tb.inv[j], dk = (double)k;
  double q = fma(u, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(u, q, 0.2);
  q = fma(u, q, -0.25);
  q = fma(u, q, 1.0 / 3.0);
  q = fma(u, q, -0.5);
  q = fma(u, q, 1.0);
  const double L_hi = 0x1.62e42fefa3800p-1, L_lo = 0x1.ef35793c76730p-45;
  return fma(dk, L_hi, tb.ln[j]) + fma(dk, L_lo, u * q);
}

// Double -> float rounded to nearest even, from the double's high and low words
// to the float's bits, for the doubles outside the normal float range: zeros,
// values whose float is subnormal or zero, values beyond the largest float, and
// infinities and NaN (the canonical NaN 0x7fffffff). Integer operations only, so
// that the fast conversion of the kernels (the bit-field move of d2f_int) needs
// no FP64 instruction on any path. A normal double below the float range is
// F 2^(eb - 1075) with the 53-bit significand F = 2^52 + m; in units of the
// smallest subnormal float, 2^-149, that is F 2^(eb - 926), and the float's bits
// are that integer rounded to even (a carry into 2^23 gives the smallest normal
// float, as it should). A subnormal double is far below half the smallest
// subnormal float and rounds to a signed zero; so does any value below 2^-150.
__host__ __device__ inline unsigned d2f_edge_bits(unsigned hi, unsigned lo) {
  const unsigned s = hi & 0x80000000u;
  const int eb = (int)((hi >> 20) & 0x7ffu);
  const unsigned mh = hi & 0xfffffu;
  if (eb == 0x7ff) return (mh | lo) != 0u ? 0x7fffffffu : (s | 0x7f800000u);
  if (eb - 1023 + 127 >= 255) return s | 0x7f800000u;
  const int sh = 926 - eb;  // at least 30 for a double below the float range
  if (eb == 0 || sh > 54) return s;
  const unsigned long long F = (1ull << 52) | ((unsigned long long)mh << 32) | lo;
  const unsigned long long q = F >> sh, rem = F & ((1ull << sh) - 1ull);
  const unsigned long long half = 1ull << (sh - 1);
  const unsigned long long up = (rem > half || (rem == half && (q & 1ull) != 0ull)) ? 1ull : 0ull;
  return s | (unsigned)(q + up);
}

}  // namespace adg
