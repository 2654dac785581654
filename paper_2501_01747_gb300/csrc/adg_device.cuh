// Device code of the ADG hot path (sm_103a), included by the translation units
// that instantiate it (one per precision variant, one for the unsynchronised
// mode), so that they compile in parallel.
//
// Per RK stage two kernels run. The stage kernel comes in three precision
// variants PREC (include/adg.h): ADG_FP64; ADG_MIXED, FP32 for the flux and the
// DG operator, FP64 for the Gauss-point temperature, the Arrhenius and
// equilibrium exponents and exponentials, the AT level sums and the
// accumulation of the conserved state, and float pairs (about 48 bits) for the
// mass action and production rates from the FP64 rate constants;
// ADG_MIXED_F32CHEM, as ADG_MIXED but with the chemistry's exponents as float
// pairs and its exponentials, products and sums in FP32. The limiter has an FP64
// and an FP32 variant (MIX), the latter for both mixed variants.
//   stage_kernel<Q,PREC>: one CTA per tile of TE consecutive elements of one
//                      instance (stage_body).
//   limiter_kernel<Q,G,MIX,EPB>: the troubled-cell indicator and, on troubled
//                      cells, the (AT-)WENO reconstruction of Eq. (9)-(11)
//                      (limiter_body). The stage kernel writes the pre-limit
//                      output twice (limiter input and next-stage buffer) so that
//                      the limiter only rewrites troubled cells.
// The constant tables are per translation unit (static); each unit uploads its
// own copy (upload_unit_tables).
#pragma once
#include <cstdio>
#include <type_traits>

#include "adg_internal.cuh"
#include "adg_math.cuh"

namespace adg {

static __constant__ Basis c_basis[ADG_MAX_P];     // index p-1
static __constant__ BasisF c_basis_f[ADG_MAX_P];  // the same, rounded to float

static __constant__ IExpTable c_iexp = {ADG_IEXP_TABLE, ADG_IEXP_TABLE32};
static __constant__ LogTable c_ltab = {ADG_LOG_TABLE_LN, ADG_LOG_TABLE_INV};

// Upload the DG/WENO tables to this translation unit's constant memory.
static cudaError_t upload_unit_tables(const Basis *tables) {
  cudaError_t e = cudaMemcpyToSymbol(c_basis, tables, sizeof(Basis) * ADG_MAX_P);
  if (e != cudaSuccess) return e;
  BasisF f[ADG_MAX_P];
  for (int p = 0; p < ADG_MAX_P; ++p)
    for (int i = 0; i < MAXQ; ++i)
      for (int j = 0; j < MAXQ; ++j) {
        f[p].B[i][j] = (float)tables[p].B[i][j];
        f[p].Sl[i][j] = (float)tables[p].Sl[i][j];
        f[p].Sr[i][j] = (float)tables[p].Sr[i][j];
        f[p].WdP[i][j] = (float)tables[p].WdP[i][j];
        f[p].WPh[i][j] = (float)tables[p].WPh[i][j];
      }
  return cudaMemcpyToSymbol(c_basis_f, f, sizeof(BasisF) * ADG_MAX_P);
}

// Limiter shared memory per CTA for EPB elements.
template <int Q, int G, bool MIX, int EPB>
static size_t limiter_smem_bytes(int nv, int ns);

template <bool MIX>
using dg_t = typename std::conditional<MIX, float, double>::type;

// The stage kernel's precision variant: arithmetic of the flux and the DG
// operator (float in both mixed variants) and of the chemistry (float only in
// ADG_MIXED_F32CHEM).
template <int PREC>
struct Prec {
  static constexpr bool mix = PREC != ADG_FP64;
  static constexpr bool fchem = PREC == ADG_MIXED_F32CHEM;
  static constexpr bool dfchem = PREC == ADG_MIXED;  // mass action in float pairs
  using dg = dg_t<mix>;
  using ct = typename std::conditional<fchem, float,
                                       typename std::conditional<dfchem, DF, double>::type>::type;
};

// Shared-memory footprint (bytes) of a stage tile of TE elements with up to O AT
// levels per face. FP64 region: species fields, exp table, basis values, modal
// tile with halo, w^n of the tile, nodal state, ln T, 1/T, u, P. Region in the
// chemistry's type: concentrations, rates of progress, production rates,
// incidence coefficients. Region in the flux's type: face, level and trace
// fluxes; the mixed variants add an FP32 copy of the species fields and the
// point flux (the FP64 variant writes the flux over the nodal state). Integers:
// delay per face, species-reaction incidence. The float-chemistry variant adds
// its df32 rate coefficients and (ln T, 1/T) pairs.
// Viscous groups append, in FP64: the tile of q = dw/dx with halo, q at the
// Gauss points (then f^d there), and per (level, face) the traces of w and q of
// both sides (then f^d of both sides).
__host__ __device__ inline size_t stage_visc_doubles(int TE, int Q, int ns, int O) {
  const size_t nv = ns + 2;
  return nv * (TE + 2) * Q + nv * (size_t)TE * Q + (size_t)O * (TE + 1) * 4 * nv +
         (size_t)TE * Q;
}

__host__ __device__ inline size_t stage_smem_bytes(int TE, int Q, int ns, int nr, int nterm,
                                                   int O, int prec, bool visc = false) {
  const bool mix = prec != ADG_FP64, fchem = prec == ADG_MIXED_F32CHEM;
  const size_t nv = ns + 2, TQ = (size_t)TE * Q, F = TE + 1;
  const size_t nd = (size_t)SP_NFIELDS * ns + sizeof(IExpTable) / 8 + MAXQ * MAXQ +
                    nv * (TE + 2) * Q + 2 * nv * TQ + 4 * TQ;
  const size_t nct = (size_t)ns * TQ + (size_t)nr * TQ + (size_t)ns * TQ + nterm;
  size_t ndg = F * nv + (size_t)O * F * nv + (size_t)O * F * 2 * nv;
  if (mix) ndg += (size_t)SP_NFIELDS * ns + nv * TQ;
  const size_t ni = F + ns + 1 + nterm;
  // float chemistry: the df32 rate coefficients [nr][6] and (ln T, 1/T) per point
  const size_t ndf = fchem ? (size_t)nr * 6 + 2 * TQ : 0;
  return (size_t)nr * sizeof(Rxn) + nd * 8 + nct * (fchem ? 4 : 8) + ndg * (mix ? 4 : 8) +
         ni * 4 + 16 + ndf * 8 + 8 + (visc ? stage_visc_doubles(TE, Q, ns, O) * 8 + 8 : 0);
}


// The items item0, item0 + step, ... of a loop over (outer, inner) pairs, the
// inner index fastest, split into (o, i) with one division per walk instead of
// one per item (an integer division by a value known only at run time costs
// about twenty instructions).
struct Walk {
  int o, i, dO, dI, n;
  __device__ __forceinline__ Walk(int item0, int step, int inner) : n(inner) {
    o = item0 / inner;
    i = item0 - o * inner;
    dO = step / inner;
    dI = step - dO * inner;
  }
  __device__ __forceinline__ void next() {
    i += dI;
    o += dO;
    if (i >= n) {
      i -= n;
      ++o;
    }
  }
};

// Copy an instance description into shared memory (by 8-byte words).
__device__ inline void load_inst(Inst &dst, const Inst *src) {
  const unsigned long long *a = reinterpret_cast<const unsigned long long *>(src);
  unsigned long long *b = reinterpret_cast<unsigned long long *>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(Inst) / 8); k += blockDim.x) b[k] = a[k];
}

// Observed delays of one PE in the unsynchronised mode: elements [first, last],
// k[0] and k[1] for the PE faces on its left and right side.
struct PeDelays {
  int first, last;
  int k[2];
};

// float -> double, exact, by moving the bit fields on the integer pipeline: on
// this GPU a precision conversion occupies the FP64 unit like a double
// instruction. Zeros and subnormal floats give a signed zero, infinities and NaN
// keep their class.
__device__ __forceinline__ double f2d_exact(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned s = u & 0x80000000u;
  const unsigned ed = (e == 255u) ? 0x7ffu : e + 896u;
  const unsigned hi = (e == 0u) ? s : (s | (ed << 20) | ((u >> 3) & 0xfffffu));
  const unsigned lo = (e == 0u) ? 0u : (u << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// The rare paths of the conversions and reciprocals below, out of line. Inline,
// the compiler may issue their instructions, predicated off, on every call: a
// hardware conversion or a division is then FP64-pipe work that each call pays
// (the stage kernel fell from 8.40 to 8.07 ms per RK stage on the ensemble
// when they moved out of line). The results are the same.
static __device__ __noinline__ unsigned d2f_edge_call(unsigned hi, unsigned lo) {
  return d2f_edge_bits(hi, lo);
}
static __device__ __noinline__ double recip_slow(double x) { return 1.0 / x; }

// double -> float, rounded to nearest even, by moving the bit fields on the
// integer pipeline (the same reason as f2d_exact). Zeros are handled inline;
// values whose float would be subnormal or overflow, and non-finite values, go
// to d2f_edge_bits (integer operations, out of line) or, with HW_EDGE, to the
// hardware conversion. The limiter, bound by the integer pipe rather than the
// FP64 one, takes HW_EDGE: there the out-of-line branch cost more than the
// predicated conversion (1.01 against 0.97 ms per RK stage).
template <bool HW_EDGE>
__device__ __forceinline__ float d2f_int_t(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int ef = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (ef <= 0 || ef >= 255) {
    if constexpr (HW_EDGE) return __double2float_rn(x);
    else return __uint_as_float(((hi << 1) | lo) == 0u ? hi : d2f_edge_call(hi, lo));
  }
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  // a mantissa carry runs into the exponent (up to infinity), as rounding should
  return __uint_as_float(((hi & 0x80000000u) | ((unsigned)ef << 23) | m) + up);
}

__device__ __forceinline__ float d2f_int(double x) { return d2f_int_t<false>(x); }

// df_split on the integer pipeline (the same pair: both conversions round to
// nearest, and the one back is exact).
__device__ __forceinline__ DF df_split_int(double x) {
  const float h = d2f_int(x);
  return DF{h, d2f_int(x - f2d_exact(h))};
}

// x as a float pair (hi + lo, about 48 significant bits) without the FP64 unit:
// hi = x rounded to float (d2f_int), lo = the remainder x - hi, which is the
// integer r formed by the 29 significand bits below float precision (less 2^29
// when hi was rounded up) times 2^(E - 52), converted to float and scaled by
// powers of two. For x outside the normal float range lo is 0 (hi is then 0, a
// subnormal float or an infinity); below about 2^-97 lo itself underflows.
__device__ __forceinline__ DF d2df_int(double x) {
  const unsigned hi32 = (unsigned)__double2hiint(x), lo32 = (unsigned)__double2loint(x);
  const int eb = (int)((hi32 >> 20) & 0x7ffu);
  const float h = d2f_int(x);
  const int ef = eb - 1023 + 127;
  if (ef <= 0 || ef >= 255) return DF{h, 0.0f};
  const unsigned rem = lo32 & 0x1fffffffu;
  const unsigned mlow = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const bool up = rem > 0x10000000u || (rem == 0x10000000u && (mlow & 1u));
  const int r = up ? (int)rem - 0x20000000 : (int)rem;
  // r 2^-52 is exact in float, and 2^(eb - 1023) is a normal float here
  float lo = __fmul_rn(__fmul_rn((float)r, 2.220446049250313e-16f), __int_as_float(ef << 23));
  if (hi32 & 0x80000000u) lo = -lo;
  return DF{h, lo};
}

// 1/x to a relative error below 2^-44, for x whose float is normal: a float
// seed (the fraction truncated to 23 bits on the integer pipeline, the
// correctly rounded float reciprocal: within 1.5 2^-23) and one Newton-Raphson
// step in FP64, r + r (1 - x r), which squares the seed's error. Two double
// operations where a full-precision division takes several times that; other x
// take the division.
__device__ __forceinline__ double recip_nr(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int ef = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (ef <= 1 || ef >= 253) return recip_slow(x);
  const float xf = __uint_as_float((hi & 0x80000000u) | ((unsigned)ef << 23) |
                                   ((hi & 0xfffffu) << 3) | (lo >> 29));
  const double r = f2d_exact(__frcp_rn(xf));
  return fma(r, fma(-x, r, 1.0), r);
}

// 1/x to about one ulp: recip_nr and a second Newton-Raphson step, which squares
// its error below the rounding of the last operation. Four double operations.
__device__ __forceinline__ double recip_nr2(double x) {
  const double r = recip_nr(x);
  return fma(r, fma(-x, r, 1.0), r);
}

// To the variant's arithmetic type without the FP64 unit.
template <typename R>
__device__ __forceinline__ R to_r(double x) {
  if constexpr (std::is_same<R, float>::value) return d2f_int(x);
  else return x;
}

// From one arithmetic type to another without the FP64 unit (float -> double
// and double -> float on the integer pipeline).
template <typename R, typename C>
__device__ __forceinline__ R conv_r(C x) {
  if constexpr (std::is_same<R, C>::value) return x;
  else if constexpr (std::is_same<C, DF>::value) return __fadd_rn(x.hi, x.lo);
  else if constexpr (std::is_same<R, float>::value) return d2f_int(x);
  else return f2d_exact(x);
}

// conv_r with the hardware conversion at the edges of the float range (the
// limiter's form, d2f_int_t<true>).
template <typename R, typename C>
__device__ __forceinline__ R conv_lim(C x) {
  if constexpr (std::is_same<R, float>::value && std::is_same<C, double>::value)
    return d2f_int_t<true>(x);
  else return conv_r<R>(x);
}

// The trace of one variable's modes w[0..Q) at xi = +1 (right = false: sum_j
// w_j) or at xi = -1 (right = true: sum_j (-1)^j w_j), in FP64 and in the order
// of the stage kernel's face phase. Every trace that enters the history ring is
// formed by it (by trace_f in ADG_MIXED), so that a face reads the same value
// from the ring as it would form itself.
template <int Q>
__device__ __forceinline__ double trace_of(const double *w, bool right) {
  double a = 0.0;
#pragma unroll
  for (int j = 0; j < Q; ++j) a += (right && (j & 1)) ? -w[j] : w[j];
  return a;
}

// The same trace in float from the modes rounded to float on the integer pipe
// (ADG_MIXED: the face flux is FP32, so its traces need no FP64 sum). A trace
// that enters the history ring in that variant is this value, exactly.
template <int Q>
__device__ __forceinline__ float trace_f(const double *w, bool right) {
  float a = 0.0f;
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    const float x = d2f_int(w[j]);
    a += (right && (j & 1)) ? -x : x;
  }
  return a;
}

// A value of the history ring. Written by another CTA of the same launch in the
// unsynchronised mode, so read from L2 (the point of coherence), not from a
// possibly stale L1 line of an earlier level in the same slot.
template <bool UNSYNC>
__device__ __forceinline__ double ring_load(const double *p) {
  if constexpr (UNSYNC) return __ldcg(p);
  else return *p;
}

// Diffusive flux of Sec. 2 at one point from the state w and its derivative
// q = dw/dx (LDG), arrays strided (variable v at w[v * ws]); fd (stride fs) gets
// (tau, tau u - q_h, -J_1 .. -J_Ns); fd may be q itself. T in closed form
// (constant c_p), the primitive derivatives by the chain rule (rho_x = sum
// q_{rho Y_i}, u_x = (q_{rho u} - u rho_x) / rho, Y_i,x = (q_{rho Y_i} - Y_i rho_x)
// / rho, T_x from the derivative of rho E - (rho u) u / 2 = sum rho Y_i e_i(T)).
// With X_i = Y_i / (W_i n), n = sum Y_j / W_j, the flux -rho D_i (Y_i / X_i) dX_i/dx
// is -(mu / (Pr Le_i)) (Y_i,x - Y_i n_x / n), and the correction velocity makes
// J_i = J_i* - Y_i sum_j J_j*. Transport: mu = mu_ref (T / T_mu)^mu_exp,
// k = mu c_p / Pr, rho D_i = k / (c_p Le_i).
// R is the arithmetic type of everything but T, which is formed in FP64 (the
// internal energy cancels against the formation energies) unless T_known > 0
// gives it; sp holds the species fields in FP64, spr in R.
// A group of G consecutive lanes (G a power of two dividing 32) evaluates it:
// the species loops are split over the lanes and the sums reduced by shuffles
// within the group. Every lane of the warp must call it; a group without work
// passes valid = false and writes nothing. Up to 4 G species.
template <typename R, int G>
__device__ inline void visc_flux_group(const double *sp, const R *spr, int ns, const Inst &I,
                                       const double *w, int ws, const double *q, int qs,
                                       double *fd, int fs, double T_known, bool valid) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & (G - 1);
  auto red = [&](auto x) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o, G);
    return x;
  };
  const R *rIW = spr + SP_INVW * ns, *rQW = spr + SP_QW * ns, *rCVW = spr + SP_CVW * ns;
  const R *rCPW = spr + SP_CPW * ns, *rIL = spr + SP_INVLE * ns;
  // this lane's species, converted once
  R rl[4], ql[4];
  int c = 0;
  for (int i = lane; i < ns; i += G, ++c) {
    rl[c] = to_r<R>(w[(2 + i) * ws]);
    ql[c] = to_r<R>(q[(2 + i) * qs]);
  }
  const R w0 = to_r<R>(w[0]), w1 = to_r<R>(w[ws]), q0 = to_r<R>(q[0]), q1 = to_r<R>(q[qs]);
  R rho = R(0), cv = R(0), rho_x = R(0), qsum = R(0);
  const bool needT = !(T_known > 0.0);
  c = 0;
  for (int i = lane; i < ns; i += G, ++c) {
    rho += rl[c];
    cv = fma(rl[c], rCVW[i], cv);
    rho_x += ql[c];
    if (needT) qsum = fma(rl[c], rQW[i], qsum);
  }
  rho = red(rho);
  cv = red(cv);
  rho_x = red(rho_x);
  R T;
  if (needT) {
    // in the variant's type: the mixed variant tolerates the cancellation here,
    // which moves f^d, a small part of the flux, by about 1e-6 of itself
    qsum = red(qsum);
    T = (w1 - R(0.5) * w0 * (w0 / rho) - qsum) / cv;
  } else {
    T = to_r<R>(T_known);
  }
  const R irho = R(1) / rho, m = w0, u = m * irho;
  const R u_x = (q0 - u * rho_x) * irho;
  R num = R(0), n = R(0), n_x = R(0), cpm = R(0);
  c = 0;
  for (int i = lane; i < ns; i += G, ++c) {
    const R rx = ql[c], Y = rl[c] * irho;
    const R Yx = (rx - Y * rho_x) * irho;
    num -= rx * fma(rCVW[i], T, rQW[i]);
    n = fma(Y, rIW[i], n);
    n_x = fma(Yx, rIW[i], n_x);
    cpm = fma(Y, rCPW[i], cpm);
  }
  num = red(num) + (q1 - R(0.5) * (q0 * u + m * u_x));
  n = red(n);
  n_x = red(n_x);
  cpm = red(cpm);
  const R T_x = num / cv;
  R mu;
  if constexpr (std::is_same<R, float>::value)
    mu = (float)I.mu_ref * expf((float)I.mu_exp * (logf(T) - (float)I.ln_T_mu));
  else
    mu = I.mu_ref * exp(I.mu_exp * (log(T) - I.ln_T_mu));
  const R a = mu * (R)I.inv_prandtl, kc = a * cpm, nxn = n_x / n;
  R Jsum = R(0);
  R Js_own[4];  // this lane's species (G >= ns / 4)
  c = 0;
  for (int i = lane; i < ns; i += G, ++c) {
    const R Y = rl[c] * irho;
    const R Yx = (ql[c] - Y * rho_x) * irho;
    Js_own[c] = -a * rIL[i] * (Yx - Y * nxn);
    Jsum += Js_own[c];
  }
  Jsum = red(Jsum);
  R qh = R(0);
  c = 0;
  for (int i = lane; i < ns; i += G, ++c) {
    const R J = Js_own[c] - rl[c] * irho * Jsum;
    qh = fma(fma(rCPW[i], T, rQW[i]), J, qh);
    if (valid) fd[(2 + i) * fs] = (double)(-J);
  }
  qh = red(qh) - kc * T_x;
  if (valid && lane == 0) {
    const R tau = R(4.0 / 3.0) * mu * u_x;
    fd[0] = (double)tau;
    fd[fs] = (double)(tau * u - qh);
  }
}

// The diffusive flux at every Gauss point of a tile (over its nodal q), G lanes
// per point; w, q [v][TQ], T [TQ] (the point temperatures).
template <typename R, int G>
__device__ inline void visc_points(const double *sp, const R *spr, int ns, const Inst &I,
                                   const double *w, double *q, const double *T, int TQ,
                                   int teq) {
  const int ngr = blockDim.x / G, g = threadIdx.x / G;
  for (int base = 0; base < teq; base += ngr) {
    const int t = base + g;
    const bool valid = t < teq;
    const int tt = valid ? t : 0;
    if (!__any_sync(0xffffffffu, valid)) continue;  // warp-uniform: no point here
    visc_flux_group<R, G>(sp, spr, ns, I, w + tt, TQ, q + tt, TQ, q + tt, TQ, T[tt], valid);
  }
}

// The diffusive flux of both sides of every face level of a tile, G lanes per
// (level, face, side): from the traces vt = (w_l, w_r, q_l, q_r) of the level,
// f^d over q_l and q_r. Levels beyond the first only at delayed PE faces.
template <typename R, int G>
__device__ inline void visc_faces(const double *sp, const R *spr, int ns, const Inst &I,
                                  double *sqt, const int *sk, int te, int NF, int O) {
  const int nv = ns + 2, ngr = blockDim.x / G, g = threadIdx.x / G;
  const int total = O * (te + 1) * 2;
  for (int base = 0; base < total; base += ngr) {
    int it = base + g;
    bool valid = it < total;
    if (!valid) it = 0;
    const int side = it & 1, mf = it >> 1, m = mf / (te + 1), f = mf - m * (te + 1);
    valid = valid && m < (sk[f] > 0 ? I.at_order : 1);
    if (!__any_sync(0xffffffffu, valid)) continue;  // warp-uniform: no level here
    double *vt = sqt + ((size_t)m * NF + f) * 4 * nv;
    visc_flux_group<R, G>(sp, spr, ns, I, vt + side * nv, 1, vt + (2 + side) * nv, 1,
                          vt + (2 + side) * nv, 1, 0.0, valid);
  }
}


// The rate of progress of reaction Rx at point t in FP64, for an item whose
// rate constant kf or kr lies beyond the float range (ADG_MIXED), from the
// float-pair concentrations scc [species][TQ]. Out of line, like the other rare
// paths: inline, its FP64 products could be issued, predicated off, for every
// item.
static __device__ __noinline__ DF rate_fp64(const Rxn &Rx, const DF *scc, int TQ, int t, double f,
                                            double r) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (Rx.rn[k] == 0) break;
    const DF c = scc[(size_t)Rx.rs[k] * TQ + t];
    const double cd = f2d_exact(c.hi) + f2d_exact(c.lo);
    f *= cd;
    if (Rx.rn[k] > 1) f *= cd;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (Rx.pn[k] == 0) break;
    const DF c = scc[(size_t)Rx.ps[k] * TQ + t];
    const double cd = f2d_exact(c.hi) + f2d_exact(c.lo);
    r *= cd;
    if (Rx.pn[k] > 1) r *= cd;
  }
  return d2df_int(f - r);
}

// Stage s of one tile: elements [e0, e0 + te) of instance I at step level nstep.
// With UNSYNC the PE faces of the tile take the delays pd->k observed by a PE
// that runs without synchronisation and read both sides from the history ring,
// also at delay 0; the stage input's traces there are published beforehand by
// the caller, not written in phase 6.
template <int Q, int PREC, bool UNSYNC, bool VISC = false>
__device__ __forceinline__ void stage_body(const Mech &M, const StageArgs &A, const Inst &I,
                                           const int e0, const int te, const int64_t nstep,
                                           const PeDelays *pd) {
  constexpr bool MIX = Prec<PREC>::mix, FCHEM = Prec<PREC>::fchem, DFCHEM = Prec<PREC>::dfchem;
  using DG = typename Prec<PREC>::dg;  // flux and DG operator
  using CT = typename Prec<PREC>::ct;  // chemistry
  extern __shared__ __align__(16) double sm[];
  const Basis &B = c_basis[Q - 2];
  const BasisF &BF = c_basis_f[Q - 2];
  const int nv = I.nv, ns = M.ns, nr = M.nr, N = I.n_elem, TE = A.TE;
  const int TQ = TE * Q;
  const int teq = te * Q;
  const double *A_win = stage_input(I, A.s);
  double *A_wnext = stage_output(I, A.s);
  // stages after the first also read, per element, w^n (SSP-RK3) or the LSERK
  // register dq
  const double *A_wacc = I.lserk ? I.wq : I.wn;
  const bool periodic = (I.bc_left == ADG_BC_PERIODIC);
  const int O = A.O, NF = TE + 1;
  Rxn *srx = reinterpret_cast<Rxn *>(sm);
  double *ssp = reinterpret_cast<double *>(srx + nr);         // [F][ns]
  IExpTable *stab = reinterpret_cast<IExpTable *>(ssp + SP_NFIELDS * ns);
  double *sPq = reinterpret_cast<double *>(stab + 1);         // [q][j] P_j(x_q)
  double *sw = sPq + MAXQ * MAXQ;                             // [v][TE+2][Q]
  double *snw = sw + (size_t)nv * (TE + 2) * Q;               // [v][TQ] nodal state
  double *slnT = snw + (size_t)nv * TQ;                       // [TQ]
  double *sinvT = slnT + TQ;
  double *su = sinvT + TQ;
  double *sPr = su + TQ;
  double *swn = sPr + TQ;                                     // [v][TQ] modes of w^n
  CT *scc = reinterpret_cast<CT *>(swn + (size_t)nv * TQ);    // [i][TQ] concentrations
  CT *sq = scc + (size_t)ns * TQ;                             // [j][TQ] rates of progress
  CT *swd = sq + (size_t)nr * TQ;                             // [i][TQ] production rates
  CT *scoef = swd + (size_t)ns * TQ;                          // [nterm] incidence coefficients
  DG *sfh = reinterpret_cast<DG *>(scoef + M.nterm);          // [NF][nv]
  DG *sflx = sfh + (size_t)NF * nv;                           // [O][NF][nv]
  DG *str = sflx + (size_t)O * NF * nv;                       // [O][NF][2][nv]
  DG *sspD, *sfx;                                             // species fields, point flux
  int *sk;
  if constexpr (MIX) {
    sspD = str + (size_t)O * NF * 2 * nv;
    sfx = sspD + (size_t)SP_NFIELDS * ns;
    sk = reinterpret_cast<int *>(sfx + (size_t)nv * TQ);
  } else {
    sspD = reinterpret_cast<DG *>(ssp);
    sfx = reinterpret_cast<DG *>(snw);
    sk = reinterpret_cast<int *>(str + (size_t)O * NF * 2 * nv);
  }
  int *soff = sk + NF;        // [ns + 1]
  int *sterm = soff + ns + 1;  // [nterm] reaction of each incidence term
  // float chemistry: df32 rate coefficients and (ln T, 1/T) per point, 8-byte aligned
  DF *srxf = reinterpret_cast<DF *>(
      (reinterpret_cast<uintptr_t>(sterm + M.nterm) + 7) & ~(uintptr_t)7);  // [nr][6]
  DF *sdfT = srxf + (size_t)nr * 6;                                          // [TQ][2]
  // viscous region (groups with viscous instances), FP64
  double *sqw = reinterpret_cast<double *>(FCHEM ? (void *)(sdfT + 2 * TQ) : (void *)srxf);  // [v][TE+2][Q]
  double *sqn = sqw + (size_t)nv * (TE + 2) * Q;                           // [v][TQ]
  double *sqt = sqn + (size_t)nv * TQ;                                     // [O][NF][4][nv]
  double *sTv = sqt + (size_t)O * NF * 4 * nv;                             // [TQ] T
  // viscous terms: compiled only into the viscous instances of the kernel (the
  // Euler kernels keep their register budget), run for viscous instances
  const bool visc = VISC && I.viscous;
  const int tid = threadIdx.x, nth = blockDim.x;
  // (2i+1)/dx of the assembly in the variant's type, once per CTA (per thread it
  // cost an FP64 division and Q conversions, as much FP64 work as an item's own)
  __shared__ DG s_scale[MAXQ];

  // 0. mechanism, species fields, incidence, exp table and basis values into
  // shared memory
  {
    // a thread's share of every table is loaded before any of it is stored, so
    // that its global loads are in flight together (a store in between would
    // hold the next load back: the tables' pointers may alias shared memory)
    const uint4 *src = reinterpret_cast<const uint4 *>(M.rx);
    uint4 *dst = reinterpret_cast<uint4 *>(srx);
    const int n_rx4 = nr * (int)(sizeof(Rxn) / 16), n_sp = SP_NFIELDS * ns;
    const int n_rxf = FCHEM ? nr * 6 : 0, n_term = M.nterm;
    const int n_all = max(max(max(n_rx4, n_sp), max(n_rxf, n_term)), max(max(32, Q * Q), ns + 1));
    for (int k = tid; k < n_all; k += nth) {
      uint4 rx4 = {};
      double spv = 0.0;
      DF rf = {};
      int term = 0, off = 0;
      if (k < n_rx4) rx4 = src[k];
      if (k < n_sp) spv = M.sp[k];
      if (k < n_rxf) rf = M.rxf[k];
      if (k < n_term) term = M.sx[k];
      if (k <= ns) off = M.sx_off[k];
      if (k < n_rx4) dst[k] = rx4;
      if (k < n_sp) {
        ssp[k] = spv;
        if constexpr (MIX) sspD[k] = conv_r<DG>(spv);
      }
      if constexpr (FCHEM) {
        if (k < n_rxf) srxf[k] = rf;
      }
      if (k < n_term) {
        sterm[k] = term >> 8;
        if constexpr (DFCHEM) scoef[k] = DF{(float)(signed char)(term & 0xff), 0.0f};
        else scoef[k] = (CT)(signed char)(term & 0xff);
      }
      if (k <= ns) soff[k] = off;
      if (k < 32) {
        stab->t[k] = c_iexp.t[k];
        stab->t32[k] = c_iexp.t32[k];
        if constexpr (FCHEM)
          iexp_table_df(c_iexp.t32[k], &stab->tf[2 * k], &stab->tf[2 * k + 1]);
      }
      if (k < Q * Q) sPq[k] = B.P[k / Q][k % Q];
      if (k < Q) s_scale[k] = conv_r<DG>((2.0 * k + 1.0) * (1.0 / I.dx));
    }
  }
  // 1. tile of modal coefficients with a one-element halo on each side and, for
  // stages after the first, the tile's modes of w^n or dq (batches of loads in
  // flight)
  {
    constexpr int BATCH = 8;
    const int span = (te + 2) * Q, n_tile = nv * span;
    const int n_wn = (A.s == 0) ? 0 : nv * te * Q;
    const int total = n_tile + n_wn;
    // (variable, position) of this thread's loads in the tile, without a
    // division per load; the w^n region takes its own walk from its first load
    Walk wt(tid, nth, span);
    const int k0 = tid + ((n_tile - tid + nth - 1) / nth) * nth - n_tile;
    Walk ww(k0 > 0 ? k0 : 0, nth, te * Q);
    for (int base = tid; base < total; base += BATCH * nth) {
      double xs[BATCH];
      double *dst[BATCH];
#pragma unroll
      for (int b = 0; b < BATCH; ++b) {
        const int idx = base + b * nth;
        dst[b] = nullptr;
        if (idx < n_tile) {
          const int v = wt.o, r = wt.i;
          wt.next();
          const int le = r / Q, j = r - le * Q;
          int e = e0 - 1 + le;
          if (e < 0) e = periodic ? e + N : 0;
          if (e >= N) e = periodic ? e - N : N - 1;
          xs[b] = A_win[((size_t)v * N + e) * Q + j];
          dst[b] = sw + ((size_t)v * (TE + 2) + le) * Q + j;
        } else if (idx < total) {
          const int v = ww.o, r = ww.i;
          ww.next();
          xs[b] = A_wacc[((size_t)v * N + e0) * Q + r];
          dst[b] = swn + (size_t)v * TQ + r;
        }
      }
#pragma unroll
      for (int b = 0; b < BATCH; ++b)
        if (dst[b]) *dst[b] = xs[b];
    }
  }
  // the tile of q = dw/dx with the same halo (viscous instances)
  if (visc) {
    const int span = (te + 2) * Q;
    for (int idx = tid; idx < nv * span; idx += nth) {
      const int v = idx / span, r = idx - v * span, le = r / Q, j = r - le * Q;
      int e = e0 - 1 + le;
      if (e < 0) e = periodic ? e + N : 0;
      if (e >= N) e = periodic ? e - N : N - 1;
      sqw[((size_t)v * (TE + 2) + le) * Q + j] = I.qx[((size_t)v * N + e) * Q + j];
    }
  }
  __syncthreads();

  // 2a. conserved state at the Gauss points, one (variable, point) per item;
  // then (inviscid) the two sides' traces of every face of the tile at level 0,
  // one (side, variable, face) per item: w(+1) = sum_j w_j of the left element,
  // w(-1) = sum_j (-1)^j w_j of the right one (a delayed face's item in phase 2b
  // overwrites them with the history's)
  const int n_trace = visc ? 0 : 2 * nv * (te + 1);
  Walk w2a(tid, nth, teq);
  for (int item = tid; item < nv * teq + n_trace; item += nth, w2a.next()) {
    if (item >= nv * teq) {
      const int r = item - nv * teq, side = r & 1, vf = r >> 1;
      const int v = vf / (te + 1), f = vf - v * (te + 1);
      const double *wi = sw + ((size_t)v * (TE + 2) + f + side) * Q;
      if constexpr (DFCHEM) {
        str[(size_t)f * 2 * nv + side * nv + v] = trace_f<Q>(wi, side);
      } else {
        double a = 0.0;
#pragma unroll
        for (int j = 0; j < Q; ++j) a += (side && (j & 1)) ? -wi[j] : wi[j];
        str[(size_t)f * 2 * nv + side * nv + v] = conv_r<DG>(a);
      }
      continue;
    }
    const int v = w2a.o, t = w2a.i;
    const int e = t / Q, q = t - e * Q;
    const double *wi = sw + ((size_t)v * (TE + 2) + e + 1) * Q;
    const double *Pq = sPq + q * Q;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < Q; ++j) acc += wi[j] * Pq[j];
    snw[(size_t)v * TQ + t] = acc;
    if constexpr (MIX) sfx[(size_t)v * TQ + t] = conv_r<DG>(acc);  // converted once, for phase 2c
    if (visc) {
      const double *qi = sqw + ((size_t)v * (TE + 2) + e + 1) * Q;
      double aq = 0.0;
#pragma unroll
      for (int j = 0; j < Q; ++j) aq += qi[j] * Pq[j];
      sqn[(size_t)v * TQ + t] = aq;
    }
  }
  __syncthreads();
  // The face fluxes of the tile (local face f between local elements f and f+1),
  // one (level, face) per item: the plain flux of the traces of phase 2a (a
  // viscous instance's item sums its own, with those of q), or one delayed
  // level of the AT flux (Eq. 7) with both sides at the common level n-k-m from
  // the history ring. They run in phase 2b on the warps after those
  // of the thermodynamics (they were the critical path of the chemistry phase).
  const int n_face = O * (te + 1);
  auto face_item = [&](const int item) {
    const int m = item / (te + 1), f = item - m * (te + 1);
    const int g = e0 + f;  // global face index
    const int pf = (g < N) ? I.pf_of_left[g] : I.pf_of_right[N - 1];
    int k = 0;
    if (pf >= 0) {
      if constexpr (UNSYNC) k = pd->k[g == pd->first ? 0 : 1];
      else k = effective_delay(I, nstep, pf);
    }
    if (m == 0) sk[f] = k;
    DG *fl = sflx + ((size_t)m * NF + f) * nv;
    DG *wl = str + ((size_t)m * NF + f) * 2 * nv, *wr = wl + nv;
    if (k > 0 || (UNSYNC && pf >= 0)) {
      if (m >= (k > 0 ? I.at_order : 1)) return;
      const int64_t lv = nstep - k - m;
      const double *bl = I.ring_in + ring_trace(I, lv, A.s, pf, 0);
      const double *br = I.ring_in + ring_trace(I, lv, A.s, pf, 1);
      if constexpr (MIX || UNSYNC) {
        for (int v = 0; v < nv; ++v) {
          wl[v] = conv_r<DG>(ring_load<UNSYNC>(bl + v));
          wr[v] = conv_r<DG>(ring_load<UNSYNC>(br + v));
        }
        num_flux_t<DG>(sspD, ns, I.flux, wl, wr, fl);
      } else {
        num_flux_t<double>(ssp, ns, I.flux, bl, br, fl);
      }
      if (visc) {
        // minus the central mean of f^d from the traces of w and q at this level
        double *vt = sqt + ((size_t)m * NF + f) * 4 * nv;  // w_l, w_r, q_l, q_r
        const double *ql = I.ring_q + ring_trace(I, lv, A.s, pf, 0);
        const double *qr = I.ring_q + ring_trace(I, lv, A.s, pf, 1);
        for (int v = 0; v < nv; ++v) {
          vt[v] = ring_load<UNSYNC>(bl + v);
          vt[nv + v] = ring_load<UNSYNC>(br + v);
          vt[2 * nv + v] = ring_load<UNSYNC>(ql + v);
          vt[3 * nv + v] = ring_load<UNSYNC>(qr + v);
        }
        // f^d of both sides: in phase 4, subtracted in the AT sum of phase 5
      }
      return;
    }
    if (m > 0) return;
    double *vt = sqt + (size_t)f * 4 * nv;
    if (visc) {
      // the traces of w (phase 2a leaves them to this item) and of q
      for (int v = 0; v < nv; ++v) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < Q; ++j) {
          a += sw[((size_t)v * (TE + 2) + f) * Q + j];
          b += ((j & 1) ? -1.0 : 1.0) * sw[((size_t)v * (TE + 2) + f + 1) * Q + j];
        }
        wl[v] = (DG)a;
        wr[v] = (DG)b;
        double qa = 0.0, qb = 0.0;
        for (int j = 0; j < Q; ++j) {
          qa += sqw[((size_t)v * (TE + 2) + f) * Q + j];
          qb += ((j & 1) ? -1.0 : 1.0) * sqw[((size_t)v * (TE + 2) + f + 1) * Q + j];
        }
        vt[v] = a;
        vt[nv + v] = b;
        vt[2 * nv + v] = qa;
        vt[3 * nv + v] = qb;
      }
    }
    // physical boundary: the ghost is the mirror image at a reflecting wall (rho u
    // negated; of q, d(rho u)/dx kept and the others negated) or a copy (outflow)
    if (!periodic && g == 0) {
      const bool refl = I.bc_left == ADG_BC_REFLECT;
      for (int v = 0; v < nv; ++v) wl[v] = wr[v];
      if (refl) wl[0] = -wr[0];
      if (visc)
        for (int v = 0; v < nv; ++v) {
          vt[v] = (refl && v == 0) ? -vt[nv] : vt[nv + v];
          vt[2 * nv + v] = (refl && v > 0) ? -vt[3 * nv + v] : vt[3 * nv + v];
        }
    } else if (!periodic && g == N) {
      const bool refl = I.bc_right == ADG_BC_REFLECT;
      for (int v = 0; v < nv; ++v) wr[v] = wl[v];
      if (refl) wr[0] = -wl[0];
      if (visc)
        for (int v = 0; v < nv; ++v) {
          vt[nv + v] = (refl && v == 0) ? -vt[0] : vt[v];
          vt[3 * nv + v] = (refl && v > 0) ? -vt[2 * nv + v] : vt[2 * nv + v];
        }
    }
    num_flux_t<DG>(sspD, ns, I.flux, wl, wr, fl);
  };

  // 2b. temperature from the internal energy (the closed form of the Newton step
  // for constant c_p), ln T, 1/T, velocity and pressure, in FP64; the face items
  {
    const double *sQW = ssp + SP_QW * ns, *sCVW = ssp + SP_CVW * ns, *sRW = ssp + SP_RW * ns;
    // A large mechanism's species sums run on L lanes per point (lane g takes
    // species g, g + L, ...; a shuffle tree adds the lanes up), so that a tile
    // of few points does not leave the CTA waiting at the next barrier on a
    // long serial chain. L depends on the mechanism only, so the result does
    // not depend on the launch configuration.
    const int L = !MIX ? 1 : (ns >= 32 ? 8 : (ns >= 16 ? 4 : 1));
    const int lsh = L == 8 ? 3 : (L == 4 ? 2 : 0);
    const int npl = teq << lsh;
    // the face items start on a warp boundary: a warp holding points and faces
    // ran both paths one after the other and was the phase's critical path
    const int fb = (npl + 31) & ~31;
    for (int it = tid; it < fb + n_face; it += nth) {
      if (it >= fb) {
        face_item(it - fb);
        continue;
      }
      // a warp of the point region: all its lanes take part in the shuffles
      const bool act = it < npl;
      const int t = act ? (it >> lsh) : 0, g = it & (L - 1);
      const double *wq = snw + t;
      double rho = 0.0, qsum = 0.0, cv = 0.0, Rm = 0.0;
      if (act)
        for (int i = g; i < ns; i += L) {
          const double r = wq[(size_t)(2 + i) * TQ];
          rho += r;
          qsum = fma(r, sQW[i], qsum);
          cv = fma(r, sCVW[i], cv);
          Rm = fma(r, sRW[i], Rm);
        }
      for (int o = L >> 1; o > 0; o >>= 1) {
        rho += __shfl_xor_sync(0xffffffffu, rho, o, L);
        qsum += __shfl_xor_sync(0xffffffffu, qsum, o, L);
        cv += __shfl_xor_sync(0xffffffffu, cv, o, L);
        Rm += __shfl_xor_sync(0xffffffffu, Rm, o, L);
      }
      if (!act || g != 0) continue;
      const double m = wq[0];
      double u, num, T;
      if constexpr (FCHEM) {
        // ln T and 1/T feed float-float arguments (about 1e-12): reciprocals
        // by one Newton step from a float seed, Tang's table logarithm, the
        // float pairs split on the integer pipeline
        u = m * recip_nr(rho);
        num = wq[TQ] - 0.5 * m * u - qsum;
        const double inum = recip_nr(num);
        T = num * recip_nr(cv);
        sdfT[2 * t] = df_split_int(log_tab(T, c_ltab));
        sdfT[2 * t + 1] = df_split_int(cv * inum);
      } else if constexpr (MIX) {
        // FP64 to about one ulp for the FP64 chemistry: reciprocals by two Newton
        // steps from a float seed, Tang's table logarithm (within 1.4 ulp)
        u = m * recip_nr2(rho);
        num = wq[TQ] - 0.5 * m * u - qsum;
        T = num * recip_nr2(cv);
        slnT[t] = log_tab(T, c_ltab);
        sinvT[t] = cv * recip_nr2(num);
      } else {
        u = m / rho;
        num = wq[TQ] - 0.5 * m * u - qsum;
        T = num / cv;
        slnT[t] = log(T);
        sinvT[t] = cv / num;
      }
      // rho > 0, 0 < T < inf and m finite, on the bit patterns (integer pipe): a
      // positive double (+inf included) is 1 .. 0x7FF0000000000000, a positive
      // finite one 1 .. 0x7FEFFFFFFFFFFFFF; NaNs and negatives lie above
      const unsigned long long brho = (unsigned long long)__double_as_longlong(rho);
      const unsigned long long bT = (unsigned long long)__double_as_longlong(T);
      const unsigned long long bm = (unsigned long long)__double_as_longlong(m);
      if (!(brho - 1ull < 0x7FF0000000000000ull) || !(bT - 1ull < 0x7FEFFFFFFFFFFFFFull) ||
          (bm & 0x7FF0000000000000ull) == 0x7FF0000000000000ull)
        report_error(I, ADG_ERR_NONPHYSICAL, e0 + t / Q, A.s, nstep);
      if constexpr (MIX) {
        // FP32 copies for phase 2c, in the storage of su (2 TQ floats)
        float *suf = reinterpret_cast<float *>(su);
        suf[t] = d2f_int(u);
        suf[TQ + t] = d2f_int(T * Rm);
      } else {
        su[t] = u;
        sPr[t] = T * Rm;
      }
      if (visc) sTv[t] = T;
    }
  }
  // the diffusive flux at every point, over its q, by groups of lanes
  if constexpr (VISC) {
    if (visc) {
      __syncthreads();
      if (ns <= 16) visc_points<DG, 4>(ssp, sspD, ns, I, snw, sqn, sTv, TQ, teq);
      else visc_points<DG, 16>(ssp, sspD, ns, I, snw, sqn, sTv, TQ, teq);
    }
  }
  __syncthreads();
  // 2c. per (variable, point): the flux, and for a species its concentration
  // (law of mass action on non-negative concentrations: clipped at zero by the
  // sign bit)
  if constexpr (MIX) {
    // the flux in FP32 throughout, on the copies of phases 2a and 2b; the
    // concentrations in the chemistry's type (FP64 from the FP64 nodal state)
    const float *sIW = sspD + SP_INVW * ns, *suf = reinterpret_cast<const float *>(su);
    Walk wk(tid, nth, teq);
    for (int item = tid; item < nv * teq; item += nth, wk.next()) {
      const int v = wk.o, t = wk.i;
      const size_t at = (size_t)v * TQ + t;
      const float w = sfx[at], u = suf[t];
      float f;
      if (v >= 2) {
        const int i = v - 2;
        if constexpr (FCHEM) {
          const float r = (__float_as_int(w) < 0) ? 0.0f : w;
          scc[(size_t)i * TQ + t] = r * sIW[i];
        } else {
          // rho Y_i / W_i as a float pair from the FP64 nodal value, no FP64 op
          const double wd = snw[at];
          const DF r = (__double2hiint(wd) < 0) ? DF{0.0f, 0.0f} : d2df_int(wd);
          scc[(size_t)i * TQ + t] = df_mul(r, d2df_int(ssp[SP_INVW * ns + i]));
        }
        f = u * w;
      } else if (v == 0) {
        f = fmaf(w, u, suf[TQ + t]);
      } else {
        f = u * (w + suf[TQ + t]);
      }
      // f = f^c - f^d
      if (visc) f -= d2f_int(sqn[at]);
      sfx[at] = f;
    }
  } else {
    const double *sIW = ssp + SP_INVW * ns;
    Walk wk(tid, nth, teq);
    for (int item = tid; item < nv * teq; item += nth, wk.next()) {
      const int v = wk.o, t = wk.i;
      const size_t at = (size_t)v * TQ + t;
      const double w = snw[at], u = su[t];
      if (v >= 2) {
        const int i = v - 2;
        const double r = (__double2hiint(w) < 0) ? 0.0 : w;
        scc[(size_t)i * TQ + t] = r * sIW[i];
        snw[at] = u * w;
      } else if (v == 0) {
        snw[at] = w * u + sPr[t];
      } else {
        snw[at] = u * (w + sPr[t]);
      }
      // f = f^c - f^d
      if (visc) snw[at] -= sqn[at];
    }
  }
  __syncthreads();

  // 3. the chemistry, one (reaction, point) per item: the reversible rate of
  // progress from the Arrhenius and the equilibrium exponentials (the face fluxes
  // ran in phase 2b).
  Walk w3(tid, nth, teq);
  for (int item = tid; item < nr * teq; item += nth, w3.next()) {
    const int j = w3.o, t = w3.i;
    const Rxn &Rx = srx[j];
    if constexpr (DFCHEM) {
      // FP64 arguments and FP64 exponentials (integer pipeline); the mass action
      // in float pairs (48 bits) on the FP32 pipe, so that k_f and k_r reach
      // the rate of progress unrounded without FP64 products
      const double lnT = slnT[t], invT = sinvT[t];
      const double kf = iexp(fma(Rx.mEaR, invT, fma(Rx.b, lnT, Rx.lnA)), *stab);
      const double kr = iexp(fma(Rx.kr2, invT, fma(Rx.kr1, lnT, Rx.kr0)), *stab);
      DF fwd = d2df_int(kf), rev = d2df_int(kr);
      if (!(fabsf(fwd.hi) < 3.0e38f) || !(fabsf(rev.hi) < 3.0e38f)) {
        // a rate constant beyond the float range: this item in FP64
        sq[(size_t)j * TQ + t] = rate_fp64(Rx, scc, TQ, t, kf, kr);
        continue;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (Rx.rn[k] == 0) break;
        const DF c = scc[(size_t)Rx.rs[k] * TQ + t];
        fwd = df_mul(fwd, c);
        if (Rx.rn[k] > 1) fwd = df_mul(fwd, c);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (Rx.pn[k] == 0) break;
        const DF c = scc[(size_t)Rx.ps[k] * TQ + t];
        rev = df_mul(rev, c);
        if (Rx.pn[k] > 1) rev = df_mul(rev, c);
      }
      sq[(size_t)j * TQ + t] = df_sub(fwd, rev);
    } else {
      CT fwd, rev;
      if constexpr (FCHEM) {
        // arguments in df32 and the FP32-pipe exp: no FP64 instruction and no
        // precision conversion per item
        const DF lnT = sdfT[2 * t], invT = sdfT[2 * t + 1], *c = srxf + 6 * j;
        fwd = exp_df(df_fma(c[2], invT, df_fma(c[1], lnT, c[0])), stab->tf);
        rev = exp_df(df_fma(c[5], invT, df_fma(c[4], lnT, c[3])), stab->tf);
      } else {
        // FP64 arguments, the FP64 exponential on the integer pipeline
        const double lnT = slnT[t], invT = sinvT[t];
        fwd = iexp(fma(Rx.mEaR, invT, fma(Rx.b, lnT, Rx.lnA)), *stab);
        rev = iexp(fma(Rx.kr2, invT, fma(Rx.kr1, lnT, Rx.kr0)), *stab);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (Rx.rn[k] == 0) break;
        CT cc = scc[(size_t)Rx.rs[k] * TQ + t];
        fwd *= cc;
        if (Rx.rn[k] > 1) fwd *= cc;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (Rx.pn[k] == 0) break;
        CT cc = scc[(size_t)Rx.ps[k] * TQ + t];
        rev *= cc;
        if (Rx.pn[k] > 1) rev *= cc;
      }
      sq[(size_t)j * TQ + t] = fwd - rev;
    }
  }
  __syncthreads();

  // 4. production rates, one (species, point) per item: the net stoichiometric
  // sum over the species' reactions, in ascending reaction order
  Walk w4(tid, nth, teq);
  for (int item = tid; item < ns * teq; item += nth, w4.next()) {
    const int i = w4.o, t = w4.i;
    if constexpr (DFCHEM) {
      DF acc = {0.0f, 0.0f};
      for (int k = soff[i]; k < soff[i + 1]; ++k)
        acc = df_fma(scoef[k], sq[(size_t)sterm[k] * TQ + t], acc);
      swd[(size_t)i * TQ + t] = acc;
    } else {
      CT acc = CT(0);
      for (int k = soff[i]; k < soff[i + 1]; ++k)
        acc = fma(scoef[k], sq[(size_t)sterm[k] * TQ + t], acc);
      swd[(size_t)i * TQ + t] = acc;
    }
  }
  // the diffusive flux of both sides of every face level, by groups of lanes
  if constexpr (VISC) {
    if (visc) {
      if (ns <= 16) visc_faces<DG, 4>(ssp, sspD, ns, I, sqt, sk, te, NF, O);
      else visc_faces<DG, 16>(ssp, sspD, ns, I, sqt, sk, te, NF, O);
    }
    __syncthreads();
  }
  // 5. the AT sum over levels, m = 0..o-1 in order, in FP64, of the Riemann flux
  // minus (viscous) the central mean of f^d
  Walk w5(tid, nth, nv);
  for (int item = tid; item < (te + 1) * nv; item += nth, w5.next()) {
    const int f = w5.o, v = w5.i;
    const int k = sk[f];
    auto level = [&](int m) {
      double x = conv_r<double>(sflx[((size_t)m * NF + f) * nv + v]);
      if (visc) {
        const double *vt = sqt + ((size_t)m * NF + f) * 4 * nv;
        x -= 0.5 * (vt[2 * nv + v] + vt[3 * nv + v]);
      }
      return x;
    };
    double acc = level(0);
    if (k > 0) {
      acc *= I.at[k][0];
      for (int m = 1; m < I.at_order; ++m) acc = fma(I.at[k][m], level(m), acc);
    }
    sfh[(size_t)f * nv + v] = conv_r<DG>(acc);
  }
  __syncthreads();
  // The successor (the limiter) is released only now: released at entry, its
  // CTAs, resident while they wait, piled onto the few SMs with room beside
  // two stage CTAs and then ran their FP64 work there, several to an SM.
  if constexpr (!UNSYNC) pdl_trigger();

  // 6. assembly of Eq. (5) (in the variant's arithmetic) and the SSP-RK3
  // combination (FP64); history ring writes
  const int slot_ok = (I.npf > 0);
  const DG *scale = s_scale;
  Walk w6(tid, nth, te);
  for (int item = tid; item < nv * te; item += nth, w6.next()) {
    const int v = w6.o, e = w6.i, ge = e0 + e, le = e + 1;
    const double *wi = sw + ((size_t)v * (TE + 2) + le) * Q;
    const DG *fq = sfx + (size_t)v * TQ + e * Q;
    const CT *sqv = (v >= 2) ? swd + (size_t)(v - 2) * TQ + e * Q : nullptr;
    const DG Wv = (v >= 2) ? sspD[SP_W * ns + v - 2] : DG(0);
    const DG fr = sfh[(size_t)(e + 1) * nv + v], fl = sfh[(size_t)e * nv + v];
    DG fqr[Q], sqr[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      fqr[q] = fq[q];
      // the production rates in the flux's type (on the integer pipeline)
      sqr[q] = (v >= 2) ? conv_r<DG>(sqv[q]) : DG(0);
    }
    double out[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      DG V = 0, S = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if constexpr (MIX) {
          V = fma(BF.WdP[q][i], fqr[q], V);
          S = fma(BF.WPh[q][i], sqr[q], S);
        } else {
          V = fma(B.WdP[q][i], fqr[q], V);
          S = fma(B.WPh[q][i], sqr[q], S);
        }
      }
      DG surf = (i & 1) ? (V - fr - fl) : (V - fr + fl);
      double r;
      if constexpr (MIX) r = f2d_exact(fmaf(scale[i], surf, Wv * S));
      else r = fma(scale[i], surf, Wv * S);
      size_t gi = ((size_t)v * N + ge) * Q + i;
      double o;
      if (I.lserk) {
        // 2N-storage LSERK: dq <- A_s dq + dt L, w <- w + B_s dq (A_0 = 0)
        const double dq =
            (A.s == 0) ? I.dt * r : fma(I.rk_a[A.s], swn[(size_t)v * TQ + e * Q + i], I.dt * r);
        I.wq[gi] = dq;
        o = fma(I.rk_b[A.s], dq, wi[i]);
      } else if (A.s == 0) {
        o = fma(I.dt, r, wi[i]);  // the stage input is w^n
      } else {
        const double wn = swn[(size_t)v * TQ + e * Q + i];
        if (A.s == 1) o = fma(0.25, fma(I.dt, r, wi[i]), 0.75 * wn);
        else o = fma(2.0 / 3.0, fma(I.dt, r, wi[i]), (1.0 / 3.0) * wn);
      }
      out[i] = o;
      I.wpre[gi] = o;
      A_wnext[gi] = o;
    }
    if (slot_ok) {
      int pr = I.pf_of_right[ge], pl = I.pf_of_left[ge];
      if (pr >= 0) {
        // left element of the PE face: its trace at xi = +1
        size_t b = ring_block(I, nstep, A.s, pr, 0) + (size_t)v * Q;
        for (int i = 0; i < Q; ++i) I.ring_pre[b + i] = out[i];
        if constexpr (!UNSYNC)
          I.ring_in[ring_trace(I, nstep, A.s, pr, 0) + v] =
              (DFCHEM && !visc) ? f2d_exact(trace_f<Q>(wi, false)) : trace_of<Q>(wi, false);
      }
      if (pl >= 0) {
        // right element of the PE face: its trace at xi = -1
        size_t b = ring_block(I, nstep, A.s, pl, 1) + (size_t)v * Q;
        for (int i = 0; i < Q; ++i) I.ring_pre[b + i] = out[i];
        if constexpr (!UNSYNC)
          I.ring_in[ring_trace(I, nstep, A.s, pl, 1) + v] =
              (DFCHEM && !visc) ? f2d_exact(trace_f<Q>(wi, true)) : trace_of<Q>(wi, true);
      }
    }
  }
}

template <int Q, int PREC, bool VISC>
__global__ void __launch_bounds__(stage_max_threads(PREC, VISC)) stage_kernel(Mech M, StageArgs A) {
  pdl_wait();
  __shared__ Inst sI;
  const int2 tile = A.tiles[blockIdx.x];
  load_inst(sI, A.insts + tile.x);
  __syncthreads();
  stage_body<Q, PREC, false, VISC>(M, A, sI, tile.y, min(A.TE, sI.n_elem - tile.y), *sI.step,
                                   nullptr);
}

template <typename R>
__device__ inline R minmod3(R a, R b, R c) {
  if (a > R(0) && b > R(0) && c > R(0)) return fmin(a, fmin(b, c));
  if (a < R(0) && b < R(0) && c < R(0)) return fmax(a, fmax(b, c));
  return R(0);
}

// Threads per limiter CTA. A CTA limits EPB = 32 elements (4 lanes per element
// in the indicator) or, for small mixed-precision groups, EPB = 16 (8 lanes), so
// that small meshes still spread over every SM; all threads stage the tile and
// run the WENO phase.
constexpr int LIM_THREADS = 128;
constexpr int LIM_EPB_MAX = 32;

// Shared memory (words of the arithmetic type) per troubled element in the WENO
// phase: the element and its two neighbours, the limited characteristic modes,
// gradP.w, the partial-density sums and momenta of the three blocks, phi_k, two
// mode sums.
__host__ __device__ inline int limiter_elem_words(int nv, int ns, int Q) {
  return 3 * nv * Q + nv * Q + 3 * 3 * Q + ns + 2 * Q + 2;
}

// Where the values of a neighbour of element e (side 0 left, 1 right) come from:
// the AT extrapolation of the neighbour's pre-limit history across a delayed PE
// face (Eq. 11, delay k > 0 at PE face pf), or the pre-limit field of element
// src, mirrored at a reflecting wall (the boundary ghost is the element itself).
struct Neighbour {
  int pf, k, ring, src, ghost, side;
};

// ring: the values come from the pre-limit history ring (a delayed PE face, or
// any PE face of the unsynchronised mode, whose delays pd->k the PE observed).
template <bool UNSYNC>
__device__ inline Neighbour neighbour_of(const Inst &I, int64_t nstep, int e, int side,
                                         const PeDelays *pd) {
  Neighbour nb;
  const int N = I.n_elem;
  nb.side = side;
  nb.pf = side == 0 ? I.pf_of_left[e] : I.pf_of_right[e];
  nb.k = 0;
  nb.ring = 0;
  if (nb.pf >= 0) {
    if constexpr (UNSYNC) nb.k = pd->k[side];
    else nb.k = effective_delay(I, nstep, nb.pf);
    nb.ring = (UNSYNC || nb.k > 0) ? 1 : 0;
  }
  nb.src = side == 0 ? e - 1 : e + 1;
  nb.ghost = 0;
  if (nb.src < 0 || nb.src >= N) {
    if (I.bc_left == ADG_BC_PERIODIC) {
      nb.src = (nb.src + N) % N;
    } else {
      nb.src = e;
      nb.ghost = ((side == 0 ? I.bc_left : I.bc_right) == ADG_BC_REFLECT) ? 1 : 0;
    }
  }
  return nb;
}

// Mode j of variable v of a neighbour (from the ring: the sum of the AT levels
// in FP64).
template <bool UNSYNC>
__device__ inline double neighbour_mode(const Inst &I, const double *wpre, int s, int64_t nstep,
                                        const Neighbour &nb, int v, int j, int Q) {
  if (nb.ring) {
    double acc = 0.0;
    for (int m = 0; m < (nb.k > 0 ? I.at_order : 1); ++m)
      acc += I.at[nb.k][m] * ring_load<UNSYNC>(I.ring_pre + ring_block(I, nstep - nb.k - m, s,
                                                                        nb.pf, nb.side) +
                                               (size_t)v * Q + j);
    return acc;
  }
  double x = wpre[((size_t)v * I.n_elem + nb.src) * Q + j];
  if (nb.ghost && (((j & 1) != 0) != (v == 0))) x = -x;
  return x;
}


// Troubled-cell indicator of element e (Sec. 3.3), a group of L lanes, in the
// arithmetic type R. In each characteristic field of L(wbar_e) the face
// deviations v(+1) - vbar and vbar - v(-1) go through the TVB-modified minmod
// with the neighbours' mean differences; deviations below I.ind_floor of the
// field's magnitude sum_v |L_kv| sigma_v count as zero (the rounding guard of
// indicator_guard: the paper's TVD criterion has no threshold). Three passes
// over the variables, the species and the fields split over the group's lanes:
// the thermodynamics of the cell average; gradP.w, the partial-density sum and the
// momentum of the data the test compares; the characteristic values per field,
// with the branch-free coefficients (A, B, C, D) described at the limiter
// kernel. Every lane of the warp calls it (shuffles); the result is the same on
// the group's lanes.
// FP64: the data are the values at five points (own average, faces +1 and -1,
// neighbours' averages), and the test takes their differences in
// characteristic space. FP32: the transform is linear, so it is applied to the
// four differences themselves, formed before any rounding to float can cancel:
// the face deviations are sums of the modes >= 1 (sum_j w_j and
// -sum_j (-1)^j w_j), and the neighbours' mean differences are taken on the
// double means carried as float pairs (hi, lo). A float run then resolves
// deviations far below the float rounding of the means themselves.
// own: modes of variable 0 of the element in the staged tile (variables vs
// apart, the neighbours' modes Q before and after, halo ghosts included);
// own_lo (FP32): low parts of the element's means (variables ls apart,
// neighbours 1 before and after); spf: species fields in R; atl, atr (and
// atl_lo, atr_lo): the AT-extrapolated averages [nv] of a neighbour across a
// delayed PE face, or null.
template <int Q, int L, typename R>
__device__ bool troubled_cell(const Mech &M, const Inst &I, int s, int64_t nstep, int e,
                              const R *own, int vs, const R *spf, const R *atl, const R *atr,
                              const R *own_lo = nullptr, int ls = 0, const R *atl_lo = nullptr,
                              const R *atr_lo = nullptr) {
  constexpr bool DIFF = std::is_same<R, float>::value;
  constexpr int NP = DIFF ? 4 : 5;  // data per variable
  const int ns = M.ns, nv = ns + 2;
  const int lane = threadIdx.x & 31, li = lane % L;
  const unsigned FULL = 0xffffffffu;
  const R *qW = spf + SP_QW * ns, *cvW = spf + SP_CVW * ns;
  const R *RW = spf + SP_RW * ns, *cpW = spf + SP_CPW * ns;
  auto allsum = [&](R x) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o, L);
    return x;
  };
  // the data of variable v: FP64, the values at the five points; FP32, the
  // differences (v(+1) - vbar, vbar - v(-1), vbar_R - vbar, vbar - vbar_L)
  auto points = [&](int v, R *x) {
    const R *w = own + (size_t)v * vs;
    if constexpr (DIFF) {
      R sp = 0, sm = 0;
#pragma unroll
      for (int j = 1; j < Q; ++j) {
        sp += w[j];
        sm += (j & 1) ? w[j] : -w[j];
      }
      const R *lo = own_lo + (size_t)v * ls;
      const R rh = atr ? atr[v] : w[Q], rl = atr ? atr_lo[v] : lo[1];
      const R lh = atl ? atl[v] : w[-Q], ll = atl ? atl_lo[v] : lo[-1];
      x[0] = sp;
      x[1] = sm;
      x[2] = (rh - w[0]) + (rl - lo[0]);
      x[3] = (w[0] - lh) + (lo[0] - ll);
    } else {
      R sp = 0, sm = 0;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        sp += w[j];
        sm += (j & 1) ? -w[j] : w[j];
      }
      x[0] = w[0];
      x[1] = sp;
      x[2] = sm;
      x[3] = atl ? atl[v] : w[-Q];
      x[4] = atr ? atr[v] : w[Q];
    }
  };
  // 1. thermodynamics of the cell average
  R rho = 0, qsum = 0, cv = 0, Rm = 0, cpm = 0;
  for (int i = li; i < ns; i += L) {
    R r = own[(size_t)(2 + i) * vs];
    rho += r;
    qsum = fma(r, qW[i], qsum);
    cv = fma(r, cvW[i], cv);
    Rm = fma(r, RW[i], Rm);
    cpm = fma(r, cpW[i], cpm);
  }
  rho = allsum(rho);
  qsum = allsum(qsum);
  cv = allsum(cv);
  Rm = allsum(Rm);
  cpm = allsum(cpm);
  const R irho = R(1) / rho, icv = R(1) / cv;
  const R m0 = own[0], E0 = own[vs];
  const R u = m0 * irho;
  const R T = (E0 - R(0.5) * m0 * u - qsum) * icv;
  const R P = T * Rm;
  const R gam = cpm * icv, g = gam - R(1);
  const R a = sqrt(gam * P * irho);
  const R ia2 = R(1) / (a * a), ha2 = R(0.5) * ia2;
  if (li == 0 && (!(rho > R(0)) || !(T > R(0)) || !isfinite(T)))
    report_error(I, ADG_ERR_NONPHYSICAL, e, s, nstep);
  auto phi_of = [&](int i) { return fma(g, fma(-cvW[i], T, R(0.5) * u * u - qW[i]), T * RW[i]); };
  // 2. gradP.w, sum rho Y and rho u of the data; sums of |phi|
  R gp[NP], rs[NP], mm[NP], x[NP];
  R sphi = 0, sphm = 0, sphp = 0;
  points(0, mm);
  points(1, x);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    gp[p] = li == 0 ? g * fma(-u, mm[p], x[p]) : R(0);
    rs[p] = 0;
  }
  for (int i = li; i < ns; i += L) {
    const R ph = phi_of(i);
    sphi += fabs(ph);
    sphm += fabs(ph - a * u);
    sphp += fabs(ph + a * u);
    points(2 + i, x);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      gp[p] = fma(ph, x[p], gp[p]);
      rs[p] += x[p];
    }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    gp[p] = allsum(gp[p]);
    rs[p] = allsum(rs[p]);
  }
  sphi = allsum(sphi);
  sphm = allsum(sphm);
  sphp = allsum(sphp);
  // 3. the characteristic fields, k = 0 and nv-1 acoustic, k = 1..ns species k-1
  const R sig0 = fma(rho, a, fabs(m0)), sig1 = fabs(E0), sigr = rho;
  const R tvb = conv_lim<R>(I.tvb), tau = conv_lim<R>(I.ind_floor), taup = conv_lim<R>(I.ind_floor_p);
  bool tr = false;
  for (int k = li; k < nv; k += L) {
    R v[NP], scale, scale_p;  // the field's magnitude, and its momentum and energy part
    if (k == 0 || k == nv - 1) {
      const R sgn = k == 0 ? R(-1) : R(1);
      const R cA = ha2, cB = sgn * a * ha2, cC = -sgn * a * u * ha2;
#pragma unroll
      for (int p = 0; p < NP; ++p) v[p] = fma(cA, gp[p], fma(cB, mm[p], cC * rs[p]));
      const R srr = cA * (k == 0 ? sphp : sphm);
      scale_p = fma(fabs(fma(cA, -u * g, cB)), sig0, fabs(cA * g) * sig1);
      scale = fma(srr, sigr, scale_p);
    } else {
      const int i = k - 1;
      points(2 + i, x);
      const R cA = -own[(size_t)(2 + i) * vs] * irho * ia2;
      const R ph = phi_of(i);
#pragma unroll
      for (int p = 0; p < NP; ++p) v[p] = fma(cA, gp[p], x[p]);
      const R srr = fabs(fma(cA, ph, R(1))) + fabs(cA) * (sphi - fabs(ph));
      scale_p = fma(fabs(cA * -u * g), sig0, fabs(cA * g) * sig1);
      scale = fma(srr, sigr, scale_p);
    }
    R ut, utt, dp, dm;
    if constexpr (DIFF) {
      ut = v[0];
      utt = v[1];
      dp = v[2];
      dm = v[3];
    } else {
      ut = v[1] - v[0];
      utt = v[0] - v[2];
      dp = v[4] - v[0];
      dm = v[0] - v[3];
    }
    const R fl = fma(tau, scale, taup * scale_p);
    if (fabs(ut) > fl && fabs(ut) > tvb && minmod3(ut, dp, dm) != ut) tr = true;
    if (fabs(utt) > fl && fabs(utt) > tvb && minmod3(utt, dp, dm) != utt) tr = true;
  }
  const unsigned bal = __ballot_sync(FULL, tr);
  const unsigned gm = ((1u << L) - 1u) << (lane - li);
  return (bal & gm) != 0u;
}

// Troubled-cell indicator and (AT-)WENO limiter (Sec. 3.3, Eq. 9-11), in the
// arithmetic type of the precision variant. Phase 1: one element per thread
// runs the indicator and writes its flag; troubled elements go to a list in
// shared memory. Phase 2: a group of G lanes per troubled element (G = 16 when
// nv <= 16, else 32) reconstructs its characteristic fields with WENO and
// writes modes >= 1 of the next stage's input (the stage kernel wrote the
// pre-limit output there for every element already).
// Eigen-structure of the frozen Jacobian at the cell average: right vectors
// r_-/+ = (u -/+ a, H -/+ u a, Y), species r_k = (u, u^2 - phi_k/g, e_k); left
// vectors l_-/+ = (gradP -/+ a (1, 0, -u..-u)) / (2 a^2), l_k = e_k - Y_k gradP/a^2,
// gradP = (-u g, g, phi_1..phi_ns), g = gamma - 1, phi_k = g (u^2/2 - e_k) + R T / W_k.
// Every characteristic value is written in one branch-free form,
// v = A gradP.w + B (rho u)_w + C (sum rho Y)_w + D (rho Y_k)_w,
// with (A, B, C, D) = (1/2a^2, -/+ a/2a^2, +/- a u/2a^2, 0) for the acoustic fields
// and (-Y_k/a^2, 0, 0, 1) for species k.
// Limiting of one block: elements [e0, e0 + te) of instance I, stage s, step
// level nstep, LIM_THREADS threads. With UNSYNC the PE faces take the delays
// pd->k observed by a PE that runs without synchronisation.
template <int Q, int G, bool MIX, int EPB, bool UNSYNC>
__device__ __forceinline__ void limiter_body(const Mech &M, const LimArgs &A, const Inst &I,
                                             const int e0, const int te, const int64_t nstep,
                                             const PeDelays *pd) {
  // lanes per element in the indicator: every thread in the mixed variant; in
  // FP64 two warps, since a warp instruction costs the FP64 pipe the same with
  // one lane per element or four: 4 lanes for CTAs of 16 elements (groups too
  // small for two CTAs of 32 per SM, where the element's serial chain bounds
  // the time), 2 for CTAs of 32 (FP64 throughput bounds it)
  constexpr int LIM_L = MIX ? LIM_THREADS / EPB : (EPB == LIM_EPB_MAX ? 2 : 4);
  static_assert((EPB * LIM_L) % 32 == 0 && EPB * LIM_L <= LIM_THREADS, "indicator warps");
  using DG = dg_t<MIX>;
  extern __shared__ __align__(16) double lsm_raw[];
  DG *lsm = reinterpret_cast<DG *>(lsm_raw);
  __shared__ int s_list[EPB];
  __shared__ int s_n;
  __shared__ Neighbour s_nb[2][EPB];
  if (I.limiter == ADG_LIM_NONE) return;
  if (threadIdx.x == 0) s_n = 0;
  const int N = I.n_elem, nv = I.nv, ns = M.ns;

  // 1. stage the CTA's elements with a one-element halo (ghosts at walls) and
  // the species fields in the variant's type; then the indicator, one element
  // per thread
  const int vs = (EPB + 2) * Q, ls = EPB + 2;
  constexpr int LO = MIX ? 1 : 0;                  // FP32: low parts of the means
  DG *spf = lsm;                                   // [SP_NFIELDS][ns]
  DG *atn = spf + SP_NFIELDS * ns;                 // [2][EPB][nv] AT neighbour averages
  DG *tile = atn + 2 * EPB * nv;                   // [nv][EPB + 2][Q]
  DG *tlo = tile + (size_t)nv * vs;                // [nv][EPB + 2] (FP32) mean - (float) mean
  DG *alo = tlo + (size_t)LO * nv * ls;            // [2][EPB][nv] (FP32) the same of atn
  DG *wsp = alo + (size_t)LO * 2 * EPB * nv;       // WENO workspace
  for (int k = threadIdx.x; k < SP_NFIELDS * ns; k += blockDim.x) spf[k] = conv_lim<DG>(M.sp[k]);
  if ((int)threadIdx.x < 2 * te) {
    const int side = threadIdx.x / te, le = threadIdx.x - side * te;
    s_nb[side][le] = neighbour_of<UNSYNC>(I, nstep, e0 + le, side, pd);
  }
  {
    // batches of loads in flight per thread before they are used
    constexpr int BATCH = 8;
    const bool periodic = (I.bc_left == ADG_BC_PERIODIC);
    const int span = (te + 2) * Q, total = nv * span, nth = blockDim.x;
    Walk wk(threadIdx.x, nth, span);  // (variable, position in the span) of each load
    for (int base = threadIdx.x; base < total; base += BATCH * nth) {
      double xs[BATCH];
      int dst[BATCH], mean[BATCH];  // tile index; index of the mean's low part, or -1
#pragma unroll
      for (int b = 0; b < BATCH; ++b) {
        const int idx = base + b * nth;
        const int v = wk.o, r = wk.i;
        wk.next();
        dst[b] = -1;
        mean[b] = -1;
        xs[b] = 0.0;
        if (idx < total) {
          const int le = r / Q, j = r - le * Q;
          if (j == 0) mean[b] = v * ls + le;
          int src = e0 - 1 + le;
          bool mirror = false;
          if (src < 0 || src >= N) {
            if (periodic) {
              src = (src + N) % N;
            } else {
              const bool left = src < 0;
              src = left ? 0 : N - 1;
              mirror = ((left ? I.bc_left : I.bc_right) == ADG_BC_REFLECT);
            }
          }
          xs[b] = I.wpre[((size_t)v * N + src) * Q + j];
          if (mirror && (((j & 1) != 0) != (v == 0))) xs[b] = -xs[b];
          dst[b] = v * vs + le * Q + j;
        }
      }
#pragma unroll
      for (int b = 0; b < BATCH; ++b)
        if (dst[b] >= 0) {
          const DG hi = conv_lim<DG>(xs[b]);
          tile[dst[b]] = hi;
          if constexpr (MIX) {
            if (mean[b] >= 0) tlo[mean[b]] = conv_lim<DG>(xs[b] - f2d_exact(hi));
          }
        }
    }
  }
  __syncthreads();
  // averages of the neighbours across delayed PE faces (Eq. 11), one
  // (side, element, variable) per item
  for (int item = threadIdx.x; item < 2 * te * nv; item += blockDim.x) {
    const int side = item / (te * nv), r = item - side * te * nv, le = r / nv, v = r - le * nv;
    const Neighbour &nb = s_nb[side][le];
    if (nb.ring) {
      const double x = neighbour_mode<UNSYNC>(I, I.wpre, A.s, nstep, nb, v, 0, Q);
      const DG hi = conv_lim<DG>(x);
      atn[(side * EPB + le) * nv + v] = hi;
      if constexpr (MIX) alo[(side * EPB + le) * nv + v] = conv_lim<DG>(x - f2d_exact(hi));
    }
  }
  __syncthreads();
  if (threadIdx.x < EPB * LIM_L) {
    // the first EPB LIM_L threads (whole warps) run the indicator, every lane of
    // them (shuffles); groups past the last element work on the first element
    // and write nothing
    const int le = threadIdx.x / LIM_L;
    const bool valid = le < te;
    const int lv = valid ? le : 0, e = e0 + lv;
    const DG *atl = s_nb[0][lv].ring ? atn + lv * nv : nullptr;
    const DG *atr = s_nb[1][lv].ring ? atn + (EPB + lv) * nv : nullptr;
    const bool t = troubled_cell<Q, LIM_L, DG>(
        M, I, A.s, nstep, e, tile + (lv + 1) * Q, vs, spf, atl, atr,
        MIX ? tlo + lv + 1 : nullptr, ls, MIX ? alo + lv * nv : nullptr,
        MIX ? alo + (EPB + lv) * nv : nullptr);
    if (valid && threadIdx.x % LIM_L == 0) {
      I.flags[(size_t)A.s * N + e] = t ? 1 : 0;
      if (t) {
        I.count[e] += 1;
        s_list[atomicAdd(&s_n, 1)] = e;
      }
    }
  }
  __syncthreads();
  const int n_tr = s_n;
  if (n_tr == 0) return;

  // 2. WENO (Eq. 9-10) on the troubled elements, G lanes each
  const Basis &B = c_basis[Q - 2];
  const BasisF &BF = c_basis_f[Q - 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane % G, gw = lane / G;
  constexpr int EPW = 32 / G;
  constexpr int NWARP = LIM_THREADS / 32;
  const int slot = warp * EPW + gw;
  double *A_wout = stage_output(I, A.s);
  const double *A_wpre = I.wpre;
  const unsigned FULL = 0xffffffffu;
  const unsigned gmask = (G == 32) ? FULL : (0xffffu << (16 * gw));
  const size_t VS = (size_t)N * Q;
  const int NB = nv * Q;
  DG *blk = wsp + (size_t)slot * limiter_elem_words(nv, ns, Q);  // [3][nv][Q]
  DG *vlim = blk + 3 * NB;                                        // [nv][Q]
  DG *gpv = vlim + NB;                                            // [3][Q]
  DG *rsv = gpv + 3 * Q;                                          // [3][Q]
  DG *mmv = rsv + 3 * Q;                                          // [3][Q]
  DG *phi = mmv + 3 * Q;                                          // [ns]
  DG *sums = phi + ns;                                            // [2][Q]
  const DG *qWd = spf + SP_QW * ns, *cvWd = spf + SP_CVW * ns;
  const DG *RWd = spf + SP_RW * ns, *cpWd = spf + SP_CPW * ns;
  for (int base = 0; base < n_tr; base += NWARP * EPW) {
    const int idx = base + slot;
    const bool valid = idx < n_tr;
    const int e = valid ? s_list[idx] : 0;
    // the element and its neighbours (pre-limit, AT-extrapolated or ghost)
    if (valid) {
      const Neighbour nl = neighbour_of<UNSYNC>(I, nstep, e, 0, pd),
                      nr = neighbour_of<UNSYNC>(I, nstep, e, 1, pd);
      for (int t = gl; t < NB; t += G) {
        const int v = t / Q, j = t - v * Q;
        blk[t] = conv_lim<DG>(A_wpre[(size_t)v * VS + (size_t)e * Q + j]);
        blk[NB + t] = conv_lim<DG>(neighbour_mode<UNSYNC>(I, A_wpre, A.s, nstep, nl, v, j, Q));
        blk[2 * NB + t] = conv_lim<DG>(neighbour_mode<UNSYNC>(I, A_wpre, A.s, nstep, nr, v, j, Q));
      }
    }
    __syncwarp();
    // cell-average thermo and eigen-quantities (species sums split over lanes)
    DG rho = 0, qsum = 0, cv = 0, Rm = 0, cpm = 0;
    if (valid)
      for (int i = gl; i < ns; i += G) {
        DG r = blk[(2 + i) * Q];
        rho += r;
        qsum = fma(r, qWd[i], qsum);
        cv = fma(r, cvWd[i], cv);
        Rm = fma(r, RWd[i], Rm);
        cpm = fma(r, cpWd[i], cpm);
      }
    for (int o = G / 2; o > 0; o >>= 1) {
      rho += __shfl_xor_sync(FULL, rho, o, G);
      qsum += __shfl_xor_sync(FULL, qsum, o, G);
      cv += __shfl_xor_sync(FULL, cv, o, G);
      Rm += __shfl_xor_sync(FULL, Rm, o, G);
      cpm += __shfl_xor_sync(FULL, cpm, o, G);
    }
    if (!valid) {
      rho = 1;
      cv = 1;
      cpm = 2;
      Rm = 1;
    }
    const DG irho = DG(1) / rho, icv = DG(1) / cv;
    const DG m0 = valid ? blk[0] : DG(0), E0 = valid ? blk[Q] : DG(1);
    const DG u = m0 * irho;
    const DG T = (E0 - DG(0.5) * m0 * u - qsum) * icv;
    const DG P = T * Rm;
    const DG gam = cpm * icv, g = gam - DG(1);
    const DG a = sqrt(gam * P * irho);
    const DG H = (E0 + P) * irho;
    const DG ia2 = DG(1) / (a * a);
    if (valid)
      for (int i = gl; i < ns; i += G)
        phi[i] = fma(g, fma(-cvWd[i], T, DG(0.5) * u * u - qWd[i]), T * RWd[i]);
    __syncwarp();
    if (valid)
      for (int t = gl; t < 3 * Q; t += G) {
        int b = t / Q, j = t - b * Q;
        const DG *x = blk + b * NB;
        DG acc = g * fma(-u, x[j], x[Q + j]), sr = 0;
        for (int i = 0; i < ns; ++i) {
          DG r = x[(2 + i) * Q + j];
          acc = fma(phi[i], r, acc);
          sr += r;
        }
        gpv[t] = acc;
        rsv[t] = sr;
        mmv[t] = x[j];
      }
    __syncwarp();
    const DG ha2 = DG(0.5) * ia2;
    auto coef = [&](int k, DG &cA, DG &cB, DG &cC, DG &cD, int &ri) {
      bool ac = (k == 0) || (k == nv - 1);
      DG sgn = (k == 0) ? DG(-1) : DG(1);
      ri = ac ? 0 : k - 1;
      DG Yk = ac ? DG(0) : blk[(2 + ri) * Q] * irho;
      cA = ac ? ha2 : -Yk * ia2;
      cB = ac ? sgn * a * ha2 : DG(0);
      cC = ac ? -sgn * a * u * ha2 : DG(0);
      cD = ac ? DG(0) : DG(1);
    };
    auto val = [&](DG cA, DG cB, DG cC, DG cD, int ri, int b, int j) {
      return fma(cA, gpv[b * Q + j],
                 fma(cB, mmv[b * Q + j], fma(cC, rsv[b * Q + j], cD * blk[b * NB + (2 + ri) * Q + j])));
    };
    // WENO per characteristic field, the group's lanes over fields
    const DG gmw[3] = {DG(0.001), DG(0.998), DG(0.001)};
    const DG eps = DG(1e-6);
    if (valid)
      for (int k = gl; k < nv; k += G) {
        DG cA, cB, cC, cD;
        int ri;
        coef(k, cA, cB, cC, cD, ri);
        DG vo[Q], vl0[Q], vr0[Q], vl[Q], vr[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          vo[j] = val(cA, cB, cC, cD, ri, 0, j);
          vl0[j] = val(cA, cB, cC, cD, ri, 1, j);
          vr0[j] = val(cA, cB, cC, cD, ri, 2, j);
        }
        // neighbours continued into this cell, their mean replaced by the own mean
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          DG al = 0, ar = 0;
#pragma unroll
          for (int j = 0; j < Q; ++j) {
            if constexpr (MIX) {
              al = fma(BF.Sl[i][j], vl0[j], al);
              ar = fma(BF.Sr[i][j], vr0[j], ar);
            } else {
              al = fma(B.Sl[i][j], vl0[j], al);
              ar = fma(B.Sr[i][j], vr0[j], ar);
            }
          }
          vl[i] = al;
          vr[i] = ar;
        }
        vl[0] = vo[0];
        vr[0] = vo[0];
        DG be[3] = {0, 0, 0};
#pragma unroll
        for (int i = 1; i < Q; ++i)
#pragma unroll
          for (int j = 1; j < Q; ++j) {
            DG bij = MIX ? (DG)BF.B[i][j] : (DG)B.B[i][j];
            be[0] = fma(vl[i] * bij, vl[j], be[0]);
            be[1] = fma(vo[i] * bij, vo[j], be[1]);
            be[2] = fma(vr[i] * bij, vr[j], be[2]);
          }
        DG wt[3], sw = 0;
        if constexpr (MIX) {
          // the same normalised weights written as ratios, safe from overflow in FP32
          DG dmin = fmin(eps + be[0], fmin(eps + be[1], eps + be[2]));
          for (int t = 0; t < 3; ++t) {
            DG rr = dmin / (eps + be[t]);
            wt[t] = gmw[t] * rr * rr;
            sw += wt[t];
          }
        } else {
          for (int t = 0; t < 3; ++t) {
            DG d = eps + be[t];
            wt[t] = gmw[t] / (d * d);
            sw += wt[t];
          }
        }
        DG isw = DG(1) / sw;
        vlim[k * Q] = vo[0];
#pragma unroll
        for (int i = 1; i < Q; ++i)
          vlim[k * Q + i] = (wt[0] * vl[i] + wt[1] * vo[i] + wt[2] * vr[i]) * isw;
      }
    __syncwarp();
    // back to conserved variables with R (modes >= 1; the cell average is kept)
    if (valid)
      for (int i = gl; i < Q; i += G) {
        DG s1 = 0, s2 = 0;
        for (int k = 1; k < nv - 1; ++k) {
          DG x = vlim[k * Q + i];
          s1 += x;
          s2 = fma(x, u * u - phi[k - 1] / g, s2);
        }
        sums[i] = s1;
        sums[Q + i] = s2;
      }
    __syncwarp();
    if (valid) {
      double *out = A_wout + (size_t)e * Q;
      for (int t = gl; t < NB; t += G) {
        int v = t / Q, i = t - v * Q;
        if (i == 0) continue;
        DG lm = vlim[i], lp = vlim[(nv - 1) * Q + i];
        DG o;
        if (v == 0) o = lm * (u - a) + lp * (u + a) + u * sums[i];
        else if (v == 1) o = lm * (H - u * a) + lp * (H + u * a) + sums[Q + i];
        else o = (lm + lp) * (blk[v * Q] * irho) + vlim[(v - 1) * Q + i];
        out[(size_t)v * VS + i] = conv_r<double>(o);
      }
    }
    __syncwarp();
  }
  (void)gmask;
}

// The mixed variants are held to 64 registers a thread (eight 128-thread CTAs,
// 32 warps, per SM instead of five at 96 registers): their limiter waits on
// instruction latency, and the extra warps hide it (1.12 -> 0.97 ms per RK
// stage on the 512-instance ensemble, a few bytes of spills). The FP64 limiter
// is bound by the FP64 pipe; with a hint of four CTAs per SM (at most 128
// registers, a few bytes of spills at p = 4) it took 4.30 ms per RK stage
// against 4.40 without a hint and 4.87 with a hint of one, which lets its
// allocation grow by up to 30 registers.
template <int Q, int G, bool MIX, int EPB>
__global__ void __launch_bounds__(LIM_THREADS, MIX ? 8 : 4) limiter_kernel(Mech M, LimArgs A) {
  pdl_enter();
  __shared__ Inst sI;
  const int2 blkid = A.blocks[blockIdx.x];
  load_inst(sI, A.insts + blkid.x);
  __syncthreads();
  limiter_body<Q, G, MIX, EPB, false>(M, A, sI, blkid.y, min(EPB, sI.n_elem - blkid.y),
                                      *sI.step, nullptr);
}

template <int Q, int G, bool MIX, int EPB>
static size_t limiter_smem_bytes(int nv, int ns) {
  constexpr int EPW = 32 / G;
  size_t smem = ((size_t)SP_NFIELDS * ns + (size_t)2 * EPB * nv + (size_t)nv * (EPB + 2) * Q +
                 (MIX ? (size_t)nv * (EPB + 2) + (size_t)2 * EPB * nv : 0) +
                 (size_t)(LIM_THREADS / 32) * EPW * limiter_elem_words(nv, ns, Q)) *
                (MIX ? sizeof(float) : sizeof(double));
  return (smem + 15) & ~(size_t)15;
}

// Launchers and set-up of one precision variant (instantiated by the unit of
// that variant only).
template <int Q, int PREC, bool VISC>
static cudaError_t launch_stage_q(const Mech &M, const StageArgs &A, int n_tiles,
                                  cudaStream_t st) {
  if ((A.visc != 0) != VISC) return cudaErrorInvalidValue;
  size_t smem = stage_smem_bytes(A.TE, Q, M.ns, M.nr, M.nterm, A.O, PREC, VISC);
  if (A.NT < 32 || A.NT > stage_max_threads(PREC, VISC) || A.NT % 32) return cudaErrorInvalidValue;
  return launch_pdl(stage_kernel<Q, PREC, VISC>, dim3(n_tiles), dim3(A.NT), smem, st, M, A);
}

template <int PREC, bool VISC>
static cudaError_t launch_stage_variant(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                                        cudaStream_t st) {
  switch (Q) {
    case 2: return launch_stage_q<2, PREC, VISC>(M, A, n_tiles, st);
    case 3: return launch_stage_q<3, PREC, VISC>(M, A, n_tiles, st);
    case 4: return launch_stage_q<4, PREC, VISC>(M, A, n_tiles, st);
    case 5: return launch_stage_q<5, PREC, VISC>(M, A, n_tiles, st);
  }
  return cudaErrorInvalidValue;
}

// Raise the dynamic shared-memory limit of the stage kernels of one variant.
template <int PREC, bool VISC>
static cudaError_t prepare_stage_variant() {
  const int lim = 200 * 1024;
  cudaError_t e = cudaSuccess;
  const void *k[4] = {(const void *)stage_kernel<2, PREC, VISC>,
                      (const void *)stage_kernel<3, PREC, VISC>,
                      (const void *)stage_kernel<4, PREC, VISC>,
                      (const void *)stage_kernel<5, PREC, VISC>};
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    e = cudaFuncSetAttribute(k[i], cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e;
}

template <int Q, int G, bool MIX, int EPB>
static cudaError_t launch_limiter_qge(const Mech &M, const LimArgs &A, int nv, int n_blocks,
                                      cudaStream_t st) {
  const size_t smem = limiter_smem_bytes<Q, G, MIX, EPB>(nv, M.ns);
  return launch_pdl(limiter_kernel<Q, G, MIX, EPB>, dim3(n_blocks), dim3(LIM_THREADS), smem, st,
                    M, A);
}

template <int Q, bool MIX>
static cudaError_t launch_limiter_q(const Mech &M, const LimArgs &A, int nv, int n_blocks,
                                    cudaStream_t st) {
  if constexpr (MIX) {
    if (A.EPB == 8) {
      if (nv <= 16) return launch_limiter_qge<Q, 16, MIX, 8>(M, A, nv, n_blocks, st);
      return launch_limiter_qge<Q, 32, MIX, 8>(M, A, nv, n_blocks, st);
    }
  }
  if (A.EPB == 16) {
    if (nv <= 16) return launch_limiter_qge<Q, 16, MIX, 16>(M, A, nv, n_blocks, st);
    return launch_limiter_qge<Q, 32, MIX, 16>(M, A, nv, n_blocks, st);
  }
  if (A.EPB != LIM_EPB_MAX) return cudaErrorInvalidValue;
  if (nv <= 16) return launch_limiter_qge<Q, 16, MIX, LIM_EPB_MAX>(M, A, nv, n_blocks, st);
  return launch_limiter_qge<Q, 32, MIX, LIM_EPB_MAX>(M, A, nv, n_blocks, st);
}

template <bool MIX>
static cudaError_t launch_limiter_variant(const Mech &M, const LimArgs &A, int Q, int nv,
                                          int n_blocks, cudaStream_t st) {
  switch (Q) {
    case 2: return launch_limiter_q<2, MIX>(M, A, nv, n_blocks, st);
    case 3: return launch_limiter_q<3, MIX>(M, A, nv, n_blocks, st);
    case 4: return launch_limiter_q<4, MIX>(M, A, nv, n_blocks, st);
    case 5: return launch_limiter_q<5, MIX>(M, A, nv, n_blocks, st);
  }
  return cudaErrorInvalidValue;
}

// Raise the dynamic shared-memory limit of every limiter kernel of the variant
// (before any launch or stream capture).
template <bool MIX>
static cudaError_t prepare_limiter_variant() {
  const int lim = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define ADG_SET(...) \
  if (e == cudaSuccess) \
  e = cudaFuncSetAttribute(__VA_ARGS__, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
  if constexpr (MIX) {
    ADG_SET(limiter_kernel<2, 16, MIX, 8>);
    ADG_SET(limiter_kernel<3, 16, MIX, 8>);
    ADG_SET(limiter_kernel<4, 16, MIX, 8>);
    ADG_SET(limiter_kernel<5, 16, MIX, 8>);
    ADG_SET(limiter_kernel<2, 32, MIX, 8>);
    ADG_SET(limiter_kernel<3, 32, MIX, 8>);
    ADG_SET(limiter_kernel<4, 32, MIX, 8>);
    ADG_SET(limiter_kernel<5, 32, MIX, 8>);
  }
  ADG_SET(limiter_kernel<2, 16, MIX, 16>);
  ADG_SET(limiter_kernel<3, 16, MIX, 16>);
  ADG_SET(limiter_kernel<4, 16, MIX, 16>);
  ADG_SET(limiter_kernel<5, 16, MIX, 16>);
  ADG_SET(limiter_kernel<2, 32, MIX, 16>);
  ADG_SET(limiter_kernel<3, 32, MIX, 16>);
  ADG_SET(limiter_kernel<4, 32, MIX, 16>);
  ADG_SET(limiter_kernel<5, 32, MIX, 16>);
  ADG_SET(limiter_kernel<2, 16, MIX, LIM_EPB_MAX>);
  ADG_SET(limiter_kernel<3, 16, MIX, LIM_EPB_MAX>);
  ADG_SET(limiter_kernel<4, 16, MIX, LIM_EPB_MAX>);
  ADG_SET(limiter_kernel<5, 16, MIX, LIM_EPB_MAX>);
  ADG_SET(limiter_kernel<2, 32, MIX, LIM_EPB_MAX>);
  ADG_SET(limiter_kernel<3, 32, MIX, LIM_EPB_MAX>);
  ADG_SET(limiter_kernel<4, 32, MIX, LIM_EPB_MAX>);
  ADG_SET(limiter_kernel<5, 32, MIX, LIM_EPB_MAX>);
#undef ADG_SET
  return e;
}

}  // namespace adg
