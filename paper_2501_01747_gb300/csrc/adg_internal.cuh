// Device-side data structures and physics of the ADG hot path.
//
// Layout in HBM (per instance): modal state [nv][n_elem][p+1] FP64, SoA by
// variable, so that a tile of consecutive elements of one variable is one
// contiguous span; history ring [depth][RK stages][PE faces][2 sides][nv][p+1].
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/adg.h"
#include "adg_math.cuh"

namespace adg {

constexpr double RU = 8.314462618;   // J/mol/K
constexpr double TREF = 298.15;      // K
constexpr double PATM = 101325.0;    // Pa
constexpr int MAXQ = ADG_MAX_P + 1;
constexpr int MAXO = ADG_MAX_AT_ORDER;
constexpr int MAXD = ADG_MAX_DELAY;
constexpr int SIDE = 4;              // species slots per reaction side
constexpr int NET = 8;               // species slots of the net stoichiometry

// Species data (structure of arrays, field f of species i at sp[f * ns + i]).
enum SpeciesField {
  SP_W = 0,     // kg/mol
  SP_INVW,      // 1/W
  SP_QW,        // (h_f - c_p T_ref)/W   : e_i(T) = qW_i + cvW_i T
  SP_CVW,       // (c_p - R)/W
  SP_RW,        // R/W
  SP_CPW,       // c_p/W
  SP_G0,        // (h_f - c_p T_ref)/R   : g_i/(R T) = G0/T + G1 - cpR ln T
  SP_G1,        // c_p/R (1 + ln T_ref) - s0/R
  SP_CPR,       // c_p/R
  SP_INVLE,     // 1/Le (viscous runs)
  SP_NFIELDS
};

// One reversible reaction, 64 bytes. With g_i/(R T) = G0_i/T + G1_i - CPR_i ln T
// (constant c_p), both rate constants are linear in (1, ln T, 1/T):
//   ln k_f = lnA + b ln T - EaR / T,
//   ln k_r = ln k_f + sum_i nu_i g_i/(R T) + dnu ln(R T / P_atm)
//          = kr0 + kr1 ln T + kr2 / T,
// kr0 = lnA + dnu ln(R/P_atm) + sum_i nu_i G1_i, kr1 = b + dnu - sum_i nu_i CPR_i,
// kr2 = -EaR + sum_i nu_i G0_i (nu the net coefficients, dnu their sum).
struct alignas(16) Rxn {
  double lnA, b, mEaR;    // ln k_f = lnA + b ln T + mEaR / T
  double kr0, kr1, kr2;   // ln k_r = kr0 + kr1 ln T + kr2 / T
  uint8_t rs[4], rn[4];   // reactants: species, coefficient (rn = 0 ends)
  uint8_t ps[4], pn[4];   // products
};
static_assert(sizeof(Rxn) == 64, "reaction record is 64 bytes");

// Species -> reaction incidence (the transpose of the net stoichiometry): the
// terms of species i are sx[sx_off[i] .. sx_off[i+1]), each (j << 8) | (nu_ij & 0xff)
// with nu_ij the species' nonzero net coefficient in reaction j, ascending in j.
struct Mech {
  int ns, nr, nterm;
  const double *sp;   // [SP_NFIELDS][ns]
  const Rxn *rx;      // [nr]
  const DF *rxf;      // [nr][6] lnA, b, mEaR, kr0, kr1, kr2 as df32 (mixed variant)
  const int *sx_off;  // [ns + 1]
  const int *sx;      // [nterm]
};

// Host: the device tables of a mechanism. Fills sp [SP_NFIELDS * ns], rx [nr],
// sx_off [ns + 1] and sx [nr * NET]; returns the number of incidence terms, or
// ADG_ERR_ARG for a reaction the tables cannot hold.
int pack_mechanism(const adg_mechanism *m, double *sp, Rxn *rx, int *sx_off, int *sx);
// Host: the rate coefficients of nr reactions as df32, [nr][6].
void pack_rxf(const Rxn *rx, int nr, DF *rxf);

// Per-instance description, passed by value to the kernels.
struct Inst {
  int n_elem, p, nv, npf, depth, at_order;
  int n_stages, lserk;                  // RK stages per step; 2N-storage LSERK scheme
  int viscous, pad0;                    // with the diffusive flux (LDG)
  double mu_ref, ln_T_mu, mu_exp, inv_prandtl;  // synthetic transport model
  double rk_a[ADG_MAX_STAGES], rk_b[ADG_MAX_STAGES];  // its A_s, B_s
  int bc_left, bc_right, flux, limiter, delay_mode, max_delay;
  double dx, dt, tvb;
  uint64_t seed;
  double cum[MAXD + 1];                 // cumulative SAA probabilities
  double at[MAXD + 1][MAXO];            // AT weights c_m(k)
  double *wn, *wa, *wb, *wpre;          // [nv][N][Q]: w^n, stage inputs, pre-limit
  double *wq;                           // [nv][N][Q]: the LSERK register dq (or null)
  double *qx;                           // [nv][N][Q]: LDG auxiliary q = dw/dx (or null)
  double *ring_q;    // history of the PE-face traces of q [depth][S][npf][2][nv] (or null)
  double *ring_in;   // history of the stage inputs' face traces [depth][S][npf][2][nv]
  double *ring_pre;  // history of the pre-limit outputs [depth][S][npf][2][nv][p+1]
  uint8_t *flags;                       // [S][N]
  int32_t *count;                       // [N]
  const int *pf_of_left;                // per element: PE face on its left face or -1
  const int *pf_of_right;               // per element: PE face on its right face or -1
  const int *pf_elem;                   // per PE face: [left element, right element]
  int *err;                             // [4] code, element, stage, step (low bits)
  int64_t *step;                        // step counter of this instance (device)
  int instance;
  int mixed;                            // precision (ADG_FP64, ADG_MIXED, ADG_MIXED_F32CHEM):
                                        // nonzero for FP32 flux, DG operator, limiter
  int face_base, npf_draw;              // PE face f is face (f + face_base) mod npf_draw of
                                        // the whole domain (a subdomain; else 0 and npf)
  double ind_floor, ind_floor_p;        // rounding guards of the indicator (indicator_guard)
};

// Rounding guards of the troubled-cell indicator (Sec. 3.3 gives a TVD test with
// no threshold): a face deviation of characteristic field k counts as zero below
// ind_floor * |field k| + ind_floor_p * |field k|_p, with |field k| =
// sum_v |L_kv| sigma_v its magnitude and |field k|_p the part of it that comes
// from the momentum and the energy.
// FP64 data: 1e-10 of the magnitude, far above its rounding, and nothing else.
// The mixed variants compute the flux and the DG operator in FP32. Their state
// then differs from the FP64 state by about 1e-6 of the momentum and energy (the
// pressure) and by a few 1e-8 of the partial densities, and a deviation below
// that difference is not resolved by them: their guard is 3e-8 of the magnitude
// plus 1e-6 of its momentum-and-energy part. A species field then keeps a guard
// far below the deviations that the FP64 scheme limits (1e-7 and more on the
// workloads here), while a field that carries the pressure ignores that noise.
constexpr double kGuardFP64 = 1e-10;
constexpr double kGuardMixed = 3e-8;
constexpr double kGuardMixedP = 1e-6;
inline double indicator_guard(int precision) {
  return precision == ADG_FP64 ? kGuardFP64 : kGuardMixed;
}
inline double indicator_guard_p(int precision) {
  return precision == ADG_FP64 ? 0.0 : kGuardMixedP;
}

// Programmatic dependent launch for the kernels of a step: each is launched so
// that it may be scheduled while its predecessor drains, waits at entry until
// the predecessor grid has completed and its writes are visible, and lets its
// own successor be scheduled once every one of its CTAs has passed the
// trigger. Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Wait, then release the successor at once: for kernels whose successor's
// waiting CTAs cannot crowd them out of an SM.
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_trigger();
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Delay of PE face f at step n (Sec. 4.1 CAA, Sec. 4.2 SAA).
__host__ __device__ inline int draw_delay(int mode, int max_delay, uint64_t seed,
                                          const double *cum, int64_t n, int f) {
  if (mode == ADG_SYNC) return 0;
  if (mode == ADG_CAA) return (int)(n % (int64_t)(max_delay + 1));
  uint64_t key = seed ^ (((uint64_t)n << 32) + (uint64_t)(uint32_t)f);
  double r = (double)(splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
  for (int k = 0; k <= max_delay; ++k)
    if (r < cum[k]) return k;
  return max_delay;
}

// The whole domain's number of PE face f of an instance (a subdomain numbers its
// own faces from its first cut face; the delays are those of the whole domain).
__host__ __device__ inline int face_number(int f, int face_base, int npf_draw) {
  if (npf_draw <= 0) return f;
  const int g = (f + face_base) % npf_draw;
  return g < 0 ? g + npf_draw : g;
}

// Delay in force: synchronous until the ring holds levels n-k-(o-1).
__device__ inline int effective_delay(const Inst &I, int64_t n, int f) {
  int k = draw_delay(I.delay_mode, I.max_delay, I.seed, I.cum, n,
                     face_number(f, I.face_base, I.npf_draw));
  return (n >= (int64_t)k + I.at_order - 1) ? k : 0;
}

__host__ __device__ inline size_t ring_block(const Inst &I, int64_t level, int s, int pf, int side) {
  int slot = (int)(level % I.depth);
  return ((((size_t)slot * I.n_stages + s) * I.npf + pf) * 2 + side) * (size_t)I.nv * (I.p + 1);
}

// Stage buffers: stage s reads w^n (s = 0) or the previous stage's output, and
// writes the next stage's input, the last stage w^{n+1}; the two intermediate
// buffers alternate (3 stages: w^n -> wa -> wb -> w^n; 5 stages: w^n -> wa ->
// wb -> wa -> wb -> w^n).
__host__ __device__ inline const double *stage_input(const Inst &I, int s) {
  return s == 0 ? I.wn : (s & 1) ? I.wa : I.wb;
}
__host__ __device__ inline double *stage_output(const Inst &I, int s) {
  return s == I.n_stages - 1 ? I.wn : (s & 1) ? I.wb : I.wa;
}

// Offset of the face-trace record (nv values) of one side of a PE face.
__device__ inline size_t ring_trace(const Inst &I, int64_t level, int s, int pf, int side) {
  int slot = (int)(level % I.depth);
  return ((((size_t)slot * I.n_stages + s) * I.npf + pf) * 2 + side) * (size_t)I.nv;
}

__device__ inline void report_error(const Inst &I, int code, int elem, int stage, int64_t n) {
  if (atomicCAS(I.err, 0, code) == 0) {
    I.err[1] = elem;
    I.err[2] = stage;
    I.err[3] = (int)n;
  }
}

// Thermodynamic state of a conserved vector w (stride `st` between variables),
// in the arithmetic type R (double, or float for the mixed-precision flux).
template <typename R>
struct ThermoT {
  R rho, u, T, P, a, gm1;
};
using Thermo = ThermoT<double>;

// T from the internal energy: e(T) is linear for constant c_p, so the Newton
// iteration on e(T) = e reaches its root in one step from any guess; that step
// is this closed form. sp: species fields (shared or global memory).
template <typename R>
__device__ inline ThermoT<R> thermo_t(const R *sp, int ns, const R *w, int st) {
  ThermoT<R> t;
  R rho = 0, qsum = 0, cv = 0, Rm = 0, cpm = 0;
  for (int i = 0; i < ns; ++i) {
    R r = w[(2 + i) * st];
    rho += r;
    qsum = fma(r, sp[SP_QW * ns + i], qsum);
    cv = fma(r, sp[SP_CVW * ns + i], cv);
    Rm = fma(r, sp[SP_RW * ns + i], Rm);
    cpm = fma(r, sp[SP_CPW * ns + i], cpm);
  }
  const R irho = R(1) / rho, icv = R(1) / cv;
  R m = w[0], E = w[st];
  t.rho = rho;
  t.u = m * irho;
  R rhoe = E - R(0.5) * m * t.u;
  t.T = (rhoe - qsum) * icv;
  t.P = t.T * Rm;
  R gam = cpm * icv;
  t.gm1 = gam - R(1);
  t.a = sqrt(gam * t.P * irho);
  return t;
}

__device__ inline Thermo thermo_of(const double *sp, int ns, const double *w, int st) {
  return thermo_t<double>(sp, ns, w, st);
}

// Physical flux component v of w (Eq. 2).
template <typename R>
__device__ inline R phys_flux_t(const R *w, int st, int v, const ThermoT<R> &t) {
  if (v == 0) return w[0] * t.u + t.P;
  if (v == 1) return t.u * (w[st] + t.P);
  return t.u * w[v * st];
}

__device__ inline double phys_flux(const double *w, int st, int v, const Thermo &t) {
  return phys_flux_t<double>(w, st, v, t);
}

// Numerical flux (Sec. 3.1): local Lax-Friedrichs or HLLC (Toro 1994, wave
// speeds S_L = min(u_L - a_L, u_R - a_R), S_R = max(u_L + a_L, u_R + a_R)).
// out[v] for v = 0..nv-1; wl, wr with unit stride.
template <typename R>
__device__ inline void num_flux_t(const R *sp, int ns, int kind, const R *wl, const R *wr,
                                  R *out) {
  const int nv = ns + 2;
  ThermoT<R> L = thermo_t<R>(sp, ns, wl, 1), Rt = thermo_t<R>(sp, ns, wr, 1);
  if (kind == ADG_FLUX_LF) {
    R lam = fmax(fabs(L.u) + L.a, fabs(Rt.u) + Rt.a);
    for (int v = 0; v < nv; ++v)
      out[v] = R(0.5) * (phys_flux_t<R>(wl, 1, v, L) + phys_flux_t<R>(wr, 1, v, Rt) -
                         lam * (wr[v] - wl[v]));
    return;
  }
  R SL = fmin(L.u - L.a, Rt.u - Rt.a);
  R SR = fmax(L.u + L.a, Rt.u + Rt.a);
  R SM = (Rt.P - L.P + L.rho * L.u * (SL - L.u) - Rt.rho * Rt.u * (SR - Rt.u)) /
         (L.rho * (SL - L.u) - Rt.rho * (SR - Rt.u));
  for (int v = 0; v < nv; ++v) {
    R f;
    if (R(0) <= SL) {
      f = phys_flux_t<R>(wl, 1, v, L);
    } else if (R(0) <= SM) {
      R c = L.rho * (SL - L.u) / (SL - SM);
      R us;
      if (v == 0) us = c * SM;
      else if (v == 1) us = c * (wl[1] / L.rho + (SM - L.u) * (SM + L.P / (L.rho * (SL - L.u))));
      else us = c * (wl[v] / L.rho);
      f = phys_flux_t<R>(wl, 1, v, L) + SL * (us - wl[v]);
    } else if (R(0) <= SR) {
      R c = Rt.rho * (SR - Rt.u) / (SR - SM);
      R us;
      if (v == 0) us = c * SM;
      else if (v == 1) us = c * (wr[1] / Rt.rho + (SM - Rt.u) * (SM + Rt.P / (Rt.rho * (SR - Rt.u))));
      else us = c * (wr[v] / Rt.rho);
      f = phys_flux_t<R>(wr, 1, v, Rt) + SR * (us - wr[v]);
    } else {
      f = phys_flux_t<R>(wr, 1, v, Rt);
    }
    out[v] = f;
  }
}

// Gauss-Legendre tables (points, weights, P_j and P_j' at the points) per Q.
struct Basis {
  double x[MAXQ], w[MAXQ];
  double P[MAXQ][MAXQ];   // P[q][j]
  double dP[MAXQ][MAXQ];  // dP[q][j]
  double B[MAXQ][MAXQ];   // smoothness-indicator quadratic form
  double Sl[MAXQ][MAXQ];  // left neighbour continued into the cell
  double Sr[MAXQ][MAXQ];  // right neighbour continued into the cell
  double WdP[MAXQ][MAXQ]; // w_q P_i'(x_q)            (volume integral)
  double WPh[MAXQ][MAXQ]; // w_q P_i(x_q) (2i+1)/2     (source projection)
};

// The same tables rounded to float, for the mixed-precision kernels.
struct BasisF {
  float B[MAXQ][MAXQ], Sl[MAXQ][MAXQ], Sr[MAXQ][MAXQ], WdP[MAXQ][MAXQ], WPh[MAXQ][MAXQ];
};

// Arguments of one stage-kernel launch. A launch covers every instance of one
// polynomial degree: CTA b works on elements [tiles[b].y, tiles[b].y + TE) of
// instance tiles[b].x. Stage s reads w^n (wn) and its input (wn, wa, wb for
// s = 0, 1, 2), writes the pre-limit output to wpre and to the next stage's
// buffer (wa, wb, wn), and reads the step level from the instance's counter.
struct StageArgs {
  const Inst *insts;
  const int2 *tiles;
  int s;
  int TE;     // elements per tile
  int NT;     // threads per CTA
  int O;      // AT levels provided for (largest AT order of the group)
  int visc;   // the group has viscous instances (shared memory holds the viscous region)
};

// Arguments of one limiter launch: CTA b limits the elements of instance
// blocks[b].x starting at blocks[b].y (LIM_WARPS warps, 32/G elements a warp).
struct LimArgs {
  const Inst *insts;
  const int2 *blocks;
  int s;
  int EPB;    // elements per CTA (limiter_elems_per_block)
};

void make_tables(Basis *tables);
cudaError_t upload_basis(const Basis *tables);
int stage_tile(const Mech &M, int Q, int O, int prec, bool visc);
int stage_threads(int TE, int Q, int nr);
// Largest CTA of the stage kernel: 1024 threads for the inviscid mixed variants
// (they fit in 64 registers a thread, so that a tile too large for two CTAs per
// SM can still keep 32 warps resident), 512 otherwise (FP64 and the viscous
// terms need up to 128 registers).
__host__ __device__ constexpr int stage_max_threads(int prec, bool visc) {
  return (prec != ADG_FP64 && !visc) ? 1024 : 512;
}
size_t stage_smem(const Mech &M, int TE, int Q, int O, int prec, bool visc);
cudaError_t prepare_kernels(int nv, int ns, int nr);
cudaError_t launch_stage(const Mech &M, const StageArgs &A, int Q, int prec, int n_tiles,
                         cudaStream_t st);
cudaError_t launch_limiter(const Mech &M, const LimArgs &A, int Q, bool mixed, int nv,
                           int n_blocks, cudaStream_t st);
cudaError_t launch_advance(int64_t *steps, int n, cudaStream_t st);
// A neighbour subdomain's boundary block [nv][Q] into the buffer element at one
// side of a subdomain instance (the stage input of `stage`, or its pre-limit
// output, which also goes into the cut face's pre-limit history at the step the
// device counter holds, so that the copy may be replayed from a graph).
cudaError_t launch_part_import(const Inst *inst, int what, int side, int stage,
                               const double *blk, int nv, int Q, cudaStream_t st);
// Every instance's current state to (to_host) or from a flat host buffer the
// device can address (pinned and mapped): offs[k] is instance k's first double
// in it, offs[n] the total.
cudaError_t launch_states_copy(const Inst *insts, const int64_t *offs, int n, double *host,
                               bool to_host, cudaStream_t st);
cudaError_t launch_aux(const LimArgs &A, int Q, int n_blocks, cudaStream_t st);
// per-variant units (adg_k64.cu, adg_k32.cu, adg_k32f.cu)
cudaError_t launch_stage_fp64(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                              cudaStream_t st);
cudaError_t launch_stage_mixed(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                               cudaStream_t st);
cudaError_t launch_stage_f32chem(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                                 cudaStream_t st);
cudaError_t launch_limiter_fp64(const Mech &M, const LimArgs &A, int Q, int nv, int n_blocks,
                                cudaStream_t st);
cudaError_t launch_limiter_mixed(const Mech &M, const LimArgs &A, int Q, int nv, int n_blocks,
                                 cudaStream_t st);
cudaError_t prepare_fp64();
cudaError_t prepare_mixed();
cudaError_t prepare_f32chem();
// viscous stage kernels (adg_v64.cu, adg_v32.cu)
cudaError_t launch_stage_visc_fp64(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                                   cudaStream_t st);
cudaError_t launch_stage_visc_mixed(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                                    cudaStream_t st);
cudaError_t prepare_visc_fp64();
cudaError_t prepare_visc_mixed();
cudaError_t upload_tables_visc_fp64(const Basis *tables);
cudaError_t upload_tables_visc_mixed(const Basis *tables);
cudaError_t upload_tables_fp64(const Basis *tables);
cudaError_t upload_tables_mixed(const Basis *tables);
cudaError_t upload_tables_f32chem(const Basis *tables);
int limiter_elems_per_block(int64_t n_elem_group, bool mixed);
// the unsynchronised mode (adg_unsync.cuh): one cooperative launch per instance
struct UnsyncArgs {
  const Inst *inst;               // the instance's device record
  int n_pe, npf, n_steps, TE, O;  // PEs, PE faces, steps, elements per stage tile, AT levels
  int EPB;                        // elements per limiter block (as the group's launches)
  int *pub_in, *pub_pre;          // [n_pe] stages published (stage inputs, pre-limit outputs)
  unsigned long long *agree;      // [npf][ADG_MAX_STAGES][MAXD + 1] common flux level:
                                  // (level + 1) << 8 | k
  unsigned long long *hist;       // [2][MAXD + 1] delays observed: flux, limiter
  long long spin_limit;           // polls of a counter before a wait gives up
  int withheld;                   // a PE that never publishes (tests the timeout), or -1
  int slow_pe, slow_us;           // a PE that idles slow_us microseconds per stage, or -1
};
cudaError_t launch_unsync(const Mech &M, const UnsyncArgs &U, int Q, bool mixed, int nv,
                          cudaStream_t st);
cudaError_t prepare_unsync();
cudaError_t upload_tables_unsync(const Basis *tables);
cudaError_t launch_unsync_fp64(const Mech &M, const UnsyncArgs &U, int Q, int nv,
                               cudaStream_t st);
cudaError_t launch_unsync_mixed(const Mech &M, const UnsyncArgs &U, int Q, int nv,
                                cudaStream_t st);
cudaError_t prepare_unsync_fp64();
cudaError_t prepare_unsync_mixed();
cudaError_t upload_tables_unsync_fp64(const Basis *tables);
cudaError_t upload_tables_unsync_mixed(const Basis *tables);
cudaError_t launch_advance_by(int64_t *step, int64_t n, cudaStream_t st);
cudaError_t launch_project(const Mech &M, const Inst &I, const double *prim, double *w,
                           cudaStream_t st);
cudaError_t launch_temperature(const Mech &M, const Inst &I, const double *w, double *T,
                               cudaStream_t st, int what = 0);

}  // namespace adg
