// CUDA kernels of the ADG hot path (sm_103a).
//
// Per RK stage two kernels run, each in an FP64 and a mixed-precision variant
// (MIX: FP32 for the flux, the DG operator and the limiter; FP64 for the
// Gauss-point temperature, the Arrhenius and equilibrium exponentials, the AT
// level sums and the accumulation of the conserved state):
//   stage_kernel<Q,MIX>  : one CTA per tile of TE consecutive elements of one
//                      instance. Loads the tile plus a one-element halo into
//                      shared memory (coalesced per variable); Gauss-point
//                      thermo and flux, one thread per point; chemistry, R
//                      chunks of reactions per point; the TE+1 face fluxes of the
//                      tile (AT levels on separate threads); Eq. (5) assembly and
//                      the SSP-RK3 combination; writes the pre-limit output and
//                      the history ring of PE-boundary elements.
//   limiter_kernel<Q,G,MIX>: G lanes per element: troubled-cell indicator in the
//                      characteristic fields of the cell average and, on troubled
//                      cells, the (AT-)WENO reconstruction of Eq. (9)-(11). The
//                      stage kernel writes the pre-limit output twice (limiter
//                      input and next-stage buffer) so that the limiter only
//                      rewrites troubled cells.
#include <cstdio>
#include <type_traits>

#include "adg_internal.cuh"
#include "adg_math.cuh"

namespace adg {

__constant__ Basis c_basis[ADG_MAX_P];     // index p-1
__constant__ BasisF c_basis_f[ADG_MAX_P];  // the same, rounded to float

__constant__ ExpTable c_exp;

template <bool MIX>
using dg_t = typename std::conditional<MIX, float, double>::type;

// Shared-memory footprint (bytes) of a stage tile of TE elements, R chemistry
// chunks per Gauss point and up to O AT levels per face. In the FP64 variant the
// flux overwrites the nodal state and the summed rates stay in chunk 0; the
// mixed variant keeps both in separate FP32 arrays.
__host__ __device__ inline size_t stage_smem_bytes(int TE, int Q, int nv, int ns, int nr, int R,
                                                   int O, bool mix) {
  size_t TQ = (size_t)TE * Q, F = TE + 1;
  size_t nd = (size_t)SP_NFIELDS * ns      // species fields
              + 34                         // exp table and ln2/32 split
              + (size_t)nv * (TE + 2) * Q  // modal tile with halo        [v][le][j]
              + (size_t)nv * TQ            // nodal state (FP64: then flux) [v][t]
              + (size_t)ns * TQ * 2        // concentrations, g/RT        [i][t]
              + (size_t)R * ns * TQ        // production rates per chunk  [c][i][t]
              + 2 * TQ;                    // ln T, 1/T                   [t]
  size_t nr_ = F * nv                      // face fluxes                 [f][v]
               + (size_t)O * F * nv        // level fluxes                [m][f][v]
               + (size_t)O * F * 2 * nv;   // traces per (level, face)    [m][f][2][v]
  size_t extra = mix ? ((size_t)SP_NFIELDS * ns + (size_t)nv * TQ + (size_t)ns * TQ) : 0;
  size_t bytes = nd * 8 + (nr_ + extra) * (mix ? 4 : 8) + F * 4 + 16;
  return bytes + (size_t)nr * sizeof(Rxn);
}

// Copy an instance description into shared memory (by 8-byte words).
__device__ inline void load_inst(Inst &dst, const Inst *src) {
  const unsigned long long *a = reinterpret_cast<const unsigned long long *>(src);
  unsigned long long *b = reinterpret_cast<unsigned long long *>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(Inst) / 8); k += blockDim.x) b[k] = a[k];
}

template <int Q, bool MIX>
__global__ void __launch_bounds__(256) stage_kernel(Mech M, StageArgs A) {
  using DG = dg_t<MIX>;
  extern __shared__ __align__(16) double sm[];
  __shared__ Inst sI;
  const int2 tile = A.tiles[blockIdx.x];
  load_inst(sI, A.insts + tile.x);
  __syncthreads();
  const Inst &I = sI;
  const Basis &B = c_basis[Q - 2];
  const BasisF &BF = c_basis_f[Q - 2];
  const int nv = I.nv, ns = M.ns, nr = M.nr, N = I.n_elem, TE = A.TE;
  const int TQ = TE * Q;
  const int e0 = tile.y;
  const int te = min(TE, N - e0);
  const int64_t nstep = *I.step;
  const double *A_win = (A.s == 0) ? I.wn : (A.s == 1) ? I.wa : I.wb;
  double *A_wnext = (A.s == 0) ? I.wa : (A.s == 1) ? I.wb : I.wn;
  const bool periodic = (I.bc_left == ADG_BC_PERIODIC);
  const int R = A.R, O = A.O, NF = TE + 1;
  Rxn *srx = reinterpret_cast<Rxn *>(sm);
  double *ssp = reinterpret_cast<double *>(srx + nr);       // [F][ns]
  ExpTable *stab = reinterpret_cast<ExpTable *>(ssp + SP_NFIELDS * ns);
  double *sw = reinterpret_cast<double *>(stab + 1);        // [v][TE+2][Q]
  double *snw = sw + (size_t)nv * (TE + 2) * Q;             // [v][TQ]  nodal state
  double *sconc = snw + (size_t)nv * TQ;                    // [i][TQ]
  double *sg = sconc + (size_t)ns * TQ;                     // [i][TQ]
  double *swd = sg + (size_t)ns * TQ;                       // [R][i][TQ]
  double *slnT = swd + (size_t)R * ns * TQ;                 // [TQ]
  double *sinvT = slnT + TQ;                                // [TQ]
  DG *sfh = reinterpret_cast<DG *>(sinvT + TQ);             // [NF][nv]
  DG *sflx = sfh + (size_t)NF * nv;                         // [O][NF][nv]
  DG *str = sflx + (size_t)O * NF * nv;                     // [O][NF][2][nv]
  DG *sspD, *sfx, *swdD;                                    // species, flux, rates in DG
  if constexpr (MIX) {
    sspD = str + (size_t)O * NF * 2 * nv;
    sfx = sspD + (size_t)SP_NFIELDS * ns;
    swdD = sfx + (size_t)nv * TQ;
  } else {
    sspD = reinterpret_cast<DG *>(ssp);
    sfx = reinterpret_cast<DG *>(snw);
    swdD = reinterpret_cast<DG *>(swd);
  }
  int *sk = MIX ? reinterpret_cast<int *>(swdD + (size_t)ns * TQ)
                : reinterpret_cast<int *>(str + (size_t)O * NF * 2 * nv);   // [NF]
  const int tid = threadIdx.x, nth = blockDim.x;

  // 0. mechanism, species fields and exp table into shared memory
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(M.rx);
    uint4 *dst = reinterpret_cast<uint4 *>(srx);
    for (int k = tid; k < nr * (int)(sizeof(Rxn) / 16); k += nth) dst[k] = src[k];
    for (int k = tid; k < SP_NFIELDS * ns; k += nth) {
      double x = M.sp[k];
      ssp[k] = x;
      if constexpr (MIX) sspD[k] = (DG)x;
    }
    const double *et = reinterpret_cast<const double *>(&c_exp);
    double *dt = reinterpret_cast<double *>(stab);
    for (int k = tid; k < 34; k += nth) dt[k] = et[k];
  }
  // 1. tile of modal coefficients with a one-element halo on each side
  const int span = (te + 2) * Q;
  for (int idx = tid; idx < nv * span; idx += nth) {
    int v = idx / span, r = idx - v * span;
    int le = r / Q, j = r - le * Q;
    int e = e0 - 1 + le;
    if (e < 0) e = periodic ? e + N : 0;
    if (e >= N) e = periodic ? e - N : N - 1;
    sw[((size_t)v * (TE + 2) + le) * Q + j] = A_win[((size_t)v * N + e) * Q + j];
  }
  __syncthreads();

  // 2a. Gauss points: conserved state and temperature (FP64), concentrations,
  // g_i/(R T), and the flux
  const double *sIW = ssp + SP_INVW * ns;
  const double *sG0 = ssp + SP_G0 * ns, *sG1 = ssp + SP_G1 * ns, *sCR = ssp + SP_CPR * ns;
  const double LN_R_PATM = log(RU / PATM);
  const int teq = te * Q;
  for (int t = tid; t < teq; t += nth) {
    int e = t / Q, q = t - e * Q, le = e + 1;
    double *wq = snw + t;   // stride TQ between variables
    for (int v = 0; v < nv; ++v) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < Q; ++j) acc += sw[((size_t)v * (TE + 2) + le) * Q + j] * B.P[q][j];
      wq[(size_t)v * TQ] = acc;
    }
    Thermo th = thermo_of(ssp, ns, wq, TQ);
    if (!(th.rho > 0.0) || !(th.T > 0.0) || !isfinite(th.T) || !isfinite(wq[0]))
      report_error(I, ADG_ERR_NONPHYSICAL, e0 + e, A.s, nstep);
    const double lnT = log(th.T), invT = 1.0 / th.T;
    slnT[t] = lnT;
    sinvT[t] = invT;
    double *cq = sconc + t, *gq = sg + t;
    for (int i = 0; i < ns; ++i) {
      double r = wq[(size_t)(2 + i) * TQ];
      // law of mass action on non-negative concentrations: clip at zero by the
      // sign bit (no FP64 instruction)
      r = (__double2hiint(r) < 0) ? 0.0 : r;
      cq[(size_t)i * TQ] = r * sIW[i];
      gq[(size_t)i * TQ] = fma(-sCR[i], lnT, fma(sG0[i], invT, sG1[i]));
    }
    if constexpr (MIX) {
      const DG u = (DG)th.u, P = (DG)th.P;
      DG *fq = sfx + t;
      fq[0] = (DG)wq[0] * u + P;
      fq[TQ] = u * ((DG)wq[TQ] + P);
      for (int v = 2; v < nv; ++v) fq[(size_t)v * TQ] = u * (DG)wq[(size_t)v * TQ];
    } else {
      double f0 = phys_flux(wq, TQ, 0, th), f1 = phys_flux(wq, TQ, 1, th);
      for (int v = 2; v < nv; ++v) wq[(size_t)v * TQ] = th.u * wq[(size_t)v * TQ];
      wq[0] = f0;
      wq[TQ] = f1;
    }
  }
  __syncthreads();

  // 2b. chemistry (FP64), the reactions of every Gauss point split into R
  // chunks: reversible rates from the species' Gibbs energies, two exponentials
  for (int item = tid; item < R * teq; item += nth) {
    int c = item / teq, t = item - c * teq;
    const double lnT = slnT[t], invT = sinvT[t];
    const double *cq = sconc + t, *gq = sg + t;
    double *wd = swd + (size_t)c * ns * TQ + t;
    for (int i = 0; i < ns; ++i) wd[(size_t)i * TQ] = 0.0;
    const double lr = lnT + LN_R_PATM;
    const int j0 = c * nr / R, j1 = (c + 1) * nr / R;
    for (int j = j0; j < j1; ++j) {
      const Rxn &Rx = srx[j];
      double lkf = fma(-Rx.EaR, invT, fma(Rx.b, lnT, Rx.lnA));
      double dg = Rx.dnu * lr;
      const int nx = Rx.nx;
      for (int k = 0; k < nx; ++k) dg = fma(Rx.xc[k], gq[(size_t)Rx.xs[k] * TQ], dg);
      double fwd = fexp(lkf, *stab), rev = fexp(lkf + dg, *stab);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (Rx.rn[k] == 0) break;
        double cc = cq[(size_t)Rx.rs[k] * TQ];
        fwd *= cc;
        if (Rx.rn[k] > 1) fwd *= cc;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (Rx.pn[k] == 0) break;
        double cc = cq[(size_t)Rx.ps[k] * TQ];
        rev *= cc;
        if (Rx.pn[k] > 1) rev *= cc;
      }
      double qj = fwd - rev;
      for (int k = 0; k < nx; ++k)
        wd[(size_t)Rx.xs[k] * TQ] = fma(Rx.xc[k], qj, wd[(size_t)Rx.xs[k] * TQ]);
    }
  }
  __syncthreads();

  // 2c. sum of the chunks' rates (into chunk 0, or the FP32 copy)
  if (MIX || R > 1)
    for (int item = tid; item < ns * teq; item += nth) {
      int i = item / teq, t = item - i * teq;
      double acc = swd[(size_t)i * TQ + t];
      for (int c = 1; c < R; ++c) acc += swd[((size_t)c * ns + i) * TQ + t];
      if constexpr (MIX) swdD[(size_t)i * TQ + t] = (DG)acc;
      else swd[(size_t)i * TQ + t] = acc;
    }
  // 3a. face fluxes of the tile (local face f between local elements f and f+1),
  // one thread per (level, face): the plain flux, or one delayed level of the AT
  // flux (Eq. 7) with both sides at the common level n-k-m
  for (int job = tid; job < O * (te + 1); job += nth) {
    int m = job / (te + 1), f = job - m * (te + 1);
    int g = e0 + f;  // global face index
    int pf = (g < N) ? I.pf_of_left[g] : I.pf_of_right[N - 1];
    int k = (pf >= 0) ? effective_delay(I, nstep, pf) : 0;
    if (m == 0) sk[f] = k;
    DG *fl = sflx + ((size_t)m * NF + f) * nv;
    DG *wl = str + ((size_t)m * NF + f) * 2 * nv, *wr = wl + nv;
    if (k > 0) {
      if (m >= I.at_order) continue;
      int64_t lv = nstep - k - m;
      const double *bl = I.ring_in + ring_trace(I, lv, A.s, pf, 0);
      const double *br = I.ring_in + ring_trace(I, lv, A.s, pf, 1);
      if constexpr (MIX) {
        for (int v = 0; v < nv; ++v) {
          wl[v] = (DG)bl[v];
          wr[v] = (DG)br[v];
        }
        num_flux_t<DG>(sspD, ns, I.flux, wl, wr, fl);
      } else {
        num_flux_t<double>(ssp, ns, I.flux, bl, br, fl);
      }
      continue;
    }
    if (m > 0) continue;
    for (int v = 0; v < nv; ++v) {
      double a = 0.0, b = 0.0;
      for (int j = 0; j < Q; ++j) {
        a += sw[((size_t)v * (TE + 2) + f) * Q + j];
        b += ((j & 1) ? -1.0 : 1.0) * sw[((size_t)v * (TE + 2) + f + 1) * Q + j];
      }
      wl[v] = (DG)a;
      wr[v] = (DG)b;
    }
    if (!periodic && g == 0) {
      for (int v = 0; v < nv; ++v) wl[v] = wr[v];
      if (I.bc_left == ADG_BC_REFLECT) wl[0] = -wr[0];
    } else if (!periodic && g == N) {
      for (int v = 0; v < nv; ++v) wr[v] = wl[v];
      if (I.bc_right == ADG_BC_REFLECT) wr[0] = -wl[0];
    }
    num_flux_t<DG>(sspD, ns, I.flux, wl, wr, fl);
  }
  __syncthreads();
  // 3b. the AT sum over levels, m = 0..o-1 in order, in FP64
  for (int item = tid; item < (te + 1) * nv; item += nth) {
    int f = item / nv, v = item - f * nv;
    int k = sk[f];
    double acc = (double)sflx[(size_t)f * nv + v];
    if (k > 0) {
      acc *= I.at[k][0];
      for (int m = 1; m < I.at_order; ++m)
        acc = fma(I.at[k][m], (double)sflx[((size_t)m * NF + f) * nv + v], acc);
    }
    sfh[(size_t)f * nv + v] = (DG)acc;
  }
  __syncthreads();

  // 4. assembly of Eq. (5) (in DG arithmetic) and the SSP-RK3 combination (FP64);
  // history ring writes
  const int slot_ok = (I.npf > 0);
  const double inv_dx = 1.0 / I.dx;
  const double *sW = ssp + SP_W * ns;
  for (int item = tid; item < nv * te; item += nth) {
    int v = item / te, e = item - v * te, ge = e0 + e, le = e + 1;
    const double *wi = sw + ((size_t)v * (TE + 2) + le) * Q;
    const DG *fq = sfx + (size_t)v * TQ + e * Q;
    const DG *sq = (v >= 2) ? swdD + (size_t)(v - 2) * TQ + e * Q : nullptr;
    const DG Wv = (v >= 2) ? (DG)sW[v - 2] : DG(0);
    const DG fr = sfh[(size_t)(e + 1) * nv + v], fl = sfh[(size_t)e * nv + v];
    DG fqr[Q], sqr[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      fqr[q] = fq[q];
      sqr[q] = (v >= 2) ? sq[q] : DG(0);
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
      double r = (double)fma((DG)((2.0 * i + 1.0) * inv_dx), surf, Wv * S);
      size_t gi = ((size_t)v * N + ge) * Q + i;
      double o;
      if (A.s == 0) o = fma(I.dt, r, I.wn[gi]);
      else if (A.s == 1) o = fma(0.25, fma(I.dt, r, wi[i]), 0.75 * I.wn[gi]);
      else o = fma(2.0 / 3.0, fma(I.dt, r, wi[i]), (1.0 / 3.0) * I.wn[gi]);
      out[i] = o;
      I.wpre[gi] = o;
      A_wnext[gi] = o;
    }
    if (slot_ok) {
      int pr = I.pf_of_right[ge], pl = I.pf_of_left[ge];
      if (pr >= 0) {
        // left element of the PE face: its trace at xi = +1
        size_t b = ring_block(I, nstep, A.s, pr, 0) + (size_t)v * Q;
        double tr = 0.0;
        for (int i = 0; i < Q; ++i) {
          tr += wi[i];
          I.ring_pre[b + i] = out[i];
        }
        I.ring_in[ring_trace(I, nstep, A.s, pr, 0) + v] = tr;
      }
      if (pl >= 0) {
        // right element of the PE face: its trace at xi = -1
        size_t b = ring_block(I, nstep, A.s, pl, 1) + (size_t)v * Q;
        double tr = 0.0;
        for (int i = 0; i < Q; ++i) {
          tr += ((i & 1) ? -1.0 : 1.0) * wi[i];
          I.ring_pre[b + i] = out[i];
        }
        I.ring_in[ring_trace(I, nstep, A.s, pl, 1) + v] = tr;
      }
    }
  }
}

template <typename R>
__device__ inline R minmod3(R a, R b, R c) {
  if (a > R(0) && b > R(0) && c > R(0)) return fmin(a, fmin(b, c));
  if (a < R(0) && b < R(0) && c < R(0)) return fmax(a, fmax(b, c));
  return R(0);
}

// Shared memory (words of the arithmetic type) per element of the limiter: the
// element and its two neighbours, the limited characteristic modes, gradP.w, the
// partial-density sums and momenta of the three blocks, phi_k, two mode sums and
// the mode sums of block 0.
__host__ __device__ inline int limiter_elem_words(int nv, int ns, int Q) {
  return 3 * nv * Q + nv * Q + 3 * 3 * Q + ns + 2 * Q + 8;
}
constexpr int LIM_WARPS = 8;

// Troubled-cell indicator and (AT-)WENO limiter (Sec. 3.3, Eq. 9-11), a group of
// G lanes per element (G = 16 when nv <= 16, else 32), in the arithmetic type of
// the precision variant.
// Eigen-structure of the frozen Jacobian at the cell average: right vectors
// r_-/+ = (u -/+ a, H -/+ u a, Y), species r_k = (u, u^2 - phi_k/g, e_k); left
// vectors l_-/+ = (gradP -/+ a (1, 0, -u..-u)) / (2 a^2), l_k = e_k - Y_k gradP/a^2,
// gradP = (-u g, g, phi_1..phi_ns), g = gamma - 1, phi_k = g (u^2/2 - e_k) + R T / W_k.
// Every characteristic value is written in one branch-free form,
// v = A gradP.w + B (rho u)_w + C (sum rho Y)_w + D (rho Y_k)_w,
// with (A, B, C, D) = (1/2a^2, -/+ a/2a^2, +/- a u/2a^2, 0) for the acoustic fields
// and (-Y_k/a^2, 0, 0, 1) for species k, so that all lanes run the same code.
template <int Q, int G, bool MIX>
__global__ void __launch_bounds__(32 * LIM_WARPS) limiter_kernel(Mech M, LimArgs A) {
  using DG = dg_t<MIX>;
  extern __shared__ __align__(16) double lsm_raw[];
  DG *lsm = reinterpret_cast<DG *>(lsm_raw);
  __shared__ Inst sI;
  const int2 blkid = A.blocks[blockIdx.x];
  load_inst(sI, A.insts + blkid.x);
  __syncthreads();
  const Inst &I = sI;
  if (I.limiter == ADG_LIM_NONE) return;
  const Basis &B = c_basis[Q - 2];
  const BasisF &BF = c_basis_f[Q - 2];
  const int N = I.n_elem, nv = I.nv, ns = M.ns;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane % G, gw = lane / G;
  constexpr int EPW = 32 / G;
  const int slot = warp * EPW + gw;
  const int e = blkid.y + slot;
  const bool valid = e < N;
  const int64_t nstep = *I.step;
  double *A_wout = (A.s == 0) ? I.wa : (A.s == 1) ? I.wb : I.wn;
  const double *A_wpre = I.wpre;
  const unsigned FULL = 0xffffffffu;
  const unsigned gmask = (G == 32) ? FULL : (0xffffu << (16 * gw));
  const size_t VS = (size_t)N * Q;
  const int NB = nv * Q;
  DG *blk = lsm + (size_t)slot * limiter_elem_words(nv, ns, Q);  // [3][nv][Q]
  DG *vlim = blk + 3 * NB;                                        // [nv][Q]
  DG *gpv = vlim + NB;                                            // [3][Q]
  DG *rsv = gpv + 3 * Q;                                          // [3][Q]
  DG *mmv = rsv + 3 * Q;                                          // [3][Q]
  DG *phi = mmv + 3 * Q;                                          // [ns]
  DG *sums = phi + ns;                                            // [2][Q]
  DG *ssum = sums + 2 * Q;   // mode sums of block 0: gp, mm, rs (plain, alternating)
  const bool periodic = (I.bc_left == ADG_BC_PERIODIC);

  // 1. the element (block 0) and its neighbours (1 left, 2 right): the pre-limit
  //    field, the AT extrapolation of the neighbour's pre-limit history across a
  //    delayed PE face (Eq. 11, summed in FP64), or a boundary ghost
  if (valid) {
    for (int d = 0; d < 3; ++d) {
      DG *dst = blk + d * NB;
      int src = e, ghost = 0, k = 0, pf = -1;
      if (d > 0) {
        pf = d == 1 ? I.pf_of_left[e] : I.pf_of_right[e];
        k = (pf >= 0) ? effective_delay(I, nstep, pf) : 0;
        src = d == 1 ? e - 1 : e + 1;
        if (src < 0 || src >= N) {
          if (periodic) {
            src = (src + N) % N;
          } else {
            src = e;
            ghost = ((d == 1 ? I.bc_left : I.bc_right) == ADG_BC_REFLECT) ? 1 : 0;
          }
        }
      }
      if (k > 0) {
        int side = d == 1 ? 0 : 1;
        for (int t = gl; t < NB; t += G) {
          double acc = 0.0;
          for (int m = 0; m < I.at_order; ++m)
            acc += I.at[k][m] * I.ring_pre[ring_block(I, nstep - k - m, A.s, pf, side) + t];
          dst[t] = (DG)acc;
        }
      } else {
        for (int t = gl; t < NB; t += G) {
          int v = t / Q, j = t - v * Q;
          double x = A_wpre[(size_t)v * VS + (size_t)src * Q + j];
          if (ghost && (((j & 1) != 0) != (v == 0))) x = -x;
          dst[t] = (DG)x;
        }
      }
    }
  }
  __syncwarp();

  // 2. cell average: thermo and eigen-quantities (species sums split over lanes)
  const double *qWd = M.sp + SP_QW * ns, *cvWd = M.sp + SP_CVW * ns;
  const double *RWd = M.sp + SP_RW * ns, *cpWd = M.sp + SP_CPW * ns;
  DG rho = 0, qsum = 0, cv = 0, Rm = 0, cpm = 0;
  if (valid)
    for (int i = gl; i < ns; i += G) {
      DG r = blk[(2 + i) * Q];
      rho += r;
      qsum = fma(r, (DG)qWd[i], qsum);
      cv = fma(r, (DG)cvWd[i], cv);
      Rm = fma(r, (DG)RWd[i], Rm);
      cpm = fma(r, (DG)cpWd[i], cpm);
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
  if (valid && gl == 0 && (!(rho > DG(0)) || !(T > DG(0)) || !isfinite(T)))
    report_error(I, ADG_ERR_NONPHYSICAL, e, A.s, nstep);
  // phi_k, and the sums of |phi_i|, |phi_i - a u|, |phi_i + a u| for the noise floor
  DG sphi = 0, sphm = 0, sphp = 0;
  if (valid) {
    for (int i = gl; i < ns; i += G) {
      DG ph = fma(g, fma(-(DG)cvWd[i], T, DG(0.5) * u * u - (DG)qWd[i]), T * (DG)RWd[i]);
      phi[i] = ph;
      sphi += fabs(ph);
      sphm += fabs(ph - a * u);
      sphp += fabs(ph + a * u);
    }
  }
  for (int o = G / 2; o > 0; o >>= 1) {
    sphi += __shfl_xor_sync(FULL, sphi, o, G);
    sphm += __shfl_xor_sync(FULL, sphm, o, G);
    sphp += __shfl_xor_sync(FULL, sphp, o, G);
  }
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
  if (valid && gl < 6) {
    const DG *src = (gl % 3 == 0) ? gpv : (gl % 3 == 1) ? mmv : rsv;
    DG acc = 0;
    for (int j = 0; j < Q; ++j) acc += (gl >= 3 && (j & 1)) ? -src[j] : src[j];
    ssum[gl] = acc;
  }
  __syncwarp();

  // coefficients of field k and its value for block b, mode j
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

  // 3. indicator: the lanes of a group test the fields
  const DG sig0 = fma(rho, a, fabs(m0)), sig1 = fabs(E0), sigr = rho;
  // noise floor 1e-5 of the field's magnitude in both precisions: above the
  // single-precision rounding, so both variants select the same troubled cells
  const DG tvb = (DG)I.tvb, tau = DG(1e-5);
  bool mine = false;
  if (valid)
    for (int k = gl; k < nv; k += G) {
      DG cA, cB, cC, cD;
      int ri;
      coef(k, cA, cB, cC, cD, ri);
      // the face values v(+1), v(-1) from the mode sums (linear in the modes)
      const DG *rk = blk + (2 + ri) * Q;
      DG rsum = 0, ralt = 0;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        rsum += rk[j];
        ralt += (j & 1) ? -rk[j] : rk[j];
      }
      DG vb = val(cA, cB, cC, cD, ri, 0, 0);
      DG vp = fma(cA, ssum[0], fma(cB, ssum[1], fma(cC, ssum[2], cD * rsum)));
      DG vm = fma(cA, ssum[3], fma(cB, ssum[4], fma(cC, ssum[5], cD * ralt)));
      DG vL = val(cA, cB, cC, cD, ri, 1, 0), vR = val(cA, cB, cC, cD, ri, 2, 0);
      // sum_v |L_kv| sigma_v in closed form: for species k, |1 + A phi_k| plus
      // |A| (sum |phi| - |phi_k|); for the acoustic fields A sum |phi_i -/+ a u|
      bool ac = (k == 0) || (k == nv - 1);
      DG srr = ac ? cA * (k == 0 ? sphp : sphm)
                  : fabs(fma(cA, phi[ri], DG(1))) + fabs(cA) * (sphi - fabs(phi[ri]));
      DG scale = fma(fabs(fma(cA, -u * g, cB)), sig0, fma(fabs(cA * g), sig1, srr * sigr));
      DG ut = vp - vb, utt = vb - vm, dp = vR - vb, dm = vb - vL;
      DG fl = tau * scale;
      if (fabs(ut) > fl && fabs(ut) > tvb && minmod3(ut, dp, dm) != ut) mine = true;
      if (fabs(utt) > fl && fabs(utt) > tvb && minmod3(utt, dp, dm) != utt) mine = true;
    }
  unsigned bal = __ballot_sync(FULL, mine) & gmask;
  const bool troubled = valid && bal != 0u && I.limiter != ADG_LIM_NONE;
  if (valid && gl == 0) {
    I.flags[(size_t)A.s * N + e] = troubled ? 1 : 0;
    if (troubled) I.count[e] += 1;
  }
  if (!troubled) return;

  // 4. WENO (Eq. 9-10) per characteristic field, the group's lanes over fields
  const DG gmw[3] = {DG(0.001), DG(0.998), DG(0.001)};
  const DG eps = DG(1e-6);
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
  __syncwarp(gmask);
  // 5. back to conserved variables with R (modes >= 1; the cell average is kept)
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
  __syncwarp(gmask);
  double *out = A_wout + (size_t)e * Q;
  for (int t = gl; t < NB; t += G) {
    int v = t / Q, i = t - v * Q;
    if (i == 0) continue;
    DG lm = vlim[i], lp = vlim[(nv - 1) * Q + i];
    DG o;
    if (v == 0) o = lm * (u - a) + lp * (u + a) + u * sums[i];
    else if (v == 1) o = lm * (H - u * a) + lp * (H + u * a) + sums[Q + i];
    else o = (lm + lp) * (blk[v * Q] * irho) + vlim[(v - 1) * Q + i];
    out[(size_t)v * VS + i] = (double)o;
  }
}

// L2 projection of primitive values at the Gauss points (Sec. 3.1): one thread
// per (element, variable); prim layout [ns+3][N][Q] (T, P, u, Y_i).
template <int Q>
__global__ void project_kernel(Mech M, Inst I, const double *prim, double *w) {
  const Basis &B = c_basis[Q - 2];
  const int N = I.n_elem, ns = M.ns, nv = I.nv;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * nv) return;
  int v = idx / N, e = idx - v * N;
  double val[Q];
  for (int q = 0; q < Q; ++q) {
    double T = prim[(size_t)e * Q + q];
    double P = prim[((size_t)N + e) * Q + q];
    double u = prim[((size_t)2 * N + e) * Q + q];
    double sYW = 0.0, ey = 0.0;
    for (int i = 0; i < ns; ++i) {
      double Y = prim[((size_t)(3 + i) * N + e) * Q + q];
      sYW += Y * M.sp[SP_INVW * ns + i];
      ey += Y * (M.sp[SP_QW * ns + i] + M.sp[SP_CVW * ns + i] * T);
    }
    double rho = P / (RU * T * sYW);
    if (v == 0) val[q] = rho * u;
    else if (v == 1) val[q] = rho * (ey + 0.5 * u * u);
    else val[q] = rho * prim[((size_t)(1 + v) * N + e) * Q + q];
  }
  for (int j = 0; j < Q; ++j) {
    double acc = 0.0;
    for (int q = 0; q < Q; ++q) acc += B.w[q] * val[q] * B.P[q][j];
    w[((size_t)v * N + e) * Q + j] = 0.5 * (2.0 * j + 1.0) * acc;
  }
}

template <int Q>
__global__ void temperature_kernel(Mech M, Inst I, const double *w, double *T) {
  const Basis &B = c_basis[Q - 2];
  const int N = I.n_elem, nv = I.nv;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * Q) return;
  int e = t / Q, q = t - e * Q;
  double wq[ADG_MAX_SPECIES + 2];
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int j = 0; j < Q; ++j) acc += w[((size_t)v * N + e) * Q + j] * B.P[q][j];
    wq[v] = acc;
  }
  T[t] = thermo_of(M.sp, M.ns, wq, 1).T;
}

// ---------------------------------------------------------------------------
// host-side launchers

cudaError_t upload_basis(const Basis *tables) {
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

int stage_tile(int Q, int nv, int ns, int nr, int R, int O, bool mixed) {
  // elements per tile: up to 256 Gauss-point threads, at most ~96 KB of tile
  int TE = 256 / Q;
  while (TE > 2 && stage_smem_bytes(TE, Q, nv, ns, nr, R, O, mixed) > 96 * 1024) TE /= 2;
  return TE;
}

int stage_chunks(int TE, int Q, int nr) {
  // chemistry chunks per Gauss point that best fill the CTA's threads
  int TQ = TE * Q, nth = ((TQ + 31) / 32) * 32;
  int best = 1;
  double best_fill = 0.0;
  for (int R = 1; R <= 8 && R <= (nr > 0 ? nr : 1); ++R) {
    int items = TQ * R;
    int rounds = (items + nth - 1) / nth;
    double fill = (double)items / (rounds * nth);
    if (fill > best_fill + 0.02) {
      best_fill = fill;
      best = R;
    }
  }
  return best;
}

size_t stage_smem(int TE, int Q, int nv, int ns, int nr, int R, int O, bool mixed) {
  return stage_smem_bytes(TE, Q, nv, ns, nr, R, O, mixed);
}

cudaError_t upload_exp_table(const ExpTable *t) {
  return cudaMemcpyToSymbol(c_exp, t, sizeof(ExpTable));
}

template <int Q, bool MIX>
static cudaError_t launch_stage_qm(const Mech &M, const StageArgs &A, int n_tiles,
                                   cudaStream_t st) {
  int nv = M.ns + 2;
  size_t smem = stage_smem_bytes(A.TE, Q, nv, M.ns, M.nr, A.R, A.O, MIX);
  int nth = ((A.TE * Q + 31) / 32) * 32;
  stage_kernel<Q, MIX><<<n_tiles, nth, smem, st>>>(M, A);
  return cudaGetLastError();
}

cudaError_t launch_stage(const Mech &M, const StageArgs &A, int Q, bool mixed, int n_tiles,
                         cudaStream_t st) {
  switch (Q * 2 + (mixed ? 1 : 0)) {
    case 4: return launch_stage_qm<2, false>(M, A, n_tiles, st);
    case 5: return launch_stage_qm<2, true>(M, A, n_tiles, st);
    case 6: return launch_stage_qm<3, false>(M, A, n_tiles, st);
    case 7: return launch_stage_qm<3, true>(M, A, n_tiles, st);
    case 8: return launch_stage_qm<4, false>(M, A, n_tiles, st);
    case 9: return launch_stage_qm<4, true>(M, A, n_tiles, st);
    case 10: return launch_stage_qm<5, false>(M, A, n_tiles, st);
    case 11: return launch_stage_qm<5, true>(M, A, n_tiles, st);
  }
  return cudaErrorInvalidValue;
}

int limiter_elems_per_block(int nv) { return LIM_WARPS * (nv <= 16 ? 2 : 1); }

template <int Q, int G, bool MIX>
static cudaError_t launch_limiter_qgm(const Mech &M, const LimArgs &A, int nv, int n_blocks,
                                      cudaStream_t st) {
  constexpr int EPW = 32 / G;
  size_t smem = (size_t)LIM_WARPS * EPW * limiter_elem_words(nv, M.ns, Q) *
                (MIX ? sizeof(float) : sizeof(double));
  smem = (smem + 15) & ~(size_t)15;
  limiter_kernel<Q, G, MIX><<<n_blocks, 32 * LIM_WARPS, smem, st>>>(M, A);
  return cudaGetLastError();
}

template <int Q, bool MIX>
static cudaError_t launch_limiter_qm(const Mech &M, const LimArgs &A, int nv, int n_blocks,
                                     cudaStream_t st) {
  if (nv <= 16) return launch_limiter_qgm<Q, 16, MIX>(M, A, nv, n_blocks, st);
  return launch_limiter_qgm<Q, 32, MIX>(M, A, nv, n_blocks, st);
}

cudaError_t launch_limiter(const Mech &M, const LimArgs &A, int Q, bool mixed, int nv,
                           int n_blocks, cudaStream_t st) {
  switch (Q * 2 + (mixed ? 1 : 0)) {
    case 4: return launch_limiter_qm<2, false>(M, A, nv, n_blocks, st);
    case 5: return launch_limiter_qm<2, true>(M, A, nv, n_blocks, st);
    case 6: return launch_limiter_qm<3, false>(M, A, nv, n_blocks, st);
    case 7: return launch_limiter_qm<3, true>(M, A, nv, n_blocks, st);
    case 8: return launch_limiter_qm<4, false>(M, A, nv, n_blocks, st);
    case 9: return launch_limiter_qm<4, true>(M, A, nv, n_blocks, st);
    case 10: return launch_limiter_qm<5, false>(M, A, nv, n_blocks, st);
    case 11: return launch_limiter_qm<5, true>(M, A, nv, n_blocks, st);
  }
  return cudaErrorInvalidValue;
}

// Raise the dynamic shared-memory limit of every kernel instance (before any
// launch or stream capture).
cudaError_t prepare_kernels(int nv, int ns, int nr) {
  (void)nv;
  (void)ns;
  (void)nr;
  const int lim = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define SET(...) \
  if (e == cudaSuccess)     \
  e = cudaFuncSetAttribute(__VA_ARGS__, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
  SET(stage_kernel<2, false>);
  SET(stage_kernel<3, false>);
  SET(stage_kernel<4, false>);
  SET(stage_kernel<5, false>);
  SET(stage_kernel<2, true>);
  SET(stage_kernel<3, true>);
  SET(stage_kernel<4, true>);
  SET(stage_kernel<5, true>);
  SET(limiter_kernel<2, 16, false>);
  SET(limiter_kernel<3, 16, false>);
  SET(limiter_kernel<4, 16, false>);
  SET(limiter_kernel<5, 16, false>);
  SET(limiter_kernel<2, 32, false>);
  SET(limiter_kernel<3, 32, false>);
  SET(limiter_kernel<4, 32, false>);
  SET(limiter_kernel<5, 32, false>);
  SET(limiter_kernel<2, 16, true>);
  SET(limiter_kernel<3, 16, true>);
  SET(limiter_kernel<4, 16, true>);
  SET(limiter_kernel<5, 16, true>);
  SET(limiter_kernel<2, 32, true>);
  SET(limiter_kernel<3, 32, true>);
  SET(limiter_kernel<4, 32, true>);
  SET(limiter_kernel<5, 32, true>);
#undef SET
  return e;
}

__global__ void advance_kernel(int64_t *steps, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) steps[i] += 1;
}

cudaError_t launch_advance(int64_t *steps, int n, cudaStream_t st) {
  advance_kernel<<<(n + 127) / 128, 128, 0, st>>>(steps, n);
  return cudaGetLastError();
}

cudaError_t launch_project(const Mech &M, const Inst &I, const double *prim, double *w,
                           cudaStream_t st) {
  int n = I.n_elem * I.nv;
  int nblk = (n + 127) / 128;
  switch (I.p + 1) {
    case 2: project_kernel<2><<<nblk, 128, 0, st>>>(M, I, prim, w); break;
    case 3: project_kernel<3><<<nblk, 128, 0, st>>>(M, I, prim, w); break;
    case 4: project_kernel<4><<<nblk, 128, 0, st>>>(M, I, prim, w); break;
    case 5: project_kernel<5><<<nblk, 128, 0, st>>>(M, I, prim, w); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_temperature(const Mech &M, const Inst &I, const double *w, double *T,
                               cudaStream_t st) {
  int n = I.n_elem * (I.p + 1);
  int nblk = (n + 127) / 128;
  switch (I.p + 1) {
    case 2: temperature_kernel<2><<<nblk, 128, 0, st>>>(M, I, w, T); break;
    case 3: temperature_kernel<3><<<nblk, 128, 0, st>>>(M, I, w, T); break;
    case 4: temperature_kernel<4><<<nblk, 128, 0, st>>>(M, I, w, T); break;
    case 5: temperature_kernel<5><<<nblk, 128, 0, st>>>(M, I, w, T); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace adg
