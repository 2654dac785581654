// CUDA kernels of the ADG hot path (sm_103a), FP64.
//
// Per RK stage two kernels run:
//   stage_kernel<Q>  : one CTA per tile of TE consecutive elements. Loads the tile
//                      plus a one-element halo into shared memory (coalesced per
//                      variable), evaluates every Gauss point (thermo, flux,
//                      chemistry) with one thread per point, computes the TE+1 face
//                      fluxes of the tile (AT flux at delayed PE faces), assembles
//                      Eq. (5) and the SSP-RK3 combination, writes the pre-limit
//                      stage output and the history ring of PE-boundary elements.
//   limiter_kernel<Q>: 16 or 32 lanes per element: troubled-cell indicator in the
//                      characteristic fields of the cell average and, on troubled
//                      cells, the (AT-)WENO reconstruction of Eq. (9)-(11). The
//                      stage kernel writes the pre-limit output twice (limiter
//                      input and next-stage buffer) so that the limiter only
//                      rewrites troubled cells.
#include <cstdio>

#include "adg_internal.cuh"
#include "adg_math.cuh"

namespace adg {

__constant__ Basis c_basis[ADG_MAX_P];   // index p-1

__constant__ ExpTable c_exp;

// Shared-memory footprint (bytes) of a stage tile of TE elements.
__host__ __device__ inline size_t stage_smem_bytes(int TE, int Q, int nv, int ns, int nr) {
  size_t n = (size_t)SP_NFIELDS * ns      // species fields
             + 34                         // exp table and ln2/32 split
             + (size_t)nv * (TE + 2) * Q  // modal tile with halo    [v][le][j]
             + (size_t)nv * TE * Q        // nodal state, then flux  [v][t]
             + (size_t)ns * TE * Q * 3    // conc, g/RT, rates        [i][t]
             + (size_t)(TE + 1) * nv      // face fluxes             [f][v]
             + (size_t)(TE + 1) * 2 * nv; // face traces             [f][2][v]
  return n * sizeof(double) + (size_t)nr * sizeof(Rxn);
}

template <int Q>
__global__ void __launch_bounds__(256) stage_kernel(Mech M, Inst I, StageArgs A) {
  extern __shared__ __align__(16) double sm[];
  const Basis &B = c_basis[Q - 2];
  const int nv = I.nv, ns = M.ns, nr = M.nr, N = I.n_elem, TE = A.TE;
  const int TQ = TE * Q;
  const int e0 = blockIdx.x * TE;
  const int te = min(TE, N - e0);
  const bool periodic = (I.bc_left == ADG_BC_PERIODIC);
  Rxn *srx = reinterpret_cast<Rxn *>(sm);
  double *ssp = reinterpret_cast<double *>(srx + nr);       // [F][ns]
  ExpTable *stab = reinterpret_cast<ExpTable *>(ssp + SP_NFIELDS * ns);
  double *sw = reinterpret_cast<double *>(stab + 1);        // [v][TE+2][Q]
  double *snode = sw + (size_t)nv * (TE + 2) * Q;           // [v][TQ]
  double *sconc = snode + (size_t)nv * TQ;                  // [i][TQ]
  double *sg = sconc + (size_t)ns * TQ;                     // [i][TQ]
  double *swd = sg + (size_t)ns * TQ;                       // [i][TQ]
  double *sfh = swd + (size_t)ns * TQ;                      // [TE+1][nv]
  double *str = sfh + (size_t)(TE + 1) * nv;                // [TE+1][2][nv]
  const int tid = threadIdx.x, nth = blockDim.x;

  // 0. mechanism, species fields and exp table into shared memory
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(M.rx);
    uint4 *dst = reinterpret_cast<uint4 *>(srx);
    for (int k = tid; k < nr * (int)(sizeof(Rxn) / 16); k += nth) dst[k] = src[k];
    for (int k = tid; k < SP_NFIELDS * ns; k += nth) ssp[k] = M.sp[k];
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
    sw[((size_t)v * (TE + 2) + le) * Q + j] = A.win[((size_t)v * N + e) * Q + j];
  }
  __syncthreads();

  // 2. Gauss points: conserved state, thermo, chemistry, flux
  const double *sW = ssp + SP_W * ns, *sIW = ssp + SP_INVW * ns;
  const double *sG0 = ssp + SP_G0 * ns, *sG1 = ssp + SP_G1 * ns, *sCR = ssp + SP_CPR * ns;
  const double LN_R_PATM = log(RU / PATM);
  for (int t = tid; t < te * Q; t += nth) {
    int e = t / Q, q = t - e * Q, le = e + 1;
    double *wq = snode + t;   // stride TQ between variables
    for (int v = 0; v < nv; ++v) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < Q; ++j) acc += sw[((size_t)v * (TE + 2) + le) * Q + j] * B.P[q][j];
      wq[(size_t)v * TQ] = acc;
    }
    Thermo th = thermo_of(ssp, ns, wq, TQ);
    if (!(th.rho > 0.0) || !(th.T > 0.0) || !isfinite(th.T) || !isfinite(wq[0]))
      report_error(I, ADG_ERR_NONPHYSICAL, e0 + e, A.s, A.n);
    // chemistry: law of mass action on non-negative concentrations, reversible
    // rates from the species' Gibbs energies (2 exponentials per reaction)
    const double lnT = log(th.T), invT = 1.0 / th.T;
    double *cq = sconc + t, *gq = sg + t, *wd = swd + t;
    for (int i = 0; i < ns; ++i) {
      double r = wq[(size_t)(2 + i) * TQ];
      // clip at zero by the sign bit (no FP64 instruction)
      r = (__double2hiint(r) < 0) ? 0.0 : r;
      cq[(size_t)i * TQ] = r * sIW[i];
      gq[(size_t)i * TQ] = fma(-sCR[i], lnT, fma(sG0[i], invT, sG1[i]));
      wd[(size_t)i * TQ] = 0.0;
    }
    const double lr = lnT + LN_R_PATM;
    for (int j = 0; j < nr; ++j) {
      const Rxn &R = srx[j];
      double lkf = fma(-R.EaR, invT, fma(R.b, lnT, R.lnA));
      double dg = R.dnu * lr;
      const int nx = R.nx;
      for (int k = 0; k < nx; ++k) dg = fma(R.xc[k], gq[(size_t)R.xs[k] * TQ], dg);
      double fwd = fexp(lkf, *stab), rev = fexp(lkf + dg, *stab);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (R.rn[k] == 0) break;
        double c = cq[(size_t)R.rs[k] * TQ];
        fwd *= c;
        if (R.rn[k] > 1) fwd *= c;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (R.pn[k] == 0) break;
        double c = cq[(size_t)R.ps[k] * TQ];
        rev *= c;
        if (R.pn[k] > 1) rev *= c;
      }
      double qj = fwd - rev;
      for (int k = 0; k < nx; ++k)
        wd[(size_t)R.xs[k] * TQ] = fma(R.xc[k], qj, wd[(size_t)R.xs[k] * TQ]);
    }
    double f0 = phys_flux(wq, TQ, 0, th), f1 = phys_flux(wq, TQ, 1, th);
    for (int v = 2; v < nv; ++v) wq[(size_t)v * TQ] = th.u * wq[(size_t)v * TQ];
    wq[0] = f0;
    wq[TQ] = f1;
  }

  // 3. face fluxes of the tile: local face f sits between local elements f and f+1
  for (int f = tid; f <= te; f += nth) {
    int g = e0 + f;  // global face index
    double *fh = sfh + (size_t)f * nv;
    double *wl = str + (size_t)f * 2 * nv, *wr = wl + nv;
    int pf = (g < N) ? I.pf_of_left[g] : I.pf_of_right[N - 1];
    int k = (pf >= 0) ? effective_delay(I, A.n, pf) : 0;
    if (k > 0) {
      // AT flux (Eq. 7): both sides at the common delayed levels n-k-m
      for (int mm = 0; mm < I.at_order; ++mm) {
        int64_t lv = A.n - k - mm;
        const double *bl = I.ring_in + ring_block(I, lv, A.s, pf, 0);
        const double *br = I.ring_in + ring_block(I, lv, A.s, pf, 1);
        for (int v = 0; v < nv; ++v) {
          double a = 0.0, b = 0.0;
          for (int j = 0; j < Q; ++j) {
            a += bl[v * Q + j];
            b += ((j & 1) ? -1.0 : 1.0) * br[v * Q + j];
          }
          wl[v] = a;
          wr[v] = b;
        }
        num_flux(ssp, ns, I.flux, wl, wr, fh, I.at[k][mm], mm > 0);
        if (mm == 0)
          for (int v = 0; v < nv; ++v) fh[v] *= I.at[k][0];
      }
      continue;
    }
    for (int v = 0; v < nv; ++v) {
      double a = 0.0, b = 0.0;
      for (int j = 0; j < Q; ++j) {
        a += sw[((size_t)v * (TE + 2) + f) * Q + j];
        b += ((j & 1) ? -1.0 : 1.0) * sw[((size_t)v * (TE + 2) + f + 1) * Q + j];
      }
      wl[v] = a;
      wr[v] = b;
    }
    if (!periodic && g == 0) {
      for (int v = 0; v < nv; ++v) wl[v] = wr[v];
      if (I.bc_left == ADG_BC_REFLECT) wl[0] = -wr[0];
    } else if (!periodic && g == N) {
      for (int v = 0; v < nv; ++v) wr[v] = wl[v];
      if (I.bc_right == ADG_BC_REFLECT) wr[0] = -wl[0];
    }
    num_flux(ssp, ns, I.flux, wl, wr, fh, 1.0, false);
  }
  __syncthreads();

  // 4. assembly of Eq. (5) and the SSP-RK3 combination; history ring writes
  const int slot_ok = (I.npf > 0);
  const double inv_dx = 1.0 / I.dx;
  for (int item = tid; item < nv * te; item += nth) {
    int v = item / te, e = item - v * te, ge = e0 + e, le = e + 1;
    const double *wi = sw + ((size_t)v * (TE + 2) + le) * Q;
    const double *fq = snode + (size_t)v * TQ + e * Q;
    const double *sq = (v >= 2) ? swd + (size_t)(v - 2) * TQ + e * Q : nullptr;
    const double Wv = (v >= 2) ? sW[v - 2] : 0.0;
    const double fr = sfh[(size_t)(e + 1) * nv + v], fl = sfh[(size_t)e * nv + v];
    double fqr[Q], sqr[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      fqr[q] = fq[q];
      sqr[q] = (v >= 2) ? sq[q] : 0.0;
    }
    double out[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double V = 0.0, S = 0.0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        V = fma(B.WdP[q][i], fqr[q], V);
        S = fma(B.WPh[q][i], sqr[q], S);
      }
      double surf = (i & 1) ? (V - fr - fl) : (V - fr + fl);
      double r = fma((2.0 * i + 1.0) * inv_dx, surf, Wv * S);
      size_t gi = ((size_t)v * N + ge) * Q + i;
      double o;
      if (A.s == 0) o = fma(I.dt, r, A.w0[gi]);
      else if (A.s == 1) o = fma(0.25, fma(I.dt, r, wi[i]), 0.75 * A.w0[gi]);
      else o = fma(2.0 / 3.0, fma(I.dt, r, wi[i]), (1.0 / 3.0) * A.w0[gi]);
      out[i] = o;
      A.wout[gi] = o;
      A.wnext[gi] = o;
    }
    if (slot_ok) {
      int pr = I.pf_of_right[ge], pl = I.pf_of_left[ge];
      if (pr >= 0) {
        size_t b = ring_block(I, A.n, A.s, pr, 0) + (size_t)v * Q;
        for (int i = 0; i < Q; ++i) {
          I.ring_in[b + i] = wi[i];
          I.ring_pre[b + i] = out[i];
        }
      }
      if (pl >= 0) {
        size_t b = ring_block(I, A.n, A.s, pl, 1) + (size_t)v * Q;
        for (int i = 0; i < Q; ++i) {
          I.ring_in[b + i] = wi[i];
          I.ring_pre[b + i] = out[i];
        }
      }
    }
  }
}

__device__ inline double minmod3(double a, double b, double c) {
  if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
  return 0.0;
}

// Shared memory (doubles) per element of the limiter: the element and its two
// neighbours, the limited characteristic modes, gradP.w, the partial-density
// sums and momenta of the three blocks, the per-species phi_k, two mode sums.
__host__ __device__ inline int limiter_elem_doubles(int nv, int ns, int Q) {
  return 3 * nv * Q + nv * Q + 3 * 3 * Q + ns + 2 * Q;
}
constexpr int LIM_WARPS = 8;

// Troubled-cell indicator and (AT-)WENO limiter (Sec. 3.3, Eq. 9-11), a group of
// G lanes per element (G = 16 when nv <= 16, else 32).
// Eigen-structure of the frozen Jacobian at the cell average: right vectors
// r_-/+ = (u -/+ a, H -/+ u a, Y), species r_k = (u, u^2 - phi_k/g, e_k); left
// vectors l_-/+ = (gradP -/+ a (1, 0, -u..-u)) / (2 a^2), l_k = e_k - Y_k gradP/a^2,
// gradP = (-u g, g, phi_1..phi_ns), g = gamma - 1, phi_k = g (u^2/2 - e_k) + R T / W_k.
// Every characteristic value is written in one branch-free form,
// v = A gradP.w + B (rho u)_w + C (sum rho Y)_w + D (rho Y_k)_w,
// with (A, B, C, D) = (1/2a^2, -/+ a/2a^2, +/- a u/2a^2, 0) for the acoustic fields
// and (-Y_k/a^2, 0, 0, 1) for species k, so that all lanes run the same FP64 code.
// The stage kernel has already written the pre-limit values into the output;
// only troubled cells are rewritten here.
template <int Q, int G>
__global__ void __launch_bounds__(32 * LIM_WARPS) limiter_kernel(Mech M, Inst I, LimArgs A) {
  extern __shared__ __align__(16) double lsm[];
  const Basis &B = c_basis[Q - 2];
  const int N = I.n_elem, nv = I.nv, ns = M.ns;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane % G, gw = lane / G;
  constexpr int EPW = 32 / G;
  const int slot = warp * EPW + gw;
  const int e = blockIdx.x * (LIM_WARPS * EPW) + slot;
  const bool valid = e < N;
  const unsigned FULL = 0xffffffffu;
  const unsigned gmask = (G == 32) ? FULL : (0xffffu << (16 * gw));
  const size_t VS = (size_t)N * Q;
  const int NB = nv * Q;
  double *blk = lsm + (size_t)slot * limiter_elem_doubles(nv, ns, Q);  // [3][nv][Q]
  double *vlim = blk + 3 * NB;                                          // [nv][Q]
  double *gpv = vlim + NB;                                              // [3][Q]
  double *rsv = gpv + 3 * Q;                                            // [3][Q]
  double *mmv = rsv + 3 * Q;                                            // [3][Q]
  double *phi = mmv + 3 * Q;                                            // [ns]
  double *sums = phi + ns;                                              // [2][Q]
  const bool periodic = (I.bc_left == ADG_BC_PERIODIC);

  // 1. the element (block 0) and its neighbours (1 left, 2 right): the pre-limit
  //    field, the AT extrapolation of the neighbour's pre-limit history across a
  //    delayed PE face (Eq. 11), or a boundary ghost
  if (valid) {
    for (int d = 0; d < 3; ++d) {
      double *dst = blk + d * NB;
      int src = e, ghost = 0, k = 0, pf = -1;
      if (d > 0) {
        pf = d == 1 ? I.pf_of_left[e] : I.pf_of_right[e];
        k = (pf >= 0) ? effective_delay(I, A.n, pf) : 0;
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
            acc += I.at[k][m] * I.ring_pre[ring_block(I, A.n - k - m, A.s, pf, side) + t];
          dst[t] = acc;
        }
      } else {
        for (int t = gl; t < NB; t += G) {
          int v = t / Q, j = t - v * Q;
          double x = A.wpre[(size_t)v * VS + (size_t)src * Q + j];
          if (ghost && (((j & 1) != 0) != (v == 0))) x = -x;
          dst[t] = x;
        }
      }
    }
  }
  __syncwarp();

  // 2. cell average: thermo and eigen-quantities (species sums split over lanes)
  const double *qW = M.sp + SP_QW * ns, *cvW = M.sp + SP_CVW * ns;
  const double *RW = M.sp + SP_RW * ns, *cpW = M.sp + SP_CPW * ns;
  double rho = 0.0, qsum = 0.0, cv = 0.0, Rm = 0.0, cpm = 0.0;
  if (valid)
    for (int i = gl; i < ns; i += G) {
      double r = blk[(2 + i) * Q];
      rho += r;
      qsum = fma(r, qW[i], qsum);
      cv = fma(r, cvW[i], cv);
      Rm = fma(r, RW[i], Rm);
      cpm = fma(r, cpW[i], cpm);
    }
  for (int o = G / 2; o > 0; o >>= 1) {
    rho += __shfl_xor_sync(FULL, rho, o, G);
    qsum += __shfl_xor_sync(FULL, qsum, o, G);
    cv += __shfl_xor_sync(FULL, cv, o, G);
    Rm += __shfl_xor_sync(FULL, Rm, o, G);
    cpm += __shfl_xor_sync(FULL, cpm, o, G);
  }
  if (!valid) {
    rho = 1.0;
    cv = 1.0;
    cpm = 2.0;
    Rm = 1.0;
  }
  const double irho = 1.0 / rho, icv = 1.0 / cv;
  const double m0 = valid ? blk[0] : 0.0, E0 = valid ? blk[Q] : 1.0;
  const double u = m0 * irho;
  const double T = (E0 - 0.5 * m0 * u - qsum) * icv;
  const double P = T * Rm;
  const double gam = cpm * icv, g = gam - 1.0;
  const double a = sqrt(gam * P * irho);
  const double H = (E0 + P) * irho;
  const double ia2 = 1.0 / (a * a);
  if (valid && gl == 0 && (!(rho > 0.0) || !(T > 0.0) || !isfinite(T)))
    report_error(I, ADG_ERR_NONPHYSICAL, e, A.s, A.n);
  if (valid) {
    for (int i = gl; i < ns; i += G)
      phi[i] = fma(g, fma(-cvW[i], T, 0.5 * u * u - qW[i]), T * RW[i]);
  }
  __syncwarp();
  if (valid)
    for (int t = gl; t < 3 * Q; t += G) {
      int b = t / Q, j = t - b * Q;
      const double *x = blk + b * NB;
      double acc = g * fma(-u, x[j], x[Q + j]), sr = 0.0;
      for (int i = 0; i < ns; ++i) {
        double r = x[(2 + i) * Q + j];
        acc = fma(phi[i], r, acc);
        sr += r;
      }
      gpv[t] = acc;
      rsv[t] = sr;
      mmv[t] = x[j];
    }
  __syncwarp();

  // coefficients of field k and its value for block b, mode j
  const double ha2 = 0.5 * ia2;
  auto coef = [&](int k, double &cA, double &cB, double &cC, double &cD, int &ri) {
    bool ac = (k == 0) || (k == nv - 1);
    double sgn = (k == 0) ? -1.0 : 1.0;
    ri = ac ? 0 : k - 1;
    double Yk = ac ? 0.0 : blk[(2 + ri) * Q] * irho;
    cA = ac ? ha2 : -Yk * ia2;
    cB = ac ? sgn * a * ha2 : 0.0;
    cC = ac ? -sgn * a * u * ha2 : 0.0;
    cD = ac ? 0.0 : 1.0;
  };
  auto val = [&](double cA, double cB, double cC, double cD, int ri, int b, int j) {
    return fma(cA, gpv[b * Q + j],
               fma(cB, mmv[b * Q + j], fma(cC, rsv[b * Q + j], cD * blk[b * NB + (2 + ri) * Q + j])));
  };

  // 3. indicator: the lanes of a group test the fields
  const double sig0 = fma(rho, a, fabs(m0)), sig1 = fabs(E0), sigr = rho;
  const double tvb = I.tvb, tau = 1e-10;
  bool mine = false;
  if (valid)
    for (int k = gl; k < nv; k += G) {
      double cA, cB, cC, cD;
      int ri;
      coef(k, cA, cB, cC, cD, ri);
      double vb = val(cA, cB, cC, cD, ri, 0, 0), vp = vb, vm = vb;
#pragma unroll
      for (int j = 1; j < Q; ++j) {
        double x = val(cA, cB, cC, cD, ri, 0, j);
        vp += x;
        vm += (j & 1) ? -x : x;
      }
      double vL = val(cA, cB, cC, cD, ri, 1, 0), vR = val(cA, cB, cC, cD, ri, 2, 0);
      double scale = fabs(fma(cA, -u * g, cB)) * sig0 + fabs(cA * g) * sig1;
      for (int i = 0; i < ns; ++i) {
        double l = fma(cA, phi[i], cC) + ((i == ri) ? cD : 0.0);
        scale = fma(fabs(l), sigr, scale);
      }
      double ut = vp - vb, utt = vb - vm, dp = vR - vb, dm = vb - vL;
      double fl = tau * scale;
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
  const double gmw[3] = {0.001, 0.998, 0.001};
  const double eps = 1e-6;
  for (int k = gl; k < nv; k += G) {
    double cA, cB, cC, cD;
    int ri;
    coef(k, cA, cB, cC, cD, ri);
    double vo[Q], vl0[Q], vr0[Q], vl[Q], vr[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      vo[j] = val(cA, cB, cC, cD, ri, 0, j);
      vl0[j] = val(cA, cB, cC, cD, ri, 1, j);
      vr0[j] = val(cA, cB, cC, cD, ri, 2, j);
    }
    // neighbours continued into this cell, their mean replaced by the own mean
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double al = 0.0, ar = 0.0;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        al = fma(B.Sl[i][j], vl0[j], al);
        ar = fma(B.Sr[i][j], vr0[j], ar);
      }
      vl[i] = al;
      vr[i] = ar;
    }
    vl[0] = vo[0];
    vr[0] = vo[0];
    double be[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 1; i < Q; ++i)
#pragma unroll
      for (int j = 1; j < Q; ++j) {
        be[0] = fma(vl[i] * B.B[i][j], vl[j], be[0]);
        be[1] = fma(vo[i] * B.B[i][j], vo[j], be[1]);
        be[2] = fma(vr[i] * B.B[i][j], vr[j], be[2]);
      }
    double wt[3], sw = 0.0;
    for (int t = 0; t < 3; ++t) {
      double d = eps + be[t];
      wt[t] = gmw[t] / (d * d);
      sw += wt[t];
    }
    double isw = 1.0 / sw;
    vlim[k * Q] = vo[0];
#pragma unroll
    for (int i = 1; i < Q; ++i)
      vlim[k * Q + i] = (wt[0] * vl[i] + wt[1] * vo[i] + wt[2] * vr[i]) * isw;
  }
  __syncwarp(gmask);
  // 5. back to conserved variables with R (modes >= 1; the cell average is kept)
  for (int i = gl; i < Q; i += G) {
    double s1 = 0.0, s2 = 0.0;
    for (int k = 1; k < nv - 1; ++k) {
      double x = vlim[k * Q + i];
      s1 += x;
      s2 = fma(x, u * u - phi[k - 1] / g, s2);
    }
    sums[i] = s1;
    sums[Q + i] = s2;
  }
  __syncwarp(gmask);
  double *out = A.wout + (size_t)e * Q;
  for (int t = gl; t < NB; t += G) {
    int v = t / Q, i = t - v * Q;
    if (i == 0) continue;
    double lm = vlim[i], lp = vlim[(nv - 1) * Q + i];
    double o;
    if (v == 0) o = lm * (u - a) + lp * (u + a) + u * sums[i];
    else if (v == 1) o = lm * (H - u * a) + lp * (H + u * a) + sums[Q + i];
    else o = (lm + lp) * (blk[v * Q] * irho) + vlim[(v - 1) * Q + i];
    out[(size_t)v * VS + i] = o;
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
  return cudaMemcpyToSymbol(c_basis, tables, sizeof(Basis) * ADG_MAX_P);
}

int stage_tile(int Q, int nv, int ns, int nr) {
  // elements per tile: up to 256 Gauss-point threads, at most ~96 KB of tile
  int TE = 256 / Q;
  while (TE > 2 && stage_smem_bytes(TE, Q, nv, ns, nr) > 96 * 1024) TE /= 2;
  return TE;
}

size_t stage_smem(int TE, int Q, int nv, int ns, int nr) {
  return stage_smem_bytes(TE, Q, nv, ns, nr);
}

cudaError_t upload_exp_table(const ExpTable *t) {
  return cudaMemcpyToSymbol(c_exp, t, sizeof(ExpTable));
}

template <int Q>
static cudaError_t launch_stage_q(const Mech &M, const Inst &I, const StageArgs &A,
                                  cudaStream_t st) {
  size_t smem = stage_smem_bytes(A.TE, Q, I.nv, M.ns, M.nr);
  static bool attr_set[4] = {false, false, false, false};
  if (!attr_set[Q - 2]) {
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<Q>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set[Q - 2] = true;
  }
  int nblk = (I.n_elem + A.TE - 1) / A.TE;
  int nth = A.TE * Q;
  nth = ((nth + 31) / 32) * 32;
  stage_kernel<Q><<<nblk, nth, smem, st>>>(M, I, A);
  return cudaGetLastError();
}

cudaError_t launch_stage(const Mech &M, const Inst &I, const StageArgs &A, cudaStream_t st) {
  switch (I.p + 1) {
    case 2: return launch_stage_q<2>(M, I, A, st);
    case 3: return launch_stage_q<3>(M, I, A, st);
    case 4: return launch_stage_q<4>(M, I, A, st);
    case 5: return launch_stage_q<5>(M, I, A, st);
  }
  return cudaErrorInvalidValue;
}

template <int Q, int G>
static cudaError_t launch_limiter_qg(const Mech &M, const Inst &I, const LimArgs &A,
                                     cudaStream_t st) {
  constexpr int EPW = 32 / G;
  size_t smem = (size_t)LIM_WARPS * EPW * limiter_elem_doubles(I.nv, M.ns, Q) * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(limiter_kernel<Q, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int per = LIM_WARPS * EPW;
  int nblk = (I.n_elem + per - 1) / per;
  limiter_kernel<Q, G><<<nblk, 32 * LIM_WARPS, smem, st>>>(M, I, A);
  return cudaGetLastError();
}

template <int Q>
static cudaError_t launch_limiter_q(const Mech &M, const Inst &I, const LimArgs &A,
                                    cudaStream_t st) {
  if (I.nv <= 16) return launch_limiter_qg<Q, 16>(M, I, A, st);
  return launch_limiter_qg<Q, 32>(M, I, A, st);
}

cudaError_t launch_limiter(const Mech &M, const Inst &I, const LimArgs &A, cudaStream_t st) {
  switch (I.p + 1) {
    case 2: return launch_limiter_q<2>(M, I, A, st);
    case 3: return launch_limiter_q<3>(M, I, A, st);
    case 4: return launch_limiter_q<4>(M, I, A, st);
    case 5: return launch_limiter_q<5>(M, I, A, st);
  }
  return cudaErrorInvalidValue;
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
