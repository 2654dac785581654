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
//   limiter_kernel<Q>: one thread per element: troubled-cell indicator in the
//                      characteristic fields of the cell average and, on troubled
//                      cells, the (AT-)WENO reconstruction of Eq. (9)-(11).
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
      cq[(size_t)i * TQ] = fmax(wq[(size_t)(2 + i) * TQ], 0.0) * sIW[i];
      gq[(size_t)i * TQ] = fma(sG0[i], invT, sG1[i]) - sCR[i] * lnT;
      wd[(size_t)i * TQ] = 0.0;
    }
    const double lr = lnT + LN_R_PATM;
    for (int j = 0; j < nr; ++j) {
      const Rxn &R = srx[j];
      double lkf = fma(R.b, lnT, R.lnA) - R.EaR * invT;
      double dg = R.dnu * lr;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (R.xn[k] == 0) break;
        dg = fma((double)R.xn[k], gq[(size_t)R.xs[k] * TQ], dg);
      }
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
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (R.xn[k] == 0) break;
        wd[(size_t)R.xs[k] * TQ] = fma((double)R.xn[k], qj, wd[(size_t)R.xs[k] * TQ]);
      }
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
  for (int item = tid; item < nv * te; item += nth) {
    int v = item / te, e = item - v * te, ge = e0 + e, le = e + 1;
    const double *wi = sw + ((size_t)v * (TE + 2) + le) * Q;
    const double *fq = snode + (size_t)v * TQ + e * Q;
    const double *sq = (v >= 2) ? swd + (size_t)(v - 2) * TQ + e * Q : nullptr;
    const double Wv = (v >= 2) ? sW[v - 2] : 0.0;
    double out[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double V = 0.0, S = 0.0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        V += B.w[q] * fq[q] * B.dP[q][i];
        if (v >= 2) S += B.w[q] * (Wv * sq[q]) * B.P[q][i];
      }
      double sgn = (i & 1) ? -1.0 : 1.0;
      double surf = V - sfh[(size_t)(e + 1) * nv + v] + sgn * sfh[(size_t)e * nv + v];
      double r = (2.0 * i + 1.0) / I.dx * surf + 0.5 * (2.0 * i + 1.0) * S;
      size_t gi = ((size_t)v * N + ge) * Q + i;
      double o;
      if (A.s == 0) o = A.w0[gi] + I.dt * r;
      else if (A.s == 1) o = 0.75 * A.w0[gi] + 0.25 * (wi[i] + I.dt * r);
      else o = (1.0 / 3.0) * A.w0[gi] + (2.0 / 3.0) * (wi[i] + I.dt * r);
      out[i] = o;
      A.wout[gi] = o;
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

// Access to a neighbour block for the limiter: the pre-limit field, the AT
// extrapolation of the neighbour's pre-limit history (Eq. 11), or a boundary ghost.
struct Nb {
  const double *direct;     // pointer to variable 0, mode 0 of the element; stride N*Q per var
  size_t vstride;
  const double *lev[MAXO];  // ring blocks (stride Q per var)
  double c[MAXO];
  int nlev;
  int ghost;                // 0 none, 1 mirror (reflecting wall)
  __device__ inline double get(int v, int j, int Q) const {
    if (nlev > 0) {
      double acc = 0.0;
      for (int m = 0; m < nlev; ++m) acc += c[m] * lev[m][v * Q + j];
      return acc;
    }
    double x = direct[v * vstride + j];
    if (ghost == 1) {
      double sg = (j & 1) ? -1.0 : 1.0;
      if (v == 0) sg = -sg;
      x *= sg;
    }
    return x;
  }
};

__device__ inline double minmod3(double a, double b, double c) {
  if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
  return 0.0;
}

// Eigen-structure of the frozen Jacobian at the cell average (Sec. 3.3):
// right vectors r_-/+ = (u -/+ a, H -/+ u a, Y), species r_k = (u, u^2 - phi_k/g, e_k),
// left vectors l_-/+ = (gradP -/+ a (1, 0, -u..-u)) / (2 a^2), l_k = e_k - Y_k gradP / a^2,
// gradP = (-u g, g, phi_1..phi_ns), g = gamma - 1,
// phi_k = g (u^2/2 - e_k) + R_u T / W_k.
template <int Q>
__global__ void __launch_bounds__(128) limiter_kernel(Mech M, Inst I, LimArgs A) {
  const Basis &B = c_basis[Q - 2];
  const int N = I.n_elem, nv = I.nv, ns = M.ns;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  const size_t VS = (size_t)N * Q;
  const double *own = A.wpre + (size_t)e * Q;
  const bool periodic = (I.bc_left == ADG_BC_PERIODIC);
  // neighbours
  Nb nb[2];
  for (int d = 0; d < 2; ++d) {
    Nb &x = nb[d];
    x.nlev = 0;
    x.ghost = 0;
    x.vstride = VS;
    int pf = d == 0 ? I.pf_of_left[e] : I.pf_of_right[e];
    int k = (pf >= 0) ? effective_delay(I, A.n, pf) : 0;
    if (k > 0) {
      int side = d == 0 ? 0 : 1;
      x.nlev = I.at_order;
      for (int m = 0; m < I.at_order; ++m) {
        x.lev[m] = I.ring_pre + ring_block(I, A.n - k - m, A.s, pf, side);
        x.c[m] = I.at[k][m];
      }
      x.direct = nullptr;
      continue;
    }
    int nbe = d == 0 ? e - 1 : e + 1;
    if (nbe < 0 || nbe >= N) {
      if (periodic) {
        nbe = (nbe + N) % N;
      } else {
        nbe = e;
        int bc = d == 0 ? I.bc_left : I.bc_right;
        x.ghost = (bc == ADG_BC_REFLECT) ? 1 : 0;
      }
    }
    x.direct = A.wpre + (size_t)nbe * Q;
  }

  // cell average and eigen-quantities
  double wbar[2];
  wbar[0] = own[0];
  wbar[1] = own[VS];
  double rho = 0.0, qsum = 0.0, cv = 0.0, Rm = 0.0, cpm = 0.0;
  const double *qW = M.sp + SP_QW * ns, *cvW = M.sp + SP_CVW * ns;
  const double *RW = M.sp + SP_RW * ns, *cpW = M.sp + SP_CPW * ns;
  for (int i = 0; i < ns; ++i) {
    double r = own[(2 + i) * VS];
    rho += r;
    qsum += r * qW[i];
    cv += r * cvW[i];
    Rm += r * RW[i];
    cpm += r * cpW[i];
  }
  const double u = wbar[0] / rho;
  const double T = (wbar[1] - 0.5 * wbar[0] * wbar[0] / rho - qsum) / cv;
  const double P = T * Rm;
  const double g = cpm / cv - 1.0;
  const double a = sqrt(cpm / cv * P / rho);
  const double H = (wbar[1] + P) / rho;
  const double ia2 = 1.0 / (a * a);
  if (!(rho > 0.0) || !(T > 0.0) || !isfinite(T)) {
    report_error(I, ADG_ERR_NONPHYSICAL, e, A.s, A.n);
  }
  // gradP . w, sum of partial densities and momentum, for every mode of the three
  // blocks (0 own, 1 left, 2 right)
  double gp[3][Q], rs[3][Q], mm[3][Q];
  for (int b = 0; b < 3; ++b)
    for (int j = 0; j < Q; ++j) {
      double m_, E_;
      if (b == 0) {
        m_ = own[j];
        E_ = own[VS + j];
      } else {
        m_ = nb[b - 1].get(0, j, Q);
        E_ = nb[b - 1].get(1, j, Q);
      }
      double acc = -u * g * m_ + g * E_, sr = 0.0;
      for (int i = 0; i < ns; ++i) {
        double r = (b == 0) ? own[(2 + i) * VS + j] : nb[b - 1].get(2 + i, j, Q);
        double phi = g * (0.5 * u * u - (qW[i] + cvW[i] * T)) + T * RW[i];
        acc += phi * r;
        sr += r;
      }
      gp[b][j] = acc;
      rs[b][j] = sr;
      mm[b][j] = m_;
    }
  // per-variable magnitudes of the noise floor
  const double sig0 = rho * a + fabs(wbar[0]), sig1 = fabs(wbar[1]), sigr = rho;
  const double tvb = I.tvb;
  const double tau = 1e-10;
  // field values of a block-mode combination: v_k = l_k . w
  auto acoustic = [&](int b, int j, double sgn) {
    return (gp[b][j] + sgn * a * (mm[b][j] - u * rs[b][j])) * 0.5 * ia2;
  };
  // gradP magnitudes for the floor of the acoustic and species fields
  double sum_abs_grad = fabs(u * g) * sig0 + fabs(g) * sig1;
  bool troubled = false;
  // acoustic fields
  for (int f = 0; f < 2 && !troubled; ++f) {
    double sgn = f == 0 ? -1.0 : 1.0;
    double vb = acoustic(0, 0, sgn), vp = 0.0, vm = 0.0;
    for (int j = 0; j < Q; ++j) {
      double x = acoustic(0, j, sgn);
      vp += x;
      vm += (j & 1) ? -x : x;
    }
    double vL = acoustic(1, 0, sgn), vR = acoustic(2, 0, sgn);
    double scale = (fabs(-u * g + sgn * a) * sig0 + fabs(g) * sig1) * 0.5 * ia2;
    for (int i = 0; i < ns; ++i) {
      double phi = g * (0.5 * u * u - (qW[i] + cvW[i] * T)) + T * RW[i];
      scale += fabs(phi - sgn * a * u) * sigr * 0.5 * ia2;
    }
    double ut = vp - vb, utt = vb - vm, dp = vR - vb, dm = vb - vL;
    double fl = tau * scale;
    if (fabs(ut) > fl && fabs(ut) > tvb && minmod3(ut, dp, dm) != ut) troubled = true;
    if (fabs(utt) > fl && fabs(utt) > tvb && minmod3(utt, dp, dm) != utt) troubled = true;
  }
  // species fields
  for (int k = 0; k < ns && !troubled; ++k) {
    double Yk = own[(2 + k) * VS] / rho;
    auto fieldv = [&](int b, int j) {
      double r = (b == 0) ? own[(2 + k) * VS + j] : nb[b - 1].get(2 + k, j, Q);
      return r - Yk * gp[b][j] * ia2;
    };
    double vb = fieldv(0, 0), vp = 0.0, vm = 0.0;
    for (int j = 0; j < Q; ++j) {
      double x = fieldv(0, j);
      vp += x;
      vm += (j & 1) ? -x : x;
    }
    double vL = fieldv(1, 0), vR = fieldv(2, 0);
    double scale = fabs(Yk) * ia2 * sum_abs_grad;
    for (int i = 0; i < ns; ++i) {
      double phi = g * (0.5 * u * u - (qW[i] + cvW[i] * T)) + T * RW[i];
      double l = (i == k ? 1.0 : 0.0) - Yk * phi * ia2;
      scale += fabs(l) * sigr;
    }
    double ut = vp - vb, utt = vb - vm, dp = vR - vb, dm = vb - vL;
    double fl = tau * scale;
    if (fabs(ut) > fl && fabs(ut) > tvb && minmod3(ut, dp, dm) != ut) troubled = true;
    if (fabs(utt) > fl && fabs(utt) > tvb && minmod3(utt, dp, dm) != utt) troubled = true;
  }
  if (I.limiter == ADG_LIM_NONE) troubled = false;
  I.flags[(size_t)A.s * N + e] = troubled ? 1 : 0;
  if (troubled) I.count[e] += 1;
  double *out = A.wout + (size_t)e * Q;
  if (!troubled) {
    for (int v = 0; v < nv; ++v)
      for (int j = 0; j < Q; ++j) out[v * VS + j] = own[v * VS + j];
    return;
  }
  // WENO (Eq. 9-10) in the characteristic fields, reconstructed with R
  const double gam[3] = {0.001, 0.998, 0.001};
  const double eps = 1e-6;
  auto weno_field = [&](double *vo, double *vl0, double *vr0, double *vlim) {
    // continue the neighbours into this cell, replace their mean by the own mean
    double vl[Q], vr[Q];
    for (int i = 0; i < Q; ++i) {
      double al = 0.0, ar = 0.0;
      for (int j = 0; j < Q; ++j) {
        al += B.Sl[i][j] * vl0[j];
        ar += B.Sr[i][j] * vr0[j];
      }
      vl[i] = al;
      vr[i] = ar;
    }
    vl[0] = vo[0];
    vr[0] = vo[0];
    double be[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) {
        be[0] += vl[i] * B.B[i][j] * vl[j];
        be[1] += vo[i] * B.B[i][j] * vo[j];
        be[2] += vr[i] * B.B[i][j] * vr[j];
      }
    double wt[3], sw = 0.0;
    for (int t = 0; t < 3; ++t) {
      wt[t] = gam[t] / ((eps + be[t]) * (eps + be[t]));
      sw += wt[t];
    }
    for (int t = 0; t < 3; ++t) wt[t] /= sw;
    vlim[0] = vo[0];
    for (int i = 1; i < Q; ++i) vlim[i] = wt[0] * vl[i] + wt[1] * vo[i] + wt[2] * vr[i];
  };
  double lm[Q], lp[Q];
  {
    double vo[Q], vl[Q], vr[Q];
    for (int j = 0; j < Q; ++j) {
      vo[j] = acoustic(0, j, -1.0);
      vl[j] = acoustic(1, j, -1.0);
      vr[j] = acoustic(2, j, -1.0);
    }
    weno_field(vo, vl, vr, lm);
    for (int j = 0; j < Q; ++j) {
      vo[j] = acoustic(0, j, 1.0);
      vl[j] = acoustic(1, j, 1.0);
      vr[j] = acoustic(2, j, 1.0);
    }
    weno_field(vo, vl, vr, lp);
  }
  double sm_[Q], se_[Q];
  for (int i = 0; i < Q; ++i) {
    sm_[i] = 0.0;
    se_[i] = 0.0;
  }
  for (int k = 0; k < ns; ++k) {
    double Yk = own[(2 + k) * VS] / rho;
    double ek = qW[k] + cvW[k] * T;
    double phik = g * (0.5 * u * u - ek) + T * RW[k];
    double vo[Q], vl[Q], vr[Q], lim[Q];
    for (int j = 0; j < Q; ++j) {
      vo[j] = own[(2 + k) * VS + j] - Yk * gp[0][j] * ia2;
      vl[j] = nb[0].get(2 + k, j, Q) - Yk * gp[1][j] * ia2;
      vr[j] = nb[1].get(2 + k, j, Q) - Yk * gp[2][j] * ia2;
    }
    weno_field(vo, vl, vr, lim);
    out[(2 + k) * VS] = own[(2 + k) * VS];
    for (int i = 1; i < Q; ++i) {
      out[(2 + k) * VS + i] = (lm[i] + lp[i]) * Yk + lim[i];
      sm_[i] += lim[i];
      se_[i] += lim[i] * (u * u - phik / g);
    }
  }
  out[0] = own[0];
  out[VS] = own[VS];
  for (int i = 1; i < Q; ++i) {
    out[i] = lm[i] * (u - a) + lp[i] * (u + a) + u * sm_[i];
    out[VS + i] = lm[i] * (H - u * a) + lp[i] * (H + u * a) + se_[i];
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

cudaError_t launch_limiter(const Mech &M, const Inst &I, const LimArgs &A, cudaStream_t st) {
  int nblk = (I.n_elem + 127) / 128;
  switch (I.p + 1) {
    case 2: limiter_kernel<2><<<nblk, 128, 0, st>>>(M, I, A); break;
    case 3: limiter_kernel<3><<<nblk, 128, 0, st>>>(M, I, A); break;
    case 4: limiter_kernel<4><<<nblk, 128, 0, st>>>(M, I, A); break;
    case 5: limiter_kernel<5><<<nblk, 128, 0, st>>>(M, I, A); break;
    default: return cudaErrorInvalidValue;
  }
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
