/* Plain FP64 CPU oracle of the asynchronous discontinuous Galerkin (ADG) scheme
 * for the 1D reacting Euler equations (arXiv 2501.01747).
 *
 * TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it to check and time the CUDA path. It shares no code with
 * the CUDA library. Every routine is the plain definition or the paper's steps in
 * their order, with no blocking, fusion or reordering. Built with
 * -O2 -ffp-contract=off so that no multiply-add is fused behind the reader's back.
 *
 * Where the paper leaves a choice open, this file takes the reading stated next to
 * the routine (modal Legendre basis with p+1 Gauss points, constant-cp species,
 * SSP-RK3 stages, one delay per PE face per step, and so on).
 */
#include "adg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define RU 8.314462618   /* J/mol/K */
#define TREF 298.15      /* K, reference temperature of h_f and s0 */
#define PATM 101325.0    /* Pa, standard-state pressure of s0 and K_c */
#define MAXV 64
#define MAXQ 8

/* ------------------------------------------------------------------------- */
/* Basis (Sec. 3.1: basis polynomials phi_j of degree <= N_p; reading: Legendre). */

void or_legendre(int n, double x, double *P, double *dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (n >= 1) {
    P[1] = x;
    dP[1] = 1.0;
  }
  for (int j = 1; j < n; ++j) {
    /* Bonnet: (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1};  P'_{j+1} = P'_{j-1} + (2j+1) P_j */
    P[j + 1] = ((2.0 * j + 1.0) * x * P[j] - j * P[j - 1]) / (j + 1.0);
    dP[j + 1] = dP[j - 1] + (2.0 * j + 1.0) * P[j];
  }
}

/* Gauss-Legendre points and weights on [-1,1], ascending: Newton on P_q. */
int or_gauss(int q, double *x, double *w) {
  double P[MAXQ + 2], dP[MAXQ + 2];
  if (q < 1 || q > MAXQ) return -1;
  for (int i = 0; i < q; ++i) {
    double t = -cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      or_legendre(q, t, P, dP);
      double dt = P[q] / dP[q];
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    or_legendre(q, t, P, dP);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dP[q] * dP[q]);
  }
  return 0;
}

/* Monomial coefficients of P_j, j = 0..n: C[j*(n+1) + k] is the coefficient of x^k. */
static void legendre_monomials(int n, double *C) {
  memset(C, 0, sizeof(double) * (n + 1) * (n + 1));
  C[0] = 1.0;
  if (n >= 1) C[(n + 1) + 1] = 1.0;
  for (int j = 1; j < n; ++j) {
    for (int k = 0; k <= n; ++k) {
      double v = -j * C[(j - 1) * (n + 1) + k];
      if (k >= 1) v += (2.0 * j + 1.0) * C[j * (n + 1) + k - 1];
      C[(j + 1) * (n + 1) + k] = v / (j + 1.0);
    }
  }
}

/* exact integral over [-1,1] of x^k */
static double mono_int(int k) { return (k % 2) ? 0.0 : 2.0 / (k + 1.0); }

/* Smoothness-indicator matrix (Eq. 10): beta = sum_s int_{Omega_e} dx^{2s-1} (d^s v/dx^s)^2 dx
 * = sum_s 2^{2s-1} int_{-1}^{1} (d^s v/d xi^s)^2 d xi, a quadratic form in the modal
 * coefficients: beta = v^T B v, B is (p+1)x(p+1), row/column 0 zero. */
void or_beta_matrix(int p, double *B) {
  int n = p + 1;
  double C[MAXQ * MAXQ];
  legendre_monomials(p, C);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int s = 1; s <= p; ++s) {
        /* s-th derivative of P_i and P_j as monomials, then the exact integral */
        double di[MAXQ], dj[MAXQ];
        for (int k = 0; k < n; ++k) {
          di[k] = 0.0;
          dj[k] = 0.0;
        }
        for (int k = s; k < n; ++k) {
          double f = 1.0;
          for (int t = 0; t < s; ++t) f *= (double)(k - t);
          di[k - s] = C[i * n + k] * f;
          dj[k - s] = C[j * n + k] * f;
        }
        double in = 0.0;
        for (int a = 0; a < n; ++a)
          for (int b = 0; b < n; ++b) in += di[a] * dj[b] * mono_int(a + b);
        acc += ldexp(1.0, 2 * s - 1) * in;
      }
      B[i * n + j] = acc;
    }
}

/* Neighbour polynomial continued into the cell (the WENO stencil of Eq. 9 and the
 * reading that v_{e+-1} are the neighbours' polynomials evaluated on Omega_e):
 * dir = -1: left neighbour, whose coordinate is xi' = xi + 2; dir = +1: right
 * neighbour, xi' = xi - 2. S[i*(p+1)+j] = (2i+1)/2 int P_j(xi') P_i(xi) d xi. */
void or_shift_matrix(int p, int dir, double *S) {
  int n = p + 1;
  double C[MAXQ * MAXQ];
  double c = -2.0 * dir;
  legendre_monomials(p, C);
  for (int j = 0; j < n; ++j) {
    /* monomials of P_j(xi + c) */
    double sh[MAXQ];
    for (int k = 0; k < n; ++k) sh[k] = 0.0;
    for (int k = 0; k < n; ++k) {
      double a = C[j * n + k];
      if (a == 0.0) continue;
      /* (xi + c)^k = sum_t binom(k,t) xi^t c^{k-t} */
      double binom = 1.0;
      for (int t = 0; t <= k; ++t) {
        sh[t] += a * binom * pow(c, k - t);
        binom = binom * (k - t) / (t + 1.0);
      }
    }
    for (int i = 0; i < n; ++i) {
      double in = 0.0;
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) in += sh[a] * C[i * n + b] * mono_int(a + b);
      S[i * n + j] = 0.5 * (2.0 * i + 1.0) * in;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* AT coefficients (Sec. 3.2, Eq. 7-8, Table 1): the weights c_m of the levels
 * n-k-m, m = 0..o-1, that cancel the Taylor terms of order 1..o-1. This is the
 * Lagrange extrapolation to t_n from the levels t_n - (k+m) dt:
 * c_m = prod_{j != m} (k+j)/(j-m). */
void or_at_coeffs(int order, int k, double *c) {
  for (int m = 0; m < order; ++m) {
    double v = 1.0;
    for (int j = 0; j < order; ++j)
      if (j != m) v *= (double)(k + j) / (double)(j - m);
    c[m] = v;
  }
}

/* SplitMix64 finaliser applied to one counter (Steele, Lea and Flood 2014). */
uint64_t or_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Delay of PE face `face` at step `step`.
 * CAA (Sec. 4.1): the delay grows by one each step and resets when n % L == 0,
 * i.e. k = n mod L with L = max_delay + 1.
 * SAA (Sec. 4.2): a uniform draw r in [0,1) is matched to the bins of the
 * cumulative probabilities {p_0, .., p_{L-1}}; the draw is SplitMix64 of
 * seed XOR (step * 2^32 + face), top 53 bits (face counted from cfg->face0). */
int or_delay(const or_cfg *cfg, int64_t step, int face) {
  if (cfg->delay_mode == 0) return 0;
  if (cfg->delay_mode == 1) return (int)(step % (cfg->max_delay + 1));
  uint64_t key = cfg->seed ^ (((uint64_t)step << 32) + (uint64_t)(uint32_t)(face + cfg->face0));
  double r = (double)(or_splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
  double acc = 0.0;
  for (int k = 0; k <= cfg->max_delay; ++k) {
    acc += cfg->delay_probs[k];
    if (r < acc) return k;
  }
  return cfg->max_delay;
}

/* ------------------------------------------------------------------------- */
/* Thermodynamics (Sec. 2: E = u^2/2 - P/rho + h, h = sum Y_i h_i; P = rho R T / W).
 * Reading: constant molar c_p per species,
 *   h_i(T) = [h_f,i + c_p,i (T - T_ref)] / W_i,  e_i = h_i - R_u T / W_i,
 *   s_i(T) = s0_i + c_p,i ln(T / T_ref). */

static double sp_e(const or_mech *m, int i, double T) {
  return (m->hf[i] + m->cp[i] * (T - TREF) - RU * T) / m->W[i];
}

/* Temperature from the internal energy per volume rho*e = sum_i r_i e_i(T):
 * Newton from Tguess, stop when |dT| <= 1e-10 T, at most 20 iterations. */
int or_temperature(const or_mech *m, const double *r, double rhoe, double Tguess,
                   double *T) {
  double t = Tguess;
  for (int it = 0; it < 20; ++it) {
    double g = -rhoe, dg = 0.0;
    for (int i = 0; i < m->ns; ++i) {
      g += r[i] * sp_e(m, i, t);
      dg += r[i] * (m->cp[i] - RU) / m->W[i];
    }
    double dT = g / dg;
    t -= dT;
    if (fabs(dT) <= 1e-10 * fabs(t)) {
      *T = t;
      return it + 1;
    }
  }
  *T = t;
  return -1;
}

/* rho, u, T, P and the frozen sound speed a^2 = gamma P / rho,
 * gamma = sum r_i cp_i/W_i / sum r_i (cp_i - R_u)/W_i. */
void or_state(const or_mech *m, const double *w, double *rho, double *u, double *T,
              double *P, double *a) {
  const double *r = w + 2;
  double rh = 0.0;
  for (int i = 0; i < m->ns; ++i) rh += r[i];
  double uu = w[0] / rh;
  double rhoe = w[1] - 0.5 * w[0] * w[0] / rh;
  double t;
  or_temperature(m, r, rhoe, 1000.0, &t);
  double Rm = 0.0, cpm = 0.0, cvm = 0.0;
  for (int i = 0; i < m->ns; ++i) {
    Rm += r[i] * RU / m->W[i];
    cpm += r[i] * m->cp[i] / m->W[i];
    cvm += r[i] * (m->cp[i] - RU) / m->W[i];
  }
  double p = t * Rm;
  *rho = rh;
  *u = uu;
  *T = t;
  *P = p;
  *a = sqrt(cpm / cvm * p / rh);
}

void or_cons_from_prim(const or_mech *m, double T, double P, double u, const double *Y,
                       double *w) {
  double sYW = 0.0;
  for (int i = 0; i < m->ns; ++i) sYW += Y[i] / m->W[i];
  double rho = P / (RU * T * sYW);
  double e = 0.0;
  for (int i = 0; i < m->ns; ++i) e += Y[i] * sp_e(m, i, T);
  w[0] = rho * u;
  w[1] = rho * (e + 0.5 * u * u);
  for (int i = 0; i < m->ns; ++i) w[2 + i] = rho * Y[i];
}

/* ------------------------------------------------------------------------- */
/* Kinetics (Sec. 2, source s = (0, 0, 0, W_i omega_i)).
 * k_f = A T^b exp(-E_a / (R_u T)); K_c = exp(-dG / (R_u T)) (P_atm / (R_u T))^{sum nu},
 * dG = sum_i nu_i g_i(T), g_i = h_i - T s_i (molar), nu = nu'' - nu'; k_r = k_f / K_c;
 * q = k_f prod c^nu' - k_r prod c^nu''; omega_i = sum_j nu_ij q_j. */
void or_rates(const or_mech *m, double T, int j, double *kf, double *Kc) {
  *kf = m->A[j] * pow(T, m->b[j]) * exp(-m->Ea[j] / (RU * T));
  double dG = 0.0;
  int dnu = 0;
  for (int i = 0; i < m->ns; ++i) {
    int nu = m->nu_r[j * m->ns + i] - m->nu_f[j * m->ns + i];
    if (nu == 0) continue;
    double h = m->hf[i] + m->cp[i] * (T - TREF);
    double s = m->s0[i] + m->cp[i] * log(T / TREF);
    dG += nu * (h - T * s);
    dnu += nu;
  }
  *Kc = exp(-dG / (RU * T)) * pow(PATM / (RU * T), (double)dnu);
}

void or_wdot(const or_mech *m, double T, const double *conc, double *wdot) {
  for (int i = 0; i < m->ns; ++i) wdot[i] = 0.0;
  for (int j = 0; j < m->nr; ++j) {
    double kf, Kc;
    or_rates(m, T, j, &kf, &Kc);
    double fwd = kf, rev = kf / Kc;
    for (int i = 0; i < m->ns; ++i) {
      for (int k = 0; k < m->nu_f[j * m->ns + i]; ++k) fwd *= conc[i];
      for (int k = 0; k < m->nu_r[j * m->ns + i]; ++k) rev *= conc[i];
    }
    double q = fwd - rev;
    for (int i = 0; i < m->ns; ++i)
      wdot[i] += (m->nu_r[j * m->ns + i] - m->nu_f[j * m->ns + i]) * q;
  }
}

/* ------------------------------------------------------------------------- */
/* Fluxes: convective flux f^c of Eq. (2) in the variables (rho u, rho E, rho Y_i). */
void or_phys_flux(const or_mech *m, const double *w, double *f) {
  double rho, u, T, P, a;
  or_state(m, w, &rho, &u, &T, &P, &a);
  f[0] = w[0] * u + P;
  f[1] = u * (w[1] + P);
  for (int i = 0; i < m->ns; ++i) f[2 + i] = u * w[2 + i];
}

/* Mixture transport (Sec. 2 names the viscosity mu, the conductivity k and the
 * mixture-averaged diffusion coefficients D_i^mix; the paper takes them from
 * Cantera). Reading, a synthetic model: mu = mu_ref (T/T_mu)^mu_exp for the
 * mixture, k = mu cp / Pr with cp the mixture's specific heat per unit mass, and
 * D_i = k / (rho cp Le_i) with a Lewis number per species. */
void or_transport(const or_mech *m, const or_cfg *cfg, double rho, double T, const double *Y,
                  double *mu, double *kc, double *D) {
  double cpm = 0.0;
  for (int i = 0; i < m->ns; ++i) cpm += Y[i] * m->cp[i] / m->W[i];
  *mu = cfg->mu_ref * pow(T / cfg->T_mu, cfg->mu_exp);
  *kc = *mu * cpm / cfg->prandtl;
  for (int i = 0; i < m->ns; ++i) D[i] = *kc / (rho * cpm * (m->Le ? m->Le[i] : 1.0));
}

/* Diffusive flux of Sec. 2 at one point, from the conserved state w and its
 * x-derivative q (the LDG auxiliary variable): (tau, tau u - q_h, -J_1 .. -J_Ns)
 * with tau = 4/3 mu du/dx, q_h = -k dT/dx + sum h_i J_i, J_i = rho Y_i V_i and
 * V_i = -(D_i / X_i) dX_i/dx. Reading: the correction velocity
 * V_c = -sum Y_j V_j is added to every V_i so that sum J_i = 0, as the density
 * equation carries no diffusive flux. The primitive derivatives follow from q by
 * the chain rule: rho_x = sum q_{rho Y_i}, u_x = (q_{rho u} - u rho_x) / rho,
 * Y_i,x = (q_{rho Y_i} - Y_i rho_x) / rho, and from
 * rho E - (rho u) u / 2 = sum rho Y_i e_i(T):
 * T_x = (q_{rho E} - (q_{rho u} u + rho u u_x) / 2 - sum q_{rho Y_i} e_i(T))
 *       / sum rho Y_i c_v,i.
 * X_i = (Y_i / W_i) / n with n = sum Y_j / W_j, so Y_i / X_i = W_i n and
 * J_i = -rho D_i W_i n dX_i/dx, with dX_i/dx = (Y_i,x / W_i - X_i n_x) / n. */
void or_visc_flux(const or_mech *m, const or_cfg *cfg, const double *w, const double *q,
                  double *fd) {
  int ns = m->ns;
  const double *r = w + 2, *qr = q + 2;
  double rho = 0.0, rho_x = 0.0;
  for (int i = 0; i < ns; ++i) {
    rho += r[i];
    rho_x += qr[i];
  }
  double u = w[0] / rho;
  double u_x = (q[0] - u * rho_x) / rho;
  double Y[MAXV], Yx[MAXV], D[MAXV], J[MAXV];
  for (int i = 0; i < ns; ++i) {
    Y[i] = r[i] / rho;
    Yx[i] = (qr[i] - Y[i] * rho_x) / rho;
  }
  double T;
  or_temperature(m, r, w[1] - 0.5 * w[0] * u, 1000.0, &T);
  double num = q[1] - 0.5 * (q[0] * u + w[0] * u_x), den = 0.0;
  for (int i = 0; i < ns; ++i) {
    num -= qr[i] * sp_e(m, i, T);
    den += r[i] * (m->cp[i] - RU) / m->W[i];
  }
  double T_x = num / den;
  double n = 0.0, n_x = 0.0;
  for (int i = 0; i < ns; ++i) {
    n += Y[i] / m->W[i];
    n_x += Yx[i] / m->W[i];
  }
  double mu, kc;
  or_transport(m, cfg, rho, T, Y, &mu, &kc, D);
  double Jsum = 0.0;
  for (int i = 0; i < ns; ++i) {
    double X = Y[i] / (m->W[i] * n);
    double X_x = (Yx[i] / m->W[i] - X * n_x) / n;
    J[i] = -rho * D[i] * m->W[i] * n * X_x;
    Jsum += J[i];
  }
  double qh = -kc * T_x;
  for (int i = 0; i < ns; ++i) {
    J[i] -= Y[i] * Jsum; /* correction velocity */
    qh += (m->hf[i] + m->cp[i] * (T - TREF)) / m->W[i] * J[i];
  }
  double tau = 4.0 / 3.0 * mu * u_x;
  fd[0] = tau;
  fd[1] = tau * u - qh;
  for (int i = 0; i < ns; ++i) fd[2 + i] = -J[i];
}

/* kind 0: local Lax-Friedrichs (Sec. 3.1), lambda = max(|u|+a) of both sides.
 * kind 1: HLLC (Toro 1994) with wave speeds S_L = min(u_L - a_L, u_R - a_R),
 *         S_R = max(u_L + a_L, u_R + a_R); species ride with the contact. */
void or_num_flux(const or_mech *m, int kind, const double *wl, const double *wr,
                 double *f) {
  int nv = m->ns + 2;
  double fl[MAXV], fr[MAXV];
  double rl, ul, Tl, Pl, al, rr, ur, Tr, Pr, ar;
  or_state(m, wl, &rl, &ul, &Tl, &Pl, &al);
  or_state(m, wr, &rr, &ur, &Tr, &Pr, &ar);
  or_phys_flux(m, wl, fl);
  or_phys_flux(m, wr, fr);
  if (kind == 0) {
    double lam = fmax(fabs(ul) + al, fabs(ur) + ar);
    for (int v = 0; v < nv; ++v) f[v] = 0.5 * (fl[v] + fr[v] - lam * (wr[v] - wl[v]));
    return;
  }
  double SL = fmin(ul - al, ur - ar);
  double SR = fmax(ul + al, ur + ar);
  double SM = (Pr - Pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) /
              (rl * (SL - ul) - rr * (SR - ur));
  if (0.0 <= SL) {
    for (int v = 0; v < nv; ++v) f[v] = fl[v];
  } else if (0.0 <= SM) {
    double coef = rl * (SL - ul) / (SL - SM);
    double us[MAXV];
    us[0] = coef * SM;
    us[1] = coef * (wl[1] / rl + (SM - ul) * (SM + Pl / (rl * (SL - ul))));
    for (int i = 0; i < m->ns; ++i) us[2 + i] = coef * (wl[2 + i] / rl);
    for (int v = 0; v < nv; ++v) f[v] = fl[v] + SL * (us[v] - wl[v]);
  } else if (0.0 <= SR) {
    double coef = rr * (SR - ur) / (SR - SM);
    double us[MAXV];
    us[0] = coef * SM;
    us[1] = coef * (wr[1] / rr + (SM - ur) * (SM + Pr / (rr * (SR - ur))));
    for (int i = 0; i < m->ns; ++i) us[2 + i] = coef * (wr[2 + i] / rr);
    for (int v = 0; v < nv; ++v) f[v] = fr[v] + SR * (us[v] - wr[v]);
  } else {
    for (int v = 0; v < nv; ++v) f[v] = fr[v];
  }
}

/* ------------------------------------------------------------------------- */
/* Eigenvectors of A = df^c/dw = R Lambda L, Lambda = diag(u-a, u, .., u, u+a)
 * (Sec. 3.3). Columns of R (variables rho u, rho E, rho Y_i):
 *   u -/+ a : (u -/+ a, H -/+ u a, Y_1..Y_ns),  H = (rho E + P)/rho
 *   u (species k): (u, u^2 - phi_k/(gamma-1), unit vector k),
 *     phi_k = dP/d(rho Y_k) = (gamma-1)(u^2/2 - e_k) + R_u T / W_k.
 * L is R^{-1}, by Gauss-Jordan elimination with partial pivoting. */
static int invert(int n, const double *Ain, double *X) {
  double A[MAXV * MAXV];
  memcpy(A, Ain, sizeof(double) * n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) X[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return -1;
    if (piv != c) {
      for (int j = 0; j < n; ++j) {
        double t = A[c * n + j];
        A[c * n + j] = A[piv * n + j];
        A[piv * n + j] = t;
        t = X[c * n + j];
        X[c * n + j] = X[piv * n + j];
        X[piv * n + j] = t;
      }
    }
    double d = A[c * n + c];
    for (int j = 0; j < n; ++j) {
      A[c * n + j] /= d;
      X[c * n + j] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[r * n + j] -= f * A[c * n + j];
        X[r * n + j] -= f * X[c * n + j];
      }
    }
  }
  return 0;
}

void or_eigen(const or_mech *m, const double *wbar, double *R, double *L, double *lam) {
  int ns = m->ns, nv = ns + 2;
  double rho, u, T, P, a;
  or_state(m, wbar, &rho, &u, &T, &P, &a);
  double cpm = 0.0, cvm = 0.0;
  for (int i = 0; i < ns; ++i) {
    cpm += wbar[2 + i] * m->cp[i] / m->W[i];
    cvm += wbar[2 + i] * (m->cp[i] - RU) / m->W[i];
  }
  double gm1 = cpm / cvm - 1.0;
  double H = (wbar[1] + P) / rho;
  for (int i = 0; i < nv * nv; ++i) R[i] = 0.0;
  /* column 0: u - a */
  R[0 * nv + 0] = u - a;
  R[1 * nv + 0] = H - u * a;
  for (int i = 0; i < ns; ++i) R[(2 + i) * nv + 0] = wbar[2 + i] / rho;
  /* column nv-1: u + a */
  R[0 * nv + nv - 1] = u + a;
  R[1 * nv + nv - 1] = H + u * a;
  for (int i = 0; i < ns; ++i) R[(2 + i) * nv + nv - 1] = wbar[2 + i] / rho;
  /* columns 1..ns: species waves */
  for (int k = 0; k < ns; ++k) {
    double ek = sp_e(m, k, T);
    double phik = gm1 * (0.5 * u * u - ek) + RU * T / m->W[k];
    R[0 * nv + 1 + k] = u;
    R[1 * nv + 1 + k] = u * u - phik / gm1;
    R[(2 + k) * nv + 1 + k] = 1.0;
  }
  invert(nv, R, L);
  lam[0] = u - a;
  for (int k = 0; k < ns; ++k) lam[1 + k] = u;
  lam[nv - 1] = u + a;
}

/* ------------------------------------------------------------------------- */
/* The scheme. */

struct or_ctx {
  or_cfg cfg;
  or_mech m;
  double *mbuf;          /* owned copies of the mechanism arrays */
  signed char *nubuf;
  double *probs;
  int nv, np1, ne, depth, npf;
  double dx;
  double xq[MAXQ], wq[MAXQ], Pq[MAXQ * MAXQ], dPq[MAXQ * MAXQ];
  double B[MAXQ * MAXQ], Sl[MAXQ * MAXQ], Sr[MAXQ * MAXQ];
  int *pf_left, *pf_right; /* per PE face: element on its left / right */
  int *face_pf;            /* per mesh face 0..ne: PE face id or -1 */
  int *elem_pf_right;      /* per element: PE face on its right or -1 */
  int *elem_pf_left;       /* per element: PE face on its left or -1 */
  int S;                 /* RK stages per step */
  double *w, *w0, *win, *wpre, *rhs, *fhat;
  double *dq;            /* LSERK register (2N storage) */
  double *qx;            /* LDG auxiliary variable q = dw/dx of the stage input */
  double *what;          /* [ne+1][nv] central face values of w for q */
  double *ring_in, *ring_pre; /* [depth][S][npf][2][nv*np1] */
  double *ring_q;        /* history of q of the PE-boundary elements, same layout */
  int64_t *ring_level;
  int *keff;
  /* subdomain (pe_end > 0): buffer elements at the cut sides, the whole domain's
   * index of local element 0, and the whole domain's number of local PE face f:
   * (f + face_base) mod npf_draw */
  int cut_l, cut_r, elem0, face_base, npf_draw;
  int64_t n;
  uint8_t *flags_last;
  int32_t *flag_count;
};

static double *ring_at(or_ctx *c, double *ring, int64_t level, int s, int pf, int side) {
  int slot = (int)(level % c->depth);
  size_t blk = (size_t)c->nv * c->np1;
  return ring + ((((size_t)slot * c->S + s) * c->npf + pf) * 2 + side) * blk;
}

/* Low-storage explicit RK in Williamson's 2N form (Sec. 3.1 cites Williamson
 * 1980 and Kennedy, Carpenter & Lewis 2000): per stage s,
 *   dq <- A_s dq + dt L(w),  w <- w + B_s dq,  at time t_n + C_s dt.
 * 1: Williamson's 3-stage 3rd-order scheme; 2: the 5-stage 4th-order scheme of
 * Carpenter & Kennedy (1994), the coefficients as published (rational
 * approximations of the optimised values). */
int or_rk_stages(int integrator) {
  return integrator == 1 ? 3 : integrator == 2 ? 5 : 3;
}

int or_lserk_coeffs(int integrator, double *A, double *B, double *C) {
  if (integrator == 1) {
    const double a[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
    const double b[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    const double cc[3] = {0.0, 1.0 / 3.0, 3.0 / 4.0};
    for (int s = 0; s < 3; ++s) {
      A[s] = a[s];
      B[s] = b[s];
      C[s] = cc[s];
    }
    return 3;
  }
  if (integrator == 2) {
    const double a[5] = {0.0, -567301805773.0 / 1357537059087.0,
                         -2404267990393.0 / 2016746695238.0,
                         -3550918686646.0 / 2091501179385.0,
                         -1275806237668.0 / 842570457699.0};
    const double b[5] = {1432997174477.0 / 9575080441755.0,
                         5161836677717.0 / 13612068292357.0,
                         1720146321549.0 / 2090206949498.0,
                         3134564353537.0 / 4481467310338.0,
                         2277821191437.0 / 14882151754819.0};
    const double cc[5] = {0.0, 1432997174477.0 / 9575080441755.0,
                          2526269341429.0 / 6820363962896.0,
                          2006345519317.0 / 3224310063776.0,
                          2802321613138.0 / 2924317926251.0};
    for (int s = 0; s < 5; ++s) {
      A[s] = a[s];
      B[s] = b[s];
      C[s] = cc[s];
    }
    return 5;
  }
  return 0;
}

or_ctx *or_create(const or_cfg *cfg, const or_mech *m) {
  if (cfg->p < 0 || cfg->p + 1 > MAXQ || m->ns + 2 > MAXV || cfg->n_elem < 1 ||
      cfg->n_pe < 1 || cfg->n_pe > cfg->n_elem || cfg->at_order < 1 ||
      (cfg->viscous && (!(cfg->mu_ref >= 0.0) || !(cfg->T_mu > 0.0) || !(cfg->prandtl > 0.0))) ||
      cfg->integrator < 0 || cfg->integrator > 2)
    return NULL;
  const int part = cfg->pe_end > 0 && !(cfg->pe_begin == 0 && cfg->pe_end == cfg->n_pe);
  if (cfg->pe_end > 0 && (cfg->pe_begin < 0 || cfg->pe_begin >= cfg->pe_end ||
                          cfg->pe_end > cfg->n_pe || (part && (cfg->viscous || cfg->face0))))
    return NULL;
  or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
  c->cfg = *cfg;
  int ns = m->ns, nr = m->nr;
  c->mbuf = (double *)malloc(sizeof(double) * (5 * ns + 3 * (nr > 0 ? nr : 1)));
  c->nubuf = (signed char *)malloc((size_t)2 * (nr > 0 ? nr : 1) * ns);
  double *mb = c->mbuf;
  memcpy(mb, m->W, sizeof(double) * ns);
  memcpy(mb + ns, m->cp, sizeof(double) * ns);
  memcpy(mb + 2 * ns, m->hf, sizeof(double) * ns);
  memcpy(mb + 3 * ns, m->s0, sizeof(double) * ns);
  if (nr > 0) {
    memcpy(mb + 4 * ns, m->A, sizeof(double) * nr);
    memcpy(mb + 4 * ns + nr, m->b, sizeof(double) * nr);
    memcpy(mb + 4 * ns + 2 * nr, m->Ea, sizeof(double) * nr);
    memcpy(c->nubuf, m->nu_f, (size_t)nr * ns);
    memcpy(c->nubuf + (size_t)nr * ns, m->nu_r, (size_t)nr * ns);
  }
  c->m.ns = ns;
  c->m.nr = nr;
  c->m.W = mb;
  c->m.cp = mb + ns;
  c->m.hf = mb + 2 * ns;
  c->m.s0 = mb + 3 * ns;
  c->m.A = mb + 4 * ns;
  c->m.b = mb + 4 * ns + nr;
  c->m.Ea = mb + 4 * ns + 2 * nr;
  {
    double *le = mb + 4 * ns + 3 * (nr > 0 ? nr : 1);
    for (int i = 0; i < ns; ++i) le[i] = m->Le ? m->Le[i] : 1.0;
    c->m.Le = le;
  }
  c->m.nu_f = c->nubuf;
  c->m.nu_r = c->nubuf + (size_t)nr * ns;
  c->probs = (double *)malloc(sizeof(double) * (cfg->max_delay + 1));
  for (int k = 0; k <= cfg->max_delay; ++k)
    c->probs[k] = (cfg->delay_mode == 2 && cfg->delay_probs) ? cfg->delay_probs[k] : 0.0;
  c->cfg.delay_probs = c->probs;

  c->nv = ns + 2;
  c->np1 = cfg->p + 1;
  c->ne = cfg->n_elem;
  c->dx = cfg->length / cfg->n_elem;
  /* a subdomain: PEs [pb, pe) own elements [E0, E1) of the whole domain's N
   * (PE k owns [floor(k N / P), floor((k+1) N / P))), plus a buffer element at
   * each cut side; the local mesh ends in outflow boundaries beyond the buffers
   * (their updates are discarded: the exchange overwrites them) */
  int pb = 0, pe = cfg->n_pe;
  if (part) {
    int64_t N = cfg->n_elem, P = cfg->n_pe;
    pb = cfg->pe_begin;
    pe = cfg->pe_end;
    int gper = (cfg->bc_left == 0);
    c->cut_l = (pb > 0 || gper);
    c->cut_r = (pe < P || gper);
    c->elem0 = (int)((pb * N) / P) - c->cut_l;
    c->ne = (int)((pe * N) / P - (pb * N) / P) + c->cut_l + c->cut_r;
    if (c->cut_l) c->cfg.bc_left = 2;
    if (c->cut_r) c->cfg.bc_right = 2;
  }
  c->depth = cfg->max_delay + cfg->at_order;
  c->S = or_rk_stages(cfg->integrator);
  int q = c->np1;
  or_gauss(q, c->xq, c->wq);
  for (int k = 0; k < q; ++k) {
    double P[MAXQ + 1], dP[MAXQ + 1];
    or_legendre(cfg->p, c->xq[k], P, dP);
    for (int j = 0; j < q; ++j) {
      c->Pq[k * q + j] = P[j];
      c->dPq[k * q + j] = dP[j];
    }
  }
  or_beta_matrix(cfg->p, c->B);
  or_shift_matrix(cfg->p, -1, c->Sl);
  or_shift_matrix(cfg->p, +1, c->Sr);

  /* PE partition (Sec. 4): PE k owns elements [floor(k N/P), floor((k+1) N/P)).
   * PE face k sits between PE k and PE k+1; with periodic boundaries the face
   * between the last and the first element is PE face P-1. */
  int P = cfg->n_pe, ne = c->ne;
  int periodic = (cfg->bc_left == 0);
  c->npf = (P > 1) ? (periodic ? P : P - 1) : 0;
  c->face_base = 0;
  c->npf_draw = c->npf;
  if (part) {
    /* the cut faces and the faces between the subdomain's own PEs, in order:
     * whole-domain faces pb - cut_l .. pe - 1 + cut_r - 1 (mod npf) */
    c->npf = c->cut_l + (pe - pb - 1) + c->cut_r;
    c->face_base = pb - c->cut_l;
  }
  c->pf_left = (int *)malloc(sizeof(int) * (c->npf > 0 ? c->npf : 1));
  c->pf_right = (int *)malloc(sizeof(int) * (c->npf > 0 ? c->npf : 1));
  c->face_pf = (int *)malloc(sizeof(int) * (ne + 1));
  c->elem_pf_right = (int *)malloc(sizeof(int) * ne);
  c->elem_pf_left = (int *)malloc(sizeof(int) * ne);
  for (int i = 0; i <= ne; ++i) c->face_pf[i] = -1;
  for (int e = 0; e < ne; ++e) c->elem_pf_right[e] = c->elem_pf_left[e] = -1;
  for (int k = 0; k < c->npf; ++k) {
    int first_next, face, el;
    if (part) {
      /* local face k is whole-domain face g = pb - cut_l + k, which sits left of
       * the first element of PE g + 1: the buffer element and the first owned
       * element for the left cut, the last owned element and the buffer for the
       * right cut */
      int g = pb - c->cut_l + k;
      if (c->cut_l && k == 0)
        first_next = 1;
      else if (c->cut_r && k == c->npf - 1)
        first_next = ne - 1;
      else
        first_next = (int)(((int64_t)(g + 1) * cfg->n_elem) / P) - c->elem0;
      face = first_next;
      el = face - 1;
    } else {
      first_next = (int)(((int64_t)((k + 1) % P) * ne) / P);
      face = (k == P - 1) ? 0 : first_next;
      el = (face == 0) ? ne - 1 : face - 1;
    }
    c->pf_left[k] = el;
    c->pf_right[k] = first_next;
    c->face_pf[face] = k;
    if (face == 0) c->face_pf[ne] = k;
    c->elem_pf_right[el] = k;
    c->elem_pf_left[first_next] = k;
  }
  size_t sz = (size_t)c->nv * ne * q;
  c->w = (double *)calloc(sz, sizeof(double));
  c->w0 = (double *)calloc(sz, sizeof(double));
  c->win = (double *)calloc(sz, sizeof(double));
  c->wpre = (double *)calloc(sz, sizeof(double));
  c->rhs = (double *)calloc(sz, sizeof(double));
  c->dq = (double *)calloc(sz, sizeof(double));
  c->qx = (double *)calloc(sz, sizeof(double));
  c->what = (double *)calloc((size_t)(ne + 1) * c->nv, sizeof(double));
  c->fhat = (double *)calloc((size_t)(ne + 1) * c->nv, sizeof(double));
  size_t rsz = (size_t)c->depth * c->S * (c->npf > 0 ? c->npf : 1) * 2 * c->nv * q;
  c->ring_in = (double *)calloc(rsz, sizeof(double));
  c->ring_pre = (double *)calloc(rsz, sizeof(double));
  c->ring_q = (double *)calloc(rsz, sizeof(double));
  c->ring_level = (int64_t *)malloc(sizeof(int64_t) * c->depth);
  for (int s = 0; s < c->depth; ++s) c->ring_level[s] = -1;
  c->keff = (int *)calloc(c->npf > 0 ? c->npf : 1, sizeof(int));
  c->flags_last = (uint8_t *)calloc((size_t)c->S * ne, 1);
  c->flag_count = (int32_t *)calloc(ne, sizeof(int32_t));
  c->n = 0;
  return c;
}

void or_destroy(or_ctx *c) {
  if (!c) return;
  free(c->mbuf);
  free(c->nubuf);
  free(c->probs);
  free(c->pf_left);
  free(c->pf_right);
  free(c->face_pf);
  free(c->elem_pf_right);
  free(c->elem_pf_left);
  free(c->w);
  free(c->w0);
  free(c->win);
  free(c->wpre);
  free(c->rhs);
  free(c->dq);
  free(c->qx);
  free(c->what);
  free(c->ring_q);
  free(c->fhat);
  free(c->ring_in);
  free(c->ring_pre);
  free(c->ring_level);
  free(c->keff);
  free(c->flags_last);
  free(c->flag_count);
  free(c);
}

#define W_(arr, v, e, j) (arr)[((size_t)(v) * c->ne + (e)) * c->np1 + (j)]

/* L2 projection of the primitive initial data given at the Gauss points
 * (prim layout [ns+3][ne][p+1]: T, P, u, Y_i): conserved values at the points,
 * then w_j = (2j+1)/2 sum_q w_q w(xi_q) P_j(xi_q). */
int or_set_primitive(or_ctx *c, const double *prim) {
  int ns = c->m.ns, nv = c->nv, q = c->np1, ne = c->ne;
  double Y[MAXV], wn[MAXQ][MAXV];
  for (int e = 0; e < ne; ++e) {
    for (int k = 0; k < q; ++k) {
      double T = prim[((size_t)0 * ne + e) * q + k];
      double P = prim[((size_t)1 * ne + e) * q + k];
      double u = prim[((size_t)2 * ne + e) * q + k];
      for (int i = 0; i < ns; ++i) Y[i] = prim[((size_t)(3 + i) * ne + e) * q + k];
      or_cons_from_prim(&c->m, T, P, u, Y, wn[k]);
    }
    for (int v = 0; v < nv; ++v)
      for (int j = 0; j < q; ++j) {
        double acc = 0.0;
        for (int k = 0; k < q; ++k) acc += c->wq[k] * wn[k][v] * c->Pq[k * q + j];
        W_(c->w, v, e, j) = 0.5 * (2.0 * j + 1.0) * acc;
      }
  }
  c->n = 0;
  for (int s = 0; s < c->depth; ++s) c->ring_level[s] = -1;
  memset(c->flag_count, 0, sizeof(int32_t) * ne);
  return 0;
}

int or_set_state(or_ctx *c, const double *w) {
  memcpy(c->w, w, sizeof(double) * c->nv * c->ne * c->np1);
  c->n = 0;
  for (int s = 0; s < c->depth; ++s) c->ring_level[s] = -1;
  memset(c->flag_count, 0, sizeof(int32_t) * c->ne);
  return 0;
}

int or_get_state(const or_ctx *c, double *w) {
  memcpy(w, c->w, sizeof(double) * c->nv * c->ne * c->np1);
  return 0;
}

int64_t or_steps_done(const or_ctx *c) { return c->n; }

int or_get_flags(const or_ctx *c, uint8_t *last, int32_t *count) {
  if (last) memcpy(last, c->flags_last, (size_t)c->S * c->ne);
  if (count) memcpy(count, c->flag_count, sizeof(int32_t) * c->ne);
  return 0;
}

/* trace of a modal element at xi = +1 (side 1) or -1 (side 0) */
static void trace_of(const or_ctx *c, const double *blk, int right, double *out) {
  for (int v = 0; v < c->nv; ++v) {
    double acc = 0.0;
    for (int j = 0; j < c->np1; ++j) {
      double s = (right || (j % 2 == 0)) ? 1.0 : -1.0;
      acc += s * blk[v * c->np1 + j];
    }
    out[v] = acc;
  }
}

static void elem_block(const or_ctx *c, const double *arr, int e, double *blk) {
  for (int v = 0; v < c->nv; ++v)
    for (int j = 0; j < c->np1; ++j) blk[v * c->np1 + j] = W_(arr, v, e, j);
}

/* boundary ghost of a trace: reflecting wall (u -> -u) or outflow (copy) */
static void ghost_trace(const or_ctx *c, int bc, const double *in, double *out) {
  for (int v = 0; v < c->nv; ++v) out[v] = in[v];
  if (bc == 1) out[0] = -in[0];
}

/* boundary ghost of a derivative trace: the x-derivative of the mirror image
 * (reflecting wall: d(rho u)/dx kept, the others negated) or a copy (outflow) */
static void ghost_qtrace(const or_ctx *c, int bc, const double *in, double *out) {
  for (int v = 0; v < c->nv; ++v) out[v] = (bc == 1 && v > 0) ? -in[v] : in[v];
}

/* The LDG auxiliary variable q = dw/dx (Sec. 3.1: evaluated like w with a
 * central flux) of the stage input, per element and mode:
 *   (dx / (2i+1)) q_i = w_hat_{e+1} - (-1)^i w_hat_e - sum_k omega_k w(xi_k) P_i'(xi_k),
 * w_hat the mean of the two traces at a face; at a PE face with delay k > 0 the
 * AT extrapolation (Eq. 7) of the means at the common delayed levels n-k-m; at a
 * physical boundary the mean with the ghost (reflecting wall: mirror image;
 * outflow: a copy, so the interior trace). */
static int aux_eval(or_ctx *c, const double *win, int s, int use_hist) {
  int nv = c->nv, q = c->np1, ne = c->ne;
  double blk[MAXV * MAXQ], wl[MAXV], wr[MAXV], g[MAXV], cm[16];
  int periodic = (c->cfg.bc_left == 0);
  for (int i = 0; i <= ne; ++i) {
    double *wh = c->what + (size_t)i * nv;
    if (periodic && i == ne) {
      memcpy(wh, c->what, sizeof(double) * nv);
      continue;
    }
    int pf = c->face_pf[i];
    int k = (use_hist && pf >= 0) ? c->keff[pf] : 0;
    if (k > 0) {
      int o = c->cfg.at_order;
      or_at_coeffs(o, k, cm);
      for (int v = 0; v < nv; ++v) wh[v] = 0.0;
      for (int mm = 0; mm < o; ++mm) {
        int64_t lv = c->n - k - mm;
        if (c->ring_level[lv % c->depth] != lv) return -3;
        trace_of(c, ring_at(c, c->ring_in, lv, s, pf, 0), 1, wl);
        trace_of(c, ring_at(c, c->ring_in, lv, s, pf, 1), 0, wr);
        for (int v = 0; v < nv; ++v) wh[v] += cm[mm] * 0.5 * (wl[v] + wr[v]);
      }
      continue;
    }
    if (i == 0 && !periodic) {
      elem_block(c, win, 0, blk);
      trace_of(c, blk, 0, wr);
      ghost_trace(c, c->cfg.bc_left, wr, g);
      for (int v = 0; v < nv; ++v) wh[v] = 0.5 * (g[v] + wr[v]);
    } else if (i == ne && !periodic) {
      elem_block(c, win, ne - 1, blk);
      trace_of(c, blk, 1, wl);
      ghost_trace(c, c->cfg.bc_right, wl, g);
      for (int v = 0; v < nv; ++v) wh[v] = 0.5 * (wl[v] + g[v]);
    } else {
      elem_block(c, win, (i == 0) ? ne - 1 : i - 1, blk);
      trace_of(c, blk, 1, wl);
      elem_block(c, win, i, blk);
      trace_of(c, blk, 0, wr);
      for (int v = 0; v < nv; ++v) wh[v] = 0.5 * (wl[v] + wr[v]);
    }
  }
  for (int e = 0; e < ne; ++e)
    for (int v = 0; v < nv; ++v)
      for (int i = 0; i < q; ++i) {
        double vol = 0.0;
        for (int k = 0; k < q; ++k) {
          double wk = 0.0;
          for (int j = 0; j < q; ++j) wk += W_(win, v, e, j) * c->Pq[k * q + j];
          vol += c->wq[k] * wk * c->dPq[k * q + i];
        }
        double sgn = (i % 2 == 0) ? 1.0 : -1.0;
        W_(c->qx, v, e, i) = (2.0 * i + 1.0) / c->dx *
                             (c->what[(size_t)(e + 1) * nv + v] - sgn * c->what[(size_t)e * nv + v] -
                              vol);
      }
  return 0;
}

static int check_state(const or_ctx *c, const double *w) {
  double rho = 0.0;
  for (int i = 0; i < c->m.ns; ++i) rho += w[2 + i];
  if (!(rho > 0.0) || !isfinite(w[0]) || !isfinite(w[1])) return -1;
  return 0;
}

/* Numerical flux of the total flux f = f^c - f^d (Sec. 3.1) between two traces:
 * the Riemann flux (LF or HLLC) of the convective part, minus the central mean of
 * the diffusive part in viscous runs. */
static void face_flux(const or_ctx *c, const double *wl, const double *ql, const double *wr,
                      const double *qr, double *fh) {
  or_num_flux(&c->m, c->cfg.flux, wl, wr, fh);
  if (!c->cfg.viscous) return;
  double dl[MAXV], dr[MAXV];
  or_visc_flux(&c->m, &c->cfg, wl, ql, dl);
  or_visc_flux(&c->m, &c->cfg, wr, qr, dr);
  for (int v = 0; v < c->nv; ++v) fh[v] -= 0.5 * (dl[v] + dr[v]);
}

/* Semi-discrete right-hand side (Eq. 5) of stage s at step level n:
 * dw_i/dt = (2i+1)/dx [ sum_q w_q f(xi_q) P_i'(xi_q) - fhat_{e+1} + (-1)^i fhat_e ]
 *           + (2i+1)/2 sum_q w_q s(xi_q) P_i(xi_q),
 * f = f^c - f^d(w, q) (q = c->qx in viscous runs).
 * At a PE face with delay k > 0 the flux is the AT flux (Eq. 7) of the fluxes at the
 * common delayed levels n-k-m (both sides of the face at the same level). */
static int rhs_eval(or_ctx *c, const double *win, int s, int use_hist) {
  int ns = c->m.ns, nv = c->nv, q = c->np1, ne = c->ne;
  const int visc = c->cfg.viscous;
  double wn[MAXV], f[MAXV], conc[MAXV], wdot[MAXV], qn[MAXV], fd[MAXV];
  double V[MAXV][MAXQ], Sv[MAXV][MAXQ];
  int err = 0;
  /* volume and source terms */
  for (int e = 0; e < ne; ++e) {
    for (int v = 0; v < nv; ++v)
      for (int i = 0; i < q; ++i) V[v][i] = Sv[v][i] = 0.0;
    for (int k = 0; k < q; ++k) {
      for (int v = 0; v < nv; ++v) {
        double acc = 0.0;
        for (int j = 0; j < q; ++j) acc += W_(win, v, e, j) * c->Pq[k * q + j];
        wn[v] = acc;
      }
      if (check_state(c, wn)) err = -1;
      double rho, u, T, P, a;
      or_state(&c->m, wn, &rho, &u, &T, &P, &a);
      if (!(T > 0.0) || !isfinite(T)) err = -1;
      or_phys_flux(&c->m, wn, f);
      if (visc) {
        for (int v = 0; v < nv; ++v) {
          double acc = 0.0;
          for (int j = 0; j < q; ++j) acc += W_(c->qx, v, e, j) * c->Pq[k * q + j];
          qn[v] = acc;
        }
        or_visc_flux(&c->m, &c->cfg, wn, qn, fd);
        for (int v = 0; v < nv; ++v) f[v] -= fd[v];
      }
      /* law of mass action on non-negative concentrations: the polynomial of a
       * trace species may dip below zero at a Gauss point */
      for (int i = 0; i < ns; ++i) conc[i] = fmax(wn[2 + i], 0.0) / c->m.W[i];
      or_wdot(&c->m, T, conc, wdot);
      for (int i = 0; i < q; ++i)
        for (int v = 0; v < nv; ++v) {
          V[v][i] += c->wq[k] * f[v] * c->dPq[k * q + i];
          double src = (v >= 2) ? c->m.W[v - 2] * wdot[v - 2] : 0.0;
          Sv[v][i] += c->wq[k] * src * c->Pq[k * q + i];
        }
    }
    for (int v = 0; v < nv; ++v)
      for (int i = 0; i < q; ++i) {
        W_(c->rhs, v, e, i) = V[v][i];
        W_(c->wpre, v, e, i) = 0.5 * (2.0 * i + 1.0) * Sv[v][i]; /* projected source */
      }
  }
  /* face fluxes */
  double blk[MAXV * MAXQ], wl[MAXV], wr[MAXV], g[MAXV], fa[MAXV], cm[16];
  double ql[MAXV], qr[MAXV], qg[MAXV];
  int periodic = (c->cfg.bc_left == 0);
  for (int i = 0; i <= ne; ++i) {
    double *fh = c->fhat + (size_t)i * nv;
    if (periodic && i == ne) {
      memcpy(fh, c->fhat, sizeof(double) * nv);
      continue;
    }
    int pf = c->face_pf[i];
    int k = (use_hist && pf >= 0) ? c->keff[pf] : 0;
    if (k > 0) {
      int o = c->cfg.at_order;
      or_at_coeffs(o, k, cm);
      for (int v = 0; v < nv; ++v) fh[v] = 0.0;
      for (int mm = 0; mm < o; ++mm) {
        int64_t lv = c->n - k - mm;
        double *bl = ring_at(c, c->ring_in, lv, s, pf, 0);
        double *br = ring_at(c, c->ring_in, lv, s, pf, 1);
        if (c->ring_level[lv % c->depth] != lv) return -3;
        trace_of(c, bl, 1, wl);
        trace_of(c, br, 0, wr);
        if (visc) {
          trace_of(c, ring_at(c, c->ring_q, lv, s, pf, 0), 1, ql);
          trace_of(c, ring_at(c, c->ring_q, lv, s, pf, 1), 0, qr);
        }
        face_flux(c, wl, ql, wr, qr, fa);
        for (int v = 0; v < nv; ++v) fh[v] += cm[mm] * fa[v];
      }
      continue;
    }
    if (i == 0 && !periodic) {
      elem_block(c, win, 0, blk);
      trace_of(c, blk, 0, wr);
      ghost_trace(c, c->cfg.bc_left, wr, g);
      if (visc) {
        elem_block(c, c->qx, 0, blk);
        trace_of(c, blk, 0, qr);
        ghost_qtrace(c, c->cfg.bc_left, qr, qg);
      }
      face_flux(c, g, qg, wr, qr, fh);
    } else if (i == ne && !periodic) {
      elem_block(c, win, ne - 1, blk);
      trace_of(c, blk, 1, wl);
      ghost_trace(c, c->cfg.bc_right, wl, g);
      if (visc) {
        elem_block(c, c->qx, ne - 1, blk);
        trace_of(c, blk, 1, ql);
        ghost_qtrace(c, c->cfg.bc_right, ql, qg);
      }
      face_flux(c, wl, ql, g, qg, fh);
    } else {
      int el = (i == 0) ? ne - 1 : i - 1;
      elem_block(c, win, el, blk);
      trace_of(c, blk, 1, wl);
      elem_block(c, win, i, blk);
      trace_of(c, blk, 0, wr);
      if (visc) {
        elem_block(c, c->qx, el, blk);
        trace_of(c, blk, 1, ql);
        elem_block(c, c->qx, i, blk);
        trace_of(c, blk, 0, qr);
      }
      face_flux(c, wl, ql, wr, qr, fh);
    }
  }
  /* assembly: rhs <- (2i+1)/dx (V_i - fhat_{e+1} + (-1)^i fhat_e) + source_i */
  for (int e = 0; e < ne; ++e)
    for (int v = 0; v < nv; ++v)
      for (int i = 0; i < q; ++i) {
        double sgn = (i % 2 == 0) ? 1.0 : -1.0;
        double surf = W_(c->rhs, v, e, i) - c->fhat[(size_t)(e + 1) * nv + v] +
                      sgn * c->fhat[(size_t)e * nv + v];
        W_(c->rhs, v, e, i) = (2.0 * i + 1.0) / c->dx * surf + W_(c->wpre, v, e, i);
      }
  return err;
}

static double minmod3(double a, double b, double d) {
  if (a > 0.0 && b > 0.0 && d > 0.0) return fmin(a, fmin(b, d));
  if (a < 0.0 && b < 0.0 && d < 0.0) return fmax(a, fmax(b, d));
  return 0.0;
}

/* Neighbour (modal block) of element e on side dir (-1 left, +1 right), taken from
 * the pre-limit field `arr`; across a PE face with delay k > 0 it is the AT
 * extrapolation (Eq. 11) of the neighbour's pre-limit values at levels n-k-m;
 * at a physical boundary it is the ghost element (outflow: a copy; reflecting:
 * the mirror image with the momentum negated). */
static int neighbour(or_ctx *c, const double *arr, int e, int dir, int s, double *blk) {
  int ne = c->ne, nv = c->nv, q = c->np1;
  int periodic = (c->cfg.bc_left == 0);
  int pf = (dir > 0) ? c->elem_pf_right[e] : c->elem_pf_left[e];
  if (pf >= 0 && c->keff[pf] > 0) {
    int k = c->keff[pf], o = c->cfg.at_order;
    double cm[16];
    or_at_coeffs(o, k, cm);
    int side = (dir > 0) ? 1 : 0;
    for (int t = 0; t < nv * q; ++t) blk[t] = 0.0;
    for (int mm = 0; mm < o; ++mm) {
      int64_t lv = c->n - k - mm;
      if (c->ring_level[lv % c->depth] != lv) return -3;
      double *src = ring_at(c, c->ring_pre, lv, s, pf, side);
      for (int t = 0; t < nv * q; ++t) blk[t] += cm[mm] * src[t];
    }
    return 0;
  }
  int nb = e + dir;
  if (nb >= 0 && nb < ne) {
    elem_block(c, arr, nb, blk);
    return 0;
  }
  if (periodic) {
    elem_block(c, arr, (nb + ne) % ne, blk);
    return 0;
  }
  int bc = (dir < 0) ? c->cfg.bc_left : c->cfg.bc_right;
  elem_block(c, arr, e, blk);
  if (bc == 1) {
    for (int v = 0; v < nv; ++v)
      for (int j = 0; j < q; ++j) {
        double sg = (j % 2 == 0) ? 1.0 : -1.0;
        if (v == 0) sg = -sg;
        blk[v * q + j] *= sg;
      }
  }
  return 0;
}

/* Troubled-cell indicator and WENO limiter (Sec. 3.3, Eq. 9-11).
 * Indicator (reading of "TVD slope limiters as in Zhong-Shu"): in each
 * characteristic field of L(wbar_e), the face deviations v(+1)-vbar and
 * vbar-v(-1) are passed through the TVB-modified minmod with the neighbours'
 * average differences; the cell is troubled if any deviation is modified.
 * The paper's criterion is TVD (M = 0) and has no threshold; deviations below
 * 1e-10 of the field's magnitude sum_v |L_kv| sigma_v count as zero, with
 * sigma = (rho a + |rho u|, |rho E|, rho, .., rho) of the cell average. That is
 * a rounding guard only: double-precision data that is flat up to rounding has
 * deviations of about 1e-16 of that magnitude times the conditioning of the
 * characteristic transform, far below it, so flat data never flags a cell on
 * the strength of its rounding.
 * Limiter: v_lim = w_-1 vt_{e-1} + w_0 v_e + w_1 vt_{e+1} with vt = the neighbour
 * polynomial on Omega_e with its mean there replaced by the mean of v_e; linear
 * weights (0.001, 0.998, 0.001), eps = 1e-6; w_lim = R v_lim on modes >= 1, the
 * cell average is kept. */
static int limit_stage(or_ctx *c, int s, uint8_t *flags) {
  int nv = c->nv, q = c->np1, ne = c->ne;
  const double gam[3] = {0.001, 0.998, 0.001};
  const double eps = 1e-6;
  const double tau = 1e-10;
  double R[MAXV * MAXV], L[MAXV * MAXV], lam[MAXV];
  double own[MAXV * MAXQ], nbl[MAXV * MAXQ], nbr[MAXV * MAXQ];
  double shl[MAXV * MAXQ], shr[MAXV * MAXQ];
  double vo[MAXV * MAXQ], vl[MAXV * MAXQ], vr[MAXV * MAXQ], vlim[MAXV * MAXQ];
  double wbar[MAXV], wp[MAXV], wm[MAXV];
  double tvb = c->cfg.tvb_M * c->dx * c->dx;
  /* the limited field goes to c->win; neighbours are read from c->wpre */
  memcpy(c->win, c->wpre, sizeof(double) * nv * ne * q);
  for (int e = 0; e < ne; ++e) {
    elem_block(c, c->wpre, e, own);
    if (neighbour(c, c->wpre, e, -1, s, nbl)) return -3;
    if (neighbour(c, c->wpre, e, +1, s, nbr)) return -3;
    for (int v = 0; v < nv; ++v) wbar[v] = own[v * q];
    if (check_state(c, wbar)) return -1;
    or_eigen(&c->m, wbar, R, L, lam);
    trace_of(c, own, 1, wp);
    trace_of(c, own, 0, wm);
    /* per-variable magnitudes for the noise floor: momentum on the scale of
     * rho a + |rho u|, energy on |rho E|, every partial density on rho */
    double sig[MAXV];
    {
      double rho = 0.0;
      for (int i = 0; i < c->m.ns; ++i) rho += wbar[2 + i];
      double a = fmax(fabs(lam[nv - 1] - lam[0]) * 0.5, 0.0);
      sig[0] = rho * a + fabs(wbar[0]);
      sig[1] = fabs(wbar[1]);
      for (int i = 0; i < c->m.ns; ++i) sig[2 + i] = rho;
    }
    int troubled = 0;
    for (int k = 0; k < nv && !troubled; ++k) {
      double vb = 0, vp = 0, vm = 0, vR = 0, vL = 0, scale = 0;
      for (int v = 0; v < nv; ++v) {
        double l = L[k * nv + v];
        vb += l * wbar[v];
        vp += l * wp[v];
        vm += l * wm[v];
        vR += l * nbr[v * q];
        vL += l * nbl[v * q];
        scale += fabs(l) * sig[v];
      }
      double ut = vp - vb, utt = vb - vm, dp = vR - vb, dm = vb - vL;
      double fl = tau * scale;
      if (fabs(ut) > fl && fabs(ut) > tvb && minmod3(ut, dp, dm) != ut) troubled = 1;
      if (fabs(utt) > fl && fabs(utt) > tvb && minmod3(utt, dp, dm) != utt) troubled = 1;
    }
    flags[e] = (uint8_t)troubled;
    if (!troubled || !c->cfg.limiter) continue;
    /* neighbours continued into Omega_e */
    for (int v = 0; v < nv; ++v)
      for (int i = 0; i < q; ++i) {
        double al = 0, ar = 0;
        for (int j = 0; j < q; ++j) {
          al += c->Sl[i * q + j] * nbl[v * q + j];
          ar += c->Sr[i * q + j] * nbr[v * q + j];
        }
        shl[v * q + i] = al;
        shr[v * q + i] = ar;
      }
    for (int k = 0; k < nv; ++k)
      for (int i = 0; i < q; ++i) {
        double a0 = 0, al = 0, ar = 0;
        for (int v = 0; v < nv; ++v) {
          a0 += L[k * nv + v] * own[v * q + i];
          al += L[k * nv + v] * shl[v * q + i];
          ar += L[k * nv + v] * shr[v * q + i];
        }
        vo[k * q + i] = a0;
        vl[k * q + i] = al;
        vr[k * q + i] = ar;
      }
    for (int k = 0; k < nv; ++k) {
      vl[k * q] = vo[k * q];
      vr[k * q] = vo[k * q];
      double be[3] = {0, 0, 0};
      const double *vv[3] = {vl + k * q, vo + k * q, vr + k * q};
      for (int t = 0; t < 3; ++t)
        for (int i = 0; i < q; ++i)
          for (int j = 0; j < q; ++j) be[t] += vv[t][i] * c->B[i * q + j] * vv[t][j];
      double wt[3], sw = 0;
      for (int t = 0; t < 3; ++t) {
        wt[t] = gam[t] / ((eps + be[t]) * (eps + be[t]));
        sw += wt[t];
      }
      for (int t = 0; t < 3; ++t) wt[t] /= sw;
      vlim[k * q] = vo[k * q];
      for (int i = 1; i < q; ++i)
        vlim[k * q + i] = wt[0] * vl[k * q + i] + wt[1] * vo[k * q + i] + wt[2] * vr[k * q + i];
    }
    for (int v = 0; v < nv; ++v)
      for (int i = 1; i < q; ++i) {
        double acc = 0;
        for (int k = 0; k < nv; ++k) acc += R[v * nv + k] * vlim[k * q + i];
        W_(c->win, v, e, i) = acc;
      }
  }
  return 0;
}

/* One step of SSP-RK3 (Shu-Osher form) with limiting after every stage:
 *   w1 = w0 + dt L(w0);  w2 = 3/4 w0 + 1/4 (w1 + dt L(w1));
 *   w^{n+1} = 1/3 w0 + 2/3 (w2 + dt L(w2)),
 * or of an LSERK scheme (or_lserk_coeffs) with limiting after every stage:
 *   dq = A_s dq + dt L(w_s),  w_{s+1} = w_s + B_s dq.
 * Stage s of step n reads stage s of the delayed steps (one delay per PE face per
 * step, common to both sides and to all stages: CAA skips the exchange of every
 * intermediate stage of a delayed step, Sec. 4.1; synchronous until the history
 * holds the levels the AT stencil needs). The step is split into its stages'
 * halves (or_stage) so that a subdomain can exchange its boundary elements
 * between them. */

/* the whole domain's number of local PE face f (the SAA draws use it) */
static int face_number(const or_ctx *c, int f) {
  if (c->npf_draw <= 0) return f;
  int g = (f + c->face_base) % c->npf_draw;
  return g < 0 ? g + c->npf_draw : g;
}

static void step_begin(or_ctx *c) {
  size_t sz = (size_t)c->nv * c->ne * c->np1;
  int64_t n = c->n;
  for (int f = 0; f < c->npf; ++f) {
    int k = or_delay(&c->cfg, n, face_number(c, f));
    c->keff[f] = (n >= (int64_t)k + c->cfg.at_order - 1) ? k : 0;
  }
  c->ring_level[(int)(n % c->depth)] = n;
  memcpy(c->w0, c->w, sizeof(double) * sz);
  memcpy(c->win, c->w, sizeof(double) * sz);
}

/* half 0 of stage s: history of the stage input, L(w_s), the pre-limit output
 * and its history */
static int stage_rhs(or_ctx *c, int s) {
  int ne = c->ne;
  size_t sz = (size_t)c->nv * ne * c->np1;
  double dt = c->cfg.dt;
  int64_t n = c->n;
  double lsA[5], lsB[5], lsC[5];
  const int lserk = or_lserk_coeffs(c->cfg.integrator, lsA, lsB, lsC) > 0;
  /* history of the stage input (for the AT flux) */
  for (int f = 0; f < c->npf; ++f) {
    elem_block(c, c->win, c->pf_left[f], ring_at(c, c->ring_in, n, s, f, 0));
    elem_block(c, c->win, c->pf_right[f], ring_at(c, c->ring_in, n, s, f, 1));
  }
  if (c->cfg.viscous) {
    /* the auxiliary variable of the stage input, and its history */
    int aerr = aux_eval(c, c->win, s, 1);
    if (aerr) return aerr;
    for (int f = 0; f < c->npf; ++f) {
      elem_block(c, c->qx, c->pf_left[f], ring_at(c, c->ring_q, n, s, f, 0));
      elem_block(c, c->qx, c->pf_right[f], ring_at(c, c->ring_q, n, s, f, 1));
    }
  }
  int err = rhs_eval(c, c->win, s, 1);
  if (err) return err;
  for (size_t t = 0; t < sz; ++t) {
    double r = c->rhs[t];
    if (lserk) {
      c->dq[t] = lsA[s] * c->dq[t] + dt * r;
      c->wpre[t] = c->win[t] + lsB[s] * c->dq[t];
    } else if (s == 0)
      c->wpre[t] = c->w0[t] + dt * r;
    else if (s == 1)
      c->wpre[t] = 0.75 * c->w0[t] + 0.25 * (c->win[t] + dt * r);
    else
      c->wpre[t] = (1.0 / 3.0) * c->w0[t] + (2.0 / 3.0) * (c->win[t] + dt * r);
  }
  /* history of the pre-limit stage output (for the AT-WENO stencil) */
  for (int f = 0; f < c->npf; ++f) {
    elem_block(c, c->wpre, c->pf_left[f], ring_at(c, c->ring_pre, n, s, f, 0));
    elem_block(c, c->wpre, c->pf_right[f], ring_at(c, c->ring_pre, n, s, f, 1));
  }
  return 0;
}

/* half 1 of stage s: the limited stage output becomes the next stage input */
static int stage_limit(or_ctx *c, int s) {
  int ne = c->ne;
  size_t sz = (size_t)c->nv * ne * c->np1;
  if (c->cfg.limiter) {
    int err = limit_stage(c, s, c->flags_last + (size_t)s * ne);
    if (err) return err;
    for (int e = 0; e < ne; ++e) c->flag_count[e] += c->flags_last[(size_t)s * ne + e];
  } else {
    memcpy(c->win, c->wpre, sizeof(double) * sz);
    memset(c->flags_last + (size_t)s * ne, 0, ne);
  }
  return 0;
}

static void step_end(or_ctx *c) {
  memcpy(c->w, c->win, sizeof(double) * (size_t)c->nv * c->ne * c->np1);
  c->n += 1;
}

int or_stage(or_ctx *c, int s, int half) {
  if (s < 0 || s >= c->S || half < 0 || half > 1) return -2;
  if (half == 0) {
    if (s == 0) step_begin(c);
    return stage_rhs(c, s);
  }
  int err = stage_limit(c, s);
  if (err) return err;
  if (s == c->S - 1) step_end(c);
  return 0;
}

int or_step(or_ctx *c, int n_steps) {
  for (int it = 0; it < n_steps; ++it)
    for (int s = 0; s < c->S; ++s)
      for (int half = 0; half < 2; ++half) {
        int err = or_stage(c, s, half);
        if (err) return err;
      }
  return 0;
}

int or_part_layout(const or_ctx *c, int *n_local, int *elem0, int *cut_left, int *cut_right) {
  if (n_local) *n_local = c->ne;
  if (elem0) *elem0 = c->elem0;
  if (cut_left) *cut_left = c->cut_l;
  if (cut_right) *cut_right = c->cut_r;
  return 0;
}

int or_part_block(or_ctx *c, int what, int side, int s, double *blk, int import) {
  if (what < 0 || what > 1 || side < 0 || side > 1 || s < 0 || s >= c->S) return -2;
  if (!(side == 0 ? c->cut_l : c->cut_r)) return -2;
  int nv = c->nv, q = c->np1;
  /* the stage input of stage 0 is the state at the start of the step */
  double *arr = (what == 1) ? c->wpre : (s == 0) ? c->w : c->win;
  int e = import ? (side == 0 ? 0 : c->ne - 1) : (side == 0 ? 1 : c->ne - 2);
  if (!import) {
    elem_block(c, arr, e, blk);
    return 0;
  }
  for (int v = 0; v < nv; ++v)
    for (int j = 0; j < q; ++j) W_(arr, v, e, j) = blk[v * q + j];
  if (what == 1) {
    /* the buffer side of the cut face's pre-limit history */
    int pf = (side == 0) ? 0 : c->npf - 1;
    memcpy(ring_at(c, c->ring_pre, c->n, s, pf, side), blk, sizeof(double) * nv * q);
  }
  return 0;
}

/* Temperature at every Gauss point of the current state, layout [ne][p+1]. */
int or_get_temperature(const or_ctx *c, double *T) {
  int nv = c->nv, q = c->np1, ne = c->ne;
  double wn[MAXV];
  for (int e = 0; e < ne; ++e)
    for (int k = 0; k < q; ++k) {
      for (int v = 0; v < nv; ++v) {
        double acc = 0.0;
        for (int j = 0; j < q; ++j) acc += W_(c->w, v, e, j) * c->Pq[k * q + j];
        wn[v] = acc;
      }
      double rho, u, t, P, a;
      or_state(&c->m, wn, &rho, &u, &t, &P, &a);
      T[(size_t)e * q + k] = t;
    }
  return 0;
}

/* One synchronous right-hand side of Eq. (5), for tests. */
int or_rhs_sync(const or_cfg *cfg, const or_mech *m, const double *w, double *rhs) {
  or_ctx *c = or_create(cfg, m);
  if (!c) return -2;
  size_t sz = (size_t)c->nv * c->ne * c->np1;
  memcpy(c->win, w, sizeof(double) * sz);
  int err = c->cfg.viscous ? aux_eval(c, c->win, 0, 0) : 0;
  if (!err) err = rhs_eval(c, c->win, 0, 0);
  memcpy(rhs, c->rhs, sizeof(double) * sz);
  or_destroy(c);
  return err;
}

/* The troubled-cell indicator and WENO limiter of Sec. 3.3 applied once to a
 * state (no delays: every neighbour is the adjacent element or a boundary
 * ghost), for tests: flags[n_elem] gets the indicator's decision, wout the
 * limited state (equal to w where the cell is not troubled or cfg->limiter is
 * off). */
int or_limit_sync(const or_cfg *cfg, const or_mech *m, const double *w, double *wout,
                  uint8_t *flags) {
  or_ctx *c = or_create(cfg, m);
  if (!c) return -2;
  size_t sz = (size_t)c->nv * c->ne * c->np1;
  memcpy(c->wpre, w, sizeof(double) * sz);
  int err = limit_stage(c, 0, flags);
  memcpy(wout, c->win, sizeof(double) * sz);
  or_destroy(c);
  return err;
}

/* The LDG auxiliary variable of a state, for tests (no delays). */
int or_aux_sync(const or_cfg *cfg, const or_mech *m, const double *w, double *qout) {
  or_ctx *c = or_create(cfg, m);
  if (!c) return -2;
  size_t sz = (size_t)c->nv * c->ne * c->np1;
  memcpy(c->win, w, sizeof(double) * sz);
  int err = aux_eval(c, c->win, 0, 0);
  memcpy(qout, c->qx, sizeof(double) * sz);
  or_destroy(c);
  return err;
}

/* Constant-volume, adiabatic, homogeneous reactor (no flow): d(rho Y_i)/dt =
 * W_i omega_i with rho e fixed, integrated with the same SSP-RK3 stages. */
int or_reactor0d(const or_mech *m, double *r, double rhoe, double dt, int n_steps) {
  int ns = m->ns;
  double r0[MAXV], r1[MAXV], k[MAXV], conc[MAXV], wd[MAXV];
  for (int it = 0; it < n_steps; ++it) {
    for (int i = 0; i < ns; ++i) r0[i] = r[i];
    for (int s = 0; s < 3; ++s) {
      double T;
      if (or_temperature(m, r, rhoe, 1000.0, &T) < 0) return -1;
      for (int i = 0; i < ns; ++i) conc[i] = fmax(r[i], 0.0) / m->W[i];
      or_wdot(m, T, conc, wd);
      for (int i = 0; i < ns; ++i) k[i] = m->W[i] * wd[i];
      for (int i = 0; i < ns; ++i) {
        if (s == 0)
          r1[i] = r0[i] + dt * k[i];
        else if (s == 1)
          r1[i] = 0.75 * r0[i] + 0.25 * (r[i] + dt * k[i]);
        else
          r1[i] = (1.0 / 3.0) * r0[i] + (2.0 / 3.0) * (r[i] + dt * k[i]);
      }
      for (int i = 0; i < ns; ++i) r[i] = r1[i];
    }
  }
  return 0;
}
