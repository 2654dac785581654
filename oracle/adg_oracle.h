/* Plain FP64 CPU oracle of the asynchronous discontinuous Galerkin (ADG) scheme
 * for the 1D reacting Euler equations (arXiv 2501.01747).
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA path: only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code with the CUDA library (no headers, helpers or tables).
 *
 * Conventions (the oracle's own; the C-ABI of the CUDA library is separate):
 *   state w: modal Legendre coefficients, layout [nv][n_elem][p+1], nv = ns + 2,
 *   variable 0 = rho*u, 1 = rho*E, 2+i = rho*Y_i. Density is the sum of the
 *   partial densities.
 */
#ifndef ADG_ORACLE_H
#define ADG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int ns, nr;
  const double *W, *cp, *hf, *s0;  /* [ns] kg/mol, J/mol/K, J/mol, J/mol/K */
  const signed char *nu_f, *nu_r;  /* [nr][ns] */
  const double *A, *b, *Ea;        /* [nr] SI, -, J/mol */
  const double *Le;                /* [ns] Lewis numbers (viscous runs; NULL: all 1) */
} or_mech;

typedef struct {
  int n_elem, p, n_pe;
  double x0, length, dt;
  int bc_left, bc_right; /* 0 periodic, 1 reflecting, 2 outflow */
  int flux;              /* 0 local Lax-Friedrichs, 1 HLLC */
  int limiter;           /* 0 none, 1 WENO (AT-WENO at delayed PE faces) */
  int at_order;          /* >= 1 */
  int delay_mode;        /* 0 synchronous, 1 CAA, 2 SAA */
  int max_delay;
  const double *delay_probs; /* [max_delay+1] (SAA) */
  uint64_t seed;
  double tvb_M;
  int integrator;        /* 0 SSP-RK3 (Shu-Osher), 1 LSERK 3-stage 3rd order
                            (Williamson 1980), 2 LSERK 5-stage 4th order
                            (Carpenter-Kennedy, 2N storage) */
  int viscous;           /* 0 Euler; 1 with the diffusive flux f^d (Sec. 2, LDG) */
  double mu_ref, T_mu, mu_exp, prandtl; /* mu = mu_ref (T/T_mu)^mu_exp, k = mu cp/Pr */
  int face0;             /* number of the first PE face in the SAA draws (0; a window
                            of a larger run passes the larger run's number of its
                            first PE face, so both draw the same delays) */
  int pe_begin, pe_end;  /* 0, 0: the whole domain. pe_end > 0: the subdomain of PEs
                            [pe_begin, pe_end) of the domain the other fields
                            describe (n_elem, n_pe, length, bcs of the whole), with a
                            buffer element at each side that borders another
                            subdomain (see or_part_layout) */
} or_cfg;

typedef struct or_ctx or_ctx;

/* quadrature and basis */
void or_legendre(int n, double x, double *P, double *dP);
int or_gauss(int q, double *x, double *w);
/* stages of an integrator, and the 2N-storage coefficients A_s, B_s, C_s of an
 * LSERK scheme (returns the number of stages, 0 for SSP-RK3) */
int or_rk_stages(int integrator);
int or_lserk_coeffs(int integrator, double *A, double *B, double *C);
/* AT coefficients c_m(k), m = 0..order-1 (Eq. 7-8) */
void or_at_coeffs(int order, int k, double *c);
int or_delay(const or_cfg *cfg, int64_t step, int face);
uint64_t or_splitmix64(uint64_t x);

/* thermo and kinetics */
int or_temperature(const or_mech *m, const double *r, double rhoe, double Tguess,
                   double *T);
void or_state(const or_mech *m, const double *w, double *rho, double *u, double *T,
              double *P, double *a);
void or_cons_from_prim(const or_mech *m, double T, double P, double u, const double *Y,
                       double *w);
void or_rates(const or_mech *m, double T, int j, double *kf, double *Kc);
void or_wdot(const or_mech *m, double T, const double *conc, double *wdot);
void or_phys_flux(const or_mech *m, const double *w, double *f);
void or_num_flux(const or_mech *m, int kind, const double *wl, const double *wr,
                 double *f);
void or_eigen(const or_mech *m, const double *wbar, double *R, double *L, double *lam);
/* transport (mu, k, D_i) and the diffusive flux f^d(w, q) at one point, q = dw/dx */
void or_transport(const or_mech *m, const or_cfg *cfg, double rho, double T, const double *Y,
                  double *mu, double *kc, double *D);
void or_visc_flux(const or_mech *m, const or_cfg *cfg, const double *w, const double *q,
                  double *fd);

/* DG tables for degree p (shift: neighbour polynomial continued into the cell) */
void or_beta_matrix(int p, double *B);
void or_shift_matrix(int p, int dir, double *S);

/* full scheme */
or_ctx *or_create(const or_cfg *cfg, const or_mech *m);
void or_destroy(or_ctx *c);
int or_set_primitive(or_ctx *c, const double *prim);
int or_set_state(or_ctx *c, const double *w);
int or_get_state(const or_ctx *c, double *w);
int or_step(or_ctx *c, int n_steps);
int64_t or_steps_done(const or_ctx *c);
/* troubled-cell flags: stages of the last step [stages][n_elem] and per-element count */
int or_get_flags(const or_ctx *c, uint8_t *last, int32_t *count);
int or_get_temperature(const or_ctx *c, double *T);

/* Domain decomposition (Sec. 3.1: the subdomains of the PEs exchange the DoFs of
 * their boundary elements with the buffer elements of their neighbours; Sec. 3.2:
 * the buffers may hold delayed levels, the flux uses the common delayed level;
 * Sec. 3.3: the limiter's neighbours are exchanged after every stage; Sec. 4:
 * CAA and SAA decide the delays). A context made with pe_end > 0 holds the
 * subdomain's elements plus one buffer element at each cut side (a side that
 * borders another subdomain): local element 0 and/or n_local - 1. Its PE faces
 * are the subdomain's own plus the cut faces, with the delays of the whole
 * domain's face numbers, and dx is the whole domain's. The buffer elements are
 * computed like the others, but their data is overwritten by the exchange
 * before it is used, so the owned elements follow the whole-domain scheme
 * exactly. Viscous subdomains are not supported (NULL from or_create).
 *
 * or_part_layout: n_local elements, global index of local element 0, and which
 * sides are cut. */
int or_part_layout(const or_ctx *c, int *n_local, int *elem0, int *cut_left, int *cut_right);
/* One half of RK stage s of the current step: half 0 (at s = 0 it first starts
 * the step: delays, history level, w0) the history writes of the stage input and
 * the right-hand side, giving the pre-limit output; half 1 the limiter (or the
 * copy without one), and at the last stage the end of the step. or_step(c, 1) is
 * the same sequence without the exchange calls in between. */
int or_stage(or_ctx *c, int s, int half);
/* The exchange at one side (0 left, 1 right) for stage s, one block [nv][p+1]:
 * what 0 = the stage input (at s = 0 the state at the start of the step), what 1
 * = the pre-limit output of stage s. Export (import = 0) copies the owned
 * boundary element of that side into blk; import (1) writes blk into that side's
 * buffer element, and for what 1 also into the history of the cut face. The
 * order per stage: import what 0 before half 0, import what 1 between half 0 and
 * half 1. -2 for a side that is not cut. */
int or_part_block(or_ctx *c, int what, int side, int s, double *blk, int import);
/* one synchronous right-hand side L(w) (Eq. 5), no delays */
int or_rhs_sync(const or_cfg *cfg, const or_mech *m, const double *w, double *rhs);
/* the troubled-cell indicator and WENO limiter (Sec. 3.3) applied once to a state,
 * no delays: flags [n_elem], limited state wout */
int or_limit_sync(const or_cfg *cfg, const or_mech *m, const double *w, double *wout,
                  uint8_t *flags);
/* the LDG auxiliary variable q = dw/dx of a state (central trace, no delays) */
int or_aux_sync(const or_cfg *cfg, const or_mech *m, const double *w, double *q);
int or_reactor0d(const or_mech *m, double *r, double rhoe, double dt, int n_steps);

#ifdef __cplusplus
}
#endif
#endif
