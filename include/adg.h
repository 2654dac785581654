/* adg.h — C ABI of the GB300 library for the asynchronous discontinuous Galerkin
 * (ADG) right-hand side of the 1D multicomponent reacting Euler equations
 * (arXiv 2501.01747), with PE boundaries emulated on one GPU.
 *
 * The operation every call serves is one explicit time step of the semi-discrete
 * DG system, Eq. (5) of Sec. 3.1:
 *     dw_i/dt = (2i+1)/dx [ int f(w) P_i' - fhat_{e+1} + (-1)^i fhat_e ] + proj_i(s),
 * advanced with three SSP-RK3 stages, where fhat is the local Lax-Friedrichs or
 * HLLC flux (Sec. 3.1), replaced at PE faces by the asynchrony-tolerant flux of
 * Eq. (7) at a common delayed level (Sec. 3.2), and every stage is followed by the
 * troubled-cell indicator and (AT-)WENO limiter of Sec. 3.3 (Eq. 9-11). Delays are
 * CAA (Sec. 4.1) or SAA (Sec. 4.2) draws, one per PE face per step.
 *
 * Conventions for every function:
 *  - return 0 (ADG_OK) on success, a negative ADG_ERR_* code otherwise;
 *    adg_error_string() names it. No function aborts the process.
 *  - state arrays are FP64 modal Legendre coefficients in the layout
 *    [nv][n_elem][p+1], nv = n_species + 2, variable 0 = rho*u, 1 = rho*E,
 *    2+i = rho*Y_i (the density is the sum of the partial densities).
 *  - pointers named *_host are host memory owned by the caller and only read or
 *    written during the call; pointers named *_dev are device memory owned by the
 *    caller. The context owns every buffer it allocated.
 *  - all work is enqueued on the CUDA stream passed to adg_step (0 = legacy
 *    default stream); the get/set functions synchronise that stream.
 */
#ifndef ADG_H
#define ADG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADG_OK 0
#define ADG_ERR_ARG -1          /* invalid argument or configuration */
#define ADG_ERR_CUDA -2         /* a CUDA runtime call failed */
#define ADG_ERR_NOMEM -3        /* device allocation failed or workspace too small */
#define ADG_ERR_NONPHYSICAL -4  /* density, temperature or state not finite/positive */
#define ADG_ERR_HISTORY -5      /* a delayed level is missing from the history ring */
#define ADG_ERR_NOLIB -6        /* no CUDA device is available */
#define ADG_ERR_TIMEOUT -7      /* a wait of the unsynchronised mode gave up */

#define ADG_BC_PERIODIC 0
#define ADG_BC_REFLECT 1
#define ADG_BC_OUTFLOW 2
#define ADG_FLUX_LF 0
#define ADG_FLUX_HLLC 1
#define ADG_LIM_NONE 0
#define ADG_LIM_WENO 1
#define ADG_SYNC 0
#define ADG_CAA 1
#define ADG_SAA 2
/* Time integrator, with limiting after every stage. ADG_RK_SSP3: SSP-RK3 in
 * Shu-Osher form. The low-storage explicit RK schemes (LSERK) of Sec. 3.1, in
 * Williamson's 2N form dq <- A_s dq + dt L(w), w <- w + B_s dq: ADG_RK_LS3,
 * Williamson's (1980) 3-stage 3rd-order scheme; ADG_RK_LS4, the 5-stage
 * 4th-order scheme of Carpenter and Kennedy (1994), the family of Kennedy,
 * Carpenter and Lewis (2000). Stage s of step n reads stage s of the delayed
 * steps; CAA skips the exchange at every stage of a delayed step (Sec. 4.1). */
#define ADG_RK_SSP3 0
#define ADG_RK_LS3 1
#define ADG_RK_LS4 2
#define ADG_MAX_STAGES 5
/* Arithmetic of the RK-stage right-hand side. The paper runs in double
 * precision; the mixed variants keep double where the stability of the
 * reacting system needs it. The state arrays stay double in every variant.
 * ADG_FP64: every step in double precision.
 * ADG_MIXED: the numerical flux, the DG volume/surface/source assembly and the
 * troubled-cell indicator and WENO reconstruction in float; in double the
 * state at the Gauss points, the temperature from the internal energy (T, ln T
 * and 1/T to about one ulp), the Arrhenius and equilibrium exponents and their
 * exponentials, the AT level sums and the RK accumulation; the mass-action
 * products, rates of progress and production rates in float pairs (about 48
 * significant bits) from the double rate constants, so that no rate constant
 * is rounded to float before it is used.
 * ADG_MIXED_F32CHEM: as ADG_MIXED, but the Arrhenius and equilibrium exponents
 * as float pairs (about 1e-12 absolute), their exponentials rounded once to
 * float, and the mass-action products and production rates in float. Not
 * offered with viscous terms or in the unsynchronised mode (ADG_ERR_ARG). */
#define ADG_FP64 0
#define ADG_MIXED 1
#define ADG_MIXED_F32CHEM 2

#define ADG_MAX_P 4        /* polynomial degree 1..4 */
#define ADG_MAX_SPECIES 60
#define ADG_MAX_DELAY 7
#define ADG_MAX_AT_ORDER 6

/* Mechanism (Sec. 2, Eq. 1-2: source W_i omega_i). Constant-c_p species;
 * reversible reactions with k_f = A T^b exp(-E_a/(R T)) and k_r = k_f / K_c. */
typedef struct {
  int n_species, n_reactions;
  const double *W;                  /* [n_species] kg/mol */
  const double *cp;                 /* [n_species] J/mol/K */
  const double *h_f;                /* [n_species] J/mol at 298.15 K */
  const double *s0;                 /* [n_species] J/mol/K at 298.15 K, 1 atm */
  const signed char *nu_f, *nu_r;   /* [n_reactions][n_species] >= 0 */
  const double *A, *b, *Ea;         /* [n_reactions] SI, -, J/mol */
  const double *Le;                 /* [n_species] Lewis numbers, used by viscous
                                       instances only; NULL: all 1 */
} adg_mechanism;

/* One instance (one 1D domain [x0, x0+length] cut into n_pe PEs). */
typedef struct {
  int n_elem, p, n_pe;
  double x0, length, dt;
  int bc_left, bc_right;   /* ADG_BC_*; periodic must be on both sides */
  int flux;                /* ADG_FLUX_* */
  int limiter;             /* ADG_LIM_* (AT-WENO at delayed PE faces) */
  int at_order;            /* 1..ADG_MAX_AT_ORDER; p+1 keeps the design order */
  int delay_mode;          /* ADG_SYNC | ADG_CAA | ADG_SAA */
  int max_delay;           /* 0..ADG_MAX_DELAY */
  const double *delay_probs; /* host [max_delay+1], SAA only (may be NULL otherwise) */
  uint64_t seed;           /* SAA delay seed */
  double tvb_M;            /* TVB constant of the indicator (0 = TVD) */
  int precision;           /* ADG_FP64 | ADG_MIXED | ADG_MIXED_F32CHEM */
  int integrator;          /* ADG_RK_SSP3 | ADG_RK_LS3 | ADG_RK_LS4 */
  /* Viscous terms (Sec. 2: f^d with the shear stress tau = 4/3 mu du/dx, the
   * heat flux q = -k dT/dx + sum h_i J_i and mixture-averaged diffusion
   * J_i = rho Y_i V_i, V_i = -(D_i/X_i) dX_i/dx, plus the correction velocity
   * that makes sum J_i = 0), discretised by the local DG method of Sec. 3.1:
   * q = dw/dx from a central trace of w, the Riemann flux of f^c minus the
   * central mean of f^d at faces; at a delayed PE face both the trace of w for
   * q and the face flux are AT-extrapolated. The transport model is synthetic
   * (the paper's comes from Cantera): mu = mu_ref (T/T_mu)^mu_exp,
   * k = mu c_p / prandtl (c_p of the mixture per unit mass) and
   * D_i = k / (rho c_p Le_i) with the mechanism's Lewis numbers. viscous = 0
   * ignores the other four fields. */
  int viscous;             /* 0: Euler; 1: with f^d */
  double mu_ref, T_mu, mu_exp, prandtl; /* Pa s, K, -, - (T_mu, prandtl > 0) */
  /* Subdomain (Sec. 3.1: each PE's subdomain exchanges its boundary elements
   * with its neighbours' buffer elements). pe_end = 0: the whole domain.
   * pe_end > 0: the PEs [pe_begin, pe_end) of the domain the fields above
   * describe (n_elem, n_pe, length and boundaries of the WHOLE domain), as an
   * instance of its own with a buffer element at each side that borders another
   * subdomain; see adg_part_layout and adg_part_block. Not with viscous terms,
   * the unsynchronised mode or adg_step_noalloc. */
  int pe_begin, pe_end;
} adg_config;

typedef struct adg_ctx adg_ctx;

/* Bytes of device memory adg_create needs for these instances (ring buffers,
 * state and stage buffers, flags, tables). Sec. 3.2 (history of delayed levels). */
int adg_workspace_bytes(const adg_mechanism *mech, const adg_config *cfgs, int n_instances,
                        size_t *bytes);

/* Create a context holding n_instances independent problems, each the setting
 * of Sec. 3.1 and 3.2: the domain [x0, x0+length] cut into n_elem elements with
 * the modal basis of degree p (Sec. 3.1, Eq. 4), split into n_pe contiguous PEs
 * whose boundary faces take the AT flux of Eq. (7) at the delays of Sec. 4
 * (CAA, Sec. 4.1; SAA, Sec. 4.2), with one reacting mixture (Sec. 2, the
 * mechanism) for all instances. workspace_dev: NULL lets the library cudaMalloc
 * what it needs; otherwise a caller-owned device buffer of at least
 * adg_workspace_bytes bytes, 256-byte aligned, that must outlive the context.
 * The mechanism and configs (and delay_probs) are copied; *out receives the
 * context (NULL on error). The state of every instance starts at zero: set it
 * with adg_set_primitive or adg_set_state. Errors: ADG_ERR_ARG (NULL pointer,
 * unsupported p, species count, delay, order, or a reaction with more than 4
 * species on one side), ADG_ERR_NOMEM, ADG_ERR_CUDA, ADG_ERR_NOLIB (no device). */
int adg_create(const adg_mechanism *mech, const adg_config *cfgs, int n_instances,
               void *workspace_dev, size_t workspace_bytes, adg_ctx **out);
/* Free the context and every device buffer it allocated (a caller-owned
 * workspace is left alone). Call it once the context's work has completed
 * (after adg_status, adg_get_state or a synchronisation of its stream). The
 * paper has no counterpart: this is resource management. NULL is ignored. */
void adg_destroy(adg_ctx *ctx);

/* Initial condition from primitive values at the p+1 Gauss-Legendre points of
 * every element: prim_host layout [n_species+3][n_elem][p+1] with rows T (K),
 * P (Pa), u (m/s), Y_1..Y_ns. L2-projects the conserved variables onto the modal
 * basis (Sec. 3.1) on the device, and resets the step counter and history. */
int adg_set_primitive(adg_ctx *ctx, int instance, const double *prim_host);

/* Copy a modal state in and reset the step counter and the history ring, so
 * that the next steps are synchronous until the history holds the delayed
 * levels (the state is the vector of modal DOFs w_j^e of Sec. 3.1, Eq. 4, in the
 * layout of the conventions above). w_host: host memory, copied during the
 * call (synchronous); w_dev: device memory, copied on `stream`.
 * Errors: ADG_ERR_ARG (NULL or bad instance), ADG_ERR_CUDA. */
int adg_set_state(adg_ctx *ctx, int instance, const double *w_host);
int adg_set_state_device(adg_ctx *ctx, int instance, const double *w_dev, void *stream);

/* Overwrite the current state of a running instance from host memory,
 * asynchronously on `stream`, keeping the step counter and the history ring (a
 * restart of a continuing run). w_host should be pinned for a true async copy
 * and must stay valid until the stream reaches the copy. */
int adg_write_state(adg_ctx *ctx, int instance, const double *w_host, void *stream);

/* Read the current state into host memory asynchronously on `stream` (no
 * synchronisation; the data is valid once the stream has passed the copy). */
int adg_read_state(adg_ctx *ctx, int instance, double *w_host, void *stream);

/* adg_write_state and adg_read_state for every instance with one call: w_host
 * holds the states of instances 0, 1, ... in order, each [nv][n_elem][p+1]
 * (adg_states_doubles gives the total length, which the buffer must hold). A
 * pinned buffer mapped into the device's address space (cudaHostAlloc or
 * cudaHostRegister memory under unified addressing) is read or written by one
 * kernel over the host link; other host memory by one copy per instance. Both
 * are enqueued on `stream`; the same rules on validity apply.
 * Errors: ADG_ERR_ARG (NULL), ADG_ERR_CUDA. */
int adg_write_states(adg_ctx *ctx, const double *w_host, void *stream);
int adg_read_states(adg_ctx *ctx, double *w_host, void *stream);
int64_t adg_states_doubles(const adg_ctx *ctx);

/* One time step (Sec. 3.1, Eq. 5; the step of adg_step) of every instance
 * from new host states to host results: the same as adg_write_states(w_in),
 * adg_step(1) and adg_read_states(w_out) on `stream`, with the same results to
 * the bit, but with the copies overlapped with the stages (the instances of one
 * degree and precision form a group and share the stage and limiter
 * launches; each group without viscous terms is cut into up to four parts of
 * its instances). The copies in run part after part, one copy per instance on the
 * copy engines; the parts step one after another, each once its own states
 * are in, and a part's states go out while the next part steps.
 * w_in and w_out: pinned host buffers (cudaHostAlloc or cudaHostRegister
 * memory) in adg_write_states' layout, adg_states_doubles long each, valid
 * until the stream passes the step; they may be the same buffer only if the
 * caller does not need w_in afterwards. The first call for a pair of buffers
 * captures a CUDA graph for it (later calls with the same pair replay it; a
 * new pair, or a new launch configuration, captures again). With one group,
 * pageable buffers or kernel timing on, the call runs the three calls in
 * sequence. Errors: ADG_ERR_ARG (NULL), ADG_ERR_CUDA. */
int adg_step_io(adg_ctx *ctx, const double *w_in, double *w_out, void *stream);

/* Copy the current modal state out: the DOFs w_j^e of Sec. 3.1 (Eq. 4) after the
 * steps done, in the layout of the conventions above. Synchronises the
 * context's last stream first, so the result is the state after every step
 * enqueued so far. w_host: host memory the caller owns, [nv][n_elem][p+1];
 * w_dev: device memory, written on `stream`. Errors: ADG_ERR_ARG (NULL or bad
 * instance), ADG_ERR_CUDA. */
int adg_get_state(adg_ctx *ctx, int instance, double *w_host);
int adg_get_state_device(adg_ctx *ctx, int instance, double *w_dev, void *stream);

/* Advance every instance by n_steps time steps of its integrator on `stream` (a
 * cudaStream_t; NULL = default stream). Each stage evaluates the semi-discrete
 * right-hand side of Eq. (5) (Sec. 3.1: volume and source quadrature, LF or
 * HLLC fluxes at element faces, the AT flux of Eq. (7)-(8) at delayed PE faces,
 * Sec. 3.2), updates the state (SSP-RK3, or the LSERK schemes of Sec. 3.1), and
 * applies the troubled-cell indicator and (AT-)WENO limiter of Sec. 3.3
 * (Eq. 9-11); the delay of each PE face is drawn once per step (Sec. 4).
 * Asynchronous: returns after enqueueing one replay of the captured step graph
 * per step. n_steps = 0 does nothing. Errors: ADG_ERR_ARG (NULL, n_steps < 0),
 * ADG_ERR_CUDA; non-physical states and missing history levels found on the
 * device are reported by adg_status. */
int adg_step(adg_ctx *ctx, int n_steps, void *stream);

/* ---- Domain decomposition (Sec. 3.1, Fig. 1: the PE boundary elements' DoFs go
 * to the neighbours' buffer elements; Sec. 3.2: the buffers may hold delayed
 * levels and the flux at a PE face uses the common delayed level; Sec. 3.3: the
 * limiter's neighbours are exchanged after every stage; Sec. 4: the delays).
 *
 * A subdomain instance (adg_config.pe_end > 0) holds the elements of its PEs,
 * [floor(pe_begin N / P), floor(pe_end N / P)) of the whole domain's N elements
 * and P PEs, plus one buffer element at each cut side (a side that borders
 * another subdomain, also across a periodic boundary). Its PE faces are its
 * own PEs' plus the cut faces; their delays are the whole domain's (SAA draws
 * by the whole domain's face number), and dx is the whole domain's. Beyond a
 * buffer element the subdomain ends in an outflow boundary: the buffers are
 * computed like the other elements, but the exchange overwrites their data
 * before any owned element reads it, so that the owned elements advance exactly
 * as in the whole-domain instance. Its arrays (states, primitives, flags) are
 * [..][n_local][..] with the buffers included.
 *
 * adg_part_layout: for a config, the subdomain's element count n_local, the
 * whole domain's index of its local element 0 (modulo n_elem: -1 for a
 * periodic subdomain that starts at PE 0), and which sides are cut (0/1).
 * The whole domain (pe_end = 0, or all PEs) gives n_elem, 0, 0, 0.
 * Errors: ADG_ERR_ARG (NULL config, bad PE range). */
int adg_part_layout(const adg_config *cfg, int *n_local, int *elem0, int *cut_left,
                    int *cut_right);

/* One half of RK stage `stage` of the current step of every instance, enqueued on
 * `stream` as plain launches (no graph): half 0 the stage kernels (Eq. 5 and the
 * RK update, giving the pre-limit output), half 1 the troubled-cell indicator
 * and limiter (Sec. 3.3), and after the last stage the step counters' advance.
 * The halves of stages 0..S-1 in order are one adg_step. Between them the
 * caller moves the subdomains' boundary blocks (adg_part_block): before half 0
 * of stage s the stage inputs, before half 1 the pre-limit outputs.
 * Errors: ADG_ERR_ARG (NULL, stage or half out of range), ADG_ERR_CUDA. */
int adg_step_stage(adg_ctx *ctx, int stage, int half, void *stream);

/* Move one boundary block, [nv][p+1] doubles in caller-owned device memory
 * blk_dev, of instance `instance` at side `side` (0 left, 1 right) for stage
 * `stage` of the current step, on `stream` (asynchronous, device-to-device).
 * what = ADG_PART_INPUT: the stage input (at stage 0 the state at the start of
 * the step); ADG_PART_PRELIMIT: the pre-limit output of that stage.
 * import = 0 (export): copies the owned element at that side (the neighbour's
 * buffer) into blk_dev; import = 1: writes blk_dev into the buffer element at
 * that side, and for ADG_PART_PRELIMIT also into the cut face's pre-limit
 * history (the levels the AT-WENO neighbour of Eq. 11 reads), at the step the
 * device's step counter holds when the copy runs. Exports are device copies,
 * imports a small kernel; both only enqueue work on `stream`, so the halves
 * and the block moves of a step can be captured in a CUDA graph and replayed
 * (adg_steps_done then counts only the calls made, not the replays). Call the
 * exports of a stage's pre-limit output after its half 0 and the imports
 * before its half 1; the stage inputs' before half 0 of the stage.
 * Errors: ADG_ERR_ARG (NULL, bad instance, side that is not cut, bad what or
 * stage), ADG_ERR_CUDA. */
#define ADG_PART_INPUT 0
#define ADG_PART_PRELIMIT 1
int adg_part_block(adg_ctx *ctx, int instance, int what, int side, int stage, double *blk_dev,
                   int import, void *stream);

/* Synchronise and report the first device-side error since the last reset
 * (ADG_ERR_NONPHYSICAL or ADG_ERR_HISTORY), with the instance, element, step and
 * stage where it happened (any pointer may be NULL); clears it. */
int adg_status(adg_ctx *ctx, int *instance, int *element, int64_t *step, int *stage);

/* Troubled-cell flags of the stages of the last step ([stages][n_elem] bytes:
 * 3 stages for ADG_RK_SSP3 and ADG_RK_LS3, 5 for ADG_RK_LS4) and per-element
 * counts of flagged stages since the last set ([n_elem] int32). */
int adg_get_flags(adg_ctx *ctx, int instance, uint8_t *last_host, int32_t *count_host);

/* Temperature at the Gauss points of the current state, [n_elem][p+1]. */
int adg_get_temperature(adg_ctx *ctx, int instance, double *T_host);

/* One auxiliary field of an instance's current state (synchronous):
 * ADG_AUX_TEMPERATURE and ADG_AUX_PRESSURE at every Gauss point (double
 * [n_elem][p+1]; T from e as in Sec. 2, P = rho R_u T sum_i Y_i/W_i), or
 * ADG_AUX_FLAGS, the troubled-cell flags of the last step's stages (uint8
 * [stages][n_elem], as adg_get_flags). ADG_ERR_ARG for another `what`. */
#define ADG_AUX_TEMPERATURE 0
#define ADG_AUX_PRESSURE 1
#define ADG_AUX_FLAGS 2
int adg_get_aux(adg_ctx *ctx, int instance, int what, void *out_host);

int64_t adg_steps_done(const adg_ctx *ctx, int instance);

/* Delays the context draws (Sec. 4.1 CAA: k = n mod (max_delay+1); Sec. 4.2 SAA:
 * SplitMix64 of seed ^ (step << 32 + face), top 53 bits, matched to the bins of
 * the cumulative probabilities), for steps [step0, step0+n_steps) and every PE
 * face: out_host [n_steps][n_pe_faces] bytes. n_pe_faces = n_pe (periodic) or
 * n_pe - 1 (bounded), 0 when n_pe == 1. */
int adg_delay_table(const adg_config *cfg, int64_t step0, int n_steps, uint8_t *out_host);

/* Per-kernel timing (on = 1 starts a new measurement). While it is on, adg_step
 * runs a variant of the step graph with a CUDA event pair around every kernel,
 * waits for each step, and adds the kernels' times up; adg_step is then
 * synchronous. adg_kernel_times returns, per kind (0: stage RHS/update kernel,
 * 1: limiter kernel, 2: whole step from the graph's first to its last node),
 * the summed milliseconds and counts since enabling; ms and launches point to
 * arrays of 3. Without timing, adg_step replays a captured CUDA graph of the
 * step and returns at once. */
int adg_enable_kernel_timing(adg_ctx *ctx, int on);
int adg_kernel_times(adg_ctx *ctx, double *ms, int64_t *launches);

/* Autotuner of the launch configuration, per group of instances: times the
 * stage kernel for every (elements per stage tile, threads per stage CTA)
 * candidate that fits in shared memory, then the limiter for every number of
 * elements per limiter CTA it is built for (8, 16, 32 in the mixed variants;
 * 16, 32 in FP64), on `stream`; keeps the fastest and drops the captured step
 * graphs. The trial launches leave the trajectory as it was: they only rewrite
 * buffers the next step rewrites, and the flags and flag counts the trial
 * limiter launches write are put back. The configuration chosen may change the
 * rounding of the limiter's sums (its lanes per element follow the elements per
 * CTA), not the stage kernel's. Synchronous. Instances are grouped by
 * degree, precision and number of RK stages. adg_get_tuning fills
 * tuning[ADG_TUNING_FIELDS * g + {0..6}] with the degree, precision, tile
 * elements, threads per CTA, tile count, RK stages and limiter elements per CTA
 * of group g (at most ADG_MAX_GROUPS groups). */
#define ADG_MAX_GROUPS (6 * ADG_MAX_P)
#define ADG_TUNING_FIELDS 7
int adg_autotune(adg_ctx *ctx, void *stream);
int adg_get_tuning(const adg_ctx *ctx, int *n_groups, int *tuning);
/* Set the launch configuration of group g directly (for instance one that an
 * earlier adg_autotune found): elements per stage tile >= 2, threads per CTA a
 * multiple of 32 in [32, 512], or up to 1024 for a group of the mixed variants
 * without viscous terms. Synchronous; drops the captured step graphs.
 * ADG_ERR_ARG for a bad group or a tile whose shared memory exceeds 200 KB. */
int adg_set_tuning(adg_ctx *ctx, int group, int elements_per_tile, int threads_per_cta);
/* Set the limiter's elements per CTA of group g (8, 16 or 32 in the mixed
 * variants, 16 or 32 in FP64; ADG_ERR_ARG otherwise). Synchronous; drops the
 * captured step graphs. */
int adg_set_limiter_tuning(adg_ctx *ctx, int group, int elements_per_cta);

/* Number of kernel launches one adg_step(ctx, 1, ...) enqueues. */
int adg_launches_per_step(const adg_ctx *ctx);

/* A NUL-terminated description of an ADG_* return code ("unknown error" for
 * other values), never NULL and owned by the library; for ADG_ERR_CUDA, the
 * text of the last failed CUDA call (a buffer shared by all threads). The paper
 * has no counterpart. */
const char *adg_error_string(int code);

/* Truly unsynchronised mode (the emulated PEs run without any lockstep; the
 * seeded CAA/SAA delays of Sec. 4 are replaced by the delays that actually
 * occur). adg_step_unsync advances instance `instance` by n_steps SSP-RK3 steps
 * in one cooperative launch with one CTA per PE. A PE publishes, per step and
 * stage, its stage input's traces at its PE faces and the pre-limit output of
 * its PE-boundary elements to the history rings, and observes the delay
 * k = max(0, n - L) of the newest level L its neighbour has published. The
 * flux at a PE face (Eq. 7) uses one delay on both sides, the common (older)
 * level of Sec. 3.2: the first side to reach step n and stage s fixes k from
 * the other side's newest level and the second adopts it, so the flux stays
 * single-valued and the scheme conservative. The AT-WENO neighbour (Eq. 11) of
 * each side takes the delay that side observed. No PE runs more than the
 * config's max_delay steps ahead of a neighbour (it waits); until the levels an
 * AT extrapolation needs exist, it waits for k = 0. The result depends on
 * timing and is not reproducible; with max_delay = 0 it reproduces adg_step's
 * synchronous result exactly. Asynchronous on `stream`; the instance's step
 * counter advances by n_steps. One unsynchronised launch per context may be in
 * flight at a time. ADG_ERR_ARG for a bad instance or more PEs than fit on the
 * GPU at once; a wait that does not end within the bound set by
 * adg_set_unsync_wait stops the launch and reports ADG_ERR_TIMEOUT through
 * adg_status.
 * adg_unsync_delays copies the histogram of the delays used since the last
 * call into hist[2][ADG_MAX_DELAY + 1] (row 0: flux, row 1: limiter; one count
 * per PE face side and stage) and clears it (synchronous). */
int adg_step_unsync(adg_ctx *ctx, int instance, int n_steps, void *stream);
int adg_unsync_delays(adg_ctx *ctx, uint64_t *hist);

/* Bound of every wait of the unsynchronised mode, in polls of a counter
 * (default 2^22, a few seconds), and a PE that never publishes anything
 * (withheld_pe >= 0; -1, the default, for none): with it set, the PEs that wait
 * on it give up after max_polls polls and the launch ends with ADG_ERR_TIMEOUT,
 * which is how the timeout path is tested. ADG_ERR_ARG for max_polls < 0 or
 * withheld_pe < -1. */
int adg_set_unsync_wait(adg_ctx *ctx, long long max_polls, int withheld_pe);

/* Emulated load imbalance for the unsynchronised mode (Sec. 3.2 names load
 * imbalance as a source of delays): PE slow_pe idles about slow_us microseconds
 * per stage before it publishes, so its neighbours run ahead of it and observe
 * delays up to max_delay. slow_pe = -1 (the default) for none. ADG_ERR_ARG for
 * slow_pe < -1 or slow_us outside [0, 10000]. */
int adg_set_unsync_imbalance(adg_ctx *ctx, int slow_pe, int slow_us);

/* ---------------------------------------------------------------------------
 * Time step without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, for instance a
 * plugin inside a host application whose own allocator owns all device
 * memory, a runtime that forbids device allocation once it is running, or a
 * caller under a fixed device-memory budget. adg_create would allocate its
 * workspace (or need one handed in); this call needs none.
 *
 * adg_step_noalloc advances one instance (mechanism and config as for
 * adg_create) by n_steps SSP-RK3 steps from the modal state w_in_dev to
 * w_out_dev (both caller-owned device arrays [nv][n_elem][p+1]; they may be the
 * same array). Like adg_set_state followed by adg_step, it starts from step 0
 * with an empty history, so the first steps are synchronous. All scratch (stage
 * buffers, history ring, tables, flags) lives in one static device array of
 * ADG_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the library holds
 * until the process exits; it calls no cudaMalloc, cudaFree or other
 * allocating routine, and allocates nothing on the host heap. The mechanism
 * tables and the instance record reach the device as parameters of small copy
 * kernels, so after the first call on a device the call only enqueues work on
 * `stream` (kernels and one device-to-device copy when the arrays differ) and
 * returns without waiting for it.
 *
 * - The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) and uploads the constant tables, synchronously;
 *   make that first call before any stream capture on that device.
 * - A problem whose scratch does not fit returns ADG_ERR_NOMEM (nothing is
 *   enqueued); more than ADG_NOALLOC_MAX_REACTIONS reactions, an integrator
 *   other than ADG_RK_SSP3 or viscous terms return ADG_ERR_ARG.
 * - Every call reuses the same array and leaves its contents there; each call
 *   clears what must start at zero (history, flags, step counter, error word).
 *   Calls that overlap on the GPU (on different streams, or from several host
 *   threads without ordering) race and corrupt each other's results.
 * - The host side stages the tables in static storage under a lock, so calls
 *   from several host threads are serialised while they enqueue.
 * - Non-physical states found on the device are not reported (there is no
 *   context to query); check the output. */
#define ADG_NOALLOC_SCRATCH_BYTES (16u << 20)
#define ADG_NOALLOC_MAX_REACTIONS 512
int adg_step_noalloc(const adg_mechanism *mech, const adg_config *cfg, const double *w_in_dev,
                     double *w_out_dev, int n_steps, void *stream);

#ifdef __cplusplus
}
#endif
#endif
