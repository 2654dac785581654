// Host runtime of the ADG library: context, device memory, tables, C ABI.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "adg_internal.cuh"
#include "adg_math.cuh"


using namespace adg;

// ---------------------------------------------------------------------------
// Basis tables of the modal Legendre DG method (Sec. 3.1) and of the WENO
// limiter (Sec. 3.3), computed on the host in FP64.

static void legendre_all(int n, double x, double *P) {
  P[0] = 1.0;
  if (n >= 1) P[1] = x;
  for (int j = 1; j < n; ++j) P[j + 1] = ((2 * j + 1) * x * P[j] - j * P[j - 1]) / (j + 1);
}

// s-th derivatives of P_0..P_n at x by differentiating the three-term recurrence:
// (j+1) P_{j+1}^(s) = (2j+1) (x P_j^(s) + s P_j^(s-1)) - j P_{j-1}^(s).
static void legendre_deriv(int n, int s, double x, double *D) {
  double prev[MAXQ + 1], cur[MAXQ + 1];
  legendre_all(n, x, prev);
  for (int d = 1; d <= s; ++d) {
    cur[0] = 0.0;
    if (n >= 1) cur[1] = (d == 1) ? 1.0 : 0.0;
    for (int j = 1; j < n; ++j)
      cur[j + 1] = ((2 * j + 1) * (x * cur[j] + d * prev[j]) - j * cur[j - 1]) / (j + 1);
    for (int j = 0; j <= n; ++j) prev[j] = cur[j];
  }
  for (int j = 0; j <= n; ++j) D[j] = prev[j];
}

static void gauss_points(int Q, double *x, double *w) {
  double P[MAXQ + 2], D[MAXQ + 2];
  for (int i = 0; i < Q; ++i) {
    double t = -cos(M_PI * (2 * i + 1) / (2.0 * Q));
    for (int it = 0; it < 200; ++it) {
      legendre_all(Q, t, P);
      legendre_deriv(Q, 1, t, D);
      double d = P[Q] / D[Q];
      t -= d;
      if (fabs(d) <= 1e-17) break;
    }
    legendre_deriv(Q, 1, t, D);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * D[Q] * D[Q]);
  }
}

static void make_basis(int p, Basis *B) {
  int Q = p + 1;
  memset(B, 0, sizeof(Basis));
  gauss_points(Q, B->x, B->w);
  for (int q = 0; q < Q; ++q) {
    double P[MAXQ + 1], D[MAXQ + 1];
    legendre_all(p, B->x[q], P);
    legendre_deriv(p, 1, B->x[q], D);
    for (int j = 0; j < Q; ++j) {
      B->P[q][j] = P[j];
      B->dP[q][j] = D[j];
    }
  }
  // beta = sum_s 2^(2s-1) int (d^s v/dxi^s)^2: Gauss rule with Q points is exact
  for (int s = 1; s <= p; ++s) {
    for (int q = 0; q < Q; ++q) {
      double D[MAXQ + 1];
      legendre_deriv(p, s, B->x[q], D);
      for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) B->B[i][j] += ldexp(1.0, 2 * s - 1) * B->w[q] * D[i] * D[j];
    }
  }
  for (int q = 0; q < Q; ++q)
    for (int i = 0; i < Q; ++i) {
      B->WdP[q][i] = B->w[q] * B->dP[q][i];
      B->WPh[q][i] = B->w[q] * B->P[q][i] * 0.5 * (2 * i + 1);
    }
  // neighbour polynomials continued into the cell: left uses xi' = xi + 2
  for (int q = 0; q < Q; ++q) {
    double Pl[MAXQ + 1], Pr[MAXQ + 1], P[MAXQ + 1];
    legendre_all(p, B->x[q] + 2.0, Pl);
    legendre_all(p, B->x[q] - 2.0, Pr);
    legendre_all(p, B->x[q], P);
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) {
        B->Sl[i][j] += 0.5 * (2 * i + 1) * B->w[q] * Pl[j] * P[i];
        B->Sr[i][j] += 0.5 * (2 * i + 1) * B->w[q] * Pr[j] * P[i];
      }
  }
}

// All constant tables: the DG/WENO basis for p = 1..ADG_MAX_P.
void adg::make_tables(Basis *tables) {
  for (int p = 1; p <= ADG_MAX_P; ++p) make_basis(p, &tables[p - 1]);
}

// Species fields (constant c_p thermo, Sec. 2), packed reactions and the
// species -> reaction incidence of the net stoichiometry.
void adg::pack_rxf(const Rxn *rx, int nr, DF *rxf) {
  for (int j = 0; j < nr; ++j) {
    const double c[6] = {rx[j].lnA, rx[j].b, rx[j].mEaR, rx[j].kr0, rx[j].kr1, rx[j].kr2};
    for (int k = 0; k < 6; ++k) rxf[6 * j + k] = df_split(c[k]);
  }
}

int adg::pack_mechanism(const adg_mechanism *m, double *sp, Rxn *rx, int *sx_off, int *sx) {
  const int ns = m->n_species, nr = m->n_reactions;
  for (int i = 0; i < ns; ++i) {
    double W = m->W[i], cp = m->cp[i], hf = m->h_f[i], s0 = m->s0[i];
    sp[SP_W * ns + i] = W;
    sp[SP_INVW * ns + i] = 1.0 / W;
    sp[SP_QW * ns + i] = (hf - cp * TREF) / W;
    sp[SP_CVW * ns + i] = (cp - RU) / W;
    sp[SP_RW * ns + i] = RU / W;
    sp[SP_CPW * ns + i] = cp / W;
    sp[SP_G0 * ns + i] = (hf - cp * TREF) / RU;
    sp[SP_G1 * ns + i] = cp / RU * (1.0 + log(TREF)) - s0 / RU;
    sp[SP_CPR * ns + i] = cp / RU;
    sp[SP_INVLE * ns + i] = m->Le ? 1.0 / m->Le[i] : 1.0;
  }
  for (int j = 0; j < nr; ++j) {
    Rxn &R = rx[j];
    memset(&R, 0, sizeof(Rxn));
    if (!(m->A[j] > 0.0)) return ADG_ERR_ARG;
    R.lnA = log(m->A[j]);
    R.b = m->b[j];
    R.mEaR = -m->Ea[j] / RU;
    int a = 0, b = 0, x = 0, dnu = 0;
    double g0 = 0.0, g1 = 0.0, cpr = 0.0;
    for (int i = 0; i < ns; ++i) {
      int f = m->nu_f[j * ns + i], r = m->nu_r[j * ns + i];
      if (f < 0 || r < 0 || f > 2 || r > 2) return ADG_ERR_ARG;
      if (f > 0) {
        if (a == SIDE) return ADG_ERR_ARG;
        R.rs[a] = (uint8_t)i;
        R.rn[a++] = (uint8_t)f;
      }
      if (r > 0) {
        if (b == SIDE) return ADG_ERR_ARG;
        R.ps[b] = (uint8_t)i;
        R.pn[b++] = (uint8_t)r;
      }
      if (r != f) {
        if (++x > NET) return ADG_ERR_ARG;
        const double nu = (double)(r - f);
        dnu += r - f;
        g0 = fma(nu, sp[SP_G0 * ns + i], g0);
        g1 = fma(nu, sp[SP_G1 * ns + i], g1);
        cpr = fma(nu, sp[SP_CPR * ns + i], cpr);
      }
    }
    R.kr0 = R.lnA + (double)dnu * log(RU / PATM) + g1;
    R.kr1 = R.b + (double)dnu - cpr;
    R.kr2 = R.mEaR + g0;
  }
  int n = 0;
  for (int i = 0; i < ns; ++i) {
    sx_off[i] = n;
    for (int j = 0; j < nr; ++j) {
      int c = m->nu_r[j * ns + i] - m->nu_f[j * ns + i];
      if (c != 0) sx[n++] = (j << 8) | (c & 0xff);
    }
  }
  sx_off[ns] = n;
  return n;
}

namespace {
// Number of species-reaction incidence terms (nonzero net coefficients).
int count_terms(const adg_mechanism *m) {
  int n = 0;
  for (int k = 0; k < m->n_species * m->n_reactions; ++k) n += (m->nu_r[k] != m->nu_f[k]);
  return n;
}
}  // namespace

// AT weights (Eq. 7-8): extrapolation to t_n from levels t_n - (k+m) dt.
static void at_weights(int order, int k, double *c) {
  for (int m = 0; m < order; ++m) {
    double v = 1.0;
    for (int j = 0; j < order; ++j)
      if (j != m) v *= (double)(k + j) / (double)(j - m);
    c[m] = v;
  }
}

// ---------------------------------------------------------------------------

// A subdomain instance (adg_config.pe_end > 0): the PEs [pb, pe) of a domain of N
// elements and P PEs, PE q owning elements [floor(q N / P), floor((q+1) N / P)),
// plus a buffer element at each cut side (a side that borders another
// subdomain). Its PE faces, in order, are the whole domain's faces
// pb - cut_l .. pe - 1 - (1 - cut_r) (mod the whole domain's face count).
struct PartInfo {
  bool part = false;
  int pb = 0, pe = 0;
  int n_local = 0;    // elements with the buffers
  int elem0 = 0;      // whole-domain index of local element 0 (may be -1: periodic)
  int cut_l = 0, cut_r = 0;
  int npf = 0;        // PE faces of the instance
  int face_base = 0;  // local face f is whole-domain face (f + face_base) mod npf_draw
  int npf_draw = 0;   // PE faces of the whole domain
  double dx = 0.0;    // the whole domain's element size
};

struct InstHost {
  Inst d;         // device view (a copy lives in the device instance table)
  int64_t n;      // steps done (host mirror of the device counter)
  double *prim;   // staging for projection / temperature
  int n_pe;       // PEs of the instance
  PartInfo part;  // subdomain layout (part = false: the whole domain)
};

// Instances of one polynomial degree and precision share the stage and limiter
// launches.
struct Group {
  int Q = 0;
  int prec = ADG_FP64;          // precision variant of the stage kernel
  bool mixed = false;           // FP32 limiter (both mixed variants)
  int S = 3;                    // RK stages per step
  bool visc = false;            // has viscous instances (LDG auxiliary kernel per stage)
  int TE = 0;                   // elements per stage tile
  int NT = 128;                 // threads per stage CTA
  int EPB = 32;                 // elements per limiter CTA
  int O = 1;                    // largest AT order of the group
  int n_tiles = 0, n_blocks = 0;
  int2 *d_tiles = nullptr;      // (instance, first element) per stage CTA
  int2 *d_blocks = nullptr;     // (instance, first element) per limiter CTA
  bool any_limiter = false;
  std::vector<int> members;     // the group's instances (adg_step_io's copies)
};

// Parts per group of adg_step_io's pipeline (at most; groups without viscous
// terms and with that many instances).
constexpr int kIoParts = 4;

struct adg_ctx {
  std::vector<cudaEvent_t> ev;   // timing events: a pair around every kernel of one step
  std::vector<int> ev_kind;      // kernel kind of each pair
  size_t ev_used;                // events recorded while capturing the timing graph
  bool timing;                   // steps run the timing graph and accumulate kernel times
  bool capturing_timed;          // enqueue_step is recording event pairs
  double kms[3];
  int64_t kcount[3];
  cudaEvent_t span[2];           // first and last node of the timing graph
  cudaGraph_t tgraph;            // the step with event pairs
  cudaGraphExec_t texec;
  int n_inst;
  int ns, nr;
  Mech mech;
  std::vector<InstHost> inst;
  Group groups[ADG_MAX_GROUPS];
  int n_groups;
  Inst *d_insts;                 // device instance table
  int64_t *d_offs;               // [n_inst + 1] first double of each state in a flat buffer
  int64_t *d_steps;              // device step counters [n_inst]
  void *mem;
  bool owns_mem;
  size_t bytes;
  int *err_all;   // device error words [n_inst][4]
  int *pub_in, *pub_pre;         // unsynchronised mode: stages published per PE [max PEs]
  unsigned long long *agree;     // unsynchronised mode: common flux levels [max PEs][3][MAXD + 1]
  unsigned long long *delay_hist;  // unsynchronised mode: delays observed [2][MAXD + 1]
  long long unsync_polls;        // unsynchronised mode: polls before a wait gives up
  int unsync_withheld;           // unsynchronised mode: PE that never publishes, or -1
  int unsync_slow_pe, unsync_slow_us;  // unsynchronised mode: emulated load imbalance
  cudaStream_t last_stream;
  cudaStream_t cap_stream;       // private stream for graph capture
  // one stream per group for the concurrent branches of the plain step graph,
  // and the events that fork them from and join them to the capture stream
  cudaStream_t branch[ADG_MAX_GROUPS];
  cudaEvent_t fork_ev, join_ev[ADG_MAX_GROUPS];
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool graph_ok;
  // adg_step_io: the step with every state copy, for one pair of pinned host
  // buffers, in parts of up to kIoParts per group: the copies in run part after part
  // on io_stream (io_ev[j]: part j's states are in), the parts' stages one after
  // another on the capture stream (done_ev[j]: part j's step is done), the
  // copies out on out_stream
  cudaStream_t io_stream, out_stream;
  cudaEvent_t io_ev[kIoParts * ADG_MAX_GROUPS], done_ev[kIoParts * ADG_MAX_GROUPS];
  cudaGraph_t io_graph;
  cudaGraphExec_t io_exec;
  const double *io_in;
  double *io_out;
};

// The streams and events of the concurrent branches (those created).
static void destroy_branches(adg_ctx *ctx) {
  for (int g = 0; g < ADG_MAX_GROUPS; ++g) {
    if (ctx->branch[g]) cudaStreamDestroy(ctx->branch[g]);
    if (ctx->join_ev[g]) cudaEventDestroy(ctx->join_ev[g]);
    ctx->branch[g] = nullptr;
    ctx->join_ev[g] = nullptr;
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  ctx->fork_ev = nullptr;
}

namespace {

constexpr int kMinTile = 2;   // smallest stage tile (elements) the autotuner tries

struct Carver {
  char *base;
  size_t off, cap;
  bool dry;
  void *take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    void *p = dry ? nullptr : base + off;
    off += n;
    return p;
  }
};

int check_args(const adg_mechanism *m, const adg_config *cfgs, int n) {
  if (!m || !cfgs || n < 1) return ADG_ERR_ARG;
  if (m->n_species < 1 || m->n_species > ADG_MAX_SPECIES || m->n_reactions < 0) return ADG_ERR_ARG;
  if (!m->W || !m->cp || !m->h_f || !m->s0) return ADG_ERR_ARG;
  if (m->n_reactions > 0 && (!m->nu_f || !m->nu_r || !m->A || !m->b || !m->Ea)) return ADG_ERR_ARG;
  for (int i = 0; i < m->n_species; ++i)
    if (!(m->W[i] > 0.0) || !(m->cp[i] > RU) || (m->Le && !(m->Le[i] > 0.0))) return ADG_ERR_ARG;
  for (int j = 0; j < m->n_reactions; ++j) {
    int nf = 0, nr = 0, nx = 0;
    for (int i = 0; i < m->n_species; ++i) {
      int a = m->nu_f[j * m->n_species + i], b = m->nu_r[j * m->n_species + i];
      if (a < 0 || b < 0 || a > 2 || b > 2) return ADG_ERR_ARG;
      nf += a > 0;
      nr += b > 0;
      nx += (b - a) != 0;
    }
    if (nf > SIDE || nr > SIDE || nx > NET) return ADG_ERR_ARG;
    if (!(m->A[j] > 0.0)) return ADG_ERR_ARG;
  }
  for (int k = 0; k < n; ++k) {
    const adg_config &c = cfgs[k];
    if (c.p < 1 || c.p > ADG_MAX_P || c.n_elem < 1 || c.n_pe < 1 || c.n_pe > c.n_elem)
      return ADG_ERR_ARG;
    if (!(c.length > 0.0) || !(c.dt > 0.0)) return ADG_ERR_ARG;
    if (c.at_order < 1 || c.at_order > ADG_MAX_AT_ORDER) return ADG_ERR_ARG;
    if (c.max_delay < 0 || c.max_delay > ADG_MAX_DELAY) return ADG_ERR_ARG;
    if (c.delay_mode < ADG_SYNC || c.delay_mode > ADG_SAA) return ADG_ERR_ARG;
    if (c.delay_mode == ADG_SAA && !c.delay_probs) return ADG_ERR_ARG;
    if (c.flux != ADG_FLUX_LF && c.flux != ADG_FLUX_HLLC) return ADG_ERR_ARG;
    if (c.limiter != ADG_LIM_NONE && c.limiter != ADG_LIM_WENO) return ADG_ERR_ARG;
    bool lp = c.bc_left == ADG_BC_PERIODIC, rp = c.bc_right == ADG_BC_PERIODIC;
    if (lp != rp) return ADG_ERR_ARG;
    if (c.bc_left < 0 || c.bc_left > 2 || c.bc_right < 0 || c.bc_right > 2) return ADG_ERR_ARG;
    if (c.precision != ADG_FP64 && c.precision != ADG_MIXED && c.precision != ADG_MIXED_F32CHEM)
      return ADG_ERR_ARG;
    if (c.precision == ADG_MIXED_F32CHEM && c.viscous) return ADG_ERR_ARG;
    if (c.integrator < ADG_RK_SSP3 || c.integrator > ADG_RK_LS4) return ADG_ERR_ARG;
    if (c.viscous != 0 && c.viscous != 1) return ADG_ERR_ARG;
    if (c.viscous && (!(c.mu_ref >= 0.0) || !(c.T_mu > 0.0) || !(c.prandtl > 0.0) ||
                      !isfinite(c.mu_exp)))
      return ADG_ERR_ARG;
    if ((int64_t)c.n_elem * (c.p + 1) * (m->n_species + 3) > (int64_t)1 << 31) return ADG_ERR_ARG;
  }
  return ADG_OK;
}

// RK stages per step, and the 2N-storage coefficients of an LSERK scheme
// (Sec. 3.1: Williamson 1980; Carpenter and Kennedy's 5-stage 4th-order scheme of
// the Kennedy-Carpenter-Lewis family), as published. Returns 0 for SSP-RK3.
int rk_stages(int integrator) { return integrator == ADG_RK_LS4 ? 5 : 3; }

static int lserk_coefficients(int integrator, double *a, double *b) {
  if (integrator == ADG_RK_LS3) {
    const double A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
    const double B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    for (int s = 0; s < 3; ++s) {
      a[s] = A[s];
      b[s] = B[s];
    }
    return 3;
  }
  if (integrator == ADG_RK_LS4) {
    const double A[5] = {0.0, -567301805773.0 / 1357537059087.0,
                         -2404267990393.0 / 2016746695238.0,
                         -3550918686646.0 / 2091501179385.0,
                         -1275806237668.0 / 842570457699.0};
    const double B[5] = {1432997174477.0 / 9575080441755.0,
                         5161836677717.0 / 13612068292357.0,
                         1720146321549.0 / 2090206949498.0,
                         3134564353537.0 / 4481467310338.0,
                         2277821191437.0 / 14882151754819.0};
    for (int s = 0; s < 5; ++s) {
      a[s] = A[s];
      b[s] = B[s];
    }
    return 5;
  }
  return 0;
}

int n_pe_faces(const adg_config &c) {
  if (c.n_pe <= 1) return 0;
  return c.bc_left == ADG_BC_PERIODIC ? c.n_pe : c.n_pe - 1;
}

// Layout of a config's (sub)domain; false for a bad PE range.
bool part_info(const adg_config &c, PartInfo *out) {
  PartInfo r;
  const int64_t N = c.n_elem, P = c.n_pe;
  const bool per = c.bc_left == ADG_BC_PERIODIC;
  r.n_local = c.n_elem;
  r.npf = r.npf_draw = n_pe_faces(c);
  r.dx = c.length / c.n_elem;
  if (c.pe_end == 0) {
    if (c.pe_begin != 0) return false;
  } else {
    if (c.pe_begin < 0 || c.pe_begin >= c.pe_end || c.pe_end > c.n_pe) return false;
    if (!(c.pe_begin == 0 && c.pe_end == c.n_pe)) {
      r.part = true;
      r.pb = c.pe_begin;
      r.pe = c.pe_end;
      r.cut_l = (c.pe_begin > 0 || per) ? 1 : 0;
      r.cut_r = (c.pe_end < c.n_pe || per) ? 1 : 0;
      const int64_t e0 = (int64_t)c.pe_begin * N / P, e1 = (int64_t)c.pe_end * N / P;
      r.elem0 = (int)e0 - r.cut_l;
      r.n_local = (int)(e1 - e0) + r.cut_l + r.cut_r;
      r.npf = r.cut_l + (c.pe_end - c.pe_begin - 1) + r.cut_r;
      r.face_base = c.pe_begin - r.cut_l;
    }
  }
  *out = r;
  return true;
}

// The instance each config describes: a subdomain becomes a bounded mesh of its
// n_local elements whose cut sides end in outflow boundaries beyond the buffer
// elements, with npf + 1 "PEs" so that n_pe_faces counts its PE faces (the PE
// table itself comes from part_info, not from the even split).
int localise(const adg_config *cfgs, int n, std::vector<adg_config> &lc,
             std::vector<PartInfo> &pi) {
  lc.assign(cfgs, cfgs + n);
  pi.resize(n);
  for (int k = 0; k < n; ++k) {
    if (!part_info(cfgs[k], &pi[k])) return ADG_ERR_ARG;
    if (!pi[k].part) continue;
    if (cfgs[k].viscous) return ADG_ERR_ARG;
    adg_config &c = lc[k];
    c.n_elem = pi[k].n_local;
    c.n_pe = pi[k].npf + 1;
    if (pi[k].cut_l) c.bc_left = ADG_BC_OUTFLOW;
    if (pi[k].cut_r) c.bc_right = ADG_BC_OUTFLOW;
  }
  return ADG_OK;
}

// Lay out every buffer; with dry = true only measures.
size_t layout(adg_ctx *ctx, const adg_config *cfgs, Carver &cv) {
  int ns = ctx->ns, nr = ctx->nr, nv = ns + 2;
  int nrr = nr > 0 ? nr : 1;
  Mech &M = ctx->mech;
  M.sp = (const double *)cv.take(sizeof(double) * SP_NFIELDS * ns);
  M.rx = (const Rxn *)cv.take(sizeof(Rxn) * nrr);
  M.rxf = (const DF *)cv.take(sizeof(DF) * 6 * nrr);
  M.sx_off = (const int *)cv.take(sizeof(int) * (ns + 1));
  M.sx = (const int *)cv.take(sizeof(int) * (M.nterm > 0 ? M.nterm : 1));
  ctx->err_all = (int *)cv.take(sizeof(int) * 4 * ctx->n_inst);
  ctx->d_insts = (Inst *)cv.take(sizeof(Inst) * ctx->n_inst);
  ctx->d_steps = (int64_t *)cv.take(sizeof(int64_t) * ctx->n_inst);
  ctx->d_offs = (int64_t *)cv.take(sizeof(int64_t) * (ctx->n_inst + 1));
  int max_pe = 1;
  for (int k = 0; k < ctx->n_inst; ++k) max_pe = cfgs[k].n_pe > max_pe ? cfgs[k].n_pe : max_pe;
  ctx->pub_in = (int *)cv.take(sizeof(int) * max_pe);
  ctx->pub_pre = (int *)cv.take(sizeof(int) * max_pe);
  ctx->agree = (unsigned long long *)cv.take(sizeof(unsigned long long) * max_pe *
                                              ADG_MAX_STAGES * (MAXD + 1));
  ctx->delay_hist = (unsigned long long *)cv.take(sizeof(unsigned long long) * 2 * (MAXD + 1));
  // groups of equal degree and precision: tile sizes and tables
  ctx->n_groups = 0;
  for (int gk = 0; gk < ADG_MAX_GROUPS; ++gk) {
    const int r = gk % (3 * ADG_MAX_P), S = gk < 3 * ADG_MAX_P ? 3 : 5;
    const int Q = 2 + r / 3, prec = r % 3;
    auto member = [&](int k) {
      return cfgs[k].p + 1 == Q && cfgs[k].precision == prec &&
             rk_stages(cfgs[k].integrator) == S;
    };
    int64_t total = 0, tiles = 0, blocks = 0;
    bool lim = false, any = false;
    int O = 1;
    for (int k = 0; k < ctx->n_inst; ++k)
      if (member(k)) {
        any = true;
        total += cfgs[k].n_elem;
        lim = lim || cfgs[k].limiter != ADG_LIM_NONE;
        if (cfgs[k].at_order > O) O = cfgs[k].at_order;
      }
    if (!any) continue;
    Group &G = ctx->groups[ctx->n_groups++];
    G.Q = Q;
    G.prec = prec;
    G.mixed = prec != ADG_FP64;
    G.S = S;
    G.O = O;
    for (int k = 0; k < ctx->n_inst; ++k)
      if (member(k) && cfgs[k].viscous) G.visc = true;
    G.TE = stage_tile(M, Q, O, G.prec, G.visc);
    // smaller tiles when the group would not fill two CTAs per SM
    int64_t target = (total + 2 * 152 - 1) / (2 * 152);
    if (target < G.TE) G.TE = target < 4 ? 4 : (int)target;
    G.NT = stage_threads(G.TE, Q, nr);
    G.EPB = limiter_elems_per_block(total, G.mixed);
    const int epb = G.EPB, epb_min = G.mixed ? 8 : 16;
    int64_t max_tiles = 0, max_blocks = 0;
    for (int k = 0; k < ctx->n_inst; ++k)
      if (member(k)) {
        tiles += (cfgs[k].n_elem + G.TE - 1) / G.TE;
        max_tiles += (cfgs[k].n_elem + kMinTile - 1) / kMinTile;
        blocks += (cfgs[k].n_elem + epb - 1) / epb;
        max_blocks += (cfgs[k].n_elem + epb_min - 1) / epb_min;
      }
    G.n_tiles = (int)tiles;
    G.n_blocks = (int)blocks;
    G.any_limiter = lim;
    // room for the tile and block tables of the smallest tile and limiter block
    // the autotuner may pick
    G.d_tiles = (int2 *)cv.take(sizeof(int2) * max_tiles);
    G.d_blocks = (int2 *)cv.take(sizeof(int2) * max_blocks);
  }
  for (int k = 0; k < ctx->n_inst; ++k) {
    const adg_config &c = cfgs[k];
    InstHost &h = ctx->inst[k];
    Inst &I = h.d;
    int N = c.n_elem, Q = c.p + 1, npf = n_pe_faces(c);
    size_t st = (size_t)nv * N * Q;
    I.wn = (double *)cv.take(sizeof(double) * st);
    I.wa = (double *)cv.take(sizeof(double) * st);
    I.wb = (double *)cv.take(sizeof(double) * st);
    I.wpre = (double *)cv.take(sizeof(double) * st);
    const int S = rk_stages(c.integrator);
    I.wq = (c.integrator != ADG_RK_SSP3) ? (double *)cv.take(sizeof(double) * st) : nullptr;
    // ring depth 2d + o: the synchronous modes need d + o levels, the
    // unsynchronised one up to 2d + o (a neighbour may run d steps ahead)
    size_t rs = (size_t)(2 * c.max_delay + c.at_order) * S * (npf > 0 ? npf : 1) * 2 * nv;
    I.ring_in = (double *)cv.take(sizeof(double) * rs);
    I.ring_pre = (double *)cv.take(sizeof(double) * rs * Q);
    I.qx = c.viscous ? (double *)cv.take(sizeof(double) * st) : nullptr;
    I.ring_q = c.viscous ? (double *)cv.take(sizeof(double) * rs) : nullptr;
    I.flags = (uint8_t *)cv.take((size_t)S * N);
    I.count = (int32_t *)cv.take(sizeof(int32_t) * N);
    I.pf_of_left = (const int *)cv.take(sizeof(int) * N);
    I.pf_of_right = (const int *)cv.take(sizeof(int) * N);
    I.pf_elem = (const int *)cv.take(sizeof(int) * 2 * (npf > 0 ? npf : 1));
    h.prim = (double *)cv.take(sizeof(double) * (size_t)(ns + 3) * N * Q);
    I.err = ctx->err_all ? ctx->err_all + 4 * k : nullptr;
  }
  return cv.off;
}

thread_local char g_last_error[256];

}  // namespace

// Stage tile table of a group for its current tile size.
static cudaError_t upload_tiles(adg_ctx *ctx, Group &G) {
  std::vector<int2> tl;
  for (int k = 0; k < ctx->n_inst; ++k) {
    const Inst &I = ctx->inst[k].d;
    if (I.p + 1 != G.Q || I.mixed != G.prec || I.n_stages != G.S) continue;
    for (int e = 0; e < I.n_elem; e += G.TE) tl.push_back(make_int2(k, e));
  }
  G.n_tiles = (int)tl.size();
  return cudaMemcpy(G.d_tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice);
}

// Limiter block table of a group for its current elements per CTA.
static cudaError_t upload_blocks(adg_ctx *ctx, Group &G) {
  std::vector<int2> bl;
  for (int k = 0; k < ctx->n_inst; ++k) {
    const Inst &I = ctx->inst[k].d;
    if (I.p + 1 != G.Q || I.mixed != G.prec || I.n_stages != G.S) continue;
    for (int e = 0; e < I.n_elem; e += G.EPB) bl.push_back(make_int2(k, e));
  }
  G.n_blocks = (int)bl.size();
  return cudaMemcpy(G.d_blocks, bl.data(), sizeof(int2) * bl.size(), cudaMemcpyHostToDevice);
}

// Elements per limiter CTA that the limiter is built for: 8, 16 and 32 in the
// mixed variants, 16 and 32 in FP64.
static bool limiter_block_ok(const Group &G, int epb) {
  return epb == 16 || epb == 32 || (G.mixed && epb == 8);
}

extern "C" {

const char *adg_error_string(int code) {
  switch (code) {
    case ADG_OK: return "ok";
    case ADG_ERR_ARG: return "invalid argument";
    case ADG_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case ADG_ERR_NOMEM: return "out of device memory or workspace too small";
    case ADG_ERR_NONPHYSICAL: return "non-physical state (density or temperature)";
    case ADG_ERR_HISTORY: return "delayed level missing from the history ring";
    case ADG_ERR_NOLIB: return "no CUDA device";
    case ADG_ERR_TIMEOUT: return "a wait of the unsynchronised mode gave up";
  }
  return "unknown error";
}

static int cuda_fail(cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "CUDA error: %s", cudaGetErrorString(e));
  return ADG_ERR_CUDA;
}

#define CK(x)                              \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

int adg_workspace_bytes(const adg_mechanism *mech, const adg_config *cfgs_in, int n,
                        size_t *bytes) {
  int rc = check_args(mech, cfgs_in, n);
  if (rc) return rc;
  if (!bytes) return ADG_ERR_ARG;
  std::vector<adg_config> lc;
  std::vector<PartInfo> pi;
  rc = localise(cfgs_in, n, lc, pi);
  if (rc) return rc;
  const adg_config *cfgs = lc.data();
  adg_ctx tmp;
  tmp.n_inst = n;
  tmp.ns = mech->n_species;
  tmp.nr = mech->n_reactions;
  tmp.mech.ns = tmp.ns;
  tmp.mech.nr = tmp.nr;
  tmp.mech.nterm = count_terms(mech);
  tmp.inst.resize(n);
  tmp.err_all = nullptr;
  Carver cv{nullptr, 0, 0, true};
  *bytes = layout(&tmp, cfgs, cv) + 256;
  return ADG_OK;
}

int adg_delay_table(const adg_config *c, int64_t step0, int n_steps, uint8_t *out) {
  if (!c || !out || n_steps < 0 || c->max_delay < 0 || c->max_delay > ADG_MAX_DELAY)
    return ADG_ERR_ARG;
  if (c->delay_mode == ADG_SAA && !c->delay_probs) return ADG_ERR_ARG;
  double cum[MAXD + 1];
  double acc = 0.0;
  for (int k = 0; k <= c->max_delay; ++k) {
    acc += (c->delay_mode == ADG_SAA) ? c->delay_probs[k] : 0.0;
    cum[k] = acc;
  }
  PartInfo pt;
  if (!part_info(*c, &pt)) return ADG_ERR_ARG;
  const int npf = pt.npf;
  for (int s = 0; s < n_steps; ++s)
    for (int f = 0; f < npf; ++f)
      out[(size_t)s * npf + f] =
          (uint8_t)draw_delay(c->delay_mode, c->max_delay, c->seed, cum, step0 + s,
                              face_number(f, pt.face_base, pt.npf_draw));
  return ADG_OK;
}

int adg_create(const adg_mechanism *mech, const adg_config *cfgs_in, int n, void *workspace,
               size_t ws_bytes, adg_ctx **out) {
  if (!out) return ADG_ERR_ARG;
  *out = nullptr;
  int rc = check_args(mech, cfgs_in, n);
  if (rc) return rc;
  // subdomains become instances of their local elements (buffers included)
  std::vector<adg_config> lc;
  std::vector<PartInfo> pinfo;
  rc = localise(cfgs_in, n, lc, pinfo);
  if (rc) return rc;
  const adg_config *cfgs = lc.data();
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return ADG_ERR_NOLIB;
  adg_ctx *ctx = new (std::nothrow) adg_ctx();
  if (!ctx) return ADG_ERR_NOMEM;
  ctx->n_inst = n;
  ctx->ns = mech->n_species;
  ctx->nr = mech->n_reactions;
  ctx->mech.ns = ctx->ns;
  ctx->mech.nr = ctx->nr;
  ctx->mech.nterm = count_terms(mech);
  ctx->inst.resize(n);
  for (int k = 0; k < n; ++k) ctx->inst[k].part = pinfo[k];
  ctx->last_stream = 0;
  ctx->unsync_polls = 1ll << 22;  // polls of ~0.5 us: a few seconds
  ctx->unsync_withheld = -1;
  ctx->unsync_slow_pe = -1;
  ctx->unsync_slow_us = 0;
  ctx->err_all = nullptr;
  ctx->ev_used = 0;
  ctx->timing = false;
  ctx->capturing_timed = false;
  ctx->kms[0] = ctx->kms[1] = ctx->kms[2] = 0.0;
  ctx->kcount[0] = ctx->kcount[1] = ctx->kcount[2] = 0;
  ctx->span[0] = ctx->span[1] = nullptr;
  ctx->tgraph = nullptr;
  ctx->texec = nullptr;
  ctx->cap_stream = nullptr;
  ctx->fork_ev = nullptr;
  for (int g = 0; g < ADG_MAX_GROUPS; ++g) {
    ctx->branch[g] = nullptr;
    ctx->join_ev[g] = nullptr;
  }
  ctx->graph = nullptr;
  ctx->exec = nullptr;
  ctx->graph_ok = false;
  ctx->io_stream = ctx->out_stream = nullptr;
  for (int j = 0; j < kIoParts * ADG_MAX_GROUPS; ++j) ctx->io_ev[j] = ctx->done_ev[j] = nullptr;
  ctx->io_graph = nullptr;
  ctx->io_exec = nullptr;
  ctx->io_in = nullptr;
  ctx->io_out = nullptr;
  Carver dry{nullptr, 0, 0, true};
  size_t need = layout(ctx, cfgs, dry) + 256;
  if (workspace) {
    if (ws_bytes < need || ((uintptr_t)workspace & 255)) {
      delete ctx;
      return ADG_ERR_NOMEM;
    }
    ctx->mem = workspace;
    ctx->owns_mem = false;
  } else {
    if (cudaMalloc(&ctx->mem, need) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return ADG_ERR_NOMEM;
    }
    ctx->owns_mem = true;
  }
  ctx->bytes = need;
  Carver cv{(char *)ctx->mem, 0, need, false};
  layout(ctx, cfgs, cv);
  int ns = ctx->ns, nr = ctx->nr, nv = ns + 2;
  Mech &M = ctx->mech;
  M.ns = ns;
  M.nr = nr;
  // mechanism tables: species fields, packed reactions, species-reaction incidence
  int rc2 = ADG_OK;
  {
    std::vector<double> sp(SP_NFIELDS * ns);
    std::vector<Rxn> rx(nr > 0 ? nr : 1);
    std::vector<int> sx_off(ns + 1), sx(M.nterm > 0 ? M.nterm : 1);
    if (pack_mechanism(mech, sp.data(), rx.data(), sx_off.data(), sx.data()) != M.nterm)
      rc2 = ADG_ERR_ARG;
    std::vector<DF> rxf(6 * (nr > 0 ? nr : 1));
    pack_rxf(rx.data(), nr, rxf.data());
    if (cudaMemcpy((void *)M.sp, sp.data(), sizeof(double) * sp.size(), cudaMemcpyHostToDevice) ||
        (nr > 0 && cudaMemcpy((void *)M.rx, rx.data(), sizeof(Rxn) * nr, cudaMemcpyHostToDevice)) ||
        (nr > 0 &&
         cudaMemcpy((void *)M.rxf, rxf.data(), sizeof(DF) * 6 * nr, cudaMemcpyHostToDevice)) ||
        cudaMemcpy((void *)M.sx_off, sx_off.data(), sizeof(int) * (ns + 1),
                   cudaMemcpyHostToDevice) ||
        (M.nterm > 0 && cudaMemcpy((void *)M.sx, sx.data(), sizeof(int) * M.nterm,
                                   cudaMemcpyHostToDevice)))
      rc2 = ADG_ERR_CUDA;
  }
  if (cudaMemset(ctx->err_all, 0, sizeof(int) * 4 * n) ||
      cudaMemset(ctx->delay_hist, 0, sizeof(unsigned long long) * 2 * (MAXD + 1)))
    rc2 = ADG_ERR_CUDA;
  // basis tables in constant memory
  {
    Basis tables[ADG_MAX_P];
    make_tables(tables);
    if (upload_basis(tables) != cudaSuccess) rc2 = ADG_ERR_CUDA;
  }
  // instances
  for (int k = 0; k < n && rc2 == ADG_OK; ++k) {
    const adg_config &c = cfgs[k];
    InstHost &h = ctx->inst[k];
    Inst &I = h.d;
    int N = c.n_elem, Q = c.p + 1, npf = n_pe_faces(c);
    I.n_elem = N;
    I.p = c.p;
    I.nv = nv;
    I.npf = npf;
    I.depth = 2 * c.max_delay + c.at_order;
    I.n_stages = rk_stages(c.integrator);
    for (int s = 0; s < ADG_MAX_STAGES; ++s) I.rk_a[s] = I.rk_b[s] = 0.0;
    I.lserk = lserk_coefficients(c.integrator, I.rk_a, I.rk_b) > 0;
    I.viscous = c.viscous;
    I.pad0 = 0;
    I.mu_ref = c.viscous ? c.mu_ref : 0.0;
    I.ln_T_mu = c.viscous ? log(c.T_mu) : 0.0;
    I.mu_exp = c.viscous ? c.mu_exp : 0.0;
    I.inv_prandtl = c.viscous ? 1.0 / c.prandtl : 0.0;
    I.at_order = c.at_order;
    I.bc_left = c.bc_left;
    I.bc_right = c.bc_right;
    I.flux = c.flux;
    I.limiter = c.limiter;
    I.delay_mode = c.delay_mode;
    I.max_delay = c.max_delay;
    I.dx = h.part.part ? h.part.dx : c.length / N;
    I.dt = c.dt;
    I.tvb = c.tvb_M * I.dx * I.dx;
    I.mixed = c.precision;
    I.face_base = h.part.face_base;
    I.npf_draw = h.part.part ? h.part.npf_draw : npf;
    I.ind_floor = indicator_guard(c.precision);
    I.ind_floor_p = indicator_guard_p(c.precision);
    I.seed = c.seed;
    I.instance = k;
    double acc = 0.0;
    for (int d = 0; d <= MAXD; ++d) {
      if (d <= c.max_delay) acc += (c.delay_mode == ADG_SAA) ? c.delay_probs[d] : 0.0;
      I.cum[d] = acc;
    }
    for (int d = 0; d <= MAXD; ++d) {
      double w[MAXO];
      for (int m = 0; m < MAXO; ++m) w[m] = 0.0;
      if (d <= c.max_delay) at_weights(c.at_order, d, w);
      for (int m = 0; m < MAXO; ++m) I.at[d][m] = w[m];
    }
    // PE partition (Sec. 4): PE q owns elements [q N / P, (q+1) N / P)
    std::vector<int> pl(N, -1), pr(N, -1), pe(2 * (npf > 0 ? npf : 1), -1);
    int P = c.n_pe;
    const PartInfo &pt = h.part;
    for (int f = 0; f < npf; ++f) {
      int right;
      if (!pt.part)
        right = (int)(((int64_t)((f + 1) % P) * N) / P);
      else if (pt.cut_l && f == 0)
        right = 1;  // the left buffer | the first owned element
      else if (pt.cut_r && f == npf - 1)
        right = N - 1;  // the last owned element | the right buffer
      else  // whole-domain face g sits left of the first element of PE g + 1
        right = (int)(((int64_t)(pt.pb - pt.cut_l + f + 1) * cfgs_in[k].n_elem) /
                      cfgs_in[k].n_pe) - pt.elem0;
      int left = (right == 0) ? N - 1 : right - 1;
      pr[left] = f;
      pl[right] = f;
      pe[2 * f] = left;
      pe[2 * f + 1] = right;
    }
    if (cudaMemcpy((void *)I.pf_of_left, pl.data(), sizeof(int) * N, cudaMemcpyHostToDevice) ||
        cudaMemcpy((void *)I.pf_of_right, pr.data(), sizeof(int) * N, cudaMemcpyHostToDevice) ||
        cudaMemcpy((void *)I.pf_elem, pe.data(), sizeof(int) * pe.size(), cudaMemcpyHostToDevice) ||
        cudaMemset(I.flags, 0, (size_t)I.n_stages * N) || cudaMemset(I.count, 0, sizeof(int32_t) * N) ||
        cudaMemset(I.wn, 0, sizeof(double) * (size_t)nv * N * Q) ||
        (I.qx && cudaMemset(I.qx, 0, sizeof(double) * (size_t)nv * N * Q)))
      rc2 = ADG_ERR_CUDA;
    h.n = 0;
    h.n_pe = c.n_pe;
    I.step = ctx->d_steps + k;
  }
  if (rc2 == ADG_OK) {
    std::vector<Inst> hi(n);
    for (int k = 0; k < n; ++k) hi[k] = ctx->inst[k].d;
    std::vector<int64_t> offs(n + 1, 0);
    for (int k = 0; k < n; ++k)
      offs[k + 1] = offs[k] + (int64_t)hi[k].nv * hi[k].n_elem * (hi[k].p + 1);
    if (cudaMemcpy(ctx->d_insts, hi.data(), sizeof(Inst) * n, cudaMemcpyHostToDevice) ||
        cudaMemcpy(ctx->d_offs, offs.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice) ||
        cudaMemset(ctx->d_steps, 0, sizeof(int64_t) * n))
      rc2 = ADG_ERR_CUDA;
    // each group's instances (adg_step_io's copies)
    for (int gi = 0; gi < ctx->n_groups; ++gi) {
      Group &G = ctx->groups[gi];
      G.members.clear();
      for (int k = 0; k < n; ++k)
        if (cfgs[k].p + 1 == G.Q && cfgs[k].precision == G.prec &&
            rk_stages(cfgs[k].integrator) == G.S)
          G.members.push_back(k);
    }
    for (int gi = 0; gi < ctx->n_groups && rc2 == ADG_OK; ++gi) {
      Group &G = ctx->groups[gi];
      if (upload_tiles(ctx, G) != cudaSuccess || upload_blocks(ctx, G) != cudaSuccess)
        rc2 = ADG_ERR_CUDA;
    }
    if (prepare_kernels(nv, ns, nr) != cudaSuccess) rc2 = ADG_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      rc2 = ADG_ERR_CUDA;
    if (ctx->n_groups > 1 && rc2 == ADG_OK) {
      if (cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess)
        rc2 = ADG_ERR_CUDA;
      for (int g = 0; g < ctx->n_groups && rc2 == ADG_OK; ++g)
        if (cudaStreamCreateWithFlags(&ctx->branch[g], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->join_ev[g], cudaEventDisableTiming) != cudaSuccess)
          rc2 = ADG_ERR_CUDA;
    }
  }
  if (rc2 != ADG_OK) {
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    destroy_branches(ctx);
    if (ctx->owns_mem) cudaFree(ctx->mem);
    delete ctx;
    return rc2;
  }
  *out = ctx;
  return ADG_OK;
}

void adg_destroy(adg_ctx *ctx) {
  if (!ctx) return;
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
  if (ctx->texec) cudaGraphExecDestroy(ctx->texec);
  for (cudaEvent_t e : ctx->span)
    if (e) cudaEventDestroy(e);
  if (ctx->tgraph) cudaGraphDestroy(ctx->tgraph);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  if (ctx->io_exec) cudaGraphExecDestroy(ctx->io_exec);
  if (ctx->io_graph) cudaGraphDestroy(ctx->io_graph);
  for (int j = 0; j < kIoParts * ADG_MAX_GROUPS; ++j) {
    if (ctx->io_ev[j]) cudaEventDestroy(ctx->io_ev[j]);
    if (ctx->done_ev[j]) cudaEventDestroy(ctx->done_ev[j]);
  }
  if (ctx->io_stream) cudaStreamDestroy(ctx->io_stream);
  if (ctx->out_stream) cudaStreamDestroy(ctx->out_stream);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  destroy_branches(ctx);
  if (ctx->owns_mem) cudaFree(ctx->mem);
  delete ctx;
}

static int inst_ok(adg_ctx *ctx, int k) {
  return ctx && k >= 0 && k < ctx->n_inst;
}

// Step counter to 0 (the history ring is then never read before it is written
// again) and flags cleared.
static cudaError_t reset_history(adg_ctx *ctx, int k, cudaStream_t st) {
  InstHost &h = ctx->inst[k];
  h.n = 0;
  cudaError_t e = cudaMemsetAsync(ctx->d_steps + k, 0, sizeof(int64_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h.d.count, 0, sizeof(int32_t) * h.d.n_elem, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h.d.flags, 0, (size_t)h.d.n_stages * h.d.n_elem, st);
  return e;
}

int adg_set_primitive(adg_ctx *ctx, int k, const double *prim) {
  if (!inst_ok(ctx, k) || !prim) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  size_t n = (size_t)(ctx->ns + 3) * h.d.n_elem * (h.d.p + 1);
  CK(cudaMemcpy(h.prim, prim, sizeof(double) * n, cudaMemcpyHostToDevice));
  CK(launch_project(ctx->mech, h.d, h.prim, h.d.wn, 0));
  CK(reset_history(ctx, k, 0));
  CK(cudaDeviceSynchronize());
  return ADG_OK;
}

int adg_set_state(adg_ctx *ctx, int k, const double *w) {
  if (!inst_ok(ctx, k) || !w) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  size_t n = (size_t)h.d.nv * h.d.n_elem * (h.d.p + 1);
  CK(cudaMemcpyAsync(h.d.wn, w, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->last_stream));
  CK(reset_history(ctx, k, ctx->last_stream));
  CK(cudaStreamSynchronize(ctx->last_stream));
  return ADG_OK;
}

int adg_set_state_device(adg_ctx *ctx, int k, const double *w, void *stream) {
  if (!inst_ok(ctx, k) || !w) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  size_t n = (size_t)h.d.nv * h.d.n_elem * (h.d.p + 1);
  CK(cudaMemcpyAsync(h.d.wn, w, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                     (cudaStream_t)stream));
  CK(reset_history(ctx, k, (cudaStream_t)stream));
  ctx->last_stream = (cudaStream_t)stream;
  return ADG_OK;
}

int adg_get_state(adg_ctx *ctx, int k, double *w) {
  if (!inst_ok(ctx, k) || !w) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  size_t n = (size_t)h.d.nv * h.d.n_elem * (h.d.p + 1);
  CK(cudaMemcpyAsync(w, h.d.wn, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->last_stream));
  CK(cudaStreamSynchronize(ctx->last_stream));
  return ADG_OK;
}

int adg_get_state_device(adg_ctx *ctx, int k, double *w, void *stream) {
  if (!inst_ok(ctx, k) || !w) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  size_t n = (size_t)h.d.nv * h.d.n_elem * (h.d.p + 1);
  CK(cudaMemcpyAsync(w, h.d.wn, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                     (cudaStream_t)stream));
  return ADG_OK;
}

// Event pair around one launch while the timing graph is captured.
static cudaError_t timed_begin(adg_ctx *ctx, int kind, cudaStream_t st) {
  if (!ctx->capturing_timed) return cudaSuccess;
  while (ctx->ev_used + 2 > ctx->ev.size()) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ctx->ev.push_back(e);
    ctx->ev_kind.push_back(0);
  }
  ctx->ev_kind[ctx->ev_used] = kind;
  // external record: an event node of the graph, readable after each replay
  return cudaEventRecordWithFlags(ctx->ev[ctx->ev_used], st, cudaEventRecordExternal);
}

static cudaError_t timed_end(adg_ctx *ctx, cudaStream_t st) {
  if (!ctx->capturing_timed) return cudaSuccess;
  cudaError_t r = cudaEventRecordWithFlags(ctx->ev[ctx->ev_used + 1], st, cudaEventRecordExternal);
  ctx->ev_used += 2;
  return r;
}

// Arguments of the auxiliary kernel of a group: its limiter block table.
static LimArgs aux_args(const adg_ctx *ctx, const Group &G, int s) {
  LimArgs L;
  L.insts = ctx->d_insts;
  L.blocks = G.d_blocks;
  L.s = s;
  L.EPB = G.EPB;
  return L;
}

// A part of a group's launches: stage tiles [tile0, tile0 + n_tiles) and
// limiter blocks [blk0, blk0 + n_blocks) of its tables (n_tiles < 0: all).
// Tiles and blocks never span instances, so the instances of a part step
// independently of the rest of the group.
struct Part {
  int tile0 = 0, n_tiles = -1, blk0 = 0, n_blocks = -1;
};

// The stages of one group's step: per RK stage, the auxiliary kernel (viscous
// groups), the stage kernel and the limiter; half 0 only the first two, half 1
// only the limiter, any other value all three. `part` limits the launches to a
// range of the group's instances (inviscid groups only).
static int enqueue_group(adg_ctx *ctx, int gi, int s, cudaStream_t st, int half = -1,
                         Part part = Part()) {
  const Group &G = ctx->groups[gi];
  if (s >= G.S) return ADG_OK;
  const int n_tiles = part.n_tiles < 0 ? G.n_tiles : part.n_tiles;
  const int n_blocks = part.n_tiles < 0 ? G.n_blocks : part.n_blocks;
  if (half != 1) {
    StageArgs A;
    A.insts = ctx->d_insts;
    A.tiles = G.d_tiles + part.tile0;
    A.s = s;
    A.TE = G.TE;
    A.NT = G.NT;
    A.O = G.O;
    A.visc = G.visc;
    CK(timed_begin(ctx, 0, st));
    // viscous groups: the LDG auxiliary variable of the stage input first
    // (timed with the stage kernel)
    if (G.visc) CK(launch_aux(aux_args(ctx, G, s), G.Q, G.n_blocks, st));
    CK(launch_stage(ctx->mech, A, G.Q, G.prec, n_tiles, st));
    CK(timed_end(ctx, st));
  }
  if (half == 0 || !G.any_limiter) return ADG_OK;
  LimArgs L;
  L.insts = ctx->d_insts;
  L.blocks = G.d_blocks + part.blk0;
  L.s = s;
  L.EPB = G.EPB;
  CK(timed_begin(ctx, 1, st));
  CK(launch_limiter(ctx->mech, L, G.Q, G.mixed, ctx->ns + 2, n_blocks, st));
  CK(timed_end(ctx, st));
  return ADG_OK;
}

// One step of every instance, then the step counters advance. Groups hold
// independent instances, so in the plain graph (concurrent) each group's
// stages form a branch of their own, forked from and joined to `st`: the GPU
// runs the groups side by side and fills one group's wave tails with another's
// CTAs. The timing graph runs the groups one after the other, so that every
// kernel's time is its own.
static int enqueue_step(adg_ctx *ctx, cudaStream_t st, bool concurrent) {
  int max_s = 0;
  for (int gi = 0; gi < ctx->n_groups; ++gi)
    max_s = ctx->groups[gi].S > max_s ? ctx->groups[gi].S : max_s;
  if (concurrent && ctx->n_groups > 1 && ctx->fork_ev) {
    CK(cudaEventRecord(ctx->fork_ev, st));
    for (int gi = 0; gi < ctx->n_groups; ++gi) {
      cudaStream_t b = ctx->branch[gi];
      CK(cudaStreamWaitEvent(b, ctx->fork_ev, 0));
      for (int s = 0; s < ctx->groups[gi].S; ++s) {
        int rc = enqueue_group(ctx, gi, s, b);
        if (rc != ADG_OK) return rc;
      }
      CK(cudaEventRecord(ctx->join_ev[gi], b));
      CK(cudaStreamWaitEvent(st, ctx->join_ev[gi], 0));
    }
  } else {
    for (int s = 0; s < max_s; ++s)
      for (int gi = 0; gi < ctx->n_groups; ++gi) {
        int rc = enqueue_group(ctx, gi, s, st);
        if (rc != ADG_OK) return rc;
      }
  }
  CK(launch_advance(ctx->d_steps, ctx->n_inst, st));
  return ADG_OK;
}

// The step as a CUDA graph, captured once on the context's private stream;
// the timing variant records an event pair around every kernel.
static int capture(adg_ctx *ctx, bool timed, cudaGraph_t *graph, cudaGraphExec_t *exec) {
  ctx->capturing_timed = timed;
  ctx->ev_used = 0;
  if (timed && !ctx->span[0]) {
    CK(cudaEventCreate(&ctx->span[0]));
    CK(cudaEventCreate(&ctx->span[1]));
  }
  CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = ADG_OK;
  if (timed && cudaEventRecordWithFlags(ctx->span[0], ctx->cap_stream,
                                        cudaEventRecordExternal) != cudaSuccess)
    rc = ADG_ERR_CUDA;
  if (rc == ADG_OK) rc = enqueue_step(ctx, ctx->cap_stream, !timed);
  if (rc == ADG_OK && timed &&
      cudaEventRecordWithFlags(ctx->span[1], ctx->cap_stream, cudaEventRecordExternal) !=
          cudaSuccess)
    rc = ADG_ERR_CUDA;
  // the capture always ends, so that the private stream is usable again
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  ctx->capturing_timed = false;
  if (rc != ADG_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != ADG_OK ? rc : cuda_fail(e);
  }
  e = cudaGraphInstantiate(exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e);
  }
  *graph = g;
  return ADG_OK;
}

static int ensure_graph(adg_ctx *ctx) {
  if (ctx->graph_ok) return ADG_OK;
  int rc = capture(ctx, false, &ctx->graph, &ctx->exec);
  if (rc == ADG_OK) ctx->graph_ok = true;
  return rc;
}

int adg_step(adg_ctx *ctx, int n_steps, void *stream) {
  if (!ctx || n_steps < 0) return ADG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  if (n_steps == 0) return ADG_OK;
  if (ctx->timing) {
    // the timing graph, one step at a time: wait for it and add up its kernels
    if (!ctx->texec) {
      int rc = capture(ctx, true, &ctx->tgraph, &ctx->texec);
      if (rc != ADG_OK) return rc;
    }
    for (int it = 0; it < n_steps; ++it) {
      CK(cudaGraphLaunch(ctx->texec, st));
      CK(cudaStreamSynchronize(st));
      for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]));
        ctx->kms[ctx->ev_kind[i]] += t;
        ctx->kcount[ctx->ev_kind[i]] += 1;
      }
      float t = 0.0f;
      CK(cudaEventElapsedTime(&t, ctx->span[0], ctx->span[1]));
      ctx->kms[2] += t;
      ctx->kcount[2] += 1;
    }
  } else {
    int rc = ensure_graph(ctx);
    if (rc != ADG_OK) return rc;
    for (int it = 0; it < n_steps; ++it) CK(cudaGraphLaunch(ctx->exec, st));
  }
  for (InstHost &h : ctx->inst) h.n += n_steps;
  return ADG_OK;
}

int adg_part_layout(const adg_config *cfg, int *n_local, int *elem0, int *cut_left,
                    int *cut_right) {
  if (!cfg || cfg->n_elem < 1 || cfg->n_pe < 1 || cfg->n_pe > cfg->n_elem || !(cfg->length > 0.0))
    return ADG_ERR_ARG;
  PartInfo pt;
  if (!part_info(*cfg, &pt)) return ADG_ERR_ARG;
  if (n_local) *n_local = pt.n_local;
  if (elem0) *elem0 = pt.elem0;
  if (cut_left) *cut_left = pt.cut_l;
  if (cut_right) *cut_right = pt.cut_r;
  return ADG_OK;
}

int adg_step_stage(adg_ctx *ctx, int stage, int half, void *stream) {
  if (!ctx || stage < 0 || half < 0 || half > 1) return ADG_ERR_ARG;
  int max_s = 0;
  for (int gi = 0; gi < ctx->n_groups; ++gi)
    max_s = ctx->groups[gi].S > max_s ? ctx->groups[gi].S : max_s;
  if (stage >= max_s) return ADG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  for (int gi = 0; gi < ctx->n_groups; ++gi) {
    int rc = enqueue_group(ctx, gi, stage, st, half);
    if (rc != ADG_OK) return rc;
  }
  if (half == 1 && stage == max_s - 1) {
    CK(launch_advance(ctx->d_steps, ctx->n_inst, st));
    for (InstHost &h : ctx->inst) h.n += 1;
  }
  return ADG_OK;
}

int adg_part_block(adg_ctx *ctx, int k, int what, int side, int stage, double *blk, int import,
                   void *stream) {
  if (!inst_ok(ctx, k) || !blk || side < 0 || side > 1 ||
      (what != ADG_PART_INPUT && what != ADG_PART_PRELIMIT))
    return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  const PartInfo &pt = h.part;
  const Inst &I = h.d;
  if (!pt.part || !(side == 0 ? pt.cut_l : pt.cut_r) || stage < 0 || stage >= I.n_stages)
    return ADG_ERR_ARG;
  const int N = I.n_elem, Q = I.p + 1, nv = I.nv;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  // [nv][N][Q]: one element's block is nv rows of Q doubles, N Q apart
  double *arr = (what == ADG_PART_PRELIMIT) ? I.wpre : const_cast<double *>(stage_input(I, stage));
  const size_t row = sizeof(double) * Q, pitch = sizeof(double) * (size_t)N * Q;
  if (!import) {
    const int e = side == 0 ? 1 : N - 2;  // the owned boundary element
    CK(cudaMemcpy2DAsync(blk, row, arr + (size_t)e * Q, pitch, row, nv, cudaMemcpyDeviceToDevice,
                         st));
    return ADG_OK;
  }
  // the buffer element, and for a pre-limit block the buffer's side of the cut
  // face in the pre-limit history of the current step: by a kernel that reads
  // the step from the device counter, so that a captured exchange replays
  CK(launch_part_import(ctx->d_insts + k, what, side, stage, blk, nv, Q, st));
  return ADG_OK;
}

// Drop the captured graphs (after the launch configuration changed).
static void drop_graphs(adg_ctx *ctx) {
  if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  if (ctx->texec) cudaGraphExecDestroy(ctx->texec);
  if (ctx->tgraph) cudaGraphDestroy(ctx->tgraph);
  ctx->exec = ctx->texec = nullptr;
  ctx->graph = ctx->tgraph = nullptr;
  ctx->graph_ok = false;
  if (ctx->io_exec) cudaGraphExecDestroy(ctx->io_exec);
  if (ctx->io_graph) cudaGraphDestroy(ctx->io_graph);
  ctx->io_exec = nullptr;
  ctx->io_graph = nullptr;
}

// The limiter's elements per CTA for one group: times a limiter launch of stage
// 0 (on the pre-limit output the stage kernel's trial launches left) for every
// block size the limiter is built for, and keeps the fastest. The trial
// launches also write the group's flags and add to its flag counts, which are
// saved before and put back after.
static int tune_limiter(adg_ctx *ctx, Group &G, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  std::vector<int> members;
  std::vector<std::vector<int32_t>> counts;
  std::vector<std::vector<uint8_t>> flags;
  CK(cudaStreamSynchronize(st));
  for (int k = 0; k < ctx->n_inst; ++k) {
    const Inst &I = ctx->inst[k].d;
    if (I.p + 1 != G.Q || I.mixed != G.prec || I.n_stages != G.S) continue;
    members.push_back(k);
    counts.emplace_back(I.n_elem);
    flags.emplace_back((size_t)I.n_stages * I.n_elem);
    CK(cudaMemcpy(counts.back().data(), I.count, sizeof(int32_t) * I.n_elem,
                  cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(flags.back().data(), I.flags, flags.back().size(), cudaMemcpyDeviceToHost));
  }
  // the best of three rounds of three launches per size (a launch of a small
  // group takes some 20 us, where one round is noisy); another size replaces
  // the rule's only when it is 3 % faster
  const int rule = G.EPB;
  const int cand[3] = {8, 16, 32};
  int best_epb = rule;
  float best = 1e30f, at_rule = 1e30f;
  for (int epb : cand) {
    if (!limiter_block_ok(G, epb)) continue;
    G.EPB = epb;
    CK(upload_blocks(ctx, G));
    LimArgs L;
    L.insts = ctx->d_insts;
    L.blocks = G.d_blocks;
    L.s = 0;
    L.EPB = epb;
    CK(launch_limiter(ctx->mech, L, G.Q, G.mixed, ctx->ns + 2, G.n_blocks, st));
    float round_best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      CK(cudaEventRecord(e0, st));
      for (int w = 0; w < 3; ++w)
        CK(launch_limiter(ctx->mech, L, G.Q, G.mixed, ctx->ns + 2, G.n_blocks, st));
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < round_best) round_best = ms;
    }
    if (epb == rule) at_rule = round_best;
    if (round_best < best) {
      best = round_best;
      best_epb = epb;
    }
  }
  if (best_epb != rule && best > 0.97f * at_rule) best_epb = rule;
  G.EPB = best_epb;
  CK(upload_blocks(ctx, G));
  for (size_t m = 0; m < members.size(); ++m) {
    const Inst &I = ctx->inst[members[m]].d;
    CK(cudaMemcpy(I.count, counts[m].data(), sizeof(int32_t) * I.n_elem, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(I.flags, flags[m].data(), flags[m].size(), cudaMemcpyHostToDevice));
  }
  return ADG_OK;
}

int adg_autotune(adg_ctx *ctx, void *stream) {
  if (!ctx) return ADG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(ctx->last_stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  static const int kTE[] = {2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 32, 40, 48, 64};
  static const int kNT[] = {64, 128, 192, 256, 384, 512, 768, 1024};
  int rc = ADG_OK;
  for (int gi = 0; gi < ctx->n_groups && rc == ADG_OK; ++gi) {
    Group &G = ctx->groups[gi];
    int bestTE = G.TE, bestNT = G.NT;
    float best = 1e30f;
    for (int te : kTE) {
      if (te < kMinTile) continue;
      if (stage_smem(ctx->mech, te, G.Q, G.O, G.prec, G.visc) > 200 * 1024) continue;
      G.TE = te;
      if (upload_tiles(ctx, G) != cudaSuccess) {
        rc = ADG_ERR_CUDA;
        break;
      }
      for (int nt : kNT) {
        if (nt > stage_max_threads(G.prec, G.visc)) continue;
        StageArgs A;
        A.insts = ctx->d_insts;
        A.tiles = G.d_tiles;
        A.s = 0;
        A.TE = te;
        A.NT = nt;
        A.O = G.O;
        A.visc = G.visc;
        // stage 0 alone rewrites only buffers that the next step rewrites again
        // (stage buffers, q, the ring slots of the current level), so the
        // trajectory is unchanged
        bool ok = true;
        if (G.visc) ok = launch_aux(aux_args(ctx, G, 0), G.Q, G.n_blocks, st) == cudaSuccess;
        ok = ok && launch_stage(ctx->mech, A, G.Q, G.prec, G.n_tiles, st) == cudaSuccess;
        ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
        for (int w = 0; w < 2 && ok; ++w)
          ok = launch_stage(ctx->mech, A, G.Q, G.prec, G.n_tiles, st) == cudaSuccess;
        ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.0f;
        if (!ok || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = ADG_ERR_CUDA;
          break;
        }
        if (ms < best) {
          best = ms;
          bestTE = te;
          bestNT = nt;
        }
      }
      if (rc != ADG_OK) break;
    }
    G.TE = bestTE;
    G.NT = bestNT;
    if (upload_tiles(ctx, G) != cudaSuccess) rc = ADG_ERR_CUDA;
    if (rc == ADG_OK && G.any_limiter) rc = tune_limiter(ctx, G, st, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graphs(ctx);
  if (rc == ADG_ERR_CUDA) return cuda_fail(cudaGetLastError());
  return rc;
}

int adg_set_tuning(adg_ctx *ctx, int group, int elements_per_tile, int threads_per_cta) {
  if (!ctx || group < 0 || group >= ctx->n_groups) return ADG_ERR_ARG;
  Group &G = ctx->groups[group];
  const int te = elements_per_tile, nt = threads_per_cta;
  if (te < kMinTile || nt < 32 || nt > stage_max_threads(G.prec, G.visc) || nt % 32)
    return ADG_ERR_ARG;
  if (stage_smem(ctx->mech, te, G.Q, G.O, G.prec, G.visc) > 200 * 1024) return ADG_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->last_stream));
  G.TE = te;
  G.NT = nt;
  CK(upload_tiles(ctx, G));
  drop_graphs(ctx);
  return ADG_OK;
}

int adg_set_limiter_tuning(adg_ctx *ctx, int group, int elements_per_cta) {
  if (!ctx || group < 0 || group >= ctx->n_groups) return ADG_ERR_ARG;
  Group &G = ctx->groups[group];
  if (!limiter_block_ok(G, elements_per_cta)) return ADG_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->last_stream));
  G.EPB = elements_per_cta;
  CK(upload_blocks(ctx, G));
  drop_graphs(ctx);
  return ADG_OK;
}

int adg_get_tuning(const adg_ctx *ctx, int *n_groups, int *tuning) {
  if (!ctx || !n_groups || !tuning) return ADG_ERR_ARG;
  *n_groups = ctx->n_groups;
  for (int gi = 0; gi < ctx->n_groups; ++gi) {
    const Group &G = ctx->groups[gi];
    int *t = tuning + ADG_TUNING_FIELDS * gi;
    t[0] = G.Q - 1;
    t[1] = G.prec;
    t[2] = G.TE;
    t[3] = G.NT;
    t[4] = G.n_tiles;
    t[5] = G.S;
    t[6] = G.EPB;
  }
  return ADG_OK;
}

int adg_step_unsync(adg_ctx *ctx, int instance, int n_steps, void *stream) {
  if (!ctx || instance < 0 || instance >= ctx->n_inst || n_steps < 0) return ADG_ERR_ARG;
  if (n_steps == 0) return ADG_OK;
  InstHost &h = ctx->inst[instance];
  const Inst &I = h.d;
  if (I.viscous) return ADG_ERR_ARG;  // the unsynchronised mode runs the Euler terms only
  if (h.part.part) return ADG_ERR_ARG;  // and whole domains only
  // the unsynchronised mode offers the FP64 and the ADG_MIXED stage arithmetic
  if (I.mixed == ADG_MIXED_F32CHEM) return ADG_ERR_ARG;
  const int Q = I.p + 1;
  const bool mixed = I.mixed != ADG_FP64;
  const Group *G = nullptr;
  for (int gi = 0; gi < ctx->n_groups; ++gi)
    if (ctx->groups[gi].Q == Q && ctx->groups[gi].prec == I.mixed &&
        ctx->groups[gi].S == I.n_stages)
      G = &ctx->groups[gi];
  if (!G) return ADG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  UnsyncArgs U;
  U.inst = ctx->d_insts + instance;
  U.n_pe = h.n_pe;
  U.npf = I.npf;
  U.n_steps = n_steps;
  U.TE = G->TE;
  U.O = G->O;
  U.EPB = G->EPB;
  U.pub_in = ctx->pub_in;
  U.pub_pre = ctx->pub_pre;
  U.agree = ctx->agree;
  U.hist = ctx->delay_hist;
  U.spin_limit = ctx->unsync_polls;
  U.withheld = ctx->unsync_withheld;
  U.slow_pe = ctx->unsync_slow_pe;
  U.slow_us = ctx->unsync_slow_us;
  cudaError_t e = launch_unsync(ctx->mech, U, Q, mixed, I.nv, st);
  if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorInvalidValue) {
    cudaGetLastError();
    return ADG_ERR_ARG;
  }
  CK(e);
  CK(launch_advance_by(I.step, n_steps, st));
  h.n += n_steps;
  return ADG_OK;
}

int adg_set_unsync_wait(adg_ctx *ctx, long long max_polls, int withheld_pe) {
  if (!ctx || max_polls < 0 || withheld_pe < -1) return ADG_ERR_ARG;
  ctx->unsync_polls = max_polls;
  ctx->unsync_withheld = withheld_pe;
  return ADG_OK;
}

int adg_set_unsync_imbalance(adg_ctx *ctx, int slow_pe, int slow_us) {
  if (!ctx || slow_pe < -1 || slow_us < 0 || slow_us > 10000) return ADG_ERR_ARG;
  ctx->unsync_slow_pe = slow_pe;
  ctx->unsync_slow_us = slow_us;
  return ADG_OK;
}

int adg_unsync_delays(adg_ctx *ctx, uint64_t *hist) {
  if (!ctx || !hist) return ADG_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->last_stream));
  CK(cudaMemcpy(hist, ctx->delay_hist, sizeof(uint64_t) * 2 * (MAXD + 1), cudaMemcpyDeviceToHost));
  CK(cudaMemset(ctx->delay_hist, 0, sizeof(uint64_t) * 2 * (MAXD + 1)));
  return ADG_OK;
}

int adg_launches_per_step(const adg_ctx *ctx) {
  if (!ctx) return 0;
  int n = 1;
  for (int gi = 0; gi < ctx->n_groups; ++gi)
    n += ctx->groups[gi].S *
         ((ctx->groups[gi].any_limiter ? 2 : 1) + (ctx->groups[gi].visc ? 1 : 0));
  return n;
}

int adg_enable_kernel_timing(adg_ctx *ctx, int on) {
  if (!ctx) return ADG_ERR_ARG;
  ctx->timing = on != 0;
  ctx->kms[0] = ctx->kms[1] = ctx->kms[2] = 0.0;
  ctx->kcount[0] = ctx->kcount[1] = ctx->kcount[2] = 0;
  return ADG_OK;
}

int adg_kernel_times(adg_ctx *ctx, double *ms, int64_t *launches) {
  if (!ctx || !ms || !launches) return ADG_ERR_ARG;
  for (int k = 0; k < 3; ++k) {
    ms[k] = ctx->kms[k];
    launches[k] = ctx->kcount[k];
  }
  return ADG_OK;
}

int adg_write_state(adg_ctx *ctx, int k, const double *w, void *stream) {
  if (!inst_ok(ctx, k) || !w) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  size_t n = (size_t)h.d.nv * h.d.n_elem * (h.d.p + 1);
  CK(cudaMemcpyAsync(h.d.wn, w, sizeof(double) * n, cudaMemcpyHostToDevice,
                     (cudaStream_t)stream));
  ctx->last_stream = (cudaStream_t)stream;
  return ADG_OK;
}

int64_t adg_states_doubles(const adg_ctx *ctx) {
  if (!ctx) return 0;
  int64_t n = 0;
  for (const InstHost &h : ctx->inst) n += (int64_t)h.d.nv * h.d.n_elem * (h.d.p + 1);
  return n;
}

// The device address of a host buffer the GPU can read and write directly
// (pinned and mapped into the device's address space), or null.
static double *mapped_host(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? (double *)at.devicePointer : nullptr;
}

int adg_write_states(adg_ctx *ctx, const double *w, void *stream) {
  if (!ctx || !w) return ADG_ERR_ARG;
  ctx->last_stream = (cudaStream_t)stream;
  // a mapped pinned buffer: one kernel reads it over the host link
  if (double *dw = mapped_host(w)) {
    CK(launch_states_copy(ctx->d_insts, ctx->d_offs, ctx->n_inst, dw, false,
                          (cudaStream_t)stream));
    return ADG_OK;
  }
  for (const InstHost &h : ctx->inst) {
    const size_t n = (size_t)h.d.nv * h.d.n_elem * (h.d.p + 1);
    CK(cudaMemcpyAsync(h.d.wn, w, sizeof(double) * n, cudaMemcpyHostToDevice,
                       (cudaStream_t)stream));
    w += n;
  }
  ctx->last_stream = (cudaStream_t)stream;
  return ADG_OK;
}

int adg_read_states(adg_ctx *ctx, double *w, void *stream) {
  if (!ctx || !w) return ADG_ERR_ARG;
  ctx->last_stream = (cudaStream_t)stream;
  if (double *dw = mapped_host(w)) {
    CK(launch_states_copy(ctx->d_insts, ctx->d_offs, ctx->n_inst, dw, true,
                          (cudaStream_t)stream));
    return ADG_OK;
  }
  for (const InstHost &h : ctx->inst) {
    const size_t n = (size_t)h.d.nv * h.d.n_elem * (h.d.p + 1);
    CK(cudaMemcpyAsync(w, h.d.wn, sizeof(double) * n, cudaMemcpyDeviceToHost,
                       (cudaStream_t)stream));
    w += n;
  }
  ctx->last_stream = (cudaStream_t)stream;
  return ADG_OK;
}

// The step with its state copies as one graph (adg_step_io). Each inviscid
// group is cut into up to kIoParts parts of about equal bytes (its instances
// in order; tiles and limiter blocks never span instances), so the first
// part's copies in and the last part's copies out, the only copies no stage
// hides, are a fraction of a group's. The copies in run part after part on io_stream, one copy per
// instance on the copy engines (kernels over the mapped buffers would take SM
// slots from the stage kernels); the parts step one after another on the
// capture stream, each once its own states are in; each part's states go out
// on out_stream while the next part steps. Every instance still reads only its
// own new input and is read only after its own step, as in adg_write_states +
// adg_step + adg_read_states.
static int capture_io(adg_ctx *ctx, const double *w_in, double *w_out) {
  if (ctx->io_exec) cudaGraphExecDestroy(ctx->io_exec);
  if (ctx->io_graph) cudaGraphDestroy(ctx->io_graph);
  ctx->io_exec = nullptr;
  ctx->io_graph = nullptr;
  if (!ctx->io_stream) CK(cudaStreamCreateWithFlags(&ctx->io_stream, cudaStreamNonBlocking));
  if (!ctx->out_stream) CK(cudaStreamCreateWithFlags(&ctx->out_stream, cudaStreamNonBlocking));
  // the first double of each instance's state in the host buffers
  std::vector<int64_t> offs(ctx->n_inst + 1, 0);
  for (int k = 0; k < ctx->n_inst; ++k) {
    const Inst &I = ctx->inst[k].d;
    offs[k + 1] = offs[k] + (int64_t)I.nv * I.n_elem * (I.p + 1);
  }
  auto bytes = [&](int k) { return sizeof(double) * (size_t)(offs[k + 1] - offs[k]); };
  // the parts: (group, members [m0, m1), tile and block ranges)
  struct IoPart {
    int g, m0, m1;
    Part r;
  };
  std::vector<IoPart> parts;
  for (int g = 0; g < ctx->n_groups; ++g) {
    const Group &G = ctx->groups[g];
    const int nm = (int)G.members.size();
    // ends of the parts: about equal bytes each, every part non-empty
    std::vector<int> ends;
    if (!G.visc && nm > 1) {
      const int P = nm < kIoParts ? nm : kIoParts;
      int64_t tot = 0, acc = 0;
      for (int k : G.members) tot += offs[k + 1] - offs[k];
      int j = 1;
      for (int m = 0; m + 1 < nm && j < P; ++m) {
        acc += offs[G.members[m] + 1] - offs[G.members[m]];
        if (acc * P >= tot * j || nm - (m + 1) == P - j) {
          ends.push_back(m + 1);
          ++j;
        }
      }
    }
    ends.push_back(nm);
    int t0 = 0, b0 = 0, m0 = 0;
    for (int cut : ends) {
      IoPart P{g, m0, cut, Part()};
      if (!(m0 == 0 && cut == nm)) {
        int nt = 0, nb = 0;
        for (int m = m0; m < cut; ++m) {
          const int ne = ctx->inst[G.members[m]].d.n_elem;
          nt += (ne + G.TE - 1) / G.TE;
          nb += (ne + G.EPB - 1) / G.EPB;
        }
        P.r.tile0 = t0;
        P.r.n_tiles = nt;
        P.r.blk0 = b0;
        P.r.n_blocks = nb;
        t0 += nt;
        b0 += nb;
      }
      parts.push_back(P);
      m0 = cut;
    }
    // the parts must cover the group's tables exactly; otherwise one part
    if (t0 != 0 && (t0 != G.n_tiles || b0 != G.n_blocks)) {
      while (!parts.empty() && parts.back().g == g) parts.pop_back();
      parts.push_back(IoPart{g, 0, nm, Part()});
    }
  }
  const int np = (int)parts.size();
  for (int j = 0; j < np; ++j) {
    if (!ctx->io_ev[j]) CK(cudaEventCreateWithFlags(&ctx->io_ev[j], cudaEventDisableTiming));
    if (!ctx->done_ev[j]) CK(cudaEventCreateWithFlags(&ctx->done_ev[j], cudaEventDisableTiming));
  }
  cudaStream_t st = ctx->cap_stream;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = ADG_OK;
  cudaError_t e = cudaEventRecord(ctx->fork_ev, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->io_stream, ctx->fork_ev, 0);
  for (int j = 0; j < np && e == cudaSuccess; ++j) {
    const IoPart &P = parts[j];
    for (int m = P.m0; m < P.m1 && e == cudaSuccess; ++m) {
      const int k = ctx->groups[P.g].members[m];
      e = cudaMemcpyAsync(ctx->inst[k].d.wn, w_in + offs[k], bytes(k), cudaMemcpyHostToDevice,
                          ctx->io_stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->io_ev[j], ctx->io_stream);
  }
  for (int j = 0; j < np && e == cudaSuccess && rc == ADG_OK; ++j) {
    const IoPart &P = parts[j];
    e = cudaStreamWaitEvent(st, ctx->io_ev[j], 0);
    for (int s = 0; s < ctx->groups[P.g].S && e == cudaSuccess && rc == ADG_OK; ++s)
      rc = enqueue_group(ctx, P.g, s, st, -1, P.r);
    if (e == cudaSuccess && rc == ADG_OK) e = cudaEventRecord(ctx->done_ev[j], st);
    if (e == cudaSuccess && rc == ADG_OK) e = cudaStreamWaitEvent(ctx->out_stream, ctx->done_ev[j], 0);
    for (int m = P.m0; m < P.m1 && e == cudaSuccess && rc == ADG_OK; ++m) {
      const int k = ctx->groups[P.g].members[m];
      e = cudaMemcpyAsync(w_out + offs[k], ctx->inst[k].d.wn, bytes(k), cudaMemcpyDeviceToHost,
                          ctx->out_stream);
    }
  }
  if (e == cudaSuccess && rc == ADG_OK) e = launch_advance(ctx->d_steps, ctx->n_inst, st);
  // the copy streams join the capture through their last events
  if (e == cudaSuccess && rc == ADG_OK) e = cudaEventRecord(ctx->join_ev[0], ctx->out_stream);
  if (e == cudaSuccess && rc == ADG_OK) e = cudaStreamWaitEvent(st, ctx->join_ev[0], 0);
  if (e == cudaSuccess && rc == ADG_OK) e = cudaStreamWaitEvent(st, ctx->io_ev[np - 1], 0);
  cudaGraph_t gr = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &gr);
  if (rc != ADG_OK || e != cudaSuccess || e2 != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    if (rc != ADG_OK) return rc;
    return cuda_fail(e != cudaSuccess ? e : e2);
  }
  e = cudaGraphInstantiate(&ctx->io_exec, gr, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(gr);
    ctx->io_exec = nullptr;
    return cuda_fail(e);
  }
  ctx->io_graph = gr;
  ctx->io_in = w_in;
  ctx->io_out = w_out;
  return ADG_OK;
}

int adg_step_io(adg_ctx *ctx, const double *w_in, double *w_out, void *stream) {
  if (!ctx || !w_in || !w_out) return ADG_ERR_ARG;
  // pinned host memory (the graph's copies need it), seen through its mapping
  const bool pinned = mapped_host(w_in) && mapped_host(w_out);
  if (!pinned || ctx->timing || ctx->n_groups < 2 || !ctx->fork_ev) {
    // one group (nothing to overlap), pageable buffers or kernel timing: the
    // three calls one after the other
    int rc = adg_write_states(ctx, w_in, stream);
    if (rc == ADG_OK) rc = adg_step(ctx, 1, stream);
    if (rc == ADG_OK) rc = adg_read_states(ctx, w_out, stream);
    return rc;
  }
  if (!ctx->io_exec || ctx->io_in != w_in || ctx->io_out != w_out) {
    int rc = capture_io(ctx, w_in, w_out);
    if (rc != ADG_OK) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = st;
  CK(cudaGraphLaunch(ctx->io_exec, st));
  for (InstHost &h : ctx->inst) h.n += 1;
  return ADG_OK;
}

int adg_read_state(adg_ctx *ctx, int k, double *w, void *stream) {
  if (!inst_ok(ctx, k) || !w) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  size_t n = (size_t)h.d.nv * h.d.n_elem * (h.d.p + 1);
  CK(cudaMemcpyAsync(w, h.d.wn, sizeof(double) * n, cudaMemcpyDeviceToHost,
                     (cudaStream_t)stream));
  ctx->last_stream = (cudaStream_t)stream;
  return ADG_OK;
}

int64_t adg_steps_done(const adg_ctx *ctx, int k) {
  if (!ctx || k < 0 || k >= ctx->n_inst) return -1;
  return ctx->inst[k].n;
}

int adg_status(adg_ctx *ctx, int *instance, int *element, int64_t *step, int *stage) {
  if (!ctx) return ADG_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->last_stream));
  std::vector<int> h(4 * ctx->n_inst);
  CK(cudaMemcpy(h.data(), ctx->err_all, sizeof(int) * h.size(), cudaMemcpyDeviceToHost));
  for (int k = 0; k < ctx->n_inst; ++k) {
    if (h[4 * k] != 0) {
      if (instance) *instance = k;
      if (element) *element = h[4 * k + 1];
      if (stage) *stage = h[4 * k + 2];
      if (step) *step = h[4 * k + 3];
      int code = h[4 * k];
      CK(cudaMemset(ctx->err_all, 0, sizeof(int) * h.size()));
      return code;
    }
  }
  return ADG_OK;
}

int adg_get_flags(adg_ctx *ctx, int k, uint8_t *last, int32_t *count) {
  if (!inst_ok(ctx, k)) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  CK(cudaStreamSynchronize(ctx->last_stream));
  if (last)
    CK(cudaMemcpy(last, h.d.flags, (size_t)h.d.n_stages * h.d.n_elem, cudaMemcpyDeviceToHost));
  if (count)
    CK(cudaMemcpy(count, h.d.count, sizeof(int32_t) * h.d.n_elem, cudaMemcpyDeviceToHost));
  return ADG_OK;
}

int adg_get_temperature(adg_ctx *ctx, int k, double *T) {
  if (!inst_ok(ctx, k) || !T) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  CK(cudaStreamSynchronize(ctx->last_stream));
  CK(launch_temperature(ctx->mech, h.d, h.d.wn, h.prim, 0));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(T, h.prim, sizeof(double) * h.d.n_elem * (h.d.p + 1), cudaMemcpyDeviceToHost));
  return ADG_OK;
}

int adg_get_aux(adg_ctx *ctx, int k, int what, void *out) {
  if (!inst_ok(ctx, k) || !out) return ADG_ERR_ARG;
  if (what == ADG_AUX_FLAGS) return adg_get_flags(ctx, k, (uint8_t *)out, nullptr);
  if (what != ADG_AUX_TEMPERATURE && what != ADG_AUX_PRESSURE) return ADG_ERR_ARG;
  InstHost &h = ctx->inst[k];
  CK(cudaStreamSynchronize(ctx->last_stream));
  CK(launch_temperature(ctx->mech, h.d, h.d.wn, h.prim, 0, what == ADG_AUX_PRESSURE ? 1 : 0));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(out, h.prim, sizeof(double) * h.d.n_elem * (h.d.p + 1), cudaMemcpyDeviceToHost));
  return ADG_OK;
}

}  // extern "C"
