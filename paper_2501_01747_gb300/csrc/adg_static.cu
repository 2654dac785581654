// adg_step_noalloc: the ADG time step for callers that cannot allocate device
// memory. All scratch (mechanism tables, stage buffers, history ring, flags,
// PE maps, error word) lives in one file-scope device array of fixed size.
#include <cmath>
#include <cstring>
#include <mutex>

#include "adg_internal.cuh"
#include "adg_math.cuh"

namespace adg {

// The scratch. Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ADG_NOALLOC_SCRATCH_BYTES];

// PE maps of one instance computed on the device (PE q owns elements
// [q N / P, (q+1) N / P); the element e belongs to PE ((e+1) P - 1) / N).
__global__ void noalloc_maps_kernel(int N, int P, int npf, int periodic, int *pf_left,
                                    int *pf_right, int32_t *count, uint8_t *flags, int *err,
                                    int64_t *step, int TE, int2 *tiles, int EPB, int2 *blocks) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) {
    for (int k = 0; k < 4; ++k) err[k] = 0;
    *step = 0;
  }
  if (e >= N) return;
  if (e % TE == 0) tiles[e / TE] = make_int2(0, e);
  if (e % EPB == 0) blocks[e / EPB] = make_int2(0, e);
  count[e] = 0;
  flags[e] = flags[N + e] = flags[2 * N + e] = 0;
  int l = -1, r = -1;
  if (npf > 0) {
    int64_t q = (((int64_t)e + 1) * P - 1) / N;
    int64_t first = q * N / P;
    int64_t next = (q + 1) * N / P;
    if (e == first) {
      if (q > 0) l = (int)(q - 1);
      else if (periodic) l = P - 1;
    }
    if (e == next - 1) {
      if (q < P - 1) r = (int)q;
      else if (periodic) r = P - 1;
    }
  }
  pf_left[e] = l;
  pf_right[e] = r;
}

// Bytes that one launch of noalloc_put_kernel copies into the scratch. They
// travel as the kernel's parameter, taken by value at launch, so no host buffer
// has to outlive the call and no copy from pageable host memory is enqueued.
constexpr int kPutBytes = 2048;
struct PutChunk {
  unsigned long long off;  // destination offset in the scratch
  unsigned n, pad;         // bytes used of b
  unsigned char b[kPutBytes];
};

__global__ void noalloc_put_kernel(unsigned char *base, PutChunk c) {
  for (unsigned i = threadIdx.x; i < c.n; i += blockDim.x) base[c.off + i] = c.b[i];
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_ptr[kMaxDevices];
bool g_ready[kMaxDevices];

// Host staging of the mechanism tables, at file scope (neither the heap nor a
// large stack frame); used only while g_mutex is held.
struct HostTables {
  double sp[SP_NFIELDS * ADG_MAX_SPECIES];
  Rxn rx[ADG_NOALLOC_MAX_REACTIONS > 0 ? ADG_NOALLOC_MAX_REACTIONS : 1];
  DF rxf[6 * (ADG_NOALLOC_MAX_REACTIONS > 0 ? ADG_NOALLOC_MAX_REACTIONS : 1)];
  int sx_off[ADG_MAX_SPECIES + 1];
  int sx[ADG_NOALLOC_MAX_REACTIONS * NET];
};
HostTables g_host;

// Copy n bytes from host memory to base + off on stream s, kPutBytes per launch.
cudaError_t put(unsigned char *base, size_t off, const void *src, size_t n, cudaStream_t s) {
  PutChunk c;
  const unsigned char *p = static_cast<const unsigned char *>(src);
  for (size_t k = 0; k < n; k += kPutBytes) {
    c.off = off + k;
    c.n = (unsigned)(n - k < (size_t)kPutBytes ? n - k : (size_t)kPutBytes);
    c.pad = 0;
    memcpy(c.b, p + k, c.n);
    noalloc_put_kernel<<<1, 256, 0, s>>>(base, c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

struct Cursor {
  unsigned char *base;
  size_t off;
  size_t take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    size_t at = off;
    off += n;
    return at;
  }
};

}  // namespace
}  // namespace adg

using namespace adg;

extern "C" int adg_step_noalloc(const adg_mechanism *mech, const adg_config *cfg,
                                const double *w_in_dev, double *w_out_dev, int n_steps,
                                void *stream) {
  if (!mech || !cfg || !w_in_dev || !w_out_dev || n_steps < 0) return ADG_ERR_ARG;
  const adg_config &c = *cfg;
  const int ns = mech->n_species, nr = mech->n_reactions;
  if (ns < 1 || ns > ADG_MAX_SPECIES || nr < 0 || nr > ADG_NOALLOC_MAX_REACTIONS)
    return ADG_ERR_ARG;
  if (c.p < 1 || c.p > ADG_MAX_P || c.n_elem < 1 || c.n_pe < 1 || c.n_pe > c.n_elem ||
      !(c.length > 0.0) || !(c.dt > 0.0) || c.at_order < 1 || c.at_order > ADG_MAX_AT_ORDER ||
      c.max_delay < 0 || c.max_delay > ADG_MAX_DELAY || c.delay_mode < ADG_SYNC ||
      c.delay_mode > ADG_SAA || (c.delay_mode == ADG_SAA && !c.delay_probs) ||
      (c.flux != ADG_FLUX_LF && c.flux != ADG_FLUX_HLLC) ||
      (c.limiter != ADG_LIM_NONE && c.limiter != ADG_LIM_WENO) || c.bc_left < 0 ||
      c.bc_left > 2 || c.bc_right < 0 || c.bc_right > 2 ||
      ((c.bc_left == ADG_BC_PERIODIC) != (c.bc_right == ADG_BC_PERIODIC)) ||
      (c.precision != ADG_FP64 && c.precision != ADG_MIXED && c.precision != ADG_MIXED_F32CHEM) ||
      c.integrator != ADG_RK_SSP3 ||
      c.viscous != 0 || c.pe_begin != 0 || c.pe_end != 0)
    return ADG_ERR_ARG;
  if (!mech->W || !mech->cp || !mech->h_f || !mech->s0) return ADG_ERR_ARG;
  if (nr > 0 && (!mech->nu_f || !mech->nu_r || !mech->A || !mech->b || !mech->Ea))
    return ADG_ERR_ARG;
  for (int i = 0; i < ns; ++i)
    if (!(mech->W[i] > 0.0) || !(mech->cp[i] > RU)) return ADG_ERR_ARG;
  const int N = c.n_elem, Q = c.p + 1, nv = ns + 2;
  const bool periodic = c.bc_left == ADG_BC_PERIODIC;
  const int npf = c.n_pe <= 1 ? 0 : (periodic ? c.n_pe : c.n_pe - 1);
  const int depth = c.max_delay + c.at_order;

  Mech M;
  M.ns = ns;
  M.nr = nr;
  M.nterm = 0;
  for (int k = 0; k < ns * nr; ++k) M.nterm += (mech->nu_r[k] != mech->nu_f[k]);

  // layout of the scratch; reject problems that do not fit
  Cursor cur{nullptr, 0};
  size_t o_sp = cur.take(sizeof(double) * SP_NFIELDS * ns);
  size_t o_rx = cur.take(sizeof(Rxn) * (nr > 0 ? nr : 1));
  size_t o_rxf = cur.take(sizeof(DF) * 6 * (nr > 0 ? nr : 1));
  size_t o_sxo = cur.take(sizeof(int) * (ns + 1));
  size_t o_sx = cur.take(sizeof(int) * (M.nterm > 0 ? M.nterm : 1));
  size_t o_err = cur.take(sizeof(int) * 4);
  size_t st = (size_t)nv * N * Q;
  size_t o_wa = cur.take(sizeof(double) * st);
  size_t o_wb = cur.take(sizeof(double) * st);
  size_t o_wpre = cur.take(sizeof(double) * st);
  size_t rs = (size_t)depth * 3 * (npf > 0 ? npf : 1) * 2 * nv;
  size_t o_rin = cur.take(sizeof(double) * rs);
  size_t o_rpre = cur.take(sizeof(double) * rs * Q);
  size_t o_flags = cur.take((size_t)3 * N);
  size_t o_count = cur.take(sizeof(int32_t) * N);
  size_t o_pl = cur.take(sizeof(int) * N);
  size_t o_pr = cur.take(sizeof(int) * N);
  const bool mixed = c.precision != ADG_FP64;
  int TE = stage_tile(M, Q, c.at_order, c.precision, false);
  int target = (N + 2 * 152 - 1) / (2 * 152);
  if (target < TE) TE = target < 4 ? 4 : target;
  const int NT = stage_threads(TE, Q, nr);
  const int EPB = limiter_elems_per_block(N, mixed);
  const int n_tiles = (N + TE - 1) / TE, n_blocks = (N + EPB - 1) / EPB;
  size_t o_inst = cur.take(sizeof(Inst));
  size_t o_step = cur.take(sizeof(int64_t));
  size_t o_tiles = cur.take(sizeof(int2) * n_tiles);
  size_t o_blocks = cur.take(sizeof(int2) * n_blocks);
  if (cur.off > (size_t)ADG_NOALLOC_SCRATCH_BYTES) return ADG_ERR_NOMEM;

  // the host staging of the tables and every launch below under one lock
  std::lock_guard<std::mutex> lock(g_mutex);
  HostTables &ht = g_host;
  if (pack_mechanism(mech, ht.sp, ht.rx, ht.sx_off, ht.sx) != M.nterm) return ADG_ERR_ARG;
  pack_rxf(ht.rx, nr, ht.rxf);

  // once per device: the scratch address and the constant tables. This is the
  // only set-up; it runs on the first call on each device.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADG_ERR_CUDA;
  {
    if (!g_ready[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return ADG_ERR_CUDA;
      Basis tables[ADG_MAX_P];
      make_tables(tables);
      if (upload_basis(tables) != cudaSuccess || prepare_kernels(nv, ns, nr) != cudaSuccess)
        return ADG_ERR_CUDA;
      g_ptr[dev] = (unsigned char *)p;
      g_ready[dev] = true;
    }
  }
  unsigned char *base = g_ptr[dev];
  cudaStream_t s = (cudaStream_t)stream;

  M.sp = (const double *)(base + o_sp);
  M.rx = (const Rxn *)(base + o_rx);
  M.rxf = (const DF *)(base + o_rxf);
  M.sx_off = (const int *)(base + o_sxo);
  M.sx = (const int *)(base + o_sx);
  Inst I;
  memset(&I, 0, sizeof(I));
  I.n_elem = N;
  I.p = c.p;
  I.nv = nv;
  I.npf = npf;
  I.npf_draw = npf;  // the whole domain: face f draws as face f (face_base 0)
  I.depth = depth;
  I.n_stages = 3;  // SSP-RK3 (memset left lserk = 0, wq = null)
  I.at_order = c.at_order;
  I.bc_left = c.bc_left;
  I.bc_right = c.bc_right;
  I.flux = c.flux;
  I.limiter = c.limiter;
  I.delay_mode = c.delay_mode;
  I.max_delay = c.max_delay;
  I.dx = c.length / N;
  I.dt = c.dt;
  I.tvb = c.tvb_M * I.dx * I.dx;
  I.mixed = c.precision;
  I.ind_floor = indicator_guard(c.precision);
  I.ind_floor_p = indicator_guard_p(c.precision);
  I.seed = c.seed;
  double acc = 0.0;
  for (int d = 0; d <= MAXD; ++d) {
    if (d <= c.max_delay) acc += (c.delay_mode == ADG_SAA) ? c.delay_probs[d] : 0.0;
    I.cum[d] = acc;
  }
  for (int d = 0; d <= MAXD; ++d)
    for (int m = 0; m < MAXO; ++m) {
      double v = 0.0;
      if (d <= c.max_delay && m < c.at_order) {
        v = 1.0;
        for (int j = 0; j < c.at_order; ++j)
          if (j != m) v *= (double)(d + j) / (double)(j - m);
      }
      I.at[d][m] = v;
    }
  I.wn = w_out_dev;
  I.wa = (double *)(base + o_wa);
  I.wb = (double *)(base + o_wb);
  I.wpre = (double *)(base + o_wpre);
  I.ring_in = (double *)(base + o_rin);
  I.ring_pre = (double *)(base + o_rpre);
  I.flags = (uint8_t *)(base + o_flags);
  I.count = (int32_t *)(base + o_count);
  I.pf_of_left = (const int *)(base + o_pl);
  I.pf_of_right = (const int *)(base + o_pr);
  I.pf_elem = nullptr;
  I.err = (int *)(base + o_err);
  I.step = (int64_t *)(base + o_step);
  I.instance = 0;

#define NA_CK(x)                               \
  do {                                         \
    if ((x) != cudaSuccess) return ADG_ERR_CUDA; \
  } while (0)
  NA_CK(put(base, o_sp, ht.sp, sizeof(double) * SP_NFIELDS * ns, s));
  if (nr > 0) NA_CK(put(base, o_rx, ht.rx, sizeof(Rxn) * nr, s));
  if (nr > 0) NA_CK(put(base, o_rxf, ht.rxf, sizeof(DF) * 6 * nr, s));
  NA_CK(put(base, o_sxo, ht.sx_off, sizeof(int) * (ns + 1), s));
  if (M.nterm > 0) NA_CK(put(base, o_sx, ht.sx, sizeof(int) * M.nterm, s));
  if (w_out_dev != w_in_dev)
    NA_CK(cudaMemcpyAsync(w_out_dev, w_in_dev, sizeof(double) * st, cudaMemcpyDeviceToDevice, s));
  NA_CK(put(base, o_inst, &I, sizeof(Inst), s));
  noalloc_maps_kernel<<<(N + 127) / 128, 128, 0, s>>>(
      N, c.n_pe, npf, periodic ? 1 : 0, (int *)I.pf_of_left, (int *)I.pf_of_right, I.count,
      I.flags, I.err, I.step, TE, (int2 *)(base + o_tiles), EPB, (int2 *)(base + o_blocks));
  NA_CK(cudaGetLastError());
  for (int64_t n = 0; n < n_steps; ++n) {
    for (int stg = 0; stg < 3; ++stg) {
      StageArgs A;
      A.insts = (const Inst *)(base + o_inst);
      A.tiles = (const int2 *)(base + o_tiles);
      A.s = stg;
      A.TE = TE;
      A.NT = NT;
      A.O = c.at_order;
      A.visc = 0;
      NA_CK(launch_stage(M, A, Q, c.precision, n_tiles, s));
      if (I.limiter != ADG_LIM_NONE) {
        LimArgs L;
        L.insts = (const Inst *)(base + o_inst);
        L.blocks = (const int2 *)(base + o_blocks);
        L.s = stg;
        L.EPB = EPB;
        NA_CK(launch_limiter(M, L, Q, mixed, nv, n_blocks, s));
      }
    }
    NA_CK(launch_advance(I.step, 1, s));
  }
#undef NA_CK
  return ADG_OK;
}
