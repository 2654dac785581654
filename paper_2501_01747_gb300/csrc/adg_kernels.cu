// Host-side dispatch of the ADG kernels and the set-up kernels (projection of
// primitive values, temperature, step counters). The stage and limiter kernels
// of each precision variant live in adg_k64.cu and adg_k32.cu.
#include "adg_device.cuh"

namespace adg {

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

// Temperature (what = 0) or pressure (what = 1, P = rho R_u T sum Y_i / W_i) at
// every Gauss point, [n_elem][p+1].
template <int Q>
__global__ void temperature_kernel(Mech M, Inst I, const double *w, double *T, int what) {
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
  const double Tt = thermo_of(M.sp, M.ns, wq, 1).T;
  if (what == 1) {
    double Rm = 0.0;
    for (int i = 0; i < M.ns; ++i) Rm = fma(wq[2 + i], M.sp[SP_RW * M.ns + i], Rm);
    T[t] = Tt * Rm;
  } else {
    T[t] = Tt;
  }
}

// Central value of variable v of the stage input at face g (between elements
// g-1 and g) for the LDG auxiliary variable: the mean of the two traces; at a PE
// face with delay k > 0 the AT extrapolation (Eq. 7) of the means at the common
// delayed levels n-k-m from the trace ring; at a physical boundary the mean with
// the ghost (reflecting wall: rho u -> 0, the others the interior trace;
// outflow: the interior trace).
template <int Q>
__device__ double face_mean(const Inst &I, const double *win, int64_t nstep, int s, int g, int v,
                            bool periodic) {
  const int N = I.n_elem;
  const int pf = (g < N) ? I.pf_of_left[g] : I.pf_of_right[N - 1];
  const int k = pf >= 0 ? effective_delay(I, nstep, pf) : 0;
  if (k > 0) {
    double acc = 0.0;
    for (int m = 0; m < I.at_order; ++m) {
      const int64_t lv = nstep - k - m;
      const double l = I.ring_in[ring_trace(I, lv, s, pf, 0) + v];
      const double r = I.ring_in[ring_trace(I, lv, s, pf, 1) + v];
      acc = fma(I.at[k][m], 0.5 * (l + r), acc);
    }
    return acc;
  }
  if (!periodic && (g == 0 || g == N)) {
    const bool left = g == 0;
    const double *w = win + ((size_t)v * N + (left ? 0 : N - 1)) * Q;
    double tr = 0.0;
    for (int j = 0; j < Q; ++j) tr += (left && (j & 1)) ? -w[j] : w[j];
    const bool refl = (left ? I.bc_left : I.bc_right) == ADG_BC_REFLECT;
    return (refl && v == 0) ? 0.0 : tr;
  }
  const int el = (g == 0) ? N - 1 : g - 1, er = (g == N) ? 0 : g;
  const double *wl = win + ((size_t)v * N + el) * Q, *wr = win + ((size_t)v * N + er) * Q;
  double a = 0.0, b = 0.0;
  for (int j = 0; j < Q; ++j) {
    a += wl[j];
    b += ((j & 1) ? -1.0 : 1.0) * wr[j];
  }
  return 0.5 * (a + b);
}

// The LDG auxiliary variable q = dw/dx of stage s (Sec. 3.1: like w, with a
// central flux) for the viscous instances of a group, one (element, variable)
// per item over the group's block table:
//   q_i = (2i+1)/dx (w_hat_{e+1} - (-1)^i w_hat_e - 2 sum_{j < i, i-j odd} w_j),
// the last sum being the integral of w P_i' (int P_j P_i' = 2 for j < i with i-j
// odd, 0 otherwise). Writes q and, for a PE-boundary element, the trace of q at
// its PE face to the q ring (level n, stage s).
template <int Q>
__global__ void __launch_bounds__(128) aux_kernel(LimArgs A) {
  pdl_enter();
  __shared__ Inst sI;
  const int2 blk = A.blocks[blockIdx.x];
  load_inst(sI, A.insts + blk.x);
  __syncthreads();
  const Inst &I = sI;
  if (!I.viscous) return;
  const int N = I.n_elem, nv = I.nv, e0 = blk.y, te = min(A.EPB, N - e0);
  const int64_t nstep = *I.step;
  const double *win = stage_input(I, A.s);
  const bool periodic = I.bc_left == ADG_BC_PERIODIC;
  const double inv_dx = 1.0 / I.dx;
  for (int item = threadIdx.x; item < te * nv; item += blockDim.x) {
    const int v = item / te, e = e0 + (item - v * te);
    const double *we = win + ((size_t)v * N + e) * Q;
    double w[Q], q[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) w[j] = we[j];
    const double whl = face_mean<Q>(I, win, nstep, A.s, e, v, periodic);
    const double whr = face_mean<Q>(I, win, nstep, A.s, e + 1, v, periodic);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double vol = 0.0;
      for (int j = i - 1; j >= 0; j -= 2) vol += w[j];
      q[i] = (2.0 * i + 1.0) * inv_dx * (whr - ((i & 1) ? -whl : whl) - 2.0 * vol);
    }
    double *qe = I.qx + ((size_t)v * N + e) * Q;
#pragma unroll
    for (int i = 0; i < Q; ++i) qe[i] = q[i];
    if (I.npf > 0) {
      const int pr = I.pf_of_right[e], pl = I.pf_of_left[e];
      if (pr >= 0) {
        double tr = 0.0;
        for (int i = 0; i < Q; ++i) tr += q[i];
        I.ring_q[ring_trace(I, nstep, A.s, pr, 0) + v] = tr;
      }
      if (pl >= 0) {
        double tr = 0.0;
        for (int i = 0; i < Q; ++i) tr += ((i & 1) ? -1.0 : 1.0) * q[i];
        I.ring_q[ring_trace(I, nstep, A.s, pl, 1) + v] = tr;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host-side launchers

cudaError_t launch_aux(const LimArgs &A, int Q, int n_blocks, cudaStream_t st) {
  switch (Q) {
    case 2: return launch_pdl(aux_kernel<2>, dim3(n_blocks), dim3(128), 0, st, A);
    case 3: return launch_pdl(aux_kernel<3>, dim3(n_blocks), dim3(128), 0, st, A);
    case 4: return launch_pdl(aux_kernel<4>, dim3(n_blocks), dim3(128), 0, st, A);
    case 5: return launch_pdl(aux_kernel<5>, dim3(n_blocks), dim3(128), 0, st, A);
  }
  return cudaErrorInvalidValue;
}

cudaError_t upload_basis(const Basis *tables) {
  cudaError_t e = upload_unit_tables(tables);
  if (e == cudaSuccess) e = upload_tables_fp64(tables);
  if (e == cudaSuccess) e = upload_tables_mixed(tables);
  if (e == cudaSuccess) e = upload_tables_f32chem(tables);
  if (e == cudaSuccess) e = upload_tables_unsync(tables);
  if (e == cudaSuccess) e = upload_tables_visc_fp64(tables);
  if (e == cudaSuccess) e = upload_tables_visc_mixed(tables);
  return e;
}

cudaError_t launch_stage(const Mech &M, const StageArgs &A, int Q, int prec, int n_tiles,
                         cudaStream_t st) {
  if (A.visc) {
    if (prec == ADG_FP64) return launch_stage_visc_fp64(M, A, Q, n_tiles, st);
    if (prec == ADG_MIXED) return launch_stage_visc_mixed(M, A, Q, n_tiles, st);
    return cudaErrorInvalidValue;  // no viscous float-chemistry variant
  }
  if (prec == ADG_FP64) return launch_stage_fp64(M, A, Q, n_tiles, st);
  if (prec == ADG_MIXED) return launch_stage_mixed(M, A, Q, n_tiles, st);
  if (prec == ADG_MIXED_F32CHEM) return launch_stage_f32chem(M, A, Q, n_tiles, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_limiter(const Mech &M, const LimArgs &A, int Q, bool mixed, int nv,
                           int n_blocks, cudaStream_t st) {
  return mixed ? launch_limiter_mixed(M, A, Q, nv, n_blocks, st)
               : launch_limiter_fp64(M, A, Q, nv, n_blocks, st);
}

cudaError_t launch_unsync(const Mech &M, const UnsyncArgs &U, int Q, bool mixed, int nv,
                          cudaStream_t st) {
  return mixed ? launch_unsync_mixed(M, U, Q, nv, st) : launch_unsync_fp64(M, U, Q, nv, st);
}

cudaError_t prepare_unsync() {
  cudaError_t e = prepare_unsync_fp64();
  if (e == cudaSuccess) e = prepare_unsync_mixed();
  return e;
}

cudaError_t upload_tables_unsync(const Basis *tables) {
  cudaError_t e = upload_tables_unsync_fp64(tables);
  if (e == cudaSuccess) e = upload_tables_unsync_mixed(tables);
  return e;
}

// Raise the dynamic shared-memory limit of every kernel instance (before any
// launch or stream capture).
cudaError_t prepare_kernels(int nv, int ns, int nr) {
  (void)nv;
  (void)ns;
  (void)nr;
  cudaError_t e = prepare_fp64();
  if (e == cudaSuccess) e = prepare_mixed();
  if (e == cudaSuccess) e = prepare_f32chem();
  if (e == cudaSuccess) e = prepare_unsync();
  if (e == cudaSuccess) e = prepare_visc_fp64();
  if (e == cudaSuccess) e = prepare_visc_mixed();
  return e;
}

int stage_tile(const Mech &M, int Q, int O, int prec, bool visc) {
  // elements per tile: up to 256 Gauss points, at most ~96 KB of tile
  int TE = 256 / Q;
  while (TE > 2 && stage_smem_bytes(TE, Q, M.ns, M.nr, M.nterm, O, prec, visc) > 96 * 1024)
    TE /= 2;
  return TE;
}

int stage_threads(int TE, int Q, int nr) {
  // enough threads for the (reaction, point) items of the chemistry in a few rounds
  int items = TE * Q * (nr > 0 ? nr : 1);
  int nt = ((items / 4 + 31) / 32) * 32;
  return nt < 128 ? 128 : (nt > 512 ? 512 : nt);
}

size_t stage_smem(const Mech &M, int TE, int Q, int O, int prec, bool visc) {
  return stage_smem_bytes(TE, Q, M.ns, M.nr, M.nterm, O, prec, visc);
}

int limiter_elems_per_block(int64_t n_elem_group, bool mixed) {
  // fewer elements per CTA (more lanes each) while 32 would give fewer than two
  // CTAs per SM: 16 (8 lanes), or 8 (16 lanes) while 16 would too; in FP64 16
  // (4 lanes) or 32 (2 lanes), as the limiter body sets its indicator lanes
  if (!mixed) return n_elem_group < (int64_t)2 * 152 * LIM_EPB_MAX ? 16 : LIM_EPB_MAX;
  if (n_elem_group < (int64_t)2 * 152 * 16) return 8;
  return n_elem_group < (int64_t)2 * 152 * LIM_EPB_MAX ? 16 : LIM_EPB_MAX;
}

__global__ void advance_kernel(int64_t *steps, int n) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) steps[i] += 1;
}

__global__ void advance_by_kernel(int64_t *step, int64_t n) { *step += n; }

cudaError_t launch_advance_by(int64_t *step, int64_t n, cudaStream_t st) {
  advance_by_kernel<<<1, 1, 0, st>>>(step, n);
  return cudaGetLastError();
}

__global__ void part_import_kernel(const Inst *inst, int what, int side, int stage,
                                   const double *blk) {
  const Inst &I = *inst;
  const int Q = I.p + 1, n = I.nv * Q, N = I.n_elem;
  const int e = side == 0 ? 0 : N - 1;  // the buffer element
  double *arr = what == ADG_PART_PRELIMIT ? I.wpre : const_cast<double *>(stage_input(I, stage));
  const int pf = side == 0 ? 0 : I.npf - 1;
  const int64_t nstep = *I.step;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int v = t / Q, j = t - v * Q;
    const double x = blk[t];
    arr[((size_t)v * N + e) * Q + j] = x;
    if (what == ADG_PART_PRELIMIT) I.ring_pre[ring_block(I, nstep, stage, pf, side) + t] = x;
  }
}

cudaError_t launch_part_import(const Inst *inst, int what, int side, int stage,
                               const double *blk, int nv, int Q, cudaStream_t st) {
  const int n = nv * Q, threads = n < 512 ? ((n + 31) / 32) * 32 : 512;
  part_import_kernel<<<1, threads, 0, st>>>(inst, what, side, stage, blk);
  return cudaGetLastError();
}

// A flat buffer of all states <-> the instances' w^n, one double per item in
// grid-stride order (consecutive threads touch consecutive doubles on both
// sides); the instance of an item comes from a binary search of the offsets,
// staged in shared memory when they fit.
__global__ void states_copy_kernel(const Inst *insts, const int64_t *offs, int n, double *host,
                                   int to_host) {
  constexpr int MAXS = 2048;
  __shared__ int64_t so[MAXS + 1];
  const bool staged = n < MAXS;
  if (staged)
    for (int k = threadIdx.x; k <= n; k += blockDim.x) so[k] = offs[k];
  __syncthreads();
  const int64_t *o = staged ? so : offs;
  const int64_t total = o[n];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n - 1;  // the instance k with o[k] <= i < o[k + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (o[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    double *w = insts[lo].wn + (i - o[lo]);
    if (to_host) host[i] = *w;
    else *w = host[i];
  }
}

cudaError_t launch_states_copy(const Inst *insts, const int64_t *offs, int n, double *host,
                               bool to_host, cudaStream_t st) {
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  states_copy_kernel<<<n_sm * 8, 256, 0, st>>>(insts, offs, n, host, to_host ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *steps, int n, cudaStream_t st) {
  return launch_pdl(advance_kernel, dim3((n + 127) / 128), dim3(128), 0, st, steps, n);
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
                               cudaStream_t st, int what) {
  int n = I.n_elem * (I.p + 1);
  int nblk = (n + 127) / 128;
  switch (I.p + 1) {
    case 2: temperature_kernel<2><<<nblk, 128, 0, st>>>(M, I, w, T, what); break;
    case 3: temperature_kernel<3><<<nblk, 128, 0, st>>>(M, I, w, T, what); break;
    case 4: temperature_kernel<4><<<nblk, 128, 0, st>>>(M, I, w, T, what); break;
    case 5: temperature_kernel<5><<<nblk, 128, 0, st>>>(M, I, w, T, what); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace adg
