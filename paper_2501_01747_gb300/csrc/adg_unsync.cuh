// The truly unsynchronised mode: the PEs of one instance advance on their own,
// each reading the newest level of its neighbours that is present.
//
// The seeded modes (Sec. 4.1 CAA, Sec. 4.2 SAA) draw the delay of each PE face
// at each step and run every PE in lockstep. Here one CTA owns one PE, all CTAs
// of the instance run in one cooperative launch (so they are co-resident), and
// each CTA loops over steps and stages without any grid-wide barrier. A CTA
// publishes, per (step, stage), first the traces of its stage input at its PE
// faces (to the trace ring) and, after the stage, the pre-limit output of its
// PE-boundary elements (to the pre-limit ring), each followed by a counter of
// published stages. The newest level L of a neighbour published for the same
// stage gives the delay k = max(0, n - L) that side observes.
//
// Flux (Eq. 7): both sides of a PE face use one common delayed level, the
// older of the two (Sec. 3.2), so that the face flux stays single-valued: the
// first side to reach (n, s) records its observed k in the face's agreement
// slot, and the other side adopts the recorded k. Every level either side then
// reads is already published. AT-WENO neighbour (Eq. 11): no conservation is at
// stake, so each side uses the delay it observed.
//
// Waits: a CTA waits while a neighbour lags by more than the maximum delay d,
// or while the levels an AT extrapolation needs (L down to L - o + 1) do not
// exist yet. So a neighbour is never more than d steps ahead while a CTA reads
// its levels, the oldest level read is 2d + o - 1 levels below the newest one
// being written, and a ring of depth 2d + o keeps every level still needed.
// The slowest CTA never waits (its neighbours have published its level), so
// the launch cannot deadlock. Each wait polls a bounded number of times; past
// the bound the CTA reports ADG_ERR_TIMEOUT through the instance's error word
// and returns, and its neighbours time out in turn.
//
// Template code, instantiated per precision variant by adg_u64.cu (FP64) and
// adg_u32.cu (mixed) with the limiter's elements per CTA of the synchronous
// launches, so that with maximum delay 0 both modes do the same arithmetic.
//
// One PE may be made slower by a fixed idle time per stage (emulated load
// imbalance, one of the sources of delay named in Sec. 3.2), which makes its
// neighbours run ahead and observe delays up to d.
#pragma once
#include "adg_device.cuh"

namespace adg {

namespace {

// Newest level with stage s published by a neighbour that has published `done`
// stages (S n + s + 1 after stage s of step n, S stages per step), and the
// usable delay at step n: k = max(0, n - L) when k = 0, or k <= d with levels
// L - o + 1 .. L present; else -1 (wait).
__device__ inline int usable_delay(int done, long long n, int s, int S, int d, int o) {
  const long long L = done >= s + 1 ? (long long)(done - s - 1) / S : -1;
  const long long k = L >= n ? 0 : n - L;
  if (k == 0) return 0;
  if (k <= d && L >= o - 1) return (int)k;
  return -1;
}

// Spin (thread 0) until the neighbour's counter gives a usable delay.
__device__ inline int wait_delay(const int *pub, long long n, int s, int S, int d, int o,
                                 long long limit) {
  for (long long it = 0; it <= limit; ++it) {
    const int done = *(const volatile int *)pub;
    const int k = usable_delay(done, n, s, S, d, o);
    if (k >= 0) {
      __threadfence();  // what the neighbour wrote before its counter is now visible
      return k;
    }
    __nanosleep(128);
  }
  return -1;
}

// The common delay of the flux at one PE face for (n, s): the slot holds
// (n + 1) << 8 | k once a side has recorded k for step n. The first side to
// arrive records its own k; a later one (or one that loses the race) adopts
// the recorded k. A slot is reused every MAXD + 1 steps, which the other side
// cannot reach while this one is at n (it is at most d <= MAXD steps ahead).
__device__ inline int agree_delay(unsigned long long *slot, long long n, int k) {
  const unsigned long long tag = (unsigned long long)(n + 1) << 8;
  unsigned long long cur = *(volatile unsigned long long *)slot;
  for (int t = 0; t < 4; ++t) {
    if ((cur & ~0xffull) == tag) {
      __threadfence();  // the recording side's published levels are visible
      return (int)(cur & 0xff);
    }
    const unsigned long long prev = atomicCAS(slot, cur, tag | (unsigned long long)k);
    if (prev == cur) return k;
    cur = prev;
  }
  return -1;
}

__device__ inline unsigned long long *agree_slot(const UnsyncArgs &U, int pf, int s,
                                                 long long n) {
  return U.agree + ((size_t)pf * ADG_MAX_STAGES + s) * (MAXD + 1) + (size_t)(n % (MAXD + 1));
}

}  // namespace

template <int Q, int G, bool MIX, int EPB>
__global__ void __launch_bounds__(LIM_THREADS) unsync_kernel(Mech M, UnsyncArgs U) {
  __shared__ Inst sI;
  __shared__ PeDelays pdi, pdp;  // delays used by the flux and by the limiter
  __shared__ int s_abort;
  load_inst(sI, U.inst);
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();
  const Inst &I = sI;
  const int N = I.n_elem, P = U.n_pe, q = blockIdx.x, nv = I.nv;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int first = (int)((long long)q * N / P), last = (int)((long long)(q + 1) * N / P) - 1;
  const int pfl = I.pf_of_left[first], pfr = I.pf_of_right[last];
  const int ql = (q + P - 1) % P, qr = (q + 1) % P;
  const int d = I.max_delay, o = I.at_order, S = I.n_stages;
  const long long n0 = *I.step;
  if (tid == 0) {
    pdi.first = pdp.first = first;
    pdi.last = pdp.last = last;
  }
  StageArgs A;
  A.insts = nullptr;
  A.tiles = nullptr;
  A.TE = U.TE;
  A.NT = nth;
  A.O = U.O;
  A.visc = 0;  // viscous instances are not run unsynchronised
  LimArgs L;
  L.insts = nullptr;
  L.blocks = nullptr;
  L.EPB = EPB;
  for (long long n = n0; n < n0 + U.n_steps; ++n) {
    for (int s = 0; s < S; ++s) {
      const int c = (int)(S * n + s);
      const double *win = stage_input(I, s);
      // a. the traces of the stage input at the PE faces: the first element's at
      // xi = -1 (right side of the left PE face), the last element's at xi = +1
      // (left side of the right PE face), formed as the stage kernel forms them
      for (int t = tid; t < 2 * nv; t += nth) {
        const int side = t / nv, v = t - side * nv;
        if (side == 0 && pfl >= 0) {
          const double *w = win + ((size_t)v * N + first) * Q;
          I.ring_in[ring_trace(I, n, s, pfl, 1) + v] =
              MIX ? f2d_exact(trace_f<Q>(w, true)) : trace_of<Q>(w, true);
        } else if (side == 1 && pfr >= 0) {
          const double *w = win + ((size_t)v * N + last) * Q;
          I.ring_in[ring_trace(I, n, s, pfr, 0) + v] =
              MIX ? f2d_exact(trace_f<Q>(w, false)) : trace_of<Q>(w, false);
        }
      }
      __syncthreads();
      // b. publish them (after the emulated extra work of a slow PE), observe
      // the neighbours' stage inputs, and agree on the common level of each PE
      // face's flux
      if (tid == 0) {
        if (q == U.slow_pe)
          for (int t = 0; t < U.slow_us; ++t) __nanosleep(1000);
        if (q != U.withheld) {
          __threadfence();
          atomicExch(&U.pub_in[q], c + 1);
        }
        int kl = 0, kr = 0;
        if (pfl >= 0) {
          kl = wait_delay(&U.pub_in[ql], n, s, S, d, o, U.spin_limit);
          if (kl >= 0) kl = agree_delay(agree_slot(U, pfl, s, n), n, kl);
        }
        if (pfr >= 0 && kl >= 0) {
          kr = wait_delay(&U.pub_in[qr], n, s, S, d, o, U.spin_limit);
          if (kr >= 0) kr = agree_delay(agree_slot(U, pfr, s, n), n, kr);
        }
        pdi.k[0] = kl;
        pdi.k[1] = kr;
        if (kl < 0 || kr < 0) {
          s_abort = 1;
          report_error(I, ADG_ERR_TIMEOUT, first, s, n);
        } else {
          if (pfl >= 0) atomicAdd(&U.hist[kl], 1ull);
          if (pfr >= 0) atomicAdd(&U.hist[kr], 1ull);
        }
      }
      __syncthreads();
      if (s_abort) return;
      // c. the stage, tile by tile
      A.s = s;
      for (int e0 = first; e0 <= last; e0 += U.TE) {
        stage_body<Q, MIX ? ADG_MIXED : ADG_FP64, true>(M, A, I, e0, min(U.TE, last + 1 - e0),
                                                        n, &pdi);
        __syncthreads();
      }
      // d. publish the pre-limit outputs, and observe the neighbours'
      if (tid == 0) {
        if (q != U.withheld) {
          __threadfence();
          atomicExch(&U.pub_pre[q], c + 1);
        }
        int kl = 0, kr = 0;
        if (pfl >= 0) kl = wait_delay(&U.pub_pre[ql], n, s, S, d, o, U.spin_limit);
        if (pfr >= 0 && kl >= 0) kr = wait_delay(&U.pub_pre[qr], n, s, S, d, o, U.spin_limit);
        pdp.k[0] = kl;
        pdp.k[1] = kr;
        if (kl < 0 || kr < 0) {
          s_abort = 1;
          report_error(I, ADG_ERR_TIMEOUT, first, s, n);
        } else {
          if (pfl >= 0) atomicAdd(&U.hist[MAXD + 1 + kl], 1ull);
          if (pfr >= 0) atomicAdd(&U.hist[MAXD + 1 + kr], 1ull);
        }
      }
      __syncthreads();
      if (s_abort) return;
      // e. the limiter, block by block
      L.s = s;
      for (int e0 = first; e0 <= last; e0 += EPB) {
        limiter_body<Q, G, MIX, EPB, true>(M, L, I, e0, min(EPB, last + 1 - e0), n, &pdp);
        __syncthreads();
      }
    }
  }
}

// Counters of every PE: all stages before the instance's current step
// published; agreement slots of every PE face empty.
static __global__ void unsync_reset_kernel(const Inst *inst, int *pub_in, int *pub_pre,
                                    unsigned long long *agree, int n_pe, int npf) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n_pe) {
    const int c = (int)(inst->n_stages * *inst->step);
    pub_in[q] = c;
    pub_pre[q] = c;
  }
  if (q < npf * ADG_MAX_STAGES * (MAXD + 1)) agree[q] = 0ull;
}

template <int Q, int G, bool MIX, int EPB>
cudaError_t unsync_launch_q(const Mech &M, const UnsyncArgs &U, int nv, cudaStream_t st) {
  const size_t smem_stage =
      stage_smem_bytes(U.TE, Q, M.ns, M.nr, M.nterm, U.O, MIX ? ADG_MIXED : ADG_FP64);
  const size_t smem_lim = limiter_smem_bytes<Q, G, MIX, EPB>(nv, M.ns);
  const size_t smem = smem_stage > smem_lim ? smem_stage : smem_lim;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  int per_sm = 0, dev = 0, n_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, unsync_kernel<Q, G, MIX, EPB>, LIM_THREADS, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if ((long long)per_sm * n_sm < U.n_pe) return cudaErrorCooperativeLaunchTooLarge;
  const int n_agree = U.npf * ADG_MAX_STAGES * (MAXD + 1);
  const int n_reset = U.n_pe > n_agree ? U.n_pe : n_agree;
  unsync_reset_kernel<<<(n_reset + 127) / 128, 128, 0, st>>>(U.inst, U.pub_in, U.pub_pre,
                                                             U.agree, U.n_pe, U.npf);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Mech m = M;
  UnsyncArgs u = U;
  void *args[] = {&m, &u};
  return cudaLaunchCooperativeKernel((const void *)unsync_kernel<Q, G, MIX, EPB>, dim3(U.n_pe),
                                     dim3(LIM_THREADS), args, smem, st);
}

template <int Q, bool MIX, int EPB>
cudaError_t unsync_launch_qe(const Mech &M, const UnsyncArgs &U, int nv, cudaStream_t st) {
  if (nv <= 16) return unsync_launch_q<Q, 16, MIX, EPB>(M, U, nv, st);
  return unsync_launch_q<Q, 32, MIX, EPB>(M, U, nv, st);
}

// One variant (precision MIX, limiter CTAs of EPB elements) of the mode.
template <bool MIX, int EPB>
cudaError_t unsync_launch_variant(const Mech &M, const UnsyncArgs &U, int Q, int nv,
                                  cudaStream_t st) {
  switch (Q) {
    case 2: return unsync_launch_qe<2, MIX, EPB>(M, U, nv, st);
    case 3: return unsync_launch_qe<3, MIX, EPB>(M, U, nv, st);
    case 4: return unsync_launch_qe<4, MIX, EPB>(M, U, nv, st);
    case 5: return unsync_launch_qe<5, MIX, EPB>(M, U, nv, st);
  }
  return cudaErrorInvalidValue;
}

template <bool MIX, int EPB>
cudaError_t unsync_prepare_variant() {
  const int lim = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define ADG_SET(...) \
  if (e == cudaSuccess) \
  e = cudaFuncSetAttribute(__VA_ARGS__, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
  ADG_SET(unsync_kernel<2, 16, MIX, EPB>);
  ADG_SET(unsync_kernel<3, 16, MIX, EPB>);
  ADG_SET(unsync_kernel<4, 16, MIX, EPB>);
  ADG_SET(unsync_kernel<5, 16, MIX, EPB>);
  ADG_SET(unsync_kernel<2, 32, MIX, EPB>);
  ADG_SET(unsync_kernel<3, 32, MIX, EPB>);
  ADG_SET(unsync_kernel<4, 32, MIX, EPB>);
  ADG_SET(unsync_kernel<5, 32, MIX, EPB>);
#undef ADG_SET
  return e;
}

}  // namespace adg
