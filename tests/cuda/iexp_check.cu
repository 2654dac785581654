// Test harness (not part of the library): the library's integer-pipeline exp
// (csrc/adg_math.cuh) on the GPU, against the same function compiled for the
// host (bit for bit), and both it and CUDA's exp against expl in extended
// precision on the host; the mixed variant's table logarithm likewise (against
// its host build and logl), and its Newton-Raphson reciprocal (csrc/adg_device.cuh)
// against the exact reciprocal, and its two-step reciprocal and integer-pipe
// split of a double into a float pair; its integer-pipe double -> float
// conversion at the edges of the float range against the host's conversion.
// Prints one JSON line.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../paper_2501_01747_gb300/csrc/adg_device.cuh"
#include "d2f_edge_values.h"

__global__ void eval(const double *x, double *mine, double *cuda_ref, int n, adg::IExpTable tab) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  mine[i] = adg::iexp(x[i], tab);
  cuda_ref[i] = exp(x[i]);
}

__global__ void eval_log(const double *x, double *ln, double *rc, int n, adg::LogTable tb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ln[i] = adg::log_tab(x[i], tb);
  rc[i] = adg::recip_nr(x[i]);
}

__global__ void eval_split(const double *x, float *hi, float *lo, double *rc2, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const adg::DF d = adg::d2df_int(x[i]);
  hi[i] = d.hi;
  lo[i] = d.lo;
  rc2[i] = adg::recip_nr2(x[i]);
}

__global__ void eval_d2f(const double *x, float *f, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  f[i] = adg::d2f_int(x[i]);
}

static double ulp_err(double got, long double ref) {
  double rd = (double)ref;
  double ulp = std::nextafter(rd, INFINITY) - rd;
  return (double)fabsl((long double)got - ref) / ulp;
}

int main() {
  const int n = 1 << 21;
  std::vector<double> x(n);
  srand(12345);
  for (int i = 0; i < n; ++i) {
    double u = (double)rand() / RAND_MAX;
    if (i % 5 == 0) x[i] = -700.0 + 1400.0 * u;        // whole range
    else if (i % 5 == 1) x[i] = -80.0 + 120.0 * u;     // Arrhenius arguments
    else if (i % 5 == 2) x[i] = (u - 0.5) * 1e-3;      // near zero
    else if (i % 5 == 3) x[i] = ldexp(u - 0.5, -(i % 60));  // tiny arguments
    else x[i] = (double)((i / 5) % 2000 - 1000) * (0.6931471805599453 / 32.0);  // table nodes
  }
  const adg::IExpTable tab = {ADG_IEXP_TABLE, ADG_IEXP_TABLE32};
  double *dx, *dm, *dr;
  if (cudaMalloc(&dx, n * 8) || cudaMalloc(&dm, n * 8) || cudaMalloc(&dr, n * 8)) return 2;
  cudaMemcpy(dx, x.data(), n * 8, cudaMemcpyHostToDevice);
  eval<<<(n + 255) / 256, 256>>>(dx, dm, dr, n, tab);
  std::vector<double> m(n), r(n);
  cudaMemcpy(m.data(), dm, n * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(r.data(), dr, n * 8, cudaMemcpyDeviceToHost);
  cudaError_t err = cudaGetLastError();
  long long mismatch = 0;
  double max_ulp = 0.0, cuda_max_ulp = 0.0;
  for (int i = 0; i < n; ++i) {
    if (m[i] != adg::iexp(x[i], tab)) ++mismatch;
    long double ref = expl((long double)x[i]);
    double e = ulp_err(m[i], ref), ec = ulp_err(r[i], ref);
    if (e > max_ulp) max_ulp = e;
    if (ec > cuda_max_ulp) cuda_max_ulp = ec;
  }
  // the table logarithm (outside [1/2, 2), where it takes the library's) and the
  // reciprocal: temperatures, then positive and negative values over 60 decades
  std::vector<double> y(n);
  for (int i = 0; i < n; ++i) {
    double u = (double)rand() / RAND_MAX;
    if (i % 2 == 0) y[i] = 50.0 + 9950.0 * u;
    else y[i] = ldexp(0.5 + 0.5 * u, (i / 2) % 200 - 100);
    if (y[i] >= 0.5 && y[i] < 2.0) y[i] *= 4.0;
    if (i % 4 == 3) y[i] = -y[i];  // the reciprocal's sign; the logarithm skips these
  }
  double *dy, *dl, *dc;
  if (cudaMalloc(&dy, n * 8) || cudaMalloc(&dl, n * 8) || cudaMalloc(&dc, n * 8)) return 2;
  cudaMemcpy(dy, y.data(), n * 8, cudaMemcpyHostToDevice);
  const adg::LogTable ltab = {ADG_LOG_TABLE_LN, ADG_LOG_TABLE_INV};
  eval_log<<<(n + 255) / 256, 256>>>(dy, dl, dc, n, ltab);
  std::vector<double> l(n), c(n);
  cudaMemcpy(l.data(), dl, n * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(c.data(), dc, n * 8, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) err = cudaGetLastError();
  long long log_mismatch = 0;
  double log_max_ulp = 0.0, recip_max_rel = 0.0;
  for (int i = 0; i < n; ++i) {
    if (y[i] > 0.0) {
      if (l[i] != adg::log_tab(y[i], ltab)) ++log_mismatch;
      const long double ref = logl((long double)y[i]);
      const double rd = fabs((double)ref);
      const double ulp = std::nextafter(rd, INFINITY) - rd;
      log_max_ulp = fmax(log_max_ulp, (double)(fabsl((long double)l[i] - ref) / ulp));
    }
    const long double rr = 1.0L / (long double)y[i];
    recip_max_rel = fmax(recip_max_rel, (double)fabsl(((long double)c[i] - rr) / rr));
  }
  // the float-pair split and the two-step reciprocal, on the same values and on
  // rate-constant-like magnitudes over the float range
  for (int i = 0; i < n; i += 3) y[i] = ldexp(0.5 + (double)rand() / RAND_MAX, (i / 3) % 216 - 96);
  float *dh, *dlo;
  double *dc2;
  if (cudaMalloc(&dh, n * 4) || cudaMalloc(&dlo, n * 4) || cudaMalloc(&dc2, n * 8)) return 2;
  cudaMemcpy(dy, y.data(), n * 8, cudaMemcpyHostToDevice);
  eval_split<<<(n + 255) / 256, 256>>>(dy, dh, dlo, dc2, n);
  std::vector<float> hh(n), ll(n);
  std::vector<double> c2(n);
  cudaMemcpy(hh.data(), dh, n * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(ll.data(), dlo, n * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(c2.data(), dc2, n * 8, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) err = cudaGetLastError();
  long long split_hi_mismatch = 0;
  double split_max_rel = 0.0, recip2_max_rel = 0.0;
  for (int i = 0; i < n; ++i) {
    if (hh[i] != (float)y[i]) ++split_hi_mismatch;
    const long double sum = (long double)hh[i] + (long double)ll[i];
    split_max_rel = fmax(split_max_rel, (double)fabsl((sum - (long double)y[i]) / y[i]));
    const long double rr = 1.0L / (long double)y[i];
    recip2_max_rel = fmax(recip2_max_rel, (double)fabsl(((long double)c2[i] - rr) / rr));
  }
  // the conversion at the edges of the float range, bit for bit (NaN as NaN)
  const std::vector<double> ev = d2f_edge_values(1 << 18);
  const int ne = (int)ev.size();
  double *dev_e;
  float *dev_f;
  if (cudaMalloc(&dev_e, ne * 8) || cudaMalloc(&dev_f, ne * 4)) return 2;
  cudaMemcpy(dev_e, ev.data(), ne * 8, cudaMemcpyHostToDevice);
  eval_d2f<<<(ne + 255) / 256, 256>>>(dev_e, dev_f, ne);
  std::vector<float> ef(ne);
  cudaMemcpy(ef.data(), dev_f, ne * 4, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) err = cudaGetLastError();
  long long edge_mismatch = 0;
  for (int i = 0; i < ne; ++i) {
    const float ref = (float)ev[i];
    if (std::isnan(ev[i])) {
      if (!std::isnan(ef[i])) ++edge_mismatch;
    } else if (std::memcmp(&ef[i], &ref, 4) != 0) {
      ++edge_mismatch;
    }
  }
  printf("{\"n\": %d, \"edge_n\": %d, \"edge_mismatch\": %lld, \"host_mismatch\": %lld, \"max_ulp\": %.4f, \"cuda_exp_max_ulp\": %.4f, "
         "\"log_host_mismatch\": %lld, \"log_max_ulp\": %.4f, \"recip_max_rel\": %.3g, "
         "\"recip2_max_rel\": %.3g, \"split_hi_mismatch\": %lld, \"split_max_rel\": %.3g, "
         "\"cuda\": \"%s\"}\n", n, ne, edge_mismatch, mismatch, max_ulp, cuda_max_ulp, log_mismatch, log_max_ulp,
         recip_max_rel, recip2_max_rel, split_hi_mismatch, split_max_rel, cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}
