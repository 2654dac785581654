// Test harness (not part of the library): evaluates the library's table-driven
// exp (csrc/adg_math.cuh) and CUDA's exp on the same arguments and prints the
// largest difference in units in the last place as one JSON line.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2501_01747_gb300/csrc/adg_math.cuh"

using adg::ExpTable;

__global__ void eval(const double *x, double *mine, double *ref, int n, ExpTable tab) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  mine[i] = adg::fexp(x[i], tab);
  ref[i] = exp(x[i]);
}

int main() {
  const int n = 1 << 20;
  std::vector<double> x(n);
  srand(12345);
  for (int i = 0; i < n; ++i) {
    double u = (double)rand() / RAND_MAX;
    if (i % 4 == 0) x[i] = -700.0 + 1400.0 * u;        // whole range
    else if (i % 4 == 1) x[i] = -80.0 + 120.0 * u;     // Arrhenius arguments
    else if (i % 4 == 2) x[i] = (u - 0.5) * 1e-3;      // near zero
    else x[i] = (double)((i / 4) % 2000 - 1000) * (0.6931471805599453 / 32.0);  // table nodes
  }
  ExpTable tab;
  for (int j = 0; j < 32; ++j) tab.t[j] = (double)exp2l((long double)j / 32.0L);
  long double l = logl(2.0L) / 32.0L;
  int ex;
  long double mant = frexpl(l, &ex);
  long double hi = ldexpl(floorl(ldexpl(mant, 32)), ex - 32);
  tab.l_hi = (double)hi;
  tab.l_lo = (double)(l - hi);
  double *dx, *dm, *dr;
  if (cudaMalloc(&dx, n * 8) || cudaMalloc(&dm, n * 8) || cudaMalloc(&dr, n * 8)) return 2;
  cudaMemcpy(dx, x.data(), n * 8, cudaMemcpyHostToDevice);
  eval<<<(n + 255) / 256, 256>>>(dx, dm, dr, n, tab);
  std::vector<double> m(n), r(n);
  cudaMemcpy(m.data(), dm, n * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(r.data(), dr, n * 8, cudaMemcpyDeviceToHost);
  cudaError_t err = cudaGetLastError();
  double max_ulp = 0.0, max_rel = 0.0;
  for (int i = 0; i < n; ++i) {
    double ulp = std::nextafter(r[i], INFINITY) - r[i];
    double d = std::fabs(m[i] - r[i]);
    if (d / ulp > max_ulp) max_ulp = d / ulp;
    if (d / r[i] > max_rel) max_rel = d / r[i];
  }
  printf("{\"n\": %d, \"max_ulp\": %.3f, \"max_rel\": %.3e, \"cuda\": \"%s\"}\n", n, max_ulp,
         max_rel, cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}
