// FMA throughput of this GPU's FP64 and FP32 pipes, the ALU denominators of
// the stage kernel's roofline (build: nvcc -O3 -gencode
// arch=compute_103a,code=sm_103a fma_peak.cu -o fma_peak).
//
// Every thread runs CH independent FMA chains of ITER steps each, so the pipe,
// not the dependency latency, bounds the rate; the grid holds WAVES full waves
// of 256-thread CTAs on every SM. The chains' results are summed and written,
// so that no chain can be dropped. Prints one line per type:
//   fp64 <TFLOP/s> <ms> and fp32 <TFLOP/s> <ms>, counting an FMA as 2 flops,
// best of 5 launches after a warm-up launch, timed with CUDA events.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int CH = 8, ITER = 4096, THREADS = 256, WAVES = 8;

template <typename T>
__global__ void fma_chains(T *out, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < ITER; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int run(const char *name, int n_sm) {
  const int blocks = n_sm * WAVES * (2048 / THREADS);
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * THREADS) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<blocks, THREADS>>>(out, (T)0.999999, (T)1e-7);
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    fma_chains<T><<<blocks, THREADS>>>(out, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  if (cudaGetLastError() != cudaSuccess) return 1;
  const double flops = 2.0 * CH * ITER * (double)blocks * THREADS;
  printf("%s %.4f %.4f\n", name, flops / (best * 1e-3) / 1e12, best);
  cudaFree(out);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return 0;
}

int main() {
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (run<double>("fp64", n_sm)) return 1;
  if (run<float>("fp32", n_sm)) return 1;
  return 0;
}
