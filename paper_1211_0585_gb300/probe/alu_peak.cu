// Arithmetic-pipe throughput probe: FP64 and FP32 FMA rates of the GPU it
// runs on (the roofline denominators of the ALU-bound kernels). Each thread
// runs 8 independent FMA chains; prints one JSON line.
#include <cstdio>
#include <cuda_runtime.h>

template <typename T>
__global__ void fma_loop(T *out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
double tflops(int blocks, int threads, int iters) {
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_loop<T><<<blocks, threads>>>(out, 10, (T)0.999, (T)1e-3);
  cudaDeviceSynchronize();
  double best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    fma_loop<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-3);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double f = 2.0 * 8 * 16 * (double)iters * blocks * threads / (ms * 1e9);
    if (f > best) best = f;
  }
  cudaFree(out);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

int main() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) { printf("{\"error\": \"no device\"}\n"); return 1; }
  const int sms = p.multiProcessorCount;
  const double f64 = tflops<double>(sms * 4, 256, 1000);
  const double f32 = tflops<float>(sms * 8, 256, 10000);
  printf("{\"device\": \"%s\", \"sms\": %d, \"fp64_tflops\": %.4f, \"fp32_tflops\": %.4f}\n", p.name, sms, f64, f32);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
