// FMA throughput of one GPU: the arithmetic ceiling ("alu" roofline) for the
// FP64 kernels and the issue ceiling of the FP32 FFT passes.  Each thread runs
// 8 independent fused multiply-add chains (no memory traffic but one store per
// thread); 8 blocks of 256 threads per SM; best of 5 launches timed with CUDA
// events; a FMA counts as 2 floating-point operations.  Not part of the
// library: build and run with
//   nvcc -O3 -gencode arch=compute_103a,code=sm_103a paper_2105_03297_gb300/alu_peak.cu -o alu_peak && ./alu_peak
#include <cstdio>
#include <cuda_runtime.h>
template <typename T, int CH>
__global__ void __launch_bounds__(256) fma_loop(T* out, T a, T b, int it) {
  T v[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < it; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <typename T, int CH> void run(const char* name, int it, int nsm) {
  const int blocks = nsm * 8, threads = 256;
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  fma_loop<T, CH><<<blocks, threads>>>(out, (T)0.999999, (T)1e-7, it);
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    fma_loop<T, CH><<<blocks, threads>>>(out, (T)0.999999, (T)1e-7, it);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
  }
  const double flops = 2.0 * CH * (double)it * blocks * threads;
  printf("%s: %.3f ms, %.2f TFLOP/s (%d blocks x %d threads, %d chains, %d iterations) err=%s\n", name, best,
         flops / best / 1e9, blocks, threads, CH, it, cudaGetErrorString(cudaGetLastError()));
  cudaFree(out);
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("%s, %d SMs, max SM clock %d MHz\n", p.name, p.multiProcessorCount, clk / 1000);
  run<double, 8>("fp64 fma", 4096, p.multiProcessorCount);
  run<float, 8>("fp32 fma", 65536, p.multiProcessorCount);
  return 0;
}
