// Floating-point issue-rate microbenchmark: the denominator of the FP64 (and
// FP32) roofline for the ERI kernels, which run on the CUDA-core pipes.
//
// Every thread runs ILP independent fused multiply-add chains for ITERS
// iterations.  The kernel records clock64() per block so that the per-SM rate
// (lane-FMAs per SM clock) is obtained independently of the clock the GPU ran
// at; CUDA events give the wall-clock rate.  Prints one JSON object.
//
// Usage: fp_peak [iters]
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <algorithm>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
  fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
  exit(1); } } while (0)

template <typename T, int ILP>
__global__ void fma_chains(T* sink, long long* cycles, int iters, T b, T c) {
  T a[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
      for (int i = 0; i < ILP; ++i) a[i] = fma(a[i], b, c);
    }
  }
  long long t1 = clock64();
  T s = 0;
#pragma unroll
  for (int i = 0; i < ILP; ++i) s += a[i];
  if (s == (T)12345.678) sink[0] = s;  // never true: keeps the chains alive
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

struct Result { double tflops; double per_sm_clk; double ms; };

template <typename T, int ILP>
Result run(int nsm, int blocks_per_sm, int threads, int iters) {
  int nblk = nsm * blocks_per_sm;
  T* sink; long long* cyc;
  CK(cudaMalloc(&sink, sizeof(T)));
  CK(cudaMalloc(&cyc, sizeof(long long) * nblk));
  T b = (T)0.999999, c = (T)1e-7;
  for (int w = 0; w < 2; ++w) fma_chains<T, ILP><<<nblk, threads>>>(sink, cyc, iters / 4 + 1, b, c);
  CK(cudaDeviceSynchronize());
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0));
  fma_chains<T, ILP><<<nblk, threads>>>(sink, cyc, iters, b, c);
  CK(cudaEventRecord(e1));
  CK(cudaEventSynchronize(e1));
  CK(cudaGetLastError());
  float ms = 0; CK(cudaEventElapsedTime(&ms, e0, e1));
  std::vector<long long> h(nblk);
  CK(cudaMemcpy(h.data(), cyc, sizeof(long long) * nblk, cudaMemcpyDeviceToHost));
  long long cmax = *std::max_element(h.begin(), h.end());
  double fmas = (double)nblk * threads * iters * 8.0 * ILP;
  Result r;
  r.ms = ms;
  r.tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  // lane-FMAs per SM per clock, all blocks of an SM resident together
  r.per_sm_clk = (double)blocks_per_sm * threads * iters * 8.0 * ILP / (double)cmax;
  CK(cudaFree(sink)); CK(cudaFree(cyc));
  CK(cudaEventDestroy(e0)); CK(cudaEventDestroy(e1));
  return r;
}

int main(int argc, char** argv) {
  int iters = argc > 1 ? atoi(argv[1]) : 4096;
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, 0));
  int nsm = p.multiProcessorCount;
  int clk_khz = 0; CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0));
  printf("{\"gpu\": \"%s\", \"sm_count\": %d, \"cc\": \"%d.%d\", \"attr_clock_mhz\": %.0f,\n", p.name, nsm,
         p.major, p.minor, clk_khz / 1e3);
  printf(" \"fp64\": [\n");
  const int warps[] = {4, 8, 16, 32};
  bool first = true;
  for (int wi = 0; wi < 4; ++wi) {
    int thr = warps[wi] * 32;
    Result r1 = run<double, 1>(nsm, 1, thr, iters / 16);
    Result r4 = run<double, 4>(nsm, 1, thr, iters / 16);
    Result r8 = run<double, 8>(nsm, 1, thr, iters / 16);
    printf("%s  {\"warps_per_sm\": %d, \"ilp1\": [%.4f, %.3f], \"ilp4\": [%.4f, %.3f], \"ilp8\": [%.4f, %.3f]}",
           first ? "" : ",\n", warps[wi], r1.tflops, r1.per_sm_clk, r4.tflops, r4.per_sm_clk, r8.tflops,
           r8.per_sm_clk);
    first = false;
  }
  printf("\n ],\n \"fp32\": [\n");
  first = true;
  for (int wi = 0; wi < 4; ++wi) {
    int thr = warps[wi] * 32;
    Result r4 = run<float, 4>(nsm, 1, thr, iters);
    Result r8 = run<float, 8>(nsm, 1, thr, iters);
    printf("%s  {\"warps_per_sm\": %d, \"ilp4\": [%.3f, %.3f], \"ilp8\": [%.3f, %.3f]}", first ? "" : ",\n",
           warps[wi], r4.tflops, r4.per_sm_clk, r8.tflops, r8.per_sm_clk);
    first = false;
  }
  printf("\n ],\n \"units\": \"each pair is [TFLOP/s from CUDA events, lane-FMAs per SM per SM-clock]\"}\n");
  return 0;
}
