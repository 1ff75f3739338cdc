// Arithmetic-pipe peaks of the GPU this library runs on, measured in the same
// process as the products they are compared with: FP32 FMA, FP64 FMA and
// FP64 tensor-core (mma.sync m8n8k4) throughput.  These are the denominators
// of the rooflines of the kernels that are bound by arithmetic rather than by
// HBM (the FP64 products and the FP32 tree).  Built as its own small library
// (libhm_probe.so); nothing in the product path calls it.
//
// Each probe launches SMs x blocks_per_sm blocks of `threads` threads; every
// thread (or warp, for mma) runs `iters` iterations over 8 independent
// accumulation chains, so the pipe, not a dependency, bounds the rate.  The
// kernels touch memory only to store one value per thread at the end (so the
// compiler keeps the arithmetic).  Time: CUDA events around one launch after
// a warm-up launch, best of `repeats`.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int CH = 8;   // independent chains per thread

__global__ void k_ffma(float* out, int iters, float a, float b) {
  float x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < CH; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double* out, int iters, double a, double b) {
  double x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// D = A B + C for one 8x8x4 tile per warp and chain (row-major A, column-major
// B; each lane holds one element of A and B and two of C/D).
__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void k_dmma(double* out, int iters, double a, double b) {
  double d[CH][2];
#pragma unroll
  for (int c = 0; c < CH; ++c) { d[c][0] = threadIdx.x * 1e-3; d[c][1] = c; }
  const double av = a + threadIdx.x * 1e-9, bv = b - threadIdx.x * 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) dmma(d[c][0], d[c][1], av, bv);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += d[c][0] + d[c][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

// which: 0 FP32 FMA, 1 FP64 FMA, 2 FP64 mma.sync.  On success writes the
// achieved TFLOP/s (2 flops per multiply-add), the best launch time in
// milliseconds and the number of SMs, and returns 0; returns the CUDA error
// code otherwise.
int hm_probe_peak(int which, int blocks_per_sm, int threads, int iters, int repeats, double* tflops,
                  double* best_ms, int* sms_out) {
  if (which < 0 || which > 2 || blocks_per_sm < 1 || threads < 32 || threads > 1024 || (threads & 31) ||
      iters < 1 || repeats < 1 || !tflops || !best_ms)
    return static_cast<int>(cudaErrorInvalidValue);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return static_cast<int>(e);
  const int blocks = sms * blocks_per_sm;
  void* out = nullptr;
  e = cudaMalloc(&out, static_cast<size_t>(blocks) * threads * sizeof(double));
  if (e != cudaSuccess) return static_cast<int>(e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&]() {
    if (which == 0) k_ffma<<<blocks, threads>>>(static_cast<float*>(out), iters, 0.9999999f, 1e-7f);
    else if (which == 1) k_dfma<<<blocks, threads>>>(static_cast<double*>(out), iters, 0.9999999, 1e-7);
    else k_dmma<<<blocks, threads>>>(static_cast<double*>(out), iters, 0.999, 1e-3);
  };
  launch();
  e = cudaDeviceSynchronize();
  float best = 1e30f;
  for (int rep = 0; rep < repeats && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return static_cast<int>(e);
  double flops;
  if (which == 2) flops = 2.0 * 8 * 8 * 4 * CH * static_cast<double>(iters) * blocks * (threads / 32);
  else flops = 2.0 * 4 * CH * static_cast<double>(iters) * blocks * threads;
  *best_ms = best;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (sms_out) *sms_out = sms;
  return 0;
}

}  // extern "C"
