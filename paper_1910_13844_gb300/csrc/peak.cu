// Measured FP32 throughput of the current device (ls_fp32_peak): the denominator of the FP32-pipe
// roofline of the FFT passes.  Three kernels of known operation counts -- scalar FFMA, scalar FMUL
// and packed add.f32x2 -- each run eight independent dependency chains per thread over a grid of
// eight 256-thread blocks per SM, eight dependent steps per chain and loop iteration, timed with
// CUDA events after one untimed launch.
#include <cuda_runtime.h>

#include "common.cuh"

namespace lsgpu {

constexpr int kPeakIters = 1024;
constexpr int kPeakChains = 8;
constexpr int kPeakReps = 8;   // dependent steps of each chain per loop iteration (loop overhead < 3%)

template <int OP>
__global__ void __launch_bounds__(256) k_peak(float seed, float* sink) {
  float a[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) a[j] = seed + threadIdx.x * 1e-7f + j;
  const float b = 0.999999f, c = 1e-7f;
  if constexpr (OP == 2) {
    // packed adds: each instruction adds two float lanes
    unsigned long long p[kPeakChains / 2];
#pragma unroll
    for (int j = 0; j < kPeakChains / 2; ++j)
      asm("mov.b64 %0, {%1, %2};" : "=l"(p[j]) : "f"(a[2 * j]), "f"(a[2 * j + 1]));
    unsigned long long q;
    asm("mov.b64 %0, {%1, %2};" : "=l"(q) : "f"(c), "f"(-c));
#pragma unroll 1
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
      for (int r = 0; r < kPeakReps; ++r)
#pragma unroll
        for (int j = 0; j < kPeakChains / 2; ++j) asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(p[j]) : "l"(q));
    }
#pragma unroll
    for (int j = 0; j < kPeakChains / 2; ++j) asm("mov.b64 {%0, %1}, %2;" : "=f"(a[2 * j]), "=f"(a[2 * j + 1]) : "l"(p[j]));
  } else {
#pragma unroll 1
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
      for (int r = 0; r < kPeakReps; ++r)
#pragma unroll
        for (int j = 0; j < kPeakChains; ++j) {
          if constexpr (OP == 0) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[j]) : "f"(b), "f"(c));
          else asm volatile("mul.rn.f32 %0, %0, %1;" : "+f"(a[j]) : "f"(b));
        }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += a[j];
  if (s == 12345.678f) *sink = s;   // keeps the chains live; never true for these inputs
}

}  // namespace lsgpu

using namespace lsgpu;

extern "C" int ls_fp32_peak(double* out, void* stream) {
  if (!out) { set_last_error("null argument"); return LS_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  LS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* sink = nullptr;
  LS_CUDA_TRY(cudaMallocAsync((void**)&sink, sizeof(float), st));
  cudaEvent_t e0, e1;
  LS_CUDA_TRY(cudaEventCreate(&e0));
  LS_CUDA_TRY(cudaEventCreate(&e1));
  const int blocks = 8 * sms, threads = 256;
  // lane operations per thread and iteration: reps * chains (FFMA, FMUL: reps * chains instructions of one
  // lane-op; packed add: reps * chains / 2 instructions of two)
  const double lane_ops = (double)blocks * threads * kPeakIters * kPeakReps * kPeakChains;
  int rc = LS_OK;
  for (int op = 0; op < 3 && rc == LS_OK; ++op) {
    auto launch = [&] {
      if (op == 0) k_peak<0><<<blocks, threads, 0, st>>>(1.0f, sink);
      else if (op == 1) k_peak<1><<<blocks, threads, 0, st>>>(1.0f, sink);
      else k_peak<2><<<blocks, threads, 0, st>>>(1.0f, sink);
    };
    launch();
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5; ++r) launch();
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
      set_last_error("FP32 peak timing failed: %s", cudaGetErrorString(cudaGetLastError()));
      rc = LS_ECUDA;
      break;
    }
    out[op] = 5.0 * lane_ops / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  if (rc == LS_OK) LS_CUDA_TRY(cudaStreamSynchronize(st));
  return rc;
}
