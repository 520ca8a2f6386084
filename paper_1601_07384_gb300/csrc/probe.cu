// Throughput probe of the arithmetic pipes the operator kernels are rated against: independent chains
// of binary64 FMAs and of binary32 FMAs, every SM filled, timed with CUDA events.  The binary64 rate
// bounds the plain FP64 operator kernel; the binary32 rate, divided by the 12 FP32 operations of one
// binary64-accurate pair product, bounds the pair kernel.
#include <chrono>

#include "solver.h"

namespace stdg {

constexpr int kProbeChains = 8;      // independent accumulators per thread
constexpr int kProbeIters = 4096;    // FMAs per chain

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T a, T b, T* out) {
  T acc[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += acc[c];
  if (s == (T)-1) out[0] = s;        // keeps the chains live; never true for these inputs
}

template <typename T>
static double probe_tflops(int nsm, cudaStream_t st, T* sink, float* ms_out) {
  const int blocks = nsm * 8, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  k_fma_probe<T><<<blocks, threads, 0, st>>>((T)0.999, (T)1e-3, sink);      // warm-up
  cudaEventRecord(e0, st);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) k_fma_probe<T><<<blocks, threads, 0, st>>>((T)0.999, (T)1e-3, sink);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  *ms_out = ms / reps;
  const double flops = 2.0 * (double)blocks * threads * kProbeChains * kProbeIters;
  return flops / (ms / reps * 1e-3) / 1e12;
}

}  // namespace stdg

using namespace stdg;

extern "C" stdg_status stdg_fma_probe(double* tflops_fp64, double* tflops_fp32, void* stream) {
  if (!tflops_fp64 || !tflops_fp32) { set_error("stdg_fma_probe: NULL argument"); return STDG_EINVAL; }
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_error("stdg_fma_probe: no CUDA device");
    return STDG_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* sink = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess) { set_error("stdg_fma_probe: cudaMalloc failed"); return STDG_ENOMEM; }
  float ms64 = 0.0f, ms32 = 0.0f;
  *tflops_fp64 = probe_tflops<double>(nsm, st, sink, &ms64);
  *tflops_fp32 = probe_tflops<float>(nsm, st, reinterpret_cast<float*>(sink), &ms32);
  const cudaError_t e = cudaGetLastError();
  cudaFree(sink);
  if (e != cudaSuccess) { set_error("stdg_fma_probe: %s", cudaGetErrorString(e)); return STDG_ECUDA; }
  return STDG_OK;
}
