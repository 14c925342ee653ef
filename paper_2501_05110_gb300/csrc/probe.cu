// FMA throughput probe: the arithmetic roof against which the operator apply is reported.
//
// Every thread runs eight independent chains of fused multiply-adds (enough to cover the FMA pipe's
// latency) for a fixed number of iterations; the grid fills every SM several times over.  The chains
// cannot be folded away: their results feed one store per thread.
#include <cuda_runtime.h>

#include "sap_internal.h"

namespace sap {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* out, int iters, T a, T b) {
  T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
  T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

template <typename T>
cudaError_t run_probe(double* flops_per_s) {
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  const int blocks = sms * 16, threads = 256;
  const int iters = sizeof(T) == 8 ? 64 : 2048;
  T* out = nullptr;
  if ((err = cudaMalloc(&out, sizeof(T) * blocks * threads)) != cudaSuccess) return err;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_probe_kernel<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));  // warm-up
  cudaEventRecord(e0);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) fma_probe_kernel<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
  cudaEventRecord(e1);
  err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return err;
  const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads * reps;
  *flops_per_s = flops / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace
}  // namespace sap

extern "C" sap_status sap_probe_fma(int prec, double* flops_per_s) {
  if (!flops_per_s || (prec != SAP_PREC_FP64 && prec != SAP_PREC_FP32)) return SAP_EINVAL;
  const cudaError_t err = prec == SAP_PREC_FP64 ? sap::run_probe<double>(flops_per_s) : sap::run_probe<float>(flops_per_s);
  return err == cudaSuccess ? SAP_OK : SAP_ECUDA;
}
