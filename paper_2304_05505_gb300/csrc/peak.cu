// The FP64 FMA rate of this device, measured: the peak the FP64 build's
// stages are reported against (their GEMMs run on the FP64 pipe of the CUDA
// cores).  Each thread runs eight independent chains of fused multiply-adds
// (enough in flight to cover the pipe's latency); the grid fills every SM
// with four 256-thread blocks.  Nothing is changed on the device.
#include "thc_internal.cuh"

namespace {

constexpr int CHAINS = 8, ITERS = 4096, THREADS = 256;

__global__ void __launch_bounds__(THREADS) dfma_kernel(double m, double c, double* out) {
  double a[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; j++) a[j] = 1e-3 * (threadIdx.x + j);
#pragma unroll 4
  for (int i = 0; i < ITERS; i++) {
#pragma unroll
    for (int j = 0; j < CHAINS; j++) a[j] = fma(a[j], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < CHAINS; j++) s += a[j];
  if (threadIdx.x == 0) out[blockIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" thc_status thc_measure_fp64_rate(void* stream, double* tflops_host) {
  if (!tflops_host) return THC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return THC_ERR_CUDA;
  const int blocks = 4 * nsm;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  thc_status st = THC_OK;
  float ms = 0.0f;
  if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess) return THC_ERR_OOM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { st = THC_ERR_CUDA; goto done; }
  for (int rep = 0; rep < 2; rep++) {   // the first launch warms up
    cudaEventRecord(e0, s);
    dfma_kernel<<<blocks, THREADS, 0, s>>>(0.9999999, 1e-7, out);
    cudaEventRecord(e1, s);
  }
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f)) {
    st = THC_ERR_CUDA;
    goto done;
  }
  *tflops_host = 2.0 * CHAINS * (double)ITERS * THREADS * blocks / (ms * 1e-3) / 1e12;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}
