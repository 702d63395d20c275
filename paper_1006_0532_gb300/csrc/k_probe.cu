// Throughput of the GPU's FP64 pipe, the bound of the FP64 form's advance: a fused
// multiply-add rate measured with a kernel of independent FMA chains (no memory traffic),
// timed with CUDA events on the caller's stream.
#include "pdfx_internal.h"

namespace pdfx {
namespace {

constexpr int kChains = 8;        // independent accumulators per thread
constexpr int kProbeThreads = 256;

__device__ double g_probe_sink[32];   // keeps the chains' results live

__global__ void __launch_bounds__(kProbeThreads) fma_chain_kernel(int iters, double a, double b) {
  double acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = static_cast<double>(threadIdx.x + k) * 1e-3;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k];
  if (threadIdx.x == 0) g_probe_sink[blockIdx.x & 31] = s;
}

}  // namespace
}  // namespace pdfx

extern "C" int pdfx_measure_fp64_rate(double* flops_per_s, void* stream) {
  using namespace pdfx;
  if (!flops_per_s) return PDFX_ERR_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PDFX_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PDFX_ERR_CUDA;
  const int blocks = 8 * sms;
  const int iters = 256;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PDFX_ERR_CUDA;
  // a = 1 - 2^-20 and b small keep the accumulators finite and away from subnormals
  const double a = 1.0 - 9.5367431640625e-07, b = 1e-6;
  fma_chain_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, a, b);   // warm-up
  cudaEventRecord(e0, s);
  fma_chain_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, a, b);
  cudaEventRecord(e1, s);
  float ms = 0.0f;
  int rc = PDFX_OK;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
    rc = PDFX_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PDFX_OK) return rc;
  const double fmas = static_cast<double>(blocks) * kProbeThreads * iters * 16.0 * kChains;
  *flops_per_s = 2.0 * fmas / (static_cast<double>(ms) * 1e-3);
  return cudaGetLastError() == cudaSuccess ? PDFX_OK : PDFX_ERR_CUDA;
}
