// FP64 throughput probe: the denominator of the roofline of the FP64-bound
// phases (column-pivoted QR, small LUs), measured on the device the library runs
// on.  Every thread runs eight independent chains of fused multiply-adds on
// registers, so the loop issues nothing but DFMA and its loop counter; the grid
// is 8 CTAs of 256 threads per SM.  The paper has no counterpart: this is part
// of measuring the path, not of the path.
#include <cuda_runtime.h>

#include "internal.h"

namespace {

constexpr int PR_CHAINS = 8;

__global__ void __launch_bounds__(256) k_dfma_probe(double* out, int iters, double a, double b) {
  double x[PR_CHAINS];
#pragma unroll
  for (int c = 0; c < PR_CHAINS; ++c) x[c] = threadIdx.x * 1e-9 + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PR_CHAINS; ++c) s += x[c];
  if (s == 12345.678) out[blockIdx.x] = s;   // keeps the chains live; practically never true
}

}  // namespace

extern "C" rss_status rss_probe_fp64(double* tflops, double* ms, void* stream) {
  if (!tflops) {
    rss_set_error("rss_probe_fp64: tflops is NULL");
    return RSS_EINVAL;
  }
  int dev = 0, sms = 0;
  RSS_CUDA(cudaGetDevice(&dev));
  RSS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* out = nullptr;
  RSS_CUDA(pool_malloc(reinterpret_cast<void**>(&out), sizeof(double) * 8 * sms, st));
  const int blocks = 8 * sms, threads = 256, iters = 1 << 14;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RSS_CUDA(cudaEventCreate(&e0));
  RSS_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 6; ++rep) {   // the first launch warms the clocks up
    RSS_CUDA(cudaEventRecord(e0, st));
    k_dfma_probe<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
    RSS_LAUNCHED();
    RSS_CUDA(cudaEventRecord(e1, st));
    RSS_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    RSS_CUDA(cudaEventElapsedTime(&t, e0, e1));
    if (rep > 0 && t < best) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pool_free(out, st);
  const double flops = 2.0 * PR_CHAINS * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return RSS_OK;
}
