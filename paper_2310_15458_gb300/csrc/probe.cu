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

namespace {

// Eight independent accumulator chains of m8n8k4 FP64 tensor-core products per
// warp (each product is 2 x 8 x 8 x 4 = 512 flops).
__global__ void __launch_bounds__(256) k_dmma_probe(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-9, b = 0.999999;
  double c[PR_CHAINS][2];
#pragma unroll
  for (int q = 0; q < PR_CHAINS; ++q) c[q][0] = c[q][1] = q * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < PR_CHAINS; ++q)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c[q][0]), "+d"(c[q][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < PR_CHAINS; ++q) s += c[q][0] + c[q][1];
  if (s == 12345.678) out[blockIdx.x] = s;
}

}  // namespace

extern "C" rss_status rss_probe_dmma(double* tflops, double* ms, void* stream) {
  if (!tflops) {
    rss_set_error("rss_probe_dmma: tflops is NULL");
    return RSS_EINVAL;
  }
  int dev = 0, sms = 0;
  RSS_CUDA(cudaGetDevice(&dev));
  RSS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* out = nullptr;
  RSS_CUDA(pool_malloc(reinterpret_cast<void**>(&out), sizeof(double) * 8 * sms, st));
  const int blocks = 8 * sms, threads = 256, iters = 1 << 11;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RSS_CUDA(cudaEventCreate(&e0));
  RSS_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 6; ++rep) {
    RSS_CUDA(cudaEventRecord(e0, st));
    k_dmma_probe<<<blocks, threads, 0, st>>>(out, iters);
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
  const double flops = 512.0 * PR_CHAINS * (double)iters * blocks * (threads / 32);
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return RSS_OK;
}
