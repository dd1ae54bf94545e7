// Device self-tests that need no input data: the bounded wait every persistent
// kernel relies on (it must give up and report, never hang), and the FP32 FMA
// peak that bounds the complex64 CUDA-core path.
#include <cuda_runtime.h>

#include "tc_kernel.cuh"

namespace tn {
namespace {

// one thread waits on an mbarrier that nothing arrives on: the wait must end
// after limit_ns with the error flag raised
__global__ void bounded_wait_kernel(int* err, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  wait_bounded_ns(&bar, 0, err, limit_ns);
}

// independent FMA chains per thread (enough in flight to fill the FP32 pipes)
constexpr int kChains = 8;
__global__ void __launch_bounds__(256) ffma_kernel(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1234.5f) out[0] = s;  // keeps the chains alive; practically never taken
}

}  // namespace

bool selftest_bounded_wait(uint64_t limit_ns, cudaStream_t s) {
  int* d_err = nullptr;
  TN_CUDA(cudaMalloc(&d_err, sizeof(int)));
  int h = 0;
  try {
    TN_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    bounded_wait_kernel<<<1, 1, 0, s>>>(d_err, limit_ns);
    TN_CUDA(cudaGetLastError());
    TN_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TN_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    cudaFree(d_err);
    throw;
  }
  cudaFree(d_err);
  return h != 0;
}

double selftest_fp32_peak(cudaStream_t s) {
  int dev = 0, sms = 0;
  TN_CUDA(cudaGetDevice(&dev));
  TN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* out = nullptr;
  TN_CUDA(cudaMalloc(&out, sizeof(float)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double tflops = 0;
  try {
    TN_CUDA(cudaEventCreate(&e0));
    TN_CUDA(cudaEventCreate(&e1));
    const unsigned blocks = (unsigned)sms * 8;
    const int iters = 1 << 14;
    ffma_kernel<<<blocks, 256, 0, s>>>(out, 1 << 10, 0.999f, 0.001f);  // warm-up
    TN_CUDA(cudaEventRecord(e0, s));
    ffma_kernel<<<blocks, 256, 0, s>>>(out, iters, 0.999f, 0.001f);
    TN_CUDA(cudaEventRecord(e1, s));
    TN_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    TN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    tflops = 2.0 * kChains * (double)iters * blocks * 256 / (ms * 1e-3) / 1e12;
  } catch (...) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return tflops;
}

}  // namespace tn
