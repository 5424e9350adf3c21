// fsi_probe_peaks: measured ALU and memory ceilings of the current GPU, the
// denominators of the operators' rooflines (timing support; the paper has none).
//
// FMA rate: every thread runs 8 independent fused multiply-add chains (enough to
// cover the pipeline latency) for a fixed count, on a grid of 8 CTAs of 256 threads
// per SM; flops = 2 x chains x count x threads.  Read bandwidth: a grid-stride sum
// of a 2 GiB float4 buffer (only reads reach HBM; the sums are written once per
// thread).  Copy bandwidth: the same buffer copied into a second one (read + write
// bytes counted).  Each figure is the best of five timed launches after a warm-up.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace fsi {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_kernel(T a, T b, int count, T* sink) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = a + T(threadIdx.x + i);
  for (int k = 0; k < count; ++k) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], b, a);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == T(-12345.678)) sink[0] = s;  // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(256) read_kernel(const float4* __restrict__ a, int64_t n, float* sink) {
  float s = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const float4 v = __ldcs(a + i);
    s += (v.x + v.y) + (v.z + v.w);
  }
  if (s == -12345.678f) sink[0] = s;
}

__global__ void __launch_bounds__(256) copy_kernel(const float4* __restrict__ a, float4* __restrict__ b, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) __stcs(b + i, __ldcs(a + i));
}

template <class F>
int best_ms(F launch, float* best) {
  cudaEvent_t e0, e1;
  FSI_CUDA(cudaEventCreate(&e0));
  FSI_CUDA(cudaEventCreate(&e1));
  launch();
  FSI_CUDA(cudaGetLastError());
  FSI_CUDA(cudaDeviceSynchronize());
  *best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    FSI_CUDA(cudaEventRecord(e0));
    launch();
    FSI_CUDA(cudaEventRecord(e1));
    FSI_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    FSI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *best = std::min(*best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return FSI_OK;
}

}  // namespace
}  // namespace fsi

using namespace fsi;

extern "C" int fsi_probe_peaks(double* fp32_tflops, double* fp64_tflops, double* read_gbs, double* copy_gbs) {
  if (!fp32_tflops || !fp64_tflops || !read_gbs || !copy_gbs) return set_error(FSI_EINVAL, "fsi_probe_peaks: null");
  int dev = 0, sms = 0;
  FSI_CUDA(cudaGetDevice(&dev));
  FSI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  const double thr = (double)blocks * threads;
  float* sink = nullptr;
  FSI_CUDA(cudaMalloc(&sink, 64));
  float ms = 0.f;
  int rc;
  const int n32 = 4096, n64 = 256;
  if ((rc = best_ms([&] { fma_kernel<float><<<blocks, threads>>>(1.0f, 0.999f, n32, sink); }, &ms))) goto done;
  *fp32_tflops = 2.0 * 8 * n32 * thr / (ms * 1e-3) / 1e12;
  if ((rc = best_ms([&] { fma_kernel<double><<<blocks, threads>>>(1.0, 0.999, n64, reinterpret_cast<double*>(sink)); },
                    &ms)))
    goto done;
  *fp64_tflops = 2.0 * 8 * n64 * thr / (ms * 1e-3) / 1e12;
  {
    const int64_t bytes = (int64_t)2 << 30;  // 2 GiB per buffer
    float4 *a = nullptr, *b = nullptr;
    cudaError_t e = cudaMalloc(&a, bytes);
    if (e != cudaSuccess) { rc = cuda_check(e, "fsi_probe_peaks: cudaMalloc"); goto done; }
    e = cudaMalloc(&b, bytes);
    if (e != cudaSuccess) { cudaFree(a); rc = cuda_check(e, "fsi_probe_peaks: cudaMalloc"); goto done; }
    const int64_t n = bytes / (int64_t)sizeof(float4);
    e = cudaMemset(a, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(b, 0, bytes);
    if (e != cudaSuccess) {
      cudaFree(a);
      cudaFree(b);
      rc = cuda_check(e, "fsi_probe_peaks: cudaMemset");
      goto done;
    }
    rc = best_ms([&] { read_kernel<<<sms * 8, threads>>>(a, n, sink); }, &ms);
    if (!rc) *read_gbs = (double)bytes / (ms * 1e-3) / 1e9;
    if (!rc) rc = best_ms([&] { copy_kernel<<<sms * 8, threads>>>(a, b, n); }, &ms);
    if (!rc) *copy_gbs = 2.0 * (double)bytes / (ms * 1e-3) / 1e9;
    cudaFree(a);
    cudaFree(b);
  }
done:
  cudaFree(sink);
  return rc;
}
