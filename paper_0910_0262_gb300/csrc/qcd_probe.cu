// Device-limit probes: the denominators of the kernels' rooflines that no vendor figure gives for
// this part (its FP64 / FP32 FMA rate under the clocks it actually runs at, and the bandwidth of a
// copy whose working set stays in L2).  The paper has no counterpart: it quotes the Cell's peak
// figures (Sec. 2) and measures its own DMA bandwidths (Sec. 3); these play that role here.
#include <cuda_runtime.h>

#include "qcd.h"
#include "qcd_api_scope.h"
#include "qcd_kernels.h"

namespace qcd {

QCD_DEBUG_TAKE(debug_take_probe)
namespace {

constexpr int FMA_CHAINS = 8;      // independent dependency chains per thread
constexpr int FMA_BLOCK = 256;
constexpr int FMA_BLOCKS_PER_SM = 8;

// FMA_CHAINS independent chains x <- x a + b per thread, `iters` times; the sum is stored only when
// it equals a value it never takes, so that the compiler keeps the work and nothing is written.
template <typename R>
__global__ void __launch_bounds__(FMA_BLOCK) fma_probe_kernel(R* sink, int iters, R a, R b) {
  R x[FMA_CHAINS];
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; k++) x[k] = R(threadIdx.x) * R(1e-3) + R(k);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; k++) x[k] = fma(x[k], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; k++) s += x[k];
  if (s == R(-1.25)) sink[blockIdx.x] = s;
}

// dst = src over n float4 (loads through L2 only), grid-stride, `passes` times over the buffer
__global__ void copy_probe_kernel(float4* __restrict__ dst, const float4* __restrict__ src, size_t n, int passes) {
  for (int k = 0; k < passes; k++)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
      dst[i] = __ldcg(src + i);
}

// device time of `reps` back-to-back runs of launch(), after one untimed run
template <typename F>
cudaError_t time_launches(cudaStream_t st, int reps, F launch, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  launch();
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; r++) launch();
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace
}  // namespace qcd

using namespace qcd;

extern "C" {

qcd_status qcd_probe_fma_peak(int precision, void* cuda_stream, double* tflops) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(QCD_ERR_CUDA, "no CUDA device");
  ApiScope scope("qcd_probe_fma_peak", dev);
  if (scope.status() != QCD_OK) return scope.status();
  if (!tflops) return set_error(QCD_ERR_ARG, "null pointer");
  if (precision != 64 && precision != 32) return set_error(QCD_ERR_ARG, "precision must be 64 or 32");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int blocks = sms * FMA_BLOCKS_PER_SM;
  // FP64 runs at a small fraction of the FP32 rate on this part: fewer iterations keep it near 20 ms
  const int iters = precision == 64 ? 4096 : 65536;
  void* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(double) * blocks);
  if (e != cudaSuccess) return set_error(QCD_ERR_NOMEM, cudaGetErrorString(e));
  float ms = 0.f;
  const int reps = 5;
  if (precision == 64)
    e = time_launches(st, reps, [&] {
      fma_probe_kernel<double><<<blocks, FMA_BLOCK, 0, st>>>(static_cast<double*>(sink), iters, 0.999999, 1e-7);
    }, &ms);
  else
    e = time_launches(st, reps, [&] {
      fma_probe_kernel<float><<<blocks, FMA_BLOCK, 0, st>>>(static_cast<float*>(sink), iters, 0.9999f, 1e-5f);
    }, &ms);
  g_kernel_launches += reps + 1;
  cudaFree(sink);
  if (e != cudaSuccess) return set_error(QCD_ERR_CUDA, cudaGetErrorString(e));
  const double flops = 2.0 * FMA_CHAINS * (double)iters * FMA_BLOCK * blocks * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return QCD_OK;
}

qcd_status qcd_probe_copy_bandwidth(size_t bytes, int reps, void* cuda_stream, double* gbs) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(QCD_ERR_CUDA, "no CUDA device");
  ApiScope scope("qcd_probe_copy_bandwidth", dev);
  if (scope.status() != QCD_OK) return scope.status();
  if (!gbs || reps < 1 || bytes < 16 || bytes % 16) return set_error(QCD_ERR_ARG, "need gbs, reps >= 1, bytes a multiple of 16");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void *src = nullptr, *dst = nullptr;
  cudaError_t e = cudaMalloc(&src, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&dst, bytes);
  if (e != cudaSuccess) {
    if (src) cudaFree(src);
    cudaGetLastError();
    return set_error(QCD_ERR_NOMEM, cudaGetErrorString(e));
  }
  cudaMemsetAsync(src, 0, bytes, st);
  const size_t n = bytes / 16;
  // an L2-resident copy takes microseconds: repeat it inside the launch so the launch gap does not count
  const int passes = bytes <= ((size_t)64 << 20) ? 32 : 1;
  float ms = 0.f;
  e = time_launches(st, reps, [&] {
    copy_probe_kernel<<<sms * 8, 256, 0, st>>>(static_cast<float4*>(dst), static_cast<const float4*>(src), n,
                                               passes);
  }, &ms);
  g_kernel_launches += reps + 1;
  cudaFree(src);
  cudaFree(dst);
  if (e != cudaSuccess) return set_error(QCD_ERR_CUDA, cudaGetErrorString(e));
  *gbs = 2.0 * (double)bytes * passes * reps / (ms * 1e-3) / 1e9;
  return QCD_OK;
}

}  // extern "C"
