// Measurement utility (no counterpart in the paper): the FMA throughput of this GPU in
// FP64 or FP32, the denominator of the ALU rooflines of the Jacobi and transform
// kernels.  Every thread runs eight independent multiply-add chains x <- x a + b
// (a = 1 - 2^-20, b = 2^-20: the chains stay near 1 and never overflow or go
// subnormal), so the FMA pipe, not a dependency, bounds the issue rate.  The grid is
// four CTAs of 512 threads per SM; the kernel runs once to warm up and is then timed
// over three launches with CUDA events; GFLOP/s counts an FMA as two flops.
#include "lt_internal.cuh"

namespace lt {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads)
fma_probe_kernel(T a, T b, int iters, T* __restrict__ sink) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (T)1 + (T)(threadIdx.x + j) * b;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  // a store the compiler cannot drop; never true for chains that stay near 1
  if (s == (T)-1) sink[blockIdx.x] = s;
}

template <typename T>
lt_status measure(int iters, double* gflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return LT_ERR_CUDA;
  const int grid = 4 * sms;
  const T a = (T)1 - (T)9.5367431640625e-07, b = (T)9.5367431640625e-07;  // 2^-20
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return LT_ERR_CUDA;
  }
  fma_probe_kernel<T><<<grid, kProbeThreads, 0, st>>>(a, b, iters, nullptr);
  cudaEventRecord(e0, st);
  for (int r = 0; r < 3; ++r) fma_probe_kernel<T><<<grid, kProbeThreads, 0, st>>>(a, b, iters, nullptr);
  cudaEventRecord(e1, st);
  float ms = 0.f;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.f)) return LT_ERR_CUDA;
  const double flops = 3.0 * 2.0 * kChains * (double)iters * grid * kProbeThreads;
  *gflops = flops / (ms * 1e-3) / 1e9;
  return LT_OK;
}

}  // namespace
}  // namespace lt

extern "C" lt_status lt_measure_fma_peak(lt_precision prec, double* gflops, void* stream) {
  if (gflops == nullptr) return LT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == LT_FP64) return lt::measure<double>(1 << 14, gflops, st);
  if (prec == LT_FP32) return lt::measure<float>(1 << 18, gflops, st);
  return LT_ERR_ARG;
}
