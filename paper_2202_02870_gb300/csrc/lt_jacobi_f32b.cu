// Instantiations of the SVT Jacobi kernel for float (split across translation units so
// that they compile in parallel).
#include "lt_jacobi_svt.cuh"

namespace lt {
namespace jac {

template <int G, int E>
static cudaError_t go(const JArgs& a, int grid, cudaStream_t st) {
  auto k = jacobi_svt_kernel<float, G, E, kMaxThreadsF32>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.jp.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, a.jp.threads, a.jp.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_svt_f32_g16_32(const JArgs& a, int grid, cudaStream_t st) {
  const int key = a.jp.G * 1000 + a.jp.E;
  switch (key) {
    case 16014: return go<16, 14>(a, grid, st);
    case 16016: return go<16, 16>(a, grid, st);
    case 16018: return go<16, 18>(a, grid, st);
    case 16020: return go<16, 20>(a, grid, st);
    case 16024: return go<16, 24>(a, grid, st);
    case 32014: return go<32, 14>(a, grid, st);
    case 32016: return go<32, 16>(a, grid, st);
    case 32018: return go<32, 18>(a, grid, st);
    case 32020: return go<32, 20>(a, grid, st);
    case 32024: return go<32, 24>(a, grid, st);
    case 32028: return go<32, 28>(a, grid, st);
    case 32032: return go<32, 32>(a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace jac
}  // namespace lt
