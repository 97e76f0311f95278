// Instantiations of the SVT Jacobi kernel (float), one of several translation units so
// that they compile in parallel.  Key: G * 10000 + B * 100 + E.
#include "lt_jacobi_svt.cuh"

namespace lt {
namespace jac {

template <int G, int E, int B>
static cudaError_t go(const JArgs& a, int grid, cudaStream_t st) {
  auto k = jacobi_svt_kernel<float, G, E, B, kMaxThreadsF32>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.jp.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, a.jp.threads, a.jp.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_svt_f32_pw_b(const JArgs& a, int grid, cudaStream_t st) {
  switch (a.jp.G * 10000 + a.jp.B * 100 + a.jp.E) {
    case 160116: return go<16, 16, 1>(a, grid, st);
    case 160124: return go<16, 24, 1>(a, grid, st);
    case 320120: return go<32, 20, 1>(a, grid, st);
    case 320124: return go<32, 24, 1>(a, grid, st);
    case 320128: return go<32, 28, 1>(a, grid, st);
    case 320132: return go<32, 32, 1>(a, grid, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace jac
}  // namespace lt
