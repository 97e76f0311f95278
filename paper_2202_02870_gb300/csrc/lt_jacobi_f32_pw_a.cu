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

cudaError_t launch_svt_f32_pw_a(const JArgs& a, int grid, cudaStream_t st) {
  switch (a.jp.G * 10000 + a.jp.B * 100 + a.jp.E) {
    case 80102: return go<8, 2, 1>(a, grid, st);
    case 80104: return go<8, 4, 1>(a, grid, st);
    case 80106: return go<8, 6, 1>(a, grid, st);
    case 80108: return go<8, 8, 1>(a, grid, st);
    case 80112: return go<8, 12, 1>(a, grid, st);
    case 80118: return go<8, 18, 1>(a, grid, st);
    case 80124: return go<8, 24, 1>(a, grid, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace jac
}  // namespace lt
