// Instantiations of the SVT Jacobi kernel (double), one of several translation units so
// that they compile in parallel.  Key: G * 10000 + B * 100 + E.
#include "lt_jacobi_svt.cuh"

namespace lt {
namespace jac {

template <int G, int E, int B>
static cudaError_t go(const JArgs& a, int grid, cudaStream_t st) {
  auto k = jacobi_svt_kernel<double, G, E, B, kMaxThreadsF64>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.jp.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, a.jp.threads, a.jp.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_svt_f64_b(const JArgs& a, int grid, cudaStream_t st) {
  switch (a.jp.G * 10000 + a.jp.B * 100 + a.jp.E) {
    case 80108: return go<8, 8, 1>(a, grid, st);
    case 80110: return go<8, 10, 1>(a, grid, st);
    case 80112: return go<8, 12, 1>(a, grid, st);
    case 80114: return go<8, 14, 1>(a, grid, st);
    case 80116: return go<8, 16, 1>(a, grid, st);
    case 80118: return go<8, 18, 1>(a, grid, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace jac
}  // namespace lt
