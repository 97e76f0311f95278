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

cudaError_t launch_svt_f64_c(const JArgs& a, int grid, cudaStream_t st) {
  switch (a.jp.G * 10000 + a.jp.B * 100 + a.jp.E) {
    case 160108: return go<16, 8, 1>(a, grid, st);
    case 160110: return go<16, 10, 1>(a, grid, st);
    case 160112: return go<16, 12, 1>(a, grid, st);
    case 160114: return go<16, 14, 1>(a, grid, st);
    case 320108: return go<32, 8, 1>(a, grid, st);
    case 320112: return go<32, 12, 1>(a, grid, st);
    case 320116: return go<32, 16, 1>(a, grid, st);
    case 320118: return go<32, 18, 1>(a, grid, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace jac
}  // namespace lt
